/*
 * ptk.h -- C ABI of libptk, a GB300 (sm_103a) implementation of the row-wise
 * ALS update of P-Tucker for sparse Tucker factorisation (Oh, Park, Sael,
 * Kang, "Scalable Tucker Factorization for Sparse Tensors -- Algorithms and
 * Discoveries", arXiv 1710.02261).
 *
 * Problem (Sec. 2.2, Definition "Sparse Tucker Factorization", Eq. TF_PARTIAL):
 * given the observed entries Omega of an N-order tensor X, find a core G
 * (J_1 x ... x J_N) and factors A^(n) (I_n x J_n) minimising
 *     sum_{alpha in Omega} (X_alpha - sum_beta G_beta prod_n a^(n)_{i_n j_n})^2
 *       + lambda sum_n ||A^(n)||^2 .
 *
 * Conventions shared by every call
 *   - Every call returns ptk_status; no C++ exception crosses the ABI.  The
 *     message of the last failure on the calling host thread is returned by
 *     ptk_last_error().
 *   - Array pointers are DEVICE pointers owned by the caller unless the
 *     argument name ends in _h (host).  The library never frees them.
 *   - Work is enqueued on the given stream and is asynchronous unless a call
 *     says otherwise.  A context serialises its own scratch buffers: issue the
 *     calls of one context on one stream at a time (use one context per
 *     concurrent stream).
 *   - Indices are 0-based int32 (the paper is 1-based, Sec. 2.1).  The core is
 *     dense in C order over (j_1..j_N), last index fastest.  Factor A^(n) is
 *     row-major with leading dimension ld[n] >= J[n] (elements).
 *   - lambda must be > 0, so that B + lambda I is positive definite (Sec. 3.2).
 *   - Omega is a list: duplicate coordinates are allowed and each counts once
 *     per occurrence.
 *   - nnz must be < 2^31.
 */
#ifndef PTK_H
#define PTK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ptk_stream_t; /* the same handle type as cudaStream_t */

#define PTK_MAX_ORDER 10
#define PTK_MAX_RANK 16

typedef enum ptk_status {
    PTK_OK = 0,
    PTK_ERR_INVALID_ARG = 1,   /* bad sizes, null pointers, lambda <= 0, index out of range */
    PTK_ERR_OUT_OF_MEMORY = 2, /* scratch allocation failed (nothing was enqueued) */
    PTK_ERR_CUDA = 3,          /* a CUDA runtime call or a kernel launch failed */
    PTK_ERR_UNSUPPORTED = 4,   /* valid request the library does not implement (e.g. Cache + Approx) */
    PTK_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    PTK_ERR_BUSY = 6,          /* admission refused (serving) */
    PTK_ERR_NUMERIC = 7        /* a row system was not positive definite or produced non-finite values */
} ptk_status;

typedef enum ptk_dtype { PTK_F32 = 0, PTK_F64 = 1 } ptk_dtype;

/* Arithmetic of the delta contraction (Eq. delta).  B_i, c_i are accumulated in
 * FP32 for the FP32/TF32/BF16 settings (FP64 for PTK_PREC_FP64); the J x J
 * solve is FP64 in every setting. */
typedef enum ptk_precision {
    PTK_PREC_FP64 = 0, /* CUDA-core FP64 throughout (model dtype must be PTK_F64) */
    PTK_PREC_FP32 = 1, /* CUDA-core FP32 delta ("plain FP32 GPU form") */
    PTK_PREC_TF32 = 2, /* tcgen05 tensor cores, TF32 operands, FP32 accumulation in TMEM */
    PTK_PREC_BF16 = 3, /* tcgen05 tensor cores, BF16 operands, FP32 accumulation in TMEM */
    PTK_PREC_BF16X3 = 4 /* tcgen05 tensor cores, each FP32 operand split into BF16 high + low parts;
                           three MMAs (hi*hi + hi*lo + lo*hi) per product, FP32 accumulation:
                           products within ~2^-16 relative, near-FP32 accuracy */
} ptk_precision;

/* Sec. 3.3: P-Tucker (plain), P-Tucker-Cache, P-Tucker-Approx. */
typedef enum ptk_variant { PTK_PLAIN = 0, PTK_CACHE = 1, PTK_APPROX = 2 } ptk_variant;

/* Alg. 4 criterion: remove the core entries with the largest partial
 * reconstruction error R(beta) (Eq. recon_partial, the paper's rule), or the
 * ones with the smallest |G_beta| (the magnitude rule Sec. 3.3 contrasts with). */
typedef enum ptk_trunc_rule { PTK_TRUNC_R_BETA = 0, PTK_TRUNC_MAGNITUDE = 1 } ptk_trunc_rule;

/* How the row sums B_i, c_i (Eqs. rowB, rowC) are spread over the GPU.
 * Sec. 3.4 gives rows to threads with dynamic scheduling because slice sizes
 * are uneven.  PTK_SCHED_ENTRIES splits the work by entries instead: equal
 * tiles of consecutive slice-ordered entries, with rows that cross tiles merged
 * afterwards, so one huge row is shared by many blocks.  The two row schedules
 * give every row to a single warp, dealt in turn (row r to warp r mod W, the
 * naive static split) or taken from a shared counter (dynamic scheduling).
 * PTK_SCHED_AUTO (the default) takes, per mode, PTK_SCHED_TENSOR for FP32
 * layouts with J <= 15 whose rows of 64 entries or more hold at least half of
 * the entries, otherwise the
 * static row schedule when the longest row of the mode holds at most a
 * quarter of one warp's even share of the entries (short, even rows: no
 * merges, fewer instructions per entry) and the entry split otherwise.  Every schedule sums each row in a fixed
 * order (deterministic); the orders differ between schedules, so FP32 results
 * agree to the accumulators' rounding, not bit for bit. */
typedef enum ptk_schedule {
    PTK_SCHED_AUTO = 0,
    PTK_SCHED_ENTRIES = 1,
    PTK_SCHED_ROWS_STATIC = 2,
    PTK_SCHED_ROWS_DYNAMIC = 3,
    PTK_SCHED_TENSOR = 4  /* FP32, J <= 15: rows of >= 64 entries on the tensor cores in chunks of
                             512 entries (each Delta value split into four 7-bit BF16 digits, exact
                             products and chunk sums, double-float combination), chunks shared
                             out by entries; shorter rows one per warp as PTK_SCHED_ROWS_STATIC */
} ptk_schedule;

typedef struct ptk_ctx ptk_ctx;       /* opaque: device, scratch buffers, error flags */
typedef struct ptk_slices ptk_slices; /* opaque: slice layout of one mode */

/* Observed entries Omega (Table 1). */
typedef struct ptk_coo {
    int32_t order;                /* N, 1 <= N <= PTK_MAX_ORDER */
    int64_t dims[PTK_MAX_ORDER];  /* I_1..I_N (host values) */
    int64_t nnz;                  /* |Omega| */
    const int32_t* idx;           /* device [nnz][order] */
    const void* vals;             /* device [nnz] of dtype */
    ptk_dtype dtype;
} ptk_coo;

/* Tucker model: core G and factors A^(n). */
typedef struct ptk_model {
    int32_t order;
    int32_t J[PTK_MAX_ORDER];     /* core dimensions, 1 <= J_n <= PTK_MAX_RANK */
    int64_t dims[PTK_MAX_ORDER];  /* I_n: rows of A^(n) */
    void* core;                   /* device, dense C order, dtype */
    void* factors[PTK_MAX_ORDER]; /* device, row-major [dims[n]][ld[n]], dtype */
    int64_t ld[PTK_MAX_ORDER];    /* leading dimension of A^(n) in elements, >= J[n] */
    ptk_dtype dtype;
} ptk_model;

typedef struct ptk_als_opts {
    ptk_variant variant;
    ptk_precision precision;
    double lambda;                /* regularisation (paper default 0.01, Sec. 5.1) */
    double trunc_rate;            /* Approx: p, 0 < p < 1 (paper default 0.2) */
    ptk_trunc_rule trunc_rule;
    int32_t error_pass;           /* 1: compute the error after the sweep (Alg. 2) */
    ptk_schedule schedule;        /* work split of the row sums (0: chosen per mode) */
} ptk_als_opts;

/* Filled after a sweep when error_pass is set (host struct; the call then
 * synchronises the stream before returning). */
typedef struct ptk_sweep_stats {
    double sse;          /* sum over Omega of squared residuals */
    double error;        /* sqrt(sse), Eq. (reconfull) */
    double rmse;         /* sqrt(sse / nnz) */
    double loss;         /* sse + lambda sum_n ||A^(n)||_F^2, Eq. (TF_PARTIAL) */
    int64_t core_nnz;    /* non-zero core entries after this sweep (Approx truncates) */
    int64_t bad_rows;    /* row systems that were not positive definite */
} ptk_sweep_stats;

/* ---- context ------------------------------------------------------------ */
ptk_status ptk_create(ptk_ctx** ctx, int device);
void ptk_destroy(ptk_ctx* ctx);
/* Message of the last failure on this host thread ("" if none). */
const char* ptk_last_error(void);
/* Library version string. */
const char* ptk_version(void);

/* ---- tracing --------------------------------------------------------------
 * Kernel groups whose device time the context can record with CUDA events on
 * the launching stream. */
typedef enum ptk_timer {
    PTK_T_SLICES = 0, /* slice layout: radix sort, row pointers, gathers */
    PTK_T_DELTA = 1,  /* Eq. (delta) contraction (CUDA-core or tensor-core) */
    PTK_T_GRAM = 2,   /* Eqs. (rowB), (rowC) segmented sums */
    PTK_T_SOLVE = 3,  /* Eq. (rowupdate) batched FP64 solves */
    PTK_T_ERROR = 4,  /* Eq. (reconfull) error pass and norms */
    PTK_T_CACHE = 5,  /* P-Tucker-Cache table build and rescale */
    PTK_T_APPROX = 6, /* Eq. (recon_partial) scores and Alg. 4 truncation */
    PTK_T_QR = 7,     /* QR finalisation */
    PTK_T_FOLDIN = 8, /* fold-in and prediction */
    PTK_T_COUNT = 9
} ptk_timer;

/* enable != 0: record an event pair around every kernel group from now on. */
ptk_status ptk_set_timing(ptk_ctx* ctx, int32_t enable);
/* Per group since the last read: device milliseconds (ms_h), kernel launches
 * (launches_h, counted even with timing off) and timed group instances
 * (groups_h).  Each pointer may be NULL; arrays have PTK_T_COUNT entries.
 * Waits for the recorded events, then resets the counters. */
ptk_status ptk_read_timers(ptk_ctx* ctx, double* ms_h, int64_t* launches_h, int64_t* groups_h);
/* Kernel launches issued through libptk in this process so far. */
int64_t ptk_launch_count(void);

/* ---- a1: slice layout (Table 1, Omega^(n)_{i_n}; Alg. 3 slice loop) ------
 * Groups the entries by their mode-`mode` index with a stable device radix
 * sort: perm lists the entry ids of row 0, then row 1, ..., each row in input
 * order; row_ptr[I_n + 1] holds the row boundaries.  The layout also keeps a
 * slice-ordered copy of every coordinate column and of the values (converted
 * to the compute type `dtype`).  The handle owns that device memory, taken
 * from the context's stream-ordered memory pool (blocks freed by
 * ptk_slices_destroy are reused by the next layout without a driver
 * allocation).  Synchronous: it waits for `stream` to check the coordinates
 * (INVALID_ARG when one is out of range) and to record the longest row, which
 * the default row-sum schedule of ptk_als_sweep uses. */
ptk_status ptk_build_mode_slices(ptk_ctx* ctx, const ptk_coo* x, int32_t mode, ptk_dtype compute,
                                 ptk_slices** out, ptk_stream_t stream);
/* Waits for the device to be idle (as cudaFree does) and returns the arrays
 * to the pool.  May be called after the context is destroyed. */
void ptk_slices_destroy(ptk_slices* s);
/* Device views of a slice layout: perm [nnz] int32, row_ptr [dims[mode]+1]
 * int64, rid [nnz] int32 (row of each slice-ordered entry). */
ptk_status ptk_slices_view(const ptk_slices* s, const int32_t** perm, const int64_t** row_ptr,
                           const int32_t** rid, int64_t* nnz, int64_t* rows);
/* Copies perm and row_ptr into caller-owned device buffers (either may be
 * NULL), asynchronously on `stream`. */
ptk_status ptk_slices_export(const ptk_slices* s, int32_t* perm_out, int64_t* row_ptr_out, ptk_stream_t stream);

/* ---- a2..a7: one iteration of Alg. 2 -----------------------------------
 * Alg. 3 for modes 1..N in order (every row i of A^(n) is replaced by
 * c_i (B_i + lambda I)^{-1}, Eqs. rowupdate/rowB/rowC/delta), then, if
 * opts->error_pass, the error of Eq. (reconfull) on the device (copied to
 * stats_h, with a stream synchronisation, when stats_h is not NULL), then for
 * PTK_APPROX the core truncation of Alg. 4 (the core is modified in place).
 * A PTK_APPROX sweep first reads nnz(G) back to the host (one 8-byte copy and
 * a stream synchronisation): below a share of |G| that depends on the order,
 * its FP32 CUDA-core delta and its R(beta) sums then visit only the non-zero
 * core entries (Sec. 3.3: the iteration gets cheaper as the core empties).
 * slices[n] must come from ptk_build_mode_slices of the same x with mode n.
 * The core is read-only for PTK_PLAIN / PTK_CACHE.  PTK_CACHE keeps the
 * |Omega| x |G| table Pres (FP32) in context scratch for the sweep.
 * Errors: INVALID_ARG (shape mismatch), UNSUPPORTED (precision/dtype
 * combination), OUT_OF_MEMORY, CUDA; NUMERIC when stats_h is given and some
 * row system failed (the factors are still written; such rows are zero). */
ptk_status ptk_als_sweep(ptk_ctx* ctx, const ptk_coo* x, ptk_slices* const* slices, ptk_model* m,
                         const ptk_als_opts* opts, ptk_sweep_stats* stats_h, ptk_stream_t stream);

/* ---- Alg. 3 for one mode, on the rows one caller owns ----------------------
 * Rows of A^(n) are independent given the other factors (Sec. 3.2): the
 * update of rows [row_lo, row_hi) of mode `mode` needs only the observed
 * entries of those rows.  x holds those entries (any entries of other rows
 * are processed but change nothing), s is x's slice layout of mode `mode`
 * (ptk_build_mode_slices), and every row i in [row_lo, row_hi) becomes
 * c_i (B_i + lambda I)^{-1} (Eq. rowupdate; a row without entries in x
 * becomes zero).  Rows outside the range are left as they are.  This is the
 * step each process of a row-sharded sweep runs before the updated rows are
 * exchanged.  Plain variant only (UNSUPPORTED for Cache / Approx);
 * asynchronous on `stream`. */
ptk_status ptk_als_mode(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, ptk_model* m, int32_t mode,
                        int64_t row_lo, int64_t row_hi, const ptk_als_opts* opts, ptk_stream_t stream);

/* Statistics of the last ptk_als_sweep of this context that ran with
 * opts->error_pass set (computed on the device during that sweep); waits for
 * `stream`.  Lets a caller keep the sweep itself free of host syncs. */
ptk_status ptk_sweep_stats_read(ptk_ctx* ctx, ptk_sweep_stats* stats_h, ptk_stream_t stream);

/* ---- a3: row sums alone, Eqs. (rowB), (rowC) ------------------------------
 * For slice-ordered Delta rows z = [delta_0..delta_{J-1}, x] (device, dtype,
 * [nnz][ld] with ld = J + 1 rounded up to an odd number), row boundaries
 * row_ptr (device int64 [rows + 1], from 0 to nnz) and the row of every
 * entry rid (device int32 [nnz], non-decreasing), writes for every row i
 *     out[i] = [B_i upper triangle, row-major (j <= k); c_i]
 * with B_i = sum z_j z_k and c_i = sum x z_k over the row's entries (device
 * FP64 [rows][J(J+1)/2 + J]; empty rows get zeros), using `schedule` as
 * ptk_als_sweep would (FP32 sums are double-float or, with
 * PTK_SCHED_TENSOR, exact chunk products on the tensor cores; FP64 plain).
 * digits: for PTK_SCHED_TENSOR, the BF16 digits per value, 4 (28 bits; 0
 * means 4) or 3 (21 bits, what ptk_als_sweep takes for tensor-core deltas).
 * The inputs are read, not kept.  Synchronous.  Errors: INVALID_ARG (sizes,
 * ld, row_ptr not spanning 0..nnz), UNSUPPORTED (PTK_SCHED_TENSOR without
 * FP32, J <= 15 and a row of >= 64 entries), OUT_OF_MEMORY, TIMEOUT. */
ptk_status ptk_row_sums(ptk_ctx* ctx, const void* delta, ptk_dtype dtype, int32_t ld, int32_t J, const int64_t* row_ptr,
                        const int32_t* rid, int64_t rows, int64_t nnz, ptk_schedule schedule, int32_t digits,
                        double* out, ptk_stream_t stream);

/* ---- a2: delta vectors, Eq. (delta) ---------------------------------------
 * For each of the n coordinates (device int32 [n][order]; the mode column is
 * ignored) writes delta(j) = sum_{beta: j_mode = j} G_beta prod_{k != mode}
 * a^(k)_{i_k j_k} to out[n][J[mode]] (model dtype, device).  `precision`
 * picks the arithmetic: PTK_PREC_FP64 needs a PTK_F64 model; TF32 / BF16 run on
 * the tensor cores where ptk_delta_tc_supported says so, otherwise in FP32 on
 * CUDA cores. */
ptk_status ptk_delta(ptk_ctx* ctx, const ptk_model* m, int32_t mode, const int32_t* coords, int64_t n,
                     ptk_precision precision, void* out, ptk_stream_t stream);
/* 1 when the tensor-core delta kernel covers mode `mode` of this model shape
 * at this precision (orders 3-5, equal ranks J with J*J <= 128 and a Kronecker
 * group of at most 256 elements, FP32 model), else 0. */
int ptk_delta_tc_supported(const ptk_model* m, int32_t mode, ptk_precision precision);

/* ---- allocation-free delta ------------------------------------------------
 * The paper has no counterpart to this entry point.  It computes the same
 * delta vectors as ptk_delta on CUDA cores (FP32 or FP64, per the model dtype)
 * for callers that cannot allocate device memory: serving threads on a fixed
 * memory budget, where a cudaMalloc may fail or stall the whole device at the
 * worst moment, and runtimes that embed the library and own every byte of
 * device memory themselves, so that no other component may allocate.  It needs
 * no ptk_ctx and calls no cudaMalloc, cudaFree or allocating library routine.
 * Its scratch (the core permuted for `mode`) is a static device array of
 * 512 KiB that every GPU loading the library holds until the process exits; a
 * core whose permuted copy needs more (about 131072 FP32 or 65536 FP64
 * elements) returns PTK_ERR_INVALID_ARG.  It runs on the calling thread's
 * current device.  Set-up: the first call with n > 0 on a device looks up the
 * array's device address and raises the shared-memory limit of the kernels it
 * launches (once per device, under a lock); make that first call before any
 * stream capture.  n == 0 returns PTK_OK without touching the device.  Every
 * call shares the array, and each call rewrites what it reads: calls that
 * overlap on the GPU (other streams, other host threads) race on it, so
 * serialise them.  coords: device int32 [n][order] (mode column ignored);
 * every other column k must lie in [0, dims[k]): unlike ptk_delta, which
 * reports bad coordinates through its context, this call has no status word
 * on the device and does not check them (an out-of-range coordinate reads
 * outside the factor).  out: device [n][J[mode]] of the model dtype. */
ptk_status ptk_delta_noalloc(const ptk_model* m, int32_t mode, const int32_t* coords, int64_t n, void* out,
                             ptk_stream_t stream);

/* ---- a6: error pass on any entry set (training or held-out test set) ----
 * sse, error, rmse of Eq. (reconfull) over x (loss uses lambda).  Synchronous. */
ptk_status ptk_error(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, double lambda,
                     ptk_sweep_stats* stats_h, ptk_stream_t stream);

/* ---- a7: partial reconstruction error, Eq. (recon_partial) --------------
 * R_out (device, double [|G|], C order) receives R(beta) for every core entry
 * (0 for entries already removed, G_beta = 0): the squared-error change that
 * core entry beta is responsible for, computed with the current factors.
 * Alg. 4 removes the entries with the largest values.  FP32 model and values. */
ptk_status ptk_partial_error(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, double* R_out,
                             ptk_stream_t stream);

/* ---- Alg. 2 driver -------------------------------------------------------
 * Runs up to max_sweeps iterations of ptk_als_sweep on each problem, stopping
 * early when |err_t - err_{t-1}| / err_{t-1} < tol (tol <= 0: never), then,
 * if finalize_qr, orthogonalises every A^(n) = Q R, A^(n) <- Q,
 * G <- G x_n R (Alg. 2 final loop; requires I_n >= J_n).  The model holds the
 * initial values on entry (Alg. 2 initialises with U(0,1) draws; the caller
 * provides them).
 *
 * Batching: the problems are independent (different orders, sizes, ranks);
 * they are spread over `lanes` CUDA streams (each with its own scratch), the
 * largest first, each to the least-loaded lane, so that small problems fill
 * the GPU together.  With graphs = 1 every sweep after the first runs inside
 * one CUDA graph per problem whose device-side loop (a conditional WHILE
 * node) applies the stopping rule on the GPU: no host round trip between
 * sweeps.  The first sweep runs eagerly and sizes the lane's scratch.
 * lanes <= 0 picks min(count, 8).  Each problem's arithmetic is the same
 * whatever its lane, so results do not depend on lanes or graphs.
 *
 * errors_h[count][max_sweeps] (nullable) receives the error (Eq. reconfull)
 * after each sweep; sweeps_h[count] (nullable) the sweeps run.  The problems'
 * arrays must be distinct.  Synchronous: returns after every problem is done;
 * PTK_ERR_TIMEOUT if a bounded device wait gave up in any sweep (rows whose
 * system was not positive definite are left to ptk_als_sweep's statistics). */
typedef struct ptk_problem {
    ptk_coo x;
    ptk_slices* slices[PTK_MAX_ORDER];
    ptk_model model;
} ptk_problem;

typedef struct ptk_fit_opts {
    ptk_als_opts als;
    int32_t max_sweeps;
    double tol;
    int32_t finalize_qr;
    int32_t lanes;    /* concurrent streams (<= 0: min(count, 8); at most 16) */
    int32_t graphs;   /* 1: sweeps 2.. as one CUDA graph per problem with a device-side loop */
    int32_t autotune; /* 1: tune the delta launch shape of every untuned problem class first
                         (ptk_autotune_delta on the class's largest problem, mode 1, 2^18 entries) */
} ptk_fit_opts;

ptk_status ptk_fit(ptk_ctx* ctx, ptk_problem* probs, int32_t count, const ptk_fit_opts* opts,
                   double* errors_h, int32_t* sweeps_h, ptk_stream_t stream);

/* ---- failure detection self-test -----------------------------------------
 * Every device wait in libptk is bounded: a kernel that gives up records a
 * timeout, lets its in-flight copies land, frees what it holds and returns,
 * and the call returns PTK_ERR_TIMEOUT with the context still usable.  This
 * call exercises that path on purpose: one block waits on a barrier that
 * nothing completes, for `limit` polls (1 .. 2^20), and the call must return
 * PTK_ERR_TIMEOUT.  The paper has no counterpart.  Synchronous. */
ptk_status ptk_selftest_wait(ptk_ctx* ctx, int64_t limit, ptk_stream_t stream);

/* ---- launch-shape autotuner for Eq. (delta) ------------------------------
 * Times every candidate launch shape of the delta contraction for the model's
 * class (dtype, precision, order, ranks) on the first max_entries entries
 * (<= 0: all) of slice layout `s` (its mode is the free mode), reps launches
 * each after one warm-up, and stores the fastest in the context's table;
 * every later delta launch of that class in this context (and in the lanes of
 * its batched fits) uses it.  Candidates: the tensor-core kernel (TF32/BF16,
 * where supported) and the CUDA-core kernel (FP32/FP64, never less precise)
 * with shared-memory chunk sizes for cores larger than shared memory, blocks
 * per SM and entries per thread.  The paper has no counterpart (its kernels are CPU loops).
 * out_h (nullable) receives every candidate's time.  Synchronous. */
#define PTK_TUNE_MAX 16
typedef struct ptk_tune_report {
    int32_t candidates;
    int32_t best;                       /* index of the fastest */
    int64_t entries;                    /* entries each launch processed */
    int32_t backend[PTK_TUNE_MAX];      /* 1: CUDA cores, 2: tensor cores */
    int32_t chunk_kb[PTK_TUNE_MAX];     /* CUDA cores: chunk of a streamed core (0: core fits) */
    int32_t ctas_per_sm[PTK_TUNE_MAX];  /* CUDA cores: blocks per SM (0: occupancy limit) */
    int32_t entries_per_thread[PTK_TUNE_MAX];  /* CUDA cores: entries per thread (2 or 4) */
    float ms[PTK_TUNE_MAX];             /* mean time of one launch */
} ptk_tune_report;

ptk_status ptk_autotune_delta(ptk_ctx* ctx, const ptk_slices* s, const ptk_model* m, ptk_precision prec,
                              int64_t max_entries, int32_t reps, ptk_tune_report* out_h, ptk_stream_t stream);
/* Forgets every tuned class of the context (later launches use the defaults). */
void ptk_autotune_clear(ptk_ctx* ctx);

/* ---- a8: QR finalisation alone (Alg. 2 final loop) ----------------------- */
ptk_status ptk_qr_finalize(ptk_ctx* ctx, ptk_model* m, ptk_stream_t stream);

/* ---- a9: prediction, Eq. (recon2) ----------------------------------------
 * out[e] = sum_beta G_beta prod_n a^(n)_{coords[e][n] j_n} for e < n. */
ptk_status ptk_predict(ptk_ctx* ctx, const ptk_model* m, const int32_t* coords, int64_t n, void* out,
                       ptk_stream_t stream);

/* ---- a9: fold-in ---------------------------------------------------------
 * Each request is a new slice of mode `mode`: its observed entries give a new
 * row by the row update of Eq. (rowupdate) with G and the other factors fixed
 * (Theorem 1), and the row predicts the request's query coordinates by
 * Eq. (recon2).  obs_idx / query_idx rows are full coordinates [order]; their
 * mode column is ignored, except that an observed entry whose mode column is
 * -1 is padding and contributes nothing.  Offsets are device int64 [count + 1]. */
typedef struct ptk_foldin_batch {
    int32_t count;
    const int64_t* obs_ptr;     /* device [count+1] */
    const int32_t* obs_idx;     /* device [obs_ptr[count]][order] */
    const void* obs_vals;       /* device [obs_ptr[count]], model dtype */
    const int64_t* query_ptr;   /* device [count+1] */
    const int32_t* query_idx;   /* device [query_ptr[count]][order] */
    void* rows_out;             /* device [count][J[mode]], model dtype */
    void* preds_out;            /* device [query_ptr[count]], model dtype */
    int64_t total_obs;          /* host copy of obs_ptr[count] */
    int64_t total_query;        /* host copy of query_ptr[count] */
} ptk_foldin_batch;

ptk_status ptk_foldin(ptk_ctx* ctx, const ptk_model* m, int32_t mode, const ptk_foldin_batch* batch,
                      double lambda, ptk_precision precision, ptk_stream_t stream);

/* ---- serving: continuous-batching fold-in --------------------------------
 * A server answers fold-in requests (see ptk_foldin) for new slices of mode
 * opts->mode of a fixed model.  A worker thread keeps up to opts->slots
 * batches on the GPU, each on its own stream: requests that arrive while
 * batches run are admitted, in arrival order, into the next batch as slots and
 * device memory free up (the bytes of the batches in flight stay under
 * opts->memory_cap_bytes).  Each request's entries are placed at a Gram-tile
 * boundary, so its result is bit-identical alone and in any mix.  The model's
 * device arrays must stay valid and unchanged while the server exists. */
typedef struct ptk_server ptk_server;

typedef struct ptk_server_opts {
    int32_t mode;                 /* the requests are new slices of this mode */
    double lambda;
    ptk_precision precision;      /* delta arithmetic (PTK_PREC_FP64 needs a PTK_F64 model) */
    int32_t max_batch_requests;   /* requests per batch */
    int64_t max_batch_entries;    /* observed entries per batch (before tile padding) */
    int64_t max_batch_queries;    /* query coordinates per batch */
    int64_t memory_cap_bytes;     /* device bytes of the batches in flight (admission) */
    int32_t slots;                /* batches in flight, 1..8 */
    int32_t max_queue;            /* queued requests before submit returns PTK_ERR_BUSY */
} ptk_server_opts;

typedef struct ptk_server_stats {
    int64_t submitted, completed, rejected, batches, queued, inflight_bytes, max_inflight_bytes;
} ptk_server_stats;

/* Creates the server on `device` (allocates its batch buffers; synchronous). */
ptk_status ptk_server_create(const ptk_model* m, int device, const ptk_server_opts* opts, ptk_server** out);
/* Queues one request (host arrays, copied before returning): m observed entries
 * (coordinates [m][order], mode column ignored; values of the model dtype) and
 * q query coordinates [q][order].  *ticket identifies it.  PTK_ERR_BUSY when
 * the queue is full or the request alone exceeds the memory cap;
 * PTK_ERR_INVALID_ARG for out-of-range coordinates. */
ptk_status ptk_server_submit(ptk_server* s, const int32_t* obs_idx_h, const void* obs_vals_h, int64_t m,
                             const int32_t* query_idx_h, int64_t q, uint64_t* ticket);
/* Non-blocking.  When the request is done: *done = 1, row_h[J[mode]] and
 * preds_h[q] (host, model dtype) are filled, *latency_ms is the time from
 * submit to completion, and the ticket is released.  Otherwise *done = 0. */
ptk_status ptk_server_poll(ptk_server* s, uint64_t ticket, void* row_h, void* preds_h, int32_t* done,
                           double* latency_ms);
ptk_status ptk_server_read_stats(ptk_server* s, ptk_server_stats* out_h);
/* Stops the worker after the batches in flight, drops queued requests, frees everything. */
void ptk_server_destroy(ptk_server* s);

/* ---- serving with a device-resident request loop --------------------------
 * The same fold-in as ptk_foldin (Theorem 1: the row update of Eq. rowupdate
 * for a new slice of mode opts->mode with G and the other factors fixed, and
 * predictions by Eq. recon2), served by a loop that runs on the GPU: `workers`
 * persistent CTAs poll a ring of request descriptors in host-mapped pinned
 * memory and each takes the next published request and runs it to the end
 * (delta per entry on CUDA cores in the model dtype, the row sums in
 * double-float for an FP32 model or FP64, an FP64 Cholesky solve with one
 * refinement step, the predictions), writing the row and predictions back to
 * mapped memory.  Requests are admitted in arrival order while their data
 * fits in the arena (opts->arena_bytes of pinned memory the GPU reads in
 * place) and the ring has a free slot; requests that arrive while others run
 * are taken by idle CTAs at once, so requests of every size overlap on the
 * device, and each request's arithmetic (hence its result bits) does not
 * depend on what else is in flight.  A CTA with no work for opts->idle_ms
 * (GPU global timer) leaves, and the kernel ends with the last one; a host
 * thread relaunches it when requests wait.  The model's device arrays must
 * stay valid and unchanged while the server exists; the core (permuted for
 * the mode), one row buffer per thread and a tile of 256 delta rows must fit
 * in one CTA's shared memory (UNSUPPORTED otherwise).  The paper serves no
 * requests; Sec. 3's row update is what each request computes. */
typedef struct ptk_dserver ptk_dserver;

typedef struct ptk_dserver_opts {
    int32_t mode;          /* the requests are new slices of this mode */
    double lambda;
    int32_t ring;          /* descriptors in the request ring (requests in flight at most), 1..65536 */
    int64_t arena_bytes;   /* pinned bytes for the data of the requests in flight (admission) */
    int64_t max_queries;   /* query coordinates per request, at most */
    int64_t max_pending;   /* requests waiting for admission before submit returns PTK_ERR_BUSY */
    int32_t workers;       /* persistent CTAs (<= 0: one per SM) */
    double idle_ms;        /* a CTA leaves after this long without a request */
} ptk_dserver_opts;

typedef struct ptk_dserver_stats {
    int64_t submitted, completed, rejected;
    int64_t launches;          /* launches of the loop kernel (the first, and relaunches after idle exits) */
    int64_t idle_exits;        /* CTAs that left after idle_ms without work */
    int64_t served_on_device;  /* requests the device loop has finished */
    int64_t bad_rows;          /* rows whose system was not positive definite (returned as zero) */
    int64_t pending, inflight; /* waiting for admission; published and not yet collected */
    int32_t running;           /* 1 while the loop kernel runs */
} ptk_dserver_stats;

/* Creates the server on `device` (synchronous: copies the permuted core,
 * allocates the ring, arena and results in pinned mapped host memory) and
 * starts its host thread; the loop kernel starts with the first request. */
ptk_status ptk_dserver_create(const ptk_model* m, int device, const ptk_dserver_opts* opts, ptk_dserver** out);
/* Queues one request (host arrays, copied before returning): m observed
 * entries (coordinates [m][order], mode column ignored; values of the model
 * dtype) and q <= max_queries query coordinates [q][order].  arrival_s: the
 * request's arrival time in seconds on ptk_clock_seconds()'s clock (<= 0:
 * now); latencies run from it.  PTK_ERR_BUSY when the request alone exceeds
 * the arena or max_pending requests wait; PTK_ERR_INVALID_ARG for
 * out-of-range coordinates. */
ptk_status ptk_dserver_submit(ptk_dserver* s, const int32_t* obs_idx_h, const void* obs_vals_h, int64_t m,
                              const int32_t* query_idx_h, int64_t q, double arrival_s, uint64_t* ticket);
/* Non-blocking.  When the request is done: *done = 1, row_h[J[mode]] and
 * preds_h[q] (host, model dtype) are filled, *latency_ms is the time from its
 * arrival to the host seeing its result, and the ticket is released. */
ptk_status ptk_dserver_poll(ptk_dserver* s, uint64_t ticket, void* row_h, void* preds_h, int32_t* done,
                            double* latency_ms);
ptk_status ptk_dserver_read_stats(ptk_dserver* s, ptk_dserver_stats* out_h);
/* Sets the stop word, waits for the loop to leave, frees everything. */
void ptk_dserver_destroy(ptk_dserver* s);
/* Seconds on the steady clock the servers time latencies with. */
double ptk_clock_seconds(void);

#ifdef __cplusplus
}
#endif
#endif /* PTK_H */
