// common.cuh -- shared internals of libptk (context, scratch, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <memory>
#include <unordered_map>
#include <vector>

#include "ptk.h"

namespace ptk {

// ---------------------------------------------------------------------------
// errors
void set_error(const char* fmt, ...);
const char* get_error();

#define PTK_CHECK_ARG(cond, ...)            \
    do {                                    \
        if (!(cond)) {                      \
            ::ptk::set_error(__VA_ARGS__);  \
            return PTK_ERR_INVALID_ARG;     \
        }                                   \
    } while (0)

#define PTK_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::ptk::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                       \
            return PTK_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

#define PTK_LAUNCH_CHECK()                                                                    \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess) {                                                              \
            ::ptk::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),      \
                             __FILE__, __LINE__);                                             \
            return PTK_ERR_CUDA;                                                              \
        }                                                                                     \
    } while (0)

#define PTK_TRY(...)                      \
    do {                                  \
        ptk_status s_ = (__VA_ARGS__);    \
        if (s_ != PTK_OK) return s_;      \
    } while (0)

// True while `st` is being captured into a CUDA graph.
inline bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Raises a kernel's dynamic shared-memory limit to `bytes` and, with
// `carveout`, asks for the largest shared-memory carveout.  The limit only
// grows, so a graph captured for a larger launch of the same kernel keeps
// launching; while `st` is capturing nothing is changed (the uncaptured run
// that precedes every capture has set it).
inline ptk_status smem_attr(const void* kern, size_t bytes, cudaStream_t st, bool carveout = false) {
    if (capturing(st)) return PTK_OK;
    cudaFuncAttributes fa;
    PTK_CUDA(cudaFuncGetAttributes(&fa, kern));
    if ((size_t)fa.maxDynamicSharedSizeBytes < bytes)
        PTK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (carveout && fa.preferredShmemCarveout != (int)cudaSharedmemCarveoutMaxShared)
        PTK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    return PTK_OK;
}

// ---------------------------------------------------------------------------
// device-side status words (one int per kind, in context memory)
enum DevFlag : int {
    FLAG_BAD_ROWS = 0,   // row systems that were not positive definite / non-finite
    FLAG_BAD_INDEX = 1,  // coordinates out of range
    FLAG_TIMEOUT = 2,    // a bounded wait gave up
    FLAG_SPARSE = 3,     // a compacted core list outgrew the count it was sized for
    FLAG_COUNT = 8
};

// Scratch slots: each grows on demand and is reused across calls.
enum Slot : int {
    SLOT_DELTA = 0,     // Delta [E][ld]
    SLOT_ROWBUF,        // per-row B/c sums
    SLOT_PARTIAL,       // per-tile edge partials
    SLOT_PARTIAL_ROW,   // per-tile edge rows
    SLOT_GPERM,         // permuted core
    SLOT_GPERM_TC,      // tensor-core image of the permuted core
    SLOT_RED,           // reduction partials
    SLOT_PRES,          // Cache table
    SLOT_AOLD,          // Cache: previous A^(n)
    SLOT_APPROX,        // Approx accumulators / keys
    SLOT_SORT0,
    SLOT_SORT1,
    SLOT_SORT2,
    SLOT_SORT3,
    SLOT_SCAN,
    SLOT_MISC,
    SLOT_FOLD0,
    SLOT_FOLD1,
    SLOT_QR,
    SLOT_TC_COORDS,     // tensor-core delta: coordinate columns copied to 16-byte aligned SoA
    SLOT_TC_PLAN,       // tensor-core Gram: chunk plan built for a caller's rows
    SLOT_SPARSE,        // sparse-core delta: compacted core lists
    SLOT_COUNT
};

// Launch shape of the delta contraction chosen by the autotuner for a class
// of problems (model dtype, precision, order, ranks).
enum TuneBackend : int { TUNE_DEFAULT = 0, TUNE_SIMT = 1, TUNE_TC = 2 };
struct TuneCfg {
    int backend = TUNE_DEFAULT;
    int chunk_kb = 0;       // CUDA cores, streamed core: shared-memory chunk (0: 48 KB)
    int ctas_per_sm = 0;    // CUDA cores: resident blocks per SM in the grid (0: occupancy limit)
    int dent = 0;           // CUDA cores: entries per thread, 2 or 4 (0: by core size)
};
using TuneTable = std::unordered_map<uint64_t, TuneCfg>;

}  // namespace ptk

struct ptk_timer_rec {
    int id;
    cudaEvent_t e0, e1;
};

struct ptk_ctx {
    int timing = 0;
    int last_order = 0;          // shape of the last sweep (for its statistics)
    int64_t last_nnz = 0;
    double last_lambda = 0.0;
    std::vector<ptk_timer_rec> pending;
    double acc_ms[PTK_T_COUNT] = {};
    int64_t acc_launch[PTK_T_COUNT] = {};
    int64_t acc_groups[PTK_T_COUNT] = {};
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    void* slot_ptr[ptk::SLOT_COUNT] = {};
    size_t slot_bytes[ptk::SLOT_COUNT] = {};
    int* d_flags = nullptr;      // [FLAG_COUNT]
    double* d_stats = nullptr;   // [16] device reduction results
    double* h_stats = nullptr;   // pinned mirror
    int* h_flags = nullptr;      // pinned mirror
    // streams and child contexts that ptk_fit runs independent problems on
    std::vector<std::pair<cudaStream_t, ptk_ctx*>> lanes;
    bool in_capture = false;     // a graph capture is recording this context's launches
    // stream-ordered pool for per-call arrays (slice layouts): freed blocks stay
    // cached for the next call instead of going back to the driver
    cudaMemPool_t pool = nullptr;
    // a second stream for work that overlaps the main stream's kernels
    // (forked from and joined to the calling stream with these events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::shared_ptr<ptk::TuneTable> tune = std::make_shared<ptk::TuneTable>();  // shared with the lanes
};

struct ptk_slices {
    int32_t mode = 0;
    int32_t order = 0;
    int64_t nnz = 0;
    int64_t rows = 0;
    ptk_dtype dtype = PTK_F32;    // type of the slice-ordered values
    int32_t* perm = nullptr;      // [nnz] entry id in input order
    int64_t* row_ptr = nullptr;   // [rows + 1]
    int32_t* cols[PTK_MAX_ORDER] = {};  // slice-ordered coordinate columns; cols[mode] = row id
    void* vals = nullptr;         // [nnz] slice-ordered values (dtype)
    int device = 0;
    bool pooled = false;          // arrays come from the context's memory pool
    int64_t max_row = 0;          // entries of the longest row
    // chunks of the rows long enough for the tensor-core Gram (FP32 layouts):
    // (row, first entry, entries, long-row entries before it) per chunk
    int4* tc_plan = nullptr;
    int64_t tc_nchunks = 0;
    int64_t tc_long_entries = 0;
};

namespace ptk {

// process-wide count of kernel launches issued by libptk
extern std::atomic<int64_t> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Records an event pair around a kernel group (when timing is on) and the
// launches issued inside it.
struct TimerScope {
    ptk_ctx* c;
    int id;
    cudaStream_t st;
    int64_t l0;
    cudaEvent_t e0 = nullptr;
    TimerScope(ptk_ctx* c_, int id_, cudaStream_t st_) : c(c_), id(id_), st(st_), l0(g_launches.load()) {
        if (c->timing && cudaEventCreate(&e0) == cudaSuccess) cudaEventRecord(e0, st);
    }
    ~TimerScope() {
        c->acc_launch[id] += g_launches.load() - l0;
        if (e0) {
            cudaEvent_t e1;
            if (cudaEventCreate(&e1) == cudaSuccess) {
                cudaEventRecord(e1, st);
                c->pending.push_back({id, e0, e1});
            } else {
                cudaEventDestroy(e0);
            }
        }
    }
};

// Scratch allocation: returns nullptr (with the error set) on failure.
void* scratch(ptk_ctx* ctx, int slot, size_t bytes);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t dtype_size(ptk_dtype t) { return t == PTK_F64 ? 8 : 4; }

ptk_status check_model(const ptk_model* m);
ptk_status check_coo(const ptk_coo* x, const ptk_model* m);

// ---------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Gives up after ~`limit` polls, records
// FLAG_TIMEOUT and returns false; the caller must then stop using the buffer.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* flags,
                                                  long long limit = (1ll << 26)) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    if (flags) atomicAdd(&flags[FLAG_TIMEOUT], 1);
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion signalled as
// transaction bytes on `bar`.  Addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)

// sort.cu
ptk_status build_slices_impl(ptk_ctx* ctx, const ptk_coo* x, int mode, ptk_dtype compute, ptk_slices* s,
                             cudaStream_t st);
ptk_status radix_sort_u64_desc_stable(ptk_ctx* ctx, uint64_t* keys, uint32_t* vals, int64_t n,
                                      cudaStream_t st);
// exclusive prefix sum of n uint32 values (in may equal out)
ptk_status excl_scan_u32(ptk_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t st);

// delta (SIMT and tensor-core)
struct DeltaJob {
    int64_t n = 0;                        // entries
    int order = 0;
    int mode = 0;                         // the free mode n
    const int32_t* col[PTK_MAX_ORDER] = {};  // coordinate k of entry e: col[k][e * cstride]
    int64_t cstride = 1;
    const void* factors[PTK_MAX_ORDER] = {};
    int64_t ld[PTK_MAX_ORDER] = {};
    int J[PTK_MAX_ORDER] = {};
    const void* core = nullptr;           // dense C order (model dtype)
    const void* vals = nullptr;           // optional x values (written to slot J_n)
    void* out = nullptr;                  // Delta [n][out_ld]
    int out_ld = 0;
    ptk_dtype dtype = PTK_F32;            // storage/compute dtype (F32 or F64)
    bool padded = false;                  // col/vals arrays have >= 16 bytes of slack past the end
    int chunk_kb = 0;                     // launch shape (see TuneCfg)
    int ctas_per_sm = 0;
    int dent = 0;
    int64_t core_nnz = -1;                // non-zero core entries when known (Approx), else -1
};
int delta_out_ld(int Jn);
// A delta job over n entries of `m` for free mode `mode` (coordinates and output unset).
DeltaJob make_job(const ptk_model* m, int mode, int64_t n);
// Class of a delta job for the autotuner's table.
uint64_t tune_key(const DeltaJob& job, ptk_precision prec);
// Eq. (delta) for `job` in `prec`, with the launch shape the autotuner chose
// for its class (tensor cores for TF32/BF16 where supported, unless the tuner
// found the FP32 CUDA-core kernel faster; CUDA cores otherwise).
ptk_status delta_run(ptk_ctx* ctx, DeltaJob job, ptk_precision prec, cudaStream_t st);
ptk_status delta_simt(ptk_ctx* ctx, const DeltaJob& job, cudaStream_t st);
ptk_status delta_tc(ptk_ctx* ctx, const DeltaJob& job, ptk_precision prec, cudaStream_t st);
bool delta_tc_supported(const DeltaJob& job, ptk_precision prec);

// gram.cu
struct GramJob {
    int64_t n = 0;            // entries (slice order)
    int64_t rows = 0;
    int J = 0;
    const void* delta = nullptr;  // [n][ld] with x at slot J
    int ld = 0;
    const int32_t* rid = nullptr; // [n] row of each entry (non-decreasing)
    const int64_t* row_ptr = nullptr;
    void* rowbuf = nullptr;       // [rows][nout]: FP64 sums, or (s, lo) double-float FP32 pairs (entry tiles)
    ptk_dtype dtype = PTK_F32;
    int schedule = PTK_SCHED_ENTRIES;  // ptk_schedule
    int64_t max_row = 0;               // entries of the longest row (PTK_SCHED_AUTO)
    int* wrote_f64 = nullptr;          // if set: 1 when the sums were stored as FP64 (row schedules)
    const int4* tc_plan = nullptr;     // chunk plan of the slice layout (tensor-core Gram)
    int64_t tc_nchunks = 0;
    int64_t tc_long_entries = 0;
    int64_t rows_below = 0;            // row kernels: only rows with fewer entries (0: every row)
    int digits = 4;                    // tensor-core Gram: 4 digits (28 bits), or 3 (21 bits) for deltas
                                       // from tensor-core products
};
int gram_nout(int J);
// entries per Gram tile (a request aligned to it sums in the same order anywhere)
int gram_tile_entries(int J, ptk_dtype dtype);
ptk_status gram(ptk_ctx* ctx, const GramJob& job, cudaStream_t st);

// gram_tc.cu: tensor-core Gram of the rows with at least gram_tc_min_row()
// entries (FP64 sums into job.rowbuf; the other rows are left untouched)
int gram_tc_min_row();
int64_t gram_tc_plan_capacity(int64_t nnz);
ptk_status gram_tc_plan(ptk_ctx* ctx, const int64_t* row_ptr, int64_t rows, int64_t nnz, int4* plan,
                        int64_t* nchunks_h, int64_t* long_entries_h, cudaStream_t st);
bool gram_tc_supported(const GramJob& job);
ptk_status gram_tc(ptk_ctx* ctx, const GramJob& job, cudaStream_t st);

// solve.cu
struct SolveJob {
    int64_t rows = 0;
    int J = 0;
    const void* rowbuf = nullptr;     // [rows][nout] (gram accumulators)
    ptk_dtype buf_dtype = PTK_F32;
    const int64_t* row_ptr = nullptr; // emptiness test
    double lambda = 0.01;
    void* out = nullptr;              // [rows][ld] (out dtype)
    int64_t ld = 0;
    ptk_dtype out_dtype = PTK_F32;
};
ptk_status solve_rows(ptk_ctx* ctx, const SolveJob& job, cudaStream_t st);

// error.cu
ptk_status error_from_delta(ptk_ctx* ctx, const void* delta, int ld, int Jn, const int32_t* row_col,
                            int64_t row_stride, int64_t n, const void* factor, int64_t fld, ptk_dtype dtype,
                            double* d_out, cudaStream_t st);
ptk_status sumsq_factors(ptk_ctx* ctx, const ptk_model* m, double* d_out, cudaStream_t st);
ptk_status dot_rows(ptk_ctx* ctx, const void* delta, int ld, int Jn, const int32_t* row_of, const int32_t* row_col,
                    int64_t row_stride, int64_t n, const void* factor, int64_t fld, ptk_dtype dtype, void* out,
                    cudaStream_t st);
ptk_status count_nonzero(ptk_ctx* ctx, const void* core, int64_t size, ptk_dtype dtype, double* d_out,
                         cudaStream_t st);

// cache.cu
ptk_status cache_build(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, float* pres, cudaStream_t st);
ptk_status cache_delta(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, const ptk_model* m, const float* pres,
                       void* delta, int ld, cudaStream_t st);
ptk_status cache_rescale(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, int mode, const void* aold,
                         float* pres, cudaStream_t st);

// approx.cu
ptk_status partial_error_impl(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, const float* vals, double* d_R,
                              cudaStream_t st);
// Residual source for R(beta): a Delta array of mode `dmode` (x in slot
// J_dmode) and the coordinates of the same entries in the same order.
struct UVSource {
    const float* delta = nullptr;
    int ld = 0;
    int dmode = 0;
    const int32_t* col[PTK_MAX_ORDER] = {};
    int64_t cstride = 1;
};
// core_nnz: nnz(G) when known (the sweep counts it), else -1
ptk_status approx_truncate(ptk_ctx* ctx, const ptk_coo* x, ptk_model* m, double p, ptk_trunc_rule rule,
                           cudaStream_t st, const UVSource* from_sweep = nullptr, int64_t core_nnz = -1);

// qr.cu
ptk_status qr_finalize_impl(ptk_ctx* ctx, ptk_model* m, cudaStream_t st);

}  // namespace ptk
