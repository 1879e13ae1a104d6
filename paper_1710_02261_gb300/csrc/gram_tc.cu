// gram_tc.cu -- Eqs. (rowB) and (rowC) on the tensor cores, for rows with many
// entries:
//     B_i = sum_{alpha in Omega_i} delta_alpha delta_alpha^T ,
//     c_i = sum_{alpha in Omega_i} x_alpha delta_alpha .
// With the value x appended as column J, both are the upper triangle of the
// Gram matrix Z^T Z of the row's Delta rows z = [delta_0..delta_{J-1}, x].
//
// Exact products on BF16 tensor cores (the splitting scheme of Ozaki, Ogita,
// Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication", 2012).  A row's entries are
// taken in chunks of up to CH = 512 consecutive entries.  For each column j
// the chunk's largest |z_j| fixes a power of two 2^{e_j} > max |z_j|, and
// every z_j is written as S = 4 signed digits (3 for deltas from tensor-core
// products, whose own error is 2^-16 or more):
//     z_j = 2^{e_j - 7} (d0 + d1 + d2 + d3),  d_s = q_s 2^{-7s},  |q_s| <= 128,
// each rounded to nearest, so only the last one rounds z (by at most 2^-29 of
// the column's largest value with four digits, 2^-22 with three; below FP32's
// own rounding of delta for values within a factor 16 of it).  Digits hold at most 8 significant bits, exact
// in BF16; the product of two is exact in the FP32 accumulator, and a chunk's
// 512 products of one digit pair are multiples of 2^{-7(s+t)} of magnitude at
// most 2^{23-7(s+t)}, so every MMA result D[(s,j),(t,k)] = sum_alpha
// d_s(alpha,j) d_t(alpha,k) is exact.  The chunk's Gram entry is then
//     G_jk = 2^{e_j + e_k - 14} sum_{s,t} D[(s,j),(t,k)],
// combined in double-float arithmetic (exact over t, ~2^-48 relative over s)
// and added to the row's double-float sums.  So the sums are those of the
// Delta rows themselves to about 2^-48 of sum |z_j z_k|: the accuracy of the
// CUDA-core double-float kernel (gram.cu), with the products on tensor cores.
//
// Operands: the 64 digit rows (s, j) of a chunk, K-major over entries, form
// one shared-memory matrix Q [64][CH] (BF16).  One tcgen05.mma per 16
// entries computes D = Q Q^T: A is Q read as 128 rows (rows 64..127 read the
// next 8-entry block's rows 0..63 and land in accumulator rows never read),
// B is Q's 64 rows, N = 64.  The accumulator (128 lanes x 64 columns FP32)
// lives in tensor memory; lane (s, j) holds D[(s,j), :].
//
// Work split: the rows with at least TLONG entries are cut into chunks by the
// slice layout (a plan of (row, first entry, entries, long-row entries
// before it) per chunk).  Each CTA takes a contiguous range of chunks holding an equal share
// of the work, counted as the entries plus a fixed cost per chunk.  A row that lies inside one CTA's range
// is written by it; a row split between CTAs leaves its pieces in per-CTA
// slots, added in CTA order by gram_tc_fixup.  Rows with fewer entries go to
// the row-per-warp CUDA-core kernel (gram.cu).  Every sum is taken in a fixed
// order: results are deterministic.
//
// Roles (384 threads): warps 0-7 split the chunk into digits (Q); warps 8-9
// read the accumulator (TMEM lanes 0-63) and combine; warp 10 owns TMEM and
// streams chunks into shared memory with bulk copies; warp 11 issues the MMAs.
// Two digit stages and accumulators, two or three chunk stages; every wait is
// bounded (FLAG_TIMEOUT).
#include "common.cuh"
#include "tc_ptx.cuh"

namespace ptk {

namespace {

using namespace ::ptk::tc;

constexpr int GT_CH = 512;                  // entries per chunk
constexpr int GT_TLONG = 64;                // rows with at least this many entries use the tensor cores
constexpr int GT_SMAX = 4;                  // digits per value, at most
constexpr int GT_C = 16;                    // columns per digit block (J + 1 <= 16)
constexpr int GT_KC = GT_CH / 8;            // 8-entry blocks per chunk
constexpr int GT_QBYTES = GT_KC * 1024 + 1024;  // Q stage + the block read past its end by rows 64..127
constexpr int GT_NSL = 8;                   // digit warps
constexpr int GT_SLT = GT_NSL * 32;         // digit threads
constexpr int GT_WC = GT_NSL;               // first combiner warp (TMEM lanes 0-31; the next: 32-63)
constexpr int GT_WL = GT_NSL + 2;           // loader / TMEM owner warp
constexpr int GT_WM = GT_NSL + 3;           // MMA warp
constexpr int GT_THREADS = (GT_NSL + 4) * 32;
static_assert(GT_NSL % 4 == 0, "combiner warps must sit on TMEM lane quadrants 0 and 1");
constexpr int GT_NCOL = 64;                 // accumulator columns (t, k)
// work of one chunk beside its entries, in entries, for the CTA split: the
// chunk's fixed costs (three barriers, the accumulator round trip, the
// combination) measured as worth about 1.5k entries of digit work
constexpr int GT_K0 = 1536;

__host__ __device__ constexpr int gt_ld(int J) { return ((J + 1) & 1) ? (J + 1) : (J + 2); }
// a chunk of up to CH entries starting up to 3 entries into the stage, plus
// the zeroed tail up to the next 16-entry boundary
__host__ __device__ constexpr int gt_dstage(int J) { return ((GT_CH + 24) * gt_ld(J) * 4 + 127) / 128 * 128; }
// chunk stages in flight: three (the loader two chunks ahead) where they fit
// beside two digit stages and the static arrays, else two
__host__ __device__ constexpr int gt_nds(int J) {
    return 2 * GT_QBYTES + 3 * gt_dstage(J) + 128 + 18 * 1024 <= 227 * 1024 ? 3 : 2;
}
__host__ __device__ constexpr int gt_smem(int J) { return 2 * GT_QBYTES + gt_nds(J) * gt_dstage(J) + 128; }

// ---- the chunk plan (built once per slice layout) ---------------------------
__global__ void plan_count(const int64_t* __restrict__ row_ptr, int64_t rows, int64_t tlong,
                           uint32_t* __restrict__ nchunk, uint32_t* __restrict__ nent) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= rows; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c = 0, e = 0;
        if (r < rows) {
            const int64_t m = row_ptr[r + 1] - row_ptr[r];
            if (m >= tlong) {
                c = (uint32_t)((m + GT_CH - 1) / GT_CH);
                e = (uint32_t)m;
            }
        }
        nchunk[r] = c;
        nent[r] = e;
    }
}

// one thread per chunk (a Zipf head row has thousands): its row is the one
// whose chunk range holds it; a row of m >= tlong entries has ceil(m / CH)
// chunks of equal size (+-1)
__global__ void plan_emit(const int64_t* __restrict__ row_ptr, int64_t rows, int64_t cap,
                          const uint32_t* __restrict__ coff, const uint32_t* __restrict__ eoff,
                          int4* __restrict__ plan) {
    const int64_t total = coff[rows];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total && c < cap;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = rows;  // first row r with coff[r] > c, minus one
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)coff[mid] <= c)
                lo = mid + 1;
            else
                hi = mid;
        }
        const int64_t r = lo - 1;
        const int64_t b = row_ptr[r], m = row_ptr[r + 1] - b;
        const int64_t nc = (m + GT_CH - 1) / GT_CH, q = c - coff[r];
        const int64_t s0 = q * m / nc, s1 = (q + 1) * m / nc;
        plan[c] = make_int4((int)r, (int)(b + s0), (int)(s1 - s0), (int)(eoff[r] + (uint32_t)s0));
    }
}

// ---- double-float helpers ----------------------------------------------------
struct DF {
    float h, l;
};
// a + b = s.h + s.l exactly (Knuth's TwoSum); the _rn intrinsics keep nvcc
// from contracting the error terms into FMAs
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.h, b.h);
    const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s.h, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s.h))};
}
// 2^n for -126 <= n <= 127
__device__ __forceinline__ float pow2i(int n) { return __int_as_float((n + 127) << 23); }
// v * 2^E, exact unless the result leaves the FP32 range; -254 <= E <= 242
// here (E < -250 only for values below 2^-250, which flush to zero)
__device__ __forceinline__ DF df_scale(DF v, int E) {
    if (E < -250) return {0.f, 0.f};
    const int e1 = E / 2, e2 = E - e1;
    const float a = pow2i(e1), b = pow2i(e2);
    return {__fmul_rn(__fmul_rn(v.h, a), b), __fmul_rn(__fmul_rn(v.l, a), b)};
}

struct GtParams {
    const float* delta;      // [n][ld]: delta_0..delta_{J-1}, x
    const int4* plan;        // [nchunks]: row, first entry, entries, long-row entries before it
    int64_t nchunks;
    int64_t long_entries;
    int64_t k0;              // work of one chunk's combination, in entries (CTA balance)
    double* rowbuf;          // [rows][nout] FP64
    float2* slotL;           // [grid][nout] the first run of a CTA when its row began earlier
    float2* slotR;           // [grid][nout] the last run of a CTA when its row goes on
    int* meta;               // [grid][5]: first chunk, end chunk, left row, left passes through, right row
    int* flags;
};

// first chunk c whose work before it, long-row entries + k0 c, is >= target
__device__ int64_t plan_lower_bound(const int4* plan, int64_t n, int64_t k0, int64_t target) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(uint32_t)plan[mid].w + k0 * mid < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// output index of Gram entry (j, k), j <= k, of the columns [delta, x]:
// B upper triangle row-major, then c; -1 for (x, x)
template <int J>
__device__ __forceinline__ int gt_out(int j, int k) {
    if (k < J) return j * J - j * (j - 1) / 2 + (k - j);
    return j < J ? J * (J + 1) / 2 + j : -1;
}

// S digits per value: 4 (28 bits) for FP32 deltas, 3 (21 bits) where the
// deltas come from tensor-core products (errors of 2^-16 or more)
template <int J, int S>
__global__ void __launch_bounds__(GT_THREADS, 1) gram_tc_kernel(const GtParams p) {
    constexpr int LD = gt_ld(J), C = J + 1, DST = gt_dstage(J), NDS = gt_nds(J), NOUT = J * (J + 1) / 2 + J;
    static_assert(C <= GT_C, "J + 1 columns must fit a digit block");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint64_t dfull[3], dempty[3], qfull[2], qempty[2], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    __shared__ int64_t c0_s, c1_s;
    __shared__ float sRed[GT_NSL][GT_C];   // per-warp column maxima
    __shared__ float sScale[2][GT_C];      // 2^{7 - e_j} per stage (0: zero column)
    __shared__ int sExp[4][GT_C];          // e_j per chunk (ring of 4; INT_MIN: zero column)
    __shared__ int4 sChunk[8];             // plan entries in flight (ring of 8, written by the loader)
    __shared__ DF sP[2][S][GT_C][GT_C];    // combiner exchange: P_s(j, q) at [s][q][j], per stage

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int cta = blockIdx.x;

    if (tid == 0) {
        for (int b = 0; b < NDS; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], GT_SLT);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&qfull[b], GT_SLT);
            mbar_init(&qempty[b], 1);
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 64);
        }
        fence_mbar_init();
        abort_s = 0;
        // this CTA's chunks: an equal share of the work (entries + K0 per chunk)
        const int64_t G = gridDim.x;
        const int64_t W = p.long_entries + p.k0 * p.nchunks;
        const int64_t lo = W * cta / G, hi = W * (cta + 1) / G;
        const int64_t c0 = plan_lower_bound(p.plan, p.nchunks, p.k0, lo);
        const int64_t c1 = cta + 1 == G ? p.nchunks : plan_lower_bound(p.plan, p.nchunks, p.k0, hi);
        c0_s = c0;
        c1_s = c1;
        int* m = p.meta + 5 * cta;
        m[0] = (int)c0;
        m[1] = (int)c1;
        m[2] = -1;
        m[3] = 0;
        m[4] = -1;
    }
    if (warp == GT_WL) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(2 * GT_NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int64_t c0 = c0_s, nk = c1_s - c0_s;

    if (warp < GT_NSL) {
        // ---------------- digits ----------------
        for (int64_t k = 0; k < nk; ++k) {
            const int b = (int)(k & 1);
            const unsigned ph = (unsigned)((k >> 1) & 1);
            const int bd = (int)(k % NDS);
            const unsigned phd = (unsigned)((k / NDS) & 1);
            bool ok = !abort_s && mbar_wait_bounded(&qempty[b], ph ^ 1, p.flags, 1ll << 24) &&
                      mbar_wait_bounded(&dfull[bd], phd, p.flags, 1ll << 24);
            if (named_bar_or(1, GT_SLT, !ok)) {
                abort_s = 1;
                break;
            }
            const int4 ch = sChunk[k & 7];  // published by the loader before dfull completed
            const int m = ch.z;
            const int off = ch.y & 3;  // the stage starts at the 4-entry boundary below the chunk
            float* D = reinterpret_cast<float*>(smem + 2 * GT_QBYTES + bd * DST) + off * LD;
            const int nblk = 2 * ((m + 15) >> 4);  // 8-entry blocks the MMA reads
            // zero the entries between the chunk's end and the last block's
            for (int i = tid; i < (nblk * 8 - m) * C; i += GT_SLT) D[(m + i / C) * LD + i % C] = 0.f;
            // column maxima: thread (j = tid & 15, g8 = tid >> 4) takes entries g8, g8 + 8, ...
            {
                constexpr int GS = GT_SLT / 16;  // threads per column
                const int j = tid & 15, g8 = tid >> 4;
                float mx = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
                if (j < C) {
                    int e = g8;
                    for (; e + 3 * GS < m; e += 4 * GS) {
                        mx = fmaxf(mx, fabsf(D[e * LD + j]));
                        m1 = fmaxf(m1, fabsf(D[(e + GS) * LD + j]));
                        m2 = fmaxf(m2, fabsf(D[(e + 2 * GS) * LD + j]));
                        m3 = fmaxf(m3, fabsf(D[(e + 3 * GS) * LD + j]));
                    }
                    for (; e < m; e += GS) mx = fmaxf(mx, fabsf(D[e * LD + j]));
                }
                mx = fmaxf(fmaxf(mx, m1), fmaxf(m2, m3));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
                if (lane < 16) sRed[warp][j] = mx;
            }
            named_bar_or(1, GT_SLT, false);
            if (tid < GT_C) {
                float mx = sRed[0][tid];
#pragma unroll
                for (int w = 1; w < GT_NSL; ++w) mx = fmaxf(mx, sRed[w][tid]);
                const int be = (int)((__float_as_uint(mx) >> 23) & 255);
                // 2^e > max|z| with e = be - 126; columns below 2^-121 (or empty) count as zero
                const int e = be - 126;
                const bool zero = be == 0 || e < -120;
                sScale[b][tid] = zero ? 0.f : pow2i(7 - e);
                sExp[k & 3][tid] = zero ? INT_MIN : e;
            }
            named_bar_or(1, GT_SLT, false);
            // digits: items (column j < C, 8-entry block g), 2 ceil(m / 16) blocks.
            // y = z 2^{7-e} (|y| < 128) is split as y = d0 + d1 + d2 + d3, d_s a
            // multiple of 2^{-7s} with |d_s| <= 2^{7-7s} (rounding to nearest by
            // adding and removing 1.5 * 2^{23-7s}); each d_s has at most 8
            // significant bits, so its BF16 image is the top half of its FP32
            // bits.  Pairs of entries go through the packed FP32x2 instructions.
            uint8_t* Q = smem + b * GT_QBYTES;
            const float2 neg1 = make_float2(-1.f, -1.f);
            const int nit = C * nblk;
            auto item = [&](int it, uint32_t (&w)[S][4]) {
                const int j = it % C, g = it / C;
                const float sc = sScale[b][j];
                const float2 sc2 = make_float2(sc, sc);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int e = g * 8 + 2 * h;
                    float2 r = __fmul2_rn(make_float2(D[e * LD + j], D[(e + 1) * LD + j]), sc2);  // exact
#pragma unroll
                    for (int q = 0; q < S; ++q) {
                        const float Ms = 1.5f * (float)(1 << 23) / (float)(1 << (7 * q));  // 1.5 * 2^{23-7q}
                        const float2 t = __fadd2_rn(r, make_float2(Ms, Ms));
                        const float2 d = __fadd2_rn(t, make_float2(-Ms, -Ms));  // r rounded to a multiple of 2^{-7q}
                        w[q][h] = __byte_perm(__float_as_uint(d.x), __float_as_uint(d.y), 0x7632);
                        if (q + 1 < S) r = __ffma2_rn(d, neg1, r);  // r - d, exact
                    }
                }
            };
            auto store = [&](int it, const uint32_t (&w)[S][4]) {
                const int j = it % C, g = it / C;
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    const int row = q * GT_C + j;
                    *reinterpret_cast<uint4*>(Q + g * 1024 + (row >> 3) * 128 + (row & 7) * 16) =
                        make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
                }
            };
            // two items at a time: independent chains for the latency of each
            int it = tid;
            for (; it + GT_SLT < nit; it += 2 * GT_SLT) {
                uint32_t w0[S][4], w1[S][4];
                item(it, w0);
                item(it + GT_SLT, w1);
                store(it, w0);
                store(it + GT_SLT, w1);
            }
            if (it < nit) {
                uint32_t w0[S][4];
                item(it, w0);
                store(it, w0);
            }
            fence_proxy_async_smem();  // the digits are read by the tensor cores
            mbar_arrive(&qfull[b]);
            mbar_arrive(&dempty[bd]);
        }
    } else if (warp < GT_WC + 2) {
        // ---------------- accumulator -> double-float row sums ----------------
        // Lane (s, j) of TMEM holds D[(s,j), (t,q)]; it forms P_s(j, q) =
        // sum_t D[(s,j),(t,q)] exactly and leaves it in shared memory.  Then
        // thread T of the 64 owns outputs T, T + 64, T + 128 of the row (Gram
        // entry (j, q)): it adds the four P_s, scales by 2^{e_j + e_q - 14}
        // and keeps the row's double-float sum.
        const int L = tid - GT_WC * 32;
        const int s = L >> 4, j = L & 15;
        constexpr int PER = (NOUT + 63) / 64;
        int oj[PER], oq[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int o = L + 64 * u;
            oj[u] = -1;
            oq[u] = 0;
            if (o < J * (J + 1) / 2) {
                int a = 0, first = 0;
                while (o >= first + (J - a)) {
                    first += J - a;
                    ++a;
                }
                oj[u] = a;
                oq[u] = a + (o - first);
            } else if (o < NOUT) {
                oj[u] = o - J * (J + 1) / 2;  // c_k = sum x delta_k: Gram entry (k, J)
                oq[u] = J;
            }
        }
        DF acc[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) acc[u] = {0.f, 0.f};
        int run_row = -1;
        int64_t run_first = 0;
        auto flush = [&](int64_t last) {
            // the run of chunks [run_first, last] (CTA-relative) of row run_row
            const int64_t cf = c0 + run_first, cl = c0 + last;
            const bool before = run_first == 0 && cf > 0 && p.plan[cf - 1].x == run_row;
            const bool after = last == nk - 1 && cl + 1 < p.nchunks && p.plan[cl + 1].x == run_row;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int o = L + 64 * u;
                if (oj[u] < 0) continue;
                if (!before && !after)
                    p.rowbuf[(int64_t)run_row * NOUT + o] = (double)acc[u].h + (double)acc[u].l;
                else if (before)
                    p.slotL[(int64_t)cta * NOUT + o] = make_float2(acc[u].h, acc[u].l);
                else
                    p.slotR[(int64_t)cta * NOUT + o] = make_float2(acc[u].h, acc[u].l);
            }
            if (L == 0) {
                int* mt = p.meta + 5 * cta;
                if (before) {
                    mt[2] = run_row;
                    mt[3] = after ? 1 : 0;
                } else if (after) {
                    mt[4] = run_row;
                }
            }
        };
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        int row_next = nk > 0 ? p.plan[c0].x : -1;
        for (int64_t k = 0; k < nk; ++k) {
            const int b = (int)(k & 1);
            const unsigned ph = (unsigned)((k >> 1) & 1);
            const bool ok = !abort_s && mbar_wait_bounded(&tfull[b], ph, p.flags, 1ll << 24);
            if (named_bar_or(2, 64, !ok)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            float d[S * GT_C];
            const uint32_t taddr = tmem_base_s + lane_off + (uint32_t)(b * GT_NCOL);
#pragma unroll
            for (int c = 0; c < S * GT_C; c += 16) tmem_ld16(taddr + c, d + c);
            tmem_ld_wait();
            const int row = row_next;
            if (k + 1 < nk) row_next = p.plan[c0 + k + 1].x;  // in flight while this chunk is combined
            int exj[PER], exq[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                exj[u] = oj[u] >= 0 ? sExp[k & 3][oj[u]] : INT_MIN;
                exq[u] = oj[u] >= 0 ? sExp[k & 3][oq[u]] : INT_MIN;
            }
            tc_fence_before();
            mbar_arrive(&tempty[b]);
            // P_s(j, q) = sum_t D[(s,j),(t,q)]: exact in double-float
            if (s < S) {
#pragma unroll
                for (int q = 0; q < C; ++q) {
                    DF v = two_sum(d[q], d[GT_C + q]);
#pragma unroll
                    for (int t = 2; t < S; ++t) {
                        const DF w = two_sum(v.h, d[t * GT_C + q]);
                        v = {w.h, __fadd_rn(v.l, w.l)};
                    }
                    sP[b][s][q][j] = v;
                }
            }
            named_bar_or(2, 64, false);
            if (row != run_row) {
                if (run_row >= 0) flush(k - 1);
#pragma unroll
                for (int u = 0; u < PER; ++u) acc[u] = {0.f, 0.f};
                run_row = row;
                run_first = k;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (oj[u] < 0 || exj[u] == INT_MIN || exq[u] == INT_MIN) continue;
                const int jj = oj[u], qq = oq[u];
                DF t = sP[b][0][qq][jj];
#pragma unroll
                for (int u2 = 1; u2 < S; ++u2) t = df_add(t, sP[b][u2][qq][jj]);
                acc[u] = df_add(acc[u], df_scale(t, exj[u] + exq[u] - 14));
            }
        }
        if (!abort_s && run_row >= 0) flush(nk - 1);
    } else if (warp == GT_WL) {
        // ---------------- chunk loader ----------------
        if (lane == 0) {
            for (int64_t k = 0; k < nk; ++k) {
                const int bd = (int)(k % NDS);
                const unsigned phd = (unsigned)((k / NDS) & 1);
                if (abort_s || !mbar_wait_bounded(&dempty[bd], phd ^ 1, p.flags, 1ll << 24)) {
                    abort_s = 1;
                    break;
                }
                const int4 ch = p.plan[c0 + k];
                sChunk[k & 7] = ch;  // visible to the waiters of dfull[bd] (released by its arrive)
                const int64_t a0 = ch.y & ~3;
                const int64_t a1 = ((int64_t)ch.y + ch.z + 3) & ~3ll;
                const unsigned bytes = (unsigned)((a1 - a0) * LD * 4);  // a multiple of 16: 4 | (a1 - a0)
                mbar_expect_tx(&dfull[bd], bytes);
                bulk_g2s(smem + 2 * GT_QBYTES + bd * DST, p.delta + a0 * LD, bytes, &dfull[bd]);
            }
        }
    } else if (tid == GT_WM * 32) {
        // ---------------- MMA issue ----------------
        const uint32_t idesc = instr_desc(1, 128, S * GT_C);  // N: the digit rows (t, q)
        for (int64_t k = 0; k < nk; ++k) {
            const int b = (int)(k & 1);
            const unsigned ph = (unsigned)((k >> 1) & 1);
            if (abort_s || !mbar_wait_bounded(&qfull[b], ph, p.flags, 1ll << 24) ||
                !mbar_wait_bounded(&tempty[b], ph ^ 1, p.flags, 1ll << 24)) {
                abort_s = 1;
                break;
            }
            tc_fence_after();
            const int ksteps = (sChunk[k & 7].z + 15) >> 4;
            const uint32_t tmem = tmem_base_s + (uint32_t)(b * GT_NCOL);
            for (int ks = 0; ks < ksteps; ++ks) {
                // K-block pair (2 ks, 2 ks + 1): 8-row groups 128 bytes apart, K-blocks 1024
                const uint64_t dsc = smem_desc(smem + b * GT_QBYTES + ks * 2048, 1024, 128);
                mma<false>(tmem, dsc, dsc, idesc, ks > 0);
            }
            mma_commit(&tfull[b]);
            mma_commit(&qempty[b]);
        }
    }
    __syncthreads();
    if (warp == GT_WL) {
        if (abort_s) {
            // let issued copies and MMAs land before TMEM is freed (bounded)
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&tfull[b], 0, nullptr, 1 << 20);
            for (int b = 0; b < NDS; ++b) mbar_wait_bounded(&dfull[b], 0, nullptr, 1 << 20);
        }
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(2 * GT_NCOL)
                     : "memory");
    }
}

// Rows split between CTAs: the right piece of the CTA where the row begins,
// then the left pieces of the following CTAs up to the one where it ends, in
// CTA order.  One block per CTA slot; only slots that end a row do work.
__global__ void gram_tc_fixup(GtParams p, int nout) {
    const int c = blockIdx.x;
    const int* mc = p.meta + 5 * c;
    const int r = mc[2];
    if (r < 0 || mc[3]) return;
    int d = c - 1;
    while (d >= 0) {
        const int* md = p.meta + 5 * d;
        if (md[0] == md[1] || (md[2] == r && md[3])) {
            --d;
            continue;
        }
        break;
    }
    if (d < 0 || p.meta[5 * d + 4] != r) {
        if (threadIdx.x == 0) atomicAdd(&p.flags[FLAG_BAD_ROWS], 1);  // not reachable with a valid plan
        return;
    }
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        const float2 v0 = p.slotR[(int64_t)d * nout + o];
        DF acc = {v0.x, v0.y};
        for (int e = d + 1; e <= c; ++e) {
            const int* me = p.meta + 5 * e;
            if (me[0] == me[1]) continue;
            const float2 v = p.slotL[(int64_t)e * nout + o];
            acc = df_add(acc, {v.x, v.y});
        }
        p.rowbuf[(int64_t)r * nout + o] = (double)acc.h + (double)acc.l;
    }
}

template <int J, int S>
ptk_status launch_tc(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    constexpr int NOUT = J * (J + 1) / 2 + J;
    if (job.ld != gt_ld(J)) {
        set_error("gram_tc: Delta row length %d, expected %d", job.ld, gt_ld(J));
        return PTK_ERR_INVALID_ARG;
    }
    auto kern = gram_tc_kernel<J, S>;
    PTK_TRY(smem_attr((const void*)kern, gt_smem(J), st, true));
    const int grid = ctx->sm_count;
    const size_t slot_bytes = sizeof(float2) * (size_t)grid * NOUT;
    char* part = (char*)scratch(ctx, SLOT_PARTIAL, 2 * slot_bytes + sizeof(int) * 5 * (size_t)grid + 64);
    if (!part) return PTK_ERR_OUT_OF_MEMORY;
    GtParams p;
    p.delta = (const float*)job.delta;
    p.plan = job.tc_plan;
    p.nchunks = job.tc_nchunks;
    p.long_entries = job.tc_long_entries;
    p.k0 = GT_K0;
    p.rowbuf = (double*)job.rowbuf;
    p.slotL = (float2*)part;
    p.slotR = (float2*)(part + slot_bytes);
    p.meta = (int*)(part + 2 * slot_bytes);
    p.flags = ctx->d_flags;
    { kern<<<grid, GT_THREADS, gt_smem(J), st>>>(p); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    { gram_tc_fixup<<<grid, 128, 0, st>>>(p, NOUT); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

}  // namespace

int gram_tc_min_row() { return GT_TLONG; }

ptk_status gram_tc_plan(ptk_ctx* ctx, const int64_t* row_ptr, int64_t rows, int64_t nnz, int4* plan,
                        int64_t* nchunks_h, int64_t* long_entries_h, cudaStream_t st) {
    uint32_t* cnt = (uint32_t*)scratch(ctx, SLOT_SORT2, sizeof(uint32_t) * 2 * (size_t)(rows + 1));
    if (!cnt) return PTK_ERR_OUT_OF_MEMORY;
    uint32_t* ent = cnt + rows + 1;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows + 1, 256), (int64_t)ctx->sm_count * 16));
    { plan_count<<<g, 256, 0, st>>>(row_ptr, rows, gram_tc_min_row(), cnt, ent); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    PTK_TRY(excl_scan_u32(ctx, cnt, cnt, rows + 1, st));
    PTK_TRY(excl_scan_u32(ctx, ent, ent, rows + 1, st));
    const int64_t cap = gram_tc_plan_capacity(nnz);
    const int gc = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cap, 256), (int64_t)ctx->sm_count * 16));
    { plan_emit<<<gc, 256, 0, st>>>(row_ptr, rows, cap, cnt, ent, plan); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    uint32_t tot[2];
    PTK_CUDA(cudaMemcpyAsync(&tot[0], cnt + rows, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaMemcpyAsync(&tot[1], ent + rows, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PTK_CUDA(cudaStreamSynchronize(st));
    *nchunks_h = tot[0];
    *long_entries_h = tot[1];
    return PTK_OK;
}

// capacity of a plan for `nnz` entries: a row of m >= TLONG entries has at
// most m / TLONG chunks
int64_t gram_tc_plan_capacity(int64_t nnz) { return nnz / gram_tc_min_row() + 1; }

bool gram_tc_supported(const GramJob& job) {
    return job.dtype == PTK_F32 && job.J >= 1 && job.J <= GT_C - 1 && job.tc_plan != nullptr && job.tc_nchunks > 0;
}

ptk_status gram_tc(ptk_ctx* ctx, const GramJob& job, cudaStream_t st) {
    if (!gram_tc_supported(job)) {
        set_error("gram_tc: needs FP32 sums, J <= 15 and a chunk plan with at least one chunk");
        return PTK_ERR_UNSUPPORTED;
    }
    switch (job.J) {
#define PTK_CASE(J) \
    case J:         \
        return job.digits == 3 ? launch_tc<J, 3>(ctx, job, st) : launch_tc<J, 4>(ctx, job, st);
        PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
        PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15)
#undef PTK_CASE
        default:
            return PTK_ERR_UNSUPPORTED;
    }
}

}  // namespace ptk
