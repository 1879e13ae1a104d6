// delta_simt.cu -- Eq. (delta) on CUDA cores (FP32 or FP64).
//
// For the free mode n, every entry e gets
//     delta_e(j) = sum_{beta: j_n = j} G_beta prod_{k != n} a^(k)_{i_k j_k}.
// The core is permuted once per mode to Gp[j_n][q][j_L], where L is the last
// mode other than n and q runs over the remaining ("middle") modes in C order.
// Each thread evaluates two entries: for every q it forms the middle product
// w_q (one multiply per q with the innermost middle row), contracts the core
// fibre Gp[j_n][q][:] with the last-mode row (a J_L dot product) and adds
// w_q * dot to delta(j_n).  Core fibres are shared by the warp (broadcast
// shared-memory loads), so one 16-byte load feeds 8 FMAs.
#include <mutex>
#include <utility>

#include "common.cuh"

namespace ptk {

int delta_out_ld(int Jn) {
    // J_n values then x; an odd row length keeps the Gram kernel's per-thread
    // row walks free of shared-memory bank conflicts.
    int ld = Jn + 1;
    return (ld & 1) ? ld : ld + 1;
}

namespace {

constexpr int DT = 128;   // threads per block
// entries per thread: DN (2 or 4, a template parameter): each shared-memory
// core fibre feeds DN entries, more registers per thread
constexpr int MAXM = PTK_MAX_ORDER - 2;

template <typename T>
struct DeltaParams {
    int64_t n;
    const int32_t* col_last;
    const int32_t* col_inner;
    const int32_t* col_outer[MAXM];
    int64_t cstride;
    const T* f_last;
    int64_t ld_last;
    const T* f_inner;
    int64_t ld_inner;
    const T* f_outer[MAXM];
    int64_t ld_outer[MAXM];
    int J_outer[MAXM];
    int n_outer;          // outer middle modes (middle modes minus the innermost)
    int has_inner;        // 0 when the order is 2
    int jn, jl, ji;       // runtime sizes
    int64_t Q;            // product of middle-mode sizes
    int64_t Qouter;       // Q / ji
    int JLp;              // padded fibre length
    const T* Gp;          // [jn][Q][JLp]
    int use_smem;         // 1: the whole core is staged in shared memory once per block
    int64_t qo_chunk;     // else: outer-q indices per chunk streamed through shared memory
    int ctas_per_sm;      // grid: resident blocks per SM (0: occupancy limit)
    int dent;             // entries per thread (2 or 4)
    int64_t g_elems;
    const T* vals;
    T* out;
    int out_ld;
};

struct Dims8 {
    int J[PTK_MAX_ORDER];
};

template <typename T>
__global__ void permute_core(const T* __restrict__ G, int order, const Dims8 J8, int mode, int last, int64_t Q,
                             int JLp, T* __restrict__ Gp, int64_t total) {
    const int* J = J8.J;
    // Gp[jn][q][jl]; q digits are the middle modes in increasing mode order
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int jl = (int)(t % JLp);
        int64_t r = t / JLp;
        int64_t q = r % Q;
        int jn = (int)(r / Q);
        if (jl >= J[last]) {
            Gp[t] = T(0);
            continue;
        }
        int jj[PTK_MAX_ORDER];
        jj[mode] = jn;
        jj[last] = jl;
        int64_t rem = q;
        for (int k = order - 1; k >= 0; --k) {
            if (k == mode || k == last) continue;
            jj[k] = (int)(rem % J[k]);
            rem /= J[k];
        }
        int64_t src = 0;
        for (int k = 0; k < order; ++k) src = src * J[k] + jj[k];
        Gp[t] = G[src];
    }
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int W = 2;
};

template <typename T, int JN, int JL, int JI, bool EXACT, int DENT>
__global__ void __launch_bounds__(DT) delta_simt_kernel(const DeltaParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = Vec<T>::W;
    constexpr int JLV = (JL + W - 1) / W;  // vector loads per fibre
    using V = typename Vec<T>::V;
    T* sG = reinterpret_cast<T*>(smem_raw);
    const T* G = p.Gp;
    if (p.use_smem) {
        const V* src = reinterpret_cast<const V*>(p.Gp);
        V* dst = reinterpret_cast<V*>(sG);
        for (int64_t i = threadIdx.x; i < p.g_elems / W; i += DT) dst[i] = src[i];
        __syncthreads();
        G = sG;
    }
    const int jn_rt = EXACT ? JN : p.jn;
    const int jl_rt = EXACT ? JL : p.jl;
    const int ji_rt = EXACT ? JI : p.ji;
    const int64_t Q = p.Q;
    const int JLp = p.JLp;
    // A core larger than shared memory is streamed through it in chunks of
    // outer-q slabs (all j_n, all inner indices); each chunk serves the block's
    // DT * DENT entries before the next one is loaded.
    const int64_t QOC = p.use_smem ? p.Qouter : p.qo_chunk;
    for (int64_t tile = blockIdx.x; tile * (DT * DENT) < p.n; tile += gridDim.x) {
        int64_t e[DENT];
        bool ok[DENT];
        T al[DENT][JL];
        T acc[DENT][JN];
        const T* rin[DENT];
        const T* rout[DENT][MAXM];
#pragma unroll
        for (int i = 0; i < DENT; ++i) {
            e[i] = tile * (DT * DENT) + i * DT + threadIdx.x;
            ok[i] = e[i] < p.n;
            int64_t ee = ok[i] ? e[i] : 0;
            const T* rl = p.f_last + (int64_t)p.col_last[ee * p.cstride] * p.ld_last;
#pragma unroll
            for (int j = 0; j < JL; ++j) al[i][j] = (EXACT || j < jl_rt) ? rl[j] : T(0);
#pragma unroll
            for (int j = 0; j < JN; ++j) acc[i][j] = T(0);
            rin[i] = p.has_inner ? p.f_inner + (int64_t)p.col_inner[ee * p.cstride] * p.ld_inner : nullptr;
            for (int m = 0; m < p.n_outer; ++m)
                rout[i][m] = p.f_outer[m] + (int64_t)p.col_outer[m][ee * p.cstride] * p.ld_outer[m];
        }
        for (int64_t qo0 = 0; qo0 < p.Qouter; qo0 += QOC) {
            const int64_t qo1 = qo0 + QOC < p.Qouter ? qo0 + QOC : p.Qouter;
            int64_t Qs = Q, qbase = 0;  // q stride and first q of the fibres G points at
            if (!p.use_smem) {
                const int64_t qn = (qo1 - qo0) * ji_rt;
                __syncthreads();  // every thread is done with the previous chunk
                for (int jn = 0; jn < jn_rt; ++jn) {
                    const V* src = reinterpret_cast<const V*>(p.Gp + ((int64_t)jn * Q + qo0 * ji_rt) * JLp);
                    V* dst = reinterpret_cast<V*>(sG + (int64_t)jn * qn * JLp);
                    for (int64_t i = threadIdx.x; i < qn * JLp / W; i += DT) dst[i] = src[i];
                }
                __syncthreads();
                G = sG;
                Qs = qn;
                qbase = qo0 * ji_rt;
            }
            for (int64_t qo = qo0; qo < qo1; ++qo) {
                T pre[DENT];
#pragma unroll
                for (int i = 0; i < DENT; ++i) pre[i] = T(1);
                {
                    int64_t rem = qo;
                    for (int m = p.n_outer - 1; m >= 0; --m) {
                        int d = (int)(rem % p.J_outer[m]);
                        rem /= p.J_outer[m];
#pragma unroll
                        for (int i = 0; i < DENT; ++i) pre[i] *= rout[i][m][d];
                    }
                }
#pragma unroll 1
                for (int oi = 0; oi < ji_rt; ++oi) {
                    T w[DENT];
#pragma unroll
                    for (int i = 0; i < DENT; ++i) w[i] = p.has_inner ? pre[i] * rin[i][oi] : pre[i];
                    const int64_t q = qo * ji_rt + oi - qbase;
#pragma unroll
                    for (int jn = 0; jn < JN; ++jn) {
                        if (!EXACT && jn >= jn_rt) break;
                        const V* g = reinterpret_cast<const V*>(G + ((int64_t)jn * Qs + q) * JLp);
                        T gv[JLV * W];
#pragma unroll
                        for (int v = 0; v < JLV; ++v) {
                            // the fibre holds JLp = roundup(jl, W) elements: never read past it
                            V x;
                            if (EXACT || v * W < jl_rt) {
                                x = g[v];
                            } else {
                                if constexpr (W == 4) x = make_float4(0.f, 0.f, 0.f, 0.f);
                                else x = make_double2(0.0, 0.0);
                            }
                            if constexpr (W == 4) {
                                gv[4 * v + 0] = x.x; gv[4 * v + 1] = x.y; gv[4 * v + 2] = x.z; gv[4 * v + 3] = x.w;
                            } else {
                                gv[2 * v + 0] = x.x; gv[2 * v + 1] = x.y;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < DENT; ++i) {
                            T t = T(0);
#pragma unroll
                            for (int j = 0; j < JL; ++j) t = fma(gv[j], al[i][j], t);
                            acc[i][jn] = fma(w[i], t, acc[i][jn]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < DENT; ++i) {
            if (!ok[i]) continue;
            T* o = p.out + e[i] * p.out_ld;
#pragma unroll
            for (int j = 0; j < JN; ++j)
                if (EXACT || j < jn_rt) o[j] = acc[i][j];
            if (p.vals) o[jn_rt] = p.vals[e[i]];
        }
    }
}

// ---- sparse core ---------------------------------------------------------------
// P-Tucker-Approx (Sec. 3.3, Alg. 4) zeroes a share of the core entries every
// sweep so that the delta of Eq. (delta) costs time in proportion to nnz(G),
// not |G|: the sum runs over the non-zero beta only, each a product of N - 1
// factor entries and G_beta.  The dense kernel above streams every core fibre
// whatever it holds; this path visits the non-zeros.  The permuted core
// Gp[j_n][q][j_L] is compacted once per launch into records of its non-zero
// entries, ordered by j_n: G_beta and the positions, in a thread's rows, of
// the N - 1 factor entries it multiplies (j_L in the last mode's row, the q
// digits in the middle modes' rows).  Each thread copies the factor rows of
// its SP_W entries to its own block of shared memory, their values of one
// row element side by side, and for every j_n sums G_beta times the
// product of the N - 1 row values over that j_n's records: per record one
// broadcast load, N - 1 vector loads (all the thread's entries at once) and N - 1
// multiplies per entry, with no per-fibre state or branch.
constexpr int SP_THREADS = 1024;  // compaction block
constexpr int SP_MAXF = 12;       // factor positions a record holds (N - 1 <= PTK_MAX_ORDER - 1)
constexpr int SP_W = 2;           // entries per thread: one 8-byte vector per row element

// Orders up to 4 (at most three factors): the factors' byte offsets in a
// thread's rows as words; higher orders: their positions as bytes.
struct SpRec {
    float g;
    union {
        int off[3];
        uint8_t pos[SP_MAXF];
    };
};
static_assert(sizeof(SpRec) == 16, "one record per 16-byte load");

// middle modes in q digit order (outer modes, then the inner mode, fastest)
struct SpDigits {
    int J[PTK_MAX_ORDER];
    int off[PTK_MAX_ORDER];  // position of the mode's row in a thread's rows
    int n;
};

// One block.  For each j_n in turn, thread t takes q in [Q t / B, Q (t + 1) / B)
// and writes its non-zeros after those of the threads before it; jstart[j] is
// the first record of j_n = j.  More than cap records: none are kept, jstart
// stays zero (no delta terms) and FLAG_SPARSE is raised.
__global__ void __launch_bounds__(SP_THREADS) compact_core(const float* __restrict__ Gp, int jn, int64_t Q, int JLp,
                                                           int jl, SpDigits dg, SpRec* __restrict__ rec,
                                                           int* __restrict__ jstart, int cap, int* __restrict__ flags) {
    __shared__ int sc[SP_THREADS];
    __shared__ int base_s;
    const int t = threadIdx.x;
    const int64_t q0 = Q * t / SP_THREADS, q1 = Q * (t + 1) / SP_THREADS;
    if (t == 0) base_s = 0;
    for (int j = 0; j <= jn; ++j)
        if (t == 0) jstart[j] = 0;
    __syncthreads();
    for (int j = 0; j < jn; ++j) {
        const float* f = Gp + (int64_t)j * Q * JLp;
        int c = 0;
        for (int64_t q = q0; q < q1; ++q)
            for (int l = 0; l < jl; ++l) c += f[q * JLp + l] != 0.f;
        sc[t] = c;
        __syncthreads();
        for (int off = 1; off < SP_THREADS; off <<= 1) {  // inclusive scan
            const int v = t >= off ? sc[t - off] : 0;
            __syncthreads();
            sc[t] += v;
            __syncthreads();
        }
        const int base = base_s, total = sc[SP_THREADS - 1];
        if (base + total > cap) {
            if (t == 0) {
                for (int k = 0; k <= jn; ++k) jstart[k] = 0;
                atomicAdd(&flags[FLAG_SPARSE], 1);
            }
            return;  // uniform: every thread read the same totals
        }
        int w = base + sc[t] - c;
        for (int64_t q = q0; q < q1; ++q)
            for (int l = 0; l < jl; ++l) {
                const float g = f[q * JLp + l];
                if (g == 0.f) continue;
                int pos[SP_MAXF];
                pos[0] = l;  // the last mode's row starts at position 0
                int64_t rem = q;
                for (int m = dg.n - 1; m >= 0; --m) {
                    pos[1 + m] = dg.off[m] + (int)(rem % dg.J[m]);
                    rem /= dg.J[m];
                }
                SpRec r;
                r.g = g;
                for (int k = 0; k < SP_MAXF; ++k) r.pos[k] = 0;
                if (dg.n + 1 <= 3) {
                    for (int k = 0; k <= dg.n; ++k) r.off[k] = 4 * SP_W * pos[k];  // byte offsets of row vectors
                } else {
                    for (int k = 0; k <= dg.n; ++k) r.pos[k] = (uint8_t)pos[k];
                }
                rec[w++] = r;
            }
        __syncthreads();  // every thread has read base_s and sc
        if (t == 0) {
            base_s = base + total;
            jstart[j + 1] = base + total;
        }
        __syncthreads();
    }
}

struct SpLayout {
    int cap;       // records the shared-memory layout holds
    int off_rows;  // byte offset of the rows (after the records and jstart), a multiple of 16
    int nf;        // factors per record: N - 1
    int RL;        // row elements per entry: J_L + middle-mode ranks
    int RS;        // row vectors per thread (odd, >= RL)
    int off_inner;
    int off_outer[PTK_MAX_ORDER];
};

// SP_W = 2 entries per thread: one float2 per row element (a thread's rows
// then take half the shared memory of four entries: about twice the resident
// warps, for a walk that waits on its dependent loads).  NF = N - 1 factors
// per record (0: taken from the layout at run time).
template <int JN, int NF>
__global__ void __launch_bounds__(DT) delta_sparse_kernel(const DeltaParams<float> p, const SpLayout L,
                                                          const SpRec* __restrict__ rec,
                                                          const int* __restrict__ jstart) {
    constexpr int W = SP_W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpRec* sRec = reinterpret_cast<SpRec*>(smem_raw);
    int* sJ = reinterpret_cast<int*>(sRec + L.cap);
    float2* sRow = reinterpret_cast<float2*>(smem_raw + L.off_rows);
    const int nrec = jstart[p.jn];
    for (int i = threadIdx.x; i < nrec; i += DT) sRec[i] = rec[i];
    for (int i = threadIdx.x; i <= p.jn; i += DT) sJ[i] = jstart[i];
    __syncthreads();
    const int nf = NF > 0 ? NF : L.nf;
    float2* const mine = sRow + (int64_t)threadIdx.x * L.RS;  // element r of the W entries at mine[r]
    float* const mine_s = reinterpret_cast<float*>(mine);
    for (int64_t tile = blockIdx.x; tile * (DT * W) < p.n; tile += gridDim.x) {
        int64_t e[W];
        bool ok[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            e[i] = tile * (DT * W) + i * DT + threadIdx.x;
            ok[i] = e[i] < p.n;
            const int64_t ee = ok[i] ? e[i] : 0;
            const float* rl = p.f_last + (int64_t)p.col_last[ee * p.cstride] * p.ld_last;
            for (int j = 0; j < p.jl; ++j) mine_s[j * W + i] = rl[j];
            if (p.has_inner) {
                const float* ri = p.f_inner + (int64_t)p.col_inner[ee * p.cstride] * p.ld_inner;
                for (int j = 0; j < p.ji; ++j) mine_s[(L.off_inner + j) * W + i] = ri[j];
            }
            for (int m = 0; m < p.n_outer; ++m) {
                const float* ro = p.f_outer[m] + (int64_t)p.col_outer[m][ee * p.cstride] * p.ld_outer[m];
                for (int j = 0; j < p.J_outer[m]; ++j) mine_s[(L.off_outer[m] + j) * W + i] = ro[j];
            }
        }
        float acc[W][JN];
        const unsigned char* const mb = reinterpret_cast<const unsigned char*>(mine);
        auto row = [&](const SpRec& r, int k) -> float2 {
            if constexpr (NF >= 1 && NF <= 3)
                return *reinterpret_cast<const float2*>(mb + r.off[k]);
            else
                return mine[r.pos[k]];
        };
        auto term = [&](const SpRec& r, float2& t) {  // t += G_beta * prod of the record's row values
            float2 v = row(r, 0);
            float2 pr = make_float2(r.g * v.x, r.g * v.y);
#pragma unroll
            for (int k = 1; k < (NF > 0 ? NF : SP_MAXF); ++k) {
                if (NF == 0 && k >= nf) break;
                v = row(r, k);
                pr.x *= v.x;
                pr.y *= v.y;
            }
            t.x += pr.x;
            t.y += pr.y;
        };
#pragma unroll
        for (int j = 0; j < JN; ++j) {
            float2 t0 = make_float2(0.f, 0.f), t1 = t0;
            if (j < p.jn) {
                int r = sJ[j];
                const int r1 = sJ[j + 1];
                for (; r + 1 < r1; r += 2) {  // two independent sums
                    const SpRec a = sRec[r], b = sRec[r + 1];
                    term(a, t0);
                    term(b, t1);
                }
                if (r < r1) term(sRec[r], t0);
            }
            acc[0][j] = t0.x + t1.x;
            acc[1][j] = t0.y + t1.y;
        }
#pragma unroll
        for (int i = 0; i < W; ++i) {
            if (!ok[i]) continue;
            float* o = p.out + e[i] * p.out_ld;
#pragma unroll
            for (int j = 0; j < JN; ++j)
                if (j < p.jn) o[j] = acc[i][j];
            if (p.vals) o[p.jn] = p.vals[e[i]];
        }
    }
}

// Streamed core: as many outer-q slabs (all j_n and inner indices) per chunk
// as `kb` KB of shared memory hold (kb <= 0: 48 KB).
template <typename T>
void set_chunk(DeltaParams<T>& p, int kb) {
    const size_t slab = (size_t)p.jn * p.ji * p.JLp * sizeof(T);
    const size_t budget = (size_t)(kb > 0 ? kb : 48) * 1024;
    p.qo_chunk = std::max<int64_t>(1, std::min<int64_t>(p.Qouter, (int64_t)(budget / slab)));
}

// What a launch needs to know about the device.  `raised`: every kernel
// instantiation this launch can reach already accepts kMaxStagedCore bytes of
// dynamic shared memory (set once per device), so no attribute is read or set.
struct LaunchLimits {
    int sm_count = 0;
    size_t smem_optin = 0;
    bool raised = false;
};
inline LaunchLimits limits_of(const ptk_ctx* ctx) {
    LaunchLimits l;
    l.sm_count = ctx->sm_count;
    l.smem_optin = ctx->smem_optin;
    return l;
}
// largest core staged whole in shared memory (larger cores are streamed in
// chunks of at most 48 KB unless the autotuner picked a larger chunk)
constexpr size_t kMaxStagedCore = 100 * 1024;

template <typename T, int JN, int JL, int JI, bool EXACT, int DENT>
ptk_status launch_delta(const LaunchLimits& lim, const DeltaParams<T>& p, cudaStream_t st) {
    const size_t smem = p.use_smem ? (size_t)p.g_elems * sizeof(T)
                                   : (size_t)p.jn * p.qo_chunk * p.ji * p.JLp * sizeof(T);
    auto kern = delta_simt_kernel<T, JN, JL, JI, EXACT, DENT>;
    if (smem > 48 * 1024 && !lim.raised) PTK_TRY(smem_attr((const void*)kern, smem, st));
    int per_sm = 0;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DT, smem));
    if (per_sm < 1) per_sm = 1;
    if (p.ctas_per_sm > 0) per_sm = std::min(per_sm, p.ctas_per_sm);
    int64_t tiles = ceil_div(p.n, DT * DENT);
    int64_t grid = std::min<int64_t>(tiles, (int64_t)lim.sm_count * per_sm);
    if (grid < 1) grid = 1;
    { kern<<<(unsigned)grid, DT, smem, st>>>(p); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

template <typename T, int DENT>
ptk_status dispatch_dent(const LaunchLimits& lim, const DeltaParams<T>& p, bool uniform, cudaStream_t st) {
    if (uniform) {
        switch (p.jn) {
#define PTK_CASE(J) \
    case J:         \
        return launch_delta<T, J, J, J, true, DENT>(lim, p, st);
            PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
            PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15)
            PTK_CASE(16)
#undef PTK_CASE
            default: break;
        }
    }
    return launch_delta<T, PTK_MAX_RANK, PTK_MAX_RANK, PTK_MAX_RANK, false, DENT>(lim, p, st);
}

// Four entries per thread halve the shared-memory core reads per entry and
// pay off once the core is large; FP64 (small problems) keeps two.
template <typename T>
ptk_status dispatch(const LaunchLimits& lim, const DeltaParams<T>& p, bool uniform, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        const int dent = p.dent > 0 ? p.dent : (p.g_elems >= 4096 ? 4 : 2);
        if (dent == 4) return dispatch_dent<T, 4>(lim, p, uniform, st);
    }
    return dispatch_dent<T, 2>(lim, p, uniform, st);
}

// The sparse path where it pays: the records and every thread's rows fit in
// shared memory and the non-zeros are few.  The walk is bound by shared-memory
// bandwidth: per entry and record it reads N - 1 row values (4 bytes each) of
// the entry's own rows, 128 bytes per cycle per SM, so at most 32 / (N - 1)
// entry-records per SM cycle (10.7 at order 4; 8.6 measured on the 4-order
// Zipf workload).  The dense kernel keeps the rows in registers and reads the
// core by broadcast: about 100 entry-elements per SM cycle measured (one FMA
// and a little per element).  So the walk is taken when nnz(G) (N - 1) * 3.1
// < 0.9 |G|: below about 15 % of the core at order 3, 10 % at order 4.
constexpr double kSparseCostPerFactor = 3.1;

template <int JN, int NF>
ptk_status launch_sparse(ptk_ctx* ctx, const DeltaParams<float>& p, const SpLayout& L, const SpRec* rec,
                         const int* jstart, size_t smem, cudaStream_t st) {
    auto kern = delta_sparse_kernel<JN, NF>;
    if (smem > 48 * 1024) PTK_TRY(smem_attr((const void*)kern, smem, st));
    int per_sm = 0;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DT, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = ceil_div(p.n, DT * SP_W);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->sm_count * per_sm));
    { kern<<<(unsigned)grid, DT, smem, st>>>(p, L, rec, jstart); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

template <int JN>
ptk_status launch_sparse_nf(ptk_ctx* ctx, const DeltaParams<float>& p, const SpLayout& L, const SpRec* rec,
                            const int* jstart, size_t smem, cudaStream_t st) {
    if (L.nf == 1) return launch_sparse<JN, 1>(ctx, p, L, rec, jstart, smem, st);
    if (L.nf == 2) return launch_sparse<JN, 2>(ctx, p, L, rec, jstart, smem, st);
    if (L.nf == 3) return launch_sparse<JN, 3>(ctx, p, L, rec, jstart, smem, st);
    return launch_sparse<JN, 0>(ctx, p, L, rec, jstart, smem, st);  // positions as bytes, N - 1 > 3
}

// PTK_OK with *taken = false when the sparse path does not apply.
ptk_status run_sparse(ptk_ctx* ctx, const DeltaParams<float>& p, int order, int64_t core_nnz, bool* taken,
                      cudaStream_t st) {
    *taken = false;
    const int nf = order - 1;
    const int64_t cells = (int64_t)p.jn * p.Q * p.jl;  // |G|
    const double sparse_cost = (double)core_nnz * nf * kSparseCostPerFactor, dense_cost = (double)cells;
    if (core_nnz < 0 || sparse_cost > 0.9 * dense_cost || nf > SP_MAXF || p.jn > 16 || p.Q > (1ll << 30))
        return PTK_OK;
    SpDigits dg{};
    SpLayout L{};
    int nmid = 0;
    L.RL = p.jl;
    if (p.has_inner) {
        int pos = p.jl + p.ji;  // outer middle rows follow the last-mode and inner rows
        for (int m = 0; m < p.n_outer; ++m) {
            dg.J[nmid] = p.J_outer[m];
            dg.off[nmid] = pos;
            L.off_outer[m] = pos;
            pos += p.J_outer[m];
            ++nmid;
        }
        dg.J[nmid] = p.ji;  // the inner mode is the fastest q digit
        dg.off[nmid] = p.jl;
        L.off_inner = p.jl;
        ++nmid;
        L.RL = pos;
    }
    dg.n = nmid;
    if (L.RL > 255 || 1 + nmid != nf) return PTK_OK;
    L.nf = nf;
    L.RS = L.RL | 1;  // odd: a warp's vector loads at one position hit distinct banks
    L.cap = (int)std::max<int64_t>(core_nnz, 1);
    L.off_rows = (int)(((size_t)L.cap * sizeof(SpRec) + (size_t)(p.jn + 1) * sizeof(int) + 15) / 16 * 16);
    const size_t smem = (size_t)L.off_rows + (size_t)DT * L.RS * 4 * SP_W;
    if (smem > ctx->smem_optin) return PTK_OK;
    unsigned char* buf = (unsigned char*)scratch(ctx, SLOT_SPARSE, (size_t)L.off_rows + 64);
    if (!buf) return PTK_ERR_OUT_OF_MEMORY;
    SpRec* rec = reinterpret_cast<SpRec*>(buf);
    int* jstart = reinterpret_cast<int*>(buf + (size_t)L.cap * sizeof(SpRec));
    { compact_core<<<1, SP_THREADS, 0, st>>>(p.Gp, p.jn, p.Q, p.JLp, p.jl, dg, rec, jstart, L.cap, ctx->d_flags);
      ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    *taken = true;
    if (p.jn <= 4) return launch_sparse_nf<4>(ctx, p, L, rec, jstart, smem, st);
    if (p.jn <= 8) return launch_sparse_nf<8>(ctx, p, L, rec, jstart, smem, st);
    if (p.jn <= 12) return launch_sparse_nf<12>(ctx, p, L, rec, jstart, smem, st);
    return launch_sparse_nf<16>(ctx, p, L, rec, jstart, smem, st);
}

template <typename T>
ptk_status run(ptk_ctx* ctx, const DeltaJob& job, cudaStream_t st) {
    const int N = job.order, n = job.mode;
    int others[PTK_MAX_ORDER], no = 0;
    for (int k = 0; k < N; ++k)
        if (k != n) others[no++] = k;
    if (no < 1) {
        set_error("delta: order must be >= 2");
        return PTK_ERR_INVALID_ARG;
    }
    const int last = others[no - 1];
    DeltaParams<T> p{};
    p.n = job.n;
    p.cstride = job.cstride;
    p.col_last = job.col[last];
    p.f_last = (const T*)job.factors[last];
    p.ld_last = job.ld[last];
    p.jn = job.J[n];
    p.jl = job.J[last];
    p.Q = 1;
    for (int m = 0; m < no - 1; ++m) p.Q *= job.J[others[m]];
    if (no >= 2) {
        int inner = others[no - 2];
        p.has_inner = 1;
        p.col_inner = job.col[inner];
        p.f_inner = (const T*)job.factors[inner];
        p.ld_inner = job.ld[inner];
        p.ji = job.J[inner];
        p.n_outer = no - 2;
        for (int m = 0; m < no - 2; ++m) {
            p.col_outer[m] = job.col[others[m]];
            p.f_outer[m] = (const T*)job.factors[others[m]];
            p.ld_outer[m] = job.ld[others[m]];
            p.J_outer[m] = job.J[others[m]];
        }
    } else {
        p.has_inner = 0;
        p.ji = 1;
        p.n_outer = 0;
    }
    p.Qouter = p.Q / p.ji;
    constexpr int W = Vec<T>::W;
    p.JLp = (p.jl + W - 1) / W * W;
    p.g_elems = (int64_t)p.jn * p.Q * p.JLp;
    T* Gp = (T*)scratch(ctx, SLOT_GPERM, sizeof(T) * (size_t)p.g_elems + 64);
    if (!Gp) return PTK_ERR_OUT_OF_MEMORY;
    Dims8 dJ;
    for (int k = 0; k < PTK_MAX_ORDER; ++k) dJ.J[k] = job.J[k];
    {
        int64_t total = p.g_elems;
        int64_t g = std::min<int64_t>(ceil_div(total, 256), (int64_t)ctx->sm_count * 8);
        { permute_core<T><<<(unsigned)std::max<int64_t>(g, 1), 256, 0, st>>>((const T*)job.core, N, dJ, n, last, p.Q,
                                                                          p.JLp, Gp, total); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
    }
    p.Gp = Gp;
    p.use_smem = (size_t)p.g_elems * sizeof(T) <= std::min<size_t>(ctx->smem_optin, kMaxStagedCore);
    set_chunk(p, job.chunk_kb);
    p.ctas_per_sm = job.ctas_per_sm;
    p.dent = job.dent;
    p.vals = (const T*)job.vals;
    p.out = (T*)job.out;
    p.out_ld = job.out_ld;
    if (p.n == 0) return PTK_OK;
    if constexpr (sizeof(T) == 4) {
        if (job.core_nnz >= 0) {  // a truncated core (Approx, FP32): walk its non-zeros where that is shorter
            bool taken = false;
            PTK_TRY(run_sparse(ctx, p, N, job.core_nnz, &taken, st));
            if (taken) return PTK_OK;
        }
    }
    bool uniform = p.jn == p.jl && (p.has_inner ? p.ji == p.jn : false);
    return dispatch<T>(limits_of(ctx), p, uniform, st);
}

}  // namespace

ptk_status delta_simt(ptk_ctx* ctx, const DeltaJob& job, cudaStream_t st) {
    if (job.dtype == PTK_F64) return run<double>(ctx, job, st);
    return run<float>(ctx, job, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the CUDA-core delta launch.  The permuted core,
// which delta_simt keeps in context scratch, lives here in a file-scope device
// array instead, so a call allocates and frees nothing.  The array is shared by
// every call on a device and keeps the previous call's contents; permute_core
// rewrites every element the kernel reads (including the zero padding), so
// nothing has to be cleared.  Calls that overlap on the GPU (different streams
// or threads) race on the array.
namespace {

constexpr size_t kStaticCoreBytes = 512 * 1024;
__device__ __align__(256) unsigned char g_static_core[kStaticCoreBytes];

struct StaticDevice {
    bool ready = false;
    void* core = nullptr;  // device address of g_static_core on this device
    LaunchLimits lim;      // SM count, shared-memory limit; attributes raised
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;

// Lets one kernel instantiation take `bytes` of dynamic shared memory.
template <typename T, int JN, int JL, int JI, bool EXACT, int DENT>
ptk_status raise_one(int bytes) {
    PTK_CUDA(cudaFuncSetAttribute((const void*)delta_simt_kernel<T, JN, JL, JI, EXACT, DENT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return PTK_OK;
}
// Every instantiation dispatch<T> can reach: uniform ranks 1..16 and the
// general kernel, for each entries-per-thread count of the type.
template <typename T, int DENT, int... Js>
ptk_status raise_dent(int bytes, std::integer_sequence<int, Js...>) {
    ptk_status s = raise_one<T, PTK_MAX_RANK, PTK_MAX_RANK, PTK_MAX_RANK, false, DENT>(bytes);
    ((s = (s == PTK_OK ? raise_one<T, Js + 1, Js + 1, Js + 1, true, DENT>(bytes) : s)), ...);
    return s;
}
ptk_status raise_all(int bytes) {
    const auto ranks = std::make_integer_sequence<int, PTK_MAX_RANK>{};
    ptk_status s = raise_dent<float, 2>(bytes, ranks);
    if (s == PTK_OK) s = raise_dent<float, 4>(bytes, ranks);
    if (s == PTK_OK) s = raise_dent<double, 2>(bytes, ranks);
    return s;
}

// Once per device, with that device current: the array's device address (the
// host-side symbol is only a stand-in), the launch limits, and the shared-
// memory attribute of every reachable kernel, so that later calls read or set
// no attribute.
ptk_status static_device(int dev, StaticDevice** out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device %d out of range", dev);
        return PTK_ERR_INVALID_ARG;
    }
    StaticDevice& d = g_static_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        PTK_CUDA(cudaGetSymbolAddress(&ptr, g_static_core));
        int sms = 0, optin = 0;
        PTK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PTK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // the largest staged core run_static can ask for (streamed chunks stay at 48 KB)
        PTK_TRY(raise_all((int)std::min<size_t>((size_t)optin, kMaxStagedCore)));
        d.core = ptr;
        d.lim.sm_count = sms;
        d.lim.smem_optin = (size_t)optin;
        d.lim.raised = true;
        d.ready = true;
    }
    *out = &d;
    return PTK_OK;
}

template <typename T>
ptk_status run_static(const StaticDevice& sd, const DeltaJob& job, cudaStream_t st) {
    const int N = job.order, n = job.mode;
    int others[PTK_MAX_ORDER], no = 0;
    for (int k = 0; k < N; ++k)
        if (k != n) others[no++] = k;
    const int last = others[no - 1];
    DeltaParams<T> p{};
    p.n = job.n;
    p.cstride = job.cstride;
    p.col_last = job.col[last];
    p.f_last = (const T*)job.factors[last];
    p.ld_last = job.ld[last];
    p.jn = job.J[n];
    p.jl = job.J[last];
    p.Q = 1;
    for (int m = 0; m < no - 1; ++m) p.Q *= job.J[others[m]];
    if (no >= 2) {
        const int inner = others[no - 2];
        p.has_inner = 1;
        p.col_inner = job.col[inner];
        p.f_inner = (const T*)job.factors[inner];
        p.ld_inner = job.ld[inner];
        p.ji = job.J[inner];
        p.n_outer = no - 2;
        for (int m = 0; m < no - 2; ++m) {
            p.col_outer[m] = job.col[others[m]];
            p.f_outer[m] = (const T*)job.factors[others[m]];
            p.ld_outer[m] = job.ld[others[m]];
            p.J_outer[m] = job.J[others[m]];
        }
    } else {
        p.has_inner = 0;
        p.ji = 1;
        p.n_outer = 0;
    }
    p.Qouter = p.Q / p.ji;
    constexpr int W = Vec<T>::W;
    p.JLp = (p.jl + W - 1) / W * W;
    p.g_elems = (int64_t)p.jn * p.Q * p.JLp;
    if ((size_t)p.g_elems * sizeof(T) > kStaticCoreBytes) {
        set_error("ptk_delta_noalloc: the permuted core needs %lld bytes, the static scratch holds %zu",
                  (long long)((size_t)p.g_elems * sizeof(T)), kStaticCoreBytes);
        return PTK_ERR_INVALID_ARG;
    }
    T* Gp = (T*)sd.core;
    Dims8 dJ;
    for (int k = 0; k < PTK_MAX_ORDER; ++k) dJ.J[k] = job.J[k];
    {
        const int64_t total = p.g_elems;
        const int64_t g = std::min<int64_t>(ceil_div(total, 256), (int64_t)sd.lim.sm_count * 8);
        { permute_core<T><<<(unsigned)std::max<int64_t>(g, 1), 256, 0, st>>>((const T*)job.core, N, dJ, n, last,
                                                                            p.Q, p.JLp, Gp, total); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
    }
    p.Gp = Gp;
    p.use_smem = (size_t)p.g_elems * sizeof(T) <= std::min<size_t>(sd.lim.smem_optin, kMaxStagedCore);
    set_chunk(p, 0);
    p.ctas_per_sm = 0;
    p.dent = 0;
    p.vals = nullptr;
    p.out = (T*)job.out;
    p.out_ld = job.out_ld;
    const bool uniform = p.jn == p.jl && (p.has_inner ? p.ji == p.jn : false);
    return dispatch<T>(sd.lim, p, uniform, st);
}

}  // namespace
}  // namespace ptk

extern "C" ptk_status ptk_delta_noalloc(const ptk_model* m, int32_t mode, const int32_t* coords, int64_t n, void* out,
                                        ptk_stream_t stream) {
    using namespace ptk;
    PTK_TRY(check_model(m));
    PTK_CHECK_ARG(mode >= 0 && mode < m->order, "mode out of range");
    PTK_CHECK_ARG(n >= 0 && n < (1ll << 31), "n out of range");
    if (n == 0) return PTK_OK;  // nothing to compute: no set-up, no launch, the array is untouched
    PTK_CHECK_ARG(coords && out, "null arrays");
    int dev = 0;
    PTK_CUDA(cudaGetDevice(&dev));
    StaticDevice* sd = nullptr;
    PTK_TRY(static_device(dev, &sd));
    DeltaJob job;
    job.n = n;
    job.order = m->order;
    job.mode = mode;
    for (int k = 0; k < m->order; ++k) {
        job.col[k] = coords + k;
        job.factors[k] = m->factors[k];
        job.ld[k] = m->ld[k];
        job.J[k] = m->J[k];
    }
    job.cstride = m->order;
    job.core = m->core;
    job.out = out;
    job.out_ld = m->J[mode];
    job.dtype = m->dtype;
    if (m->dtype == PTK_F64) return run_static<double>(*sd, job, (cudaStream_t)stream);
    return run_static<float>(*sd, job, (cudaStream_t)stream);
}
