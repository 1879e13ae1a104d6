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
