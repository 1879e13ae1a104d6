// delta_tc.cu -- Eq. (delta) on the 5th-generation tensor cores (tcgen05).
//
// For the free mode n, split the other modes into a Kronecker group K (all of
// them but the last) and the last other mode L.  Then
//     delta_e(j_n) = sum_{j_L} a^(L)_{i_L j_L} * D_e(j_n, j_L),
//     D_e(j_n, j_L) = sum_k A_e(k) Gb((j_n, j_L), k),
// where A_e(k) = prod_{m in K} a^(m)_{i_m k_m} is the Kronecker product of the
// entry's K-group factor rows and Gb is the core reshaped to [(j_n, j_L)][k].
// D = A Gb^T is a dense contraction: a 128-entry tile is one
// tcgen05.mma (M = 128, N = J_n*J_L padded to 16, K = prod_{m in K} J_m
// padded to the instruction K) with BF16 or TF32 operands and FP32
// accumulation in tensor memory.  CUDA cores build A (one entry per thread,
// written straight into shared memory in the canonical K-major no-swizzle
// layout) and contract D with the L-mode row after tcgen05.ld.
//
// Pipeline: two warpgroups per CTA take alternate tiles, each with its own A
// buffer and TMEM accumulator, so one group's MMAs run while the other builds
// its next operand or runs its epilogue.  Gb is copied to shared memory once
// per CTA.  Every wait is bounded: on timeout the kernel records
// FLAG_TIMEOUT, drains, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "common.cuh"

namespace ptk {
namespace {

constexpr int TC_M = 128;          // entries per tile (MMA M)
constexpr int TC_THREADS = 256;    // two warpgroups
constexpr long long TC_SPIN = 1ll << 24;

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    // tcgen05 shared-memory descriptor: start, leading / stride byte offsets
    // (>> 4), descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
    const uint32_t a = smem_u32(p);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// kind::f16 / kind::tf32 instruction descriptor: FP32 accumulator, A and B
// of type `ab` (1 = BF16, 2 = TF32), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int ab, int M, int N) {
    return (1u << 4) | ((uint32_t)ab << 7) | ((uint32_t)ab << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t to_tf32(float a) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return r;
}

// ---- shapes -----------------------------------------------------------------
// Layout of a K-major operand with R rows: 16-byte chunks of KPG elements;
// chunk (row, kc) at (row/8)*SBO + kc*128 + (row%8)*16 with SBO = KCH*128.
template <bool TF32>
struct Elt {
    static constexpr int ESZ = TF32 ? 4 : 2;
    static constexpr int KPG = 16 / ESZ;      // elements per 16-byte chunk
    static constexpr int MMA_K = TF32 ? 8 : 16;
};

struct TcParams {
    int64_t n;
    const int32_t* col_k[3];     // coordinate columns of the K-group modes
    const float* f_k[3];
    int64_t ld_k[3];
    const int32_t* col_l;
    const float* f_l;
    int64_t ld_l;
    int64_t cstride;
    const float* vals;
    float* out;
    int out_ld;
    const uint8_t* b_image;      // Gb in the shared-memory layout
    int b_bytes;
    int* flags;
};

template <int J, int NK, bool TF32>
struct TcCfg {
    using E = Elt<TF32>;
    static constexpr int K = NK == 1 ? J : (NK == 2 ? J * J : J * J * J);
    static constexpr int KP = (K + E::MMA_K - 1) / E::MMA_K * E::MMA_K;
    static constexpr int KCH = KP / E::KPG;            // 16-byte chunks per row
    static constexpr int NN = J * J;                   // (j_n, j_L) pairs
    static constexpr int NP = (NN + 15) / 16 * 16;     // MMA N
    static constexpr int NCOL = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);  // TMEM columns per accumulator
    static constexpr int SBO = KCH * 128;
    static constexpr int A_BYTES = TC_M * KP * E::ESZ;
    static constexpr int B_BYTES = NP * KP * E::ESZ;
    static constexpr int SMEM = B_BYTES + 2 * A_BYTES + 128;
    static constexpr int KSTEPS = KP / E::MMA_K;
    static_assert(NP <= 128, "accumulator wider than 128 columns");
};

template <int J, int NK, bool TF32>
__global__ void __launch_bounds__(TC_THREADS, 2) delta_tc_kernel(const TcParams p) {
    using C = TcCfg<J, NK, TF32>;
    using E = typename C::E;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* sB = smem;
    uint8_t* sA0 = smem + C::B_BYTES;
    __shared__ uint64_t bar_done[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int tid = threadIdx.x;
    const int g = tid >> 7;            // warpgroup
    const int tg = tid & 127;          // row of the tile
    const int warp = tid >> 5;
    uint8_t* sA = sA0 + g * C::A_BYTES;

    // Gb -> shared memory (plain 16-byte copies, then hand it to the async proxy)
    for (int i = tid * 16; i < p.b_bytes; i += TC_THREADS * 16)
        *reinterpret_cast<uint4*>(sB + i) = *reinterpret_cast<const uint4*>(p.b_image + i);
    if (tid == 0) {
        mbar_init(&bar_done[0], 1);
        mbar_init(&bar_done[1], 1);
        fence_mbar_init();
        abort_s = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(2 * C::NCOL)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s + (uint32_t)(g * C::NCOL);
    const uint32_t idesc = instr_desc(TF32 ? 2 : 1, TC_M, C::NP);

    const int64_t ntiles = ceil_div_dev(p.n, TC_M);
    int it = 0;
    bool ok = true;
    for (int64_t tile = (int64_t)blockIdx.x * 2 + g; tile < ntiles; tile += (int64_t)gridDim.x * 2, ++it) {
        const int64_t e = tile * TC_M + tg;
        const bool valid = e < p.n;
        const int64_t ee = valid ? e : 0;
        // ---- gather the entry's rows ------------------------------------
        float rk[NK][J];
#pragma unroll
        for (int m = 0; m < NK; ++m) {
            const float* r = p.f_k[m] + (int64_t)p.col_k[m][ee * p.cstride] * p.ld_k[m];
#pragma unroll
            for (int j = 0; j < J; ++j) rk[m][j] = valid ? r[j] : 0.f;
        }
        float al[J];
        {
            const float* r = p.f_l + (int64_t)p.col_l[ee * p.cstride] * p.ld_l;
#pragma unroll
            for (int j = 0; j < J; ++j) al[j] = r[j];
        }
        const float xval = (valid && p.vals) ? p.vals[e] : 0.f;
        // ---- A row: Kronecker product of the K-group rows ----------------
        uint8_t* arow = sA + (tg >> 3) * C::SBO + (tg & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < C::KCH; ++kc) {
            float v[E::KPG];
#pragma unroll
            for (int t = 0; t < E::KPG; ++t) {
                const int k = kc * E::KPG + t;
                float a = 0.f;
                if (k < C::K) {
                    if constexpr (NK == 1) {
                        a = rk[0][k];
                    } else if constexpr (NK == 2) {
                        a = rk[0][k / J] * rk[1][k % J];
                    } else {
                        a = rk[0][k / (J * J)] * rk[1][(k / J) % J] * rk[2][k % J];
                    }
                }
                v[t] = a;
            }
            uint4 w;
            if constexpr (TF32) {
                w = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
            } else {
                w = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                               pack_bf16(v[6], v[7]));
            }
            *reinterpret_cast<uint4*>(arow + kc * 128) = w;
        }
        fence_proxy_async_smem();
        named_bar(1 + g, 128);
        // ---- MMAs of this tile (one thread of the group) -------------------
        if (tg == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < C::KSTEPS; ++ks) {
                const uint64_t ad = smem_desc(sA + ks * 256, 128, C::SBO);
                const uint64_t bd = smem_desc(sB + ks * 256, 128, C::SBO);
                mma<TF32>(tmem, ad, bd, idesc, ks > 0);
            }
            mma_commit(&bar_done[g]);
        }
        // ---- epilogue --------------------------------------------------------
        if (!mbar_wait_bounded(&bar_done[g], (unsigned)(it & 1), p.flags, TC_SPIN)) {
            ok = false;
            break;
        }
        tc_fence_after();
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        float dl[J];
#pragma unroll
        for (int jn = 0; jn < J; ++jn) dl[jn] = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < C::NP; c0 += 16) {
            float d[16];
            tmem_ld16(lane_addr + c0, d);
            tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int c = c0 + t;  // column (j_n, j_L) = (c / J, c % J)
                if (c < J * J) dl[c / J] = fmaf(d[t], al[c % J], dl[c / J]);
            }
        }
        tc_fence_before();
        if (valid) {
            float* o = p.out + e * p.out_ld;
#pragma unroll
            for (int jn = 0; jn < J; ++jn) o[jn] = dl[jn];
            if (p.vals) o[J] = xval;
        }
    }
    if (!ok) atomicExch(&abort_s, 1);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base_s), "r"(2 * C::NCOL)
                     : "memory");
    }
}

// Gb in the layout above: row r = j_n * J + j_L, column k over the K-group
// modes (C order), zero padded.
template <bool TF32>
__global__ void build_b_image(const float* __restrict__ G, int order, int mode, int lmode, int J, int NK,
                              const int* __restrict__ kmodes_unused, int K, int NP, int KP, uint8_t* __restrict__ img) {
    using E = Elt<TF32>;
    const int KCH = KP / E::KPG;
    const int SBO = KCH * 128;
    const int total = NP * KP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int r = t / KP, k = t % KP;
        float v = 0.f;
        if (r < J * J && k < K) {
            const int jn = r / J, jl = r % J;
            int jj[PTK_MAX_ORDER];
            jj[mode] = jn;
            jj[lmode] = jl;
            // K-group modes in increasing order, the last one fastest in k
            int rem = k;
            for (int m = order - 1; m >= 0; --m) {
                if (m == mode || m == lmode) continue;
                jj[m] = rem % J;
                rem /= J;
            }
            int src = 0;
            for (int m = 0; m < order; ++m) src = src * J + jj[m];
            v = G[src];
        }
        const int off = (r >> 3) * SBO + (k / E::KPG) * 128 + (r & 7) * 16 + (k % E::KPG) * E::ESZ;
        if constexpr (TF32) {
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
            *reinterpret_cast<uint32_t*>(img + off) = u;
        } else {
            *reinterpret_cast<__nv_bfloat16*>(img + off) = __float2bfloat16_rn(v);
        }
    }
}

struct Shape {
    bool ok = false;
    int J = 0, NK = 0;
    int kmodes[3] = {};
    int lmode = -1;
};

Shape shape_of(const DeltaJob& job) {
    Shape s;
    const int N = job.order;
    if (job.dtype != PTK_F32 || N < 3 || N > 5) return s;
    const int J = job.J[0];
    for (int k = 0; k < N; ++k)
        if (job.J[k] != J) return s;
    if (J * J > 128 || J < 2) return s;
    s.J = J;
    s.NK = N - 2;
    int o = 0;
    for (int k = 0; k < N; ++k) {
        if (k == job.mode) continue;
        if (o < s.NK)
            s.kmodes[o] = k;
        else
            s.lmode = k;
        ++o;
    }
    // the K extent must fit the shared-memory budget (A double buffer + Gb)
    int K = 1;
    for (int m = 0; m < s.NK; ++m) K *= J;
    if (K > 256) return s;
    s.ok = true;
    return s;
}

template <int J, int NK, bool TF32>
ptk_status launch_tc(ptk_ctx* ctx, const DeltaJob& job, const Shape& sh, cudaStream_t st) {
    using C = TcCfg<J, NK, TF32>;
    uint8_t* img = (uint8_t*)scratch(ctx, SLOT_GPERM_TC, C::B_BYTES);
    if (!img) return PTK_ERR_OUT_OF_MEMORY;
    {
        const int total = C::NP * C::KP;
        build_b_image<TF32><<<(total + 255) / 256, 256, 0, st>>>((const float*)job.core, job.order, job.mode,
                                                                 sh.lmode, J, NK, nullptr, C::K, C::NP, C::KP, img);
        ::ptk::note_launch();
    }
    PTK_LAUNCH_CHECK();
    TcParams p{};
    p.n = job.n;
    for (int m = 0; m < NK; ++m) {
        p.col_k[m] = job.col[sh.kmodes[m]];
        p.f_k[m] = (const float*)job.factors[sh.kmodes[m]];
        p.ld_k[m] = job.ld[sh.kmodes[m]];
    }
    p.col_l = job.col[sh.lmode];
    p.f_l = (const float*)job.factors[sh.lmode];
    p.ld_l = job.ld[sh.lmode];
    p.cstride = job.cstride;
    p.vals = (const float*)job.vals;
    p.out = (float*)job.out;
    p.out_ld = job.out_ld;
    p.b_image = img;
    p.b_bytes = C::B_BYTES;
    p.flags = ctx->d_flags;
    auto kern = delta_tc_kernel<J, NK, TF32>;
    PTK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    PTK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 1;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_THREADS, C::SMEM));
    per_sm = std::max(1, std::min(per_sm, 512 / (2 * C::NCOL)));  // TMEM: 512 columns per SM
    const int64_t tiles = ceil_div(job.n, TC_M);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(tiles, 2), (int64_t)ctx->sm_count * per_sm));
    { kern<<<(unsigned)grid, TC_THREADS, C::SMEM, st>>>(p); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

template <bool TF32>
ptk_status dispatch_tc(ptk_ctx* ctx, const DeltaJob& job, const Shape& sh, cudaStream_t st) {
#define PTK_TC(JJ, KK) \
    if (sh.J == JJ && sh.NK == KK) return launch_tc<JJ, KK, TF32>(ctx, job, sh, st);
    PTK_TC(10, 2) PTK_TC(10, 1) PTK_TC(5, 1) PTK_TC(5, 2) PTK_TC(5, 3)
    PTK_TC(2, 1) PTK_TC(3, 1) PTK_TC(4, 1) PTK_TC(6, 1) PTK_TC(7, 1) PTK_TC(8, 1) PTK_TC(9, 1) PTK_TC(11, 1)
    PTK_TC(2, 2) PTK_TC(3, 2) PTK_TC(4, 2) PTK_TC(6, 2) PTK_TC(7, 2) PTK_TC(8, 2) PTK_TC(9, 2) PTK_TC(11, 2)
    PTK_TC(2, 3) PTK_TC(3, 3) PTK_TC(4, 3) PTK_TC(6, 3)
#undef PTK_TC
    set_error("tensor-core delta: no kernel for J=%d, order %d", sh.J, sh.NK + 2);
    return PTK_ERR_UNSUPPORTED;
}

}  // namespace

bool delta_tc_supported(const DeltaJob& job, ptk_precision prec) {
    if (prec != PTK_PREC_BF16 && prec != PTK_PREC_TF32) return false;
    Shape s = shape_of(job);
    if (!s.ok) return false;
    if (s.NK == 3 && s.J > 6) return false;
    return true;
}

ptk_status delta_tc(ptk_ctx* ctx, const DeltaJob& job, ptk_precision prec, cudaStream_t st) {
    Shape s = shape_of(job);
    if (!s.ok || !delta_tc_supported(job, prec)) {
        set_error("tensor-core delta is not available for this shape");
        return PTK_ERR_UNSUPPORTED;
    }
    if (job.n == 0) return PTK_OK;
    if (prec == PTK_PREC_TF32) return dispatch_tc<true>(ctx, job, s, st);
    return dispatch_tc<false>(ctx, job, s, st);
}

}  // namespace ptk

extern "C" int ptk_delta_tc_supported(const ptk_model* m, int32_t mode, ptk_precision prec) {
    if (!m || mode < 0 || mode >= m->order) return 0;
    ptk::DeltaJob j;
    j.order = m->order;
    j.mode = mode;
    for (int k = 0; k < m->order; ++k) j.J[k] = m->J[k];
    j.dtype = m->dtype;
    return ptk::delta_tc_supported(j, prec) ? 1 : 0;
}
