// cache.cu -- P-Tucker-Cache (Alg. 3 with the table Pres, Sec. 3.3).
//   build:   Pres[alpha][beta] = G_beta prod_{k=1..N} a^(k)_{i_k j_k}
//   delta:   delta(j) = sum_{beta: j_n = j} Pres[alpha][beta] / a^(n)_{i_n j}
//            (the divisor is the same for every beta with j_n = j, so the
//            sum is divided once); when a^(n)_{i_n j} is exactly 0 the
//            products are taken as plain P-Tucker does.
//   rescale: after mode n, Pres[alpha][beta] *= a_new / a_old, recomputed
//            from the factors when a_old is exactly 0.
// Pres is |Omega| x |G| FP32 in input entry order (row alpha contiguous), so
// every pass streams it from HBM: 4|G| bytes per entry to build, 4|G| to read
// for delta and 8|G| to rescale.  One warp works on one entry at a time.
#include "common.cuh"

namespace ptk {
namespace {

constexpr int CW = 8;  // warps per block

struct CoreShape {
    int order;
    int J[PTK_MAX_ORDER];
    int64_t stride[PTK_MAX_ORDER];  // C-order strides of the core
    int64_t size;
};

struct Facs {
    const float* A[PTK_MAX_ORDER];
    int64_t ld[PTK_MAX_ORDER];
};

CoreShape shape_of(const ptk_model* m) {
    CoreShape s;
    s.order = m->order;
    int64_t st = 1;
    for (int k = m->order - 1; k >= 0; --k) {
        s.J[k] = m->J[k];
        s.stride[k] = st;
        st *= m->J[k];
    }
    s.size = st;
    return s;
}

Facs facs_of(const ptk_model* m) {
    Facs f;
    for (int k = 0; k < m->order; ++k) {
        f.A[k] = (const float*)m->factors[k];
        f.ld[k] = m->ld[k];
    }
    return f;
}

// G_beta * prod_{k != skip} a^(k)_{i_k j_k(beta)}  (skip = -1: all modes)
__device__ __forceinline__ float fresh_product(const CoreShape& cs, const Facs& f, const float* __restrict__ G,
                                               const int32_t* coord, int64_t beta, int skip) {
    float p = G[beta];
    for (int k = 0; k < cs.order; ++k) {
        int j = (int)((beta / cs.stride[k]) % cs.J[k]);
        if (k != skip) p *= f.A[k][(int64_t)coord[k] * f.ld[k] + j];
    }
    return p;
}

__global__ void __launch_bounds__(CW * 32) pres_build(const int32_t* __restrict__ idx, int64_t E, CoreShape cs, Facs f,
                                                      const float* __restrict__ G, float* __restrict__ pres) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < E; a += nwarps) {
        const int32_t* co = idx + a * cs.order;
        float* row = pres + a * cs.size;
        for (int64_t b = lane; b < cs.size; b += 32) row[b] = fresh_product(cs, f, G, co, b, -1);
    }
}

__global__ void __launch_bounds__(CW * 32) pres_delta(const int32_t* __restrict__ idx, const int32_t* __restrict__ perm,
                                                      const float* __restrict__ svals, int64_t E, int mode, CoreShape cs,
                                                      Facs f, const float* __restrict__ G,
                                                      const float* __restrict__ pres, float* __restrict__ delta,
                                                      int out_ld) {
    __shared__ float acc_s[CW][PTK_MAX_RANK][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Jn = cs.J[mode];
    const int64_t U = cs.stride[mode];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < E; e += nwarps) {
        const int64_t a = perm[e];
        const int32_t* co = idx + a * cs.order;
        const float* row = pres + a * cs.size;
        for (int j = 0; j < Jn; ++j) acc_s[w][j][lane] = 0.f;
        __syncwarp();
        for (int64_t b = lane; b < cs.size; b += 32) {
            int j = (int)((b / U) % Jn);
            acc_s[w][j][lane] += row[b];
        }
        __syncwarp();
        const float* arow = f.A[mode] + (int64_t)co[mode] * f.ld[mode];
        float* out = delta + e * out_ld;
        for (int j = 0; j < Jn; ++j) {
            float s = warp_sum(acc_s[w][j][lane]);
            const float aj = arow[j];
            if (aj != 0.f) {
                if (lane == 0) out[j] = s / aj;
            } else {
                // plain products for this j (Sec. 3.3 fallback)
                float t = 0.f;
                const int64_t cnt = cs.size / Jn;
                for (int64_t r = lane; r < cnt; r += 32) {
                    int64_t o = r / U, u = r % U;
                    int64_t b = (o * Jn + j) * U + u;
                    t += fresh_product(cs, f, G, co, b, mode);
                }
                t = warp_sum(t);
                if (lane == 0) out[j] = t;
            }
        }
        if (lane == 0) out[Jn] = svals[e];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(CW * 32) pres_rescale(const int32_t* __restrict__ idx, int64_t E, int mode,
                                                        CoreShape cs, Facs f, const float* __restrict__ G,
                                                        const float* __restrict__ aold, float* __restrict__ pres) {
    __shared__ float ratio_s[CW][PTK_MAX_RANK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Jn = cs.J[mode];
    const int64_t U = cs.stride[mode];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < E; a += nwarps) {
        const int32_t* co = idx + a * cs.order;
        const float* ao = aold + (int64_t)co[mode] * f.ld[mode];
        const float* an = f.A[mode] + (int64_t)co[mode] * f.ld[mode];
        if (lane < Jn) ratio_s[w][lane] = ao[lane] != 0.f ? an[lane] / ao[lane] : 0.f;
        __syncwarp();
        float* row = pres + a * cs.size;
        for (int64_t b = lane; b < cs.size; b += 32) {
            int j = (int)((b / U) % Jn);
            if (ao[j] != 0.f)
                row[b] *= ratio_s[w][j];
            else
                row[b] = fresh_product(cs, f, G, co, b, -1);
        }
        __syncwarp();
    }
}

int grid_warps(ptk_ctx* ctx, int64_t n) {
    int64_t g = ceil_div(std::max<int64_t>(n, 1), CW);
    return (int)std::min<int64_t>(g, (int64_t)ctx->sm_count * 8);
}

}  // namespace

ptk_status cache_build(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, float* pres, cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    { pres_build<<<grid_warps(ctx, x->nnz), CW * 32, 0, st>>>(x->idx, x->nnz, shape_of(m), facs_of(m),
                                                            (const float*)m->core, pres); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status cache_delta(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, const ptk_model* m, const float* pres,
                       void* delta, int ld, cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    { pres_delta<<<grid_warps(ctx, x->nnz), CW * 32, 0, st>>>(x->idx, s->perm, (const float*)s->vals, x->nnz, s->mode,
                                                            shape_of(m), facs_of(m), (const float*)m->core, pres,
                                                            (float*)delta, ld); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status cache_rescale(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, int mode, const void* aold, float* pres,
                         cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    { pres_rescale<<<grid_warps(ctx, x->nnz), CW * 32, 0, st>>>(x->idx, x->nnz, mode, shape_of(m), facs_of(m),
                                                              (const float*)m->core, (const float*)aold, pres); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

}  // namespace ptk
