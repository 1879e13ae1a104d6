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
// for delta and 8|G| to rescale.  One warp works on one entry at a time with
// coalesced 128-byte accesses, CU of them in flight per lane.  The core index
// splits as beta = h * Klo + l (h over the leading modes, l over the rest,
// balanced), so the build multiplies G_beta by two small per-entry tables of
// factor-row products and the free mode's digit of beta comes from a table
// over h or l; no per-element integer division.
#include "common.cuh"

namespace ptk {
namespace {

constexpr int CW = 8;   // warps per block
constexpr int CU = 8;   // loads in flight per lane

struct CoreShape {
    int order;
    int J[PTK_MAX_ORDER];
    int64_t stride[PTK_MAX_ORDER];  // C-order strides of the core
    int64_t size;
    // beta = h * Klo + l: h runs over modes [0, s), l over modes [s, N)
    int s, Khi, Klo;
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
    // the split that balances the two halves
    int64_t best = INT64_MAX;
    s.s = 1;
    for (int c = 1; c < m->order; ++c) {
        const int64_t lo = s.stride[c - 1];   // prod J[c..N-1]
        const int64_t hi = st / lo;
        if (std::max(hi, lo) < best) {
            best = std::max(hi, lo);
            s.s = c;
        }
    }
    s.Klo = (int)s.stride[s.s - 1];
    s.Khi = (int)(st / s.Klo);
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

// G_beta * prod_{k != skip} a^(k)_{i_k j_k(beta)}  (skip = -1: all modes);
// the exact-zero fallbacks only.
__device__ __forceinline__ float fresh_product(const CoreShape& cs, const Facs& f, const float* __restrict__ G,
                                               const int32_t* coord, int64_t beta, int skip) {
    float p = G[beta];
    for (int k = 0; k < cs.order; ++k) {
        int j = (int)((beta / cs.stride[k]) % cs.J[k]);
        if (k != skip) p *= f.A[k][(int64_t)coord[k] * f.ld[k] + j];
    }
    return p;
}

// P[t] = prod over modes k0..k1-1 of a^(k)_{i_k j_k(t)}, t in C order over
// those modes (one warp).
__device__ __forceinline__ void kron_rows(float* P, int K, int k0, int k1, const CoreShape& cs, const Facs& f,
                                          const int32_t* co, int lane) {
    for (int t = lane; t < K; t += 32) {
        int rem = t;
        float p = 1.f;
        for (int k = k1 - 1; k >= k0; --k) {
            const int j = rem % cs.J[k];
            rem /= cs.J[k];
            p *= f.A[k][(int64_t)co[k] * f.ld[k] + j];
        }
        P[t] = p;
    }
}

// Digit of the free mode n as a function of h (n < s) or of l (n >= s).
__device__ __forceinline__ void digit_table(uint8_t* jt, const CoreShape& cs, int n) {
    const bool lo = n >= cs.s;
    const int K = lo ? cs.Klo : cs.Khi;
    const int64_t st = lo ? cs.stride[n] : cs.stride[n] / cs.Klo;
    for (int t = threadIdx.x; t < K; t += blockDim.x) jt[t] = (uint8_t)((t / st) % cs.J[n]);
}

// Pres[alpha][h * Klo + l] = G[h * Klo + l] * Phi[h] * Plo[l]
__global__ void __launch_bounds__(CW * 32) pres_build(const int32_t* __restrict__ idx, int64_t E, CoreShape cs, Facs f,
                                                      const float* __restrict__ G, float* __restrict__ pres) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* Phi = sm + (size_t)w * (cs.Khi + cs.Klo);
    float* Plo = Phi + cs.Khi;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < E; a += nwarps) {
        const int32_t* co = idx + a * cs.order;
        __syncwarp();
        kron_rows(Phi, cs.Khi, 0, cs.s, cs, f, co, lane);
        kron_rows(Plo, cs.Klo, cs.s, cs.order, cs, f, co, lane);
        __syncwarp();
        float* row = pres + a * cs.size;
        int h = 0, l = lane;
        while (l >= cs.Klo) l -= cs.Klo, ++h;
        for (int64_t b = lane; b < cs.size; b += 32) {
            row[b] = G[b] * (Phi[h] * Plo[l]);
            l += 32;
            while (l >= cs.Klo) l -= cs.Klo, ++h;
        }
    }
}

__global__ void __launch_bounds__(CW * 32) pres_delta(const int32_t* __restrict__ idx, const int32_t* __restrict__ perm,
                                                      const float* __restrict__ svals, int64_t E, int mode, CoreShape cs,
                                                      Facs f, const float* __restrict__ G,
                                                      const float* __restrict__ pres, float* __restrict__ delta,
                                                      int out_ld) {
    __shared__ float acc_s[CW][PTK_MAX_RANK][33];
    __shared__ uint8_t jt[4096];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Jn = cs.J[mode];
    const bool nlo = mode >= cs.s;
    digit_table(jt, cs, mode);
    __syncthreads();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = warp; e < E; e += nwarps) {
        const int64_t a = perm[e];
        const int32_t* co = idx + a * cs.order;
        const float* row = pres + a * cs.size;
        for (int j = 0; j < Jn; ++j) acc_s[w][j][lane] = 0.f;
        __syncwarp();
        int h = 0, l = lane;
        while (l >= cs.Klo) l -= cs.Klo, ++h;
        for (int64_t b0 = 0; b0 < cs.size; b0 += 32 * CU) {
            float v[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int64_t b = b0 + 32 * u + lane;
                v[u] = b < cs.size ? __ldcs(row + b) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                if (b0 + 32 * u + lane < cs.size) acc_s[w][nlo ? jt[l] : jt[h]][lane] += v[u];
                l += 32;
                while (l >= cs.Klo) l -= cs.Klo, ++h;
            }
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
                const int64_t U = cs.stride[mode];
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
    __shared__ uint8_t jt[4096];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Jn = cs.J[mode];
    const bool nlo = mode >= cs.s;
    digit_table(jt, cs, mode);
    __syncthreads();
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < E; a += nwarps) {
        const int32_t* co = idx + a * cs.order;
        const float* ao = aold + (int64_t)co[mode] * f.ld[mode];
        const float* an = f.A[mode] + (int64_t)co[mode] * f.ld[mode];
        __syncwarp();
        const bool zero = lane < Jn && ao[lane] == 0.f;
        if (lane < Jn) ratio_s[w][lane] = zero ? 0.f : an[lane] / ao[lane];
        const bool any_zero = __any_sync(0xffffffffu, zero);
        __syncwarp();
        float* row = pres + a * cs.size;
        int h = 0, l = lane;
        while (l >= cs.Klo) l -= cs.Klo, ++h;
        for (int64_t b0 = 0; b0 < cs.size; b0 += 32 * CU) {
            float v[CU];
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int64_t b = b0 + 32 * u + lane;
                v[u] = b < cs.size ? row[b] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int64_t b = b0 + 32 * u + lane;
                if (b < cs.size) {
                    const int j = nlo ? jt[l] : jt[h];
                    if (any_zero && ao[j] == 0.f)
                        row[b] = fresh_product(cs, f, G, co, b, -1);
                    else
                        __stcs(row + b, v[u] * ratio_s[w][j]);
                }
                l += 32;
                while (l >= cs.Klo) l -= cs.Klo, ++h;
            }
        }
    }
}

int grid_warps(ptk_ctx* ctx, int64_t n, int per_sm) {
    int64_t g = ceil_div(std::max<int64_t>(n, 1), CW);
    return (int)std::min<int64_t>(g, (int64_t)ctx->sm_count * per_sm);
}

}  // namespace

ptk_status cache_build(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, float* pres, cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    const CoreShape cs = shape_of(m);
    const size_t smem = sizeof(float) * CW * (size_t)(cs.Khi + cs.Klo);
    if (smem > ctx->smem_optin) {
        set_error("P-Tucker-Cache: core %lld too large for the table builder", (long long)cs.size);
        return PTK_ERR_UNSUPPORTED;
    }
    PTK_TRY(smem_attr((const void*)pres_build, smem, st));
    int per_sm = 1;
    PTK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pres_build, CW * 32, smem));
    { pres_build<<<grid_warps(ctx, x->nnz, std::max(per_sm, 1)), CW * 32, smem, st>>>(
          x->idx, x->nnz, cs, facs_of(m), (const float*)m->core, pres); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status cache_delta(ptk_ctx* ctx, const ptk_coo* x, const ptk_slices* s, const ptk_model* m, const float* pres,
                       void* delta, int ld, cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    const CoreShape cs = shape_of(m);
    if (std::max(cs.Khi, cs.Klo) > 4096) {
        set_error("P-Tucker-Cache: core %lld too large", (long long)cs.size);
        return PTK_ERR_UNSUPPORTED;
    }
    { pres_delta<<<grid_warps(ctx, x->nnz, 8), CW * 32, 0, st>>>(x->idx, s->perm, (const float*)s->vals, x->nnz,
                                                               s->mode, cs, facs_of(m), (const float*)m->core, pres,
                                                               (float*)delta, ld); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status cache_rescale(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, int mode, const void* aold, float* pres,
                         cudaStream_t st) {
    if (x->nnz == 0) return PTK_OK;
    const CoreShape cs = shape_of(m);
    if (std::max(cs.Khi, cs.Klo) > 4096) {
        set_error("P-Tucker-Cache: core %lld too large", (long long)cs.size);
        return PTK_ERR_UNSUPPORTED;
    }
    { pres_rescale<<<grid_warps(ctx, x->nnz, 8), CW * 32, 0, st>>>(x->idx, x->nnz, mode, cs, facs_of(m),
                                                                 (const float*)m->core, (const float*)aold, pres); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

}  // namespace ptk
