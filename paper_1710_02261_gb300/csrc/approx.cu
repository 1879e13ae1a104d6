// approx.cu -- P-Tucker-Approx (Sec. 3.3, Alg. 4).
// Partial reconstruction error of core entry beta, Eq. (recon_partial):
//     R(beta) = sum_alpha p_ab (-2 x_a + p_ab + 2 sum_{g != beta} p_ag)
//             = -2 G_beta u_beta - G_beta^2 v_beta,
//     u_beta = sum_alpha r_alpha K_alpha(beta),  v_beta = sum_alpha K_alpha(beta)^2,
// with p_ab = G_beta K_alpha(beta), K_alpha(beta) = prod_n a^(n)_{i_n j_n} and the
// residual r_alpha = x_alpha - X_hat(alpha).  The two |G|-sized sums are taken
// in one pass over the entries; then the non-zero entries are ranked (largest
// R first, or smallest |G| first) by a stable radix sort with the C-order index
// as tie-break, and the first floor(p * nnz) of them are set to zero.
#include "common.cuh"

namespace ptk {
namespace {

constexpr int AT = 256;      // threads per block
constexpr int ACH = 32;      // entries staged per step
constexpr int AMAXG = 8192;  // core entries per pass

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct UVParams {
    const float* delta0;   // [E][ld0]: delta for mode dmode with x in slot J_dmode
    int ld0;
    int dmode;
    const int32_t* col[PTK_MAX_ORDER];  // coordinate k of entry e: col[k][e * cstride]
    int64_t cstride;
    int64_t E;
    int order;
    int J[PTK_MAX_ORDER];
    const float* A[PTK_MAX_ORDER];
    int64_t lda[PTK_MAX_ORDER];
    int64_t gsize;
    int64_t b0, b1;        // core-entry range of this pass
    float* part;           // [grid][b1-b0][2]
};

// Staged chunk: for each entry the factor rows of all modes, then the residual.
__device__ __forceinline__ void stage_chunk(const UVParams& p, const int* rowoff, int estride, int64_t c0, int cn,
                                            float* ent) {
    const int N = p.order;
    for (int t = threadIdx.x; t < cn * estride; t += blockDim.x) {
        const int e = t / estride, q = t % estride;
        const int64_t ge = c0 + e;
        float v;
        if (q < rowoff[N]) {
            int k = 0;
            while (q >= rowoff[k + 1]) ++k;
            const int j = q - rowoff[k];
            v = p.A[k][(int64_t)p.col[k][ge * p.cstride] * p.lda[k] + j];
        } else {
            const int dm = p.dmode;
            const float* d = p.delta0 + ge * p.ld0;
            const float* a0 = p.A[dm] + (int64_t)p.col[dm][ge * p.cstride] * p.lda[dm];
            float xh = 0.f;
            for (int j = 0; j < p.J[dm]; ++j) xh = fmaf(d[j], a0[j], xh);
            v = d[p.J[dm]] - xh;
        }
        ent[e * estride + q] = v;
    }
}

// All core entries of the pass at once (prefixes <= AT): thread (pf, g) keeps
// u and v of the JL core entries with prefix pf in registers over the block's
// whole entry range, taking every G_E-th entry of each staged chunk; the
// groups are summed in a fixed order at the end.  A chunk holds, per entry,
// the factor rows of all modes and the residual; the next chunk's rows are
// fetched into registers (one (entry, mode) item per thread and round) while
// the current chunk is consumed.
constexpr int ACH2 = 128;
constexpr int UV_ITEMS = 3;  // (entry, mode) items per thread per chunk: ACH2 * (N + 1) <= AT * UV_ITEMS

struct Items {
    float v[UV_ITEMS][PTK_MAX_RANK];
};

__device__ __forceinline__ void fetch_items(const UVParams& p, int64_t c0, int cn, Items& it) {
    const int N = p.order;
#pragma unroll
    for (int u = 0; u < UV_ITEMS; ++u) {
        const int item = threadIdx.x + u * AT;
        const int e = item / (N + 1), k = item % (N + 1);
        if (e >= cn) continue;
        const int64_t ge = c0 + e;
        if (k < N) {
            const float* row = p.A[k] + (int64_t)p.col[k][ge * p.cstride] * p.lda[k];
#pragma unroll
            for (int j = 0; j < PTK_MAX_RANK; ++j)
                if (j < p.J[k]) it.v[u][j] = row[j];
        } else {
            const int dm = p.dmode;
            const float* d = p.delta0 + ge * p.ld0;
            const float* a0 = p.A[dm] + (int64_t)p.col[dm][ge * p.cstride] * p.lda[dm];
            float xh = 0.f;
#pragma unroll
            for (int j = 0; j < PTK_MAX_RANK; ++j)
                if (j < p.J[dm]) xh = fmaf(d[j], a0[j], xh);
            it.v[u][0] = d[p.J[dm]] - xh;
        }
    }
}

__device__ __forceinline__ void store_items(const UVParams& p, const int* rowoff, int estride, int cn,
                                            const Items& it, float* ent) {
    const int N = p.order;
#pragma unroll
    for (int u = 0; u < UV_ITEMS; ++u) {
        const int item = threadIdx.x + u * AT;
        const int e = item / (N + 1), k = item % (N + 1);
        if (e >= cn) continue;
        float* dst = ent + e * estride + rowoff[k];
        if (k < N) {
#pragma unroll
            for (int j = 0; j < PTK_MAX_RANK; ++j)
                if (j < p.J[k]) dst[j] = it.v[u][j];
        } else {
            dst[0] = it.v[u][0];
        }
    }
}

__global__ void __launch_bounds__(AT) uv_accumulate_reg(const UVParams p) {
    extern __shared__ __align__(16) float sm[];
    const int N = p.order;
    int rowoff[PTK_MAX_ORDER + 1];
    rowoff[0] = 0;
    for (int k = 0; k < N; ++k) rowoff[k + 1] = rowoff[k] + p.J[k];
    const int estride = rowoff[N] + 1;
    const int JL = p.J[N - 1];
    const int64_t pf0 = p.b0 / JL, pf1 = (p.b1 + JL - 1) / JL;
    const int npf = (int)(pf1 - pf0);
    const int GE = AT / npf;                 // entry groups (>= 1)
    const int tid = threadIdx.x;
    const int g = tid / npf;
    const int64_t pf = pf0 + tid % npf;
    const bool active = g < GE;
    float* ent = sm;                         // [ACH2][estride]
    float* red = sm + ACH2 * estride;        // [GE][npf][JL][2] for the final reduction
    int off[PTK_MAX_ORDER];
    {
        int64_t rem = pf;
        for (int k = N - 2; k >= 0; --k) {
            off[k] = rowoff[k] + (int)(rem % p.J[k]);
            rem /= p.J[k];
        }
    }
    float ua[PTK_MAX_RANK], va[PTK_MAX_RANK];
#pragma unroll
    for (int l = 0; l < PTK_MAX_RANK; ++l) {
        ua[l] = 0.f;
        va[l] = 0.f;
    }
    const int64_t per_block = ceil_div_dev(p.E, gridDim.x);
    const int64_t e_begin = blockIdx.x * per_block;
    const int64_t e_end = min(p.E, e_begin + per_block);
    Items it;
    if (e_begin < e_end) fetch_items(p, e_begin, (int)min((int64_t)ACH2, e_end - e_begin), it);
    for (int64_t c0 = e_begin; c0 < e_end; c0 += ACH2) {
        const int cn = (int)min((int64_t)ACH2, e_end - c0);
        __syncthreads();  // the previous chunk is consumed
        store_items(p, rowoff, estride, cn, it, ent);
        __syncthreads();
        if (c0 + ACH2 < e_end) fetch_items(p, c0 + ACH2, (int)min((int64_t)ACH2, e_end - c0 - ACH2), it);
        if (active) {
            for (int e = g; e < cn; e += GE) {
                const float* er = ent + e * estride;
                float pre = 1.f;
                for (int k = 0; k < N - 1; ++k) pre *= er[off[k]];
                const float r = er[rowoff[N]];
                const float* al = er + rowoff[N - 1];
#pragma unroll
                for (int l = 0; l < PTK_MAX_RANK; ++l) {
                    if (l < JL) {
                        const float K = pre * al[l];
                        ua[l] = fmaf(r, K, ua[l]);
                        va[l] = fmaf(K, K, va[l]);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (active)
        for (int l = 0; l < JL; ++l) {
            red[((g * npf + tid % npf) * JL + l) * 2] = ua[l];
            red[((g * npf + tid % npf) * JL + l) * 2 + 1] = va[l];
        }
    __syncthreads();
    const int64_t nb = p.b1 - p.b0;
    float* out = p.part + (int64_t)blockIdx.x * nb * 2;
    for (int64_t t = tid; t < nb; t += AT) {
        const int64_t b = p.b0 + t;
        const int q = (int)(b / JL - pf0), l = (int)(b % JL);
        float u = 0.f, v = 0.f;
        for (int gg = 0; gg < GE; ++gg) {
            u += red[((gg * npf + q) * JL + l) * 2];
            v += red[((gg * npf + q) * JL + l) * 2 + 1];
        }
        out[2 * t] = u;
        out[2 * t + 1] = v;
    }
}

// one pass over all entries for core entries [b0, b1)
__global__ void __launch_bounds__(AT) uv_accumulate(const UVParams p) {
    extern __shared__ __align__(16) float sm[];
    const int N = p.order;
    int rowoff[PTK_MAX_ORDER + 1];
    rowoff[0] = 0;
    for (int k = 0; k < N; ++k) rowoff[k + 1] = rowoff[k] + p.J[k];
    const int estride = rowoff[N] + 1;  // factor rows of all modes, then r
    float* ent = sm;                          // [ACH][estride]
    float* us = sm + ACH * estride;           // [nb]
    float* vs = us + (p.b1 - p.b0);           // [nb]
    const int64_t nb = p.b1 - p.b0;
    const int JL = p.J[N - 1];
    for (int64_t t = threadIdx.x; t < nb; t += AT) {
        us[t] = 0.f;
        vs[t] = 0.f;
    }
    // prefixes of this pass: beta = prefix * JL + l
    const int64_t pf0 = p.b0 / JL, pf1 = (p.b1 + JL - 1) / JL;
    const int64_t per_block = ceil_div_dev(p.E, gridDim.x);
    const int64_t e_begin = blockIdx.x * per_block;
    const int64_t e_end = min(p.E, e_begin + per_block);
    __syncthreads();
    for (int64_t c0 = e_begin; c0 < e_end; c0 += ACH) {
        const int cn = (int)min((int64_t)ACH, e_end - c0);
        // stage factor rows and residuals of the chunk
        stage_chunk(p, rowoff, estride, c0, cn, ent);
        __syncthreads();
        for (int64_t pf = pf0 + threadIdx.x; pf < pf1; pf += AT) {
            int dig[PTK_MAX_ORDER];
            int64_t rem = pf;
            for (int k = N - 2; k >= 0; --k) {
                dig[k] = (int)(rem % p.J[k]);
                rem /= p.J[k];
            }
            float ua[PTK_MAX_RANK], va[PTK_MAX_RANK];
            for (int l = 0; l < JL; ++l) {
                ua[l] = 0.f;
                va[l] = 0.f;
            }
            for (int e = 0; e < cn; ++e) {
                const float* er = ent + e * estride;
                float pre = 1.f;
                for (int k = 0; k < N - 1; ++k) pre *= er[rowoff[k] + dig[k]];
                const float r = er[rowoff[N]];
                const float* al = er + rowoff[N - 1];
#pragma unroll
                for (int l = 0; l < PTK_MAX_RANK; ++l) {
                    if (l < JL) {
                        const float K = pre * al[l];
                        ua[l] = fmaf(r, K, ua[l]);
                        va[l] = fmaf(K, K, va[l]);
                    }
                }
            }
            for (int l = 0; l < JL; ++l) {
                const int64_t b = pf * JL + l;
                if (b >= p.b0 && b < p.b1) {
                    us[b - p.b0] += ua[l];
                    vs[b - p.b0] += va[l];
                }
            }
        }
        __syncthreads();
    }
    float* out = p.part + (int64_t)blockIdx.x * nb * 2;
    for (int64_t t = threadIdx.x; t < nb; t += AT) {
        out[2 * t] = us[t];
        out[2 * t + 1] = vs[t];
    }
}

__global__ void uv_finish(const float* __restrict__ part, int nblocks, int64_t b0, int64_t nb,
                          const float* __restrict__ G, double* __restrict__ R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        double u = 0.0, v = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            u += (double)part[((int64_t)b * nb + t) * 2];
            v += (double)part[((int64_t)b * nb + t) * 2 + 1];
        }
        const double g = (double)G[b0 + t];
        R[b0 + t] = g == 0.0 ? 0.0 : -2.0 * g * u - g * g * v;
    }
}

__device__ __forceinline__ uint64_t ord_key(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void make_keys(const float* __restrict__ G, const double* __restrict__ R, int64_t n, int rule,
                          uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[t];
        uint64_t k;
        if (g == 0.f)
            k = ~0ull;                        // removed entries rank last
        else if (rule == PTK_TRUNC_R_BETA)
            k = ~ord_key(R[t]);               // descending R
        else
            k = ord_key(fabs((double)g));     // ascending |G|
        if (k == ~0ull && g != 0.f) k = ~0ull - 1;
        keys[t] = k;
        vals[t] = (uint32_t)t;
    }
}

__global__ void zero_selected(const double* __restrict__ nnz_d, double p, const uint32_t* __restrict__ order,
                              float* __restrict__ G) {
    const int64_t nnz = (int64_t)nnz_d[0];
    const int64_t k = (int64_t)floor(p * (double)nnz);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < k; t += (int64_t)gridDim.x * blockDim.x)
        G[order[t]] = 0.f;
}

}  // namespace

// u, v and R(beta) for every core entry into d_R (double, |G|), from the
// residuals of `src`.
static ptk_status uv_pass(ptk_ctx* ctx, const ptk_model* m, int64_t E, const UVSource& src, double* d_R,
                          cudaStream_t st) {
    const int N = m->order;
    int64_t gsize = 1;
    for (int k = 0; k < N; ++k) gsize *= m->J[k];
    UVParams p;
    p.delta0 = src.delta;
    p.ld0 = src.ld;
    p.dmode = src.dmode;
    for (int k = 0; k < N; ++k) p.col[k] = src.col[k];
    p.cstride = src.cstride;
    p.E = E;
    p.order = N;
    int estride = 1;
    for (int k = 0; k < N; ++k) {
        p.J[k] = m->J[k];
        p.A[k] = (const float*)m->factors[k];
        p.lda[k] = m->ld[k];
        estride += m->J[k];
    }
    p.gsize = gsize;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(E, 4096), 1), (int64_t)ctx->sm_count * 2);
    const int JL = m->J[N - 1];
    // passes of at most AT core prefixes (JL core entries each) use the
    // register-resident kernel; each pass re-reads the entries
    const bool reg_ok = ACH2 * (N + 1) <= AT * UV_ITEMS;
    const int64_t pass = reg_ok ? std::min<int64_t>(gsize, (int64_t)(AT - 1) * JL) : std::min<int64_t>(gsize, AMAXG);
    float* part = (float*)scratch(ctx, SLOT_APPROX, sizeof(float) * (size_t)grid * pass * 2);
    if (!part) return PTK_ERR_OUT_OF_MEMORY;
    p.part = part;
    for (int64_t b0 = 0; b0 < gsize; b0 += pass) {
        p.b0 = b0;
        p.b1 = std::min<int64_t>(gsize, b0 + pass);
        const int64_t npf = (p.b1 + JL - 1) / JL - p.b0 / JL;
        if (npf <= AT && reg_ok) {
            const int GE = AT / (int)npf;
            const size_t smem = sizeof(float) * ((size_t)ACH2 * estride + (size_t)GE * npf * JL * 2);
            PTK_TRY(smem_attr((const void*)uv_accumulate_reg, smem, st));
            { uv_accumulate_reg<<<grid, AT, smem, st>>>(p); ::ptk::note_launch(); }
        } else {
            const size_t smem = sizeof(float) * ((size_t)ACH * estride + 2 * (size_t)(p.b1 - p.b0));
            PTK_TRY(smem_attr((const void*)uv_accumulate, smem, st));
            { uv_accumulate<<<grid, AT, smem, st>>>(p); ::ptk::note_launch(); }
        }
        PTK_LAUNCH_CHECK();
        { uv_finish<<<(unsigned)std::max<int64_t>(1, ceil_div(p.b1 - p.b0, 256)), 256, 0, st>>>(
            part, grid, b0, p.b1 - p.b0, (const float*)m->core, d_R); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
    }
    return PTK_OK;
}

// R(beta) for every core entry into d_R (double, |G|), from the entries of x
// (their residuals from a fresh delta pass for mode 1).
ptk_status partial_error_impl(ptk_ctx* ctx, const ptk_coo* x, const ptk_model* m, const float* vals, double* d_R,
                              cudaStream_t st) {
    const int N = m->order;
    const int64_t E = x->nnz;
    DeltaJob job;
    job.n = E;
    job.order = N;
    job.mode = 0;
    for (int k = 0; k < N; ++k) {
        job.col[k] = x->idx + k;
        job.factors[k] = m->factors[k];
        job.ld[k] = m->ld[k];
        job.J[k] = m->J[k];
    }
    job.cstride = N;
    job.core = m->core;
    job.vals = vals;
    job.dtype = PTK_F32;
    job.out_ld = delta_out_ld(m->J[0]);
    void* d0 = scratch(ctx, SLOT_DELTA, sizeof(float) * (size_t)std::max<int64_t>(E, 1) * job.out_ld);
    if (!d0) return PTK_ERR_OUT_OF_MEMORY;
    job.out = d0;
    if (E > 0) PTK_TRY(delta_simt(ctx, job, st));
    UVSource src;
    src.delta = (const float*)d0;
    src.ld = job.out_ld;
    src.dmode = 0;
    for (int k = 0; k < N; ++k) src.col[k] = x->idx + k;
    src.cstride = N;
    return uv_pass(ctx, m, E, src, d_R, st);
}

ptk_status approx_truncate(ptk_ctx* ctx, const ptk_coo* x, ptk_model* m, double prate, ptk_trunc_rule rule,
                           cudaStream_t st, const UVSource* from_sweep) {
    if (m->dtype != PTK_F32) {
        set_error("P-Tucker-Approx is implemented for the FP32 model only");
        return PTK_ERR_UNSUPPORTED;
    }
    int64_t gsize = 1;
    for (int k = 0; k < m->order; ++k) gsize *= m->J[k];
    char* buf = (char*)scratch(ctx, SLOT_FOLD1, (sizeof(uint64_t) + sizeof(uint32_t) + sizeof(double)) * gsize + 64);
    if (!buf) return PTK_ERR_OUT_OF_MEMORY;
    uint64_t* keys = (uint64_t*)buf;
    double* R = (double*)(buf + sizeof(uint64_t) * gsize);
    uint32_t* vals = (uint32_t*)(buf + (sizeof(uint64_t) + sizeof(double)) * gsize);
    if (rule == PTK_TRUNC_R_BETA) {
        const void* xv = x->vals;
        if (x->dtype != PTK_F32) {
            set_error("Approx needs FP32 values");
            return PTK_ERR_UNSUPPORTED;
        }
        if (from_sweep)  // the sweep's last Delta already holds every residual's delta
            PTK_TRY(uv_pass(ctx, m, x->nnz, *from_sweep, R, st));
        else
            PTK_TRY(partial_error_impl(ctx, x, m, (const float*)xv, R, st));
    }
    const int g = (int)std::min<int64_t>(ceil_div(gsize, 256), (int64_t)ctx->sm_count * 8);
    { make_keys<<<g, 256, 0, st>>>((const float*)m->core, R, gsize, (int)rule, keys, vals); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    PTK_TRY(count_nonzero(ctx, m->core, gsize, PTK_F32, ctx->d_stats + 13, st));
    PTK_TRY(radix_sort_u64_desc_stable(ctx, keys, vals, gsize, st));
    { zero_selected<<<g, 256, 0, st>>>(ctx->d_stats + 13, prate, vals, (float*)m->core); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

}  // namespace ptk
