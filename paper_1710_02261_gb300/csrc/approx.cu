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

// ---- u, v over the non-zero core entries -------------------------------------
// R(beta) matters only for the entries still in the core (a zero entry ranks
// last whatever its R), so once most of the core is truncated the two sums
// are taken for the non-zeros only.  The non-zeros are compacted (C order)
// into records: beta and the positions, in a staged entry's rows, of its N
// factor entries.  A thread keeps u and v of UV_RPT records over its block's
// entries; per entry and record that is N shared-memory loads, N - 1
// multiplies and two FMAs, against about 2.5 instructions per entry and core
// entry for the dense pass, so this pass is taken below about a fifth of the
// core (the record loop has no branch per zero, the dense one has no zeros to
// skip).
constexpr int UV_RPT = 4;  // records per thread
constexpr int UV_CT = 1024;  // compaction block

struct UVRec {
    int beta;
    uint8_t pos[12];  // factor-entry positions in a staged entry's rows (< 256)
};
static_assert(sizeof(UVRec) == 16, "one record per 16-byte load");

// One block; thread t takes beta in [|G| t / B, |G| (t + 1) / B); records in
// C order; n_out = their number (at most cap, else none and FLAG_SPARSE).
struct UVDims {
    int J[PTK_MAX_ORDER];
};

__global__ void __launch_bounds__(UV_CT) uv_compact(const float* __restrict__ G, int64_t gsize, int order, UVDims J,
                                                    UVRec* __restrict__ rec, int* __restrict__ n_out, int cap,
                                                    int* __restrict__ flags) {
    __shared__ int sc[UV_CT];
    const int t = threadIdx.x;
    const int64_t b0 = gsize * t / UV_CT, b1 = gsize * (t + 1) / UV_CT;
    int c = 0;
    for (int64_t b = b0; b < b1; ++b) c += G[b] != 0.f;
    sc[t] = c;
    __syncthreads();
    for (int off = 1; off < UV_CT; off <<= 1) {
        const int v = t >= off ? sc[t - off] : 0;
        __syncthreads();
        sc[t] += v;
        __syncthreads();
    }
    const int total = sc[UV_CT - 1];
    if (total > cap) {
        if (t == 0) {
            *n_out = 0;
            atomicAdd(&flags[FLAG_SPARSE], 1);
        }
        return;
    }
    if (t == 0) *n_out = total;
    int w = sc[t] - c;
    int rowoff[PTK_MAX_ORDER];
    rowoff[0] = 0;
    for (int k = 1; k < order; ++k) rowoff[k] = rowoff[k - 1] + J.J[k - 1];
    for (int64_t b = b0; b < b1; ++b) {
        if (G[b] == 0.f) continue;
        UVRec r;
        r.beta = (int)b;
        for (int k = 0; k < 12; ++k) r.pos[k] = 0;
        int64_t rem = b;
        for (int k = order - 1; k >= 0; --k) {  // C order: the last mode's index is fastest
            r.pos[k] = (uint8_t)(rowoff[k] + (int)(rem % J.J[k]));
            rem /= J.J[k];
        }
        rec[w++] = r;
    }
}

// block (x, y): entries of slice x, records [y * AT * UV_RPT, (y + 1) * AT * UV_RPT) of the list
template <int N>
__global__ void __launch_bounds__(AT) uv_sparse(const UVParams p, const UVRec* __restrict__ rec,
                                                const int* __restrict__ n_rec, float* __restrict__ part) {
    extern __shared__ __align__(16) float sm[];
    int rowoff[N + 1];
    rowoff[0] = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) rowoff[k + 1] = rowoff[k] + p.J[k];
    const int estride = rowoff[N] + 1;
    float* ent = sm;  // [ACH2][estride]
    const int nrec = *n_rec;
    const int r0 = blockIdx.y * AT * UV_RPT;
    int pos[UV_RPT][N];
    bool has[UV_RPT];
#pragma unroll
    for (int q = 0; q < UV_RPT; ++q) {
        const int ri = r0 + q * AT + threadIdx.x;
        has[q] = ri < nrec;
        const UVRec r = has[q] ? rec[ri] : rec[0];
#pragma unroll
        for (int k = 0; k < N; ++k) pos[q][k] = has[q] ? r.pos[k] : 0;
    }
    float ua[UV_RPT], va[UV_RPT];
#pragma unroll
    for (int q = 0; q < UV_RPT; ++q) {
        ua[q] = 0.f;
        va[q] = 0.f;
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
        for (int e = 0; e < cn; ++e) {
            const float* er = ent + e * estride;
            const float r = er[rowoff[N]];
#pragma unroll
            for (int q = 0; q < UV_RPT; ++q) {
                if (!has[q]) continue;  // past the list's end (the last block row's tail)
                float K = er[pos[q][0]];
#pragma unroll
                for (int k = 1; k < N; ++k) K *= er[pos[q][k]];
                ua[q] = fmaf(r, K, ua[q]);
                va[q] = fmaf(K, K, va[q]);
            }
        }
    }
    // part[x][record][2]; records past the list are never read
#pragma unroll
    for (int q = 0; q < UV_RPT; ++q) {
        const int ri = r0 + q * AT + threadIdx.x;
        if (!has[q]) continue;
        part[((int64_t)blockIdx.x * nrec + ri) * 2] = ua[q];
        part[((int64_t)blockIdx.x * nrec + ri) * 2 + 1] = va[q];
    }
}

// R of the records (the blocks' partial sums in block order, in FP64); every
// other core entry is zero and keeps R = 0 (set before)
__global__ void uv_sparse_finish(const float* __restrict__ part, int nblocks, const UVRec* __restrict__ rec,
                                 const int* __restrict__ n_rec, const float* __restrict__ G, double* __restrict__ R) {
    const int nrec = *n_rec;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nrec; t += gridDim.x * blockDim.x) {
        double u = 0.0, v = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            u += (double)part[((int64_t)b * nrec + t) * 2];
            v += (double)part[((int64_t)b * nrec + t) * 2 + 1];
        }
        const int beta = rec[t].beta;
        const double g = (double)G[beta];
        R[beta] = -2.0 * g * u - g * g * v;
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

template <int N>
ptk_status launch_uv_sparse(const UVParams& p, const UVRec* rec, const int* n_rec, float* part, int grid, int ny,
                            size_t smem, cudaStream_t st) {
    PTK_TRY(smem_attr((const void*)uv_sparse<N>, smem, st));
    { uv_sparse<N><<<dim3((unsigned)grid, (unsigned)ny), AT, smem, st>>>(p, rec, n_rec, part); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

// u, v and R(beta) over the non-zero core entries only (core_nnz of them);
// PTK_OK with *taken = false where the dense pass is the cheaper one
static ptk_status uv_pass_sparse(ptk_ctx* ctx, const ptk_model* m, const UVParams& p, int64_t core_nnz,
                                 double* d_R, bool* taken, cudaStream_t st) {
    *taken = false;
    const int N = m->order;
    int64_t gsize = 1;
    for (int k = 0; k < N; ++k) gsize *= m->J[k];
    int rowlen = 1;
    for (int k = 0; k < N; ++k) rowlen += m->J[k];
    // the chunk staging (fetch_items) covers ACH2 entries of up to five modes
    if (core_nnz < 0 || N < 3 || ACH2 * (N + 1) > AT * UV_ITEMS || rowlen > 255 ||
        (double)core_nnz * (2 * N + 1) > 0.9 * 2.5 * (double)gsize)
        return PTK_OK;
    const int cap = (int)std::max<int64_t>(core_nnz, 1);
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(p.E, 4096), 1), (int64_t)ctx->sm_count * 2);
    const int ny = (int)ceil_div(cap, (int64_t)AT * UV_RPT);
    const size_t rbytes = ((size_t)cap * sizeof(UVRec) + 15) / 16 * 16;
    char* buf = (char*)scratch(ctx, SLOT_SPARSE, rbytes + 64 + sizeof(float) * 2 * (size_t)grid * cap);
    if (!buf) return PTK_ERR_OUT_OF_MEMORY;
    UVRec* rec = reinterpret_cast<UVRec*>(buf);
    int* n_rec = reinterpret_cast<int*>(buf + rbytes);
    float* part = reinterpret_cast<float*>(buf + rbytes + 64);
    UVDims dj{};
    for (int k = 0; k < N; ++k) dj.J[k] = m->J[k];
    { uv_compact<<<1, UV_CT, 0, st>>>((const float*)m->core, gsize, N, dj, rec, n_rec, cap, ctx->d_flags);
      ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    PTK_CUDA(cudaMemsetAsync(d_R, 0, sizeof(double) * (size_t)gsize, st));
    const size_t smem = sizeof(float) * (size_t)ACH2 * rowlen;
    *taken = true;
    switch (N) {
        case 3: PTK_TRY(launch_uv_sparse<3>(p, rec, n_rec, part, grid, ny, smem, st)); break;
        case 4: PTK_TRY(launch_uv_sparse<4>(p, rec, n_rec, part, grid, ny, smem, st)); break;
        default: PTK_TRY(launch_uv_sparse<5>(p, rec, n_rec, part, grid, ny, smem, st)); break;
    }
    { uv_sparse_finish<<<(unsigned)std::max<int64_t>(1, ceil_div(cap, 256)), 256, 0, st>>>(
          part, grid, rec, n_rec, (const float*)m->core, d_R); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

// u, v and R(beta) for every core entry into d_R (double, |G|), from the
// residuals of `src`; with core_nnz >= 0 (nnz(G), known) over the non-zero
// entries alone where that is cheaper.
static ptk_status uv_pass(ptk_ctx* ctx, const ptk_model* m, int64_t E, const UVSource& src, double* d_R,
                          cudaStream_t st, int64_t core_nnz = -1) {
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
    if (E > 0) {
        bool taken = false;
        PTK_TRY(uv_pass_sparse(ctx, m, p, core_nnz, d_R, &taken, st));
        if (taken) return PTK_OK;
    }
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
                           cudaStream_t st, const UVSource* from_sweep, int64_t core_nnz) {
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
            PTK_TRY(uv_pass(ctx, m, x->nnz, *from_sweep, R, st, core_nnz));
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
