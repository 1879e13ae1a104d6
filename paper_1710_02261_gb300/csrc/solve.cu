// solve.cu -- Eq. (rowupdate): a_i = c_i (B_i + lambda I)^{-1} for every row,
// as the solution of the symmetric positive-definite system
// (B_i + lambda I) a_i^T = c_i^T (Alg. 3, matrix inverse and row update).
// Batched, one thread per row, in FP64: Cholesky L L^T, forward/back
// substitution, then one step of iterative refinement with the residual
// recomputed from the stored B_i, c_i.  An empty slice (B = 0, c = 0) gives the
// zero row, the exact minimiser of lambda ||a||^2.
//
// Also the reductions of the error pass, Eq. (reconfull): residuals from the
// last mode's Delta rows, sums of squares, and predictions from Delta rows.
#include "common.cuh"

namespace ptk {
namespace {

template <int J>
__device__ __forceinline__ int uidx(int j, int k) {  // upper triangle, row-major, j <= k
    return j * J - (j * (j - 1)) / 2 + (k - j);
}

// Row-buffer entry q as FP64: FP32 sums are stored as double-float pairs
// (s, lo) with value s + lo, FP64 sums as plain doubles.
__device__ __forceinline__ double rb(const float* b, int q) { return (double)b[2 * q] + (double)b[2 * q + 1]; }
__device__ __forceinline__ double rb(const double* b, int q) { return b[q]; }
template <typename TB>
constexpr int rb_width() { return sizeof(TB) == 4 ? 2 : 1; }

template <typename TB, typename TO, int J>
__global__ void __launch_bounds__(128) solve_kernel(const TB* __restrict__ rowbuf, const int64_t* __restrict__ row_ptr,
                                                   int64_t rows, double lambda, TO* __restrict__ out, int64_t ld,
                                                   int* flags) {
    constexpr int NTRI = J * (J + 1) / 2;
    constexpr int NOUT = NTRI + J;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        TO* o = out + r * ld;
        if (row_ptr[r + 1] == row_ptr[r]) {
#pragma unroll
            for (int j = 0; j < J; ++j) o[j] = TO(0);
            continue;
        }
        const TB* b = rowbuf + r * NOUT * rb_width<TB>();
        double L[NTRI];  // packed lower triangle, row-major: L(i,j) at i(i+1)/2 + j
        double inv[J];
        bool ok = true;
#pragma unroll
        for (int i = 0; i < J; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                double s = rb(b, uidx<J>(j, i));
                if (i == j) s += lambda;
#pragma unroll
                for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
                if (i == j) {
                    if (!(s > 0.0)) {
                        ok = false;
                        s = 1.0;
                    }
                    double d = sqrt(s);
                    L[i * (i + 1) / 2 + i] = d;
                    inv[i] = 1.0 / d;
                } else {
                    L[i * (i + 1) / 2 + j] = s * inv[j];
                }
            }
        }
        double x[J], y[J];
        auto chol_solve = [&](const double* rhs, double* sol) {
#pragma unroll
            for (int i = 0; i < J; ++i) {
                double s = rhs[i];
#pragma unroll
                for (int k = 0; k < i; ++k) s -= L[i * (i + 1) / 2 + k] * y[k];
                y[i] = s * inv[i];
            }
#pragma unroll
            for (int i = J - 1; i >= 0; --i) {
                double s = y[i];
#pragma unroll
                for (int k = i + 1; k < J; ++k) s -= L[k * (k + 1) / 2 + i] * sol[k];
                sol[i] = s * inv[i];
            }
        };
        double c[J];
#pragma unroll
        for (int j = 0; j < J; ++j) c[j] = rb(b, NTRI + j);
        chol_solve(c, x);
        // one refinement step: res = c - (B + lambda I) x, x += (B + lambda I)^{-1} res
        double res[J], dx[J];
#pragma unroll
        for (int i = 0; i < J; ++i) {
            double s = c[i] - lambda * x[i];
#pragma unroll
            for (int k = 0; k < J; ++k) {
                const int q = i <= k ? uidx<J>(i, k) : uidx<J>(k, i);
                s -= rb(b, q) * x[k];
            }
            res[i] = s;
        }
        chol_solve(res, dx);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            x[j] += dx[j];
            if (!isfinite(x[j])) ok = false;
        }
        if (!ok) {
            atomicAdd(&flags[FLAG_BAD_ROWS], 1);
#pragma unroll
            for (int j = 0; j < J; ++j) x[j] = 0.0;
        }
#pragma unroll
        for (int j = 0; j < J; ++j) o[j] = (TO)x[j];
    }
}

template <typename TB, typename TO, int J>
ptk_status launch_solve(ptk_ctx* ctx, const SolveJob& job, cudaStream_t st) {
    int64_t grid = std::min<int64_t>(ceil_div(job.rows, 128), (int64_t)ctx->sm_count * 8);
    if (grid < 1) return PTK_OK;
    { solve_kernel<TB, TO, J><<<(unsigned)grid, 128, 0, st>>>((const TB*)job.rowbuf, job.row_ptr, job.rows, job.lambda,
                                                           (TO*)job.out, job.ld, ctx->d_flags); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

template <typename TB, typename TO>
ptk_status dispatch_solve(ptk_ctx* ctx, const SolveJob& job, cudaStream_t st) {
    switch (job.J) {
#define PTK_CASE(J) \
    case J:         \
        return launch_solve<TB, TO, J>(ctx, job, st);
        PTK_CASE(1) PTK_CASE(2) PTK_CASE(3) PTK_CASE(4) PTK_CASE(5) PTK_CASE(6) PTK_CASE(7) PTK_CASE(8)
        PTK_CASE(9) PTK_CASE(10) PTK_CASE(11) PTK_CASE(12) PTK_CASE(13) PTK_CASE(14) PTK_CASE(15) PTK_CASE(16)
#undef PTK_CASE
        default:
            set_error("solve: J=%d unsupported", job.J);
            return PTK_ERR_UNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// reductions: per-thread partials, per-block FP64, then one ordered block.
constexpr int RT = 256;

__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    __syncthreads();
    return s;
}

__global__ void final_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    double s = block_sum_d(v, sh);
    if (threadIdx.x == 0) *out = s;
}

// residual^2 of slice-ordered entries: x - <delta_e, a^(n)_{rid(e)}>
template <typename T>
__global__ void resid_sq(const T* __restrict__ delta, int ld, int Jn, const int32_t* __restrict__ row_col,
                         int64_t row_stride, int64_t n, const T* __restrict__ A, int64_t fld, double* __restrict__ part) {
    __shared__ double sh[32];
    T acc = T(0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const T* d = delta + e * ld;
        const T* a = A + (int64_t)row_col[e * row_stride] * fld;
        T xh = T(0);
        for (int j = 0; j < Jn; ++j) xh = fma(d[j], a[j], xh);
        T r = d[Jn] - xh;
        acc = fma(r, r, acc);
    }
    double s = block_sum_d((double)acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void sumsq_rows(const T* __restrict__ A, int64_t rows, int J, int64_t ld, double* __restrict__ part) {
    __shared__ double sh[32];
    T acc = T(0);
    const int64_t total = rows * J;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        T v = A[(t / J) * ld + (t % J)];
        acc = fma(v, v, acc);
    }
    double s = block_sum_d((double)acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void nonzero_count(const T* __restrict__ G, int64_t size, double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < size; t += (int64_t)gridDim.x * blockDim.x)
        acc += G[t] != T(0) ? 1.0 : 0.0;
    double s = block_sum_d(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[e] = <delta_e, a_{row(e)}>, row(e) = row_of[e] or row_col[e * row_stride]
template <typename T>
__global__ void dot_rows_kernel(const T* __restrict__ delta, int ld, int Jn, const int32_t* __restrict__ row_of,
                                const int32_t* __restrict__ row_col, int64_t row_stride, int64_t n,
                                const T* __restrict__ A, int64_t fld, T* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of ? row_of[e] : row_col[e * row_stride];
        const T* d = delta + e * ld;
        const T* a = A + (int64_t)r * fld;
        T xh = T(0);
        for (int j = 0; j < Jn; ++j) xh = fma(d[j], a[j], xh);
        out[e] = xh;
    }
}

int red_grid(ptk_ctx* ctx, int64_t n) {
    int64_t g = std::min<int64_t>(ceil_div(n > 0 ? n : 1, RT), (int64_t)ctx->sm_count * 4);
    return (int)std::max<int64_t>(g, 1);
}

}  // namespace

ptk_status solve_rows(ptk_ctx* ctx, const SolveJob& job, cudaStream_t st) {
    if (job.buf_dtype == PTK_F64) {
        if (job.out_dtype == PTK_F64) return dispatch_solve<double, double>(ctx, job, st);
        return dispatch_solve<double, float>(ctx, job, st);
    }
    if (job.out_dtype == PTK_F64) return dispatch_solve<float, double>(ctx, job, st);
    return dispatch_solve<float, float>(ctx, job, st);
}

ptk_status error_from_delta(ptk_ctx* ctx, const void* delta, int ld, int Jn, const int32_t* row_col,
                            int64_t row_stride, int64_t n, const void* factor, int64_t fld, ptk_dtype dtype,
                            double* d_out, cudaStream_t st) {
    int g = red_grid(ctx, n);
    double* part = (double*)scratch(ctx, SLOT_RED, sizeof(double) * (size_t)g);
    if (!part) return PTK_ERR_OUT_OF_MEMORY;
    if (dtype == PTK_F64)
        { resid_sq<double><<<g, RT, 0, st>>>((const double*)delta, ld, Jn, row_col, row_stride, n,
                                           (const double*)factor, fld, part); ::ptk::note_launch(); }
    else
        { resid_sq<float><<<g, RT, 0, st>>>((const float*)delta, ld, Jn, row_col, row_stride, n,
                                          (const float*)factor, fld, part); ::ptk::note_launch(); }
    { final_sum<<<1, RT, 0, st>>>(part, g, d_out); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status sumsq_factors(ptk_ctx* ctx, const ptk_model* m, double* d_out, cudaStream_t st) {
    // d_out[n] = ||A^(n)||_F^2 for each mode
    for (int n = 0; n < m->order; ++n) {
        int64_t total = m->dims[n] * m->J[n];
        int g = red_grid(ctx, total);
        double* part = (double*)scratch(ctx, SLOT_RED, sizeof(double) * (size_t)g);
        if (!part) return PTK_ERR_OUT_OF_MEMORY;
        if (m->dtype == PTK_F64)
            { sumsq_rows<double><<<g, RT, 0, st>>>((const double*)m->factors[n], m->dims[n], m->J[n], m->ld[n], part); ::ptk::note_launch(); }
        else
            { sumsq_rows<float><<<g, RT, 0, st>>>((const float*)m->factors[n], m->dims[n], m->J[n], m->ld[n], part); ::ptk::note_launch(); }
        { final_sum<<<1, RT, 0, st>>>(part, g, d_out + n); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
    }
    return PTK_OK;
}

ptk_status count_nonzero(ptk_ctx* ctx, const void* core, int64_t size, ptk_dtype dtype, double* d_out,
                         cudaStream_t st) {
    int g = red_grid(ctx, size);
    double* part = (double*)scratch(ctx, SLOT_RED, sizeof(double) * (size_t)g);
    if (!part) return PTK_ERR_OUT_OF_MEMORY;
    if (dtype == PTK_F64)
        { nonzero_count<double><<<g, RT, 0, st>>>((const double*)core, size, part); ::ptk::note_launch(); }
    else
        { nonzero_count<float><<<g, RT, 0, st>>>((const float*)core, size, part); ::ptk::note_launch(); }
    { final_sum<<<1, RT, 0, st>>>(part, g, d_out); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

ptk_status dot_rows(ptk_ctx* ctx, const void* delta, int ld, int Jn, const int32_t* row_of, const int32_t* row_col,
                    int64_t row_stride, int64_t n, const void* factor, int64_t fld, ptk_dtype dtype, void* out,
                    cudaStream_t st) {
    if (n == 0) return PTK_OK;
    int g = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->sm_count * 16);
    if (dtype == PTK_F64)
        { dot_rows_kernel<double><<<g, 256, 0, st>>>((const double*)delta, ld, Jn, row_of, row_col, row_stride, n,
                                                   (const double*)factor, fld, (double*)out); ::ptk::note_launch(); }
    else
        { dot_rows_kernel<float><<<g, 256, 0, st>>>((const float*)delta, ld, Jn, row_of, row_col, row_stride, n,
                                                  (const float*)factor, fld, (float*)out); ::ptk::note_launch(); }
    PTK_LAUNCH_CHECK();
    return PTK_OK;
}

}  // namespace ptk
