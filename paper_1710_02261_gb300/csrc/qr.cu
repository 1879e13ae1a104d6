// qr.cu -- Alg. 2 final loop: A^(n) = Q^(n) R^(n), A^(n) <- Q^(n),
// G <- G x_n R^(n) for n = 1..N (Sec. 3.1).  The thin QR of the tall I_n x J_n
// factor is taken as CholeskyQR2 in FP64: W = A^T A, W = R^T R (Cholesky),
// A <- A R^{-1}, done twice, with R = R_2 R_1 (positive diagonal, the same R as
// a Householder QR normalised to a positive diagonal).  The n-mode product of
// Sec. 2.1 with U = R: (G x_n R)_{..k..} = sum_j G_{..j..} R[k][j].
#include "common.cuh"

namespace ptk {
namespace {

constexpr int QT = 256;

template <typename T>
__global__ void ata_partial(const T* __restrict__ A, int64_t rows, int J, int64_t ld, double* __restrict__ part) {
    __shared__ double tile[QT][PTK_MAX_RANK + 1];
    const int ntri = J * (J + 1) / 2;
    // (j,k) pair of this thread
    int pj = 0, pk = 0;
    if ((int)threadIdx.x < ntri) {
        int t = threadIdx.x, j = 0;
        while (t >= J - j) {
            t -= J - j;
            ++j;
        }
        pj = j;
        pk = j + t;
    }
    double acc = 0.0;
    for (int64_t r0 = (int64_t)blockIdx.x * QT; r0 < rows; r0 += (int64_t)gridDim.x * QT) {
        const int64_t r = r0 + threadIdx.x;
        for (int j = 0; j < J; ++j) tile[threadIdx.x][j] = r < rows ? (double)A[r * ld + j] : 0.0;
        __syncthreads();
        if ((int)threadIdx.x < ntri) {
            const int cnt = (int)min((int64_t)QT, rows - r0);
            for (int i = 0; i < cnt; ++i) acc += tile[i][pj] * tile[i][pk];
        }
        __syncthreads();
    }
    if ((int)threadIdx.x < ntri) part[(int64_t)blockIdx.x * ntri + threadIdx.x] = acc;
}

// Cholesky of W (summed from the block partials): W = R^T R, R upper; also R^{-1}.
// Rtot <- R * Rtot (or R when first).
__global__ void chol_upper(const double* __restrict__ part, int nblocks, int J, double* __restrict__ R,
                           double* __restrict__ Rinv, double* __restrict__ Rtot, int first, int* flags) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int ntri = J * (J + 1) / 2;
    double W[PTK_MAX_RANK][PTK_MAX_RANK];
    for (int t = 0, j = 0; j < J; ++j)
        for (int k = j; k < J; ++k, ++t) {
            double s = 0.0;
            for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * ntri + t];
            W[j][k] = s;
            W[k][j] = s;
        }
    // R^T R = W, R upper (row-major R[i][j], i <= j)
    for (int i = 0; i < J; ++i)
        for (int j = 0; j < J; ++j) R[i * J + j] = 0.0;
    for (int i = 0; i < J; ++i) {
        double s = W[i][i];
        for (int k = 0; k < i; ++k) s -= R[k * J + i] * R[k * J + i];
        if (!(s > 0.0)) {
            atomicAdd(&flags[FLAG_BAD_ROWS], 1);
            s = 1e-300;
        }
        const double d = sqrt(s);
        R[i * J + i] = d;
        for (int j = i + 1; j < J; ++j) {
            double t = W[i][j];
            for (int k = 0; k < i; ++k) t -= R[k * J + i] * R[k * J + j];
            R[i * J + j] = t / d;
        }
    }
    // R^{-1} (upper) by back substitution on columns of I
    for (int c = 0; c < J; ++c) {
        for (int i = J - 1; i >= 0; --i) {
            double s = i == c ? 1.0 : 0.0;
            for (int k = i + 1; k < J; ++k) s -= R[i * J + k] * Rinv[k * J + c];
            Rinv[i * J + c] = s / R[i * J + i];
        }
    }
    double tmp[PTK_MAX_RANK * PTK_MAX_RANK];
    for (int i = 0; i < J; ++i)
        for (int j = 0; j < J; ++j) {
            double s = 0.0;
            if (first)
                s = R[i * J + j];
            else
                for (int k = 0; k < J; ++k) s += R[i * J + k] * Rtot[k * J + j];
            tmp[i * J + j] = s;
        }
    for (int t = 0; t < J * J; ++t) Rtot[t] = tmp[t];
}

template <typename T>
__global__ void apply_rinv(T* __restrict__ A, int64_t rows, int J, int64_t ld, const double* __restrict__ Rinv) {
    __shared__ double Ri[PTK_MAX_RANK * PTK_MAX_RANK];
    for (int t = threadIdx.x; t < J * J; t += blockDim.x) Ri[t] = Rinv[t];
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        double a[PTK_MAX_RANK], o[PTK_MAX_RANK];
        for (int j = 0; j < J; ++j) a[j] = (double)A[r * ld + j];
        for (int j = 0; j < J; ++j) {
            double s = 0.0;
            for (int k = 0; k <= j; ++k) s += a[k] * Ri[k * J + j];
            o[j] = s;
        }
        for (int j = 0; j < J; ++j) A[r * ld + j] = (T)o[j];
    }
}

struct Shape8 {
    int order;
    int J[PTK_MAX_ORDER];
};

template <typename T>
__global__ void core_times_r(const T* __restrict__ G, T* __restrict__ Gout, Shape8 s, int mode,
                             const double* __restrict__ R, int64_t size) {
    int64_t stride = 1;
    for (int k = s.order - 1; k > mode; --k) stride *= s.J[k];
    const int Jn = s.J[mode];
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < size; b += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)((b / stride) % Jn);
        const int64_t base = b - (int64_t)k * stride;
        double acc = 0.0;
        for (int j = 0; j < Jn; ++j) acc += (double)G[base + (int64_t)j * stride] * R[k * Jn + j];
        Gout[b] = (T)acc;
    }
}

template <typename T>
ptk_status run(ptk_ctx* ctx, ptk_model* m, cudaStream_t st) {
    int64_t gsize = 1;
    Shape8 sh;
    sh.order = m->order;
    for (int k = 0; k < m->order; ++k) {
        gsize *= m->J[k];
        sh.J[k] = m->J[k];
    }
    const int nb = ctx->sm_count * 2;
    const int JJ = PTK_MAX_RANK * PTK_MAX_RANK;
    double* buf = (double*)scratch(ctx, SLOT_QR, sizeof(double) * ((size_t)nb * 136 + 3 * JJ));
    T* gtmp = (T*)scratch(ctx, SLOT_GPERM, sizeof(T) * (size_t)gsize);
    if (!buf || !gtmp) return PTK_ERR_OUT_OF_MEMORY;
    double* part = buf;
    double* R = buf + (size_t)nb * 136;
    double* Rinv = R + JJ;
    double* Rtot = Rinv + JJ;
    for (int n = 0; n < m->order; ++n) {
        const int J = m->J[n];
        T* A = (T*)m->factors[n];
        const int64_t rows = m->dims[n];
        const int g = (int)std::min<int64_t>(ceil_div(rows, QT), nb);
        for (int pass = 0; pass < 2; ++pass) {
            { ata_partial<T><<<g, QT, 0, st>>>(A, rows, J, m->ld[n], part); ::ptk::note_launch(); }
            { chol_upper<<<1, 32, 0, st>>>(part, g, J, R, Rinv, Rtot, pass == 0, ctx->d_flags); ::ptk::note_launch(); }
            { apply_rinv<T><<<(int)std::min<int64_t>(ceil_div(rows, 256), ctx->sm_count * 8), 256, 0, st>>>(
                A, rows, J, m->ld[n], Rinv); ::ptk::note_launch(); }
            PTK_LAUNCH_CHECK();
        }
        { core_times_r<T><<<(int)std::min<int64_t>(ceil_div(gsize, 256), ctx->sm_count * 8), 256, 0, st>>>(
            (const T*)m->core, gtmp, sh, n, Rtot, gsize); ::ptk::note_launch(); }
        PTK_LAUNCH_CHECK();
        PTK_CUDA(cudaMemcpyAsync(m->core, gtmp, sizeof(T) * (size_t)gsize, cudaMemcpyDeviceToDevice, st));
    }
    return PTK_OK;
}

}  // namespace

ptk_status qr_finalize_impl(ptk_ctx* ctx, ptk_model* m, cudaStream_t st) {
    if (m->dtype == PTK_F64) return run<double>(ctx, m, st);
    return run<float>(ctx, m, st);
}

}  // namespace ptk
