/*
 * ptk_oracle.c -- plain, slow, FP64 CPU oracle for P-Tucker (Oh, Park, Sael,
 * Kang, "Scalable Tucker Factorization for Sparse Tensors -- Algorithms and
 * Discoveries", arXiv 1710.02261).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark load this file.  It shares no code, header, table
 * or helper with the CUDA library; neither side includes the other.
 *
 * Conventions: indices are 0-based (the paper is 1-based, Sec. 2.1); the core
 * G is dense in C order over (j_1..j_N) (last index fastest); factor A^(n) is
 * row-major [I_n][J_n]; the observed set Omega is a list idx[E][N] + vals[E]
 * (duplicates allowed, each one counts as an observation).  Everything is
 * double precision and every loop follows the paper's order of operations:
 * products are taken as G_beta * a^(1) * a^(2) * ... (mode order), sums run
 * over entries in slice order and over core entries in C order.
 *
 * Every function below is pinned by a test that does not call the function it
 * checks (brute-force dense reconstruction, closed-form ridge regression, the
 * paper's invariants); the header comment of each names its passage.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAX_ORDER 16

static int64_t core_size(int N, const int32_t* J) {
    int64_t s = 1;
    for (int k = 0; k < N; ++k) s *= J[k];
    return s;
}

/* multi-index of core entry beta (C order) */
static void core_index(int N, const int32_t* J, int64_t beta, int32_t* j) {
    for (int k = N - 1; k >= 0; --k) {
        j[k] = (int32_t)(beta % J[k]);
        beta /= J[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Omega^(n)_{i_n}: entries whose n-th index is i_n (Table 1; Alg. 3, the loop
 * over alpha in Omega^(n)_{i_n}).  Stable grouping by counting: perm lists the
 * entry ids of row 0, then row 1, ..., each in input order; row_ptr[I_n+1]. */
int ora_slices(int N, const int64_t* dims, int64_t E, const int32_t* idx, int mode,
               int64_t* perm, int64_t* row_ptr) {
    int64_t I = dims[mode];
    for (int64_t i = 0; i <= I; ++i) row_ptr[i] = 0;
    for (int64_t e = 0; e < E; ++e) {
        int32_t i = idx[e * N + mode];
        if (i < 0 || i >= I) return -1;
        row_ptr[i + 1] += 1;
    }
    for (int64_t i = 0; i < I; ++i) row_ptr[i + 1] += row_ptr[i];
    int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I > 0 ? I : 1));
    if (!cursor) return -2;
    for (int64_t i = 0; i < I; ++i) cursor[i] = row_ptr[i];
    for (int64_t e = 0; e < E; ++e) perm[cursor[idx[e * N + mode]]++] = e;
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (delta): delta(j) = sum over beta with j_n = j of G_beta * prod_{k!=n}
 * a^(k)_{i_k j_k}.  Zero core entries (truncated by P-Tucker-Approx) are
 * skipped, which leaves the sum unchanged. */
void ora_delta(int N, const int32_t* J, const double* G, double* const* A,
               const int32_t* coord, int mode, double* delta) {
    int64_t Gs = core_size(N, J);
    int32_t j[ORA_MAX_ORDER];
    for (int t = 0; t < J[mode]; ++t) delta[t] = 0.0;
    for (int64_t b = 0; b < Gs; ++b) {
        if (G[b] == 0.0) continue;
        core_index(N, J, b, j);
        double p = G[b];
        for (int k = 0; k < N; ++k) {
            if (k == mode) continue;
            p *= A[k][(int64_t)coord[k] * J[k] + j[k]];
        }
        delta[j[mode]] += p;
    }
}

/* Eq. (recon2): X_hat(alpha) = sum_beta G_beta prod_n a^(n)_{i_n j_n}. */
static double predict_one(int N, const int32_t* J, const double* G, double* const* A,
                          const int32_t* coord) {
    int64_t Gs = core_size(N, J);
    int32_t j[ORA_MAX_ORDER];
    double s = 0.0;
    for (int64_t b = 0; b < Gs; ++b) {
        if (G[b] == 0.0) continue;
        core_index(N, J, b, j);
        double p = G[b];
        for (int k = 0; k < N; ++k) p *= A[k][(int64_t)coord[k] * J[k] + j[k]];
        s += p;
    }
    return s;
}

void ora_predict(int N, const int32_t* J, const double* G, double* const* A, int64_t n,
                 const int32_t* coords, double* out) {
    for (int64_t e = 0; e < n; ++e) out[e] = predict_one(N, J, G, A, coords + e * N);
}

/* Eq. (reconfull) squared: sum over Omega of (X_alpha - X_hat(alpha))^2. */
double ora_sse(int N, const int32_t* J, const double* G, double* const* A, int64_t E,
               const int32_t* idx, const double* vals) {
    double s = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        double r = vals[e] - predict_one(N, J, G, A, idx + e * N);
        s += r * r;
    }
    return s;
}

/* Eq. (TF_PARTIAL): sse + lambda * sum_n ||A^(n)||_F^2. */
double ora_loss(int N, const int64_t* dims, const int32_t* J, const double* G, double* const* A,
                int64_t E, const int32_t* idx, const double* vals, double lambda) {
    double reg = 0.0;
    for (int k = 0; k < N; ++k)
        for (int64_t t = 0; t < dims[k] * J[k]; ++t) reg += A[k][t] * A[k][t];
    return ora_sse(N, J, G, A, E, idx, vals) + lambda * reg;
}

/* ------------------------------------------------------------------------ */
/* Row update, Eq. (rowupdate): a = c (B + lambda I)^{-1}.  B + lambda I is
 * symmetric positive definite (Sec. 3.2), so the row is the solution of
 * (B + lambda I) a^T = c^T, taken here by a textbook Cholesky factorisation
 * L L^T followed by forward and back substitution.  Returns 0, or 1 when a
 * pivot is not positive. */
int ora_spd_solve(int n, const double* B, const double* c, double lambda, double* a) {
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    double* y = (double*)calloc((size_t)n, sizeof(double));
    if (!L || !y) { free(L); free(y); return 2; }
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = B[i * n + j] + (i == j ? lambda : 0.0);
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) { bad = 1; s = 1.0; }
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = c[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * a[k];
        a[i] = s / L[i * n + i];
    }
    free(L);
    free(y);
    return bad;
}

/* Eqs. (rowB), (rowC): B = sum_alpha delta delta^T, c = sum_alpha x_alpha delta
 * over the given entries (in the given order), then the row by Eq. (rowupdate).
 * B (J_n x J_n, full) and c may be NULL. */
int ora_row_update(int N, const int32_t* J, const double* G, double* const* A, int mode,
                   int64_t m, const int64_t* entries, const int32_t* idx, const double* vals,
                   double lambda, double* row, double* B_out, double* c_out) {
    int Jn = J[mode];
    double* B = (double*)calloc((size_t)Jn * Jn, sizeof(double));
    double* c = (double*)calloc((size_t)Jn, sizeof(double));
    double* d = (double*)calloc((size_t)Jn, sizeof(double));
    if (!B || !c || !d) { free(B); free(c); free(d); return 2; }
    for (int64_t t = 0; t < m; ++t) {
        int64_t e = entries ? entries[t] : t;
        ora_delta(N, J, G, A, idx + e * N, mode, d);
        for (int p = 0; p < Jn; ++p) {
            for (int q = 0; q < Jn; ++q) B[p * Jn + q] += d[p] * d[q];
            c[p] += vals[e] * d[p];
        }
    }
    int rc = ora_spd_solve(Jn, B, c, lambda, row);
    if (B_out) memcpy(B_out, B, sizeof(double) * Jn * Jn);
    if (c_out) memcpy(c_out, c, sizeof(double) * Jn);
    free(B); free(c); free(d);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 for one mode n (plain P-Tucker): every row i_n of A^(n) is replaced
 * by its row-update result over Omega^(n)_{i_n}.  Rows are independent
 * (Sec. 3.2), so they run in parallel with dynamic scheduling (Sec. 3.4); each
 * row's arithmetic is sequential, so the result does not depend on the thread
 * count.  An empty slice gives B = 0, c = 0 and hence the zero row. */
int ora_update_mode(int N, const int64_t* dims, const int32_t* J, int64_t E, const int32_t* idx,
                    const double* vals, const double* G, double** A, int mode, double lambda,
                    int nthreads) {
    int64_t I = dims[mode];
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I + 1));
    if (!perm || !rp) { free(perm); free(rp); return 2; }
    if (ora_slices(N, dims, E, idx, mode, perm, rp) != 0) { free(perm); free(rp); return 1; }
    int bad = 0;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : bad)
    for (int64_t i = 0; i < I; ++i) {
        double row[64];
        int rc = ora_row_update(N, J, G, (double* const*)A, mode, rp[i + 1] - rp[i], perm + rp[i],
                                idx, vals, lambda, row, NULL, NULL);
        bad += rc != 0;
        for (int j = 0; j < J[mode]; ++j) A[mode][i * J[mode] + j] = row[j];
    }
    free(perm);
    free(rp);
    return bad ? 3 : 0;
}

/* ------------------------------------------------------------------------ */
/* P-Tucker-Cache (Alg. 3 with the cache table Pres, Sec. 3.3):
 *   Pres[alpha][beta] = G_beta prod_{k=1..N} a^(k)_{i_k j_k}   (precompute)
 *   delta(j_n) += Pres[alpha][beta] / a^(n)_{i_n j_n}          (O(1) per pair)
 *   after mode n: Pres[alpha][beta] = Pres / a_old * a_new
 * When the divisor a is exactly 0 the products are taken as plain P-Tucker
 * does (Sec. 3.3).  Pres is E x |G| doubles. */
static double pres_fresh(int N, const int32_t* J, const double* G, double* const* A,
                         const int32_t* coord, int64_t b, const int32_t* j) {
    double p = G[b];
    for (int k = 0; k < N; ++k) p *= A[k][(int64_t)coord[k] * J[k] + j[k]];
    return p;
}

int ora_sweep_cache(int N, const int64_t* dims, const int32_t* J, int64_t E, const int32_t* idx,
                    const double* vals, const double* G, double** A, double lambda, int nthreads) {
    int64_t Gs = core_size(N, J);
    double* pres = (double*)malloc(sizeof(double) * (size_t)(E * Gs > 0 ? E * Gs : 1));
    if (!pres) return 2;
    (void)nthreads;
    /* precompute the table Pres (P-Tucker-Cache, before the mode loop), rows split evenly over threads */
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t e = 0; e < E; ++e) {
        int32_t j[ORA_MAX_ORDER];
        for (int64_t b = 0; b < Gs; ++b) {
            core_index(N, J, b, j);
            pres[e * Gs + b] = pres_fresh(N, J, G, (double* const*)A, idx + e * N, b, j);
        }
    }
    int bad = 0;
    for (int n = 0; n < N; ++n) {
        int64_t I = dims[n];
        int Jn = J[n];
        int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
        int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(I + 1));
        double* aold = (double*)malloc(sizeof(double) * (size_t)(I * Jn > 0 ? I * Jn : 1));
        if (!perm || !rp || !aold) { free(perm); free(rp); free(aold); free(pres); return 2; }
        ora_slices(N, dims, E, idx, n, perm, rp);
        memcpy(aold, A[n], sizeof(double) * (size_t)(I * Jn));
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : bad)
        for (int64_t i = 0; i < I; ++i) {
            double B[64 * 64], c[64], d[64], row[64];
            int32_t j[ORA_MAX_ORDER];
            for (int p = 0; p < Jn * Jn; ++p) B[p] = 0.0;
            for (int p = 0; p < Jn; ++p) c[p] = 0.0;
            for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
                int64_t e = perm[t];
                const int32_t* co = idx + e * N;
                for (int p = 0; p < Jn; ++p) d[p] = 0.0;
                for (int64_t b = 0; b < Gs; ++b) {
                    core_index(N, J, b, j);
                    double a = A[n][(int64_t)co[n] * Jn + j[n]];
                    if (a != 0.0) {
                        d[j[n]] += pres[e * Gs + b] / a;
                    } else {
                        double p = G[b];
                        for (int k = 0; k < N; ++k)
                            if (k != n) p *= A[k][(int64_t)co[k] * J[k] + j[k]];
                        d[j[n]] += p;
                    }
                }
                for (int p = 0; p < Jn; ++p) {
                    for (int q = 0; q < Jn; ++q) B[p * Jn + q] += d[p] * d[q];
                    c[p] += vals[e] * d[p];
                }
            }
            bad += ora_spd_solve(Jn, B, c, lambda, row) != 0;
            for (int p = 0; p < Jn; ++p) A[n][i * Jn + p] = row[p];
        }
        /* update Pres with the old and new A^(n) (P-Tucker-Cache, after the mode's row updates) */
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t e = 0; e < E; ++e) {
            int32_t j[ORA_MAX_ORDER];
            const int32_t* co = idx + e * N;
            for (int64_t b = 0; b < Gs; ++b) {
                core_index(N, J, b, j);
                double ao = aold[(int64_t)co[n] * Jn + j[n]];
                double an = A[n][(int64_t)co[n] * Jn + j[n]];
                if (ao != 0.0)
                    pres[e * Gs + b] = pres[e * Gs + b] / ao * an;
                else
                    pres[e * Gs + b] = pres_fresh(N, J, G, (double* const*)A, co, b, j);
            }
        }
        free(perm); free(rp); free(aold);
    }
    free(pres);
    return bad ? 3 : 0;
}

/* Alg. 3, plain variant: modes in order 1..N (Gauss-Seidel across modes). */
int ora_sweep(int N, const int64_t* dims, const int32_t* J, int64_t E, const int32_t* idx,
              const double* vals, const double* G, double** A, double lambda, int nthreads) {
    int rc = 0;
    for (int n = 0; n < N; ++n) {
        int r = ora_update_mode(N, dims, J, E, idx, vals, G, A, n, lambda, nthreads);
        if (r) rc = r;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* P-Tucker-Approx, Eq. (recon_partial).  R(beta) is the part of the squared
 * reconstruction error that core entry beta is responsible for.
 *   literal:    sum_alpha [ (x - sum_gamma p_gamma)^2 - (x - sum_{gamma!=beta} p_gamma)^2 ]
 *   simplified: sum_alpha p_beta ( -2 x + p_beta + 2 sum_{gamma!=beta} p_gamma )
 * with p_gamma = G_gamma prod_n a^(n)_{i_n j_n}.  Entries already removed
 * (G_beta = 0) get R = 0.  The literal form costs O(E |G|^2) (tiny inputs). */
void ora_partial_error(int N, const int32_t* J, const double* G, double* const* A, int64_t E,
                       const int32_t* idx, const double* vals, int literal, double* R) {
    int64_t Gs = core_size(N, J);
    int32_t j[ORA_MAX_ORDER];
    double* p = (double*)malloc(sizeof(double) * (size_t)Gs);
    for (int64_t b = 0; b < Gs; ++b) R[b] = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* co = idx + e * N;
        double x = vals[e];
        for (int64_t b = 0; b < Gs; ++b) {
            core_index(N, J, b, j);
            p[b] = pres_fresh(N, J, G, A, co, b, j);
        }
        if (literal) {
            double full = 0.0;
            for (int64_t g = 0; g < Gs; ++g) full += p[g];
            for (int64_t b = 0; b < Gs; ++b) {
                if (G[b] == 0.0) continue;
                double rest = 0.0;
                for (int64_t g = 0; g < Gs; ++g)
                    if (g != b) rest += p[g];
                R[b] += (x - full) * (x - full) - (x - rest) * (x - rest);
            }
        } else {
            double full = 0.0;
            for (int64_t g = 0; g < Gs; ++g) full += p[g];
            for (int64_t b = 0; b < Gs; ++b) {
                if (G[b] == 0.0) continue;
                double others = full - p[b];
                R[b] += p[b] * (-2.0 * x + p[b] + 2.0 * others);
            }
        }
    }
    free(p);
}

/* Alg. 4, the truncation step: among the current non-zero core entries, remove (set to
 * 0) floor(p * nnz) of them -- the largest R(beta) first (rule 0), or the
 * smallest |G_beta| first (rule 1, the truncated-SVD-like criterion the paper
 * contrasts with in Sec. 3.3).  Ties go to the lower C-order index.  Returns
 * the number removed. */
typedef struct { double key; int64_t b; } ora_kv;
static int cmp_desc(const void* x, const void* y) {
    const ora_kv* a = (const ora_kv*)x; const ora_kv* c = (const ora_kv*)y;
    if (a->key > c->key) return -1;
    if (a->key < c->key) return 1;
    return (a->b > c->b) - (a->b < c->b);
}
static int cmp_asc(const void* x, const void* y) {
    const ora_kv* a = (const ora_kv*)x; const ora_kv* c = (const ora_kv*)y;
    if (a->key < c->key) return -1;
    if (a->key > c->key) return 1;
    return (a->b > c->b) - (a->b < c->b);
}
int64_t ora_truncate(int N, const int32_t* J, double* G, const double* R, double p, int rule,
                     int64_t* removed) {
    int64_t Gs = core_size(N, J), nnz = 0;
    ora_kv* kv = (ora_kv*)malloc(sizeof(ora_kv) * (size_t)Gs);
    for (int64_t b = 0; b < Gs; ++b) {
        if (G[b] == 0.0) continue;
        kv[nnz].key = rule == 0 ? R[b] : fabs(G[b]);
        kv[nnz].b = b;
        ++nnz;
    }
    qsort(kv, (size_t)nnz, sizeof(ora_kv), rule == 0 ? cmp_desc : cmp_asc);
    int64_t k = (int64_t)floor(p * (double)nnz);
    for (int64_t t = 0; t < k; ++t) {
        G[kv[t].b] = 0.0;
        if (removed) removed[t] = kv[t].b;
    }
    free(kv);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2, the finalisation after the sweeps: A^(n) = Q R (Householder, Golub & Van Loan Alg. 5.2.1,
 * R with a positive diagonal), A^(n) <- Q, G <- G x_n R, for n = 1..N in
 * order.  The n-mode product follows Sec. 2.1: (G x_n R)_{..k..} = sum_j
 * G_{..j..} R[k][j].  Requires I_n >= J_n; returns 1 otherwise. */
static void householder_qr(int64_t m, int n, double* A, double* R) {
    /* A (m x n, row-major) is overwritten by the thin Q */
    double* V = (double*)calloc((size_t)(m * n), sizeof(double));
    double* W = (double*)malloc(sizeof(double) * (size_t)m);
    double* beta = (double*)calloc((size_t)n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        double norm = 0.0;
        for (int64_t i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
        norm = sqrt(norm);
        double x0 = A[k * n + k];
        double alpha = x0 >= 0 ? -norm : norm;
        for (int64_t i = 0; i < m; ++i) W[i] = 0.0;
        for (int64_t i = k; i < m; ++i) W[i] = A[i * n + k];
        W[k] = x0 - alpha;
        double vv = 0.0;
        for (int64_t i = k; i < m; ++i) vv += W[i] * W[i];
        beta[k] = vv > 0 ? 2.0 / vv : 0.0;
        for (int64_t i = k; i < m; ++i) V[i * n + k] = W[i];
        for (int c = k; c < n; ++c) {
            double s = 0.0;
            for (int64_t i = k; i < m; ++i) s += W[i] * A[i * n + c];
            s *= beta[k];
            for (int64_t i = k; i < m; ++i) A[i * n + c] -= s * W[i];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) R[r * n + c] = c >= r ? A[r * n + c] : 0.0;
    /* thin Q = H_0 H_1 ... H_{n-1} [I_n; 0] */
    for (int64_t i = 0; i < m; ++i)
        for (int c = 0; c < n; ++c) A[i * n + c] = (i == c) ? 1.0 : 0.0;
    for (int k = n - 1; k >= 0; --k) {
        for (int c = 0; c < n; ++c) {
            double s = 0.0;
            for (int64_t i = k; i < m; ++i) s += V[i * n + k] * A[i * n + c];
            s *= beta[k];
            for (int64_t i = k; i < m; ++i) A[i * n + c] -= s * V[i * n + k];
        }
    }
    /* positive diagonal of R */
    for (int r = 0; r < n; ++r) {
        if (R[r * n + r] < 0) {
            for (int c = 0; c < n; ++c) R[r * n + c] = -R[r * n + c];
            for (int64_t i = 0; i < m; ++i) A[i * n + r] = -A[i * n + r];
        }
    }
    free(V); free(W); free(beta);
}

int ora_qr_finalize(int N, const int64_t* dims, const int32_t* J, double* G, double** A) {
    int64_t Gs = core_size(N, J);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)Gs);
    int32_t j[ORA_MAX_ORDER];
    for (int n = 0; n < N; ++n) {
        if (dims[n] < J[n]) { free(tmp); return 1; }
        int Jn = J[n];
        double* R = (double*)malloc(sizeof(double) * (size_t)(Jn * Jn));
        householder_qr(dims[n], Jn, A[n], R);
        /* G <- G x_n R */
        for (int64_t b = 0; b < Gs; ++b) {
            core_index(N, J, b, j);
            int k = j[n];
            double s = 0.0;
            int64_t stride = 1;
            for (int t = N - 1; t > n; --t) stride *= J[t];
            int64_t base = b - (int64_t)k * stride;
            for (int q = 0; q < Jn; ++q) s += G[base + (int64_t)q * stride] * R[k * Jn + q];
            tmp[b] = s;
        }
        memcpy(G, tmp, sizeof(double) * (size_t)Gs);
        free(R);
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: repeat { Alg. 3; error by Eq. (reconfull); Approx: Alg. 4 } until
 * max_sweeps, or until the relative change of the error falls below tol
 * (tol <= 0 disables the test); then, if finalize, the QR step.
 * variant: 0 plain, 1 cache, 2 approx.  errors_out[max_sweeps] receives the
 * error after each sweep (before truncation).  Returns the sweeps run, or a
 * negative code. */
int ora_fit(int N, const int64_t* dims, const int32_t* J, int64_t E, const int32_t* idx,
            const double* vals, double* G, double** A, double lambda, int variant,
            int max_sweeps, double tol, double trunc_p, int trunc_rule, int finalize,
            int nthreads, double* errors_out) {
    int64_t Gs = core_size(N, J);
    double prev = -1.0;
    int s;
    for (s = 0; s < max_sweeps; ++s) {
        int rc = variant == 1 ? ora_sweep_cache(N, dims, J, E, idx, vals, G, A, lambda, nthreads)
                              : ora_sweep(N, dims, J, E, idx, vals, G, A, lambda, nthreads);
        if (rc == 2) return -2;
        double err = sqrt(ora_sse(N, J, G, (double* const*)A, E, idx, vals));
        if (errors_out) errors_out[s] = err;
        if (variant == 2) {
            double* R = (double*)malloc(sizeof(double) * (size_t)Gs);
            if (trunc_rule == 0)
                ora_partial_error(N, J, G, (double* const*)A, E, idx, vals, 0, R);
            ora_truncate(N, J, G, R, trunc_p, trunc_rule, NULL);
            free(R);
        }
        if (tol > 0 && prev > 0 && fabs(err - prev) / prev < tol) { ++s; break; }
        prev = err;
    }
    if (finalize && ora_qr_finalize(N, dims, J, G, A) != 0) return -1;
    return s;
}

int ora_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
