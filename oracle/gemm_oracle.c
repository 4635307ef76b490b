/*
 * FP64 CPU oracle for generalized matrix multiplication, C = alpha*A*B + beta*C
 * (the Tiramisu paper's running example, Section I; also its sgemm benchmark,
 * Section VI-A).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load this file's shared object.  It shares no code, header
 * or constant with the CUDA library and never calls it.
 *
 * What it computes is the plain definition, element by element:
 *     out[i][j] = alpha * sum_k A[i][k] * B[k][j] + beta * C0[i][j]
 * with every FP32 input widened to double and the sum taken in double, k in
 * increasing order (an i-k-j loop nest), rows split over OpenMP threads.
 * Each product of two widened floats is exact in double (24 + 24 < 53 bits).
 *
 * BLAS conventions (the paper does not state them; reference-BLAS reading):
 *   - matrices are row-major: A is M x K (lda >= K), B is K x N (ldb >= N),
 *     C0 is M x N (ldc >= N);
 *   - beta == 0: C0 is not read, so NaN/Inf in it do not propagate;
 *   - alpha == 0 or K == 0: A and B are not read and the result is beta*C0.
 */
#include <stdint.h>
#include <stddef.h>

static void oracle_row(int64_t i, int64_t N, int64_t K, double alpha,
                       const float* A, int64_t lda, const float* B, int64_t ldb,
                       double beta, const float* C0, int64_t ldc, double* orow)
{
    for (int64_t j = 0; j < N; ++j) orow[j] = 0.0;
    if (alpha != 0.0) {
        for (int64_t k = 0; k < K; ++k) {
            const double a = (double)A[i * lda + k];
            const float* brow = B + k * ldb;
            for (int64_t j = 0; j < N; ++j) orow[j] += a * (double)brow[j];
        }
    }
    for (int64_t j = 0; j < N; ++j) {
        double v = (alpha != 0.0) ? alpha * orow[j] : 0.0;
        if (beta != 0.0) v += beta * (double)C0[i * ldc + j];
        orow[j] = v;
    }
}

/* Full result: out is M x N with leading dimension ldo. */
void oracle_gemm_f64(int64_t M, int64_t N, int64_t K, float alpha,
                     const float* A, int64_t lda, const float* B, int64_t ldb,
                     float beta, const float* C0, int64_t ldc,
                     double* out, int64_t ldo)
{
    const double da = (double)alpha, db = (double)beta;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < M; ++i)
        oracle_row(i, N, K, da, A, lda, B, ldb, db, C0, ldc, out + i * ldo);
}

/* Selected rows only (for sampled checks at sizes where the full product is
 * too slow on a CPU): out is nrows x N, row r holds result row rows[r]. */
void oracle_gemm_f64_rows(int64_t N, int64_t K, float alpha,
                          const float* A, int64_t lda, const float* B, int64_t ldb,
                          float beta, const float* C0, int64_t ldc,
                          const int64_t* rows, int64_t nrows, double* out)
{
    const double da = (double)alpha, db = (double)beta;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r)
        oracle_row(rows[r], N, K, da, A, lda, B, ldb, db, C0, ldc, out + r * N);
}

/* The last step of the definition on its own: out = alpha * P + beta * C0,
 * where P holds the sums sum_k A[i][k] * B[k][j] in double (oracle_gemm_f64
 * with alpha = 1, beta = 0 computes them: 1 * sum is exact).  The same
 * arithmetic as oracle_row's last loop, so that the two steps give the
 * one-step result bit for bit; one product then serves several (alpha,
 * beta) pairs.  C0 is not read when beta == 0; alpha == 0 ignores P. */
void oracle_axpby_f64(int64_t M, int64_t N, float alpha, const double* P, int64_t ldp,
                      float beta, const float* C0, int64_t ldc, double* out, int64_t ldo)
{
    const double da = (double)alpha, db = (double)beta;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            double v = (da != 0.0) ? da * P[i * ldp + j] : 0.0;
            if (db != 0.0) v += db * (double)C0[i * ldc + j];
            out[i * ldo + j] = v;
        }
    }
}

/* The same definition evaluated in FP32 arithmetic, the accuracy of a plain
 * single-precision gemm: for each element, acc = 0 and, k in increasing
 * order, acc = fl(acc + fl(a_ik * b_kj)) (every operation rounded to nearest
 * FP32, no fused multiply-add: the file is compiled with -ffp-contract=off);
 * then out = fl(fl(alpha * acc) + fl(beta * c0)), or fl(alpha * acc) when
 * beta == 0.  Its error against the FP64 result is bounded by the classical
 * recursive-summation bound gamma_(K+2) * (|alpha| sum_k |a||b| + |beta c0|),
 * gamma_n = n u / (1 - n u), u = 2^-24.  out is M x N float (ldo). */
void oracle_gemm_f32_seq(int64_t M, int64_t N, int64_t K, float alpha,
                         const float* A, int64_t lda, const float* B, int64_t ldb,
                         float beta, const float* C0, int64_t ldc,
                         float* out, int64_t ldo)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            float acc = 0.0f;
            if (alpha != 0.0f) {
                for (int64_t k = 0; k < K; ++k) {
                    const float p = A[i * lda + k] * B[k * ldb + j];
                    acc = acc + p;
                }
            }
            float v = (alpha != 0.0f) ? alpha * acc : 0.0f;
            if (beta != 0.0f) {
                const float c = beta * C0[i * ldc + j];
                v = v + c;
            }
            out[i * ldo + j] = v;
        }
    }
}

/* Relative Frobenius error ||got - ref||_F / ||ref||_F, in double.  When the
 * reference is all zero the absolute Frobenius norm of the difference is
 * returned instead.  got is M x N float (ldg), ref M x N double (ldr). */
double oracle_rel_frob(int64_t M, int64_t N, const float* got, int64_t ldg,
                       const double* ref, int64_t ldr)
{
    double num = 0.0, den = 0.0;
    #pragma omp parallel for reduction(+:num,den) schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            const double r = ref[i * ldr + j];
            const double d = (double)got[i * ldg + j] - r;
            num += d * d;
            den += r * r;
        }
    }
    if (den == 0.0) return __builtin_sqrt(num);
    return __builtin_sqrt(num / den);
}

/* Sets the number of OpenMP threads of the loops above (for timing the
 * oracle on one core and on all of them). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Threads the OpenMP loops above use (for reporting the CPU baseline). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
