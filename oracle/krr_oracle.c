/*
 * Plain CPU oracle for Gaussian-kernel ridge regression on genotype data.
 *
 * TEST INFRASTRUCTURE ONLY.  The parity tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this library; the product path (the
 * CUDA library and its Python binding) never does, and shares no code with it.
 *
 * Everything is written the obvious way: int64 for integer sums, IEEE double
 * for every floating-point quantity, loops in the order the definitions read.
 * OpenMP (when available) only splits independent outer loops.
 *
 * Layouts: row-major.  A genotype matrix with n rows (patients) and m columns
 * (SNPs) has element (i,k) at g[i*ld + k].  Dense square matrices have
 * element (i,j) at a[i*n + j].
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Squared Euclidean distance between every row of G1 and every row of G2,
 * summed term by term: d_ij = sum_k (g1_ik - g2_jk)^2.
 * This is the definition of the distance used by the Gaussian kernel
 * (Alg. 5, first branch) and the quantity the paper's distance section
 * (Sec. IV-B, "Engaging INT8 Tensor Cores for Distance Calculations")
 * writes out element by element.  Exact in int64.
 */
void oracle_sqdist_bruteforce(const int8_t *g1, int64_t n1, int64_t ld1,
                              const int8_t *g2, int64_t n2, int64_t ld2,
                              int64_t m, int64_t *d) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n1; ++i) {
        const int8_t *a = g1 + i * ld1;
        for (int64_t j = 0; j < n2; ++j) {
            const int8_t *b = g2 + j * ld2;
            int64_t s = 0;
            for (int64_t k = 0; k < m; ++k) {
                int64_t t = (int64_t)a[k] - (int64_t)b[k];
                s += t * t;
            }
            d[i * n2 + j] = s;
        }
    }
}

/*
 * The same distances through the paper's Gram identity (Sec. IV-B worked
 * example): a matrix holding the squared row norms down its columns, plus
 * its transpose, minus twice the Gram matrix G1 G2^T.
 * Here n_i = sum_k g1_ik^2, q_j = sum_k g2_jk^2, s_ij = sum_k g1_ik g2_jk and
 * d_ij = n_i + q_j - 2 s_ij.  Exact in int64.  The tests check that it
 * agrees with the term-by-term definition above.
 */
void oracle_sqdist_gram(const int8_t *g1, int64_t n1, int64_t ld1,
                        const int8_t *g2, int64_t n2, int64_t ld2,
                        int64_t m, int64_t *d) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n1; ++i) {
        const int8_t *a = g1 + i * ld1;
        int64_t ni = 0;
        for (int64_t k = 0; k < m; ++k) ni += (int64_t)a[k] * a[k];
        for (int64_t j = 0; j < n2; ++j) {
            const int8_t *b = g2 + j * ld2;
            int64_t qj = 0, s = 0;
            for (int64_t k = 0; k < m; ++k) {
                qj += (int64_t)b[k] * b[k];
                s += (int64_t)a[k] * b[k];
            }
            d[i * n2 + j] = ni + qj - 2 * s;
        }
    }
}

/*
 * Gaussian kernel of Alg. 5: K_ij = exp(-gamma * d_ij), in double with the
 * C library exp.
 */
void oracle_gaussian_kernel(const int64_t *d, int64_t count, double gamma,
                            double *k) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) k[t] = exp(-gamma * (double)d[t]);
}

/*
 * Cholesky factorisation A = L L^T of a symmetric positive definite n x n
 * matrix (Alg. 3, "Factorize").  Column-by-column (left-looking) form:
 *   L_jj = sqrt(A_jj - sum_{p<j} L_jp^2)
 *   L_ij = (A_ij - sum_{p<j} L_ip L_jp) / L_jj     for i > j.
 * Reads the lower triangle of a, writes L into the lower triangle and zeros
 * above the diagonal.  Returns -1 on success, else the first column whose
 * pivot is not positive (a is then partly overwritten).
 */
int64_t oracle_cholesky(double *a, int64_t n) {
    for (int64_t j = 0; j < n; ++j) {
        double *rj = a + j * n;
        double s = rj[j];
        for (int64_t p = 0; p < j; ++p) s -= rj[p] * rj[p];
        if (!(s > 0.0)) return j;
        double ljj = sqrt(s);
        rj[j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double *ri = a + i * n;
            double t = ri[j];
            for (int64_t p = 0; p < j; ++p) t -= ri[p] * rj[p];
            ri[j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) a[i * n + j] = 0.0;
    return -1;
}

/*
 * Forward substitution L Z = Y for p right-hand sides (first half of Alg. 3,
 * "Solve").  L is n x n lower triangular (row-major, as written by
 * oracle_cholesky); y is n x p row-major and is overwritten by Z.
 */
void oracle_forward_subst(const double *l, int64_t n, double *y, int64_t p) {
    for (int64_t i = 0; i < n; ++i) {
        const double *ri = l + i * n;
        for (int64_t c = 0; c < p; ++c) {
            double t = y[i * p + c];
            for (int64_t k = 0; k < i; ++k) t -= ri[k] * y[k * p + c];
            y[i * p + c] = t / ri[i];
        }
    }
}

/*
 * Backward substitution L^T X = Z for p right-hand sides (second half of
 * Alg. 3, "Solve").  z is n x p row-major and is overwritten by X.
 */
void oracle_backward_subst(const double *l, int64_t n, double *z, int64_t p) {
    for (int64_t i = n - 1; i >= 0; --i) {
        for (int64_t c = 0; c < p; ++c) {
            double t = z[i * p + c];
            for (int64_t k = i + 1; k < n; ++k) t -= l[k * n + i] * z[k * p + c];
            z[i * p + c] = t / l[i * n + i];
        }
    }
}

/*
 * Plain matrix product C = A B with A (r x q) and B (q x p), row-major,
 * double accumulation in index order.  Used for the prediction product of
 * Alg. 4 and for residuals.
 */
void oracle_matmul(const double *a, int64_t r, int64_t q, const double *b,
                   int64_t p, double *c) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < r; ++i) {
        for (int64_t j = 0; j < p; ++j) c[i * p + j] = 0.0;
        for (int64_t k = 0; k < q; ++k) {
            double aik = a[i * q + k];
            for (int64_t j = 0; j < p; ++j) c[i * p + j] += aik * b[k * p + j];
        }
    }
}

/*
 * Rows of the kernel matrix against a fixed set of training rows, computed
 * straight from the definition: out[s*n2 + j] = exp(-gamma * d(g1_s, g2_j))
 * for each requested row index rows[s] of G1.  Lets a test check a residual
 * on a sample of rows of a problem too large to build whole.
 */
void oracle_kernel_rows(const int8_t *g1, int64_t ld1, const int64_t *rows,
                        int64_t nrows, const int8_t *g2, int64_t n2, int64_t ld2,
                        int64_t m, double gamma, double *out) {
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
    for (int64_t s = 0; s < nrows; ++s) {
        for (int64_t j = 0; j < n2; ++j) {
            const int8_t *a = g1 + rows[s] * ld1;
            const int8_t *b = g2 + j * ld2;
            int64_t t = 0;
            for (int64_t k = 0; k < m; ++k) {
                int64_t u = (int64_t)a[k] - (int64_t)b[k];
                t += u * u;
            }
            out[s * n2 + j] = exp(-gamma * (double)t);
        }
    }
}

/*
 * Identity-by-state allele counts (Alg. 5, second branch): for each pair of
 * rows, the number of alleles the two patients share identical by state,
 * summed over the m loci.  At one locus genotypes a and b (copies of the
 * minor allele, 0..2) share 2 - |a - b| alleles: the same genotype shares
 * both, genotypes one apart share one, opposite homozygotes share none.
 * Exact in int64.
 */
void oracle_ibs_count(const int8_t *g1, int64_t n1, int64_t ld1,
                      const int8_t *g2, int64_t n2, int64_t ld2,
                      int64_t m, int64_t *out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n1; ++i) {
        const int8_t *a = g1 + i * ld1;
        for (int64_t j = 0; j < n2; ++j) {
            const int8_t *b = g2 + j * ld2;
            int64_t s = 0;
            for (int64_t k = 0; k < m; ++k) {
                int64_t t = (int64_t)a[k] - (int64_t)b[k];
                s += 2 - (t < 0 ? -t : t);
            }
            out[i * n2 + j] = s;
        }
    }
}

/*
 * Squared Euclidean distances between real-valued confounder rows (age,
 * sex, principal components, ...), term by term in double:
 * dc_ij = sum_q (c1_iq - c2_jq)^2.  The paper adds these to the integer
 * genotype distances before the exponential of the Gaussian kernel
 * (Sec. IV-B, distance section).
 */
void oracle_conf_sqdist(const double *c1, int64_t n1, int64_t ld1,
                        const double *c2, int64_t n2, int64_t ld2,
                        int64_t nc, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n1; ++i) {
        for (int64_t j = 0; j < n2; ++j) {
            double s = 0.0;
            for (int64_t q = 0; q < nc; ++q) {
                double t = c1[i * ld1 + q] - c2[j * ld2 + q];
                s += t * t;
            }
            out[i * n2 + j] = s;
        }
    }
}
