/*
 * kpm_oracle.c -- CPU oracle for the KPM moment sweep.  TEST INFRASTRUCTURE
 * ONLY: it is called by the tests, by smoke() and by the benchmark's CPU
 * baseline, never by the library.  It shares no code with the CUDA path.
 *
 * Plain, slow, obviously correct FP64 code that follows the paper
 * (Lin, Saad, Yang, "Approximating spectral densities of large matrices"):
 *
 *  - random start vectors: Theorem 3.1 needs E[v] = 0, E[v v^T] = I
 *    (eq. stochasticcondition).  Rademacher +-1 entries satisfy it.  The signs
 *    come from the splitmix64 generator (Steele, Lea, Flood, OOPSLA 2014),
 *    written here from its published definition.
 *  - the shift/scale B = (A - cI)/d with c = (lb+ub)/2, d = (ub-lb)/2
 *    (eq. cd, Section 3.1).
 *  - the Chebyshev three-term recurrence v_{k+1} = 2 B v_k - v_{k-1},
 *    v_1 = B v_0 (eq. 3term, Algorithm 1).
 *  - moments, "direct" mode: zeta_k = v_0^T v_k for k = 0..M (Algorithm 1).
 *  - moments, "doubling" mode (Appendix A): with p = ceil(k/2), q = k - p,
 *    T_{p+q} = 2 T_p T_q - T_{|p-q|}, hence
 *    v_0^T T_k(B) v_0 = 2 v_p^T v_q - v_0^T T_{|p-q|}(B) v_0.
 *    (The paper prints the sign of the last term as "+"; the product formula
 *    T_p T_q = (T_{p+q} + T_{|p-q|})/2 fixes it as "-".)
 *  - Legendre moments (Algorithm DGL, Section 3.1.3): v_1 = B v_0,
 *    v_{k+1} = ((2k+1) B v_k - k v_{k-1}) / (k+1), nu_k = v_0^T v_k.
 *
 * Normalisation: each vector's moment is mu_k^(l) = v_l^T T_k(B) v_l / n, so
 * that the average over the n_v vectors is
 * mu_k = (1/(n n_v)) sum_l v_l^T T_k(B) v_l.  The paper's coefficient
 * (2 - delta_k0)/pi (eq. expmu, eq. muEst) is applied at reconstruction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_GAMMA 0x9e3779b97f4a7c15ULL

/* splitmix64: the state advances by the golden-ratio increment, and the
 * output is the state passed through two xor-shift-multiply rounds. */
uint64_t oracle_splitmix64_next(uint64_t *state) {
    uint64_t z;
    *state += ORACLE_GAMMA;
    z = *state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* The +-1 entry of start vector l of matrix b at (original) row i.
 * A 64-bit word is the splitmix64 output number ctr+1 of the stream seeded
 * with `seed` (i.e. the state seed + (ctr+1)*gamma), where
 * ctr = b * 2^48 + floor(l/64) * 2^32 + i; the entry takes bit (l mod 64)
 * of that word: 0 -> +1, 1 -> -1. */
double oracle_rademacher(uint64_t seed, uint64_t b, uint64_t l, uint64_t i) {
    uint64_t ctr = (b << 48) + ((l >> 6) << 32) + i;
    uint64_t state = seed + ctr * ORACLE_GAMMA; /* next() adds one more gamma */
    uint64_t word = oracle_splitmix64_next(&state);
    return ((word >> (l & 63)) & 1ULL) ? -1.0 : 1.0;
}

/* The n x n_v block of start vectors, row-major: out[i*n_v + l]. */
void oracle_start_block(int64_t n, int64_t n_v, int64_t vec_offset, uint64_t seed,
                        uint64_t batch_index, double *out) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t l = 0; l < n_v; ++l)
            out[i * n_v + l] = oracle_rademacher(seed, batch_index, (uint64_t)(vec_offset + l), (uint64_t)i);
}

/* y = A x for a CSR matrix. */
static void spmv(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                 const double *val, const double *x, double *y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * x[col_idx[e]];
        y[i] = s;
    }
}

/* y = B x with B = (A - cI)/d. */
static void apply_B(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *val, double c, double d, const double *x, double *y) {
    spmv(n, row_ptr, col_idx, val, x, y);
    for (int64_t i = 0; i < n; ++i) y[i] = (y[i] - c * x[i]) / d;
}

/* x^T y; `reverse` sums from the last row to the first (used only to measure
 * how much the rounding order alone moves the result). */
static double dot(int64_t n, const double *x, const double *y, int reverse) {
    double s = 0.0;
    if (!reverse) {
        for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
    } else {
        for (int64_t i = n - 1; i >= 0; --i) s += x[i] * y[i];
    }
    return s;
}

/*
 * Per-vector moments mu_per_vec[l*(M+1) + k] = v_l^T T_k(B) v_l / n for
 * l = 0..n_v-1 (start vector index vec_offset + l of matrix `batch_index`).
 * mode 0 = direct (M matrix-vector products), 1 = doubling (ceil(M/2)),
 * 2 = Legendre: mu_per_vec[l*(M+1) + k] = v_l^T L_k(B) v_l / n (M products).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_kpm_moments(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *val, double lb, double ub, int M, int64_t n_v,
                       int64_t vec_offset, uint64_t seed, uint64_t batch_index, int mode,
                       int reverse, int nthreads, double *mu_per_vec) {
    if (n <= 0 || M < 0 || n_v <= 0 || !(ub > lb) || (mode < 0 || mode > 2)) return -1;
    const double c = 0.5 * (lb + ub);
    const double d = 0.5 * (ub - lb);
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t l = 0; l < n_v; ++l) {
        double *v0 = malloc(sizeof(double) * n);
        double *vprev = malloc(sizeof(double) * n);
        double *vcur = malloc(sizeof(double) * n);
        double *vnext = malloc(sizeof(double) * n);
        double *mu = mu_per_vec + l * (int64_t)(M + 1);
        if (!v0 || !vprev || !vcur || !vnext) {
            failed = 1;
        } else {
            for (int64_t i = 0; i < n; ++i)
                v0[i] = oracle_rademacher(seed, batch_index, (uint64_t)(vec_offset + l), (uint64_t)i);
            double dn = (double)n;
            if (mode == 0) {
                /* Algorithm 1: zeta_k = v_0^T v_k, v_{k+1} = 2 B v_k - v_{k-1}. */
                memcpy(vcur, v0, sizeof(double) * n);
                mu[0] = dot(n, v0, vcur, reverse) / dn;
                if (M >= 1) {
                    apply_B(n, row_ptr, col_idx, val, c, d, v0, vnext);   /* v_1 = B v_0 */
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                    mu[1] = dot(n, v0, vcur, reverse) / dn;
                }
                for (int k = 1; k < M; ++k) {
                    apply_B(n, row_ptr, col_idx, val, c, d, vcur, vnext);
                    for (int64_t i = 0; i < n; ++i) vnext[i] = 2.0 * vnext[i] - vprev[i];
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                    mu[k + 1] = dot(n, v0, vcur, reverse) / dn;
                }
            } else if (mode == 2) {
                /* Algorithm DGL: the Legendre three-term recurrence, direct dots. */
                memcpy(vcur, v0, sizeof(double) * n);
                mu[0] = dot(n, v0, vcur, reverse) / dn;
                if (M >= 1) {
                    apply_B(n, row_ptr, col_idx, val, c, d, v0, vnext);   /* v_1 = B v_0 */
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                    mu[1] = dot(n, v0, vcur, reverse) / dn;
                }
                for (int k = 1; k < M; ++k) {
                    apply_B(n, row_ptr, col_idx, val, c, d, vcur, vnext);
                    const double a = (2.0 * k + 1.0) / (k + 1.0), b = (double)k / (k + 1.0);
                    for (int64_t i = 0; i < n; ++i) vnext[i] = a * vnext[i] - b * vprev[i];
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                    mu[k + 1] = dot(n, v0, vcur, reverse) / dn;
                }
            } else {
                /* Appendix A doubling: after v_j is formed, the moments whose
                 * p = ceil(k/2) equals j are k = 2j-1 (q = j-1, |p-q| = 1) and
                 * k = 2j (q = j, |p-q| = 0). */
                memcpy(vcur, v0, sizeof(double) * n);
                mu[0] = dot(n, v0, v0, reverse) / dn;
                if (M >= 1) {
                    apply_B(n, row_ptr, col_idx, val, c, d, v0, vnext);   /* v_1 */
                    mu[1] = dot(n, vnext, v0, reverse) / dn;
                    if (M >= 2) mu[2] = 2.0 * dot(n, vnext, vnext, reverse) / dn - mu[0];
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                }
                for (int j = 2; 2 * j - 1 <= M; ++j) {
                    apply_B(n, row_ptr, col_idx, val, c, d, vcur, vnext);
                    for (int64_t i = 0; i < n; ++i) vnext[i] = 2.0 * vnext[i] - vprev[i];
                    /* vnext = v_j, vcur = v_{j-1} */
                    mu[2 * j - 1] = 2.0 * dot(n, vnext, vcur, reverse) / dn - mu[1];
                    if (2 * j <= M) mu[2 * j] = 2.0 * dot(n, vnext, vnext, reverse) / dn - mu[0];
                    memcpy(vprev, vcur, sizeof(double) * n);
                    memcpy(vcur, vnext, sizeof(double) * n);
                }
            }
        }
        free(v0);
        free(vprev);
        free(vcur);
        free(vnext);
    }
    return failed ? -1 : 0;
}

/* Gershgorin discs: every eigenvalue lies in some [a_ii - r_i, a_ii + r_i]
 * with r_i = sum_{j != i} |a_ij| (a textbook bound; the paper instead derives
 * its bounds from a short Lanczos run, Section 3.1). */
void oracle_gershgorin(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *val, double *lb, double *ub) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double center = 0.0, radius = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if ((int64_t)col_idx[e] == i) center += val[e];
            else radius += fabs(val[e]);
        }
        if (center - radius < lo) lo = center - radius;
        if (center + radius > hi) hi = center + radius;
    }
    *lb = lo;
    *ub = hi;
}

/* Plain CSR y = A x, exposed for the Lanczos oracle. */
void oracle_spmv(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                 const double *val, const double *x, double *y) {
    spmv(n, row_ptr, col_idx, val, x, y);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
