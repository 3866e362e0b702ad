// KPML and the Delta-Gauss-Legendre method (Sections 3.1.1, 3.1.3, Appendix B), FP64.
//
// Legendre moments from Chebyshev moments.  For fixed start vectors
// nu_k = (1/(n n_v)) sum_l v_l^T L_k(B) v_l is linear in the Chebyshev moments
// mu_j of the same vectors through the Chebyshev expansion of L_k:
//     L_k(t) = sum_{m=0}^{floor(k/2)} e_{k-2m} h_m h_{k-m} T_{k-2m}(t),
//     h_m = (2m)! / (4^m (m!)^2) = prod_{i<m} (2i+1)/(2i+2),  e_0 = 1, e_j = 2.
// (Check: L_2 = (3/4) T_2 + 1/4, L_3 = (5/8) T_3 + (3/8) T_1.)  All coefficients
// are non-negative and sum to L_k(1) = 1, so nu_k is a convex combination of
// mu_0..mu_k: the doubling Chebyshev sweep gives in ceil(M/2) passes what the
// Legendre recurrence of Algorithm DGL gives in M.
//
// KPML: phi_L(t) = sum_k (k + 1/2) nu_k L_k(t) by the forward three-term
// recurrence (k+1) L_{k+1} = (2k+1) t L_k - k L_{k-1} (|L_k| <= 1 on [-1, 1]),
// with the coefficients (2k+1)/(k+1) and k/(k+1) from a table.
//
// DGL: gamma_k(t) by Eq. gam0 and the joint recurrence of Eq. Leg3, stopped by
// Eq. StopRecur, one thread per point.
//
// Gauss-Legendre nodes for blurring KPML: Newton's method on L_N from the
// asymptotic first guess cos(pi (i + 3/4) / (N + 1/2)), with
// L_N'(x) = N (x L_N - L_{N-1}) / (x^2 - 1) and weights 2 / ((1 - x^2) L_N'(x)^2).
#include <cuda_runtime.h>
#include <math.h>

#include "dos_internal.h"

namespace dos {
namespace {

int grid_for_points(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// h[m] for m = 0..M, sequential products (M+1 values, one thread).
__global__ void leg_h_kernel(int M, double *__restrict__ h) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double v = 1.0;
    h[0] = v;
    for (int m = 0; m < M; ++m) {
        v *= (2.0 * m + 1.0) / (2.0 * m + 2.0);
        h[m + 1] = v;
    }
}

// nu[r][k] = sum_m e_{k-2m} h_m h_{k-m} mu[r][k-2m], m ascending.
__global__ void cheb_to_leg_kernel(const double *__restrict__ mu, int64_t count, int M,
                                   const double *__restrict__ h, double *__restrict__ nu) {
    const int64_t per = (int64_t)M + 1, total = count * per;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / per;
        const int k = (int)(q - r * per);
        const double *m_row = mu + r * per;
        double s = 0.0;
        for (int m = 0; 2 * m <= k; ++m) {
            const int j = k - 2 * m;
            s = fma((j == 0 ? 1.0 : 2.0) * h[m] * h[k - m], m_row[j], s);
        }
        nu[q] = s;
    }
}

// ab[2k] = (2k+1)/(k+1), ab[2k+1] = k/(k+1): the recurrence coefficients, so the
// per-point loops below need no FP64 division (a long dependent sequence here).
__global__ void leg_coef_kernel(int K, double *__restrict__ ab) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        ab[2 * k] = (2.0 * k + 1.0) / (k + 1.0);
        ab[2 * k + 1] = (double)k / (k + 1.0);
    }
}

__device__ __forceinline__ double kpml_at(const double *__restrict__ nu, int M,
                                          const double *__restrict__ ab, double t) {
    double Lp = 0.0, Lc = 1.0;      // L_{k-1}, L_k
    double s = 0.5 * nu[0];
    for (int k = 0; k < M; ++k) {
        const double Ln = fma(ab[2 * k] * t, Lc, -ab[2 * k + 1] * Lp);
        Lp = Lc;
        Lc = Ln;
        s = fma((k + 1.5) * nu[k + 1], Lc, s);
    }
    return s;
}

// out_t[i] = phi_L(t_i) (times w[i] if given), out_l[i] = phi_L(t_i) / d.
__global__ void kpml_kernel(const double *__restrict__ nu, int M, const double *__restrict__ ab,
                            const double *__restrict__ t, const double *__restrict__ w, int N,
                            double inv_d, double *__restrict__ out_t, double *__restrict__ out_l) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double ti = t ? t[i] : -cospi((i + 0.5) / (double)N);
        const double v = kpml_at(nu, M, ab, ti);
        out_t[i] = w ? w[i] * v : v;
        if (out_l) out_l[i] = v * inv_d;
    }
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]; y[i] = c + d t[i].
__global__ void gauss_legendre_kernel(int N, const double *__restrict__ ab, double c, double d,
                                      double *__restrict__ t, double *__restrict__ w,
                                      double *__restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double x = cospi((i + 0.75) / (N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;    // L_0, L_1
            for (int k = 1; k < N; ++k) {
                const double p2 = fma(ab[2 * k] * x, p1, -ab[2 * k + 1] * p0);
                p0 = p1;
                p1 = p2;
            }
            dp = N * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) <= 5e-16) break;
        }
        // one more evaluation at the converged node for the weight
        double p0 = 1.0, p1 = x;
        for (int k = 1; k < N; ++k) {
            const double p2 = fma(ab[2 * k] * x, p1, -ab[2 * k + 1] * p0);
            p0 = p1;
            p1 = p2;
        }
        dp = N * (x * p1 - p0) / (x * x - 1.0);
        const int o = N - 1 - i;
        t[o] = x;
        w[o] = 2.0 / ((1.0 - x * x) * dp * dp);
        if (y) y[o] = c + d * x;
    }
}

// DGL at points x (eigenvalue units, or the uniform grid x0 + m h).
__global__ void dgl_kernel(const double *__restrict__ nu, int M, double c, double d, double sigma,
                           double tol, const double *__restrict__ x, double x0, double h, int N,
                           double *__restrict__ phi, int *__restrict__ used) {
    const double s = sigma / d, s2 = s * s, r = M_SQRT2 * s;
    const double pref = 1.0 / (sqrt(2.0 * M_PI) * s * d);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double xi = x ? x[i] : x0 + i * h;
        const double t = (xi - c) / d;
        const double g0 = s * sqrt(0.5 * M_PI) * (erf((1.0 - t) / r) + erf((1.0 + t) / r));
        const double ep = exp(-0.5 * ((1.0 - t) / s) * ((1.0 - t) / s));
        const double em = exp(-0.5 * ((1.0 + t) / s) * ((1.0 + t) / s));
        double gp = 0.0, gc = g0;          // gamma_{k-1}, gamma_k
        double pp = 0.0, pc = 0.0;         // psi_{k-1}, psi_k
        double acc = 0.5 * g0 * nu[0];
        int k = 0;
        while (k < M) {
            const double zeta = (k & 1) ? ep + em : ep - em;
            const double gn = ((2.0 * k + 1.0) * (s2 * (pc - zeta) + t * gc) - k * gp) / (k + 1.0);
            const double pn = (2.0 * k + 1.0) * gc + pp;
            gp = gc;
            gc = gn;
            pp = pc;
            pc = pn;
            ++k;
            acc = fma((k + 0.5) * gc, nu[k], acc);
            if (tol > 0.0 && fabs(gp) + fabs(gc) <= k * tol) break;
        }
        phi[i] = pref * acc;
        if (used) used[i] = k;
    }
}

}  // namespace

void launch_cheb_to_legendre(const double *mu, int64_t count, int M, double *h_scratch,
                             double *nu, cudaStream_t s) {
    leg_h_kernel<<<1, 32, 0, s>>>(M, h_scratch);
    DOS_LAUNCHED();
    cheb_to_leg_kernel<<<grid_for_points(count * (M + 1), 256, 152 * 16), 256, 0, s>>>(
        mu, count, M, h_scratch, nu);
    DOS_LAUNCHED();
}

void launch_kpml(const double *nu, int M, const double *t, const double *w, int N, double inv_d,
                 double *out_t, double *out_l, double *coef_scratch, cudaStream_t s) {
    leg_coef_kernel<<<grid_for_points(M + 1, 256, 152 * 4), 256, 0, s>>>(M + 1, coef_scratch);
    DOS_LAUNCHED();
    kpml_kernel<<<grid_for_points(N, 128, 152 * 16), 128, 0, s>>>(nu, M, coef_scratch, t, w, N,
                                                                  inv_d, out_t, out_l);
    DOS_LAUNCHED();
}

void launch_gauss_legendre(int N, double c, double d, double *t, double *w, double *y,
                           double *coef_scratch, cudaStream_t s) {
    leg_coef_kernel<<<grid_for_points(N + 1, 256, 152 * 4), 256, 0, s>>>(N + 1, coef_scratch);
    DOS_LAUNCHED();
    gauss_legendre_kernel<<<grid_for_points(N, 128, 152 * 16), 128, 0, s>>>(N, coef_scratch, c, d,
                                                                           t, w, y);
    DOS_LAUNCHED();
}

void launch_dgl(const double *nu, int M, double c, double d, double sigma, double tol,
                const double *x, double x0, double h, int N, double *phi, int *used,
                cudaStream_t s) {
    dgl_kernel<<<grid_for_points(N, 128, 152 * 16), 128, 0, s>>>(nu, M, c, d, sigma, tol, x, x0,
                                                                 h, N, phi, used);
    DOS_LAUNCHED();
}

}  // namespace dos
