// Reconstruction (step a6) and the smoothed error metric (step a7), FP64.
//
// Coefficients a_k = (2 - delta_k0) g_k mu_k with g_k the Jackson factors of
// Appendix A (Eq. jackson, alpha_M = pi/(M+2)) or 1; the polynomial
// P(t) = sum_k a_k T_k(t) is evaluated by Clenshaw's recurrence, and
//     phi_hat(t) = P(t) / (pi sqrt(1 - t^2))           (Eq. tdosFinal, Eq. expmu).
// The blurred KPM density <phi_tilde, g_sigma(. - x)> is the Gauss-Chebyshev sum
//     (1/N_q) sum_i P(t_i) g_sigma(x - c - d t_i),  t_i = cos(pi (i + 1/2)/N_q),
// the blurred exact density (1/n) sum_j g_sigma(x - lambda_j) (Eq. blurphi with
// the 1/n of Eq. DOS0), g_sigma the Gaussian of Eq. gauss.
#include <cuda_runtime.h>
#include <math.h>

#include "dos_internal.h"

namespace dos {
namespace {

__global__ void coef_kernel(const double *__restrict__ mu, int M, int damping,
                            double *__restrict__ a) {
    const double alpha = M_PI / (double)(M + 2);
    const double sa = sin(alpha), ca = cos(alpha);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= M; k += gridDim.x * blockDim.x) {
        double g = 1.0;
        if (damping == DOS_DAMP_JACKSON) {
            const double ka = k * alpha;
            g = ((1.0 - (double)k / (M + 2)) * sa * cos(ka) + ca * sin(ka) / (M + 2)) / sa;
        }
        a[k] = (k == 0 ? 1.0 : 2.0) * g * mu[k];
    }
}

__device__ __forceinline__ double clenshaw(const double *__restrict__ a, int M, double t) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = M; k >= 1; --k) {
        const double b0 = fma(2.0 * t, b1, a[k] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(t, b1, a[0] - b2);
}

__global__ void reconstruct_kernel(const double *__restrict__ a, int M, double d,
                                   const double *__restrict__ t, int N_t,
                                   double *__restrict__ phi_hat, double *__restrict__ phi_lambda) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_t; i += gridDim.x * blockDim.x) {
        const double ti = t ? t[i] : -cospi((i + 0.5) / (double)N_t);
        const double v = clenshaw(a, M, ti) / (M_PI * sqrt((1.0 - ti) * (1.0 + ti)));
        phi_hat[i] = v;
        if (phi_lambda) phi_lambda[i] = v / d;
    }
}

// Many moment rows at once: row b of mu (stride ldm) -> coefficients (stride M+1)
// -> phi_hat row b (stride N_t), the same arithmetic as the single-row kernels.
__global__ void coef_rows_kernel(const double *__restrict__ mu, int64_t ldm, int B, int M,
                                 int damping, double *__restrict__ a) {
    const double alpha = M_PI / (double)(M + 2);
    const double sa = sin(alpha), ca = cos(alpha);
    const int64_t total = (int64_t)B * (M + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / (M + 1);
        const int k = (int)(e - b * (M + 1));
        double g = 1.0;
        if (damping == DOS_DAMP_JACKSON) {
            const double ka = k * alpha;
            g = ((1.0 - (double)k / (M + 2)) * sa * cos(ka) + ca * sin(ka) / (M + 2)) / sa;
        }
        a[e] = (k == 0 ? 1.0 : 2.0) * g * mu[b * ldm + k];
    }
}

__global__ void reconstruct_rows_kernel(const double *__restrict__ a, int B, int M,
                                        const double *__restrict__ t, int N_t,
                                        double *__restrict__ phi_hat) {
    const int64_t total = (int64_t)B * N_t;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / N_t;
        const int i = (int)(e - b * N_t);
        const double ti = t ? t[i] : -cospi((i + 0.5) / (double)N_t);
        phi_hat[e] = clenshaw(a + b * (M + 1), M, ti) / (M_PI * sqrt((1.0 - ti) * (1.0 + ti)));
    }
}

// P(t_i) and the node's position c + d t_i in eigenvalue units.
__global__ void nodes_kernel(const double *__restrict__ a, int M, int N_q, double c, double d,
                             double *__restrict__ P, double *__restrict__ Y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N_q; i += gridDim.x * blockDim.x) {
        const double t = cospi((i + 0.5) / (double)N_q);
        P[i] = clenshaw(a, M, t);
        Y[i] = c + d * t;
    }
}

__device__ __forceinline__ double gauss(double u, double inv_sigma, double norm) {
    const double z = u * inv_sigma;
    return norm * exp(-0.5 * z * z);
}

// One block per grid point x_m; fixed-order block sums (reproducible).
__device__ __forceinline__ double block_sum_d(double s) {
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    __syncthreads();
    return tot;
}

__global__ void blur_kpm_kernel(const double *__restrict__ P, const double *__restrict__ Y, int N_q,
                                double sigma, double x0, double h, int N_x, double *out) {
    const double inv_s = 1.0 / sigma, norm = 1.0 / sqrt(2.0 * M_PI * sigma * sigma);
    // nodes beyond 12 sigma weigh less than exp(-72) ~ 5e-32 of the peak: skipped
    // (the exponential is evaluated in FP64, the slow pipe on this GPU)
    const double cut = 12.0 * sigma;
    for (int m = blockIdx.x; m < N_x; m += gridDim.x) {
        const double x = x0 + m * h;
        double s = 0.0;
        for (int i = threadIdx.x; i < N_q; i += blockDim.x) {
            const double u = x - Y[i];
            if (fabs(u) < cut) s += P[i] * gauss(u, inv_s, norm);
        }
        s = block_sum_d(s);
        if (threadIdx.x == 0) out[m] = s / N_q;
    }
}

__global__ void blur_eigs_kernel(const double *__restrict__ eig, int64_t n_eig, double sigma,
                                 double x0, double h, int N_x, double *out) {
    const double inv_s = 1.0 / sigma, norm = 1.0 / sqrt(2.0 * M_PI * sigma * sigma);
    for (int m = blockIdx.x; m < N_x; m += gridDim.x) {
        const double x = x0 + m * h;
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n_eig; j += blockDim.x) {
            const double u = x - eig[j];
            if (fabs(u) < 12.0 * sigma) s += gauss(u, inv_s, norm);  // beyond: < 5e-32 of the peak
        }
        s = block_sum_d(s);
        if (threadIdx.x == 0) out[m] = s / (double)n_eig;
    }
}

__global__ void error_norms_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                   int N_x, double h, double *out) {
    __shared__ double smax[32];
    double s = 0.0, mx = 0.0;
    for (int m = threadIdx.x; m < N_x; m += blockDim.x) {
        const double v = fabs(a[m] - b[m]);
        s += (m == 0 || m == N_x - 1) ? 0.5 * v : v;
        mx = fmax(mx, v);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
    s = block_sum_d(s);
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, smax[w]);
        out[0] = h * s;
        out[1] = mx;
    }
}

// mu_k = (pi/N) sum_i sqrt(1 - t_i^2) phi(t_i) T_k(t_i), t_i = -cos(pi (i+1/2)/N):
// one block per k, T_k(t_i) = cos(k theta_i) with theta_i the node angle
// pi - pi (i + 1/2)/N, fixed-order block sum.
__global__ void grid_moments_kernel(const double *__restrict__ phi, int N, int M,
                                    double *__restrict__ mu) {
    for (int k = blockIdx.x; k <= M; k += gridDim.x) {
        double s = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const double x = (i + 0.5) / (double)N;  // t_i = -cos(pi x) = cos(pi (1 - x))
            const double w = sinpi(x);               // sqrt(1 - t_i^2)
            // T_k(t_i) = cos(k pi (1 - x)); reduce k (1 - x) mod 2 exactly enough
            const double arg = fmod((double)k * (1.0 - x), 2.0);
            s += w * phi[i] * cospi(arg);
        }
        s = block_sum_d(s);
        if (threadIdx.x == 0) mu[k] = M_PI * s / N;
    }
}

// Heat-capacity kernel of Eq. gfunc up to its constant factor:
// g(lambda) = x^2 e^{-x} / (1 - e^{-x})^2 with x = beta sqrt(max(lambda, 0)); g -> 1 as x -> 0.
__device__ __forceinline__ double heat_kernel(double lambda, double beta) {
    const double x = beta * sqrt(fmax(lambda, 0.0));
    if (x < 1e-6) return 1.0 - x * x / 12.0;
    const double em = exp(-x);
    const double den = -expm1(-x);  // 1 - e^{-x}
    return x * x * em / (den * den);
}

// out[b] = sum_j w_j g(p_j; beta_b) * scale; one block per beta, fixed-order sums.
__global__ void heat_points_kernel(const double *__restrict__ pts, const double *__restrict__ w,
                                   int64_t n_pts, double scale, const double *__restrict__ betas,
                                   int n_beta, double *__restrict__ out) {
    for (int b = blockIdx.x; b < n_beta; b += gridDim.x) {
        const double beta = betas[b];
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n_pts; j += blockDim.x) s += w[j] * heat_kernel(pts[j], beta);
        s = block_sum_d(s);
        if (threadIdx.x == 0) out[b] = s * scale;
    }
}

int grid_cap(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void launch_reconstruct(const double *mu, int M, int damping, double lb, double ub,
                        const double *t, int N_t, double *coef_scratch, double *phi_hat,
                        double *phi_lambda, cudaStream_t s) {
    coef_kernel<<<grid_cap(M + 1, 256, 1024), 256, 0, s>>>(mu, M, damping, coef_scratch);
    DOS_LAUNCHED();
    reconstruct_kernel<<<grid_cap(N_t, 256, 4096), 256, 0, s>>>(
        coef_scratch, M, 0.5 * (ub - lb), t, N_t, phi_hat, phi_lambda);
    DOS_LAUNCHED();
}

void launch_reconstruct_rows(const double *mu, int64_t ldm, int B, int M, int damping,
                             const double *t, int N_t, double *coef_scratch, double *phi_hat,
                             cudaStream_t s) {
    coef_rows_kernel<<<grid_cap((int64_t)B * (M + 1), 256, 4096), 256, 0, s>>>(
        mu, ldm, B, M, damping, coef_scratch);
    DOS_LAUNCHED();
    reconstruct_rows_kernel<<<grid_cap((int64_t)B * N_t, 256, 8192), 256, 0, s>>>(
        coef_scratch, B, M, t, N_t, phi_hat);
    DOS_LAUNCHED();
}

// poly_scratch: (M+1) coefficients, N_q node values, N_q node positions.
void launch_blur_kpm(const double *mu, int M, int damping, double lb, double ub, double sigma,
                     int N_q, double x0, double h, int N_x, double *poly_scratch, double *out,
                     cudaStream_t s) {
    double *a = poly_scratch, *P = poly_scratch + (M + 1), *Y = P + N_q;
    coef_kernel<<<grid_cap(M + 1, 256, 1024), 256, 0, s>>>(mu, M, damping, a);
    DOS_LAUNCHED();
    nodes_kernel<<<grid_cap(N_q, 256, 4096), 256, 0, s>>>(a, M, N_q, 0.5 * (lb + ub),
                                                          0.5 * (ub - lb), P, Y);
    DOS_LAUNCHED();
    blur_kpm_kernel<<<N_x < 65535 ? N_x : 65535, 256, 0, s>>>(P, Y, N_q, sigma, x0, h, N_x, out);
    DOS_LAUNCHED();
}

void launch_blur_eigs(const double *eig, int64_t n_eig, double sigma, double x0, double h,
                      int N_x, double *out, cudaStream_t s) {
    blur_eigs_kernel<<<N_x < 65535 ? N_x : 65535, 256, 0, s>>>(eig, n_eig, sigma, x0, h, N_x,
                                                                out);
    DOS_LAUNCHED();
}

// KPM: P(t_i) at N_q Gauss-Chebyshev nodes (positions Y) then the quadrature
// (1/N_q) sum_i P(t_i) g(Y_i); scratch: (M+1) + 2 N_q doubles.
void launch_heat_kpm(const double *mu, int M, int damping, double lb, double ub, int N_q,
                     const double *betas, int n_beta, double *scratch, double *out,
                     cudaStream_t s) {
    double *a = scratch, *P = scratch + (M + 1), *Y = P + N_q;
    coef_kernel<<<grid_cap(M + 1, 256, 1024), 256, 0, s>>>(mu, M, damping, a);
    DOS_LAUNCHED();
    nodes_kernel<<<grid_cap(N_q, 256, 4096), 256, 0, s>>>(a, M, N_q, 0.5 * (lb + ub),
                                                          0.5 * (ub - lb), P, Y);
    DOS_LAUNCHED();
    heat_points_kernel<<<n_beta < 65535 ? n_beta : 65535, 256, 0, s>>>(Y, P, N_q, 1.0 / N_q,
                                                                      betas, n_beta, out);
    DOS_LAUNCHED();
}

void launch_heat_points(const double *pts, const double *w, int64_t n_pts, double scale,
                        const double *betas, int n_beta, double *out, cudaStream_t s) {
    heat_points_kernel<<<n_beta < 65535 ? n_beta : 65535, 256, 0, s>>>(pts, w, n_pts, scale, betas,
                                                                      n_beta, out);
    DOS_LAUNCHED();
}

void launch_grid_moments(const double *phi, int N, int M, double *mu, cudaStream_t s) {
    grid_moments_kernel<<<M + 1 < 4096 ? M + 1 : 4096, 256, 0, s>>>(phi, N, M, mu);
    DOS_LAUNCHED();
}

void launch_error_norms(const double *a, const double *b, int N_x, double h, double *out,
                        cudaStream_t s) {
    error_norms_kernel<<<1, 1024, 0, s>>>(a, b, N_x, h, out);
    DOS_LAUNCHED();
}

}  // namespace dos
