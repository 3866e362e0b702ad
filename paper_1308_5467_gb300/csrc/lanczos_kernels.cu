// Lanczos DOS (Section 3.2.1, Eq. landos): n_v independent M-step Lanczos runs
// advanced together as a block, Ritz values and Gauss weights per run, and the
// Gaussian-blurred DOS from them.  FP64 throughout.
//
// Block layout as in the moment sweep: Q[i*ld + l].  The Lanczos vectors are kept
// unnormalised, q_j = s_j u_j with one factor per column, so that no pass has to
// rescale a block.  With w_j = A q_j - beta_{j-1} q_{j-1} and W = w_j / s_j, step j:
//   W = A u_j - c_j u_{j-1}                 (SpMM pass, lanczos_team_spmm_kernel in
//                                            kpm_kernels.cu; W overwrites u_{j-1})
//   alpha_j = q_j . w_j = s_j^2 u_j . W      (per-vector partials, fixed-order reduce)
//   u_{j+1} = t_j (W - alpha_j u_j)          (vector pass, partial ||u_{j+1}||^2)
//   beta_j = ||w_j - alpha_j q_j|| = s_j ||u_{j+1}|| / t_j
// with t_j = 1 / beta_{j-1}, s_{j+1} = s_j / (t_j beta_j), c_{j+1} = beta_j s_j / s_{j+1}
// (s_0 = t_0 = 1).  t_j keeps |u_j| of the order of beta_j / beta_0, and every
// per-element pass does the work it did with normalised vectors.
// A run whose beta_j falls to 1e-12 times its running norm estimate has reached
// an invariant subspace; the host keeps its first j+1 coefficients only.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dos_internal.h"

namespace dos {
namespace {

constexpr int kThreads = 256;

// w <- t (w - alpha u) per column, partial ||w||^2 per column (t NULL: 1)
__global__ void lanczos_axpy_kernel(int64_t n, int ld, const double *__restrict__ alpha,
                                    const double *__restrict__ t_fac,
                                    const double *__restrict__ q, double *__restrict__ w,
                                    double *__restrict__ part, int n_vec) {
    extern __shared__ double sh[];
    const int cols = ld;
    const int rows_per_block = blockDim.x / cols;
    const int rloc = threadIdx.x / cols, l = threadIdx.x % cols;
    const double a = alpha[l];
    const double t = t_fac ? t_fac[l] : 1.0;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * rows_per_block + rloc; i < n;
         i += (int64_t)gridDim.x * rows_per_block) {
        const size_t o = (size_t)i * ld + l;
        const double v = (w[o] - a * q[o]) * t;
        w[o] = v;
        if (l < n_vec) acc = fma(v, v, acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < cols) {
        double s = 0.0;
        for (int r = 0; r < rows_per_block; ++r) s += sh[r * cols + threadIdx.x];
        part[(size_t)blockIdx.x * cols + threadIdx.x] = s;
    }
}

// Sum over blocks of part[b][l] for column l = blockIdx.x: each thread sums a
// strided slice in order, then a fixed shuffle tree and a fixed warp order, so
// the result is reproducible.  Thread 0 returns the total.
__device__ double column_total(const double *__restrict__ part, int n_blocks, int ld, int l) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) s += part[(size_t)b * ld + l];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

// alpha_j = s_j^2 (u_j . w) per column (s NULL: 1).  One block per column.
__global__ void lanczos_alpha_kernel(const double *__restrict__ part, int n_blocks, int ld,
                                     const double *__restrict__ s_fac,
                                     double *__restrict__ alpha) {
    const int l = blockIdx.x;
    const double t = column_total(part, n_blocks, ld, l);
    if (threadIdx.x == 0) {
        const double sj = s_fac ? s_fac[l] : 1.0;
        alpha[l] = t * sj * sj;
    }
}

// From v^2 = ||u_{j+1}||^2 (partials) per column, with s = s_j and bp = beta_{j-1}
// (both NULL at j = 0: 1):  beta_j = s bp v, and the factors of the next step,
// s_{j+1} = s bp / beta_j, c_{j+1} = beta_j^2 / bp (the SpMM's coefficient of u_j)
// and t_{j+1} = 1 / beta_j (the axpy's rescale).  A zero beta_j leaves the run's
// later vectors at zero.  One block per column; s may be s_next (in place).
__global__ void lanczos_beta_kernel(const double *__restrict__ part, int n_blocks, int ld,
                                    const double *s_fac, const double *__restrict__ beta_prev,
                                    double *__restrict__ beta, double *s_next,
                                    double *__restrict__ c_next, double *__restrict__ t_next) {
    const int l = blockIdx.x;
    const double t = column_total(part, n_blocks, ld, l);
    if (threadIdx.x == 0) {
        const double sj = s_fac ? s_fac[l] : 1.0;
        const double bp = beta_prev ? beta_prev[l] : 1.0;
        const double b = sj * bp * sqrt(t);
        beta[l] = b;
        const double ib = b > 0.0 ? 1.0 / b : 0.0;
        s_next[l] = sj * bp * ib;
        c_next[l] = bp > 0.0 ? b * b / bp : 0.0;
        t_next[l] = ib;
    }
}

// start block: Rademacher vector columns divided by sqrt(n)
__global__ void unit_scale_kernel(int64_t n, int ld, int n_vec, double *__restrict__ q) {
    const double inv = 1.0 / sqrt((double)n);
    const int64_t total = n * ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        q[t] = (t % ld) < n_vec ? q[t] * inv : 0.0;
}

// Used for the Lanczos bounds (one thread; work arrays in global scratch).
// Implicit QL with Wilkinson-style shifts (the classical tql1/tql2 iteration) on
// the symmetric tridiagonal (dd: diagonal, ee: off-diagonal, ee[m-1] = 0),
// applying every plane rotation to one row zz of the eigenvector matrix (start
// from e_1 for first components, from e_m for last components).  On return
// dd holds the eigenvalues (unsorted) and zz that row's entries.
__device__ void ql_one_row(int m, double *__restrict__ dd, double *__restrict__ ee,
                           double *__restrict__ zz) {
    for (int lo = 0; lo < m; ++lo) {
        for (int iter = 0; iter < 60; ++iter) {
            int mm = lo;
            for (; mm < m - 1; ++mm) {
                const double dsum = fabs(dd[mm]) + fabs(dd[mm + 1]);
                if (fabs(ee[mm]) <= 2.2e-16 * dsum) break;
            }
            if (mm == lo) break;
            double g = (dd[lo + 1] - dd[lo]) / (2.0 * ee[lo]);
            double r = hypot(g, 1.0);
            g = dd[mm] - dd[lo] + ee[lo] / (g + (g >= 0.0 ? fabs(r) : -fabs(r)));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = mm - 1;
            bool underflow = false;
            // The sweep reads d[i], z[i], e[i] and rewrites d[i+1], z[i+1], e[i+1]; d[i]
            // is next step's d[i+1] unchanged and z[i] is passed on rotated, so both are
            // carried in registers and the loads stay off the dependent FP64 chain.
            double d_next = dd[mm], z_next = zz[mm];  // d[i+1], z[i+1] of step i
            for (; i >= lo; --i) {
                const double e_i = ee[i], d_i = dd[i], z_i = zz[i];
                const double f = s * e_i, b = c * e_i;
                // r = hypot(f, g), s = f / r, c = g / r through one reciprocal square
                // root (FP64 division and hypot are long dependent sequences here);
                // |f|, |g| are of the order of the entries of T, far from overflow.
                const double h2 = fma(f, f, g * g);
                if (h2 == 0.0) {
                    ee[i + 1] = 0.0;
                    dd[i + 1] = d_next - p;
                    zz[i + 1] = z_next;
                    ee[mm] = 0.0;
                    underflow = true;
                    break;
                }
                const double ir = rsqrt(h2);
                r = h2 * ir;
                ee[i + 1] = r;
                s = f * ir;
                c = g * ir;
                g = d_next - p;
                r = (d_i - g) * s + 2.0 * c * b;
                p = s * r;
                dd[i + 1] = g + p;
                g = c * r - b;
                zz[i + 1] = s * z_i + c * z_next;
                z_next = c * z_i - s * z_next;
                d_next = d_i;
            }
            if (underflow) continue;
            zz[lo] = z_next;
            dd[lo] -= p;
            ee[lo] = g;
            ee[mm] = 0.0;
        }
    }
}

// ---- Ritz pairs of the n_v Lanczos tridiagonals (Golub–Welsch quadrature) --------
// Nodes: the eigenvalues of each run's T (diagonal alpha_0..alpha_{m-1}, off-diagonal
// beta_0..beta_{m-2}), by bisection on Sturm counts, one thread per eigenvalue.
// Weights: the Gauss weight of node lambda_j is the residue of
// r(z) = e_1^T (zI - T)^{-1} e_1 at lambda_j, i.e. the square of the first component
// of its unit eigenvector.  It is taken as the contour integral
// (1/2 pi i) \oint r(z) dz over a circle around lambda_j, by the trapezoid rule on
// K = 64 points (one lane per conjugate pair), with r(z) the Stieltjes continued
// fraction 1 / (z - alpha_0 - beta_0^2 / (z - alpha_1 - ...)) evaluated from the
// bottom up.  Off the real axis every partial denominator has |Im t_i| >= |Im z|,
// so the evaluation is stable and bounded.  Eigenvalues closer than 1e-8 of the
// spectral scale (the copies that loss of orthogonality produces), or closer than
// twice the width of a neighbouring group, are merged into one group: its total
// weight, at its weight centroid (from the second integral \oint (z - c) r(z) dz),
// goes to the member just below the centroid, the others get weight 0.  The total and the centroid are
// well-conditioned where the split is not, and they keep the blurred DOS and the
// quadrature's moments to second order in the group's width.  Each circle's radius is half the
// distance from the group's centre to the nearest other node, so every other pole
// is at least twice the radius away and every member within 0.4 of it: the
// trapezoid error is below 2^-60 of a neighbouring weight.
// Both kernels first scale T by a power of two so its Gershgorin bound is in
// [1, 2) (exact; the results are scaled back), which keeps the Sturm recurrence
// and the continued fraction far from overflow.
constexpr int kRitzPoints = 64;  // K, trapezoid points on each circle (32 lanes x 2)

// Loads run l's tridiagonal into shared memory, scaled: a[i] = f alpha_i,
// b2[i] = (f beta_i)^2; returns f and the scaled Gershgorin interval.
__device__ void load_scaled_tridiagonal(const double *__restrict__ alpha,
                                        const double *__restrict__ beta, int l, int m, int ld,
                                        double *a, double *b2, double *sc /* f, lo, hi */) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[i] = alpha[(size_t)i * ld + l];
        b2[i] = i + 1 < m ? beta[(size_t)i * ld + l] : 0.0;  // raw beta for now
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < m; ++i) {
            const double r = (i > 0 ? fabs(b2[i - 1]) : 0.0) + fabs(b2[i]);
            lo = fmin(lo, a[i] - r);
            hi = fmax(hi, a[i] + r);
        }
        const double scale = fmax(fabs(lo), fabs(hi));
        double f = 1.0;
        if (scale >= 2.2250738585072014e-308 && scale < INFINITY) {
            int e;
            frexp(scale, &e);    // scale = q 2^e, q in [0.5, 1)
            f = ldexp(1.0, 1 - e);  // f scale in [1, 2)
        }
        sc[0] = f;
        sc[1] = lo * f;
        sc[2] = hi * f;
    }
    __syncthreads();
    const double f = sc[0];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        a[i] *= f;
        const double bb = b2[i] * f;
        b2[i] = bb * bb;
    }
    __syncthreads();
}

// Number of eigenvalues of T below x: m minus the sign changes of the leading
// principal minors D_i = det(x I - T_i) (D_0 = 1, D_1 = x - a_0,
// D_i = (x - a_{i-1}) D_{i-1} - b2_{i-2} D_{i-2}).  A zero minor counts as positive;
// for an unreduced T an interior zero is flanked by opposite signs, so either
// choice gives the same count.  The last two minors are rescaled together by an
// exact power of two (the larger into [1, 2)) whenever the larger leaves
// [2^-400, 2^400]; the exponents are read as integers, off the FP64 chain.
__device__ int sturm_below(const double *a, const double *b2, int m, double x) {
    double p0 = 1.0, p1 = x - a[0];
    int changes = p1 < 0.0 ? 1 : 0;
    for (int i = 1; i < m; ++i) {
        const double p2 = fma(x - a[i], p1, -b2[i - 1] * p0);
        changes += (p2 < 0.0) != (p1 < 0.0) ? 1 : 0;
        p0 = p1;
        p1 = p2;
        const int e = max((int)((__double_as_longlong(p0) >> 52) & 0x7ff),
                          (int)((__double_as_longlong(p1) >> 52) & 0x7ff));
        if (e > 1023 + 400 || (e < 1023 - 400 && e != 0)) {
            const double s = __longlong_as_double((long long)(2046 - e) << 52);  // 2^(1023-e)
            p0 *= s;
            p1 *= s;
        }
    }
    return m - changes;
}

__global__ void ritz_bisect_kernel(const double *__restrict__ alpha,
                                   const double *__restrict__ beta,
                                   const int *__restrict__ m_used, int M, int ld, int n_vec,
                                   double *__restrict__ theta) {
    extern __shared__ double rz_sm[];
    __shared__ double sc[3];
    const int l = blockIdx.x;
    if (l >= n_vec) return;
    const int m = m_used[l];
    double *th = theta + (size_t)l * M;
    for (int j = max(m, 0) + threadIdx.x; j < M; j += blockDim.x) th[j] = 0.0;
    if (m <= 0) return;
    double *a = rz_sm, *b2 = rz_sm + M;
    load_scaled_tridiagonal(alpha, beta, l, m, ld, a, b2, sc);
    const double f = sc[0];
    const double scale = fmax(fabs(sc[1]), fabs(sc[2]));
    const double eps = 2.220446049250313e-16;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double lo = sc[1] - 2.0 * eps * scale, hi = sc[2] + 2.0 * eps * scale;
        for (int it = 0; it < 128; ++it) {
            if (hi - lo <= fmax(4.0 * eps * fmax(fabs(lo), fabs(hi)), eps * scale)) break;
            const double mid = 0.5 * (lo + hi);
            if (sturm_below(a, b2, m, mid) > j) hi = mid;
            else lo = mid;
        }
        th[j] = 0.5 * (lo + hi) / f;
    }
}

__global__ void ritz_weight_kernel(const double *__restrict__ alpha,
                                   const double *__restrict__ beta,
                                   const int *__restrict__ m_used, int M, int ld, int n_vec,
                                   double *__restrict__ theta, double *__restrict__ weight) {
    extern __shared__ double rz_sm[];
    __shared__ double sc[3];
    __shared__ int n_groups;
    const int l = blockIdx.x;
    if (l >= n_vec) return;
    const int m = m_used[l];
    double *wt = weight + (size_t)l * M;
    for (int j = max(m, 0) + threadIdx.x; j < M; j += blockDim.x) wt[j] = 0.0;
    if (m <= 0) return;
    double *a = rz_sm, *b2 = rz_sm + M, *lam = rz_sm + 2 * (size_t)M;
    int *gs = reinterpret_cast<int *>(rz_sm + 3 * (size_t)M), *ge = gs + M;
    load_scaled_tridiagonal(alpha, beta, l, m, ld, a, b2, sc);
    const double f = sc[0];
    const double scale = fmax(fabs(sc[1]), fabs(sc[2]));
    for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = theta[(size_t)l * M + i] * f;
    __syncthreads();
    if (threadIdx.x == 0) {
        // groups of the (ascending) nodes, merged left to right on a stack until every
        // gap is at least 1e-8 scale and twice the wider of its two groups
        int top = 0;
        for (int j = 0; j < m; ++j) {
            int s = j, e = j;
            while (top > 0) {
                const int ps = gs[top - 1], pe = ge[top - 1];
                const double gap = lam[s] - lam[pe];
                const double wd = fmax(lam[pe] - lam[ps], lam[e] - lam[s]);
                if (gap < 1e-8 * scale || gap < 2.0 * wd) {
                    s = ps;
                    --top;
                } else {
                    break;
                }
            }
            gs[top] = s;
            ge[top] = e;
            ++top;
        }
        n_groups = top;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    double sn, cs;
    sincospi((2.0 * lane + 1.0) / kRitzPoints, &sn, &cs);  // this lane's point (upper half)
    const int ng = n_groups;
    for (int g = warp; g < ng; g += n_warps) {
        const int s = gs[g], e = ge[g];
        const double c = 0.5 * (lam[s] + lam[e]), width = lam[e] - lam[s];
        double D = INFINITY;
        if (g > 0) D = fmin(D, c - lam[ge[g - 1]]);
        if (g + 1 < ng) D = fmin(D, lam[gs[g + 1]] - c);
        const double rho = D < INFINITY ? 0.5 * D : fmax(fmax(2.0 * width, scale), 1.0);
        const double zr = c + rho * cs, zi = rho * sn;
        double tr = zr - a[m - 1], ti = zi;
        for (int i = m - 2; i >= 0; --i) {
            const double q = b2[i] / fma(tr, tr, ti * ti);
            tr = zr - a[i] - q * tr;
            ti = zi + q * ti;
        }
        // r = 1 / t; with zeta = z - c = rho e^{i th}, this point and its conjugate
        // contribute 2 Re(r zeta) / K to the weight and 2 Re(r zeta^2) / K to the
        // first moment about c
        const double inv = 1.0 / fma(tr, tr, ti * ti);
        double v = rho * inv * fma(tr, cs, ti * sn);
        double v1 = rho * rho * inv * fma(tr, fma(cs, cs, -sn * sn), ti * (2.0 * sn * cs));
        for (int off = 16; off > 0; off >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, off);
            v1 += __shfl_down_sync(0xffffffffu, v1, off);
        }
        // lane 0 holds the sums; the group's node goes to the member just below its
        // centroid, which keeps the Ritz values ascending
        const double W = __shfl_sync(0xffffffffu, v, 0) * (2.0 / kRitzPoints);
        const double M1 = __shfl_sync(0xffffffffu, v1, 0) * (2.0 / kRitzPoints);
        int k = s;
        double cc = lam[s];
        if (e > s && W > 0.0) {
            cc = fmin(fmax(c + M1 / W, lam[s]), lam[e]);
            while (k < e && lam[k + 1] <= cc) ++k;
        }
        for (int q = s + lane; q <= e; q += 32) wt[q] = q == k ? W : 0.0;
        if (lane == 0 && e > s) theta[(size_t)l * M + k] = cc / f;
    }
}

// phi(x_i) = (1/n_vec) sum_{l,k} weight[l,k] g_sigma(x_i - theta[l,k]); one block per point.
__global__ void weighted_gauss_kernel(const double *__restrict__ pts, const double *__restrict__ w,
                                      int64_t n_pts, double scale, double sigma,
                                      const double *__restrict__ x, double x0, double h, int N_x,
                                      double *__restrict__ out) {
    __shared__ double sh[32];
    const double inv_s = 1.0 / sigma, norm = 1.0 / sqrt(2.0 * M_PI * sigma * sigma);
    for (int m = blockIdx.x; m < N_x; m += gridDim.x) {
        const double xm = x ? x[m] : x0 + m * h;
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n_pts; j += blockDim.x) {
            const double z = (xm - pts[j]) * inv_s;
            if (fabs(z) < 12.0) s += w[j] * norm * exp(-0.5 * z * z);  // beyond: < 5e-32 of the peak
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
            out[m] = t * scale;
        }
        __syncthreads();
    }
}

// Haydock (Section 3.2.2): phi(x) = scale * sum w (eta/pi) / ((x - theta)^2 + eta^2),
// the imaginary part of the M-step continued fraction e_1^T (z - T)^{-1} e_1 at
// z = x + i eta written through the Ritz pairs.
__global__ void weighted_lorentz_kernel(const double *__restrict__ pts,
                                        const double *__restrict__ w, int64_t n_pts, double scale,
                                        double eta, const double *__restrict__ x, int N_x,
                                        double *__restrict__ out) {
    __shared__ double sh[32];
    const double c = eta / M_PI, e2 = eta * eta;
    for (int m = blockIdx.x; m < N_x; m += gridDim.x) {
        const double xm = x[m];
        double s = 0.0;
        for (int64_t j = threadIdx.x; j < n_pts; j += blockDim.x) {
            const double u = xm - pts[j];
            s += w[j] * c / (u * u + e2);
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
            out[m] = t * scale;
        }
        __syncthreads();
    }
}

int block_threads_for(int ld) { return (kThreads / ld) * ld; }  // ld <= 256

// Lanczos bounds (Section 3.1.1): the run stops at an invariant subspace
// (beta_j <= 1e-12 times the running estimate max(|alpha_i| + beta_i + beta_{i-1})
// of ||A||); the extreme Ritz values theta of the k-step tridiagonal widened by
// ||f|| |y_last| (f the residual, y the unit Ritz vector).  One thread.
// out: lo, hi, and the number of steps kept.
__global__ void lanczos_bounds_kernel(const double *__restrict__ alpha,
                                      const double *__restrict__ beta, int k,
                                      double *__restrict__ work, double *__restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int kk = k;
    double scale = 0.0;
    bool finite = true;
    for (int j = 0; j < k; ++j) {
        finite = finite && isfinite(alpha[j]) && isfinite(beta[j]);
        scale = fmax(scale, fabs(alpha[j]) + beta[j] + (j ? beta[j - 1] : 0.0));
        if (!(beta[j] > 1e-12 * scale)) {
            kk = j + 1;
            break;
        }
    }
    if (!finite) {
        out[0] = out[1] = NAN;
        out[2] = kk;
        return;
    }
    double *dd = work, *ee = work + kk, *zz = work + 2 * kk;
    for (int i = 0; i < kk; ++i) {
        dd[i] = alpha[i];
        ee[i] = i + 1 < kk ? beta[i] : 0.0;
        zz[i] = i == kk - 1 ? 1.0 : 0.0;
    }
    ql_one_row(kk, dd, ee, zz);
    int jmin = 0, jmax = 0;
    for (int i = 1; i < kk; ++i) {
        if (dd[i] < dd[jmin]) jmin = i;
        if (dd[i] > dd[jmax]) jmax = i;
    }
    const double f = beta[kk - 1];
    out[0] = dd[jmin] - f * fabs(zz[jmin]);
    out[1] = dd[jmax] + f * fabs(zz[jmax]);
    out[2] = kk;
}

// w <- w / sum(w) in place (one block: fixed-order partial sums, a fixed shuffle
// tree, then the division); sum_out[0] = the sum, for the caller's check.
__global__ void normalize_weights_kernel(double *__restrict__ w, int64_t n,
                                         double *__restrict__ sum_out) {
    __shared__ double sh[32];
    __shared__ double total;
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s += w[j];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
        total = t;
        sum_out[0] = t;
    }
    __syncthreads();
    const double t = total;
    if (t > 0.0 && isfinite(t))
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) w[j] /= t;
}

// Steps each Lanczos run keeps: a run ends at an invariant subspace, beta_j <= 1e-12
// times the running estimate max(|alpha_i| + beta_i + beta_{i-1}) of ||A|| (the
// paper is silent on breakdown); -1 marks a run with a non-finite coefficient.
__global__ void lanczos_steps_kernel(const double *__restrict__ alpha,
                                     const double *__restrict__ beta, int M, int ld, int n_vec,
                                     int *__restrict__ m_used) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_vec) return;
    double scale = 0.0;
    int m = M;
    for (int j = 0; j < M; ++j) {
        const double al = alpha[(size_t)j * ld + l], be = beta[(size_t)j * ld + l];
        const double bp = j ? beta[(size_t)(j - 1) * ld + l] : 0.0;
        if (!isfinite(al) || !isfinite(be)) {
            m = -1;
            break;
        }
        scale = fmax(scale, fabs(al) + be + bp);
        if (!(be > 1e-12 * scale)) {
            m = j + 1;
            break;
        }
    }
    m_used[l] = m;
}

}  // namespace

int lanczos_blocks(int num_sms, int64_t n, int ld) {
    const int bt = block_threads_for(ld);
    const int rows = bt / ld;
    int64_t b = (n + rows - 1) / rows;
    const int64_t cap = (int64_t)num_sms * 8;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

void launch_lanczos_block_axpy(int64_t n, int ld, int n_vec, const double *alpha,
                               const double *t_fac, const double *q, double *w, double *part,
                               int n_blocks, cudaStream_t s) {
    const int bt = block_threads_for(ld);
    lanczos_axpy_kernel<<<n_blocks, bt, bt * sizeof(double), s>>>(n, ld, alpha, t_fac, q, w,
                                                                   part, n_vec);
    DOS_LAUNCHED();
}

void launch_lanczos_alpha(const double *part, int n_blocks, int ld, const double *s_fac,
                          double *alpha, cudaStream_t s) {
    lanczos_alpha_kernel<<<ld, 256, 0, s>>>(part, n_blocks, ld, s_fac, alpha);
    DOS_LAUNCHED();
}

void launch_lanczos_beta(const double *part, int n_blocks, int ld, const double *s_fac,
                         const double *beta_prev, double *beta, double *s_next, double *c_next,
                         double *t_next, cudaStream_t s) {
    lanczos_beta_kernel<<<ld, 256, 0, s>>>(part, n_blocks, ld, s_fac, beta_prev, beta, s_next,
                                           c_next, t_next);
    DOS_LAUNCHED();
}

void launch_unit_scale(int64_t n, int ld, int n_vec, double *q, int num_sms, cudaStream_t s) {
    int64_t g = (n * ld + kThreads - 1) / kThreads;
    if (g > (int64_t)num_sms * 16) g = (int64_t)num_sms * 16;
    unit_scale_kernel<<<(int)std::max<int64_t>(g, 1), kThreads, 0, s>>>(n, ld, n_vec, q);
    DOS_LAUNCHED();
}

void launch_tridiag_ritz(const double *alpha, const double *beta, const int *m_used, int M, int ld,
                         int n_vec, double *theta, double *weight, cudaStream_t s) {
    // M <= 4096: bisection 64 KB, weights 96 KB + 32 KB of shared memory at most
    const size_t sm_b = 2 * (size_t)M * sizeof(double);
    const size_t sm_w = 3 * (size_t)M * sizeof(double) + 2 * (size_t)M * sizeof(int);
    if (sm_b > 48 * 1024)
        DOS_CUDA_TRY(cudaFuncSetAttribute((const void *)ritz_bisect_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_b));
    if (sm_w > 48 * 1024)
        DOS_CUDA_TRY(cudaFuncSetAttribute((const void *)ritz_weight_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_w));
    const int tb = M < 1024 ? (M + 31) / 32 * 32 : 1024;
    ritz_bisect_kernel<<<n_vec, tb, sm_b, s>>>(alpha, beta, m_used, M, ld, n_vec, theta);
    DOS_LAUNCHED();
    ritz_weight_kernel<<<n_vec, 512, sm_w, s>>>(alpha, beta, m_used, M, ld, n_vec, theta, weight);
    DOS_LAUNCHED();
}

void launch_weighted_lorentz(const double *pts, const double *w, int64_t n_pts, double scale,
                             double eta, const double *x, int N_x, double *out, cudaStream_t s) {
    weighted_lorentz_kernel<<<N_x < 65535 ? N_x : 65535, 256, 0, s>>>(pts, w, n_pts, scale, eta, x,
                                                                      N_x, out);
    DOS_LAUNCHED();
}

void launch_weighted_gauss(const double *pts, const double *w, int64_t n_pts, double scale,
                           double sigma, const double *x, double x0, double h, int N_x,
                           double *out, cudaStream_t s) {
    weighted_gauss_kernel<<<N_x < 65535 ? N_x : 65535, 256, 0, s>>>(pts, w, n_pts, scale, sigma, x,
                                                                    x0, h, N_x, out);
    DOS_LAUNCHED();
}

void launch_lanczos_bounds(const double *alpha, const double *beta, int k, double *work,
                           double *out, cudaStream_t s) {
    lanczos_bounds_kernel<<<1, 32, 0, s>>>(alpha, beta, k, work, out);
    DOS_LAUNCHED();
}

void launch_normalize_weights(double *w, int64_t n, double *sum_out, cudaStream_t s) {
    normalize_weights_kernel<<<1, 1024, 0, s>>>(w, n, sum_out);
    DOS_LAUNCHED();
}

void launch_lanczos_steps(const double *alpha, const double *beta, int M, int ld, int n_vec,
                          int *m_used, cudaStream_t s) {
    lanczos_steps_kernel<<<(n_vec + 63) / 64, 64, 0, s>>>(alpha, beta, M, ld, n_vec, m_used);
    DOS_LAUNCHED();
}

}  // namespace dos
