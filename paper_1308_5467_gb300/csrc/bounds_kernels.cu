// Kernels for the spectrum bounds (step a1, Section 3.1 around Eq. cd).
//
// Gershgorin: one pass over the CSR, each row gives the disc
// [a_ii - r_i, a_ii + r_i], r_i = sum_{j != i} |a_ij|; block min/max partials
// are combined by a single-block kernel.
//
// Lanczos: plain k-step Lanczos in FP64 on one vector (no reorthogonalisation,
// as in Eq. lanfact), each step as
//     w = A q_j - beta_{j-1} q_{j-1};  alpha_j = q_j . w;  w -= alpha_j q_j;
//     beta_j = ||w||;  q_{j+1} = w / beta_j.
// Dot products use fixed-order block partials plus a single-block sum, so the
// result is reproducible.  alpha/beta stay on the device until the end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dos_internal.h"

namespace dos {
namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ double load_val(const void *val, int64_t e) {
    return (double)reinterpret_cast<const T *>(val)[e];
}

__device__ __forceinline__ void block_minmax(double &lo, double &hi) {
    __shared__ double slo[32], shi[32];
    for (int off = 16; off > 0; off >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, off));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { slo[warp] = lo; shi[warp] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
    }
}

// Fixed-order block sum; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double s) {
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    __syncthreads();
    return tot;
}

template <typename T>
__global__ void gershgorin_kernel(int64_t n, const int32_t *__restrict__ row_ptr,
                                  const int32_t *__restrict__ col_idx, const void *val,
                                  double *part) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double center = 0.0, radius = 0.0;
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const double a = load_val<T>(val, e);
            if (col_idx[e] == i) center += a; else radius += fabs(a);
        }
        lo = fmin(lo, center - radius);
        hi = fmax(hi, center + radius);
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = lo;
        part[2 * blockIdx.x + 1] = hi;
    }
}

__global__ void minmax_final_kernel(const double *part, int n_blocks, double *out) {
    double lo = INFINITY, hi = -INFINITY;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        lo = fmin(lo, part[2 * b]);
        hi = fmax(hi, part[2 * b + 1]);
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        out[0] = lo;
        out[1] = hi;
    }
}

// Start vector l = 0 of matrix b = 0 (the same generator as the sweep's start
// vectors), divided by its norm sqrt(n).
__global__ void lanczos_start_kernel(int64_t n, uint64_t seed, double *q) {
    const double nrm = sqrt((double)n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + ((uint64_t)i + 1ULL) * 0x9e3779b97f4a7c15ULL;  // ctr = i
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        q[i] = ((z & 1ULL) ? -1.0 : 1.0) / nrm;
    }
}

template <typename T>
__global__ void lanczos_matvec_kernel(int64_t n, const int32_t *__restrict__ row_ptr,
                                      const int32_t *__restrict__ col_idx, const void *val,
                                      const double *__restrict__ q,
                                      const double *__restrict__ q_prev,
                                      const double *__restrict__ beta_prev, double *__restrict__ w,
                                      double *part) {
    const double bp = beta_prev ? *beta_prev : 0.0;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double y = 0.0;
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) y += load_val<T>(val, e) * q[col_idx[e]];
        y -= bp * q_prev[i];
        w[i] = y;
        s += q[i] * y;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_final_kernel(const double *part, int n_blocks, double *out, int take_sqrt) {
    double s = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) s += part[b];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : s;
}

__global__ void lanczos_axpy_kernel(int64_t n, const double *__restrict__ alpha,
                                    const double *__restrict__ q, double *__restrict__ w,
                                    double *part) {
    const double a = *alpha;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = w[i] - a * q[i];
        w[i] = v;
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void lanczos_next_kernel(int64_t n, const double *__restrict__ beta,
                                    double *__restrict__ q, double *__restrict__ q_prev,
                                    const double *__restrict__ w) {
    const double b = *beta;
    if (!(b > 0.0)) return;  // invariant subspace: the host stops here
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        q_prev[i] = q[i];
        q[i] = w[i] / b;
    }
}

// Order-preserving map of a double to an unsigned 64-bit key (negative numbers
// have all bits flipped, non-negative ones the sign bit set), so integer
// atomicMin/atomicMax give the exact floating-point min/max in any order.
__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

template <typename T>
__global__ void gershgorin_batched_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                                          const int32_t *__restrict__ col_idx, const void *val,
                                          int B, const int32_t *__restrict__ seg_row0,
                                          unsigned long long *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = B;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg_row0[mid] <= i) lo = mid; else hi = mid;
        }
        const int64_t local = i - seg_row0[lo];
        double center = 0.0, radius = 0.0;
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const double a = load_val<T>(val, e);
            if (col_idx[e] == local) center += a; else radius += fabs(a);
        }
        atomicMin(keys + 2 * lo, order_key(center - radius));
        atomicMax(keys + 2 * lo + 1, order_key(center + radius));
    }
}

__global__ void keys_to_double_kernel(const unsigned long long *keys, int count, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
        out[i] = __longlong_as_double((long long)b);
    }
}

__global__ void keys_init_kernel(unsigned long long *keys, int B) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        keys[2 * i] = ~0ULL;     // min accumulator
        keys[2 * i + 1] = 0ULL;  // max accumulator
    }
}

}  // namespace

void launch_gershgorin_batched(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                               const void *val, int dtype, int B, const int32_t *seg_row0,
                               unsigned long long *keys, double *out, int num_sms,
                               cudaStream_t s) {
    keys_init_kernel<<<(B + 255) / 256, 256, 0, s>>>(keys, B);
    DOS_LAUNCHED();
    const int grid = reduce_blocks(num_sms, n_rows);
    if (dtype == DOS_F64)
        gershgorin_batched_kernel<double><<<grid, kThreads, 0, s>>>(n_rows, row_ptr, col_idx, val,
                                                                    B, seg_row0, keys);
    else
        gershgorin_batched_kernel<float><<<grid, kThreads, 0, s>>>(n_rows, row_ptr, col_idx, val,
                                                                   B, seg_row0, keys);
    DOS_LAUNCHED();
    keys_to_double_kernel<<<(2 * B + 255) / 256, 256, 0, s>>>(keys, 2 * B, out);
    DOS_LAUNCHED();
}

int gershgorin_blocks(int num_sms) { return num_sms * 4; }
int reduce_blocks(int num_sms, int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > num_sms * 4) b = num_sms * 4;
    return b < 1 ? 1 : (int)b;
}

void launch_gershgorin(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const void *val, int dtype, double *part, int n_blocks, cudaStream_t s) {
    if (dtype == DOS_F64)
        gershgorin_kernel<double><<<n_blocks, kThreads, 0, s>>>(n, row_ptr, col_idx, val, part);
    else
        gershgorin_kernel<float><<<n_blocks, kThreads, 0, s>>>(n, row_ptr, col_idx, val, part);
    DOS_LAUNCHED();
}

void launch_minmax_final(const double *part, int n_blocks, double *out, cudaStream_t s) {
    minmax_final_kernel<<<1, kThreads, 0, s>>>(part, n_blocks, out);
    DOS_LAUNCHED();
}

void launch_lanczos_start(int64_t n, uint64_t seed, double *q, cudaStream_t s) {
    lanczos_start_kernel<<<reduce_blocks(152, n), kThreads, 0, s>>>(n, seed, q);
    DOS_LAUNCHED();
}

void launch_lanczos_matvec(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                           const void *val, int dtype, const double *q, const double *q_prev,
                           const double *beta_prev, double *w, double *part, int n_blocks,
                           cudaStream_t s) {
    if (dtype == DOS_F64)
        lanczos_matvec_kernel<double><<<n_blocks, kThreads, 0, s>>>(n, row_ptr, col_idx, val, q,
                                                                    q_prev, beta_prev, w, part);
    else
        lanczos_matvec_kernel<float><<<n_blocks, kThreads, 0, s>>>(n, row_ptr, col_idx, val, q,
                                                                   q_prev, beta_prev, w, part);
    DOS_LAUNCHED();
}

void launch_sum_final(const double *part, int n_blocks, double *out, int take_sqrt,
                      cudaStream_t s) {
    sum_final_kernel<<<1, kThreads, 0, s>>>(part, n_blocks, out, take_sqrt);
    DOS_LAUNCHED();
}

void launch_lanczos_axpy(int64_t n, const double *alpha, const double *q, double *w,
                         double *part, int n_blocks, cudaStream_t s) {
    lanczos_axpy_kernel<<<n_blocks, kThreads, 0, s>>>(n, alpha, q, w, part);
    DOS_LAUNCHED();
}

void launch_lanczos_next(int64_t n, const double *beta, double *q, double *q_prev,
                         const double *w, cudaStream_t s) {
    lanczos_next_kernel<<<reduce_blocks(152, n), kThreads, 0, s>>>(n, beta, q, q_prev, w);
    DOS_LAUNCHED();
}

}  // namespace dos
