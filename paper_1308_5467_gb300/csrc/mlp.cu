// The learned part (not in the paper): a 3-layer perceptron from low-order
// Chebyshev moments to a DOS on a grid, trained and run entirely by these
// kernels.  Matrix products use the tensor cores through warp-level
// mma.sync m16n8k16 (bfloat16 operands, FP32 accumulation) with fused
// epilogues (bias + ReLU, ReLU-mask back-propagation); the loss, bias
// gradients and Adam run in FP32.  All reductions have a fixed order, so a
// training run is bitwise reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/dos_mlp.h"
#include "dos_internal.h"

using namespace dos;
typedef __nv_bfloat16 bf16;

struct dos_mlp {
    dos_ctx *ctx = nullptr;
    int n_in = 0, nh = 0, n_out = 0;
    int64_t n_params = 0;
    int64_t off[6] = {0};  // W1, b1, W2, b2, W3, b3 inside the flat arrays
    int64_t wsz[3] = {0};  // element counts of W1, W2, W3
    Buffer state;          // params | grads | adam m | adam v (FP32), bf16 weight copies
    Buffer acts;           // per-batch activations
    Buffer in_stage;       // dos_mlp_infer: a host input slice copied to the device
    int cap_B = 0;
    int64_t step = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb = nullptr;    // W1 | W2 | W3 in bfloat16
    // batch buffers (cap_B rows)
    float *xf = nullptr, *tf = nullptr, *y = nullptr, *dyf = nullptr, *dh2f = nullptr,
          *dh1f = nullptr, *loss_part = nullptr;
    bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dyb = nullptr, *dh2b = nullptr,
         *dh1b = nullptr;
};

namespace {

constexpr int kLossBlocks = 64;

// ---- initialisation ------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// He-uniform weights: U(-sqrt(6/fan_in), sqrt(6/fan_in)); biases zero.
__global__ void init_params_kernel(float *p, int64_t n, int64_t o0, int64_t s0, int fan0,
                                   int64_t o1, int64_t s1, int fan1, int64_t o2, int64_t s2,
                                   int fan2, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int fan = 0;
        if (i >= o0 && i < o0 + s0) fan = fan0;
        else if (i >= o1 && i < o1 + s1) fan = fan1;
        else if (i >= o2 && i < o2 + s2) fan = fan2;
        if (fan == 0) {
            p[i] = 0.f;
        } else {
            const uint64_t z = mix64(seed + ((uint64_t)i + 1) * 0x9e3779b97f4a7c15ULL);
            const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0,1)
            p[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / fan));
        }
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ in, bf16 *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// ---- tensor-core GEMM -------------------------------------------------------------
// C(m, n) = sum_k A(m, k) * B(n, k), with A(m, k) = TA ? A[k*lda + m] : A[m*lda + k] and
// B(n, k) = TB ? B[k*ldb + n] : B[n*ldb + k].  64x64 block tile, 32-deep k
// slices staged in shared memory, 4 warps of 32x32, each as 2x4 m16n8k16 MMAs.
enum Epi { EPI_BIAS_RELU_BF16 = 0, EPI_BIAS_F32 = 1, EPI_MASK = 2, EPI_F32 = 3 };

__device__ __forceinline__ uint32_t ld_pair(const bf16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, const bf16 *__restrict__ A,
                                                   int lda, const bf16 *__restrict__ B, int ldb,
                                                   const float *__restrict__ bias,
                                                   const bf16 *__restrict__ mask, int ldm,
                                                   float *__restrict__ Cf, bf16 *__restrict__ Cb,
                                                   int ldc) {
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];
    const int bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    const bf16 zero = __float2bfloat16_rn(0.f);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int idx = tid; idx < 64 * 32; idx += 128) {
            int r, k;
            if (TA) { r = idx & 63; k = idx >> 6; } else { k = idx & 31; r = idx >> 5; }
            const int gm = bm + r, gk = k0 + k;
            bf16 val = zero;
            if (gm < M && gk < K) val = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[r][k] = val;
        }
        for (int idx = tid; idx < 64 * 32; idx += 128) {
            int r, k;
            if (TB) { r = idx & 63; k = idx >> 6; } else { k = idx & 31; r = idx >> 5; }
            const int gn = bn + r, gk = k0 + k;
            bf16 val = zero;
            if (gn < N && gk < K) val = TB ? B[(size_t)gk * ldb + gn] : B[(size_t)gn * ldb + gk];
            Bs[r][k] = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 32; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16;
                a[i][0] = ld_pair(&As[r + g][kk + 2 * t]);
                a[i][1] = ld_pair(&As[r + g + 8][kk + 2 * t]);
                a[i][2] = ld_pair(&As[r + g][kk + 2 * t + 8]);
                a[i][3] = ld_pair(&As[r + g + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8;
                b[j][0] = ld_pair(&Bs[c + g][kk + 2 * t]);
                b[j][1] = ld_pair(&Bs[c + g][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int row = bm + wm + i * 16 + g + h * 8;
                    const int col = bn + wn + j * 8 + 2 * t + e;
                    if (row >= M || col >= N) continue;
                    float v = acc[i][j][h * 2 + e];
                    const size_t o = (size_t)row * ldc + col;
                    if (EPI == EPI_BIAS_RELU_BF16) {
                        v = fmaxf(v + bias[col], 0.f);
                        Cb[o] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_BIAS_F32) {
                        Cf[o] = v + bias[col];
                    } else if (EPI == EPI_MASK) {
                        v = __bfloat162float(mask[(size_t)row * ldm + col]) > 0.f ? v : 0.f;
                        Cf[o] = v;
                        Cb[o] = __float2bfloat16_rn(v);
                    } else {
                        Cf[o] = v;
                    }
                }
}

template <bool TA, bool TB, int EPI>
void gemm(int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, const float *bias,
          const bf16 *mask, int ldm, float *Cf, bf16 *Cb, int ldc, cudaStream_t s) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TA, TB, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, bias, mask, ldm, Cf,
                                                   Cb, ldc);
    DOS_LAUNCHED();
}

// ---- loss, gradients, optimiser -----------------------------------------------------
// dy = sign(y - target) / (B n_out) (FP32 and bfloat16); per-block sums of |y - target|.
__global__ void l1_loss_kernel(const float *__restrict__ y, const float *__restrict__ target,
                               int64_t count, float scale, float *__restrict__ dyf,
                               bf16 *__restrict__ dyb, float *__restrict__ part) {
    __shared__ float sh[32];
    float s = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - target[i];
        s += fabsf(d);
        const float gsgn = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        dyf[i] = gsgn;
        dyb[i] = __float2bfloat16_rn(gsgn);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        part[blockIdx.x] = tot;
    }
}

__global__ void loss_final_kernel(const float *part, int n, float scale, float *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = (float)(s * scale);
    }
}

// db[j] = sum_b D[b*ld + j]  (fixed order over b)
__global__ void colsum_kernel(const float *__restrict__ D, int B, int N, int ld,
                              float *__restrict__ db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += D[(size_t)b * ld + j];
    db[j] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            bf16 *__restrict__ wb, int64_t o0, int64_t s0, int64_t o1,
                            int64_t s1, int64_t o2, int64_t s2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        int64_t w = -1;
        if (i >= o0 && i < o0 + s0) w = i - o0;
        else if (i >= o1 && i < o1 + s1) w = s0 + (i - o1);
        else if (i >= o2 && i < o2 + s2) w = s0 + s1 + (i - o2);
        if (w >= 0) wb[w] = __float2bfloat16_rn(pi);
    }
}

int grid1(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

int mfail(dos_mlp *mlp, const Error &e) {
    if (mlp && mlp->ctx) mlp->ctx->last_error = e.msg;
    return e.status;
}

template <typename F>
int mguard(dos_mlp *mlp, F &&f) {
    if (!mlp) return DOS_EINVAL;
    try {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != mlp->ctx->device) DOS_CUDA_TRY(cudaSetDevice(mlp->ctx->device));
        f();
        if (prev >= 0 && prev != mlp->ctx->device) cudaSetDevice(prev);
        mlp->ctx->last_error.clear();
        return DOS_OK;
    } catch (const Error &e) {
        return mfail(mlp, e);
    } catch (const std::bad_alloc &) {
        return mfail(mlp, Error{DOS_ENOMEM, "host allocation failed"});
    }
}

void refresh_bf16_weights(dos_mlp *mlp, cudaStream_t s) {
    to_bf16_kernel<<<grid1(mlp->wsz[0]), 256, 0, s>>>(mlp->params + mlp->off[0], mlp->wb,
                                                      mlp->wsz[0]);
    DOS_LAUNCHED();
    to_bf16_kernel<<<grid1(mlp->wsz[1]), 256, 0, s>>>(mlp->params + mlp->off[2],
                                                      mlp->wb + mlp->wsz[0], mlp->wsz[1]);
    DOS_LAUNCHED();
    to_bf16_kernel<<<grid1(mlp->wsz[2]), 256, 0, s>>>(mlp->params + mlp->off[4],
                                                      mlp->wb + mlp->wsz[0] + mlp->wsz[1],
                                                      mlp->wsz[2]);
    DOS_LAUNCHED();
}

void ensure_batch(dos_mlp *mlp, int B) {
    if (B <= mlp->cap_B) return;
    const size_t nb = (size_t)B;
    const size_t f32 = nb * (mlp->n_in + 3 * (size_t)mlp->n_out + 2 * (size_t)mlp->nh) +
                       kLossBlocks + 1;
    const size_t b16 = nb * ((size_t)mlp->n_in + 4 * (size_t)mlp->nh + mlp->n_out);
    uint8_t *base = (uint8_t *)mlp->acts.get(f32 * 4 + b16 * 2 + 64);
    float *f = (float *)base;
    mlp->xf = f; f += nb * mlp->n_in;
    mlp->tf = f; f += nb * mlp->n_out;
    mlp->y = f; f += nb * mlp->n_out;
    mlp->dyf = f; f += nb * mlp->n_out;
    mlp->dh2f = f; f += nb * mlp->nh;
    mlp->dh1f = f; f += nb * mlp->nh;
    mlp->loss_part = f; f += kLossBlocks + 1;
    bf16 *h = (bf16 *)(((uintptr_t)f + 15) & ~uintptr_t(15));
    mlp->xb = h; h += nb * mlp->n_in;
    mlp->h1 = h; h += nb * mlp->nh;
    mlp->h2 = h; h += nb * mlp->nh;
    mlp->dyb = h; h += nb * mlp->n_out;
    mlp->dh2b = h; h += nb * mlp->nh;
    mlp->dh1b = h;
    mlp->cap_B = B;
}

void stage_input(dos_mlp *mlp, const float *x, int B, const float *target, cudaStream_t s) {
    DOS_REQUIRE(x != nullptr, "x is NULL");
    DOS_REQUIRE(B >= 1 && B <= 65536, "B must be in [1, 65536]");
    ensure_batch(mlp, B);
    DOS_CUDA_TRY(cudaMemcpyAsync(mlp->xf, x, (size_t)B * mlp->n_in * 4, cudaMemcpyDefault, s));
    if (target)
        DOS_CUDA_TRY(cudaMemcpyAsync(mlp->tf, target, (size_t)B * mlp->n_out * 4,
                                     cudaMemcpyDefault, s));
    to_bf16_kernel<<<grid1((int64_t)B * mlp->n_in), 256, 0, s>>>(mlp->xf, mlp->xb,
                                                                 (int64_t)B * mlp->n_in);
    DOS_LAUNCHED();
}

// Input rows of any stride and element type to the bfloat16 operand, through
// FP32 (the type of the network's input): xb[r, j] = bf16(float(x[r * ldx + j])).
template <typename T>
__global__ void stage_rows_kernel(const T *__restrict__ x, int64_t ldx, int n_in, int B,
                                  bf16 *__restrict__ xb) {
    const int64_t total = (int64_t)B * n_in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n_in;
        const int j = (int)(e - r * n_in);
        xb[e] = __float2bfloat16_rn((float)x[r * ldx + j]);
    }
}

void forward(dos_mlp *mlp, int B, cudaStream_t s) {
    const bf16 *W1 = mlp->wb, *W2 = mlp->wb + mlp->wsz[0], *W3 = W2 + mlp->wsz[1];
    const float *p = mlp->params;
    gemm<false, false, EPI_BIAS_RELU_BF16>(B, mlp->nh, mlp->n_in, mlp->xb, mlp->n_in, W1,
                                           mlp->n_in, p + mlp->off[1], nullptr, 0, nullptr,
                                           mlp->h1, mlp->nh, s);
    gemm<false, false, EPI_BIAS_RELU_BF16>(B, mlp->nh, mlp->nh, mlp->h1, mlp->nh, W2, mlp->nh,
                                           p + mlp->off[3], nullptr, 0, nullptr, mlp->h2,
                                           mlp->nh, s);
    gemm<false, false, EPI_BIAS_F32>(B, mlp->n_out, mlp->nh, mlp->h2, mlp->nh, W3, mlp->nh,
                                     p + mlp->off[5], nullptr, 0, mlp->y, nullptr, mlp->n_out, s);
}

// loss into loss_part[kLossBlocks], gradients into mlp->grads
void loss_backward(dos_mlp *mlp, int B, cudaStream_t s) {
    const int64_t cnt = (int64_t)B * mlp->n_out;
    const float scale = (float)(1.0 / (double)cnt);
    l1_loss_kernel<<<kLossBlocks, 256, 0, s>>>(mlp->y, mlp->tf, cnt, scale, mlp->dyf, mlp->dyb,
                                               mlp->loss_part);
    DOS_LAUNCHED();
    loss_final_kernel<<<1, 32, 0, s>>>(mlp->loss_part, kLossBlocks, scale,
                                       mlp->loss_part + kLossBlocks);
    DOS_LAUNCHED();
    const bf16 *W2 = mlp->wb + mlp->wsz[0], *W3 = W2 + mlp->wsz[1];
    float *g = mlp->grads;
    const int H = mlp->nh;
    // layer 3: dW3 = dy^T h2, db3 = sum dy, dh2 = (dy W3) * [h2 > 0]
    gemm<true, true, EPI_F32>(mlp->n_out, H, B, mlp->dyb, mlp->n_out, mlp->h2, H, nullptr,
                              nullptr, 0, g + mlp->off[4], nullptr, H, s);
    colsum_kernel<<<(mlp->n_out + 255) / 256, 256, 0, s>>>(mlp->dyf, B, mlp->n_out, mlp->n_out,
                                                            g + mlp->off[5]);
    DOS_LAUNCHED();
    gemm<false, true, EPI_MASK>(B, H, mlp->n_out, mlp->dyb, mlp->n_out, W3, H, nullptr, mlp->h2,
                                H, mlp->dh2f, mlp->dh2b, H, s);
    // layer 2
    gemm<true, true, EPI_F32>(H, H, B, mlp->dh2b, H, mlp->h1, H, nullptr, nullptr, 0,
                              g + mlp->off[2], nullptr, H, s);
    colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh2f, B, H, H, g + mlp->off[3]);
    DOS_LAUNCHED();
    gemm<false, true, EPI_MASK>(B, H, H, mlp->dh2b, H, W2, H, nullptr, mlp->h1, H, mlp->dh1f,
                                mlp->dh1b, H, s);
    // layer 1
    gemm<true, true, EPI_F32>(H, mlp->n_in, B, mlp->dh1b, H, mlp->xb, mlp->n_in, nullptr,
                              nullptr, 0, g + mlp->off[0], nullptr, mlp->n_in, s);
    colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh1f, B, H, H, g + mlp->off[1]);
    DOS_LAUNCHED();
}

bool is_host_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
}

// ---- checkpoint file ----------------------------------------------------------------
// Little-endian encoding written byte by byte, so the bytes do not depend on the
// host; FNV-1a (64-bit) over everything before the trailing hash.
constexpr unsigned char kMagic[8] = {'D', 'O', 'S', 'M', 'L', 'P', 0, 1};
constexpr size_t kHeaderBytes = 8 + 4 * 4 + 8 + 8;

void put_u32(std::vector<unsigned char> &b, uint32_t v) {
    for (int i = 0; i < 4; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
void put_u64(std::vector<unsigned char> &b, uint64_t v) {
    for (int i = 0; i < 8; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
uint32_t get_u32(const unsigned char *p) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
uint64_t get_u64(const unsigned char *p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}
uint64_t fnv1a64(const unsigned char *p, size_t n) {
    uint64_t h = 14695981039346656037ULL;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}
int64_t count_params(int64_t n_in, int64_t nh, int64_t n_out) {
    return nh * n_in + nh + nh * nh + nh + n_out * nh + n_out;
}

}  // namespace

extern "C" {

int dos_mlp_create(dos_ctx *ctx, int n_in, int n_hidden, int n_out, uint64_t seed,
                   dos_mlp **out) {
    if (!ctx || !out) return DOS_EINVAL;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 8192 || n_hidden > 8192 || n_out > 8192) {
        ctx->last_error = "layer sizes must be in [1, 8192]";
        return DOS_EINVAL;
    }
    dos_mlp *mlp = new (std::nothrow) dos_mlp();
    if (!mlp) return DOS_ENOMEM;
    mlp->ctx = ctx;
    mlp->n_in = n_in;
    mlp->nh = n_hidden;
    mlp->n_out = n_out;
    mlp->wsz[0] = (int64_t)n_hidden * n_in;
    mlp->wsz[1] = (int64_t)n_hidden * n_hidden;
    mlp->wsz[2] = (int64_t)n_out * n_hidden;
    const int64_t sizes[6] = {mlp->wsz[0], n_hidden, mlp->wsz[1], n_hidden, mlp->wsz[2], n_out};
    int64_t o = 0;
    for (int i = 0; i < 6; ++i) {
        mlp->off[i] = o;
        o += sizes[i];
    }
    mlp->n_params = o;
    int rc = mguard(mlp, [&] {
        const int64_t np = mlp->n_params;
        const int64_t nw = mlp->wsz[0] + mlp->wsz[1] + mlp->wsz[2];
        uint8_t *base = (uint8_t *)mlp->state.get(np * 16 + nw * 2 + 64);
        mlp->params = (float *)base;
        mlp->grads = mlp->params + np;
        mlp->m = mlp->grads + np;
        mlp->v = mlp->m + np;
        mlp->wb = (bf16 *)(((uintptr_t)(mlp->v + np) + 15) & ~uintptr_t(15));
        DOS_CUDA_TRY(cudaMemset(mlp->grads, 0, 3 * np * sizeof(float)));
        init_params_kernel<<<grid1(np), 256>>>(mlp->params, np, mlp->off[0], mlp->wsz[0], n_in,
                                               mlp->off[2], mlp->wsz[1], n_hidden, mlp->off[4],
                                               mlp->wsz[2], n_hidden, seed);
        DOS_LAUNCHED();
        refresh_bf16_weights(mlp, 0);
        DOS_CUDA_TRY(cudaDeviceSynchronize());
    });
    if (rc != DOS_OK) {
        mlp->state.release();
        delete mlp;
        return rc;
    }
    *out = mlp;
    return DOS_OK;
}

int dos_mlp_destroy(dos_mlp *mlp) {
    if (!mlp) return DOS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(mlp->ctx->device);
    cudaDeviceSynchronize();
    mlp->state.release();
    mlp->acts.release();
    mlp->in_stage.release();
    if (prev >= 0) cudaSetDevice(prev);
    cudaGetLastError();
    delete mlp;
    return DOS_OK;
}

int dos_mlp_num_params(const dos_mlp *mlp, int64_t *count) {
    if (!mlp || !count) return DOS_EINVAL;
    *count = mlp->n_params;
    return DOS_OK;
}

int dos_mlp_set_params(dos_mlp *mlp, const float *params, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(params != nullptr, "params is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        DOS_CUDA_TRY(cudaMemcpyAsync(mlp->params, params, mlp->n_params * 4, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemsetAsync(mlp->m, 0, 2 * mlp->n_params * 4, s));
        mlp->step = 0;
        refresh_bf16_weights(mlp, s);
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_mlp_get_params(dos_mlp *mlp, float *params, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(params != nullptr, "params is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        DOS_CUDA_TRY(cudaMemcpyAsync(params, mlp->params, mlp->n_params * 4, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_mlp_forward(dos_mlp *mlp, const float *x, int B, float *y, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(y != nullptr, "y is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        stage_input(mlp, x, B, nullptr, s);
        forward(mlp, B, s);
        DOS_CUDA_TRY(cudaMemcpyAsync(y, mlp->y, (size_t)B * mlp->n_out * 4, cudaMemcpyDefault, s));
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, y) != cudaSuccess) cudaGetLastError();
        else if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_mlp_infer(dos_mlp *mlp, const void *x, int x_dtype, int64_t ldx, int64_t B, float *y,
                  int max_rows, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(x != nullptr && y != nullptr, "x / y is NULL");
        DOS_REQUIRE(x_dtype == DOS_F32 || x_dtype == DOS_F64, "x_dtype must be DOS_F32 or DOS_F64");
        DOS_REQUIRE(B >= 1, "B must be >= 1");
        DOS_REQUIRE(max_rows >= 0 && max_rows <= 65536, "max_rows must be in [0, 65536]");
        if (ldx == 0) ldx = mlp->n_in;
        DOS_REQUIRE(ldx >= mlp->n_in, "ldx must be >= n_in");
        const int rows = max_rows ? max_rows : 8192;
        const size_t esz = x_dtype == DOS_F64 ? 8 : 4;
        const bool x_host = is_host_ptr(x);
        cudaStream_t s = (cudaStream_t)stream;
        for (int64_t r0 = 0; r0 < B; r0 += rows) {
            const int b = (int)std::min<int64_t>(rows, B - r0);
            ensure_batch(mlp, b);
            const uint8_t *src = (const uint8_t *)x + (size_t)r0 * ldx * esz;
            if (x_host) {  // the slice's rows, copied as one block
                const size_t bytes = ((size_t)(b - 1) * ldx + mlp->n_in) * esz;
                void *d = mlp->in_stage.get(bytes);
                DOS_CUDA_TRY(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
                src = (const uint8_t *)d;
            }
            if (x_dtype == DOS_F64)
                stage_rows_kernel<double><<<grid1((int64_t)b * mlp->n_in), 256, 0, s>>>(
                    (const double *)src, ldx, mlp->n_in, b, mlp->xb);
            else
                stage_rows_kernel<float><<<grid1((int64_t)b * mlp->n_in), 256, 0, s>>>(
                    (const float *)src, ldx, mlp->n_in, b, mlp->xb);
            DOS_LAUNCHED();
            forward(mlp, b, s);
            DOS_CUDA_TRY(cudaMemcpyAsync(y + r0 * mlp->n_out, mlp->y,
                                         (size_t)b * mlp->n_out * 4, cudaMemcpyDefault, s));
            // the next slice overwrites the staging and activation buffers: with a host
            // output the copy above must finish first (stream order covers device ones)
            if (x_host || is_host_ptr(y)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
        }
    });
}

int dos_mlp_save(dos_mlp *mlp, const char *path, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(path != nullptr, "path is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t np = mlp->n_params;
        std::vector<float> host((size_t)(3 * np));
        // params, then the Adam moments m and v (adjacent after the gradients)
        DOS_CUDA_TRY(cudaMemcpyAsync(host.data(), mlp->params, np * 4, cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(host.data() + np, mlp->m, 2 * np * 4, cudaMemcpyDeviceToHost,
                                     s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<unsigned char> b;
        b.reserve(kHeaderBytes + (size_t)(12 * np) + 8);
        b.insert(b.end(), kMagic, kMagic + 8);
        put_u32(b, (uint32_t)mlp->n_in);
        put_u32(b, (uint32_t)mlp->nh);
        put_u32(b, (uint32_t)mlp->n_out);
        put_u32(b, 0u);
        put_u64(b, (uint64_t)mlp->step);
        put_u64(b, (uint64_t)np);
        for (float f : host) {
            uint32_t u;
            memcpy(&u, &f, 4);
            put_u32(b, u);
        }
        put_u64(b, fnv1a64(b.data(), b.size()));
        const std::string tmp = std::string(path) + ".partial";
        FILE *f = fopen(tmp.c_str(), "wb");
        if (!f) throw Error{DOS_EIO, std::string("cannot open ") + tmp + " for writing"};
        const size_t w = fwrite(b.data(), 1, b.size(), f);
        const int cl = fclose(f);
        if (w != b.size() || cl != 0) {
            remove(tmp.c_str());
            throw Error{DOS_EIO, std::string("short write to ") + tmp};
        }
        if (rename(tmp.c_str(), path) != 0) {
            remove(tmp.c_str());
            throw Error{DOS_EIO, std::string("cannot rename ") + tmp + " to " + path};
        }
    });
}

int dos_mlp_load(dos_ctx *ctx, const char *path, dos_mlp **out, void *stream) {
    if (!ctx || !out || !path) return DOS_EINVAL;
    *out = nullptr;
    std::vector<unsigned char> b;
    {
        FILE *f = fopen(path, "rb");
        if (!f) {
            ctx->last_error = std::string("cannot open ") + path;
            return DOS_EIO;
        }
        unsigned char chunk[1 << 16];
        size_t got;
        while ((got = fread(chunk, 1, sizeof(chunk), f)) > 0) b.insert(b.end(), chunk, chunk + got);
        const bool err = ferror(f) != 0;
        fclose(f);
        if (err) {
            ctx->last_error = std::string("read error on ") + path;
            return DOS_EIO;
        }
    }
    auto bad = [&](const char *why) {
        ctx->last_error = std::string(path) + ": " + why;
        return DOS_EIO;
    };
    if (b.size() < kHeaderBytes + 8) return bad("too short for a network file");
    if (memcmp(b.data(), kMagic, 8) != 0) return bad("not a network file of format version 1");
    const uint32_t n_in = get_u32(&b[8]), nh = get_u32(&b[12]), n_out = get_u32(&b[16]);
    const uint64_t step = get_u64(&b[24]), np = get_u64(&b[32]);
    if (n_in < 1 || nh < 1 || n_out < 1 || n_in > 8192 || nh > 8192 || n_out > 8192)
        return bad("layer sizes out of range");
    if (np != (uint64_t)count_params(n_in, nh, n_out)) return bad("parameter count disagrees");
    if (b.size() != kHeaderBytes + 12 * np + 8) return bad("length disagrees with the sizes");
    if (fnv1a64(b.data(), b.size() - 8) != get_u64(&b[b.size() - 8])) return bad("hash mismatch");
    std::vector<float> host((size_t)(3 * np));
    for (size_t i = 0; i < host.size(); ++i) {
        const uint32_t u = get_u32(&b[kHeaderBytes + 4 * i]);
        memcpy(&host[i], &u, 4);
    }
    dos_mlp *mlp = nullptr;
    int rc = dos_mlp_create(ctx, (int)n_in, (int)nh, (int)n_out, 0, &mlp);
    if (rc != DOS_OK) return rc;
    rc = mguard(mlp, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        DOS_CUDA_TRY(cudaMemcpyAsync(mlp->params, host.data(), np * 4, cudaMemcpyHostToDevice, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(mlp->m, host.data() + np, 2 * np * 4,
                                     cudaMemcpyHostToDevice, s));
        mlp->step = (int64_t)step;
        refresh_bf16_weights(mlp, s);
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
    if (rc != DOS_OK) {
        dos_mlp_destroy(mlp);
        return rc;
    }
    *out = mlp;
    return DOS_OK;
}

int dos_mlp_loss_grad(dos_mlp *mlp, const float *x, const float *target, int B, float *loss,
                      float *grads, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(target != nullptr, "target is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        stage_input(mlp, x, B, target, s);
        forward(mlp, B, s);
        loss_backward(mlp, B, s);
        if (grads)
            DOS_CUDA_TRY(cudaMemcpyAsync(grads, mlp->grads, mlp->n_params * 4, cudaMemcpyDefault, s));
        float h = 0.f;
        DOS_CUDA_TRY(cudaMemcpyAsync(&h, mlp->loss_part + kLossBlocks, 4, cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (loss) *loss = h;
    });
}

int dos_mlp_train_step(dos_mlp *mlp, const float *x, const float *target, int B, float lr,
                       float *loss, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(target != nullptr, "target is NULL");
        DOS_REQUIRE(isfinite(lr) && lr > 0.f, "lr must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        stage_input(mlp, x, B, target, s);
        forward(mlp, B, s);
        loss_backward(mlp, B, s);
        mlp->step += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 - pow(b1, (double)mlp->step));
        const float c2 = (float)(1.0 - pow(b2, (double)mlp->step));
        adam_kernel<<<grid1(mlp->n_params), 256, 0, s>>>(
            mlp->params, mlp->grads, mlp->m, mlp->v, mlp->n_params, lr, (float)b1, (float)b2,
            1e-8f, c1, c2, mlp->wb, mlp->off[0], mlp->wsz[0], mlp->off[2], mlp->wsz[1],
            mlp->off[4], mlp->wsz[2]);
        DOS_LAUNCHED();
        if (loss) {
            float h = 0.f;
            DOS_CUDA_TRY(cudaMemcpyAsync(&h, mlp->loss_part + kLossBlocks, 4,
                                         cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
            *loss = h;
        }
    });
}

}  // extern "C"
