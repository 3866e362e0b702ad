// The learned part (not in the paper): a 3-layer perceptron from low-order
// Chebyshev moments to a DOS on a grid, trained and run entirely by these
// kernels.  The nine matrix products of a training step (three forward, six
// backward) run on the fifth-generation tensor cores (mlp_tc.cu: TMA-fed
// tcgen05.mma with the FP32 accumulator in tensor memory, bfloat16 operands)
// with fused epilogues (bias + ReLU, ReLU-mask back-propagation).  Every product
// is C = A B^T with both operands K-contiguous, so the kernels that produce an
// operand also write the transposed copy the backward pass needs (activations,
// output gradient, weights).  The loss, bias gradients and Adam run in FP32.
// All reductions have a fixed order, so a training run is bitwise reproducible.
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
    Buffer flags;          // status word of the bounded waits of the tensor-core kernels
    int cap_B = 0;
    int64_t step = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    // bfloat16 weights with leading dimensions padded to 8 (tensor-map rows), and
    // the transposes of W2 and W3 for the backward products
    bf16 *W1b = nullptr, *W2b = nullptr, *W2t = nullptr, *W3b = nullptr, *W3t = nullptr;
    int *status = nullptr;
    // batch buffers (cap_B rows; bf16 operands with padded leading dimensions)
    float *xf = nullptr, *tf = nullptr, *y = nullptr, *dyf = nullptr, *dh2f = nullptr,
          *dh1f = nullptr, *loss_part = nullptr;
    bf16 *xb = nullptr, *xbt = nullptr, *h1 = nullptr, *h1t = nullptr, *h2 = nullptr,
         *h2t = nullptr, *dyb = nullptr, *dybt = nullptr, *dh2b = nullptr, *dh2t = nullptr,
         *dh1t = nullptr;
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

// Leading dimension of a bfloat16 operand with k contiguous elements per row:
// rows of a tensor map must be multiples of 16 bytes.
inline int pad8(int k) { return (k + 7) / 8 * 8; }

// FP32 rows x cols matrix (contiguous) -> bf16 with leading dimension ld and,
// when out_t is given, the transpose (cols x rows, leading dimension ld_t).
__global__ void to_bf16_pad_kernel(const float *__restrict__ in, int rows, int cols,
                                   bf16 *__restrict__ out, int ld, bf16 *__restrict__ out_t,
                                   int ld_t) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
        const bf16 h = __float2bfloat16_rn(in[e]);
        out[(size_t)r * ld + c] = h;
        if (out_t) out_t[(size_t)c * ld_t + r] = h;
    }
}

// ---- loss, gradients, optimiser -----------------------------------------------------
// dy = sign(y - target) / (B n_out): FP32 (for the bias gradient) and bfloat16, row-major
// and transposed (operands of the two layer-3 products); per-block sums of |y - target|.
__global__ void l1_loss_kernel(const float *__restrict__ y, const float *__restrict__ target,
                               int B, int n_out, float scale, float *__restrict__ dyf,
                               bf16 *__restrict__ dyb, int ldb, bf16 *__restrict__ dybt,
                               int ldt, float *__restrict__ part) {
    __shared__ float sh[32];
    float s = 0.f;
    const int64_t count = (int64_t)B * n_out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / n_out), o = (int)(i - (int64_t)b * n_out);
        const float d = y[i] - target[i];
        s += fabsf(d);
        const float gsgn = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        dyf[i] = gsgn;
        const bf16 h = __float2bfloat16_rn(gsgn);
        dyb[(size_t)b * ldb + o] = h;
        dybt[(size_t)o * ldt + b] = h;
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
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
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
    const int nh = mlp->nh, n_in = mlp->n_in, n_out = mlp->n_out;
    to_bf16_pad_kernel<<<grid1(mlp->wsz[0]), 256, 0, s>>>(mlp->params + mlp->off[0], nh, n_in,
                                                          mlp->W1b, pad8(n_in), nullptr, 0);
    DOS_LAUNCHED();
    to_bf16_pad_kernel<<<grid1(mlp->wsz[1]), 256, 0, s>>>(mlp->params + mlp->off[2], nh, nh,
                                                          mlp->W2b, pad8(nh), mlp->W2t, pad8(nh));
    DOS_LAUNCHED();
    to_bf16_pad_kernel<<<grid1(mlp->wsz[2]), 256, 0, s>>>(mlp->params + mlp->off[4], n_out, nh,
                                                          mlp->W3b, pad8(nh), mlp->W3t,
                                                          pad8(n_out));
    DOS_LAUNCHED();
}

// Bump allocator over one device buffer; every piece 256-byte aligned (TMA needs 16).
struct Carve {
    uint8_t *p;
    template <typename T>
    T *take(size_t count) {
        T *r = (T *)p;
        p += (count * sizeof(T) + 255) / 256 * 256;
        return r;
    }
};

void ensure_batch(dos_mlp *mlp, int B) {
    if (B <= mlp->cap_B) return;
    const size_t nb = (size_t)B, pb = (size_t)pad8(B);
    const size_t ni = mlp->n_in, nh = mlp->nh, no = mlp->n_out;
    const size_t pi = pad8(mlp->n_in), ph = pad8(mlp->nh), po = pad8(mlp->n_out);
    const size_t f32 = nb * (ni + 3 * no + 2 * ph) + kLossBlocks + 1;
    const size_t b16 = nb * (pi + 2 * ph + po + ph) + pb * (ni + 2 * nh + no + 2 * nh);
    Carve c{(uint8_t *)mlp->acts.get(f32 * 4 + b16 * 2 + 20 * 256)};
    mlp->xf = c.take<float>(nb * ni);
    mlp->tf = c.take<float>(nb * no);
    mlp->y = c.take<float>(nb * no);
    mlp->dyf = c.take<float>(nb * no);
    mlp->dh2f = c.take<float>(nb * ph);
    mlp->dh1f = c.take<float>(nb * ph);
    mlp->loss_part = c.take<float>(kLossBlocks + 1);
    mlp->xb = c.take<bf16>(nb * pi);
    mlp->h1 = c.take<bf16>(nb * ph);
    mlp->h2 = c.take<bf16>(nb * ph);
    mlp->dyb = c.take<bf16>(nb * po);
    mlp->dh2b = c.take<bf16>(nb * ph);
    mlp->xbt = c.take<bf16>(ni * pb);
    mlp->h1t = c.take<bf16>(nh * pb);
    mlp->h2t = c.take<bf16>(nh * pb);
    mlp->dybt = c.take<bf16>(no * pb);
    mlp->dh2t = c.take<bf16>(nh * pb);
    mlp->dh1t = c.take<bf16>(nh * pb);
    mlp->cap_B = B;
}

// Input rows of any stride and element type to the bfloat16 operand (leading
// dimension ld), through FP32 (the type of the network's input):
// xb[r, j] = bf16(float(x[r * ldx + j])); with xbt, also the transpose.
template <typename T>
__global__ void stage_rows_kernel(const T *__restrict__ x, int64_t ldx, int n_in, int B,
                                  bf16 *__restrict__ xb, int ld, bf16 *__restrict__ xbt,
                                  int ldt) {
    const int64_t total = (int64_t)B * n_in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n_in;
        const int j = (int)(e - r * n_in);
        const bf16 h = __float2bfloat16_rn((float)x[r * ldx + j]);
        xb[r * ld + j] = h;
        if (xbt) xbt[(size_t)j * ldt + r] = h;
    }
}

// Training-batch input: x (B x n_in FP32, host or device) and optional target.
void stage_input(dos_mlp *mlp, const float *x, int B, const float *target, bool train,
                 cudaStream_t s) {
    DOS_REQUIRE(x != nullptr, "x is NULL");
    DOS_REQUIRE(B >= 1 && B <= 65536, "B must be in [1, 65536]");
    ensure_batch(mlp, B);
    DOS_CUDA_TRY(cudaMemcpyAsync(mlp->xf, x, (size_t)B * mlp->n_in * 4, cudaMemcpyDefault, s));
    if (target)
        DOS_CUDA_TRY(cudaMemcpyAsync(mlp->tf, target, (size_t)B * mlp->n_out * 4,
                                     cudaMemcpyDefault, s));
    stage_rows_kernel<float><<<grid1((int64_t)B * mlp->n_in), 256, 0, s>>>(
        mlp->xf, mlp->n_in, mlp->n_in, B, mlp->xb, pad8(mlp->n_in), train ? mlp->xbt : nullptr,
        pad8(B));
    DOS_LAUNCHED();
}

constexpr long long kSpinCycles = 4000000000LL;  // about two seconds at 2 GHz

TcGemm tc(dos_mlp *mlp, int M, int N, int K, int epi) {
    TcGemm g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.status = mlp->status;
    g.spin = kSpinCycles;
    return g;
}

// With train, the products also write the transposed activations the backward
// products read.
void forward(dos_mlp *mlp, int B, bool train, cudaStream_t s) {
    const float *p = mlp->params;
    const int pi = pad8(mlp->n_in), ph = pad8(mlp->nh), pb = pad8(B);
    TcGemm g = tc(mlp, B, mlp->nh, mlp->n_in, TC_EPI_BIAS_RELU_BF16);
    g.bias = p + mlp->off[1];
    g.Cb = mlp->h1;
    g.ldc = ph;
    g.Ct = train ? mlp->h1t : nullptr;
    g.ldt = pb;
    launch_gemm_tc(g, mlp->xb, pi, mlp->W1b, pi, s);
    g = tc(mlp, B, mlp->nh, mlp->nh, TC_EPI_BIAS_RELU_BF16);
    g.bias = p + mlp->off[3];
    g.Cb = mlp->h2;
    g.ldc = ph;
    g.Ct = train ? mlp->h2t : nullptr;
    g.ldt = pb;
    launch_gemm_tc(g, mlp->h1, ph, mlp->W2b, ph, s);
    g = tc(mlp, B, mlp->n_out, mlp->nh, TC_EPI_BIAS_F32);
    g.bias = p + mlp->off[5];
    g.Cf = mlp->y;
    g.ldc = mlp->n_out;
    launch_gemm_tc(g, mlp->h2, ph, mlp->W3b, ph, s);
}

// loss into loss_part[kLossBlocks], gradients into mlp->grads
void loss_backward(dos_mlp *mlp, int B, cudaStream_t s) {
    const int64_t cnt = (int64_t)B * mlp->n_out;
    const float scale = (float)(1.0 / (double)cnt);
    const int H = mlp->nh, pb = pad8(B), ph = pad8(H), po = pad8(mlp->n_out);
    l1_loss_kernel<<<kLossBlocks, 256, 0, s>>>(mlp->y, mlp->tf, B, mlp->n_out, scale, mlp->dyf,
                                               mlp->dyb, po, mlp->dybt, pb, mlp->loss_part);
    DOS_LAUNCHED();
    loss_final_kernel<<<1, 32, 0, s>>>(mlp->loss_part, kLossBlocks, scale,
                                       mlp->loss_part + kLossBlocks);
    DOS_LAUNCHED();
    float *gr = mlp->grads;
    // layer 3: dW3 = dy^T h2, db3 = sum dy, dh2 = (dy W3) * [h2 > 0]
    TcGemm g = tc(mlp, mlp->n_out, H, B, TC_EPI_F32);
    g.Cf = gr + mlp->off[4];
    g.ldc = H;
    launch_gemm_tc(g, mlp->dybt, pb, mlp->h2t, pb, s);
    colsum_kernel<<<(mlp->n_out + 255) / 256, 256, 0, s>>>(mlp->dyf, B, mlp->n_out, mlp->n_out,
                                                            gr + mlp->off[5]);
    DOS_LAUNCHED();
    g = tc(mlp, B, H, mlp->n_out, TC_EPI_MASK);
    g.mask = mlp->h2;
    g.ldm = ph;
    g.Cf = mlp->dh2f;
    g.Cb = mlp->dh2b;
    g.ldc = ph;
    g.Ct = mlp->dh2t;
    g.ldt = pb;
    launch_gemm_tc(g, mlp->dyb, po, mlp->W3t, po, s);
    // layer 2: dW2 = dh2^T h1, db2 = sum dh2, dh1 = (dh2 W2) * [h1 > 0]
    g = tc(mlp, H, H, B, TC_EPI_F32);
    g.Cf = gr + mlp->off[2];
    g.ldc = H;
    launch_gemm_tc(g, mlp->dh2t, pb, mlp->h1t, pb, s);
    colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh2f, B, H, ph, gr + mlp->off[3]);
    DOS_LAUNCHED();
    g = tc(mlp, B, H, H, TC_EPI_MASK);
    g.mask = mlp->h1;
    g.ldm = ph;
    g.Cf = mlp->dh1f;
    g.ldc = ph;
    g.Ct = mlp->dh1t;
    g.ldt = pb;
    launch_gemm_tc(g, mlp->dh2b, ph, mlp->W2t, ph, s);
    // layer 1: dW1 = dh1^T x, db1 = sum dh1
    g = tc(mlp, H, mlp->n_in, B, TC_EPI_F32);
    g.Cf = gr + mlp->off[0];
    g.ldc = mlp->n_in;
    launch_gemm_tc(g, mlp->dh1t, pb, mlp->xbt, pb, s);
    colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(mlp->dh1f, B, H, ph, gr + mlp->off[1]);
    DOS_LAUNCHED();
}

// The tensor-core products' bounded waits (status bit 8): read after a sync.
void check_status(dos_mlp *mlp, cudaStream_t s) {
    int h = 0;
    DOS_CUDA_TRY(cudaMemcpyAsync(&h, mlp->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DOS_CUDA_TRY(cudaStreamSynchronize(s));
    if (h & 8) {
        DOS_CUDA_TRY(cudaMemsetAsync(mlp->status, 0, sizeof(int), s));
        throw Error{DOS_ETIMEOUT, "a bounded wait of the tensor-core product ran out"};
    }
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
        const size_t pi = pad8(n_in), ph = pad8(n_hidden), po = pad8(n_out);
        const size_t nwb = (size_t)n_hidden * pi + 2 * (size_t)n_hidden * ph +
                           (size_t)n_out * ph + (size_t)n_hidden * po;
        Carve c{(uint8_t *)mlp->state.get(np * 16 + nwb * 2 + 8 * 256)};
        mlp->params = c.take<float>(4 * np);  // params | grads | m | v, adjacent
        mlp->grads = mlp->params + np;
        mlp->m = mlp->grads + np;
        mlp->v = mlp->m + np;
        mlp->W1b = c.take<bf16>((size_t)n_hidden * pi);
        mlp->W2b = c.take<bf16>((size_t)n_hidden * ph);
        mlp->W2t = c.take<bf16>((size_t)n_hidden * ph);
        mlp->W3b = c.take<bf16>((size_t)n_out * ph);
        mlp->W3t = c.take<bf16>((size_t)n_hidden * po);
        mlp->status = (int *)mlp->flags.get(sizeof(int));
        DOS_CUDA_TRY(cudaMemset(mlp->status, 0, sizeof(int)));
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
        mlp->flags.release();
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
    mlp->flags.release();
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
        check_status(mlp, s);
    });
}

int dos_mlp_forward(dos_mlp *mlp, const float *x, int B, float *y, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(y != nullptr, "y is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        stage_input(mlp, x, B, nullptr, false, s);
        forward(mlp, B, false, s);
        DOS_CUDA_TRY(cudaMemcpyAsync(y, mlp->y, (size_t)B * mlp->n_out * 4, cudaMemcpyDefault, s));
        if (is_host_ptr(y)) check_status(mlp, s);
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
            const int pi = pad8(mlp->n_in);
            if (x_dtype == DOS_F64)
                stage_rows_kernel<double><<<grid1((int64_t)b * mlp->n_in), 256, 0, s>>>(
                    (const double *)src, ldx, mlp->n_in, b, mlp->xb, pi, nullptr, 0);
            else
                stage_rows_kernel<float><<<grid1((int64_t)b * mlp->n_in), 256, 0, s>>>(
                    (const float *)src, ldx, mlp->n_in, b, mlp->xb, pi, nullptr, 0);
            DOS_LAUNCHED();
            forward(mlp, b, false, s);
            DOS_CUDA_TRY(cudaMemcpyAsync(y + r0 * mlp->n_out, mlp->y,
                                         (size_t)b * mlp->n_out * 4, cudaMemcpyDefault, s));
            // the next slice overwrites the staging and activation buffers: with a host
            // output the copy above must finish first (stream order covers device ones)
            if (x_host || is_host_ptr(y)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (x_host || is_host_ptr(y)) check_status(mlp, s);
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
        check_status(mlp, s);   // synchronises; no checkpoint of a step whose products timed out
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
        stage_input(mlp, x, B, target, true, s);
        forward(mlp, B, true, s);
        loss_backward(mlp, B, s);
        if (grads)
            DOS_CUDA_TRY(cudaMemcpyAsync(grads, mlp->grads, mlp->n_params * 4, cudaMemcpyDefault, s));
        float h = 0.f;
        DOS_CUDA_TRY(cudaMemcpyAsync(&h, mlp->loss_part + kLossBlocks, 4, cudaMemcpyDeviceToHost, s));
        check_status(mlp, s);
        if (loss) *loss = h;
    });
}

int dos_mlp_train_step(dos_mlp *mlp, const float *x, const float *target, int B, float lr,
                       float *loss, void *stream) {
    return mguard(mlp, [&] {
        DOS_REQUIRE(target != nullptr, "target is NULL");
        DOS_REQUIRE(isfinite(lr) && lr > 0.f, "lr must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        stage_input(mlp, x, B, target, true, s);
        forward(mlp, B, true, s);
        loss_backward(mlp, B, s);
        mlp->step += 1;
        const double b1 = 0.9, b2 = 0.999;
        const float c1 = (float)(1.0 - pow(b1, (double)mlp->step));
        const float c2 = (float)(1.0 - pow(b2, (double)mlp->step));
        adam_kernel<<<grid1(mlp->n_params), 256, 0, s>>>(
            mlp->params, mlp->grads, mlp->m, mlp->v, mlp->n_params, lr, (float)b1, (float)b2,
            1e-8f, c1, c2);
        DOS_LAUNCHED();
        refresh_bf16_weights(mlp, s);
        if (loss) {
            float h = 0.f;
            DOS_CUDA_TRY(cudaMemcpyAsync(&h, mlp->loss_part + kLossBlocks, 4,
                                         cudaMemcpyDeviceToHost, s));
            check_status(mlp, s);
            *loss = h;
        }
    });
}

}  // extern "C"
