// Dense products of the learned network on the fifth-generation tensor cores.
//
//   C = epilogue(A B^T),  A: M x K and B: N x K bfloat16, row-major with K
//   contiguous (leading dimensions multiples of 8 elements), FP32 accumulation.
//
// One CTA of 128 threads computes a 128 x 128 tile of C:
//   * one thread streams K-slices of 64 elements (128 bytes of a row) of A and B
//     into a ring of shared-memory stages with TMA (cp.async.bulk.tensor, 128-byte
//     swizzle, rows past M, N or K filled with zeros), each completing on the
//     stage's "full" mbarrier;
//   * the same thread issues tcgen05.mma (kind::f16: BF16 operands, FP32
//     accumulator in tensor memory, M = N = 128, K = 16 per instruction, four per
//     slice) and tcgen05.commit to the stage's "empty" mbarrier, which fires when
//     the MMAs reading the stage are done; the stage of the previous slice is
//     refilled while the current slice's MMAs run;
//   * a last commit to "done" releases the four warps, which read the
//     accumulator with tcgen05.ld (warp w owns tensor-memory lanes 32w..32w+31,
//     the tile's rows) into an FP32 tile in the (now idle) stage memory, padded to
//     129 columns so that neither a thread writing its row nor a warp reading a
//     row or a column conflicts on banks; the epilogue then leaves the tile in two
//     coalesced passes, row by row for the row-major outputs (bias and mask read
//     along the row) and column by column for the transposed bf16 copy.
// Every mbarrier wait is bounded (spin cycles): a wait that runs out sets status
// bit 8, the CTA waits (bounded again) for what it issued, frees its tensor
// memory and skips the stores.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "dos_internal.h"

namespace dos {
namespace {

typedef __nv_bfloat16 bf16;

// Three stages (99 KB of shared memory) leave room for two CTAs per SM, so one
// tile's epilogue overlaps another's loads and products.
constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3, kThreads = 128;
constexpr uint32_t kTileBytes = kBM * kBK * 2;     // one operand slice: 128 rows x 128 B
constexpr uint32_t kStageBytes = 2 * kTileBytes;   // A and B (kBN == kBM)
constexpr uint32_t kTmemCols = kBN;                // FP32 accumulator: one column per n
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + 256;

// Instruction descriptor of tcgen05.mma .kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand slice in the 128-byte
// swizzled layout TMA writes (rows of 128 bytes, groups of eight rows 1024 bytes
// apart): start address >> 4 in bits 0-13, leading-dimension offset (not used by
// swizzled K-major layouts) 1 in bits 16-29, stride offset 1024 >> 4 in bits 32-45,
// descriptor version 1 in bits 46-47, swizzle mode 2 (128-byte) in bits 61-63.
// Stepping K by 16 within the 128-byte row adds 32 bytes to the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(saddr(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}
// 32 consecutive FP32 columns of this thread's lane (warp w: lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

template <int EPI>
__global__ void __launch_bounds__(kThreads, 2)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a,
                   const __grid_constant__ CUtensorMap map_b, const TcGemm g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_fail;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + (size_t)kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int nk = (g.K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        auto load = [&](int kc) {
            const int s = kc % kStages;
            uint8_t *sa = smem + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            tma_load_2d(sa, &map_a, kc * kBK, m0, &full[s]);
            tma_load_2d(sa + kTileBytes, &map_b, kc * kBK, n0, &full[s]);
        };
        const int pre = nk < kStages ? nk : kStages;
        for (int kc = 0; kc < pre; ++kc) load(kc);
        int issued = pre, consumed = 0;
        bool ok = true;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % kStages;
            if (!mbar_wait(&full[s], (kc / kStages) & 1, g.spin)) {
                ok = false;
                break;
            }
            consumed = kc + 1;
            const uint32_t sa = saddr(smem + (size_t)s * kStageBytes), sb = sa + kTileBytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32),
                         (kc | kk) != 0 ? 1u : 0u);
            mma_commit(&empty[s]);
            if (kc >= 1 && kc - 1 + kStages < nk) {  // refill the previous slice's stage
                const int p = kc - 1;
                if (!mbar_wait(&empty[p % kStages], (p / kStages) & 1, g.spin)) {
                    ok = false;
                    break;
                }
                load(p + kStages);
                issued = p + kStages + 1;
            }
        }
        mma_commit(done);  // fires once every MMA issued above has completed
        if (!ok) {
            atomicOr(g.status, 8);
            s_fail = 1;
            for (int kc = consumed; kc < issued; ++kc)  // loads still writing shared memory
                mbar_wait(&full[kc % kStages], (kc / kStages) & 1, g.spin);
        }
    }
    bool waited = mbar_wait(done, 0, g.spin);
    if (!waited) waited = mbar_wait(done, 0, g.spin);  // once more before giving up
    if (!waited && lane == 0) atomicOr(g.status, 8);
    const int bad = __syncthreads_or(!waited || s_fail);
    tc_fence_after();

    constexpr int kLd = kBN + 1;  // staged tile row stride (floats)
    float *tile = reinterpret_cast<float *>(smem);
    if (!bad) {
        const int r = warp * 32 + lane;  // tile row of this thread's TMEM lane
#pragma unroll 1
        for (int c = 0; c < kBN / 32; ++c) {
            if (n0 + c * 32 >= g.N) break;  // warp-uniform
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[r * kLd + c * 32 + j] = v[j];
        }
    }
    __syncthreads();
    if (!bad) {
        const int rows = min(kBM, g.M - m0), cols = min(kBN, g.N - n0);
        // row-major outputs: a warp walks one row, lanes over consecutive columns
        for (int idx = threadIdx.x; idx < rows * kBN; idx += kThreads) {
            const int rr = idx / kBN, cc = idx - rr * kBN;
            if (cc >= cols) continue;
            const int row = m0 + rr, col = n0 + cc;
            float x = tile[rr * kLd + cc];
            const size_t o = (size_t)row * g.ldc + col;
            if (EPI == TC_EPI_BIAS_RELU_BF16) {
                x = fmaxf(x + g.bias[col], 0.f);
                ((bf16 *)g.Cb)[o] = __float2bfloat16_rn(x);
            } else if (EPI == TC_EPI_BIAS_F32) {
                g.Cf[o] = x + g.bias[col];
            } else if (EPI == TC_EPI_MASK) {
                x = __bfloat162float(((const bf16 *)g.mask)[(size_t)row * g.ldm + col]) > 0.f
                        ? x : 0.f;
                g.Cf[o] = x;
                if (g.Cb) ((bf16 *)g.Cb)[o] = __float2bfloat16_rn(x);
            } else {
                g.Cf[o] = x;
            }
            tile[rr * kLd + cc] = x;  // the epilogue's value, for the transposed pass
        }
        if (g.Ct) {
            __syncthreads();
            // transposed bf16 copy: a warp walks one column, lanes over consecutive rows
            for (int idx = threadIdx.x; idx < cols * kBM; idx += kThreads) {
                const int cc = idx / kBM, rr = idx - cc * kBM;
                if (rr >= rows) continue;
                ((bf16 *)g.Ct)[(size_t)(n0 + cc) * g.ldt + m0 + rr] =
                    __float2bfloat16_rn(tile[rr * kLd + cc]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

// Tensor map of a rows x K bfloat16 matrix (leading dimension ld elements) with
// boxes of 128 rows x 64 elements, 128-byte swizzle, zero fill outside.
CUtensorMap bf16_map(const void *base, int K, int rows, int ld) {
    EncodeFn enc = encode_fn();
    if (!enc) throw Error{DOS_ECUDA, "cuTensorMapEncodeTiled is not available"};
    DOS_REQUIRE(((uintptr_t)base & 15) == 0 && ld % 8 == 0 && ld >= K,
                "tensor-core operand: 16-byte aligned base and ld a multiple of 8 >= K");
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{DOS_ECUDA, "cuTensorMapEncodeTiled rejected an operand"};
    return m;
}

template <int EPI>
void launch_epi(const CUtensorMap &ma, const CUtensorMap &mb, const TcGemm &g, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(gemm_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemBytes);
    });
    DOS_CUDA_TRY(attr);
    const dim3 grid((g.N + kBN - 1) / kBN, (g.M + kBM - 1) / kBM);
    gemm_tc_kernel<EPI><<<grid, kThreads, kSmemBytes, s>>>(ma, mb, g);
    DOS_LAUNCHED();
}

}  // namespace

void launch_gemm_tc(const TcGemm &g, const void *A, int lda, const void *B, int ldb,
                    cudaStream_t s) {
    DOS_REQUIRE(g.M >= 1 && g.N >= 1 && g.K >= 1 && g.M <= 65535 * kBM, "GEMM sizes");
    const CUtensorMap ma = bf16_map(A, g.K, g.M, lda);
    const CUtensorMap mb = bf16_map(B, g.K, g.N, ldb);
    switch (g.epi) {
        case TC_EPI_BIAS_RELU_BF16: launch_epi<TC_EPI_BIAS_RELU_BF16>(ma, mb, g, s); break;
        case TC_EPI_BIAS_F32: launch_epi<TC_EPI_BIAS_F32>(ma, mb, g, s); break;
        case TC_EPI_MASK: launch_epi<TC_EPI_MASK>(ma, mb, g, s); break;
        default: launch_epi<TC_EPI_F32>(ma, mb, g, s); break;
    }
}

}  // namespace dos
