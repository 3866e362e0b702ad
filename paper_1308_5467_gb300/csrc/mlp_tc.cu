// Dense products of the learned network on the fifth-generation tensor cores.
//
//   C = epilogue(A B^T),  A: M x K and B: N x K bfloat16, row-major with K
//   contiguous (leading dimensions multiples of 8 elements), FP32 accumulation.
//
// Persistent, warp-specialised kernel: one CTA of ten warps per SM walks the
// 128 x 128 output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (row-block
// major, so CTAs running together share the A rows of a row block in L2):
//   * warp 0 (one thread) streams K-slices of 64 elements (128 bytes of a row) of
//     A and B into a ring of four shared-memory stages with TMA
//     (cp.async.bulk.tensor, 128-byte swizzle, rows past M, N or K filled with
//     zeros), each completing on the stage's "full" mbarrier;
//   * warp 1 (one thread) issues tcgen05.mma (kind::f16: BF16 operands, FP32
//     accumulator in tensor memory, M = N = 128, K = 16 per instruction, four per
//     slice) and tcgen05.commit to the stage's "empty" mbarrier, which frees the
//     stage when its MMAs are done; two accumulators (2 x 128 tensor-memory
//     columns) alternate between tiles, and a commit to the accumulator's "full"
//     mbarrier hands a finished tile to the epilogue;
//   * warps 2-9 read the accumulator with tcgen05.ld (warp w reaches tensor-memory
//     lanes 32 (w mod 4) .. +31, the tile's rows, and takes half of the columns),
//     apply the epilogue and store each thread's 32 consecutive columns with
//     16-byte vector stores (the transposed bf16 copy column by column,
//     consecutive lanes on consecutive rows), then release the accumulator on its
//     "empty" mbarrier -- so one tile's epilogue overlaps the next tile's loads
//     and products.
// Every mbarrier wait is bounded (spin cycles) and also gives up when another
// role has: a wait that runs out sets status bit 8 and an abort flag that ends
// every role's loop; the CTA then waits (bounded again) for the copies and
// products it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "dos_internal.h"

namespace dos {
namespace {

typedef __nv_bfloat16 bf16;

// Four stages of operands (128 KB of shared memory): one CTA per SM (six stages
// measured the same).  Eight epilogue warps: two per tensor-memory lane quadrant,
// each taking half the columns.
constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 4, kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTileBytes = kBM * kBK * 2;     // one operand slice: 128 rows x 128 B
constexpr uint32_t kStageBytes = 2 * kTileBytes;   // A and B (kBN == kBM)
constexpr uint32_t kTmemCols = 2 * kBN;            // two FP32 accumulators, one column per n
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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
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

// Bounded wait that also gives up once another role has set the abort flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity,
                                                   long long limit, volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
__device__ __forceinline__ void fail(volatile int *abort, int *status) {
    *abort = 1;
    atomicOr(status, 8);
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Epilogue of one thread: row `row` (< M), the 32 columns c0 .. c0+31 (those < N)
// of the accumulator in v.
template <int EPI>
__device__ __forceinline__ void epilogue_row(const TcGemm &g, int row, int c0, float (&v)[32]) {
    const int ncol = min(32, g.N - c0);
    const bool full = ncol == 32;
    if (EPI == TC_EPI_BIAS_RELU_BF16 || EPI == TC_EPI_BIAS_F32) {
        float b[32];
        if (full && (((uintptr_t)(g.bias + c0) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(g.bias + c0) + q);
                b[4 * q] = b4.x;
                b[4 * q + 1] = b4.y;
                b[4 * q + 2] = b4.z;
                b[4 * q + 3] = b4.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) b[j] = j < ncol ? __ldg(g.bias + c0 + j) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
            v[j] = EPI == TC_EPI_BIAS_RELU_BF16 ? fmaxf(v[j] + b[j], 0.f) : v[j] + b[j];
    } else if (EPI == TC_EPI_MASK) {
        const bf16 *mrow = (const bf16 *)g.mask + (size_t)row * g.ldm + c0;
        if (full && ((g.ldm & 7) == 0) && (((uintptr_t)g.mask & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 m = __ldg(reinterpret_cast<const uint4 *>(mrow) + q);
                const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162 *>(&w[h]);
                    if (!(__low2float(p2) > 0.f)) v[q * 8 + 2 * h] = 0.f;
                    if (!(__high2float(p2) > 0.f)) v[q * 8 + 2 * h + 1] = 0.f;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < ncol && !(__bfloat162float(mrow[j]) > 0.f)) v[j] = 0.f;
        }
    }
    const size_t o = (size_t)row * g.ldc + c0;
    // FP32 output
    if (EPI != TC_EPI_BIAS_RELU_BF16) {
        float *dst = g.Cf + o;
        if (full && ((g.ldc & 3) == 0) && (((uintptr_t)g.Cf & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                reinterpret_cast<float4 *>(dst)[q] =
                    make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < ncol) dst[j] = v[j];
        }
    }
    // bf16 output (always for BIAS_RELU_BF16; for MASK when Cb is given)
    if (EPI == TC_EPI_BIAS_RELU_BF16 || (EPI == TC_EPI_MASK && g.Cb)) {
        bf16 *dst = (bf16 *)g.Cb + o;
        if (full && ((g.ldc & 7) == 0) && (((uintptr_t)g.Cb & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                reinterpret_cast<uint4 *>(dst)[q] = make_uint4(
                    pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                    pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < ncol) dst[j] = __float2bfloat16_rn(v[j]);
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap map_a,
                   const __grid_constant__ CUtensorMap map_b, const TcGemm g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ volatile int s_abort;
    __shared__ int s_issued, s_consumed;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + (size_t)kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;   // 2: accumulator b holds a finished tile
    uint64_t *acc_empty = acc_full + 2;     // 2: the epilogue has read accumulator b
    uint64_t *drain = acc_empty + 2;        // every MMA issued has completed
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + kBK - 1) / kBK;
    const int tiles_n = (g.N + kBN - 1) / kBN;
    const int n_tiles = ((g.M + kBM - 1) / kBM) * tiles_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);   // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: TMA loads of A and B slices into the stage ring ----
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < n_tiles && !s_abort; t += gridDim.x) {
                const int m0 = (t / tiles_n) * kBM, n0 = (t % tiles_n) * kBN;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kStages;
                    if (!mbar_wait_or_abort(&empty[s], ((it / kStages) & 1) ^ 1, g.spin, &s_abort)) {
                        if (!s_abort) fail(&s_abort, g.status);
                        break;
                    }
                    uint8_t *sa = smem + (size_t)s * kStageBytes;
                    mbar_expect_tx(&full[s], kStageBytes);
                    tma_load_2d(sa, &map_a, kc * kBK, m0, &full[s]);
                    tma_load_2d(sa + kTileBytes, &map_b, kc * kBK, n0, &full[s]);
                    s_issued = it + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer: products of each tile into accumulator (tile count & 1) ----
        if (lane == 0) {
            int it = 0, tc = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < n_tiles && ok && !s_abort; t += gridDim.x, ++tc) {
                const int b = tc & 1;
                if (!mbar_wait_or_abort(&acc_empty[b], ((tc >> 1) & 1) ^ 1, g.spin, &s_abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kBN);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % kStages;
                    if (!mbar_wait_or_abort(&full[s], (it / kStages) & 1, g.spin, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    s_consumed = it + 1;
                    const uint32_t sa = saddr(smem + (size_t)s * kStageBytes), sb = sa + kTileBytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)
                        mma_bf16(d, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32),
                                 (kc | kk) != 0 ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[b]);
            }
            if (!ok && !s_abort) fail(&s_abort, g.status);
            mma_commit(drain);  // fires once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---- epilogue: warps 2-9; warp w reads accumulator lanes 32 (w % 4) .. +31
        // (tcgen05.ld reaches only its own quadrant) and column chunks 2h, 2h + 1 of
        // the four, h = (w - 2) / 4 ----
        const int quad = warp & 3, half = (warp - 2) >> 2;
        int tc = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tc) {
            const int b = tc & 1;
            const bool got = mbar_wait_or_abort(&acc_full[b], (tc >> 1) & 1, g.spin, &s_abort);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0 && !s_abort) fail(&s_abort, g.status);
                break;
            }
            tc_fence_after();
            const int m0 = (t / tiles_n) * kBM, n0 = (t % tiles_n) * kBN;
            const int row = m0 + quad * 32 + lane;
#pragma unroll 1
            for (int c = 2 * half; c < 2 * half + 2; ++c) {
                const int c0 = n0 + c * 32;
                if (c0 >= g.N) break;  // warp-uniform
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * kBN + c * 32), v);
                if (row < g.M) {
                    epilogue_row<EPI>(g, row, c0, v);
                    if (g.Ct) {  // transposed bf16 copy: lanes write consecutive rows
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c0 + j < g.N)
                                ((bf16 *)g.Ct)[(size_t)(c0 + j) * g.ldt + row] =
                                    __float2bfloat16_rn(v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }

    __syncthreads();
    // Teardown: wait (bounded) for the products and copies this CTA issued, then
    // free the tensor memory.
    if (threadIdx.x == 32) {
        if (!mbar_wait(drain, 0, g.spin)) {
            if (!mbar_wait(drain, 0, g.spin)) atomicOr(g.status, 8);
        }
    }
    if (threadIdx.x == 0 && s_abort) {
        for (int it = s_consumed; it < s_issued; ++it)  // loads still writing shared memory
            mbar_wait(&full[it % kStages], (it / kStages) & 1, g.spin);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
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
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        DOS_CUDA_TRY(cudaGetDevice(&dev));
        DOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int64_t tiles = (int64_t)((g.N + kBN - 1) / kBN) * ((g.M + kBM - 1) / kBM);
    const int grid = (int)std::min<int64_t>(tiles, sms);
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
