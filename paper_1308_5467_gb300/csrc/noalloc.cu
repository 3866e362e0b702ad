// dos_kpm_moments_noalloc: the moment sweep for callers that cannot allocate
// device memory.  Some callers must not call cudaMalloc while they run:
// applications whose device memory is reserved up front by their own pool
// allocator (a framework's caching allocator holds nearly all of it, so a
// library's cudaMalloc fails or evicts the pool's cache), and services with a
// fixed memory budget or latency target, where cudaMalloc/cudaFree may
// synchronise the device and stall unrelated work.  This entry point takes the
// caller's inputs and output and keeps every intermediate (the two vector
// blocks, tiles, partial sums, status) in one file-scope device array of fixed
// size instead.  The paper has no counterpart; it is deployment plumbing
// around the same kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dos_internal.h"

namespace {

// 64 MiB: the first MiB holds the control data, the rest the two vector blocks.
constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr size_t kControlBytes = size_t(1) << 20;
constexpr int kMaxTiles = 2048;
constexpr int kSlots = 16;       // partial-sum slices reduced every kSlots steps
constexpr int kMaxSteps = 10000; // M <= 20000
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once with that device current.
std::atomic<void *> g_scratch_addr[kMaxDevices];

__global__ void noalloc_setup_kernel(int32_t *row0, int32_t *tile_begin, double *seg_c,
                                     double *seg_inv_d, int *status, int n, int tiles, double c,
                                     double inv_d) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        row0[0] = 0;
        row0[1] = n;
        tile_begin[0] = 0;
        tile_begin[1] = tiles;
        seg_c[0] = c;
        seg_inv_d[0] = inv_d;
        status[0] = 0;
        status[1] = 0;
    }
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int dos_kpm_moments_noalloc(const dos_csr *A, double lb, double ub, int M, int n_v,
                                       uint64_t seed, int precision, double *mu, void *stream) {
    using namespace dos;
    if (!A || !mu) return DOS_EINVAL;
    if (A->location != DOS_DEVICE || A->n < 1 || A->n >= (int64_t(1) << 31) || A->nnz < 0 ||
        A->nnz >= (int64_t(1) << 31) || !A->row_ptr || (A->nnz && (!A->col_idx || !A->val)))
        return DOS_EINVAL;
    if (!(isfinite(lb) && isfinite(ub) && ub > lb) || M < 0 || n_v < 1 || n_v > 256)
        return DOS_EINVAL;
    if (precision == DOS_PREC_F64 ? A->dtype != DOS_F64
                                  : (precision != DOS_PREC_F32_ACC64 || A->dtype != DOS_F32))
        return DOS_EINVAL;
    // size limits of the fixed scratch
    const int vpt = precision == DOS_PREC_F64 ? 2 : 4;
    const int esz = precision == DOS_PREC_F64 ? 8 : 4;
    const int ld = (n_v + vpt - 1) / vpt * vpt;
    const int S = M < 2 ? 1 : (M + 1) / 2;
    if (S > kMaxSteps) return DOS_ENOMEM;
    if (2 * (size_t)A->n * ld * esz > kScratchBytes - kControlBytes) return DOS_ENOMEM;
    // every array the kernels read or write must be device memory: a host
    // address handed to a kernel would fault instead of returning an error
    if (!on_device(mu) || !on_device(A->row_ptr)) return DOS_EINVAL;
    if (A->nnz && (!on_device(A->col_idx) || !on_device(A->val))) return DOS_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DOS_ECUDA;
    }
    // One-time set-up on this device: the host-side name g_scratch is only a
    // stand-in; the kernels need its device address.
    void *base = g_scratch_addr[dev].load();
    if (!base) {
        if (cudaGetSymbolAddress(&base, g_scratch) != cudaSuccess || !base) {
            cudaGetLastError();
            return DOS_ECUDA;
        }
        g_scratch_addr[dev].store(base);
    }
    cudaStream_t s = (cudaStream_t)stream;
    try {
        int dev_sms = 0;
        DOS_CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev));
        Shape sh = default_shape(precision, ld, dev_sms, A->n);
        if (sh.tiles > kMaxTiles) sh.tiles = kMaxTiles;
        const int T = sh.tiles;
        // control region layout
        uint8_t *p = (uint8_t *)base;
        int32_t *row0 = (int32_t *)p;            // 2
        int32_t *tile_begin = row0 + 2;          // 2
        int *status = (int *)(row0 + 4);         // 4
        double *seg_c = (double *)(p + 64);
        double *seg_inv_d = seg_c + 1;
        int4 *tiles = (int4 *)(p + 256);                             // T * 16 B
        double *partial = (double *)(p + 256 + kMaxTiles * 16);      // kSlots * T * 2
        double *partial0 = partial + (size_t)kSlots * kMaxTiles * 2; // T
        double *dotsum = partial0 + kMaxTiles;                       // S * 2
        double *dotsum0 = dotsum + 2 * (size_t)kMaxSteps;            // 1
        uint8_t *xb = p + kControlBytes;
        const double c = 0.5 * (lb + ub), inv_d = 1.0 / (0.5 * (ub - lb));
        noalloc_setup_kernel<<<1, 32, 0, s>>>(row0, tile_begin, seg_c, seg_inv_d, status,
                                             (int)A->n, T, c, inv_d);
        DOS_LAUNCHED();
        // structure check before any kernel reads through the indices
        launch_validate_csr(A->n, A->nnz, A->row_ptr, A->col_idx, 1, row0, status + 1, s);
        int bad = 0;
        DOS_CUDA_TRY(cudaMemcpyAsync(&bad, status + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (bad) return DOS_EINVAL;
        launch_make_tiles(A->row_ptr, 1, row0, tile_begin, T, 3, tiles, s);
        SweepArgs a{};
        a.precision = precision;
        a.row_ptr = A->row_ptr;
        a.col_idx = A->col_idx;
        a.val = A->val;
        a.n_rows = A->n;
        a.nnz = A->nnz;
        a.n_v = n_v;
        a.ld = ld;
        a.B = 1;
        a.seg_row0 = row0;
        a.seg_c = seg_c;
        a.seg_inv_d = seg_inv_d;
        a.tiles = tiles;
        a.n_tiles = T;
        a.x0 = xb;
        a.x1 = xb + (size_t)A->n * ld * esz;
        a.partial = partial;
        a.partial0 = partial0;
        a.per_vec = 0;
        a.seed = seed;
        a.vec_offset = 0;
        a.batch_index = 0;
        a.shape = sh;
        a.status = status;
        launch_init_vectors(a, s);
        int k0 = 0;
        for (int k = 0; k < S; ++k) {
            launch_step(a, k, k % kSlots, s);
            if ((k + 1) % kSlots == 0 || k == S - 1) {
                launch_reduce(partial, T, 1, 1, 1, tile_begin, k0, k + 1 - k0, k0 % kSlots,
                              kSlots, S, 0, 1, 0, dotsum, s);
                k0 = k + 1;
            }
        }
        launch_reduce0(partial0, 1, 1, 1, tile_begin, 0, 1, 0, dotsum0, s);
        launch_finalize(dotsum, dotsum0, row0, 1, M, S, n_v, 1, mu, nullptr,
                        precision == DOS_PREC_F64 ? 1e-8 : 1e-3, status, s);
        int h = 0;
        DOS_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (h & 2) return DOS_ESPECTRUM;
    } catch (const Error &e) {
        return e.status;
    }
    return DOS_OK;
}
