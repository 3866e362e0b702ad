// Internal declarations shared by the translation units of libdos.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dos.h"

namespace dos {

// ---- error plumbing ----------------------------------------------------------
struct Error {
    int status;
    std::string msg;
};

#define DOS_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            throw ::dos::Error{DOS_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
    } while (0)

#define DOS_REQUIRE(cond, msg)                                                          \
    do {                                                                                \
        if (!(cond)) throw ::dos::Error{DOS_EINVAL, (msg)};                             \
    } while (0)

// ---- device scratch owned by a context -----------------------------------------
struct Buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    void *get(size_t need) {  // grow-only
        if (need <= bytes) return ptr;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        size_t cap = need + need / 8 + 256;
        cudaError_t e = cudaMalloc(&ptr, cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{DOS_ENOMEM, "cudaMalloc of " + std::to_string(cap) + " bytes failed"};
        }
        bytes = cap;
        return ptr;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

struct PinnedBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    void *get(size_t need) {
        if (need <= bytes) return ptr;
        if (ptr) cudaFreeHost(ptr);
        ptr = nullptr;
        bytes = 0;
        if (cudaMallocHost(&ptr, need) != cudaSuccess) {
            cudaGetLastError();
            throw Error{DOS_ENOMEM, "cudaMallocHost failed"};
        }
        bytes = need;
        return ptr;
    }
    void release() {
        if (ptr) cudaFreeHost(ptr);
        ptr = nullptr;
        bytes = 0;
    }
};

// Launch shape of the fused step kernel.
struct Shape {
    int team = 0, chunks = 0, block = 0, tiles = 0;
    int staged = 0;  // 0 direct loads, 1 TMA-staged row panels (step_staged_kernel),
                     // 2 TMA gathers of the X_k rows (step_tmag_kernel),
                     // 3 direct loads with the tile's CSR staged (step_csrs_kernel)
    int cb = 16;     // bytes per chunk: 16, or 32 (direct loads, staged 0 or 3)
    int depth = 0;   // TMA gathers: batches in flight per team (2, 4, 8; 0: by shared memory)
    int panel = 0;   // vectors per pass over A (0: up to 256)
};

// Cached CUDA graph for one sweep configuration.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> key;      // configuration of `exec`
    std::vector<uint64_t> pending;  // configuration of the previous direct-launch call
    int64_t kernel_nodes = 0;
    cudaStream_t stream = nullptr;  // replay stream (ordered after the caller's by events)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

}  // namespace dos

struct dos_ctx {
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    // CSR staging (host-resident inputs, FP32 copies of FP64 values)
    dos::Buffer csr_rowptr, csr_colidx, csr_val, val_f32;
    // sweep scratch
    dos::Buffer xbuf, partial, dotsum, tiles, segs, status, mu_dev, mupv_dev;
    // bounds scratch
    dos::Buffer bnd_vec, bnd_part, bnd_out;
    // Lanczos DOS scratch
    dos::Buffer lz_buf;
    // Legendre (KPML / DGL) scratch: moments, conversion table, nodes and grids
    dos::Buffer leg_buf, leg_aux;
    // reconstruct / error scratch
    dos::Buffer rec_in, rec_out, err_buf;
    dos::PinnedBuffer host_stage;
    // autotuner cache: (rows, nnz, B, n_v, precision) -> shape
    std::map<std::tuple<int64_t, int64_t, int, int, int>, dos::Shape> tuned;
    dos::GraphCache graph;
    // profiling counters (dos_profile_enable / dos_profile_read)
    bool profiling = false;
    std::vector<cudaEvent_t> prof_events;  // two per vector panel
    double prof_step_ms = 0.0;
    int64_t prof_step_launches = 0, prof_sweeps = 0;
};

namespace dos {
// Count of kernel launches issued by the library (all contexts, this process).
extern std::atomic<int64_t> g_launch_count;
inline void count_launches(int64_t n) { g_launch_count.fetch_add(n, std::memory_order_relaxed); }
#define DOS_LAUNCHED()                       \
    do {                                     \
        ::dos::count_launches(1);            \
        DOS_CUDA_TRY(cudaGetLastError());    \
    } while (0)
}  // namespace dos

namespace dos {

// ---- kernels (launchers live in the .cu files) --------------------------------

// CSR structure check; sets *flag (device int) nonzero on failure.
void launch_validate_csr(int64_t n_rows, int64_t nnz, const int32_t *row_ptr,
                         const int32_t *col_idx, int B, const int32_t *seg_row0, int *flag,
                         cudaStream_t s);
void launch_f64_to_f32(const double *in, float *out, int64_t count, cudaStream_t s);

// Sweep plan: one tile per block; tiles never cross a segment (matrix) boundary.
// tiles[t] = {row_begin, row_end, segment, 0}; seg_tile_begin has B+1 entries.
void launch_make_tiles(const int32_t *row_ptr, int B, const int32_t *seg_row0,
                       const int32_t *seg_tile_begin, int n_tiles, int row_cost, int4 *tiles,
                       cudaStream_t s);

struct SweepArgs {
    int precision;  // DOS_PREC_*
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const void *val;  // double* (F64) or float* (F32)
    int64_t n_rows;   // total rows (all segments)
    int64_t nnz;      // nonzeros (all segments)
    int n_v, ld;      // vectors, padded row length of the vector blocks
    int B;            // segments
    const int32_t *seg_row0;  // device, B+1
    const double *seg_c;      // device, B
    const double *seg_inv_d;  // device, B
    const int4 *tiles;
    int n_tiles;
    void *x0, *x1;            // the two vector blocks (n_rows x ld each)
    double *partial;          // [steps_in_chunk][n_tiles][2][pv]
    double *partial0;         // [n_tiles][pv] for mu_0
    int per_vec;              // pv = ld if per_vec else 1
    uint64_t seed;
    int64_t vec_offset;
    uint64_t batch_index;     // counter field b for segment 0 (segment s uses b + s)
    Shape shape;
    int *status = nullptr;    // device flags: bit 1 spectrum, bit 2 wait timeout
    long long spin_cycles = 0;  // bounded-wait limit (0: about one second)
    int stall_test = 0;       // tests only: make the staged kernel's first wait run out
    int pdl = 1;              // programmatic dependent launch of the direct step kernel
};

// Occupancy-derived default shape for (precision, ld).
Shape default_shape(int precision, int ld, int num_sms, int64_t n_rows);
bool shape_supported(int precision, const Shape &sh, int ld);
int max_active_blocks(int precision, const Shape &sh, int ld);
// Ring depth of the TMA-gather kernel for this shape (asked: 0 = by shared memory).
int tmag_depth(int block, int team, int ld, int esz, int asked);

void launch_init_vectors(const SweepArgs &a, cudaStream_t s);
// Step k (0-based): reads x_cur = blocks[k%2], writes blocks[(k+1)%2]; partial slice `slot`.
void launch_step(const SweepArgs &a, int k, int slot, cudaStream_t s);
// Deterministic reduction over tiles of the step slices [k0, k0+count), stored at
// partial slots (slot0 + i) % slots, into dotsum[seg][k][2][dst_pv] (columns
// col_offset .. col_offset+ncols-1 when pv > 1; += when accumulate and pv == 1).
void launch_reduce(const double *partial, int n_tiles, int pv, int ncols, int B,
                   const int32_t *seg_tile_begin, int k0, int count, int slot0, int slots,
                   int steps_total, int col_offset, int dst_pv, int accumulate, double *dotsum,
                   cudaStream_t s);
void launch_reduce0(const double *part0, int pv, int ncols, int B, const int32_t *seg_tile_begin,
                    int col_offset, int dst_pv, int accumulate, double *dotsum0, cudaStream_t s);
// Moments from the reduced dot products; writes mu[seg][M+1] and optional per-vector
// moments mu_pv[(seg*n_v + l)*(M+1) + k]; sets bit 1 of *status on |mu_k| > mu_0 (1 + tol)
// or a non-finite moment.  pvt = n_v (per-vector dot sums) or 1 (totals).
void launch_finalize(const double *dotsum, const double *dotsum0, const int32_t *seg_row0, int B,
                     int M, int steps_total, int n_v, int pvt, double *mu, double *mu_pv,
                     double tol, int *status, cudaStream_t s);

// Bounds
void launch_gershgorin(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                       const void *val, int dtype, double *part, int n_blocks, cudaStream_t s);
void launch_minmax_final(const double *part, int n_blocks, double *out, cudaStream_t s);
// Per-segment Gershgorin min/max: out[2b] = lower, out[2b+1] = upper; keys: 2B scratch.
void launch_gershgorin_batched(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                               const void *val, int dtype, int B, const int32_t *seg_row0,
                               unsigned long long *keys, double *out, int num_sms,
                               cudaStream_t s);
int gershgorin_blocks(int num_sms);
void launch_lanczos_start(int64_t n, uint64_t seed, double *q, cudaStream_t s);
// w = A q - beta_prev * q_prev; partial dots q.w per block
void launch_lanczos_matvec(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                           const void *val, int dtype, const double *q, const double *q_prev,
                           const double *beta_prev, double *w, double *part, int n_blocks,
                           cudaStream_t s);
// out[idx] = sum of part (fixed order); optional sqrt
void launch_sum_final(const double *part, int n_blocks, double *out, int take_sqrt,
                      cudaStream_t s);
// w -= alpha q ; partial norms of w
void launch_lanczos_axpy(int64_t n, const double *alpha, const double *q, double *w,
                         double *part, int n_blocks, cudaStream_t s);
// q_prev <- q ; q <- w / beta  (beta > 0 checked on device: beta==0 -> leave q)
void launch_lanczos_next(int64_t n, const double *beta, double *q, double *q_prev,
                         const double *w, cudaStream_t s);
int reduce_blocks(int num_sms, int64_t n);

// Reconstruction and the error metric
// coef_scratch: M+1 doubles
void launch_reconstruct(const double *mu, int M, int damping, double lb, double ub,
                        const double *t, int N_t, double *coef_scratch, double *phi_hat,
                        double *phi_lambda, cudaStream_t s);
// The learned network's tensor-core product (mlp_tc.cu): C = epilogue(A B^T) with
// A (M x K) and B (N x K) bfloat16, K contiguous, leading dimensions multiples of 8.
enum TcEpi { TC_EPI_BIAS_RELU_BF16 = 0, TC_EPI_BIAS_F32 = 1, TC_EPI_MASK = 2, TC_EPI_F32 = 3 };
struct TcGemm {
    int M, N, K, epi;
    const float *bias;   // N: TC_EPI_BIAS_RELU_BF16 (relu(acc + b) in bf16), TC_EPI_BIAS_F32
    const void *mask;    // bf16 M x N (ld ldm): TC_EPI_MASK keeps acc where mask > 0
    int ldm;
    float *Cf;           // FP32 output (ld ldc): TC_EPI_BIAS_F32, TC_EPI_MASK, TC_EPI_F32
    void *Cb;            // bf16 output (ld ldc) or null
    int ldc;
    void *Ct;            // bf16 transposed output, N x M (ld ldt), or null
    int ldt;
    int *status;         // bit 8: a bounded wait ran out
    long long spin;      // wait limit in SM clock cycles
};
void launch_gemm_tc(const TcGemm &g, const void *A, int lda, const void *B, int ldb,
                    cudaStream_t s);

// B rows of moments (row stride ldm) -> B x N_t phi_hat; coef_scratch: B (M+1) doubles
void launch_reconstruct_rows(const double *mu, int64_t ldm, int B, int M, int damping,
                             const double *t, int N_t, double *coef_scratch, double *phi_hat,
                             cudaStream_t s);
void launch_blur_kpm(const double *mu, int M, int damping, double lb, double ub, double sigma,
                     int N_q, double x0, double h, int N_x, double *poly_scratch, double *out,
                     cudaStream_t s);
void launch_blur_eigs(const double *eig, int64_t n_eig, double sigma, double x0, double h,
                      int N_x, double *out, cudaStream_t s);
void launch_error_norms(const double *a, const double *b, int N_x, double h, double *out,
                        cudaStream_t s);
void launch_grid_moments(const double *phi, int N, int M, double *mu, cudaStream_t s);
void launch_heat_kpm(const double *mu, int M, int damping, double lb, double ub, int N_q,
                     const double *betas, int n_beta, double *scratch, double *out,
                     cudaStream_t s);
void launch_heat_points(const double *pts, const double *w, int64_t n_pts, double scale,
                        const double *betas, int n_beta, double *out, cudaStream_t s);

// KPML / DGL (FP64).  h_scratch: M+1 doubles.
void launch_cheb_to_legendre(const double *mu, int64_t count, int M, double *h_scratch,
                             double *nu, cudaStream_t s);
// out_t[i] = phi_L(t_i) (times w[i] when w is given; t NULL: Chebyshev nodes),
// out_l[i] = phi_L(t_i) * inv_d when out_l is given.  coef_scratch: 2 (M+1) doubles.
void launch_kpml(const double *nu, int M, const double *t, const double *w, int N, double inv_d,
                 double *out_t, double *out_l, double *coef_scratch, cudaStream_t s);
// Gauss-Legendre nodes t (ascending), weights w, positions y = c + d t (y may be NULL).
// coef_scratch: 2 (N+1) doubles.
void launch_gauss_legendre(int N, double c, double d, double *t, double *w, double *y,
                           double *coef_scratch, cudaStream_t s);
// DGL density at x[i] (or x0 + i h when x is NULL); used may be NULL.
void launch_dgl(const double *nu, int M, double c, double d, double sigma, double tol,
                const double *x, double x0, double h, int N, double *phi, int *used,
                cudaStream_t s);

// Lanczos DOS (block of n_vec independent runs, FP64)
// Block product with the fused step's team mapping (kpm_kernels.cu): w = A q -
// beta_prev q_prev over q_prev, per-block alpha partials [n_blocks][ld].
int lanczos_team_blocks(int num_sms, int64_t n, int ld);
// W = A u_j - c_j u_{j-1} over u_{j-1} (c_prev: c_j per column, NULL: no previous
// term); part gets the partial sums of u_j . W
void launch_lanczos_team_spmm(int64_t n, int ld, const int32_t *row_ptr, const int32_t *col_idx,
                              const double *val, const double *q, double *qprev_w,
                              const double *c_prev, double *part, int n_blocks,
                              cudaStream_t s);
int lanczos_blocks(int num_sms, int64_t n, int ld);
void launch_lanczos_block_axpy(int64_t n, int ld, int n_vec, const double *alpha,
                               const double *t_fac, const double *q, double *w, double *part,
                               int n_blocks, cudaStream_t s);
void launch_lanczos_alpha(const double *part, int n_blocks, int ld, const double *s_fac,
                          double *alpha, cudaStream_t s);
void launch_lanczos_beta(const double *part, int n_blocks, int ld, const double *s_fac,
                         const double *beta_prev, double *beta, double *s_next, double *c_next,
                         double *t_next, cudaStream_t s);
void launch_unit_scale(int64_t n, int ld, int n_vec, double *q, int num_sms, cudaStream_t s);
// w <- w / sum(w) on the device; sum_out[0] receives the sum.
void launch_normalize_weights(double *w, int64_t n, double *sum_out, cudaStream_t s);
// m_used[l]: steps run l keeps (invariant-subspace rule), -1 for non-finite values.
void launch_lanczos_steps(const double *alpha, const double *beta, int M, int ld, int n_vec,
                          int *m_used, cudaStream_t s);
// Extreme-Ritz-value bounds of a k-step Lanczos run: out = {lo, hi, steps kept};
// work: 3 k doubles.
void launch_lanczos_bounds(const double *alpha, const double *beta, int k, double *work,
                           double *out, cudaStream_t s);
// work: 3 * n_vec * M doubles
void launch_tridiag_ritz(const double *alpha, const double *beta, const int *m_used, int M, int ld,
                         int n_vec, double *theta, double *weight, cudaStream_t s);
void launch_weighted_gauss(const double *pts, const double *w, int64_t n_pts, double scale,
                           double sigma, const double *x, double x0, double h, int N_x,
                           double *out, cudaStream_t s);
void launch_weighted_lorentz(const double *pts, const double *w, int64_t n_pts, double scale,
                             double eta, const double *x, int N_x, double *out, cudaStream_t s);

}  // namespace dos
