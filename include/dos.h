/*
 * dos.h -- C ABI of libdos, a GB300 (sm_103a) library for the Kernel
 * Polynomial Method (KPM) estimate of the density of states (DOS) of a large
 * sparse real symmetric matrix, after Lin, Saad and Yang, "Approximating
 * spectral densities of large matrices" (SIAM Review 58(1), 2016;
 * arXiv:1308.5467).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: DOS_OK (0) or one of the DOS_E*
 *    codes below.  dos_last_error(ctx) gives a one-line message for the last
 *    failure on that context.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is queued on it; the functions that return results in host
 *    memory, or that must check a device-side status, synchronise the stream
 *    before returning (each function says which).
 *  - Buffers are owned by the caller; the library never frees caller memory.
 *    Scratch (vector blocks, partial sums, staging copies) is owned by the
 *    context, allocated on first use and grown on demand; a context is not
 *    thread-safe: use one context per host thread.
 *  - Output arrays documented as "host or device" may be either: the library
 *    asks the CUDA runtime which kind of memory the pointer refers to.
 *  - Matrices are CSR with int32 row pointers and column indices (so nnz <
 *    2^31), column indices sorted or not, FP64 or FP32 values.  A matrix must
 *    be symmetric for the method to make sense; symmetry is not checked.
 *    Structural validity (row_ptr[0] = 0, row_ptr non-decreasing,
 *    row_ptr[n] = nnz, 0 <= col_idx < n) IS checked on the device before any
 *    kernel reads through the indices; a failure returns DOS_EINVAL.
 *  - Start vectors (Theorem 3.1: E[v] = 0, E[v v^T] = I) are Rademacher +-1
 *    entries.  Entry (row i, vector l) of matrix b is bit (l mod 64) of the
 *    64-bit splitmix64 output number ctr+1 of the stream seeded with `seed`,
 *    ctr = b*2^48 + floor(l/64)*2^32 + i  (0 -> +1, 1 -> -1).  Results are
 *    therefore reproducible for a given (seed, matrix, n_v).
 */
#ifndef DOS_H
#define DOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define DOS_OK 0
#define DOS_EINVAL 1     /* bad argument, or a CSR that fails validation */
#define DOS_ENOMEM 2     /* device or host allocation failed */
#define DOS_ECUDA 3      /* a CUDA runtime call failed (message in dos_last_error) */
#define DOS_ESPECTRUM 4  /* |mu_k| > mu_0 (1 + tol) or a non-finite moment: the
                            bounds did not enclose the spectrum (Section 3.1:
                            T_k(B) v_0 then grows exponentially) */
#define DOS_ETIMEOUT 5   /* a bounded device-side wait ran out */
#define DOS_EIO 6        /* a file could not be opened, read or written, or is not
                            a file of the expected format (dos_mlp_save / load) */

/* ---- enumerations ---------------------------------------------------------- */
#define DOS_F64 0               /* value / vector element type */
#define DOS_F32 1

#define DOS_DEVICE 0            /* where a dos_csr's arrays live */
#define DOS_HOST 1

#define DOS_PREC_F64 0          /* values, vectors, products and dot products in FP64 */
#define DOS_PREC_F32_ACC64 1    /* values, vectors and the recurrence in FP32; each
                                   moment dot product formed from exact FP32 products,
                                   accumulated per thread as an unevaluated float pair
                                   (about 2^-48 relative) and summed across threads and
                                   blocks, and stored, in FP64 */

#define DOS_BOUNDS_GERSHGORIN 0 /* disc bound, one pass over the matrix */
#define DOS_BOUNDS_LANCZOS 1    /* k-step Lanczos with residual bounds (Section 3.1) */

#define DOS_DAMP_NONE 0         /* plain truncated expansion, Eq. tdosFinal */
#define DOS_DAMP_JACKSON 1      /* Jackson damping factors, Appendix A Eq. jackson */

/* flags of dos_kpm_opts.flags */
#define DOS_OPT_NO_VALIDATE 1u      /* skip the CSR structure check (caller vouches) */
#define DOS_OPT_NO_SPECTRUM_CHECK 2u/* do not synchronise to check |mu_k| <= mu_0 */
#define DOS_OPT_NO_GRAPH 4u         /* launch the sweep kernel by kernel instead of
                                       replaying a cached CUDA graph */
#define DOS_OPT_AUTOTUNE 8u         /* time the candidate launch shapes on this matrix
                                       once and cache the fastest (see dos_tune) */
#define DOS_OPT_TEST_STALL_WAIT 16u /* failure-detection tests only: the TMA kernels'
                                       waits can never complete and must run out
                                       (staged 2 and 4 expect 16 bytes more than they
                                       copy; staged 3 arms its barrier without issuing
                                       the gather) */
#define DOS_OPT_NO_PDL 32u          /* launch consecutive sweep steps with plain stream
                                       order instead of programmatic dependent launch
                                       (the next step's blocks are scheduled while the
                                       current one drains and wait on the device for its
                                       completion before touching memory) */

typedef struct dos_ctx dos_ctx;

/* A CSR matrix descriptor.  `location` says whether the three arrays are in
 * device memory (used in place) or host memory (copied to context-owned device
 * memory inside the call, on `stream`). */
typedef struct {
    int64_t n;               /* rows = columns, >= 1 */
    int64_t nnz;             /* nonzeros, < 2^31 */
    const int32_t *row_ptr;  /* n + 1 entries */
    const int32_t *col_idx;  /* nnz entries */
    const void *val;         /* nnz entries of type `dtype` */
    int32_t dtype;           /* DOS_F64 or DOS_F32 */
    int32_t location;        /* DOS_DEVICE or DOS_HOST */
} dos_csr;

/* Launch shape of the fused sweep kernel.  Zero fields mean "choose". */
typedef struct {
    int32_t team;            /* threads that share one matrix row (1..32, power of 2) */
    int32_t chunks;          /* vector chunks per thread (1, 2 or 4) */
    int32_t block;           /* threads per block (64..1024, multiple of 32) */
    int32_t tiles;           /* row tiles = blocks per sweep step */
    int32_t staged;          /* 1: rows of X_k / X_{k-1} loaded by the threads;
                                2: row panels of X_k and X_{k-1} staged in shared memory
                                by bulk asynchronous (TMA) copies;
                                3: the gathered rows X_k[j] of each four nonzeros loaded
                                by one TMA gather (tile::gather4) into shared memory;
                                4: as 1, with each row tile's CSR slice (row_ptr,
                                column indices, values) staged in shared memory by bulk
                                asynchronous copies first; needs col_idx and val
                                16-byte aligned (0: choose) */
    int32_t chunk_bytes;     /* bytes per chunk: 16, or 32 (256-bit loads and stores;
                                with staged 1 or 4 only, and rows of whole 32-byte
                                chunks)
                                (0: 16, or the autotuned choice) */
    int32_t depth;           /* staged 3 only: batches of four gathers each team keeps in
                                flight (2, 4 or 8); 0: the deepest of 8, 4, 2 whose
                                stages leave room for two blocks per SM */
    int32_t panel;           /* vectors per pass over A, 0..4096: the n_v vectors are
                                swept in ceil(n_v / w) consecutive passes of at most
                                w = min(panel, 256) vectors (equal widths, the last
                                possibly narrower), each pass reading A once; the two
                                vector blocks take 2 n w' s bytes of device memory
                                (w' = the pass width rounded up to 16 bytes of the
                                element size s), so narrower passes fit larger n.
                                The moments do not depend on it beyond the rounding
                                of their FP64 sums.  0: w = 256 (the autotuner keeps
                                0: narrower passes measured slower) */
} dos_launch;

/* Optional arguments of the _ex / _batched entry points (NULL = defaults). */
typedef struct {
    uint32_t flags;          /* DOS_OPT_* */
    int64_t vec_offset;      /* first start-vector index l (default 0): a run with
                                vec_offset = o and n_v = k computes exactly vectors
                                o..o+k-1 of a larger run, so runs can be sharded */
    uint64_t batch_index;    /* matrix index b used by the start-vector counter
                                (single-matrix calls; default 0) */
    dos_launch launch;       /* launch shape override (zeros = autotuned/default) */
    int64_t wait_limit_cycles; /* limit of each device-side wait of the staged kernel, in
                                SM clock cycles (0 = about one second); a wait that runs
                                out makes the call return DOS_ETIMEOUT */
} dos_kpm_opts;

/* ---- context --------------------------------------------------------------- */

/* Create a context bound to CUDA device `device`; it owns all scratch memory.
 * Errors: DOS_EINVAL (ctx NULL or no such device), DOS_ENOMEM, DOS_ECUDA. */
int dos_ctx_create(dos_ctx **ctx, int device);

/* Free the context and all scratch memory it owns (synchronises the device).
 * NULL is accepted. */
int dos_ctx_destroy(dos_ctx *ctx);

/* Message for the last failure on `ctx` (never NULL; "" if none). */
const char *dos_last_error(const dos_ctx *ctx);

/* Short name of a status code ("DOS_OK", "DOS_EINVAL", ...). */
const char *dos_status_string(int status);

/* Kernel timing.  While enabled, every sweep records CUDA events on its stream
 * just before its first and just after its last fused-step launch (per vector
 * panel) and adds the elapsed time and the number of step launches to the
 * context's counters; each sweep then synchronises its stream at the end.
 * dos_lanczos_ritz counts the same way around each of its block-SpMM launches
 * (its dominant kernel), as one "sweep" of M step launches.
 * dos_profile_enable resets the counters.  The paper has no counterpart: this
 * is measurement plumbing. */
int dos_profile_enable(dos_ctx *ctx, int on);
/* step_ms: summed event time over the step launches; step_launches: how many;
 * sweeps: how many sweeps contributed; launches: all kernel launches issued by
 * the library since enabling.  Any pointer may be NULL. */
int dos_profile_read(dos_ctx *ctx, double *step_ms, int64_t *step_launches, int64_t *sweeps,
                     int64_t *launches);

/* Check a CSR's structure on the device (see the conventions above); returns
 * DOS_OK or DOS_EINVAL.  Synchronises `stream`. */
int dos_validate_csr(dos_ctx *ctx, const dos_csr *A, void *stream);

/* ---- step a2: start vectors ------------------------------------------------ */
/*
 * Write the n x n_v block of Rademacher start vectors that dos_kpm_moments
 * uses (Theorem 3.1's E[v] = 0, E[v v^T] = I; Algorithm 1 "select a new random
 * vector"), row-major out[i*n_v + l] = entry (row i, vector vec_offset + l) of
 * matrix batch_index, as +1/-1 in `dtype` (DOS_F64 or DOS_F32).  out: host or
 * device.  Synchronises `stream` when out is host memory.
 * Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_start_vectors(dos_ctx *ctx, int64_t n, int n_v, uint64_t seed, uint64_t batch_index,
                      int64_t vec_offset, int dtype, void *out, void *stream);

/* ---- step a1: spectrum bounds ---------------------------------------------- */
/*
 * Lower and upper bounds lb <= lambda_min(A), ub >= lambda_max(A) for the
 * shift/scale of Eq. cd (Section 3.1), each widened by pad_frac * (ub - lb).
 *   method DOS_BOUNDS_GERSHGORIN: min/max over rows of a_ii -+ sum_{j!=i}|a_ij|
 *          (`steps`, `seed` unused).
 *   method DOS_BOUNDS_LANCZOS: `steps`-step Lanczos (1 <= steps <= 512, stops
 *          early at an invariant subspace) from the normalised start vector
 *          l = 0 of `seed`; lb = theta_min - ||f|| |y_min(last)|,
 *          ub = theta_max + ||f|| |y_max(last)| with f the Lanczos residual and
 *          y the unit Ritz vectors of the tridiagonal T_k (Eq. lanfact).  The
 *          paper notes this is a heuristic (not a guaranteed enclosure), hence
 *          the pad.  Runs in FP64 whatever the value dtype.
 * lb, ub: host pointers.  Synchronises `stream`.
 * Errors: DOS_EINVAL (bad args/CSR), DOS_ENOMEM, DOS_ECUDA.
 */
int dos_bounds(dos_ctx *ctx, const dos_csr *A, int method, int steps, uint64_t seed,
               double pad_frac, double *lb, double *ub, void *stream);

/*
 * Gershgorin bounds of B matrices concatenated as in dos_kpm_moments_batched
 * (one pass over all rows, one launch): lb[b], ub[b] (host arrays of B) are
 * min/max over the rows of matrix b of a_ii -+ sum_{j!=i}|a_ij|, widened by
 * pad_frac * (ub - lb) (a matrix with a single eigenvalue gets +-0.5).
 * Synchronises `stream`.  Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_bounds_batched(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows,
                       double pad_frac, double *lb, double *ub, void *stream);

/* ---- steps a2-a5: the Chebyshev moment sweep ------------------------------- */
/*
 * Stochastic Chebyshev moments of B = (A - cI)/d, c = (lb+ub)/2, d = (ub-lb)/2
 * (Eq. cd), for k = 0..M:
 *     mu_k = (1/(n n_v)) sum_{l=0}^{n_v-1} v_l^T T_k(B) v_l
 * (Eqs. expmu, nuk, muEst without the factor (2 - delta_k0)/pi, which
 * dos_reconstruct applies; so mu_0 = 1).  The recurrence v_{k+1} = 2 B v_k -
 * v_{k-1}, v_1 = B v_0 (Eq. 3term, Algorithm 1) runs on all n_v vectors at
 * once as a block SpMM, fused in one pass over A with the shift/scale and with
 * the dot products of the doubling identity (Appendix A, sign corrected):
 *     mu_{2k}   = 2 v_k^T v_k / n     - mu_0,
 *     mu_{2k+1} = 2 v_{k+1}^T v_k / n - mu_1,
 * so ceil(M/2) passes over A give all M+1 moments.
 *   M: degree, 0 <= M <= 100000.  n_v: vectors, 1 <= n_v <= 4096.
 *   precision: DOS_PREC_F64 (needs A->dtype == DOS_F64) or DOS_PREC_F32_ACC64
 *      (an FP64 matrix is rounded to FP32 on the device first).
 *   mu: M+1 doubles, host or device.
 *   mu_per_vec: NULL, or n_v*(M+1) doubles, host or device: the moments of
 *      each start vector, mu_per_vec[l*(M+1) + k] = v_l^T T_k(B) v_l / n.
 * Synchronises `stream` (to read the status) unless DOS_OPT_NO_SPECTRUM_CHECK
 * is set and both outputs are device memory.
 * Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA, DOS_ESPECTRUM (moments are still
 * written).
 */
int dos_kpm_moments(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                    uint64_t seed, int precision, double *mu, double *mu_per_vec, void *stream);

/* dos_kpm_moments with options (vector offset for sharding, launch shape, flags). */
int dos_kpm_moments_ex(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                       uint64_t seed, int precision, double *mu, double *mu_per_vec,
                       const dos_kpm_opts *opts, void *stream);

/*
 * Batched sweep: B independent matrices of uneven size advanced together, one
 * kernel launch per Chebyshev step for all of them (the step sequence is
 * captured once in a CUDA graph and replayed).  The matrices are concatenated
 * row-wise in one CSR descriptor: A->row_ptr is global and non-decreasing over
 * all rows, A->col_idx is LOCAL to each matrix (0 <= col < n_b), A->n is the
 * total row count.  seg_rows (host, B+1 int64) gives the first row of each
 * matrix (seg_rows[0] = 0, seg_rows[B] = A->n, every n_b >= 1).  lb, ub: host
 * arrays of B bounds.  Matrix b uses start vectors with counter field b.
 * mu: B*(M+1) doubles (host or device), mu[b*(M+1) + k].
 * mu_per_vec: NULL or B*n_v*(M+1) doubles, [(b*n_v + l)*(M+1) + k].
 * Synchronises `stream`.  Errors as dos_kpm_moments.
 */
int dos_kpm_moments_batched(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows,
                            const double *lb, const double *ub, int M, int n_v, uint64_t seed,
                            int precision, double *mu, double *mu_per_vec,
                            const dos_kpm_opts *opts, void *stream);

/*
 * dos_kpm_moments without any memory allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc while they
 * run -- applications whose device memory is reserved up front by their own
 * pool allocator (so a library's cudaMalloc fails or evicts the pool's cache),
 * and services held to a fixed memory budget or latency target, where
 * cudaMalloc / cudaFree may synchronise the device.  It computes the same
 * moments mu_0..mu_M as dos_kpm_moments (single matrix, start-vector counter
 * b = 0, vector offset 0) but keeps all intermediates in one fixed 64 MiB
 * device array that is part of the library image (every GPU that loads the
 * library holds it until the process exits), so the caller passes only inputs
 * and outputs and no context is needed.  It works on the calling thread's current device.
 *   A: all three arrays in DEVICE memory (checked: a host array returns
 *      DOS_EINVAL before any work is queued); values FP64 for DOS_PREC_F64,
 *      FP32 for DOS_PREC_F32_ACC64 (no conversion copy is made).
 *   mu: M+1 doubles in device memory.
 *   Limits: n_v <= 256, M <= 20000, and 2 * n * ld * element_size <= 63 MiB
 *      with ld = n_v rounded up to 2 (FP64) or 4 (FP32) -- e.g. n <= 129024
 *      rows at n_v = 64 in FP32.  Larger problems return DOS_ENOMEM before any
 *      work is queued.
 *   The first call on a device looks up the array's device address with
 *   cudaGetSymbolAddress (in host code the array's name is only a stand-in for
 *   it); make that first call before any stream capture.  Every call uses the
 *   same array and leaves its contents behind (the kernels re-initialise what
 *   they read); calls that overlap on the GPU
 *   -- from several host threads or streams -- race on it and must be
 *   serialised by the caller.  Synchronises `stream` (to check the CSR
 *   structure and the spectrum).
 * Errors: DOS_EINVAL (bad argument or CSR, host pointers), DOS_ENOMEM (sizes
 * beyond the limits), DOS_ECUDA, DOS_ESPECTRUM.  No message is recorded.
 */
int dos_kpm_moments_noalloc(const dos_csr *A, double lb, double ub, int M, int n_v,
                            uint64_t seed, int precision, double *mu, void *stream);

/*
 * Autotuner: time each candidate launch shape of the fused sweep kernel for a
 * few steps on this matrix (and segment layout, B >= 1; seg_rows as in
 * dos_kpm_moments_batched, NULL when B == 1) and cache the fastest in the
 * context under the key (total rows, nnz, B, n_v, precision).  Later sweeps
 * with the same key use it unless a launch override is given.  `best`
 * (host, may be NULL) receives the choice; `best_ms` (may be NULL) its time per
 * step.  Synchronises `stream`.
 */
int dos_tune(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows, int n_v,
             int precision, dos_launch *best, double *best_ms, void *stream);

/* ---- step a6: reconstruction ----------------------------------------------- */
/*
 * DOS on a t-grid from moments normalised as above (Eq. tdosFinal with the
 * coefficients of Eq. expmu, and, for DOS_DAMP_JACKSON, the factors g_k^M of
 * Appendix A Eq. jackson):
 *     phi_hat(t) = [g_0 mu_0 + 2 sum_{k=1}^M g_k mu_k T_k(t)] / (pi sqrt(1 - t^2)),
 * and in eigenvalue units phi(lambda) = phi_hat((lambda - c)/d) / d.
 *   mu: M+1 doubles (host or device).  t: N_t points in (-1, 1) (host or
 *   device) or NULL for the Chebyshev nodes t_i = -cos(pi (i + 1/2) / N_t).
 *   phi_hat: N_t doubles (host or device).  phi_lambda: NULL or N_t doubles,
 *   which needs ub > lb.
 * Computed on the device in FP64.  Synchronises `stream` when an output is host
 * memory.  Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_reconstruct(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                    const double *t, int N_t, double *phi_hat, double *phi_lambda, void *stream);

/*
 * dos_reconstruct for B moment rows at once (the output of
 * dos_kpm_moments_batched): mu is B x (M+1) doubles, row-major; phi_hat is
 * B x N_t doubles, row b the density in t of row b of mu (Eq. tdosFinal with
 * the coefficients of Eq. expmu and, for DOS_DAMP_JACKSON, Appendix A's
 * factors), on the points t (N_t, in (-1, 1)) or, when t is NULL, the Chebyshev
 * nodes.  Each row equals dos_reconstruct's output for that row bit for bit.
 * Host or device arrays; synchronises `stream` when phi_hat is host memory.
 * 1 <= B <= 2^20, B N_t <= 2^31.  Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_reconstruct_batched(dos_ctx *ctx, const double *mu, int B, int M, int damping,
                            const double *t, int N_t, double *phi_hat, void *stream);

/*
 * Inverse of dos_reconstruct on the Chebyshev grid: given phi_hat at the N_t
 * nodes t_i = -cos(pi (i + 1/2) / N_t) (host or device), the moments
 *     mu_k = integral phi_hat(t) T_k(t) dt = (pi/N_t) sum_i sqrt(1 - t_i^2) phi_hat(t_i) T_k(t_i)
 * for k = 0..M_out, 0 <= M_out < N_t (Gauss-Chebyshev quadrature: exact when
 * sqrt(1 - t^2) phi_hat(t) is a polynomial of degree <= 2 N_t - 1 - M_out).
 * With DOS_DAMP_NONE and M_out = N_t - 1, dos_reconstruct of these moments on
 * the same grid returns phi_hat again: the cosine-transform pair behind the
 * paper's spectroscopic view of KPM (Section 3.1.2).  Used to score a DOS
 * given on a grid (e.g. the network of dos_mlp.h) with dos_smoothed_error.
 * mu: M_out+1 doubles, host or device.
 * Synchronises `stream` when mu is host memory.
 */
int dos_moments_from_grid(dos_ctx *ctx, const double *phi_hat, int N_t, int M_out, double *mu,
                          void *stream);

/* ---- step a7: accuracy metric ---------------------------------------------- */
/*
 * Error of the KPM DOS at resolution sigma (eigenvalue units), in the paper's
 * metric: both densities blurred by the Gaussian g_sigma (Eq. gauss), the
 * reference as phi_sigma(x) = (1/n) sum_j g_sigma(x - lambda_j) (Eq. blurphi
 * with the 1/n of Eq. DOS0), the KPM DOS as <phi_tilde, g_sigma(. - x)>
 * evaluated by Gauss-Chebyshev quadrature on N_q = max(4(M'+1), ceil(40 d /
 * sigma)) nodes (M' = max(M, M_ref)).  On a uniform grid of N_x points over
 * [lb - 6 sigma, ub + 6 sigma]:
 *     err_l1  = trapezoid integral of |difference|   (Eq. err2, p = 1),
 *     err_inf = max |difference|                      (Eq. errormetric).
 * Reference: `eig` (n_eig exact eigenvalues, host or device) if not NULL,
 * else `ref_mu` (M_ref+1 moments for the same lb, ub, with damping
 * ref_damping).  N_x in [2, 10^6].  err_l1, err_inf: host pointers (either may
 * be NULL).  Synchronises `stream`.
 */
int dos_smoothed_error(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                       const double *eig, int64_t n_eig, const double *ref_mu, int M_ref,
                       int ref_damping, double sigma, int N_x, double *err_l1, double *err_inf,
                       void *stream);

/* ---- the Lanczos DOS (Section 3.2.1) -------------------------------------- */
/*
 * n_v independent M-step Lanczos runs (Eq. lanfact, plain three-term
 * recurrence without reorthogonalisation, FP64) from the unit-normalised
 * Rademacher start vectors l = 0..n_v-1 of `seed` (the vectors of
 * dos_kpm_moments), advanced together as one block SpMM per step.  For each
 * run the eigenvalues theta (Ritz values, ascending) of its tridiagonal T and the
 * squared first components of the unit eigenvectors (weights, summing to one)
 * are computed on the device (Golub-Welsch: the nodes by bisection on Sturm
 * counts, each weight as the residue of e_1^T (zI - T)^{-1} e_1 by a contour
 * integral): the quadrature of Eq. landist / Eq. tauexpand.  Ritz values closer
 * than 1e-8 of the spectral scale (the copies that loss of orthogonality makes)
 * are reported as one node: the entry just below the group's weight centroid
 * holds the group's total weight at that centroid, the other entries keep their
 * Ritz value with weight 0 (theta stays ascending).  A run
 * that reaches an invariant subspace
 * (beta_j <= 1e-12 * its running norm estimate) stops after j+1 steps: its
 * remaining entries are 0 and m_used[l] = j+1.
 *   A: FP64 values.  1 <= M <= min(n, 4096), 1 <= n_v <= 256.
 *   theta, weight: n_v*M doubles, [l*M + k], host or device.
 *   m_used: NULL or n_v ints (host).
 * Synchronises `stream`.  Errors: DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA.
 */
int dos_lanczos_ritz(dos_ctx *ctx, const dos_csr *A, int M, int n_v, uint64_t seed,
                     double *theta, double *weight, int *m_used, void *stream);

/*
 * The Lanczos DOS of Eq. landos at N_x points x (host or device):
 *   phi(x) = (1/n_v) sum_l sum_k weight[l*M+k] g_sigma(x - theta[l*M+k])
 * (the paper's extra 1/n belongs to unnormalised start vectors; with unit ones
 * each run's weights sum to one and phi integrates to one).  phi: N_x doubles,
 * host or device.  Synchronises `stream` when phi is host memory.
 */
int dos_lanczos_dos(dos_ctx *ctx, const double *theta, const double *weight, int n_v, int M,
                    double sigma, const double *x, int N_x, double *phi, void *stream);

/*
 * Haydock's method (Section 3.2.2): the Lorentzian-blurred DOS
 *   phi_eta(x) = (1/n_v) sum_l sum_k weight[l*M+k] (eta/pi) / ((x - theta[l*M+k])^2 + eta^2),
 * which is -(1/pi) Im of the runs' M-step continued fraction
 * e_1^T ((x + i eta) I - T_M)^{-1} e_1 averaged over the runs, written through the
 * Ritz pairs of dos_lanczos_ritz (unit start vectors: no extra 1/n; the 1/pi
 * normalises the Lorentzian).  x: N_x points (host or device); phi: N_x doubles,
 * host or device.  Synchronises `stream` when phi is host memory.
 */
int dos_haydock_dos(dos_ctx *ctx, const double *theta, const double *weight, int n_v, int M,
                    double eta, const double *x, int N_x, double *phi, void *stream);

/*
 * dos_smoothed_error for an approximation given as weighted points (e.g. the
 * Ritz values and weights of dos_lanczos_ritz): the approximate density is
 * sum_j w_j g_sigma(x - p_j) / sum_j w_j, blurred by nothing further (the
 * Gaussian is already the blur); the reference, grid and norms are those of
 * dos_smoothed_error.  pts, wts: n_pts doubles, host or device.  err_l1,
 * err_inf: host (may be NULL).  Synchronises `stream`.
 */
int dos_points_error(dos_ctx *ctx, const double *pts, const double *wts, int64_t n_pts,
                     double lb, double ub, const double *eig, int64_t n_eig, const double *ref_mu,
                     int M_ref, int ref_damping, double sigma, int N_x, double *err_l1,
                     double *err_inf, void *stream);

/* ---- KPML and the Delta-Gauss-Legendre method (Sections 3.1.1, 3.1.3, App. B) */
/*
 * Legendre moments nu_k = (1/(n n_v)) sum_l v_l^T L_k(B) v_l, k = 0..M, of the
 * same start vectors and B as dos_kpm_moments (Algorithm DGL, with Rademacher
 * vectors in place of normalised ones, hence the 1/n; nu_0 = 1).
 * Algorithm DGL forms them from M passes of the Legendre recurrence
 * (k+1) v_{k+1} = (2k+1) B v_k - k v_{k-1}; here they come from the Chebyshev
 * sweep (ceil(M/2) passes with the doubling identity) and the exact expansion
 *     L_k(t) = sum_{m=0}^{floor(k/2)} e_{k-2m} h_m h_{k-m} T_{k-2m}(t),
 *     h_m = (2m)! / (4^m (m!)^2),  e_0 = 1, e_j = 2 (j > 0),
 * whose coefficients are non-negative and sum to L_k(1) = 1, so each nu_k is a
 * convex combination of mu_0..mu_k and inherits their rounding error.
 * Arguments, precision, options and errors as dos_kpm_moments_ex; nu: M+1
 * doubles, nu_per_vec: NULL or n_v*(M+1) doubles [l*(M+1) + k] (host or device).
 */
int dos_legendre_moments(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                         uint64_t seed, int precision, double *nu, double *nu_per_vec,
                         const dos_kpm_opts *opts, void *stream);

/*
 * The expansion above applied to `count` rows of M+1 Chebyshev moments
 * (mu[r*(M+1) + j], normalised as dos_kpm_moments) giving Legendre moments
 * nu[r*(M+1) + k].  mu, nu: host or device, distinct.  0 <= M <= 100000.
 * Synchronises `stream` when nu is host memory.  Errors: DOS_EINVAL,
 * DOS_ENOMEM, DOS_ECUDA.
 */
int dos_cheb_to_legendre(dos_ctx *ctx, const double *mu, int64_t count, int M, double *nu,
                         void *stream);

/*
 * KPML: the Legendre expansion of the DOS (Section 3.1.1; undamped -- the paper
 * gives no damping for Legendre polynomials):
 *     phi_L(t) = sum_{k=0}^{M} (k + 1/2) nu_k L_k(t),
 * and phi(lambda) = phi_L((lambda - c)/d) / d.  nu: M+1 doubles; t: N_t points
 * in [-1, 1] or NULL for the nodes t_i = -cos(pi (i + 1/2) / N_t); phi_t: N_t
 * doubles; phi_lambda: NULL or N_t doubles (needs ub > lb).  All host or
 * device.  Synchronises `stream` when an output is host memory.
 */
int dos_kpml_reconstruct(dos_ctx *ctx, const double *nu, int M, double lb, double ub,
                         const double *t, int N_t, double *phi_t, double *phi_lambda,
                         void *stream);

/*
 * DGL (Eq. dglexpansion, Algorithm DGL): at each x (eigenvalue units) with
 * t = (x - c)/d and s = sigma/d,
 *     phi(x) = (1/d) (2 pi s^2)^{-1/2} sum_{k=0}^{M_x} (k + 1/2) gamma_k(t) nu_k,
 *     gamma_k(t) = int_{-1}^{1} L_k(u) exp(-((u - t)/s)^2 / 2) du   (Eq. DGLcoeff),
 * gamma_0 from Eq. gam0 (erf), the rest from the joint recurrence of Eq. Leg3
 * (psi_0 = 0, psi_1 = gamma_0, zeta_k of Eq. eta), stopped at the first k >= 1
 * with |gamma_{k-1}| + |gamma_k| <= k tol (Eq. StopRecur; tol <= 0: never) or
 * at M: M_x = that k.  phi approximates the Gaussian-blurred DOS
 * (1/n) sum_j g_sigma(x - lambda_j) directly.
 *   nu: M+1 doubles; x: N_x points, or NULL for the metric's grid of
 *   dos_smoothed_error (N_x points over [lb - 6 sigma, ub + 6 sigma]);
 *   phi: N_x doubles; m_used: NULL or N_x ints.  All host or device.
 * Synchronises `stream` when an output is host memory.
 */
int dos_dgl(dos_ctx *ctx, const double *nu, int M, double lb, double ub, double sigma, double tol,
            const double *x, int N_x, double *phi, int *m_used, void *stream);

/*
 * dos_smoothed_error for the Legendre methods: method DOS_LEG_KPML blurs phi_L
 * as <phi_L, g_sigma(. - x)> by Gauss-Legendre quadrature on
 * N_q = max(4(M'+1), ceil(40 d / sigma)) nodes of [-1, 1] (nodes by Newton's
 * method on L_{N_q}); method DOS_LEG_DGL uses phi of dos_dgl as is (the paper
 * compares DGL with the sup-norm of Eq. err2).  Reference, grid, norms and
 * outputs as dos_smoothed_error.  Synchronises `stream`.
 */
enum { DOS_LEG_KPML = 0, DOS_LEG_DGL = 1 };
int dos_legendre_error(dos_ctx *ctx, const double *nu, int M, int method, double lb, double ub,
                       double sigma, double tol, const double *eig, int64_t n_eig,
                       const double *ref_mu, int M_ref, int ref_damping, int N_x, double *err_l1,
                       double *err_inf, void *stream);

/* ---- an observable: the heat capacity (Section 4.3) ------------------------ */
/*
 * <phi, g_beta> for each beta in betas (n_beta values, host or device) with the
 * heat-capacity kernel of Eq. gfunc up to its constant factor,
 *     g_beta(lambda) = x^2 e^{-x} / (1 - e^{-x})^2,  x = beta sqrt(max(lambda, 0))
 * (beta = hbar c / (k_B T); the paper normalises C_v to a maximum of one, so
 * constants do not matter; g -> 1 as x -> 0).  The density is either
 *   - KPM moments mu (M+1, host or device, normalised as dos_kpm_moments) with
 *     damping, integrated by Gauss-Chebyshev quadrature on max(4(M+1), 2048)
 *     nodes of [lb, ub]: (1/N_q) sum_i P(t_i) g(c + d t_i); pts must be NULL;
 *   - or weighted points (Ritz values and weights of dos_lanczos_ritz, or exact
 *     eigenvalues with equal weights): sum_j w_j g(p_j) / sum_j w_j; mu NULL.
 * The error of an estimate is Eq. errormetric_g: |<phi,g> - <phi_tilde,g>|.
 * cv: n_beta doubles (host or device).  Synchronises `stream`.
 */
int dos_heat_capacity(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                      const double *pts, const double *wts, int64_t n_pts, const double *betas,
                      int n_beta, double *cv, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DOS_H */
