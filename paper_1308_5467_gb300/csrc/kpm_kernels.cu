// Kernels of the Chebyshev moment sweep (steps a2-a5 of the KPM path).
//
// Data layout in HBM
//   vector blocks X (two of them): row-major, n_rows x ld, element (i, l) at
//   X[i*ld + l]; ld = n_v rounded up to a 16-byte multiple, pad columns zero.
//   A nonzero a_ij therefore feeds all n_v right-hand sides from one
//   contiguous row X[j, :], read with 16-byte vector loads by a "team" of
//   threads that shares the matrix row.
//   The recurrence writes X_{k+1} over X_{k-1} in place (same thread reads the
//   old value and writes the new one), so two blocks suffice.
//
// One launch per Chebyshev step k computes, in a single pass over A:
//   X_{k+1} = 2 (A X_k - c X_k)/d - X_{k-1}        (k >= 1, Eq. 3term with B = (A-cI)/d)
//   X_1     =   (A X_0 - c X_0)/d                   (k = 0, Algorithm 1)
// and the per-vector dot products of the doubling identity (Appendix A):
//   r_k = X_{k+1} . X_k  -> mu_{2k+1} = 2 r_k/n - mu_1   (mu_1 = r_0/n)
//   s_k = X_{k+1} . X_{k+1} -> mu_{2k+2} = 2 s_k/n - mu_0
//   z   = X_0 . X_0 (k = 0 only) -> mu_0.
// Partial sums are written per tile (one tile per block) and reduced later in
// a fixed order, so results are bitwise reproducible for a given launch shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "dos_internal.h"

namespace dos {
namespace {

constexpr int kBlock = 256;

// ---- splitmix64 (Steele, Lea, Flood 2014), device side -------------------------
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return z;
}
// Word number ctr+1 of the stream seeded with `seed`.
__device__ __forceinline__ uint64_t rademacher_word(uint64_t seed, uint64_t b, uint64_t word,
                                                    uint64_t row) {
    const uint64_t ctr = (b << 48) + (word << 32) + row;
    return sm64_mix(seed + (ctr + 1ULL) * 0x9e3779b97f4a7c15ULL);
}

// ---- unevaluated float pair accumulator ---------------------------------------
// sum = hi + lo.  Each product x*y of two floats is split exactly into
// p + pe (fma), p is added to hi with Knuth's branch-free two-sum, and both
// rounding errors go to lo.  The __f*_rn intrinsics keep the compiler from
// contracting the error-free steps into fused operations.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add_prod(FF &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = fmaf(x, y, -p);
    const float s = __fadd_rn(a.hi, p);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(e, pe));
}
// Add a float to the pair with the same two-sum (no product split).
__device__ __forceinline__ void ff_add(FF &a, float v) {
    const float s = __fadd_rn(a.hi, v);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ double acc_value(const FF &a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ void acc_zero(FF &a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void acc_add_prod(FF &a, float x, float y) { ff_add_prod(a, x, y); }
__device__ __forceinline__ void acc_add(FF &a, float v) { ff_add(a, v); }

__device__ __forceinline__ double acc_value(const double &a) { return a; }
__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_add_prod(double &a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_add(double &a, double v) { a += v; }

// ---- the affine map of B = (A - cI)/d --------------------------------------------
// (y - c x) / d for y = (A X)[i, l], x = X[i, l].  In FP32, c and 1/d are each
// carried as an unevaluated pair hi + lo (lo = the FP32 rounding of the
// remainder), so the FP32 form applies B itself to about 2^-48 instead of the
// operator built from c and 1/d rounded to FP32.  That rounding would move
// every eigenvalue of B by up to 2^-24 relative, an error of mu_k that does not
// average out over rows and vectors and grows like k 2^-24 at a point mass of
// the spectrum near +-1; what is left is the rounding of each step's result.
template <typename T>
struct Affine {
    T c, c_lo, s, s_lo;
    __device__ __forceinline__ Affine(double cd, double sd) {
        c = (T)cd;
        s = (T)sd;
        c_lo = (T)(cd - (double)c);
        s_lo = (T)(sd - (double)s);
    }
    __device__ __forceinline__ T operator()(T y, T x) const {
        T t = fma(-c, x, y);
        if constexpr (sizeof(T) == 4) t = fma(-c_lo, x, t);
        T r = t * s;
        if constexpr (sizeof(T) == 4) r = fma(t, s_lo, r);
        return r;
    }
};

template <typename T> struct Traits;
template <> struct Traits<float> {
    static constexpr int VPT = 4;
    using Acc = FF;
};
template <> struct Traits<double> {
    static constexpr int VPT = 2;
    using Acc = double;
};

template <typename T>
__device__ __forceinline__ void load16(const T *p, T (&v)[Traits<T>::VPT]) {
    if constexpr (sizeof(T) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
}
template <typename T>
__device__ __forceinline__ void store16(T *p, const T (&v)[Traits<T>::VPT]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
}

// A chunk is the W consecutive vector entries one thread moves with one
// instruction: 16 bytes (float4 / double2) or 32 bytes (the 256-bit
// ld.global.v8.f32 / .v4.f64 and st.global forms of this GPU).  The 32-byte
// forms are inline PTX marked volatile so that none of them is moved above the
// grid-dependency wait at the top of the step kernel.
template <typename T, int W>
__device__ __forceinline__ void load_chunk(const T *p, T (&v)[W]) {
    static_assert(sizeof(T) * W == 16 || sizeof(T) * W == 32, "16- or 32-byte chunks");
    if constexpr (sizeof(T) * W == 16) {
        load16(p, v);
    } else if constexpr (sizeof(T) == 4) {
        asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                       "=f"(v[6]), "=f"(v[7])
                     : "l"(p));
    } else {
        asm volatile("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
                     : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                     : "l"(p));
    }
}
// X_{k-1}[i]: read once, then overwritten by the same thread (no L1 allocation
// for the 32-byte form, so the stream does not evict gathered rows of X_k).
template <typename T, int W>
__device__ __forceinline__ void load_chunk_prev(const T *p, T (&v)[W]) {
    if constexpr (sizeof(T) * W == 16) {
        load16(p, v);
    } else if constexpr (sizeof(T) == 4) {
        asm volatile("ld.global.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                       "=f"(v[6]), "=f"(v[7])
                     : "l"(p));
    } else {
        asm volatile("ld.global.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                     : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                     : "l"(p));
    }
}
template <typename T, int W>
__device__ __forceinline__ void store_chunk(T *p, const T (&v)[W]) {
    if constexpr (sizeof(T) * W == 16) {
        store16(p, v);
    } else if constexpr (sizeof(T) == 4) {
        asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
                     "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
    } else {
        asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                     "d"(v[2]), "d"(v[3]));
    }
}

// ---- start vectors (step a2) ---------------------------------------------------
template <typename T>
__global__ void init_vectors_kernel(T *__restrict__ x, int64_t n_rows, int ld, int n_v, int B,
                                    const int32_t *__restrict__ seg_row0, uint64_t seed,
                                    int64_t vec_offset, uint64_t b0) {
    constexpr int VPT = Traits<T>::VPT;
    const int chunks = ld / VPT;
    const int64_t total = n_rows * chunks;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / chunks;
        const int ch = (int)(t - row * chunks);
        // segment of this row
        int lo = 0, hi = B;  // seg_row0[lo] <= row < seg_row0[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg_row0[mid] <= row) lo = mid; else hi = mid;
        }
        const uint64_t local = (uint64_t)(row - seg_row0[lo]);
        T v[VPT];
        uint64_t cached_word = ~0ULL, bits = 0;
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            const int l = ch * VPT + j;
            if (l < n_v) {
                const uint64_t gl = (uint64_t)(vec_offset + l);
                if ((gl >> 6) != cached_word) {
                    cached_word = gl >> 6;
                    bits = rademacher_word(seed, b0 + (uint64_t)lo, cached_word, local);
                }
                v[j] = ((bits >> (gl & 63)) & 1ULL) ? T(-1) : T(1);
            } else {
                v[j] = T(0);
            }
        }
        store16(x + row * ld + ch * VPT, v);
    }
}

// ---- fused step (steps a3, a4) ---------------------------------------------------
template <typename T>
struct StepParams {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const T *val;
    const T *xc;  // X_k
    T *xn;        // X_{k-1} on entry, X_{k+1} on exit
    int ld, n_chunks, pv, first;
    const int4 *tiles;
    const int32_t *seg_row0;
    const double *seg_c, *seg_inv_d;
    double *part;   // [n_tiles][2][pv]
    double *part0;  // [n_tiles][pv]
    int *status;    // bit 2 (value 4): a bounded device-side wait ran out
    int panel_rows; // staged kernel: rows per shared-memory panel
    long long spin_cycles;  // staged kernel: wait limit in SM clock cycles
    int stall_test; // staged kernel, tests only: over-count the expected bytes so a
                    // wait never completes and must run out
    int rev;        // direct kernel: walk each tile's rows from its last row down
};

// Deterministic block reduction of one accumulator set into out[0..pv).
// red: shared scratch of (blockDim/32) * ld doubles.
template <typename Acc, int G, int CPT, int VPT>
__device__ __forceinline__ void block_reduce_store(const Acc (&acc)[CPT][VPT], double *out,
                                                   int ld, int n_chunks, int pv, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    const int g = lane % G;
    double v[CPT][VPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int j = 0; j < VPT; ++j) v[c][j] = acc_value(acc[c][j]);
    // sum over the teams of this warp (fixed tree)
#pragma unroll
    for (int off = G; off < 32; off <<= 1)
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
            for (int j = 0; j < VPT; ++j) v[c][j] += __shfl_down_sync(0xffffffffu, v[c][j], off);
    if (lane < G) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int ch = g + c * G;
            if (ch < n_chunks)
#pragma unroll
                for (int j = 0; j < VPT; ++j) red[warp * ld + ch * VPT + j] = v[c][j];
        }
    }
    __syncthreads();
    if (pv > 1) {
        for (int col = threadIdx.x; col < ld; col += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < n_warps; ++w) s += red[w * ld + col];
            out[col] = s;
        }
    } else {
        // columns summed over warps, then over columns by warp 0 (fixed order)
        for (int col = threadIdx.x; col < ld; col += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < n_warps; ++w) s += red[w * ld + col];
            red[col] = s;  // column `col` of warp 0's row is only read by this thread
        }
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
            for (int col = lane; col < ld; col += 32) s += red[col];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) out[0] = s;
        }
    }
    __syncthreads();
}

// One block per row tile; a team of G threads shares a matrix row, thread g of
// the team owning the 16-byte chunks g, g+G, ..., g+(CPT-1)G of the rows of X.
// Per row the independent loads are issued before anything waits on them: the
// row's own X_k[i] and X_{k-1}[i] chunks and the next row's extents first, then
// the gathers X_k[j] of up to 8 nonzeros at a time; so a row costs about one
// memory latency instead of a chain of four.
// The next U (column, value) pairs of the team's row, starting at entry e
// (entries at or past e1 come back as column 0, value 0).  Thread g of the team
// loads entries e + g, e + g + G, ... once, and the team exchanges them by
// shuffles among its own lanes (mask), instead of every thread loading all U.
template <typename T, int G, int U>
__device__ __forceinline__ void team_fetch(const int32_t *__restrict__ col_idx,
                                           const T *__restrict__ val, int e, int e1, int g,
                                           int team_base, unsigned mask, int (&col)[U],
                                           T (&a)[U]) {
    constexpr int PER = (U + G - 1) / G;
    int mc[PER];
    T ma[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int idx = e + g + q * G;
        const bool ok = (g + q * G < U) && idx < e1;
        mc[q] = ok ? __ldg(col_idx + idx) : 0;
        ma[q] = ok ? __ldg(val + idx) : T(0);
    }
    if constexpr (G == 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            col[u] = mc[u];
            a[u] = ma[u];
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            col[u] = __shfl_sync(mask, mc[u / G], team_base + (u % G));
            a[u] = __shfl_sync(mask, ma[u / G], team_base + (u % G));
        }
    }
}

// Deterministic block sum of one value per thread into *out (red: >= 32 doubles).
template <typename Acc>
__device__ __forceinline__ void block_reduce_scalar(const Acc &acc, double *out, double *red) {
    double v = acc_value(acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s;
    }
    __syncthreads();
}

// PV: keep one accumulator per vector (per-vector moments requested); otherwise
// each thread first sums its row's products over its own vectors in the
// working precision (at most 4*CPT terms, an error at the level of the FP32
// rounding of the vectors themselves) and accumulates those row sums.
// FIRST: the step X_1 = B X_0 (no X_{k-1}; also accumulates X_0 . X_0).  Being a
// template parameter, the 249-of-250 ordinary steps carry no branch on it, which
// frees registers and lets the compiler schedule the gathers of a batch together.
// Threads that hold at most 32 bytes of a row (CPT * CB <= 32) fit in 64 registers:
// four blocks per SM; wider ones keep their batch of gathers in up to 80: three.
template <typename T, int G, int CPT, bool PV, int CB, bool FIRST>
__global__ void __launch_bounds__(kBlock, CPT * CB <= 32 ? 4 : 3)
    step_kernel(const StepParams<T> p) {
    constexpr int VPT = CB / (int)sizeof(T);  // vector entries per chunk
    using Acc = typename Traits<T>::Acc;
    constexpr int TPW = 32 / G;  // teams per warp
    constexpr int U = CPT * CB >= 64 ? 4 : 8;  // nonzeros per gather batch (bounded registers)
    extern __shared__ double red[];

    // Programmatic dependent launch: let the next step's grid be scheduled now,
    // and wait until the previous grid has completed and its writes are visible
    // before reading anything it produced.  Both are no-ops for a plain launch.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const int4 tl = p.tiles[blockIdx.x];
    const int rb = tl.x, re = tl.y, seg = tl.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % G;
    const int n_teams = (blockDim.x >> 5) * TPW;
    const int team = warp * TPW + lane / G;
    const int team_base = (lane / G) * G;
    const unsigned team_mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << team_base);
    const Affine<T> shift(p.seg_c[seg], p.seg_inv_d[seg]);
    const int ld = p.ld;
    const T *__restrict__ xseg = p.xc + (size_t)p.seg_row0[seg] * ld;
    const T *__restrict__ xc = p.xc;
    const int32_t *__restrict__ row_ptr = p.row_ptr;
    const int32_t *__restrict__ col_idx = p.col_idx;
    const T *__restrict__ val = p.val;
    T *xn = p.xn;

    constexpr bool first = FIRST;
    constexpr int NA = PV ? CPT : 1, NJ = PV ? VPT : 1;
    Acc accR[NA][NJ], accS[NA][NJ], acc0[NA][NJ];
#pragma unroll
    for (int cc = 0; cc < NA; ++cc)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            acc_zero(accR[cc][j]);
            acc_zero(accS[cc][j]);
            acc_zero(acc0[cc][j]);
        }

    bool valid[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) valid[cc] = (g + cc * G) < p.n_chunks;

    // Row idx of the tile (idx = team, team + n_teams, ...) is tile row rb + idx, or
    // re - 1 - idx on steps that walk the tile backwards: consecutive steps then meet
    // first the rows the previous step wrote last, while they are still in L2.
    const int cnt = re - rb;
    const int rdir = p.rev ? -1 : 1, rorg = p.rev ? re - 1 : rb;
    int idx = team;
    int row = rorg + rdir * idx;
    int e0 = 0, e1 = 0;
    if (idx < cnt) {
        e0 = __ldg(row_ptr + row);
        e1 = __ldg(row_ptr + row + 1);
    }
    while (idx < cnt) {
        const size_t roff = (size_t)row * ld;
        T xk[CPT][VPT], xo[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (valid[cc]) {
                const int off = (g + cc * G) * VPT;
                load_chunk(xc + roff + off, xk[cc]);
                if (!first) load_chunk_prev(xn + roff + off, xo[cc]);
            }
        }
        const int nidx = idx + n_teams;
        const int nrow = rorg + rdir * nidx;
        int ne0 = 0, ne1 = 0;
        if (nidx < cnt) {
            ne0 = __ldg(row_ptr + nrow);
            ne1 = __ldg(row_ptr + nrow + 1);
        }
        T y[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
            for (int j = 0; j < VPT; ++j) y[cc][j] = T(0);
        for (int e = e0; e < e1; e += U) {
            int col[U];
            T a[U];
            team_fetch<T, G, U>(col_idx, val, e, e1, g, team_base, team_mask, col, a);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e + u < e1) {
                    const T *src = xseg + (size_t)col[u] * ld;
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        if (valid[cc]) {
                            T xv[VPT];
                            load_chunk(src + (g + cc * G) * VPT, xv);
#pragma unroll
                            for (int j = 0; j < VPT; ++j) y[cc][j] = fma(a[u], xv[j], y[cc][j]);
                        }
                    }
                }
            }
        }
        T rr = T(0), ss = T(0), zz = T(0);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (!valid[cc]) continue;
            const int off = (g + cc * G) * VPT;
            T xnew[VPT];
            if (first) {
#pragma unroll
                for (int j = 0; j < VPT; ++j) xnew[j] = shift(y[cc][j], xk[cc][j]);
            } else {
#pragma unroll
                for (int j = 0; j < VPT; ++j)
                    xnew[j] = fma(T(2), shift(y[cc][j], xk[cc][j]), -xo[cc][j]);
            }
            store_chunk(xn + roff + off, xnew);
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if constexpr (PV) {
                    acc_add_prod(accR[cc][j], xnew[j], xk[cc][j]);
                    acc_add_prod(accS[cc][j], xnew[j], xnew[j]);
                    if (first) acc_add_prod(acc0[cc][j], xk[cc][j], xk[cc][j]);
                } else {
                    rr = fma(xnew[j], xk[cc][j], rr);
                    ss = fma(xnew[j], xnew[j], ss);
                    zz = fma(xk[cc][j], xk[cc][j], zz);
                }
            }
        }
        if constexpr (!PV) {
            acc_add(accR[0][0], rr);
            acc_add(accS[0][0], ss);
            if (first) acc_add(acc0[0][0], zz);
        }
        idx = nidx;
        row = nrow;
        e0 = ne0;
        e1 = ne1;
    }

    if constexpr (PV) {
        double *out = p.part + (size_t)blockIdx.x * 2 * p.pv;
        block_reduce_store<Acc, G, CPT, VPT>(accR, out, ld, p.n_chunks, p.pv, red);
        block_reduce_store<Acc, G, CPT, VPT>(accS, out + p.pv, ld, p.n_chunks, p.pv, red);
        if (first)
            block_reduce_store<Acc, G, CPT, VPT>(acc0, p.part0 + (size_t)blockIdx.x * p.pv, ld,
                                                 p.n_chunks, p.pv, red);
    } else {
        double *out = p.part + (size_t)blockIdx.x * 2;
        block_reduce_scalar(accR[0][0], out, red);
        block_reduce_scalar(accS[0][0], out + 1, red);
        if (first) block_reduce_scalar(acc0[0][0], p.part0 + blockIdx.x, red);
    }
}

// ---- TMA-staged variant -----------------------------------------------------------
// The tile is walked in panels of R consecutive rows.  One elected thread
// copies the panel's slabs X_k[r0:r0+R, :] and X_{k-1}[r0:r0+R, :] (contiguous,
// 16-byte aligned) into shared memory with bulk asynchronous copies
// (cp.async.bulk, the Tensor Memory Accelerator's 1-D form) that complete on an
// mbarrier, two stages deep, so the next panel streams in while this one is
// computed and the streaming loads hold no registers.  The gathers X_k[j] of
// the SpMM still go through L1/L2.  Every wait is bounded: past
// `spin_cycles` the block agrees (syncthreads_or) to stop, sets status bit 4
// and returns after waiting, again bounded, for its copies in flight.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait for phase `parity` of `bar`; false if `limit` cycles passed first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

template <typename T, int G, int CPT, bool PV>
__global__ void __launch_bounds__(kBlock, 2) step_staged_kernel(const StepParams<T> p) {
    constexpr int VPT = Traits<T>::VPT;
    using Acc = typename Traits<T>::Acc;
    constexpr int TPW = 32 / G;
    constexpr int U = CPT >= 4 ? 4 : 8;
    extern __shared__ __align__(128) unsigned char smem[];
    const int ld = p.ld;
    const int R = p.panel_rows;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);          // 2 barriers
    T *slab = reinterpret_cast<T *>(smem + 128);                  // [2 stages][cur, prev][R*ld]
    double *red = reinterpret_cast<double *>(smem + 128 + 4 * (size_t)R * ld * sizeof(T));

    const int4 tl = p.tiles[blockIdx.x];
    const int rb = tl.x, re = tl.y, seg = tl.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % G;
    const int n_teams = (blockDim.x >> 5) * TPW;
    const int team = warp * TPW + lane / G;
    const int team_base = (lane / G) * G;
    const unsigned team_mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << team_base);
    const Affine<T> shift(p.seg_c[seg], p.seg_inv_d[seg]);
    const T *__restrict__ xseg = p.xc + (size_t)p.seg_row0[seg] * ld;
    const int32_t *__restrict__ row_ptr = p.row_ptr;
    const int32_t *__restrict__ col_idx = p.col_idx;
    const T *__restrict__ val = p.val;
    T *xn = p.xn;
    const bool first = p.first != 0;
    const int n_panels = (re - rb + R - 1) / R;

    constexpr int NA = PV ? CPT : 1, NJ = PV ? VPT : 1;
    Acc accR[NA][NJ], accS[NA][NJ], acc0[NA][NJ];
#pragma unroll
    for (int cc = 0; cc < NA; ++cc)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            acc_zero(accR[cc][j]);
            acc_zero(accS[cc][j]);
            acc_zero(acc0[cc][j]);
        }
    bool valid[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) valid[cc] = (g + cc * G) < p.n_chunks;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int panel, int stage) {
        const int r0 = rb + panel * R;
        const int rows = min(R, re - r0);
        const uint32_t bytes = (uint32_t)((size_t)rows * ld * sizeof(T));
        T *dst = slab + (size_t)stage * 2 * R * ld;
        mbar_expect_tx(&bar[stage], (first ? bytes : 2 * bytes) + (p.stall_test ? 16u : 0u));
        bulk_copy_g2s(dst, p.xc + (size_t)r0 * ld, bytes, &bar[stage]);
        if (!first) bulk_copy_g2s(dst + (size_t)R * ld, xn + (size_t)r0 * ld, bytes, &bar[stage]);
    };
    if (threadIdx.x == 0 && n_panels > 0) issue(0, 0);
    int issued = n_panels > 0 ? 1 : 0, consumed = 0;
    bool timed_out = false;
    for (int pi = 0; pi < n_panels; ++pi) {
        const int stage = pi & 1;
        if (threadIdx.x == 0 && pi + 1 < n_panels) issue(pi + 1, stage ^ 1);
        if (pi + 1 < n_panels) ++issued;
        const bool ok = mbar_wait_bounded(&bar[stage], (pi >> 1) & 1, p.spin_cycles);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        ++consumed;
        const T *scur = slab + (size_t)stage * 2 * R * ld;
        const T *sprev = scur + (size_t)R * ld;
        const int r0 = rb + pi * R;
        const int rows = min(R, re - r0);
        int j = team;
        int e0 = 0, e1 = 0;
        if (j < rows) {
            e0 = __ldg(row_ptr + r0 + j);
            e1 = __ldg(row_ptr + r0 + j + 1);
        }
        while (j < rows) {
            const int row = r0 + j;
            const int nj = j + n_teams;
            int ne0 = 0, ne1 = 0;
            if (nj < rows) {
                ne0 = __ldg(row_ptr + r0 + nj);
                ne1 = __ldg(row_ptr + r0 + nj + 1);
            }
            T y[CPT][VPT];
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
                for (int q = 0; q < VPT; ++q) y[cc][q] = T(0);
            for (int e = e0; e < e1; e += U) {
                int col[U];
                T a[U];
                team_fetch<T, G, U>(col_idx, val, e, e1, g, team_base, team_mask, col, a);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (e + u < e1) {
                        const T *src = xseg + (size_t)col[u] * ld;
#pragma unroll
                        for (int cc = 0; cc < CPT; ++cc) {
                            if (valid[cc]) {
                                T xv[VPT];
                                load16(src + (g + cc * G) * VPT, xv);
#pragma unroll
                                for (int q = 0; q < VPT; ++q) y[cc][q] = fma(a[u], xv[q], y[cc][q]);
                            }
                        }
                    }
                }
            }
            T rr = T(0), ss = T(0), zz = T(0);
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                if (!valid[cc]) continue;
                const int off = (g + cc * G) * VPT;
                T xk[VPT], xo[VPT], xnew[VPT];
                load16(scur + (size_t)j * ld + off, xk);
                if (first) {
#pragma unroll
                    for (int q = 0; q < VPT; ++q) xnew[q] = shift(y[cc][q], xk[q]);
                } else {
                    load16(sprev + (size_t)j * ld + off, xo);
#pragma unroll
                    for (int q = 0; q < VPT; ++q)
                        xnew[q] = fma(T(2), shift(y[cc][q], xk[q]), -xo[q]);
                }
                store16(xn + (size_t)row * ld + off, xnew);
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    if constexpr (PV) {
                        acc_add_prod(accR[cc][q], xnew[q], xk[q]);
                        acc_add_prod(accS[cc][q], xnew[q], xnew[q]);
                        if (first) acc_add_prod(acc0[cc][q], xk[q], xk[q]);
                    } else {
                        rr = fma(xnew[q], xk[q], rr);
                        ss = fma(xnew[q], xnew[q], ss);
                        zz = fma(xk[q], xk[q], zz);
                    }
                }
            }
            if constexpr (!PV) {
                acc_add(accR[0][0], rr);
                acc_add(accS[0][0], ss);
                if (first) acc_add(acc0[0][0], zz);
            }
            j = nj;
            e0 = ne0;
            e1 = ne1;
        }
        __syncthreads();  // this stage is refilled in the next iteration
    }
    if (timed_out) {
        // drain: wait (bounded) for the copies this block issued and never consumed
        if (threadIdx.x == 0) {
            atomicOr(p.status, 4);
            for (int k = consumed; k < issued; ++k)
                mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1, p.spin_cycles);
        }
        __syncthreads();
        return;
    }
    if constexpr (PV) {
        double *out = p.part + (size_t)blockIdx.x * 2 * p.pv;
        block_reduce_store<Acc, G, CPT, VPT>(accR, out, ld, p.n_chunks, p.pv, red);
        block_reduce_store<Acc, G, CPT, VPT>(accS, out + p.pv, ld, p.n_chunks, p.pv, red);
        if (first)
            block_reduce_store<Acc, G, CPT, VPT>(acc0, p.part0 + (size_t)blockIdx.x * p.pv, ld,
                                                 p.n_chunks, p.pv, red);
    } else {
        double *out = p.part + (size_t)blockIdx.x * 2;
        block_reduce_scalar(accR[0][0], out, red);
        block_reduce_scalar(accS[0][0], out + 1, red);
        if (first) block_reduce_scalar(acc0[0][0], p.part0 + blockIdx.x, red);
    }
}

// ---- TMA-gather variant -------------------------------------------------------------
// The gathers X_k[j, :] of the SpMM are issued as tensor-memory-accelerator
// gathers: one elected lane per team loads the rows of four nonzeros with a single
// cp.async.bulk.tensor ... tile::gather4 (a 2-D tensor map of the vector block,
// boxes one row high) into a per-team shared-memory stage, completing on that
// stage's mbarrier.  Each team owns a ring of `depth` stages and walks its rows as
// one stream of batches (four nonzeros each, padded with column 0 / value 0 past a
// row's end): the producer side runs up to depth batches ahead of the consumer,
// across row boundaries, so the gathers of the next rows are in flight while this
// row is summed.  The gathered rows hold no registers and no L1 miss slots.
// X_k[i] and X_{k-1}[i] are thread loads as in the direct kernel.  Used for steps
// k >= 1 (the first step runs the direct first-step instance).  Every wait is
// bounded: past spin_cycles a team stops, sets status bit 4 and waits (bounded
// again) for its gathers in flight before the block ends.  The wait test
// (stall_test) arms the barrier without issuing the gather.
// The tensor-map type and cuTensorMapEncodeTiled's signature (driver API).
#include <cuda.h>
#include <cudaTypedefs.h>

__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *tmap, int r0, int r1,
                                            int r2, int r3, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared memory: [depth barriers per team][4 values per stage][pad to 128 B]
// [depth stages per team, each the 4 gathered rows packed (row u at u * ld), rounded
// up to 128 B][reduction scratch].
__host__ __device__ inline size_t tmag_stage_bytes(int ld, int esz) {
    return ((size_t)4 * ld * esz + 127) / 128 * 128;
}
__host__ __device__ inline size_t tmag_head_bytes(int n_teams, int depth, int esz) {
    return ((size_t)n_teams * depth * (sizeof(uint64_t) + 4 * esz) + 127) / 128 * 128;
}
size_t tmag_smem(int block, int team, int ld, int esz, int depth) {
    const int n_teams = (block / 32) * (32 / team);
    return tmag_head_bytes(n_teams, depth, esz) +
           (size_t)n_teams * depth * tmag_stage_bytes(ld, esz) +
           (size_t)(block / 32) * ld * sizeof(double);
}
// Ring depth: the one asked for, else the deepest of 8, 4, 2 that leaves room for
// two blocks per SM.
int tmag_ring_depth(int block, int team, int ld, int esz, int asked) {
    if (asked) return asked;
    for (int d = 8; d > 2; d >>= 1)
        if (tmag_smem(block, team, ld, esz, d) <= (size_t)112 * 1024) return d;
    return 2;
}

template <typename T, int G, int CPT, bool PV>
__global__ void __launch_bounds__(kBlock, 2) step_tmag_kernel(const StepParams<T> p,
                                                             const __grid_constant__ CUtensorMap tmap,
                                                             const int log2_depth) {
    constexpr int VPT = Traits<T>::VPT;
    using Acc = typename Traits<T>::Acc;
    constexpr int TPW = 32 / G;
    extern __shared__ __align__(128) unsigned char smem[];

    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const int ld = p.ld;
    const int depth = 1 << log2_depth;
    const uint32_t ring_mask = (uint32_t)depth - 1u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % G;
    const int n_teams = (blockDim.x >> 5) * TPW;
    const int team = warp * TPW + lane / G;
    const int team_base = (lane / G) * G;
    const unsigned team_mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << team_base);
    const size_t stage_elems = tmag_stage_bytes(ld, (int)sizeof(T)) / sizeof(T);
    const size_t head = tmag_head_bytes(n_teams, depth, (int)sizeof(T));
    uint64_t *tbar = reinterpret_cast<uint64_t *>(smem) + (size_t)team * depth;
    T *tval = reinterpret_cast<T *>(smem + (size_t)n_teams * depth * sizeof(uint64_t)) +
              (size_t)team * depth * 4;
    T *tbuf = reinterpret_cast<T *>(smem + head) + (size_t)team * depth * stage_elems;
    double *red = reinterpret_cast<double *>(smem + head +
                                             (size_t)n_teams * depth * stage_elems * sizeof(T));

    const int4 tl = p.tiles[blockIdx.x];
    const int rb = tl.x, re = tl.y, seg = tl.z;
    const Affine<T> shift(p.seg_c[seg], p.seg_inv_d[seg]);
    const int row0 = p.seg_row0[seg];
    const T *__restrict__ xc = p.xc;
    const int32_t *__restrict__ row_ptr = p.row_ptr;
    const int32_t *__restrict__ col_idx = p.col_idx;
    const T *__restrict__ val = p.val;
    T *xn = p.xn;
    const uint32_t batch_bytes = 4u * (uint32_t)ld * (uint32_t)sizeof(T);

    constexpr int NA = PV ? CPT : 1, NJ = PV ? VPT : 1;
    Acc accR[NA][NJ], accS[NA][NJ];
#pragma unroll
    for (int cc = 0; cc < NA; ++cc)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            acc_zero(accR[cc][j]);
            acc_zero(accS[cc][j]);
        }
    bool valid[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) valid[cc] = (g + cc * G) < p.n_chunks;

    if (g == 0) {
        for (int st = 0; st < depth; ++st) mbar_init(&tbar[st], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // Producer position: row p_row, its entries [p_e, p_e1); all team-uniform.
    int p_row = rb + team, p_e = 0, p_e1 = 0;
    if (p_row < re) {
        p_e = __ldg(row_ptr + p_row);
        p_e1 = __ldg(row_ptr + p_row + 1);
    }
    uint32_t n_issued = 0, n_done = 0;
    // Issue batches until the ring is full or the team's rows are exhausted.
    auto produce = [&]() {
        while (n_issued - n_done <= ring_mask) {
            while (p_row < re && p_e >= p_e1) {
                p_row += n_teams;
                if (p_row < re) {
                    p_e = __ldg(row_ptr + p_row);
                    p_e1 = __ldg(row_ptr + p_row + 1);
                }
            }
            if (p_row >= re) return;
            int col[4];
            T a[4];
            team_fetch<T, G, 4>(col_idx, val, p_e, p_e1, g, team_base, team_mask, col, a);
            const uint32_t st = n_issued & ring_mask;
            __syncwarp(team_mask);  // the stage's previous batch has been read by the team
            if (g == 0) {
#pragma unroll
                for (int u = 0; u < 4; ++u) tval[st * 4 + u] = a[u];
                fence_proxy_async_smem();
                mbar_expect_tx(&tbar[st], batch_bytes);
                // tests only: the gather is left out, so the wait runs out with
                // nothing in flight
                if (!p.stall_test)
                    tma_gather4(tbuf + (size_t)st * stage_elems, &tmap, row0 + col[0],
                                row0 + col[1], row0 + col[2], row0 + col[3], &tbar[st]);
            }
            ++n_issued;
            p_e += 4;
        }
    };

    bool timed_out = false;
    for (int row = rb + team; row < re; row += n_teams) {
        const size_t roff = (size_t)row * ld;
        T xk[CPT][VPT], xo[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (valid[cc]) {
                const int off = (g + cc * G) * VPT;
                load16(xc + roff + off, xk[cc]);
                load16(xn + roff + off, xo[cc]);
            }
        }
        const int e0 = __ldg(row_ptr + row), e1 = __ldg(row_ptr + row + 1);
        const int nb = (e1 - e0 + 3) >> 2;
        T y[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
            for (int j = 0; j < VPT; ++j) y[cc][j] = T(0);
        for (int b = 0; b < nb; ++b) {
            produce();
            const uint32_t st = n_done & ring_mask;
            const bool ok = mbar_wait_bounded(&tbar[st], (n_done >> log2_depth) & 1u,
                                              p.spin_cycles);
            if (__any_sync(team_mask, !ok)) {  // the team leaves together
                timed_out = true;
                break;
            }
            const T *buf = tbuf + (size_t)st * stage_elems;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T au = tval[st * 4 + u];
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    if (valid[cc]) {
                        T xv[VPT];
                        load16(buf + (size_t)u * ld + (g + cc * G) * VPT, xv);
#pragma unroll
                        for (int j = 0; j < VPT; ++j) y[cc][j] = fma(au, xv[j], y[cc][j]);
                    }
                }
            }
            ++n_done;
        }
        if (timed_out) break;
        T rr = T(0), ss = T(0);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (!valid[cc]) continue;
            const int off = (g + cc * G) * VPT;
            T xnew[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j)
                xnew[j] = fma(T(2), shift(y[cc][j], xk[cc][j]), -xo[cc][j]);
            store16(xn + roff + off, xnew);
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if constexpr (PV) {
                    acc_add_prod(accR[cc][j], xnew[j], xk[cc][j]);
                    acc_add_prod(accS[cc][j], xnew[j], xnew[j]);
                } else {
                    rr = fma(xnew[j], xk[cc][j], rr);
                    ss = fma(xnew[j], xnew[j], ss);
                }
            }
        }
        if constexpr (!PV) {
            acc_add(accR[0][0], rr);
            acc_add(accS[0][0], ss);
        }
    }
    if (timed_out) {
        // a wait ran out: record it and let the gathers still in flight land (bounded)
        if (g == 0) atomicOr(p.status, 4);
        while (n_done < n_issued) {
            if (!mbar_wait_bounded(&tbar[n_done & ring_mask], (n_done >> log2_depth) & 1u,
                                   p.spin_cycles))
                break;
            ++n_done;
        }
    }
    if constexpr (PV) {
        double *out = p.part + (size_t)blockIdx.x * 2 * p.pv;
        block_reduce_store<Acc, G, CPT, VPT>(accR, out, ld, p.n_chunks, p.pv, red);
        block_reduce_store<Acc, G, CPT, VPT>(accS, out + p.pv, ld, p.n_chunks, p.pv, red);
    } else {
        double *out = p.part + (size_t)blockIdx.x * 2;
        block_reduce_scalar(accR[0][0], out, red);
        block_reduce_scalar(accS[0][0], out + 1, red);
    }
}

// ---- CSR-staged variant -------------------------------------------------------------
// The tile's slice of the matrix is copied into shared memory before its rows are
// walked: row_ptr[rb..re] by the block's threads (coalesced), the column indices and
// values of its nonzeros by two bulk asynchronous copies (cp.async.bulk, the Tensor
// Memory Accelerator's 1-D form) issued by one thread and completing on an mbarrier
// (bounded wait, as in the other staged variants).  A row's nonzeros are then read
// from shared memory -- the same address across a team, a broadcast -- so every
// gather address of a row is known at once: the dependent chain per row shrinks from
// (CSR fetch, then gathers) for every batch of nonzeros to the gathers alone, and the
// CSR registers and shuffles of the direct kernel go away.  The copies run while the
// other blocks resident on the SM compute.  A tile whose slice exceeds the staging
// capacity (kCsrsNnz nonzeros, kCsrsRows rows) reads its CSR from global memory with
// the same arithmetic.  Bulk copies need 16-byte aligned ends: the slice is widened
// to whole 16-byte groups of 4 entries (never past the arrays' last whole group; the
// entries after it are loaded by plain loads).  The capacity is kept small: shared
// memory taken from the L1 costs the gathers their L1 hits (a 4096-entry slice, 45 KB
// per block, dropped the 64^3 lattice's L1 hit rate from 38% to 21%), and the tuner
// picks tile counts whose slices fit.
constexpr int kCsrsNnz = 1024;
constexpr int kCsrsRows = 512;

template <typename T>
__host__ __device__ inline size_t csrs_head_bytes() {
    return 16 + (size_t)(kCsrsRows + 4) * 4 + (size_t)(kCsrsNnz + 8) * 4 +
           (size_t)(kCsrsNnz + 8) * sizeof(T);
}
size_t csrs_smem(int block, int ld, int esz) {
    const size_t head = 16 + (size_t)(kCsrsRows + 4) * 4 + (size_t)(kCsrsNnz + 8) * 4 +
                        (size_t)(kCsrsNnz + 8) * esz;
    return (head + 15) / 16 * 16 + (size_t)(block / 32) * ld * sizeof(double);
}

template <typename T, int G, int CPT, bool PV, int CB>
__global__ void __launch_bounds__(kBlock, 3) step_csrs_kernel(const StepParams<T> p,
                                                              int64_t nnz) {
    constexpr int VPT = CB / (int)sizeof(T);
    using Acc = typename Traits<T>::Acc;
    constexpr int TPW = 32 / G;
    constexpr int U = CPT * CB >= 64 ? 4 : 8;
    extern __shared__ __align__(16) unsigned char csmem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(csmem);
    int32_t *rp_s = reinterpret_cast<int32_t *>(csmem + 16);
    int32_t *col_s = rp_s + kCsrsRows + 4;
    T *val_s = reinterpret_cast<T *>(col_s + kCsrsNnz + 8);
    double *red = reinterpret_cast<double *>(csmem + (csrs_head_bytes<T>() + 15) / 16 * 16);
    __shared__ int s_stop;

    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const int4 tl = p.tiles[blockIdx.x];
    const int rb = tl.x, re = tl.y, seg = tl.z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % G;
    const int n_teams = (blockDim.x >> 5) * TPW;
    const int team = warp * TPW + lane / G;
    const Affine<T> shift(p.seg_c[seg], p.seg_inv_d[seg]);
    const int ld = p.ld;
    const T *__restrict__ xseg = p.xc + (size_t)p.seg_row0[seg] * ld;
    const T *__restrict__ xc = p.xc;
    const int32_t *__restrict__ row_ptr = p.row_ptr;
    T *xn = p.xn;

    // ---- stage the tile's CSR slice ----
    const bool rows_fit = re - rb <= kCsrsRows;
    if (rows_fit)
        for (int r = threadIdx.x; r <= re - rb; r += blockDim.x) rp_s[r] = __ldg(row_ptr + rb + r);
    if (threadIdx.x == 0) s_stop = 0;
    __syncthreads();
    const int64_t e_lo = rows_fit ? rp_s[0] : 0, e_hi = rows_fit ? rp_s[re - rb] : 0;
    const int64_t a0 = e_lo & ~int64_t(3);                    // first staged entry
    const int64_t whole = nnz & ~int64_t(3);                  // end of the last whole group
    const bool staged = rows_fit && (e_hi - a0) <= kCsrsNnz;
    if (staged) {
        const int64_t a1 = min((e_hi + 3) & ~int64_t(3), whole);  // bulk part [a0, a1)
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
            const uint32_t n4 = a1 > a0 ? (uint32_t)(a1 - a0) : 0u;
            // (stall_test: expect 16 bytes that never arrive, so the wait must run out)
            mbar_expect_tx(bar, n4 * (4u + (uint32_t)sizeof(T)) + (p.stall_test ? 16u : 0u));
            if (n4) {
                bulk_copy_g2s(col_s, p.col_idx + a0, n4 * 4u, bar);
                bulk_copy_g2s(val_s, p.val + a0, n4 * (uint32_t)sizeof(T), bar);
            }
        }
        // entries past the last whole group of 4 (at most 3): plain loads
        const int64_t t0 = max(a0, whole);
        if (threadIdx.x < 4 && t0 + threadIdx.x < e_hi) {
            const int64_t e = t0 + threadIdx.x;
            col_s[e - a0] = __ldg(p.col_idx + e);
            val_s[e - a0] = __ldg(p.val + e);
        }
        __syncthreads();  // the barrier is initialised before anyone waits on it
        if (!mbar_wait_bounded(bar, 0, p.spin_cycles)) {
            // give the copies in flight a second (bounded) chance to land before the
            // block moves on and, at exit, hands its shared memory back
            mbar_wait_bounded(bar, 0, p.spin_cycles);
            atomicOr(p.status, 4);
            s_stop = 1;
        }
        __syncthreads();
    }
    const bool stop = s_stop != 0;

    constexpr int NA = PV ? CPT : 1, NJ = PV ? VPT : 1;
    Acc accR[NA][NJ], accS[NA][NJ];
#pragma unroll
    for (int cc = 0; cc < NA; ++cc)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            acc_zero(accR[cc][j]);
            acc_zero(accS[cc][j]);
        }
    bool valid[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) valid[cc] = (g + cc * G) < p.n_chunks;

    for (int row = rb + team; row < re && !stop; row += n_teams) {
        int e0, e1;
        if (staged) {
            e0 = rp_s[row - rb];
            e1 = rp_s[row - rb + 1];
        } else {
            e0 = __ldg(row_ptr + row);
            e1 = __ldg(row_ptr + row + 1);
        }
        const size_t roff = (size_t)row * ld;
        T xk[CPT][VPT], xo[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (valid[cc]) {
                const int off = (g + cc * G) * VPT;
                load_chunk(xc + roff + off, xk[cc]);
                load_chunk_prev(xn + roff + off, xo[cc]);
            }
        }
        T y[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
#pragma unroll
            for (int j = 0; j < VPT; ++j) y[cc][j] = T(0);
        for (int e = e0; e < e1; e += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e + u < e1) {
                    int col;
                    T a;
                    if (staged) {
                        col = col_s[e + u - a0];
                        a = val_s[e + u - a0];
                    } else {
                        col = __ldg(p.col_idx + e + u);
                        a = __ldg(p.val + e + u);
                    }
                    const T *src = xseg + (size_t)col * ld;
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        if (valid[cc]) {
                            T xv[VPT];
                            load_chunk(src + (g + cc * G) * VPT, xv);
#pragma unroll
                            for (int j = 0; j < VPT; ++j) y[cc][j] = fma(a, xv[j], y[cc][j]);
                        }
                    }
                }
            }
        }
        T rr = T(0), ss = T(0);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (!valid[cc]) continue;
            const int off = (g + cc * G) * VPT;
            T xnew[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j)
                xnew[j] = fma(T(2), shift(y[cc][j], xk[cc][j]), -xo[cc][j]);
            store_chunk(xn + roff + off, xnew);
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                if constexpr (PV) {
                    acc_add_prod(accR[cc][j], xnew[j], xk[cc][j]);
                    acc_add_prod(accS[cc][j], xnew[j], xnew[j]);
                } else {
                    rr = fma(xnew[j], xk[cc][j], rr);
                    ss = fma(xnew[j], xnew[j], ss);
                }
            }
        }
        if constexpr (!PV) {
            acc_add(accR[0][0], rr);
            acc_add(accS[0][0], ss);
        }
    }

    if constexpr (PV) {
        double *out = p.part + (size_t)blockIdx.x * 2 * p.pv;
        block_reduce_store<Acc, G, CPT, VPT>(accR, out, ld, p.n_chunks, p.pv, red);
        block_reduce_store<Acc, G, CPT, VPT>(accS, out + p.pv, ld, p.n_chunks, p.pv, red);
    } else {
        double *out = p.part + (size_t)blockIdx.x * 2;
        block_reduce_scalar(accR[0][0], out, red);
        block_reduce_scalar(accS[0][0], out + 1, red);
    }
}

// ---- kernel table --------------------------------------------------------------
template <typename T>
using StepFn = void (*)(const StepParams<T>);

template <typename T>
using CsrsFn = void (*)(const StepParams<T>, int64_t);

template <typename T>
CsrsFn<T> pick_csrs(int G, int CPT, bool per_vec, int cb) {
#define DOS_CASE(GG, CC, BB)                                                                  \
    if (G == GG && CPT == CC && cb == BB)                                                    \
        return per_vec ? step_csrs_kernel<T, GG, CC, true, BB>                               \
                       : step_csrs_kernel<T, GG, CC, false, BB>;
    DOS_CASE(4, 1, 16) DOS_CASE(8, 1, 16) DOS_CASE(16, 1, 16) DOS_CASE(32, 1, 16)
    DOS_CASE(8, 2, 16) DOS_CASE(16, 2, 16) DOS_CASE(32, 2, 16) DOS_CASE(32, 4, 16)
    DOS_CASE(2, 1, 32) DOS_CASE(4, 1, 32) DOS_CASE(4, 2, 32) DOS_CASE(8, 1, 32)
    DOS_CASE(8, 2, 32) DOS_CASE(16, 1, 32) DOS_CASE(16, 2, 32) DOS_CASE(32, 1, 32)
#undef DOS_CASE
    return nullptr;
}

template <typename T>
StepFn<T> pick_staged(int G, int CPT, bool per_vec) {
#define DOS_CASE(GG, CC)                                                                     \
    if (G == GG && CPT == CC)                                                                \
        return per_vec ? step_staged_kernel<T, GG, CC, true> : step_staged_kernel<T, GG, CC, false>;
    DOS_CASE(4, 1) DOS_CASE(8, 1) DOS_CASE(16, 1) DOS_CASE(32, 1)
    DOS_CASE(8, 2) DOS_CASE(16, 2) DOS_CASE(32, 2) DOS_CASE(32, 4)
#undef DOS_CASE
    return nullptr;
}

template <typename T>
using TmagFn = void (*)(const StepParams<T>, const CUtensorMap, int);

template <typename T>
TmagFn<T> pick_tmag(int G, int CPT, bool per_vec) {
#define DOS_CASE(GG, CC)                                                                     \
    if (G == GG && CPT == CC)                                                                \
        return per_vec ? step_tmag_kernel<T, GG, CC, true> : step_tmag_kernel<T, GG, CC, false>;
    DOS_CASE(4, 1) DOS_CASE(8, 1) DOS_CASE(16, 1) DOS_CASE(32, 1)
    DOS_CASE(8, 2) DOS_CASE(16, 2) DOS_CASE(32, 2) DOS_CASE(32, 4)
#undef DOS_CASE
    return nullptr;
}

// The tensor map of one vector block for the gathers: 2-D, n_rows x ld elements,
// row pitch ld * size, boxes of one full row (the TMA box limit of 256 elements
// per dimension holds: panels are at most 256 vectors wide).
using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    });
    return fn;
}
template <typename T>
static CUtensorMap vector_block_map(const T *x, int64_t n_rows, int ld) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) throw Error{DOS_ECUDA, "cuTensorMapEncodeTiled is not available"};
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n_rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
    const cuuint32_t box[2] = {(cuuint32_t)ld, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = enc(&m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                             : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           2, const_cast<T *>(x), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{DOS_ECUDA, "cuTensorMapEncodeTiled rejected the vector block"};
    return m;
}

// Rows per panel of the staged kernel: a multiple of the team count with the four
// slabs within ~64 KB, at most 4 rows per team.
int staged_panel_rows(int block, int team, int ld, int esz) {
    const int n_teams = (block / 32) * (32 / team);
    int rpt = 4;
    while (rpt > 1 && (size_t)4 * n_teams * rpt * ld * esz > (size_t)64 * 1024) --rpt;
    return n_teams * rpt;
}
size_t staged_smem(int block, int team, int ld, int esz) {
    const int R = staged_panel_rows(block, team, ld, esz);
    return 128 + (size_t)4 * R * ld * esz + (size_t)(block / 32) * ld * sizeof(double);
}

template <typename T>
StepFn<T> pick(int G, int CPT, bool per_vec, int cb = 16) {
#define DOS_CASE(GG, CC, BB)                                                                  \
    if (G == GG && CPT == CC && cb == BB)                                                    \
        return per_vec ? step_kernel<T, GG, CC, true, BB, false>                             \
                       : step_kernel<T, GG, CC, false, BB, false>;
#define DOS_CASES(GG) DOS_CASE(GG, 1, 16) DOS_CASE(GG, 2, 16) DOS_CASE(GG, 4, 16)
    DOS_CASES(1) DOS_CASES(2) DOS_CASES(4) DOS_CASES(8) DOS_CASES(16) DOS_CASES(32)
    // 32-byte chunks: the team shapes that cover 32 to 1024 vector bytes per row
    DOS_CASE(1, 1, 32) DOS_CASE(2, 1, 32) DOS_CASE(2, 2, 32) DOS_CASE(4, 1, 32)
    DOS_CASE(4, 2, 32) DOS_CASE(8, 1, 32) DOS_CASE(8, 2, 32) DOS_CASE(16, 1, 32)
    DOS_CASE(16, 2, 32) DOS_CASE(32, 1, 32)
#undef DOS_CASES
#undef DOS_CASE
    return nullptr;
}

// The first step (k = 0) of a sweep with direct loads: one fixed shape that
// covers any panel (teams of 32 threads, 16-byte chunks: 256 floats or doubles
// per row), the same tiles and partial-sum layout as the shape of the later steps.
constexpr int kFirstTeam = 32;
template <typename T>
constexpr int first_chunks() { return sizeof(T) == 4 ? 2 : 4; }
template <typename T>
StepFn<T> pick_first(bool per_vec) {
    return per_vec ? step_kernel<T, kFirstTeam, first_chunks<T>(), true, 16, true>
                   : step_kernel<T, kFirstTeam, first_chunks<T>(), false, 16, true>;
}

size_t step_smem(int block, int ld) { return (size_t)(block / 32) * ld * sizeof(double); }

// ---- tiles ---------------------------------------------------------------------
__device__ __forceinline__ int64_t tile_boundary(const int32_t *row_ptr, int R0, int R1, int j,
                                                 int T, int row_cost) {
    if (j <= 0) return R0;
    if (j >= T) return R1;
    const int64_t base = row_ptr[R0];
    const int64_t total = (int64_t)(row_ptr[R1] - base) + (int64_t)row_cost * (R1 - R0);
    // smallest r in [R0, R1] with cost(r) * T >= j * total
    int lo = R0, hi = R1;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const int64_t cost = (int64_t)(row_ptr[mid] - base) + (int64_t)row_cost * (mid - R0);
        if (cost * T >= (int64_t)j * total) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__global__ void make_tiles_kernel(const int32_t *__restrict__ row_ptr, int B,
                                  const int32_t *__restrict__ seg_row0,
                                  const int32_t *__restrict__ seg_tile_begin, int n_tiles,
                                  int row_cost, int4 *__restrict__ tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    int lo = 0, hi = B;  // seg_tile_begin[lo] <= t < seg_tile_begin[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (seg_tile_begin[mid] <= t) lo = mid; else hi = mid;
    }
    const int T = seg_tile_begin[lo + 1] - seg_tile_begin[lo];
    const int j = t - seg_tile_begin[lo];
    const int R0 = seg_row0[lo], R1 = seg_row0[lo + 1];
    tiles[t] = make_int4((int)tile_boundary(row_ptr, R0, R1, j, T, row_cost),
                         (int)tile_boundary(row_ptr, R0, R1, j + 1, T, row_cost), lo, 0);
}

// ---- reduction over tiles (step a5) ---------------------------------------------
// grid.x = count*2 (step, dot), grid.y = segment.  partial slices are [slot][tile][2][pv].
__global__ void reduce_kernel(const double *__restrict__ partial, int n_tiles, int pv, int ncols,
                              const int32_t *__restrict__ seg_tile_begin, int k0, int slot0,
                              int slots, int steps_total, int col_offset, int dst_pv,
                              int accumulate, double *__restrict__ dotsum) {
    __shared__ double sh[32];
    const int kk = blockIdx.x >> 1, dot = blockIdx.x & 1, seg = blockIdx.y;
    const int k = k0 + kk;
    const int slot = (slot0 + kk) % slots;
    const int tb = seg_tile_begin[seg], te = seg_tile_begin[seg + 1];
    const double *src = partial + (size_t)slot * n_tiles * 2 * pv;
    double *dst = dotsum + (((size_t)seg * steps_total + k) * 2 + dot) * dst_pv;
    if (pv > 1) {
        for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
            double s = 0.0;
            for (int t = tb; t < te; ++t) s += src[((size_t)t * 2 + dot) * pv + col];
            dst[col_offset + col] = s;
        }
    } else {
        double s = 0.0;
        for (int t = tb + threadIdx.x; t < te; t += blockDim.x) s += src[(size_t)t * 2 + dot];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
            dst[0] = accumulate ? dst[0] + tot : tot;
        }
    }
}

// mu_0 partials: [tile][pv] -> dotsum0[seg][dst_pv]
__global__ void reduce0_kernel(const double *__restrict__ part0, int pv, int ncols,
                               const int32_t *__restrict__ seg_tile_begin, int col_offset,
                               int dst_pv, int accumulate, double *__restrict__ dotsum0) {
    __shared__ double sh[32];
    const int seg = blockIdx.x;
    const int tb = seg_tile_begin[seg], te = seg_tile_begin[seg + 1];
    double *dst = dotsum0 + (size_t)seg * dst_pv;
    if (pv > 1) {
        for (int col = threadIdx.x; col < ncols; col += blockDim.x) {
            double s = 0.0;
            for (int t = tb; t < te; ++t) s += part0[(size_t)t * pv + col];
            dst[col_offset + col] = s;
        }
    } else {
        double s = 0.0;
        for (int t = tb + threadIdx.x; t < te; t += blockDim.x) s += part0[t];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
            dst[0] = accumulate ? dst[0] + tot : tot;
        }
    }
}

// ---- moments from dot products (step a5) -------------------------------------------
// dotsum[seg][k][2][pvt], dotsum0[seg][pvt]; pvt = n_v (per-vector) or 1 (totals).
__device__ __forceinline__ double moment_from(int k, double z, const double *ds, int pvt,
                                              int col, double N, double mu0, double mu1) {
    if (k == 0) return z / N;
    const int step = (k - 1) >> 1;       // step producing mu_k
    const int dot = (k & 1) ? 0 : 1;     // odd k: r (X_{s+1}.X_s), even: s (X_{s+1}.X_{s+1})
    const double v = ds[((size_t)step * 2 + dot) * pvt + col];
    if (k == 1) return v / N;
    return 2.0 * v / N - ((k & 1) ? mu1 : mu0);
}

__global__ void finalize_kernel(const double *__restrict__ dotsum,
                                const double *__restrict__ dotsum0,
                                const int32_t *__restrict__ seg_row0, int M, int steps_total,
                                int n_v, int pvt, double *__restrict__ mu,
                                double *__restrict__ mu_pv, double tol, int *status) {
    const int seg = blockIdx.x;
    const double n = (double)(seg_row0[seg + 1] - seg_row0[seg]);
    const double *ds = dotsum + (size_t)seg * steps_total * 2 * pvt;
    const double *d0 = dotsum0 + (size_t)seg * pvt;
    // totals
    __shared__ double tot_z, tot_r0;
    if (threadIdx.x == 0) {
        double z = 0.0, r0 = 0.0;
        for (int l = 0; l < pvt; ++l) {
            z += d0[l];
            r0 += ds[l];  // step 0, dot 0
        }
        tot_z = z;
        tot_r0 = r0;
    }
    __syncthreads();
    const double N = n * (double)n_v;
    const double mu0 = tot_z / N, mu1 = tot_r0 / N;
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
        double m;
        if (pvt == 1) {
            m = moment_from(k, tot_z, ds, 1, 0, N, mu0, mu1);
        } else if (k == 0) {
            m = mu0;
        } else {
            const int step = (k - 1) >> 1, dot = (k & 1) ? 0 : 1;
            double v = 0.0;
            for (int l = 0; l < pvt; ++l) v += ds[((size_t)step * 2 + dot) * pvt + l];
            m = (k == 1) ? v / N : 2.0 * v / N - ((k & 1) ? mu1 : mu0);
        }
        mu[(size_t)seg * (M + 1) + k] = m;
        if (!(fabs(m) <= mu0 * (1.0 + tol))) atomicOr(status, 2);
    }
    if (mu_pv != nullptr) {  // per-vector dot sums are stored (pvt == n_v, also when 1)
        for (int idx = threadIdx.x; idx < n_v * (M + 1); idx += blockDim.x) {
            const int l = idx / (M + 1), k = idx - l * (M + 1);
            const double z = d0[l];
            const double m0 = z / n, m1 = ds[l] / n;
            mu_pv[((size_t)seg * n_v + l) * (M + 1) + k] =
                moment_from(k, z, ds, pvt, l, n, m0, m1);
        }
    }
}

__global__ void f64_to_f32_kernel(const double *__restrict__ in, float *__restrict__ out,
                                  int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void validate_kernel(int64_t n_rows, int64_t nnz, const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col_idx, int B,
                                const int32_t *__restrict__ seg_row0, int *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[i], b = row_ptr[i + 1];
        if (i == 0 && a != 0) { atomicOr(flag, 1); continue; }
        if (i == n_rows - 1 && b != nnz) { atomicOr(flag, 1); continue; }
        if (b < a || a < 0 || b > nnz) { atomicOr(flag, 1); continue; }
        int lo = 0, hi = B;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (seg_row0[mid] <= i) lo = mid; else hi = mid;
        }
        const int64_t n_seg = seg_row0[lo + 1] - seg_row0[lo];
        for (int64_t e = a; e < b; ++e) {
            const int32_t cidx = col_idx[e];
            if (cidx < 0 || cidx >= n_seg) { atomicOr(flag, 1); break; }
        }
    }
}

int grid_for(int64_t work, int block, int cap) {
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int tmag_depth(int block, int team, int ld, int esz, int asked) {
    return tmag_ring_depth(block, team, ld, esz, asked);
}

// ---- launchers -------------------------------------------------------------------
void launch_validate_csr(int64_t n_rows, int64_t nnz, const int32_t *row_ptr,
                         const int32_t *col_idx, int B, const int32_t *seg_row0, int *flag,
                         cudaStream_t s) {
    validate_kernel<<<grid_for(n_rows, 256, 65535), 256, 0, s>>>(n_rows, nnz, row_ptr, col_idx,
                                                                  B, seg_row0, flag);
    DOS_LAUNCHED();
}

void launch_f64_to_f32(const double *in, float *out, int64_t count, cudaStream_t s) {
    f64_to_f32_kernel<<<grid_for(count, 256, 65535), 256, 0, s>>>(in, out, count);
    DOS_LAUNCHED();
}

void launch_make_tiles(const int32_t *row_ptr, int B, const int32_t *seg_row0,
                       const int32_t *seg_tile_begin, int n_tiles, int row_cost, int4 *tiles,
                       cudaStream_t s) {
    make_tiles_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(row_ptr, B, seg_row0, seg_tile_begin,
                                                            n_tiles, row_cost, tiles);
    DOS_LAUNCHED();
}

bool shape_supported(int precision, const Shape &sh, int ld) {
    const int esz = precision == DOS_PREC_F64 ? 8 : 4;
    if (sh.block != kBlock) return false;
    if (sh.team < 1 || sh.team > 32 || (sh.team & (sh.team - 1))) return false;
    if (sh.chunks != 1 && sh.chunks != 2 && sh.chunks != 4) return false;
    if (sh.tiles < 1) return false;
    if (sh.staged < 0 || sh.staged > 3) return false;
    if (sh.cb != 16 && sh.cb != 32) return false;
    const int vpt = sh.cb / esz;
    if (sh.cb == 32) {  // 256-bit accesses: direct loads, rows of whole 32-byte chunks
        if ((sh.staged != 0 && sh.staged != 3) || ld % vpt != 0) return false;
        if (sh.staged == 0 &&
            !(precision == DOS_PREC_F64 ? (void *)pick<double>(sh.team, sh.chunks, false, 32)
                                        : (void *)pick<float>(sh.team, sh.chunks, false, 32)))
            return false;
    }
    if (sh.staged == 3 &&
        !(precision == DOS_PREC_F64 ? (void *)pick_csrs<double>(sh.team, sh.chunks, false, sh.cb)
                                    : (void *)pick_csrs<float>(sh.team, sh.chunks, false, sh.cb)))
        return false;
    if (sh.staged == 1 &&
        !(precision == DOS_PREC_F64 ? (void *)pick_staged<double>(sh.team, sh.chunks, false)
                                    : (void *)pick_staged<float>(sh.team, sh.chunks, false)))
        return false;
    if (sh.staged == 2) {  // TMA gathers: 16-byte chunks, rows of at most 256 elements
        if (sh.cb != 16 || ld > 256) return false;
        if (!(precision == DOS_PREC_F64 ? (void *)pick_tmag<double>(sh.team, sh.chunks, false)
                                        : (void *)pick_tmag<float>(sh.team, sh.chunks, false)))
            return false;
        if (sh.depth != 0 && sh.depth != 2 && sh.depth != 4 && sh.depth != 8) return false;
        const int depth = tmag_ring_depth(sh.block, sh.team, ld, esz, sh.depth);
        if (tmag_smem(sh.block, sh.team, ld, esz, depth) > (size_t)227 * 1024) return false;
    } else if (sh.depth != 0) {
        return false;  // the ring depth belongs to the TMA-gather variant
    }
    return sh.team * sh.chunks * vpt >= ld;
}

// Opt in to more than 48 KB of dynamic shared memory (per kernel, per device;
// remembered so the driver is asked once per size).
static void allow_smem_fn(const void *fn, size_t bytes);
template <typename T>
static void allow_smem(StepFn<T> fn, size_t bytes) {
    allow_smem_fn((const void *)fn, bytes);
}
static void allow_smem_fn(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int>, size_t> granted;
    int dev = 0;
    DOS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t &g = granted[std::make_tuple((const void *)fn, dev)];
    if (g >= bytes) return;
    DOS_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
    g = bytes;
}

template <typename T>
static int occupancy_t(const Shape &sh, int ld) {
    int nb = 0;
    if (sh.staged == 1) {
        auto fn = pick_staged<T>(sh.team, sh.chunks, false);
        if (!fn) return 0;
        const size_t sm = staged_smem(sh.block, sh.team, ld, sizeof(T));
        allow_smem<T>(fn, sm);
        DOS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.block, sm));
    } else if (sh.staged == 2) {
        auto fn = pick_tmag<T>(sh.team, sh.chunks, false);
        if (!fn) return 0;
        const int esz = (int)sizeof(T);
        const size_t sm = tmag_smem(sh.block, sh.team, ld, esz,
                                    tmag_ring_depth(sh.block, sh.team, ld, esz, sh.depth));
        allow_smem_fn((const void *)fn, sm);
        DOS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.block, sm));
    } else if (sh.staged == 3) {
        auto fn = pick_csrs<T>(sh.team, sh.chunks, false, sh.cb);
        if (!fn) return 0;
        const size_t sm = csrs_smem(sh.block, ld, (int)sizeof(T));
        allow_smem_fn((const void *)fn, sm);
        DOS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.block, sm));
    } else {
        auto fn = pick<T>(sh.team, sh.chunks, false, sh.cb);
        if (!fn) return 0;
        DOS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sh.block,
                                                                    step_smem(sh.block, ld)));
    }
    return nb;
}

int max_active_blocks(int precision, const Shape &sh, int ld) {
    return precision == DOS_PREC_F64 ? occupancy_t<double>(sh, ld) : occupancy_t<float>(sh, ld);
}

Shape default_shape(int precision, int ld, int num_sms, int64_t n_rows) {
    const int vpt = precision == DOS_PREC_F64 ? 2 : 4;
    const int chunks = ld / vpt;
    Shape sh;
    sh.block = kBlock;
    if (chunks <= 32) {
        int g = 1;
        while (g < chunks) g <<= 1;
        sh.team = g;
        sh.chunks = 1;
    } else {
        sh.team = 32;
        sh.chunks = chunks <= 64 ? 2 : 4;
    }
    const int occ = max_active_blocks(precision, sh, ld);
    const int teams = (kBlock / 32) * (32 / sh.team);
    int64_t tiles = (int64_t)num_sms * (occ > 0 ? occ : 1);
    const int64_t max_tiles = (n_rows + teams - 1) / teams;
    if (tiles > max_tiles) tiles = max_tiles;
    if (tiles < 1) tiles = 1;
    sh.tiles = (int)tiles;
    return sh;
}

void launch_init_vectors(const SweepArgs &a, cudaStream_t s) {
    const int vpt = a.precision == DOS_PREC_F64 ? 2 : 4;
    const int64_t work = a.n_rows * (a.ld / vpt);
    const int grid = grid_for(work, 256, 152 * 32);
    if (a.precision == DOS_PREC_F64)
        init_vectors_kernel<double><<<grid, 256, 0, s>>>((double *)a.x0, a.n_rows, a.ld, a.n_v,
                                                         a.B, a.seg_row0, a.seed, a.vec_offset,
                                                         a.batch_index);
    else
        init_vectors_kernel<float><<<grid, 256, 0, s>>>((float *)a.x0, a.n_rows, a.ld, a.n_v, a.B,
                                                        a.seg_row0, a.seed, a.vec_offset,
                                                        a.batch_index);
    DOS_LAUNCHED();
}

template <typename T>
static void launch_step_t(const SweepArgs &a, int k, int slot, cudaStream_t s) {
    StepParams<T> p;
    p.row_ptr = a.row_ptr;
    p.col_idx = a.col_idx;
    p.val = (const T *)a.val;
    T *blk[2] = {(T *)a.x0, (T *)a.x1};
    p.xc = blk[k & 1];
    p.xn = blk[(k + 1) & 1];
    p.ld = a.ld;
    p.n_chunks = a.ld / (a.shape.cb / (int)sizeof(T));
    p.pv = a.per_vec ? a.ld : 1;
    p.first = k == 0;
    p.tiles = a.tiles;
    p.seg_row0 = a.seg_row0;
    p.seg_c = a.seg_c;
    p.seg_inv_d = a.seg_inv_d;
    p.part = a.partial + (size_t)slot * a.n_tiles * 2 * p.pv;
    p.part0 = a.partial0;
    p.status = a.status;
    p.spin_cycles = a.spin_cycles > 0 ? a.spin_cycles : 2000000000LL;  // ~1 s
    p.stall_test = a.stall_test;
    p.rev = k & 1;
    if (a.shape.staged == 1) {
        auto fn = pick_staged<T>(a.shape.team, a.shape.chunks, a.per_vec != 0);
        if (!fn) throw Error{DOS_EINVAL, "unsupported staged launch shape"};
        p.panel_rows = staged_panel_rows(a.shape.block, a.shape.team, a.ld, sizeof(T));
        const size_t sm = staged_smem(a.shape.block, a.shape.team, a.ld, sizeof(T));
        allow_smem<T>(fn, sm);
        fn<<<a.n_tiles, a.shape.block, sm, s>>>(p);
    } else if (a.shape.staged == 3 && k > 0) {
        auto fn = pick_csrs<T>(a.shape.team, a.shape.chunks, a.per_vec != 0, a.shape.cb);
        if (!fn) throw Error{DOS_EINVAL, "unsupported CSR-staged launch shape"};
        if (((uintptr_t)a.col_idx & 15) || ((uintptr_t)a.val & 15))
            throw Error{DOS_EINVAL, "the CSR-staged variant needs col_idx and val 16-byte aligned"};
        p.panel_rows = 0;
        const size_t sm = csrs_smem(a.shape.block, a.ld, (int)sizeof(T));
        allow_smem_fn((const void *)fn, sm);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)a.n_tiles);
        cfg.blockDim = dim3((unsigned)a.shape.block);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = a.pdl ? 1 : 0;
        DOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, p, (int64_t)a.nnz));
    } else if (a.shape.staged == 2 && k > 0) {
        auto fn = pick_tmag<T>(a.shape.team, a.shape.chunks, a.per_vec != 0);
        if (!fn) throw Error{DOS_EINVAL, "unsupported TMA-gather launch shape"};
        p.panel_rows = 0;
        const CUtensorMap tmap = vector_block_map<T>(p.xc, a.n_rows, a.ld);
        const int esz = (int)sizeof(T);
        const int depth = tmag_ring_depth(a.shape.block, a.shape.team, a.ld, esz, a.shape.depth);
        const int log2_depth = depth == 8 ? 3 : depth == 4 ? 2 : 1;
        const size_t sm = tmag_smem(a.shape.block, a.shape.team, a.ld, esz, depth);
        allow_smem_fn((const void *)fn, sm);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)a.n_tiles);
        cfg.blockDim = dim3((unsigned)a.shape.block);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = a.pdl ? 1 : 0;
        DOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, p, tmap, log2_depth));
    } else {
        // direct loads; also the first step of the TMA-gather variant
        auto fn = k == 0 ? pick_first<T>(a.per_vec != 0)
                         : pick<T>(a.shape.team, a.shape.chunks, a.per_vec != 0, a.shape.cb);
        if (!fn) throw Error{DOS_EINVAL, "unsupported launch shape"};
        if (k == 0) {
            if (kFirstTeam * first_chunks<T>() * (16 / (int)sizeof(T)) < a.ld)
                throw Error{DOS_EINVAL, "vector panel wider than the first-step kernel covers"};
            p.n_chunks = a.ld / (16 / (int)sizeof(T));
        }
        p.panel_rows = 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)a.n_tiles);
        cfg.blockDim = dim3((unsigned)a.shape.block);
        cfg.dynamicSmemBytes = step_smem(a.shape.block, a.ld);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = a.pdl ? 1 : 0;
        DOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, p));
    }
    DOS_LAUNCHED();
}

// ---- block Lanczos product (Section 3.2.1) with the fused step's data mapping -----
// w = A u_j - c_j u_{j-1} for n_vec runs at once (FP64), written over u_{j-1}, and
// per-block partial sums of u_j . w per column (c_prev: c_j per column, NULL for
// no previous term).  The Lanczos loop keeps its vectors unnormalised
// (q_j = s_j u_j), so with the right c_j this is q_j's product divided by s_j:
// one FMA per element after the gathers, as for normalised vectors.  A team
// of G threads shares a matrix row, each thread owning CPT chunks of CB bytes of
// the row of Q; CSR entries are fetched once per team and shared by shuffles.
template <int G, int CPT, int CB>
__global__ void __launch_bounds__(kBlock, 3) lanczos_team_spmm_kernel(
    int64_t n, int ld, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
    const double *__restrict__ val, const double *__restrict__ q, double *__restrict__ qprev_w,
    const double *__restrict__ c_prev, double *__restrict__ part) {
    constexpr int VPT = CB / 8;
    constexpr int TPW = 32 / G;
    constexpr int U = CPT * CB >= 64 ? 4 : 8;
    extern __shared__ double red[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % G;
    const int n_teams = (blockDim.x >> 5) * TPW;
    const int team = warp * TPW + lane / G;
    const int team_base = (lane / G) * G;
    const unsigned team_mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << team_base);
    const int n_chunks = ld / VPT;
    bool valid[CPT];
    double bp[CPT][VPT], acc[CPT][VPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        valid[cc] = (g + cc * G) < n_chunks;
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            bp[cc][j] = (c_prev && valid[cc]) ? c_prev[(g + cc * G) * VPT + j] : 0.0;
            acc[cc][j] = 0.0;
        }
    }
    for (int64_t row = (int64_t)blockIdx.x * n_teams + team; row < n;
         row += (int64_t)gridDim.x * n_teams) {
        const size_t roff = (size_t)row * ld;
        const int e0 = __ldg(row_ptr + row), e1 = __ldg(row_ptr + row + 1);
        double xk[CPT][VPT], xo[CPT][VPT], y[CPT][VPT];
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (valid[cc]) {
                const int off = (g + cc * G) * VPT;
                load_chunk(q + roff + off, xk[cc]);
                load_chunk_prev(qprev_w + roff + off, xo[cc]);
            }
#pragma unroll
            for (int j = 0; j < VPT; ++j) y[cc][j] = 0.0;
        }
        for (int e = e0; e < e1; e += U) {
            int col[U];
            double a[U];
            team_fetch<double, G, U>(col_idx, val, e, e1, g, team_base, team_mask, col, a);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e + u < e1) {
                    const double *src = q + (size_t)col[u] * ld;
#pragma unroll
                    for (int cc = 0; cc < CPT; ++cc) {
                        if (valid[cc]) {
                            double xv[VPT];
                            load_chunk(src + (g + cc * G) * VPT, xv);
#pragma unroll
                            for (int j = 0; j < VPT; ++j) y[cc][j] = fma(a[u], xv[j], y[cc][j]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            if (!valid[cc]) continue;
            double w[VPT];
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                w[j] = y[cc][j] - bp[cc][j] * xo[cc][j];
                acc[cc][j] = fma(xk[cc][j], w[j], acc[cc][j]);
            }
            store_chunk(qprev_w + roff + (g + cc * G) * VPT, w);
        }
    }
    block_reduce_store<double, G, CPT, VPT>(acc, part + (size_t)blockIdx.x * ld, ld, n_chunks, ld,
                                            red);
}

using LanczosFn = void (*)(int64_t, int, const int32_t *, const int32_t *, const double *,
                           const double *, double *, const double *, double *);
static LanczosFn pick_lanczos(int G, int CPT, int CB) {
#define DOS_LZ(GG, CC, BB) \
    if (G == GG && CPT == CC && CB == BB) return lanczos_team_spmm_kernel<GG, CC, BB>;
    DOS_LZ(1, 1, 16) DOS_LZ(2, 1, 16) DOS_LZ(4, 1, 16) DOS_LZ(8, 1, 16) DOS_LZ(16, 1, 16)
    DOS_LZ(32, 1, 16) DOS_LZ(32, 2, 16) DOS_LZ(32, 4, 16)
    DOS_LZ(1, 1, 32) DOS_LZ(2, 1, 32) DOS_LZ(4, 1, 32) DOS_LZ(8, 1, 32) DOS_LZ(16, 1, 32)
    DOS_LZ(32, 1, 32) DOS_LZ(32, 2, 32)
#undef DOS_LZ
    return nullptr;
}

// Smallest team (then chunk count) covering the padded row: 32-byte chunks when
// the row is whole 32-byte chunks.
static void lanczos_shape(int ld, int *G, int *CPT, int *CB) {
    *CB = ld % 4 == 0 ? 32 : 16;
    const int chunks = ld / (*CB / 8);
    int g = 1;
    while (g < chunks && g < 32) g <<= 1;
    int c = 1;
    while (g * c < chunks) c <<= 1;
    *G = g;
    *CPT = c;
}

int lanczos_team_blocks(int num_sms, int64_t n, int ld) {
    int G, CPT, CB;
    lanczos_shape(ld, &G, &CPT, &CB);
    const int64_t teams = (int64_t)(kBlock / 32) * (32 / G);
    const int64_t b = (n + teams - 1) / teams;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 6));
}

void launch_lanczos_team_spmm(int64_t n, int ld, const int32_t *row_ptr, const int32_t *col_idx,
                              const double *val, const double *q, double *qprev_w,
                              const double *c_prev, double *part, int n_blocks,
                              cudaStream_t s) {
    int G, CPT, CB;
    lanczos_shape(ld, &G, &CPT, &CB);
    LanczosFn fn = pick_lanczos(G, CPT, CB);
    if (!fn) throw Error{DOS_EINVAL, "no Lanczos product kernel for this vector block"};
    fn<<<n_blocks, kBlock, step_smem(kBlock, ld), s>>>(n, ld, row_ptr, col_idx, val, q, qprev_w,
                                                       c_prev, part);
    DOS_LAUNCHED();
}

void launch_step(const SweepArgs &a, int k, int slot, cudaStream_t s) {
    if (a.precision == DOS_PREC_F64) launch_step_t<double>(a, k, slot, s);
    else launch_step_t<float>(a, k, slot, s);
}

void launch_reduce(const double *partial, int n_tiles, int pv, int ncols, int B,
                   const int32_t *seg_tile_begin, int k0, int count, int slot0, int slots,
                   int steps_total, int col_offset, int dst_pv, int accumulate, double *dotsum,
                   cudaStream_t s) {
    if (count <= 0) return;
    dim3 grid(count * 2, B);
    reduce_kernel<<<grid, 256, 0, s>>>(partial, n_tiles, pv, ncols, seg_tile_begin, k0, slot0,
                                       slots, steps_total, col_offset, dst_pv, accumulate, dotsum);
    DOS_LAUNCHED();
}

void launch_reduce0(const double *part0, int pv, int ncols, int B, const int32_t *seg_tile_begin,
                    int col_offset, int dst_pv, int accumulate, double *dotsum0, cudaStream_t s) {
    reduce0_kernel<<<B, 256, 0, s>>>(part0, pv, ncols, seg_tile_begin, col_offset, dst_pv,
                                     accumulate, dotsum0);
    DOS_LAUNCHED();
}

void launch_finalize(const double *dotsum, const double *dotsum0, const int32_t *seg_row0, int B,
                     int M, int steps_total, int n_v, int pvt, double *mu, double *mu_pv,
                     double tol, int *status, cudaStream_t s) {
    finalize_kernel<<<B, 256, 0, s>>>(dotsum, dotsum0, seg_row0, M, steps_total, n_v, pvt, mu,
                                      mu_pv, tol, status);
    DOS_LAUNCHED();
}

}  // namespace dos
