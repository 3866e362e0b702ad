// Host side of the C ABI declared in include/dos.h: argument checks, CSR
// staging and validation, the sweep plan (tiles, vector panels, partial-sum
// slots), launch sequencing, the CUDA-graph cache and the autotuner.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "dos_internal.h"

using namespace dos;

std::atomic<int64_t> dos::g_launch_count{0};

namespace {

constexpr int kPanelMax = 256;        // vectors per pass over A
constexpr int kRowCost = 3;           // tile cost of one row, in nonzeros
constexpr size_t kPartialCap = size_t(512) << 20;  // bytes of per-step partial sums kept

int fail(dos_ctx *ctx, const Error &e) {
    if (ctx) ctx->last_error = e.msg;
    return e.status;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) DOS_CUDA_TRY(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename F>
int guarded(dos_ctx *ctx, F &&f) {
    if (!ctx) return DOS_EINVAL;
    try {
        DeviceGuard g(ctx->device);
        f();
        ctx->last_error.clear();
        return DOS_OK;
    } catch (const Error &e) {
        return fail(ctx, e);
    } catch (const std::bad_alloc &) {
        return fail(ctx, Error{DOS_ENOMEM, "host allocation failed"});
    }
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from device scratch to a caller buffer of either kind.
void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    DOS_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

struct DevCSR {
    int64_t n, nnz;
    const int32_t *row_ptr, *col_idx;
    const void *val;
    int dtype;
    const int32_t *host_row_ptr;  // non-null when the caller passed host arrays
};

DevCSR stage_csr(dos_ctx *ctx, const dos_csr *A, cudaStream_t s) {
    DOS_REQUIRE(A != nullptr, "matrix descriptor is NULL");
    DOS_REQUIRE(A->n >= 1 && A->n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    DOS_REQUIRE(A->nnz >= 0 && A->nnz < (int64_t(1) << 31), "nnz must be in [0, 2^31)");
    DOS_REQUIRE(A->dtype == DOS_F64 || A->dtype == DOS_F32, "dtype must be DOS_F64 or DOS_F32");
    DOS_REQUIRE(A->location == DOS_DEVICE || A->location == DOS_HOST, "bad location");
    DOS_REQUIRE(A->row_ptr != nullptr, "row_ptr is NULL");
    DOS_REQUIRE(A->nnz == 0 || (A->col_idx != nullptr && A->val != nullptr),
                "col_idx / val is NULL");
    DevCSR d{A->n, A->nnz, A->row_ptr, A->col_idx, A->val, A->dtype, nullptr};
    if (A->location == DOS_HOST) {
        const size_t es = A->dtype == DOS_F64 ? 8 : 4;
        void *rp = ctx->csr_rowptr.get((A->n + 1) * sizeof(int32_t));
        void *ci = ctx->csr_colidx.get(std::max<int64_t>(A->nnz, 1) * sizeof(int32_t));
        void *va = ctx->csr_val.get(std::max<int64_t>(A->nnz, 1) * es);
        DOS_CUDA_TRY(cudaMemcpyAsync(rp, A->row_ptr, (A->n + 1) * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, s));
        if (A->nnz) {
            DOS_CUDA_TRY(cudaMemcpyAsync(ci, A->col_idx, A->nnz * sizeof(int32_t),
                                         cudaMemcpyHostToDevice, s));
            DOS_CUDA_TRY(cudaMemcpyAsync(va, A->val, A->nnz * es, cudaMemcpyHostToDevice, s));
        }
        d.row_ptr = (const int32_t *)rp;
        d.col_idx = (const int32_t *)ci;
        d.val = va;
        d.host_row_ptr = A->row_ptr;
    }
    return d;
}

// Segment table on the device: seg_row0 (B+1 int32), seg_tile_begin (B+1 int32),
// seg_c (B doubles), seg_inv_d (B doubles), validation/status flags (4 ints).
struct SegDev {
    int32_t *row0, *tile_begin;
    double *c, *inv_d;
};

SegDev upload_segments(dos_ctx *ctx, const std::vector<int32_t> &row0,
                       const std::vector<int32_t> &tile_begin, const std::vector<double> &c,
                       const std::vector<double> &inv_d, cudaStream_t s) {
    const int B = (int)c.size();
    const size_t ints = ((2 * (size_t)(B + 1)) + 1) & ~size_t(1);  // keep doubles 8-aligned
    const size_t bytes = ints * 4 + 2 * (size_t)B * 8;
    uint8_t *dev = (uint8_t *)ctx->segs.get(bytes);
    uint8_t *host = (uint8_t *)ctx->host_stage.get(bytes);
    memcpy(host, row0.data(), (B + 1) * 4);
    memcpy(host + (B + 1) * 4, tile_begin.data(), (B + 1) * 4);
    memcpy(host + ints * 4, c.data(), B * 8);
    memcpy(host + ints * 4 + B * 8, inv_d.data(), B * 8);
    DOS_CUDA_TRY(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s));
    // the pinned staging buffer is reused by the next call: wait for the copy
    DOS_CUDA_TRY(cudaStreamSynchronize(s));
    SegDev d;
    d.row0 = (int32_t *)dev;
    d.tile_begin = (int32_t *)(dev + (B + 1) * 4);
    d.c = (double *)(dev + ints * 4);
    d.inv_d = (double *)(dev + ints * 4 + B * 8);
    return d;
}

int *status_flags(dos_ctx *ctx) { return (int *)ctx->status.get(4 * sizeof(int)); }

// Under stream capture an event record must be flagged "external" to become an
// event node of the graph (otherwise it only marks a capture-internal
// dependency); outside capture that flag is rejected, so pick per call.
void record_timing_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    DOS_CUDA_TRY(cudaStreamIsCapturing(s, &st));
    if (st == cudaStreamCaptureStatusActive)
        DOS_CUDA_TRY(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else
        DOS_CUDA_TRY(cudaEventRecord(e, s));
}

void validate_on_device(dos_ctx *ctx, const DevCSR &A, int B, const int32_t *seg_row0_dev,
                        cudaStream_t s) {
    int *flag = status_flags(ctx) + 1;
    DOS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    launch_validate_csr(A.n, A.nnz, A.row_ptr, A.col_idx, B, seg_row0_dev, flag, s);
    int h = 0;
    DOS_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    DOS_CUDA_TRY(cudaStreamSynchronize(s));
    DOS_REQUIRE(h == 0, "CSR structure check failed (row_ptr not monotone / not ending at nnz, "
                        "or a column index out of range)");
}

struct SweepRequest {
    int B;
    std::vector<int64_t> seg_rows;  // B+1
    std::vector<double> lb, ub;     // B
    int M, n_v;
    uint64_t seed;
    int precision;
    double *mu, *mu_pv;
    dos_kpm_opts opts;
};

Shape tune_shape(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows, int n_v,
                 int precision, double *best_ms, cudaStream_t s);

// Vector panels: the n_v vectors are swept in n_panels consecutive passes over
// A of panel_nv vectors each (the last may be narrower); ld is a panel's row
// length in elements, rounded up to whole 16-byte chunks of the sweep precision.
struct Panels {
    int n_panels, panel_nv, ld;
};
Panels panels_of(int n_v, int width, int precision) {
    const int vpt = precision == DOS_PREC_F64 ? 2 : 4;
    const int w = std::min(width > 0 ? width : kPanelMax, kPanelMax);
    Panels p;
    p.n_panels = (n_v + w - 1) / w;
    p.panel_nv = (n_v + p.n_panels - 1) / p.n_panels;
    p.ld = (p.panel_nv + vpt - 1) / vpt * vpt;
    return p;
}

Shape choose_shape(dos_ctx *ctx, const SweepRequest &r, const dos_csr *Adesc, int64_t n_rows,
                   int64_t nnz, cudaStream_t s) {
    const dos_launch &o = r.opts.launch;
    if (o.team || o.chunks || o.block || o.tiles || o.staged || o.chunk_bytes || o.depth ||
        o.panel) {
        DOS_REQUIRE(o.panel >= 0 && o.panel <= 4096, "launch.panel must be in [0, 4096]");
        const int ld = panels_of(r.n_v, o.panel, r.precision).ld;
        Shape d = default_shape(r.precision, ld, ctx->num_sms, n_rows);
        Shape sh;
        sh.panel = o.panel;
        sh.team = o.team ? o.team : d.team;
        sh.chunks = o.chunks ? o.chunks : d.chunks;
        sh.block = o.block ? o.block : d.block;
        DOS_REQUIRE(o.staged >= 0 && o.staged <= 4, "launch.staged must be 0, 1, 2, 3 or 4");
        sh.staged = o.staged ? o.staged - 1 : d.staged;
        DOS_REQUIRE(o.chunk_bytes == 0 || o.chunk_bytes == 16 || o.chunk_bytes == 32,
                    "launch.chunk_bytes must be 0, 16 or 32");
        sh.cb = o.chunk_bytes ? o.chunk_bytes : 16;
        DOS_REQUIRE(o.depth == 0 || ((o.depth == 2 || o.depth == 4 || o.depth == 8) && o.staged == 3),
                    "launch.depth must be 0, or 2, 4 or 8 with staged 3");
        sh.depth = o.depth;
        sh.tiles = 1;
        DOS_REQUIRE(shape_supported(r.precision, sh, ld),
                    "launch override does not cover the vector block (team*chunks*chunk_bytes >= row) "
                    "or uses an unsupported team/chunks/block/staged/chunk_bytes combination");
        if (o.tiles) {
            sh.tiles = o.tiles;
        } else {
            const int occ = std::max(1, max_active_blocks(r.precision, sh, ld));
            const int teams = (sh.block / 32) * (32 / sh.team);
            sh.tiles = (int)std::max<int64_t>(
                1, std::min<int64_t>((int64_t)ctx->num_sms * occ, (n_rows + teams - 1) / teams));
        }
        return sh;
    }
    const int ld = panels_of(r.n_v, 0, r.precision).ld;
    auto it = ctx->tuned.find(std::make_tuple(n_rows, nnz, r.B, std::min(r.n_v, kPanelMax),
                                              r.precision));
    if (it != ctx->tuned.end() && shape_supported(r.precision, it->second, ld)) return it->second;
    if (r.opts.flags & DOS_OPT_AUTOTUNE) {
        Shape sh = tune_shape(ctx, Adesc, r.B, r.seg_rows.data(), r.n_v, r.precision, nullptr, s);
        if (shape_supported(r.precision, sh, ld)) return sh;
    }
    return default_shape(r.precision, ld, ctx->num_sms, n_rows);
}

struct Plan {
    int n_tiles;
    std::vector<int32_t> row0, tile_begin;
};

Plan make_plan(const SweepRequest &r, const DevCSR &A, const Shape &sh, cudaStream_t s) {
    Plan p;
    const int B = r.B;
    p.row0.resize(B + 1);
    for (int b = 0; b <= B; ++b) p.row0[b] = (int32_t)r.seg_rows[b];
    p.tile_begin.assign(B + 1, 0);
    if (B == 1) {
        p.tile_begin[1] = sh.tiles;
    } else {
        // nnz at the segment boundaries
        std::vector<int32_t> rp(B + 1);
        if (A.host_row_ptr) {
            for (int b = 0; b <= B; ++b) rp[b] = A.host_row_ptr[r.seg_rows[b]];
        } else {
            for (int b = 0; b <= B; ++b)
                DOS_CUDA_TRY(cudaMemcpyAsync(&rp[b], A.row_ptr + r.seg_rows[b], sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
        }
        std::vector<double> cost(B);
        double total = 0.0;
        for (int b = 0; b < B; ++b) {
            cost[b] = (double)(rp[b + 1] - rp[b]) + kRowCost * (double)(r.seg_rows[b + 1] - r.seg_rows[b]);
            total += cost[b];
        }
        const double target = std::max<double>(sh.tiles, B);
        for (int b = 0; b < B; ++b) {
            const int64_t rows = r.seg_rows[b + 1] - r.seg_rows[b];
            int64_t t = (int64_t)llround(target * cost[b] / total);
            t = std::max<int64_t>(1, std::min<int64_t>(t, rows));
            p.tile_begin[b + 1] = p.tile_begin[b] + (int32_t)t;
        }
    }
    p.n_tiles = p.tile_begin[B];
    return p;
}

void run_sweep(dos_ctx *ctx, const dos_csr *Adesc, SweepRequest &r, cudaStream_t s) {
    DOS_REQUIRE(r.M >= 0 && r.M <= 100000, "M must be in [0, 100000]");
    DOS_REQUIRE(r.n_v >= 1 && r.n_v <= 4096, "n_v must be in [1, 4096]");
    DOS_REQUIRE(r.precision == DOS_PREC_F64 || r.precision == DOS_PREC_F32_ACC64,
                "precision must be DOS_PREC_F64 or DOS_PREC_F32_ACC64");
    DOS_REQUIRE(r.mu != nullptr, "mu is NULL");
    DOS_REQUIRE(r.opts.vec_offset >= 0 && r.opts.vec_offset + r.n_v <= (int64_t(1) << 16) * 64,
                "vec_offset + n_v out of range");
    DevCSR A = stage_csr(ctx, Adesc, s);
    DOS_REQUIRE(!(r.precision == DOS_PREC_F64 && A.dtype != DOS_F64),
                "DOS_PREC_F64 needs FP64 matrix values");
    const int B = r.B;
    DOS_REQUIRE(B >= 1 && B <= (1 << 16), "B must be in [1, 65536]");
    DOS_REQUIRE(r.seg_rows[0] == 0 && r.seg_rows[B] == A.n, "seg_rows must start at 0 and end at n");
    for (int b = 0; b < B; ++b) {
        DOS_REQUIRE(r.seg_rows[b + 1] > r.seg_rows[b], "every matrix needs at least one row");
        DOS_REQUIRE(isfinite(r.lb[b]) && isfinite(r.ub[b]) && r.ub[b] > r.lb[b],
                    "bounds must be finite with ub > lb");
    }
    DOS_REQUIRE(r.opts.batch_index + (uint64_t)B <= (uint64_t(1) << 16), "batch index out of range");

    // values in the sweep precision
    const void *val = A.val;
    if (r.precision == DOS_PREC_F32_ACC64 && A.dtype == DOS_F64 && A.nnz > 0) {
        float *v32 = (float *)ctx->val_f32.get(A.nnz * sizeof(float));
        launch_f64_to_f32((const double *)A.val, v32, A.nnz, s);
        val = v32;
    }

    const int esz = r.precision == DOS_PREC_F64 ? 8 : 4;
    const Shape sh = choose_shape(ctx, r, Adesc, A.n, A.nnz, s);
    // vector panels of the chosen width
    const Panels pan = panels_of(r.n_v, sh.panel, r.precision);
    const int n_panels = pan.n_panels, panel_nv = pan.panel_nv, ld = pan.ld;
    Plan plan = make_plan(r, A, sh, s);

    std::vector<double> c(B), inv_d(B);
    for (int b = 0; b < B; ++b) {
        c[b] = 0.5 * (r.lb[b] + r.ub[b]);
        inv_d[b] = 1.0 / (0.5 * (r.ub[b] - r.lb[b]));
    }
    SegDev seg = upload_segments(ctx, plan.row0, plan.tile_begin, c, inv_d, s);
    if (!(r.opts.flags & DOS_OPT_NO_VALIDATE)) validate_on_device(ctx, A, B, seg.row0, s);

    const int S = std::max(1, (r.M + 1) / 2);  // ceil(M/2), at least one step
    const bool per_vec = r.mu_pv != nullptr;
    const int pv = per_vec ? ld : 1;
    const int pvt = per_vec ? r.n_v : 1;
    const size_t per_step = (size_t)plan.n_tiles * 2 * pv * sizeof(double);
    const int slots = (int)std::max<size_t>(1, std::min<size_t>(S, kPartialCap / per_step));

    int4 *tiles = (int4 *)ctx->tiles.get(plan.n_tiles * sizeof(int4));
    launch_make_tiles(A.row_ptr, B, seg.row0, seg.tile_begin, plan.n_tiles, kRowCost, tiles, s);

    uint8_t *xb = (uint8_t *)ctx->xbuf.get(2 * (size_t)A.n * ld * esz);
    double *partial = (double *)ctx->partial.get(per_step * slots +
                                                 (size_t)plan.n_tiles * pv * sizeof(double));
    double *partial0 = partial + (size_t)slots * plan.n_tiles * 2 * pv;
    double *dotsum = (double *)ctx->dotsum.get(((size_t)B * S * 2 * pvt + (size_t)B * pvt) *
                                               sizeof(double));
    double *dotsum0 = dotsum + (size_t)B * S * 2 * pvt;
    double *mu_dev = (double *)ctx->mu_dev.get((size_t)B * (r.M + 1) * sizeof(double));
    double *mupv_dev = per_vec ? (double *)ctx->mupv_dev.get((size_t)B * r.n_v * (r.M + 1) *
                                                             sizeof(double))
                               : nullptr;
    int *status = status_flags(ctx);

    SweepArgs a;
    a.precision = r.precision;
    a.row_ptr = A.row_ptr;
    a.col_idx = A.col_idx;
    a.val = val;
    a.n_rows = A.n;
    a.nnz = A.nnz;
    a.ld = ld;
    a.B = B;
    a.seg_row0 = seg.row0;
    a.seg_c = seg.c;
    a.seg_inv_d = seg.inv_d;
    a.tiles = tiles;
    a.n_tiles = plan.n_tiles;
    a.x0 = xb;
    a.x1 = xb + (size_t)A.n * ld * esz;
    a.partial = partial;
    a.partial0 = partial0;
    a.per_vec = per_vec;
    a.seed = r.seed;
    a.batch_index = r.opts.batch_index;
    a.shape = sh;
    a.status = status;
    a.spin_cycles = r.opts.wait_limit_cycles;
    a.stall_test = (r.opts.flags & DOS_OPT_TEST_STALL_WAIT) ? 1 : 0;
    a.pdl = (r.opts.flags & DOS_OPT_NO_PDL) ? 0 : 1;

    const double tol = r.precision == DOS_PREC_F64 ? 1e-8 : 1e-3;
    const bool profiling = ctx->profiling;
    if (profiling) {  // two events per panel, around its step launches
        while ((int)ctx->prof_events.size() < 2 * n_panels) {
            cudaEvent_t e;
            DOS_CUDA_TRY(cudaEventCreate(&e));
            ctx->prof_events.push_back(e);
        }
    }
    // Everything from here to the moments is pure device work on stream s, so it
    // can be captured once into a CUDA graph and replayed.
    auto enqueue = [&](cudaStream_t s) {
        DOS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
        for (int p = 0; p < n_panels; ++p) {
            const int off = p * panel_nv;
            const int width = std::min(panel_nv, r.n_v - off);
            a.n_v = width;
            a.vec_offset = r.opts.vec_offset + off;
            launch_init_vectors(a, s);
            int k0 = 0;
            if (profiling) record_timing_event(ctx->prof_events[2 * p], s);
            for (int k = 0; k < S; ++k) {
                launch_step(a, k, k % slots, s);
                if (profiling && k == S - 1)
                    record_timing_event(ctx->prof_events[2 * p + 1], s);
                if ((k + 1) % slots == 0 || k == S - 1) {
                    launch_reduce(partial, plan.n_tiles, pv, width, B, seg.tile_begin, k0,
                                  k + 1 - k0, k0 % slots, slots, S, off, pvt, p > 0, dotsum, s);
                    k0 = k + 1;
                }
            }
            launch_reduce0(partial0, pv, width, B, seg.tile_begin, off, pvt, p > 0, dotsum0, s);
        }
        launch_finalize(dotsum, dotsum0, seg.row0, B, r.M, S, r.n_v, pvt, mu_dev, mupv_dev, tol,
                        status, s);
    };
    // Graph policy: the first call with a given configuration launches kernel by
    // kernel and remembers the configuration; an identical second call captures a
    // graph, and later identical calls replay it.
    const std::vector<uint64_t> key = {
        (uint64_t)r.precision, (uint64_t)(uintptr_t)A.row_ptr, (uint64_t)(uintptr_t)A.col_idx,
        (uint64_t)(uintptr_t)val, (uint64_t)A.n, (uint64_t)A.nnz, (uint64_t)B, (uint64_t)ld,
        (uint64_t)r.n_v, (uint64_t)r.M, r.seed, (uint64_t)r.opts.vec_offset, r.opts.batch_index,
        (uint64_t)sh.team, (uint64_t)sh.chunks, (uint64_t)sh.block, (uint64_t)plan.n_tiles,
        (uint64_t)sh.staged, (uint64_t)sh.cb, (uint64_t)sh.depth, (uint64_t)sh.panel,
        (uint64_t)per_vec, (uint64_t)slots, (uint64_t)(uintptr_t)xb, (uint64_t)(uintptr_t)partial,
        (uint64_t)(uintptr_t)dotsum, (uint64_t)(uintptr_t)mu_dev, (uint64_t)(uintptr_t)mupv_dev,
        (uint64_t)(uintptr_t)tiles, (uint64_t)(uintptr_t)seg.row0, (uint64_t)(uintptr_t)status,
        (uint64_t)profiling, (uint64_t)(uintptr_t)s, (uint64_t)a.pdl};
    GraphCache &gc = ctx->graph;
    const bool use_graph = !(r.opts.flags & DOS_OPT_NO_GRAPH);
    // The graph runs on a context-owned stream ordered after `s` by events, so
    // callers on the legacy default stream (which cannot be captured) get it too.
    auto launch_graph = [&]() {
        DOS_CUDA_TRY(cudaEventRecord(gc.ev_in, s));
        DOS_CUDA_TRY(cudaStreamWaitEvent(gc.stream, gc.ev_in, 0));
        DOS_CUDA_TRY(cudaGraphLaunch(gc.exec, gc.stream));
        DOS_CUDA_TRY(cudaEventRecord(gc.ev_out, gc.stream));
        DOS_CUDA_TRY(cudaStreamWaitEvent(s, gc.ev_out, 0));
        count_launches(gc.kernel_nodes);
    };
    if (use_graph && gc.exec && gc.key == key) {
        launch_graph();
    } else if (use_graph && gc.pending == key) {
        if (!gc.stream) {
            DOS_CUDA_TRY(cudaStreamCreateWithFlags(&gc.stream, cudaStreamNonBlocking));
            DOS_CUDA_TRY(cudaEventCreateWithFlags(&gc.ev_in, cudaEventDisableTiming));
            DOS_CUDA_TRY(cudaEventCreateWithFlags(&gc.ev_out, cudaEventDisableTiming));
        }
        if (gc.exec) {
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            gc.key.clear();
        }
        const int64_t before = g_launch_count.load();
        DOS_CUDA_TRY(cudaStreamBeginCapture(gc.stream, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue(gc.stream);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(gc.stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        cudaGraph_t g = nullptr;
        DOS_CUDA_TRY(cudaStreamEndCapture(gc.stream, &g));
        gc.kernel_nodes = g_launch_count.load() - before;
        g_launch_count.fetch_sub(gc.kernel_nodes);
        cudaError_t ie = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        DOS_CUDA_TRY(ie);
        gc.key = key;
        launch_graph();
    } else {
        enqueue(s);
        gc.pending = key;
    }
    copy_out(r.mu, mu_dev, (size_t)B * (r.M + 1) * sizeof(double), s);
    if (per_vec) copy_out(r.mu_pv, mupv_dev, (size_t)B * r.n_v * (r.M + 1) * sizeof(double), s);

    const bool host_out = !is_device_ptr(r.mu) || (per_vec && !is_device_ptr(r.mu_pv));
    if (!(r.opts.flags & DOS_OPT_NO_SPECTRUM_CHECK) || host_out || profiling) {
        int h = 0;
        DOS_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (profiling) {
            for (int p = 0; p < n_panels; ++p) {
                float ms = 0.f;
                DOS_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->prof_events[2 * p],
                                                  ctx->prof_events[2 * p + 1]));
                ctx->prof_step_ms += ms;
                ctx->prof_step_launches += S;
            }
            ctx->prof_sweeps += 1;
        }
        if (h & 4)
            throw Error{DOS_ETIMEOUT,
                        "a bounded device-side wait of the staged sweep kernel ran out"};
        if (!(r.opts.flags & DOS_OPT_NO_SPECTRUM_CHECK) && (h & 2))
            throw Error{DOS_ESPECTRUM,
                        "a moment exceeds mu_0 in magnitude or is not finite: the bounds do not "
                        "enclose the spectrum"};
    }
}

dos_kpm_opts default_opts() {
    dos_kpm_opts o;
    memset(&o, 0, sizeof(o));
    return o;
}

// Autotuner: for every launch shape that covers the vector block without more
// than 2x idle lanes, and tile counts of 1x to 32x the resident blocks, time
// sweeps of 16 and 48 Chebyshev steps with CUDA events; the difference / 32 is
// the per-step time (fixed per-call costs cancel).  Best of three runs (one when
// a step takes more than 2 ms).  Vector panels narrower than 256 (launch.panel)
// are not searched: on the lattice and on the power-law graph every narrower
// width measured slower per step of all n_v vectors (each pass re-reads A and
// pays the per-nonzero costs again), so they are left to callers short of
// device memory.
static int panel_ld(int n_v, int precision) { return panels_of(n_v, 0, precision).ld; }

Shape tune_shape(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows, int n_v,
                 int precision, double *best_ms, cudaStream_t s) {
    DOS_REQUIRE(n_v >= 1 && n_v <= 4096, "n_v must be in [1, 4096]");
    DOS_REQUIRE(precision == DOS_PREC_F64 || precision == DOS_PREC_F32_ACC64, "bad precision");
    const int esz = precision == DOS_PREC_F64 ? 8 : 4;
    const int pw = std::min(n_v, kPanelMax);
    const int ld = panel_ld(n_v, precision);
    std::vector<int64_t> rows;
    if (B == 1) rows = {0, A->n};
    else rows.assign(seg_rows, seg_rows + B + 1);
    // Timing only: the moments are discarded and the spectrum check is off, so
    // any bounds do (values may grow; the kernels' speed does not depend on them).
    std::vector<double> lb(B, -1.0), ub(B, 1.0);
    double *mu_scratch = (double *)ctx->rec_out.get((size_t)B * 97 * sizeof(double));
    // timing events, released on every exit path (a failing candidate throws)
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    DOS_CUDA_TRY(cudaEventCreate(&ev.a));
    DOS_CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    Shape best;
    double best_t = INFINITY;
    bool first = true;
    // variants: direct loads, TMA panels and TMA gathers (16-byte chunks), and
    // direct loads with 32-byte chunks
    const int variants[6][2] = {{0, 16}, {1, 16}, {2, 16}, {0, 32}, {3, 16}, {3, 32}};
    for (int G = 1; G <= 32; G <<= 1) {
        for (int C : {1, 2, 4})
        for (const auto &var : variants) {
            const int cb = var[1];
            if (ld % (cb / esz) != 0) continue;
            const int chunks = ld / (cb / esz);
            const int cover = G * C;
            if (cover < chunks || (cover > 1 && cover / 2 >= chunks)) continue;
            Shape sh;
            sh.team = G;
            sh.chunks = C;
            sh.block = 256;
            sh.staged = var[0];
            sh.cb = cb;
            sh.tiles = 1;
            if (!shape_supported(precision, sh, ld)) continue;
            const int occ = max_active_blocks(precision, sh, ld);
            if (occ <= 0) continue;
            const int teams = (256 / 32) * (32 / G);
            const int64_t max_tiles = std::max<int64_t>(B, (A->n + teams - 1) / teams);
            for (int mult : {1, 2, 4, 8, 16, 32}) {
                sh.tiles = (int)std::min<int64_t>((int64_t)ctx->num_sms * occ * mult, max_tiles);
                double per_step = INFINITY;
                for (int rep = 0; rep < 3; ++rep) {
                    float ms[2];
                    for (int which = 0; which < 2; ++which) {
                        SweepRequest r;
                        r.B = B;
                        r.seg_rows = rows;
                        r.lb = lb;
                        r.ub = ub;
                        r.M = which ? 96 : 32;
                        r.n_v = pw;
                        r.seed = 1;
                        r.precision = precision;
                        r.mu = mu_scratch;
                        r.mu_pv = nullptr;
                        r.opts = default_opts();
                        r.opts.flags = DOS_OPT_NO_SPECTRUM_CHECK | (first ? 0u : DOS_OPT_NO_VALIDATE);
                        r.opts.launch.team = sh.team;
                        r.opts.launch.chunks = sh.chunks;
                        r.opts.launch.block = sh.block;
                        r.opts.launch.tiles = sh.tiles;
                        r.opts.launch.staged = sh.staged + 1;
                        r.opts.launch.chunk_bytes = sh.cb;
                        r.opts.launch.depth = sh.depth;
                        DOS_CUDA_TRY(cudaEventRecord(e0, s));
                        run_sweep(ctx, A, r, s);
                        DOS_CUDA_TRY(cudaEventRecord(e1, s));
                        DOS_CUDA_TRY(cudaEventSynchronize(e1));
                        DOS_CUDA_TRY(cudaEventElapsedTime(&ms[which], e0, e1));
                        first = false;
                    }
                    per_step = std::min(per_step, (double)(ms[1] - ms[0]) / 32.0);
                    if (per_step > 2.0) break;  // large problems: one repetition is enough
                }
                if (getenv("DOS_TUNE_VERBOSE"))
                    fprintf(stderr,
                            "dos_tune: team %d chunks %d staged %d chunk_bytes %d tiles %d: "
                            "%.4f ms/step\n",
                            sh.team, sh.chunks, sh.staged, sh.cb, sh.tiles, per_step);
                if (per_step < best_t) {
                    best_t = per_step;
                    best = sh;
                }
                if (sh.tiles == max_tiles) break;
            }
        }
    }
    DOS_REQUIRE(best.team > 0, "no launch shape fits this vector block");
    int64_t nnz = A->nnz;
    ctx->tuned[std::make_tuple((int64_t)A->n, nnz, B, pw, precision)] = best;
    if (best_ms) *best_ms = best_t;
    return best;
}


}  // namespace

// ============================================================================
extern "C" {

const char *dos_status_string(int status) {
    switch (status) {
        case DOS_OK: return "DOS_OK";
        case DOS_EINVAL: return "DOS_EINVAL";
        case DOS_ENOMEM: return "DOS_ENOMEM";
        case DOS_ECUDA: return "DOS_ECUDA";
        case DOS_ESPECTRUM: return "DOS_ESPECTRUM";
        case DOS_ETIMEOUT: return "DOS_ETIMEOUT";
        case DOS_EIO: return "DOS_EIO";
        default: return "DOS_UNKNOWN";
    }
}

int dos_ctx_create(dos_ctx **out, int device) {
    if (!out) return DOS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return DOS_ECUDA;
    }
    if (device < 0 || device >= count) return DOS_EINVAL;
    dos_ctx *ctx = new (std::nothrow) dos_ctx();
    if (!ctx) return DOS_ENOMEM;
    ctx->device = device;
    int rc = guarded(ctx, [&] {
        DOS_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    });
    if (rc != DOS_OK) {
        delete ctx;
        return rc;
    }
    *out = ctx;
    return DOS_OK;
}

int dos_ctx_destroy(dos_ctx *ctx) {
    if (!ctx) return DOS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (Buffer *b : {&ctx->csr_rowptr, &ctx->csr_colidx, &ctx->csr_val, &ctx->val_f32, &ctx->xbuf,
                      &ctx->partial, &ctx->dotsum, &ctx->tiles, &ctx->segs, &ctx->status,
                      &ctx->mu_dev, &ctx->mupv_dev, &ctx->bnd_vec, &ctx->bnd_part, &ctx->bnd_out,
                      &ctx->rec_in, &ctx->rec_out, &ctx->err_buf, &ctx->lz_buf})
        b->release();
    ctx->host_stage.release();
    if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
    if (ctx->graph.stream) cudaStreamDestroy(ctx->graph.stream);
    if (ctx->graph.ev_in) cudaEventDestroy(ctx->graph.ev_in);
    if (ctx->graph.ev_out) cudaEventDestroy(ctx->graph.ev_out);
    for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
    if (prev >= 0) cudaSetDevice(prev);
    cudaGetLastError();
    delete ctx;
    return DOS_OK;
}

const char *dos_last_error(const dos_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int dos_profile_enable(dos_ctx *ctx, int on) {
    return guarded(ctx, [&] {
        ctx->profiling = on != 0;
        ctx->prof_step_ms = 0.0;
        ctx->prof_step_launches = 0;
        ctx->prof_sweeps = 0;
        g_launch_count.store(0);
    });
}

int dos_profile_read(dos_ctx *ctx, double *step_ms, int64_t *step_launches, int64_t *sweeps,
                     int64_t *launches) {
    if (!ctx) return DOS_EINVAL;
    if (step_ms) *step_ms = ctx->prof_step_ms;
    if (step_launches) *step_launches = ctx->prof_step_launches;
    if (sweeps) *sweeps = ctx->prof_sweeps;
    if (launches) *launches = g_launch_count.load();
    return DOS_OK;
}

int dos_validate_csr(dos_ctx *ctx, const dos_csr *Adesc, void *stream) {
    return guarded(ctx, [&] {
        cudaStream_t s = (cudaStream_t)stream;
        DevCSR A = stage_csr(ctx, Adesc, s);
        std::vector<int32_t> row0 = {0, (int32_t)A.n}, tb = {0, 1};
        SegDev seg = upload_segments(ctx, row0, tb, {0.0}, {1.0}, s);
        validate_on_device(ctx, A, 1, seg.row0, s);
    });
}

int dos_start_vectors(dos_ctx *ctx, int64_t n, int n_v, uint64_t seed, uint64_t batch_index,
                      int64_t vec_offset, int dtype, void *out, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(out != nullptr, "out is NULL");
        DOS_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
        DOS_REQUIRE(n_v >= 1 && n_v <= 4096, "n_v must be in [1, 4096]");
        DOS_REQUIRE(vec_offset >= 0 && vec_offset + n_v <= (int64_t(1) << 16) * 64,
                    "vec_offset + n_v out of range");
        DOS_REQUIRE(batch_index < (uint64_t(1) << 16), "batch_index out of range");
        DOS_REQUIRE(dtype == DOS_F64 || dtype == DOS_F32, "bad dtype");
        cudaStream_t s = (cudaStream_t)stream;
        const int prec = dtype == DOS_F64 ? DOS_PREC_F64 : DOS_PREC_F32_ACC64;
        const int vpt = dtype == DOS_F64 ? 2 : 4;
        const int esz = dtype == DOS_F64 ? 8 : 4;
        const int ld = (n_v + vpt - 1) / vpt * vpt;
        std::vector<int32_t> row0 = {0, (int32_t)n}, tb = {0, 1};
        SegDev seg = upload_segments(ctx, row0, tb, {0.0}, {1.0}, s);
        void *x = ctx->xbuf.get((size_t)n * ld * esz);
        SweepArgs a{};
        a.precision = prec;
        a.n_rows = n;
        a.n_v = n_v;
        a.ld = ld;
        a.B = 1;
        a.seg_row0 = seg.row0;
        a.x0 = x;
        a.seed = seed;
        a.vec_offset = vec_offset;
        a.batch_index = batch_index;
        launch_init_vectors(a, s);
        DOS_CUDA_TRY(cudaMemcpy2DAsync(out, (size_t)n_v * esz, x, (size_t)ld * esz,
                                       (size_t)n_v * esz, (size_t)n, cudaMemcpyDefault, s));
        if (!is_device_ptr(out)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_kpm_moments_ex(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                       uint64_t seed, int precision, double *mu, double *mu_per_vec,
                       const dos_kpm_opts *opts, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(A != nullptr, "matrix descriptor is NULL");
        SweepRequest r;
        r.B = 1;
        r.seg_rows = {0, A->n};
        r.lb = {lb};
        r.ub = {ub};
        r.M = M;
        r.n_v = n_v;
        r.seed = seed;
        r.precision = precision;
        r.mu = mu;
        r.mu_pv = mu_per_vec;
        r.opts = opts ? *opts : default_opts();
        run_sweep(ctx, A, r, (cudaStream_t)stream);
    });
}

int dos_kpm_moments(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                    uint64_t seed, int precision, double *mu, double *mu_per_vec, void *stream) {
    return dos_kpm_moments_ex(ctx, A, lb, ub, M, n_v, seed, precision, mu, mu_per_vec, nullptr,
                              stream);
}

int dos_kpm_moments_batched(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows,
                            const double *lb, const double *ub, int M, int n_v, uint64_t seed,
                            int precision, double *mu, double *mu_per_vec,
                            const dos_kpm_opts *opts, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(B >= 1 && B <= (1 << 16), "B must be in [1, 65536]");
        DOS_REQUIRE(seg_rows && lb && ub, "seg_rows / lb / ub is NULL");
        SweepRequest r;
        r.B = B;
        r.seg_rows.assign(seg_rows, seg_rows + B + 1);
        r.lb.assign(lb, lb + B);
        r.ub.assign(ub, ub + B);
        r.M = M;
        r.n_v = n_v;
        r.seed = seed;
        r.precision = precision;
        r.mu = mu;
        r.mu_pv = mu_per_vec;
        r.opts = opts ? *opts : default_opts();
        r.opts.batch_index = opts ? opts->batch_index : 0;
        run_sweep(ctx, A, r, (cudaStream_t)stream);
    });
}

int dos_tune(dos_ctx *ctx, const dos_csr *A, int B, const int64_t *seg_rows, int n_v,
             int precision, dos_launch *best, double *best_ms, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(A != nullptr, "matrix descriptor is NULL");
        DOS_REQUIRE(B >= 1 && B <= (1 << 16), "B must be in [1, 65536]");
        DOS_REQUIRE(B == 1 || seg_rows != nullptr, "seg_rows is NULL");
        Shape sh = tune_shape(ctx, A, B, seg_rows, n_v, precision, best_ms, (cudaStream_t)stream);
        if (best) {
            best->team = sh.team;
            best->chunks = sh.chunks;
            best->block = sh.block;
            best->tiles = sh.tiles;
            best->staged = sh.staged + 1;
            best->chunk_bytes = sh.cb;
            best->depth = sh.staged == 2 ? tmag_depth(sh.block, sh.team, panel_ld(n_v, precision),
                                                      precision == DOS_PREC_F64 ? 8 : 4, sh.depth)
                                         : 0;
            best->panel = 0;
        }
    });
}

int dos_bounds(dos_ctx *ctx, const dos_csr *Adesc, int method, int steps, uint64_t seed,
               double pad_frac, double *lb, double *ub, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(lb && ub, "lb / ub is NULL");
        DOS_REQUIRE(method == DOS_BOUNDS_GERSHGORIN || method == DOS_BOUNDS_LANCZOS, "bad method");
        DOS_REQUIRE(isfinite(pad_frac) && pad_frac >= 0.0, "pad_frac must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        DevCSR A = stage_csr(ctx, Adesc, s);
        {
            std::vector<int32_t> row0 = {0, (int32_t)A.n}, tb = {0, 1};
            SegDev seg = upload_segments(ctx, row0, tb, {0.0}, {1.0}, s);
            validate_on_device(ctx, A, 1, seg.row0, s);
        }
        double lo, hi;
        if (method == DOS_BOUNDS_GERSHGORIN) {
            const int nb = gershgorin_blocks(ctx->num_sms);
            double *part = (double *)ctx->bnd_part.get((2 * (size_t)nb + 2) * sizeof(double));
            double *out = part + 2 * nb;
            launch_gershgorin(A.n, A.row_ptr, A.col_idx, A.val, A.dtype, part, nb, s);
            launch_minmax_final(part, nb, out, s);
            double h[2];
            DOS_CUDA_TRY(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
            lo = h[0];
            hi = h[1];
        } else {
            DOS_REQUIRE(steps >= 1 && steps <= 512, "steps must be in [1, 512]");
            const int k = (int)std::min<int64_t>(steps, A.n);
            const int nb = reduce_blocks(ctx->num_sms, A.n);
            double *vec = (double *)ctx->bnd_vec.get(3 * (size_t)A.n * sizeof(double));
            double *q = vec, *q_prev = vec + A.n, *w = vec + 2 * A.n;
            double *part = (double *)ctx->bnd_part.get(((size_t)nb + 2 * (size_t)k) * sizeof(double));
            double *alpha = part + nb, *beta = alpha + k;
            DOS_CUDA_TRY(cudaMemsetAsync(q_prev, 0, A.n * sizeof(double), s));
            launch_lanczos_start(A.n, seed, q, s);
            for (int j = 0; j < k; ++j) {
                launch_lanczos_matvec(A.n, A.row_ptr, A.col_idx, A.val, A.dtype, q, q_prev,
                                      j ? beta + j - 1 : nullptr, w, part, nb, s);
                launch_sum_final(part, nb, alpha + j, 0, s);
                launch_lanczos_axpy(A.n, alpha + j, q, w, part, nb, s);
                launch_sum_final(part, nb, beta + j, 1, s);
                if (j + 1 < k) launch_lanczos_next(A.n, beta + j, q, q_prev, w, s);
            }
            // the tridiagonal's extreme Ritz values and the last components of their
            // unit Ritz vectors, on the device (implicit QL)
            double *work = (double *)ctx->bnd_out.get((3 * (size_t)k + 3) * sizeof(double));
            double *res = work + 3 * (size_t)k;
            launch_lanczos_bounds(alpha, beta, k, work, res, s);
            double h[3];
            DOS_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
            DOS_REQUIRE(isfinite(h[0]) && isfinite(h[1]), "Lanczos produced non-finite values");
            lo = h[0];
            hi = h[1];
        }
        DOS_REQUIRE(isfinite(lo) && isfinite(hi), "bounds are not finite (non-finite values?)");
        const double w = hi - lo;
        *lb = lo - pad_frac * w;
        *ub = hi + pad_frac * w;
        if (!(*ub > *lb)) {  // a matrix with a single eigenvalue: widen to a unit interval
            *lb = lo - 0.5;
            *ub = hi + 0.5;
        }
    });
}

int dos_bounds_batched(dos_ctx *ctx, const dos_csr *Adesc, int B, const int64_t *seg_rows,
                       double pad_frac, double *lb, double *ub, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(lb && ub && seg_rows, "lb / ub / seg_rows is NULL");
        DOS_REQUIRE(B >= 1 && B <= (1 << 16), "B must be in [1, 65536]");
        DOS_REQUIRE(isfinite(pad_frac) && pad_frac >= 0.0, "pad_frac must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        DevCSR A = stage_csr(ctx, Adesc, s);
        DOS_REQUIRE(seg_rows[0] == 0 && seg_rows[B] == A.n, "seg_rows must start at 0 and end at n");
        std::vector<int32_t> row0(B + 1), tb(B + 1, 0);
        for (int b = 0; b <= B; ++b) {
            if (b < B) DOS_REQUIRE(seg_rows[b + 1] > seg_rows[b], "every matrix needs a row");
            row0[b] = (int32_t)seg_rows[b];
        }
        SegDev seg = upload_segments(ctx, row0, tb, std::vector<double>(B, 0.0),
                                     std::vector<double>(B, 1.0), s);
        validate_on_device(ctx, A, B, seg.row0, s);
        uint8_t *buf = (uint8_t *)ctx->bnd_part.get((size_t)B * 32);
        unsigned long long *keys = (unsigned long long *)buf;
        double *out = (double *)(buf + (size_t)B * 16);
        launch_gershgorin_batched(A.n, A.row_ptr, A.col_idx, A.val, A.dtype, B, seg.row0, keys,
                                  out, ctx->num_sms, s);
        std::vector<double> h(2 * (size_t)B);
        DOS_CUDA_TRY(cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) {
            const double lo = h[2 * b], hi = h[2 * b + 1];
            DOS_REQUIRE(isfinite(lo) && isfinite(hi), "bounds are not finite");
            const double w = hi - lo;
            lb[b] = lo - pad_frac * w;
            ub[b] = hi + pad_frac * w;
            if (!(ub[b] > lb[b])) {
                lb[b] = lo - 0.5;
                ub[b] = hi + 0.5;
            }
        }
    });
}

int dos_reconstruct(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                    const double *t, int N_t, double *phi_hat, double *phi_lambda, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(mu && phi_hat, "mu / phi_hat is NULL");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(N_t >= 1 && N_t <= (1 << 26), "N_t must be in [1, 2^26]");
        DOS_REQUIRE(damping == DOS_DAMP_NONE || damping == DOS_DAMP_JACKSON, "bad damping");
        DOS_REQUIRE(!phi_lambda || (isfinite(lb) && isfinite(ub) && ub > lb), "need ub > lb");
        cudaStream_t s = (cudaStream_t)stream;
        // device staging: mu | coefficients | t | phi_hat | phi_lambda
        const size_t nd = 2 * (size_t)(M + 1) + 3 * (size_t)N_t;
        double *buf = (double *)ctx->rec_in.get(nd * sizeof(double));
        double *dmu = buf, *coef = buf + (M + 1), *dt = coef + (M + 1);
        double *dphi = dt + N_t, *dphl = dphi + N_t;
        DOS_CUDA_TRY(cudaMemcpyAsync(dmu, mu, (M + 1) * sizeof(double), cudaMemcpyDefault, s));
        if (t) DOS_CUDA_TRY(cudaMemcpyAsync(dt, t, N_t * sizeof(double), cudaMemcpyDefault, s));
        launch_reconstruct(dmu, M, damping, lb, ub, t ? dt : nullptr, N_t, coef, dphi,
                           phi_lambda ? dphl : nullptr, s);
        copy_out(phi_hat, dphi, N_t * sizeof(double), s);
        if (phi_lambda) copy_out(phi_lambda, dphl, N_t * sizeof(double), s);
        if (!is_device_ptr(phi_hat) || (phi_lambda && !is_device_ptr(phi_lambda)))
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_reconstruct_batched(dos_ctx *ctx, const double *mu, int B, int M, int damping,
                            const double *t, int N_t, double *phi_hat, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(mu && phi_hat, "mu / phi_hat is NULL");
        DOS_REQUIRE(B >= 1 && B <= (1 << 20), "B must be in [1, 2^20]");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(N_t >= 1 && N_t <= (1 << 20), "N_t must be in [1, 2^20]");
        DOS_REQUIRE((int64_t)B * N_t <= (int64_t(1) << 31), "B * N_t must be <= 2^31");
        DOS_REQUIRE(damping == DOS_DAMP_NONE || damping == DOS_DAMP_JACKSON, "bad damping");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t nmu = (size_t)B * (M + 1);
        const bool mu_dev = is_device_ptr(mu), out_dev = is_device_ptr(phi_hat);
        // device staging: coefficients | mu (if host) | t (if given) | phi_hat (if host)
        const size_t nd = nmu + (mu_dev ? 0 : nmu) + (t ? N_t : 0) +
                          (out_dev ? 0 : (size_t)B * N_t);
        double *buf = (double *)ctx->rec_in.get(nd * sizeof(double));
        double *coef = buf, *p = buf + nmu;
        const double *dmu = mu;
        if (!mu_dev) {
            DOS_CUDA_TRY(cudaMemcpyAsync(p, mu, nmu * sizeof(double), cudaMemcpyHostToDevice, s));
            dmu = p;
            p += nmu;
        }
        const double *dt = nullptr;
        if (t) {
            DOS_CUDA_TRY(cudaMemcpyAsync(p, t, N_t * sizeof(double), cudaMemcpyDefault, s));
            dt = p;
            p += N_t;
        }
        double *dphi = out_dev ? phi_hat : p;
        launch_reconstruct_rows(dmu, M + 1, B, M, damping, dt, N_t, coef, dphi, s);
        if (!out_dev) {
            DOS_CUDA_TRY(cudaMemcpyAsync(phi_hat, dphi, (size_t)B * N_t * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
        }
    });
}

int dos_lanczos_ritz(dos_ctx *ctx, const dos_csr *Adesc, int M, int n_v, uint64_t seed,
                     double *theta, double *weight, int *m_used, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(theta && weight, "theta / weight is NULL");
        DOS_REQUIRE(n_v >= 1 && n_v <= 256, "n_v must be in [1, 256]");
        DOS_REQUIRE(M >= 1 && M <= 4096, "M must be in [1, 4096]");
        cudaStream_t s = (cudaStream_t)stream;
        DevCSR A = stage_csr(ctx, Adesc, s);
        DOS_REQUIRE(A.dtype == DOS_F64, "the Lanczos DOS runs in FP64: FP64 values needed");
        DOS_REQUIRE(M <= A.n, "M must not exceed n");
        std::vector<int32_t> row0 = {0, (int32_t)A.n}, tb = {0, 1};
        SegDev seg = upload_segments(ctx, row0, tb, {0.0}, {1.0}, s);
        validate_on_device(ctx, A, 1, seg.row0, s);
        const int ld = (n_v + 1) / 2 * 2;
        const int nb_axpy = lanczos_blocks(ctx->num_sms, A.n, ld);
        const int nb_spmm = lanczos_team_blocks(ctx->num_sms, A.n, ld);
        const int nb = std::max(nb_axpy, nb_spmm);  // rows of the partial-sum buffer
        // scratch: two vector blocks | partials | alpha, beta [M][ld] | out | s, c, t [ld]
        // | m_used
        const size_t nvec = (size_t)A.n * ld;
        const size_t n_dbl = 2 * nvec + (size_t)nb * ld + 2 * (size_t)M * ld + 3 * (size_t)ld +
                             2 * (size_t)n_v * M + n_v;
        double *buf = (double *)ctx->lz_buf.get(n_dbl * sizeof(double));
        double *q0 = buf, *q1 = q0 + nvec, *part = q1 + nvec, *alpha = part + (size_t)nb * ld;
        double *beta = alpha + (size_t)M * ld;
        double *th = beta + (size_t)M * ld, *wt = th + (size_t)n_v * M;
        double *s_fac = wt + (size_t)n_v * M, *c_fac = s_fac + ld, *t_fac = c_fac + ld;
        int *mu_dev = (int *)(t_fac + ld);
        SweepArgs a{};
        a.precision = DOS_PREC_F64;
        a.n_rows = A.n;
        a.n_v = n_v;
        a.ld = ld;
        a.B = 1;
        a.seg_row0 = seg.row0;
        a.x0 = q0;
        a.seed = seed;
        launch_init_vectors(a, s);
        launch_unit_scale(A.n, ld, n_v, q0, ctx->num_sms, s);
        DOS_CUDA_TRY(cudaMemsetAsync(q1, 0, nvec * sizeof(double), s));
        double *cur = q0, *prev = q1;
        const double *val = (const double *)A.val;
        const bool profiling = ctx->profiling;
        if (profiling) {  // two events per step, around its block-SpMM launch
            while ((int)ctx->prof_events.size() < 2 * M) {
                cudaEvent_t e;
                DOS_CUDA_TRY(cudaEventCreate(&e));
                ctx->prof_events.push_back(e);
            }
        }
        for (int j = 0; j < M; ++j) {
            if (profiling) DOS_CUDA_TRY(cudaEventRecord(ctx->prof_events[2 * j], s));
            // cur = u_j, prev = u_{j-1} of q_j = s_j u_j; the factors s_j, c_j, t_j
            // (per column, written by the previous step's beta kernel) are 1 / absent
            // at j = 0
            const double *sj = j ? s_fac : nullptr;
            launch_lanczos_team_spmm(A.n, ld, A.row_ptr, A.col_idx, val, cur, prev,
                                     j ? c_fac : nullptr, part, nb_spmm, s);
            if (profiling) DOS_CUDA_TRY(cudaEventRecord(ctx->prof_events[2 * j + 1], s));
            launch_lanczos_alpha(part, nb_spmm, ld, sj, alpha + (size_t)j * ld, s);
            launch_lanczos_block_axpy(A.n, ld, n_v, alpha + (size_t)j * ld, j ? t_fac : nullptr,
                                      cur, prev, part, nb_axpy, s);
            launch_lanczos_beta(part, nb_axpy, ld, sj, j ? beta + (size_t)(j - 1) * ld : nullptr,
                                beta + (size_t)j * ld, s_fac, c_fac, t_fac, s);
            std::swap(cur, prev);  // cur now holds u_{j+1}, prev u_j
        }
        // steps kept per run (invariant-subspace rule) and the Ritz pairs, on the device
        launch_lanczos_steps(alpha, beta, M, ld, n_v, mu_dev, s);
        launch_tridiag_ritz(alpha, beta, mu_dev, M, ld, n_v, th, wt, s);
        copy_out(theta, th, (size_t)n_v * M * sizeof(double), s);
        copy_out(weight, wt, (size_t)n_v * M * sizeof(double), s);
        std::vector<int> mus(n_v);
        DOS_CUDA_TRY(cudaMemcpyAsync(mus.data(), mu_dev, n_v * sizeof(int), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (profiling) {
            for (int j = 0; j < M; ++j) {
                float ms = 0.f;
                DOS_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->prof_events[2 * j],
                                                  ctx->prof_events[2 * j + 1]));
                ctx->prof_step_ms += ms;
            }
            ctx->prof_step_launches += M;
            ctx->prof_sweeps += 1;
        }
        for (int l = 0; l < n_v; ++l)
            DOS_REQUIRE(mus[l] >= 1, "Lanczos produced non-finite values");
        if (m_used) memcpy(m_used, mus.data(), n_v * sizeof(int));
    });
}

int dos_lanczos_dos(dos_ctx *ctx, const double *theta, const double *weight, int n_v, int M,
                    double sigma, const double *x, int N_x, double *phi, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(theta && weight && x && phi, "NULL argument");
        DOS_REQUIRE(n_v >= 1 && M >= 1 && (int64_t)n_v * M <= (int64_t(1) << 28), "bad n_v / M");
        DOS_REQUIRE(N_x >= 1 && N_x <= 10000000, "N_x must be in [1, 10^7]");
        DOS_REQUIRE(isfinite(sigma) && sigma > 0.0, "sigma must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t np = (size_t)n_v * M;
        double *buf = (double *)ctx->err_buf.get((2 * np + 2 * (size_t)N_x) * sizeof(double));
        double *dp = buf, *dw = dp + np, *dx = dw + np, *dphi = dx + N_x;
        DOS_CUDA_TRY(cudaMemcpyAsync(dp, theta, np * 8, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(dw, weight, np * 8, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(dx, x, (size_t)N_x * 8, cudaMemcpyDefault, s));
        launch_weighted_gauss(dp, dw, (int64_t)np, 1.0 / n_v, sigma, dx, 0.0, 0.0, N_x, dphi, s);
        copy_out(phi, dphi, (size_t)N_x * 8, s);
        if (!is_device_ptr(phi)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_haydock_dos(dos_ctx *ctx, const double *theta, const double *weight, int n_v, int M,
                    double eta, const double *x, int N_x, double *phi, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(theta && weight && x && phi, "NULL argument");
        DOS_REQUIRE(n_v >= 1 && M >= 1 && (int64_t)n_v * M <= (int64_t(1) << 28), "bad n_v / M");
        DOS_REQUIRE(N_x >= 1 && N_x <= 10000000, "N_x must be in [1, 10^7]");
        DOS_REQUIRE(isfinite(eta) && eta > 0.0, "eta must be > 0");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t np = (size_t)n_v * M;
        double *buf = (double *)ctx->err_buf.get((2 * np + 2 * (size_t)N_x) * sizeof(double));
        double *dp = buf, *dw = dp + np, *dx = dw + np, *dphi = dx + N_x;
        DOS_CUDA_TRY(cudaMemcpyAsync(dp, theta, np * 8, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(dw, weight, np * 8, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(dx, x, (size_t)N_x * 8, cudaMemcpyDefault, s));
        launch_weighted_lorentz(dp, dw, (int64_t)np, 1.0 / n_v, eta, dx, N_x, dphi, s);
        copy_out(phi, dphi, (size_t)N_x * 8, s);
        if (!is_device_ptr(phi)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_points_error(dos_ctx *ctx, const double *pts, const double *wts, int64_t n_pts,
                     double lb, double ub, const double *eig, int64_t n_eig, const double *ref_mu,
                     int M_ref, int ref_damping, double sigma, int N_x, double *err_l1,
                     double *err_inf, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(pts && wts && n_pts >= 1, "points / weights missing");
        DOS_REQUIRE(isfinite(lb) && isfinite(ub) && ub > lb, "need ub > lb");
        DOS_REQUIRE(isfinite(sigma) && sigma > 0.0, "sigma must be > 0");
        DOS_REQUIRE(N_x >= 2 && N_x <= 1000000, "N_x must be in [2, 10^6]");
        DOS_REQUIRE(eig ? n_eig >= 1 : (ref_mu != nullptr && M_ref >= 0 && M_ref <= 100000),
                    "need eigenvalues or reference moments");
        cudaStream_t s = (cudaStream_t)stream;
        const double d = 0.5 * (ub - lb);
        const int Mr = eig ? 0 : M_ref;
        const int64_t nq64 = std::max<int64_t>(4 * (int64_t)(Mr + 1), (int64_t)ceil(40.0 * d / sigma));
        const int N_q = (int)std::min<int64_t>(nq64, 1 << 24);
        const double x0 = lb - 6.0 * sigma, h = (ub - lb + 12.0 * sigma) / (N_x - 1);
        const size_t n_ref = eig ? 0 : (size_t)M_ref + 1;
        const size_t neig = eig ? (size_t)n_eig : 0;
        const size_t nd = 2 * (size_t)n_pts + n_ref + (size_t)(Mr + 1) + 2 * (size_t)N_q +
                          2 * (size_t)N_x + 3 + neig;
        double *buf = (double *)ctx->err_buf.get(nd * sizeof(double));
        double *dp = buf, *dw = dp + n_pts, *dref = dw + n_pts, *poly = dref + n_ref;
        double *approx = poly + (Mr + 1) + 2 * (size_t)N_q, *ref = approx + N_x, *out = ref + N_x;
        double *wsum = out + 2, *deig = wsum + 1;
        DOS_CUDA_TRY(cudaMemcpyAsync(dp, pts, (size_t)n_pts * 8, cudaMemcpyDefault, s));
        DOS_CUDA_TRY(cudaMemcpyAsync(dw, wts, (size_t)n_pts * 8, cudaMemcpyDefault, s));
        launch_normalize_weights(dw, n_pts, wsum, s);  // the weights as a probability measure
        launch_weighted_gauss(dp, dw, n_pts, 1.0, sigma, nullptr, x0, h, N_x, approx, s);
        if (eig) {
            DOS_CUDA_TRY(cudaMemcpyAsync(deig, eig, neig * 8, cudaMemcpyDefault, s));
            launch_blur_eigs(deig, n_eig, sigma, x0, h, N_x, ref, s);
        } else {
            DOS_CUDA_TRY(cudaMemcpyAsync(dref, ref_mu, n_ref * 8, cudaMemcpyDefault, s));
            launch_blur_kpm(dref, M_ref, ref_damping, lb, ub, sigma, N_q, x0, h, N_x, poly, ref, s);
        }
        launch_error_norms(approx, ref, N_x, h, out, s);
        double hv[3];
        DOS_CUDA_TRY(cudaMemcpyAsync(hv, out, sizeof(hv), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        DOS_REQUIRE(hv[2] > 0.0 && isfinite(hv[2]), "weights must have a positive finite sum");
        if (err_l1) *err_l1 = hv[0];
        if (err_inf) *err_inf = hv[1];
    });
}

int dos_heat_capacity(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                      const double *pts, const double *wts, int64_t n_pts, const double *betas,
                      int n_beta, double *cv, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(betas && cv && n_beta >= 1 && n_beta <= (1 << 20), "betas / cv / n_beta");
        DOS_REQUIRE((mu != nullptr) != (pts != nullptr), "give either moments or points");
        cudaStream_t s = (cudaStream_t)stream;
        if (mu) {
            DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
            DOS_REQUIRE(isfinite(lb) && isfinite(ub) && ub > lb, "need ub > lb");
            DOS_REQUIRE(damping == DOS_DAMP_NONE || damping == DOS_DAMP_JACKSON, "bad damping");
            const int N_q = std::max(4 * (M + 1), 2048);
            const size_t nd = (size_t)(M + 1) + (M + 1) + 2 * (size_t)N_q + 2 * (size_t)n_beta;
            double *buf = (double *)ctx->err_buf.get(nd * sizeof(double));
            double *dmu = buf, *scr = dmu + (M + 1), *db = scr + (M + 1) + 2 * (size_t)N_q;
            double *dout = db + n_beta;
            DOS_CUDA_TRY(cudaMemcpyAsync(dmu, mu, (M + 1) * 8, cudaMemcpyDefault, s));
            DOS_CUDA_TRY(cudaMemcpyAsync(db, betas, n_beta * 8, cudaMemcpyDefault, s));
            launch_heat_kpm(dmu, M, damping, lb, ub, N_q, db, n_beta, scr, dout, s);
            copy_out(cv, dout, n_beta * 8, s);
        } else {
            DOS_REQUIRE(wts && n_pts >= 1, "weights / n_pts");
            const size_t nd = 2 * (size_t)n_pts + 2 * (size_t)n_beta + 1;
            double *buf = (double *)ctx->err_buf.get(nd * sizeof(double));
            double *dp = buf, *dw = dp + n_pts, *db = dw + n_pts, *dout = db + n_beta;
            double *wsum = dout + n_beta;
            DOS_CUDA_TRY(cudaMemcpyAsync(dp, pts, (size_t)n_pts * 8, cudaMemcpyDefault, s));
            DOS_CUDA_TRY(cudaMemcpyAsync(dw, wts, (size_t)n_pts * 8, cudaMemcpyDefault, s));
            DOS_CUDA_TRY(cudaMemcpyAsync(db, betas, n_beta * 8, cudaMemcpyDefault, s));
            launch_normalize_weights(dw, n_pts, wsum, s);
            launch_heat_points(dp, dw, n_pts, 1.0, db, n_beta, dout, s);
            double hsum = 0.0;
            DOS_CUDA_TRY(cudaMemcpyAsync(&hsum, wsum, sizeof(double), cudaMemcpyDeviceToHost, s));
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
            DOS_REQUIRE(hsum > 0.0 && isfinite(hsum), "weights must have a positive finite sum");
            copy_out(cv, dout, n_beta * 8, s);
        }
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_moments_from_grid(dos_ctx *ctx, const double *phi_hat, int N_t, int M_out, double *mu,
                          void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(phi_hat && mu, "phi_hat / mu is NULL");
        DOS_REQUIRE(N_t >= 1 && N_t <= (1 << 24), "N_t must be in [1, 2^24]");
        DOS_REQUIRE(M_out >= 0 && M_out < N_t, "M_out must be in [0, N_t)");
        cudaStream_t s = (cudaStream_t)stream;
        double *buf = (double *)ctx->rec_in.get(((size_t)N_t + M_out + 1) * sizeof(double));
        double *dphi = buf, *dmu = buf + N_t;
        DOS_CUDA_TRY(cudaMemcpyAsync(dphi, phi_hat, N_t * sizeof(double), cudaMemcpyDefault, s));
        launch_grid_moments(dphi, N_t, M_out, dmu, s);
        copy_out(mu, dmu, (M_out + 1) * sizeof(double), s);
        if (!is_device_ptr(mu)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_smoothed_error(dos_ctx *ctx, const double *mu, int M, int damping, double lb, double ub,
                       const double *eig, int64_t n_eig, const double *ref_mu, int M_ref,
                       int ref_damping, double sigma, int N_x, double *err_l1, double *err_inf,
                       void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(mu != nullptr, "mu is NULL");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(isfinite(lb) && isfinite(ub) && ub > lb, "need ub > lb");
        DOS_REQUIRE(isfinite(sigma) && sigma > 0.0, "sigma must be > 0");
        DOS_REQUIRE(N_x >= 2 && N_x <= 1000000, "N_x must be in [2, 10^6]");
        DOS_REQUIRE(eig ? n_eig >= 1 : (ref_mu != nullptr && M_ref >= 0 && M_ref <= 100000),
                    "need eigenvalues or reference moments");
        DOS_REQUIRE(damping == DOS_DAMP_NONE || damping == DOS_DAMP_JACKSON, "bad damping");
        DOS_REQUIRE(eig || ref_damping == DOS_DAMP_NONE || ref_damping == DOS_DAMP_JACKSON,
                    "bad ref_damping");
        cudaStream_t s = (cudaStream_t)stream;
        const int Meff = eig ? M : std::max(M, M_ref);
        const double d = 0.5 * (ub - lb);
        const int64_t nq64 = std::max<int64_t>(4 * (int64_t)(Meff + 1),
                                               (int64_t)ceil(40.0 * d / sigma));
        DOS_REQUIRE(nq64 <= (1 << 24), "sigma too small for the quadrature (N_q > 2^24)");
        const int N_q = (int)nq64;
        const double x0 = lb - 6.0 * sigma;
        const double h = (ub - lb + 12.0 * sigma) / (N_x - 1);
        // scratch: mu | ref_mu | poly (M'+1 + 2 N_q) | approx (N_x) | ref (N_x) | out (2) | eig
        const size_t n_ref = eig ? 0 : (size_t)M_ref + 1;
        const size_t neig = eig ? (size_t)n_eig : 0;
        const size_t nd = (size_t)(M + 1) + n_ref + (size_t)(Meff + 1) + 2 * (size_t)N_q +
                          2 * (size_t)N_x + 2 + neig;
        double *buf = (double *)ctx->err_buf.get(nd * sizeof(double));
        double *dmu = buf, *dref = dmu + (M + 1), *poly = dref + n_ref;
        double *approx = poly + (Meff + 1) + 2 * (size_t)N_q, *ref = approx + N_x, *out = ref + N_x;
        double *deig = out + 2;
        DOS_CUDA_TRY(cudaMemcpyAsync(dmu, mu, (M + 1) * sizeof(double), cudaMemcpyDefault, s));
        launch_blur_kpm(dmu, M, damping, lb, ub, sigma, N_q, x0, h, N_x, poly, approx, s);
        if (eig) {
            DOS_CUDA_TRY(cudaMemcpyAsync(deig, eig, neig * sizeof(double), cudaMemcpyDefault, s));
            launch_blur_eigs(deig, n_eig, sigma, x0, h, N_x, ref, s);
        } else {
            DOS_CUDA_TRY(cudaMemcpyAsync(dref, ref_mu, n_ref * sizeof(double), cudaMemcpyDefault, s));
            launch_blur_kpm(dref, M_ref, ref_damping, lb, ub, sigma, N_q, x0, h, N_x, poly, ref, s);
        }
        launch_error_norms(approx, ref, N_x, h, out, s);
        double hv[2];
        DOS_CUDA_TRY(cudaMemcpyAsync(hv, out, sizeof(hv), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (err_l1) *err_l1 = hv[0];
        if (err_inf) *err_inf = hv[1];
    });
}

// ---- KPML and DGL (Sections 3.1.1, 3.1.3, Appendix B) -------------------------

int dos_legendre_moments(dos_ctx *ctx, const dos_csr *A, double lb, double ub, int M, int n_v,
                         uint64_t seed, int precision, double *nu, double *nu_per_vec,
                         const dos_kpm_opts *opts, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(A != nullptr, "matrix descriptor is NULL");
        DOS_REQUIRE(nu != nullptr, "nu is NULL");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(n_v >= 1 && n_v <= (1 << 20), "n_v must be in [1, 2^20]");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t per = (size_t)M + 1;
        const size_t rows = 1 + (nu_per_vec ? (size_t)n_v : 0);
        // scratch: Chebyshev moments (averaged row, then per-vector rows) | Legendre | h
        double *buf = (double *)ctx->leg_buf.get((2 * rows * per + per) * sizeof(double));
        double *dmu = buf, *dnu = buf + rows * per, *h = dnu + rows * per;
        SweepRequest r;
        r.B = 1;
        r.seg_rows = {0, A->n};
        r.lb = {lb};
        r.ub = {ub};
        r.M = M;
        r.n_v = n_v;
        r.seed = seed;
        r.precision = precision;
        r.mu = dmu;
        r.mu_pv = nu_per_vec ? dmu + per : nullptr;
        r.opts = opts ? *opts : default_opts();
        run_sweep(ctx, A, r, s);
        launch_cheb_to_legendre(dmu, (int64_t)rows, M, h, dnu, s);
        copy_out(nu, dnu, per * sizeof(double), s);
        if (nu_per_vec) copy_out(nu_per_vec, dnu + per, (size_t)n_v * per * sizeof(double), s);
        if (!is_device_ptr(nu) || (nu_per_vec && !is_device_ptr(nu_per_vec)))
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_cheb_to_legendre(dos_ctx *ctx, const double *mu, int64_t count, int M, double *nu,
                         void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(mu && nu && mu != nu, "mu / nu is NULL or aliased");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(count >= 1 && count * ((int64_t)M + 1) <= (int64_t(1) << 30),
                    "count * (M+1) must be in [1, 2^30]");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t tot = (size_t)count * (M + 1);
        double *buf = (double *)ctx->leg_buf.get((2 * tot + M + 1) * sizeof(double));
        double *dmu = buf, *dnu = buf + tot, *h = dnu + tot;
        DOS_CUDA_TRY(cudaMemcpyAsync(dmu, mu, tot * sizeof(double), cudaMemcpyDefault, s));
        launch_cheb_to_legendre(dmu, count, M, h, dnu, s);
        copy_out(nu, dnu, tot * sizeof(double), s);
        if (!is_device_ptr(nu)) DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_kpml_reconstruct(dos_ctx *ctx, const double *nu, int M, double lb, double ub,
                         const double *t, int N_t, double *phi_t, double *phi_lambda,
                         void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(nu && phi_t, "nu / phi_t is NULL");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(N_t >= 1 && N_t <= (1 << 26), "N_t must be in [1, 2^26]");
        DOS_REQUIRE(!phi_lambda || (isfinite(lb) && isfinite(ub) && ub > lb), "need ub > lb");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t per = (size_t)M + 1;
        double *buf = (double *)ctx->leg_buf.get((3 * per + 3 * (size_t)N_t) * sizeof(double));
        double *dnu = buf, *dt = buf + per, *dphi = dt + N_t, *dphl = dphi + N_t;
        double *coef = dphl + N_t;
        DOS_CUDA_TRY(cudaMemcpyAsync(dnu, nu, per * sizeof(double), cudaMemcpyDefault, s));
        if (t) DOS_CUDA_TRY(cudaMemcpyAsync(dt, t, N_t * sizeof(double), cudaMemcpyDefault, s));
        const double inv_d = phi_lambda ? 1.0 / (0.5 * (ub - lb)) : 0.0;
        launch_kpml(dnu, M, t ? dt : nullptr, nullptr, N_t, inv_d, dphi,
                    phi_lambda ? dphl : nullptr, coef, s);
        copy_out(phi_t, dphi, N_t * sizeof(double), s);
        if (phi_lambda) copy_out(phi_lambda, dphl, N_t * sizeof(double), s);
        if (!is_device_ptr(phi_t) || (phi_lambda && !is_device_ptr(phi_lambda)))
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_dgl(dos_ctx *ctx, const double *nu, int M, double lb, double ub, double sigma, double tol,
            const double *x, int N_x, double *phi, int *m_used, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(nu && phi, "nu / phi is NULL");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(isfinite(lb) && isfinite(ub) && ub > lb, "need ub > lb");
        DOS_REQUIRE(isfinite(sigma) && sigma > 0.0, "sigma must be > 0");
        DOS_REQUIRE(isfinite(tol), "tol must be finite");
        DOS_REQUIRE(N_x >= (x ? 1 : 2) && N_x <= 1000000, "N_x must be in [1 (2 for the grid), 10^6]");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t per = (size_t)M + 1;
        double *buf = (double *)ctx->leg_buf.get((per + 2 * (size_t)N_x) * sizeof(double) +
                                                 (size_t)N_x * sizeof(int));
        double *dnu = buf, *dx = buf + per, *dphi = dx + N_x;
        int *dused = (int *)(dphi + N_x);
        DOS_CUDA_TRY(cudaMemcpyAsync(dnu, nu, per * sizeof(double), cudaMemcpyDefault, s));
        if (x) DOS_CUDA_TRY(cudaMemcpyAsync(dx, x, N_x * sizeof(double), cudaMemcpyDefault, s));
        const double x0 = lb - 6.0 * sigma;
        const double h = x ? 0.0 : (ub - lb + 12.0 * sigma) / (N_x - 1);
        launch_dgl(dnu, M, 0.5 * (lb + ub), 0.5 * (ub - lb), sigma, tol, x ? dx : nullptr, x0, h,
                   N_x, dphi, m_used ? dused : nullptr, s);
        copy_out(phi, dphi, N_x * sizeof(double), s);
        if (m_used) copy_out(m_used, dused, N_x * sizeof(int), s);
        if (!is_device_ptr(phi) || (m_used && !is_device_ptr(m_used)))
            DOS_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int dos_legendre_error(dos_ctx *ctx, const double *nu, int M, int method, double lb, double ub,
                       double sigma, double tol, const double *eig, int64_t n_eig,
                       const double *ref_mu, int M_ref, int ref_damping, int N_x, double *err_l1,
                       double *err_inf, void *stream) {
    return guarded(ctx, [&] {
        DOS_REQUIRE(nu != nullptr, "nu is NULL");
        DOS_REQUIRE(method == DOS_LEG_KPML || method == DOS_LEG_DGL, "bad method");
        DOS_REQUIRE(M >= 0 && M <= 100000, "M must be in [0, 100000]");
        DOS_REQUIRE(isfinite(lb) && isfinite(ub) && ub > lb, "need ub > lb");
        DOS_REQUIRE(isfinite(sigma) && sigma > 0.0, "sigma must be > 0");
        DOS_REQUIRE(isfinite(tol), "tol must be finite");
        DOS_REQUIRE(N_x >= 2 && N_x <= 1000000, "N_x must be in [2, 10^6]");
        DOS_REQUIRE(eig ? n_eig >= 1 : (ref_mu != nullptr && M_ref >= 0 && M_ref <= 100000),
                    "need eigenvalues or reference moments");
        DOS_REQUIRE(eig || ref_damping == DOS_DAMP_NONE || ref_damping == DOS_DAMP_JACKSON,
                    "bad ref_damping");
        cudaStream_t s = (cudaStream_t)stream;
        const int Meff = eig ? M : std::max(M, M_ref);
        const double c = 0.5 * (lb + ub), d = 0.5 * (ub - lb);
        const int64_t nq64 = std::max<int64_t>(4 * (int64_t)(Meff + 1),
                                               (int64_t)ceil(40.0 * d / sigma));
        // Gauss-Legendre nodes cost O(N_q^2); the Chebyshev reference takes up to 2^24
        DOS_REQUIRE(nq64 <= (method == DOS_LEG_KPML ? (1 << 17) : (1 << 24)),
                    "sigma too small for the quadrature");
        const int N_q = (int)nq64;
        const double x0 = lb - 6.0 * sigma, h = (ub - lb + 12.0 * sigma) / (N_x - 1);
        const size_t per = (size_t)M + 1, n_ref = eig ? 0 : (size_t)M_ref + 1;
        const size_t neig = eig ? (size_t)n_eig : 0;
        // scratch: nu | ref_mu | blur_kpm scratch | approx | ref | out | eig | GL t, w, y, P
        const size_t n_coef = 2 * ((size_t)std::max(M, N_q) + 1);
        const size_t nd = per + n_ref + (size_t)(Meff + 1) + 2 * (size_t)N_q + 2 * (size_t)N_x +
                          2 + neig + 4 * (size_t)N_q + n_coef;
        double *buf = (double *)ctx->leg_aux.get(nd * sizeof(double));
        double *dnu = buf, *dref = dnu + per, *poly = dref + n_ref;
        double *approx = poly + (Meff + 1) + 2 * (size_t)N_q, *ref = approx + N_x;
        double *out = ref + N_x, *deig = out + 2, *gt = deig + neig, *gw = gt + N_q;
        double *gy = gw + N_q, *gP = gy + N_q, *coef = gP + N_q;
        DOS_CUDA_TRY(cudaMemcpyAsync(dnu, nu, per * sizeof(double), cudaMemcpyDefault, s));
        if (method == DOS_LEG_KPML) {
            launch_gauss_legendre(N_q, c, d, gt, gw, gy, coef, s);
            launch_kpml(dnu, M, gt, gw, N_q, 0.0, gP, nullptr, coef, s);
            launch_weighted_gauss(gy, gP, N_q, 1.0, sigma, nullptr, x0, h, N_x, approx, s);
        } else {
            launch_dgl(dnu, M, c, d, sigma, tol, nullptr, x0, h, N_x, approx, nullptr, s);
        }
        if (eig) {
            DOS_CUDA_TRY(cudaMemcpyAsync(deig, eig, neig * sizeof(double), cudaMemcpyDefault, s));
            launch_blur_eigs(deig, n_eig, sigma, x0, h, N_x, ref, s);
        } else {
            DOS_CUDA_TRY(cudaMemcpyAsync(dref, ref_mu, n_ref * sizeof(double), cudaMemcpyDefault, s));
            launch_blur_kpm(dref, M_ref, ref_damping, lb, ub, sigma, N_q, x0, h, N_x, poly, ref, s);
        }
        launch_error_norms(approx, ref, N_x, h, out, s);
        double hv[2];
        DOS_CUDA_TRY(cudaMemcpyAsync(hv, out, sizeof(hv), cudaMemcpyDeviceToHost, s));
        DOS_CUDA_TRY(cudaStreamSynchronize(s));
        if (err_l1) *err_l1 = hv[0];
        if (err_inf) *err_inf = hv[1];
    });
}

}  // extern "C"
