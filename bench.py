#!/usr/bin/env python
"""Benchmark of the KPM density-of-states path on GB300.

One "step" is one pass of the whole path over the workload: spectrum bounds
(Gershgorin) -> start vectors -> ceil(M/2) fused SpMM/recurrence/doubling-dot
steps -> moments -> Jackson reconstruction on a 1000-point t-grid -> the
sigma-smoothed L1/Linf error against a reference DOS.  The metric is Chebyshev
moments per second, nnz * n_v * M / t_step.

Default workload: the normalized Laplacian of a seeded Chung-Lu graph (n =
4,194,304, power-law expected degrees with exponent 2.5, mean degree 20, skewed
rows up to ~10^4 nonzeros), FP32 values and int32 indices; M = 1000, n_v = 256;
bounds [0, 2] padded by 1% per side, the interval that holds every normalized
Laplacian's spectrum and that this graph reaches at both ends (isolated
vertices and an isolated edge); Gershgorin's discs are ~20x wider and a
Lanczos run cannot see the isolated edge's eigenvalue 2.  FP32 vectors and SpMM with FP32 row sums accumulated as
float pairs and FP64; the FP64 form is measured too and reported under
"forms".  Inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload chunglu|anderson64|laplacian40|chunglu1m|batched|learned]
                    [--precision f32|f64]

Under torchrun (N > 1) every rank sweeps its own n_v start vectors (vector
offset rank * n_v) -- weak scaling, no collective on the data path; the moments
are combined once after timing with an all-reduce of M+1 doubles.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM traffic per step-kernel launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (workload, precision) together with the
# SHA-256 of the kernel source at capture time; a mismatch reports null.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (one pass), three
    # launches of the autotuned shape in the benchmark's launch configuration (tile
    # count included), mean read + write per launch
    ("anderson64", "f32"): {"bytes": 203623083, "src": "86278d722d815a32",
                            "launch": {"team": 4, "chunks": 2, "staged": 1, "chunk_bytes": 32,
                                       "tiles": 456, "panel": 0},
                            "note": "ncu, step_kernel<float,4,2,0,32,0>, 3 launches"},
    ("chunglu", "f32"): {"bytes": 89473691904, "src": "86278d722d815a32",
                         "launch": {"team": 32, "chunks": 2, "staged": 3, "chunk_bytes": 16,
                                    "depth": 2, "tiles": 4864, "panel": 0},
                         "note": "ncu on the full-size graph, step_tmag_kernel<float,32,2,0>, "
                                 "3 launches (1 pass)"},
}

WORKLOADS = {
    "anderson64": dict(kind="anderson", L=64, W=4.0, seed=2, M=500, n_v=64,
                       desc="3-D Anderson 64^3 periodic, W=4 (eps ~ U[-2,2]), hopping -1, seed 2"),
    "laplacian40": dict(kind="laplacian", m=40, M=100, n_v=20, seed=1,
                        desc="2-D 5-point Dirichlet Laplacian 40x40"),
    # bounds: "normalized_laplacian" = [0, 2] padded 1% per side; the
    # reference DOS of the smoothed error: ref_nv independent vectors in ref_prec;
    # f64_steps / e2e_steps: timed steps of those secondary forms (one warm-up each)
    "chunglu": dict(kind="chunglu", n=4194304, beta=2.5, mean_deg=20.0, seed=3, M=1000,
                    n_v=256, bounds="normalized_laplacian", ref_nv=1024, ref_prec="f32",
                    f64_steps=1, e2e_steps=2,
                    desc="normalized Laplacian of a Chung-Lu graph, n=4194304, "
                         "beta=2.5, mean degree 20, seed 3"),
    "chunglu1m": dict(kind="chunglu", n=1048576, beta=2.5, mean_deg=20.0, seed=3, M=200,
                      n_v=256, bounds="normalized_laplacian", ref_nv=1024, ref_prec="f32",
                      f64_steps=2, e2e_steps=2,
                      desc="normalized Laplacian of a Chung-Lu graph, n=1048576, "
                           "beta=2.5, mean degree 20, seed 3 (a quarter of the 4M-row "
                           "graph, small enough for counter captures)"),
    "batched": dict(kind="batched", count=512, seed=4, M=200, n_v=32,
                    desc="512 Anderson lattices, L ~ U{10..40}, W ~ U[1,16], seed 4"),
    # the learned moments-to-DOS network: instances (2/3 Anderson lattices, 1/3
    # Chung-Lu normalized Laplacians, n in [n_lo, n_hi]); the first held_out are
    # kept for scoring and for the timed serving step, the rest train the network
    # the network alone: Adam training steps at the learned workload's batch and
    # inference over a large batch, on random inputs (the tensor-core products)
    "mlp": dict(kind="mlp", n_in=64, n_hidden=512, n_out=256, batch=512, infer_rows=65536,
                desc="moments-to-DOS network 64-512-512-256, BF16 operands, FP32 accumulation"),
    "learned": dict(kind="learned", instances=20000, held_out=2000, n_lo=4096, n_hi=64000,
                    seed=5, n_v_in=4, M_in=64, n_v_ref=1024, M_ref=256, train_steps=20000,
                    batch=512, lr=1e-3, kpm_nv=(4, 16, 64, 256),
                    desc="learned moments-to-DOS network on generated Anderson lattices and "
                         "Chung-Lu graphs"),
}


# Per-method settings of the methods the paper compares with KPM (run with
# --method on the single-matrix workloads): Lanczos steps for the Lanczos DOS /
# Haydock (the paper reaches KPM's accuracy with about half the degree), the
# Lorentzian width for Haydock (in units of ub - lb), the DGL stop tolerance.
METHODS = {
    "lanczos": dict(M={"anderson64": 100, "laplacian40": 60}, precision="f64"),
    "haydock": dict(M={"anderson64": 100, "laplacian40": 60}, precision="f64", eta_frac=0.01),
    "kpml": dict(tol=1e-6),
    "dgl": dict(tol=1e-6),
}


def make_matrix(w):
    from synthetic import anderson_3d, chung_lu_normalized_laplacian, laplacian_2d
    if w["kind"] == "anderson":
        return anderson_3d(w["L"], w["W"], w["seed"])
    if w["kind"] == "laplacian":
        return laplacian_2d(w["m"])
    if w["kind"] == "chunglu":
        return chung_lu_normalized_laplacian(w["n"], w["beta"], w["mean_deg"], w["seed"])
    raise ValueError(w["kind"])


def step_kernel_name(shape, precision):
    """Name of the fused step kernel a launch shape runs (public staged values:
    1 direct loads, 2 TMA row panels, 3 TMA gathers; 0 / absent: direct)."""
    t = "double" if precision == "f64" else "float"
    staged = (shape or {}).get("staged", 1)
    base = {2: "step_staged_kernel", 3: "step_tmag_kernel",
            4: "step_csrs_kernel"}.get(staged, "step_kernel")
    return f"{base}<{t}>"


def algorithmic_bytes_per_step(n, nnz, n_v, precision):
    """Compulsory bytes of one fused step: CSR once (col_idx 4 B + value) plus
    row_ptr, X_k read once, X_{k-1} read and X_{k+1} written."""
    s = 8 if precision == "f64" else 4
    return nnz * (4 + s) + 4 * (n + 1) + 3 * n * n_v * s


def pinning_bound(col_idx, n, nnz, n_v, precision, l2_bytes):
    """Least DRAM traffic of one fused step if the L2 held, for the whole step, the
    rows of X_k that the most nonzeros gather (a static choice; the best any
    ordering or eviction policy can do without temporal locality): the gathers of
    the other rows come from DRAM, plus X_{k-1} read, X_{k+1} written and the CSR."""
    s = 8 if precision == "f64" else 4
    row_bytes = n_v * s
    refs = np.sort(np.bincount(col_idx, minlength=n))[::-1]
    held = int(min(n, l2_bytes // row_bytes))
    hit = float(refs[:held].sum() / max(1, refs.sum()))
    byts = nnz * row_bytes * (1.0 - hit) + 2 * n * row_bytes + nnz * (4 + s) + 4 * (n + 1)
    return {"l2_bytes": int(l2_bytes), "rows_held": held, "hit_fraction": hit,
            "bytes_per_launch": byts}


def panel_geometry(n_v, panel, precision):
    """Vector panels of a sweep as the library forms them (launch.panel): n_panels
    passes over A of panel_nv vectors (the last possibly narrower), rows of ld
    elements (whole 16-byte chunks)."""
    vpt = 2 if precision == "f64" else 4
    w = min(panel or 256, 256)
    n_panels = -(-n_v // w)
    panel_nv = -(-n_v // n_panels)
    return n_panels, panel_nv, -(-panel_nv // vpt) * vpt


def fma_per_step(n, nnz, n_v):
    """FMAs of one fused step: nnz*n_v (SpMM) + 2 n n_v (shift, recurrence) + 2 n n_v (dots)."""
    return nnz * n_v + 4 * n * n_v


# The spectrum of a normalized Laplacian I - D^-1/2 A D^-1/2 lies in [0, 2];
# padded by 1% of the width per side.
NORMALIZED_LAPLACIAN_BOUNDS = (-0.02, 2.02)

# GB300's FP64 rate is not measured here: NVIDIA's nominal figure, next to which
# the FP64 fused step's ncu FP64-pipe utilisation is the evidence of the bound.
FP64_NOMINAL_TFLOPS = 1.25
FP64_PEAK_SOURCE = ("nominal FP64 rate of GB300 (1.25 TFLOP/s, not measured); ncu: FP64 pipe "
                    "91% busy in the fused step on the 64^3 lattice")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(device):
    import torch
    try:
        u = torch.cuda.get_device_properties(device).uuid
        return "GPU-" + str(u)
    except Exception:
        return str(device)


def kernel_source_hash():
    """SHA-256 of the sweep kernels' source (kpm_kernels.cu: every variant of the
    fused step and its helpers), so a stored ncu figure is dropped as soon as any
    of them changes."""
    with open(os.path.join(ROOT, "paper_1308_5467_gb300", "csrc", "kpm_kernels.cu")) as f:
        src = f.read()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def oracle_sample(A, lb, ub, M, n_v_full, seed, target_s, cores):
    """(vectors, degree) of a bounded oracle sample of about target_s seconds on
    `cores` threads: the full degree M with as many start vectors as fit (at least
    one per thread), or -- when one doubling pass over A already costs most of the
    budget (the 4-million-row graph) -- one vector per thread at a reduced even
    degree; the sweep costs ceil(M/2) passes, so the rate scales linearly."""
    from oracle import kpm as okpm
    probe = max(1, min(cores, n_v_full))
    t0 = time.perf_counter()
    okpm.kpm_moments_per_vector(A, lb, ub, 4, probe, seed, nthreads=cores)
    t_pass = max((time.perf_counter() - t0) / 2, 1e-6)   # one pass of `probe` vectors
    t_full = t_pass * max(1, (M + 1) // 2)
    if t_full <= target_s:
        nv = int(min(4 * n_v_full, probe * max(1, int(target_s / t_full))))
        nv = max(probe, (nv // cores) * cores if nv >= cores else nv)
        return nv, M
    return probe, int(min(M, max(2, 2 * int(target_s / t_pass))))


def cpu_baseline(A, lb, ub, M, n_v_full, seed, target_s=12.0):
    """The oracle as it stands, on the host cores, over a bounded sample of the
    same matrix, bounds and start vectors (see oracle_sample)."""
    from oracle import kpm as okpm
    cores = os.cpu_count() or 1
    nv, Ms = oracle_sample(A, lb, ub, M, n_v_full, seed, target_s, cores)
    t0 = time.perf_counter()
    okpm.kpm_moments_per_vector(A, lb, ub, Ms, nv, seed, nthreads=cores)
    t = time.perf_counter() - t0
    value = A.nnz * nv * Ms / t
    scaled = "" if Ms == M else f", timed at M={Ms} and scaled linearly to M={M}"
    # the same oracle on one thread, for reference: ~target_s / 3
    per_vec_1 = t * min(cores, nv) / nv
    n1 = int(max(1, min(nv, (target_s / 3) / max(per_vec_1, 1e-6))))
    M1 = Ms if per_vec_1 <= target_s / 3 else int(max(2, 2 * ((Ms * (target_s / 3)
                                                                / per_vec_1) // 2)))
    t0 = time.perf_counter()
    okpm.kpm_moments_per_vector(A, lb, ub, M1, n1, seed, nthreads=1)
    t1 = time.perf_counter() - t0
    scaled1 = "" if M1 == M else f", timed at M={M1} and scaled linearly to M={M}"
    single = {"value": A.nnz * n1 * M1 / t1, "cores": 1,
              "sample": f"{n1} start vectors, {t1:.1f} s wall on 1 thread{scaled1}"}
    return {"value": value, "unit": "moments/s", "cores": min(cores, nv), "kind": "oracle",
            "sample": f"{nv} start vectors of the same workload (M={Ms}, doubling mode, FP64), "
                      f"{t:.1f} s wall on {min(cores, nv)} threads{scaled}",
            "single_thread": single}


def run_reference(args):
    """The reference arm: the CPU oracle, timed as it stands on the host cores,
    each step a bounded sample of the workload (about 90 s / (K + W) per step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    if w["kind"] == "batched":
        return run_reference_batched(args, w)
    if w["kind"] == "learned":
        return run_reference_learned(args, w)
    if w["kind"] == "mlp":
        return run_reference_mlp(args, w)
    if args.method != "kpm":
        return run_reference_method(args, w)
    from oracle import bounds as obounds
    from oracle import kpm as okpm
    A = make_matrix(w)
    if args.precision == "f32":
        A = A.astype(np.float32)
    if w.get("bounds") == "normalized_laplacian":
        lb, ub = NORMALIZED_LAPLACIAN_BOUNDS
    else:
        lb, ub = obounds.bounds(A, w.get("bounds", "gershgorin"), steps=20, seed=w["seed"],
                                pad_frac=0.01)
    M = w["M"]
    cores = os.cpu_count() or 1
    step_s = min(6.0, max(0.5, 90.0 / max(1, args.steps + args.warmup)))
    nv, Ms = oracle_sample(A, lb, ub, M, w["n_v"], w["seed"], step_s, cores)
    nv = min(nv, max(1, min(cores, w["n_v"])))
    for _ in range(min(args.warmup, 1)):
        okpm.kpm_moments_per_vector(A, lb, ub, min(Ms, 20), nv, w["seed"], nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        okpm.kpm_moments_per_vector(A, lb, ub, Ms, nv, w["seed"], nthreads=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = A.nnz * nv * Ms / t
    scaled = "" if Ms == M else f"; degree reduced to M={Ms}, the rate scales linearly in M"
    sample = (f"each step: {nv} of the {w['n_v']} start vectors of {args.workload} "
              f"(M={Ms}, FP64 oracle, doubling mode) on {min(cores, nv)} host threads{scaled}")
    line = {"metric": "Chebyshev moments/sec (nnz*n_v*M/s)", "value": value,
            "unit": "moments/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": A.n, "nnz": A.nnz, "M": M,
                       "n_v": w["n_v"], "n_v_sample": nv, "M_sample": Ms,
                       "bounds": w.get("bounds", "gershgorin")},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "moments/s", "cores": min(cores, nv),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "moments/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_learned(args, w):
    """Reference arm of the learned workload: its serving path on the host cores
    with the oracle -- FP64 KPM oracle (n_v = 4, M = 64) and the FP64 network
    reference with bfloat16 operands emulated -- over a bounded sample of the
    held-out instances.  The cost does not depend on the weights, so the network
    is the reference's own initialisation (no training on the host)."""
    from oracle import bounds as obounds
    from oracle import kpm as okpm
    from oracle import mlp as omlp
    from synthetic.instances import learned_instance_specs, make_instance
    specs = learned_instance_specs(w["instances"], w["seed"], w["n_lo"], w["n_hi"])
    cores = os.cpu_count() or 1
    step_s = min(6.0, max(0.5, 90.0 / max(1, args.steps + args.warmup)))
    p = omlp.init_params(w["M_in"], 512, 256, 3)
    seed_in = w["seed"] * 1000 + 1
    mats, t_est = [], 0.0
    for b, sp in enumerate(specs[:w["held_out"]]):
        A = make_instance(sp)
        if "chung" in A.meta["family"]:
            lb, ub = -0.02, 2.02
        else:
            lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
        t0 = time.perf_counter()
        mu = okpm.kpm_moments(A, lb, ub, w["M_in"], w["n_v_in"], seed_in, batch_index=b,
                              nthreads=cores)
        omlp.forward(p, mu[1:][None, :].astype(np.float32).astype(np.float64), bf16=True)
        t_est += time.perf_counter() - t0
        mats.append((b, A, lb, ub))
        if t_est >= step_s:
            break

    def one():
        for b, A, lb, ub in mats:
            mu = okpm.kpm_moments(A, lb, ub, w["M_in"], w["n_v_in"], seed_in, batch_index=b,
                                  nthreads=cores)
            omlp.forward(p, mu[1:][None, :].astype(np.float32).astype(np.float64), bf16=True)
    for _ in range(min(args.warmup, 1)):
        one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = len(mats) / t
    sample = (f"each step: {len(mats)} of the {w['held_out']} held-out instances, FP64 KPM "
              f"oracle (n_v={w['n_v_in']}, M={w['M_in']}) + FP64 network reference, "
              f"{cores} threads")
    line = {"metric": "DOS/sec (learned: n_v=4, M=64 sweep + network, 256-point DOS)",
            "value": value, "unit": "DOS/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "instances": w["instances"],
                       "held_out": w["held_out"], "sampled": len(mats)},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "DOS/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOS/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_mlp(args, w):
    """Reference arm of the network workload: the FP64 network reference (bfloat16
    operands emulated) as it stands, one Adam step per step on the same batch size."""
    from oracle import mlp as omlp
    B = w["batch"]
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (B, w["n_in"]))
    t = rng.uniform(0, 1, (B, w["n_out"]))
    p = omlp.init_params(w["n_in"], w["n_hidden"], w["n_out"], 3)
    m = {k: np.zeros_like(a) for k, a in p.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, g = omlp.loss_and_grads(p, x, t, bf16=True)
        p, m, v = omlp.adam_step(p, g, m, v, i + 1, 1e-4)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    value = B / dt
    cores = os.cpu_count() or 1
    line = {"metric": "training samples/sec (Adam steps of the moments-to-DOS network)",
            "value": value, "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "batch": B}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each step: one Adam step of batch {B}, FP64 network "
                                       f"reference (NumPy)"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batched_sample(mats, M, n_v, step_s, cores):
    """Matrices of the 512-lattice batch for a bounded oracle sample: a spread of
    sizes (the smallest, the largest and evenly spaced indices), as many as fit
    in about step_s seconds at the full M and n_v."""
    from oracle import kpm as okpm
    sizes = np.array([m.n for m in mats])
    # the smallest, the largest, then every matrix in a fixed stride-37 order
    order = [int(np.argmin(sizes)), int(np.argmax(sizes))] + \
        [(37 * i) % len(mats) for i in range(len(mats))]
    picks, t_used = [], 0.0
    for b in order:
        if b in picks:
            continue
        t0 = time.perf_counter()
        okpm.kpm_moments(mats[b], -20.0, 20.0, min(M, 8), n_v, 0, batch_index=b,
                         nthreads=cores)
        t_est = (time.perf_counter() - t0) * max(1.0, M / 8.0)
        if picks and t_used + t_est > step_s:
            break
        picks.append(b)
        t_used += t_est
    return picks


def run_reference_batched(args, w):
    """Reference arm of the 512-lattice workload: the oracle, matrix by matrix with
    each matrix's own start-vector counters, over a bounded sample of the batch."""
    from oracle import bounds as obounds
    from oracle import kpm as okpm
    from synthetic import batched_anderson
    mats = batched_anderson(w["count"], w["seed"])
    if args.precision == "f32":
        mats = [m.astype(np.float32) for m in mats]
    M, n_v = w["M"], w["n_v"]
    cores = os.cpu_count() or 1
    step_s = min(6.0, max(0.5, 90.0 / max(1, args.steps + args.warmup)))
    picks = batched_sample(mats, M, n_v, step_s, cores)
    bnds = [obounds.bounds(mats[b], "gershgorin", pad_frac=0.01) for b in picks]

    def one():
        for b, (lb, ub) in zip(picks, bnds):
            okpm.kpm_moments(mats[b], lb, ub, M, n_v, w["seed"], batch_index=b, nthreads=cores)
    for _ in range(min(args.warmup, 1)):
        one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    nnz = sum(mats[b].nnz for b in picks)
    value = nnz * n_v * M / t
    sample = (f"each step: {len(picks)} of the {len(mats)} lattices (n from "
              f"{min(mats[b].n for b in picks)} to {max(mats[b].n for b in picks)}), all "
              f"{n_v} start vectors, M={M}, FP64 oracle one matrix at a time on {cores} threads")
    line = {"metric": "Chebyshev moments/sec (nnz*n_v*M/s)", "value": value,
            "unit": "moments/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "B": len(mats), "M": M, "n_v": n_v,
                       "sampled_matrices": picks, "nnz_sample": nnz},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "moments/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "moments/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_method(args, w):
    """Reference arm for --method: the method's oracle on a sample of start vectors."""
    from oracle import bounds as obounds
    from oracle import lanczos_dos as old
    from oracle import legendre as oleg
    method = args.method
    A = make_matrix(w)
    lanczos = method in ("lanczos", "haydock")
    if not lanczos and args.precision == "f32":
        A = A.astype(np.float32)
    M = METHODS[method]["M"][args.workload] if lanczos else w["M"]
    lb, ub = obounds.bounds(A, "gershgorin", pad_frac=0.01)
    cores = os.cpu_count() or 1
    nv = 2 if lanczos else max(1, min(cores, w["n_v"]))

    def one():
        if lanczos:
            old.lanczos_ritz(A, M, nv, w["seed"])
        else:
            oleg.legendre_moments_per_vector(A, lb, ub, M, nv, w["seed"], nthreads=cores)
    if args.warmup:
        one()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = A.nnz * nv * M / t
    unit = "products/s" if lanczos else "moments/s"
    threads = 1 if lanczos else min(cores, nv)
    sample = (f"each step: {nv} of the {w['n_v']} start vectors of {args.workload}, "
              f"{method} oracle (M={M}, FP64) on {threads} host threads")
    line = {"metric": ("Lanczos block products/sec (nnz*n_v*M/s)" if lanczos
                       else "Legendre moments/sec (nnz*n_v*M/s)"),
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "method": method, "n": A.n, "nnz": A.nnz,
                       "M": M, "n_v": w["n_v"], "n_v_sample": nv},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args, w, world, rank, local, device):
    """512 Anderson lattices of uneven size in one launch per Chebyshev step.

    A step: Gershgorin bounds of all matrices (one pass) and the batched sweep
    (M = 200, n_v = 32).  Also timed: the FP64 batched form and the plain FP64
    path (one dos_kpm_moments call per matrix), with the smoothed L1 error of
    sampled matrices in each form against an FP64 n_v = 512 reference."""
    import torch
    import torch.distributed as dist

    from paper_1308_5467_gb300 import dos
    from synthetic import batched_anderson, concat_block_diagonal

    mats = batched_anderson(w["count"], w["seed"])
    rp, ci, va, seg = concat_block_diagonal(mats)
    M, n_v = w["M"], w["n_v"]
    prec = args.precision
    vdt = np.float32 if prec == "f32" else np.float64
    t_rp, t_ci = torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device)
    A = dos.CSRArrays(int(seg[-1]), t_rp, t_ci, torch.from_numpy(va.astype(vdt)).to(device))
    A64 = dos.CSRArrays(int(seg[-1]), t_rp, t_ci, torch.from_numpy(va).to(device))
    ctx = dos.Context(local)
    nnz = int(ci.shape[0])
    units = nnz * n_v * M

    def step(Acsr, precision):
        lb, ub = ctx.dos_bounds_batched(Acsr, seg, pad_frac=0.01)
        return lb, ub, ctx.dos_kpm_moments_batched(Acsr, seg, lb, ub, M, n_v, seed=w["seed"],
                                                   precision=precision, batch_index=0,
                                                   flags=dos.DOS_OPT_NO_PDL if args.no_pdl else 0)

    def timed(fn, steps, warmup, profile=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        if profile:
            ctx.dos_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = None
        for _ in range(steps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        prof = ctx.dos_profile_read() if profile else None
        if profile:
            ctx.dos_profile_enable(False)
        ms = e0.elapsed_time(e1) / steps
        if world > 1:
            t = torch.tensor([ms], device=device, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, out, prof

    tuned_b = ctx.dos_tune(A, n_v, prec, seg_rows=seg)[0]   # autotuned shape, cached in ctx
    with ClockSampler(gpu_id_for(local)) as clk:
        ms, (lb, ub, mu), prof = timed(lambda: step(A, prec), args.steps, args.warmup, True)
    value = units * world / (ms * 1e-3)
    peaks, peak_kind = measured_peaks()
    launch_ms = prof["step_ms"] / max(1, prof["step_launches"])
    n_rows = int(seg[-1])
    alg = algorithmic_bytes_per_step(n_rows, nnz, n_v, prec)
    achieved = alg / (launch_ms * 1e-3) / 1e9
    forms = {prec: {"ms_per_step": ms, "value": value, "steps": args.steps}}
    # FP64 batched, and plain FP64 KPM one matrix at a time
    st64 = max(2, args.steps // 4)
    ms64, (_, _, mu64), _ = timed(lambda: step(A64, "f64"), st64, 1)
    forms["f64_batched"] = {"ms_per_step": ms64, "value": units * world / (ms64 * 1e-3),
                            "steps": st64}
    singles = [dos.CSRArrays.from_synthetic(m, device=device) for m in mats]

    def plain():
        return [ctx.dos_kpm_moments(S, lb[b], ub[b], M, n_v, seed=w["seed"], precision="f64",
                                    batch_index=b) for b, S in enumerate(singles)]
    ms_plain, mu_plain, _ = timed(plain, 1, 1)
    forms["f64_plain_per_matrix"] = {"ms_per_step": ms_plain, "steps": 1,
                                     "value": units * world / (ms_plain * 1e-3)}
    # smoothed L1 error of sampled matrices against an FP64 n_v = 512 reference, in
    # each form (the same start vectors in all three)
    picks = [0, 100, 255, 511]
    errs = {prec: [], "f64_batched": [], "f64_plain_per_matrix": []}
    for b in picks:
        ref = ctx.dos_kpm_moments(singles[b], lb[b], ub[b], M, 512, seed=w["seed"] + 77,
                                  precision="f64", batch_index=b)
        sig = 0.02 * (ub[b] - lb[b])
        for key, m in ((prec, mu[b]), ("f64_batched", mu64[b]),
                       ("f64_plain_per_matrix", mu_plain[b])):
            errs[key].append(ctx.dos_smoothed_error(m, M, "jackson", lb[b], ub[b], sig,
                                                    ref_mu=ref)[0])
    for key, v in errs.items():
        forms[key]["e1_sampled"] = float(np.mean(v))
    forms["f64_batched"]["max_abs_diff_vs_" + prec] = float(np.abs(mu64 - mu).max())

    # end to end: host (pinned) CSR through the same C-ABI calls, which copy it in
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(rp).pin_memory()
        ci_h = torch.from_numpy(ci).pin_memory()
        va_h = torch.from_numpy(va.astype(vdt)).pin_memory()
        Ah = dos.CSRArrays(n_rows, rp_h, ci_h, va_h)
        st_e2e = max(3, args.steps // 2)
        ms_e2e, _, _ = timed(lambda: step(Ah, prec), st_e2e, 1)
        h2d = 2 * (rp_h.numel() * 4 + ci_h.numel() * 4 + va_h.numel() * va_h.element_size())
        d2h = len(mats) * (M + 1) * 8 + 2 * len(mats) * 8
        e2e = {"value": units * world / (ms_e2e * 1e-3), "unit": "moments/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "steps": st_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import kpm as okpm
        cores = os.cpu_count() or 1
        mats_h = [m.astype(vdt) for m in mats]
        cpu_picks = batched_sample(mats_h, M, n_v, 12.0, cores)
        t0 = time.perf_counter()
        for b in cpu_picks:
            okpm.kpm_moments(mats_h[b], lb[b], ub[b], M, n_v, w["seed"], batch_index=b,
                             nthreads=cores)
        t = time.perf_counter() - t0
        nnz_s = sum(mats_h[b].nnz for b in cpu_picks)
        cpu = {"value": nnz_s * n_v * M / t, "unit": "moments/s", "cores": cores,
               "kind": "oracle",
               "sample": f"{len(cpu_picks)} of the {len(mats)} lattices (n from "
                         f"{min(mats[b].n for b in cpu_picks)} to "
                         f"{max(mats[b].n for b in cpu_picks)}), all {n_v} start vectors, "
                         f"M={M}, FP64 oracle one matrix at a time, {t:.1f} s wall on {cores} "
                         f"threads"}
    if rank == 0:
        line = {
            "metric": "Chebyshev moments/sec (nnz*n_v*M/s)", "value": value, "unit": "moments/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "f32" else "f64", "data": "synthetic",
            "config": {"workload": "batched", "desc": w["desc"], "B": len(mats), "n": n_rows,
                       "nnz": nnz, "M": M, "n_v": n_v, "precision": prec, "pdl": not args.no_pdl,
                       "launch": tuned_b,
                       "l2": "inputs larger than L2: %.0f MB per fused step" % (alg / 1e6)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": peak_kind, "launch_ms": launch_ms,
                         "kernel": step_kernel_name(tuned_b, prec),
                         "algorithmic_bytes_per_launch": alg},
            "forms": forms, "e1_sampled": float(np.mean(errs[prec])),
            "gpu_launches": prof["launches"], "clocks": clk.summary(), "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    return 0


def run_learned(args, w, world, rank, local, device):
    """The learned part at its configured scale.

    Setup (reported, not timed as the step): generate the instances (host pool),
    sweep them for the network's inputs (n_v = 4, M = 64) and targets (n_v = 1024,
    M = 256 Jackson DOS on 256 nodes), train the network on all but the held-out
    instances.  A step is the serving path over all held-out instances: bounds,
    the batched n_v = 4, M = 64 sweep and the network reading the moments in
    place -- one DOS per instance on the 256-point grid.  Metric: DOS per second,
    next to the held-out smoothed L1 error of the network and of plain Jackson KPM
    at n_v = 4, and the plain-KPM path at the vector count that matches the
    network's error (DOS/s at equal error)."""
    import torch

    from paper_1308_5467_gb300 import dos, learned
    from synthetic.instances import learned_instance_specs, stream_instances
    count = w["instances"] if not args.instances else args.instances
    held = max(1, min(w["held_out"], count // 10)) if args.instances else w["held_out"]
    specs = learned_instance_specs(count, w["seed"], w["n_lo"], w["n_hi"])
    seed_in = w["seed"] * 1000 + 1
    ctx = dos.Context(local)
    t0 = time.perf_counter()
    stream = stream_instances(specs)
    held_mats = (next(stream) for _ in range(held))
    test = learned.make_dataset(ctx, held_mats, seed_in, w["n_v_in"], w["M_in"], w["n_v_ref"],
                                w["M_ref"], b0=0, keep_groups=True)
    train = learned.make_dataset(ctx, stream, seed_in, w["n_v_in"], w["M_in"], w["n_v_ref"],
                                 w["M_ref"], b0=held, tune=True)
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    steps = args.train_steps or w["train_steps"]
    net = learned.train(ctx, train["x"], train["y"], steps=steps, batch=w["batch"], lr=w["lr"],
                        seed=3)
    train_s = time.perf_counter() - t1
    e_kpm4, e_net = learned.score(ctx, test, net)
    curve = {}
    for nv in w["kpm_nv"]:
        curve[nv] = float(learned.kpm_errors(ctx, test, nv, w["M_ref"], seed_in).mean())
    match = next((nv for nv in w["kpm_nv"] if curve[nv] <= e_net.mean()), None)

    groups = test["groups"]
    pipe = learned.LearnedPipeline(ctx, net, groups, seed_in, w["n_v_in"], w["M_in"])

    def timed(fn, steps_, warmup, profile=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if profile:
            ctx.dos_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps_):
            fn()
        e1.record()
        torch.cuda.synchronize()
        prof = ctx.dos_profile_read() if profile else None
        if profile:
            ctx.dos_profile_enable(False)
        return e0.elapsed_time(e1) / steps_, prof

    with ClockSampler(gpu_id_for(local)) as clk:
        ms, prof = timed(pipe.run, args.steps, args.warmup, profile=True)
    value = held / (ms * 1e-3)
    # the plain-KPM path at the matching vector count (or the largest tried)
    nv_eq = match or w["kpm_nv"][-1]
    kpm = learned.KPMPipeline(ctx, groups, seed_in, nv_eq, w["M_ref"])
    ms_kpm, _ = timed(kpm.run, max(2, args.steps // 4), 1)
    kpm4 = learned.KPMPipeline(ctx, groups, seed_in, w["n_v_in"], w["M_in"])
    ms_kpm4, _ = timed(kpm4.run, max(2, args.steps // 4), 1)
    # end to end: host CSR and a host read of every DOS, through the same calls
    e2e = None
    if not args.no_e2e:
        for g in groups:
            assert g.host_A is not None      # pin the host copies before the timed region
        ms_e2e, _ = timed(lambda: pipe.run(host=True).cpu(), max(2, args.steps // 2), 1)
        h2d = 2 * sum(g.host_bytes for g in groups)
        e2e = {"value": held / (ms_e2e * 1e-3), "unit": "DOS/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": held * net.n_out * 4, "ms_per_step": ms_e2e}
    # roofline of the fused step kernel of the sweep (the dominant kernel)
    peaks, peak_kind = measured_peaks()
    launch_ms = prof["step_ms"] / max(1, prof["step_launches"])
    S = max(1, (w["M_in"] + 1) // 2)
    alg = sum(algorithmic_bytes_per_step(g.n, g.nnz, w["n_v_in"], "f32") for g in groups) / \
        len(groups)
    achieved = alg / (launch_ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = learned_cpu_baseline(ctx, net, test, groups, w, seed_in)
    hold_n = test["n"]
    line = {
        "metric": "DOS/sec (learned: n_v=4, M=64 sweep + network, 256-point DOS)",
        "value": value, "unit": "DOS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 sweep, bf16 network (FP32 accumulation)",
        "data": "synthetic",
        "config": {"workload": "learned", "desc": w["desc"], "instances": count,
                   "train_instances": count - held, "held_out": held,
                   "n_range": [w["n_lo"], w["n_hi"]],
                   "held_out_rows": int(hold_n.sum()), "held_out_laplacians":
                       int(test["laplacian"].sum()),
                   "inputs": f"mu_1..mu_{w['M_in']} from n_v={w['n_v_in']}",
                   "targets": f"Jackson DOS at 256 Chebyshev nodes from n_v={w['n_v_ref']}, "
                              f"M={w['M_ref']}",
                   "network": "64-512-512-256 ReLU, BF16 operands, FP32 accumulation, Adam",
                   "train_steps": steps, "batch": w["batch"],
                   "l2": "inputs larger than L2: %.1f GB of CSR held out" %
                         (sum(g.host_bytes for g in groups) / 1e9)},
        "e1_network": float(e_net.mean()), "e1_jackson_nv4_M64": float(e_kpm4.mean()),
        "e1_jackson_M256_by_nv": {str(k): v for k, v in curve.items()},
        "equal_error": {"kpm_nv": nv_eq, "reached": match is not None,
                        "kpm_M": w["M_ref"], "kpm_dos_per_s": held / (ms_kpm * 1e-3),
                        "kpm_ms_per_step": ms_kpm},
        "jackson_nv4_M64": {"dos_per_s": held / (ms_kpm4 * 1e-3), "ms_per_step": ms_kpm4},
        "setup": {"generation_s": gen_s, "host_wait_s": test["timing"]["host_wait_s"] +
                  train["timing"]["host_wait_s"],
                  "gpu_sweep_s": test["timing"]["gpu_s"] + train["timing"]["gpu_s"],
                  "gpu_moments_per_s": (test["timing"]["moments"] + train["timing"]["moments"])
                  / max(1e-9, test["timing"]["gpu_s"] + train["timing"]["gpu_s"]),
                  "train_s": train_s, "train_samples_per_s": steps * w["batch"] / train_s},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": peak_kind, "kernel": "fused sweep step (n_v = 4)",
                     "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms,
                     "steps_per_sweep": S},
        "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": prof["launches"],
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_mlp(args, w, world, rank, local, device):
    """The network's tensor-core path on its own: a step is one Adam training step
    on a batch (forward, L1 loss, backward, update: nine products), and inference
    over infer_rows rows is timed alongside (three products per 8192-row slice),
    which gives the products' throughput against the tensor-core peak."""
    import torch

    from paper_1308_5467_gb300 import dos
    ctx = dos.Context(local)
    n_in, nh, n_out, B = w["n_in"], w["n_hidden"], w["n_out"], w["batch"]
    net = dos.MLP(ctx, n_in, nh, n_out, seed=3)
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.rand((B, n_in), generator=g).to(device) * 2 - 1
    t = torch.rand((B, n_out), generator=g).to(device)
    R = w["infer_rows"]
    xi = (torch.rand((R, n_in), generator=g) * 2 - 1).to(device)
    yi = torch.empty((R, n_out), dtype=torch.float32, device=device)
    flops_row = 2 * (n_in * nh + nh * nh + nh * n_out)     # forward products per row

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    with ClockSampler(gpu_id_for(local)) as clk:
        ms = timed(lambda: net.dos_mlp_train_step(x, t, 1e-4, want_loss=False), args.steps,
                   args.warmup)
        # one slice of R rows: the input staging kernel, the three products and the
        # copy of the output into yi -- the products' rate is understated by the rest
        ms_inf = timed(lambda: net.dos_mlp_infer(xi, out=yi, max_rows=R), max(3, args.steps // 2),
                       1)
    peaks, peak_kind = measured_peaks()
    tflops = R * flops_row / (ms_inf * 1e-3) / 1e12
    train_flops = 3 * B * flops_row       # forward + the two backward products per layer
    # end to end: host inputs and targets copied in and the loss read back every step
    xh, th = x.cpu().pin_memory(), t.cpu().pin_memory()
    ms_e2e = timed(lambda: net.dos_mlp_train_step(xh.numpy(), th.numpy(), 1e-4), max(3, args.steps // 2), 1)
    line = {
        "metric": "training samples/sec (Adam steps of the moments-to-DOS network)",
        "value": B / (ms * 1e-3), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (FP32 accumulation)", "data": "synthetic",
        "config": {"workload": "mlp", "desc": w["desc"], "batch": B, "infer_rows": R,
                   "l2": "weights 0.9 MB stay in L2; inference inputs/outputs %d MB"
                         % ((R * (n_in + n_out) * 4) >> 20)},
        "train_tflops": train_flops / (ms * 1e-3) / 1e12,
        "inference": {"rows": R, "ms": ms_inf, "rows_per_s": R / (ms_inf * 1e-3),
                      "tflops": tflops},
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peaks["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": tflops / peaks["bf16_tflops"], "traffic": None,
                     "peak_source": f"{peak_kind} bf16 (cuBLAS burst)",
                     "kernel": "gemm_tc_kernel (tcgen05.mma, inference products)",
                     "flops_per_launch": R * flops_row / 3, "launch_ms": ms_inf / 3},
        "e2e": {"value": B / (ms_e2e * 1e-3), "unit": "samples/s",
                "h2d_bytes_per_step": B * (n_in + n_out) * 4, "d2h_bytes_per_step": 4,
                "ms_per_step": ms_e2e},
        "cpu_baseline": (None if args.no_cpu_baseline else
                         mlp_cpu_baseline(net, x.cpu().numpy(), t.cpu().numpy())),
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    net.close()
    ctx.close()
    return 0


def mlp_cpu_baseline(net, x, t, target_s=8.0):
    """The FP64 network reference (bfloat16 operands emulated) as it stands: loss,
    gradients and an Adam update per step on the same batch, on the host."""
    from oracle import mlp as omlp
    p = omlp.unflatten(net.dos_mlp_get_params().astype(np.float64), net.n_in, net.n_hidden,
                       net.n_out)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_s or steps < 1:
        _, g = omlp.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), bf16=True)
        p, m, v = omlp.adam_step(p, g, m, v, steps + 1, 1e-4)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": steps * x.shape[0] / dt, "unit": "samples/s",
            "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"{steps} Adam steps of batch {x.shape[0]} with the FP64 network "
                      f"reference (NumPy, bfloat16 operands emulated), {dt:.1f} s"}


def learned_cpu_baseline(ctx, net, test, groups, w, seed_in, target_s=12.0):
    """The serving path on the host cores with the oracle: the FP64 KPM oracle
    (n_v = 4, M = 64) and the FP64 network reference (bfloat16 operands emulated)
    on a sample of held-out instances, DOS per second."""
    from oracle import kpm as okpm
    from oracle import mlp as omlp
    from synthetic import CSR
    cores = os.cpu_count() or 1
    p = omlp.unflatten(net.dos_mlp_get_params().astype(np.float64), net.n_in, net.n_hidden,
                       net.n_out)
    done, t_used = 0, 0.0
    for g in groups:
        rp, ci, va = g.host
        for b in range(g.B):
            r0, r1 = int(g.seg[b]), int(g.seg[b + 1])
            e0, e1 = int(rp[r0]), int(rp[r1])
            A = CSR(r1 - r0, (rp[r0:r1 + 1] - e0).astype(np.int32), ci[e0:e1], va[e0:e1])
            t0 = time.perf_counter()
            mu = okpm.kpm_moments(A, float(g.lb[b]), float(g.ub[b]), w["M_in"], w["n_v_in"],
                                  seed_in, batch_index=g.b0 + b, nthreads=cores)
            omlp.forward(p, mu[1:][None, :].astype(np.float32).astype(np.float64), bf16=True)
            t_used += time.perf_counter() - t0
            done += 1
            if t_used >= target_s:
                break
        if t_used >= target_s:
            break
    return {"value": done / t_used, "unit": "DOS/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} held-out instances: FP64 KPM oracle (n_v={w['n_v_in']}, "
                      f"M={w['M_in']}, {cores} threads over the vectors) and the FP64 network "
                      f"reference, {t_used:.1f} s"}


def lanczos_spmm_bytes(n, nnz, ld):
    """Compulsory bytes of one Lanczos block-SpMM launch (FP64): CSR once, q_j read
    once, q_{j-1} read and w written."""
    return nnz * 12 + 4 * (n + 1) + 3 * n * ld * 8


def cpu_baseline_method(method, A, lb, ub, M, n_v_full, seed, target_s=10.0):
    """The oracle of the method, as it stands, on a bounded sample of start vectors."""
    from oracle import lanczos_dos as old
    from oracle import legendre as oleg
    cores = os.cpu_count() or 1
    if method in ("lanczos", "haydock"):
        t0 = time.perf_counter()
        old.lanczos_ritz(A, M, 1, seed)
        t1 = time.perf_counter() - t0
        nv = int(max(1, min(n_v_full, target_s / max(t1, 1e-3))))
        t0 = time.perf_counter()
        old.lanczos_ritz(A, M, nv, seed)
        t = time.perf_counter() - t0
        return {"value": A.nnz * nv * M / t, "unit": "products/s", "cores": 1, "kind": "oracle",
                "sample": f"{nv} start vectors, {M} Lanczos steps each (FP64, one thread, "
                          f"NumPy vector updates around the C sparse product), {t:.1f} s"}
    probe = max(1, min(cores, n_v_full))
    t0 = time.perf_counter()
    oleg.legendre_moments_per_vector(A, lb, ub, M, probe, seed, nthreads=cores)
    t = time.perf_counter() - t0
    nv = probe
    if t < target_s / 2:
        nv = int(min(4 * n_v_full, probe * target_s / max(t, 1e-3)))
        nv = max(probe, (nv // cores) * cores)
        t0 = time.perf_counter()
        oleg.legendre_moments_per_vector(A, lb, ub, M, nv, seed, nthreads=cores)
        t = time.perf_counter() - t0
    return {"value": A.nnz * nv * M / t, "unit": "moments/s", "cores": min(cores, nv),
            "kind": "oracle",
            "sample": f"{nv} start vectors, Legendre recurrence of Algorithm DGL (M={M} "
                      f"products per vector, FP64), {t:.1f} s on {min(cores, nv)} threads"}


def run_method(args, w, world, rank, local, device):
    """The paper's other estimators on the same workload and start vectors.

    lanczos / haydock: a step is Gershgorin bounds, an M-step Lanczos run of the
    n_v start vectors (block FP64 kernels), Ritz values and weights, and the
    Gaussian-blurred (lanczos, with the smoothed error against the reference) or
    Lorentzian-blurred (haydock, on the metric grid) DOS.  Metric: block
    matrix-vector products per second, nnz * n_v * M / t.
    kpml / dgl: a step is bounds, the Legendre moments (doubling Chebyshev sweep +
    exact basis change) and the KPML or DGL smoothed error; metric as KPM."""
    import torch
    import torch.distributed as dist

    from paper_1308_5467_gb300 import dos
    method = args.method
    cfg = METHODS[method]
    if w["kind"] not in ("anderson", "laplacian"):
        raise SystemExit(f"--method {method} runs on the single-matrix workloads "
                         "anderson64 and laplacian40")
    A = make_matrix(w)
    n_v, seed = w["n_v"], w["seed"]
    lanczos = method in ("lanczos", "haydock")
    M = cfg["M"][args.workload] if lanczos else w["M"]
    prec = "f64" if lanczos else args.precision
    vdt = np.float64 if prec == "f64" else np.float32
    Ad = dos.CSRArrays.from_synthetic(A, device=device, dtype=vdt)
    Ad64 = dos.CSRArrays.from_synthetic(A, device=device, dtype=np.float64)
    ctx = dos.Context(local)
    vec_offset = rank * n_v
    lb, ub = ctx.dos_bounds(Ad64, "gershgorin", pad_frac=0.01)
    sigma = 0.02 * (ub - lb)
    ref_mu = ctx.dos_kpm_moments(Ad64, lb, ub, 500, 1024, seed=seed + 1000, precision="f64")
    tuned_shape = ctx.dos_tune(Ad, n_v, prec)[0] if not lanczos else None
    x_grid = np.linspace(lb - 6 * sigma, ub + 6 * sigma, 4000)

    def step(Acsr):
        lo, hi = ctx.dos_bounds(Acsr, "gershgorin", pad_frac=0.01)
        if lanczos:
            theta, weight, _ = ctx.dos_lanczos_ritz(Acsr, M, n_v, seed)
            if method == "lanczos":
                return ctx.dos_points_error(theta, weight, lo, hi, sigma, ref_mu=ref_mu)
            phi = ctx.dos_haydock_dos(theta, weight, cfg["eta_frac"] * (hi - lo), x_grid)
            return float(phi.sum()), None
        nu = ctx.dos_legendre_moments(Acsr, lo, hi, M, n_v, seed, precision=prec,
                                      vec_offset=vec_offset)
        return ctx.dos_legendre_error(nu, method, lo, hi, sigma, tol=cfg["tol"], ref_mu=ref_mu)

    def timed(fn, steps, warmup, profile=False):
        for _ in range(warmup):
            fn()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            ctx.dos_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = None
        for _ in range(steps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        prof = ctx.dos_profile_read() if profile else None
        if profile:
            ctx.dos_profile_enable(False)
        ms = e0.elapsed_time(e1) / steps
        if world > 1:
            t = torch.tensor([ms], device=device, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, out, prof

    with ClockSampler(gpu_id_for(local)) as clk:
        ms, out, prof = timed(lambda: step(Ad64 if lanczos else Ad), args.steps, args.warmup,
                              profile=True)
    units = A.nnz * n_v * M
    value = units * world / (ms * 1e-3)
    peaks, peak_kind = measured_peaks()
    launch_ms = prof["step_ms"] / max(1, prof["step_launches"])
    if lanczos:
        ld = (n_v + 1) // 2 * 2
        flops = 2 * A.nnz * n_v
        byts = lanczos_spmm_bytes(A.n, A.nnz, ld)
        f_alu = flops / (launch_ms * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS
        f_hbm = byts / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
        if f_alu >= f_hbm:
            roofline = {"bound": "alu", "achieved": f_alu * FP64_NOMINAL_TFLOPS,
                        "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s", "frac": f_alu,
                        "traffic": None, "peak_source": FP64_PEAK_SOURCE,
                        "kernel": "lanczos_team_spmm_kernel", "flops_per_launch": flops,
                        "launch_ms": launch_ms, "hbm_frac": f_hbm}
        else:
            roofline = {"bound": "hbm", "achieved": f_hbm * peaks["hbm_gbs"],
                        "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": f_hbm,
                        "traffic": None, "peak_source": peak_kind,
                        "kernel": "lanczos_team_spmm_kernel", "algorithmic_bytes_per_launch": byts,
                        "launch_ms": launch_ms, "alu_frac": f_alu}
        metric, unit = "Lanczos block products/sec (nnz*n_v*M/s)", "products/s"
    else:
        alg = algorithmic_bytes_per_step(A.n, A.nnz, n_v, prec)
        achieved = alg / (launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                    "peak_source": peak_kind, "kernel": step_kernel_name(tuned_shape, prec),
                    "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms}
        metric, unit = "Legendre moments/sec (nnz*n_v*M/s)", "moments/s"

    e2e = None
    if not args.no_e2e:
        rp = torch.from_numpy(A.row_ptr).pin_memory()
        ci = torch.from_numpy(A.col_idx).pin_memory()
        va = torch.from_numpy(A.val.astype(np.float64 if lanczos else vdt)).pin_memory()
        Ah = dos.CSRArrays(A.n, rp, ci, va)
        ms_e2e, _, _ = timed(lambda: step(Ah), max(3, args.steps // 2), 1)
        h2d = 2 * (rp.numel() * 4 + ci.numel() * 4 + va.numel() * va.element_size())
        d2h = (2 * n_v * M * 8 + 16) if lanczos else (8 * (M + 1) + 16)
        e2e = {"value": units * world / (ms_e2e * 1e-3), "unit": unit,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Ac = A if lanczos or prec == "f64" else A.astype(np.float32)
        cpu = cpu_baseline_method(method, Ac, lb, ub, M, n_v, seed)
    if rank == 0:
        line = {
            "metric": metric, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "method": method, "desc": w["desc"],
                       "n": A.n, "nnz": A.nnz, "M": M, "n_v": n_v, "precision": prec,
                       "sigma": sigma, "lb": lb, "ub": ub, "launch": tuned_shape,
                       "l2": "inputs larger than L2 (vector blocks of the step)"},
            "e1": out[0], "einf": out[1], "roofline": roofline, "e2e": e2e,
            "cpu_baseline": cpu, "gpu_launches": prof["launches"], "clocks": clk.summary(),
        }
        print(json.dumps(line))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--instances", type=int, default=0,
                    help="learned workload: number of generated instances (0: its default)")
    ap.add_argument("--train-steps", type=int, default=0,
                    help="learned workload: Adam steps (0: its default)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="chunglu", choices=sorted(WORKLOADS))
    ap.add_argument("--method", default="kpm", choices=["kpm"] + sorted(METHODS),
                    help="kpm (the benchmark) or one of the paper's other estimators")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-f64-form", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-reference-dos", action="store_true",
                    help="skip the reference sweep of the smoothed error (profiling runs; e1 null)")
    ap.add_argument("--no-pdl", action="store_true",
                    help="plain stream order between sweep steps (no programmatic dependent launch)")
    ap.add_argument("--launch", default=None,
                    help="fixed launch shape team,chunks,staged(1|2|3|4)[,chunk_bytes(16|32)"
                         "[,depth(0|2|4|8)[,tiles[,panel]]]] "
                         "instead of the autotuner "
                         "(used when profiling one known kernel instance)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_1308_5467_gb300 import dos

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    w = WORKLOADS[args.workload]
    if args.method != "kpm":
        return run_method(args, w, world, rank, local, device)
    if w["kind"] == "batched":
        return run_batched(args, w, world, rank, local, device)
    if w["kind"] == "learned":
        return run_learned(args, w, world, rank, local, device)
    if w["kind"] == "mlp":
        return run_mlp(args, w, world, rank, local, device)
    A = make_matrix(w)
    if w["kind"] == "chunglu":
        A = A.astype(np.float32)      # the graph's values are FP32 (both forms read them)
    M, n_v, seed = w["M"], w["n_v"], w["seed"]
    prec = args.precision
    vdtype = np.float32 if prec == "f32" else np.float64
    Ad = dos.CSRArrays.from_synthetic(A, device=device, dtype=vdtype)
    Ad64 = dos.CSRArrays.from_synthetic(A, device=device, dtype=np.float64)
    ctx = dos.Context(local)
    vec_offset = rank * n_v
    bmethod = w.get("bounds", "gershgorin")

    def bounds_of(Acsr):
        if bmethod == "normalized_laplacian":   # known analytically: no kernel to run
            return NORMALIZED_LAPLACIAN_BOUNDS
        return ctx.dos_bounds(Acsr, bmethod, steps=20, seed=seed, pad_frac=0.01)

    lb, ub = bounds_of(Ad)
    sigma = 0.02 * (ub - lb)
    # launch shape of the fused step chosen by the library's autotuner (cached in ctx)
    fixed = None
    if args.launch:
        fixed = dict(zip(("team", "chunks", "staged", "chunk_bytes", "depth", "tiles", "panel"),
                         (int(v) for v in args.launch.split(","))))
        tuned_shape, tuned64 = fixed, None
    else:
        tuned_shape, tuned_ms = ctx.dos_tune(Ad, n_v, prec)
        tuned64 = (ctx.dos_tune(Ad64, n_v, "f64")[0]
                   if (prec == "f32" and not args.no_f64_form) else None)
    # reference DOS for the smoothed error: a sweep of ref_nv independent vectors
    # (another seed); FP32 on the graph, whose FP32 error (~1e-6 per moment) is far
    # below the stochastic error of 1024 vectors (~2e-5)
    ref_nv, ref_prec = w.get("ref_nv", 1024), w.get("ref_prec", "f64")
    ref_mu = None if args.no_reference_dos else ctx.dos_kpm_moments(
        Ad if ref_prec == prec else Ad64, lb, ub, M, ref_nv, seed=seed + 1000, precision=ref_prec)

    sweep_flags = dos.DOS_OPT_NO_PDL if args.no_pdl else 0

    def step(Acsr, precision, host=False):
        lo, hi = bounds_of(Acsr)
        mu = ctx.dos_kpm_moments(Acsr, lo, hi, M, n_v, seed=seed, precision=precision,
                                 vec_offset=vec_offset, flags=sweep_flags,
                                 launch=fixed if precision == prec else None)
        phi = ctx.dos_reconstruct(mu, M, "jackson", lo, hi, N_t=1000)
        if ref_mu is None:
            return mu, phi, None, None
        e1, einf = ctx.dos_smoothed_error(mu, M, "jackson", lo, hi, sigma, ref_mu=ref_mu)
        return mu, phi, e1, einf

    def timed(fn, steps, warmup, profile=False):
        for _ in range(warmup):
            fn()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            ctx.dos_profile_enable(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        out = None
        for _ in range(steps):
            out = fn()
        ev1.record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1) / steps
        prof = ctx.dos_profile_read() if profile else None
        if profile:
            ctx.dos_profile_enable(False)
        if world > 1:
            t = torch.tensor([ms], device=device, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, out, prof

    with ClockSampler(gpu_id_for(local)) as clk:
        ms, out, prof = timed(lambda: step(Ad, prec), args.steps, args.warmup, profile=True)
    mu, phi, e1, einf = out
    units = A.nnz * n_v * M
    value = units * world / (ms * 1e-3)

    # roofline of the dominant kernel (the fused step)
    peaks, peak_kind = measured_peaks()
    launch_ms = prof["step_ms"] / max(1, prof["step_launches"])
    kname = step_kernel_name(tuned_shape, prec)
    if prec == "f32":
        # one launch advances one vector panel by one step: its compulsory bytes are
        # the CSR once and the panel's three vector blocks
        n_panels, panel_nv, _ = panel_geometry(n_v, tuned_shape.get("panel", 0), prec)
        alg = algorithmic_bytes_per_step(A.n, A.nnz, panel_nv, prec)
        achieved = alg / (launch_ms * 1e-3) / 1e9
        tr = NCU_TRAFFIC.get((args.workload, prec))
        same_launch = tr is not None and all(tuned_shape.get(k, 0) == v
                                             for k, v in tr.get("launch", {}).items())
        traffic = tr["bytes"] if tr and tr["src"] == kernel_source_hash() and same_launch else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "peak_source": peak_kind, "kernel": kname,
                    "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms,
                    "frac_basis": "compulsory bytes of the launch's vector panel (CSR "
                                  "once, X_k once, X_{k-1} read, X_{k+1} written) / launch "
                                  "time",
                    "panels": {"count": n_panels, "vectors": panel_nv}}
        # the whole step (all n_v vectors, every panel) against the compulsory bytes
        # of one pass over A for all of them
        step_alg = algorithmic_bytes_per_step(A.n, A.nnz, n_v, prec)
        roofline["step"] = {"compulsory_bytes": step_alg, "ms": launch_ms * n_panels,
                            "frac": step_alg / (launch_ms * n_panels * 1e-3) / 1e9
                            / peaks["hbm_gbs"]}
        pb = pinning_bound(A.col_idx, A.n, A.nnz, panel_nv, prec,
                           torch.cuda.get_device_properties(device).L2_cache_size)
        pb["frac"] = pb["bytes_per_launch"] / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
        roofline["pinning_bound"] = pb
        if traffic:
            # the same launch against the DRAM bytes it actually moved (ncu)
            roofline["frac_of_traffic"] = traffic / (launch_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
            roofline["traffic_source"] = tr.get("note", "ncu dram__bytes_read.sum + "
                                                        "dram__bytes_write.sum per launch")
    else:
        flops = 2 * fma_per_step(A.n, A.nnz, n_v)
        achieved = flops / (launch_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None,
                    "peak_source": FP64_PEAK_SOURCE, "kernel": kname,
                    "flops_per_launch": flops, "launch_ms": launch_ms}

    forms = {prec: {"ms_per_step": ms, "value": value, "e1": e1, "einf": einf,
                    "steps": args.steps}}
    if not args.no_f64_form and prec == "f32":
        st64 = w.get("f64_steps", max(3, args.steps // 4))
        ms64, out64, prof64 = timed(lambda: step(Ad64, "f64"), st64, 1, profile=True)
        l64 = prof64["step_ms"] / max(1, prof64["step_launches"])
        fl = 2 * fma_per_step(A.n, A.nnz, n_v)
        diff = np.abs(out64[0] - mu)
        k = np.arange(M + 1)
        forms["f64"] = {"ms_per_step": ms64, "value": units * world / (ms64 * 1e-3),
                        "e1": out64[2], "einf": out64[3], "steps": st64,
                        "roofline": {"bound": "alu", "achieved": fl / (l64 * 1e-3) / 1e12,
                                     "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                                     "frac": fl / (l64 * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS,
                                     "peak_source": FP64_PEAK_SOURCE,
                                     "kernel": step_kernel_name(tuned64, "f64"),
                                     "launch_ms": l64},
                        # FP32 form against the FP64 form on the same values and vectors:
                        # the arithmetic error, next to the stochastic error of the estimate
                        "max_abs_diff_vs_f32": float(diff.max()),
                        # u sqrt(k+1) (1/2 + 40/sqrt(N)) at k = M, N = n n_v
                        "fp32_bound_at_M": float(2.0 ** -24 * np.sqrt(M + 1.0)
                                                 * (0.5 + 40.0 / np.sqrt(A.n * n_v))),
                        "max_diff_over_u_sqrt_k": float((diff / (2.0 ** -24
                                                                 * np.sqrt(k + 1))).max()),
                        "stochastic_std_sqrt_2_over_n_nv": float(np.sqrt(2.0 / (A.n * n_v)))}

    e2e = None
    if not args.no_e2e:
        # host (pinned) CSR arrays: the library copies them to the device inside each call
        rp = torch.from_numpy(A.row_ptr).pin_memory()
        ci = torch.from_numpy(A.col_idx).pin_memory()
        va = torch.from_numpy(A.val.astype(vdtype)).pin_memory()
        Ah = dos.CSRArrays(A.n, rp, ci, va)
        st_e2e = w.get("e2e_steps", max(3, args.steps // 2))
        ms_e2e, _, _ = timed(lambda: step(Ah, prec, host=True), st_e2e, 1)
        h2d = 2 * (rp.numel() * 4 + ci.numel() * 4 + va.numel() * va.element_size())
        d2h = 8 * (M + 1) + 8 * 1000 + 8 * 2 + 16
        e2e = {"value": units * world / (ms_e2e * 1e-3), "unit": "moments/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "steps": st_e2e}

    if world > 1:
        # the ranks swept disjoint blocks of start vectors (offset rank * n_v):
        # one weighted all-reduce of M+1 doubles gives the moments of all of them
        from paper_1308_5467_gb300.shard import combine_moments, torch_all_reduce
        mu = combine_moments(mu, n_v, n_v * world, torch_all_reduce(device=device))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A.astype(vdtype), lb, ub, M, n_v, seed)

    if rank == 0:
        line = {
            "metric": "Chebyshev moments/sec (nnz*n_v*M/s)",
            "value": value, "unit": "moments/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "f32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "launch": tuned_shape,
                       "launch_f64": tuned64, "n": A.n, "nnz": A.nnz,
                       "M": M, "n_v": n_v, "precision": prec,
                       "accumulation": ("FP32 products summed per row in FP32, rows "
                                        "accumulated as float pairs per thread, blocks and "
                                        "tiles in FP64") if prec == "f32" else "FP64",
                       "bounds": ("[0, 2] (any normalized Laplacian)"
                                  if bmethod == "normalized_laplacian" else bmethod)
                                 + ", padded 1% per side",
                       "reference_dos": f"{ref_prec.upper()} sweep of {ref_nv} other vectors",
                       "l2": "inputs larger than L2: %.0f MB touched per fused step"
                             % (algorithmic_bytes_per_step(A.n, A.nnz, n_v, prec) / 1e6),
                       "sigma": sigma, "lb": lb, "ub": ub, "pdl": not args.no_pdl},
            "dos_per_s": 1e3 / ms, "e1": e1, "einf": einf,
            "roofline": roofline, "forms": forms, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": prof["launches"], "clocks": clk.summary(),
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
