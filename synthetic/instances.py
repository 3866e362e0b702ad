"""Seeded populations of matrices for the learned moments-to-DOS network.

A population mixes the two families of the KPM workloads: 3-D Anderson
lattices (side L with L^3 in [n_lo, n_hi], disorder W ~ U[1, 16]) and
normalized Laplacians of Chung-Lu graphs (n ~ U{n_lo..n_hi}, beta = 2.5, mean
degree 20), one Chung-Lu graph for every two lattices on average.  Each
instance is described by a small tuple (its "spec") so that specs can be drawn
in the main process and the matrices built in worker processes.

Building 20,000 matrices of up to 64,000 rows holds tens of GB if kept at
once, so ``stream_instances`` builds them in a spawned process pool one
window ahead of the consumer and yields them in spec order.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from .matrices import anderson_3d, chung_lu_normalized_laplacian


def learned_instance_specs(count: int, seed: int, n_lo: int = 4096, n_hi: int = 64000,
                           chung_lu_share: float = 1.0 / 3.0) -> list[tuple]:
    """("anderson", L, W, seed) or ("chunglu", n, seed) tuples, drawn from `seed`."""
    rng = np.random.default_rng(seed)
    L_lo = int(np.ceil(round(n_lo ** (1.0 / 3.0), 9)))
    L_hi = int(np.floor(round(n_hi ** (1.0 / 3.0), 9)))
    specs = []
    for _ in range(count):
        s = int(rng.integers(1 << 30))
        if rng.random() < chung_lu_share:
            specs.append(("chunglu", int(rng.integers(n_lo, n_hi + 1)), s))
        else:
            specs.append(("anderson", int(rng.integers(L_lo, L_hi + 1)),
                          float(rng.uniform(1.0, 16.0)), s))
    return specs


def make_instance(spec: tuple):
    """The matrix of one spec, with FP32 values."""
    if spec[0] == "anderson":
        _, L, W, s = spec
        A = anderson_3d(L, W, s)
    elif spec[0] == "chunglu":
        _, n, s = spec
        A = chung_lu_normalized_laplacian(n, beta=2.5, mean_deg=20.0, seed=s)
    else:
        raise ValueError(spec)
    A = A.astype(np.float32)
    A.meta = {"family": spec[0]}   # drop per-site arrays before crossing processes
    return A


def stream_instances(specs: list[tuple], workers: int = 0, window: int = 512):
    """Yield make_instance(spec) for every spec in order, built by `workers`
    spawned processes (0: all cores) at most two windows ahead."""
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or len(specs) <= 8:
        for sp in specs:
            yield make_instance(sp)
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        chunks = [specs[i:i + window] for i in range(0, len(specs), window)]
        pending = pool.map_async(make_instance, chunks[0], chunksize=4)
        for c in range(len(chunks)):
            mats = pending.get()
            if c + 1 < len(chunks):
                pending = pool.map_async(make_instance, chunks[c + 1], chunksize=4)
            yield from mats
