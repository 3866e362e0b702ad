"""Seeded generators of the sparse symmetric matrices used as KPM workloads.

The paper's test matrices (its modified 2-D Laplacian of Section 4 and the
UF-collection matrices *shwater* and *pe3k*) are either under-specified or not
available offline, so these synthetic families stand in for them:

* ``laplacian_2d``  -- 5-point Dirichlet Laplacian on an m x m grid (diag 4,
  off-diagonal -1, row-major index ``i = a*m + b``); closed-form spectrum
  ``4 - 2cos(i pi/(m+1)) - 2cos(j pi/(m+1))``.
* ``anderson_3d``   -- Anderson tight-binding Hamiltonian on an L^3 periodic
  lattice: on-site energies uniform in [-W/2, W/2], hopping -1 to the six
  periodic neighbours; the diagonal is always stored (7 nonzeros per row).
* ``chung_lu_normalized_laplacian`` -- normalized Laplacian
  ``I - D^{-1/2} A D^{-1/2}`` of a seeded Chung-Lu random graph with a
  power-law expected-degree sequence (skewed row lengths).
* ``random_symmetric`` / ``diagonal`` -- tiny cases for brute-force checks.
* ``batched_anderson`` -- many Anderson lattices of uneven size.

All generators return a :class:`CSR` with int32 ``row_ptr``/``col_idx`` and
float64 ``val`` whose column indices are sorted within each row.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32, n+1
    col_idx: np.ndarray  # int32, nnz
    val: np.ndarray      # float64 (or float32), nnz
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.row_ptr, self.col_idx,
                   np.ascontiguousarray(self.val.astype(dtype)), dict(self.meta))

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(a, (rows, self.col_idx), self.val.astype(np.float64))
        return a


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray,
              meta: dict | None = None) -> CSR:
    """Sort COO triplets by (row, col) and pack them as CSR (no duplicates expected)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(n) + cols
    order = np.argsort(key, kind="stable")
    rows, cols, vals = rows[order], cols[order], np.asarray(vals)[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32),
               np.ascontiguousarray(vals, dtype=np.float64), meta or {})


def laplacian_2d(m: int) -> CSR:
    """5-point Dirichlet Laplacian on an m x m interior grid, n = m*m."""
    n = m * m
    a, b = np.divmod(np.arange(n, dtype=np.int64), m)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.full(n, 4.0)]
    for da, db in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        aa, bb = a + da, b + db
        ok = (aa >= 0) & (aa < m) & (bb >= 0) & (bb < m)
        rows.append(np.arange(n)[ok])
        cols.append((aa * m + bb)[ok])
        vals.append(np.full(int(ok.sum()), -1.0))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols),
                     np.concatenate(vals), {"family": "laplacian_2d", "m": m})


def anderson_3d(L: int, W: float, seed: int, hopping: float = -1.0) -> CSR:
    """Anderson model on an L^3 periodic lattice; site index i = (x*L + y)*L + z."""
    if L < 3:
        raise ValueError("L must be >= 3 so that the six periodic neighbours are distinct")
    n = L ** 3
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-W / 2.0, W / 2.0, size=n)
    idx = np.arange(n, dtype=np.int64)
    x, rem = np.divmod(idx, L * L)
    y, z = np.divmod(rem, L)
    rows = [idx]
    cols = [idx]
    vals = [eps]
    for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        j = (((x + dx) % L) * L + (y + dy) % L) * L + (z + dz) % L
        rows.append(idx)
        cols.append(j)
        vals.append(np.full(n, hopping))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                     {"family": "anderson_3d", "L": L, "W": W, "seed": seed, "eps": eps})


def _chung_lu_offset(n: int, gamma: float, mean_deg: float) -> float:
    """Index offset i0 such that the largest expected degree is sqrt(n * mean_deg).

    That is the usual admissibility condition w_max^2 <= sum(w) of the
    Chung-Lu model (every pair probability w_i w_j / sum(w) stays <= 1).
    """
    target = np.sqrt(n * mean_deg)
    i = np.arange(n, dtype=np.float64)

    def wmax(i0):
        w = (i + i0) ** (-gamma)
        return w[0] * mean_deg * n / w.sum()

    lo, hi = 1e-3, float(n)
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if wmax(mid) > target:
            new = (mid, hi)
        else:
            new = (lo, mid)
        if new == (lo, hi):   # a fixed point: further halvings change nothing
            break
        lo, hi = new
    return hi


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """np.unique(x) for a 1-D integer array, by one sort and a neighbour test."""
    s = np.sort(x)
    if s.size == 0:
        return s
    keep = np.empty(s.size, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _searchsorted_right(cdf: np.ndarray, q: np.ndarray) -> np.ndarray:
    """np.searchsorted(cdf, q, side="right") over chunks of q in threads (numpy
    releases the GIL inside the binary searches); the result is identical."""
    out = np.empty(q.shape[0], dtype=np.int64)
    bounds = np.linspace(0, q.shape[0], 33).astype(np.int64)

    def one(i):
        a, b = bounds[i], bounds[i + 1]
        out[a:b] = np.searchsorted(cdf, q[a:b], side="right")

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(32)))
    return out


def chung_lu_normalized_laplacian(n: int, beta: float = 2.5, mean_deg: float = 20.0,
                                  seed: int = 3) -> CSR:
    """Normalized Laplacian of a seeded Chung-Lu graph.

    Expected degrees w_i proportional to (i + i0)^(-1/(beta-1)), scaled to mean
    ``mean_deg``; ``round(n*mean_deg/2)`` edges are drawn with both endpoints
    sampled proportionally to w; self-loops and duplicate edges are dropped.
    ``L = I - D^{-1/2} A D^{-1/2}`` with ``L_ii = 0`` for isolated vertices; the
    diagonal is always stored.  The spectrum lies in [0, 2].
    """
    rng = np.random.default_rng(seed)
    gamma = 1.0 / (beta - 1.0)
    i0 = _chung_lu_offset(n, gamma, mean_deg)
    w = (np.arange(n, dtype=np.float64) + i0) ** (-gamma)
    w *= mean_deg * n / w.sum()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * mean_deg / 2.0))
    u = _searchsorted_right(cdf, rng.random(m))
    v = _searchsorted_right(cdf, rng.random(m))
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = _sorted_unique(lo * np.int64(n) + hi)
    lo, hi = np.divmod(key, np.int64(n))
    deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    inv_sqrt = np.zeros(n)
    nz = deg > 0
    inv_sqrt[nz] = 1.0 / np.sqrt(deg[nz].astype(np.float64))
    off = -inv_sqrt[lo] * inv_sqrt[hi]
    diag = nz.astype(np.float64)
    rows = np.concatenate([np.arange(n, dtype=np.int64), lo, hi])
    cols = np.concatenate([np.arange(n, dtype=np.int64), hi, lo])
    vals = np.concatenate([diag, off, off])
    return _from_coo(n, rows, cols, vals,
                     {"family": "chung_lu_normalized_laplacian", "beta": beta,
                      "mean_deg": mean_deg, "seed": seed, "i0": i0,
                      "max_row_len": int(deg.max()) + 1})


def random_symmetric(n: int, density: float, seed: int, empty_rows: int = 0,
                     long_row: int | None = None) -> CSR:
    """Random sparse symmetric matrix with N(0,1) entries.

    ``empty_rows`` rows (and the matching columns) are left without any entry;
    ``long_row`` (a row index) is made dense, giving one long row.
    """
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    if long_row is not None:
        mask[long_row, :] = True
        mask[:, long_row] = True
    upper = np.triu(np.where(mask, rng.standard_normal((n, n)), 0.0))
    a = upper + np.triu(upper, 1).T
    if empty_rows:
        dead = rng.choice(n, size=empty_rows, replace=False)
        a[dead, :] = 0.0
        a[:, dead] = 0.0
    rows, cols = np.nonzero(a)
    return _from_coo(n, rows, cols, a[rows, cols],
                     {"family": "random_symmetric", "density": density, "seed": seed})


def diagonal(d: np.ndarray) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return _from_coo(n, np.arange(n), np.arange(n), d, {"family": "diagonal"})


def batched_anderson(count: int, seed: int, L_range=(10, 40), W_range=(1.0, 16.0)):
    """``count`` Anderson lattices with side L ~ U{L_lo..L_hi} and W ~ U[W_lo, W_hi]."""
    rng = np.random.default_rng(seed)
    Ls = rng.integers(L_range[0], L_range[1] + 1, size=count)
    Ws = rng.uniform(W_range[0], W_range[1], size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [anderson_3d(int(L), float(W), int(s)) for L, W, s in zip(Ls, Ws, seeds)]


def concat_block_diagonal(mats: list[CSR]):
    """Concatenate CSRs row-wise for a batched sweep.

    Returns ``(row_ptr, col_idx, val, seg_rows)``: a global monotone ``row_ptr``
    over all rows, column indices kept LOCAL to each matrix, values, and the
    int64 segment row offsets (length B+1).
    """
    seg_rows = np.zeros(len(mats) + 1, dtype=np.int64)
    seg_rows[1:] = np.cumsum([m.n for m in mats])
    nnz_off = np.zeros(len(mats) + 1, dtype=np.int64)
    nnz_off[1:] = np.cumsum([m.nnz for m in mats])
    if nnz_off[-1] >= 2**31:
        raise ValueError("total nnz exceeds int32 range")
    row_ptr = np.empty(seg_rows[-1] + 1, dtype=np.int32)
    for b, m in enumerate(mats):
        row_ptr[seg_rows[b]:seg_rows[b + 1]] = m.row_ptr[:-1] + nnz_off[b]
    row_ptr[-1] = nnz_off[-1]
    col_idx = np.concatenate([m.col_idx for m in mats]).astype(np.int32)
    val = np.concatenate([m.val for m in mats])
    return row_ptr, col_idx, val, seg_rows
