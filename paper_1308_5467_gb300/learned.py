"""The learned part: dataset generation, training and evaluation of the
moments-to-DOS network, all through libdos (include/dos.h, include/dos_mlp.h).

Input of the network: mu_1..mu_64 of a matrix from n_v = 4 start vectors
(mu_0 = 1 always).  Target: the Jackson-damped DOS phi_hat at the 256
Chebyshev nodes t_i = -cos(pi (i + 1/2)/256) from a reference sweep with
n_v = 1024, M = 256 -- both produced by the library's own batched sweeps, the
start vectors of instance number b keyed by b (the sweep's batch index).
Bounds: Gershgorin discs for the Anderson lattices; for normalized Laplacians,
whose discs reach ~20x past their spectrum, the interval [0, 2] that holds any
normalized Laplacian's spectrum, padded by 1% per side.
Scoring follows the paper's metric (Section 2.2, Eq. err2 with p = 1): the
network's grid DOS is turned back into moments (dos_moments_from_grid) and
compared, blurred by a Gaussian of width sigma = 0.02 (ub - lb), with the
reference DOS; plain Jackson KPM is scored the same way.
"""
from __future__ import annotations

import time

import numpy as np

from . import dos

N_IN, N_HIDDEN, N_OUT = 64, 512, 256
NORMALIZED_LAPLACIAN_BOUNDS = (-0.02, 2.02)


def _concat(mats):
    seg = np.zeros(len(mats) + 1, dtype=np.int64)
    seg[1:] = np.cumsum([m.n for m in mats])
    nnz = np.zeros(len(mats) + 1, dtype=np.int64)
    nnz[1:] = np.cumsum([m.col_idx.shape[0] for m in mats])
    rp = np.empty(seg[-1] + 1, dtype=np.int32)
    for b, m in enumerate(mats):
        rp[seg[b]:seg[b + 1]] = m.row_ptr[:-1] + nnz[b]
    rp[-1] = nnz[-1]
    ci = np.concatenate([m.col_idx for m in mats]).astype(np.int32)
    va = np.concatenate([m.val for m in mats]).astype(np.float32)
    return rp, ci, va, seg


def _is_laplacian(m) -> bool:
    return "chung" in str(m.meta.get("family", ""))


class Group:
    """Consecutive instances concatenated for one batched sweep: the CSR (device
    or host arrays), segment rows, bounds and the first instance's index."""

    def __init__(self, ctx, mats, b0: int, device: str | None = "cuda"):
        import torch
        rp, ci, va, seg = _concat(mats)
        self.b0, self.B, self.seg = b0, len(mats), seg
        self.n, self.nnz = int(seg[-1]), int(ci.shape[0])
        self.lap = np.array([_is_laplacian(m) for m in mats])
        self.host = (rp, ci, va)
        if device is None:
            self.A = dos.CSRArrays(self.n, rp, ci, va)
        else:
            self.A = dos.CSRArrays(self.n, torch.from_numpy(rp).to(device),
                                   torch.from_numpy(ci).to(device),
                                   torch.from_numpy(va).to(device))
        self.lb, self.ub = self.bounds(ctx)
        self._host_A = None

    def bounds(self, ctx, A=None):
        lb, ub = ctx.dos_bounds_batched(self.A if A is None else A, self.seg, pad_frac=0.01)
        lb[self.lap], ub[self.lap] = NORMALIZED_LAPLACIAN_BOUNDS
        return lb, ub

    @property
    def host_A(self):
        """Pinned host copies of the CSR, for end-to-end runs through host buffers."""
        if self._host_A is None:
            import torch
            rp, ci, va = self.host
            self._host_A = dos.CSRArrays(self.n, torch.from_numpy(rp).pin_memory(),
                                         torch.from_numpy(ci).pin_memory(),
                                         torch.from_numpy(va).pin_memory())
        return self._host_A

    @property
    def host_bytes(self) -> int:
        rp, ci, va = self.host
        return rp.nbytes + ci.nbytes + va.nbytes


def make_groups(ctx, mats, b0: int = 0, group_rows: int = 4_000_000, group_max: int = 4096,
                device: str | None = "cuda"):
    """Yield Groups of consecutive matrices from any iterable (at most group_rows
    rows, except a single larger matrix, and group_max matrices each)."""
    part, rows, b = [], 0, b0
    for m in mats:
        if part and (rows + m.n > group_rows or len(part) >= group_max):
            yield Group(ctx, part, b, device)
            b += len(part)
            part, rows = [], 0
        part.append(m)
        rows += m.n
    if part:
        yield Group(ctx, part, b, device)


def make_dataset(ctx: dos.Context, mats, seed: int, n_v_in: int = 4, M_in: int = N_IN,
                 n_v_ref: int = 1024, M_ref: int = 256, n_out: int = N_OUT, b0: int = 0,
                 group_rows: int = 4_000_000, keep_groups: bool = False, tune: bool = False):
    """Features, targets and the data needed to score them, for each matrix of the
    iterable `mats` (built lazily, e.g. by synthetic.instances.stream_instances).

    Returns dict with x (count, M_in) float32, y (count, n_out) float32, mu_in
    (count, M_in+1), mu_ref (count, M_ref+1), lb, ub (count,), laplacian (count,),
    n (count,), timing {"host_wait_s", "gpu_s", "moments"} and, with keep_groups,
    the device Groups (for timing and further sweeps).  With tune, the launch
    shapes of both sweeps are autotuned on the first group and kept for the rest
    (groups differ only in the instances they hold)."""
    import torch
    xs, ys, mus, refs, lbs, ubs, laps, ns, groups = [], [], [], [], [], [], [], [], []
    shapes = None
    gpu_s, host_s, units = 0.0, 0.0, 0.0
    it = iter(make_groups(ctx, mats, b0, group_rows))
    while True:
        t0 = time.perf_counter()
        g = next(it, None)
        host_s += time.perf_counter() - t0
        if g is None:
            break
        if tune and shapes is None:
            shapes = (ctx.dos_tune(g.A, n_v_in, "f32", seg_rows=g.seg)[0],
                      ctx.dos_tune(g.A, n_v_ref, "f32", seg_rows=g.seg)[0])
            for sh in shapes:
                sh.pop("tiles")          # sized per group from its occupancy
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        mu = ctx.dos_kpm_moments_batched(g.A, g.seg, g.lb, g.ub, M_in, n_v_in, seed=seed,
                                         precision="f32", batch_index=g.b0,
                                         launch=shapes[0] if shapes else None)
        ref = ctx.dos_kpm_moments_batched(g.A, g.seg, g.lb, g.ub, M_ref, n_v_ref,
                                          seed=seed + 7919, precision="f32", batch_index=g.b0,
                                          launch=shapes[1] if shapes else None)
        y = ctx.dos_reconstruct_batched(ref, "jackson", N_t=n_out)
        torch.cuda.synchronize()
        gpu_s += time.perf_counter() - t1
        units += g.nnz * (n_v_in * M_in + n_v_ref * M_ref)
        xs.append(mu[:, 1:M_in + 1].astype(np.float32))
        ys.append(y.astype(np.float32))
        mus.append(mu)
        refs.append(ref)
        lbs.append(g.lb)
        ubs.append(g.ub)
        laps.append(g.lap)
        ns.append(np.diff(g.seg))
        if keep_groups:
            groups.append(g)
    out = {"x": np.concatenate(xs), "y": np.concatenate(ys), "mu_in": np.concatenate(mus),
           "mu_ref": np.concatenate(refs), "lb": np.concatenate(lbs), "ub": np.concatenate(ubs),
           "laplacian": np.concatenate(laps), "n": np.concatenate(ns),
           "timing": {"host_wait_s": host_s, "gpu_s": gpu_s, "moments": units},
           "shapes": shapes}
    if keep_groups:
        out["groups"] = groups
    return out


def train(ctx: dos.Context, x: np.ndarray, y: np.ndarray, steps: int = 3000, batch: int = 256,
          lr: float = 1e-3, seed: int = 0, device: str = "cuda") -> dos.MLP:
    """Adam on minibatches drawn with a seeded permutation; cosine learning-rate decay."""
    import torch
    net = dos.MLP(ctx, x.shape[1], N_HIDDEN, y.shape[1], seed=seed)
    X = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(device)
    Y = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).to(device)
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    order = rng.permutation(n)
    pos = 0
    for it in range(steps):
        if pos + batch > n:
            order = rng.permutation(n)
            pos = 0
        idx = torch.from_numpy(order[pos:pos + batch]).to(device)
        pos += batch
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        step_lr = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        net.dos_mlp_train_step(xb, yb, max(step_lr, 1e-6), want_loss=False)
    torch.cuda.synchronize()
    return net


def _e1(ctx, mu, damping, lb, ub, ref, sigma_frac):
    sigma = sigma_frac * (ub - lb)
    return ctx.dos_smoothed_error(mu, mu.shape[0] - 1, damping, lb, ub, sigma, ref_mu=ref,
                                  ref_damping="jackson")[0]


def score(ctx: dos.Context, data: dict, net: dos.MLP | None = None, sigma_frac: float = 0.02,
          n_out: int = N_OUT):
    """Smoothed L1 errors (paper metric) against the reference DOS: for the network
    (if given) and for plain Jackson KPM from the input moments."""
    e_kpm, e_net = [], []
    pred = net.dos_mlp_infer(data["x"]) if net is not None else None
    for b in range(data["x"].shape[0]):
        lb, ub = float(data["lb"][b]), float(data["ub"][b])
        ref = data["mu_ref"][b]
        e_kpm.append(_e1(ctx, data["mu_in"][b], "jackson", lb, ub, ref, sigma_frac))
        if pred is not None:
            mu_net = np.empty(n_out)
            ctx.dos_moments_from_grid(pred[b].astype(np.float64), n_out - 1, mu_net)
            e_net.append(_e1(ctx, mu_net, "none", lb, ub, ref, sigma_frac))
    return np.array(e_kpm), (np.array(e_net) if pred is not None else None)


def kpm_errors(ctx: dos.Context, data: dict, n_v: int, M: int, seed: int,
               sigma_frac: float = 0.02):
    """Smoothed L1 errors of plain Jackson KPM with n_v vectors and degree M on the
    kept groups of `data` (vectors from `seed`), against the same reference."""
    errs = []
    for g in data["groups"]:
        mu = ctx.dos_kpm_moments_batched(g.A, g.seg, g.lb, g.ub, M, n_v, seed=seed,
                                         precision="f32", batch_index=g.b0)
        for b in range(g.B):
            i = g.b0 - data["groups"][0].b0 + b
            errs.append(_e1(ctx, mu[b], "jackson", float(g.lb[b]), float(g.ub[b]),
                            data["mu_ref"][i], sigma_frac))
    return np.array(errs)


class LearnedPipeline:
    """The serving path of the learned part on a list of Groups: bounds, a batched
    sweep of n_v = 4 vectors to degree 64, and the network reading mu_1..mu_64
    in place; the DOS of every instance lands in one device array."""

    def __init__(self, ctx, net, groups, seed: int, n_v: int = 4, M: int = N_IN):
        import torch
        self.ctx, self.net, self.groups, self.seed, self.n_v, self.M = ctx, net, groups, seed, \
            n_v, M
        self.count = sum(g.B for g in groups)
        self.mu = [torch.empty((g.B, M + 1), dtype=torch.float64, device="cuda")
                   for g in groups]
        self.out = torch.empty((self.count, net.n_out), dtype=torch.float32, device="cuda")

    def run(self, host: bool = False):
        r0 = 0
        for g, mu in zip(self.groups, self.mu):
            A = g.host_A if host else g.A
            lb, ub = g.bounds(self.ctx, A)
            self.ctx.dos_kpm_moments_batched(A, g.seg, lb, ub, self.M, self.n_v, seed=self.seed,
                                             precision="f32", batch_index=g.b0, mu=mu)
            self.net.dos_mlp_infer(mu, col0=1, out=self.out[r0:r0 + g.B])
            r0 += g.B
        return self.out


class KPMPipeline:
    """Plain Jackson KPM on the same groups: bounds, a batched sweep of n_v
    vectors to degree M, and the batched reconstruction on the same grid."""

    def __init__(self, ctx, groups, seed: int, n_v: int, M: int, n_out: int = N_OUT):
        import torch
        self.ctx, self.groups, self.seed, self.n_v, self.M = ctx, groups, seed, n_v, M
        self.count = sum(g.B for g in groups)
        self.mu = [torch.empty((g.B, M + 1), dtype=torch.float64, device="cuda")
                   for g in groups]
        self.out = torch.empty((self.count, n_out), dtype=torch.float64, device="cuda")
        self.n_out = n_out

    def run(self):
        r0 = 0
        for g, mu in zip(self.groups, self.mu):
            lb, ub = g.bounds(self.ctx)
            self.ctx.dos_kpm_moments_batched(g.A, g.seg, lb, ub, self.M, self.n_v,
                                             seed=self.seed, precision="f32",
                                             batch_index=g.b0, mu=mu)
            self.ctx.dos_reconstruct_batched(mu, "jackson", N_t=self.n_out,
                                             phi_hat=self.out[r0:r0 + g.B])
            r0 += g.B
        return self.out
