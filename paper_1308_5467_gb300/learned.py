"""The learned part: dataset generation, training and evaluation of the
moments-to-DOS network, all through libdos (include/dos.h, include/dos_mlp.h).

Input of the network: mu_1..mu_64 of a matrix from n_v = 4 start vectors
(mu_0 = 1 always).  Target: the Jackson-damped DOS phi_hat at the 256
Chebyshev nodes t_i = -cos(pi (i + 1/2)/256) from a reference sweep with
n_v = 1024, M = 256 -- both produced by the library's own batched sweeps.
Scoring follows the paper's metric (Section 2.2, Eq. err2 with p = 1): the
network's grid DOS is turned back into moments (dos_moments_from_grid) and
compared, blurred by a Gaussian of width sigma = 0.02 (ub - lb), with the
reference DOS; plain Jackson KPM from the same 4 vectors is scored the same way.
"""
from __future__ import annotations

import numpy as np

from . import dos

N_IN, N_HIDDEN, N_OUT = 64, 512, 256


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


def make_dataset(ctx: dos.Context, mats, seed: int, n_v_in: int = 4, M_in: int = N_IN,
                 n_v_ref: int = 1024, M_ref: int = 256, n_out: int = N_OUT, group: int = 32,
                 device: str = "cuda"):
    """Features, targets and the data needed to score them, for each matrix.

    Returns dict with x (count, M_in) float32, y (count, n_out) float32,
    mu_in (count, M_in+1), mu_ref (count, M_ref+1), lb, ub (count,)."""
    import torch
    xs, ys, mus, refs, lbs, ubs = [], [], [], [], [], []
    for g0 in range(0, len(mats), group):
        part = mats[g0:g0 + group]
        rp, ci, va, seg = _concat(part)
        A = dos.CSRArrays(int(seg[-1]), torch.from_numpy(rp).to(device),
                          torch.from_numpy(ci).to(device), torch.from_numpy(va).to(device))
        lb, ub = ctx.dos_bounds_batched(A, seg, pad_frac=0.01)
        mu = ctx.dos_kpm_moments_batched(A, seg, lb, ub, M_in, n_v_in, seed=seed,
                                         precision="f32", batch_index=g0)
        ref = ctx.dos_kpm_moments_batched(A, seg, lb, ub, M_ref, n_v_ref, seed=seed + 7919,
                                          precision="f32", batch_index=g0)
        for b in range(len(part)):
            y = ctx.dos_reconstruct(ref[b], M_ref, "jackson", N_t=n_out)
            xs.append(mu[b, 1:].astype(np.float32))
            ys.append(y.astype(np.float32))
        mus.append(mu)
        refs.append(ref)
        lbs.append(lb)
        ubs.append(ub)
    return {"x": np.stack(xs), "y": np.stack(ys), "mu_in": np.concatenate(mus),
            "mu_ref": np.concatenate(refs), "lb": np.concatenate(lbs),
            "ub": np.concatenate(ubs)}


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


def score(ctx: dos.Context, data: dict, net: dos.MLP | None = None, sigma_frac: float = 0.02,
          n_out: int = N_OUT):
    """Smoothed L1 errors (paper metric) against the reference DOS: for the network
    (if given) and for plain Jackson KPM from the input moments."""
    e_kpm, e_net = [], []
    pred = net.dos_mlp_forward(data["x"]) if net is not None else None
    for b in range(data["x"].shape[0]):
        lb, ub = float(data["lb"][b]), float(data["ub"][b])
        sigma = sigma_frac * (ub - lb)
        ref = data["mu_ref"][b]
        M_ref = ref.shape[0] - 1
        mu = data["mu_in"][b]
        e_kpm.append(ctx.dos_smoothed_error(mu, mu.shape[0] - 1, "jackson", lb, ub, sigma,
                                            ref_mu=ref, ref_damping="jackson")[0])
        if pred is not None:
            mu_net = np.empty(n_out)
            ctx.dos_moments_from_grid(pred[b].astype(np.float64), n_out - 1, mu_net)
            e_net.append(ctx.dos_smoothed_error(mu_net, n_out - 1, "none", lb, ub, sigma,
                                                ref_mu=ref, ref_damping="jackson")[0])
        del M_ref
    return np.array(e_kpm), (np.array(e_net) if pred is not None else None)
