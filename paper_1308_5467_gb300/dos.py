"""Thin ctypes binding of libdos (include/dos.h): argument marshalling only.

Every function forwards to the C entry point of the same name; all arithmetic
runs in the library's CUDA kernels.  Arrays may be torch CUDA tensors (used in
place, on the tensor's device and the current torch stream) or numpy arrays /
CPU tensors (host memory: the library copies them).  If libdos.so is missing
this module raises ImportError -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdos.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libdos.so not found at {LIB_PATH}: build it with "
        "`python -m paper_1308_5467_gb300.build` (needs nvcc)")

_lib = C.CDLL(LIB_PATH)

DOS_OK, DOS_EINVAL, DOS_ENOMEM, DOS_ECUDA, DOS_ESPECTRUM, DOS_ETIMEOUT, DOS_EIO = range(7)
DOS_F64, DOS_F32 = 0, 1
DOS_DEVICE, DOS_HOST = 0, 1
DOS_PREC_F64, DOS_PREC_F32_ACC64 = 0, 1
DOS_BOUNDS_GERSHGORIN, DOS_BOUNDS_LANCZOS = 0, 1
DOS_DAMP_NONE, DOS_DAMP_JACKSON = 0, 1
DOS_OPT_NO_VALIDATE, DOS_OPT_NO_SPECTRUM_CHECK, DOS_OPT_NO_GRAPH, DOS_OPT_AUTOTUNE = 1, 2, 4, 8
DOS_OPT_TEST_STALL_WAIT = 16
DOS_OPT_NO_PDL = 32
DOS_LEG_KPML, DOS_LEG_DGL = 0, 1

PRECISIONS = {"f64": DOS_PREC_F64, "f32": DOS_PREC_F32_ACC64}
DAMPINGS = {"none": DOS_DAMP_NONE, "jackson": DOS_DAMP_JACKSON}
BOUNDS = {"gershgorin": DOS_BOUNDS_GERSHGORIN, "lanczos": DOS_BOUNDS_LANCZOS}
LEGENDRE_METHODS = {"kpml": DOS_LEG_KPML, "dgl": DOS_LEG_DGL}


class dos_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("dtype", C.c_int32),
                ("location", C.c_int32)]


class dos_launch(C.Structure):
    _fields_ = [("team", C.c_int32), ("chunks", C.c_int32), ("block", C.c_int32),
                ("tiles", C.c_int32), ("staged", C.c_int32), ("chunk_bytes", C.c_int32),
                ("depth", C.c_int32), ("panel", C.c_int32)]


class dos_kpm_opts(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("vec_offset", C.c_int64), ("batch_index", C.c_uint64),
                ("launch", dos_launch), ("wait_limit_cycles", C.c_int64)]


_vp, _i, _i64, _u64, _d = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
_dp = C.POINTER(C.c_double)
_SIGS = {
    "dos_ctx_create": (_i, [C.POINTER(_vp), _i]),
    "dos_ctx_destroy": (_i, [_vp]),
    "dos_last_error": (C.c_char_p, [_vp]),
    "dos_status_string": (C.c_char_p, [_i]),
    "dos_validate_csr": (_i, [_vp, C.POINTER(dos_csr), _vp]),
    "dos_start_vectors": (_i, [_vp, _i64, _i, _u64, _u64, _i64, _i, _vp, _vp]),
    "dos_profile_enable": (_i, [_vp, _i]),
    "dos_profile_read": (_i, [_vp, _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int64)]),
    "dos_bounds": (_i, [_vp, C.POINTER(dos_csr), _i, _i, _u64, _d, _dp, _dp, _vp]),
    "dos_bounds_batched": (_i, [_vp, C.POINTER(dos_csr), _i, _vp, _d, _vp, _vp, _vp]),
    "dos_kpm_moments": (_i, [_vp, C.POINTER(dos_csr), _d, _d, _i, _i, _u64, _i, _vp, _vp, _vp]),
    "dos_kpm_moments_ex": (_i, [_vp, C.POINTER(dos_csr), _d, _d, _i, _i, _u64, _i, _vp, _vp,
                                C.POINTER(dos_kpm_opts), _vp]),
    "dos_kpm_moments_batched": (_i, [_vp, C.POINTER(dos_csr), _i, _vp, _vp, _vp, _i, _i, _u64,
                                     _i, _vp, _vp, C.POINTER(dos_kpm_opts), _vp]),
    "dos_tune": (_i, [_vp, C.POINTER(dos_csr), _i, _vp, _i, _i, C.POINTER(dos_launch), _dp, _vp]),
    "dos_reconstruct": (_i, [_vp, _vp, _i, _i, _d, _d, _vp, _i, _vp, _vp, _vp]),
    "dos_reconstruct_batched": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _vp, _vp]),
    "dos_smoothed_error": (_i, [_vp, _vp, _i, _i, _d, _d, _vp, _i64, _vp, _i, _i, _d, _i, _dp,
                                _dp, _vp]),
    "dos_moments_from_grid": (_i, [_vp, _vp, _i, _i, _vp, _vp]),
    "dos_heat_capacity": (_i, [_vp, _vp, _i, _i, _d, _d, _vp, _vp, _i64, _vp, _i, _vp, _vp]),
    "dos_lanczos_ritz": (_i, [_vp, C.POINTER(dos_csr), _i, _i, _u64, _vp, _vp, _vp, _vp]),
    "dos_lanczos_dos": (_i, [_vp, _vp, _vp, _i, _i, _d, _vp, _i, _vp, _vp]),
    "dos_haydock_dos": (_i, [_vp, _vp, _vp, _i, _i, _d, _vp, _i, _vp, _vp]),
    "dos_points_error": (_i, [_vp, _vp, _vp, _i64, _d, _d, _vp, _i64, _vp, _i, _i, _d, _i, _dp,
                              _dp, _vp]),
    "dos_legendre_moments": (_i, [_vp, C.POINTER(dos_csr), _d, _d, _i, _i, _u64, _i, _vp, _vp,
                                  C.POINTER(dos_kpm_opts), _vp]),
    "dos_cheb_to_legendre": (_i, [_vp, _vp, _i64, _i, _vp, _vp]),
    "dos_kpml_reconstruct": (_i, [_vp, _vp, _i, _d, _d, _vp, _i, _vp, _vp, _vp]),
    "dos_dgl": (_i, [_vp, _vp, _i, _d, _d, _d, _d, _vp, _i, _vp, _vp, _vp]),
    "dos_legendre_error": (_i, [_vp, _vp, _i, _i, _d, _d, _d, _d, _vp, _i64, _vp, _i, _i, _i,
                                _dp, _dp, _vp]),
}
_SIGS.update({
    "dos_mlp_create": (_i, [_vp, _i, _i, _i, _u64, C.POINTER(_vp)]),
    "dos_mlp_destroy": (_i, [_vp]),
    "dos_mlp_num_params": (_i, [_vp, C.POINTER(C.c_int64)]),
    "dos_mlp_set_params": (_i, [_vp, _vp, _vp]),
    "dos_mlp_get_params": (_i, [_vp, _vp, _vp]),
    "dos_mlp_forward": (_i, [_vp, _vp, _i, _vp, _vp]),
    "dos_mlp_infer": (_i, [_vp, _vp, _i, _i64, _i64, _vp, _i, _vp]),
    "dos_mlp_save": (_i, [_vp, C.c_char_p, _vp]),
    "dos_mlp_load": (_i, [_vp, C.c_char_p, C.POINTER(_vp), _vp]),
    "dos_mlp_loss_grad": (_i, [_vp, _vp, _vp, _i, C.POINTER(C.c_float), _vp, _vp]),
    "dos_mlp_train_step": (_i, [_vp, _vp, _vp, _i, C.c_float, C.POINTER(C.c_float), _vp]),
})
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class DosError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.dos_status_string(status).decode()}: {message}")
        self.status = status


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, is_device, keepalive) of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None, False, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x.is_cuda, x
    a = np.ascontiguousarray(x)
    return a.ctypes.data, False, a


def _stream_of(*xs):
    for x in xs:
        if x is not None and _is_torch(x) and x.is_cuda:
            import torch
            return C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return C.c_void_p(0)


class CSRArrays:
    """A CSR matrix for the library: three arrays (torch CUDA tensors = device,
    numpy arrays = host) plus n.  ``val`` dtype float64 or float32."""

    def __init__(self, n: int, row_ptr, col_idx, val):
        self.n = int(n)
        self.row_ptr, self.col_idx, self.val = row_ptr, col_idx, val
        rp, dev_rp, k0 = _ptr(row_ptr)
        ci, dev_ci, k1 = _ptr(col_idx)
        va, dev_va, k2 = _ptr(val)
        if not (dev_rp == dev_ci == dev_va):
            raise ValueError("row_ptr, col_idx and val must all be on the device or all on the host")
        self._keep = (k0, k1, k2)
        vdt = str(getattr(val, "dtype", "")).replace("torch.", "")
        if vdt not in ("float64", "float32"):
            raise ValueError("val must be float64 or float32")
        nnz = int(col_idx.shape[0])
        self.desc = dos_csr(self.n, nnz, rp, ci, va, DOS_F64 if vdt == "float64" else DOS_F32,
                            DOS_DEVICE if dev_rp else DOS_HOST)
        self.on_device = dev_rp

    @classmethod
    def from_synthetic(cls, A, device=None, dtype=None):
        """From a synthetic.CSR; device=None keeps host numpy arrays."""
        val = A.val if dtype is None else A.val.astype(dtype)
        if device is None:
            return cls(A.n, np.ascontiguousarray(A.row_ptr), np.ascontiguousarray(A.col_idx),
                       np.ascontiguousarray(val))
        import torch
        return cls(A.n, torch.from_numpy(np.ascontiguousarray(A.row_ptr)).to(device),
                   torch.from_numpy(np.ascontiguousarray(A.col_idx)).to(device),
                   torch.from_numpy(np.ascontiguousarray(val)).to(device))


class Context:
    """One libdos context (dos_ctx) bound to a CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        rc = _lib.dos_ctx_create(C.byref(h), int(device))
        if rc != DOS_OK:
            raise DosError(rc, "dos_ctx_create failed")
        self._h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None):
            _lib.dos_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int):
        if rc != DOS_OK:
            raise DosError(rc, _lib.dos_last_error(self._h).decode())

    def last_error(self) -> str:
        return _lib.dos_last_error(self._h).decode()

    # ---- entry points -----------------------------------------------------------
    def dos_profile_enable(self, on: bool = True):
        self._check(_lib.dos_profile_enable(self._h, 1 if on else 0))

    def dos_profile_read(self):
        """dict(step_ms, step_launches, sweeps, launches) accumulated since enabling."""
        ms = C.c_double()
        sl, sw, la = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(_lib.dos_profile_read(self._h, C.byref(ms), C.byref(sl), C.byref(sw),
                                          C.byref(la)))
        return {"step_ms": ms.value, "step_launches": sl.value, "sweeps": sw.value,
                "launches": la.value}

    def dos_validate_csr(self, A: CSRArrays):
        self._check(_lib.dos_validate_csr(self._h, C.byref(A.desc), _stream_of(A.row_ptr)))

    def dos_start_vectors(self, n: int, n_v: int, seed: int, batch_index: int = 0,
                          vec_offset: int = 0, dtype="float64", out=None):
        """(n, n_v) block of +-1 start vectors (numpy unless `out` is given)."""
        if out is None:
            out = np.empty((n, n_v), dtype=np.dtype(dtype))
        dt = str(out.dtype).replace("torch.", "")
        po, _, k = _ptr(out)
        self._check(_lib.dos_start_vectors(self._h, int(n), int(n_v), int(seed), int(batch_index),
                                           int(vec_offset), DOS_F64 if dt == "float64" else DOS_F32,
                                           po, _stream_of(out)))
        return out

    def dos_bounds(self, A: CSRArrays, method="gershgorin", steps: int = 20, seed: int = 0,
                   pad_frac: float = 0.01):
        lb, ub = C.c_double(), C.c_double()
        m = BOUNDS[method] if isinstance(method, str) else int(method)
        self._check(_lib.dos_bounds(self._h, C.byref(A.desc), m, int(steps), int(seed),
                                    float(pad_frac), C.byref(lb), C.byref(ub),
                                    _stream_of(A.row_ptr)))
        return lb.value, ub.value

    def dos_bounds_batched(self, A: CSRArrays, seg_rows, pad_frac: float = 0.01):
        """Gershgorin (lb, ub) arrays of the B concatenated matrices."""
        seg = np.ascontiguousarray(seg_rows, dtype=np.int64)
        B = seg.shape[0] - 1
        lb = np.empty(B)
        ub = np.empty(B)
        self._check(_lib.dos_bounds_batched(self._h, C.byref(A.desc), B, seg.ctypes.data,
                                            float(pad_frac), lb.ctypes.data, ub.ctypes.data,
                                            _stream_of(A.row_ptr)))
        return lb, ub

    def _opts(self, flags=0, vec_offset=0, batch_index=0, launch=None, wait_limit_cycles=0):
        o = dos_kpm_opts()
        o.flags = int(flags)
        o.vec_offset = int(vec_offset)
        o.batch_index = int(batch_index)
        o.wait_limit_cycles = int(wait_limit_cycles)
        if launch:
            o.launch = dos_launch(*[int(launch.get(k, 0))
                                    for k in ("team", "chunks", "block", "tiles", "staged",
                                              "chunk_bytes", "depth", "panel")])
        return o

    def dos_kpm_moments(self, A: CSRArrays, lb: float, ub: float, M: int, n_v: int, seed: int,
                        precision="f64", mu=None, mu_per_vec=None, flags=0, vec_offset=0,
                        batch_index=0, launch=None, wait_limit_cycles=0):
        """Moments mu_0..mu_M (numpy float64 unless `mu` is given)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        out = np.empty(M + 1, dtype=np.float64) if mu is None else mu
        pmu, _, k0 = _ptr(out)
        ppv, _, k1 = _ptr(mu_per_vec)
        opts = self._opts(flags, vec_offset, batch_index, launch, wait_limit_cycles)
        self._check(_lib.dos_kpm_moments_ex(self._h, C.byref(A.desc), float(lb), float(ub),
                                            int(M), int(n_v), int(seed), prec, pmu, ppv,
                                            C.byref(opts), _stream_of(A.row_ptr, out)))
        return out

    def dos_kpm_moments_batched(self, A: CSRArrays, seg_rows, lb, ub, M: int, n_v: int,
                                seed: int, precision="f32", mu=None, mu_per_vec=None, flags=0,
                                batch_index=0, launch=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        seg = np.ascontiguousarray(seg_rows, dtype=np.int64)
        B = seg.shape[0] - 1
        lbv = np.ascontiguousarray(lb, dtype=np.float64)
        ubv = np.ascontiguousarray(ub, dtype=np.float64)
        out = np.empty((B, M + 1), dtype=np.float64) if mu is None else mu
        pmu, _, k0 = _ptr(out)
        ppv, _, k1 = _ptr(mu_per_vec)
        opts = self._opts(flags, 0, batch_index, launch)
        self._check(_lib.dos_kpm_moments_batched(self._h, C.byref(A.desc), B, seg.ctypes.data,
                                                 lbv.ctypes.data, ubv.ctypes.data, int(M),
                                                 int(n_v), int(seed), prec, pmu, ppv,
                                                 C.byref(opts), _stream_of(A.row_ptr, out)))
        return out

    def dos_tune(self, A: CSRArrays, n_v: int, precision="f32", seg_rows=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        best = dos_launch()
        ms = C.c_double()
        seg = None if seg_rows is None else np.ascontiguousarray(seg_rows, dtype=np.int64)
        B = 1 if seg is None else seg.shape[0] - 1
        self._check(_lib.dos_tune(self._h, C.byref(A.desc), B,
                                  None if seg is None else seg.ctypes.data, int(n_v), prec,
                                  C.byref(best), C.byref(ms), _stream_of(A.row_ptr)))
        return {"team": best.team, "chunks": best.chunks, "block": best.block,
                "tiles": best.tiles, "staged": best.staged,
                "chunk_bytes": best.chunk_bytes, "depth": best.depth,
                "panel": best.panel}, ms.value

    def dos_reconstruct(self, mu, M: int, damping="jackson", lb: float = -1.0, ub: float = 1.0,
                        t=None, N_t: int = 1000, phi_hat=None, phi_lambda=None,
                        want_lambda: bool = False):
        damp = DAMPINGS[damping] if isinstance(damping, str) else int(damping)
        if t is not None:
            N_t = int(t.shape[0])
        out = np.empty(N_t, dtype=np.float64) if phi_hat is None else phi_hat
        outl = phi_lambda
        if outl is None and want_lambda:
            outl = np.empty(N_t, dtype=np.float64)
        pmu, _, k0 = _ptr(mu)
        pt, _, k1 = _ptr(t)
        po, _, k2 = _ptr(out)
        pl, _, k3 = _ptr(outl)
        self._check(_lib.dos_reconstruct(self._h, pmu, int(M), damp, float(lb), float(ub), pt,
                                         int(N_t), po, pl, _stream_of(mu, out)))
        return (out, outl) if want_lambda or phi_lambda is not None else out

    def dos_reconstruct_batched(self, mu, damping="jackson", t=None, N_t: int = 1000,
                                phi_hat=None):
        """Rows of moments (B, M+1) -> rows of phi_hat (B, N_t)."""
        damp = DAMPINGS[damping] if isinstance(damping, str) else int(damping)
        B, M = int(mu.shape[0]), int(mu.shape[1]) - 1
        if t is not None:
            N_t = int(t.shape[0])
        out = np.empty((B, N_t), dtype=np.float64) if phi_hat is None else phi_hat
        m = mu if _is_torch(mu) else np.ascontiguousarray(mu, dtype=np.float64)
        pm, _, k0 = _ptr(m)
        pt, _, k1 = _ptr(t)
        po, _, k2 = _ptr(out)
        self._check(_lib.dos_reconstruct_batched(self._h, pm, B, M, damp, pt, int(N_t), po,
                                                 _stream_of(m, out)))
        return out

    def dos_lanczos_ritz(self, A: CSRArrays, M: int, n_v: int, seed: int):
        """(theta, weight, m_used): Ritz values / weights per run, shape (n_v, M)."""
        theta = np.empty((n_v, M))
        weight = np.empty((n_v, M))
        m_used = np.empty(n_v, dtype=np.int32)
        self._check(_lib.dos_lanczos_ritz(self._h, C.byref(A.desc), int(M), int(n_v), int(seed),
                                          theta.ctypes.data, weight.ctypes.data,
                                          m_used.ctypes.data, _stream_of(A.row_ptr)))
        return theta, weight, m_used

    def dos_lanczos_dos(self, theta, weight, sigma: float, x):
        n_v, M = theta.shape
        out = np.empty(x.shape[0])
        th = np.ascontiguousarray(theta, dtype=np.float64)
        wt = np.ascontiguousarray(weight, dtype=np.float64)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        self._check(_lib.dos_lanczos_dos(self._h, th.ctypes.data, wt.ctypes.data, int(n_v), int(M),
                                         float(sigma), xx.ctypes.data, int(xx.shape[0]),
                                         out.ctypes.data, C.c_void_p(0)))
        return out

    def dos_haydock_dos(self, theta, weight, eta: float, x):
        n_v, M = theta.shape
        out = np.empty(x.shape[0])
        th = np.ascontiguousarray(theta, dtype=np.float64)
        wt = np.ascontiguousarray(weight, dtype=np.float64)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        self._check(_lib.dos_haydock_dos(self._h, th.ctypes.data, wt.ctypes.data, int(n_v), int(M),
                                         float(eta), xx.ctypes.data, int(xx.shape[0]),
                                         out.ctypes.data, C.c_void_p(0)))
        return out

    def dos_points_error(self, pts, wts, lb: float, ub: float, sigma: float, eig=None,
                         ref_mu=None, ref_damping="jackson", N_x: int = 4000):
        p = np.ascontiguousarray(pts, dtype=np.float64).ravel()
        w = np.ascontiguousarray(wts, dtype=np.float64).ravel()
        pe, _, k1 = _ptr(eig)
        pr, _, k2 = _ptr(ref_mu)
        n_eig = 0 if eig is None else int(eig.shape[0])
        M_ref = -1 if ref_mu is None else int(ref_mu.shape[0]) - 1
        rdamp = DAMPINGS[ref_damping] if isinstance(ref_damping, str) else int(ref_damping)
        e1, einf = C.c_double(), C.c_double()
        self._check(_lib.dos_points_error(self._h, p.ctypes.data, w.ctypes.data, int(p.shape[0]),
                                          float(lb), float(ub), pe, n_eig, pr, M_ref, rdamp,
                                          float(sigma), int(N_x), C.byref(e1), C.byref(einf),
                                          C.c_void_p(0)))
        return e1.value, einf.value

    def dos_heat_capacity(self, betas, mu=None, M=None, damping="jackson", lb=-1.0, ub=1.0,
                          pts=None, wts=None):
        """<phi, g_beta> for each beta, from KPM moments or from weighted points."""
        b = np.ascontiguousarray(betas, dtype=np.float64)
        out = np.empty(b.shape[0])
        damp = DAMPINGS[damping] if isinstance(damping, str) else int(damping)
        if mu is not None:
            m = np.ascontiguousarray(mu, dtype=np.float64)
            self._check(_lib.dos_heat_capacity(self._h, m.ctypes.data,
                                               int(M if M is not None else m.shape[0] - 1), damp,
                                               float(lb), float(ub), None, None, 0,
                                               b.ctypes.data, int(b.shape[0]), out.ctypes.data,
                                               C.c_void_p(0)))
        else:
            p = np.ascontiguousarray(pts, dtype=np.float64).ravel()
            w = np.ascontiguousarray(wts, dtype=np.float64).ravel()
            self._check(_lib.dos_heat_capacity(self._h, None, 0, damp, 0.0, 1.0, p.ctypes.data,
                                               w.ctypes.data, int(p.shape[0]), b.ctypes.data,
                                               int(b.shape[0]), out.ctypes.data, C.c_void_p(0)))
        return out

    def dos_moments_from_grid(self, phi_hat, M_out: int, mu=None):
        """Moments mu_0..mu_M_out of a DOS given at the Chebyshev nodes."""
        out = np.empty(M_out + 1, dtype=np.float64) if mu is None else mu
        pp, _, k0 = _ptr(phi_hat)
        po, _, k1 = _ptr(out)
        self._check(_lib.dos_moments_from_grid(self._h, pp, int(phi_hat.shape[0]), int(M_out),
                                               po, _stream_of(phi_hat, out)))
        return out

    def dos_smoothed_error(self, mu, M: int, damping, lb: float, ub: float, sigma: float,
                           eig=None, ref_mu=None, ref_damping="jackson", N_x: int = 4000):
        damp = DAMPINGS[damping] if isinstance(damping, str) else int(damping)
        rdamp = DAMPINGS[ref_damping] if isinstance(ref_damping, str) else int(ref_damping)
        pmu, _, k0 = _ptr(mu)
        pe, _, k1 = _ptr(eig)
        pr, _, k2 = _ptr(ref_mu)
        n_eig = 0 if eig is None else int(eig.shape[0])
        M_ref = -1 if ref_mu is None else int(ref_mu.shape[0]) - 1
        e1, einf = C.c_double(), C.c_double()
        self._check(_lib.dos_smoothed_error(self._h, pmu, int(M), damp, float(lb), float(ub), pe,
                                            n_eig, pr, M_ref, rdamp, float(sigma), int(N_x),
                                            C.byref(e1), C.byref(einf), _stream_of(mu)))
        return e1.value, einf.value

    def dos_legendre_moments(self, A: CSRArrays, lb: float, ub: float, M: int, n_v: int,
                             seed: int, precision="f64", nu=None, nu_per_vec=None, flags=0,
                             vec_offset=0, batch_index=0, launch=None):
        """Legendre moments nu_0..nu_M of the same start vectors as dos_kpm_moments."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        out = np.empty(M + 1, dtype=np.float64) if nu is None else nu
        pnu, _, k0 = _ptr(out)
        ppv, _, k1 = _ptr(nu_per_vec)
        opts = self._opts(flags, vec_offset, batch_index, launch)
        self._check(_lib.dos_legendre_moments(self._h, C.byref(A.desc), float(lb), float(ub),
                                              int(M), int(n_v), int(seed), prec, pnu, ppv,
                                              C.byref(opts), _stream_of(A.row_ptr, out)))
        return out

    def dos_cheb_to_legendre(self, mu, nu=None):
        """Rows of Chebyshev moments (last axis M+1) to Legendre moments."""
        M = int(mu.shape[-1]) - 1
        count = int(np.prod(mu.shape[:-1])) if len(mu.shape) > 1 else 1
        if nu is None:
            src = np.ascontiguousarray(mu, dtype=np.float64) if not _is_torch(mu) else mu
            out = np.empty(tuple(mu.shape), dtype=np.float64) if not _is_torch(mu) else \
                mu.new_empty(mu.shape)
        else:
            src, out = mu, nu
        pm, _, k0 = _ptr(src)
        po, _, k1 = _ptr(out)
        self._check(_lib.dos_cheb_to_legendre(self._h, pm, count, M, po, _stream_of(src, out)))
        return out

    def dos_kpml_reconstruct(self, nu, lb: float = -1.0, ub: float = 1.0, t=None,
                             N_t: int = 1000, want_lambda: bool = False):
        n = np.ascontiguousarray(nu, dtype=np.float64)
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        if tt is not None:
            N_t = int(tt.shape[0])
        out = np.empty(N_t)
        outl = np.empty(N_t) if want_lambda else None
        self._check(_lib.dos_kpml_reconstruct(self._h, n.ctypes.data, int(n.shape[0]) - 1,
                                              float(lb), float(ub),
                                              None if tt is None else tt.ctypes.data, int(N_t),
                                              out.ctypes.data,
                                              None if outl is None else outl.ctypes.data,
                                              C.c_void_p(0)))
        return (out, outl) if want_lambda else out

    def dos_dgl(self, nu, lb: float, ub: float, sigma: float, tol: float = 1e-6, x=None,
                N_x: int = 4000):
        """(phi, m_used) of the DGL density at x (eigenvalue units; None: the metric grid)."""
        n = np.ascontiguousarray(nu, dtype=np.float64)
        xx = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        if xx is not None:
            N_x = int(xx.shape[0])
        phi = np.empty(N_x)
        used = np.empty(N_x, dtype=np.int32)
        self._check(_lib.dos_dgl(self._h, n.ctypes.data, int(n.shape[0]) - 1, float(lb),
                                 float(ub), float(sigma), float(tol),
                                 None if xx is None else xx.ctypes.data, int(N_x),
                                 phi.ctypes.data, used.ctypes.data, C.c_void_p(0)))
        return phi, used

    def dos_legendre_error(self, nu, method, lb: float, ub: float, sigma: float,
                           tol: float = 1e-6, eig=None, ref_mu=None, ref_damping="jackson",
                           N_x: int = 4000):
        meth = LEGENDRE_METHODS[method] if isinstance(method, str) else int(method)
        rdamp = DAMPINGS[ref_damping] if isinstance(ref_damping, str) else int(ref_damping)
        if not _is_torch(nu):
            nu = np.ascontiguousarray(nu, dtype=np.float64)
        if eig is not None and not _is_torch(eig):
            eig = np.ascontiguousarray(eig, dtype=np.float64)
        if ref_mu is not None and not _is_torch(ref_mu):
            ref_mu = np.ascontiguousarray(ref_mu, dtype=np.float64)
        pn, _, k0 = _ptr(nu)
        pe, _, k1 = _ptr(eig)
        pr, _, k2 = _ptr(ref_mu)
        n_eig = 0 if eig is None else int(eig.shape[0])
        M_ref = -1 if ref_mu is None else int(ref_mu.shape[0]) - 1
        e1, einf = C.c_double(), C.c_double()
        self._check(_lib.dos_legendre_error(self._h, pn, int(nu.shape[0]) - 1, meth, float(lb),
                                            float(ub), float(sigma), float(tol), pe, n_eig, pr,
                                            M_ref, rdamp, int(N_x), C.byref(e1), C.byref(einf),
                                            _stream_of(nu)))
        return e1.value, einf.value


class MLP:
    """dos_mlp (include/dos_mlp.h): moments -> DOS network trained by the library."""

    def __init__(self, ctx: Context, n_in: int = 64, n_hidden: int = 512, n_out: int = 256,
                 seed: int = 0, _handle=None):
        self.ctx = ctx
        if _handle is None:
            h = C.c_void_p()
            ctx._check(_lib.dos_mlp_create(ctx._h, int(n_in), int(n_hidden), int(n_out),
                                           int(seed), C.byref(h)))
        else:
            h = _handle
        self._h = h
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        cnt = C.c_int64()
        ctx._check(_lib.dos_mlp_num_params(h, C.byref(cnt)))
        self.n_params = cnt.value

    @classmethod
    def dos_mlp_load(cls, ctx: Context, path: str):
        """A network restored from a file written by dos_mlp_save."""
        h = C.c_void_p()
        ctx._check(_lib.dos_mlp_load(ctx._h, os.fsencode(path), C.byref(h), C.c_void_p(0)))
        with open(path, "rb") as f:
            head = f.read(20)
        n_in, nh, n_out = (int.from_bytes(head[8 + 4 * i:12 + 4 * i], "little")
                           for i in range(3))
        return cls(ctx, n_in, nh, n_out, _handle=h)

    def dos_mlp_save(self, path: str):
        self.ctx._check(_lib.dos_mlp_save(self._h, os.fsencode(path), C.c_void_p(0)))

    def dos_mlp_infer(self, x, out=None, max_rows: int = 0, col0: int = 0):
        """network(x[:, col0:col0 + n_in]) for any number of rows (sliced through
        bounded buffers); x float32 or float64 (e.g. the moments of a batched sweep
        with col0 = 1), host or device, rows contiguous."""
        if _is_torch(x):
            xa = x
            dt = str(x.dtype).replace("torch.", "")
        else:
            xa = np.ascontiguousarray(x)
            if xa.dtype not in (np.float32, np.float64):
                xa = xa.astype(np.float32)
            dt = str(xa.dtype)
        if _is_torch(xa) and not xa.is_contiguous():
            raise ValueError("x must be contiguous")
        B, ldx = int(xa.shape[0]), int(xa.shape[1])
        if col0 < 0 or col0 + self.n_in > ldx:
            raise ValueError("x has too few columns for n_in at col0")
        esz = 8 if dt == "float64" else 4
        y = np.empty((B, self.n_out), dtype=np.float32) if out is None else out
        px, _, k0 = _ptr(xa)
        py, _, k1 = _ptr(y)
        self.ctx._check(_lib.dos_mlp_infer(self._h, px + col0 * esz,
                                           DOS_F64 if dt == "float64" else DOS_F32, ldx, B, py,
                                           int(max_rows), _stream_of(xa, y)))
        return y

    def close(self):
        if getattr(self, "_h", None):
            _lib.dos_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dos_mlp_set_params(self, params):
        p, _, k = _ptr(np.ascontiguousarray(params, dtype=np.float32)
                       if not _is_torch(params) else params)
        self.ctx._check(_lib.dos_mlp_set_params(self._h, p, _stream_of(params)))

    def dos_mlp_get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self.ctx._check(_lib.dos_mlp_get_params(self._h, out.ctypes.data, C.c_void_p(0)))
        return out

    def dos_mlp_forward(self, x, out=None):
        xa = x if _is_torch(x) else np.ascontiguousarray(x, dtype=np.float32)
        B = int(xa.shape[0])
        y = np.empty((B, self.n_out), dtype=np.float32) if out is None else out
        px, _, k0 = _ptr(xa)
        py, _, k1 = _ptr(y)
        self.ctx._check(_lib.dos_mlp_forward(self._h, px, B, py, _stream_of(xa, y)))
        return y

    def dos_mlp_loss_grad(self, x, target, want_grads=True):
        xa = x if _is_torch(x) else np.ascontiguousarray(x, dtype=np.float32)
        ta = target if _is_torch(target) else np.ascontiguousarray(target, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32) if want_grads else None
        loss = C.c_float()
        px, _, k0 = _ptr(xa)
        pt, _, k1 = _ptr(ta)
        pg, _, k2 = _ptr(g)
        self.ctx._check(_lib.dos_mlp_loss_grad(self._h, px, pt, int(xa.shape[0]), C.byref(loss),
                                               pg, _stream_of(xa, ta)))
        return loss.value, g

    def dos_mlp_train_step(self, x, target, lr: float, want_loss: bool = True):
        xa = x if _is_torch(x) else np.ascontiguousarray(x, dtype=np.float32)
        ta = target if _is_torch(target) else np.ascontiguousarray(target, dtype=np.float32)
        px, _, k0 = _ptr(xa)
        pt, _, k1 = _ptr(ta)
        loss = C.c_float()
        self.ctx._check(_lib.dos_mlp_train_step(self._h, px, pt, int(xa.shape[0]), float(lr),
                                                C.byref(loss) if want_loss else None,
                                                _stream_of(xa, ta)))
        return loss.value if want_loss else None


def status_string(status: int) -> str:
    return _lib.dos_status_string(int(status)).decode()
