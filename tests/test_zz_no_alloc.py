"""dos_kpm_moments_noalloc: the sweep for callers that cannot allocate device
memory (their memory is reserved by their own pool allocator, or held to a fixed
budget where cudaMalloc may synchronise the device).  It must give the moments
of dos_kpm_moments, call after call, without the device's free memory moving.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

from synthetic import anderson_3d, laplacian_2d

pytestmark = pytest.mark.gpu


def _noalloc():
    from paper_1308_5467_gb300 import dos
    f = dos._lib.dos_kpm_moments_noalloc
    f.restype = C.c_int
    f.argtypes = [C.POINTER(dos.dos_csr), C.c_double, C.c_double, C.c_int, C.c_int, C.c_uint64,
                  C.c_int, C.c_void_p, C.c_void_p]
    return f


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-9)])
def test_noalloc_matches_allocating_entry_point_twice(precision, tol):
    import torch
    from paper_1308_5467_gb300 import dos
    A = anderson_3d(24, 4.0, seed=2)
    dtype = np.float64 if precision == "f64" else np.float32
    Ad = dos.CSRArrays.from_synthetic(A, device="cuda", dtype=dtype)
    lb, ub, M, n_v, seed = -8.2, 8.2, 300, 48, 5
    with dos.Context(0) as ctx:
        ref = ctx.dos_kpm_moments(Ad, lb, ub, M, n_v, seed, precision=precision)
    f = _noalloc()
    prec = dos.PRECISIONS[precision]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for call in range(2):
        mu = torch.full((M + 1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = f(C.byref(Ad.desc), lb, ub, M, n_v, seed, prec, mu.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == dos.DOS_OK, dos.status_string(rc)
        if call == 1:  # the one-time set-up is done: nothing may be allocated now
            assert torch.cuda.mem_get_info()[0] == free_before
        outs.append(mu.cpu().numpy())
    for out in outs:
        assert np.abs(out - ref).max() <= tol
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_small_matrix_then_limits():
    import torch
    from paper_1308_5467_gb300 import dos
    A = laplacian_2d(40)
    Ad = dos.CSRArrays.from_synthetic(A, device="cuda")
    with dos.Context(0) as ctx:
        ref = ctx.dos_kpm_moments(Ad, -0.08, 8.08, 100, 20, 1, precision="f64")
    f = _noalloc()
    mu = torch.empty(101, dtype=torch.float64, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert f(C.byref(Ad.desc), -0.08, 8.08, 100, 20, 1, dos.DOS_PREC_F64, mu.data_ptr(), s) == 0
    assert np.abs(mu.cpu().numpy() - ref).max() < 1e-12
    # beyond the fixed scratch: 2 * n * 256 * 8 bytes of vector blocks > 63 MiB
    big = dos.CSRArrays.from_synthetic(anderson_3d(40, 1.0, seed=1), device="cuda")
    rc = f(C.byref(big.desc), -7.0, 7.0, 10, 256, 1, dos.DOS_PREC_F64, mu.data_ptr(), s)
    assert rc == dos.DOS_ENOMEM
    # host output pointer is refused
    host = np.empty(101)
    rc = f(C.byref(Ad.desc), -0.08, 8.08, 100, 20, 1, dos.DOS_PREC_F64, host.ctypes.data, s)
    assert rc == dos.DOS_EINVAL
    # a descriptor that says "device" but holds host col_idx / val is refused on the
    # host, before any kernel could read through the host addresses
    ci_h, va_h = np.ascontiguousarray(A.col_idx), np.ascontiguousarray(A.val)
    for ci, va in ((ci_h.ctypes.data, Ad.desc.val), (Ad.desc.col_idx, va_h.ctypes.data)):
        mixed = dos.dos_csr(A.n, A.nnz, Ad.desc.row_ptr, ci, va, dos.DOS_F64, dos.DOS_DEVICE)
        rc = f(C.byref(mixed), -0.08, 8.08, 100, 20, 1, dos.DOS_PREC_F64, mu.data_ptr(), s)
        assert rc == dos.DOS_EINVAL
    # and the entry point still works afterwards
    assert f(C.byref(Ad.desc), -0.08, 8.08, 100, 20, 1, dos.DOS_PREC_F64, mu.data_ptr(), s) == 0
    assert np.abs(mu.cpu().numpy() - ref).max() < 1e-12
