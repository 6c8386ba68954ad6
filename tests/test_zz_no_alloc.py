"""The allocation-free operator entry point (rsn_apply_noalloc) against the
allocating one (rsn_apply), through the C ABI.

rsn_apply_noalloc serves callers that cannot allocate device memory while
they call the library (a pre-sized memory pool, a real-time loop, a host
framework that owns every allocation).  Its scratch is a fixed device array
shared by all calls, so the test makes two different calls in a row and checks
both, with the tolerances of the operator parity tests: FP64 to 1e-12 and FP32
to 2e-6 of the largest entry.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_1401_0782_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call(B, ctx, fn, prec, E, x):
    E = np.ascontiguousarray(E, dtype=np.float64)
    y = torch.empty_like(x)
    rc = getattr(ctx.lib, fn)(ctx.h, prec, int(E.size), E.ctypes.data, x.data_ptr(), y.data_ptr())
    assert rc == B.RSN_OK, ctx.lib.rsn_last_error(ctx.h).decode()
    return y


def test_noalloc_apply_matches_allocating_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0782_gb300 import binding as B
    j = P.molecular_junction(seed=3, nx=12, ny=12, nz=40, n_wells=4, n_cap=5)
    ctx = B.Context(0).set_junction(j)
    rng = np.random.default_rng(5)
    # before any allocating call the operator is not on the device: refused
    x0 = torch.zeros((1, j.N), dtype=torch.complex128, device="cuda")
    y0 = torch.empty_like(x0)
    E0 = np.array([0.2])
    rc = ctx.lib.rsn_apply_noalloc(ctx.h, B.RSN_FP64, 1, E0.ctypes.data, x0.data_ptr(), y0.data_ptr())
    assert rc == B.RSN_ESTATE
    for call, (prec, dtype, tol) in enumerate([(B.RSN_FP64, torch.complex128, 1e-12),
                                               (B.RSN_FP64, torch.complex128, 1e-12),
                                               (B.RSN_MIXED, torch.complex64, 2e-6),
                                               (B.RSN_MIXED, torch.complex64, 2e-6)]):
        n = 3 + call
        E = rng.uniform(-1.0, 1.5, n)
        xr = rng.standard_normal((n, j.N)) + 1j * rng.standard_normal((n, j.N))
        x = torch.tensor(xr, dtype=dtype, device="cuda")
        y_ref = _call(B, ctx, "rsn_apply", prec, E, x)
        y_na = _call(B, ctx, "rsn_apply_noalloc", prec, E, x)
        torch.cuda.synchronize()
        scale = y_ref.abs().max().item()
        assert (y_na - y_ref).abs().max().item() <= tol * scale
    # beyond the fixed scratch: a clear error, nothing launched
    big = 1 << 20
    rc = ctx.lib.rsn_apply_noalloc(ctx.h, B.RSN_FP64, big, np.zeros(1).ctypes.data, x0.data_ptr(),
                                   y0.data_ptr())
    assert rc == B.RSN_EINVAL
    assert b"fixed array" in ctx.lib.rsn_last_error(ctx.h)
    ctx.close()
