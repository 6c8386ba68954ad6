"""torch.autograd.Function wrapper: gradient of T(E) with respect to V_loc
against central finite differences of the GPU T itself and against the CPU
oracle's adjoint gradient."""
import numpy as np
import pytest

import oracle as O
from paper_1401_0782_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_0782_gb300 import binding
    return binding


@pytest.mark.parametrize("keep", [None, 0])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autograd_matches_oracle_and_finite_differences(B, prec, keep):
    # keep=None: the forward columns stay on the device and the backward pass
    # solves only the adjoints; keep=0: the backward pass solves both again
    from paper_1401_0782_gb300 import autograd as AG
    j = P.molecular_junction(seed=8, nx=10, ny=10, nz=32, n_wells=3, n_cap=4)
    E = [0.18, 0.22]
    cols = j.right_columns()[::9]
    ctx = B.Context(0).set_junction(j)
    opts = B.default_opts(B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED)
    v = torch.tensor(j.v_loc, dtype=torch.float64, device="cuda", requires_grad=True)
    T = AG.transmission(ctx, v, E, cols, opts, keep_bytes=keep)
    w = torch.tensor([1.0, -2.0], dtype=torch.float64, device="cuda")
    (T * w).sum().backward()
    g = v.grad.cpu().numpy()
    T_ref, g_ref = O.transmission_grad(j, E, cols, T_bar=[1.0, -2.0])
    tolT = 1e-9 if prec == "fp64" else 1e-6
    assert np.all(np.abs(T.detach().cpu().numpy() - T_ref) <= tolT * np.maximum(np.abs(T_ref), 1e-3))
    tolg = 1e-8 if prec == "fp64" else 1e-5
    assert np.abs(g - g_ref).max() <= tolg * np.abs(g_ref).max()
    if prec == "fp64" and keep is None:
        # central differences of the GPU T at seeded points (dV = 1e-4 Ha)
        rng = np.random.default_rng(2)
        pts = rng.choice(np.flatnonzero(np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()), 4, replace=False)
        for r in pts:
            vp = j.v_loc.copy(); vp[r] += 1e-4
            vm = j.v_loc.copy(); vm[r] -= 1e-4
            ctx.set_potential(vp)
            Tp = ctx.transmission(E, cols, opts)
            ctx.set_potential(vm)
            Tm = ctx.transmission(E, cols, opts)
            fd = ((Tp - Tm) / 2e-4) @ np.array([1.0, -2.0])
            assert abs(fd - g[r]) <= 1e-5 * np.abs(g).max() + 1e-12
    ctx.close()


def test_reused_columns_give_the_same_gradient_with_fewer_solves(B):
    j = P.molecular_junction(seed=8, nx=10, ny=10, nz=32, n_wells=3, n_cap=4)
    E = [0.18, 0.22]
    Tb = [1.0, -2.0]
    cols = j.right_columns()[::9]
    ctx = B.Context(0).set_junction(j)
    o = B.default_opts(B.RSN_FP64)
    T1, g1 = ctx.transmission_vjp(E, Tb, cols, o)
    it_both = ctx.last_stats()["krylov_iters"]
    T2, x = ctx.transmission_keep(E, cols, o)
    it_fwd = ctx.last_stats()["krylov_iters"]
    g2 = ctx.transmission_vjp_reuse(E, Tb, cols, x, o)
    it_adj = ctx.last_stats()["krylov_iters"]
    assert np.array_equal(T1, T2)
    assert np.abs(g1 - g2).max() <= 1e-10 * np.abs(g1).max()
    # the reuse path solved no forward column again
    assert it_adj < it_both and abs(it_fwd + it_adj - it_both) <= 0.05 * it_both
    ctx.close()
