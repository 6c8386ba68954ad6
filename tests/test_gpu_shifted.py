"""Shifted COCG on the GPU (rsn_solve_columns_shifted / rsn_transmission_shifted):
columns at every energy of a window from one seed Krylov space per column,
against the oracle's sparse LU at each energy (FP64: ||dx||/||x|| <= 1e-9,
certified by the oracle's operator) and against the oracle's own shifted COCG;
T(E) over a window against the oracle's LU transmission, including the
waveguide's open-channel staircase; the mixed precision is refused."""
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


def _junction():
    return P.molecular_junction(seed=3, nx=12, ny=12, nz=40, n_wells=4, n_cap=5)


def test_shifted_columns_match_lu_at_every_energy(B):
    j = _junction()
    E = np.linspace(0.15, 0.35, 9)
    cols = j.right_columns()[::71]
    ctx = B.Context(0).set_junction(j)
    x, it, rel = ctx.solve_columns_shifted(E, cols, B.default_opts(B.RSN_FP64))
    x = x.cpu().numpy()
    assert np.all(it > 0), it
    for e, En in enumerate(E):
        ref = O.solve_columns(j, En, cols).T
        err = np.linalg.norm(x[e] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 1e-9, (En, err.max())
        b = np.zeros((j.N, cols.size), complex)
        b[cols, np.arange(cols.size)] = 1
        r = np.linalg.norm(b - O.apply_operator(j, En, x[e].T), axis=0)
        assert r.max() <= 1e-11, (En, r.max())
    # one Krylov space per column: the seed ran at most as long as the slowest
    # energy, far fewer operator applications than one solve per energy
    _, it1, _ = ctx.solve_columns(E, cols, B.default_opts(B.RSN_FP64))
    assert it.max(axis=0).sum() * 3 <= it1.sum(), (it.max(axis=0), it1.sum(axis=0))
    ctx.close()


def test_shifted_columns_match_oracle_shifted_cocg(B):
    j = _junction()
    E = np.array([0.17, 0.2, 0.26, 0.31])
    col = int(j.right_columns()[40])
    ctx = B.Context(0).set_junction(j)
    x, it, _ = ctx.solve_columns_shifted(E, [col], B.default_opts(B.RSN_FP64))
    b = np.zeros(j.N, complex)
    b[col] = 1
    seed = int(np.argmin(np.abs(E - 0.5 * (E.min() + E.max()))))
    Xo, k, _, _ = O.shifted_cocg(j, E, b, seed=seed, rtol=1e-13)
    xg = x[:, 0].cpu().numpy()
    err = np.linalg.norm(xg - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
    assert err.max() <= 1e-9, err
    assert abs(int(it.max()) - k) <= 2, (it, k)  # the same recurrence, up to rounding at the stop
    ctx.close()


@pytest.mark.parametrize("name", ["waveguide", "junction"])
def test_shifted_transmission_matches_oracle(B, name):
    if name == "waveguide":
        j = P.waveguide()
        E = P.energy_grid(0.05, 2.0, 64)[::4]
        cols = None
    else:
        j = _junction()
        E = np.linspace(0.16, 0.24, 12)
        cols = j.right_columns()[::13]
    ctx = B.Context(0).set_junction(j)
    T, it = ctx.transmission_shifted(E, cols, B.default_opts(B.RSN_FP64), return_iters=True)
    T_ref = O.transmission(j, E, cols)
    assert np.all(np.abs(T - T_ref) <= 1e-9 * np.maximum(np.abs(T_ref), 1e-3)), np.abs(T - T_ref).max()
    if name == "junction":
        T_plain = ctx.transmission(E, cols, B.default_opts(B.RSN_FP64))
        assert np.all(np.abs(T - T_plain) <= 1e-9 * np.maximum(np.abs(T_ref), 1e-3))
    ctx.close()


def test_shifted_refuses_mixed_precision(B):
    j = _junction()
    ctx = B.Context(0).set_junction(j)
    with pytest.raises(B.RsnError) as e:
        ctx.transmission_shifted([0.2, 0.21], j.right_columns()[:4], B.default_opts(B.RSN_MIXED))
    assert e.value.code == B.RSN_EINVAL
    ctx.close()
