"""Parity at the benchmark sizes, on sampled outputs and on properties that
hold at any size, plus error paths.

* 24x24x120 junction (8th-order FD, 80 projectors): sampled columns certified
  by the oracle's operator (true residual), one column against the oracle's
  certified Krylov solve, the T reduction recomputed by the oracle formula from
  the GPU's own columns; per-column T contributions of 16 columns at three
  energies against the oracle's sparse-LU golden values (relative 1e-9 FP64,
  1e-6 mixed); mixed against FP64 (relative 1e-6).
* 48x48x192 junction (12th-order FD, 540 s/p/d projectors): dT/dV_loc against
  central differences of the GPU T at 32 seeded points, against the sum rule
  sum_r dT/dV_r = -dT/dE (a uniform potential shift is an energy shift) and
  against the oracle's adjoint gradient (golden values); FP64 and mixed agree.
* Error paths: empty calls, bad columns, a deadline that expires, an
  iteration cap that is too small.
"""
import os

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


@pytest.fixture(scope="module")
def junction():
    return P.molecular_junction(seed=1)


def _unit(N, cols):
    b = np.zeros((N, len(cols)), complex)
    b[cols, np.arange(len(cols))] = 1
    return b


def test_junction_columns_certified_and_T_reduction(B, junction):
    j = junction
    cols = P.column_subset(j, 8, seed=8)
    E = 0.2
    ctx = B.Context(0).set_junction(j)
    x64, it64, rr64 = ctx.solve_columns([E], cols, B.default_opts(B.RSN_FP64))
    xm, itm, rrm = ctx.solve_columns([E], cols, B.default_opts(B.RSN_MIXED))
    x64 = x64[0].cpu().numpy().T
    xm = xm[0].cpu().numpy().T
    b = _unit(j.N, cols)
    r64 = np.linalg.norm(b - O.apply_operator(j, E, x64), axis=0)
    rm = np.linalg.norm(b - O.apply_operator(j, E, xm), axis=0)
    assert r64.max() <= 2e-13 and rm.max() <= 1.5e-10, (r64.max(), rm.max())
    assert np.all(it64 > 0) and np.all(itm > 0)
    # one column against the oracle's own certified solve, at the column tolerance
    x_ref = O.solve_columns(j, E, cols[:1], method="krylov", rtol=1e-13)[:, 0]
    assert np.linalg.norm(x64[:, 0] - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # T reduction at full size: oracle formula on the GPU's columns
    T_gpu = ctx.transmission([E], cols, B.default_opts(B.RSN_FP64))[0]
    T_from_cols = 4.0 * np.sum(j.gamma_r[cols] * O.column_weights(j, x64))
    assert abs(T_gpu - T_from_cols) <= 1e-9 * abs(T_from_cols)
    ctx.close()


def _golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "junction_24x24x120_tc.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    out = {}
    for k, E, c, t, _ in rows:
        out.setdefault(float(E), ([], []))
        out[float(E)][0].append(int(c))
        out[float(E)][1].append(float(t))
    return [(E, np.array(c, np.int32), np.array(t)) for E, (c, t) in sorted(out.items())]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_junction_per_column_T_matches_oracle_lu(B, junction, prec):
    """Per-column contributions t_c = sum_L Gamma_L |x_c|^2 and their T at the
    benchmark junction and three energies of its window, against the oracle's
    sparse-LU values (tests/golden, written by make_junction_golden.py).  Every
    lead channel is closed there (T ~ 1e-19..1e-15), so only relative errors
    say anything: FP64 1e-9 for every column and for T; mixed 1e-6 for T and
    1e-3 for each column (the goal-oriented finish at tol_T = 1e-7 fixes the
    tiniest shares, ~1e-22 of the column norm, to ~1e-4; they weigh nothing
    in T)."""
    j = junction
    ctx = B.Context(0).set_junction(j)
    p = B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED
    tol = 1e-9 if prec == "fp64" else 1e-6
    tol_col = 1e-9 if prec == "fp64" else 1e-3
    gl = torch.tensor(j.gamma_l, device="cuda")
    for E, cols, t_ref in _golden():
        x, _, _ = ctx.solve_columns([E], cols, B.default_opts(p))
        tc = (gl[None, :] * x[0].abs() ** 2).sum(1).cpu().numpy()
        rel = np.abs(tc - t_ref) / t_ref
        assert rel.max() <= tol_col, (E, rel.max())
        T = ctx.transmission([E], cols, B.default_opts(p))[0]
        T_ref = 4.0 * np.sum(j.gamma_r[cols] * t_ref)
        assert abs(T - T_ref) <= tol * T_ref, (E, T, T_ref)
    ctx.close()


def test_junction_mixed_vs_fp64_transmission(B, junction):
    j = junction
    cols = P.column_subset(j, 64, seed=9)
    E = [0.17, 0.21]
    ctx = B.Context(0).set_junction(j)
    T64 = ctx.transmission(E, cols, B.default_opts(B.RSN_FP64))
    Tm = ctx.transmission(E, cols, B.default_opts(B.RSN_MIXED))
    # the goal-oriented finish (tol_T 1e-7 mixed, 3e-11 FP64) fixes T to ~1e-7 of itself
    assert np.all(np.abs(Tm - T64) <= 1e-6 * np.abs(T64)), np.abs(Tm - T64) / np.abs(T64)
    ctx.close()


def _adjoint_golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "adjoint_junction_48x48x192_grad.txt")
    if not os.path.exists(path):
        return None
    vals, pts, g = {}, [], []
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        if f[0] == "g":
            pts.append(int(f[1]))
            g.append(float(f[2]))
        else:
            vals[f[0]] = float(f[1])
    return vals, np.array(pts), np.array(g)


def test_large_adjoint_junction_fd_and_sum_rule(B):
    """48x48x192 junction (442,368 points, 12th-order FD, 540 s/p/d projectors),
    four seeded right-CAP columns at E = 0.2 Ha: dT/dV_loc from the adjoint
    against central differences of the GPU T at 32 seeded points (dV = 1e-4
    Ha), the sum rule sum_r dT/dV_r = -dT/dE, the oracle's adjoint gradient
    (tests/golden, its certified Krylov route) at 64 points, and mixed against
    FP64."""
    j = P.adjoint_junction(seed=4)
    assert j.N == 442368 and j.n_proj == 540
    cols = P.column_subset(j, 4, seed=11)
    E = 0.2
    ctx = B.Context(0).set_junction(j)
    # on this junction the FP64 COCG recurrence of the adjoint systems levels off
    # near 5e-11 (measured): they stop at 1e-10, the forward columns keep 1e-13
    o64 = B.default_opts(B.RSN_FP64, tol_adjoint=1e-10)
    T, g = ctx.transmission_vjp([E], [1.0], cols, o64)
    gs = np.abs(g).max()
    assert gs > 0
    gold = _adjoint_golden()
    if gold is not None:
        vals, gp, gv = gold
        # the oracle's forward columns stop at a relative residual of 1e-13, which
        # fixes this junction's T to ~1e-6 of itself; its adjoints at 1e-10
        assert abs(T[0] - vals["T"]) <= 1e-5 * abs(vals["T"]), (T[0], vals["T"])
        assert np.abs(g[gp] - gv).max() <= 1e-5 * vals["max_abs_g"], np.abs(g[gp] - gv).max() / vals["max_abs_g"]
        assert abs(g.sum() - vals["sum_g"]) <= 1e-5 * abs(vals["sum_g"]) + 1e-6 * vals["max_abs_g"]
        pts = gp[:32]
    else:
        rng = np.random.default_rng(4)
        pts = rng.choice(np.flatnonzero(np.abs(g) > 0.05 * gs), 32, replace=False)
    dv = 1e-4
    # a central difference to 1e-4 of max|g| needs T to ~1e-7 of itself here
    # (T 4e-8, max|g| 3e-7): the finite-difference solves stop their goal phase at 1e-9
    o_fd = B.default_opts(B.RSN_FP64, tol_adjoint=1e-10, tol_T=1e-9)
    for r in pts:
        vp = j.v_loc.copy(); vp[r] += dv
        vm = j.v_loc.copy(); vm[r] -= dv
        ctx.set_potential(vp)
        Tp = ctx.transmission([E], cols, o_fd)[0]
        ctx.set_potential(vm)
        Tm = ctx.transmission([E], cols, o_fd)[0]
        fd = (Tp - Tm) / (2 * dv)
        assert abs(fd - g[r]) <= 1e-4 * gs, (r, fd, g[r])
    ctx.set_potential(j.v_loc)
    # T(E) has a resonance of width ~3e-4 Ha here: a central difference with
    # dE = 1e-5 carries a truncation error of ~(dE / width)^2 / 6 = 2e-4
    de = 2e-6
    dTdE = (ctx.transmission([E + de], cols, o64)[0] - ctx.transmission([E - de], cols, o64)[0]) / (2 * de)
    assert abs(g.sum() + dTdE) <= 1e-4 * max(abs(dTdE), gs)
    Tm, gm = ctx.transmission_vjp([E], [1.0], cols, B.default_opts(B.RSN_MIXED))
    assert abs(Tm[0] - T[0]) <= 1e-6 * abs(T[0]) and np.abs(gm - g).max() <= 1e-4 * gs
    ctx.close()


def test_error_paths(B):
    j = P.molecular_junction(seed=3, nx=10, ny=10, nz=30, n_wells=2, n_cap=4)
    ctx = B.Context(0).set_junction(j)
    assert ctx.transmission([], j.right_columns()).size == 0
    assert np.array_equal(ctx.transmission([0.2, 0.3], []), np.zeros(2))
    with pytest.raises(B.RsnError) as e:
        ctx.transmission([0.2], [j.N])
    assert e.value.code == B.RSN_EINVAL
    # an iteration cap that is too small: the columns are reported, not hidden
    x, it, rr = ctx.solve_columns([0.2], j.right_columns()[:4], B.default_opts(B.RSN_FP64, max_iter=5),
                                  raise_on_noconv=False)
    assert np.all(it < 0) and np.all(rr > 1e-6)
    # a deadline that expires
    with pytest.raises(B.RsnError) as e:
        ctx.transmission(np.linspace(0.1, 0.3, 64), j.right_columns(), B.default_opts(B.RSN_FP64, deadline_ms=1.0,
                                                                                      graph_iters=1))
    assert e.value.code == B.RSN_ETIMEOUT
    ctx.close()
