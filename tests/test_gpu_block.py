"""GPU parity of the block COCG path (rsn_solve_columns_block /
rsn_transmission_block) against the CPU oracle.

Blocks of 4, 8 or 16 columns of one energy share one Krylov space; the block
recurrence runs in complex FP32 under FP64 outer steps, so its columns meet the
FP64 residual target of the options (mixed defaults: ||b - A x|| <= 1e-10 ||b||)
and, with the goal-oriented finish (tol_T = 1e-7), each column's T partial
t_c = sum_L Gamma_L |x_c|^2 to ~1e-7 of itself.  Bounds: columns against the
oracle's sparse LU at 1e-8 relative (residual 1e-10 times the modest condition
numbers of these small junctions), t_c and T at 1e-6 relative (the mixed-mode
bound of the plain path), the benchmark junction's golden per-column values
(tests/golden, oracle sparse LU) at 1e-6 for T and 1e-3 for each column, the
bounds of the plain mixed mode.  Blocks that lose their orthogonality hand their
columns to the plain solver, so every column meets the same targets.
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


def _tc(j, X):
    return (j.gamma_l[:, None] * np.abs(X) ** 2).sum(0)


# small cross-sections keep the oracle's sparse LU at seconds: even nx (the
# FP32 point-pair operator), odd nx and N (8-byte aligned vectors: the register
# operator), order 12 with s/p/d projectors; the benchmark junction is covered
# by its golden values below
JUNCTIONS = {
    "junction_R4": lambda: P.molecular_junction(seed=3, nx=12, ny=12, nz=40, n_wells=4, n_cap=5),
    "ragged_R3": lambda: P.molecular_junction(seed=5, nx=13, ny=11, nz=37, fd_half_order=3, n_wells=3, n_cap=4),
    "spd_R6": lambda: P.molecular_junction(seed=4, nx=12, ny=12, nz=40, fd_half_order=6, n_wells=3, lmax=2,
                                           n_cap=6, h=0.3),
}


@pytest.mark.parametrize("name", sorted(JUNCTIONS))
@pytest.mark.parametrize("blk", [4, 8, 16])
def test_block_columns_match_lu(B, name, blk):
    """Columns and T partials of blocks (the last block of each energy ragged
    and padded) against the oracle's sparse LU at two energies."""
    j = JUNCTIONS[name]()
    cols = P.column_subset(j, 2 * blk + 3, seed=11)
    E = [0.19, 0.23]
    ctx = B.Context(0).set_junction(j)
    x, tc, its, rel = ctx.solve_columns_block(E, cols, block=blk)
    x = x.cpu().numpy()
    assert np.all(its > 0) and rel.max() <= 1e-10, (its.min(), rel.max())
    T_ref = np.zeros(len(E))
    for e, En in enumerate(E):
        X_ref = O.solve_columns(j, En, cols)
        dx = np.linalg.norm(x[e].T - X_ref, axis=0) / np.linalg.norm(X_ref, axis=0)
        assert dx.max() <= 1e-8, (En, dx.max())
        t_ref = _tc(j, X_ref)
        assert np.all(np.abs(tc[e] - t_ref) <= 1e-6 * t_ref), (En, (np.abs(tc[e] - t_ref) / t_ref).max())
        # the reported partials are those of the returned columns
        assert np.allclose(tc[e], _tc(j, x[e].T), rtol=1e-12, atol=0)
        T_ref[e] = 4.0 * np.sum(j.gamma_r[cols] * t_ref)
    T = ctx.transmission_block(E, cols, block=blk)
    assert np.all(np.abs(T - T_ref) <= 1e-6 * T_ref), np.abs(T - T_ref) / T_ref
    ctx.close()


def test_block_waveguide_open_channels(B):
    """Every right-CAP column of the 8x8 waveguide in blocks of 16 at energies
    with 1, 3 and 4 open channels: T against the oracle's LU at 1e-7 relative."""
    j = P.waveguide(nx=8, ny=8, nz=48)
    E = [0.8, 1.5, 1.95]
    ctx = B.Context(0).set_junction(j)
    T = ctx.transmission_block(E, block=16)
    T_ref = O.transmission(j, E)
    assert np.all(np.abs(T - T_ref) <= 1e-7 * np.abs(T_ref)), (T, T_ref)
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


def test_block_benchmark_junction_golden(B):
    """The benchmark junction (24x24x120, every channel closed, T ~ 1e-16..1e-10)
    at three energies of its window: the 16 golden columns as one block per
    energy against the oracle's sparse-LU values, with the bounds of the plain
    mixed mode: T at 1e-6 relative, each column at 1e-3 (the goal-oriented
    finish at tol_T = 1e-7 fixes the tiniest shares, ~1e-22 of the column norm,
    to ~1e-4; they weigh nothing in T)."""
    j = P.molecular_junction(seed=1)
    ctx = B.Context(0).set_junction(j)
    gold = _golden()
    for E, cols, t_ref in gold:
        T, tc, its = ctx.transmission_block([E], cols, block=16, return_cols=True)
        rel = np.abs(tc[0] - t_ref) / t_ref
        assert rel.max() <= 1e-3, (E, rel.max())
        T_ref = 4.0 * np.sum(j.gamma_r[cols] * t_ref)
        assert abs(T[0] - T_ref) <= 1e-6 * T_ref, (E, T[0], T_ref)
        assert np.all(its > 0)
    ctx.close()


def test_block_edge_cases(B):
    j = JUNCTIONS["junction_R4"]()
    ctx = B.Context(0).set_junction(j)
    cols = P.column_subset(j, 5, seed=12)
    # one column in a block of 4: three padding members
    x1, tc1, _, _ = ctx.solve_columns_block([0.2], cols[:1], block=4)
    X_ref = O.solve_columns(j, 0.2, cols[:1])
    assert np.linalg.norm(x1[0, 0].cpu().numpy() - X_ref[:, 0]) <= 1e-8 * np.linalg.norm(X_ref[:, 0])
    # empty calls
    assert ctx.transmission_block([], cols, block=4).size == 0
    assert np.all(ctx.transmission_block([0.2, 0.3], np.array([], np.int32), block=4) == 0.0)
    # refused arguments
    for kw in ({"block": 5}, {"block": 4, "tol_inner": 1.5}):
        with pytest.raises(B.RsnError) as ei:
            ctx.transmission_block([0.2], cols, **kw)
        assert ei.value.code == B.RSN_EINVAL
    with pytest.raises(B.RsnError) as ei:
        ctx.transmission_block([0.2], cols, block=4, opts=B.default_opts(B.RSN_FP64))
    assert ei.value.code == B.RSN_EINVAL
    with pytest.raises(B.RsnError) as ei:
        ctx.transmission_block([0.2], np.array([cols[0], cols[1], cols[0]], np.int32), block=4)
    assert ei.value.code == B.RSN_EINVAL
    # the context stays usable
    T = ctx.transmission_block([0.2], cols, block=4)
    T_ref = 4.0 * np.sum(j.gamma_r[cols] * _tc(j, O.solve_columns(j, 0.2, cols)))
    assert abs(T[0] - T_ref) <= 1e-6 * T_ref
    ctx.close()
