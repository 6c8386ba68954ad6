"""Batched uneven junctions through rsn_batch_transmission (one slot pool over
all the junctions of a device): each junction's T(E) against the same junction
solved alone and against the CPU oracle (sparse LU), in FP64 and mixed
precision; error reporting per junction."""
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


def _junctions():
    # uneven cross-sections, lengths, CAP depths and well counts, 8th-order FD,
    # built as the batched workload but small enough for the oracle's LU
    specs = [(10, 32, 4, 2), (12, 40, 5, 3), (14, 36, 6, 4), (11, 48, 4, 3)]
    return [P.molecular_junction(seed=20 + k, nx=n, ny=n, nz=nz, n_cap=cap, n_wells=w)
            for k, (n, nz, cap, w) in enumerate(specs)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_single_junction_and_oracle(B, prec):
    js = _junctions()
    ctxs = [B.Context(0).set_junction(j) for j in js]
    energies = [np.linspace(0.15 + 0.02 * k, 0.35, 3) for k in range(len(js))]
    cols = [j.right_columns()[::7] for j in js]
    opts = B.default_opts(B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED)
    Tb = B.batch_transmission(ctxs, energies, cols, opts)
    assert len(Tb) == len(js)
    for k, (j, ctx) in enumerate(zip(js, ctxs)):
        T_alone = ctx.transmission(energies[k], cols[k], opts)
        T_ref = O.transmission(j, energies[k], cols[k])
        if prec == "fp64":
            tol = 1e-9 * np.maximum(np.abs(T_ref), 1e-3)
        else:
            tol = np.full(T_ref.shape, 1e-6)
        assert np.all(np.abs(Tb[k] - T_ref) <= tol), (k, Tb[k], T_ref)
        assert np.all(np.abs(Tb[k] - T_alone) <= tol), (k, Tb[k], T_alone)
    for c in ctxs:
        c.close()


def test_batch_reports_the_failing_junction(B):
    js = _junctions()[:3]
    ctxs = [B.Context(0).set_junction(j) for j in js]
    energies = [[0.2], [0.2], [0.2]]
    cols = [js[0].right_columns()[:4], np.array([js[1].N + 5], np.int32), js[2].right_columns()[:4]]
    with pytest.raises(B.RsnError) as e:
        B.batch_transmission(ctxs, energies, cols, B.default_opts(B.RSN_FP64))
    assert e.value.code == B.RSN_EINVAL and "junction 1" in str(e.value)
    # a context listed twice is refused
    with pytest.raises(B.RsnError) as e:
        B.batch_transmission([ctxs[0], ctxs[0]], [[0.2], [0.2]], None, B.default_opts(B.RSN_FP64))
    assert e.value.code == B.RSN_EINVAL
    for c in ctxs:
        c.close()


def test_one_pool_over_sixteen_uneven_junctions(B):
    # the 16 smallest of the 64 seeded uneven junctions (cross-sections 12..21,
    # odd and even, so the pool runs the point-pair and the register kernel
    # side by side): pooled T against each junction alone, and against the
    # oracle's LU on the three smallest
    js = P.batched_junctions()
    pick = sorted(range(len(js)), key=lambda k: js[k].N)[:16]
    sub = [js[k] for k in pick]
    assert len({j.nx % 2 for j in sub}) == 2
    ctxs = [B.Context(0).set_junction(j) for j in sub]
    energies = [np.array([0.18, 0.22]) for _ in sub]
    cols = [j.right_columns()[::97] for j in sub]
    for prec in (B.RSN_FP64, B.RSN_MIXED):
        o = B.default_opts(prec)
        Tb = B.batch_transmission(ctxs, energies, cols, o)
        for k, (j, ctx) in enumerate(zip(sub, ctxs)):
            T_alone = ctx.transmission(energies[k], cols[k], o)
            # the pool and the lone solve differ only by the operator tiling (rounding
            # order) and where the goal-oriented finish stops.  Where T falls below
            # ~1e-30 in FP64, or ~1e-20 in the mixed mode (long junctions with every
            # lead channel closed), the Gamma_L tail of a column sits at the
            # precision floor of its recurrence: T is rounding noise there and only
            # its smallness is checked; above it FP64 agrees to 1e-8, mixed to 1e-5
            floor, rel = (1e-30, 1e-8) if prec == B.RSN_FP64 else (1e-20, 1e-5)
            big = np.abs(T_alone) > floor
            assert np.all(np.abs(Tb[k] - T_alone)[big] <= rel * np.abs(T_alone)[big]), (k, Tb[k], T_alone)
            assert np.all(np.abs(Tb[k])[~big] <= 1e3 * floor), (k, Tb[k], T_alone)
            if prec == B.RSN_FP64 and k < 3:
                T_ref = O.transmission(j, energies[k], cols[k])
                assert np.all(np.abs(Tb[k] - T_ref) <= 1e-8 * np.abs(T_ref)), (k, Tb[k], T_ref)
    for c in ctxs:
        c.close()
