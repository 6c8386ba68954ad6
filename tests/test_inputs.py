"""The seeded synthetic inputs (shapes, value ranges, CAP profile, column sets,
batched size draws) match the recipe they are documented with, and repeat
exactly for a seed.  CPU only; the builders hold none of the method's
arithmetic."""
import numpy as np
import pytest

from paper_1401_0782_gb300 import problems as P


@pytest.fixture(scope="module")
def junction():
    return P.molecular_junction(seed=1)


def test_bench_junction_shape_and_projectors(junction):
    j = junction
    assert (j.nx, j.ny, j.nz, j.N) == (24, 24, 120, 69120)
    assert j.fd_half_order == 4 and j.h == 0.35
    assert j.n_proj == 80  # 20 atoms x (s + 3 p)
    # every projector has unit 2-norm (quadrature weight folded in) and a support
    # of the |r| <= 2 r_c ball (~2,600 points at h = 0.35)
    for p in range(j.n_proj):
        v = j.proj_val[j.proj_offsets[p]:j.proj_offsets[p + 1]]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert 2000 < v.size < 3200
    # E_KB shared by the 3 p projectors of an atom
    e = j.proj_ekb.reshape(20, 4)
    assert np.all(e[:, 1:] == e[:, 1:2]) and np.all(np.abs(e) <= 1.0)


def test_quadratic_cap_profile(junction):
    j = junction
    plane = j.nx * j.ny
    gl = j.gamma_l.reshape(j.nz, plane)
    gr = j.gamma_r.reshape(j.nz, plane)
    # uniform over each plane, mirror images, A (d / n_cap)^2 with d = n_cap at the box end
    assert np.all(gl == gl[:, :1]) and np.all(gr == gr[:, :1])
    assert np.array_equal(gl[::-1], gr)
    prof = gr[:, 0]
    n = j.n_cap
    assert n == 8 and np.count_nonzero(prof) == n
    for d in range(1, n + 1):
        assert prof[j.nz - 1 - (n - d)] == pytest.approx(0.5 * (d / n) ** 2, rel=0, abs=1e-15)
    assert j.right_columns().size == n * plane == 4608


def test_potential_walls_and_wells(junction):
    j = junction
    v = j.v_loc.reshape(j.nz, j.ny, j.nx)
    # corners of the outer lead planes (wells sit in the central third only):
    # V = 3 (1 - s^2), s = (1 + tanh((a - d) / w)) / 2 with a = 8 h (16-point
    # square), d = 11.5 h from the axis, w = 0.5 bohr
    s = 0.5 * (1.0 + np.tanh((8 * 0.35 - 11.5 * 0.35) / 0.5))
    lead = np.r_[0:j.nz // 6, 5 * j.nz // 6:j.nz]
    assert np.allclose(v[lead, 0, 0], 3.0 * (1.0 - s * s), rtol=0, atol=1e-9)
    assert np.allclose(v[lead, -1, -1], 3.0 * (1.0 - s * s), rtol=0, atol=1e-9)
    # the lead planes at the ends hold no well: centre of the soft square ~ 0
    assert abs(v[0, j.ny // 2, j.nx // 2]) < 1e-3
    # wells lower the potential in the central third only
    mid = v[j.nz // 3: 2 * j.nz // 3]
    assert mid.min() < -0.5 and v[: j.nz // 4].min() > -1e-3


def test_seeded_builders_repeat_exactly():
    a = P.molecular_junction(seed=5, nx=10, ny=10, nz=30, n_wells=3, n_cap=4)
    b = P.molecular_junction(seed=5, nx=10, ny=10, nz=30, n_wells=3, n_cap=4)
    c = P.molecular_junction(seed=6, nx=10, ny=10, nz=30, n_wells=3, n_cap=4)
    assert np.array_equal(a.v_loc, b.v_loc) and np.array_equal(a.proj_val, b.proj_val)
    assert not np.array_equal(a.v_loc, c.v_loc)


def test_column_subset_and_energy_grid(junction):
    cols = P.column_subset(junction, 256, seed=8)
    assert cols.size == 256 and np.all(np.diff(cols) > 0)
    assert np.all(np.isin(cols, junction.right_columns()))
    assert np.array_equal(cols, P.column_subset(junction, 256, seed=8))
    assert np.array_equal(P.column_subset(junction, 10**6, seed=1), junction.right_columns())
    E = P.energy_grid(0.16, 0.24, 128)
    assert E.size == 128 and E[0] == 0.16 and E[-1] == 0.24


def test_batched_junction_size_draws():
    js = P.batched_junctions(n=4)
    for k, j in enumerate(js):
        rng = np.random.default_rng(1000 + k)
        nxy, nz, cap, wells = (int(rng.integers(12, 33)), int(rng.integers(64, 193)),
                               int(rng.integers(6, 11)), int(rng.integers(5, 31)))
        assert (j.nx, j.ny, j.nz, j.n_cap) == (nxy, nxy, nz, cap)
        assert j.n_proj == 4 * wells and j.fd_half_order == 4
        assert j.name.startswith(f"batched_{k}_")


def test_batch_wrapper_checks_list_lengths():
    from paper_1401_0782_gb300 import binding as B
    with pytest.raises(ValueError):
        B.batch_transmission([], [[0.2]], None)
