"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances: FP64 mode -- columns ||dx||/||x|| <= 1e-9 and T relative 1e-9
(|dT| <= 1e-9 max(|T|, 1e-3) on the waveguide staircase); mixed mode (FP32
Krylov + FP64 refinement to relative residual 1e-10, goal-oriented finish) --
T relative 1e-6 (|dT| <= 1e-6 on the waveguide).  The operator itself is checked element-wise:
FP64 to 1e-12 relative (rounding order only), FP32 to 2e-6 relative.
"""
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


def _rand_x(rng, n, N, dtype):
    x = rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N))
    return torch.tensor(x, dtype=dtype, device="cuda")


JUNCTIONS = {
    "waveguide_R1": lambda: P.waveguide(nx=8, ny=8, nz=48),
    "junction_R4": lambda: P.molecular_junction(seed=3, nx=12, ny=12, nz=40, n_wells=4, n_cap=5),
    "ragged_R3": lambda: P.molecular_junction(seed=5, nx=13, ny=11, nz=37, fd_half_order=3, n_wells=3, n_cap=4),
    "spd_R6": lambda: P.molecular_junction(seed=4, nx=12, ny=12, nz=40, fd_half_order=6, n_wells=3, lmax=2,
                                           n_cap=6, h=0.3),
    "wide_R2": lambda: P.molecular_junction(seed=6, nx=40, ny=36, nz=20, fd_half_order=2, n_wells=2, n_cap=3),
    # the benchmark's cross-section (plane streaming above 48 KiB of shared memory)
    "bench_plane_R4": lambda: P.molecular_junction(seed=7, nx=24, ny=24, nz=30, n_wells=3, n_cap=4),
    "r5": lambda: P.molecular_junction(seed=9, nx=14, ny=14, nz=36, fd_half_order=5, n_wells=3, n_cap=4),
    # one-CTA-per-SM point-pair variant (planes of more than 576 points)
    "big_plane_R4": lambda: P.molecular_junction(seed=10, nx=32, ny=30, nz=24, n_wells=3, n_cap=4),
}


@pytest.mark.parametrize("name", sorted(JUNCTIONS))
@pytest.mark.parametrize("tiling", [(0, 0, 0), (5, 7, 2), (3, 9, 1), (0, 11, -1), (0, 13, -2), (0, 17, -3)])
def test_apply_matches_oracle_operator(B, name, tiling):
    j = JUNCTIONS[name]()
    ctx = B.Context(0).set_junction(j)
    ctx.set_tiling(*tiling)
    rng = np.random.default_rng(1)
    E = np.array([0.2, -0.7, 1.3])
    x64 = _rand_x(rng, E.size, j.N, torch.complex128)
    y64 = ctx.apply(E, x64, B.RSN_FP64).cpu().numpy()
    xh = x64.cpu().numpy()
    ref = np.stack([O.apply_operator(j, e, xh[k]) for k, e in enumerate(E)])
    scale = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= 1e-12 * scale
    x32 = x64.to(torch.complex64)
    y32 = ctx.apply(E, x32, B.RSN_MIXED).cpu().numpy()
    ref32 = np.stack([O.apply_operator(j, e, x32[k].cpu().numpy().astype(np.complex128)) for k, e in enumerate(E)])
    assert np.abs(y32 - ref32).max() <= 2e-6 * scale
    ctx.close()


@pytest.mark.parametrize("fn", ["rsn_apply", "rsn_apply_noalloc"])
@pytest.mark.parametrize("tiling", [(0, 0, 0), (0, 11, -1), (0, 13, -2), (0, 17, -3)])
def test_apply_with_unaligned_vectors(B, fn, tiling):
    # vectors 8 bytes off a 16-byte boundary cannot be bulk-copied: the apply
    # entry points fall back to a register tiling that fits the CTA limits
    j = JUNCTIONS["bench_plane_R4"]()
    ctx = B.Context(0).set_junction(j)
    ctx.set_tiling(*tiling)
    rng = np.random.default_rng(2)
    E = np.array([0.2, 0.4])
    xr = rng.standard_normal((E.size, j.N)) + 1j * rng.standard_normal((E.size, j.N))
    xb = torch.zeros(E.size * j.N + 1, dtype=torch.complex64, device="cuda")
    yb = torch.zeros_like(xb)
    x = xb[1:]
    x.copy_(torch.tensor(xr.ravel(), dtype=torch.complex64))
    y = yb[1:]
    assert x.data_ptr() % 16 == 8 and y.data_ptr() % 16 == 8
    if fn == "rsn_apply_noalloc":
        ctx.apply(E, torch.zeros((E.size, j.N), dtype=torch.complex64, device="cuda"), B.RSN_MIXED)  # upload
    rc = getattr(ctx.lib, fn)(ctx.h, B.RSN_MIXED, int(E.size), E.ctypes.data, x.data_ptr(), y.data_ptr())
    assert rc == B.RSN_OK, ctx.lib.rsn_last_error(ctx.h).decode()
    torch.cuda.synchronize()
    yh = y.cpu().numpy().reshape(E.size, j.N)
    xh = x.cpu().numpy().reshape(E.size, j.N).astype(np.complex128)
    ref = np.stack([O.apply_operator(j, e, xh[k]) for k, e in enumerate(E)])
    assert np.abs(yh - ref).max() <= 2e-6 * np.abs(ref).max()
    ctx.close()


def test_solve_columns_fp64_matches_lu(B):
    j = JUNCTIONS["junction_R4"]()
    E = [0.17, 0.23]
    cols = j.right_columns()[::37]
    ctx = B.Context(0).set_junction(j)
    x, iters, relres = ctx.solve_columns(E, cols, B.default_opts(B.RSN_FP64))
    x = x.cpu().numpy()
    for e, En in enumerate(E):
        ref = O.solve_columns(j, En, cols).T
        err = np.linalg.norm(x[e] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 1e-9, err.max()
    assert np.all(iters > 0) and np.all(relres <= 1e-13)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_columns_with_hundreds_of_tiles(B, prec):
    # one y row and one z plane per CTA: 12 x 40 = 480 operator tiles, so the
    # partial sums of mu and ||b||^2 span more entries than one CTA has threads
    j = JUNCTIONS["junction_R4"]()
    E = [0.21]
    cols = j.right_columns()[::29]
    ctx = B.Context(0).set_junction(j)
    ctx.set_tiling(1, 1, 1)
    x, iters, relres = ctx.solve_columns(E, cols, B.default_opts(B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED))
    ref = O.solve_columns(j, E[0], cols).T
    err = np.linalg.norm(x[0].cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= (1e-9 if prec == "fp64" else 1e-6), err.max()
    ctx.close()


def test_solve_columns_mixed_residual_and_ragged_tiles(B):
    j = JUNCTIONS["ragged_R3"]()
    E = [0.05, 0.31]
    cols = j.right_columns()[::11]
    ctx = B.Context(0).set_junction(j)
    ctx.set_tiling(4, 6, 2)
    x, iters, relres = ctx.solve_columns(E, cols, B.default_opts(B.RSN_MIXED))
    x = x.cpu().numpy()
    for e, En in enumerate(E):
        b = np.zeros((j.N, cols.size), complex)
        b[cols, np.arange(cols.size)] = 1
        r = b - O.apply_operator(j, En, x[e].T)
        assert (np.linalg.norm(r, axis=0) <= 1.5e-10).all()
        ref = O.solve_columns(j, En, cols).T
        err = np.linalg.norm(x[e] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 1e-6
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_waveguide_transmission_and_staircase(B, prec):
    w = P.waveguide()
    E = P.energy_grid(0.05, 2.0, 64)[::4]
    ctx = B.Context(0).set_junction(w)
    p = B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED
    T = ctx.transmission(E, None, B.default_opts(p))
    T_ref = O.transmission(w, E)
    if prec == "fp64":
        assert np.all(np.abs(T - T_ref) <= 1e-9 * np.maximum(np.abs(T_ref), 1e-3))
    else:
        assert np.all(np.abs(T - T_ref) <= 1e-6)
    th = O.channel_thresholds(8, 8, 0.5)
    for e, t in zip(E, T):
        below = th[th < e]
        if (below.size and e - below.max() >= 0.18) or (not below.size and th.min() - e >= 0.06):
            assert abs(t - O.open_channels(8, 8, 0.5, e)) <= 0.06
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vjp_matches_oracle_gradient(B, prec):
    j = JUNCTIONS["junction_R4"]()
    E = [0.16, 0.2, 0.24]
    Tb = [1.0, -0.5, 2.0]
    cols = j.right_columns()[::13]
    ctx = B.Context(0).set_junction(j)
    p = B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED
    T, g = ctx.transmission_vjp(E, Tb, cols, B.default_opts(p))
    T_ref, g_ref = O.transmission_grad(j, E, cols, T_bar=Tb)
    gs = np.abs(g_ref).max()
    # T ~ 1e-11 here (closed lead channels): relative bounds, which the
    # goal-oriented finish of the columns meets
    if prec == "fp64":
        assert np.all(np.abs(T - T_ref) <= 1e-9 * np.abs(T_ref)), np.abs(T - T_ref) / np.abs(T_ref)
        assert np.abs(g - g_ref).max() <= 1e-8 * gs
    else:
        assert np.all(np.abs(T - T_ref) <= 1e-6 * np.abs(T_ref)), np.abs(T - T_ref) / np.abs(T_ref)
        assert np.abs(g - g_ref).max() <= 1e-5 * gs
    ctx.close()


@pytest.mark.parametrize("tiling", [(0, 0, 0), (0, 13, -2), (0, 17, -3), (0, 11, -1), (4, 6, 2), "autotune"])
def test_mixed_solves_under_every_operator_kernel(B, tiling):
    # the COCG operator of the mixed solver: automatic (point-pair), point-pair,
    # plane kernel, whole-plane bulk-copy with a shifted queue, register kernel,
    # the autotuner's pick
    j = JUNCTIONS["junction_R4"]()
    E = [0.19]
    cols = j.right_columns()[::53]
    ctx = B.Context(0).set_junction(j)
    if tiling == "autotune":
        pick = ctx.autotune(B.RSN_MIXED, 64)
        assert pick["gbs"] > 0 and pick["tma"] in (0, 1, 2, 3)
    else:
        ctx.set_tiling(*tiling)
    x, iters, relres = ctx.solve_columns(E, cols, B.default_opts(B.RSN_MIXED))
    ref = O.solve_columns(j, E[0], cols).T
    err = np.linalg.norm(x[0].cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-6 and relres.max() <= 1e-10, (err.max(), relres.max())
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_open_channel_junction_relative_transmission(B, prec):
    # above the leads' first transverse levels T = O(1): the relative bound is
    # the whole story (FP64 1e-9, mixed 1e-6)
    j = JUNCTIONS["junction_R4"]()
    E = [1.5, 1.8, 2.1]
    cols = j.right_columns()[::11]
    ctx = B.Context(0).set_junction(j)
    T = ctx.transmission(E, cols, B.default_opts(B.RSN_FP64 if prec == "fp64" else B.RSN_MIXED))
    T_ref = O.transmission(j, E, cols)
    assert T_ref.min() > 1e-3, T_ref  # channels are open at these energies
    rel = 1e-9 if prec == "fp64" else 1e-6
    assert np.all(np.abs(T - T_ref) <= rel * np.abs(T_ref)), np.abs(T - T_ref) / np.abs(T_ref)
    ctx.close()


def test_fp64_is_bit_reproducible(B):
    j = JUNCTIONS["junction_R4"]()
    cols = j.right_columns()[::29]
    ctx = B.Context(0).set_junction(j)
    T1 = ctx.transmission([0.2, 0.21], cols, B.default_opts(B.RSN_FP64))
    T2 = ctx.transmission([0.2, 0.21], cols, B.default_opts(B.RSN_FP64))
    assert np.array_equal(T1, T2)
    ctx.close()
