"""Pins for the CPU oracle (no GPU).  Each check ties the oracle to something
other than itself: a published table, polynomial exactness, closed-form
eigenvalues, exact lead self-energies, the eigen-route identity of Sec. II.C,
dense inversion, invariants of Eq. complex-sym, finite differences and dense
autograd.  A few tests plant a mistake in a copy of the oracle's arithmetic
and check that the pin catches it."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1401_0782_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# finite-difference weights
# ---------------------------------------------------------------------------

def _golden_fd():
    out = {}
    with open(os.path.join(GOLDEN, "fd_coefficients.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            out[int(tok[0])] = [Fraction(t) for t in tok[1:]]
    return out


def test_fd_coefficients_match_published_table():
    gold = _golden_fd()
    assert sorted(gold) == [1, 2, 3, 4, 5, 6]
    for R, ref in gold.items():
        assert O.fd_coefficients(R) == ref


@pytest.mark.parametrize("R", [1, 2, 3, 4, 5, 6])
def test_fd_weights_exact_on_even_polynomials(R):
    # f(x) = x^(2m): f''(0) = 2 for m = 1, 0 otherwise; exact for 2m <= 2R,
    # and the first inexact moment (m = R+1) must not vanish (order exactly 2R).
    c = O.fd_coefficients(R)
    for m in range(0, R + 2):
        val = (c[0] if m == 0 else 0) + sum(c[k] * 2 * Fraction(k) ** (2 * m) for k in range(1, R + 1))
        want = 2 if m == 1 else 0
        if m <= R:
            assert val == want, (R, m, val)
        else:
            assert val != 0


def test_laplacian_second_order_sine_modes():
    # Dirichlet sine modes are exact eigenvectors of the 2nd-order stencil.
    nx, ny, nz, h = 5, 4, 7, 0.4
    lap = O.laplacian(nx, ny, nz, h, 1)
    x = np.arange(1, nx + 1)
    y = np.arange(1, ny + 1)
    z = np.arange(1, nz + 1)
    for (a, b, c) in [(1, 1, 1), (2, 3, 5), (5, 4, 7)]:
        f = np.einsum("k,j,i->kji", np.sin(c * np.pi * z / (nz + 1)),
                      np.sin(b * np.pi * y / (ny + 1)), np.sin(a * np.pi * x / (nx + 1))).ravel()
        lam = -sum((2 - 2 * np.cos(m * np.pi / (n + 1))) / h**2 for m, n in ((a, nx), (b, ny), (c, nz)))
        np.testing.assert_allclose(lap @ f, lam * f, atol=1e-11 * abs(lam))


@pytest.mark.parametrize("R", [4, 6])
def test_laplacian_high_order_anisotropic_gaussian(R):
    # An anisotropic Gaussian (different widths per axis) catches a transposed
    # grid ordering; the error at interior points shrinks like h^(2R).
    errs = []
    ax, ay, az = 1.0 / 1.5**2, 1.0 / 1.2**2, 1.0 / 1.0**2  # fixed widths (bohr)
    for h, (nx, ny, nz) in ((0.3, (30, 34, 38)), (0.15, (60, 68, 76))):
        cx, cy, cz = (nx - 1) * h / 2, (ny - 1) * h / 2, (nz - 1) * h / 2
        Z, Y, X = np.meshgrid(np.arange(nz) * h - cz, np.arange(ny) * h - cy, np.arange(nx) * h - cx, indexing="ij")
        f = np.exp(-ax * X**2 - ay * Y**2 - az * Z**2)
        exact = f * ((4 * ax**2 * X**2 - 2 * ax) + (4 * ay**2 * Y**2 - 2 * ay) + (4 * az**2 * Z**2 - 2 * az))
        lap = O.laplacian(nx, ny, nz, h, R)
        got = (lap @ f.ravel()).reshape(f.shape)
        inner = (np.abs(X) < 2.0) & (np.abs(Y) < 2.0) & (np.abs(Z) < 2.0)  # away from the walls
        errs.append(np.abs(got - exact)[inner].max() / np.abs(exact).max())
    assert errs[0] < 1e-3
    assert errs[1] < errs[0] / 2 ** (2 * R - 3)


# ---------------------------------------------------------------------------
# projectors / Hamiltonian
# ---------------------------------------------------------------------------

def test_projectors_unit_norm_and_kb_spectrum():
    # Atom centred on a grid point: s, px, py, pz are mutually orthogonal by
    # symmetry, so the nonzero eigenvalues of H_nl are exactly the E_KB values.
    nx = ny = nz = 15
    h = 0.35
    c = np.array([[7 * h, 7 * h, 7 * h]])
    ekb = np.array([[0.7, -0.4]])
    off, idx, val, e = P._kb_projectors(nx, ny, nz, h, c, 1, 1.5, ekb)
    for p in range(len(e)):
        assert abs(np.sum(val[off[p]:off[p + 1]] ** 2) - 1.0) < 1e-12
    j = P.Junction(nx, ny, nz, h, 1, np.zeros(nx * ny * nz), np.zeros(nx * ny * nz),
                   np.zeros(nx * ny * nz), off, idx, val, e)
    Hnl = O.hamiltonian(j) - O.local_hamiltonian(j)
    sup = np.unique(idx)
    w = np.linalg.eigvalsh(Hnl[sup][:, sup].toarray())
    w = np.sort(w[np.abs(w) > 1e-10])
    np.testing.assert_allclose(w, np.sort([0.7, -0.4, -0.4, -0.4]), atol=1e-12)
    assert abs(Hnl - Hnl.T).max() < 1e-15


def test_bordered_system_equals_explicit_inverse():
    j = P.tiny_junction()
    E = 0.37
    A = O.system_matrix(j, E).toarray()
    cols = j.right_columns()[::5]
    X = O.solve_columns(j, E, cols)
    G = np.linalg.inv(A)
    np.testing.assert_allclose(X, G[:, cols], rtol=0, atol=1e-11 * np.abs(G).max())
    y = O.apply_operator(j, E, X)
    assert np.abs(y[cols, np.arange(cols.size)] - 1).max() < 1e-11


# ---------------------------------------------------------------------------
# transmission: closed forms and identities
# ---------------------------------------------------------------------------

def test_channel_thresholds_closed_form_vs_dense_eigenvalues():
    nx, ny, h = 8, 8, 0.5
    def d2(n):
        return (np.diag(np.full(n, -2.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h**2
    Hxy = -0.5 * (np.kron(np.eye(ny), d2(nx)) + np.kron(d2(ny), np.eye(nx)))
    np.testing.assert_allclose(O.channel_thresholds(nx, ny, h), np.linalg.eigvalsh(Hxy), atol=1e-12)
    # thresholds inside [0.05, 2] Ha for the 8x8, h = 0.5 guide: 1, 2 and 1 new modes
    th = O.channel_thresholds(nx, ny, h)
    assert np.sum(th < 2.0) == 4 and abs(th[0] - 0.48245903) < 1e-7


@pytest.mark.parametrize("E", [0.3, 0.8, 1.5, 1.95])
def test_exact_lead_self_energy_gives_integer_channels(E):
    T = O.lead_self_energy_T(8, 8, 5, 0.5, E)
    assert abs(T - O.open_channels(8, 8, 0.5, E)) < 1e-9


def staircase_checkable(E, th):
    """Energies where a 16-plane quadratic CAP is nearly reflectionless: the
    slowest open channel carries >= 0.18 Ha of longitudinal kinetic energy, or
    no channel is open and the first threshold is >= 0.06 Ha away."""
    below = th[th < E]
    if below.size == 0:
        return th.min() - E >= 0.06
    return E - below.max() >= 0.18


def test_waveguide_cap_staircase():
    # CAP version (factor 4 coupling) against the open-channel count.  Slow
    # channels near a threshold are partly reflected by the CAP, so only
    # energies where every open channel is fast enough are compared.
    w = P.waveguide()
    E_all = P.energy_grid(0.05, 2.0, 64)
    th = O.channel_thresholds(8, 8, 0.5)
    E = np.array([e for e in E_all[::3] if staircase_checkable(e, th)])
    assert E.size >= 12
    T = O.transmission(w, E)
    N_open = np.array([O.open_channels(8, 8, 0.5, e) for e in E])
    assert np.all(np.abs(T - N_open) <= 0.06), np.c_[E, T, N_open]
    assert set(N_open) == {0, 1, 3}
    assert np.all(T >= -1e-12) and np.all(T <= N_open + 0.06)


def test_waveguide_staircase_catches_missing_factor_4():
    # planted mistake: the bare Eq. T-realspace without the coupling factor 4
    w = P.waveguide()
    X = O.solve_columns(w, 1.5, w.right_columns())
    T_wrong = np.sum(w.gamma_r[w.right_columns()] * O.column_weights(w, X))
    assert abs(T_wrong - 3) > 1.0


def test_sparse_columns_match_dense_trace_formula():
    # Eq. T (dense trace with coupling 2*CAP) == Eq. T-realspace (columns).
    j = P.tiny_junction()
    for E in (-0.2, 0.37, 1.1):
        G = np.linalg.inv(O.system_matrix(j, E).toarray())
        T_trace = O.transmission_trace(G, 2 * j.gamma_l, 2 * j.gamma_r)
        T_cols = O.transmission(j, [E])[0]
        assert abs(T_cols - T_trace) <= 1e-11 * max(1.0, abs(T_trace))


def test_eigen_route_identity():
    # Eq. T-tilde-realsp with all eigenpairs (U^T U = 1) reproduces T.
    j = P.tiny_junction(fd_half_order=3)
    E = np.array([-0.3, 0.2, 0.9])
    np.testing.assert_allclose(O.transmission_eigen(j, E), O.transmission(j, E), rtol=1e-8, atol=1e-12)


def test_invariants_symmetry_lr_and_retarded_sign():
    j = P.tiny_junction(seed=11)
    E = 0.45
    A = O.system_matrix(j, E).toarray()
    G = np.linalg.inv(A)
    assert np.abs(G - G.T).max() < 1e-12 * np.abs(G).max()  # Eq. complex-sym
    X = O.solve_columns(j, E, np.arange(j.N))
    assert np.all(np.diag(X).imag < 0)  # retarded: Im G_jj = -pi LDOS < 0
    jr = P.Junction(**{**j.__dict__, "gamma_l": j.gamma_r, "gamma_r": j.gamma_l})
    assert abs(O.transmission(j, [E])[0] - O.transmission(jr, [E])[0]) < 1e-12
    cols = j.right_columns()
    perm = np.random.default_rng(0).permutation(cols)
    assert abs(O.transmission(j, [E], cols)[0] - O.transmission(j, [E], perm)[0]) < 1e-12


def test_krylov_route_matches_lu():
    j = P.molecular_junction(nx=10, ny=10, nz=30, n_wells=3, n_cap=4)
    cols = j.right_columns()[[0, 57, 233]]
    X_lu = O.solve_columns(j, 0.2, cols, method="lu")
    X_kr = O.solve_columns(j, 0.2, cols, method="krylov", rtol=1e-13)
    assert np.linalg.norm(X_kr - X_lu) <= 1e-8 * np.linalg.norm(X_lu)


# ---------------------------------------------------------------------------
# gradient dT/dV_loc
# ---------------------------------------------------------------------------

def test_gradient_central_differences_and_sum_rule():
    j = P.tiny_junction(seed=3)
    E = [0.41]
    T, g = O.transmission_grad(j, E)
    rng = np.random.default_rng(5)
    pts = rng.choice(j.N, 12, replace=False)
    dv = 1e-4
    for r in pts:
        vp = j.v_loc.copy(); vp[r] += dv
        vm = j.v_loc.copy(); vm[r] -= dv
        fd = (O.transmission(j.with_potential(vp), E)[0] - O.transmission(j.with_potential(vm), E)[0]) / (2 * dv)
        assert abs(fd - g[r]) <= 1e-6 * max(1.0, np.abs(g).max())
    # uniform V shift == energy shift: sum_r dT/dV_r = -dT/dE
    de = 1e-5
    dTdE = (O.transmission(j, [E[0] + de])[0] - O.transmission(j, [E[0] - de])[0]) / (2 * de)
    assert abs(np.sum(g) + dTdE) <= 1e-6 * max(1.0, abs(dTdE))


def test_gradient_matches_dense_autograd():
    torch = pytest.importorskip("torch")
    j = P.tiny_junction(seed=9, lmax=0)
    E = 0.3
    T_bar = [1.7]
    T, g = O.transmission_grad(j, [E], T_bar=T_bar)
    H0 = O.hamiltonian(j).toarray() - np.diag(j.v_loc)
    V = torch.tensor(j.v_loc, dtype=torch.float64, requires_grad=True)
    A = (E * torch.eye(j.N, dtype=torch.complex128) - torch.tensor(H0, dtype=torch.complex128)
         - torch.diag(V.to(torch.complex128))
         + 1j * torch.diag(torch.tensor(j.gamma_l + j.gamma_r, dtype=torch.complex128)))
    G = torch.linalg.inv(A)
    gl = torch.tensor(j.gamma_l, dtype=torch.float64)
    gr = torch.tensor(j.gamma_r, dtype=torch.float64)
    Tt = 4.0 * torch.sum(gl[:, None] * gr[None, :] * G.abs() ** 2)
    (T_bar[0] * Tt).backward()
    assert abs(Tt.item() - T[0]) < 1e-12
    np.testing.assert_allclose(g, V.grad.numpy(), rtol=1e-8, atol=1e-12 * np.abs(g).max())


def test_gradient_pin_catches_wrong_adjoint_weight():
    # planted mistake: the conjugate of lambda instead of lambda breaks FD agreement
    j = P.tiny_junction(seed=3)
    E = 0.41
    cols = j.right_columns()
    X, s = O.solve_columns(j, E, cols, return_lu=True)
    Lam = s.solve(j.gamma_l[:, None] * np.conj(X))
    g_wrong = 8.0 * np.sum(j.gamma_r[cols][None, :] * np.real(np.conj(Lam) * X), axis=1)
    _, g = O.transmission_grad(j, [E])
    assert np.abs(g_wrong - g).max() > 1e-3 * np.abs(g).max()


# ----------------------------------------------------------------------------
# shifted COCG over an energy window (A(E) is a shift family, Eq. G)
# ----------------------------------------------------------------------------

def _shift_junction():
    return P.molecular_junction(seed=12, nx=10, ny=10, nz=30, n_wells=3, n_cap=4)


def test_shifted_cocg_matches_lu_at_every_energy():
    j = _shift_junction()
    E = np.linspace(0.15, 0.35, 5)
    col = int(j.right_columns()[17])
    b = np.zeros(j.N, complex)
    b[col] = 1.0
    for seed in (0, 2):
        X, iters, _, _ = O.shifted_cocg(j, E, b, seed=seed, rtol=1e-12)
        assert 0 < iters < 5000
        for e, En in enumerate(E):
            ref = O.solve_columns(j, En, [col])[:, 0]
            assert np.linalg.norm(X[e] - ref) <= 1e-9 * np.linalg.norm(ref), (seed, En)
            # the true residual at each energy, with the oracle's own operator
            res = np.linalg.norm(b - O.apply_operator(j, En, X[e]))
            assert res <= 1e-11, (seed, En, res)


def test_shifted_cocg_residuals_stay_collinear():
    # mid-iteration, each energy's true residual is the seed residual over pi
    j = _shift_junction()
    E = np.array([0.2, 0.12, 0.31])
    b = np.zeros(j.N, complex)
    b[int(j.right_columns()[5])] = 1.0
    X, iters, pi, r = O.shifted_cocg(j, E, b, seed=0, stop_at=25)
    assert iters == 25 and pi[0] == 1.0
    for e, En in enumerate(E):
        true_r = b - O.apply_operator(j, En, X[e])
        assert np.linalg.norm(true_r - r / pi[e]) <= 1e-9 * np.linalg.norm(true_r), En
    # the seed itself is plain COCG: 25 steps of the oracle's own recurrence
    x = np.zeros(j.N, complex)
    rr = b.copy()
    p = rr.copy()
    rho = rr @ rr
    for _ in range(25):
        q = O.apply_operator(j, 0.2, p)
        a = rho / (p @ q)
        x += a * p
        rr -= a * q
        rho_new = rr @ rr
        p = rr + (rho_new / rho) * p
        rho = rho_new
    assert np.linalg.norm(X[0] - x) <= 1e-12 * np.linalg.norm(x)


def test_shifted_cocg_pin_catches_a_wrong_shift_sign():
    # a plausible mistake: shifting by E_s - E instead of E - E_s.  Solving at the
    # energies mirrored about the seed reproduces it, and the LU pin rejects it.
    j = _shift_junction()
    E = np.array([0.2, 0.26])
    col = int(j.right_columns()[3])
    b = np.zeros(j.N, complex)
    b[col] = 1.0
    mirrored = 2 * E[0] - E
    X, _, _, _ = O.shifted_cocg(j, mirrored, b, seed=0, rtol=1e-12)
    ref = O.solve_columns(j, E[1], [col])[:, 0]
    assert np.linalg.norm(X[1] - ref) > 1e-3 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------
# Landauer current (Eq. Landauer)
# ----------------------------------------------------------------------------
def test_landauer_constant_transmission_gives_ohmic_current():
    # int (f_L - f_R) dE = mu_L - mu_R = V at any temperature: I = T V / pi.
    # kT > 0 on a fine grid; kT = 0 with the chemical potentials at cell
    # centres, where the trapezoidal rule integrates the step exactly
    E = np.linspace(-2.0, 2.0, 40001)
    V = np.array([-0.3, 0.05, 0.2, 0.5])
    I = O.landauer_current(E, np.full(E.size, 0.7), V, E_F=0.1, kT=0.01)
    assert np.allclose(I, 0.7 * V / np.pi, rtol=1e-6, atol=1e-12)
    E0 = np.arange(-20000, 20001) * 1e-4 + 0.5e-4
    I0 = O.landauer_current(E0, np.full(E0.size, 0.7), V, E_F=0.1, kT=0.0)
    assert np.allclose(I0, 0.7 * V / np.pi, rtol=1e-9, atol=1e-12)


def test_landauer_staircase_is_piecewise_linear_and_odd():
    # T(E) = number of open channels of the waveguide: at kT = 0 the current
    # is (1/pi) int_{mu_R}^{mu_L} N(E) dE, the area under the staircase
    th = O.channel_thresholds(8, 8, 0.5)
    E = np.linspace(0.0, 2.5, 250001)
    N = np.array([O.open_channels(8, 8, 0.5, e) for e in E[::50]], dtype=float)
    N = np.repeat(N, 50)[: E.size]
    E_F, V = 1.2, np.array([0.2, 0.6, 1.0])
    I = O.landauer_current(E, N, V, E_F=E_F)
    for v, i in zip(V, I):
        lo, hi = E_F - v / 2, E_F + v / 2
        area = sum(max(0.0, min(hi, t + 4.0) - max(lo, t)) for t in th)  # channel t open on (t, t + 2/h^2)
        assert abs(i - area / np.pi) <= 2e-3 * area / np.pi
    assert np.allclose(O.landauer_current(E, N, -V, E_F=E_F), -I)


def test_landauer_linear_response_is_the_transmission_at_the_fermi_level():
    # dI/dV at V = 0: (1/pi) int T(E) (-f'(E - E_F)) dE = T(E_F) / pi + O(kT^2 T'')
    # (the Landauer conductance 2e^2/h T); kT = 0.002 Ha, 200 grid cells per kT
    E = np.linspace(-1.0, 1.0, 200001)
    T = 0.3 + 0.2 * np.sin(3 * E)
    dv = 1e-4
    g = (O.landauer_current(E, T, [dv], E_F=0.2, kT=0.002) -
         O.landauer_current(E, T, [-dv], E_F=0.2, kT=0.002))[0] / (2 * dv)
    assert abs(g - (0.3 + 0.2 * np.sin(0.6)) / np.pi) <= 1e-5


def test_landauer_catches_a_missing_spin_factor():
    # a current without the factor 2 of 2e/h is half the ohmic value
    E = np.linspace(-2.0, 2.0, 4001)
    I = O.landauer_current(E, np.ones(E.size), [0.4])[0]
    assert abs(I - 0.4 / np.pi) < 1e-9 and abs(0.5 * I - 0.4 / np.pi) > 0.1 * 0.4 / np.pi
