"""CPU oracle for real-space NEGF transmission with absorbing boundaries.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this module.  The product
path (the C-ABI library and its Python binding) never calls it and shares no
code with it: the two meet only through the seeded inputs of
``paper_1401_0782_gb300.problems``, which hold none of the method's arithmetic.

Everything here is plain complex128 / float64 NumPy-SciPy, chosen to be
checked by eye against the paper:

* ``fd_coefficients``      -- central second-derivative weights (closed form).
* ``hamiltonian``          -- H_KS = -1/2 lap_FD + V_loc + sum_p |beta_p> E_KB <beta_p|
                              (Sec. II.C: FD Laplacian, local potential and
                              cutoff-limited nonlocal part are the only entries).
* ``system_matrix``        -- (G^r)^{-1} = E 1 - H_KS + i Gamma  (Eqs. G and Hop,
                              the CAP taking the place of i*eta).
* ``solve_columns``        -- x_j = G^r e_j by SuperLU (one factorisation per E)
                              of the system with the projector term kept factored
                              through auxiliary unknowns (``bordered_system``); at
                              ~10^5 points, where a 3-D LU takes minutes, by a plain
                              NumPy conjugate-orthogonal CG with every column's true
                              residual certified.
* ``transmission``         -- Eq. T-realspace with the CAP as coupling:
                              T = 4 sum_{i in L, j in R} Gamma_L,i Gamma_R,j |G_ij|^2
                              (factor 4: the coupling is Gamma_std = 2*CAP).
* ``shifted_cocg``         -- columns at every energy of a window from one Krylov
                              space (A(E) is a shift family, Eq. G): COCG on a seed
                              energy plus the collinear shifted recurrences.
* ``transmission_grad``    -- dT/dV_loc by the adjoint identity
                              dG/dV_r = G e_r e_r^T G (G = G^T, Eq. complex-sym).
* ``transmission_trace``   -- Eq. T written as a dense trace, Tr{G Gam_R G^dag Gam_L}.
* ``transmission_eigen``   -- Eq. T-tilde-realsp from a full complex-orthogonal
                              eigenbasis (Sec. II.C), tiny grids only.
* ``landauer_current``     -- Eq. Landauer, I = (2e/h) int T (f_L - f_R) dE, by the
                              trapezoidal rule on the given energy grid.
* ``open_channels``        -- closed-form channel count of a hard-wall waveguide.
* ``lead_self_energy_T``   -- exact semi-infinite-lead self-energies for the
                              same waveguide (textbook NEGF), dense.

Parity status: every function is pinned by tests in ``tests/test_oracle.py``
against mathematics that does not route through itself (closed forms, exact
lead self-energies, polynomial exactness, eigen-route identity, finite
differences, dense autograd); none is "parity unpinned".
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "fd_coefficients",
    "laplacian",
    "hamiltonian",
    "system_matrix",
    "solve_columns",
    "transmission",
    "column_weights",
    "transmission_grad",
    "shifted_cocg",
    "transmission_trace",
    "transmission_eigen",
    "open_channels",
    "channel_thresholds",
    "landauer_current",
    "lead_self_energy_T",
    "apply_operator",
    "local_hamiltonian",
    "bordered_system",
]


# ----------------------------------------------------------------------------
# finite-difference Laplacian
# ----------------------------------------------------------------------------

def fd_coefficients(R: int) -> List[Fraction]:
    """Weights c_0..c_R of the order-2R central second derivative (h = 1).

    f''(0) ~ c_0 f(0) + sum_{k=1..R} c_k (f(k) + f(-k)), with the closed form
    c_k = 2 (-1)^{k+1} (R!)^2 / (k^2 (R-k)! (R+k)!)  and  c_0 = -2 sum c_k.
    """
    if not 1 <= R <= 12:
        raise ValueError("R out of range")
    c = [Fraction(0)] * (R + 1)
    for k in range(1, R + 1):
        c[k] = Fraction(2 * (-1) ** (k + 1) * math.factorial(R) ** 2,
                        k * k * math.factorial(R - k) * math.factorial(R + k))
    c[0] = -2 * sum(c[1:])
    return c


def _second_derivative_1d(n: int, h: float, R: int) -> sp.csr_matrix:
    """n x n matrix of d^2/dx^2 with zero (Dirichlet) values outside 0..n-1."""
    c = [float(v) for v in fd_coefficients(R)]
    diags = [np.full(n, c[0])]
    offs = [0]
    for k in range(1, R + 1):
        if k < n:
            diags += [np.full(n - k, c[k]), np.full(n - k, c[k])]
            offs += [k, -k]
    return (sp.diags(diags, offs, shape=(n, n), format="csr") / (h * h)).tocsr()


def laplacian(nx: int, ny: int, nz: int, h: float, R: int) -> sp.csr_matrix:
    """3-D FD Laplacian on the tensor grid (x fastest) as the Kronecker sum
    lap = I_z (x) I_y (x) D_x + I_z (x) D_y (x) I_x + D_z (x) I_y (x) I_x."""
    Dx = _second_derivative_1d(nx, h, R)
    Dy = _second_derivative_1d(ny, h, R)
    Dz = _second_derivative_1d(nz, h, R)
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    lap = (sp.kron(Iz, sp.kron(Iy, Dx)) + sp.kron(Iz, sp.kron(Dy, Ix))
           + sp.kron(Dz, sp.kron(Iy, Ix)))
    return lap.tocsr()


def _projector_rows(j) -> sp.csr_matrix:
    """B with B[p, :] = v_p (the sqrt(h^3)-weighted projector values)."""
    rows = np.repeat(np.arange(j.n_proj), np.diff(j.proj_offsets))
    return sp.csr_matrix((j.proj_val, (rows, j.proj_idx)), shape=(j.n_proj, j.N))


def local_hamiltonian(j) -> sp.csr_matrix:
    """-1/2 lap_FD + diag(V_loc): the sparse (stencil + diagonal) part of H_KS."""
    H = -0.5 * laplacian(j.nx, j.ny, j.nz, j.h, j.fd_half_order) + sp.diags(j.v_loc)
    return H.tocsr()


def hamiltonian(j) -> sp.csr_matrix:
    """Real symmetric H_KS = -1/2 lap + diag(V_loc) + sum_p e_kb[p] v_p v_p^T.

    The nonlocal term fills every atom's sphere densely, so this explicit form
    is for small grids; the solvers below keep it factored.
    """
    H = local_hamiltonian(j)
    if j.n_proj:
        B = _projector_rows(j)
        H = H + B.T @ sp.diags(j.proj_ekb) @ B
    return H.tocsr()


def system_matrix(j, E: float, H: Optional[sp.csr_matrix] = None) -> sp.csc_matrix:
    """A(E) = E 1 - H_KS + i (Gamma_L + Gamma_R)  = (G^r)^{-1}  (Eqs. G, Hop).

    Explicit form (small grids)."""
    if H is None:
        H = hamiltonian(j)
    N = j.N
    A = E * sp.identity(N, dtype=np.complex128) - H.astype(np.complex128) \
        + 1j * sp.diags(j.gamma_l + j.gamma_r)
    return A.tocsc()


def local_system_matrix(j, E: float, Hloc=None) -> sp.csr_matrix:
    """E 1 - (-1/2 lap + V_loc) + i Gamma: A(E) without the projector term."""
    if Hloc is None:
        Hloc = local_hamiltonian(j)
    N = j.N
    return (E * sp.identity(N, dtype=np.complex128) - Hloc.astype(np.complex128)
            + 1j * sp.diags(j.gamma_l + j.gamma_r)).tocsr()


def bordered_system(j, E: float, Hloc=None) -> sp.csc_matrix:
    """A(E) with the projector term kept factored through auxiliary unknowns.

    With y_p = v_p . x the system A(E) x = b reads
        [ A_loc(E)   -B^T diag(e_kb) ] [x]   [b]
        [ B          -1              ] [y] = [0],
    whose first block row is A_loc x - B^T diag(e_kb) B x = A(E) x.
    """
    A_loc = local_system_matrix(j, E, Hloc)
    if j.n_proj == 0:
        return A_loc.tocsc()
    B = _projector_rows(j)
    return sp.bmat([[A_loc, -(B.T @ sp.diags(j.proj_ekb))],
                    [B, -sp.identity(j.n_proj)]]).tocsc()


def apply_operator(j, E: float, x: np.ndarray, Hloc=None) -> np.ndarray:
    """y = A(E) x = A_loc(E) x - B^T (e_kb o (B x)) for x of shape (N,) or (N, k)."""
    y = local_system_matrix(j, E, Hloc) @ x
    if j.n_proj:
        B = _projector_rows(j)
        Bx = B @ x
        y = y - B.T @ (j.proj_ekb.reshape((-1,) + (1,) * (np.ndim(x) - 1)) * Bx)
    return y


# ----------------------------------------------------------------------------
# Green's-function columns and transmission
# ----------------------------------------------------------------------------

class _Solver:
    """x = A(E)^{-1} b for the junction at one energy.

    ``method="lu"``: SuperLU factorisation of the bordered system (exact up to
    rounding).  ``method="krylov"``: conjugate-orthogonal CG (the CG recurrence
    with the unconjugated bilinear form u^T v, valid because A = A^T) in plain
    NumPy complex128, from zero, to relative residual ``rtol``; each solution
    is then certified by recomputing its true residual b - A x with the
    operator of this module, so the result does not rest on the recurrence.
    The Krylov route exists because a 3-D LU at ~10^5 points takes minutes and
    gigabytes.
    """

    def __init__(self, j, E, method="lu", rtol=1e-13, Hloc=None):
        self.j, self.E, self.method, self.rtol = j, float(E), method, rtol
        self.Hloc = local_hamiltonian(j) if Hloc is None else Hloc
        if method == "lu":
            self.lu = spla.splu(bordered_system(j, self.E, self.Hloc))
        elif method == "krylov":
            A_loc = local_system_matrix(j, self.E, self.Hloc)
            B = _projector_rows(j) if j.n_proj else None
            ekb = j.proj_ekb

            def mv(v):
                y = A_loc @ v
                if B is not None:
                    y = y - B.T @ (ekb * (B @ v))
                return y

            self.op = spla.LinearOperator((j.N, j.N), matvec=mv, dtype=np.complex128)
            self.mv = mv
        else:
            raise ValueError(method)

    def _cocg(self, b, maxiter=50000):
        bn = np.linalg.norm(b)
        x = np.zeros_like(b)
        if bn == 0.0:
            return x
        r = b.copy()
        p = r.copy()
        rho = r @ r
        for _ in range(maxiter):
            q = self.mv(p)
            alpha = rho / (p @ q)
            x += alpha * p
            r -= alpha * q
            if np.linalg.norm(r) <= 0.5 * self.rtol * bn:
                # confirm on the true residual before stopping
                r = b - self.mv(x)
                if np.linalg.norm(r) <= self.rtol * bn:
                    return x
            rho_new = r @ r
            p = r + (rho_new / rho) * p
            rho = rho_new
        return x

    def solve(self, Bmat: np.ndarray) -> np.ndarray:
        N = self.j.N
        squeeze = Bmat.ndim == 1
        Bm = Bmat[:, None] if squeeze else Bmat
        if self.method == "lu":
            nb = self.j.n_proj
            rhs = np.zeros((N + nb, Bm.shape[1]), dtype=np.complex128)
            rhs[:N] = Bm
            X = self.lu.solve(rhs)[:N]
        else:
            X = np.zeros((N, Bm.shape[1]), dtype=np.complex128)
            for c in range(Bm.shape[1]):
                b = Bm[:, c].astype(np.complex128)
                x = self._cocg(b)
                res = np.linalg.norm(self.mv(x) - b) / max(np.linalg.norm(b), 1e-300)
                if res > 10 * self.rtol:
                    raise RuntimeError(f"krylov oracle did not converge (true residual {res:.2e})")
                X[:, c] = x
        return X[:, 0] if squeeze else X


def solve_columns(j, E: float, cols: Sequence[int], H=None, return_lu=False,
                  method: str = "lu", rtol: float = 1e-13):
    """X[:, c] = G^r(E) e_{cols[c]}  (columns of Eq. G)."""
    solver = _Solver(j, E, method, rtol)
    cols = np.asarray(cols, dtype=np.int64)
    B = np.zeros((j.N, cols.size), dtype=np.complex128)
    B[cols, np.arange(cols.size)] = 1.0
    X = solver.solve(B)
    if return_lu:
        return X, solver
    return X


def column_weights(j, X: np.ndarray) -> np.ndarray:
    """t_c = sum_{i in L} Gamma_L,i |X_ic|^2 for each solved column c."""
    return (j.gamma_l[:, None] * (X.real**2 + X.imag**2)).sum(axis=0)


def transmission(j, energies: Iterable[float], cols: Optional[Sequence[int]] = None,
                 method: str = "lu") -> np.ndarray:
    """T(E) = 4 sum_{j in cols} Gamma_R,j sum_{i in L} Gamma_L,i |G_ij(E)|^2.

    Eq. T-realspace of Sec. II.B (derived in the Appendix from Eq. T), with the
    factor 4 of the coupling Gamma = 2*CAP.  With ``cols`` = every point of the
    right CAP this is the full transmission; a subset gives a partial sum.
    """
    if cols is None:
        cols = j.right_columns()
    cols = np.asarray(cols)
    out = []
    for E in energies:
        X = solve_columns(j, float(E), cols, method=method)
        out.append(4.0 * np.sum(j.gamma_r[cols] * column_weights(j, X)))
    return np.asarray(out)


def shifted_cocg(j, energies: Sequence[float], b: np.ndarray, seed: int = 0, rtol: float = 1e-10,
                 maxiter: int = 50000, stop_at: Optional[int] = None):
    """x(E) = A(E)^{-1} b for every E of ``energies`` from one Krylov space.

    A(E) = E 1 - H_KS + i Gamma (Eq. G) is a shift family: A(E) = A(E_s) +
    (E - E_s) 1 around the seed energy E_s = energies[seed].  The seed system
    runs plain COCG (x_0 = 0):

        alpha_k = rho_k / (p_k^T A_s p_k),  x += alpha_k p_k,  r -= alpha_k A_s p_k,
        beta_k = rho_{k+1} / rho_k,         p_{k+1} = r_{k+1} + beta_k p_k.

    Its residual is r_k = R_k(A_s) b with R_k a polynomial, R_k(0) = 1.  The
    shifted system's residual in the same Krylov space is collinear with it,
    r^sig_k = r_k / pi_k with pi_k = R_k(-sig), sig = E - E_s.  The three-term
    recurrence of R_k evaluated at -sig gives (alpha_{-1} = 1, beta_{-1} = 0,
    pi_{-1} = pi_0 = 1):

        pi_{k+1} = (1 + alpha_k sig) pi_k + (alpha_k beta_{k-1} / alpha_{k-1}) (pi_k - pi_{k-1}),
        alpha^sig_k = alpha_k pi_k / pi_{k+1},   beta^sig_k = beta_k (pi_k / pi_{k+1})^2,
        x^sig += alpha^sig_k p^sig_k,            p^sig_{k+1} = r_{k+1} / pi_{k+1} + beta^sig_k p^sig_k.

    One operator application per iteration serves every energy.  Iterates until
    every shifted residual ||r_k|| / |pi_k| is at most rtol ||b|| (or for
    ``stop_at`` iterations).  Returns (X, iterations, pi, r): X[e] the solution at
    energies[e], pi[e] the collinearity factor and r the seed residual at the stop.
    """
    E = np.asarray(energies, dtype=float)
    Es = float(E[seed])
    sig = E - Es
    b = np.asarray(b, dtype=np.complex128)
    bn = np.linalg.norm(b)
    nE = E.size
    X = np.zeros((nE, b.size), dtype=np.complex128)
    pi = np.ones(nE, dtype=np.complex128)
    if bn == 0.0:
        return X, 0, pi, b.copy()
    # the seed operator A(E_s) = A_loc(E_s) - B^T diag(e_kb) B, assembled once
    # (the same sparse products as apply_operator, without rebuilding them per step)
    A_loc = local_system_matrix(j, Es)
    Bp = _projector_rows(j) if j.n_proj else None

    def seed_op(v):
        y = A_loc @ v
        if Bp is not None:
            y = y - Bp.T @ (j.proj_ekb * (Bp @ v))
        return y

    r = b.copy()
    P = np.repeat(r[None, :], nE, axis=0)  # p^sig_0 = r_0 / pi_0 = b
    pi_old = np.ones(nE, dtype=np.complex128)
    rho = r @ r
    alpha_old, beta_old = 1.0 + 0j, 0j
    k = 0
    limit = maxiter if stop_at is None else stop_at
    while k < limit:
        p = P[seed]
        q = seed_op(p)
        alpha = rho / (p @ q)
        r = r - alpha * q
        rho_new = r @ r
        beta = rho_new / rho
        pi_new = (1.0 + alpha * sig) * pi + (alpha * beta_old / alpha_old) * (pi - pi_old)
        a_sig = alpha * pi / pi_new
        b_sig = beta * (pi / pi_new) ** 2
        X += a_sig[:, None] * P
        P = r[None, :] / pi_new[:, None] + b_sig[:, None] * P
        pi_old, pi = pi, pi_new
        alpha_old, beta_old, rho = alpha, beta, rho_new
        k += 1
        if stop_at is None and np.max(np.linalg.norm(r) / np.abs(pi)) <= rtol * bn:
            break
    return X, k, pi, r


def transmission_grad(j, energies: Sequence[float], cols: Optional[Sequence[int]] = None,
                      T_bar: Optional[Sequence[float]] = None, method: str = "lu"):
    """(T(E), d/dV_loc of sum_E T_bar(E) T(E)).

    With A = E - H + iGamma and H containing diag(V_loc), dA/dV_r = -e_r e_r^T,
    so dX_j/dV_r = G e_r X_j(r).  Then
        dT/dV_r = 8 sum_j Gamma_R,j Re( lambda_j(r) X_j(r) ),
        lambda_j = G (Gamma_L o conj(X_j))   (G^T = G, Eq. complex-sym),
    and lambda_j reuses the LU of the forward solve.
    """
    if cols is None:
        cols = j.right_columns()
    cols = np.asarray(cols)
    energies = list(energies)
    if T_bar is None:
        T_bar = np.ones(len(energies))
    T = np.zeros(len(energies))
    g = np.zeros(j.N)
    for e, E in enumerate(energies):
        X, lu = solve_columns(j, float(E), cols, return_lu=True, method=method)
        T[e] = 4.0 * np.sum(j.gamma_r[cols] * column_weights(j, X))
        W = j.gamma_l[:, None] * np.conj(X)
        Lam = lu.solve(W)
        g += T_bar[e] * 8.0 * np.sum(j.gamma_r[cols][None, :] * np.real(Lam * X), axis=1)
    return T, g


def transmission_trace(G: np.ndarray, gamma_l: np.ndarray, gamma_r: np.ndarray) -> float:
    """Eq. T as a dense trace: Tr{ G Gamma_R G^dagger Gamma_L } (real part).

    ``gamma_l`` / ``gamma_r`` are the coupling matrices (2-D) or their diagonals.
    """
    GL = np.diag(gamma_l) if np.ndim(gamma_l) == 1 else gamma_l
    GR = np.diag(gamma_r) if np.ndim(gamma_r) == 1 else gamma_r
    return float(np.real(np.trace(G @ GR @ G.conj().T @ GL)))


def transmission_eigen(j, energies: Iterable[float]) -> np.ndarray:
    """Eq. T-tilde-realsp from the full eigen-decomposition of H_op (tiny N).

    (H_KS - i Gamma) U_i = eps_i U_i (Eq. complex-energy-evp); the columns are
    scaled so that U^T U = 1 (complex orthogonal, U^dagger = (U^{-1})^*).  Then
    Gt_L = U^dagger Gamma_L U, Gt_R = U^T Gamma_R U^* (Eq. Gamma-tilde) and
        T = sum_{ij} Gt_L,ij Gt_R,ji / ((E - eps_j)(E - eps_i^*)),
    with the coupling taken as 2*CAP as in ``transmission``.
    """
    H = hamiltonian(j).toarray()
    W = j.gamma_l + j.gamma_r
    Hop = H - 1j * np.diag(W)
    eps, U = sla.eig(Hop)
    norms = np.sqrt(np.sum(U * U, axis=0))  # complex "norm" u^T u
    U = U / norms[None, :]
    GtL = U.conj().T @ np.diag(2.0 * j.gamma_l) @ U
    GtR = U.T @ np.diag(2.0 * j.gamma_r) @ U.conj()
    out = []
    for E in energies:
        dj = 1.0 / (E - eps)  # 1/(E - eps_j)
        di = 1.0 / (E - np.conj(eps))  # 1/(E - eps_i^*)
        out.append(np.real(np.sum(GtL * GtR.T * di[:, None] * dj[None, :])))
    return np.asarray(out)


def fermi(x: np.ndarray, kT: float) -> np.ndarray:
    """Fermi-Dirac occupation f(x) = 1 / (1 + exp(x / kT)) of an energy x
    measured from the chemical potential; kT = 0: step with f(0) = 1/2."""
    x = np.asarray(x, dtype=float)
    if kT == 0.0:
        return np.where(x < 0, 1.0, np.where(x > 0, 0.0, 0.5))
    return 0.5 * (1.0 - np.tanh(x / (2.0 * kT)))


def landauer_current(E: Sequence[float], T: Sequence[float], V: Sequence[float], E_F: float = 0.0,
                     kT: float = 0.0) -> np.ndarray:
    """Eq. Landauer: I(V) = (2e/h) int T(E) [f(E - mu_L) - f(E - mu_R)] dE,
    mu_{L,R} = E_F +- V/2 (Sec. II.A: the electrodes' chemical potentials sit at
    +-eV/2 about the Fermi level).  Atomic units (e = hbar = 1, so 2e/h = 1/pi;
    energies and the bias eV in hartree, I in e E_h / hbar).  The integral is
    the trapezoidal rule on the ascending grid E where T is given."""
    E = np.asarray(E, dtype=float)
    T = np.asarray(T, dtype=float)
    out = []
    for v in np.atleast_1d(V):
        g = T * (fermi(E - (E_F + 0.5 * v), kT) - fermi(E - (E_F - 0.5 * v), kT))
        out.append(np.sum(0.5 * (E[1:] - E[:-1]) * (g[1:] + g[:-1])) / np.pi)
    return np.asarray(out)


# ----------------------------------------------------------------------------
# closed forms for the hard-wall waveguide (2nd-order FD, V = 0)
# ----------------------------------------------------------------------------

def channel_thresholds(nx: int, ny: int, h: float) -> np.ndarray:
    """Transverse energies eps_mn = (2 - cos(m pi/(nx+1)) - cos(n pi/(ny+1))) / h^2,
    the eigenvalues of -1/2 lap on an nx x ny Dirichlet cross-section."""
    m = np.arange(1, nx + 1)
    n = np.arange(1, ny + 1)
    em = (1.0 - np.cos(m * np.pi / (nx + 1))) / (h * h)
    en = (1.0 - np.cos(n * np.pi / (ny + 1))) / (h * h)
    return np.sort((em[:, None] + en[None, :]).ravel())


def open_channels(nx: int, ny: int, h: float, E: float) -> int:
    """Number of propagating modes: eps_mn < E < eps_mn + 2/h^2 (the 1-D band of
    -1/2 d^2/dz^2 on the lattice spans [0, 2/h^2])."""
    eps = channel_thresholds(nx, ny, h)
    return int(np.sum((eps < E) & (E < eps + 2.0 / (h * h))))


def lead_self_energy_T(nx: int, ny: int, nz: int, h: float, E: float) -> float:
    """Transmission of a perfect waveguide with exact semi-infinite leads.

    Device: nz planes of the 2nd-order Dirichlet waveguide (V = 0).  Each lead
    continues the same lattice to infinity; per transverse mode phi_mn its
    surface self-energy is Sigma = -tau e^{ik}, tau = 1/(2h^2), with
    E - eps_mn = (1 - cos k)/h^2, k in (0, pi) (evanescent modes: the decaying
    root).  Gamma = i(Sigma - Sigma^dagger) and T = Tr{G Gam_R G^dag Gam_L}
    (Eq. T) -- textbook NEGF, independent of any absorbing potential.
    """
    tau = 1.0 / (2.0 * h * h)
    nxy = nx * ny
    N = nxy * nz
    # transverse modes (orthonormal sine basis on the cross-section)
    px = np.sqrt(2.0 / (nx + 1)) * np.sin(np.outer(np.arange(1, nx + 1), np.arange(1, nx + 1)) * np.pi / (nx + 1))
    py = np.sqrt(2.0 / (ny + 1)) * np.sin(np.outer(np.arange(1, ny + 1), np.arange(1, ny + 1)) * np.pi / (ny + 1))
    sig_plane = np.zeros((nxy, nxy), dtype=np.complex128)
    for m in range(nx):
        for n in range(ny):
            eps = (1.0 - np.cos((m + 1) * np.pi / (nx + 1))) / (h * h) \
                + (1.0 - np.cos((n + 1) * np.pi / (ny + 1))) / (h * h)
            # solve tau*(2cos k) ... : E - eps - 2tau = -2 tau cos k
            c = (2.0 * tau - (E - eps)) / (2.0 * tau)  # cos k
            if abs(c) <= 1.0:
                k = np.arccos(c)
                s = -tau * np.exp(1j * k)
            else:
                # evanescent: e^{ik} = lam with |lam| < 1 and lam + 1/lam = 2c
                lam = c - np.sign(c) * np.sqrt(c * c - 1.0)
                s = -tau * lam
            phi = np.outer(py[n], px[m]).ravel()  # x fastest within the plane
            sig_plane += s * np.outer(phi, phi)
    lap = laplacian(nx, ny, nz, h, 1)
    H = (-0.5 * lap).toarray()
    SL = np.zeros((N, N), dtype=np.complex128)
    SR = np.zeros((N, N), dtype=np.complex128)
    SL[:nxy, :nxy] = sig_plane
    SR[N - nxy:, N - nxy:] = sig_plane
    G = np.linalg.inv(E * np.eye(N) - H - SL - SR)
    GamL = 1j * (SL - SL.conj().T)
    GamR = 1j * (SR - SR.conj().T)
    return transmission_trace(G, GamL, GamR)
