"""Write golden values of T(E) and dT/dV_loc on the 48x48x192 adjoint junction.

Junction ``problems.adjoint_junction(seed=4)`` (442,368 points, h = 0.3 bohr,
12th-order FD, 60 wells, 60 atoms x 9 s/p/d KB projectors, 6-plane CAP), four
seeded right-CAP columns (``problems.column_subset(j, 4, seed=11)``), E = 0.2 Ha.
The oracle's steps of ``transmission_grad`` on its Krylov route (a sparse LU
at this size needs tens of GB): forward columns x_c = G e_c (Eq. G), then
lambda_c = G (Gamma_L o conj x_c) with the same operator (G = G^T, Eq.
complex-sym), T = 4 sum_c Gamma_R,c sum_L Gamma_L |x_c|^2 (Eq. T-realspace)
and dT/dV_r = 8 sum_c Gamma_R,c Re(lambda_c(r) x_c(r)).  Every solve is
certified by its true residual (relative 1e-13 forward, 1e-10 adjoint).  The
file keeps T, sum_r dT/dV_r, and dT/dV at 64 seeded points where the gradient
is large (the FD points of the tests among them).  Only ``oracle`` and the
input generators are used.

    python tests/golden/make_adjoint_golden.py
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "adjoint_junction_48x48x192_grad.txt")


def main() -> None:
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    from paper_1401_0782_gb300 import problems as P
    j = P.adjoint_junction(seed=4)
    cols = P.column_subset(j, 4, seed=11)
    E = 0.2
    X, solver = O.solve_columns(j, E, cols, return_lu=True, method="krylov", rtol=1e-13)
    T = 4.0 * np.sum(j.gamma_r[cols] * O.column_weights(j, X))
    solver.rtol = 1e-10
    W = j.gamma_l[:, None] * np.conj(X)
    Lam = solver.solve(W)
    g = 8.0 * np.sum(j.gamma_r[cols][None, :] * np.real(Lam * X), axis=1)
    rng = np.random.default_rng(4)
    pts = np.sort(rng.choice(np.flatnonzero(np.abs(g) > 0.05 * np.abs(g).max()), 64, replace=False))
    with open(OUT, "w") as f:
        f.write("# dT(E)/dV_loc(r) on problems.adjoint_junction(seed=4) (48x48x192), E = 0.2 Ha,\n")
        f.write(f"# columns problems.column_subset(j, 4, seed=11) = {' '.join(str(int(c)) for c in cols)}\n")
        f.write("# oracle Krylov route (forward relative residual 1e-13, adjoint 1e-10, both certified)\n")
        f.write("# written by tests/golden/make_adjoint_golden.py (oracle only)\n")
        f.write(f"T {T:.17e}\n")
        f.write(f"sum_g {g.sum():.17e}\n")
        f.write(f"max_abs_g {np.abs(g).max():.17e}\n")
        for r in pts:
            f.write(f"g {int(r)} {g[r]:.17e}\n")
    print(OUT)


if __name__ == "__main__":
    main()
