"""Write the golden per-column transmission contributions of the 24x24x120 junction.

For the benchmark junction (``problems.molecular_junction(seed=1)``: 24x24x120
points, h = 0.35 bohr, 8th-order FD, 20 atoms x 4 KB projectors, 8-plane
quadratic CAP) and three energies of the benchmark window (indices 0, 64 and 127
of linspace(0.16, 0.24, 128) Ha), this script solves 16 seeded right-CAP
columns x_c = G(E) e_c (Eq. G) with the oracle's sparse LU of the bordered
system and writes, per (E, column),

    t_c = sum_{i in L} Gamma_L,i |x_c(i)|^2          (Eq. T-realspace, one column)

so that T over these columns is 4 sum_c Gamma_R,c t_c.  Only ``oracle`` and the
input generators are used; nothing here comes from the CUDA library.  One LU
factorisation takes minutes and ~6 GB at this size, which is why the values are
stored instead of recomputed by the tests.

    python tests/golden/make_junction_golden.py  [--processes 3]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "junction_24x24x120_tc.txt")
E_INDEX = (0, 64, 127)
N_COLS = 16
COL_SEED = 8


def _energy(k: int) -> float:
    import numpy as np
    return float(np.linspace(0.16, 0.24, 128)[k])


def _columns(j):
    from paper_1401_0782_gb300 import problems as P
    return P.column_subset(j, N_COLS, seed=COL_SEED)


def _one(k: int):
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    from paper_1401_0782_gb300 import problems as P
    j = P.molecular_junction(seed=1)
    cols = _columns(j)
    E = _energy(k)
    X = O.solve_columns(j, E, cols)  # sparse LU (complex128)
    t = O.column_weights(j, X)
    # certify: relative residual of each column with the oracle's own operator
    b = np.zeros((j.N, cols.size), complex)
    b[cols, np.arange(cols.size)] = 1.0
    res = np.linalg.norm(b - O.apply_operator(j, E, X), axis=0)
    return k, E, cols, t, res


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--processes", type=int, default=len(E_INDEX))
    a = ap.parse_args()
    with mp.get_context("spawn").Pool(a.processes) as pool:
        rows = pool.map(_one, E_INDEX)
    with open(OUT, "w") as f:
        f.write("# Per-column transmission contributions t_c = sum_{i in L} Gamma_L,i |G_{i,c}(E)|^2 (Eq. T-realspace)\n")
        f.write("# junction: problems.molecular_junction(seed=1), 24x24x120, h=0.35, 8th-order FD, 80 KB projectors\n")
        f.write(f"# columns: problems.column_subset(j, {N_COLS}, seed={COL_SEED}); solver: oracle sparse LU (complex128)\n")
        f.write("# written by tests/golden/make_junction_golden.py (oracle only)\n")
        f.write("# energy_index  E_hartree  column  t_c  lu_relative_residual\n")
        for k, E, cols, t, res in rows:
            for c, tc, r in zip(cols, t, res):
                f.write(f"{k} {E:.17g} {int(c)} {tc:.17e} {r:.3e}\n")
    print(OUT)


if __name__ == "__main__":
    main()
