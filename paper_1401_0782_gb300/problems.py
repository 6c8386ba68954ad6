"""Seeded synthetic junctions: the inputs shared by the CUDA path and the oracle.

This module builds problem *data* only -- grid, local potential V_loc, the two
absorbing potentials Gamma_L / Gamma_R, Kleinman-Bylander projector values,
energy grids and the set of right-lead columns.  It holds none of the
method's arithmetic (no finite-difference coefficients, no operator, no
Green's function, no transmission); each side builds those itself.

Conventions (used by every consumer):

* Grid points ``(ix, iy, iz)`` sit at ``(ix*h, iy*h, iz*h)``; the flat index is
  ``ix + nx*(iy + ny*iz)`` (x fastest).  Outside the box the wave function is
  zero (Dirichlet) on every axis.
* The transport axis is z.  The absorbing potentials are diagonal and real,
  ``Gamma >= 0``, and enter the system matrix as ``E - H + i(Gamma_L+Gamma_R)``
  (Sec. II.B, Eq. Hop, with the CAP playing the anti-Hermitian part of the
  lead self-energy).
* Projectors are given in compressed-row form, one row per projector:
  ``proj_offsets[p]:proj_offsets[p+1]`` index ``proj_idx`` (flat grid index)
  and ``proj_val``.  The values already include the quadrature weight,
  ``val = beta(r) * sqrt(h^3)``, so the nonlocal term is
  ``H_nl = sum_p e_kb[p] * val_p val_p^T`` and each projector has unit 2-norm.
  Projectors of one atom share their support and are stored consecutively.

Workload recipes (sizes, depths and seeds) follow the synthetic junctions
used throughout the tests and the benchmark; every random draw comes from
``numpy.random.default_rng(seed)`` in the order documented in each builder.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Junction",
    "cap_quadratic",
    "cap_gaussian",
    "waveguide",
    "molecular_junction",
    "batched_junctions",
    "adjoint_junction",
    "energy_grid",
    "column_subset",
]


@dataclasses.dataclass
class Junction:
    """One real-space junction: grid, V_loc, CAPs and KB projectors."""

    nx: int
    ny: int
    nz: int
    h: float
    fd_half_order: int  # R: the Laplacian stencil reaches +-R points per axis
    v_loc: np.ndarray  # (N,) float64
    gamma_l: np.ndarray  # (N,) float64, >= 0
    gamma_r: np.ndarray  # (N,) float64, >= 0
    proj_offsets: np.ndarray  # (n_proj+1,) int64
    proj_idx: np.ndarray  # (nnz,) int32
    proj_val: np.ndarray  # (nnz,) float64, beta*sqrt(h^3)
    proj_ekb: np.ndarray  # (n_proj,) float64
    name: str = ""
    n_cap: int = 0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_proj(self) -> int:
        return int(self.proj_ekb.shape[0])

    def right_columns(self) -> np.ndarray:
        """Grid points j with Gamma_R[j] > 0, ascending (the G columns T needs)."""
        return np.flatnonzero(self.gamma_r > 0).astype(np.int32)

    def left_columns(self) -> np.ndarray:
        return np.flatnonzero(self.gamma_l > 0).astype(np.int32)

    def with_potential(self, v_loc: np.ndarray) -> "Junction":
        return dataclasses.replace(self, v_loc=np.ascontiguousarray(v_loc, dtype=np.float64))

    def nbytes_setup(self) -> int:
        """Bytes a full upload of this junction's setup arrays moves host->device."""
        return int(
            self.v_loc.nbytes
            + self.gamma_l.nbytes
            + self.gamma_r.nbytes
            + self.proj_offsets.nbytes
            + self.proj_idx.nbytes
            + self.proj_val.nbytes
            + self.proj_ekb.nbytes
        )


# ----------------------------------------------------------------------------
# absorbing potentials (diagonal, uniform across each z plane)
# ----------------------------------------------------------------------------

def cap_quadratic(nx: int, ny: int, nz: int, n_cap: int, amplitude: float):
    """Quadratic CAP over the ``n_cap`` end planes of each lead.

    Depth d counts planes into the absorbing slab from its inner edge: d = 1 on
    the innermost CAP plane and d = n_cap on the outermost (boundary) plane,
    Gamma = amplitude * (d / n_cap)^2.  Gamma_L and Gamma_R mirror each other.
    """
    if not (0 < n_cap and 2 * n_cap <= nz):
        raise ValueError("need 0 < n_cap <= nz/2")
    prof_l = np.zeros(nz)
    prof_r = np.zeros(nz)
    for iz in range(n_cap):
        d = n_cap - iz
        prof_l[iz] = amplitude * (d / n_cap) ** 2
        prof_r[nz - 1 - iz] = amplitude * (d / n_cap) ** 2
    plane = np.ones(nx * ny)
    return np.kron(prof_l, plane), np.kron(prof_r, plane)


def cap_gaussian(nx: int, ny: int, nz: int, h: float, gamma0: float, sigma: float,
                 cutoff: float = 1e-8):
    """Gaussian absorbing potential of Sec. II.B (Eq. ABC).

    Gamma_{L,R}(z) = gamma0 * exp(-(z - z_{L,R})^2 / sigma^2), centred on the
    first / last plane; the left profile covers the left half of the cell and
    the right profile the right half, each truncated where it falls below
    ``cutoff * gamma0`` so that the two supports stay disjoint.
    """
    z = np.arange(nz) * h
    zl, zr = 0.0, (nz - 1) * h
    gl = gamma0 * np.exp(-((z - zl) ** 2) / sigma**2)
    gr = gamma0 * np.exp(-((z - zr) ** 2) / sigma**2)
    half = nz // 2
    gl[half:] = 0.0
    gr[:half] = 0.0
    gl[gl < cutoff * gamma0] = 0.0
    gr[gr < cutoff * gamma0] = 0.0
    plane = np.ones(nx * ny)
    return np.kron(gl, plane), np.kron(gr, plane)


# ----------------------------------------------------------------------------
# potentials and projectors
# ----------------------------------------------------------------------------

def _coords(nx, ny, nz, h):
    ix = np.arange(nx) * h
    iy = np.arange(ny) * h
    iz = np.arange(nz) * h
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")  # x fastest after ravel
    return X.ravel(), Y.ravel(), Z.ravel()


def _soft_square_wall(nx, ny, nz, h, side_pts, v_wall, width):
    """V = v_wall * (1 - s(x) s(y)), s(u) = (1 + tanh((a - |u-u_c|)/w)) / 2."""
    X, Y, _ = _coords(nx, ny, nz, h)
    a = 0.5 * side_pts * h
    xc = 0.5 * (nx - 1) * h
    yc = 0.5 * (ny - 1) * h
    sx = 0.5 * (1.0 + np.tanh((a - np.abs(X - xc)) / width))
    sy = 0.5 * (1.0 + np.tanh((a - np.abs(Y - yc)) / width))
    return v_wall * (1.0 - sx * sy)


def _real_harmonics(l, dx, dy, dz):
    """Unnormalised real solid harmonics r^l Y_lm for l = 0, 1, 2."""
    if l == 0:
        return [np.ones_like(dx)]
    if l == 1:
        return [dx, dy, dz]
    if l == 2:
        r2 = dx * dx + dy * dy + dz * dz
        return [dx * dy, dy * dz, dz * dx, dx * dx - dy * dy, 3.0 * dz * dz - r2]
    raise ValueError(l)


def _kb_projectors(nx, ny, nz, h, centres, lmax, rc, ekb_per_l):
    """Gaussian KB projectors beta_{a,lm} = r^l Y_lm exp(-r^2/(2 rc^2)), |r| <= 2 rc.

    Each projector is normalised on the grid (h^3 sum beta^2 = 1) and stored as
    val = beta * sqrt(h^3), i.e. with unit 2-norm.  ``ekb_per_l[a][l]`` is shared
    by the 2l+1 projectors of shell l of atom a.
    """
    X, Y, Z = _coords(nx, ny, nz, h)
    offsets = [0]
    idx_list: List[np.ndarray] = []
    val_list: List[np.ndarray] = []
    ekb: List[float] = []
    for a, c in enumerate(centres):
        dx, dy, dz = X - c[0], Y - c[1], Z - c[2]
        r2 = dx * dx + dy * dy + dz * dz
        sup = np.flatnonzero(r2 <= (2.0 * rc) ** 2)
        g = np.exp(-r2[sup] / (2.0 * rc * rc))
        for l in range(lmax + 1):
            for harm in _real_harmonics(l, dx[sup], dy[sup], dz[sup]):
                beta = harm * g
                nrm = np.sqrt(np.sum(beta * beta))
                if nrm == 0.0:
                    beta = np.zeros_like(beta)
                else:
                    beta = beta / nrm
                idx_list.append(sup.astype(np.int32))
                val_list.append(beta)
                offsets.append(offsets[-1] + sup.size)
                ekb.append(float(ekb_per_l[a][l]))
    if idx_list:
        idx = np.concatenate(idx_list).astype(np.int32)
        val = np.concatenate(val_list).astype(np.float64)
    else:
        idx = np.zeros(0, np.int32)
        val = np.zeros(0, np.float64)
    return (np.asarray(offsets, np.int64), idx, val, np.asarray(ekb, np.float64))


def _no_projectors():
    return (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64),
            np.zeros(0, np.float64))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def waveguide(nx: int = 8, ny: int = 8, nz: int = 48, h: float = 0.5, n_cap: int = 16,
              cap_amplitude: float = 0.5, fd_half_order: int = 1,
              cap: str = "quadratic", gamma0: float = 0.5, sigma: Optional[float] = None) -> Junction:
    """Hard-wall free-electron waveguide: V_loc = 0, Dirichlet walls, no projectors.

    Defaults: 8x8x48 points (3,072), h = 0.5 bohr, 2nd-order Laplacian, quadratic
    CAP of amplitude 0.5 Ha over the 16 end planes of each lead.
    """
    N = nx * ny * nz
    if cap == "quadratic":
        gl, gr = cap_quadratic(nx, ny, nz, n_cap, cap_amplitude)
    elif cap == "gaussian":
        gl, gr = cap_gaussian(nx, ny, nz, h, gamma0, sigma if sigma else n_cap * h / 2.0)
    else:
        raise ValueError(cap)
    off, idx, val, ekb = _no_projectors()
    return Junction(nx, ny, nz, h, fd_half_order, np.zeros(N), gl, gr, off, idx, val, ekb,
                    name=f"waveguide_{nx}x{ny}x{nz}", n_cap=n_cap)


def molecular_junction(seed: int = 1, nx: int = 24, ny: int = 24, nz: int = 120,
                       h: float = 0.35, fd_half_order: int = 4, n_wells: int = 20,
                       lmax: int = 1, n_cap: int = 8, cap_amplitude: float = 0.5,
                       side_pts: Optional[int] = None, v_wall: float = 3.0,
                       wall_width: float = 0.5, rc: float = 1.5, sigma_well: float = 1.0,
                       central_planes: Optional[int] = None) -> Junction:
    """Synthetic molecular junction (defaults: 24x24x120, h = 0.35, 8th-order FD).

    * Lead confinement: V_wall = 3 Ha outside a centred soft square of
      ``side_pts`` points (default round(2n/3): 16 for n = 24) with tanh edges of
      width 0.5 bohr.
    * ``n_wells`` Gaussian wells exp(-r^2/(2 sigma^2)), sigma = 1 bohr, depth
      U[-2, -0.5] Ha, centres uniform in the central ``central_planes`` planes
      (default nz/3: 40 for nz = 120) and inside the soft square.
    * One atom per well centre carrying s (lmax >= 0), p (lmax >= 1) and d
      (lmax = 2) Gaussian KB projectors, r_c = 1.5 bohr, support |r| <= 2 r_c,
      E_KB ~ U[-1, 1] Ha drawn once per (atom, l).
    * Quadratic CAP of ``n_cap`` planes, amplitude 0.5 Ha, at each end.

    Draw order from default_rng(seed): well centres (n_wells x 3 uniforms in
    [0,1)), well depths (n_wells), then E_KB (n_wells x (lmax+1)).
    """
    if side_pts is None:
        side_pts = int(round(2 * nx / 3))
    if central_planes is None:
        central_planes = nz // 3
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    v = _soft_square_wall(nx, ny, nz, h, side_pts, v_wall, wall_width)
    a = 0.5 * side_pts * h
    xc, yc = 0.5 * (nx - 1) * h, 0.5 * (ny - 1) * h
    z_lo = ((nz - central_planes) // 2) * h
    z_hi = z_lo + (central_planes - 1) * h
    u = rng.random((n_wells, 3))
    centres = np.empty((n_wells, 3))
    centres[:, 0] = xc - a + 2 * a * u[:, 0]
    centres[:, 1] = yc - a + 2 * a * u[:, 1]
    centres[:, 2] = z_lo + (z_hi - z_lo) * u[:, 2]
    depth = rng.uniform(-2.0, -0.5, n_wells)
    ekb = rng.uniform(-1.0, 1.0, (n_wells, lmax + 1))
    X, Y, Z = _coords(nx, ny, nz, h)
    for c, d in zip(centres, depth):
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        v = v + d * np.exp(-r2 / (2.0 * sigma_well**2))
    off, idx, val, e = _kb_projectors(nx, ny, nz, h, centres, lmax, rc, ekb)
    gl, gr = cap_quadratic(nx, ny, nz, n_cap, cap_amplitude)
    return Junction(nx, ny, nz, h, fd_half_order, v, gl, gr, off, idx, val, e,
                    name=f"junction_{nx}x{ny}x{nz}_s{seed}", n_cap=n_cap)


def adjoint_junction(seed: int = 4) -> Junction:
    """Large junction for the adjoint: 48x48x192 (442,368 points), h = 0.3 bohr,
    12th-order FD, 60 wells, 60 atoms x 9 s/p/d projectors, 6-plane CAP."""
    return molecular_junction(seed=seed, nx=48, ny=48, nz=192, h=0.3, fd_half_order=6,
                              n_wells=60, lmax=2, n_cap=6)


def batched_junctions(n: int = 64, seed0: int = 1000, h: float = 0.35,
                      fd_half_order: int = 4) -> List[Junction]:
    """Uneven junction set: junction k uses default_rng(seed0 + k) and draws, in
    order, its cross-section n_xy ~ U{12..32}, length nz ~ U{64..192}, CAP depth
    ~ U{6..10} planes and well count ~ U{5..30}; the rest follows
    ``molecular_junction`` with the same generator state continued."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        nxy = int(rng.integers(12, 33))
        nz = int(rng.integers(64, 193))
        n_cap = int(rng.integers(6, 11))
        n_wells = int(rng.integers(5, 31))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        out.append(molecular_junction(seed=sub_seed, nx=nxy, ny=nxy, nz=nz, h=h,
                                      fd_half_order=fd_half_order, n_wells=n_wells,
                                      lmax=1, n_cap=n_cap))
        out[-1].name = f"batched_{k}_{nxy}x{nxy}x{nz}"
    return out


def energy_grid(lo: float, hi: float, n: int) -> np.ndarray:
    """n energies uniformly spaced in [lo, hi], endpoints included."""
    return np.linspace(lo, hi, n)


def column_subset(junction: Junction, n: int, seed: int) -> np.ndarray:
    """A seeded, ascending subset of n right-lead columns (all if n >= count)."""
    cols = junction.right_columns()
    if n >= cols.size:
        return cols
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(cols.size, size=n, replace=False))
    return cols[pick].astype(np.int32)


def tiny_junction(seed: int = 7, nx: int = 4, ny: int = 4, nz: int = 12, h: float = 0.5,
                  fd_half_order: int = 2, n_cap: int = 3, lmax: int = 1,
                  n_atoms: int = 2) -> Junction:
    """Small random junction for brute-force checks (dense inversion on N ~ 200)."""
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    v = rng.uniform(-0.5, 0.5, N)
    X, Y, Z = _coords(nx, ny, nz, h)
    centres = np.stack([rng.uniform(0.3, 0.7, n_atoms) * (nx - 1) * h,
                        rng.uniform(0.3, 0.7, n_atoms) * (ny - 1) * h,
                        rng.uniform(0.35, 0.65, n_atoms) * (nz - 1) * h], axis=1)
    ekb = rng.uniform(-1.0, 1.0, (n_atoms, lmax + 1))
    off, idx, val, e = _kb_projectors(nx, ny, nz, h, centres, lmax, 0.6, ekb)
    gl, gr = cap_quadratic(nx, ny, nz, n_cap, 0.5)
    return Junction(nx, ny, nz, h, fd_half_order, v, gl, gr, off, idx, val, e,
                    name=f"tiny_{nx}x{ny}x{nz}_R{fd_half_order}", n_cap=n_cap)


__all__.append("tiny_junction")
