"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the benchmark.

This module holds problem data only: the structured grid description, the seeded density field,
the reference load vector f and the set of Dirichlet (fixed) degrees of freedom.  It contains none
of the method's arithmetic (no element matrices, no solves, no eigenproblems), so both sides may
import it without sharing any computational code.

Layout conventions (the same ones the C-ABI documents):
  * element (i, j[, k]) has flat index  e = i + nelx * (j + nely * k)            (x fastest)
  * node    (i, j[, k]) has flat index  a = i + (nelx+1) * (j + (nely+1) * k)
  * DOF c of node a is  d * a + c  (node-interleaved, d = 2 in 2D, 3 in 3D)
  * every element is a unit square / unit cube.

The paper's design field is a filtered and projected density (Sec. 2, the density filter and the
relaxed Heaviside projection).  The solver takes physical densities as input; the density filter is
used here only to turn seeded Gaussian noise into smooth, design-like fields with the length scale
of the paper's examples.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np
from scipy import ndimage

__all__ = [
    "Problem",
    "density_field",
    "column_2d",
    "cantilever_3d",
    "config",
    "CONFIG_NAMES",
    "batch_configs",
]


@dataclass
class Problem:
    """A structured-grid linear-buckling problem instance (inputs only)."""

    name: str
    dim: int
    nel: Tuple[int, int, int]          # (nelx, nely, nelz); nelz = 1 in 2D (ignored)
    x: np.ndarray                      # physical densities, float64 [m]
    f: np.ndarray                      # reference load vector, float64 [n]
    fixed: np.ndarray                  # uint8 [n], 1 = Dirichlet DOF (u = 0)
    nu: float = 0.3
    E0: float = 1.0                    # solid modulus
    Emin: float = 1e-6                 # void modulus (stiffness interpolation only)
    penal: float = 3.0
    mg_levels: int = 3
    eig_level: int = 1                 # 1 = eigenproblem on the fine grid (exact LBA)
    num_modes: int = 6
    meta: dict = field(default_factory=dict)

    @property
    def nelx(self) -> int:
        return self.nel[0]

    @property
    def nely(self) -> int:
        return self.nel[1]

    @property
    def nelz(self) -> int:
        return self.nel[2] if self.dim == 3 else 1

    @property
    def num_elements(self) -> int:
        return int(self.x.size)

    @property
    def num_nodes(self) -> int:
        if self.dim == 2:
            return (self.nelx + 1) * (self.nely + 1)
        return (self.nelx + 1) * (self.nely + 1) * (self.nelz + 1)

    @property
    def num_dofs(self) -> int:
        return self.dim * self.num_nodes


# ----------------------------------------------------------------------------------------------
# density field
# ----------------------------------------------------------------------------------------------
def _cone_kernel(radius: float, dim: int) -> np.ndarray:
    r = int(np.ceil(radius)) - 1 if float(radius).is_integer() else int(np.floor(radius))
    r = max(r, 0)
    ax = np.arange(-r, r + 1, dtype=np.float64)
    if dim == 2:
        gy, gx = np.meshgrid(ax, ax, indexing="ij")
        dist = np.sqrt(gx * gx + gy * gy)
    else:
        gz, gy, gx = np.meshgrid(ax, ax, ax, indexing="ij")
        dist = np.sqrt(gx * gx + gy * gy + gz * gz)
    return np.maximum(0.0, radius - dist)


def density_field(shape_zyx: Tuple[int, ...], seed: int, radius: float, volfrac: float,
                  amplitude: float = 0.25, xmin: float = 0.01) -> np.ndarray:
    """Seeded smooth density field on an element grid, mean = volfrac (to 1e-9), values in [xmin, 1].

    Recipe: N(0,1) noise per element from numpy's PCG64 with the given seed -> cone (linear hat)
    filter of the given radius in element units, normalised by the in-domain weight sum -> scaled to
    zero mean, unit standard deviation -> x = clip(volfrac + amplitude * s + c, xmin, 1), with the
    shift c found by bisection so that mean(x) = volfrac.  Returned flat with x fastest.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape_zyx)
    ker = _cone_kernel(radius, len(shape_zyx))
    num = ndimage.convolve(noise, ker, mode="constant", cval=0.0)
    den = ndimage.convolve(np.ones_like(noise), ker, mode="constant", cval=0.0)
    s = num / den
    s = (s - s.mean()) / s.std()
    base = volfrac + amplitude * s
    lo, hi = -1.0, 1.0
    for _ in range(64):  # the bracket [-1, 1] shrinks below one unit in the last place of c
        c = 0.5 * (lo + hi)
        m = np.clip(base + c, xmin, 1.0).mean()
        if m < volfrac:
            lo = c
        else:
            hi = c
    x = np.clip(base + 0.5 * (lo + hi), xmin, 1.0)
    return np.ascontiguousarray(x.reshape(-1), dtype=np.float64)


# ----------------------------------------------------------------------------------------------
# boundary conditions and loads
# ----------------------------------------------------------------------------------------------
def column_2d(nel_long: int, nel_short: int, seed: int, radius: float, volfrac: float = 0.5,
              name: str = "column2d", mg_levels: int = 3, eig_level: int = 1, num_modes: int = 6,
              x: Optional[np.ndarray] = None) -> Problem:
    """2D Q4 plane-stress column: nel_long elements tall (y), nel_short wide (x).

    All DOFs of the base nodes (y = 0) are fixed.  A downward (compressive) load of total magnitude 1
    is spread uniformly over the top edge (y = nel_long) as consistent nodal loads: interior top nodes
    carry 1/nel_short, the two corner nodes 1/(2 nel_short).
    """
    nelx, nely = nel_short, nel_long
    if x is None:
        x = density_field((nely, nelx), seed, radius, volfrac)
    nnx, nny = nelx + 1, nely + 1
    n = 2 * nnx * nny
    f = np.zeros(n)
    top = (nny - 1) * nnx + np.arange(nnx)
    w = np.full(nnx, 1.0 / nelx)
    w[0] *= 0.5
    w[-1] *= 0.5
    f[2 * top + 1] = -w
    fixed = np.zeros(n, dtype=np.uint8)
    base = np.arange(nnx)
    fixed[2 * base] = 1
    fixed[2 * base + 1] = 1
    f[fixed == 1] = 0.0
    return Problem(name=name, dim=2, nel=(nelx, nely, 1), x=x, f=f, fixed=fixed,
                   mg_levels=mg_levels, eig_level=eig_level, num_modes=num_modes,
                   meta=dict(seed=seed, radius=radius, volfrac=volfrac))


def cantilever_3d(nelx: int, nely: int, nelz: int, seed: int, radius: float, volfrac: float,
                  name: str = "cantilever3d", mg_levels: int = 4, eig_level: int = 3,
                  num_modes: int = 12, x: Optional[np.ndarray] = None) -> Problem:
    """3D H8 cantilever: all DOFs on the face x = 0 fixed; a downward (-z) load of total magnitude 1
    spread uniformly over the top face z = nelz (each element face passes a quarter of its share to
    each of its four nodes; shares landing on fixed DOFs are dropped)."""
    if x is None:
        x = density_field((nelz, nely, nelx), seed, radius, volfrac)
    nnx, nny, nnz = nelx + 1, nely + 1, nelz + 1
    n = 3 * nnx * nny * nnz
    f = np.zeros(n)
    wx = np.ones(nnx)
    wx[0] = wx[-1] = 0.5
    wy = np.ones(nny)
    wy[0] = wy[-1] = 0.5
    wtop = np.outer(wy, wx).reshape(-1) / float(nelx * nely)
    top = (nnz - 1) * nnx * nny + np.arange(nnx * nny)
    f[3 * top + 2] = -wtop
    fixed = np.zeros(n, dtype=np.uint8)
    kk, jj = np.meshgrid(np.arange(nnz), np.arange(nny), indexing="ij")
    face = (kk * nny + jj).reshape(-1) * nnx
    for c in range(3):
        fixed[3 * face + c] = 1
    f[fixed == 1] = 0.0
    return Problem(name=name, dim=3, nel=(nelx, nely, nelz), x=x, f=f, fixed=fixed,
                   mg_levels=mg_levels, eig_level=eig_level, num_modes=num_modes,
                   meta=dict(seed=seed, radius=radius, volfrac=volfrac))


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------
CONFIG_NAMES = ("column60x20", "column480x160", "cantilever96x48x48", "cantilever128x64x64")


def config(name: str) -> Problem:
    """The named synthetic workloads.

    column60x20         2D Q4, 60 x 20, seed 0, filter radius 2, volfrac 0.5, 3 MG levels, exact
                        fine-grid eigenproblem, 6 modes.
    column480x160       2D Q4, 480 x 160, seed 1, radius 4, volfrac 0.5, 5 MG levels, eigenproblem
                        on level 3 (120 x 40), 12 modes.
    cantilever96x48x48  3D H8, 96 x 48 x 48, seed 2, radius 3, volfrac 0.3, 5 MG levels (coarsest
                        6 x 3 x 3), eigenproblem on level 3 (24 x 12 x 12), 12 modes.
    cantilever128x64x64 3D H8, 128 x 64 x 64, seed 3, radius 3, volfrac 0.3, 5 MG levels.
    """
    if name == "column60x20":
        return column_2d(60, 20, seed=0, radius=2, volfrac=0.5, name=name, mg_levels=3,
                         eig_level=1, num_modes=6)
    if name == "column480x160":
        return column_2d(480, 160, seed=1, radius=4, volfrac=0.5, name=name, mg_levels=5,
                         eig_level=3, num_modes=12)
    if name == "cantilever96x48x48":
        return cantilever_3d(96, 48, 48, seed=2, radius=3, volfrac=0.3, name=name, mg_levels=5,
                             eig_level=3, num_modes=12)
    if name == "cantilever128x64x64":
        return cantilever_3d(128, 64, 64, seed=3, radius=3, volfrac=0.3, name=name, mg_levels=5,
                             eig_level=4, num_modes=12)
    raise KeyError(name)


def batch_levels(nel_long: int, nel_short: int, coarsest_short: int = 8) -> int:
    """Multigrid levels of a batch design: halve both axes while the short side is even and larger
    than coarsest_short (and the long side stays even)."""
    levels, t, a = 1, nel_short, nel_long
    while t % 2 == 0 and t > coarsest_short and a % 2 == 0:
        t //= 2
        a //= 2
        levels += 1
    return levels


def batch_configs(count: int = 64, seed0: int = 100) -> List[Problem]:
    """Uneven batch of 2D columns: nel_long = a * nel_short with a in {2, 3, 4},
    nel_short in {32, 48, 64, ..., 256}, nel_long <= 512; volfrac ~ U[0.3, 0.6], radius in [2, 4].
    Each design coarsens until the short side has at most 8 elements (batch_levels)."""
    out = []
    rng = np.random.default_rng(seed0)
    shorts = [s for s in range(32, 257, 16)]
    for b in range(count):
        while True:
            a = int(rng.integers(2, 5))
            s = int(shorts[int(rng.integers(0, len(shorts)))])
            if a * s <= 512:
                break
        vf = float(rng.uniform(0.3, 0.6))
        r = float(rng.uniform(2.0, 4.0))
        out.append(column_2d(a * s, s, seed=seed0 + b, radius=r, volfrac=vf, name=f"batch{b}",
                             mg_levels=batch_levels(a * s, s), eig_level=1, num_modes=6))
    return out
