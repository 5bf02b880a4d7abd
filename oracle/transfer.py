"""Explicit interpolation operators between nested grids, Sec. 2.1 (I^j_{j+1}, I^{j+1}_j = (I^j_{j+1})^T).

The interpolation is the standard geometric bi/trilinear one of nested Q4/H8 grids with 2:1
coarsening: a fine node coinciding with a coarse node copies it; a fine node at an edge midpoint
averages the two edge ends; a face centre averages four; a cell centre (3D) averages eight.
Restricted to free DOFs (fixed fine rows and fixed coarse columns removed), the Galerkin operator is
K^{j+1} = P^T K^j P (Sec. 2.1 step 1; Algorithm 2 'restrict').
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import grid


def _axis_weights(nc: int) -> sp.csr_matrix:
    """1D linear interpolation from nc+1 coarse nodes to 2 nc + 1 fine nodes."""
    nf = 2 * nc
    rows, cols, vals = [], [], []
    for i in range(nf + 1):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [i // 2, i // 2 + 1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf + 1, nc + 1))


def interpolation(nel_fine, dim) -> sp.csr_matrix:
    """Full (all-DOF) interpolation P: coarse DOFs -> fine DOFs, node-interleaved, x fastest."""
    ncoarse = grid.coarse_nel(nel_fine, dim)
    Px = _axis_weights(ncoarse[0])
    Py = _axis_weights(ncoarse[1])
    if dim == 2:
        Pn = sp.kron(Py, Px)                 # node index = i + nnx * j  (x fastest)
    else:
        Pz = _axis_weights(ncoarse[2])
        Pn = sp.kron(Pz, sp.kron(Py, Px))
    return sp.kron(Pn, sp.eye(dim)).tocsr()


def free_interpolation(nel_fine, dim, fixed_fine, fixed_coarse) -> sp.csr_matrix:
    """P with fixed fine rows and fixed coarse columns removed (maps free coarse -> free fine)."""
    P = interpolation(nel_fine, dim)
    ff = np.flatnonzero(fixed_fine == 0)
    fc = np.flatnonzero(fixed_coarse == 0)
    return P[ff][:, fc].tocsr()


def hierarchy(nel, dim, fixed, levels):
    """Per level j = 1..levels: (nel_j, fixed_j) and free interpolations P_j : level j+1 -> level j."""
    nels = grid.level_nels(nel, dim, levels)
    fixeds = [np.asarray(fixed, dtype=np.uint8)]
    for j in range(levels - 1):
        fixeds.append(grid.coarse_fixed(fixeds[-1], nels[j], dim))
    Ps = [free_interpolation(nels[j], dim, fixeds[j], fixeds[j + 1]) for j in range(levels - 1)]
    return nels, fixeds, Ps
