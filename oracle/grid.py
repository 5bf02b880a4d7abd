"""Structured-grid bookkeeping for the fine grid Omega_1 and the nested coarse grids (Sec. 2, Sec. 2.1).

Numbering (x fastest): element e = i + nelx (j + nely k); node a = i + (nelx+1)(j + (nely+1) k);
DOF = dim * a + c.  Local element node order follows oracle.elements.
"""
from __future__ import annotations

import numpy as np


def node_dims(nel, dim):
    return tuple(n + 1 for n in nel[:dim])


def num_nodes(nel, dim):
    return int(np.prod(node_dims(nel, dim)))


def element_nodes(nel, dim) -> np.ndarray:
    """[m, 2^dim] global node indices of each element, in the local order of oracle.elements."""
    if dim == 2:
        nx, ny = nel[0], nel[1]
        nnx = nx + 1
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        n0 = (j * nnx + i).reshape(-1)
        return np.stack([n0, n0 + 1, n0 + 1 + nnx, n0 + nnx], axis=1)
    nx, ny, nz = nel
    nnx, nny = nx + 1, ny + 1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    n0 = ((k * nny + j) * nnx + i).reshape(-1)
    s = nnx * nny
    return np.stack([n0, n0 + 1, n0 + 1 + nnx, n0 + nnx,
                     n0 + s, n0 + s + 1, n0 + s + 1 + nnx, n0 + s + nnx], axis=1)


def element_dofs(nel, dim) -> np.ndarray:
    """[m, dim * 2^dim] global DOFs of each element (node-interleaved)."""
    en = element_nodes(nel, dim)
    return (dim * en[:, :, None] + np.arange(dim)[None, None, :]).reshape(en.shape[0], -1)


def coarse_nel(nel, dim):
    """Element counts of the next coarser grid (2:1 per axis)."""
    out = list(nel)
    for a in range(dim):
        if nel[a] % 2:
            raise ValueError("grid not divisible by 2 along axis %d" % a)
        out[a] = nel[a] // 2
    return tuple(out)


def level_nels(nel, dim, levels):
    """Element counts of levels 1..levels (level 1 = fine)."""
    out = [tuple(nel)]
    for _ in range(levels - 1):
        out.append(coarse_nel(out[-1], dim))
    return out


def coarse_fixed(fixed_fine: np.ndarray, nel_fine, dim) -> np.ndarray:
    """Dirichlet set of the next coarser grid: a coarse DOF is fixed when the fine DOF at the
    coinciding node is fixed (the paper leaves boundary conditions on coarse grids implicit)."""
    nf = node_dims(nel_fine, dim)
    F = fixed_fine.reshape(tuple(reversed(nf)) + (dim,))
    if dim == 2:
        C = F[::2, ::2, :]
    else:
        C = F[::2, ::2, ::2, :]
    return np.ascontiguousarray(C.reshape(-1)).astype(np.uint8)
