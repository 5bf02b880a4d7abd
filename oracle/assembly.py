"""Sparse assembly of K[x] and G[x, u] (Sec. 2: K_e = E_kappa(x_e) K_e0, G_e = E_sigma(x_e) G_e0[u_e])."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import elements, grid


def assemble_K(nel, dim, x, nu, penal, E0, Emin) -> sp.csr_matrix:
    """Global stiffness K[x] = sum_e E_kappa(x_e) A_e^T K_e0 A_e (all DOFs, no BCs)."""
    Ke0 = elements.stiffness_ke0(dim, nu)
    edofs = grid.element_dofs(nel, dim)
    Ek, _, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).reshape(-1)
    cols = np.tile(edofs, (1, nd)).reshape(-1)
    vals = (Ek[:, None, None] * Ke0[None, :, :]).reshape(-1)
    n = dim * grid.num_nodes(nel, dim)
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def element_stress_stiffness(nel, dim, u, nu) -> np.ndarray:
    """[m, nd, nd] unit-modulus G_e0[u_e] for every element (Sec. 2); the same formula as
    oracle.elements.stress_stiffness_ge0, evaluated for all elements at once."""
    edofs = grid.element_dofs(nel, dim)
    Ue = np.asarray(u, dtype=np.float64)[edofs]                  # [m, nd]
    D = elements.constitutive(dim, nu)
    pts, wts = elements.gauss_points(dim)
    nn = 2 ** dim
    Gs = np.zeros((edofs.shape[0], nn, nn))
    for xi, w in zip(pts, wts):
        dN = elements.shape_gradients(xi)
        sig = Ue @ (D @ elements.strain_matrix(dN)).T              # [m, nvoigt]
        S = np.zeros((edofs.shape[0], dim, dim))
        if dim == 2:
            S[:, 0, 0], S[:, 1, 1] = sig[:, 0], sig[:, 1]
            S[:, 0, 1] = S[:, 1, 0] = sig[:, 2]
        else:
            S[:, 0, 0], S[:, 1, 1], S[:, 2, 2] = sig[:, 0], sig[:, 1], sig[:, 2]
            S[:, 0, 1] = S[:, 1, 0] = sig[:, 3]
            S[:, 1, 2] = S[:, 2, 1] = sig[:, 4]
            S[:, 2, 0] = S[:, 0, 2] = sig[:, 5]
        Gs += w * elements.detJ(dim) * np.einsum("ai,mab,bj->mij", dN, S, dN)
    G = np.zeros((edofs.shape[0], dim * nn, dim * nn))
    for c in range(dim):
        G[:, c::dim, c::dim] = Gs
    return G


def assemble_G(nel, dim, x, u, nu, penal, E0, Emin) -> sp.csr_matrix:
    """Global stress stiffness G[x, u] = sum_e E_sigma(x_e) A_e^T G_e0[u_e] A_e (all DOFs)."""
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    Ge = element_stress_stiffness(nel, dim, u, nu)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).reshape(-1)
    cols = np.tile(edofs, (1, nd)).reshape(-1)
    vals = (Es[:, None, None] * Ge).reshape(-1)
    n = dim * grid.num_nodes(nel, dim)
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def restrict_free(A: sp.spmatrix, fixed: np.ndarray) -> sp.csr_matrix:
    """Rows and columns of the free DOFs (Dirichlet DOFs eliminated)."""
    free = np.flatnonzero(fixed == 0)
    return A.tocsr()[free][:, free].tocsr()


def apply_K(nel, dim, x, nu, penal, E0, Emin, V) -> np.ndarray:
    """y = K[x] v for each row v of V (all DOFs, no BCs), element by element without assembly:
    y = sum_e E_kappa(x_e) A_e^T K_e0 A_e v (Sec. 2).  For grids too large to assemble cheaply."""
    Ke0 = elements.stiffness_ke0(dim, nu)
    edofs = grid.element_dofs(nel, dim)
    Ek, _, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    n = V.shape[1]
    out = np.zeros_like(V)
    for r in range(V.shape[0]):
        Fe = Ek[:, None] * (V[r][edofs] @ Ke0.T)
        out[r] = np.bincount(edofs.reshape(-1), weights=Fe.reshape(-1), minlength=n)
    return out


def apply_G(nel, dim, x, u, nu, penal, E0, Emin, V) -> np.ndarray:
    """y = G[x, u] v for each row v of V, element by element: sum_e E_sigma(x_e) A_e^T G_e0[u_e] A_e v."""
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    Ge = element_stress_stiffness(nel, dim, u, nu)
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    n = V.shape[1]
    out = np.zeros_like(V)
    for r in range(V.shape[0]):
        Fe = Es[:, None] * np.einsum("mij,mj->mi", Ge, V[r][edofs])
        out[r] = np.bincount(edofs.reshape(-1), weights=Fe.reshape(-1), minlength=n)
    return out
