"""Adjoint systems and sensitivities of the buckling load factors and of the compliance (Sec. 2).

With phi^T K phi = 1 and lambda = -phi^T K phi / phi^T G phi (eq. minBLFcharRayleigh), differentiating
the Rayleigh quotient with u = u(x) gives

   d lambda / d x_e = -[ phi^T K' phi + lambda phi^T G' phi - lambda z^T K' u ] / (phi^T G phi),
   K z = phi^T (grad_u G) phi                                   (eq. AdjointSystem),

with K' = dE_kappa/dx_e K_e0 and G' = dE_sigma/dx_e G_e0[u_e] acting on element e only.  The bracket is
the one of eq. SensitivityLambda; that equation omits the factor -1/(phi^T G phi), which equals
lambda under the stated K-normalisation (it is 1 only when phi^T G phi = -1), so the factor is kept.
Compliance: dJ/dx_e = -dE_kappa/dx_e u_e^T K_e0 u_e.
"""
from __future__ import annotations

import numpy as np

from . import assembly, elements, grid


def adjoint_rhs(nel, dim, x, phi, nu, penal, E0, Emin) -> np.ndarray:
    """b = phi^T (grad_u G) phi: b_k = sum_e E_sigma(x_e) d/du_k (phi_e^T G_e0[u_e] phi_e), full DOF set."""
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    Pe = np.asarray(phi)[edofs]                                     # [m, nd]
    D = elements.constitutive(dim, nu)
    pts, wts = elements.gauss_points(dim)
    nn = 2 ** dim
    be = np.zeros_like(Pe)
    for xi, w in zip(pts, wts):
        dN = elements.shape_gradients(xi)
        grad = np.einsum("ai,mic->mac", dN, Pe.reshape(-1, nn, dim))   # d phi_c / d x_a
        H = np.einsum("mac,mbc->mab", grad, grad)
        if dim == 2:
            h = np.stack([H[:, 0, 0], H[:, 1, 1], 2.0 * H[:, 0, 1]], axis=1)
        else:
            h = np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], 2.0 * H[:, 0, 1],
                          2.0 * H[:, 1, 2], 2.0 * H[:, 2, 0]], axis=1)
        BtD = elements.strain_matrix(dN).T @ D
        be += w * elements.detJ(dim) * h @ BtD.T
    b = np.zeros(dim * grid.num_nodes(nel, dim))
    np.add.at(b, edofs.reshape(-1), (Es[:, None] * be).reshape(-1))
    return b


def sensitivities(op, u, lam, Phi):
    """dlambda/dx [q, m], dJ/dx [m] and the adjoint solutions Z [n, q] (full DOF set)."""
    p = op.p
    dim, nel = p.dim, p.nel
    x = np.asarray(p.x, dtype=np.float64)
    edofs = grid.element_dofs(nel, dim)
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Ke0 = elements.stiffness_ke0(dim, p.nu)
    Ge = assembly.element_stress_stiffness(nel, dim, u, p.nu)       # unit-modulus G_e0[u_e]
    G = op.G(u)
    q = Phi.shape[1]
    B = np.stack([adjoint_rhs(nel, dim, x, Phi[:, i], p.nu, p.penal, p.E0, p.Emin) for i in range(q)],
                 axis=1)
    B[op.fixed == 1] = 0.0
    Z = op.to_full(op.solve(B[op.free]))
    Ue = u[edofs]
    Ku = np.einsum("ij,mj->mi", Ke0, Ue)
    dJ = -dEk * np.einsum("mi,mi->m", Ue, Ku)
    dlam = np.zeros((q, x.size))
    for i in range(q):
        ph = Phi[:, i]
        Pe = ph[edofs]
        Ze = Z[:, i][edofs]
        pKp = np.einsum("mi,ij,mj->m", Pe, Ke0, Pe)
        pGp = np.einsum("mi,mij,mj->m", Pe, Ge, Pe)
        zKu = np.einsum("mi,mi->m", Ze, Ku)
        phiGphi = ph @ (G @ ph)
        dlam[i] = -(dEk * pKp + lam[i] * dEs * pGp - lam[i] * dEk * zKu) / phiGphi
    return dlam, dJ, Z
