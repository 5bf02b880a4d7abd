"""Consistent sensitivities of the multilevel buckling load factors (Sec. 2.1, eq. eigResidual;
Appendix A, eq. consistentSensitivity).

Test infrastructure: a plain FP64 statement of what the GPU path computes, called only by the tests and
the benchmark's CPU baseline.

The multilevel load factor of a mode depends on the densities x through the steps of Sec. 2.1:

    u = K^{-1} f,   G = G[x, u]                              (Algorithm 1 step 2; Sec. 2)
    K^l = P^T K P,  G^l = P^T G P                             (P: free interpolations Omega_l -> Omega_1)
    (K^l + mu G^l) psi = 0                                    (coarse pair, eq. eigenvalueProblemCoarseScale)
    Psi = P psi,    K phi = G Psi                             (eq. FineScaleBVP)
    lambda = -phi^T K phi / phi^T G phi                       (eq. FineScaleRQ)

and (lambda, phi) leaves the residual y = (K + lambda G) phi of eq. eigResidual.  lambda does not change
when psi is scaled, so the normalisation of the coarse mode drops out of its derivative.  With
D = -1/(phi^T G phi) the gradient of the Rayleigh quotient in phi is 2 D y, and the chain rule through
the steps above gives, for a change dK, dG of the operators (dG the total change of G[x, u(x)],
including the one through u):

    d lambda = D phi^T (dK + lambda dG) phi + 2 D y^T d phi,
    K d phi  = dG Psi + G P d psi - dK phi,
    (K^l + mu G^l) d psi = -(P^T dK P + d mu G^l + mu P^T dG P) psi.

Two adjoint systems remove d phi and d psi:

    K w = y                                                   (fine, symmetric positive definite)
    (K^l + mu G^l) c = b,  psi^T G^l c = 0,  b = P^T G w      (coarse; psi^T b = y^T phi = 0, so the
                                                               singular system is consistent)

so that 2 y^T d phi = 2 w^T (dG Psi - dK phi) - 2 (P c)^T (dK + mu dG) Psi (the constraint on c removes
d mu).  The part of dG that comes through u, G[x, du] with K du = -dK u, is a linear functional of du;
with K z = g, g = grad_v [lambda phi^T G[v] phi + (2 w - 2 mu P c)^T G[v] Psi] (the u-adjoint of
eq. AdjointSystem with a combined right-hand side) it becomes -z^T dK u.  Per element e (K_e0 and
G_e0[u_e] of unit modulus, dE_kappa and dE_sigma the SIMP derivatives):

    d lambda / d x_e = D { dE_kappa [ (phi - 2 w)^T K_e0 phi - 2 (P c)^T K_e0 Psi - z^T K_e0 u ]
                         + dE_sigma [ lambda phi^T G_e0 phi + (2 w - 2 mu P c)^T G_e0 Psi ] }.

With w = 0 and c = 0 this is eq. SensitivityLambda (its adjoint z then being lambda times that of
eq. AdjointSystem).

The printed eq. consistentSensitivity is the same derivative written with the adjoint
p = -2 (K + lambda G)^{-1} y of the residual: for phi scaled to phi^T G phi = -1 (so D = 1), and with
every derivative in it total (dG through u as well, and d y / d x_e the total change of the residual
along the method), it holds identically.  `paper_formula` evaluates that form on tiny grids, where
d y / d x_e comes from the forward (direct) differentiation of the same steps (`forward_derivative`),
and the tests check it against the adjoint form above and both against central differences of the
multilevel load factors.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import assembly, elements, grid, lba


def adjoint_rhs_pair(nel, dim, x, a, c, nu, penal, E0, Emin) -> np.ndarray:
    """g = grad_v (a^T G[x, v] c) on the full DOF set (G is linear in v, Sec. 2).

    a^T G_e0[v] c = sum_gp w|J| sum_ij S_ij(v) H_ij with H_ij = sum_k (d_i a_k)(d_j c_k) and S(v) the
    Gauss-point stress of v; S is symmetric, so in Voigt form S : H = sigma . h with
    h = (H_00, H_11, H_01 + H_10) in 2D and (H_00, H_11, H_22, H_01 + H_10, H_12 + H_21, H_20 + H_02) in
    3D, and sigma = D B v gives the element gradient sum_gp w|J| B^T D h.  For a = c it is the
    right-hand side of eq. AdjointSystem."""
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    Ae = np.asarray(a, dtype=np.float64)[edofs]
    Ce = np.asarray(c, dtype=np.float64)[edofs]
    D = elements.constitutive(dim, nu)
    pts, wts = elements.gauss_points(dim)
    nn = 2 ** dim
    ge = np.zeros_like(Ae)
    for xi, w in zip(pts, wts):
        dN = elements.shape_gradients(xi)
        ga = np.einsum("ai,mic->mac", dN, Ae.reshape(-1, nn, dim))     # d a_k / d x_i   [m, i, k]
        gc = np.einsum("ai,mic->mac", dN, Ce.reshape(-1, nn, dim))
        H = np.einsum("mik,mjk->mij", ga, gc)
        if dim == 2:
            h = np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 0, 1] + H[:, 1, 0]], axis=1)
        else:
            h = np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], H[:, 0, 1] + H[:, 1, 0],
                          H[:, 1, 2] + H[:, 2, 1], H[:, 2, 0] + H[:, 0, 2]], axis=1)
        BtD = elements.strain_matrix(dN).T @ D
        ge += w * elements.detJ(dim) * h @ BtD.T
    g = np.zeros(dim * grid.num_nodes(nel, dim))
    np.add.at(g, edofs.reshape(-1), (Es[:, None] * ge).reshape(-1))
    return g


def interpolation_chain(Ps) -> sp.csr_matrix | None:
    """P = P_1 P_2 ... P_{l-1}: free DOFs of Omega_l -> free DOFs of Omega_1 (None for l = 1)."""
    P = None
    for Pj in Ps:
        P = Pj if P is None else (P @ Pj).tocsr()
    return P


def multilevel_pairs(op: lba.Problem, u: np.ndarray, q: int, eig_level: int, dense_limit: int = 4000):
    """Sec. 2.1 steps 1-4 in the coarse modes' order, without normalising or sorting the fine modes:
    phi_i = K^{-1} G P psi_i exactly, so that the chain rule applies column by column.  Free DOFs."""
    G = op.G(u)
    Gf = assembly.restrict_free(G, op.fixed)
    Kl, Gl, Ps, _, _ = lba.galerkin_levels(op, Gf, eig_level)
    mu, psi = lba.buckling_pencil(Kl, Gl, q, dense_limit)
    P = interpolation_chain(Ps)
    Psi = psi if P is None else P @ psi
    Phi = op.solve(Gf @ Psi)
    KPhi = op.Kf @ Phi
    GPhi = Gf @ Phi
    lam = -np.einsum("ij,ij->j", Phi, KPhi) / np.einsum("ij,ij->j", Phi, GPhi)
    Y = KPhi + GPhi * lam[None, :]
    return dict(G=G, Gf=Gf, Kl=Kl, Gl=Gl, P=P, mu=mu, psi=psi, Psi=Psi, Phi=Phi, lam=lam, Y=Y)


def _bordered_solve(A: np.ndarray, v: np.ndarray, B: np.ndarray) -> np.ndarray:
    """x with A x = B and v^T x = 0, from the bordered system [[A, v], [v^T, 0]] (A singular along the
    null vector that v is not orthogonal to)."""
    n = A.shape[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A
    M[:n, n] = v
    M[n, :n] = v
    rhs = np.zeros(n + 1)
    rhs[:n] = B
    return sla.solve(M, rhs)[:n]


def consistent_sensitivities(op: lba.Problem, u: np.ndarray, q: int, eig_level: int, dense_limit: int = 4000):
    """d lambda_i / d x [q, m] of the multilevel load factors by the adjoint chain of the module
    docstring, rows in ascending order of lambda (the order of lba.multilevel_lba).  Also returns the
    adjoint fields (full DOF set, same order, each mode's vectors on the scale of phi = K^{-1} G Psi):
    W (fine adjoint), Chat = P c (coarse adjoint on Omega_1), Z (u-adjoint) and the residuals Y."""
    p = op.p
    dim, nel = p.dim, p.nel
    x = np.asarray(p.x, dtype=np.float64)
    edofs = grid.element_dofs(nel, dim)
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Ke0 = elements.stiffness_ke0(dim, p.nu)
    Ge = assembly.element_stress_stiffness(nel, dim, u, p.nu)
    mp = multilevel_pairs(op, u, q, eig_level, dense_limit)
    Gf, Kl, Gl, P = mp["Gf"], mp["Kl"], mp["Gl"], mp["P"]
    Kld, Gld = Kl.toarray(), Gl.toarray()
    W = op.solve(mp["Y"])                                               # K w = y
    B = Gf @ W
    if P is not None:
        B = P.T @ B                                                     # b = P^T G w
    Cc = np.zeros((Kld.shape[0], q))
    for i in range(q):
        ps = mp["psi"][:, i]
        Cc[:, i] = _bordered_solve(Kld + mp["mu"][i] * Gld, Gld @ ps, B[:, i])
    Chat = Cc if P is None else P @ Cc
    Psi, Phi, lam, mu = mp["Psi"], mp["Phi"], mp["lam"], mp["mu"]
    Ufull = np.asarray(u, dtype=np.float64)
    Zg = np.zeros((op.n, q))
    for i in range(q):
        a = op.to_full(2.0 * W[:, i] - 2.0 * mu[i] * Chat[:, i])
        ph = op.to_full(Phi[:, i])
        g = lam[i] * adjoint_rhs_pair(nel, dim, x, ph, ph, p.nu, p.penal, p.E0, p.Emin)
        g += adjoint_rhs_pair(nel, dim, x, a, op.to_full(Psi[:, i]), p.nu, p.penal, p.E0, p.Emin)
        Zg[:, i] = g
    Z = op.to_full(op.solve(Zg[op.free]))
    Ue = Ufull[edofs]
    Ku = np.einsum("ij,mj->mi", Ke0, Ue)
    dlam = np.zeros((q, x.size))
    for i in range(q):
        ph = op.to_full(Phi[:, i])[edofs]
        we = op.to_full(W[:, i])[edofs]
        ce = op.to_full(Chat[:, i])[edofs]
        Pe = op.to_full(Psi[:, i])[edofs]
        ze = Z[:, i][edofs]
        Dm = -1.0 / (Phi[:, i] @ (Gf @ Phi[:, i]))
        kpart = (np.einsum("mi,ij,mj->m", ph - 2.0 * we, Ke0, ph)
                 - 2.0 * np.einsum("mi,ij,mj->m", ce, Ke0, Pe)
                 - np.einsum("mi,mi->m", ze, Ku))
        ae = 2.0 * we - 2.0 * mu[i] * ce
        gpart = (lam[i] * np.einsum("mi,mij,mj->m", ph, Ge, ph)
                 + np.einsum("mi,mij,mj->m", ae, Ge, Pe))
        dlam[i] = Dm * (dEk * kpart + dEs * gpart)
    order = np.argsort(lam)
    full = lambda M: op.to_full(M[:, order])
    return dlam[order], dict(lam=lam[order], W=full(W), Chat=full(Chat), Z=Z[:, order], Y=full(mp["Y"]),
                             Phi=full(Phi), Psi=full(Psi), mu=mu[order], order=order)


def _element_operator(op: lba.Problem, e: int, Ae: np.ndarray) -> sp.csr_matrix:
    """The global matrix of one element's nd x nd block Ae, restricted to the free DOFs."""
    edofs = grid.element_dofs(op.nel, op.dim)[e]
    nd = edofs.size
    M = sp.coo_matrix((Ae.reshape(-1), (np.repeat(edofs, nd), np.tile(edofs, nd))), shape=(op.n, op.n))
    return assembly.restrict_free(M, op.fixed)


def forward_derivative(op: lba.Problem, u: np.ndarray, mp: dict, e: int):
    """Direct (forward) differentiation of the steps of Sec. 2.1 with respect to x_e, for the pairs of
    `multilevel_pairs` (coarse order): returns d lambda [q] and the total change of the residual
    d y [nf, q] and of phi, d phi [nf, q] (free DOFs)."""
    p = op.p
    x = np.asarray(p.x, dtype=np.float64)
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Ke0 = elements.stiffness_ke0(p.dim, p.nu)
    Ge = assembly.element_stress_stiffness(p.nel, p.dim, u, p.nu)
    dK = dEk[e] * _element_operator(op, e, Ke0)
    du = op.to_full(-op.solve(dK @ np.asarray(u)[op.free]))
    dG = dEs[e] * _element_operator(op, e, Ge[e]) + assembly.restrict_free(op.G(du), op.fixed)
    P = mp["P"]
    dKl = dK if P is None else P.T @ dK @ P
    dGl = dG if P is None else P.T @ dG @ P
    Kld, Gld = mp["Kl"].toarray(), mp["Gl"].toarray()
    dKl = dKl.toarray() if sp.issparse(dKl) else dKl
    dGl = dGl.toarray() if sp.issparse(dGl) else dGl
    Gf, Kf = mp["Gf"], op.Kf
    q = mp["lam"].size
    dlam = np.zeros(q)
    dY = np.zeros_like(mp["Y"])
    dPhi = np.zeros_like(mp["Phi"])
    for i in range(q):
        ps, m = mp["psi"][:, i], mp["mu"][i]
        dmu = -(ps @ (dKl @ ps) + m * (ps @ (dGl @ ps))) / (ps @ (Gld @ ps))
        dps = _bordered_solve(Kld + m * Gld, Gld @ ps, -(dKl @ ps + dmu * (Gld @ ps) + m * (dGl @ ps)))
        dPs = dps if P is None else P @ dps
        ph, Ps, lam = mp["Phi"][:, i], mp["Psi"][:, i], mp["lam"][i]
        dph = op.solve(dG @ Ps + Gf @ dPs - dK @ ph)
        Dm = -1.0 / (ph @ (Gf @ ph))
        y = mp["Y"][:, i]
        dl = Dm * (ph @ (dK @ ph) + lam * (ph @ (dG @ ph))) + 2.0 * Dm * (y @ dph)
        dlam[i] = dl
        dPhi[:, i] = dph
        dY[:, i] = dK @ ph + dl * (Gf @ ph) + lam * (dG @ ph) + Kf @ dph + lam * (Gf @ dph)
    return dlam, dY, dPhi


def paper_formula(op: lba.Problem, u: np.ndarray, mp: dict, e: int, dY: np.ndarray, use_p: bool = True):
    """eq. consistentSensitivity for the pairs of `multilevel_pairs`, element e, with phi scaled to
    phi^T G phi = -1 (the normalisation under which the printed form carries no factor D), the
    u-dependence of G through the adjoint z of eq. AdjointSystem in the first bracket, and d y / d x_e
    the given total change of the residual (of the unscaled phi; it is scaled with phi).  Every
    derivative in the p-terms is total.  use_p = False sets p = 0, which leaves eq. SensitivityLambda."""
    p = op.p
    x = np.asarray(p.x, dtype=np.float64)
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Ke0 = elements.stiffness_ke0(p.dim, p.nu)
    Ge = assembly.element_stress_stiffness(p.nel, p.dim, u, p.nu)
    dK = dEk[e] * _element_operator(op, e, Ke0)
    dGx = dEs[e] * _element_operator(op, e, Ge[e])
    du = op.to_full(-op.solve(dK @ np.asarray(u)[op.free]))
    dG = dGx + assembly.restrict_free(op.G(du), op.fixed)
    Gf, Kf = mp["Gf"], op.Kf
    uf = np.asarray(u)[op.free]
    q = mp["lam"].size
    out = np.zeros(q)
    for i in range(q):
        lam = mp["lam"][i]
        s = np.sqrt(-(mp["Phi"][:, i] @ (Gf @ mp["Phi"][:, i])))
        ph = mp["Phi"][:, i] / s
        y = (Kf @ ph) + lam * (Gf @ ph)
        dy = dY[:, i] / s
        phf = op.to_full(ph)
        g = adjoint_rhs_pair(p.nel, p.dim, x, phf, phf, p.nu, p.penal, p.E0, p.Emin)[op.free]
        z = op.solve(g)
        first = ph @ ((dK + lam * dGx) @ ph) - lam * (z @ (dK @ uf))
        if use_p:
            pv = -2.0 * np.linalg.solve((Kf + lam * Gf).toarray(), y)
            out[i] = (first + pv @ ((dK + lam * dG) @ ph) - pv @ dy) / (1.0 - pv @ (Gf @ ph))
        else:
            out[i] = first
    return out
