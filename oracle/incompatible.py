"""Incompatible-mode elements of the paper's Sec. 2 (Wilson's quadrilateral in 2D, the hexahedron
with incompatible modes in 3D), for unit squares / unit cubes, unit modulus, unit thickness in 2D.

Test infrastructure (the plain CPU oracle): nothing outside tests/ and the bench's baseline legs
imports it.

Each displacement component is interpolated by the 2^d nodal bilinear / trilinear functions N_i plus
d internal "bubble" modes P_k = 1 - xi_k^2 (k = 1..d, natural coordinates xi in [-1, 1]^d): 6
functions per component in 2D (the paper's "6-DOF Wilson quadrilateral"), 11 in 3D (the paper's
"11-DOF hexahedron").  The internal amplitudes alpha (d per component) are element-local:

    K_full = sum_gp w |J| B~^T D B~,   B~ = [B_nodal | B_internal],   (2 x 2 (x 2) Gauss)

and static condensation eliminates them: alpha = -K_aa^{-1} K_au u_e, i.e. the element acts on its
nodal DOFs through T = [I ; -K_aa^{-1} K_au]:

    K_c = T^T K_full T = K_uu - K_ua K_aa^{-1} K_au.

The paper does not say how the stress stiffness treats the internal modes.  Reading used here: the
internal modes follow the same static condensation (the standard element-level treatment), so the
Gauss-point stresses come from the enhanced strain B~ [u_e ; alpha(u_e)] and

    G_c[u_e] = T^T G_full[u_e] T,   G_full(i c, j c') = delta_cc' sum_gp w |J| grad F_i . S grad F_j,

with F the 2^d + d interpolation functions of a component.

Local node order, DOF order and Voigt order as in oracle.elements; the internal DOFs are ordered
[alpha_1 (x, y[, z] components), alpha_2 (...), ...] after the nodal ones in K_full / G_full.
"""
from __future__ import annotations

import numpy as np

from . import elements, grid


def _functions_grad(xi: np.ndarray) -> np.ndarray:
    """d F / d x at natural point xi for the 2^d nodal functions then the d bubble modes
    P_k = 1 - xi_k^2 (d/dx = 2 d/dxi on the unit element).  Returns [dim, 2^dim + dim]."""
    dim = xi.size
    dN = elements.shape_gradients(xi)
    dP = np.zeros((dim, dim))
    for k in range(dim):
        dP[k, k] = 2.0 * (-2.0 * xi[k])
    return np.concatenate([dN, dP], axis=1)


def _strain_matrix(dF: np.ndarray) -> np.ndarray:
    """Voigt strain matrix for interpolation functions with gradients dF [dim, nf], DOFs ordered
    function-major, component-minor (the order of oracle.elements.strain_matrix)."""
    return elements.strain_matrix(dF)


def stiffness_full(dim: int, nu: float) -> np.ndarray:
    """K_full [(2^d + d) d]^2 (unit modulus), nodal DOFs first, then the internal ones."""
    D = elements.constitutive(dim, nu)
    pts, wts = elements.gauss_points(dim)
    nf = 2 ** dim + dim
    K = np.zeros((dim * nf, dim * nf))
    for xi, w in zip(pts, wts):
        B = _strain_matrix(_functions_grad(xi))
        K += w * elements.detJ(dim) * B.T @ D @ B
    return K


def condensation(dim: int, nu: float) -> np.ndarray:
    """T [(2^d + d) d, 2^d d]: nodal DOFs -> (nodal DOFs, condensed internal amplitudes)."""
    K = stiffness_full(dim, nu)
    nu_ = dim * 2 ** dim
    Kaa = K[nu_:, nu_:]
    Kau = K[nu_:, :nu_]
    return np.vstack([np.eye(nu_), -np.linalg.solve(Kaa, Kau)])


def stiffness_ke0(dim: int, nu: float) -> np.ndarray:
    """Condensed unit-modulus element stiffness K_c = T^T K_full T (2^d d square)."""
    T = condensation(dim, nu)
    K = T.T @ stiffness_full(dim, nu) @ T
    return 0.5 * (K + K.T)


def stress_at_gauss_points(dim: int, nu: float, ue: np.ndarray) -> np.ndarray:
    """Unit-modulus stresses (Voigt) at the Gauss points from the enhanced strain of u_e."""
    D = elements.constitutive(dim, nu)
    full = condensation(dim, nu) @ np.asarray(ue, dtype=np.float64)
    pts, _ = elements.gauss_points(dim)
    return np.array([D @ _strain_matrix(_functions_grad(xi)) @ full for xi in pts])


def stress_stiffness_ge0(dim: int, nu: float, ue: np.ndarray) -> np.ndarray:
    """Condensed unit-modulus stress stiffness G_c[u_e] = T^T G_full[u_e] T (2^d d square)."""
    pts, wts = elements.gauss_points(dim)
    sig = stress_at_gauss_points(dim, nu, ue)
    nf = 2 ** dim + dim
    Gs = np.zeros((nf, nf))
    for xi, w, s in zip(pts, wts, sig):
        dF = _functions_grad(xi)
        S = elements._stress_tensor(dim, s)
        Gs += w * elements.detJ(dim) * dF.T @ S @ dF
    T = condensation(dim, nu)
    G = T.T @ np.kron(Gs, np.eye(dim)) @ T
    return 0.5 * (G + G.T)


# ------------------------------------------------------------------------------------------------
# assembly (all DOFs, no boundary conditions), Sec. 2: K_e = E_kappa K_c, G_e = E_sigma G_c[u_e]
# ------------------------------------------------------------------------------------------------
def _assemble(nel, dim, Ae):
    import scipy.sparse as sp
    edofs = grid.element_dofs(nel, dim)
    nd = edofs.shape[1]
    rows = np.repeat(edofs, nd, axis=1).reshape(-1)
    cols = np.tile(edofs, (1, nd)).reshape(-1)
    n = dim * grid.num_nodes(nel, dim)
    return sp.coo_matrix((Ae.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()


def assemble_K(nel, dim, x, nu, penal, E0, Emin):
    Kc = stiffness_ke0(dim, nu)
    Ek, _, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    return _assemble(nel, dim, Ek[:, None, None] * Kc[None, :, :])


def assemble_G(nel, dim, x, u, nu, penal, E0, Emin):
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    u = np.asarray(u, dtype=np.float64)
    Ge = np.stack([stress_stiffness_ge0(dim, nu, u[d]) for d in edofs])
    return _assemble(nel, dim, Es[:, None, None] * Ge)


# ------------------------------------------------------------------------------------------------
# buckling analysis and sensitivities with the incompatible-mode elements (Sec. 2 with K_c, G_c)
# ------------------------------------------------------------------------------------------------
def adjoint_element_vector(dim: int, nu: float, phie: np.ndarray) -> np.ndarray:
    """d/du_e of phi_e^T G_c[u_e] phi_e (unit modulus).  With phi~ = T phi_e (nodal and internal
    amplitudes), phi_e^T G_c[u_e] phi_e = sum_gp w |J| sigma(u_e) . h(phi~), where sigma(u_e) =
    D B~ T u_e is the enhanced stress and h the Voigt form (doubled shear) of
    H_ab = sum_c (d_a phi~_c)(d_b phi~_c); so the derivative is sum_gp w |J| (B~ T)^T D h(phi~)."""
    D = elements.constitutive(dim, nu)
    T = condensation(dim, nu)
    pts, wts = elements.gauss_points(dim)
    nf = 2 ** dim + dim
    P = (T @ np.asarray(phie, dtype=np.float64)).reshape(nf, dim)
    out = np.zeros(dim * 2 ** dim)
    for xi, w in zip(pts, wts):
        dF = _functions_grad(xi)
        grad = dF @ P                      # grad[a, c] = d phi~_c / d x_a
        H = grad @ grad.T
        if dim == 2:
            h = np.array([H[0, 0], H[1, 1], 2.0 * H[0, 1]])
        else:
            h = np.array([H[0, 0], H[1, 1], H[2, 2], 2.0 * H[0, 1], 2.0 * H[1, 2], 2.0 * H[2, 0]])
        out += w * elements.detJ(dim) * (_strain_matrix(dF) @ T).T @ D @ h
    return out


def adjoint_rhs(nel, dim, x, phi, nu, penal, E0, Emin) -> np.ndarray:
    """b = phi^T (grad_u G) phi for the condensed elements, full DOF set (eq. AdjointSystem)."""
    edofs = grid.element_dofs(nel, dim)
    _, Es, _, _ = elements.simp(np.asarray(x, dtype=np.float64), penal, E0, Emin)
    phi = np.asarray(phi, dtype=np.float64)
    b = np.zeros(dim * grid.num_nodes(nel, dim))
    for e, d in enumerate(edofs):
        np.add.at(b, d, Es[e] * adjoint_element_vector(dim, nu, phi[d]))
    return b


class Problem:
    """The oracle's problem view (the interface of oracle.lba.Problem: K, Kf, fixed, free, solve,
    to_full, G) with the incompatible-mode elements."""

    def __init__(self, prob):
        import scipy.sparse.linalg as spla
        from . import assembly
        self.p = prob
        self.dim = prob.dim
        self.nel = prob.nel
        self.fixed = np.asarray(prob.fixed, dtype=np.uint8)
        self.free = np.flatnonzero(self.fixed == 0)
        self.n = prob.num_dofs
        self.K = assemble_K(prob.nel, prob.dim, prob.x, prob.nu, prob.penal, prob.E0, prob.Emin)
        self.Kf = assembly.restrict_free(self.K, self.fixed)
        self._splu = spla.splu
        self._lu = None

    def solve(self, B: np.ndarray) -> np.ndarray:
        if self._lu is None:
            self._lu = self._splu(self.Kf.tocsc())
        return self._lu.solve(np.asarray(B, dtype=np.float64))

    def to_full(self, vf: np.ndarray) -> np.ndarray:
        out = np.zeros((self.n,) + vf.shape[1:])
        out[self.free] = vf
        return out

    def G(self, u: np.ndarray):
        p = self.p
        return assemble_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin)


def sensitivities(op: Problem, u, lam, Phi):
    """dlambda/dx [q, m], dJ/dx [m] and the adjoint solutions Z [n, q] with the condensed elements:
    the formula of oracle.sensitivity (eq. SensitivityLambda with the factor -1/(phi^T G phi)) on
    K_c and G_c[u_e]."""
    p = op.p
    dim, nel = p.dim, p.nel
    x = np.asarray(p.x, dtype=np.float64)
    edofs = grid.element_dofs(nel, dim)
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Kc = stiffness_ke0(dim, p.nu)
    Ge = np.stack([stress_stiffness_ge0(dim, p.nu, u[d]) for d in edofs])
    G = op.G(u)
    q = Phi.shape[1]
    B = np.stack([adjoint_rhs(nel, dim, x, Phi[:, i], p.nu, p.penal, p.E0, p.Emin) for i in range(q)], axis=1)
    B[op.fixed == 1] = 0.0
    Z = op.to_full(op.solve(B[op.free]))
    Ue = u[edofs]
    Ku = np.einsum("ij,mj->mi", Kc, Ue)
    dJ = -dEk * np.einsum("mi,mi->m", Ue, Ku)
    dlam = np.zeros((q, x.size))
    for i in range(q):
        ph = Phi[:, i]
        Pe = ph[edofs]
        Ze = Z[:, i][edofs]
        pKp = np.einsum("mi,ij,mj->m", Pe, Kc, Pe)
        pGp = np.einsum("mi,mij,mj->m", Pe, Ge, Pe)
        zKu = np.einsum("mi,mi->m", Ze, Ku)
        dlam[i] = -(dEk * pKp + lam[i] * dEs * pGp - lam[i] * dEk * zKu) / (ph @ (G @ ph))
    return dlam, dJ, Z
