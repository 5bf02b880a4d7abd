"""Element matrices of the bilinear Q4 (plane stress) and trilinear H8 elements.

Paper, Sec. 2: K_e = E_kappa(x_e) K_e0 and G_e = E_sigma(x_e) G_e0[u_e]; the element type here is the
plain Q4 / H8 (the paper's incompatible-mode variants are a different element).  All elements are
unit squares / unit cubes, unit Young's modulus, unit thickness in 2D.

Local node order (natural coordinates xi_i in {-1, +1}):
  Q4: (0,0) (1,0) (1,1) (0,1)
  H8: the Q4 order on z = 0, then the same on z = 1.
Local DOF order: node-interleaved [n1x, n1y, (n1z), n2x, ...].
Voigt order: 2D [xx, yy, xy]; 3D [xx, yy, zz, xy, yz, zx]; engineering shear strains.

Integration: 2 x 2 (x 2) Gauss-Legendre, exact for these bilinear/trilinear fields on a square/cube.
Parity is pinned by tests (symbolic exact integration, rigid-body null spaces, patch tests, the
textbook geometric stiffness for uniform stress).
"""
from __future__ import annotations

import numpy as np

NODES_Q4 = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=np.float64)
NODES_H8 = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
_G = 1.0 / np.sqrt(3.0)


def gauss_points(dim: int):
    """2-point Gauss rule per axis on [-1, 1]: points +-1/sqrt(3), weights 1."""
    pts = np.array([-_G, _G])
    if dim == 2:
        return [np.array([a, b]) for b in pts for a in pts], np.ones(4)
    return [np.array([a, b, c]) for c in pts for b in pts for a in pts], np.ones(8)


def shape_gradients(xi: np.ndarray) -> np.ndarray:
    """d N_i / d x at natural point xi for the unit element (x = (xi + 1) / 2, so d/dx = 2 d/dxi).

    Returns [dim, nnodes]."""
    dim = xi.size
    nodes = NODES_Q4 if dim == 2 else NODES_H8
    nn = nodes.shape[0]
    dN = np.zeros((dim, nn))
    for i in range(nn):
        for a in range(dim):
            v = nodes[i, a] / 2.0 ** dim
            for b in range(dim):
                if b != a:
                    v *= 1.0 + nodes[i, b] * xi[b]
            dN[a, i] = 2.0 * v
    return dN


def detJ(dim: int) -> float:
    """Jacobian determinant of the map from [-1,1]^d to the unit element."""
    return 0.5 ** dim


def constitutive(dim: int, nu: float) -> np.ndarray:
    """Unit-modulus elasticity matrix: plane stress (2D) or isotropic 3D, engineering shear."""
    if dim == 2:
        return np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]]) / (1.0 - nu * nu)
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def strain_matrix(dN: np.ndarray) -> np.ndarray:
    """B such that strain (Voigt, engineering shear) = B u_e."""
    dim, nn = dN.shape
    if dim == 2:
        B = np.zeros((3, 2 * nn))
        for i in range(nn):
            B[0, 2 * i] = dN[0, i]
            B[1, 2 * i + 1] = dN[1, i]
            B[2, 2 * i] = dN[1, i]
            B[2, 2 * i + 1] = dN[0, i]
        return B
    B = np.zeros((6, 3 * nn))
    for i in range(nn):
        B[0, 3 * i] = dN[0, i]
        B[1, 3 * i + 1] = dN[1, i]
        B[2, 3 * i + 2] = dN[2, i]
        B[3, 3 * i] = dN[1, i]          # xy
        B[3, 3 * i + 1] = dN[0, i]
        B[4, 3 * i + 1] = dN[2, i]      # yz
        B[4, 3 * i + 2] = dN[1, i]
        B[5, 3 * i] = dN[2, i]          # zx
        B[5, 3 * i + 2] = dN[0, i]
    return B


def stiffness_ke0(dim: int, nu: float) -> np.ndarray:
    """K_e0 = sum_gp w |J| B^T D B (unit modulus), Sec. 2."""
    D = constitutive(dim, nu)
    pts, wts = gauss_points(dim)
    nd = dim * 2 ** dim
    K = np.zeros((nd, nd))
    for xi, w in zip(pts, wts):
        B = strain_matrix(shape_gradients(xi))
        K += w * detJ(dim) * B.T @ D @ B
    return K


def stress_at_gauss_points(dim: int, nu: float, ue: np.ndarray) -> np.ndarray:
    """Unit-modulus Cauchy stresses (Voigt) at each Gauss point: sigma = D B(gp) u_e.  [ngp, nvoigt]"""
    D = constitutive(dim, nu)
    pts, _ = gauss_points(dim)
    return np.array([D @ strain_matrix(shape_gradients(xi)) @ ue for xi in pts])


def _stress_tensor(dim: int, s: np.ndarray) -> np.ndarray:
    if dim == 2:
        return np.array([[s[0], s[2]], [s[2], s[1]]])
    return np.array([[s[0], s[3], s[5]], [s[3], s[1], s[4]], [s[5], s[4], s[2]]])


def stress_stiffness_ge0(dim: int, nu: float, ue: np.ndarray) -> np.ndarray:
    """G_e0[u_e] (unit modulus), Sec. 2: the geometric (stress) stiffness of the element under the
    Gauss-point stresses of u_e,
        G_e0(i c, j c') = delta_cc' sum_gp w |J| sum_ab dN_i/dx_a S_ab(gp) dN_j/dx_b."""
    pts, wts = gauss_points(dim)
    sig = stress_at_gauss_points(dim, nu, ue)
    nn = 2 ** dim
    Gs = np.zeros((nn, nn))
    for xi, w, s in zip(pts, wts, sig):
        dN = shape_gradients(xi)
        Gs += w * detJ(dim) * dN.T @ _stress_tensor(dim, s) @ dN
    return np.kron(Gs, np.eye(dim))


def adjoint_element_vector(dim: int, nu: float, phie: np.ndarray) -> np.ndarray:
    """d/du_e of phi_e^T G_e0[u_e] phi_e (unit modulus): sum_gp w |J| B^T D h(phi_e), with
    h = Voigt form of H_ab = sum_c (d_a phi_c)(d_b phi_c) with doubled shear entries, because
    phi^T G_e0[u] phi = sum_gp w |J| sigma(u) . h(phi) and sigma(u) = D B u.  This is the element
    part of the adjoint right-hand side phi^T (grad_u G) phi of Sec. 2 (adjoint system)."""
    D = constitutive(dim, nu)
    pts, wts = gauss_points(dim)
    nn = 2 ** dim
    out = np.zeros(dim * nn)
    P = phie.reshape(nn, dim)
    for xi, w in zip(pts, wts):
        dN = shape_gradients(xi)
        grad = dN @ P            # grad[a, c] = d phi_c / d x_a
        H = grad @ grad.T        # H[a, b] = sum_c d_a phi_c d_b phi_c
        if dim == 2:
            h = np.array([H[0, 0], H[1, 1], 2.0 * H[0, 1]])
        else:
            h = np.array([H[0, 0], H[1, 1], H[2, 2], 2.0 * H[0, 1], 2.0 * H[1, 2], 2.0 * H[2, 0]])
        out += w * detJ(dim) * strain_matrix(dN).T @ D @ h
    return out


def simp(x: np.ndarray, penal: float, E0: float, Emin: float):
    """SIMP interpolations of Sec. 2 (paper's E1 -> E0 here, paper's E0 -> Emin):
    E_kappa = Emin + x^p (E0 - Emin), E_sigma = x^p E0, and their derivatives."""
    xp = x ** penal
    dxp = penal * x ** (penal - 1.0)
    return Emin + xp * (E0 - Emin), xp * E0, dxp * (E0 - Emin), dxp * E0
