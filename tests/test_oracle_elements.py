"""Pins of the oracle's element matrices against mathematics independent of its Gauss-quadrature code.

Sec. 2: K_e = E_kappa K_e0, G_e = E_sigma G_e0[u_e].  Pins: exact symbolic integration (SymPy, in
physical coordinates, no quadrature), rigid-body null spaces, the patch test, linearity of G_e0 in u,
the textbook geometric stiffness under uniform uniaxial stress, and the adjoint element vector as the
exact gradient of phi^T G_e0[u] phi.
"""
import itertools

import numpy as np
import pytest
import sympy as sy

from oracle import elements

NU = 0.3


def _sym_shape(dim):
    X = sy.symbols("x y z")[:dim]
    corners = [(0, 0), (1, 0), (1, 1), (0, 1)] if dim == 2 else [
        (0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    N = []
    for c in corners:
        f = sy.Integer(1)
        for a in range(dim):
            f *= X[a] if c[a] == 1 else (1 - X[a])
        N.append(f)
    return X, N


def _sym_integrate(expr, X):
    for x in X:
        expr = sy.integrate(expr, (x, 0, 1))
    return expr


def _sym_D(dim, nu):
    nu = sy.Rational(nu).limit_denominator(1000)
    if dim == 2:
        return sy.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    D = sy.zeros(6, 6)
    for i in range(3):
        for j in range(3):
            D[i, j] = lam
        D[i, i] = lam + 2 * mu
        D[i + 3, i + 3] = mu
    return D


def _sym_B(dim, X, N):
    nn = len(N)
    if dim == 2:
        B = sy.zeros(3, 2 * nn)
        for i, Ni in enumerate(N):
            B[0, 2 * i] = sy.diff(Ni, X[0]); B[1, 2 * i + 1] = sy.diff(Ni, X[1])
            B[2, 2 * i] = sy.diff(Ni, X[1]); B[2, 2 * i + 1] = sy.diff(Ni, X[0])
        return B
    B = sy.zeros(6, 3 * nn)
    for i, Ni in enumerate(N):
        dx, dy, dz = (sy.diff(Ni, v) for v in X)
        B[0, 3 * i] = dx; B[1, 3 * i + 1] = dy; B[2, 3 * i + 2] = dz
        B[3, 3 * i] = dy; B[3, 3 * i + 1] = dx
        B[4, 3 * i + 1] = dz; B[4, 3 * i + 2] = dy
        B[5, 3 * i] = dz; B[5, 3 * i + 2] = dx
    return B


@pytest.mark.parametrize("dim", [2, 3])
def test_ke0_equals_exact_symbolic_integral(dim):
    X, N = _sym_shape(dim)
    B = _sym_B(dim, X, N)
    D = _sym_D(dim, NU)
    integrand = B.T * D * B
    nd = integrand.shape[0]
    Ke = elements.stiffness_ke0(dim, NU)
    # integrate a polynomial matrix entrywise (upper triangle; symmetry checked separately)
    for i in range(nd):
        for j in range(i, nd):
            exact = float(_sym_integrate(sy.expand(integrand[i, j]), X))
            assert Ke[i, j] == pytest.approx(exact, rel=1e-13, abs=1e-14)
    assert np.allclose(Ke, Ke.T, atol=1e-15)


def test_ke0_q4_integer_pattern():
    """At nu = 0.3 the Q4 entries are (1/(80 (1 - nu^2))) x integers (exact symbolic value)."""
    Ke = elements.stiffness_ke0(2, NU) * 80.0 * (1.0 - NU * NU)
    assert np.allclose(Ke, np.round(Ke), atol=1e-12)
    assert np.round(Ke[0]).tolist() == [36, 13, -22, -1, -18, -13, 4, 1]


def _rigid_modes(dim):
    nodes = (elements.NODES_Q4 if dim == 2 else elements.NODES_H8 + 1.0) / 2.0
    nodes = (elements.NODES_Q4 + 1.0) / 2.0 if dim == 2 else (elements.NODES_H8 + 1.0) / 2.0
    nn = nodes.shape[0]
    modes = []
    for c in range(dim):
        t = np.zeros((nn, dim)); t[:, c] = 1.0
        modes.append(t.reshape(-1))
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (2, 0)]
    for a, b in pairs:
        r = np.zeros((nn, dim))
        r[:, a] = -nodes[:, b]
        r[:, b] = nodes[:, a]
        modes.append(r.reshape(-1))
    return np.array(modes).T


@pytest.mark.parametrize("dim,rank", [(2, 5), (3, 18)])
def test_ke0_null_space_is_rigid_body(dim, rank):
    Ke = elements.stiffness_ke0(dim, NU)
    R = _rigid_modes(dim)
    assert np.abs(Ke @ R).max() < 1e-13
    ev = np.linalg.eigvalsh(Ke)
    assert (ev > -1e-13).all()
    assert int((ev > 1e-10).sum()) == rank


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_linear_field(dim):
    """A 3 x 3 (x 3) patch of unit elements under a linear displacement field: interior nodes carry
    zero net force (the element represents constant strain exactly)."""
    from oracle import assembly, grid
    nel = (3, 3, 3) if dim == 3 else (3, 3, 1)
    K = assembly.assemble_K(nel, dim, np.ones(int(np.prod(nel[:dim]))), NU, 3.0, 1.0, 1e-6).toarray()
    nd = grid.node_dims(nel, dim)
    coords = np.array(list(itertools.product(*[range(n) for n in reversed(nd)])), dtype=float)[:, ::-1]
    rng = np.random.default_rng(5)
    A = rng.standard_normal((dim, dim))
    u = (coords @ A.T).reshape(-1)
    f = K @ u
    interior = np.all((coords > 0) & (coords < np.array(nd) - 1), axis=1)
    idx = (dim * np.flatnonzero(interior)[:, None] + np.arange(dim)).reshape(-1)
    assert np.abs(f[idx]).max() < 1e-12
    assert np.abs(f).max() > 1e-3


@pytest.mark.parametrize("dim", [2, 3])
def test_ge0_symmetric_linear_rigid(dim):
    rng = np.random.default_rng(1)
    nd = dim * 2 ** dim
    u1, u2 = rng.standard_normal(nd), rng.standard_normal(nd)
    G1 = elements.stress_stiffness_ge0(dim, NU, u1)
    G2 = elements.stress_stiffness_ge0(dim, NU, u2)
    G12 = elements.stress_stiffness_ge0(dim, NU, 2.0 * u1 - 3.0 * u2)
    assert np.allclose(G1, G1.T, atol=1e-14)
    assert np.allclose(G12, 2.0 * G1 - 3.0 * G2, atol=1e-13)
    for r in _rigid_modes(dim).T:
        assert np.abs(elements.stress_stiffness_ge0(dim, NU, r)).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_ge0_uniform_uniaxial_stress_textbook(dim):
    """Under uniform sigma_xx = s (all other stresses zero) the geometric stiffness is
    s * int (dN/dx)^T (dN/dx) dV (x) I_d, integrated exactly with SymPy."""
    # displacement giving a uniform uniaxial stress: eps = D^{-1} [s, 0, ...]
    D = elements.constitutive(dim, NU)
    nv = D.shape[0]
    sig = np.zeros(nv); sig[0] = 0.7
    eps = np.linalg.solve(D, sig)
    nodes = (elements.NODES_Q4 + 1.0) / 2.0 if dim == 2 else (elements.NODES_H8 + 1.0) / 2.0
    Gm = np.diag(eps[:dim])
    u = (nodes @ Gm.T).reshape(-1)                # normal strains only
    Ge = elements.stress_stiffness_ge0(dim, NU, u)
    X, N = _sym_shape(dim)
    nn = len(N)
    M = np.zeros((nn, nn))
    for i in range(nn):
        for j in range(nn):
            M[i, j] = float(_sym_integrate(sy.expand(sy.diff(N[i], X[0]) * sy.diff(N[j], X[0])), X))
    assert np.allclose(Ge, 0.7 * np.kron(M, np.eye(dim)), atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_element_vector_is_gradient(dim):
    """d/du_k (phi^T G_e0[u] phi) = phi^T G_e0[e_k] phi because G_e0 is linear in u."""
    rng = np.random.default_rng(2)
    nd = dim * 2 ** dim
    phi = rng.standard_normal(nd)
    g = elements.adjoint_element_vector(dim, NU, phi)
    brute = np.array([phi @ elements.stress_stiffness_ge0(dim, NU, np.eye(nd)[k]) @ phi for k in range(nd)])
    assert np.allclose(g, brute, rtol=1e-13, atol=1e-14)


def test_simp_interpolation():
    x = np.array([0.0, 0.3, 1.0])
    Ek, Es, dEk, dEs = elements.simp(x, 3.0, 1.0, 1e-6)
    assert np.allclose(Ek, [1e-6, 1e-6 + 0.027 * (1 - 1e-6), 1.0])
    assert np.allclose(Es, [0.0, 0.027, 1.0])
    h = 1e-7
    for k in range(1, 3):
        e1 = elements.simp(x[k:k + 1] + h, 3.0, 1.0, 1e-6)
        e0 = elements.simp(x[k:k + 1] - h, 3.0, 1.0, 1e-6)
        assert (e1[0] - e0[0]) / (2 * h) == pytest.approx(dEk[k], rel=1e-7)
        assert (e1[1] - e0[1]) / (2 * h) == pytest.approx(dEs[k], rel=1e-7)
