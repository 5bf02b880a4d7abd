"""Pins of the oracle's incompatible-mode elements (oracle/incompatible.py; the paper's Sec. 2
Wilson quadrilateral and incompatible-mode hexahedron): rigid-body null space and rank, constant
strain (patch) behaviour identical to Q4 / H8, exact pure-bending energy (the closed form the
incompatible modes exist for), the closed form of the 2D condensed stiffness, and the Euler column."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import elements, incompatible, lba

NU = 0.3


def _rigid_modes(dim):
    X = (elements.NODES_Q4 if dim == 2 else elements.NODES_H8 + 0.0) * 0.5  # node coordinates, centred
    modes = []
    for c in range(dim):  # translations
        m = np.zeros((X.shape[0], dim))
        m[:, c] = 1.0
        modes.append(m.reshape(-1))
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (1, 2), (2, 0)]
    for a, b in pairs:  # infinitesimal rotations
        m = np.zeros((X.shape[0], dim))
        m[:, a] = -X[:, b]
        m[:, b] = X[:, a]
        modes.append(m.reshape(-1))
    return np.array(modes).T


def _linear_fields(dim):
    """Nodal values of the 3 (2D) / 6 (3D) independent constant-strain displacement fields."""
    X = (elements.NODES_Q4 if dim == 2 else elements.NODES_H8 + 0.0) * 0.5
    out = []
    for a in range(dim):
        for b in range(a, dim):
            m = np.zeros((X.shape[0], dim))
            m[:, a] += X[:, b]
            if a != b:
                m[:, b] += X[:, a]
            out.append(m.reshape(-1))
    return np.array(out).T


@pytest.mark.parametrize("dim,rank", [(2, 5), (3, 18)])
def test_condensed_stiffness_rank_and_rigid_null_space(dim, rank):
    K = incompatible.stiffness_ke0(dim, NU)
    assert np.allclose(K, K.T, atol=1e-14)
    w = np.linalg.eigvalsh(K)
    assert np.all(w > -1e-12)
    assert int(np.sum(w > 1e-10 * w.max())) == rank
    R = _rigid_modes(dim)
    assert np.abs(K @ R).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_strain_is_untouched_by_the_internal_modes(dim):
    """The bubble modes have zero mean gradient, so a constant strain does not excite them
    (alpha = 0) and the element acts on it exactly like Q4 / H8: the patch test carries over."""
    L = _linear_fields(dim)
    Kc = incompatible.stiffness_ke0(dim, NU)
    Kp = elements.stiffness_ke0(dim, NU)
    assert np.allclose(Kc @ L, Kp @ L, atol=1e-13)
    T = incompatible.condensation(dim, NU)
    assert np.abs((T @ L)[dim * 2 ** dim:]).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_pure_bending_energy_is_exact(dim):
    """Pure bending with curvature kappa, sigma_xx = E kappa t (t = y in 2D, z in 3D), all other
    stresses zero: the field lies in the enhanced space, so the condensed element energy equals the
    exact strain energy E kappa^2 / 24 of the unit element; plain Q4 / H8 lock (larger energy)."""
    kappa = 0.37
    X = (elements.NODES_Q4 if dim == 2 else elements.NODES_H8 + 0.0) * 0.5
    if dim == 2:
        x, y = X[:, 0], X[:, 1]
        ue = np.stack([kappa * x * y, -kappa * (x ** 2 + NU * y ** 2) / 2.0], axis=1).reshape(-1)
    else:
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        ue = np.stack([kappa * x * z, -NU * kappa * y * z, -kappa * (x ** 2 + NU * z ** 2 - NU * y ** 2) / 2.0],
                      axis=1).reshape(-1)
    exact = kappa ** 2 / 24.0
    Uc = 0.5 * ue @ incompatible.stiffness_ke0(dim, NU) @ ue
    Up = 0.5 * ue @ elements.stiffness_ke0(dim, NU) @ ue
    assert Uc == pytest.approx(exact, rel=1e-12)
    assert Up > 1.2 * exact


def test_2d_condensed_stiffness_closed_form():
    """For the unit square, condensation changes only the two hourglass energies: from
    (D11 + D33)/12 per squared hourglass amplitude h (u0 - u1 + u2 - u3, same for v) in Q4 to the
    bending modulus (D11 - D12^2/D22)/12, i.e. K_Q4 - K_c = c (g_u g_u^T + g_v g_v^T) with
    c = (D11 + D33 - D11 + D12^2/D22)/12 and g the hourglass pattern."""
    D = elements.constitutive(2, NU)
    c = (D[2, 2] + D[0, 1] ** 2 / D[1, 1]) / 12.0
    gu = np.zeros(8)
    gu[0::2] = [1.0, -1.0, 1.0, -1.0]
    gv = np.zeros(8)
    gv[1::2] = [1.0, -1.0, 1.0, -1.0]
    diff = elements.stiffness_ke0(2, NU) - incompatible.stiffness_ke0(2, NU)
    assert np.allclose(diff, c * (np.outer(gu, gu) + np.outer(gv, gv)), atol=1e-14)


@pytest.mark.parametrize("nu", [0.2, 0.3, 0.45])
def test_3d_condensed_stiffness_closed_form(nu):
    """For the unit cube, condensation changes the energy only on three pairs of bilinear Walsh
    patterns (u xy with w yz, v xy with w zx, v yz with u zx; s_S = product of the node's corner
    signs over the axes in S): K_H8 - K_c = (1/64) sum over the pairs of a (v1 v1^T + v2 v2^T) +
    b (v1 v2^T + v2 v1^T), a = (4/3)(mu + lambda^2/(lambda + 2 mu)), b = (4/3) lambda^2/(lambda + 2 mu);
    the trilinear (xyz) mode and the other bilinear patterns keep their H8 energy."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    a = 4.0 / 3.0 * (mu + lam ** 2 / (lam + 2 * mu))
    b = 4.0 / 3.0 * lam ** 2 / (lam + 2 * mu)
    X = elements.NODES_H8
    pat = {"xy": X[:, 0] * X[:, 1], "yz": X[:, 1] * X[:, 2], "zx": X[:, 2] * X[:, 0]}

    def vec(S, c):
        v = np.zeros(24)
        v[c::3] = pat[S]
        return v

    F = np.zeros((24, 24))
    for (s1, c1), (s2, c2) in [(("xy", 0), ("yz", 2)), (("xy", 1), ("zx", 2)), (("yz", 1), ("zx", 0))]:
        v1, v2 = vec(s1, c1), vec(s2, c2)
        F += (a * (np.outer(v1, v1) + np.outer(v2, v2)) + b * (np.outer(v1, v2) + np.outer(v2, v1))) / 64.0
    diff = elements.stiffness_ke0(3, nu) - incompatible.stiffness_ke0(3, nu)
    assert np.allclose(diff, F, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_condensed_stress_stiffness_invariants(dim):
    rng = np.random.default_rng(3)
    nd = dim * 2 ** dim
    u1, u2 = rng.standard_normal(nd), rng.standard_normal(nd)
    G1 = incompatible.stress_stiffness_ge0(dim, NU, u1)
    G2 = incompatible.stress_stiffness_ge0(dim, NU, u2)
    G12 = incompatible.stress_stiffness_ge0(dim, NU, 2.0 * u1 - 3.0 * u2)
    assert np.allclose(G1, G1.T, atol=1e-14)
    assert np.allclose(G12, 2.0 * G1 - 3.0 * G2, atol=1e-12)          # linear in u_e
    for r in _rigid_modes(dim).T:                                        # no stress, no G
        assert np.abs(incompatible.stress_stiffness_ge0(dim, NU, r)).max() < 1e-13


def test_euler_column_with_incompatible_modes():
    """The clamped-free Euler column of the Q4 pin (width w, length 40 w, total top load 1, uniform
    solid): with the bending-exact element the first load factor is within 0.1 % of the Euler load
    already at 4 elements across (measured 0.01 %; Q4: 3.0 %), and closer than Q4 at every
    resolution (8 across: 0.02 % vs 0.74 %)."""
    errs_c, errs_p = [], []
    for across in (4, 8):
        L = 40 * across
        p = synthetic.column_2d(L, across, seed=0, radius=1, x=np.ones(L * across))
        exact = np.pi ** 2 * (across ** 3 / 12.0) / (4.0 * L ** 2)
        fixed = np.asarray(p.fixed, dtype=np.uint8)
        free = np.flatnonzero(fixed == 0)
        for assemble, errs in ((incompatible, errs_c), (None, errs_p)):
            if assemble is None:
                op = lba.Problem(p)
                u, _ = lba.linear_analysis(op)
                Kf = op.Kf
                G = op.G(u)
            else:
                K = incompatible.assemble_K(p.nel, 2, p.x, p.nu, p.penal, p.E0, p.Emin)
                Kf = K[free][:, free].tocsc()
                u = np.zeros(p.num_dofs)
                u[free] = spla.spsolve(Kf, np.asarray(p.f)[free])
                G = incompatible.assemble_G(p.nel, 2, p.x, u, p.nu, p.penal, p.E0, p.Emin)
            Gf = G[free][:, free]
            lam, _ = lba.buckling_pencil(Kf, Gf, 1, dense_limit=3000)
            errs.append(lam[0] / exact - 1.0)
    assert abs(errs_c[0]) < 1e-3
    assert all(abs(c) < abs(q) for c, q in zip(errs_c, errs_p))
    assert abs(errs_c[1]) < abs(errs_c[0]) + 1e-4


def test_adjoint_rhs_is_the_derivative_of_phi_G_phi():
    """b . w = d/dt phi^T G[u + t w] phi (G is linear in u, so the central difference is exact up to
    rounding), with the condensed elements."""
    p = synthetic.column_2d(6, 4, seed=10, radius=1.5)
    op = incompatible.Problem(p)
    u = op.to_full(op.solve(np.asarray(p.f)[op.free]))
    rng = np.random.default_rng(11)
    phi, w = rng.standard_normal(p.num_dofs), rng.standard_normal(p.num_dofs)
    b = incompatible.adjoint_rhs(p.nel, 2, p.x, phi, p.nu, p.penal, p.E0, p.Emin)
    t = 1e-3
    gp = phi @ (op.G(u + t * w) @ phi)
    gm = phi @ (op.G(u - t * w) @ phi)
    assert b @ w == pytest.approx((gp - gm) / (2 * t), rel=1e-10)


def test_incompatible_sensitivities_central_difference():
    """Exact LBA path with the condensed elements: dlambda/dx and dJ/dx against central differences
    (h = 1e-5 x_e) on 12 random elements, 1e-5 of max |.| where the load factors are separated."""
    p = synthetic.column_2d(10, 4, seed=8, radius=1.5)
    q = 3

    def values(prob):
        op = incompatible.Problem(prob)
        u = op.to_full(op.solve(np.asarray(prob.f)[op.free]))
        lam, Phi, _ = lba.exact_lba(op, u, q)
        return op, u, float(np.asarray(prob.f) @ u), lam, Phi

    op, u, J, lam, Phi = values(p)
    dlam, dJ, _ = incompatible.sensitivities(op, u, lam, Phi)
    gaps = np.minimum(np.abs(np.diff(np.r_[-np.inf, lam])), np.abs(np.diff(np.r_[lam, np.inf])))
    rng = np.random.default_rng(9)
    x0 = p.x.copy()
    for e in rng.choice(p.x.size, size=12, replace=False):
        h = 1e-5 * x0[e]
        vals = []
        for s in (+1, -1):
            p.x = x0.copy()
            p.x[e] += s * h
            _, _, Js, lams, _ = values(p)
            vals.append((Js, lams))
        p.x = x0
        assert (vals[0][0] - vals[1][0]) / (2 * h) == pytest.approx(dJ[e], abs=1e-5 * np.abs(dJ).max())
        fdl = (vals[0][1] - vals[1][1]) / (2 * h)
        for i in range(q):
            if gaps[i] / lam[i] > 1e-4:
                assert fdl[i] == pytest.approx(dlam[i, e], abs=1e-5 * np.abs(dlam[i]).max())


def test_incompatible_multilevel_rayleigh_bound_and_3d_adjoint():
    """The multilevel path (Sec. 2.1 steps 1-4) runs unchanged on the condensed elements, and its
    first load factor is a Rayleigh quotient, hence not below the exact one; the 3D adjoint
    right-hand side is the derivative of phi^T G[u] phi."""
    p = synthetic.column_2d(24, 8, seed=7, radius=2, mg_levels=3, eig_level=2, num_modes=3)
    op = incompatible.Problem(p)
    u = op.to_full(op.solve(np.asarray(p.f)[op.free]))
    ml = lba.multilevel_lba(op, u, 3, 2)
    lam_exact, _, _ = lba.exact_lba(op, u, 1)
    assert ml["lam"][0] >= lam_exact[0] * (1 - 1e-10)
    assert ml["lam"][0] <= lam_exact[0] * 1.1
    q3 = synthetic.cantilever_3d(4, 2, 2, seed=3, radius=1.5, volfrac=0.5, mg_levels=1, eig_level=1, num_modes=1)
    op3 = incompatible.Problem(q3)
    u3 = op3.to_full(op3.solve(np.asarray(q3.f)[op3.free]))
    rng = np.random.default_rng(4)
    phi, w = rng.standard_normal(q3.num_dofs), rng.standard_normal(q3.num_dofs)
    b = incompatible.adjoint_rhs(q3.nel, 3, q3.x, phi, q3.nu, q3.penal, q3.E0, q3.Emin)
    t = 1e-3
    d = (phi @ (op3.G(u3 + t * w) @ phi) - phi @ (op3.G(u3 - t * w) @ phi)) / (2 * t)
    assert b @ w == pytest.approx(d, rel=1e-10)
