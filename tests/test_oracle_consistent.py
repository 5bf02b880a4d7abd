"""Pins of oracle.consistent: the exact derivative of the multilevel load factors (Sec. 2.1,
eq. eigResidual, eq. consistentSensitivity) against central differences of lba.multilevel_lba, against
the forward differentiation of the same steps, against the printed eq. consistentSensitivity, and the
special cases that reduce to eq. SensitivityLambda."""
import numpy as np
import pytest

import synthetic
from oracle import assembly, consistent, lba, sensitivity


def _case(kind):
    if kind == "2d_l2":
        return synthetic.column_2d(16, 8, seed=8, radius=1.5, mg_levels=3), 4, 2
    if kind == "2d_l3":
        return synthetic.column_2d(16, 8, seed=12, radius=1.5, mg_levels=3), 3, 3
    return synthetic.cantilever_3d(8, 4, 4, seed=13, radius=1.5, volfrac=0.5, mg_levels=2), 3, 2


def _ml_lam(p, q, L):
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    return lba.multilevel_lba(op, u, q, eig_level=L)["lam"]


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_rhs_pair_is_the_gradient_of_the_bilinear_stress_form(dim):
    """G[x, v] is linear in v, so g . v = a^T G[x, v] c exactly, for any v; g is symmetric in (a, c)
    and equals the right-hand side of eq. AdjointSystem for a = c."""
    p = (synthetic.column_2d(6, 4, seed=10, radius=1.5) if dim == 2
         else synthetic.cantilever_3d(4, 2, 2, seed=10, radius=1.5, volfrac=0.5))
    rng = np.random.default_rng(14)
    a, c, v = (rng.standard_normal(p.num_dofs) for _ in range(3))
    args = (p.nu, p.penal, p.E0, p.Emin)
    g = consistent.adjoint_rhs_pair(p.nel, dim, p.x, a, c, *args)
    Gv = assembly.assemble_G(p.nel, dim, p.x, v, *args)
    assert g @ v == pytest.approx(a @ (Gv @ c), rel=1e-12)
    assert np.allclose(g, consistent.adjoint_rhs_pair(p.nel, dim, p.x, c, a, *args), rtol=0, atol=1e-12 * np.abs(g).max())
    gq = consistent.adjoint_rhs_pair(p.nel, dim, p.x, a, a, *args)
    assert np.allclose(gq, sensitivity.adjoint_rhs(p.nel, dim, p.x, a, *args), rtol=0, atol=1e-12 * np.abs(gq).max())


@pytest.mark.parametrize("kind", ["2d_l2", "2d_l3", "3d_l2"])
def test_consistent_sensitivities_central_difference(kind):
    """Central differences (h = 1e-4 x_e) of the multilevel load factors of lba.multilevel_lba agree
    with the adjoint chain to 1e-6 of max |d lambda_i / d x|, on modes separated from their
    neighbours; eq. SensitivityLambda applied to the same pairs misses by far more."""
    p, q, L = _case(kind)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    dl, aux = consistent.consistent_sensitivities(op, u, q, L)
    lam = aux["lam"]
    ml = lba.multilevel_lba(op, u, q, eig_level=L)
    assert np.allclose(lam, ml["lam"], rtol=1e-12)
    plain, _, _ = sensitivity.sensitivities(op, u, ml["lam"], ml["Phi"])
    gaps = np.minimum(np.abs(np.diff(np.r_[-np.inf, lam])), np.abs(np.diff(np.r_[lam, np.inf])))
    rng = np.random.default_rng(15)
    els = rng.choice(p.x.size, size=8, replace=False)
    x0 = p.x.copy()
    worst_plain = 0.0
    try:
        for e in els:
            h = 1e-4 * x0[e]
            p.x = x0.copy(); p.x[e] += h
            lp = _ml_lam(p, q, L)
            p.x = x0.copy(); p.x[e] -= h
            lm = _ml_lam(p, q, L)
            fd = (lp - lm) / (2 * h)
            for i in range(q):
                if gaps[i] / lam[i] > 1e-3:
                    scale = np.abs(dl[i]).max()
                    assert fd[i] == pytest.approx(dl[i, e], abs=1e-6 * scale)
                    worst_plain = max(worst_plain, abs(fd[i] - plain[i, e]) / scale)
    finally:
        p.x = x0
    assert worst_plain > 1e-3


@pytest.mark.parametrize("kind", ["2d_l2", "3d_l2"])
def test_forward_differentiation_and_printed_formula_equal_the_adjoint_chain(kind):
    """Forward differentiation of the steps of Sec. 2.1 gives the adjoint chain's derivative; the
    printed eq. consistentSensitivity with p = -2 (K + lambda G)^{-1} y and the forward d y / d x_e
    gives it too; with p = 0 the printed form is eq. SensitivityLambda."""
    p, q, L = _case(kind)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    dl, aux = consistent.consistent_sensitivities(op, u, q, L)
    mp = consistent.multilevel_pairs(op, u, q, L)
    order = aux["order"]
    ml = lba.multilevel_lba(op, u, q, eig_level=L)
    plain, _, _ = sensitivity.sensitivities(op, u, ml["lam"], ml["Phi"])
    rng = np.random.default_rng(16)
    for e in rng.choice(p.x.size, size=4, replace=False):
        fw, dY, _ = consistent.forward_derivative(op, u, mp, e)
        scale = np.abs(dl).max(axis=1)
        assert np.all(np.abs(fw[order] - dl[:, e]) <= 1e-9 * scale)
        pf = consistent.paper_formula(op, u, mp, e, dY)
        assert np.all(np.abs(pf[order] - dl[:, e]) <= 1e-8 * scale)
        p0 = consistent.paper_formula(op, u, mp, e, dY, use_p=False)
        assert np.all(np.abs(p0[order] - plain[:, e]) <= 1e-9 * np.abs(plain).max(axis=1))


def test_coarse_adjoint_is_consistent_and_constrained():
    """b = P^T G w is orthogonal to psi (psi^T b = y^T phi = 0 by the definition of lambda), and c meets
    psi^T G^l c = 0 and (K^l + mu G^l) c = b."""
    p, q, L = _case("2d_l2")
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    mp = consistent.multilevel_pairs(op, u, q, L)
    W = op.solve(mp["Y"])
    B = mp["P"].T @ (mp["Gf"] @ W)
    for i in range(q):
        ps = mp["psi"][:, i]
        assert abs(ps @ B[:, i]) <= 1e-12 * np.linalg.norm(ps) * np.linalg.norm(B[:, i])
        A = (mp["Kl"] + mp["mu"][i] * mp["Gl"]).toarray()
        c = consistent._bordered_solve(A, mp["Gl"] @ ps, B[:, i])
        assert abs(ps @ (mp["Gl"] @ c)) <= 1e-12 * np.linalg.norm(mp["Gl"] @ ps) * np.linalg.norm(c)
        assert np.linalg.norm(A @ c - B[:, i]) <= 1e-10 * np.linalg.norm(B[:, i])


def test_exact_pairs_reduce_to_sensitivity_lambda():
    """eig_level = 1: the coarse pairs are the fine eigenpairs, phi = -psi / lambda, y = 0, w = 0, and
    the consistent derivative is eq. SensitivityLambda of the exact LBA."""
    p = synthetic.column_2d(10, 4, seed=8, radius=1.5)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    q = 3
    dl, aux = consistent.consistent_sensitivities(op, u, q, 1)
    lam, Phi, _ = lba.exact_lba(op, u, q)
    ref, _, _ = sensitivity.sensitivities(op, u, lam, Phi)
    assert np.allclose(aux["lam"], lam, rtol=1e-10)
    assert np.abs(aux["W"]).max() <= 1e-8 * np.abs(aux["Phi"]).max()
    assert np.allclose(dl, ref, rtol=0, atol=1e-7 * np.abs(ref).max())


def test_printed_formula_pin_rejects_a_wrong_adjoint():
    """The agreement of the printed eq. consistentSensitivity with the adjoint chain depends on its
    adjoint p = -2 (K + lambda G)^{-1} y: the opposite sign of p, or dropping the factor
    1 / (1 - p^T G phi), misses the derivative by far more than the 1e-8 the correct form meets."""
    p, q, L = _case("2d_l2")
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    dl, aux = consistent.consistent_sensitivities(op, u, q, L)
    mp = consistent.multilevel_pairs(op, u, q, L)
    order = aux["order"]
    e = 5
    _, dY, _ = consistent.forward_derivative(op, u, mp, e)
    scale = np.abs(dl).max(axis=1)
    good = consistent.paper_formula(op, u, mp, e, dY)
    assert np.all(np.abs(good[order] - dl[:, e]) <= 1e-8 * scale)
    # the same formula written out here with the two plausible slips
    Gf, Kf = mp["Gf"], op.Kf
    worst_sign = worst_factor = 0.0
    x = np.asarray(p.x, dtype=np.float64)
    from oracle import elements
    _, _, dEk, dEs = elements.simp(x, p.penal, p.E0, p.Emin)
    Ke0 = elements.stiffness_ke0(p.dim, p.nu)
    Ge = assembly.element_stress_stiffness(p.nel, p.dim, u, p.nu)
    dK = dEk[e] * consistent._element_operator(op, e, Ke0)
    dGx = dEs[e] * consistent._element_operator(op, e, Ge[e])
    du = op.to_full(-op.solve(dK @ np.asarray(u)[op.free]))
    dG = dGx + assembly.restrict_free(op.G(du), op.fixed)
    uf = np.asarray(u)[op.free]
    for r in range(q):
        i = order[r]
        lam = mp["lam"][i]
        s = np.sqrt(-(mp["Phi"][:, i] @ (Gf @ mp["Phi"][:, i])))
        ph = mp["Phi"][:, i] / s
        y = Kf @ ph + lam * (Gf @ ph)
        dy = dY[:, i] / s
        phf = op.to_full(ph)
        z = op.solve(consistent.adjoint_rhs_pair(p.nel, p.dim, x, phf, phf, p.nu, p.penal, p.E0, p.Emin)[op.free])
        first = ph @ ((dK + lam * dGx) @ ph) - lam * (z @ (dK @ uf))
        pv = -2.0 * np.linalg.solve((Kf + lam * Gf).toarray(), y)
        core = first + pv @ ((dK + lam * dG) @ ph) - pv @ dy
        assert abs(core / (1.0 - pv @ (Gf @ ph)) - dl[r, e]) <= 1e-8 * scale[r]
        wrong_sign = (first - pv @ ((dK + lam * dG) @ ph) + pv @ dy) / (1.0 + pv @ (Gf @ ph))
        worst_sign = max(worst_sign, abs(wrong_sign - dl[r, e]) / scale[r])
        worst_factor = max(worst_factor, abs(core - dl[r, e]) / scale[r])
    assert worst_sign > 1e-3 and worst_factor > 1e-3, (worst_sign, worst_factor)
