"""Pins of the oracle's Algorithm 2 refinement (oracle.lba.multilevel_lba_refined: per-level
Kaczmarz smoothing and Rayleigh-Ritz, Appendix A): Kaczmarz row projections never lengthen a vector
(A psi = 0 is consistent), the Ritz load factors bound each level's exact ones from above
(Courant-Fischer for the K-definite pencil), the refinement without smoothing and projection is
Sec. 2.1 steps 1-4, and the fine load factor keeps its Rayleigh bound."""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic
from oracle import lba


def _case():
    p = synthetic.column_2d(32, 16, seed=13, radius=2.5, mg_levels=4, eig_level=3, num_modes=4)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    return p, op, u


def test_kaczmarz_projections_never_lengthen_a_vector():
    p, op, u = _case()
    A = op.Kf + 0.5 * lba.assembly.restrict_free(op.G(u), op.fixed)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((A.shape[0], 2))
    norms = [np.linalg.norm(psi, axis=0)]
    for _ in range(3):
        psi = lba.kaczmarz(A, psi, 1)
        norms.append(np.linalg.norm(psi, axis=0))
    assert all(np.all(b <= a * (1 + 1e-14)) for a, b in zip(norms, norms[1:]))


def test_reduces_to_sec_2_1_without_smoothing_and_projection():
    p, op, u = _case()
    a = lba.multilevel_lba(op, u, 4, 3)
    b = lba.multilevel_lba_refined(op, u, 4, 3, sweeps=0, ritz_projection=False)
    assert np.allclose(a["lam"], b["lam"], rtol=1e-12)


def test_ritz_load_factors_bound_each_level_and_the_fine_grid():
    p, op, u = _case()
    r = lba.multilevel_lba_refined(op, u, 4, 3, sweeps=2)
    for lv in r["levels"]:
        mu = sla.eigh(-lv["G"].toarray(), lv["K"].toarray(), eigvals_only=True)
        exact = np.sort(1.0 / mu[mu > 0])[:4]
        assert np.all(lv["lam"][:4] >= exact * (1 - 1e-10)), (lv["level"], lv["lam"], exact)
    lam_exact, _, _ = lba.exact_lba(op, u, 1)
    assert r["lam"][0] >= lam_exact[0] * (1 - 1e-10)
    # the per-level smoothing does not make the first load factor worse than Sec. 2.1's
    plain = lba.multilevel_lba(op, u, 4, 3)
    assert r["lam"][0] <= plain["lam"][0] * (1 + 1e-3)


def test_kaczmarz_single_row_is_the_orthogonal_projection():
    """One row a: the update psi - (a . psi / |a|^2) a is the orthogonal projection onto a^perp, so
    a . psi vanishes afterwards and the change is parallel to a with that exact coefficient (a row
    scaled by |a| instead of |a|^2 fails the first check)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    n = 9
    a = np.zeros(n)
    a[[1, 4, 7]] = rng.standard_normal(3) * 3.0
    A = sp.csr_matrix(a[None, :])
    psi = rng.standard_normal((n, 2))
    out = lba.kaczmarz(A, psi, 1)
    assert np.abs(a @ out).max() <= 1e-13 * np.abs(a).max() * np.abs(psi).max()
    coef = (a @ psi) / (a @ a)
    assert np.allclose(out, psi - np.outer(a, coef), rtol=0, atol=1e-14)


def test_kaczmarz_converges_to_the_null_space_projection():
    """For A psi = 0 every Kaczmarz step is an orthogonal projection onto a hyperplane that contains
    null(A), and the iterate stays in psi0 + range(A^T): the sweeps converge to the orthogonal
    projection of psi0 onto null(A), (I - A^+ A) psi0 (A^+ from the SVD); a null vector is left
    unchanged."""
    import scipy.sparse as sp
    rng = np.random.default_rng(6)
    A = rng.standard_normal((4, 10))
    psi0 = rng.standard_normal((10, 3))
    U, S, Vt = np.linalg.svd(A)
    Pnull = np.eye(10) - Vt[:4].T @ Vt[:4]
    out = lba.kaczmarz(sp.csr_matrix(A), psi0, 400)
    assert np.allclose(out, Pnull @ psi0, rtol=0, atol=1e-10)
    v = Pnull @ rng.standard_normal(10)
    assert np.allclose(lba.kaczmarz(sp.csr_matrix(A), v[:, None], 3)[:, 0], v, rtol=0, atol=1e-13)


def test_multicolour_order_is_a_permutation_with_disjoint_same_colour_supports():
    """The multicolour row order visits every free row once, and two rows of different nodes of one
    colour share no column of the level's pencil, so the rows of one colour commute: reversing the
    node order inside every colour gives bit-identical sweeps."""
    p, op, u = _case()
    nels, fixeds, Ps = lba.transfer.hierarchy(p.nel, p.dim, p.fixed, 3)
    Gf = lba.assembly.restrict_free(op.G(u), op.fixed)
    Kl, Gl = (Ps[0].T @ op.Kf @ Ps[0]).tocsr(), (Ps[0].T @ Gf @ Ps[0]).tocsr()
    A = (Kl + 0.7 * Gl).tocsr()
    order = lba.multicolour_rows(nels[1], p.dim, fixeds[1])
    assert np.array_equal(np.sort(order), np.arange(A.shape[0]))
    nd = lba.grid.node_dims(nels[1], p.dim)
    free = np.flatnonzero(fixeds[1] == 0)
    node_of = free // p.dim
    colour = (node_of % nd[0]) % 3 + 3 * ((node_of // nd[0]) % 3)
    for col in range(9):
        rows = order[colour[order] == col]
        seen = {}
        for r in rows:
            for cidx in A.indices[A.indptr[r]:A.indptr[r + 1]]:
                owner = seen.setdefault(cidx, node_of[r])
                assert owner == node_of[r], (col, r, cidx)
    # reversed node order within each colour (rows of one node kept in turn)
    rev = []
    for col in range(9):
        rows = order[colour[order] == col]
        for node in sorted(set(node_of[rows]), reverse=True):
            rev.extend(rows[node_of[rows] == node])
    psi = np.random.default_rng(2).standard_normal((A.shape[0], 3))
    a = lba.kaczmarz(A, psi, 2, order)
    b = lba.kaczmarz(A, psi, 2, np.asarray(rev))
    assert np.array_equal(a, b)


def test_inverse_iteration_steps_descend_to_the_exact_load_factor():
    """fine_steps > 1 repeats the fine solve K Phi = G Phi_prev (eq. PInvIt-GeneralInteration with
    P = K).  Under pure compression -G is positive semi-definite and every step lowers the smallest
    Rayleigh quotient (it is an inverse-iteration step of a positive semi-definite operator), never
    below the exact lambda_1; with the gap of this column the iteration converges to it."""
    from tests.test_oracle_lba import _roller_column
    p = _roller_column((8, 32), 2, 1.0, eig_level=3, mg_levels=3)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    exact, _, _ = lba.exact_lba(op, u, 2)
    prev = np.inf
    for k in (1, 2, 3, 6, 30):
        r = lba.multilevel_lba_refined(op, u, 2, 3, sweeps=0, ritz_projection=False, fine_steps=k)
        assert exact[0] * (1 - 1e-12) <= r["lam"][0] <= prev * (1 + 1e-12), (k, r["lam"][0], prev)
        prev = r["lam"][0]
    assert prev == pytest.approx(exact[0], rel=1e-8)
