"""Algorithm 2 (Appendix A) on the GPU against the oracle's multilevel_lba_refined: after every
prolongation from the eigen level down to Omega_1, multicolour Kaczmarz sweeps on
(K^j + sigma G^j) psi = 0 (sigma the smallest load factor of the level above; the rows in the
3^d node-colour order that both sides use), the Rayleigh-Ritz projection of (K^j, G^j) on span Psi^j,
then the fine solve and Rayleigh quotients, optionally repeated as inverse-iteration steps
(eq. PInvIt-GeneralInteration with P = K).  Load factors within 1e-6 where the oracle's final and
coarse load factors are isolated (relative gap > 1e-4); at most two of the q may be clustered."""
import numpy as np
import pytest

import synthetic
from oracle import lba, sensitivity
from tests.gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu


def _gaps(lam):
    lam = np.asarray(lam)
    g = np.full(lam.size, np.inf)
    for i in range(lam.size):
        if i > 0:
            g[i] = min(g[i], abs(lam[i] - lam[i - 1]) / abs(lam[i]))
        if i + 1 < lam.size:
            g[i] = min(g[i], abs(lam[i + 1] - lam[i]) / abs(lam[i]))
    return g


CASES = [
    ("col96x32_l3", lambda: synthetic.column_2d(96, 32, seed=23, radius=3, mg_levels=4, eig_level=3, num_modes=6)),
    ("col64x32_l3", lambda: synthetic.column_2d(64, 32, seed=24, radius=2, mg_levels=3, eig_level=3, num_modes=4)),
    ("cant16x8x8_l2", lambda: synthetic.cantilever_3d(16, 8, 8, seed=25, radius=2, volfrac=0.4, mg_levels=3,
                                                      eig_level=2, num_modes=4)),
]
SETTINGS = [  # (kaczmarz sweeps, Ritz projection, fine inverse-iteration steps)
    (2, 1, 1),
    (0, 0, 3),
    (1, 1, 2),
]


@pytest.mark.parametrize("sweeps,ritz,steps", SETTINGS, ids=["kaczmarz2_ritz", "inverse3", "kaczmarz1_ritz_inverse2"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_algorithm2_matches_oracle(name, make, sweeps, ritz, steps):
    torch, pkg = require_gpu()
    p = make()
    s = pkg.Solver(p, kaczmarz_sweeps=sweeps, ritz_levels=ritz, fine_steps=steps)
    s.solve_equilibrium()
    lam, info = s.compute_buckling()
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    ref = lba.multilevel_lba_refined(op, u, p.num_modes, p.eig_level, sweeps=sweeps, ritz_projection=bool(ritz),
                                     order="multicolour", fine_steps=steps)
    ok = (_gaps(ref["lam_coarse"]) > 1e-4) & (_gaps(ref["lam"]) > 1e-4)
    for lv in ref["levels"]:
        ok &= _gaps(lv["lam"][: p.num_modes]) > 1e-4
    assert ok.sum() >= p.num_modes - 2, ref["lam"]
    assert np.allclose(lam[ok], ref["lam"][ok], rtol=1e-6, atol=0), (lam, ref["lam"])
    assert np.all(np.diff(lam) >= 0)
    # the modes are K-normalised (each fine column is its own inverse-iteration step, so they are
    # not mutually K-orthogonal) and the Rayleigh bound holds
    Phi = s.get_field(pkg.TOBK_FIELD_MODES).reshape(p.num_modes, -1).T
    P = Phi[op.free]
    assert np.allclose(np.einsum("ij,ij->j", P, op.Kf @ P), 1.0, rtol=0, atol=1e-9)
    assert lam[0] >= lba.exact_lba(op, u, 1)[0][0] * (1 - 1e-9)
    # sensitivities of the refined pairs: the same formula on the oracle's refined pairs
    dlam, dJ, _ = s.compute_sensitivities()
    dlo, dJo, _ = sensitivity.sensitivities(op, u, ref["lam"], ref["Phi"])
    for i in np.flatnonzero(ok):
        assert rel_err(dlam[i], dlo[i]) < 1e-5, i
    s.close()


def test_refinement_moves_the_first_load_factor_toward_the_exact_one():
    """On a 2D column with the eigenproblem two levels down: the exact lambda_1 <= Algorithm 2's
    lambda~_1 (Kaczmarz + Ritz, or inverse-iteration steps) <= Sec. 2.1's lambda~_1, on the GPU."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(96, 32, seed=23, radius=3, mg_levels=4, eig_level=3, num_modes=6)
    lams = {}
    for key, kw in (("plain", {}), ("alg2", dict(kaczmarz_sweeps=2, ritz_levels=1)),
                    ("inverse4", dict(fine_steps=4))):
        s = pkg.Solver(p, **kw)
        s.solve_equilibrium()
        lams[key] = s.compute_buckling()[0][0]
        s.close()
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    exact = lba.exact_lba(op, u, 1)[0][0]
    assert exact * (1 - 1e-9) <= lams["inverse4"] <= lams["plain"] * (1 + 1e-9)
    assert exact * (1 - 1e-9) <= lams["alg2"] <= lams["plain"] * (1 + 1e-3)
