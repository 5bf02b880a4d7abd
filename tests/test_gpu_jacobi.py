"""The damped-Jacobi smoother z <- z + omega D^{-1}(b - K z) (omega = 0.6, two pre- and two
post-smoothing sweeps per level) as the multigrid smoother of every solve of the path, against the
oracle: linear analysis (Algorithm 1 step 2) in 2D and 3D, multilevel LBA (Sec. 2.1 steps 1-4), and
the sensitivities (eq. SensitivityLambda) from the oracle's own pairs.  Tolerances as everywhere:
relative residual 1e-8, load factors 1e-6, sensitivities 1e-5 of max |.|, modes and sensitivities
gated on isolated load factors (relative gap > 1e-4)."""
import numpy as np
import pytest

import synthetic
from oracle import lba, sensitivity
from tests.gpu_util import rel_err, require_gpu

pytestmark = pytest.mark.gpu

JACOBI = dict(smoother=0, omega=0.6, nu_pre=2, nu_post=2, max_iter=2000)


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
    ("cant16x8x8_l2", lambda: synthetic.cantilever_3d(16, 8, 8, seed=25, radius=2, volfrac=0.4, mg_levels=3,
                                                      eig_level=2, num_modes=4)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_damped_jacobi_path_matches_oracle(name, make):
    torch, pkg = require_gpu()
    p = make()
    s = pkg.Solver(p, **JACOBI)
    assert s.desc.smoother == 0
    J, info = s.solve_equilibrium()
    assert info["converged"] == 1
    u = s.get_field(pkg.TOBK_FIELD_U)
    op = lba.Problem(p)
    res = np.linalg.norm(p.f[op.free] - op.Kf @ u[op.free]) / np.linalg.norm(p.f[op.free])
    assert res <= 1e-8
    uo, Jo = lba.linear_analysis(op)
    e = u[op.free] - uo[op.free]
    assert np.sqrt(e @ (op.Kf @ e)) / np.sqrt(uo[op.free] @ (op.Kf @ uo[op.free])) < 1e-6
    assert J == pytest.approx(Jo, rel=1e-7)
    lam, binfo = s.compute_buckling()
    ml = lba.multilevel_lba(op, uo, p.num_modes, p.eig_level)
    ok = _gaps(ml["lam_coarse"]) > 1e-4
    assert ok.sum() >= p.num_modes - 2
    assert np.allclose(lam[ok], ml["lam"][ok], rtol=1e-6, atol=0), (lam, ml["lam"])
    dlam, dJ, sinfo = s.compute_sensitivities()
    assert sinfo["converged"] == 1
    dlo, dJo, _ = sensitivity.sensitivities(op, uo, ml["lam"], ml["Phi"])
    assert rel_err(dJ, dJo) < 1e-6
    for i in np.flatnonzero(ok & (_gaps(ml["lam"]) > 1e-4)):
        assert rel_err(dlam[i], dlo[i]) < 1e-5, i
    s.close()


def test_damped_jacobi_and_chebyshev_reach_the_same_solution():
    """Both smoothers precondition the same CG: the solutions agree to the stopping tolerance, and
    the Chebyshev smoother (the default) needs fewer iterations."""
    torch, pkg = require_gpu()
    p = synthetic.config("column60x20")
    sj = pkg.Solver(p, **JACOBI)
    sc = pkg.Solver(p)
    Jj, ij = sj.solve_equilibrium()
    Jc, ic = sc.solve_equilibrium()
    assert Jj == pytest.approx(Jc, rel=1e-7)
    assert ic["iterations"] <= ij["iterations"]
    sj.close(); sc.close()
