"""GPU parity of the consistent sensitivities of the multilevel load factors (Sec. 2.1, eq. eigResidual,
eq. consistentSensitivity) against oracle.consistent, whose derivative is pinned by central
differences of the multilevel load factors (tests/test_oracle_consistent.py).

Tolerances (FP64 mode): sensitivities within 1e-5 of max |d lambda_i / d x|, the adjoint fields
(fine adjoint w, prolongated coarse adjoint P c, prolongated modes Psi) within 1e-6 of their largest
entry, on modes whose coarse and fine load factors are isolated (relative gap > 1e-4), so that the
pairs and hence their derivatives are unique."""
import numpy as np
import pytest

from gpu_util import rel_err, require_gpu
import synthetic
from oracle import consistent, lba, sensitivity

pytestmark = pytest.mark.gpu

CASES = [
    ("col64x32_l3", lambda: synthetic.column_2d(64, 32, seed=31, radius=2, mg_levels=4, eig_level=3, num_modes=6)),
    ("col48x16_l2", lambda: synthetic.column_2d(48, 16, seed=33, radius=2, mg_levels=3, eig_level=2, num_modes=4)),
    ("cant16x8x8_l2", lambda: synthetic.cantilever_3d(16, 8, 8, seed=32, radius=1.5, volfrac=0.5, mg_levels=3,
                                                      eig_level=2, num_modes=4)),
]


def _gaps(lam):
    lam = np.asarray(lam)
    g = np.full(lam.size, np.inf)
    for i in range(lam.size):
        if i > 0:
            g[i] = min(g[i], abs(lam[i] - lam[i - 1]) / abs(lam[i]))
        if i + 1 < lam.size:
            g[i] = min(g[i], abs(lam[i + 1] - lam[i]) / abs(lam[i]))
    return g


def _gpu(p, **kw):
    torch, pkg = require_gpu()
    s = pkg.Solver(p, consistent_sens=1, **kw)
    s.solve_equilibrium()
    lam, _ = s.compute_buckling()
    dlam, dJ, info = s.compute_sensitivities()
    fields = {k: s.get_field(getattr(pkg, k)).reshape(p.num_modes, -1).T
              for k in ("TOBK_FIELD_MODES", "TOBK_FIELD_FINE_ADJOINT", "TOBK_FIELD_COARSE_ADJOINT",
                        "TOBK_FIELD_PROLONGATED")}
    s.close()
    return lam, dlam, dJ, info, fields


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_consistent_sensitivities_match_oracle(name, make):
    p = make()
    lam, dlam, dJ, info, F = _gpu(p)
    assert info["converged"] == 1
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    dl_o, aux = consistent.consistent_sensitivities(op, u, p.num_modes, p.eig_level)
    ok = (_gaps(aux["lam"]) > 1e-4) & (_gaps(np.sort(aux["mu"])) > 1e-4)
    assert ok.sum() >= p.num_modes - 1, (aux["lam"], aux["mu"])
    assert np.allclose(lam[ok], aux["lam"][ok], rtol=1e-6, atol=0)
    _, dJ_o, _ = sensitivity.sensitivities(op, u, aux["lam"], aux["Phi"])
    assert rel_err(dJ, dJ_o) < 1e-6
    Phi = F["TOBK_FIELD_MODES"]
    for i in np.flatnonzero(ok):
        assert rel_err(dlam[i], dl_o[i]) < 1e-5, (i, rel_err(dlam[i], dl_o[i]))
        # the GPU's fields are on the scale of its normalised mode; the oracle's on phi = K^{-1} G P psi
        sc = (Phi[:, i] @ aux["Phi"][:, i]) / (aux["Phi"][:, i] @ aux["Phi"][:, i])
        for key, ref in (("TOBK_FIELD_FINE_ADJOINT", aux["W"]), ("TOBK_FIELD_COARSE_ADJOINT", aux["Chat"]),
                         ("TOBK_FIELD_PROLONGATED", aux["Psi"])):
            assert rel_err(F[key][:, i], sc * ref[:, i]) < 1e-6, (i, key, rel_err(F[key][:, i], sc * ref[:, i]))


def test_consistent_differs_from_sensitivity_lambda_and_fp32_vcycle_agrees():
    """The consistent derivative is not eq. SensitivityLambda of the same pairs (the residual term is
    not small on a coarse eigen level); the FP32 V-cycle as preconditioner of every solve leaves the
    result within the FP64 tolerance."""
    torch, pkg = require_gpu()
    p = CASES[1][1]()
    lam, dlam, _, _, _ = _gpu(p)
    s = pkg.Solver(p)
    s.solve_equilibrium()
    s.compute_buckling()
    plain, _, _ = s.compute_sensitivities()
    s.close()
    assert max(rel_err(plain[i], dlam[i]) for i in range(p.num_modes)) > 1e-3
    lam32, dlam32, _, _, _ = _gpu(p, precision=pkg.TOBK_FP32_VCYCLE)
    ok = _gaps(lam) > 1e-4
    for i in np.flatnonzero(ok):
        assert rel_err(dlam32[i], dlam[i]) < 1e-5


def test_consistent_on_exact_path_is_sensitivity_lambda_and_invalid_combinations_are_refused():
    torch, pkg = require_gpu()
    p = synthetic.column_2d(24, 8, seed=21, radius=2, mg_levels=3, eig_level=1, num_modes=4)
    out = []
    for flag in (0, 1):
        s = pkg.Solver(p, consistent_sens=flag)
        s.solve_equilibrium()
        s.compute_buckling()
        out.append(s.compute_sensitivities()[0])
        with pytest.raises(pkg.TobkError):
            s.get_field(pkg.TOBK_FIELD_FINE_ADJOINT)
        s.close()
    assert np.array_equal(out[0], out[1])
    q = synthetic.column_2d(24, 8, seed=21, radius=2, mg_levels=3, eig_level=2, num_modes=4)
    for bad in ({"kaczmarz_sweeps": 1}, {"ritz_levels": 1}, {"fine_steps": 2}, {"element": 1}):
        with pytest.raises(pkg.TobkError) as ei:
            pkg.Solver(q, consistent_sens=1, **bad)
        assert ei.value.code == pkg.TOBK_E_ARG


def _ml_lambda(pkg, p, x):
    s = pkg.Solver(p)
    s.set_densities(x)
    s.solve_equilibrium()
    lam, _ = s.compute_buckling()
    s.close()
    return lam


@pytest.mark.parametrize("name", ["column480x160", "cantilever48x24x24"])
def test_consistent_sensitivities_are_the_derivative_of_the_gpu_load_factors_full_size(name):
    """At the benchmark's size, along a random direction d (relative to x, all elements), the
    consistent derivative equals the central difference of the GPU's own multilevel load factors
    (step h = 1e-4: rounding and solver tolerance give ~1e-6 of the difference), and eq.
    SensitivityLambda of the same pairs does not."""
    torch, pkg = require_gpu()
    if name == "column480x160":
        p = synthetic.config(name)
    else:
        p = synthetic.cantilever_3d(48, 24, 24, seed=34, radius=2, volfrac=0.4, mg_levels=4, eig_level=2, num_modes=6)
    lam, dlam, _, info, _ = _gpu(p)
    assert info["converged"] == 1
    s = pkg.Solver(p)
    s.solve_equilibrium()
    s.compute_buckling()
    plain, _, _ = s.compute_sensitivities()
    s.close()
    rng = np.random.default_rng(35)
    d = rng.standard_normal(p.x.size) * np.minimum(p.x, 1.0 - p.x)  # x +- h d stays inside (0, 1)
    h = 1e-4
    lp = _ml_lambda(pkg, p, p.x + h * d)
    lm = _ml_lambda(pkg, p, p.x - h * d)
    fd = (lp - lm) / (2 * h)
    ok = _gaps(lam) > 1e-3  # modes that cannot swap order under the perturbation
    assert ok.sum() >= p.num_modes // 2, lam
    worst_plain = 0.0
    for i in np.flatnonzero(ok):
        scale = np.abs(dlam[i]) @ np.abs(d)
        assert abs(fd[i] - dlam[i] @ d) <= 1e-5 * scale, (i, fd[i], dlam[i] @ d, plain[i] @ d)
        worst_plain = max(worst_plain, abs(fd[i] - plain[i] @ d) / scale)
    assert worst_plain > 1e-3


def test_consistent_sensitivities_graph_replay_is_bit_identical():
    """On a caller's stream the coarse adjoint's iteration pairs replay a captured CUDA graph; on the
    legacy stream they are launched directly.  Same kernels in the same order: the same bits."""
    torch, pkg = require_gpu()
    p = CASES[0][1]()
    out = []
    for stream in (None, torch.cuda.Stream()):
        # early_fine = 0: the fine solves after the eigensolve on both streams (the legacy stream has no
        # second stream to start them on)
        s = pkg.Solver(p, stream=stream, consistent_sens=1, early_fine=0)
        s.solve_equilibrium()
        s.compute_buckling()
        for _ in range(2):  # the second call replays the graph captured by the first
            dlam, _, info = s.compute_sensitivities()
        torch.cuda.synchronize()
        out.append((dlam.copy(), info["status_detail"]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] > 0


def test_consistent_sensitivities_with_the_early_fine_solve_match_oracle():
    """On a caller's stream the early fine solve supplies part of the modes (their coarse pairs taken
    when they met eig_tol); the consistent derivative then follows those pairs and still matches the
    oracle within 1e-5."""
    torch, pkg = require_gpu()
    p = CASES[0][1]()
    s = pkg.Solver(p, stream=torch.cuda.Stream(), consistent_sens=1)
    s.solve_equilibrium()
    lam, _ = s.compute_buckling()
    dlam, _, info = s.compute_sensitivities()
    torch.cuda.synchronize()
    s.close()
    assert info["converged"] == 1
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    dl_o, aux = consistent.consistent_sensitivities(op, u, p.num_modes, p.eig_level)
    ok = (_gaps(aux["lam"]) > 1e-4) & (_gaps(np.sort(aux["mu"])) > 1e-4)
    assert ok.sum() >= p.num_modes - 1
    assert np.allclose(lam[ok], aux["lam"][ok], rtol=1e-6, atol=0)
    for i in np.flatnonzero(ok):
        assert rel_err(dlam[i], dl_o[i]) < 1e-5, (i, rel_err(dlam[i], dl_o[i]))
