"""Edge and degenerate cases of the solver path against the oracle: a zero load, uniform solid and
near-void designs, a black-and-white 0.01/1 design (what a converged topology optimisation
produces: the largest stiffness contrast the density range allows, across sharp material
boundaries), small grids without coarsening, an eigen level too small for the eigensolver's block,
invalid densities and the call order of the paper's problem statement (set densities -> solve
equilibrium -> buckling -> sensitivities)."""
import numpy as np
import pytest

import synthetic
from oracle import lba
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _column(nel_long, nel_short, x=None, **kw):
    kw.setdefault("mg_levels", 3)
    kw.setdefault("eig_level", 1)
    kw.setdefault("num_modes", 3)
    return synthetic.column_2d(nel_long, nel_short, seed=31, radius=2, x=x, **kw)


def test_zero_load_gives_zero_displacement_and_compliance():
    torch, pkg = require_gpu()
    p = _column(24, 8)
    s = pkg.Solver(p)
    s.set_load(np.zeros(p.num_dofs))
    J, info = s.solve_equilibrium()
    u = s.get_field(pkg.TOBK_FIELD_U)
    assert J == 0.0 and np.all(u == 0.0) and info["converged"] == 1
    s.close()


@pytest.mark.parametrize("design", ["solid", "near_void", "binary"])
def test_degenerate_designs_match_oracle(design):
    """Uniform x = 1 and x = 0.01 (stiffness Emin + 0.01^3: a uniformly soft column, whose load
    factors scale by E_sigma / E_kappa) and a black-and-white design whose load path is solid (a
    solid core of half the width between void sides; stiffness contrast 1e6 across the material
    boundaries): equilibrium to the stated residual and load factors within 1e-6."""
    torch, pkg = require_gpu()
    base = _column(32, 16)
    xs = np.arange(16)
    core = np.tile(((xs >= 4) & (xs < 12)).astype(float), 32)  # elements x-fastest, 16 per row
    x = {"solid": np.ones_like(base.x), "near_void": np.full_like(base.x, 0.01),
         "binary": np.where(core > 0, 1.0, 0.01)}[design]
    p = _column(32, 16, x=x)
    s = pkg.Solver(p)
    J, info = s.solve_equilibrium()
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    lam, _ = s.compute_buckling()
    op = lba.Problem(p)
    u, Jo = lba.linear_analysis(op)
    assert J == pytest.approx(Jo, rel=1e-7)
    uu = s.get_field(pkg.TOBK_FIELD_U)
    assert np.abs(uu - u).max() <= 1e-7 * np.abs(u).max()
    lam_o, _, _ = lba.exact_lba(op, u, p.num_modes)
    assert np.allclose(lam, lam_o, rtol=1e-6), (lam, lam_o)
    s.close()


def test_small_grid_single_level():
    """Eight elements up and two across (48 free DOFs), no coarsening: the preconditioner is the
    dense coarsest solve alone, and the eigensolver's basis can span a large part of the space."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(8, 2, seed=3, radius=1.0, mg_levels=1, eig_level=1, num_modes=2)
    s = pkg.Solver(p)
    J, info = s.solve_equilibrium()
    lam, _ = s.compute_buckling()
    op = lba.Problem(p)
    u, Jo = lba.linear_analysis(op)
    lam_o, _, _ = lba.exact_lba(op, u, p.num_modes)
    assert J == pytest.approx(Jo, rel=1e-10)
    assert np.allclose(lam, lam_o, rtol=1e-8)
    s.close()


def test_eigen_level_smaller_than_the_block_is_reported():
    """Two elements up, one across: 8 free DOFs cannot hold the eigensolver's block of q = 9
    K-orthonormal vectors; the call reports TOBK_E_BREAKDOWN instead of returning load factors from a
    rank-deficient basis."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(2, 1, seed=3, radius=1.0, mg_levels=1, eig_level=1, num_modes=9)
    s = pkg.Solver(p)
    s.solve_equilibrium()
    with pytest.raises(pkg.TobkError) as e:
        s.compute_buckling()
    assert e.value.code == pkg.binding.TOBK_E_BREAKDOWN
    s.close()


def test_eigen_basis_spanning_the_whole_level_is_exact():
    """Two elements up, one across, q = 2: the eigensolver's basis reaches all 8 free DOFs within a
    few expansions, so its Ritz pairs are the exact ones (dense oracle)."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(2, 1, seed=3, radius=1.0, mg_levels=1, eig_level=1, num_modes=2)
    s = pkg.Solver(p)
    s.solve_equilibrium()
    lam, info = s.compute_buckling()
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    lam_o, _, _ = lba.exact_lba(op, u, 2)
    assert np.allclose(lam, lam_o, rtol=1e-8, atol=0), (lam, lam_o)
    s.close()


def test_invalid_densities_and_call_order_are_rejected():
    torch, pkg = require_gpu()
    p = _column(16, 8)
    s = pkg.Solver(p)
    for bad in (np.nan, 1.5, -0.1):
        x = p.x.copy()
        x[3] = bad
        with pytest.raises(pkg.TobkError) as e:
            s.set_densities(x)
        assert e.value.code == pkg.binding.TOBK_E_ARG
    with pytest.raises(pkg.TobkError) as e:
        s.set_densities(p.x[:-1])
    assert e.value.code == pkg.binding.TOBK_E_ARG
    s.set_densities(p.x)  # new densities invalidate u: buckling and sensitivities must wait
    with pytest.raises(pkg.TobkError) as e:
        s.compute_buckling()
    assert e.value.code == pkg.binding.TOBK_E_STATE
    s.solve_equilibrium()
    with pytest.raises(pkg.TobkError) as e:
        s.compute_sensitivities()
    assert e.value.code == pkg.binding.TOBK_E_STATE
    s.compute_buckling()
    s.compute_sensitivities()
    s.close()


# ------------------------------------------------------------------------------------------------
# failure detection: host-side causes, library status codes (nothing here can fault the GPU; every
# loop in the library is bounded by max_iter)
# ------------------------------------------------------------------------------------------------
def _raw_solve(s):
    """tobk_solve_equilibrium through the C-ABI, returning its status instead of raising."""
    import ctypes as C
    from paper_1909_13585_gb300 import binding
    J = C.c_double()
    info = binding.tobk_solve_info()
    rc = s.lib.tobk_solve_equilibrium(s.h, C.byref(J), C.byref(info))
    msg = s.lib.tobk_last_error(s.h).decode()
    return rc, J.value, info.as_dict(), msg


def test_iteration_limit_returns_not_converged_with_the_last_iterate():
    """max_iter too small: TOBK_E_NOT_CONVERGED, info filled (iterations, converged = 0, the true
    relative residual of the returned iterate), and u holds that iterate (its residual, evaluated by
    the oracle, is the one reported)."""
    torch, pkg = require_gpu()
    p = _column(48, 16)
    s = pkg.Solver(p, max_iter=4)
    rc, J, info, msg = _raw_solve(s)
    assert rc == pkg.binding.TOBK_E_NOT_CONVERGED, (rc, msg)
    assert "iteration limit" in msg
    assert info["converged"] == 0 and 1 <= info["iterations"] <= 4
    assert np.isfinite(info["rel_residual"]) and info["rel_residual"] > 1e-8
    u = s.get_field(pkg.TOBK_FIELD_U)
    op = lba.Problem(p)
    res = np.linalg.norm(p.f[op.free] - op.Kf @ u[op.free]) / np.linalg.norm(p.f[op.free])
    assert res == pytest.approx(info["rel_residual"], rel=1e-6)
    # the same handle then converges with a sufficient limit
    s2 = pkg.Solver(p)
    J2, info2 = s2.solve_equilibrium()
    assert info2["converged"] == 1
    s.close(); s2.close()


def test_no_dirichlet_dofs_ends_with_an_error_status():
    """No fixed DOF: K is singular (rigid-body modes) and the load has a net force, so K u = f has no
    solution.  The solve must come back with a failure status (breakdown, non-finite or not
    converged), not hang and not report success."""
    import time
    torch, pkg = require_gpu()
    p = _column(32, 16)
    s = pkg.Solver(p, max_iter=100)
    s.set_fixed(np.zeros(p.num_dofs, dtype=np.uint8))
    s.set_load(p.f)
    s.set_densities(p.x)
    t0 = time.perf_counter()
    rc, J, info, msg = _raw_solve(s)
    assert time.perf_counter() - t0 < 60.0
    assert rc in (pkg.binding.TOBK_E_BREAKDOWN, pkg.binding.TOBK_E_NONFINITE, pkg.binding.TOBK_E_NOT_CONVERGED), (rc, msg)
    assert info["converged"] == 0
    s.close()


def test_nan_in_the_load_is_reported_as_non_finite():
    """A NaN entry in f reaches the CG scalars; the solve stops with TOBK_E_NONFINITE."""
    torch, pkg = require_gpu()
    p = _column(32, 16)
    s = pkg.Solver(p)
    f = p.f.copy()
    f[np.flatnonzero(p.fixed == 0)[5]] = np.nan
    s.set_load(f)
    rc, J, info, msg = _raw_solve(s)
    assert rc == pkg.binding.TOBK_E_NONFINITE, (rc, msg)
    assert "non-finite" in msg
    s.close()


def test_weights_for_another_architecture_are_rejected(tmp_path):
    """A well-formed weights file whose parameter vector does not fit the network it names: a clean
    ValueError before any parameter reaches the library."""
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import learned
    z = dict(learned.read_weights(learned.WEIGHTS))
    z["channels"] = np.array([16, 32, 64, 128])
    path = str(tmp_path / "other.npz")
    np.savez(path, **z)
    with pytest.raises(ValueError, match="parameters"):
        learned.load_weights(pkg, torch, path)
    net = pkg.UNet(tuple(int(v) for v in z["nel"]), int(z["levels"]), tuple(int(v) for v in z["channels"]))
    with pytest.raises(ValueError, match="float32 of length"):
        net.set_state(torch.zeros(10, dtype=torch.float32))
    net.close()
