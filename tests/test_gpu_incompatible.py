"""The paper's incompatible-mode elements (Sec. 2: Wilson's quadrilateral, the hexahedron with 11
interpolation functions per component, internal modes condensed element by element) on the GPU
against oracle/incompatible.py: the fine K v and its Galerkin levels, the condensed stress
stiffness G v and the adjoint right-hand side (operator tests on the same inputs), then the linear
analysis, the exact and multilevel LBA and the sensitivities against the oracle's own chain, in FP64
and with the FP32 V-cycle.  Tolerances as for the plain elements."""
import numpy as np
import pytest

import synthetic
from oracle import incompatible as inc
from oracle import lba, transfer
from tests.gpu_util import rel_err, require_gpu, to_dev

pytestmark = pytest.mark.gpu
INC = 1


def _gaps(lam):
    lam = np.asarray(lam)
    g = np.full(lam.size, np.inf)
    for i in range(lam.size):
        if i > 0:
            g[i] = min(g[i], abs(lam[i] - lam[i - 1]) / abs(lam[i]))
        if i + 1 < lam.size:
            g[i] = min(g[i], abs(lam[i + 1] - lam[i]) / abs(lam[i]))
    return g


OPS = [
    ("2d_40x24", lambda: synthetic.column_2d(40, 24, seed=41, radius=2, mg_levels=3, eig_level=2, num_modes=4)),
    ("3d_12x8x4", lambda: synthetic.cantilever_3d(12, 8, 4, seed=42, radius=1.5, volfrac=0.4, mg_levels=2, eig_level=2,
                                                  num_modes=3)),
]


@pytest.mark.parametrize("name,make", OPS, ids=[c[0] for c in OPS])
def test_operators_match_condensed_assembly(name, make):
    torch, pkg = require_gpu()
    p = make()
    s = pkg.Solver(p, element=INC)
    op = inc.Problem(p)
    rng = np.random.default_rng(3)
    nr = 3
    V = rng.standard_normal((nr, p.num_dofs))
    V[:, p.fixed == 1] = 0.0
    y = torch.zeros((nr, p.num_dofs), dtype=torch.float64, device="cuda")
    s.apply_K(1, to_dev(torch, V), y, nr)
    ref = (op.K @ V.T).T
    ref[:, p.fixed == 1] = 0.0
    assert rel_err(y.cpu().numpy(), ref) < 1e-13
    # Galerkin level 2 against the explicit triple product of the condensed K
    nels, fixeds, Ps = transfer.hierarchy(p.nel, p.dim, p.fixed, 2)
    K2 = (Ps[0].T @ op.Kf @ Ps[0]).tocsr()
    info = s.level_info(2)
    v = rng.standard_normal(info["n"])
    v[fixeds[1] == 1] = 0.0
    y2 = torch.zeros(info["n"], dtype=torch.float64, device="cuda")
    s.apply_K(2, to_dev(torch, v), y2, 1)
    ref2 = np.zeros(info["n"])
    ref2[fixeds[1] == 0] = K2 @ v[fixeds[1] == 0]
    assert rel_err(y2.cpu().numpy(), ref2) < 1e-12
    # condensed stress stiffness G[u] v and its level-2 Galerkin form, on the GPU's u
    s.solve_equilibrium()
    u = s.get_field(pkg.TOBK_FIELD_U)
    G = inc.assemble_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin)
    yg = torch.zeros((nr, p.num_dofs), dtype=torch.float64, device="cuda")
    s.apply_G(1, to_dev(torch, V), yg, nr)
    refg = (G @ V.T).T
    refg[:, p.fixed == 1] = 0.0
    assert rel_err(yg.cpu().numpy(), refg) < 1e-12
    Gf = lba.assembly.restrict_free(G, p.fixed)
    G2 = (Ps[0].T @ Gf @ Ps[0]).tocsr()
    yg2 = torch.zeros(info["n"], dtype=torch.float64, device="cuda")
    s.apply_G(2, to_dev(torch, v), yg2, 1)
    refg2 = np.zeros(info["n"])
    refg2[fixeds[1] == 0] = G2 @ v[fixeds[1] == 0]
    assert rel_err(yg2.cpu().numpy(), refg2) < 1e-12
    s.close()


CHAIN = [
    ("2d_exact", lambda: synthetic.column_2d(48, 16, seed=43, radius=2, mg_levels=3, eig_level=1, num_modes=4)),
    ("2d_l3", lambda: synthetic.column_2d(96, 32, seed=23, radius=3, mg_levels=4, eig_level=3, num_modes=6)),
    ("3d_exact", lambda: synthetic.cantilever_3d(8, 4, 4, seed=22, radius=1.5, volfrac=0.5, mg_levels=2, eig_level=1,
                                                 num_modes=4)),
    ("3d_l2", lambda: synthetic.cantilever_3d(16, 8, 8, seed=25, radius=2, volfrac=0.4, mg_levels=3, eig_level=2,
                                              num_modes=4)),
]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32_vcycle"])
@pytest.mark.parametrize("name,make", CHAIN, ids=[c[0] for c in CHAIN])
def test_chain_matches_oracle(name, make, precision):
    torch, pkg = require_gpu()
    p = make()
    s = pkg.Solver(p, element=INC, precision=precision, eig_tol=0.5e-8)
    J, info = s.solve_equilibrium()
    assert info["converged"] == 1
    u = s.get_field(pkg.TOBK_FIELD_U)
    op = inc.Problem(p)
    res = np.linalg.norm(p.f[op.free] - op.Kf @ u[op.free]) / np.linalg.norm(p.f[op.free])
    assert res <= 1e-8
    uo, Jo = lba.linear_analysis(op)
    e = u[op.free] - uo[op.free]
    assert np.sqrt(e @ (op.Kf @ e)) / np.sqrt(uo[op.free] @ (op.Kf @ uo[op.free])) < 1e-6
    assert J == pytest.approx(Jo, rel=1e-7)
    lam, binfo = s.compute_buckling()
    if p.eig_level == 1:
        lam_o, Phi_o, Gf = lba.exact_lba(op, uo, p.num_modes)
        ok = _gaps(lam_o) > 1e-4
        Phi = s.get_field(pkg.TOBK_FIELD_MODES).reshape(p.num_modes, -1).T
        for i in range(p.num_modes):
            assert lba.eig_residual(op.Kf, Gf, lam[i], Phi[op.free, i]) <= 1e-8
    else:
        ml = lba.multilevel_lba(op, uo, p.num_modes, p.eig_level)
        lam_o, Phi_o = ml["lam"], ml["Phi"]
        ok = (_gaps(ml["lam_coarse"]) > 1e-4) & (_gaps(lam_o) > 1e-4)
    assert ok.sum() >= p.num_modes - 2, lam_o
    assert np.allclose(lam[ok], lam_o[ok], rtol=1e-6, atol=0), (lam, lam_o)
    dlam, dJ, sinfo = s.compute_sensitivities()
    dlo, dJo, _ = inc.sensitivities(op, uo, lam_o, Phi_o)
    assert rel_err(dJ, dJo) < 1e-6
    for i in np.flatnonzero(ok):
        assert rel_err(dlam[i], dlo[i]) < 1e-5, i
    # adjoint right-hand sides: the oracle's condensed element formula on the GPU's modes
    Phi = s.get_field(pkg.TOBK_FIELD_MODES).reshape(p.num_modes, -1)
    B = s.get_field(pkg.TOBK_FIELD_ADJOINT_RHS).reshape(p.num_modes, -1)
    for i in range(min(2, p.num_modes)):
        b = inc.adjoint_rhs(p.nel, p.dim, p.x, Phi[i], p.nu, p.penal, p.E0, p.Emin)
        b[p.fixed == 1] = 0.0
        assert rel_err(B[i], b) < 1e-11
    s.close()


def test_algorithm2_with_incompatible_elements():
    """Kaczmarz smoothing and Ritz projection on every level, including the fine grid whose stress
    stiffness is the condensed one."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(96, 32, seed=23, radius=3, mg_levels=4, eig_level=3, num_modes=6)
    s = pkg.Solver(p, element=INC, kaczmarz_sweeps=2, ritz_levels=1)
    s.solve_equilibrium()
    lam, _ = s.compute_buckling()
    op = inc.Problem(p)
    uo, _ = lba.linear_analysis(op)
    ref = lba.multilevel_lba_refined(op, uo, p.num_modes, p.eig_level, sweeps=2, ritz_projection=True,
                                     order="multicolour")
    ok = (_gaps(ref["lam_coarse"]) > 1e-4) & (_gaps(ref["lam"]) > 1e-4)
    for lv in ref["levels"]:
        ok &= _gaps(lv["lam"][: p.num_modes]) > 1e-4
    assert ok.sum() >= p.num_modes - 2
    assert np.allclose(lam[ok], ref["lam"][ok], rtol=1e-6, atol=0), (lam, ref["lam"])
    s.close()


def test_incompatible_element_is_stiffer_in_bending():
    """The Euler column of the oracle pin at 8 elements across: the incompatible-mode element removes
    the Q4's shear locking, so its lowest load factor is below the plain one (closer to Euler)."""
    torch, pkg = require_gpu()
    p = synthetic.column_2d(64, 8, seed=0, radius=1, mg_levels=3, eig_level=1, num_modes=2,
                            x=np.ones(64 * 8))
    lams = []
    for el in (0, INC):
        s = pkg.Solver(p, element=el)
        s.solve_equilibrium()
        lams.append(s.compute_buckling()[0][0])
        s.close()
    assert lams[1] < lams[0]
