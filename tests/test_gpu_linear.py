"""GPU parity of the linear part of the path against the oracle: fine-grid K v (Sec. 2), Galerkin
coarse operators (Sec. 2.1 step 1), stress stiffness G v (Sec. 2), and the mgPCG linear analysis
(Algorithm 1 step 2) to relative residual 1e-8, for Q4 (2D) and H8 (3D), several thread blocks and
ragged tails."""
import numpy as np
import pytest

import synthetic
from oracle import assembly, lba, transfer
from tests.gpu_util import rel_err, require_gpu, to_dev

pytestmark = pytest.mark.gpu

CASES_2D = [(12, 4, 2), (40, 24, 3), (96, 40, 4)]         # (nel_long, nel_short, levels)
CASES_3D = [(8, 4, 4, 2), (16, 8, 8, 3), (24, 12, 8, 3)]


def _problem(case):
    if len(case) == 3:
        return synthetic.column_2d(case[0], case[1], seed=11, radius=2, mg_levels=case[2],
                                   eig_level=1, num_modes=2)
    return synthetic.cantilever_3d(case[0], case[1], case[2], seed=12, radius=2, volfrac=0.4,
                                   mg_levels=case[3], eig_level=min(2, case[3]), num_modes=2)


@pytest.mark.parametrize("case", CASES_2D + CASES_3D)
def test_fine_Kv_matches_assembled_K(case):
    torch, pkg = require_gpu()
    p = _problem(case)
    s = pkg.Solver(p)
    rng = np.random.default_rng(1)
    nr = 3
    V = rng.standard_normal((nr, p.num_dofs))
    V[:, p.fixed == 1] = 0.0
    y = torch.zeros((nr, p.num_dofs), dtype=torch.float64, device="cuda")
    s.apply_K(1, to_dev(torch, V), y, nr)
    K = assembly.assemble_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin)
    ref = (K @ V.T).T
    ref[:, p.fixed == 1] = 0.0
    assert rel_err(y.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("case", CASES_2D + CASES_3D)
def test_galerkin_levels_match_explicit_triple_products(case):
    torch, pkg = require_gpu()
    p = _problem(case)
    s = pkg.Solver(p)
    op = lba.Problem(p)
    nels, fixeds, Ps = transfer.hierarchy(p.nel, p.dim, p.fixed, p.mg_levels)
    Kl = op.Kf
    rng = np.random.default_rng(2)
    for j in range(1, p.mg_levels):
        Kl = (Ps[j - 1].T @ Kl @ Ps[j - 1]).tocsr()
        info = s.level_info(j + 1)
        v = rng.standard_normal(info["n"])
        v[fixeds[j] == 1] = 0.0
        y = torch.zeros(info["n"], dtype=torch.float64, device="cuda")
        s.apply_K(j + 1, to_dev(torch, v), y, 1)
        free = fixeds[j] == 0
        ref = np.zeros(info["n"])
        ref[free] = Kl @ v[free]
        assert rel_err(y.cpu().numpy(), ref) < 1e-12, j


@pytest.mark.parametrize("case", CASES_2D + CASES_3D)
def test_linear_analysis_residual_and_oracle(case):
    torch, pkg = require_gpu()
    p = _problem(case)
    s = pkg.Solver(p)
    J, info = s.solve_equilibrium()
    u = s.get_field(pkg.TOBK_FIELD_U)
    op = lba.Problem(p)
    res = np.linalg.norm(p.f[op.free] - op.Kf @ u[op.free]) / np.linalg.norm(p.f[op.free])
    assert res <= 1e-8, res
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    uo, Jo = lba.linear_analysis(op)
    e = u[op.free] - uo[op.free]
    assert np.sqrt(e @ (op.Kf @ e)) / np.sqrt(uo[op.free] @ (op.Kf @ uo[op.free])) < 1e-6
    assert J == pytest.approx(Jo, rel=1e-7)
    assert np.all(u[p.fixed == 1] == 0.0)


@pytest.mark.parametrize("case", [CASES_2D[1], CASES_3D[1]])
def test_stress_stiffness_Gv(case):
    torch, pkg = require_gpu()
    p = _problem(case)
    s = pkg.Solver(p)
    s.solve_equilibrium()
    u = s.get_field(pkg.TOBK_FIELD_U)
    G = assembly.assemble_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin)
    rng = np.random.default_rng(3)
    V = rng.standard_normal((2, p.num_dofs))
    V[:, p.fixed == 1] = 0.0
    y = torch.zeros((2, p.num_dofs), dtype=torch.float64, device="cuda")
    s.apply_G(1, to_dev(torch, V), y, 2)
    ref = (G @ V.T).T
    ref[:, p.fixed == 1] = 0.0
    assert rel_err(y.cpu().numpy(), ref) < 1e-12
    if p.eig_level > 1:   # Galerkin G on level 2
        op = lba.Problem(p)
        Gf = assembly.restrict_free(G, p.fixed)
        nels, fixeds, Ps = transfer.hierarchy(p.nel, p.dim, p.fixed, 2)
        G2 = Ps[0].T @ Gf @ Ps[0]
        info = s.level_info(2)
        v = rng.standard_normal(info["n"]); v[fixeds[1] == 1] = 0.0
        y2 = torch.zeros(info["n"], dtype=torch.float64, device="cuda")
        s.apply_G(2, to_dev(torch, v), y2, 1)
        ref2 = np.zeros(info["n"]); ref2[fixeds[1] == 0] = G2 @ v[fixeds[1] == 0]
        assert rel_err(y2.cpu().numpy(), ref2) < 1e-12


@pytest.mark.parametrize("level", [1, 2])
def test_multi_rhs_solve(level):
    torch, pkg = require_gpu()
    p = _problem(CASES_2D[2])
    s = pkg.Solver(p, max_rhs=7)
    nels, fixeds, Ps = transfer.hierarchy(p.nel, p.dim, p.fixed, p.mg_levels)
    info = s.level_info(level)
    rng = np.random.default_rng(4)
    B = rng.standard_normal((7, info["n"]))
    B[:, fixeds[level - 1] == 1] = 0.0
    X = torch.zeros((7, info["n"]), dtype=torch.float64, device="cuda")
    si = s.solve(level, to_dev(torch, B), X, 7)
    op = lba.Problem(p)
    Kl = op.Kf
    for j in range(level - 1):
        Kl = Ps[j].T @ Kl @ Ps[j]
    free = fixeds[level - 1] == 0
    Xn = X.cpu().numpy()
    for r in range(7):
        res = np.linalg.norm(B[r, free] - Kl @ Xn[r, free]) / np.linalg.norm(B[r, free])
        assert res <= 1e-8
    assert si["converged"] == 1


def test_fp32_vcycle_flexible_cg_reaches_same_tolerance():
    torch, pkg = require_gpu()
    for case in (CASES_2D[2], CASES_3D[1]):
        p = _problem(case)
        s = pkg.Solver(p, precision=pkg.TOBK_FP32_VCYCLE)
        J, info = s.solve_equilibrium()
        u = s.get_field(pkg.TOBK_FIELD_U)
        op = lba.Problem(p)
        res = np.linalg.norm(p.f[op.free] - op.Kf @ u[op.free]) / np.linalg.norm(p.f[op.free])
        assert res <= 1e-8
        uo, Jo = lba.linear_analysis(op)
        assert J == pytest.approx(Jo, rel=1e-7)


def test_graph_replayed_solves_match_direct_launches():
    """On a non-default stream the CG iterations replay a captured CUDA graph; the iterates must be
    identical to the directly launched ones (same kernels, same order)."""
    torch, pkg = require_gpu()
    p = _problem(CASES_2D[2])
    s1 = pkg.Solver(p)                                   # legacy default stream: direct launches
    stream = torch.cuda.Stream()
    s2 = pkg.Solver(p, stream=stream)                    # graph replay
    J1, i1 = s1.solve_equilibrium()
    J2, i2 = s2.solve_equilibrium()
    J3, i3 = s2.solve_equilibrium()                      # second solve replays the cached graph
    u1 = s1.get_field(pkg.TOBK_FIELD_U)
    u2 = s2.get_field(pkg.TOBK_FIELD_U)
    assert i1["iterations"] == i2["iterations"] == i3["iterations"]
    assert np.array_equal(u1, u2)
    assert J1 == J2 == J3


@pytest.mark.parametrize("case", [CASES_2D[2], CASES_3D[1]])
def test_two_stream_split_solve_is_bit_identical(case):
    """A multi-RHS solve on a caller's stream runs its right-hand sides as two halves on two streams;
    every RHS is an independent CG recurrence with the same kernels, so the solutions and iteration
    counts must equal those of the single-stream launch sequence (the legacy stream, which never
    splits) bit for bit, for an odd RHS count too."""
    torch, pkg = require_gpu()
    p = _problem(case)
    rng = np.random.default_rng(7)
    for nr in (2, 5):
        B = rng.standard_normal((nr, p.num_dofs))
        B[:, p.fixed == 1] = 0.0
        out = []
        for stream in (None, torch.cuda.Stream()):
            s = pkg.Solver(p, stream=stream, max_rhs=nr)
            s.solve_equilibrium()
            X = torch.zeros((nr, p.num_dofs), dtype=torch.float64, device="cuda")
            info = s.solve(1, to_dev(torch, B), X, nr)
            info2 = s.solve(1, to_dev(torch, B), X, nr)        # replays the halves' cached graphs
            torch.cuda.synchronize()
            out.append((X.cpu().numpy(), info["iterations"], info2["iterations"]))
            s.close()
        assert out[0][1] == out[1][1] == out[1][2]
        assert np.array_equal(out[0][0], out[1][0])

