"""GPU parity at the benchmark's full sizes and launch configurations (the settings bench.py times):
column480x160 in FP64 (the headline step) against the oracle's direct solves and multilevel LBA;
cantilever96x48x48 with the FP32 V-cycle and the fused load + adjoint launch through properties that
hold at any size, evaluated with the oracle's assembly-free K v and G v (true residuals of u and of
the adjoint systems, the Rayleigh quotients and K-normalisation of the returned modes); sampled
designs of the 64-design batch."""
import numpy as np
import pytest

import synthetic
from oracle import assembly, lba, sensitivity
from tests.gpu_util import require_gpu

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


def _relres(p, U, B):
    """max over rows of ||B - K U|| / ||B|| on the free DOFs (oracle operator, no assembly)."""
    KU = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, U)
    free = p.fixed == 0
    B = np.atleast_2d(B)
    return max(np.linalg.norm((B[r] - KU[r])[free]) / np.linalg.norm(B[r][free]) for r in range(B.shape[0]))


def test_column480x160_fp64_step_matches_oracle():
    torch, pkg = require_gpu()
    p = synthetic.config("column480x160")
    s = pkg.Solver(p, stream=torch.cuda.Stream())
    J, i1 = s.solve_equilibrium()
    lam, i2 = s.compute_buckling()
    dlam, dJ, i3 = s.compute_sensitivities()
    u = s.get_field(pkg.TOBK_FIELD_U)
    assert _relres(p, u, p.f) <= 1e-8
    op = lba.Problem(p)
    uo, Jo = lba.linear_analysis(op)
    assert J == pytest.approx(Jo, rel=1e-7)
    ml = lba.multilevel_lba(op, uo, p.num_modes, p.eig_level)
    ok = _gaps(ml["lam_coarse"]) > 1e-4
    assert np.allclose(lam[ok], ml["lam"][ok], rtol=1e-6, atol=0), (lam, ml["lam"])
    # sensitivities of the well-separated pairs (same formula on the oracle's pairs)
    dlo, dJo, _ = sensitivity.sensitivities(op, uo, ml["lam"], ml["Phi"])
    assert np.abs(dJ - dJo).max() <= 1e-5 * np.abs(dJo).max()
    for i in np.flatnonzero(ok & (_gaps(ml["lam"]) > 1e-4)):
        assert np.abs(dlam[i] - dlo[i]).max() <= 1e-5 * np.abs(dlo[i]).max(), i
    s.close()


def test_cantilever96x48x48_fp32_fused_properties():
    torch, pkg = require_gpu()
    p = synthetic.config("cantilever96x48x48")
    s = pkg.Solver(p, stream=torch.cuda.Stream(), precision=pkg.TOBK_FP32_VCYCLE, fuse_load_adjoint=1)
    J, _ = s.solve_equilibrium()
    lam, info = s.compute_buckling()
    assert info["converged"] == 1
    s.compute_sensitivities()
    u = s.get_field(pkg.TOBK_FIELD_U)
    q, n = p.num_modes, p.num_dofs
    Phi = s.get_field(pkg.TOBK_FIELD_MODES).reshape(q, n)
    Z = s.get_field(pkg.TOBK_FIELD_ADJOINT).reshape(q, n)
    Bz = s.get_field(pkg.TOBK_FIELD_ADJOINT_RHS).reshape(q, n)
    assert _relres(p, u, p.f) <= 1e-8
    assert J == pytest.approx(float(p.f @ u), rel=1e-12)
    # modes: K-normalised, lambda = Rayleigh quotient -phi^T K phi / phi^T G phi (oracle operators)
    KP = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, Phi)
    GP = assembly.apply_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin, Phi)
    free = p.fixed == 0
    for i in range(q):
        kk = Phi[i][free] @ KP[i][free]
        gg = Phi[i][free] @ GP[i][free]
        assert kk == pytest.approx(1.0, rel=1e-8)
        assert lam[i] == pytest.approx(-kk / gg, rel=1e-8)
    assert np.all(np.diff(lam) >= 0) and lam[0] > 0
    # adjoint right-hand sides (oracle element formula on the GPU's modes) and adjoint solutions
    Bo = np.stack([sensitivity.adjoint_rhs(p.nel, p.dim, p.x, Phi[i], p.nu, p.penal, p.E0, p.Emin) for i in range(3)])
    Bo[:, p.fixed == 1] = 0.0
    assert np.abs(Bz[:3] - Bo).max() <= 1e-10 * np.abs(Bo).max()
    assert _relres(p, Z, Bz) <= 1e-8
    s.close()


def test_batch64_sampled_designs_against_oracle():
    torch, pkg = require_gpu()
    problems = synthetic.batch_configs(64)
    nrhs = 7
    rng = np.random.default_rng(11)
    blocks = []
    for p in problems:
        B = rng.standard_normal((nrhs, p.num_dofs))
        B[0] = p.f
        B[:, p.fixed == 1] = 0.0
        blocks.append(B)
    bt = pkg.Batch(problems, nrhs, stream=torch.cuda.Stream())
    bt.set_designs(np.concatenate([p.x for p in problems]), np.concatenate([p.fixed for p in problems]).astype(np.uint8))
    bt.autotune()
    B = torch.from_numpy(np.concatenate([b.reshape(-1) for b in blocks])).cuda()
    X = torch.zeros_like(B)
    infos, _ = bt.solve(B, X)
    assert all(i["converged"] == 1 for i in infos)
    Xh = X.cpu().numpy()
    off = bt.dof_offsets
    for d in (0, 17, 40, 63):
        p = problems[d]
        Xd = Xh[nrhs * off[d]: nrhs * off[d + 1]].reshape(nrhs, p.num_dofs)
        assert _relres(p, Xd, blocks[d]) <= 1e-8 * 1.01, d
    bt.close()
