"""GPU parity of the batched solver (many designs of uneven size in one set of grouped launches)
against the oracle: every design's K(x_d) X_d = B_d solved to relative residual 1e-8 by FP64 flexible
CG with the FP32 V-cycle (the mgPCG of Appendix A), for every autotuner variant of the grouped
smoother kernels, and the same solutions as the single-design solver."""
import numpy as np
import pytest

import synthetic
from oracle import lba
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(32, 16), (48, 16), (64, 16), (96, 32), (64, 32), (40, 8)]  # (nel_long, nel_short)


def _designs():
    out = []
    for k, (a, b) in enumerate(SHAPES):
        out.append(synthetic.column_2d(a, b, seed=300 + k, radius=2.0, volfrac=0.3 + 0.05 * k,
                                       mg_levels=synthetic.batch_levels(a, b, coarsest_short=4),
                                       eig_level=1, num_modes=2, name=f"b{k}"))
    return out


def _packed(designs, nrhs, seed=5):
    rng = np.random.default_rng(seed)
    x = np.concatenate([p.x for p in designs])
    fixed = np.concatenate([p.fixed for p in designs]).astype(np.uint8)
    blocks = []
    for p in designs:
        B = rng.standard_normal((nrhs, p.num_dofs))
        B[0] = p.f
        B[:, p.fixed == 1] = 0.0
        blocks.append(B)
    return x, fixed, blocks


def _check(designs, blocks, X, dof_off, nrhs, tol=1e-8):
    for d, p in enumerate(designs):
        op = lba.Problem(p)
        Xd = X[nrhs * dof_off[d]: nrhs * dof_off[d + 1]].reshape(nrhs, p.num_dofs)
        assert np.all(Xd[:, p.fixed == 1] == 0.0)
        for r in range(nrhs):
            b = blocks[d][r][op.free]
            res = np.linalg.norm(b - op.Kf @ Xd[r][op.free]) / np.linalg.norm(b)
            assert res <= tol * 1.01, (d, r, res)


def test_batch_solve_matches_oracle_for_every_variant():
    torch, pkg = require_gpu()
    designs = _designs()
    nrhs = 3
    x, fixed, blocks = _packed(designs, nrhs)
    bt = pkg.Batch(designs, nrhs)
    dof = bt.dof_offsets
    assert dof[-1] == sum(p.num_dofs for p in designs)
    bt.set_designs(torch.from_numpy(x).cuda(), torch.from_numpy(fixed).cuda())
    B = torch.from_numpy(np.concatenate([b.reshape(-1) for b in blocks])).cuda()
    fv, cv = bt.autotune()
    assert 0 <= fv < 4 and 0 <= cv < 3
    ref = None
    for fine in range(4):
        for coarse in range(3):
            bt.set_variants(fine, coarse)
            X = torch.zeros_like(B)
            infos, _ = bt.solve(B, X)
            for inf in infos:
                assert inf["converged"] == 1 and inf["rel_residual"] <= 1e-8
            Xh = X.cpu().numpy()
            _check(designs, blocks, Xh, dof, nrhs)
            if ref is None:
                ref = Xh
            else:  # the variants differ only in the FP32 preconditioner's blocking
                assert np.abs(Xh - ref).max() <= 1e-6 * np.abs(ref).max()
    # exact solutions from the oracle (direct solve) agree in the energy norm
    for d, p in enumerate(designs):
        op = lba.Problem(p)
        u, _ = lba.linear_analysis(op)
        ud = ref[nrhs * dof[d]: nrhs * dof[d] + p.num_dofs]
        e = ud[op.free] - u[op.free]
        assert np.sqrt(e @ (op.Kf @ e)) <= 1e-6 * np.sqrt(u[op.free] @ (op.Kf @ u[op.free]))
    bt.close()


def test_batch_host_buffers_repeat_and_match_single_design_solver():
    torch, pkg = require_gpu()
    designs = _designs()[:4]
    nrhs = 2
    x, fixed, blocks = _packed(designs, nrhs, seed=9)
    bt = pkg.Batch(designs, nrhs)
    bt.set_designs(x, fixed)
    B = np.concatenate([b.reshape(-1) for b in blocks])
    X1 = np.zeros_like(B)
    X2 = np.zeros_like(B)
    bt.solve(B, X1)
    bt.solve(B, X2)  # replayed graph: identical
    assert np.array_equal(X1, X2)
    _check(designs, blocks, X1, bt.dof_offsets, nrhs)
    dof = bt.dof_offsets
    for d, p in enumerate(designs):
        s = pkg.Solver(p, precision=pkg.TOBK_FP32_VCYCLE, max_rhs=nrhs)
        Bd = torch.from_numpy(blocks[d].copy()).cuda()
        Xd = torch.zeros_like(Bd)
        s.solve(1, Bd, Xd, nrhs)
        ref = Xd.cpu().numpy().reshape(-1)
        got = X1[nrhs * dof[d]: nrhs * dof[d + 1]]
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
        s.close()
    bt.close()


def test_batch_rejects_bad_descriptors():
    torch, pkg = require_gpu()
    p3 = synthetic.cantilever_3d(8, 4, 4, seed=1, radius=2, volfrac=0.4, mg_levels=2, eig_level=1, num_modes=2)
    with pytest.raises(pkg.TobkError):
        pkg.Batch([p3], 1)
    p2 = _designs()[0]
    with pytest.raises(pkg.TobkError):
        pkg.Batch([p2], 0)
