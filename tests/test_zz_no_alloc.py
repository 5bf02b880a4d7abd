"""The allocation-free residual check (tobk_residual_noalloc) against the handle-based solver.

tobk_residual_noalloc serves callers that may not allocate device memory (for example code running
under CUDA stream capture, or inside another framework's memory pool).  It keeps its reduction
scratch in a fixed device array of the library.  This test calls it through the C-ABI on the
solution of tobk_solve and checks that it reproduces the true relative residuals the solver reports
(tobk_solve's rel_residual is the largest of them), on two calls in a row so that reuse of the
shared scratch is covered.  The file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synthetic
from oracle import lba
from tests.gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_residual_matches_solver(dim):
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    lib = binding.load()
    if dim == 2:
        p = synthetic.column_2d(64, 32, seed=31, radius=2, mg_levels=3, eig_level=1, num_modes=2)
    else:
        p = synthetic.cantilever_3d(16, 8, 8, seed=32, radius=2, volfrac=0.4, mg_levels=2, eig_level=1,
                                    num_modes=2)
    nr = 5
    s = pkg.Solver(p, max_rhs=nr)
    rng = np.random.default_rng(7)
    Bh = rng.standard_normal((nr, p.num_dofs))
    Bh[:, p.fixed == 1] = 0.0
    B = to_dev(torch, Bh)
    X = torch.zeros((nr, p.num_dofs), dtype=torch.float64, device="cuda")
    info = s.solve(1, B, X, nr)                       # existing entry point
    assert info["converged"] == 1
    x = to_dev(torch, p.x)
    fixed = to_dev(torch, p.fixed.astype(np.uint8))
    # the oracle's own residuals of the same solutions (independent reference)
    op = lba.Problem(p)
    Xh = X.cpu().numpy()
    ref = np.array([np.linalg.norm(Bh[r, op.free] - op.Kf @ Xh[r, op.free]) / np.linalg.norm(Bh[r, op.free])
                    for r in range(nr)])
    for call in range(2):                              # two calls in a row share the scratch
        relres = torch.full((nr,), -1.0, dtype=torch.float64, device="cuda")
        rc = lib.tobk_residual_noalloc(C.byref(s.desc), x.data_ptr(), fixed.data_ptr(), B.data_ptr(),
                                       X.data_ptr(), nr, relres.data_ptr(), None)
        assert rc == binding.TOBK_OK
        torch.cuda.synchronize()
        got = relres.cpu().numpy()
        assert np.all(got > 0.0)
        assert got.max() == pytest.approx(info["rel_residual"], rel=1e-9)
        assert np.allclose(got, ref, rtol=1e-6)
        assert np.all(got <= 1e-8)
    s.close()


def _desc(binding, lib, p, **kw):
    d = binding.tobk_desc()
    lib.tobk_default_desc(C.byref(d))
    d.dim, d.nel[0], d.nel[1] = p.dim, p.nel[0], p.nel[1]
    d.nel[2] = p.nel[2] if p.dim == 3 else 1
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_noalloc_sixteen_rhs_on_a_grid_wider_than_its_block_cap():
    """nrhs = 16 (the limit) on a 2D grid of 263,425 nodes, more than the 1024 blocks x 256 threads
    of the fixed grid width (the grid-stride loop covers the rest), for arbitrary B and X: every
    relres agrees with the oracle's element-by-element K X.  Entries of X at fixed DOFs are read as
    zero, so setting them changes nothing."""
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    from oracle import assembly
    lib = binding.load()
    p = synthetic.column_2d(1024, 256, seed=33, radius=2, mg_levels=1)
    assert p.num_nodes > 1024 * 256
    nr = 16
    rng = np.random.default_rng(8)
    Bh = rng.standard_normal((nr, p.num_dofs))
    Xh = rng.standard_normal((nr, p.num_dofs))
    free = p.fixed == 0
    Xf = Xh.copy()
    Xf[:, ~free] = 0.0
    KX = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, Xf)
    ref = np.linalg.norm((Bh - KX)[:, free], axis=1) / np.linalg.norm(Bh[:, free], axis=1)
    d = _desc(binding, lib, p)
    x = to_dev(torch, p.x)
    fixed = to_dev(torch, p.fixed.astype(np.uint8))
    B, X = to_dev(torch, Bh), to_dev(torch, Xh)
    for call in range(2):
        relres = torch.full((nr,), -1.0, dtype=torch.float64, device="cuda")
        rc = lib.tobk_residual_noalloc(C.byref(d), x.data_ptr(), fixed.data_ptr(), B.data_ptr(), X.data_ptr(), nr,
                                       relres.data_ptr(), None)
        assert rc == binding.TOBK_OK
        torch.cuda.synchronize()
        assert np.allclose(relres.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_bad_arguments():
    """Null pointers, empty grids and the material checks of tobk_create are rejected with
    TOBK_E_ARG before anything is launched."""
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    lib = binding.load()
    p = synthetic.cantilever_3d(4, 2, 2, seed=1, radius=1.5, volfrac=0.5, mg_levels=1)
    buf = torch.zeros(p.num_dofs, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = to_dev(torch, p.x)
    fixed = to_dev(torch, p.fixed.astype(np.uint8))

    def call(d, xp=x.data_ptr(), bp=buf.data_ptr(), op=out.data_ptr(), nr=1):
        return lib.tobk_residual_noalloc(C.byref(d), xp, fixed.data_ptr(), bp, bp, nr, op, None)

    assert call(_desc(binding, lib, p)) == binding.TOBK_OK
    for kw in (dict(nu=0.5), dict(nu=-1.0), dict(E0=0.0), dict(Emin=-1e-6), dict(penal=0.5), dict(dim=4)):
        assert call(_desc(binding, lib, p, **kw)) == binding.TOBK_E_ARG, kw
    d = _desc(binding, lib, p)
    d.nel[1] = 0
    assert call(d) == binding.TOBK_E_ARG
    assert call(_desc(binding, lib, p), xp=None) == binding.TOBK_E_ARG
    assert call(_desc(binding, lib, p), bp=None) == binding.TOBK_E_ARG
    assert call(_desc(binding, lib, p), op=None) == binding.TOBK_E_ARG
    assert call(_desc(binding, lib, p), nr=0) == binding.TOBK_E_ARG
    torch.cuda.synchronize()


def test_noalloc_rejects_too_many_rhs():
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    lib = binding.load()
    p = synthetic.column_2d(8, 4, seed=1, radius=1.5, mg_levels=1)
    d = binding.tobk_desc()
    lib.tobk_default_desc(C.byref(d))
    d.dim, d.nel[0], d.nel[1] = 2, p.nel[0], p.nel[1]
    buf = torch.zeros(17 * p.num_dofs, dtype=torch.float64, device="cuda")
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    x = to_dev(torch, p.x)
    fixed = to_dev(torch, p.fixed.astype(np.uint8))
    rc = lib.tobk_residual_noalloc(C.byref(d), x.data_ptr(), fixed.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                   17, out.data_ptr(), None)
    assert rc == binding.TOBK_E_ARG
    assert b"between 1 and 16" in lib.tobk_last_error(None)
