"""The tensor-core Gram product of the eigensolver (tobk_gram_tc: error-free splitting of FP64
vectors into bfloat16 digit planes, exact accumulation, Ozaki et al. 2012) against exactly rounded
dot products (every product split exactly by Dekker's method, the pieces summed by math.fsum), on
ragged sizes and vectors with widely spread magnitudes; and the eigensolver with tensor-core and
with FP64 CUDA-core Gram products giving the same load factors."""
import ctypes as C
import math

import numpy as np
import pytest

import synthetic
from oracle import lba
from tests.gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _two_prod(a, b):
    """a * b = p + e exactly (Dekker's splitting, no fused multiply-add)."""
    sp = 134217729.0
    p = a * b
    ca, cb = sp * a, sp * b
    ah = ca - (ca - a)
    al = a - ah
    bh = cb - (cb - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _exact_gram(A, B):
    out = np.zeros((A.shape[0], B.shape[0]))
    for i in range(A.shape[0]):
        for j in range(B.shape[0]):
            p, e = _two_prod(A[i], B[j])
            out[i, j] = math.fsum(np.concatenate([p, e]))
    return out


def _vectors(rng, count, n, spread=True):
    X = rng.standard_normal((count, n))
    if spread:
        X *= 2.0 ** rng.integers(-30, 30, size=(count, 1))          # per-vector scale
        small = rng.random((count, n)) < 0.3                          # entries far below the vector's top
        X *= np.where(small, 2.0 ** rng.integers(-40, 1, size=(count, n)), 1.0)
    return X


SHAPES = [(1, 1, 1), (17, 24, 63), (64, 24, 64), (12, 33, 65), (64, 64, 200), (12, 12, 9922)]


@pytest.mark.parametrize("na,nb,n", SHAPES)
def test_gram_tc_matches_exactly_rounded_products(na, nb, n):
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    lib = binding.load()
    rng = np.random.default_rng(na * 1000 + nb * 10 + n)
    A = _vectors(rng, na, n)
    B = _vectors(rng, nb, n)
    if na > 3:
        A[2] = 0.0                                      # a zero vector
    C_ = torch.zeros((na, nb), dtype=torch.float64, device="cuda")
    Ad, Bd = to_dev(torch, A), to_dev(torch, B)        # keep both alive across the call
    rc = lib.tobk_gram_tc(Ad.data_ptr(), na, Bd.data_ptr(), nb, n, n, C_.data_ptr(), None)
    assert rc == binding.TOBK_OK
    got = C_.cpu().numpy()
    ref = _exact_gram(A, B)
    bound = 4 * n * 2.0 ** -53 * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :]
    assert np.all(np.abs(got - ref) <= bound), np.abs(got - ref).max()
    # as accurate as the FP64 dot product (within a factor 2 of its error, or at the bound)
    fp64 = A @ B.T
    assert np.abs(got - ref).max() <= max(2 * np.abs(fp64 - ref).max(), bound.max())


def test_gram_tc_argument_and_nonfinite_checks():
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import binding
    lib = binding.load()
    A = torch.ones((65, 100), dtype=torch.float64, device="cuda")
    Cm = torch.zeros((65, 65), dtype=torch.float64, device="cuda")
    assert lib.tobk_gram_tc(A.data_ptr(), 65, A.data_ptr(), 2, 100, 100, Cm.data_ptr(), None) == binding.TOBK_E_ARG
    assert lib.tobk_gram_tc(A.data_ptr(), 2, A.data_ptr(), 2, 100, 50, Cm.data_ptr(), None) == binding.TOBK_E_ARG
    A[1, 7] = float("nan")
    assert lib.tobk_gram_tc(A.data_ptr(), 3, A.data_ptr(), 2, 100, 100, Cm.data_ptr(), None) == binding.TOBK_E_NONFINITE


@pytest.mark.parametrize("eig_level", [1, 3])
def test_eigensolver_same_with_and_without_tensor_cores(eig_level):
    torch, pkg = require_gpu()
    p = synthetic.column_2d(96, 32, seed=23, radius=3, mg_levels=4, eig_level=eig_level, num_modes=6)
    lams = []
    for tc in (1, 0):
        s = pkg.Solver(p, eig_gram_tc=tc)
        s.solve_equilibrium()
        lam, info = s.compute_buckling()
        assert info["converged"] == 1
        lams.append(lam)
        s.close()
    assert np.allclose(lams[0], lams[1], rtol=1e-9, atol=0)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    ref = lba.exact_lba(op, u, 6)[0] if eig_level == 1 else lba.multilevel_lba(op, u, 6, eig_level)["lam"]
    assert lams[0][0] == pytest.approx(ref[0], rel=1e-6)
