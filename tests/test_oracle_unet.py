"""Pins of the learned warm start's oracle (oracle/unet.py): the 3x3x3 convolution against a
brute-force loop, the adjoint pairs (pooling / upsampling, node averaging) by inner products, and
the whole backward pass against central finite differences of the loss."""
import numpy as np
import pytest

from oracle import unet

import synthetic


def test_conv3_equals_brute_force_loops():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = unet.conv3(a, w, b)
    C, D, H, W = a.shape
    ref = np.zeros((3, D, H, W))
    for o in range(3):
        for z in range(D):
            for y in range(H):
                for x in range(W):
                    s = b[o]
                    for i in range(C):
                        for t in range(27):
                            dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if 0 <= zz < D and 0 <= yy < H and 0 <= xx < W:
                                s += w[o, i, t] * a[i, zz, yy, xx]
                    ref[o, z, y, x] = s
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_adjoint_pairs():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 4, 4, 6))
    g = rng.standard_normal((2, 2, 2, 3))
    assert np.isclose(np.sum(unet.avgpool(a) * g), np.sum(a * unet.avgpool_backward(g)))
    assert np.isclose(np.sum(unet.up(g) * a), np.sum(g * unet.up_backward(a)))
    y = rng.standard_normal((3, 2, 3, 4))
    t, cnt = unet.node_average(y)
    gt = rng.standard_normal(t.shape)
    assert np.isclose(np.sum(t * gt), np.sum(y * unet.node_average_backward(gt, y.shape, cnt)))
    assert np.allclose(cnt.max(), 8) and np.allclose(cnt.min(), 1)


def test_bf16_rounding_is_round_to_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1e-3], dtype=np.float64)
    r = unet.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] - 1e-3) <= 2 ** -8 * 1e-3


def test_bf16_activations_change_the_prediction_by_bf16_rounding_only():
    """act_bf16 rounds every 3x3x3 convolution input to bfloat16: the prediction moves by about the
    bfloat16 resolution (2^-8 relative per operand), not more, and is not identical."""
    L, ch = 2, [16, 16]
    p = synthetic.cantilever_3d(8, 4, 4, seed=4, radius=1.5, volfrac=0.4, mg_levels=1, eig_level=1, num_modes=1)
    rng = np.random.default_rng(7)
    theta = 0.15 * rng.standard_normal(unet.num_params(L, ch))
    a = unet.predict(theta, p.x, p.f, p.fixed, p.nel, L, ch, out_scale=10.0)
    b = unet.predict(theta, p.x, p.f, p.fixed, p.nel, L, ch, out_scale=10.0, act_bf16=True)
    d = np.abs(a - b).max() / np.abs(a).max()
    assert 0.0 < d < 2e-2


@pytest.mark.parametrize("loss", ["energy", "mse"])
def test_gradient_matches_central_differences(loss):
    L, ch = 2, [2, 3]
    p = synthetic.cantilever_3d(4, 2, 2, seed=3, radius=1.5, volfrac=0.4, mg_levels=1, eig_level=1,
                                num_modes=1)
    rng = np.random.default_rng(2)
    theta = 0.3 * rng.standard_normal(unet.num_params(L, ch))
    u = rng.standard_normal(p.num_dofs) * 1e2
    u[p.fixed == 1] = 0.0
    value, g = unet.gradient(theta, p.x, p.f, u, p.fixed, p.nel, L, ch, bf16=False, out_scale=3.0, loss=loss)
    assert g.shape == theta.shape and value > 0
    idx = rng.choice(theta.size, 25, replace=False)
    for k in idx:
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        lp, _ = unet.gradient(tp, p.x, p.f, u, p.fixed, p.nel, L, ch, bf16=False, out_scale=3.0, loss=loss)
        lm, _ = unet.gradient(tm, p.x, p.f, u, p.fixed, p.nel, L, ch, bf16=False, out_scale=3.0, loss=loss)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, fd, g[k])


def test_energy_loss_is_the_relative_energy_error_of_the_guess():
    """With the exact solution as target, the energy loss equals (u0 - u)^T K (u0 - u) / u^T K u of
    the guess u0 = t / s on the free DOFs, computed directly from an assembled K."""
    import synthetic
    from oracle import assembly, lba
    L, ch = 2, [2, 3]
    p = synthetic.cantilever_3d(4, 2, 2, seed=6, radius=1.5, volfrac=0.4, mg_levels=1, eig_level=1, num_modes=1)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    rng = np.random.default_rng(4)
    theta = 0.3 * rng.standard_normal(unet.num_params(L, ch))
    c = 2.5
    value, _ = unet.gradient(theta, p.x, p.f, u, p.fixed, p.nel, L, ch, out_scale=c, loss="energy")
    u0 = unet.predict(theta, p.x, p.f, p.fixed, p.nel, L, ch, out_scale=c)
    e = (u0 - u)[op.free]
    assert value == pytest.approx(e @ (op.Kf @ e) / (u[op.free] @ (op.Kf @ u[op.free])), rel=1e-10)
