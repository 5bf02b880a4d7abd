"""GPU parity of the learned warm start (the 3D U-Net's hand-written forward, backward and Adam
kernels) against the NumPy oracle (oracle/unet.py): loss, gradient of every parameter, prediction;
checkpoint round trip; and that Adam steps lower the loss."""
import numpy as np
import pytest

import synthetic
from oracle import unet as ou
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

NEL, LEVELS, CH = (16, 8, 8), 3, (16, 16, 32)


def _sample(seed=0):
    p = synthetic.cantilever_3d(*NEL, seed=seed, radius=2.0, volfrac=0.35, mg_levels=1, eig_level=1, num_modes=1)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(p.num_dofs) * 50.0
    u[p.fixed == 1] = 0.0
    return p, u


def _theta(n, seed=3, scale=0.15):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(n)).astype(np.float32)


def _smooth_target(p):
    """A smooth displacement field (cantilever-like bending) the network can fit."""
    nx, ny, nz = p.nel
    z, y, x = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    u = np.zeros((z.size, 3))
    u[:, 2] = -((x.reshape(-1) / nx) ** 2) * 100.0
    u[:, 0] = (z.reshape(-1) / nz - 0.5) * (x.reshape(-1) / nx) * 20.0
    u = u.reshape(-1)
    u[p.fixed == 1] = 0.0
    return u


@pytest.mark.parametrize("kind", ["energy", "mse"])
def test_loss_gradient_and_prediction_match_oracle(kind):
    torch, pkg = require_gpu()
    net = pkg.UNet(NEL, LEVELS, CH, loss=pkg.binding.TOBK_UNET_LOSS_ENERGY if kind == "energy" else
                   pkg.binding.TOBK_UNET_LOSS_MSE)
    assert net.num_params == ou.num_params(LEVELS, list(CH))
    theta = _theta(net.num_params)
    net.set_state(torch.from_numpy(theta).cuda())
    c = 37.5
    net.set_output_scale(c)
    assert net.output_scale() == c
    p, _ = _sample()
    rng = np.random.default_rng(5)
    u = _smooth_target(p) * (1.0 + 0.1 * rng.standard_normal(p.num_dofs))  # u . f > 0 for the energy loss
    u[p.fixed == 1] = 0.0
    x32 = torch.from_numpy(p.x.astype(np.float32)).cuda()
    f = torch.from_numpy(p.f).cuda()
    fx = torch.from_numpy(p.fixed.astype(np.uint8)).cuda()
    tgt = torch.from_numpy(u.astype(np.float32)).cuda()
    g = torch.zeros(net.num_params, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(x32, f, tgt, fx, g)
    lo, go = ou.gradient(theta.astype(np.float64), p.x.astype(np.float32).astype(np.float64), p.f,
                         u.astype(np.float32).astype(np.float64), p.fixed, p.nel, LEVELS, list(CH), out_scale=c,
                         loss=kind)
    assert loss == pytest.approx(lo, rel=1e-4)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - go).max() <= 2e-3 * np.abs(go).max()
    # per layer: relative agreement of each layer's gradient block
    k = 0
    for name, co, ci, taps in ou.layer_shapes(LEVELS, list(CH)):
        sz = co * ci * taps + co
        a, b = gg[k:k + sz], go[k:k + sz]
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b) + 1e-12, name
        k += sz
    # prediction with the FP32 direct convolution (the training forward)
    u0 = torch.zeros(p.num_dofs, dtype=torch.float64, device="cuda")
    net.set_tensor_cores(False)
    net.predict(torch.from_numpy(p.x).cuda(), f, fx, u0)
    ref = ou.predict(theta.astype(np.float64), p.x, p.f, p.fixed, p.nel, LEVELS, list(CH), out_scale=c)
    assert np.abs(u0.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()
    # prediction on the tensor cores (tcgen05, activations rounded to bfloat16): against the oracle
    # with the same roundings
    net.set_tensor_cores(2)  # every level (this grid is below the size where mode 1 would use them)
    u1 = torch.zeros(p.num_dofs, dtype=torch.float64, device="cuda")
    net.predict(torch.from_numpy(p.x).cuda(), f, fx, u1)
    ref_bf = ou.predict(theta.astype(np.float64), p.x, p.f, p.fixed, p.nel, LEVELS, list(CH), out_scale=c,
                        act_bf16=True)
    _assert_bf16_prediction(u1.cpu().numpy(), ref_bf)
    net.close()


def _assert_bf16_prediction(got, ref):
    """The two sides' FP32 / FP64 sums differ by ~1e-6, so an activation occasionally rounds to the
    neighbouring bfloat16 value (2^-8 relative) on one side only, and the difference spreads over
    the receptive field of the layers above it.  So: on average the predictions agree to 3e-4 of
    the largest value, 99.9 % of them to one bfloat16 ulp (2^-8), and none by more than 2^-6 (a
    wrong tap, channel or tile would be off by order one)."""
    d = np.abs(got - ref) / np.abs(ref).max()
    assert d.mean() <= 3e-4
    assert np.quantile(d, 0.999) <= 2.0 ** -8
    assert d.max() <= 2.0 ** -6


@pytest.mark.parametrize("cin,cout,dims", [(16, 16, (5, 7, 37)), (4, 16, (3, 9, 20)), (48, 32, (6, 8, 38)),
                                           (128, 64, (4, 6, 30)), (64, 128, (3, 4, 44)),
                                           (16, 16, (3, 4, 128)), (48, 32, (2, 3, 256)), (4, 64, (2, 2, 128))])
def test_tensor_core_conv3_matches_oracle(cin, cout, dims):
    """One 3x3x3 convolution on the tensor cores (tcgen05 implicit GEMM) against the oracle's direct
    convolution, on bfloat16-representable inputs and weights, so that both sides multiply the same
    numbers and differ only by FP32 accumulation (at most 27 * 128 products per output): several
    128-voxel tiles with a ragged last tile, input channels padded to 16, and 16 to 128 outputs; x
    extents that are multiples of 128 take the halo-slab (row) kernel, the others the per-tap gather."""
    torch, pkg = require_gpu()
    rng = np.random.default_rng(cin * 1000 + cout)
    D, H, W = dims
    a = ou.bf16_round(rng.uniform(-1.0, 1.0, (cin, D, H, W)))
    w = ou.bf16_round(rng.uniform(-0.2, 0.2, (cout, cin, 27)))
    b = ou.bf16_round(rng.uniform(-0.1, 0.1, cout))
    ref = ou.relu(ou.conv3(a, w, b))
    out = torch.zeros((cout, D, H, W), dtype=torch.float32, device="cuda")
    pkg.binding.conv3_bf16(torch.from_numpy(a.astype(np.float32)).cuda(),
                           torch.from_numpy(w.astype(np.float32)).cuda(),
                           torch.from_numpy(b.astype(np.float32)).cuda(), out, relu=True)
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    assert (got[ref == 0.0] == 0.0).mean() > 0.99  # ReLU zeros where the exact result is negative


def test_checkpoint_round_trip_and_adam_lowers_the_loss():
    torch, pkg = require_gpu()
    net = pkg.UNet(NEL, LEVELS, CH, seed=7, loss=pkg.binding.TOBK_UNET_LOSS_MSE)
    p, _ = _sample(1)
    u = _smooth_target(p)
    x32 = torch.from_numpy(p.x.astype(np.float32)).cuda()
    f = torch.from_numpy(p.f).cuda()
    fx = torch.from_numpy(p.fixed.astype(np.uint8)).cuda()
    tgt = torch.from_numpy(u.astype(np.float32)).cuda()
    sd = net.design_scale(x32, f)
    _, s_or = ou.features(p.x.astype(np.float32).astype(np.float64), p.f, p.nel)
    assert sd == pytest.approx(s_or, rel=1e-5)
    net.set_output_scale(float(np.sqrt(np.mean((sd * u[p.fixed == 0]) ** 2))))
    l0 = net.loss_grad(x32, f, tgt, fx)
    losses = [net.train_step(x32, f, tgt, fx, 1, 2e-3) for _ in range(40)]
    assert losses[-1] < 0.5 * l0
    n = net.num_params
    P, M, V = (torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(3))
    step = net.get_state(P, M, V)
    assert step == 40
    net2 = pkg.UNet(NEL, LEVELS, CH, seed=99, loss=pkg.binding.TOBK_UNET_LOSS_MSE)
    net2.set_state(P, M, V, step)
    net2.set_output_scale(net.output_scale())
    xd = torch.from_numpy(p.x).cuda()
    a = torch.zeros(p.num_dofs, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    net.predict(xd, f, fx, a)
    net2.predict(xd, f, fx, b)
    assert torch.equal(a, b)
    # both continue identically from the same optimizer state
    assert net.train_step(x32, f, tgt, fx, 1, 2e-3) == net2.train_step(x32, f, tgt, fx, 1, 2e-3)
    net.close()
    net2.close()


def test_tensor_core_prediction_on_128_wide_grid():
    """The whole tensor-core prediction on a grid whose finest level is 128 voxels wide (the row
    kernel, including the decoder's upsampled and concatenated inputs) against the oracle with
    bfloat16 activations, and against the FP32 direct convolution."""
    torch, pkg = require_gpu()
    nel, levels, ch = (128, 8, 8), 3, (16, 16, 32)
    p = synthetic.cantilever_3d(*nel, seed=2, radius=2.0, volfrac=0.35, mg_levels=1, eig_level=1, num_modes=1)
    net = pkg.UNet(nel, levels, ch)
    theta = _theta(net.num_params, seed=9, scale=0.06)  # a gain of about one per layer, as after training
    net.set_state(torch.from_numpy(theta).cuda())
    net.set_output_scale(20.0)
    net.set_tensor_cores(2)
    x = torch.from_numpy(p.x).cuda()
    f = torch.from_numpy(p.f).cuda()
    fx = torch.from_numpy(p.fixed.astype(np.uint8)).cuda()
    u_tc = torch.zeros(p.num_dofs, dtype=torch.float64, device="cuda")
    net.predict(x, f, fx, u_tc)
    ref = ou.predict(theta.astype(np.float64), p.x, p.f, p.fixed, nel, levels, list(ch), out_scale=20.0,
                     act_bf16=True)
    got = u_tc.cpu().numpy()
    _assert_bf16_prediction(got, ref)
    net.set_tensor_cores(False)
    u_fp = torch.zeros_like(u_tc)
    net.predict(x, f, fx, u_fp)
    assert np.abs(got - u_fp.cpu().numpy()).max() <= 3e-2 * np.abs(ref).max()
    net.close()
