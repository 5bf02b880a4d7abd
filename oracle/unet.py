"""Oracle (test infrastructure, not the product path) of the learned warm start: a small 3D U-Net
that maps a density field and its load to a displacement guess u0 for the MGCG solve, its loss
and the gradient of the loss with respect to every parameter.  Plain NumPy in float64: convolutions
as sums of 27 shifted slices, every backward step written out as the adjoint of its forward step.

The network is not part of the paper: the paper's solver path is multigrid-preconditioned CG
(Appendix A); the learned part only supplies the starting iterate, and plain MGCG still runs to the
same tolerance.  Parity pins: finite differences of the loss (tests/test_oracle_unet.py) and a
brute-force convolution on tiny inputs.

Architecture (levels L, channels c[0..L-1], element grid nz x ny x nx, x fastest):
  features: ch0 = 2 x - 1, ch1..3 = the nodal load summed over each element's 8 nodes, divided by
            the largest such sum over the grid
  encoder:  e_0 = R(C(R(C(features)))), e_l = R(C(R(C(avgpool(e_{l-1}))))), l = 1..L-1
  decoder:  d_{L-1} = e_{L-1}; d_l = R(C(R(C([up(d_{l+1}), e_l])))), l = L-2..0
  output:   y = H(d_0) + up^{L-1}(Hc(e_{L-1}))   (3 channels per element; H, Hc: 1x1x1 convolutions)
            the fine head H and the coarse head Hc (the coarse-correction term) share one output
  nodes:    t_a = c x (mean of y over the elements around node a (1..8 of them)), per component,
            c a fixed output scale
  guess:    u0 = t / s at free DOFs (0 at fixed DOFs), s = mean_e E_kappa(x_e) / (largest element
            load sum)
  C = 3x3x3 convolution with zero padding and bias, R = ReLU, up = nearest 2x upsampling,
  avgpool = 2x2x2 mean.
Loss of one sample with target solution u, t* = s u, K the sample's stiffness on the free DOFs:
  energy (default): (t - t*)^T K (t - t*) / t*^T K t*  (K t* = s f), the relative energy-norm error;
  mse:              sum_free (t - t*)^2 / sum_free t*^2.

Parameters, in this order, each conv as weights [Cout][Cin][27] (tap = dz*9 + dy*3 + dx over
offsets -1..1, dz slowest) then bias [Cout]: enc_l a, enc_l b for l = 0..L-1; dec_l a, dec_l b for
l = L-2..0 (decoder input channels: the upsampled coarse channels first, then the skip); head
[3][c0] + [3]; coarse head [3][c_{L-1}] + [3].  The convolutions use the parameters rounded to
bfloat16 (round to nearest even), as the GPU kernels do."""
from __future__ import annotations

import numpy as np


def layer_shapes(levels, channels, cin=4, cout=3):
    """[(name, Cout, Cin, taps)] in parameter order."""
    out = []
    prev = cin
    for l in range(levels):
        out.append((f"enc{l}a", channels[l], prev, 27))
        out.append((f"enc{l}b", channels[l], channels[l], 27))
        prev = channels[l]
    for l in range(levels - 2, -1, -1):
        out.append((f"dec{l}a", channels[l], channels[l + 1] + channels[l], 27))
        out.append((f"dec{l}b", channels[l], channels[l], 27))
    out.append(("head", cout, channels[0], 1))
    out.append(("chead", cout, channels[levels - 1], 1))
    return out


def num_params(levels, channels):
    return sum(co * ci * k + co for _, co, ci, k in layer_shapes(levels, channels))


def unpack(theta, levels, channels):
    """dict name -> (W [Cout][Cin][taps], b [Cout]) views of the flat parameter vector."""
    p, k = {}, 0
    for name, co, ci, taps in layer_shapes(levels, channels):
        w = theta[k:k + co * ci * taps].reshape(co, ci, taps)
        k += co * ci * taps
        b = theta[k:k + co]
        k += co
        p[name] = (w, b)
    return p


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------------------------------------
# building blocks (arrays [C][D][H][W])
# ------------------------------------------------------------------------------------------------
def _shift(a, dz, dy, dx):
    """b[c, z, y, x] = a[c, z + dz, y + dy, x + dx] (zero outside)."""
    C, D, H, W = a.shape
    b = np.zeros_like(a)
    zs, ze = max(0, -dz), min(D, D - dz)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    b[:, zs:ze, ys:ye, xs:xe] = a[:, zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return b


TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3(a, w, b):
    """out[o] = b[o] + sum_i sum_tap w[o, i, tap] a[i](. + tap)"""
    out = np.zeros((w.shape[0],) + a.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = _shift(a, dz, dy, dx)
        out += np.einsum("oi,izyx->ozyx", w[:, :, t], s)
    return out + b[:, None, None, None]


def conv3_backward(a, w, g):
    """Given out = conv3(a, w, b) and g = dL/dout: (dL/da, dL/dw, dL/db)."""
    ga = np.zeros_like(a)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = _shift(a, dz, dy, dx)
        gw[:, :, t] = np.einsum("ozyx,izyx->oi", g, s)
        ga += _shift(np.einsum("oi,ozyx->izyx", w[:, :, t], g), -dz, -dy, -dx)
    return ga, gw, g.sum(axis=(1, 2, 3))


def conv1(a, w, b):
    return np.einsum("oi,izyx->ozyx", w[:, :, 0], a) + b[:, None, None, None]


def conv1_backward(a, w, g):
    return (np.einsum("oi,ozyx->izyx", w[:, :, 0], g), np.einsum("ozyx,izyx->oi", g, a)[:, :, None],
            g.sum(axis=(1, 2, 3)))


def avgpool(a):
    C, D, H, W = a.shape
    return a.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def avgpool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(a, k=1):
    for _ in range(k):
        a = np.repeat(np.repeat(np.repeat(a, 2, axis=1), 2, axis=2), 2, axis=3)
    return a


def up_backward(g, k=1):
    for _ in range(k):
        C, D, H, W = g.shape
        g = g.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))
    return g


def relu(a):
    return np.maximum(a, 0.0)


def node_average(y):
    """y [3][nz][ny][nx] per element -> t [nnode][3] node-interleaved: mean over adjacent elements."""
    C, D, H, W = y.shape
    acc = np.zeros((C, D + 1, H + 1, W + 1))
    cnt = np.zeros((D + 1, H + 1, W + 1))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                acc[:, dz:dz + D, dy:dy + H, dx:dx + W] += y
                cnt[dz:dz + D, dy:dy + H, dx:dx + W] += 1.0
    t = acc / cnt
    return np.ascontiguousarray(t.reshape(C, -1).T), cnt


def node_average_backward(gt, shape, cnt):
    """gt [nnode][3] = dL/dt -> dL/dy [3][nz][ny][nx]."""
    C, D, H, W = shape
    g = (gt.T.reshape(C, D + 1, H + 1, W + 1)) / cnt
    gy = np.zeros(shape)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                gy += g[:, dz:dz + D, dy:dy + H, dx:dx + W]
    return gy


# ------------------------------------------------------------------------------------------------
# the network
# ------------------------------------------------------------------------------------------------
def features(x, f, nel, penal=3.0, E0=1.0, Emin=1e-6):
    """Input features [4][nz][ny][nx] and the scale s of the design (see the module docstring)."""
    nx, ny, nz = nel
    xe = x.reshape(nz, ny, nx)
    fn = f.reshape(nz + 1, ny + 1, nx + 1, 3)
    fe = np.zeros((3, nz, ny, nx))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                fe += np.moveaxis(fn[dz:dz + nz, dy:dy + ny, dx:dx + nx, :], 3, 0)
    fmax = np.abs(fe).max()
    fmax = fmax if fmax > 0 else 1.0
    feat = np.concatenate([(2.0 * xe - 1.0)[None], fe / fmax])
    Ek = Emin + x ** penal * (E0 - Emin)
    return feat, Ek.mean() / fmax


def forward(theta, feat, levels, channels, bf16=True, act_bf16=False):
    """Element output y [3][nz][ny][nx] and the cache for backward.  act_bf16: the input of every
    3x3x3 convolution is rounded to bfloat16 first (the operands of the tensor-core inference path;
    the 1x1x1 heads keep their FP32 inputs)."""
    P = unpack(bf16_round(theta) if bf16 else np.asarray(theta, dtype=np.float64), levels, channels)
    rq = (lambda a: bf16_round(a)) if act_bf16 else (lambda a: a)
    cache = {"in": [], "a": [], "e": [], "dpre": {}, "d": {}}
    h = feat
    for l in range(levels):
        if l > 0:
            h = avgpool(cache["e"][l - 1])
        cache["in"].append(h)
        a = relu(conv3(rq(h), *P[f"enc{l}a"]))
        cache["a"].append(a)
        cache["e"].append(relu(conv3(rq(a), *P[f"enc{l}b"])))
    d = cache["e"][levels - 1]
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([up(d), cache["e"][l]])
        a = relu(conv3(rq(cat), *P[f"dec{l}a"]))
        cache["dpre"][l] = (cat, a)
        d = relu(conv3(rq(a), *P[f"dec{l}b"]))
        cache["d"][l] = d
    d0 = d if levels > 1 else cache["e"][0]
    cache["d0"] = d0
    y = conv1(d0, *P["head"]) + up(conv1(cache["e"][levels - 1], *P["chead"]), levels - 1)
    return y, cache


def gradient(theta, x, f, u, fixed, nel, levels, channels, penal=3.0, bf16=True, out_scale=1.0, loss="energy",
             nu=0.3, E0=1.0, Emin=1e-6):
    """(loss, flat gradient) of one sample: the backward pass level by level (decoder from the top
    level 0 down to the bottleneck, then the encoder from the bottleneck up).  bf16=False uses the
    parameters unrounded (for finite-difference checks)."""
    feat, s = features(x, f, nel, penal)
    y, cache = forward(theta, feat, levels, channels, bf16)
    t, cnt = node_average(y)
    t = out_scale * t.reshape(-1)
    free = fixed == 0
    if loss == "energy":
        from . import assembly
        tf = np.where(free, t, 0.0)
        Kt = np.where(free, assembly.apply_K(nel, 3, x, nu, penal, E0, Emin, tf)[0], 0.0)
        uf = float(np.sum(np.where(free, u * f, 0.0)))
        den = s * s * uf
        value = float((tf @ Kt - 2.0 * s * (tf @ np.where(free, f, 0.0)) + s * s * uf) / den)
        gt = np.where(free, 2.0 * (Kt - s * f) / den, 0.0)
    else:
        tgt = s * u
        den = float(np.sum(tgt[free] ** 2))
        diff = np.where(free, t - tgt, 0.0)
        value = float(np.sum(diff ** 2) / den)
        gt = 2.0 * diff / den
    gy = node_average_backward((out_scale * gt).reshape(-1, 3), y.shape, cnt)
    P = unpack(bf16_round(theta) if bf16 else np.asarray(theta, dtype=np.float64), levels, channels)
    G = {}
    L = levels
    gd, gw, gb = conv1_backward(cache["d0"], P["head"][0], gy)
    G["head"] = (gw, gb)
    ge = [np.zeros_like(e) for e in cache["e"]]
    g_last, gw, gb = conv1_backward(cache["e"][L - 1], P["chead"][0], up_backward(gy, L - 1))
    G["chead"] = (gw, gb)
    ge[L - 1] += g_last
    # decoder: d_l = R(C_b(R(C_a([up(d_{l+1}), e_l])))) for l = 0 .. L-2; gd = dL/dd_l
    for l in range(0, L - 1):
        cat, a = cache["dpre"][l]
        gpost = gd * (cache["d"][l] > 0)
        ga, gw, gb = conv3_backward(a, P[f"dec{l}b"][0], gpost)
        G[f"dec{l}b"] = (gw, gb)
        gcat, gw, gb = conv3_backward(cat, P[f"dec{l}a"][0], ga * (a > 0))
        G[f"dec{l}a"] = (gw, gb)
        cu = channels[l + 1]
        ge[l] += gcat[cu:]
        gd = up_backward(gcat[:cu])  # dL/dd_{l+1}
    if L == 1:
        ge[0] += gd
    else:
        ge[L - 1] += gd  # d_{L-1} = e_{L-1}
    # encoder from the bottleneck up: e_l = R(C_b(R(C_a(in_l)))), in_l = avgpool(e_{l-1})
    for l in range(L - 1, -1, -1):
        gpost = ge[l] * (cache["e"][l] > 0)
        a = cache["a"][l]
        ga, gw, gb = conv3_backward(a, P[f"enc{l}b"][0], gpost)
        G[f"enc{l}b"] = (gw, gb)
        gin, gw, gb = conv3_backward(cache["in"][l], P[f"enc{l}a"][0], ga * (a > 0))
        G[f"enc{l}a"] = (gw, gb)
        if l > 0:
            ge[l - 1] += avgpool_backward(gin)
    flat = np.concatenate([np.concatenate([G[name][0].reshape(-1), G[name][1]])
                           for name, *_ in layer_shapes(levels, channels)])
    return value, flat


def predict(theta, x, f, fixed, nel, levels, channels, penal=3.0, out_scale=1.0, act_bf16=False):
    """u0 [n] (node-interleaved, zero at fixed DOFs)."""
    feat, s = features(x, f, nel, penal)
    y, _ = forward(theta, feat, levels, channels, act_bf16=act_bf16)
    t, _ = node_average(y)
    u0 = out_scale * t.reshape(-1) / s
    u0[fixed == 1] = 0.0
    return u0
