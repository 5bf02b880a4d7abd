"""Learned warm start for the 3D H8 cantilever: training data generated by the method itself
(mgPCG solutions of seeded random designs), training of the U-Net with the library's own forward,
backward and Adam kernels (tobk_unet_*), and its evaluation against plain mgPCG from a zero start
(iterations and time to the same relative residual).  Argument marshalling and loops only: every
step of the solver and of the network runs in libtobk.so.

    python -m paper_1909_13585_gb300.learned train --out weights.npz [--designs 2000] [--epochs 4]
    python -m paper_1909_13585_gb300.learned evaluate --weights weights.npz [--designs 50]
"""
from __future__ import annotations

import argparse
import math
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

NEL = (128, 64, 64)            # H8 elements (x, y, z) of the learned-warm-start workload
MG_LEVELS = 5
LEVELS, CHANNELS = 4, (16, 32, 64, 64)
TRAIN_SEEDS = (10000, 12000)   # [first, last) design seeds of the training set
TEST_SEEDS = (20000, 20050)    # held-out designs
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_cantilever128x64x64.npz")


def design_recipe(seed):
    """Filter radius in [2, 4] and volume fraction in [0.2, 0.5] of design `seed`."""
    rng = np.random.default_rng(seed + 7919)
    return float(rng.uniform(2.0, 4.0)), float(rng.uniform(0.2, 0.5))


def _density(args):
    seed, nel = args
    r, vf = design_recipe(seed)
    return synthetic.density_field((nel[2], nel[1], nel[0]), seed, r, vf).astype(np.float32)


def densities(seeds, nel=NEL, workers=None):
    """Densities [N][m] (float32) of the designs, generated on the host cores (spawned workers, so
    that the pool never forks a process that holds a CUDA context)."""
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    jobs = [(s, tuple(nel)) for s in seeds]
    if workers == 1 or len(jobs) < 4:
        return np.stack([_density(j) for j in jobs])
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.stack(pool.map(_density, jobs, chunksize=max(1, len(jobs) // (4 * workers))))


def problem(x, nel=NEL):
    return synthetic.cantilever_3d(*nel, seed=0, radius=2.0, volfrac=0.3, mg_levels=MG_LEVELS, eig_level=1,
                                   num_modes=1, x=np.asarray(x, dtype=np.float64))


def generate(pkg, torch, X, nel=NEL, rtol=1e-8, stream=None):
    """Solutions U [N][n] (float32, device) of K(x_i) u = f by the library's mgPCG (FP32 V-cycle)."""
    p0 = problem(X[0], nel)
    s = pkg.Solver(p0, stream=stream, precision=pkg.TOBK_FP32_VCYCLE, rtol=rtol, max_rhs=1)
    dev = torch.device("cuda")
    f = torch.from_numpy(p0.f).to(dev)
    U = torch.zeros((len(X), p0.num_dofs), dtype=torch.float32, device=dev)
    u = torch.zeros(p0.num_dofs, dtype=torch.float64, device=dev)
    iters = []
    for i in range(len(X)):
        s.set_densities(torch.from_numpy(X[i].astype(np.float64)).to(dev))
        info = s.solve(1, f, u, 1)
        iters.append(info["iterations"])
        U[i].copy_(u)
    s.close()
    return U, iters


def output_scale(net, Xd, U, fixed, f, samples=16):
    """RMS of the scaled targets s_i u_i over the free DOFs of the first samples: the network's
    outputs are then of order one."""
    free = fixed == 0
    acc = 0.0
    k = min(samples, Xd.shape[0])
    for i in range(k):
        s = net.design_scale(Xd[i], f)
        acc += float(((s * U[i][free].double()) ** 2).mean())
    return (acc / k) ** 0.5


def train(net, torch, Xd, U, f, fixed, epochs=4, batch=4, lr=2e-3, seed=0, log=None):
    """Adam on mini-batches of `batch` designs; learning rate lr, halved after every epoch."""
    N = Xd.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(N)
        tot, cnt = 0.0, 0
        for k in range(0, N - batch + 1, batch):
            idx = torch.from_numpy(order[k:k + batch]).to(Xd.device)
            xb = Xd.index_select(0, idx).contiguous()
            ub = U.index_select(0, idx).contiguous()
            tot += net.train_step(xb, f, ub, fixed, batch, lr)
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.4e} (lr {lr:.2e})")
        lr *= 0.5
    return hist


def _params_only(net, torch):
    P = torch.zeros(net.num_params, dtype=torch.float32)
    net.get_state(P)
    return P


def save_weights(net, torch, path):
    P, M, V = (torch.zeros(net.num_params, dtype=torch.float32) for _ in range(3))
    step = net.get_state(P, M, V)
    np.savez(path, params=P.numpy(), adam_m=M.numpy(), adam_v=V.numpy(), step=step,
             levels=net.levels, channels=np.array(net.channels), nel=np.array(net.nel),
             out_scale=net.output_scale())


WEIGHT_KEYS = ("nel", "levels", "channels", "params", "adam_m", "adam_v", "step", "out_scale")


def read_weights(path):
    """Reads a weights file written by save_weights and checks it on the host: a readable .npz
    archive with every key, FP32 parameter and Adam-moment vectors of one common length, finite
    values, a positive output scale.  Raises ValueError naming what is wrong."""
    try:
        with np.load(path) as z:
            data = {k: z[k] for k in z.files}
    except Exception as e:  # truncated or foreign files fail inside numpy / zipfile
        raise ValueError(f"weights file {path!r} is not a readable .npz archive ({type(e).__name__}: {e})") from None
    missing = [k for k in WEIGHT_KEYS if k not in data]
    if missing:
        raise ValueError(f"weights file {path!r} lacks {', '.join(missing)}")
    params = data["params"]
    if params.dtype != np.float32 or params.ndim != 1:
        raise ValueError(f"weights file {path!r}: params must be a 1-D float32 vector, got {params.dtype} {params.shape}")
    for k in ("adam_m", "adam_v"):
        if data[k].dtype != np.float32 or data[k].shape != params.shape:
            raise ValueError(f"weights file {path!r}: {k} does not match params ({data[k].dtype} {data[k].shape})")
    if not (np.all(np.isfinite(params)) and np.isfinite(float(data["out_scale"])) and float(data["out_scale"]) > 0):
        raise ValueError(f"weights file {path!r} holds non-finite parameters or a bad output scale")
    return data


def load_weights(pkg, torch, path, stream=None):
    """A network restored from a weights file; ValueError if the file is damaged or was written for
    another architecture (its parameter count differs from the network it describes)."""
    z = read_weights(path)
    net = pkg.UNet(tuple(int(v) for v in z["nel"]), int(z["levels"]), tuple(int(v) for v in z["channels"]),
                   stream=stream)
    if net.num_params != z["params"].size:
        n = net.num_params
        net.close()
        raise ValueError(f"weights file {path!r} holds {z['params'].size} parameters, the network it describes "
                         f"needs {n}")
    net.set_state(torch.from_numpy(z["params"]), torch.from_numpy(z["adam_m"]), torch.from_numpy(z["adam_v"]),
                  int(z["step"]))
    net.set_output_scale(float(z["out_scale"]))
    return net


def evaluate(pkg, torch, net, X, nel=NEL, rtol=1e-8, flush=None, precision=None):
    """Per held-out design: mgPCG iterations and device time from zero and from the network's guess
    (network inference included), the true relative residual of both and the relative energy-norm
    error of the guess.  Both arms go through tobk_solve_equilibrium; the plain arm is the fallback.
    `flush`: a device tensor larger than L2, zeroed before each timed arm; `precision`: the solver's
    V-cycle precision (default: the FP32 V-cycle)."""
    dev = torch.device("cuda")
    p0 = problem(X[0], nel)
    stream = net.stream  # the solver shares the network's stream, so that the guess is ordered before the solve
    prec = pkg.TOBK_FP32_VCYCLE if precision is None else precision
    s = pkg.Solver(p0, stream=stream, precision=prec, rtol=rtol, max_rhs=1)
    f = torch.from_numpy(p0.f).to(dev)
    fixed = torch.from_numpy(p0.fixed.astype(np.uint8)).to(dev)
    u0 = torch.zeros(p0.num_dofs, dtype=torch.float64, device=dev)
    out = []
    for i in range(len(X)):
        xd = torch.from_numpy(X[i].astype(np.float64)).to(dev)
        row = {}
        for arm in ("plain", "learned"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.set_densities(xd)
            if flush is not None:  # cold L2 for both arms
                flush.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            if arm == "learned":
                net.predict(xd, f, fixed, u0)
                s.set_initial_guess(u0)
            else:
                s.set_initial_guess(None)
            _, info = s.solve_equilibrium()
            e1.record(stream)
            torch.cuda.synchronize()
            row[arm] = {"iterations": info["iterations"], "ms": e0.elapsed_time(e1),
                        "rel_residual": info["rel_residual"], "converged": info["converged"]}
        # relative energy-norm error of the guess the solve started from (the network's output scaled
        # by alpha = u0^T f / u0^T K u0, as tobk_set_initial_guess does), against the converged solution
        u = torch.zeros(p0.num_dofs, dtype=torch.float64, device=dev)
        s.get_field(pkg.TOBK_FIELD_U, u)
        Ku = torch.zeros_like(u)
        Ku0 = torch.zeros_like(u)
        s.apply_K(1, u, Ku)
        s.apply_K(1, u0, Ku0)
        torch.cuda.synchronize()
        u0m = torch.where(fixed.bool(), torch.zeros_like(u0), u0)
        Ku0 = torch.where(fixed.bool(), torch.zeros_like(Ku0), Ku0)
        den = float(u0m @ Ku0)
        alpha = float(u0m @ f) / den if den > 0.0 else 0.0
        e_energy = float(u @ Ku) - 2.0 * alpha * float(u0m @ Ku) + alpha * alpha * den
        row["guess_energy_error"] = math.sqrt(max(e_energy, 0.0) / float(u @ Ku))
        row["rtol"] = rtol
        out.append(row)
    s.set_initial_guess(None)
    s.close()
    return out


def summary(rows):
    it_p = np.array([r["plain"]["iterations"] for r in rows], dtype=float)
    it_l = np.array([r["learned"]["iterations"] for r in rows], dtype=float)
    ms_p = np.array([r["plain"]["ms"] for r in rows])
    ms_l = np.array([r["learned"]["ms"] for r in rows])
    return {"designs": len(rows), "iterations_plain_mean": float(it_p.mean()),
            "iterations_learned_mean": float(it_l.mean()), "ms_plain_mean": float(ms_p.mean()),
            "ms_learned_mean": float(ms_l.mean()),
            "fallback_rate": float(np.mean([r["learned"]["iterations"] >= r["plain"]["iterations"] for r in rows])),
            "rel_residual_max": float(max(max(r["plain"]["rel_residual"], r["learned"]["rel_residual"]) for r in rows)),
            # what the guess can buy: mgPCG reduces the error by the same factor per iteration from any
            # start, rho = rtol^(1 / plain iterations), so a start with relative energy error e saves
            # about log(e) / log(rho) iterations
            "guess_energy_error_mean": float(np.mean([r["guess_energy_error"] for r in rows])),
            "iterations_saved_expected": float(np.mean([
                math.log(max(r["guess_energy_error"], 1e-300)) / math.log(r["rtol"] ** (1.0 / r["plain"]["iterations"]))
                for r in rows]))}


def main():
    import torch
    import paper_1909_13585_gb300 as pkg

    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--designs", type=int, default=None)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--init", default=None, help="weights file to start the training from")
    ap.add_argument("--data-rtol", type=float, default=1e-6,
                    help="relative residual of the training solutions (targets need not be exact)")
    args = ap.parse_args()
    log = lambda m: print(f"[{time.strftime('%H:%M:%S')}] {m}", flush=True)  # noqa: E731
    if args.cmd == "train":
        n = args.designs or (TRAIN_SEEDS[1] - TRAIN_SEEDS[0])
        t0 = time.time()
        X = densities(range(TRAIN_SEEDS[0], TRAIN_SEEDS[0] + n))
        log(f"{n} training designs generated on the host in {time.time() - t0:.1f} s")
        pkg.load()
        t0 = time.time()
        stream = torch.cuda.Stream()
        U, iters = generate(pkg, torch, X, rtol=args.data_rtol, stream=stream)
        torch.cuda.synchronize()
        log(f"{n} mgPCG solutions in {time.time() - t0:.1f} s (iterations mean {np.mean(iters):.1f})")
        p0 = problem(X[0])
        dev = torch.device("cuda")
        f = torch.from_numpy(p0.f).to(dev)
        fixed = torch.from_numpy(p0.fixed.astype(np.uint8)).to(dev)
        Xd = torch.from_numpy(X).to(dev)
        if args.init:
            net = load_weights(pkg, torch, args.init, stream=stream)
            net.set_state(_params_only(net, torch), None, None, 0)  # keep the weights, restart Adam
        else:
            net = pkg.UNet(NEL, LEVELS, CHANNELS, stream=stream)
            net.set_output_scale(output_scale(net, Xd, U, fixed, f))
        log(f"output scale {net.output_scale():.4e}")
        t0 = time.time()
        hist = train(net, torch, Xd, U, f, fixed, args.epochs, args.batch, args.lr, log=log)
        torch.cuda.synchronize()
        log(f"training: {args.epochs} epochs in {time.time() - t0:.1f} s, losses {hist}")
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        save_weights(net, torch, args.out)
        Xt = densities(range(TEST_SEEDS[0], TEST_SEEDS[1]))
        rows = evaluate(pkg, torch, net, Xt)
        print(json.dumps({"train_loss": hist, "eval": summary(rows), "rows": rows}))
    else:
        n = args.designs or (TEST_SEEDS[1] - TEST_SEEDS[0])
        X = densities(range(TEST_SEEDS[0], TEST_SEEDS[0] + n))
        net = load_weights(pkg, torch, args.weights, stream=torch.cuda.Stream())
        rows = evaluate(pkg, torch, net, X)
        print(json.dumps({"eval": summary(rows), "rows": rows}))


if __name__ == "__main__":
    main()
