#!/usr/bin/env python3
"""Benchmark of the multilevel buckling hot path: DOF x RHS solved per second to relative
residual 1e-8.

One step = one pass of the whole path over one synthetic design: set densities (SIMP moduli,
Galerkin hierarchy, coarsest inverse), linear analysis K u = f (1 RHS), stress stiffness, coarse
Galerkin eigenproblem + prolongation + fine block solve K Phi = G Psi (q RHS) + Rayleigh quotients,
adjoint right-hand sides + adjoint block solve (q RHS) + sensitivities.  DOF x RHS per step =
n * (1 + q + q) for the multilevel path (n * (1 + q) for the exact fine-grid path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic  # noqa: E402

METRIC = "DOF*RHS solved/s at rel. residual 1e-8"
UNIT = "DOF*RHS/s"
WORKLOAD = "column480x160"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the mixed-precision / 3D form measurements")
    ap.add_argument("--profile-run", action="store_true",
                    help="one untimed step only (for an external profiler's launch list)")
    ap.add_argument("--profile-classes", action="store_true",
                    help="with --profile-run: the library's kernel-class profiler on during the step, i.e. every "
                         "kernel launched directly on the solver's stream, as in the class timing of the bench line")
    ap.add_argument("--eig-gram-tc", type=int, default=0, choices=[0, 1],
                    help="eigensolver Gram products on the tensor cores (FP64-accurate splitting)")
    return ap.parse_args()


def rhs_per_step(p, fused=False):
    """Fine-grid right-hand sides solved per step: the load, the q fine-mode systems of the
    multilevel path (none for the exact path) and the q adjoint systems (+1 when the load is
    re-solved in the same block)."""
    return 1 + (p.num_modes if p.eig_level > 1 else 0) + p.num_modes + (1 if fused else 0)


def measure_form(pkg, torch, name, precision, fused, steps, warmup, dev, flush, outputs=None, **overrides):
    """The same step on another workload / precision, device-timed per step with an L2 flush.  If
    `outputs` is a dict, the last step's u, load factors and sensitivities are stored in it (host)."""
    p = synthetic.config(name)
    stream = torch.cuda.Stream(device=dev)
    s = pkg.Solver(p, stream=stream, precision=precision, fuse_load_adjoint=1 if fused else 0, **overrides)
    x_d = torch.from_numpy(p.x).to(dev)
    q, m = p.num_modes, p.num_elements
    dlam_d = torch.zeros((q, m), dtype=torch.float64, device=dev)
    dJ_d = torch.zeros(m, dtype=torch.float64, device=dev)
    info = {}

    s.phase_timing(True)

    def step():
        s.set_densities(x_d)
        _, i1 = s.solve_equilibrium()
        lam, i2 = s.compute_buckling()
        info["eigen_ms"] = s.phase_read()["eigen"]
        _, _, i3 = s.compute_sensitivities(dlam_d, dJ_d)
        info.update(la_iters=i1["iterations"], buckling_iters=i2["iterations"], adjoint_iters=i3["iterations"],
                    sensitivities_ms=i3["time_ms"])
        info["_lam"] = lam

    for _ in range(warmup):
        step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    # the consistent sensitivities solve the q fine adjoints K w = y besides (their coarse adjoints are
    # on the eigen level and not counted)
    extra = p.num_modes if overrides.get("consistent_sens") else 0
    units = p.num_dofs * (rhs_per_step(p, fused) + extra)
    lam = info.pop("_lam")
    if outputs is not None:
        outputs.update(u=s.get_field(pkg.TOBK_FIELD_U), lam=np.array(lam), dlam=dlam_d.cpu().numpy(),
                       dJ=dJ_d.cpu().numpy())
    s.close()
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "dofs": p.num_dofs,
            "rhs_per_step": rhs_per_step(p, fused) + extra, "precision": "fp64" if precision == 0 else "fp32_vcycle",
            "fused_load_adjoint": bool(fused), "steps": steps, "warmup": warmup,
            **({"consistent_sensitivities": True} if extra else {}),
            **({"smoother": "damped_jacobi", "omega": overrides.get("omega", 0.6)} if overrides.get("smoother") == 0
               else {}), **info}


def output_errors(test, ref):
    """Per-output differences of one form's results from another's (same design): relative 2-norm
    of u, largest relative load-factor difference, and the sensitivities' largest difference scaled
    by their largest magnitude (per mode, worst mode)."""
    du = float(np.linalg.norm(test["u"] - ref["u"]) / np.linalg.norm(ref["u"]))
    dl = float(np.abs(test["lam"] / ref["lam"] - 1).max())
    dd = float(max(np.abs(test["dlam"][i] - ref["dlam"][i]).max() / np.abs(ref["dlam"][i]).max()
                   for i in range(ref["dlam"].shape[0])))
    dj = float(np.abs(test["dJ"] - ref["dJ"]).max() / np.abs(ref["dJ"]).max())
    return {"u_rel_l2": du, "lambda_rel_max": dl, "dlambda_rel_max": dd, "dJ_rel_max": dj}


def measure_batch_sequential_fp64(pkg, torch, steps, warmup, dev, flush, count=64, nadj=6):
    """The batch's designs and right-hand sides solved one design at a time by the plain FP64 mgPCG
    (one handle per design, its 1 + nadj right-hand sides in one multi-RHS solve): the baseline of the
    batched form.  One step = set every design's densities + solve every design."""
    problems = synthetic.batch_configs(count)
    stream = torch.cuda.Stream(device=dev)
    B = batch_rhs(pkg, torch, problems, nadj, dev, stream)
    nr = 1 + nadj
    solvers, views, xs = [], [], []
    off = 0
    for p in problems:
        s = pkg.Solver(p, stream=stream, max_rhs=nr)
        solvers.append(s)
        views.append((B[off: off + nr * p.num_dofs], torch.zeros(nr * p.num_dofs, dtype=torch.float64, device=dev)))
        xs.append(torch.from_numpy(p.x).to(dev))
        off += nr * p.num_dofs
    its = []

    def step():
        its.clear()
        for s, (b, xo), x in zip(solvers, views, xs):
            s.set_densities(x)
            xo.zero_()
            its.append(s.solve(1, b, xo, nr)["iterations"])

    for _ in range(warmup):
        step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    dofs = int(sum(p.num_dofs for p in problems))
    for s in solvers:
        s.close()
    return {"value": dofs * nr / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "designs": count, "dofs_total": dofs,
            "rhs_per_design": nr, "precision": "fp64", "iterations_max": max(its), "steps": steps, "warmup": warmup}


def batch_rhs(pkg, torch, problems, nadj, dev, stream):
    """Right-hand sides of the batch: per design the load and nadj adjoint right-hand sides of a
    preceding buckling analysis of the same design (multilevel, eigenproblem on the second-coarsest
    level), packed [design][1 + nadj][n_d] on the device."""
    blocks = []
    for p in problems:
        q = synthetic.column_2d(p.nel[1], p.nel[0], seed=p.meta["seed"], radius=p.meta["radius"],
                                volfrac=p.meta["volfrac"], mg_levels=p.mg_levels,
                                eig_level=max(2, p.mg_levels - 1), num_modes=nadj, x=p.x)
        s = pkg.Solver(q, stream=stream, precision=pkg.TOBK_FP32_VCYCLE)
        s.solve_equilibrium()
        s.compute_buckling()
        s.compute_sensitivities()
        B = np.zeros((1 + nadj, p.num_dofs))
        B[0] = p.f
        B[1:] = s.get_field(pkg.TOBK_FIELD_ADJOINT_RHS).reshape(nadj, p.num_dofs)
        blocks.append(B.reshape(-1))
        s.close()
    return torch.from_numpy(np.concatenate(blocks)).to(dev)


def measure_batch(pkg, torch, steps, warmup, dev, flush, count=64, nadj=6):
    """Batched form: `count` uneven 2D designs, each with the load and `nadj` adjoint RHS, solved
    together (grouped launches, captured graphs, autotuned tiles, FP32 V-cycle, FP64 outer CG).
    One step = set every design's densities (hierarchy set-up) + the batched solve."""
    problems = synthetic.batch_configs(count)
    stream = torch.cuda.Stream(device=dev)
    B = batch_rhs(pkg, torch, problems, nadj, dev, stream)
    bt = pkg.Batch(problems, 1 + nadj, stream=stream)
    x = torch.from_numpy(np.concatenate([p.x for p in problems])).to(dev)
    fixed = torch.from_numpy(np.concatenate([p.fixed for p in problems]).astype(np.uint8)).to(dev)
    X = torch.zeros_like(B)
    bt.set_designs(x, fixed)
    variants = bt.autotune()
    infos = None
    for _ in range(warmup):
        bt.set_designs(x, fixed)
        infos, _ = bt.solve(B, X)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs[k][0].record(stream)
        bt.set_designs(x, fixed)
        infos, _ = bt.solve(B, X)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    dofs = int(sum(p.num_dofs for p in problems))
    units = dofs * (1 + nadj)
    bt.close()
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "designs": count, "dofs_total": dofs,
            "rhs_per_design": 1 + nadj, "precision": "fp32_vcycle", "autotuned_variants": list(variants),
            "iterations_max": max(i["iterations"] for i in infos),
            "rel_residual_max": max(i["rel_residual"] for i in infos), "steps": steps, "warmup": warmup}


def measure_learned(pkg, torch, dev, flush, designs=4):
    """Learned warm start on held-out 128 x 64 x 64 designs: network inference + mgPCG from its guess
    against plain mgPCG from zero, both to relative residual 1e-8 (one RHS per design)."""
    from paper_1909_13585_gb300 import learned
    if not os.path.exists(learned.WEIGHTS):
        return {"unavailable": "no trained weights in the package"}
    X = learned.densities(range(learned.TEST_SEEDS[0], learned.TEST_SEEDS[0] + designs), workers=1)
    net = learned.load_weights(pkg, torch, learned.WEIGHTS, stream=torch.cuda.Stream(device=dev))
    learned.evaluate(pkg, torch, net, X[:1], flush=flush)  # warm-up (graph capture, allocations)
    rows = learned.evaluate(pkg, torch, net, X, flush=flush)
    net.close()
    sm = learned.summary(rows)
    dofs = learned.problem(X[0]).num_dofs
    return {"value": dofs / (sm["ms_learned_mean"] / 1e3), "value_plain": dofs / (sm["ms_plain_mean"] / 1e3),
            "unit": UNIT, "dofs": dofs, "rhs_per_step": 1, "held_out_designs": designs, **sm}


# ------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): runs in a child process, single-threaded BLAS
# ------------------------------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import synthetic
from oracle import lba, sensitivity
p = synthetic.config({workload!r})
times = []
for k in range({reps}):
    t0 = time.perf_counter()
    op = lba.Problem(p)
    u, J = lba.linear_analysis(op)
    if p.eig_level > 1:
        ml = lba.multilevel_lba(op, u, p.num_modes, p.eig_level)
        lam, Phi = ml["lam"], ml["Phi"]
    else:
        lam, Phi, _ = lba.exact_lba(op, u, p.num_modes)
    dlam, dJ, Z = sensitivity.sensitivities(op, u, lam, Phi)
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times}}))
"""


def run_oracle(workload, reps):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, workload=workload, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])["times"]


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p = synthetic.config(args.workload)
    units = p.num_dofs * rhs_per_step(p)
    times = run_oracle(args.workload, args.warmup + args.steps)[args.warmup:]
    total = sum(times)
    value = units * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(p, "fp64"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"full step of {args.workload} per timed step (SciPy SuperLU + ARPACK, "
                                   "single-threaded BLAS)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict(p, precision):
    return {"workload": p.name, "dim": p.dim, "nel": list(p.nel[:p.dim]), "dofs": p.num_dofs,
            "mg_levels": p.mg_levels, "eig_level": p.eig_level, "modes": p.num_modes,
            "rhs_per_step": rhs_per_step(p), "precision": precision,
            "l2": "flushed between timed steps (512 MiB write)", "seed": p.meta.get("seed")}


# ------------------------------------------------------------------------------------------------
# roofline of the dominant kernel class
# ------------------------------------------------------------------------------------------------
def sources_hash(paths):
    h = hashlib.sha1()
    for f in paths:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(kclass, workload):
    """DRAM bytes per launch of the kernel class from the committed ncu summary
    profiles/<class>_<workload>.md, if the sources it lists are unchanged since the capture (their
    hash matches), else None."""
    path = os.path.join(ROOT, "profiles", f"{kclass}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    sm = re.search(r"sources:\s*(.+)", txt)
    hm = re.search(r"sources_hash:\s*([0-9a-f]+)", txt)
    if not (m and sm and hm):
        return None
    paths = sm.group(1).split()
    if not all(os.path.exists(os.path.join(ROOT, f)) for f in paths) or sources_hash(paths) != hm.group(1):
        return None
    return float(m.group(1))


# Algorithmic FP64 operations (add, multiply or fused multiply-add: one FP64-pipe issue each) per
# node and right-hand side of the fine-level factored Q4 kernels: 41 per element for the forces
# (one element per node), 6 to gather the four element contributions of a node's two DOFs, plus the
# per-DOF update: Chebyshev/Jacobi step 5 x 2, residual 1 x 2, CG direction (z + beta p, p.q) 2 x 2.
Q4_FP64_OPS_PER_NODE = {"fine_smooth": 41 + 6 + 10, "fine_residual": 41 + 6 + 2, "fine_cg_matvec": 41 + 6 + 4}
# FP64 pipe: 152 SMs x 2 FP64 instructions per clock x 2070 MHz (the maximum SM clock); a register-only
# FMA probe on this part measured 1.194 TFLOP/s at 1995 MHz, i.e. the same 2 FMA per clock per SM.
FP64_OPS_PEAK_G = 152 * 2 * 2.070


# kernel classes of the library's profiler that are one kernel each (the fine-level operator in its
# three modes); the others (coarse levels, transfers, vector and eigensolver kernels) aggregate
# several different kernels and are reported by class only
SINGLE_KERNEL_CLASSES = ("fine_smooth", "fine_residual", "fine_cg_matvec")


def roofline(prof, p, peaks, precision):
    """Roofline of the dominant kernel (the single-kernel class with the most device time):
    achieved = algorithmic work per launch (from the DOF x RHS the class processed) / average launch
    time (CUDA events on the solver's stream)."""
    name, rec = max(((k, v) for k, v in prof.items() if k in SINGLE_KERNEL_CLASSES), key=lambda kv: kv[1]["ms"])
    m, n, nnode = p.num_elements, p.num_dofs, p.num_nodes
    launches = max(rec["launches"], 1)
    per_launch_s = 1e-3 * rec["ms"] / launches
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    out = {"kernel_class": name, "launches": rec["launches"], "avg_launch_us": 1e6 * per_launch_s,
           "share_of_class_time": rec["ms"] / sum(v["ms"] for v in prof.values()),
           "largest_class": {"name": top[0], "ms": top[1]["ms"], "launches": top[1]["launches"]}}
    hbm = peaks.get("hbm_gbs", 6792.7)
    if name in Q4_FP64_OPS_PER_NODE and p.dim == 2 and precision == "fp64":
        rhs_per_launch = rec["dof_rhs"] / n / launches
        ops = rhs_per_launch * nnode * Q4_FP64_OPS_PER_NODE[name]
        # bytes: per RHS read v, b (and d_in), write y (and d_out); per node dinv, fixed; per element E
        vec_words = {"fine_smooth": 5, "fine_residual": 3, "fine_cg_matvec": 5}[name]
        bytes_ = rhs_per_launch * 8.0 * vec_words * n + 8.0 * n + n + 8.0 * m
        achieved = ops / per_launch_s / 1e9
        out.update({"bound": "alu", "achieved": achieved, "peak": FP64_OPS_PEAK_G, "unit": "G FP64 ops/s",
                    "frac": achieved / FP64_OPS_PEAK_G,
                    "peak_source": "derived: 152 SMs x 2 FP64 pipe issues/clk x 2070 MHz (measured FMA probe agrees)",
                    "algorithmic_fp64_ops_per_launch": ops, "algorithmic_bytes_per_launch": bytes_,
                    "hbm_gbs_at_same_time": bytes_ / per_launch_s / 1e9,
                    "hbm_frac_of_measured": bytes_ / per_launch_s / 1e9 / hbm})
    else:
        word = 8 if precision == "fp64" else 4
        bytes_ = 4.0 * word * rec["dof_rhs"] / launches  # read v, b, dinv-scaled update, write y per DOF x RHS
        achieved = bytes_ / per_launch_s / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "peak_source": "of measured", "algorithmic_bytes_per_launch": bytes_})
    out["traffic"] = profiled_traffic(name, p.name)
    return out


# ------------------------------------------------------------------------------------------------
# multi-rank aggregation (one process per GPU; each rank solves its own replica of the workload)
# ------------------------------------------------------------------------------------------------
def max_over_ranks(value, world, device):
    """The largest value over the ranks (the job's time is its slowest rank's time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step, steps, world, max_ms):
    """Whole-job units per second: every rank processes units_per_step in each of `steps` steps
    (weak scaling), and the job takes its slowest rank's max_ms."""
    return world * units_per_step * steps / (max_ms / 1e3)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def ours(args):
    import torch
    import paper_1909_13585_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}

    p = synthetic.config(args.workload)
    precision = pkg.TOBK_FP64 if args.precision == "fp64" else pkg.TOBK_FP32_VCYCLE
    stream = torch.cuda.Stream(device=dev)
    s = pkg.Solver(p, stream=stream, precision=precision, eig_gram_tc=args.eig_gram_tc)
    q, m, n = p.num_modes, p.num_elements, p.num_dofs
    units = n * rhs_per_step(p)

    x_d = torch.from_numpy(p.x).to(dev)
    dlam_d = torch.zeros((q, m), dtype=torch.float64, device=dev)
    dJ_d = torch.zeros(m, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step():
        s.set_densities(x_d)
        s.solve_equilibrium()
        s.compute_buckling()
        s.compute_sensitivities(dlam_d, dJ_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile_run:
        if args.profile_classes:
            s.profile(True)
        step()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_run": p.name, "gpu_launches_total": pkg.launch_count()}))
        s.close()
        return 0

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    launches0 = pkg.launch_count()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = pkg.launch_count() - launches0
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = job_throughput(units, args.steps, world, total_ms)

    # per-phase device times over K more steps (CUDA events per phase and per eigensolver iteration,
    # no per-launch events), then the kernel-class profile over K more steps (events around every
    # launch of a class, which serialises the host side: its times feed the roofline only)
    phases = {}
    s.phase_timing(True)
    for _ in range(args.steps):
        s.set_densities(x_d)
        _, i1 = s.solve_equilibrium()
        _, i2 = s.compute_buckling()
        _, _, i3 = s.compute_sensitivities(dlam_d, dJ_d)
        for k, inf in (("linear_analysis", i1), ("buckling", i2), ("sensitivities", i3)):
            phases.setdefault(k, []).append(inf["time_ms"])
            phases.setdefault(k + "_iters", []).append(inf["iterations"])
        for k, v in s.phase_read().items():
            phases.setdefault("buckling." + k, []).append(v)
    s.phase_timing(False)
    s.profile(True)
    for _ in range(args.steps):
        step()
    prof = s.profile_read()
    s.profile(False)
    roof = roofline(prof, p, peaks, args.precision)

    # end-to-end through the public API with pinned host buffers (H2D inputs, D2H outputs)
    e2e = None
    if not args.no_e2e:
        x_h = torch.from_numpy(p.x.copy()).pin_memory()
        f_h = torch.from_numpy(p.f.copy()).pin_memory()
        fx_h = torch.from_numpy(p.fixed.astype(np.uint8)).pin_memory()
        dlam_h = torch.zeros((q, m), dtype=torch.float64).pin_memory()
        dJ_h = torch.zeros(m, dtype=torch.float64).pin_memory()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        lam_sum = 0.0
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            s.set_fixed(fx_h)
            s.set_load(f_h)
            s.set_densities(x_h)
            J, _ = s.solve_equilibrium()
            lam, _ = s.compute_buckling()
            s.compute_sensitivities(dlam_h, dJ_h)
            ev[k][1].record(stream)
            lam_sum += float(lam[0]) + J
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
        e2e = {"value": job_throughput(units, args.steps, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": 8 * m + 8 * n + n, "d2h_bytes_per_step": 8 * q + 8 * q * m + 8 * m + 8}

    forms = {}
    if not args.no_forms:
        fs, fw = args.steps, max(3, args.warmup)
        forms["column480x160_fp32_vcycle"] = measure_form(pkg, torch, "column480x160", pkg.TOBK_FP32_VCYCLE, False,
                                                          fs, fw, dev, flush)
        forms["column480x160_fp64_damped_jacobi"] = measure_form(pkg, torch, "column480x160", pkg.TOBK_FP64, False,
                                                                 fs, fw, dev, flush, smoother=0, omega=0.6)
        forms["column480x160_fp64_tensor_core_gram"] = measure_form(pkg, torch, "column480x160", pkg.TOBK_FP64, False,
                                                                    fs, fw, dev, flush, eig_gram_tc=1)
        ocons, oplain = {}, {}
        forms["column480x160_fp64_consistent_sensitivities"] = measure_form(
            pkg, torch, "column480x160", pkg.TOBK_FP64, False, fs, fw, dev, flush, outputs=ocons, consistent_sens=1)
        measure_form(pkg, torch, "column480x160", pkg.TOBK_FP64, False, 1, 1, dev, flush, outputs=oplain)
        forms["column480x160_fp64_consistent_sensitivities"]["difference_from_eq_SensitivityLambda"] = \
            output_errors(ocons, oplain)
        del ocons, oplain
        forms["column60x20_fp64_exact_lba"] = measure_form(pkg, torch, "column60x20", pkg.TOBK_FP64, False,
                                                           fs, fw, dev, flush)
        o64, o32 = {}, {}
        forms["cantilever96x48x48_fp64"] = measure_form(pkg, torch, "cantilever96x48x48", pkg.TOBK_FP64, False,
                                                        fs, fw, dev, flush, outputs=o64)
        forms["cantilever96x48x48_fp32_vcycle_fused"] = measure_form(pkg, torch, "cantilever96x48x48",
                                                                     pkg.TOBK_FP32_VCYCLE, True, fs, fw, dev, flush,
                                                                     outputs=o32)
        forms["cantilever96x48x48_fp32_vcycle_fused"]["error_vs_fp64_path"] = output_errors(o32, o64)
        del o64, o32
        forms["batch64_column2d_fp32_vcycle"] = measure_batch(pkg, torch, fs, fw, dev, flush)
        forms["batch64_column2d_fp64_one_at_a_time"] = measure_batch_sequential_fp64(pkg, torch, fs, fw, dev, flush)
        forms["cantilever128x64x64_learned_warm_start"] = measure_learned(pkg, torch, dev, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times = run_oracle(args.workload, 1)
        cpu = {"value": units / times[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full step of {args.workload} ({times[0]:.1f} s: assembly, SuperLU LA, "
                         "multilevel LBA with ARPACK, adjoint sensitivities), single-threaded BLAS"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic", "config": config_dict(p, args.precision),
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "wall_s_timed_region": t_wall,
            "phases_ms": {k: statistics.median(v) for k, v in phases.items()},
            "kernel_classes": prof,
            "forms": forms,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    s.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
