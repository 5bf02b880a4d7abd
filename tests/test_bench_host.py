"""Host logic of bench.py (no GPU): the work counted per step, the roofline of the dominant kernel
from a kernel-class profile, and the committed DRAM-traffic figure's source check."""
import os
import shutil

import pytest

import bench
import synthetic


def test_rhs_per_step_counts_load_fine_modes_and_adjoints():
    p = synthetic.config("column480x160")            # multilevel: load + 12 fine-mode + 12 adjoint
    assert bench.rhs_per_step(p) == 25
    assert bench.rhs_per_step(p, fused=True) == 26   # the load re-solved with the adjoints
    e = synthetic.config("column60x20")              # exact path: no fine-mode solve
    assert bench.rhs_per_step(e) == 1 + e.num_modes


def _profile():
    # per-class device time (ms), launches and DOF x RHS processed over a profiled run
    return {"fine_smooth": {"launches": 2880, "ms": 232.3, "dof_rhs": 3726460920.0},
            "fine_residual": {"launches": 960, "ms": 68.6, "dof_rhs": 1242153640.0},
            "coarse": {"launches": 16740, "ms": 244.3, "dof_rhs": 2083931680.0},
            "vector": {"launches": 4620, "ms": 79.5, "dof_rhs": 4372461040.0}}


def test_roofline_takes_the_dominant_single_kernel_and_counts_algorithmic_work():
    p = synthetic.config("column480x160")
    prof = _profile()
    r = bench.roofline(prof, p, {"hbm_gbs": 6792.7}, "fp64")
    # the coarse class took longer but aggregates several kernels: the fine smoother is reported
    assert r["kernel_class"] == "fine_smooth" and r["largest_class"]["name"] == "coarse"
    launches, ms = prof["fine_smooth"]["launches"], prof["fine_smooth"]["ms"]
    rhs_per_launch = prof["fine_smooth"]["dof_rhs"] / p.num_dofs / launches
    ops = rhs_per_launch * p.num_nodes * bench.Q4_FP64_OPS_PER_NODE["fine_smooth"]
    assert r["algorithmic_fp64_ops_per_launch"] == pytest.approx(ops)
    assert r["achieved"] == pytest.approx(ops / (1e-3 * ms / launches) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_OPS_PEAK_G)
    assert r["bound"] == "alu" and 0.0 < r["frac"] < 1.0
    assert r["share_of_class_time"] == pytest.approx(ms / sum(v["ms"] for v in prof.values()))


def test_profiled_traffic_requires_unchanged_sources(tmp_path, monkeypatch):
    """The committed figure is used only while the kernel sources it lists hash to the recorded
    value; a changed source file makes it unavailable (null in the bench line)."""
    got = bench.profiled_traffic("fine_smooth", "column480x160")
    assert got is not None and got > 0
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), root / "profiles")
    for rel in ("paper_1909_13585_gb300/csrc",):
        shutil.copytree(os.path.join(bench.ROOT, rel), root / rel)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic("fine_smooth", "column480x160") == got
    with open(root / "paper_1909_13585_gb300/csrc/fine2d.cu", "a") as f:
        f.write("// changed\n")
    assert bench.profiled_traffic("fine_smooth", "column480x160") is None
    assert bench.profiled_traffic("no_such_class", "column480x160") is None
