"""The trained warm start on held-out designs of the 128 x 64 x 64 cantilever workload: plain mgPCG
from the network's guess reaches the same relative residual as from zero (the network can change
the iteration count, never the accepted accuracy); the guess the solve starts from (the network's
output scaled to minimise its energy-norm error, u0^T f / u0^T K u0) is closer to the solution than the
zero guess in the energy norm; what it gains or loses in iterations is reported (bench.py reports the
same on more designs)."""
import numpy as np
import pytest

from oracle import assembly
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_trained_warm_start_keeps_the_tolerance_and_reports_its_gain():
    torch, pkg = require_gpu()
    from paper_1909_13585_gb300 import learned
    X = learned.densities(range(learned.TEST_SEEDS[0], learned.TEST_SEEDS[0] + 2), workers=1)
    stream = torch.cuda.Stream()
    net = learned.load_weights(pkg, torch, learned.WEIGHTS, stream=stream)
    rows = learned.evaluate(pkg, torch, net, X)
    for r in rows:
        assert r["plain"]["converged"] == 1 and r["learned"]["converged"] == 1
        assert r["plain"]["rel_residual"] <= 1e-8 and r["learned"]["rel_residual"] <= 1e-8
        assert abs(r["learned"]["iterations"] - r["plain"]["iterations"]) <= 8
    # energy-norm error of the guess against the solution, with the oracle's operator
    p = learned.problem(X[0])
    s = pkg.Solver(p, stream=stream, precision=pkg.TOBK_FP32_VCYCLE, max_rhs=1)
    s.solve_equilibrium()
    u = s.get_field(pkg.TOBK_FIELD_U)
    dev = torch.device("cuda")
    u0 = torch.zeros(p.num_dofs, dtype=torch.float64, device=dev)
    net.predict(torch.from_numpy(p.x).to(dev), torch.from_numpy(p.f).to(dev),
                torch.from_numpy(p.fixed.astype(np.uint8)).to(dev), u0)
    torch.cuda.synchronize()
    g = u0.cpu().numpy()
    free = p.fixed == 0
    Ku = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, u)[0]
    Kg = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, g)[0]
    uKu = u[free] @ Ku[free]

    def energy_error(v, Kv):
        return float((v[free] @ Kv[free] - 2 * v[free] @ Ku[free] + uKu) / uKu)

    raw = energy_error(g, Kg)
    alpha = (g[free] @ p.f[free]) / (g[free] @ Kg[free])        # the solve's scaling of the guess
    scaled = energy_error(alpha * g, alpha * Kg)
    print(f"relative energy error of the guess {raw:.3f}, scaled by {alpha:.3f}: {scaled:.3f}; iterations plain /"
          f" learned {[r['plain']['iterations'] for r in rows]} / {[r['learned']['iterations'] for r in rows]}")
    assert np.isfinite(raw) and np.isfinite(scaled)
    assert scaled < 1.0          # the guess the solve starts from is better than zero in the energy norm
    assert scaled <= raw + 1e-12
    s.close()
    net.close()
