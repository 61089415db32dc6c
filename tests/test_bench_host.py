"""Host-side helpers of bench.py that need no GPU: the fluid fraction behind
the fluid-only MLUPS, and the oracle's CPU baseline with its single-core
sample."""
import numpy as np

import bench
from oracle import oracle as O
from paper_1903_04799_gb300 import workloads as W


def test_fluid_fraction_matches_the_oracle_classification():
    """Spheres on a node, off-node, across the periodic faces: the host count
    of solid nodes equals the oracle's classification exactly."""
    cases = [W.c1_fixed_squirmer(), W.c2_free_swimmer(n=40, R=6.3)]
    wl = W.c2_free_swimmer(n=36, R=5.5)
    wl.bodies[0].pos = (0.4, 35.7, 17.2)
    cases.append(wl)
    for wl in cases:
        s = O.OracleSim(*wl.shape, lambda_e=1.0, collision=wl.collision)
        for b in wl.bodies:
            s.add_sphere(b.pos, b.e, b.R, b.B1, b.beta, b.mobile)
        assert bench.fluid_fraction(wl) == float((s.owner() == 0).mean()), wl.name


def test_cpu_baseline_reports_single_core_and_restores_threads():
    wl = W.c2_free_swimmer(n=24, R=4.0)
    before = O.num_threads()
    r = bench.cpu_baseline(wl, budget_s=0.5, single_budget_s=0.5)
    assert O.num_threads() == before
    assert r["cores"] == before and r["kind"] == "oracle"
    assert r["value"] > 0 and r["single_core"]["value"] > 0
    assert isinstance(r["host"], str) and r["host"]
    assert np.isfinite(r["value"])
