"""Host-side helpers of bench.py (no GPU): the particle workload reaches the
volume fraction it states, and the committed DRAM-traffic table parses."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_particle_workload_volume_fraction():
    W = bench.particle_workload(64, 0.10)
    sp = W["spheres"]
    vol = 4.0 / 3.0 * np.pi * sp["radius"] ** 3
    assert len(sp["r"]) == int(round(0.10 * 64 ** 3 / vol))
    assert abs((1.0 - W["fluid"]) - 0.10) < 0.02          # discrete spheres, about the stated fraction
    assert sp["mass"] == 2.2 * vol and sp["contact"] == (10.0, 1.0)
    d = sp["r"][:, None, :] - sp["r"][None, :, :]
    d -= 64 * np.round(d / 64)
    dist = np.sqrt((d * d).sum(axis=2)) + np.eye(len(sp["r"])) * 1e9
    assert dist.min() >= 2 * sp["radius"] + 1 - 1e-9         # gaps of at least one node


def test_traffic_table_parses():
    for key in ("fp32", "fp16", "colloid_fp32", "colloid_fp16", "single_fp32", "particles_fp32"):
        v = bench.traffic_per_site(key)
        assert v is not None and 100.0 < v < 400.0, key
    assert bench.traffic_per_site("fp64") is None
