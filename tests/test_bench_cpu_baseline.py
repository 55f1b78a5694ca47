"""Host legs of bench.py: the oracle baseline on every host core (spawned
single-thread processes) on a small scene, and its failure path."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cold_state(name):
    sys.path.insert(0, ROOT)
    from oracle import contacts as oc, qp
    from synth import scene_for

    sc = scene_for(name, seed=1)
    con = oc.detect(sc)
    g, lam = qp.initial_point(con.Nc, sc.mu)
    _, P = qp.padded_size(con.Nc, 3)
    return torch.tensor(qp.to_padded(g, con.Nc, 3, P)), torch.tensor(lam)


def test_all_cores_baseline_counts_every_core():
    sys.path.insert(0, ROOT)
    import bench

    g, lam = _cold_state("pile8")
    out = bench.cpu_baseline_all_cores("pile8", g, lam, 20.0, seconds=0.5)
    assert out["cores"] == (os.cpu_count() or 1)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert np.isfinite(out["value"]) and out["value"] > 0


def test_all_cores_baseline_reports_a_failed_worker():
    sys.path.insert(0, ROOT)
    import bench

    g, lam = _cold_state("pile8")
    out = bench.cpu_baseline_all_cores("no-such-workload", g, lam, 20.0, seconds=0.5)
    assert out["value"] is None and "error" in out
