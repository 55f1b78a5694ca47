"""Host legs of bench.py: the oracle baseline on one and on every host core
(spawned single-thread processes) at given PDIP iterates of a small scene, the
oracle's own window, and the failure path."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _iterates(name, k=3):
    sys.path.insert(0, ROOT)
    import bench
    from synth import scene_for

    return bench.oracle_window(scene_for(name, seed=1), k, tol=1e-10)


def test_oracle_window_is_the_pdip_trajectory():
    sys.path.insert(0, ROOT)
    from oracle import contacts as oc, pdip, qp
    from synth import scene_for

    its = _iterates("pile8", 3)
    sc = scene_for("pile8", seed=1)
    con = oc.detect(sc)
    g0, l0 = qp.initial_point(con.Nc, sc.mu)
    assert np.array_equal(its[0][0], g0) and np.array_equal(its[0][1], l0)
    _, N, r = qp.qp_data(sc, con)
    g1, l1, _ = pdip.pdip_step(N, r, sc.mu, g0, l0)  # Cholesky: same step up to the PCG tolerance
    assert np.allclose(its[1][0], g1, rtol=1e-6, atol=1e-9 * np.abs(g1).max())


def test_cpu_baseline_one_core():
    sys.path.insert(0, ROOT)
    import bench
    from synth import scene_for

    its = _iterates("pile8", 2)
    out = bench.cpu_baseline(scene_for("pile8", seed=1), its, [0, 1], tol=1e-10)
    assert out["cores"] == 1 and out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert np.isfinite(out["value"]) and out["value"] > 0 and out["iterations_per_solve"] > 0


def test_all_cores_baseline_counts_every_core():
    sys.path.insert(0, ROOT)
    import bench

    its = _iterates("pile8", 2)
    out = bench.cpu_baseline_all_cores("pile8", its, [0, 1], tol=1e-10, seconds=0.5)
    assert out["cores"] == (os.cpu_count() or 1)
    assert out["kind"] == "oracle" and out["unit"] == bench.UNIT
    assert np.isfinite(out["value"]) and out["value"] > 0


def test_all_cores_baseline_reports_a_failed_worker():
    sys.path.insert(0, ROOT)
    import bench

    its = _iterates("pile8", 1)
    out = bench.cpu_baseline_all_cores("no-such-workload", its, [0], seconds=0.5)
    assert out["value"] is None and "error" in out
