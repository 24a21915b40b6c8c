"""Host logic of bench.py (no GPU): workload table, the far-kernel traffic
record and the roofline arithmetic."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_workloads_are_complete():
    need = {"op", "leaf", "eta", "eps", "eps_aca", "ng", "nrhs", "c"}
    for name, cfg in bench.WORKLOADS.items():
        assert need <= set(cfg), name
        assert ("level" in cfg) != ("housing" in cfg), name
        assert ("N" in cfg and "dt" in cfg) != ("gcq" in cfg), name
    assert "sphere5120_slp_bdf2_N64" in bench.WORKLOADS


def test_far_traffic_only_for_the_measured_workload():
    assert bench.far_traffic("sphere5120_slp_bdf2_N64") is None
    t = bench.far_traffic(bench.FAR_TRAFFIC["workload"])
    assert t is None or t == bench.FAR_TRAFFIC["bytes"]


def test_roofline_arithmetic():
    blocks = np.array([[0, 10, 10, 20, 0], [0, 10, 20, 40, 1]], dtype=np.int32)
    st = {"ms_singular": 1.0, "ms_near": 2.0, "ms_far": 10.0, "entries_regular": 100 * 33 + 5000,
          "entries_tube": 700}
    cfg = {"op": "SLP", "Nu": 33}
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    r = bench.roofline(st, cfg, blocks, peaks, "measured", {"sm_mhz": 2000.0}, "x", {"sfu": 4e12})
    pairs = (5000 + 700) * 49
    assert abs(r["achieved"] - pairs * 4 / 0.010 / 1e12) < 1e-12
    assert r["peak"] == 4.0 and abs(r["frac"] - r["achieved"] / 4.0) < 1e-15
    r2 = bench.roofline(st, cfg, blocks, peaks, "measured", {"sm_mhz": 2000.0}, "x", None)
    assert abs(r2["peak"] - 16 * 152 * 2000e6 / 1e12) < 1e-12


def test_oracle_samples_are_stratified_and_disjoint():
    rng = np.random.default_rng(0)
    nb = 1000
    i0 = rng.integers(0, 100, nb)
    blocks = np.stack([i0, i0 + rng.integers(1, 300, nb), i0, i0 + rng.integers(1, 300, nb),
                       rng.integers(0, 2, nb)], axis=1).astype(np.int32)
    masks = []
    for off in range(5):
        m, k = bench.oracle_sample_mask(blocks, 24, off)
        assert k == -(-nb // 24) and m.sum() == -(-nb // k)
        masks.append(m)
        # one block from each stratum of k blocks in decreasing size order
        sz = (blocks[:, 1] - blocks[:, 0]).astype(np.int64) * (blocks[:, 3] - blocks[:, 2])
        order = np.lexsort((np.arange(nb), -sz))
        for a in range(0, nb, k):
            assert m[order[a:a + k]].sum() == 1
    assert not np.any(np.sum(masks, axis=0) > 1)  # disjoint samples
    m2, _ = bench.oracle_sample_mask(blocks, 24, 3)
    assert np.array_equal(m2, masks[3])  # deterministic
