"""The roofline arithmetic of bench.py (no GPU): work per photon from the
counting build's tallies, the bytes the bounds use, and the committed ncu
counters the bench reads beside them."""
import json
import os

import pytest

import bench


def _tally(**kw):
    t = {"photons": 10, "steps": 0, "nodes_smem": 0, "nodes_global": 0, "tri_tests": 0,
         "smooth_normals": 0, "turns": 0, "detected": 0, "tracks": 0, "sphere_groups": 0,
         "rects": 0}
    t.update(kw)
    return t


def test_one_event_kind_at_a_time():
    """Each tallied event adds exactly its per-event cost, divided by the
    photons: a plain sum, checked one event kind at a time."""
    base = bench.work_per_photon(_tally())
    # the per-photon emission cost alone (one photon event per photon)
    assert base["fp32"] == pytest.approx(bench.WORK_COST["photon"]["fp32"])
    assert base["mufu"] == pytest.approx(bench.WORK_COST["photon"]["mufu"])
    for key, ev in (("nodes_global", "node"), ("tri_tests", "tri"),
                    ("smooth_normals", "normal"), ("turns", "turn"), ("detected", "detected")):
        w = bench.work_per_photon(_tally(**{key: 20}))
        for k in ("fp32", "minmax", "mufu"):
            assert w[k] - base[k] == pytest.approx(20 * bench.WORK_COST[ev][k] / 10), (key, k)
    # rectangles are tested once per step each
    w = bench.work_per_photon(_tally(steps=5, rects=3))
    c = bench.WORK_COST
    assert w["fp32"] - base["fp32"] == pytest.approx(
        5 * (c["step"]["fp32"] + c["shade_tri"]["fp32"] + 3 * c["rect"]["fp32"]) / 10)


def test_bytes_split_between_shared_memory_and_outside():
    """A node read from shared memory counts in `bytes` but not in the
    bytes read from outside it; streamed bytes are the records alone."""
    w = bench.work_per_photon(_tally(nodes_smem=10, nodes_global=5, tri_tests=3,
                                     smooth_normals=2, tracks=1, detected=1))
    B = bench.BYTES
    outside = (5 * B["node"] + 3 * B["tri"] + 2 * B["normal"] + B["track"]
               + 10 * B["perm"] + B["hit"] + B["refine_rec"]) / 10
    assert w["bytes_outside_smem"] == pytest.approx(outside)
    assert w["smem_bytes"] == pytest.approx(10 * B["node"] / 10)
    assert w["bytes"] == pytest.approx(outside + 10 * B["node"] / 10)
    assert w["bytes_streamed"] == pytest.approx(
        (B["track"] + 10 * (B["perm"] + 1) + B["hit"] + B["refine_rec"]) / 10)


def test_node_cost_matches_the_centre_extent_box_test():
    """Four children x three axes x (centre-distance FMA = 2, half-extent
    product, two adds) plus four widening products; min/max: two per child
    on each axis after the first and two for the [0, tmax] clamp."""
    assert bench.WORK_COST["node"]["fp32"] == 4 * 3 * 5 + 4
    assert bench.WORK_COST["node"]["minmax"] == 4 * 6


def test_committed_counters_are_complete():
    """The committed ncu counters name the sources they were taken from and
    carry every figure the bench reads from them."""
    prof = bench.load_profile()
    assert prof is not None
    for k in ("sources", "photons", "dram_bytes_per_launch", "lts_bytes_per_launch",
              "warp_inst_per_photon", "command", "launch"):
        assert k in prof, k
    assert len(prof["sources"]) == 16
    assert prof["dram_bytes_per_launch"] == prof["dram_read_bytes"] + prof["dram_write_bytes"]
    assert prof["warp_inst_per_photon"] == pytest.approx(
        prof["warp_inst_per_launch"] / prof["photons"], abs=0.01)
    assert "--clock-control none" in prof["command"]


def test_measured_hbm_peak_is_read_when_present():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    v = bench.measured_hbm_gbs()
    if os.path.exists(path):
        assert v == pytest.approx(float(json.load(open(path))["hbm_gbs"]))
    else:
        assert v is None
