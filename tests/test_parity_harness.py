"""The photon-by-photon parity harness (tests/parity.py) checked on the CPU:
given the oracle's own results dressed as a GPU run it passes, and each
kind of discrepancy it exists to catch, planted in that copy, makes it fail.
No GPU: the "GPU" side here is the oracle's output in the library's hit
record layout."""
import numpy as np
import pytest

import oracle
from paper_2309_12496_gb300 import rich
from paper_2309_12496_gb300 import workloads as W

import parity as P


@pytest.fixture(scope="module")
def case():
    oracle.build()
    wl = W.rich1(120, meshed=True)
    P.set_grid(wl.scene.planes)
    ref = P.run_oracle(wl)
    return wl, ref


def _as_gpu(wl, ref):
    off = ref["offsets"].astype(np.int64)
    n = int(off[-1])
    det = np.nonzero(ref["fate"] == oracle.FATE_DETECTED)[0]
    t = np.searchsorted(off, det, side="right") - 1
    hits = np.zeros(len(det), rich.HIT_DTYPE)
    hits["event"] = wl.tracks.event[t]
    hits["track"] = wl.tracks.id[t]
    hits["photon"] = det - off[t]
    for k in ("plane", "ix", "iy", "u", "v", "lambda"):
        hits[k] = ref[k][det]
    hits["n_reflections"] = ref["n_refl"][det]
    return {"n": n, "n_hits": len(det), "hits": hits, "fate": ref["fate"].copy(),
            "pixel_counts": ref["pixel_counts"].copy(), "event_sums": ref["event_sums"].copy()}


def test_identical_results_pass(case):
    wl, ref = case
    st = P.compare(_as_gpu(wl, ref), ref, wl.tracks, P.TOL_UV_REFINE)
    assert st["mismatched_photons"] == 0 and st["hits"] > 1000
    assert st["pixels_differing"] == 0 and st["event_sums_bad"] == 0


def _clean_hit(ref, gpu):
    """Index in the hit list of a detected photon the oracle does not flag."""
    h = gpu["hits"]
    off = ref["offsets"].astype(np.int64)
    for k in range(len(h)):
        g = off[int(h["track"][k])] + int(h["photon"][k])
        if ref["graze"][g] == 0:
            return k, g
    raise AssertionError


def test_pixel_of_a_clean_photon_differs(case):
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    k, g = _clean_hit(ref, gpu)
    gpu["hits"]["ix"][k] += 1
    with pytest.raises(AssertionError):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)


def test_hit_list_disagrees_with_fate_array(case):
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    k, g = _clean_hit(ref, gpu)
    gpu["hits"] = np.delete(gpu["hits"], k)
    gpu["n_hits"] -= 1
    with pytest.raises(AssertionError, match="marks detected"):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)


def test_graze_mismatches_are_counted(case):
    """Pixel changes on photons the oracle flags as grazes are excused one
    by one, but count against the allowance (here one photon)."""
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    off = ref["offsets"].astype(np.int64)
    h = gpu["hits"]
    g_of = off[h["track"].astype(np.int64)] + h["photon"].astype(np.int64)
    grazed = np.nonzero(ref["graze"][g_of] != 0)[0]
    assert len(grazed) >= 2
    # one grazing photon moved to the next pixel: allowed, its pixels excused
    gpu["hits"]["ix"][grazed[0]] ^= 1
    pc = gpu["pixel_counts"]
    ev = int(h["event"][grazed[0]])
    base = [0, 65536, 131072][int(h["plane"][grazed[0]])]
    old = base + int(h["iy"][grazed[0]]) * 256 + (int(h["ix"][grazed[0]]) ^ 1)
    new = base + int(h["iy"][grazed[0]]) * 256 + int(h["ix"][grazed[0]])
    pc[ev, old] -= 1
    pc[ev, new] += 1
    st = P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)
    assert st["mismatched_photons"] == 1 and st["pixels_unexplained"] == 0
    # a second one exceeds the allowance of this 4e4-photon case
    gpu["hits"]["ix"][grazed[1]] ^= 1
    with pytest.raises(AssertionError):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)


def test_pixel_count_off_elsewhere(case):
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    gpu["pixel_counts"][0, 12345] += 1
    with pytest.raises(AssertionError):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)


@pytest.mark.parametrize("column,delta", [(0, 1.0), (1, 1e-6), (2, 1e-6), (3, 1e-6)])
def test_event_sums_checked_in_every_column(case, column, delta):
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    gpu["event_sums"][0, 0, column] += delta * max(1.0, abs(gpu["event_sums"][0, 0, column]))
    with pytest.raises(AssertionError):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)


def test_position_error_beyond_tolerance(case):
    wl, ref = case
    gpu = _as_gpu(wl, ref)
    k, g = _clean_hit(ref, gpu)
    gpu["hits"]["u"][k] += 2e-4
    with pytest.raises(AssertionError):
        P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)
