"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
the same seeded inputs, photon by photon (marked gpu).

Bars (see tests/parity.py): fates equal except oracle-flagged grazes,
mismatches at most 1e-5 of photons (+1); hit plane and pixel equal for
non-graze photons; |du|, |dv| <= 1e-4 mm on the refined path (FP32 path
bound stated per geometry); wavelengths bit-identical; pixel counts exact
away from mismatched photons.
"""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2309_12496_gb300 import rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402

import parity as P  # noqa: E402

REPORT = os.environ.get("RICH_PARITY_REPORT")


def report(name, stats):
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": name, **stats}) + "\n")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_12496_gb300 import build
    build.build()
    oracle.build()


# ------------------------------------------------------------------ Philox
def test_philox_bitwise_vs_oracle():
    """10^6 counters: the library's Philox4x32-10 equals the oracle's."""
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(1_000_000, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x9E3779B97F4A7C15
    ctx = rich.Context(0)
    got = ctx.philox(ctr, seed)
    ref = oracle.philox(ctr, np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32))
    np.testing.assert_array_equal(got, ref)
    ctx.close()


# ------------------------------------------------------------------ emission
def test_emission_matches_oracle():
    """Materialised photons of 1000 RICH1 tracks: photon counts per track
    (keys), bit-identical wavelengths, origins and directions to FP32
    accuracy."""
    wl = W.rich1(1000)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    pb = rich.PhotonBuffers(n)
    ctx.emit(dt, wl.n_minus_1, seed=wl.seed, photons=pb)
    counts, mu, off = oracle.track_yield(wl.tracks, oracle.params(wl))
    assert n == int(off[-1]) == pb.n
    g = {k: v[:n].cpu().numpy() for k, v in pb.t.items()}
    track_of = np.repeat(np.arange(wl.tracks.n), counts.astype(np.int64))
    np.testing.assert_array_equal(g["track"].view(np.uint32), wl.tracks.id[track_of])
    j = np.arange(n) - off[track_of].astype(np.int64)
    np.testing.assert_array_equal(g["photon"].view(np.uint32), j)
    prm = oracle.params(wl)
    sample = np.random.default_rng(0).choice(n, 3000, replace=False)
    max_do = max_dd = 0.0
    for k in sample:
        o, d, lam = oracle.emit(wl.tracks, prm, int(track_of[k]), int(j[k]))
        assert np.float32(lam) == g["lambda_"][k]
        max_do = max(max_do, np.abs(o - [g["x"][k], g["y"][k], g["z"][k]]).max())
        max_dd = max(max_dd, np.abs(d - [g["dx"][k], g["dy"][k], g["dz"][k]]).max())
    report("emission_rich1", {"max_origin_err_mm": max_do, "max_dir_err": max_dd})
    assert max_do < 2e-4 and max_dd < 3e-7
    ctx.close()


def test_poisson_counts_over_wide_mean_range():
    """Photon counts of 500,000 tracks whose Frank-Tamm means span 0 to ~3000
    (CDF inversion below 10, PTRS above) equal the oracle's exactly. The
    oracle draws in FP64 with the textbook forms (three logs, lgamma); the
    kernel in double-word arithmetic (~2^-44 per operation: one table-driven
    log per trial, log k! from a table), so a count could differ only if a
    floor or a rejection test fell within ~1e-10 of its threshold."""
    n = 500_000
    rng = np.random.default_rng(11)
    tr = W.pion_tracks(n, seed=11, p_min=0.3, p_max=100.0)
    tr.length[:] = (np.exp(rng.uniform(np.log(1.0), np.log(9000.0), n))).astype(tr.length.dtype)
    dt = rich.DeviceTracks(tr)
    counts = torch.empty(n, dtype=torch.int32, device="cuda")
    offsets = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    for seed in (1, 0xDEADBEEF12345):
        rich.rich_photon_counts_static(dt, 0.0014, counts, offsets, seed=seed)
        torch.cuda.synchronize()
        got = counts.cpu().numpy().view(np.uint32)
        ref, mu, off = oracle.track_yield(tr, oracle.params(seed=seed, n_minus_1=0.0014,
                                                            lambda_min=200.0, lambda_max=600.0))
        report("poisson_wide", {"seed": seed, "tracks": n, "mu_max": float(mu.max()),
                                "below_10": int((mu < 10).sum()),
                                "mismatches": int((got != ref).sum())})
        assert mu.max() > 2000 and (mu < 10).sum() > 10_000 and (mu == 0).sum() > 1000
        np.testing.assert_array_equal(got, ref)
        assert int(offsets[-1]) == int(off[-1])


# --------------------------------------------------------------- point source
def _ring_error(hits, scene, beta=1.0):
    rect = scene.rects[0]
    hu = -float(np.dot(rect["origin"].astype(np.float64), rect["u_axis"]))
    hv = -float(np.dot(rect["origin"].astype(np.float64), rect["v_axis"]))
    r = np.hypot(hits["u"] - hu, hits["v"] - hv)
    nb = (1 + float(np.float32(0.0014))) * beta
    return float(np.abs(r - 1355.0 * math.sqrt(nb * nb - 1)).max(initial=0.0))


@pytest.mark.parametrize("precision", [rich.PREC_REFINE64, rich.PREC_FP32])
def test_point_source_parity(precision):
    wl = W.point_source(100_000)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, precision)
    tol = P.TOL_UV_REFINE if precision == rich.PREC_REFINE64 else P.TOL_UV_FP32["point_source"]
    st = P.compare(gpu, ref, wl.tracks, tol, name=f"point_source_prec{precision}")
    # closed form: every hit at (R/2) tan(theta) from the plane's axis point
    st["max_ring_err_mm"] = _ring_error(gpu["hits"], wl.scene)
    report(f"point_source_prec{precision}_ring", {"max_ring_err_mm": st["max_ring_err_mm"]})
    assert st["max_ring_err_mm"] < tol + 1e-6


def test_muon_point_source_parity():
    """The paper-scale point source (one 100 GeV/c muon at the centre of
    curvature; 10^5 of its photons here): beta < 1 from the track's FP32
    momentum and mass, every hit on the ring (R/2) tan(theta) with
    cos(theta) = 1/(n beta), and photon-by-photon parity with the oracle."""
    wl = W.point_source_muon(100_000)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    st = P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name="point_source_muon")
    p, m = float(wl.tracks.p[0]), float(wl.tracks.mass[0])
    beta = p / math.sqrt(p * p + m * m)
    st["max_ring_err_mm"] = _ring_error(gpu["hits"], wl.scene, beta)
    report("point_source_muon_ring", {"max_ring_err_mm": st["max_ring_err_mm"]})
    assert gpu["n_hits"] > 10_000
    assert st["max_ring_err_mm"] < P.TOL_UV_REFINE + 1e-6


@pytest.mark.parametrize("precision", [rich.PREC_REFINE64, rich.PREC_FP32])
def test_point_source_meshed_parity(precision):
    """The point source at the centre of curvature of the mirror as a
    smooth-normal triangle mesh (3200 triangles): the kernel's normal blend
    reflects every photon back through the centre, so its hits lie on the
    analytic ring (R/2) tan(theta) within the FP32 input bound of the mesh
    (5e-4 mm, refined), and match the oracle photon by photon."""
    wl = W.point_source(100_000, meshed=True)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, precision)
    tol = P.TOL_UV_REFINE if precision == rich.PREC_REFINE64 else P.TOL_UV_FP32["point_source"]
    st = P.compare(gpu, ref, wl.tracks, tol, name=f"point_source_meshed_prec{precision}")
    st["max_ring_err_mm"] = _ring_error(gpu["hits"], wl.scene)
    report(f"point_source_meshed_prec{precision}_ring", {"max_ring_err_mm": st["max_ring_err_mm"]})
    assert gpu["n_hits"] > 10_000
    assert st["max_ring_err_mm"] < 5e-4 + (0 if precision == rich.PREC_REFINE64 else tol)


# ---------------------------------------------------------------- RICH1
@pytest.mark.parametrize("meshed", [True, False])
@pytest.mark.parametrize("precision", [rich.PREC_REFINE64, rich.PREC_FP32])
def test_rich1_parity_full(meshed, precision):
    """The full RICH1-like workload (1000 pion tracks, ~3.5e5 photons) in
    the default launch configuration the benchmark times."""
    wl = W.rich1(1000, meshed=meshed)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, precision)
    tol = P.TOL_UV_REFINE if precision == rich.PREC_REFINE64 else P.TOL_UV_FP32["rich1"]
    P.compare(gpu, ref, wl.tracks, tol, name=f"rich1_meshed{int(meshed)}_prec{precision}")


def test_rich2_parity_subset():
    """RICH2-like meshed geometry (R = 8600 mm, ~1.5e5 triangles), 300
    tracks."""
    wl = W.rich2(300)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name="rich2_meshed_300")


def test_batched_events_sampled():
    """Batched events (256 events with Poisson(50) tracks): per-photon
    parity on every photon of 24 sampled events, and their per-event pixel
    histograms and FP64 sums."""
    wl = W.batched(256, seed=1)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    sc = oracle.Scene(wl.scene)
    prm = oracle.params(wl)
    _, _, off = oracle.track_yield(wl.tracks, prm)
    events = np.random.default_rng(0).choice(256, 24, replace=False)
    sel = np.zeros(int(off[-1]), bool)
    merged = None
    for e in events:
        idx = np.nonzero(wl.tracks.event == e)[0]
        if len(idx) == 0:
            continue
        a, b = int(idx[0]), int(idx[-1]) + 1
        r = sc.trace(wl.tracks, prm, offsets=off, track_range=(a, b), n_hist_events=256)
        sel[int(off[a]):int(off[b])] = True
        if merged is None:
            merged = r
            continue
        for k in ("fate", "plane", "ix", "iy", "u", "v", "lambda", "graze", "n_refl"):
            merged[k][int(off[a]):int(off[b])] = r[k][int(off[a]):int(off[b])]
        merged["pixel_counts"] += r["pixel_counts"]
        merged["event_sums"] += r["event_sums"]
    st = P.compare(gpu, merged, wl.tracks, P.TOL_UV_REFINE, sel=sel, name="batched_256_sampled")
    assert st["photons"] > 20_000 and "event_sums_bad" in st


# ------------------------------------------------------------- invariances
def test_external_photons_match_fused():
    """Photons materialised by rich_emit and traced as caller photons (the
    photon-vector input of Sec. 4.2) give bit-identical fates and FP32 hits
    to the fused emission. Refined hits of caller photons are exact for
    their FP32 inputs, whose direction rounding (~6e-8 rad) over the ~3 m
    lever arm of the optics moves a hit by up to ~2e-4 mm from the fused
    path's FP64 emission: bound 5e-4 mm."""
    wl = W.rich1(300)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    for prec in (rich.PREC_FP32, rich.PREC_REFINE64):
        fused = P.run_gpu(wl, prec, ctx=ctx, dtracks=dt)
        n = fused["n"]
        pb = rich.PhotonBuffers(n)
        ctx.emit(dt, wl.n_minus_1, seed=wl.seed, photons=pb)
        ext = P.run_gpu(wl, prec, ctx=ctx, dtracks=dt, photons=pb, trace_seed=wl.seed)
        np.testing.assert_array_equal(ext["fate"], fused["fate"])
        a = np.sort(fused["hits"], order=["event", "track", "photon"])
        b = np.sort(ext["hits"], order=["event", "track", "photon"])
        if prec == rich.PREC_FP32:
            np.testing.assert_array_equal(a, b)
        else:
            for k in ("event", "track", "photon", "plane", "lambda", "n_reflections"):
                np.testing.assert_array_equal(a[k], b[k])
            assert np.abs(a["u"] - b["u"]).max() < 5e-4
            assert np.abs(a["v"] - b["v"]).max() < 5e-4
    ctx.close()


@pytest.mark.parametrize("launch", [
    {"block_threads": 128, "refill_min": 1, "chunk": 32},
    {"block_threads": 256, "refill_min": 32, "chunk": 1024, "blocks_per_sm": 1},
    {"block_threads": 64, "refill_min": 8, "chunk": 7},
    # the builds of one block per SM, cold photon state in shared memory
    {"block_threads": 896, "wide_regs": 1, "bvh_smem_nodes": 256},
    {"block_threads": 1024, "bvh_smem_nodes": 768},
    {"block_threads": 320, "refill_min": 24, "chunk": 64, "bvh_smem_nodes": 0},
])
def test_results_invariant_to_launch_shape(launch):
    """Keyed random numbers: block shape, compaction interval and chunk
    size change nothing in the per-photon results."""
    wl = W.rich1(200)
    base = P.run_gpu(wl, rich.PREC_REFINE64)
    other = P.run_gpu(wl, rich.PREC_REFINE64, launch=launch)
    np.testing.assert_array_equal(base["fate"], other["fate"])
    a = np.sort(base["hits"], order=["event", "track", "photon"])
    b = np.sort(other["hits"], order=["event", "track", "photon"])
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(base["pixel_counts"], other["pixel_counts"])


def test_azimuth_order_changes_nothing():
    """The trace takes each track's photons in azimuth order once the
    context knows the photon total (a synchronised emission); a fresh
    context emitting without synchronising traces in index order. Both give
    the same fates, hits and pixel counts."""
    wl = W.rich1(300)
    res = {}
    for sync in (False, True):
        ctx = rich.Context(0)
        ctx.init_geometry(wl.scene)
        dt = rich.DeviceTracks(wl.tracks)
        n = int(ctx.emit(dt, wl.n_minus_1, seed=wl.seed, sync=True)) if sync else None
        if not sync:
            ctx.emit(dt, wl.n_minus_1, seed=wl.seed, sync=False)
            n = 400_000
        out = rich.TraceOutputs(n, wl.scene.pixels_per_event, len(wl.scene.planes), 1, n)
        ctx.trace(out, precision=rich.PREC_REFINE64)
        nh, st = ctx.hits()
        res[sync] = (st["photon_order"], st["n_photons"], out.fate[: st["n_photons"]].cpu().numpy(),
                     np.sort(out.hits_numpy(nh), order=["event", "track", "photon"]),
                     out.pixel_counts_numpy())
        ctx.close()
    assert res[False][0] == 0 and res[True][0] == 1
    assert res[False][1] == res[True][1]
    for k in (2, 3, 4):
        np.testing.assert_array_equal(res[False][k], res[True][k])


def test_mixed_track_sizes_order_invariant():
    """Tracks above 16,384 photons keep index order while the others are
    ordered by azimuth; with both kinds in one emission the trace finds each
    photon's track by search and takes the ordered tracks' photons from
    their queue entries. Fates, hits and pixel counts equal those of the
    same photons traced in index order (a fresh context emitting without
    synchronising)."""
    tracks = W.pion_tracks(6, seed=11, n_fixed=100)
    tracks.n_fixed[:] = [20_000, 300, 17_000, 1_000, 50, 4_000]
    scene = W.rich1_scene(meshed=True)
    res = {}
    for sync in (False, True):
        ctx = rich.Context(0)
        ctx.init_geometry(scene)
        dt = rich.DeviceTracks(tracks)
        if sync:
            n = int(ctx.emit(dt, 0.0014, seed=2, sync=True))
        else:
            ctx.emit(dt, 0.0014, seed=2, sync=False)
            n = 50_000
        out = rich.TraceOutputs(n, scene.pixels_per_event, len(scene.planes), 1, n)
        ctx.trace(out, precision=rich.PREC_REFINE64)
        nh, st = ctx.hits()
        res[sync] = (st["photon_order"], st["n_photons"], out.fate[: st["n_photons"]].cpu().numpy(),
                     np.sort(out.hits_numpy(nh), order=["event", "track", "photon"]),
                     out.pixel_counts_numpy())
        ctx.close()
    assert res[False][0] == 0 and res[True][0] == 1
    assert res[False][1] == res[True][1] == 42_350
    for k in (2, 3, 4):
        np.testing.assert_array_equal(res[False][k], res[True][k])


def test_deferred_scan_matches_scan_pass():
    """An unsynchronised emission leaves the count scan to the ordering pass
    (offsets and total from the group sums); a synchronised one runs the
    scan pass. On 3000 tracks (12 scan groups, a ragged last one, tracks
    below threshold with no photons), the second emission of a context is
    ordered either way and both give the same photons, fates, hits and
    pixel counts."""
    tr = W.pion_tracks(3000, seed=21, p_min=0.3, p_max=60.0)
    scene = W.rich1_scene(meshed=True)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    dt = rich.DeviceTracks(tr)
    n = int(ctx.emit(dt, 0.0014, seed=3, sync=True))
    res = []
    for sync in (True, False):
        out = rich.TraceOutputs(n, scene.pixels_per_event, len(scene.planes), 1, n)
        if sync:
            assert int(ctx.emit(dt, 0.0014, seed=3, sync=True)) == n
        else:
            ctx.emit(dt, 0.0014, seed=3, sync=False)
        ctx.trace(out, precision=rich.PREC_REFINE64)
        nh, st = ctx.hits()
        res.append((st["photon_order"], st["n_photons"], st["fate"], out.fate.cpu().numpy(),
                    np.sort(out.hits_numpy(nh), order=["event", "track", "photon"]),
                    out.pixel_counts_numpy()))
    ctx.close()
    assert res[0][0] == res[1][0] == 1
    assert res[0][1] == res[1][1] == n
    assert res[0][2] == res[1][2]
    for k in (3, 4, 5):
        np.testing.assert_array_equal(res[0][k], res[1][k])


# --------------------------------------------------------------- edge cases
def test_zero_tracks_and_empty_emission():
    wl = W.rich1(10)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    empty = W.Tracks(**{f: getattr(wl.tracks, f)[:0] for f in W.Tracks.FIELDS},
                     event=wl.tracks.event[:0], id=wl.tracks.id[:0])
    dt = rich.DeviceTracks(empty)
    assert ctx.emit(dt, 0.0014) == 0
    out = rich.TraceOutputs(1, wl.scene.pixels_per_event, 3, 1, 0)
    ctx.trace(out)
    n_hits, st = ctx.hits()
    assert n_hits == 0 and st["n_photons"] == 0 and sum(st["fate"]) == 0
    ctx.close()


def test_below_threshold_and_fixed_zero():
    """Tracks below the Cherenkov threshold and tracks with a fixed count of
    zero emit nothing; neighbours are unaffected (ragged counts)."""
    tr = W.pion_tracks(64, seed=9)
    tr.p[::3] = 1.5                           # below the 2.64 GeV/c threshold
    wl = W.Workload("ragged", W.rich1_scene(), tr, n_minus_1=0.0014)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)
    tr2 = W.pion_tracks(16, seed=9, n_fixed=5)
    tr2.n_fixed[::2] = 0
    wl2 = W.Workload("fixed", W.rich1_scene(), tr2, n_minus_1=0.0014)
    ref2 = P.run_oracle(wl2)
    gpu2 = P.run_gpu(wl2, rich.PREC_REFINE64)
    assert gpu2["n"] == 40
    P.compare(gpu2, ref2, wl2.tracks, P.TOL_UV_REFINE)


def test_hit_overflow_reports_true_count():
    wl = W.point_source(20_000)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1)
    out = rich.TraceOutputs(10, wl.scene.pixels_per_event, 1, 1, 0)
    ctx.trace(out)
    with pytest.raises(rich.RichError) as e:
        ctx.hits()
    assert e.value.status == 4
    n_hits, st = ctx.hits(allow_overflow=True)
    assert n_hits > 10 and st["n_hits"] == n_hits
    assert int(out.pixel_counts_numpy().sum()) == n_hits
    ctx.close()


def test_max_bounces_limit():
    """max_bounces = 1: photons needing a second reflection stop there."""
    wl = W.rich1(100)
    ref = P.run_oracle(wl, max_bounces=1)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    out = rich.TraceOutputs(n, wl.scene.pixels_per_event, 3, 1, n)
    ctx.trace(out, max_bounces=1)
    n_hits, st = ctx.hits()
    gpu = {"n": n, "fate": out.fate.cpu().numpy(), "hits": out.hits_numpy(n_hits)}
    assert (gpu["fate"] == 6).sum() > 0
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE)
    ctx.close()


def test_invalid_inputs_are_rejected():
    wl = W.rich1(10)
    ctx = rich.Context(0)
    with pytest.raises(rich.RichError) as e:
        ctx.trace(rich.TraceOutputs(1))
    assert e.value.status == 7                      # no geometry yet
    bad = W.rich1_scene()
    bad.materials = bad.materials.copy()
    bad.materials[0]["table"] = 99
    with pytest.raises(rich.RichError) as e:
        ctx.init_geometry(bad)
    assert e.value.status == 6
    bad = W.point_source_scene()
    bad.rects = bad.rects.copy()
    bad.rects[0]["nx"] = 100                        # grid no longer fits
    with pytest.raises(rich.RichError) as e:
        ctx.init_geometry(bad)
    assert e.value.status == 6
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    with pytest.raises(rich.RichError) as e:
        ctx.emit(dt, -1.0)
    assert e.value.status == 1
    ctx.emit(dt, 0.0014)
    with pytest.raises(rich.RichError) as e:
        ctx.trace(rich.TraceOutputs(1), max_bounces=0)
    assert e.value.status == 1
    small = rich.PhotonBuffers(3)
    with pytest.raises(rich.RichError) as e:
        ctx.emit(dt, 0.0014, photons=small)
    assert e.value.status == 4
    ctx.close()
