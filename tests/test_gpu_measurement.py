"""The measurement aids of the library (marked gpu): the microbenchmarks of
the roofline denominators, the per-kernel timing and the counting build of
the trace kernel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_12496_gb300 import rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_12496_gb300 import build
    build.build()


def test_measured_peaks_are_plausible():
    """Each measured rate lies between a quarter of and just above what the
    unit counts allow at the device's maximum clock: 128 FP32 FMA lanes per
    SM, 64 min/max lanes, 16 special-function lanes; L2 reads above the
    6.8 TB/s of HBM."""
    pk = rich.measure_peaks(0)
    f = pk["sm_clock_mhz_max"] * 1e6
    n = pk["n_sm"]
    assert 0.25 < pk["fp32_fma_flops"] / (2 * 128 * n * f) < 1.05, pk
    assert 0.25 < pk["fp32_minmax_ops"] / (128 * n * f) < 1.05, pk
    assert 0.25 < pk["mufu_ops"] / (16 * n * f) < 1.05, pk
    assert pk["l2_read_bytes"] > 6.8e12, pk


def _setup(n_tracks=300):
    scene = W.rich1_scene(meshed=True)
    tracks = W.pion_tracks(n_tracks, seed=3)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    dt = rich.DeviceTracks(tracks)
    n = ctx.emit(dt, 0.0014, seed=4, sync=True)
    return scene, ctx, dt, n


@pytest.mark.parametrize("knobs", [
    dict(block_threads=768, wide_regs=1, refill_min=32, chunk=32),
    dict(block_threads=512, blocks_per_sm=2, bvh_smem_nodes=256, refill_min=32, chunk=32),
])
def test_counting_build_gives_the_same_results_and_consistent_tallies(knobs):
    """rich_trace_work traces the last emission with the counting build (the
    72-register and the 64-register builds of one block per SM): the same
    hits and fates as rich_trace, and tallies that agree with them (one
    reflection per hit per mirror met, at least one step per photon)."""
    scene, ctx, dt, n = _setup()
    out = rich.TraceOutputs(n, scene.pixels_per_event, len(scene.planes), 1, n)
    ctx.trace(out, precision=rich.PREC_REFINE64, **knobs)
    nh, st = ctx.hits()
    ref = np.sort(out.hits_numpy(nh), order=["event", "track", "photon"])
    fate = out.fate.cpu().numpy().copy()
    ctx.emit(dt, 0.0014, seed=4, sync=True)
    out.clear()
    w = ctx.trace_work(out, **knobs)
    nh2, st2 = ctx.hits()
    got = np.sort(out.hits_numpy(nh2), order=["event", "track", "photon"])
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(out.fate.cpu().numpy(), fate)
    assert w["photons"] == n and w["detected"] == nh
    assert w["steps"] >= n
    assert w["turns"] >= int(ref["n_reflections"].astype(np.int64).sum())
    assert w["nodes_smem"] > n and w["nodes_global"] > 0 and w["tri_tests"] > n
    assert w["smooth_normals"] > 0 and w["rects"] == len(scene.rects)
    assert w["sphere_groups"] == 0 and w["tracks"] == 300
    # an unsupported form is refused
    with pytest.raises(rich.RichError):
        ctx.trace_work(out, block_threads=256)
    ctx.close()


def test_work_tallies_do_not_depend_on_the_launch():
    """A photon's steps, reflections, normal blends and detection are fixed
    by its keyed draws, so those tallies are the same for any block shape.
    Its node and triangle tests are nearly so: a lane tests its postponed
    leaf once every lane of its warp holds one, so the distance it culls
    with at a given node depends a little on its warp mates (which photons
    share a warp follows the launch); the totals agree to 0.1 %. The split
    of node tests between staged and global nodes follows the number of
    staged nodes."""
    scene, ctx, dt, n = _setup()
    out = rich.TraceOutputs(n, scene.pixels_per_event, len(scene.planes), 1, n)
    res = []
    for knobs in (dict(block_threads=896, wide_regs=1, bvh_smem_nodes=768),
                  dict(block_threads=512, blocks_per_sm=2, bvh_smem_nodes=0, chunk=64),
                  dict(block_threads=1024, bvh_smem_nodes=256, refill_min=24)):
        ctx.emit(dt, 0.0014, seed=4, sync=True)
        out.clear()
        res.append(ctx.trace_work(out, **knobs))
    for w in res[1:]:
        for k in ("photons", "steps", "smooth_normals", "turns", "detected"):
            assert w[k] == res[0][k], k
        assert w["tri_tests"] == pytest.approx(res[0]["tri_tests"], rel=1e-3)
        assert w["nodes_smem"] + w["nodes_global"] == pytest.approx(
            res[0]["nodes_smem"] + res[0]["nodes_global"], rel=1e-3)
    assert res[1]["nodes_smem"] == 0
    assert res[0]["nodes_smem"] > res[2]["nodes_smem"] > 0
    ctx.close()


def test_kernel_timing():
    """With timing on, the last emit and trace report positive kernel
    durations, the trace and refinement within the call's own event time;
    off again, nothing new is timed."""
    scene, ctx, dt, n = _setup()
    out = rich.TraceOutputs(n, scene.pixels_per_event, len(scene.planes), 1, 0)
    st = torch.cuda.current_stream()
    ctx.set_timing(True)
    ctx.emit(dt, 0.0014, seed=5, sync=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    ctx.trace(out, precision=rich.PREC_REFINE64)
    b.record(st)
    b.synchronize()
    k = ctx.kernel_times()
    assert k["yield"] > 0 and k["order"] > 0 and k["trace"] > 0 and k["refine"] > 0
    assert k["trace"] + k["refine"] <= a.elapsed_time(b) * 1.05 + 0.01
    ctx.trace(out, precision=rich.PREC_FP32)
    assert ctx.kernel_times()["refine"] == -1.0
    ctx.set_timing(False)
    ctx.trace(out, precision=rich.PREC_REFINE64)
    assert ctx.kernel_times() == {"yield": -1.0, "order": -1.0, "trace": -1.0, "refine": -1.0}
    ctx.close()
