"""Batching features on the GPU (marked gpu): the emit + trace sequence
captured as a CUDA graph, the autotuner, and chunked runs that resume from
(chunk index, accumulated histograms)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_12496_gb300 import autotune, build, rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _sorted_hits(out, n):
    return np.sort(out.hits_numpy(n), order=["event", "track", "photon"])


def test_graph_replay_matches_direct_calls():
    """Replays of the captured graph give exactly the hits, pixel counts and
    sums of a direct rich_emit + rich_trace with the same inputs."""
    wl = W.batched(64, seed=4)
    ne = 64
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    args = (n, wl.scene.pixels_per_event, len(wl.scene.planes), ne, n)
    direct = rich.TraceOutputs(*args)
    ctx.trace(direct)
    nd, _ = ctx.hits()
    graph = rich.TraceOutputs(*args)
    ctx.graph_capture(dt, graph, wl.n_minus_1, seed=wl.seed)
    for _ in range(2):
        graph.clear()
        ctx.graph_launch()
        ng, st = ctx.hits()
        assert ng == nd and st["n_photons"] == n
        np.testing.assert_array_equal(_sorted_hits(graph, ng), _sorted_hits(direct, nd))
        np.testing.assert_array_equal(graph.pixel_counts_numpy(), direct.pixel_counts_numpy())
        np.testing.assert_allclose(graph.event_sums_numpy(), direct.event_sums_numpy(),
                                   rtol=1e-12)
        np.testing.assert_array_equal(graph.fate.cpu().numpy(), direct.fate.cpu().numpy())
    ctx.close()


def test_autotuner_picks_a_candidate_and_results_do_not_change():
    wl = W.rich1(200)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    out = rich.TraceOutputs(n, wl.scene.pixels_per_event, 3, 1, n)
    space = autotune.candidates(wl.scene.n_triangles)[::5]
    knobs, ms, table = autotune.tune(ctx, out, n, rich.PREC_REFINE64, reps=1,
                                     use_cache=False, space=space)
    # every candidate runs, or is refused as a shape that does not fit
    assert knobs in space and ms > 0 and len(table) + len(autotune.failed) == len(space)
    for k, msg in autotune.failed:
        assert "does not fit" in msg or "exceed shared memory" in msg, (k, msg)
    assert len(table) >= len(space) - 2, autotune.failed
    out.clear()
    ctx.trace(out, **knobs)
    n1, _ = ctx.hits()
    a = _sorted_hits(out, n1)
    fa = out.fate.cpu().numpy()
    out.clear()
    ctx.trace(out)
    n2, _ = ctx.hits()
    np.testing.assert_array_equal(a, _sorted_hits(out, n2))
    np.testing.assert_array_equal(fa, out.fate.cpu().numpy())
    ctx.close()


def test_chunked_run_resumes_exactly():
    """Chunks are independent (keyed random numbers): histograms of chunks
    0-3 in one run equal chunks 0-1, then 2-3 resumed in a fresh context
    from the saved (chunk index, histograms)."""
    scene = W.rich2_scene(meshed=True)
    chunks = []
    for c in range(4):
        tr = W.pion_tracks(150, seed=c, length=2000.0, max_angle=0.15)
        tr.id[:] = np.arange(150) + 150 * c
        chunks.append(tr)

    def run(ctx, idx, hist=None):
        out = rich.TraceOutputs(200_000, scene.pixels_per_event, 2, 1, 0)
        if hist is not None:
            out.pixel_counts.copy_(hist)
        for c in idx:
            ctx.emit(rich.DeviceTracks(chunks[c]), 0.0005, seed=3)
            ctx.trace(out)
        torch.cuda.synchronize()
        return out.pixel_counts.clone()

    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    whole = run(ctx, range(4))
    saved = run(ctx, range(2))           # checkpoint: next chunk = 2, histograms
    ctx.close()
    ctx2 = rich.Context(0)
    ctx2.init_geometry(scene)
    resumed = run(ctx2, range(2, 4), hist=saved)
    ctx2.close()
    assert int(whole.sum()) > 1000
    assert torch.equal(whole, resumed)
