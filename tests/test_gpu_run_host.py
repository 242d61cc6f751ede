"""rich_run_host (one step from host memory) against the device-buffer path
(rich_emit + rich_trace + rich_hits on device tracks): the same hit records,
counters and fates, with the early hit copy off (first call) and on (later
calls); a host buffer smaller than the hit count (marked gpu)."""
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


def _sorted(h):
    return np.sort(h, order=["event", "track", "photon"])


@pytest.fixture(scope="module")
def setup():
    scene = W.rich1_scene(meshed=True)
    tracks = W.pion_tracks(300, seed=4)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    dt = rich.DeviceTracks(tracks)
    n = ctx.emit(dt, 0.0014, seed=9)
    cap = n // 2 + 1024
    out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, n)
    ctx.trace(out, precision=rich.PREC_REFINE64)
    nh, st = ctx.hits()
    ref = _sorted(out.hits_numpy(nh))
    ref_fate = out.fate.cpu().numpy().copy()
    yield ctx, scene, tracks, n, cap, nh, st, ref, ref_fate
    ctx.close()


def test_run_host_matches_device_path(setup):
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    ht = rich.HostTracks(tracks)
    out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, n)
    hits_host = torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    for rep in range(3):       # first call: no early copy; then the early copy
        hits_host.zero_()
        nh2, st2 = ctx.run_host(ht, out, hits_host, 0.0014, seed=9)
        assert nh2 == nh
        assert st2["n_photons"] == st["n_photons"] == n
        assert st2["fate"] == st["fate"]
        got = np.frombuffer(hits_host.numpy()[: nh2 * rich.HIT_DTYPE.itemsize].tobytes(),
                            rich.HIT_DTYPE)
        np.testing.assert_array_equal(_sorted(got), ref)
        np.testing.assert_array_equal(out.fate.cpu().numpy(), ref_fate)


def test_run_host_small_host_buffer(setup):
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    ht = rich.HostTracks(tracks)
    out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, n)
    k = 10
    hits_host = torch.zeros(k * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    with pytest.raises(rich.RichError) as e:
        ctx.run_host(ht, out, hits_host, 0.0014, seed=9)
    assert e.value.status == 4                      # RICH_ERR_OVERFLOW
    got = np.frombuffer(hits_host.numpy().tobytes(), rich.HIT_DTYPE)
    keys = set(zip(ref["event"], ref["track"], ref["photon"]))
    assert all((h["event"], h["track"], h["photon"]) in keys for h in got)
    # the context stays usable
    big = torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    nh2, _ = ctx.run_host(ht, out, big, 0.0014, seed=9)
    assert nh2 == nh


def test_run_host_counters_only(setup):
    """A NULL host buffer: counters only, no overflow status."""
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    from paper_2309_12496_gb300.rich import C, Stats, load, _emit_params, _trace_opts
    ht = rich.HostTracks(tracks)
    out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, n)
    prm = _emit_params(9, 0.0014, 200.0, 600.0)
    o = _trace_opts(0, rich.PREC_REFINE64, 8, 16, 1e-3, 0, 0, 0, 0, 0, -1, ())
    nh2 = C.c_uint64(0)
    s = Stats()
    status = load().rich_run_host(ctx.handle, C.byref(ht.desc()), C.byref(prm), C.byref(o),
                                  C.byref(out.desc()), None, 0, C.byref(nh2), C.byref(s))
    assert status == 0 and nh2.value == nh and s.n_photons == n
    # the binding's None, synchronous and pipelined
    nh3, st3 = ctx.run_host(ht, out, None, 0.0014, seed=9)
    assert nh3 == nh and st3["n_photons"] == n
    nh4, st4 = ctx.run_wait(ctx.run_host_async(ht, out, None, 0.0014, seed=9))
    assert nh4 == nh and st4["n_photons"] == n


def test_fate_array_smaller_than_the_photon_total(setup):
    """Photons at or beyond fate_capacity get no fate entry (nothing is
    written past the array); the entries below it equal a full array's."""
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    dt = rich.DeviceTracks(tracks)
    k = n // 3
    small = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 0)
    storage = torch.zeros(k + 64, dtype=torch.uint8, device="cuda")
    small.fate = storage[:k]              # the binding passes numel() as the capacity
    assert ctx.emit(dt, 0.0014, seed=9) == n
    ctx.trace(small, precision=rich.PREC_REFINE64)
    nh2, _ = ctx.hits()
    assert nh2 == nh
    torch.cuda.synchronize()
    got = storage.cpu().numpy()
    np.testing.assert_array_equal(got[:k], ref_fate[:k])
    assert not got[k:].any()              # nothing written past the capacity


def test_run_host_zero_tracks():
    scene = W.rich1_scene(meshed=False)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    empty = W.pion_tracks(0, seed=1)
    ht = rich.HostTracks(empty)
    out = rich.TraceOutputs(16, scene.pixels_per_event, len(scene.planes), 1, 0)
    hits_host = torch.empty(16 * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    nh, st = ctx.run_host(ht, out, hits_host, 0.0014, seed=1)
    assert nh == 0 and st["n_photons"] == 0
    ctx.close()


def test_run_host_async_pipeline_matches_sync(setup):
    """Two steps in flight (rich_run_host_async / rich_run_wait), each with
    its own outputs: every step equals the synchronous call of the same seed
    (counters, fates, hit records); a third step in flight is refused and a
    waited ticket is no longer in flight."""
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    ht = rich.HostTracks(tracks)
    seeds = [11, 12, 13, 14]
    # fate arrays with room for every seed's photons (the counts differ by seed)
    out_s = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 2 * n)
    host_s = torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    want = {}
    for s in seeds:
        nh_s, st_s = ctx.run_host(ht, out_s, host_s, 0.0014, seed=s)
        recs = np.frombuffer(host_s.numpy()[: nh_s * rich.HIT_DTYPE.itemsize].tobytes(),
                             rich.HIT_DTYPE)
        want[s] = (nh_s, st_s, _sorted(recs), out_s.fate[: st_s["n_photons"]].cpu().numpy())
    outs = [rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 2 * n)
            for _ in range(2)]
    hosts = [torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
             for _ in range(2)]
    tickets = [ctx.run_host_async(ht, outs[0], hosts[0], 0.0014, seed=seeds[0])]
    for k, s in enumerate(seeds):
        if k + 1 < len(seeds):
            tickets.append(ctx.run_host_async(ht, outs[(k + 1) % 2], hosts[(k + 1) % 2], 0.0014,
                                              seed=seeds[k + 1]))
        nh_k, st_k = ctx.run_wait(tickets[k])
        nh_s, st_s, recs_s, fate_s = want[s]
        assert nh_k == nh_s and st_k == st_s
        recs = np.frombuffer(hosts[k % 2].numpy()[: nh_k * rich.HIT_DTYPE.itemsize].tobytes(),
                             rich.HIT_DTYPE)
        np.testing.assert_array_equal(_sorted(recs), recs_s)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(outs[k % 2].fate[: st_k["n_photons"]].cpu().numpy(), fate_s)
    t1 = ctx.run_host_async(ht, outs[0], hosts[0], 0.0014, seed=1)
    t2 = ctx.run_host_async(ht, outs[1], hosts[1], 0.0014, seed=2)
    with pytest.raises(rich.RichError) as e:
        ctx.run_host_async(ht, outs[0], hosts[0], 0.0014, seed=3)
    assert e.value.status == 7                      # RICH_ERR_STATE
    ctx.run_wait(t1)
    ctx.run_wait(t2)
    with pytest.raises(rich.RichError) as e:
        ctx.run_wait(t2)
    assert e.value.status == 7


def test_run_host_isotropic_source_matches_device_path():
    """rich_run_host with the emission arguments of another light source
    (isotropic scintillation with a binned spectrum) gives the device-buffer
    path's photons, counters and hit records."""
    import parity as P
    wl = W.scintillation(60)
    ref = P.run_gpu(wl, want_fate=False, hist=False)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    ht = rich.HostTracks(wl.tracks)
    cap = ref["n"] + 1024
    out = rich.TraceOutputs(cap, wl.scene.pixels_per_event, len(wl.scene.planes), 0, 0)
    hits_host = torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    nh, st = ctx.run_host(ht, out, hits_host, wl.n_minus_1, wl.lambda_min, wl.lambda_max,
                          seed=wl.seed, source=wl.source, yield_per_mm=wl.yield_per_mm,
                          spectrum_table=wl.spectrum_table)
    ctx.close()
    assert st["n_photons"] == ref["n"] and nh == ref["n_hits"]
    assert st["fate"] == ref["stats"]["fate"]
    got = np.frombuffer(hits_host.numpy()[: nh * rich.HIT_DTYPE.itemsize].tobytes(),
                        rich.HIT_DTYPE)
    np.testing.assert_array_equal(_sorted(got), _sorted(ref["hits"]))


def test_run_host_follow_up_copy_when_the_early_copy_falls_short():
    """The early hit copy is sized from the previous step's count; a step
    with many more hits than that has its remaining records copied at
    completion (synchronous and pipelined). The records equal the
    device-buffer path's."""
    scene = W.rich1_scene(meshed=True)
    small, large = W.pion_tracks(20, seed=5), W.pion_tracks(400, seed=6)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    dt = rich.DeviceTracks(large)
    n = ctx.emit(dt, 0.0014, seed=4)
    cap = n // 2 + 1024
    ref_out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 0)
    ctx.trace(ref_out, precision=rich.PREC_REFINE64)
    nh_ref, _ = ctx.hits()
    ref = _sorted(ref_out.hits_numpy(nh_ref))
    hs, hl = rich.HostTracks(small), rich.HostTracks(large)
    outs = [rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 0)
            for _ in range(2)]
    hosts = [torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
             for _ in range(2)]

    def records(h, k):
        return _sorted(np.frombuffer(h.numpy()[: k * rich.HIT_DTYPE.itemsize].tobytes(),
                                     rich.HIT_DTYPE))

    # synchronous: small step, then the large one
    nh_s, _ = ctx.run_host(hs, outs[0], hosts[0], 0.0014, seed=4)
    assert 0 < nh_s and 4 * nh_s < nh_ref
    nh, _ = ctx.run_host(hl, outs[1], hosts[1], 0.0014, seed=4)
    assert nh == nh_ref
    np.testing.assert_array_equal(records(hosts[1], nh), ref)
    # pipelined: small step completed, then small + large in flight
    ctx.run_host(hs, outs[0], hosts[0], 0.0014, seed=4)
    t0 = ctx.run_host_async(hs, outs[0], hosts[0], 0.0014, seed=4)
    t1 = ctx.run_host_async(hl, outs[1], hosts[1], 0.0014, seed=4)
    assert ctx.run_wait(t0)[0] == nh_s
    nh, _ = ctx.run_wait(t1)
    assert nh == nh_ref
    np.testing.assert_array_equal(records(hosts[1], nh), ref)
    ctx.close()


def test_run_host_async_rejects_buffers_of_the_step_in_flight(setup):
    """A second step in flight may not write into the first one's device hit
    buffer or host hit buffer (the first step's trace and copies still write
    there): RICH_ERR_ARG, nothing enqueued, and the first step completes
    with its own results."""
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    ht = rich.HostTracks(tracks)
    outs = [rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, 2 * n)
            for _ in range(2)]
    hosts = [torch.empty(cap * rich.HIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
             for _ in range(2)]
    t1 = ctx.run_host_async(ht, outs[0], hosts[0], 0.0014, seed=9)
    with pytest.raises(rich.RichError) as e:
        ctx.run_host_async(ht, outs[0], hosts[1], 0.0014, seed=10)
    assert e.value.status == 1                      # RICH_ERR_ARG
    with pytest.raises(rich.RichError) as e:
        ctx.run_host_async(ht, outs[1], hosts[0], 0.0014, seed=10)
    assert e.value.status == 1
    nh1, st1 = ctx.run_wait(t1)
    assert nh1 == nh and st1["fate"] == st["fate"]
    recs = np.frombuffer(hosts[0].numpy()[: nh1 * rich.HIT_DTYPE.itemsize].tobytes(),
                         rich.HIT_DTYPE)
    np.testing.assert_array_equal(_sorted(recs), ref)
    # with the first step waited for, its buffers are free again
    t2 = ctx.run_host_async(ht, outs[0], hosts[0], 0.0014, seed=9)
    assert ctx.run_wait(t2)[0] == nh


def test_node_copy_wait_running_out_is_reported_and_harmless(setup):
    """The trace blocks wait, bounded, for the TMA copy of the top BVH nodes
    into shared memory. A wait limit that gives up at once (a negative
    wait_limit) makes every block record RICH_ERR_TIMEOUT, wait again for
    the copy in flight, and read the nodes from global memory: rich_hits
    reports the timeout, and the hits and fates equal the normal run's."""
    ctx, scene, tracks, n, cap, nh, st, ref, ref_fate = setup
    dt = rich.DeviceTracks(tracks)
    assert ctx.emit(dt, 0.0014, seed=9) == n
    out = rich.TraceOutputs(cap, scene.pixels_per_event, len(scene.planes), 1, n)
    ctx.trace(out, precision=rich.PREC_REFINE64, wait_limit=-1)
    with pytest.raises(rich.RichError) as e:
        ctx.hits()
    assert e.value.status == 5                      # RICH_ERR_TIMEOUT
    n_hits, st2 = ctx.hits(allow=(5,))
    assert st2["status"] == 5 and st2["device_status"] == 5
    assert n_hits == nh and st2["fate"] == st["fate"]
    np.testing.assert_array_equal(_sorted(out.hits_numpy(n_hits)), ref)
    np.testing.assert_array_equal(out.fate.cpu().numpy(), ref_fate)
    # the status is the last trace's: a normal trace reports none
    ctx.trace(out, precision=rich.PREC_REFINE64)
    assert ctx.hits()[0] == nh
