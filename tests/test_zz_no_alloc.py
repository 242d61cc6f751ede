"""The allocation-free entry point rich_photon_counts_static, for callers
that cannot allocate device memory (a framework whose pool allocator owns the
GPU's memory, or a simulation hook that must not call cudaMalloc), against
the counts the context path rich_emit produces. Collected last so that a run
stopping at its first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_12496_gb300 import build, rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402


def test_static_counts_match_emit_on_two_calls():
    build.build()
    wl = W.rich1(1000)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n_tr = wl.tracks.n
    counts = torch.empty(n_tr, dtype=torch.int32, device="cuda")
    offsets = torch.empty(n_tr + 1, dtype=torch.int64, device="cuda")
    for seed in (0, 12345):                        # two calls in a row
        n = ctx.emit(dt, wl.n_minus_1, seed=seed)
        pb = rich.PhotonBuffers(n)
        ctx.emit(dt, wl.n_minus_1, seed=seed, photons=pb)
        tracks_of = pb.t["track"][:n].cpu().numpy().view(np.uint32)
        ref = np.bincount(tracks_of, minlength=n_tr)   # track ids are indices here
        counts.fill_(-1)
        offsets.fill_(-1)
        rich.rich_photon_counts_static(dt, wl.n_minus_1, counts, offsets, seed=seed)
        torch.cuda.synchronize()
        c = counts.cpu().numpy().view(np.uint32)
        o = offsets.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(c, ref)
        np.testing.assert_array_equal(o[:-1], np.concatenate([[0], np.cumsum(ref)[:-1]]))
        assert int(o[-1]) == n
    ctx.close()


def test_static_counts_rejects_beyond_its_limit():
    wl = W.rich1(4)
    dt = rich.DeviceTracks(wl.tracks)
    counts = torch.empty(4, dtype=torch.int32, device="cuda")
    offsets = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(rich.RichError) as e:
        rich.rich_photon_counts_static(dt, 0.0014, counts, offsets, n=(1 << 20) + 1)
    assert e.value.status == 1
    assert "at most 1048576" in str(e.value)
