"""An emission whose photon total the host does not read next leaves the
count scan to the ordering pass (each block scans the 256-track group sums
and adds the counts before its track in its group); a synchronised emission
runs the scan as its own pass. Both must give the same photons, fates, hits
and pixel counts: on ragged inputs (tracks below the Cherenkov threshold,
fixed zero counts), one track, 4096 and 4097 tracks (a group boundary: 16
full groups, then one more track), the scintillation source and the
dispersive radiator (marked gpu)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_12496_gb300 import rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402

GROUPS_16 = 4096    # tracks in 16 full scan groups of 256


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_12496_gb300 import build
    build.build()


def _run(wl, sync):
    """Emit (synchronised: the scan pass; not: the scan inside the ordering
    pass) and trace on a context that already knows the photon total, so
    both order the photons."""
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    kw = dict(source=wl.source, yield_per_mm=wl.yield_per_mm,
              spectrum_table=wl.spectrum_table, dispersion=wl.dispersion)
    n = int(ctx.emit(dt, wl.n_minus_1, wl.lambda_min, wl.lambda_max, seed=wl.seed, sync=True,
                     **kw))
    out = rich.TraceOutputs(max(n, 1), wl.scene.pixels_per_event, len(wl.scene.planes),
                            int(wl.tracks.event.max()) + 1 if wl.tracks.n else 1, max(n, 1))
    ctx.emit(dt, wl.n_minus_1, wl.lambda_min, wl.lambda_max, seed=wl.seed, sync=sync, **kw)
    ctx.trace(out, precision=rich.PREC_REFINE64)
    nh, st = ctx.hits()
    res = (st["n_photons"], st["fate"], st["photon_order"], out.fate.cpu().numpy()[:n],
           np.sort(out.hits_numpy(nh), order=["event", "track", "photon"]),
           out.pixel_counts_numpy())
    ctx.close()
    return n, res


def _ragged(n_tracks, seed):
    tr = W.pion_tracks(n_tracks, seed=seed, p_min=0.3, p_max=60.0)
    tr.p[::5] = 1.0                       # below the 2.64 GeV/c threshold: no photons
    return W.Workload("ragged", W.rich1_scene(meshed=True), tr, n_minus_1=0.0014, seed=seed)


@pytest.mark.parametrize("case", ["one_track", "ragged_7", "ragged_1000", "fixed_zero",
                                  "groups_16", "groups_16_plus_1", "scintillation",
                                  "dispersive"])
def test_deferred_scan_matches_scan_pass_edge_cases(case):
    if case == "one_track":
        wl = W.rich1(1, seed=4)
    elif case == "ragged_7":
        wl = _ragged(7, 5)
    elif case == "ragged_1000":
        wl = _ragged(1000, 6)
    elif case == "fixed_zero":
        tr = W.pion_tracks(300, seed=8, n_fixed=50)
        tr.n_fixed[::3] = 0
        wl = W.Workload("fixed", W.rich1_scene(meshed=True), tr, n_minus_1=0.0014, seed=8)
    elif case == "groups_16":
        wl = _ragged(GROUPS_16, 9)
    elif case == "groups_16_plus_1":
        wl = _ragged(GROUPS_16 + 1, 10)
    elif case == "scintillation":
        wl = W.scintillation(300, seed=11)
    else:
        wl = W.rich1_dispersive(500, seed=12)
    n_a, a = _run(wl, sync=True)
    n_b, b = _run(wl, sync=False)
    assert n_a == n_b and a[0] == b[0] == n_a and a[1] == b[1]
    assert a[2] == b[2] == 1                       # both ordered
    for x, y in zip(a[3:], b[3:]):
        np.testing.assert_array_equal(x, y)
