"""GPU parity of photons given by the caller (the photon emitter's vectors
of positions and momenta, Sec. 4.2) against the oracle's entry point for
caller photons, photon by photon (marked gpu).

Both sides read the same FP32 origins, directions and wavelengths and draw
the reflectivity and QE uniforms from the photons' own keys (event, track,
photon) under the same seed, so the bars are those of the emitted-photon
parity (tests/parity.py): fates equal except oracle-flagged grazes (at most
1e-5 of photons), the same plane and pixel, |du|, |dv| <= 1e-4 mm on the
refined path (2e-3 mm in FP32), exact pixel counts and FP64 event sums.
"""
import math

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


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_12496_gb300 import build
    build.build()
    oracle.build()


def _gpu_ext(ctx, scene, arrays, seed, precision, n_ev):
    pb = rich.PhotonBuffers.from_arrays(**arrays)
    out = rich.TraceOutputs(max(pb.n, 1), scene.pixels_per_event, len(scene.planes), n_ev, pb.n)
    ctx.trace(out, photons=pb, precision=precision, seed=seed)
    n_hits, stats = ctx.hits()
    return {"n": pb.n, "n_hits": n_hits, "stats": stats, "hits": out.hits_numpy(n_hits),
            "fate": out.fate.cpu().numpy()[:pb.n], "pixel_counts": out.pixel_counts_numpy(),
            "event_sums": out.event_sums_numpy()}


def _oracle_ext(scene, arrays, seed, n_ev):
    sc = oracle.Scene(scene)
    prm = oracle.params(None, seed=seed, n_minus_1=0.0014, lambda_min=200.0, lambda_max=600.0)
    o = np.column_stack([arrays["x"], arrays["y"], arrays["z"]])
    d = np.column_stack([arrays["dx"], arrays["dy"], arrays["dz"]])
    return sc.trace_photons(o, d, arrays["lambda"], arrays["event"], arrays["track"],
                            arrays["photon"], prm, n_hist_events=n_ev)


def _check(scene, arrays, seed, name):
    P.set_grid(scene.planes)
    keys = (arrays["event"], arrays["track"], arrays["photon"])
    n_ev = int(arrays["event"].max()) + 1
    ref = _oracle_ext(scene, arrays, seed, n_ev)
    ctx = rich.Context(0)
    ctx.init_geometry(scene)
    stats = {}
    for prec, tol in ((rich.PREC_REFINE64, P.TOL_UV_REFINE), (rich.PREC_FP32, P.TOL_UV_FP32["rich1"])):
        gpu = _gpu_ext(ctx, scene, arrays, seed, prec, n_ev)
        stats[prec] = P.compare(gpu, ref, None, tol, keys=keys, name=f"{name}_prec{prec}")
    ctx.close()
    return stats


def test_emitted_photons_as_caller_photons_match_oracle():
    """Photons of 1000 RICH1 tracks materialised by rich_emit (FP32), then
    traced as caller photons: the oracle traces the same FP32 arrays."""
    wl = W.rich1(1000)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    pb = rich.PhotonBuffers(n)
    ctx.emit(dt, wl.n_minus_1, seed=wl.seed, photons=pb)
    arrays = {("lambda" if f == "lambda_" else f): pb.t[f][:n].cpu().numpy()
              for f in rich.PhotonBuffers.FIELDS}
    for f in rich.PhotonBuffers.KEYS:
        arrays[f] = pb.t[f][:n].cpu().numpy().view(np.uint32)
    ctx.close()
    st = _check(wl.scene, arrays, wl.seed, "ext_emitted_rich1")
    assert st[rich.PREC_REFINE64]["hits"] > 40_000


def test_arbitrary_caller_photons_match_oracle():
    """200,000 photons with origins uniform in the radiator volume
    (|x|, |y| <= 200 mm, 0 <= z <= 1000 mm), directions uniform in solid
    angle within 0.35 rad of the mirror axis, wavelengths uniform on
    [200, 600] nm, spread over 7 events, with track and photon keys chosen
    at random by the caller (not those of any emission)."""
    rng = np.random.default_rng(2024)
    n = 200_000
    ct = 1.0 - rng.random(n) * (1.0 - math.cos(0.35))
    st = np.sqrt(1 - ct * ct)
    ph = 2 * math.pi * rng.random(n)
    arrays = {
        "x": rng.uniform(-200, 200, n).astype(np.float32),
        "y": rng.uniform(-200, 200, n).astype(np.float32),
        "z": rng.uniform(0, 1000, n).astype(np.float32),
        "dx": (st * np.cos(ph)).astype(np.float32),
        "dy": (st * np.sin(ph)).astype(np.float32),
        "dz": ct.astype(np.float32),
        "lambda": rng.uniform(200, 600, n).astype(np.float32),
        "event": rng.integers(0, 7, n).astype(np.uint32),
        "track": rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32),
        "photon": np.arange(n, dtype=np.uint32) * np.uint32(2654435761),
    }
    scene = W.rich1_scene(meshed=True)
    stats = _check(scene, arrays, seed=0xC0FFEE, name="ext_arbitrary_rich1")
    assert stats[rich.PREC_REFINE64]["hits"] > 10_000
