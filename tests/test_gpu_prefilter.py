"""GPU parity of the efficiencies applied before propagation (Sec. 4.3:
the quantum efficiency and the mirror reflectivities as one accept/reject
per photon at its wavelength, rejected photons not propagated), against the
FP64 oracle on the same seeded inputs, photon by photon (marked gpu).

Bars as in test_gpu_parity.py: fates equal except oracle-flagged grazes,
hit plane and pixel equal, |du|, |dv| <= 1e-4 mm on the refined path,
pixel counts exact away from mismatched photons."""
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

# scene tables: point source (0 QE, 1 reflectivity); RICH-like scenes
# (0 QE, 1 spherical-mirror reflectivity, 2 flat-mirror reflectivity)
PRE_POINT = (0, 1)
PRE_RICH = (0, 1, 2)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2309_12496_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("precision", [rich.PREC_REFINE64, rich.PREC_FP32])
def test_point_source_prefilter_parity(precision):
    wl = W.point_source(100_000)
    ref = P.run_oracle(wl, prefilter=PRE_POINT)
    gpu = P.run_gpu(wl, precision, prefilter=PRE_POINT)
    tol = P.TOL_UV_REFINE if precision == rich.PREC_REFINE64 else P.TOL_UV_FP32["point_source"]
    P.compare(gpu, ref, wl.tracks, tol, name=f"point_source_prefilter_prec{precision}")
    f = gpu["fate"]
    assert set(np.unique(f)) <= {rich.FATE_DETECTED, rich.FATE_PREFILTERED}
    st = gpu["stats"]
    assert st["fate"][rich.FATE_PREFILTERED] == int((f == rich.FATE_PREFILTERED).sum())
    assert st["fate"][rich.FATE_DETECTED] == gpu["n_hits"]
    h = gpu["hits"]
    n = 1 + float(np.float32(0.0014))
    r = np.hypot(h["u"] - 368.64, h["v"] - 368.64)
    assert np.abs(r - 1355.0 * math.sqrt(n * n - 1)).max() < tol + 1e-6


@pytest.mark.parametrize("meshed", [True, False])
def test_rich1_prefilter_parity_full(meshed):
    """The full RICH1-like workload (1000 pion tracks, ~3.5e5 photons),
    refined, with the three efficiencies applied before propagation."""
    wl = W.rich1(1000, meshed=meshed)
    ref = P.run_oracle(wl, prefilter=PRE_RICH)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64, prefilter=PRE_RICH)
    st = P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE,
                   name=f"rich1_prefilter_meshed{int(meshed)}")
    np.testing.assert_allclose(gpu["event_sums"][..., 0], ref["event_sums"][..., 0],
                               atol=st["fate_mismatch"])
    # roughly one photon in eight passes QE x R_a x R_b
    acc = 1.0 - gpu["stats"]["fate"][rich.FATE_PREFILTERED] / gpu["n"]
    assert 0.05 < acc < 0.2


def test_prefilter_caller_photons_match_fused():
    """Caller photons (the photon-vector input of Sec. 4.2) with the prefilter
    take the same accept/reject (their keys select the QE draw) and the
    same fates as the fused emission."""
    wl = W.rich1(300)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    fused = P.run_gpu(wl, rich.PREC_FP32, ctx=ctx, dtracks=dt, prefilter=PRE_RICH)
    pb = rich.PhotonBuffers(fused["n"])
    ctx.emit(dt, wl.n_minus_1, seed=wl.seed, photons=pb)
    ext = P.run_gpu(wl, rich.PREC_FP32, ctx=ctx, dtracks=dt, photons=pb, trace_seed=wl.seed,
                    prefilter=PRE_RICH)
    np.testing.assert_array_equal(ext["fate"], fused["fate"])
    a = np.sort(fused["hits"], order=["event", "track", "photon"])
    b = np.sort(ext["hits"], order=["event", "track", "photon"])
    np.testing.assert_array_equal(a, b)
    ctx.close()


def test_prefilter_invariant_to_launch_shape_and_rejects_bad_tables():
    wl = W.rich1(200)
    base = P.run_gpu(wl, rich.PREC_REFINE64, prefilter=PRE_RICH)
    other = P.run_gpu(wl, rich.PREC_REFINE64, prefilter=PRE_RICH,
                      launch={"block_threads": 128, "refill_min": 1, "chunk": 7})
    np.testing.assert_array_equal(base["fate"], other["fate"])
    np.testing.assert_array_equal(base["pixel_counts"], other["pixel_counts"])
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = ctx.emit(dt, wl.n_minus_1, seed=wl.seed)
    out = rich.TraceOutputs(n)
    with pytest.raises(rich.RichError):
        ctx.trace(out, prefilter=(0, len(wl.scene.tables)))
    with pytest.raises(ValueError):
        ctx.trace(out, prefilter=(0, 1, 2, 0, 1))
    ctx.close()
