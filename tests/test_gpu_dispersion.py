"""GPU parity of the dispersive radiator (n(lambda) in the radiator: each
photon's Cherenkov angle at its own wavelength, the Frank-Tamm integral of
sin^2 theta(lambda) as the mean count, the wavelength law
sin^2 theta(lambda) / lambda^2) against the FP64 oracle (marked gpu).

Bars as in test_gpu_parity.py; photon counts and wavelengths bit-exact."""
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


@pytest.mark.parametrize("meshed", [True, False])
def test_rich1_dispersive_parity_full(meshed):
    """1000 pion tracks with n(lambda), refined hits."""
    wl = W.rich1_dispersive(1000, meshed=meshed)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name=f"rich1_dispersive_meshed{int(meshed)}")


def test_dispersive_point_source_ring_per_wavelength():
    """beta = 1 point source at the centre of curvature: every hit at
    (R/2) sqrt(n(lambda)^2 - 1) for its own wavelength, on the GPU."""
    wl = W.point_source(100_000)
    wl.dispersion = W.C4F10_DISPERSION
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name="point_source_dispersive")
    a, l0 = (np.float64(x) for x in W.C4F10_DISPERSION)
    h = gpu["hits"]
    half = -float(np.dot(wl.scene.rects[0]["origin"], wl.scene.rects[0]["u_axis"]))
    r = np.hypot(h["u"] - half, h["v"] - half)
    lam = h["lambda"].astype(np.float64)
    n = 1 + a / (1 / l0**2 - 1 / lam**2)
    assert np.abs(r - 1355.0 * np.sqrt(n * n - 1)).max() < 1e-4


def test_dispersive_counts_across_threshold():
    """Per-track counts equal the oracle's keyed Poisson draws of the
    closed-form mean, for 20,000 pions from 2.3 to 100 GeV/c (below, across
    and far above the threshold band 2.47-2.64 GeV/c)."""
    tr = W.pion_tracks(20_000, seed=5, p_min=2.3)
    wl = W.rich1_dispersive(1, meshed=False)
    wl.tracks = tr
    n_ref, mu, off = oracle.track_yield(tr, oracle.params(wl))
    assert (mu == 0).sum() > 100 and ((mu > 0) & (mu < 100)).sum() > 100
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(tr)
    counts = torch.empty(tr.n, dtype=torch.int32, device="cuda")
    offs = torch.empty(tr.n + 1, dtype=torch.int64, device="cuda")
    rich.rich_photon_counts_static(dt, 0.0, counts, offs, seed=wl.seed,
                                   dispersion=wl.dispersion)
    np.testing.assert_array_equal(counts.cpu().numpy().view(np.uint32), n_ref)
    n = ctx.emit(dt, 0.0, seed=wl.seed, dispersion=wl.dispersion)
    assert n == int(off[-1])
    ctx.close()


def test_dispersive_caller_photons_match_fused():
    """Materialised dispersive photons traced as caller photons: same fates
    and FP32 hits as the fused emission; wavelengths equal the oracle's."""
    wl = W.rich1_dispersive(200)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    fused = P.run_gpu(wl, rich.PREC_FP32, ctx=ctx, dtracks=dt)
    pb = rich.PhotonBuffers(fused["n"])
    ctx.emit(dt, 0.0, seed=wl.seed, photons=pb, dispersion=wl.dispersion)
    ext = P.run_gpu(wl, rich.PREC_FP32, ctx=ctx, dtracks=dt, photons=pb, trace_seed=wl.seed)
    np.testing.assert_array_equal(ext["fate"], fused["fate"])
    a = np.sort(fused["hits"], order=["event", "track", "photon"])
    b = np.sort(ext["hits"], order=["event", "track", "photon"])
    np.testing.assert_array_equal(a, b)
    ref = P.run_oracle(wl)
    np.testing.assert_array_equal(pb.t["lambda_"][: pb.n].cpu().numpy(), ref["lambda"])
    ctx.close()
