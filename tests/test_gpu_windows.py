"""GPU parity of refraction at window faces (Snell's law with the binned
index of a quartz-like window; total internal reflection) against the FP64
oracle, photon by photon (marked gpu). The paper's simplified RICH geometry
removed the detector windows (Sec. 4.1); these cases put them back.

Bars as in test_gpu_parity.py."""
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
def test_rich1_windows_parity_full(meshed):
    """1000 pion tracks, quartz windows in front of both focal planes,
    refined hits."""
    wl = W.rich1_windows(1000, meshed=meshed)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name=f"rich1_windows_meshed{int(meshed)}")


def test_rich1_windows_fp32():
    wl = W.rich1_windows(300, meshed=True)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_FP32)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_FP32["rich1"], name="rich1_windows_fp32")


def test_slab_ring_closed_form_gpu():
    """Ring radius through a 30 mm slab, 970 tan(theta) + 30 tan(theta_r),
    per photon with the index bin of its wavelength, and parity."""
    wl = W.slab_ring(20000)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name="slab_ring")
    h = gpu["hits"]
    n = 1 + float(np.float32(0.33))
    sin_t = math.sqrt(1 - 1 / n**2)
    k = np.clip(np.floor((h["lambda"] - np.float32(200)) / np.float32(25)), 0, 15).astype(int)
    sin_r = sin_t / np.asarray(W.f32(W.QUARTZ_N), np.float64)[k]
    r_exp = 970.0 * sin_t / math.sqrt(1 - sin_t**2) + 30.0 * sin_r / np.sqrt(1 - sin_r**2)
    r = np.hypot(h["u"] - 1280.0, h["v"] - 1280.0)
    assert np.abs(r - r_exp).max() < 1e-4


def test_slab_total_internal_reflection_gpu():
    """Isotropic source inside a slab of index 1.5: fates (detected,
    trapped until the direction-change limit, escaped sideways) equal the
    oracle's; detected fraction 1 - cos(theta_c)."""
    wl = W.slab_tir(100000)
    ref = P.run_oracle(wl)
    gpu = P.run_gpu(wl, rich.PREC_REFINE64)
    P.compare(gpu, ref, wl.tracks, P.TOL_UV_REFINE, name="slab_tir")
    frac = 1 - math.sqrt(1 - 1 / 1.5**2)
    assert abs(gpu["n_hits"] / 1e5 - frac) < 4 * math.sqrt(frac * (1 - frac) / 1e5)
    assert gpu["stats"]["fate"][rich.FATE_NAMES.index("max_bounces")] > 50000


def test_gradient_rejects_refracting_scene():
    wl = W.rich1_windows(10, meshed=False)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    out = rich.TraceOutputs(1000)
    tg = torch.zeros(wl.tracks.n * len(wl.scene.planes) * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(rich.RichError):
        ctx.trace_grad(dt, W.nominal_theta(wl.scene, wl.n_minus_1), tg, out)
    ctx.close()
