"""GPU adjoint (rich_trace_grad) against the oracle's dual-number gradient
of the soft ring chi^2, on the RICH1-like analytic geometry (marked gpu).

Both sides replay each detected photon along its recorded reflecting
surfaces; the GPU carries FP64 values and FP32 tangents, the oracle FP64
duals. Photons whose topology differs between the FP32 and FP64 traces
(grazes) enter one sum and not the other, which bounds the agreement of
the means at about (mismatches / hits used) of one term."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2309_12496_gb300 import build, rich  # noqa: E402
from paper_2309_12496_gb300 import workloads as W  # noqa: E402

REPORT = os.environ.get("RICH_PARITY_REPORT")
TILTED = [2e-3, -1e-3, 0.5e-3, 1.5e-3, -2e-3, 1e-3, 0.0, -0.7e-3]


def _report(name, stats):
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": name, **stats}) + "\n")


@pytest.fixture(scope="module")
def setup():
    build.build()
    oracle.build()
    wl = W.adjoint_workload(n_tracks=40, photons_per_track=2000, seed=5)
    sc = oracle.Scene(wl.scene)
    prm = oracle.params(wl)
    th0 = W.nominal_theta(wl.scene, wl.n_minus_1)
    nom = sc.trace(wl.tracks, prm)
    det = nom["fate"] == 5
    off = nom["offsets"].astype(np.int64)
    tix = np.repeat(np.arange(wl.tracks.n), np.diff(off))
    n_planes = len(wl.scene.planes)
    tg = W.ring_targets(wl.tracks.n, n_planes, tix[det], nom["plane"][det], nom["u"][det],
                        nom["v"][det])
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    tg_dev = torch.from_numpy(tg).cuda()
    n_ph = int(off[-1])
    out = rich.TraceOutputs(n_ph, wl.scene.pixels_per_event, n_planes, 1, n_ph)
    yield dict(wl=wl, sc=sc, prm=prm, th0=th0, tg=tg, ctx=ctx, dt=dt, tg_dev=tg_dev, out=out,
               n_planes=n_planes)
    ctx.close()


@pytest.mark.parametrize("point", ["nominal", "tilted"])
def test_adjoint_matches_oracle_gradient(setup, point):
    S = setup
    th = S["th0"].copy()
    if point == "tilted":
        th[:8] = TILTED
        th[8] *= 1.002
        th[9] *= 0.99
    th32 = np.float32(th).astype(np.float64)         # the GPU's FP32 parameters
    loss_g, grad_g, used_g = S["ctx"].trace_grad(S["dt"], th32, S["tg_dev"], S["out"],
                                                 sigma=1.0, seed=S["wl"].seed)
    loss_o, grad_o, _, used_o = S["sc"].grad(S["wl"].tracks, S["prm"], th32, S["tg"],
                                             sigma=1.0)
    scale = np.abs(grad_o).max()
    st = {"point": point, "used_gpu": used_g, "used_oracle": used_o, "loss_gpu": loss_g,
          "loss_oracle": loss_o, "max_grad_diff_rel_to_max": float(np.abs(grad_g - grad_o).max() / scale),
          "grad_gpu": grad_g.tolist(), "grad_oracle": grad_o.tolist()}
    _report(f"adjoint_{point}", st)
    assert abs(used_g - used_o) <= max(2, used_o // 2000)
    frac = (abs(used_g - used_o) + 1) / used_o
    assert loss_g == pytest.approx(loss_o, rel=5 * frac + 1e-6)
    assert np.abs(grad_g - grad_o).max() <= (2e-4 + 5 * frac) * scale, st


def test_forward_hits_at_theta_match_oracle(setup):
    """The forward pass of the gradient writes FP64 hit positions at theta:
    photon by photon they equal the oracle's trace at the same theta."""
    S = setup
    th = S["th0"].copy()
    th[:8] = TILTED
    th32 = np.float32(th).astype(np.float64)
    S["out"].clear()
    S["ctx"].trace_grad(S["dt"], th32, S["tg_dev"], S["out"], seed=S["wl"].seed)
    n_hits, _ = S["ctx"].hits()
    hits = S["out"].hits_numpy(n_hits)
    ref = S["sc"].trace_at(S["wl"].tracks, S["prm"], th32)
    off = ref["offsets"].astype(np.int64)
    g = off[hits["track"].astype(np.int64)] + hits["photon"].astype(np.int64)
    ok = (ref["fate"][g] == 5) & (ref["graze"][g] == 0)
    assert ok.mean() > 0.99
    du = np.abs(hits["u"][ok] - ref["u"][g[ok]])
    dv = np.abs(hits["v"][ok] - ref["v"][g[ok]])
    _report("adjoint_forward_hits", {"hits": int(ok.sum()), "max_du": float(du.max()),
                                     "max_dv": float(dv.max())})
    assert du.max() < 1e-4 and dv.max() < 1e-4


def test_autograd_function_and_descent(setup):
    """torch.autograd through the C ABI: backward gives rich_trace_grad's
    gradient; plain gradient steps on the tilts from a misaligned start
    lower the loss."""
    S = setup
    th = torch.tensor(S["th0"], dtype=torch.float64)
    th[:8] = torch.tensor(TILTED, dtype=torch.float64)
    th.requires_grad_(True)
    loss = rich.ring_chi2(S["ctx"], th, S["dt"], S["tg_dev"], S["out"], sigma=1.0,
                          seed=S["wl"].seed)
    loss.backward()
    _, grad, _ = S["ctx"].trace_grad(S["dt"], th.detach().numpy(), S["tg_dev"], S["out"],
                                     seed=S["wl"].seed)
    np.testing.assert_allclose(th.grad.numpy(), grad, rtol=1e-12, atol=0)
    losses = [float(loss)]
    x = th.detach().clone()
    for _ in range(4):
        x.requires_grad_(True)
        lo = rich.ring_chi2(S["ctx"], x, S["dt"], S["tg_dev"], S["out"], sigma=1.0,
                            seed=S["wl"].seed)
        lo.backward()
        with torch.no_grad():
            step = torch.zeros_like(x)
            step[:8] = x.grad[:8] / (x.grad[:8].norm() + 1e-30) * 4e-4
            x = (x - step).detach()
        losses.append(float(lo))
    _report("adjoint_descent", {"losses": losses})
    assert losses[-1] < losses[0]
