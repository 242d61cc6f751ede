"""GPU adjoint (rich_trace_grad) against the oracle's dual-number gradient
of the soft ring chi^2, on the RICH1-like analytic geometry (marked gpu).

Both sides replay each detected photon along its recorded reflecting
surfaces; the GPU carries double-word values (~48 bits) and FP32 tangents,
the oracle FP64 duals. Both must use the same detected photons; each
gradient component is then compared on its own (relative 1e-5, absolute
floor 1e-6 of the largest component)."""
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


def _tilted(th0):
    th = th0.copy()
    th[:8] = TILTED
    th[8] *= 1.002
    th[9] *= 0.99
    return th


def _check_gradient(loss_g, grad_g, used_g, loss_o, grad_o, used_o, name, point):
    """Per-component agreement of the GPU gradient with the oracle's: when
    both used the same detected photons, each component within a relative
    1e-5 of the oracle's (FP32 tangents over a few dozen chained operations:
    ~1e-6), with an absolute floor of 1e-6 of the largest component (a
    component that vanishes at the point), and the loss within 1e-9
    (double-word values, FP64 sums)."""
    scale = np.abs(grad_o).max()
    diff = np.abs(grad_g - grad_o)
    bound = 1e-5 * np.abs(grad_o) + 1e-6 * scale
    st = {"point": point, "used_gpu": used_g, "used_oracle": used_o, "loss_gpu": loss_g,
          "loss_oracle": loss_o, "loss_rel": abs(loss_g - loss_o) / abs(loss_o),
          "max_rel_component": float((diff / np.maximum(np.abs(grad_o), 1e-300)).max()),
          "max_diff_over_bound": float((diff / bound).max()),
          "grad_gpu": grad_g.tolist(), "grad_oracle": grad_o.tolist()}
    _report(name, st)
    assert used_g == used_o, st
    assert st["loss_rel"] <= 1e-9, st
    assert np.all(diff <= bound), st
    return st


@pytest.mark.parametrize("point", ["nominal", "tilted"])
def test_adjoint_matches_oracle_gradient(setup, point):
    S = setup
    th = S["th0"].copy() if point == "nominal" else _tilted(S["th0"])
    th32 = np.float32(th).astype(np.float64)         # the GPU's FP32 parameters
    loss_g, grad_g, used_g = S["ctx"].trace_grad(S["dt"], th32, S["tg_dev"], S["out"],
                                                 sigma=1.0, seed=S["wl"].seed)
    loss_o, grad_o, _, used_o = S["sc"].grad(S["wl"].tracks, S["prm"], th32, S["tg"],
                                             sigma=1.0)
    _check_gradient(loss_g, grad_g, used_g, loss_o, grad_o, used_o, f"adjoint_{point}", point)


def test_adjoint_full_size_matches_oracle_gradient():
    """The adjoint workload at its full size (200 tracks x 5000 photons,
    10^6 photons), at a tilted point, through the same call the benchmark
    times: every gradient component against the oracle's."""
    wl = W.adjoint_workload()
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
    th32 = np.float32(_tilted(th0)).astype(np.float64)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n_ph = int(off[-1])
    assert n_ph == 1_000_000
    out = rich.TraceOutputs(n_ph, wl.scene.pixels_per_event, n_planes, 1, 0)
    loss_g, grad_g, used_g = ctx.trace_grad(dt, th32, torch.from_numpy(tg).cuda(), out,
                                            sigma=1.0, seed=wl.seed)
    ctx.close()
    loss_o, grad_o, _, used_o = sc.grad(wl.tracks, prm, th32, tg, sigma=1.0)
    st = _check_gradient(loss_g, grad_g, used_g, loss_o, grad_o, used_o, "adjoint_full_c4",
                         "tilted")
    assert st["used_gpu"] > 100_000


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


def test_adjoint_two_tilted_tiles_per_path():
    """Every detected photon of the periscope scene reflects off two tilted
    tiles, so each hit takes a second replay for the second tile's tilts:
    the four tilt components of both tiles, R and n - 1 against the oracle."""
    wl = W.two_mirror(20_000)
    sc = oracle.Scene(wl.scene)
    prm = oracle.params(wl)
    nom = sc.trace(wl.tracks, prm)
    det = nom["fate"] == 5
    assert det.sum() > 1000 and np.all(nom["n_refl"][det] == 2)
    tg = W.ring_targets(1, 1, np.zeros(int(det.sum()), np.int64), nom["plane"][det],
                        nom["u"][det], nom["v"][det])
    th = W.nominal_theta(wl.scene, wl.n_minus_1)
    th[:4] = [2e-3, -1e-3, 1.5e-3, 0.5e-3]
    th32 = np.float32(th).astype(np.float64)
    ctx = rich.Context(0)
    ctx.init_geometry(wl.scene)
    dt = rich.DeviceTracks(wl.tracks)
    n = int(nom["offsets"][-1])
    out = rich.TraceOutputs(n, wl.scene.pixels_per_event, 1, 1, n)
    loss_g, grad_g, used_g = ctx.trace_grad(dt, th32, torch.from_numpy(tg).cuda(), out,
                                            sigma=1.0, seed=wl.seed)
    ctx.close()
    loss_o, grad_o, _, used_o = sc.grad(wl.tracks, prm, th32, tg, sigma=1.0)
    assert np.all(np.abs(grad_o[:4]) > 1e2) and np.all(grad_o[4:8] == 0.0)
    _check_gradient(loss_g, grad_g, used_g, loss_o, grad_o, used_o, "adjoint_two_tiles",
                    "tilted")
