"""Pins of the oracle's gradient of the soft ring chi^2 (dual numbers along
the recorded surface sequence) against closed forms of the point-source
optics and against central finite differences of its own forward replay."""
import math

import numpy as np
import pytest

from paper_2309_12496_gb300 import workloads as W

ETA = float(np.float32(0.0014))


def _point(n=400):
    wl = W.point_source(n)
    return wl, W.nominal_theta(wl.scene, wl.n_minus_1)


def test_ring_radius_derivative_in_n_is_exact(oracle_lib):
    """Point source at the centre of curvature: r = (R/2) tan(theta) with
    tan(theta) = sqrt(n^2 - 1) (beta = 1), so dr/dn = (R/2) n / tan(theta)
    = 25,634 mm per unit n, exactly radial (Sec. 3 angle)."""
    wl, th = _point()
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    n = 1 + ETA
    expect = 1355.0 * n / math.sqrt(n * n - 1)
    assert expect == pytest.approx(25634.0, abs=1.0)
    seen = 0
    for j in range(200):
        fate, u, v, du, dv = sc.hit_jacobian(wl.tracks, prm, th, 0, j)
        if fate != 5:
            continue
        e = np.array([u - 368.64, v - 368.64])
        e /= np.linalg.norm(e)
        assert e @ [du[9], dv[9]] == pytest.approx(expect, rel=1e-9)
        assert abs(-e[1] * du[9] + e[0] * dv[9]) < 1e-6 * expect
        seen += 1
    assert seen > 5


def test_radius_and_tilt_derivatives_match_paraxial_optics(oracle_lib):
    """Paraxial optics of a spherical mirror (focal length R/2), the source
    a distance R0 from the pole and the plane R0/2 from it: the ring radius
    moves by dr/dR = tan(theta) when only R changes (image distance
    R0 R/(2 R0 - R)), and a tilt alpha of the mirror about its pole turns
    the reflected rays by 2 alpha, shifting the ring centre by R0 alpha on
    the plane. Non-paraxial corrections at theta = 53 mrad are ~0.1 %."""
    wl, th = _point()
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    tan_t = math.sqrt((1 + ETA) ** 2 - 1)
    for j in range(200):
        fate, u, v, du, dv = sc.hit_jacobian(wl.tracks, prm, th, 0, j)
        if fate != 5:
            continue
        e = np.array([u - 368.64, v - 368.64])
        e /= np.linalg.norm(e)
        assert e @ [du[8], dv[8]] == pytest.approx(tan_t, rel=5e-3)
        # tilt about e1 (x) moves the centre along y, about e2 (y) along x
        assert math.hypot(du[0], dv[0]) == pytest.approx(2710.0, rel=5e-3)
        assert abs(dv[0]) > 100 * abs(du[0])
        assert math.hypot(du[1], dv[1]) == pytest.approx(2710.0, rel=5e-3)
        assert abs(du[1]) > 100 * abs(dv[1])
        # tiles 1..3 do not exist in this scene
        assert np.all(du[2:8] == 0) and np.all(dv[2:8] == 0)
        break


@pytest.mark.parametrize("at_nominal", [True, False])
def test_dual_gradient_matches_finite_differences(oracle_lib, at_nominal):
    """On the RICH1-like analytic geometry (4 tiles, 2 flats, 3 planes), the
    dual-number gradient of the loss equals central differences of the same
    forced-topology replay (h = 1e-6 rad, 1e-6 relative) to 1e-6 relative,
    at the nominal parameters and at a tilted, rescaled point."""
    wl = W.adjoint_workload(n_tracks=16, photons_per_track=400, seed=3)
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    th0 = W.nominal_theta(wl.scene, wl.n_minus_1)
    nom = sc.trace(wl.tracks, prm)
    det = nom["fate"] == 5
    off = nom["offsets"].astype(np.int64)
    tix = np.repeat(np.arange(wl.tracks.n), np.diff(off))
    tg = W.ring_targets(wl.tracks.n, 3, tix[det], nom["plane"][det], nom["u"][det],
                        nom["v"][det])
    th = th0.copy()
    if not at_nominal:
        th[:8] = [2e-3, -1e-3, 0.5e-3, 1.5e-3, -2e-3, 1e-3, 0.0, -0.7e-3]
        th[8] *= 1.002
        th[9] *= 0.99
    loss, g, gfd, used = sc.grad(wl.tracks, prm, th, tg, sigma=1.0, fd=True)
    assert used > 500 and np.isfinite(loss)
    scale = np.abs(gfd).max()
    for k in range(10):
        assert g[k] == pytest.approx(gfd[k], rel=1e-6, abs=1e-9 * scale), (k, g, gfd)
    # every tile tilt reaches the loss at the tilted point
    if not at_nominal:
        assert np.all(np.abs(g[:8]) > 0)


def test_replay_reproduces_forward_hits(oracle_lib):
    """The value part of the dual replay along a photon's recorded surfaces
    equals the forward trace's hit, including photons of a fixed-count track
    below the Cherenkov threshold (they leave along the track)."""
    tr = W.pion_tracks(6, seed=2, n_fixed=300)
    tr.p[0] = 2.0                     # below the 2.64 GeV/c threshold
    wl = W.Workload("g", W.rich1_scene(meshed=False), tr, n_minus_1=0.0014)
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    th = W.nominal_theta(wl.scene, wl.n_minus_1)
    out = sc.trace(wl.tracks, prm)
    off = out["offsets"].astype(np.int64)
    checked = 0
    for g in np.nonzero(out["fate"] == 5)[0][::7]:
        t = int(np.searchsorted(off, g, side="right") - 1)
        fate, u, v, du, dv = sc.hit_jacobian(wl.tracks, prm, th, t, int(g - off[t]))
        assert fate == 5
        assert abs(u - out["u"][g]) < 1e-9 and abs(v - out["v"][g]) < 1e-9
        assert np.all(np.isfinite(du)) and np.all(np.isfinite(dv))
        checked += 1
    assert checked > 20
