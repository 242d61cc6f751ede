"""Pins of the oracle's entry point for photons given by the caller (the
photon emitter's vectors of positions and momenta, Sec. 4.2), no GPU.

  * Point source at the centre of curvature: whatever direction a photon
    leaves the centre in, the mirror sends it back through the centre, so a
    caller photon from the centre with direction d (FP32) is detected on
    the plane at R/2 at the point where the line through the centre along d
    crosses it: (u, v) = z_plane (dx, dy)/dz minus the plane's corner, to
    1e-9 mm.
  * Flat mirror (image method): a photon from o with direction d reflects
    off the plane z = 1000 as if it came from the image point (ox, oy,
    2000 - oz) with direction (dx, dy, -dz), which fixes its hit on the
    plane z = 500 in closed form.
  * Caller photons carrying the keys of emitted photons draw the same
    reflectivity and QE uniforms: their fates equal those of the emission
    path, photon by photon.
"""
import math

import numpy as np
import pytest

from paper_2309_12496_gb300 import workloads as w


def _point_source_photons(oracle_lib, wl, n):
    prm = oracle_lib.params(wl)
    o = np.zeros((n, 3), np.float32)
    d = np.empty((n, 3), np.float32)
    lam = np.empty(n, np.float32)
    for j in range(n):
        _, dj, lj = oracle_lib.emit(wl.tracks, prm, 0, j)
        d[j], lam[j] = dj, lj
    return prm, o, d, lam


def test_external_point_source_hits_the_line_through_the_centre(oracle_lib):
    wl = w.point_source(3000)
    sc = oracle_lib.Scene(wl.scene)
    prm, o, d, lam = _point_source_photons(oracle_lib, wl, 3000)
    z = np.zeros(3000, np.uint32)
    out = sc.trace_photons(o, d, lam, z, z, np.arange(3000, dtype=np.uint32), prm)
    det = out["fate"] == 5
    assert det.sum() > 300
    dd = d.astype(np.float64)
    org = wl.scene.rects[0]["origin"].astype(np.float64)    # FP32 corner
    z0 = float(org[2])
    np.testing.assert_allclose(out["u"][det], z0 * dd[det, 0] / dd[det, 2] - org[0],
                               rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["v"][det], z0 * dd[det, 1] / dd[det, 2] - org[1],
                               rtol=0, atol=1e-9)
    # same keys as the emission path: same fates photon by photon
    ref = sc.trace(wl.tracks, prm)
    np.testing.assert_array_equal(out["fate"], ref["fate"][:3000])
    np.testing.assert_array_equal(out["lambda"], ref["lambda"][:3000])


def test_external_photons_flat_mirror_image_method(oracle_lib):
    """Arbitrary origins, directions, wavelengths and keys in front of a
    flat mirror: each detected hit is where the image ray meets the plane;
    reflectivity and QE are 1, so every photon that reaches the mirror
    inside it is detected."""
    b = w._Builder("flat")
    t1 = b.table_const(1.0)
    m_mir = b.material(w.MAT_MIRROR, t1)
    m_det = b.material(w.MAT_DETECTOR, t1, plane=0)
    b.rect(np.array([400.0, -400.0, 1000.0]), np.array([-1.0, 0, 0]), np.array([0, 1.0, 0]),
           800.0, 800.0, m_mir)
    half = 128 * 2.88
    b.rect((-half, -half, 500.0), (1.0, 0, 0), (0, 1.0, 0), 256 * 2.88, 256 * 2.88,
           m_det, nx=256, ny=256, pitch=2.88)
    scene = b.build()
    sc = oracle_lib.Scene(scene)
    rng = np.random.default_rng(7)
    n = 4000
    o = np.column_stack([rng.uniform(-100, 100, (n, 2)), rng.uniform(520, 980, n)]).astype(np.float32)
    ct = rng.uniform(math.cos(0.2), 1.0, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    st = np.sqrt(1 - ct * ct)
    d = np.column_stack([st * np.cos(ph), st * np.sin(ph), ct]).astype(np.float32)
    lam = rng.uniform(200, 600, n).astype(np.float32)
    ev = rng.integers(0, 5, n).astype(np.uint32)
    tk = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    pk = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    prm = oracle_lib.params(None, seed=11, n_minus_1=0.0014, lambda_min=200.0,
                            lambda_max=600.0)
    out = sc.trace_photons(o, d, lam, ev, tk, pk, prm)
    oo, dd = o.astype(np.float64), d.astype(np.float64)
    # image ray: from (ox, oy, 2000 - oz) along (dx, dy, -dz) to z = 500
    t = (2000.0 - oo[:, 2] - 500.0) / dd[:, 2]
    x = oo[:, 0] + t * dd[:, 0]
    y = oo[:, 1] + t * dd[:, 1]
    tm = (1000.0 - oo[:, 2]) / dd[:, 2]
    on_mirror = (np.abs(oo[:, 0] + tm * dd[:, 0]) < 400) & (np.abs(oo[:, 1] + tm * dd[:, 1]) < 400)
    org = scene.rects[1]["origin"].astype(np.float64)      # FP32 corner
    on_plane = (np.abs(x) < half) & (np.abs(y) < half)
    det = out["fate"] == 5
    clear = on_mirror & on_plane & (out["graze"] == 0)
    assert clear.sum() > 3000
    assert np.all(det[clear])
    np.testing.assert_allclose(out["u"][clear], x[clear] - org[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["v"][clear], y[clear] - org[1], rtol=0, atol=1e-9)
    pitch = float(scene.rects[1]["pitch"])
    np.testing.assert_array_equal(out["ix"][clear], np.floor((x[clear] - org[0]) / pitch))
    # per-event pixel counts and sums follow the caller's event keys
    for e in range(5):
        sel = det & (ev == e)
        assert out["pixel_counts"][e].sum() == sel.sum()
        assert out["event_sums"][e, 0, 1] == pytest.approx(out["u"][sel].sum(), rel=1e-12)
