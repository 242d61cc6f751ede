"""Pins of the FP64 oracle against things other than itself.

Each test checks an oracle function against a library routine, a closed
form, a textbook constant, an invariant, a statistical law or brute force,
chosen so that a plausible slip (a wrong multiplier or sign, a dropped term,
a swapped index, an off-by-one bin) fails at least one of them. None of
these tests needs a GPU.
"""
import json
import math
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_2309_12496_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")
PAPER = json.load(open(GOLDEN))
ETA_C4F10 = float(np.float32(0.0014))   # n - 1 as the FP32 input holds it
ETA_CF4 = float(np.float32(0.0005))


# ------------------------------------------------------------------ Philox
_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(c_ptr, o_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(o_ptr + 4 * i + 0, a)
    tl.store(o_ptr + 4 * i + 1, b)
    tl.store(o_ptr + 4 * i + 2, c)
    tl.store(o_ptr + 4 * i + 3, d)
z = np.load(sys.argv[1])
ctr = torch.from_numpy(z["ctr"].view(np.int32).copy())
out = torch.zeros_like(ctr)
k[(1,)](ctr, out, int(z["seed"]), N=ctr.numel() // 4)
np.save(sys.argv[2], out.numpy().view(np.uint32))
"""


def test_philox_matches_triton_library(oracle_lib):
    """Philox4x32-10 of the oracle equals Triton's tl.philox (a library
    implementation, run by Triton's CPU interpreter) on random counters and
    a 64-bit seed split into (lo, hi) key words."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = [0xFFFFFFFF] * 4
    seed = 0x0123456789ABCDEF
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "in.npz")
        dst = os.path.join(d, "out.npy")
        np.savez(src, ctr=ctr, seed=np.uint64(seed))
        env = dict(os.environ, TRITON_INTERPRET="1")
        r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, src, dst],
                           env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
        ref = np.load(dst).reshape(-1, 4)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    got = oracle_lib.philox(ctr, key)
    np.testing.assert_array_equal(got, ref)


def test_philox_bijective_and_uniform(oracle_lib):
    """Distinct counters give distinct outputs; words are uniform (chi^2 on
    256 bins) and uncorrelated across the 4 lanes."""
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = 12345
    out = oracle_lib.philox(ctr, np.array([0, 0], np.uint32))
    packed = out.view(np.uint64).reshape(n, 2)
    assert len(np.unique(packed[:, 0] ^ (packed[:, 1] << np.uint64(1)))) == n
    from scipy import stats
    for lane in range(4):
        hist = np.bincount(out[:, lane] >> 24, minlength=256)
        assert stats.chisquare(hist).pvalue > 1e-4
    c = np.corrcoef(out.astype(np.float64).T)
    assert np.abs(c - np.eye(4)).max() < 0.02


# ------------------------------------------------------------- Frank-Tamm
def test_yield_matches_pdg_constant(oracle_lib):
    """Frank-Tamm: d2N/dx dE = (alpha / hbar c) z^2 sin^2(theta), with
    alpha/(hbar c) = 369.81 eV^-1 cm^-1 (PDG review of passage of particles
    through matter) and hc = 1239.84 eV nm. For beta = 1 in C4F10 and CF4
    this gives 0.4270 and 0.1527 photons/mm over 200-600 nm."""
    def pdg(eta, beta):
        nb = (1 + eta) * beta
        s2 = 1 - 1 / nb**2 if nb > 1 else 0.0
        de = 1239.84193 / 200.0 - 1239.84193 / 600.0
        return 369.81 * s2 * de / 10.0
    for eta in (ETA_C4F10, ETA_CF4, 0.33):
        got = oracle_lib.yield_per_mm(eta, 1.0)
        assert got == pytest.approx(pdg(eta, 1.0), rel=2e-4)
    assert oracle_lib.yield_per_mm(ETA_C4F10, 1.0) == pytest.approx(0.42704, abs=1e-5)
    assert oracle_lib.yield_per_mm(ETA_CF4, 1.0) == pytest.approx(0.15272, abs=1e-5)


def test_yield_threshold(oracle_lib):
    """No light below threshold beta = 1/n: for a pion in C4F10 the
    threshold momentum is m / sqrt(n^2 - 1) = 2.637 GeV/c."""
    m = w.PION_MASS
    n = 1 + ETA_C4F10
    p_thr = m / math.sqrt(n * n - 1)
    assert p_thr == pytest.approx(2.637, abs=1e-3)
    beta = lambda p: p / math.sqrt(p * p + m * m)
    assert oracle_lib.yield_per_mm(ETA_C4F10, beta(p_thr * 0.999)) == 0.0
    assert oracle_lib.yield_per_mm(ETA_C4F10, beta(p_thr * 1.01)) > 0.0


def test_mean_photons_per_track_rich1_spectrum(oracle_lib):
    """Mean Frank-Tamm mean over the log-uniform 2-100 GeV/c pion spectrum,
    by quadrature of the closed form, equals the oracle's per-track means
    averaged over many tracks (to statistical precision)."""
    from scipy import integrate
    m, n, L = w.PION_MASS, 1 + ETA_C4F10, 1000.0
    k = 369.81 * (1239.84193 / 200 - 1239.84193 / 600) / 10.0

    def mu(lnp):
        p = math.exp(lnp)
        b = p / math.sqrt(p * p + m * m)
        s2 = max(0.0, 1 - 1 / (n * b) ** 2)
        return L * k * s2
    a, b = math.log(2.0), math.log(100.0)
    expect = integrate.quad(mu, a, b, points=[math.log(2.637)])[0] / (b - a)
    assert expect == pytest.approx(342.3, abs=0.5)
    tr = w.pion_tracks(20000, seed=3)
    wl = w.Workload("t", None, tr, n_minus_1=0.0014)
    nph, mus, off = oracle_lib.track_yield(tr, oracle_lib.params(wl))
    assert mus.mean() == pytest.approx(expect, rel=0.02)
    # Poisson counts: mean matches the means, variance ~ mean + var(mu)
    assert nph.mean() == pytest.approx(mus.mean(), rel=0.01)
    assert int(off[-1]) == int(nph.sum())


@pytest.mark.parametrize("mu", [0.7, 3.0, 9.5, 10.0, 42.0, 341.0])
def test_poisson_sampler_distribution(oracle_lib, mu):
    """The keyed Poisson draw (inversion below 10, PTRS above) follows the
    Poisson law: chi^2 against scipy's pmf over 20,000 independent keys."""
    from scipy import stats
    ks = np.array([oracle_lib.poisson(mu, seed=11, event=1, track=t)
                   for t in range(20000)])
    assert ks.mean() == pytest.approx(mu, abs=4 * math.sqrt(mu / 20000))
    lo, hi = int(max(0, mu - 4 * math.sqrt(mu) - 2)), int(mu + 4 * math.sqrt(mu) + 3)
    edges = np.arange(lo, hi + 1)
    obs = np.array([(ks == k).sum() for k in edges[:-1]] + [(ks >= edges[-1]).sum()])
    obs[0] += (ks < lo).sum()
    pmf = stats.poisson.pmf(edges[:-1], mu)
    exp = np.concatenate([pmf, [stats.poisson.sf(edges[-1] - 1, mu)]])
    exp[0] += stats.poisson.cdf(lo - 1, mu)
    exp = exp * len(ks)
    keep = exp > 5
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4


# --------------------------------------------------------------- emission
def test_emission_angle_is_cherenkov(oracle_lib):
    """Sec. 3: photons leave at cos(theta) = 1/(n beta) to the track,
    independent of azimuth; directions are unit vectors; the origin lies on
    the track segment [0, L)."""
    tr = w.pion_tracks(50, seed=5)
    wl = w.Workload("t", None, tr, n_minus_1=0.0014)
    prm = oracle_lib.params(wl)
    m = w.PION_MASS
    for i in range(0, 50, 7):
        p = float(tr.p[i])
        beta = p / math.sqrt(p * p + float(np.float32(m)) ** 2)
        if (1 + ETA_C4F10) * beta <= 1:
            continue
        t = np.array([tr.dx[i], tr.dy[i], tr.dz[i]], np.float64)
        t /= np.linalg.norm(t)
        for j in range(20):
            o, d, lam = oracle_lib.emit(tr, prm, i, j)
            assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-14)
            assert np.dot(d, t) == pytest.approx(1 / ((1 + ETA_C4F10) * beta), abs=1e-13)
            s = np.dot(o, t)
            assert 0.0 <= s < float(tr.length[i])
            assert np.linalg.norm(o - s * t) < 1e-9
            assert 200.0 <= lam <= 600.0


def test_emission_azimuth_and_wavelength_laws(oracle_lib):
    """Azimuth uniform on [0, 2 pi) (measured in a frame built here, not the
    oracle's); wavelength follows the Frank-Tamm spectrum dN/dl ~ 1/l^2 on
    [200, 600] nm, whose CDF is (1/200 - 1/l)/(1/200 - 1/600) (KS tests)."""
    from scipy import stats
    wl = w.point_source(4000)
    prm = oracle_lib.params(wl)
    phis, lams = [], []
    for j in range(4000):
        _, d, lam = oracle_lib.emit(wl.tracks, prm, 0, j)
        phis.append(math.atan2(d[1], d[0]) % (2 * math.pi))
        lams.append(lam)
    assert stats.kstest(np.array(phis) / (2 * math.pi), "uniform").pvalue > 1e-3
    cdf = lambda l: (1 / 200.0 - 1 / l) / (1 / 200.0 - 1 / 600.0)
    assert stats.kstest(np.array(lams, np.float64), cdf).pvalue > 1e-3


# ----------------------------------------------------------------- tables
def test_tables_follow_paper_binning(oracle_lib):
    """Sec. 4.3: QE histogram in 33 nm bins with its 35% peak in the bin
    containing 450 nm; reflectivity in 25 nm bins from 94% to 89% over
    200-600 nm. The oracle's lookup returns the bin holding lambda, clamped
    at the ends."""
    sc = oracle_lib.Scene(w.rich1_scene(meshed=False))
    tab = w.rich1_scene(meshed=False).tables
    assert tab[0]["p1"] == PAPER["qe_bin_width_nm"]["value"]
    assert tab[1]["p1"] == PAPER["reflectivity_bin_width_nm"]["value"]
    qe_peak = PAPER["qe_peak"]
    assert sc.table(0, qe_peak["lambda_nm"]) == pytest.approx(qe_peak["value"], abs=1e-6)
    assert max(sc.table(0, l) for l in np.arange(200, 1000, 1.0)) == pytest.approx(0.35, abs=1e-6)
    r = PAPER["reflectivity_range"]
    assert sc.table(1, 200.5) == pytest.approx(r["high"], abs=1e-6)
    assert sc.table(1, 599.5) == pytest.approx(r["low"], abs=0.0015)
    # bin edges: [200 + 25 k, 200 + 25 (k + 1)) and clamping
    vals = tab[1]["values"]
    for k in range(16):
        assert sc.table(1, 200.0 + 25 * k) == vals[k]
        assert sc.table(1, np.nextafter(np.float32(225.0 + 25 * k), np.float32(0))) == vals[k]
    assert sc.table(1, 150.0) == vals[0]
    assert sc.table(1, 700.0) == vals[15]
    # analytic Gaussian QE of the point-source scene, evaluated in FP32
    sp = oracle_lib.Scene(w.point_source_scene())
    for lam in (250.0, 400.0, 537.5):
        x = np.float32(np.float32(lam) - np.float32(400)) / np.float32(120)
        ref = np.float32(0.3) * np.exp(-np.float32(x * x), dtype=np.float32)
        assert sp.table(0, lam) == pytest.approx(float(ref), rel=3e-7)
    assert sp.table(1, 431.0) == pytest.approx(0.9, rel=1e-7)


# ------------------------------------------------- closed-form geometries
def _ring_radii(out, rect):
    det = out["fate"] == 5
    half_u = -float(np.dot(rect["origin"], rect["u_axis"]))
    half_v = -float(np.dot(rect["origin"], rect["v_axis"]))
    return det, np.hypot(out["u"][det] - half_u, out["v"][det] - half_v)


def test_point_source_ring_radius(oracle_lib):
    """Source at the mirror's centre of curvature: every reflected photon
    returns through the centre, so every hit on the plane at R/2 lies at
    radius (R/2) tan(theta) = 71.72495 mm with tan(theta) = sqrt(n^2 - 1)
    for beta = 1 (Sec. 3 angle; the ring radius measures the Cherenkov
    angle as in Sec. 6)."""
    wl = w.point_source(20000)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl))
    det, rad = _ring_radii(out, wl.scene.rects[0])
    n = 1 + ETA_C4F10
    expect = 1355.0 * math.sqrt(n * n - 1)
    assert expect == pytest.approx(71.72495, abs=2e-5)
    assert det.sum() > 1000
    assert np.abs(rad - expect).max() < 1e-9
    # every photon reaches the mirror: fates are only mirror-absorbed,
    # QE-rejected or detected
    assert set(np.unique(out["fate"])) <= {2, 4, 5}


def test_muon_point_source_ring_radius(oracle_lib):
    """One 100 GeV/c muon (m = 105.66 MeV) at the centre of curvature:
    beta = p / sqrt(p^2 + m^2) = 0.99999944 from the FP32 momentum and mass,
    cos(theta) = 1/(n beta) (Sec. 3), and every hit at (R/2) tan(theta)
    = 71.71062 mm, 0.0143 mm inside the beta = 1 ring: a dropped mass or a
    beta squared in the wrong place moves the ring by far more than the
    bound."""
    wl = w.point_source_muon(20000)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl))
    det, rad = _ring_radii(out, wl.scene.rects[0])
    p, m = float(wl.tracks.p[0]), float(wl.tracks.mass[0])
    nb = (1 + ETA_C4F10) * p / math.sqrt(p * p + m * m)
    expect = 1355.0 * math.sqrt(nb * nb - 1)
    assert expect == pytest.approx(71.71062, abs=2e-5)
    assert 1355.0 * math.sqrt((1 + ETA_C4F10) ** 2 - 1) - expect > 0.01
    assert det.sum() > 1000
    assert np.abs(rad - expect).max() < 1e-9


def test_point_source_expected_counts(oracle_lib):
    """Detected fraction = R * <QE> with <QE> the spectrum-weighted mean of
    0.3 exp(-((l - 400)/120)^2) under dN/dl ~ 1/l^2 on [200, 600] nm
    (quadrature: 0.13435); 10^5 photons give 12,092 +- 103 hits (binomial),
    and the reflectivity draw rejects 10% of photons."""
    from scipy import integrate
    num = integrate.quad(lambda l: 0.3 * math.exp(-((l - 400) / 120) ** 2) / l**2, 200, 600)[0]
    den = integrate.quad(lambda l: 1 / l**2, 200, 600)[0]
    qe = num / den
    assert qe == pytest.approx(0.13435, abs=1e-5)
    wl = w.point_source(100000)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl))
    n_det = int((out["fate"] == 5).sum())
    p = 0.9 * qe
    assert abs(n_det - 1e5 * p) < 4 * math.sqrt(1e5 * p * (1 - p))
    n_abs = int((out["fate"] == 2).sum())
    assert abs(n_abs - 1e4) < 4 * math.sqrt(1e5 * 0.09)
    # azimuth of hits uniform around the ring centre
    from scipy import stats
    det = out["fate"] == 5
    ang = np.arctan2(out["v"][det] - 368.64, out["u"][det] - 368.64)
    assert stats.kstest((ang + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3
    # histogram and per-event sums agree with the hit list
    assert out["pixel_counts"].sum() == n_det
    es = out["event_sums"][0, 0]
    assert es[0] == n_det
    assert es[1] == pytest.approx(out["u"][det].sum(), rel=1e-12)
    assert es[3] == pytest.approx(out["lambda"][det].astype(np.float64).sum(), rel=1e-12)


def _flat_mirror_scene(meshed, n_cells=1):
    """Point source at the origin, flat mirror at z = 1000 facing the source,
    detector plane at z = 500 facing +z (the mirror)."""
    b = w._Builder("flat")
    t1 = b.table_const(1.0)
    m_mir = b.material(w.MAT_MIRROR, t1)
    m_det = b.material(w.MAT_DETECTOR, t1, plane=0)
    side = 800.0
    origin = np.array([side / 2, -side / 2, 1000.0])
    u_ax, v_ax = np.array([-1.0, 0, 0]), np.array([0, 1.0, 0])
    if meshed:
        b.triangles(w._mesh_rectangle(origin, u_ax, v_ax, side, side, n_cells, n_cells),
                    None, m_mir, smooth=False)
    else:
        b.rect(origin, u_ax, v_ax, side, side, m_mir)
    half = 128 * 2.88
    b.rect((-half, -half, 500.0), (1.0, 0, 0), (0, 1.0, 0), 256 * 2.88, 256 * 2.88,
           m_det, nx=256, ny=256, pitch=2.88)
    return b.build()


@pytest.mark.parametrize("meshed,cells", [(False, 1), (True, 1), (True, 7)])
def test_flat_mirror_image_method(oracle_lib, meshed, cells):
    """Law of reflection via the image method: a flat mirror at z = 1000
    images the source at z = 2000, so the reflected cone reaches the plane
    z = 500 at radius 1500 tan(theta). Checks rectangle and triangle
    intersection (through the BVH and by brute force) and the reflection."""
    sc_ = _flat_mirror_scene(meshed, cells)
    tr = w.point_source_tracks(3000)
    wl = w.Workload("flat", sc_, tr, n_minus_1=0.0014)
    sc = oracle_lib.Scene(sc_, leaf_size=2)
    n = 1 + ETA_C4F10
    expect = 1500.0 * math.sqrt(n * n - 1)
    for bvh in (True, False):
        out = sc.trace(tr, oracle_lib.params(wl, use_bvh=bvh))
        det, rad = _ring_radii(out, sc_.rects[-1])
        assert det.sum() == 3000      # QE = R = 1
        assert np.abs(rad - expect).max() < 1e-9


def test_sphere_intersection_closed_forms(oracle_lib):
    """Ray from the centre of a sphere: t = R. Ray along the axis from
    outside, at distance D from the centre: the concave (far) side at
    t = D + R is hit only when the near point is off the tile; the convex
    back at t = D - R is hit when it is on the tile."""
    b = w._Builder("sph")
    t1 = b.table_const(1.0)
    m = b.material(w.MAT_MIRROR, t1)
    b.sphere((0.0, 0.0, 0.0), 1000.0, (0.0, 0.0, 1.0), (1.0, 0, 0), (0, 1.0, 0), m,
             cos_min=0.5)
    sc = oracle_lib.Scene(b.build())
    rng = np.random.default_rng(0)
    d = rng.normal(size=(200, 3))
    d[:, 2] = np.abs(d[:, 2]) + 2.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d[d[:, 2] > 0.55]          # inside the 60-degree cap
    t, prim = sc.raycast(np.zeros((len(d), 3)), d)
    assert len(d) > 150 and np.all(prim == 0)
    np.testing.assert_allclose(t, 1000.0, rtol=0, atol=1e-9)
    # from below (outside), aiming +z: near intersection z = -1000 is off the
    # cap (w.axis = -1), far one z = +1000 is on it
    t, prim = sc.raycast([[0.0, 0.0, -3000.0]], [[0.0, 0.0, 1.0]])
    assert prim[0] == 0 and t[0] == pytest.approx(4000.0, abs=1e-9)
    # from above (outside), aiming -z: the convex back at z = +1000
    t, prim = sc.raycast([[0.0, 0.0, 3000.0]], [[0.0, 0.0, -1.0]])
    assert prim[0] == 0 and t[0] == pytest.approx(2000.0, abs=1e-9)
    # tangent-missing ray
    t, prim = sc.raycast([[1000.5, 0.0, -3000.0]], [[0.0, 0.0, 1.0]])
    assert prim[0] == -1


def test_triangle_intersection_closed_form(oracle_lib):
    """Ray through a known barycentric point of a triangle hits at the
    distance to that point; rays outside its edges miss."""
    b = w._Builder("tri")
    t1 = b.table_const(1.0)
    m = b.material(w.MAT_ABSORBER, t1)
    V = np.array([[[0.0, 0.0, 100.0], [50.0, 0.0, 110.0], [0.0, 40.0, 95.0]]])
    b.triangles(V, None, m, smooth=False)
    sc = oracle_lib.Scene(b.build())
    rng = np.random.default_rng(1)
    for _ in range(50):
        b1, b2 = rng.random(2) * 0.5
        p = V[0, 0] + b1 * (V[0, 1] - V[0, 0]) + b2 * (V[0, 2] - V[0, 0])
        o = rng.normal(size=3) * 30.0
        d = (p - o) / np.linalg.norm(p - o)
        t, prim = sc.raycast([o], [d])
        assert prim[0] == 0
        assert t[0] == pytest.approx(np.linalg.norm(p - o), abs=1e-9)
        q = V[0, 0] + 1.05 * (V[0, 1] - V[0, 0]) + 0.2 * (V[0, 2] - V[0, 0])
        t, prim = sc.raycast([o], [(q - o) / np.linalg.norm(q - o)])
        assert prim[0] == -1


def test_bvh_matches_brute_force(oracle_lib):
    """The oracle's median-split BVH returns exactly the brute-force nearest
    hit (distance and primitive) for random rays on a ~1000-triangle patch
    of the RICH1 mesh and on the full mesh."""
    full = w.rich1_scene(meshed=True)
    for n_tri in (1000, full.n_triangles):
        sub = w.Scene("sub", full.tables, full.materials, full.spheres[:0],
                      full.rects[:0], full.tri_vertices[:n_tri],
                      full.tri_normals[:n_tri], full.tri_material[:n_tri])
        sc = oracle_lib.Scene(sub, leaf_size=3)
        rng = np.random.default_rng(2)
        n = 3000 if n_tri == 1000 else 1500
        o = rng.normal(size=(n, 3)) * 100.0
        tgt = sub.tri_vertices[rng.integers(0, n_tri, n)].mean(axis=1)
        tgt = tgt + rng.normal(size=(n, 3)) * 8.0
        d = tgt - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        t1, p1 = sc.raycast(o, d, use_bvh=True)
        t2, p2 = sc.raycast(o, d, use_bvh=False)
        np.testing.assert_array_equal(p1, p2)
        np.testing.assert_array_equal(t1, t2)
        assert (p1 >= 0).mean() > 0.3


def test_results_invariant_to_sharding(oracle_lib):
    """Keyed random numbers: tracing a sub-range of tracks reproduces the
    same per-photon results as the full run."""
    wl = w.rich1(60, meshed=False)
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    full = sc.trace(wl.tracks, prm)
    off = full["offsets"]
    part = sc.trace(wl.tracks, prm, offsets=off, track_range=(20, 45))
    a, b = int(off[20]), int(off[45])
    for k in ("fate", "plane", "ix", "iy", "u", "v", "lambda", "n_refl"):
        np.testing.assert_array_equal(part[k][a:b], full[k][a:b])
    assert np.all(part["fate"][:a] == 0)


def test_rich1_bookkeeping(oracle_lib):
    """Fates partition the photons; pixel counts and per-event sums agree
    with the hit list; hits lie inside their pixel; grazes are rare."""
    wl = w.rich1(100, meshed=True)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl))
    f = out["fate"]
    assert np.all((f >= 1) & (f <= 7))
    det = f == 5
    assert out["pixel_counts"].sum() == det.sum()
    assert out["event_sums"][0, :, 0].sum() == det.sum()
    pitch = 2.88
    u, v = out["u"][det], out["v"][det]
    ix, iy = out["ix"][det], out["iy"][det]
    assert np.all(ix * np.float64(np.float32(pitch)) <= u + 1e-12)
    assert np.all(u < (ix + 1) * np.float64(np.float32(pitch)) + 1e-12)
    assert np.all((iy >= 0) & (iy < 256))
    assert (out["graze"] != 0).mean() < 0.01
    # planes 0/1 collect light after two reflections mostly
    assert (out["n_refl"][det & (out["plane"] < 2)] == 2).mean() > 0.8


# ------------------------------- efficiencies before propagation (Sec. 4.3)
def test_prefilter_point_source_counts_and_ring(oracle_lib):
    """The three efficiencies applied as one accept/reject before
    propagation (Sec. 4.3). On the point-source scene every photon reaches
    the mirror and returns to the plane, so with the prefilter on (QE table
    x reflectivity table) every accepted photon is detected and nothing
    else is: fates are only 'detected' or 'prefiltered'. The count follows
    the same closed form as in flight, 1e5 x 0.9 x <QE> = 12,092 +- 103,
    and every hit lies on the ring of radius (R/2) tan(theta)."""
    assert PAPER["efficiencies_before_propagation"]["count"] == 3
    wl = w.point_source(100000)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl, prefilter=(0, 1)))
    f = out["fate"]
    assert set(np.unique(f)) <= {oracle_lib.FATE_DETECTED, oracle_lib.FATE_PREFILTERED}
    n_det = int((f == oracle_lib.FATE_DETECTED).sum())
    p = 0.9 * 0.13435
    assert abs(n_det - 1e5 * p) < 4 * math.sqrt(1e5 * p * (1 - p))
    det, rad = _ring_radii(out, wl.scene.rects[0])
    n = 1 + ETA_C4F10
    assert np.abs(rad - 1355.0 * math.sqrt(n * n - 1)).max() < 1e-9
    assert out["pixel_counts"].sum() == n_det
    # rejected photons are not propagated: no reflections recorded
    assert np.all(out["n_refl"][f == oracle_lib.FATE_PREFILTERED] == 0)


def test_prefilter_uses_the_qe_draw_and_switches_in_flight_tests_off(oracle_lib):
    """With the QE table alone as the prefilter, the accept decision is the
    in-flight QE decision (the same draw and table), and mirrors then
    always reflect. So a photon detected in flight is detected with the
    prefilter; a photon detected only with the prefilter failed the
    in-flight reflectivity test; a constant-one prefilter detects every
    photon."""
    wl = w.point_source(30000)
    sc = oracle_lib.Scene(wl.scene)
    fly = sc.trace(wl.tracks, oracle_lib.params(wl))["fate"]
    pre = sc.trace(wl.tracks, oracle_lib.params(wl, prefilter=(0,)))["fate"]
    D = oracle_lib.FATE_DETECTED
    assert np.all(pre[fly == D] == D)
    only = (pre == D) & (fly != D)
    assert only.sum() > 0
    assert np.all(fly[only] == 2)          # mirror-absorbed in flight
    assert np.all(pre[fly == 4] == oracle_lib.FATE_PREFILTERED)   # QE-rejected
    # a scene whose first table is the constant 1 passes every photon
    ones = wl.scene.tables.copy()
    ones[1]["p0"] = 1.0
    sc1 = oracle_lib.Scene(w.Scene(**{**wl.scene.__dict__, "tables": ones}))
    all_det = sc1.trace(wl.tracks, oracle_lib.params(wl, prefilter=(1,)))["fate"]
    assert np.all(all_det == D)


def test_prefilter_matches_in_flight_statistics_rich1(oracle_lib):
    """RICH1-like scene: photons that meet the spherical mirror, the flat
    mirror and the detector have the same detection probability
    QE x R_a x R_b whether the efficiencies are applied before propagation
    or in flight, so the detected counts on the two focal planes agree
    within statistics, and no photon is mirror-absorbed or QE-rejected
    with the prefilter."""
    wl = w.rich1(200, meshed=False)
    sc = oracle_lib.Scene(wl.scene)
    fly = sc.trace(wl.tracks, oracle_lib.params(wl))
    pre = sc.trace(wl.tracks, oracle_lib.params(wl, prefilter=(0, 1, 2)))
    assert not np.isin(pre["fate"], (2, 4)).any()
    sel = lambda o: int(((o["fate"] == 5) & (o["plane"] < 2) & (o["n_refl"] == 2)).sum())
    a, b = sel(fly), sel(pre)
    assert a > 5000
    assert abs(a - b) < 4 * math.sqrt(a + b)


# ----------------------------------------------- other light sources (Sec. 6)
def _all_detector_box(half=500.0, n_pix=64, qe=1.0):
    """Cube of six inward-facing detector planes with a constant QE."""
    b = w._Builder("detector_box")
    t = b.table_const(qe)
    mats = [b.material(w.MAT_DETECTOR, t, plane=i) for i in range(6)]
    w._box_walls(b, half, lambda k: mats[k], n_pix)
    return b.build()


def test_isotropic_emission_laws(oracle_lib):
    """Isotropic (scintillation) emission: unit directions with cos(theta)
    uniform on [-1, 1] and uniform azimuth; origins on the segment; the
    wavelength follows the binned spectrum (bin frequencies by chi^2 against
    the CDF differences, uniform inside each bin)."""
    from scipy import stats
    wl = w.scintillation(20)
    prm = oracle_lib.params(wl)
    n, mu, off = oracle_lib.track_yield(wl.tracks, prm)
    tab = wl.scene.tables[wl.spectrum_table]
    cdf = tab["values"][: tab["nbins"] + 1].astype(np.float64)
    dirs, lams, s_rel = [], [], []
    for i in range(4):
        t0 = np.array([wl.tracks.x[i], wl.tracks.y[i], wl.tracks.z[i]], np.float64)
        td = np.array([wl.tracks.dx[i], wl.tracks.dy[i], wl.tracks.dz[i]], np.float64)
        td /= np.linalg.norm(td)
        for j in range(int(n[i])):
            o, d, lam = oracle_lib.emit(wl.tracks, prm, i, j)
            dirs.append(d)
            lams.append(lam)
            r = o - t0
            s = float(np.dot(r, td))
            assert np.linalg.norm(r - s * td) < 1e-9
            s_rel.append(s / float(wl.tracks.length[i]))
    d = np.array(dirs)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-14
    assert stats.kstest((d[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest((phi + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3
    assert stats.kstest(np.array(s_rel), "uniform").pvalue > 1e-3
    lam = np.array(lams, np.float64)
    k = np.floor((lam - tab["p0"]) / tab["p1"]).astype(int)
    counts = np.bincount(k, minlength=tab["nbins"])[: tab["nbins"]]
    p = np.diff(cdf)
    big = p * len(lam) > 20
    e = p[big] * len(lam)
    chi2 = (((counts[big] - e) ** 2) / e).sum()
    assert stats.chi2.sf(chi2, big.sum() - 1) > 1e-4
    frac = (lam - tab["p0"]) / tab["p1"] - k
    assert stats.kstest(frac, "uniform").pvalue > 1e-3


def test_isotropic_yield_is_poisson_in_length(oracle_lib):
    """Photon count per segment ~ Poisson(yield x length): mean and variance
    of 400 segments of 100 mm at 20 photons/mm."""
    wl = w.scintillation(400)
    n, mu, _ = oracle_lib.track_yield(wl.tracks, oracle_lib.params(wl))
    assert np.allclose(mu, 2000.0, rtol=1e-6)
    assert abs(n.mean() - 2000.0) < 4 * math.sqrt(2000.0 / 400)
    assert 0.75 < n.var() / 2000.0 < 1.3


def test_isotropic_point_in_detector_box_solid_angle(oracle_lib):
    """An isotropic point source at the centre of a cube of detector faces
    (QE = 1): no photon escapes, each face receives 1/6 of them, and on a
    face at distance d the fraction of photons within radius rho of the
    face centre is (1 - d / sqrt(rho^2 + d^2)) / 2 (solid angle of a cone)."""
    from scipy import stats
    scene = _all_detector_box()
    tr = w._make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), p=[1.0],
                        mass=[0.0], length=[0.0], event=[0], tid=[0], n_fixed=[60000])
    wl = w.Workload("iso_point", scene, tr, n_minus_1=0.0, source=w.SOURCE_ISOTROPIC,
                    lambda_min=300.0, lambda_max=500.0)
    out = oracle_lib.Scene(scene).trace(tr, oracle_lib.params(wl))
    assert np.all(out["fate"] == 5)
    per = np.bincount(out["plane"], minlength=6)
    assert stats.chisquare(per).pvalue > 1e-3
    top = out["plane"] == 1
    rho = np.hypot(out["u"][top] - 500.0, out["v"][top] - 500.0)
    inside = rho < 500.0
    cdf = lambda r: (1 - 500.0 / np.sqrt(r * r + 500.0 ** 2)) / 2
    # conditional on rho < 500 (the inscribed disc)
    x = cdf(rho[inside]) / cdf(500.0)
    assert stats.kstest(x, "uniform").pvalue > 1e-3
    assert abs(inside.sum() / len(out["fate"]) - cdf(500.0)) < 4 * math.sqrt(cdf(500.0) / 60000)


def test_water_point_source_ring(oracle_lib):
    """Water (n = 1.33), beta = 1: a point source at the tank centre along
    +z puts every photon on the top face at radius d tan(theta) =
    2000 sqrt(n^2 - 1) = 1753.67 mm from its centre (Sec. 3 angle; the
    liquid radiators of Sec. 6); the Frank-Tamm yield per mm over 300-600 nm
    is 2 pi alpha (1 - 1/n^2)(1/300 nm - 1/600 nm)."""
    scene = w.water_tank_scene()
    tr = w._make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), p=[1e6],
                        mass=[0.0], length=[0.0], event=[0], tid=[0], n_fixed=[5000])
    wl = w.Workload("water_point", scene, tr, n_minus_1=0.33, lambda_min=300.0,
                    lambda_max=600.0)
    out = oracle_lib.Scene(scene).trace(tr, oracle_lib.params(wl))
    hit = out["fate"] == 5
    assert hit.sum() > 500
    assert np.all(out["plane"][hit] == 1)
    n = 1 + float(np.float32(0.33))
    r = np.hypot(out["u"][hit] - 2000.0, out["v"][hit] - 2000.0)
    assert np.abs(r - 2000.0 * math.sqrt(n * n - 1)).max() < 1e-9
    assert set(np.unique(out["fate"])) <= {4, 5}
    y = oracle_lib.yield_per_mm(float(np.float32(0.33)), 1.0, 300.0, 600.0)
    alpha = 1 / 137.035999
    assert y == pytest.approx(2 * math.pi * alpha * (1 - 1 / n**2) * (1e6 / 300 - 1e6 / 600),
                              rel=1e-12)
    assert 30 < y < 36


def test_scintillation_box_bookkeeping(oracle_lib):
    """Scintillation box: photons end detected on the top/bottom planes,
    QE-rejected, absorbed by a wall reflection or at the reflection limit;
    hits after k wall reflections exist for several k; counts and sums agree
    with the hit list."""
    wl = w.scintillation(30)
    out = oracle_lib.Scene(wl.scene).trace(wl.tracks, oracle_lib.params(wl))
    f = out["fate"]
    esc = (f == 1) & (out["graze"] == 0)
    assert esc.sum() == 0
    assert set(np.unique(f)) <= {1, 2, 4, 5, 6}
    det = f == 5
    assert set(np.unique(out["plane"][det])) == {0, 1}
    assert len(np.unique(out["n_refl"][det])) >= 4
    assert out["pixel_counts"].sum() == det.sum()
    assert (out["graze"] != 0).mean() < 0.01


# ------------------------------------------------------ dispersive radiator
def _n1_disp(lam_nm, a, l0):
    """n - 1 of the single-resonance form (its definition, lambda in nm)."""
    return a / (1.0 / l0**2 - 1.0 / lam_nm**2)


@pytest.mark.parametrize("p", [1000.0, 50.0, 4.0, 2.75, 2.6, 2.5, 2.4])
def test_dispersive_yield_matches_quadrature(oracle_lib, p):
    """Frank-Tamm photons per mm with n(lambda): the oracle's closed-form
    integral against numerical quadrature of
    2 pi alpha int max(0, 1 - 1/(n(lambda) beta)^2) dlambda / lambda^2 over
    200-600 nm, for pions from far above threshold to below it (between
    2.47 and 2.64 GeV/c only the shorter wavelengths emit)."""
    from scipy import integrate
    a, l0 = w.C4F10_DISPERSION
    wl = w.rich1_dispersive(1)
    prm = oracle_lib.params(wl)
    p, m = float(np.float32(p)), float(np.float32(w.PION_MASS))   # the FP32 inputs
    E = math.sqrt(p * p + m * m)
    beta = p / E
    f = lambda lam: max(0.0, 1.0 - 1.0 / ((1 + _n1_disp(lam, a, l0)) * beta) ** 2) / lam**2
    g = lambda lam: (1 + _n1_disp(lam, a, l0)) * beta - 1
    hi = 600.0
    if g(200.0) > 0 > g(600.0):       # emission stops inside the band: split there
        from scipy import optimize
        hi = optimize.brentq(g, 200.0, 600.0, xtol=1e-13)
    ref = 0.0 if g(200.0) <= 0 else 2 * math.pi / 137.035999 * integrate.quad(
        f, 200.0, hi, limit=200, epsabs=1e-15, epsrel=1e-13)[0] * 1e6
    got = oracle_lib.disp_yield_per_mm(prm, p, m)
    if ref == 0.0:
        assert got == 0.0
    else:
        assert got == pytest.approx(ref, rel=1e-8, abs=1e-12)
    if p < 2.45:
        assert got == 0.0


def test_dispersive_yield_constant_index_limit(oracle_lib):
    """With lambda0 far below the band, n - 1 = a lambda0^2 (1 + O(lambda0^2 /
    lambda^2)) is constant to 1e-5 and the yield equals the constant-index
    Frank-Tamm value (itself pinned to the PDG constant) to 1e-4."""
    wl = w.rich1_dispersive(1)
    wl.dispersion = (float(np.float32(1.4e-3)), 1.0)
    prm = oracle_lib.params(wl)
    got = oracle_lib.disp_yield_per_mm(prm, 1e6, 0.0)
    ref = oracle_lib.yield_per_mm(1.4e-3, 1.0, 200.0, 600.0)
    assert got == pytest.approx(ref, rel=1e-4)


def test_dispersive_emission_wavelength_law_and_angle(oracle_lib):
    """Photons of a beta = 1 point source with n(lambda): the wavelengths
    follow the density sin^2 theta(lambda) / lambda^2 (KS against its
    numerically integrated CDF), and every hit of the point-source scene
    lies at (R/2) tan theta(lambda) of its own wavelength (the source sits
    at the centre of curvature), tan theta = sqrt(n(lambda)^2 - 1)."""
    from scipy import integrate, stats
    a, l0 = w.C4F10_DISPERSION
    wl = w.point_source(100000)
    wl.dispersion = w.C4F10_DISPERSION
    out = oracle_lib.Scene(wl.scene).trace(wl.tracks, oracle_lib.params(wl))
    dens = lambda lam: (1.0 - 1.0 / (1 + _n1_disp(lam, a, l0)) ** 2) / lam**2
    norm = integrate.quad(dens, 200.0, 600.0)[0]
    grid = np.linspace(200.0, 600.0, 401)
    cdf_grid = np.array([integrate.quad(dens, 200.0, x)[0] / norm for x in grid])
    lam = out["lambda"].astype(np.float64)
    u = np.interp(lam, grid, cdf_grid)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # the constant-index spectrum 1/lambda^2 is rejected by the same test
    u_flat = (1 / 200.0 - 1 / lam) / (1 / 200.0 - 1 / 600.0)
    assert stats.kstest(u_flat, "uniform").pvalue < 1e-6
    det, r = _ring_radii(out, wl.scene.rects[0])
    n = 1 + _n1_disp(out["lambda"][det].astype(np.float64), np.float64(a), np.float64(l0))
    np.testing.assert_allclose(r, 1355.0 * np.sqrt(n * n - 1), rtol=0, atol=1e-9)
    assert r.max() - r.min() > 3.0        # dispersion spreads the ring


def test_dispersive_threshold_band(oracle_lib):
    """A 2.55 GeV/c pion in C4F10-like gas is above threshold only at short
    wavelengths: every photon's wavelength lies below the threshold
    wavelength where n(lambda) beta = 1."""
    a, l0 = w.C4F10_DISPERSION
    wl = w.rich1_dispersive(1, meshed=False)
    p, m = 2.55, w.PION_MASS
    wl.tracks = w._make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), p=[p],
                               mass=[m], length=[1000.0], event=[0], tid=[0], n_fixed=[3000])
    out = oracle_lib.Scene(wl.scene).trace(wl.tracks, oracle_lib.params(wl))
    pf, mf = float(np.float32(p)), float(np.float32(m))
    beta = pf / math.sqrt(pf * pf + mf * mf)
    from scipy import optimize
    lam_t = optimize.brentq(lambda lam: (1 + _n1_disp(lam, a, l0)) * beta - 1, 200.0, 600.0)
    assert lam_t < 400.0
    assert out["lambda"].max() <= lam_t * (1 + 1e-6)
    assert out["lambda"].min() >= 200.0


# ------------------------------------------------- refraction (window slab)
def test_window_slab_ring_closed_form(oracle_lib):
    """A beta = 1 Cherenkov cone (water, n = 1.33, theta = 41 degrees) from a
    point along +z crosses a 30 mm glass slab (900 < z < 930) before a
    plane at z = 1000: Snell's law at both faces gives the ring radius
    970 tan(theta) + 30 tan(theta_r), sin(theta_r) = sin(theta) / n_w(lambda)
    with the window's binned index at each photon's wavelength (paper
    Sec. 4.1 removed the windows; this puts one back)."""
    wl = w.slab_ring(5000)
    scene, tr = wl.scene, wl.tracks
    out = oracle_lib.Scene(scene).trace(tr, oracle_lib.params(wl))
    det = out["fate"] == 5
    assert det.all()
    n = 1 + float(np.float32(0.33))
    sin_t = math.sqrt(1 - 1 / n**2)
    lam = out["lambda"].astype(np.float32)
    k = np.clip(np.floor((lam - np.float32(200)) / np.float32(25)), 0, 15).astype(int)
    n_w = np.asarray(w.f32(w.QUARTZ_N), np.float64)[k]
    sin_r = sin_t / n_w
    r_exp = 970.0 * sin_t / math.sqrt(1 - sin_t**2) + 30.0 * sin_r / np.sqrt(1 - sin_r**2)
    r = np.hypot(out["u"] - 1280.0, out["v"] - 1280.0)
    np.testing.assert_allclose(r, r_exp, rtol=0, atol=1e-9)
    assert r.max() - r.min() > 0.5            # the index varies with the wavelength


def test_window_total_internal_reflection_fraction(oracle_lib):
    """An isotropic source in the middle of a 6 mm slab of index 1.5 with
    photodetector planes (QE = 1) 7 mm above and below: only photons with
    |cos(theta)| > cos(theta_c) = sqrt(1 - 1/n^2) leave through a face, so
    the detected fraction is 1 - cos(theta_c) = 0.2546; each escaping photon
    lands at 3 tan(theta_in) + 7 tan(theta_out) from the source's foot,
    sin(theta_out) = n sin(theta_in); trapped photons bounce by total
    internal reflection until the direction-change limit."""
    from scipy import stats
    N = 40000
    wl = w.slab_tir(N)
    scene, tr = wl.scene, wl.tracks
    prm = oracle_lib.params(wl)
    out = oracle_lib.Scene(scene).trace(tr, prm)
    det = out["fate"] == 5
    frac = 1 - math.sqrt(1 - 1 / 1.5**2)
    assert abs(det.mean() - frac) < 4 * math.sqrt(frac * (1 - frac) / N)
    assert set(np.unique(out["fate"][~det])) <= {1, 6}
    assert stats.chisquare(np.bincount(out["plane"][det], minlength=2)).pvalue > 1e-3
    for g in np.nonzero(det)[0][:400]:
        _, d, _ = oracle_lib.emit(tr, prm, 0, int(g))
        s_in = math.hypot(d[0], d[1])
        s_out = 1.5 * s_in
        r_exp = 3 * s_in / abs(d[2]) + 7 * s_out / math.sqrt(1 - s_out**2)
        up = d[2] > 0
        cx = 2048.0
        r = math.hypot(out["u"][g] - cx, out["v"][g] - cx)
        assert out["plane"][g] == (0 if up else 1)
        assert abs(r - r_exp) < 1e-9


def test_surface_skip_rule(oracle_lib):
    """A photon leaving a surface (one mirror segment, flat or window face:
    the triangles of one `triangles` call) is not intersected with that
    surface again at its next step. A ray starting 1e-4 mm below a flat
    meshed mirror and leaving it at a grazing angle re-enters a neighbouring
    facet when only the facet just hit is skipped, and does not when the
    whole surface is skipped; BVH and brute force agree under the rule."""
    b = w._Builder("flat")
    t = b.table_const(0.9)
    m = b.material(w.MAT_MIRROR, t)
    b.triangles(w._mesh_rectangle(np.array([-100.0, -100.0, 0.0]), np.array([1.0, 0, 0]),
                                  np.array([0, 1.0, 0]), 200.0, 200.0, 20, 20),
                None, m, smooth=False)
    with_s = b.build()
    without = w.Scene(**{**with_s.__dict__, "tri_surface": None})
    n = with_s.n_triangles
    rng = np.random.default_rng(1)
    k = rng.integers(0, n, 400)
    cen = with_s.tri_vertices[k].astype(np.float64).mean(axis=1)
    o = cen - np.array([0, 0, 1e-4])
    ang = rng.uniform(0, 2 * np.pi, 400)
    d = np.stack([np.cos(ang), np.sin(ang), np.full(400, 1e-5)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t0, p0 = oracle_lib.Scene(without).raycast(o, d, skip=k, t_min=1e-3)
    assert (p0 >= 0).sum() > 300          # neighbouring facets are re-hit
    for bvh in (True, False):
        t1, p1 = oracle_lib.Scene(with_s).raycast(o, d, skip=k, t_min=1e-3, use_bvh=bvh)
        assert np.all(p1 == -1)
