"""Pins of the oracle's smooth-normal reflection on triangle meshes and of
the graze flag of its surface-skip rule (no GPU).

A spherical mirror given as a triangle mesh carries, at each vertex, the
unit normal of the sphere there, (C - v)/R, and a hit reflects about the
barycentric blend of its triangle's vertex normals, renormalised. Because
the hit point itself is the same blend of the vertices, p = sum b_i v_i,
the blend of the normals is sum b_i (C - v_i)/R = (C - p)/R: the smooth
normal at ANY point of such a mesh points exactly at the centre of
curvature. Two consequences pin the oracle's interpolation against
geometry rather than against its own formula:

  * the normal it reflects about equals (C - p)/|C - p| at every hit, and
    the normal of the vertex itself at each vertex;
  * a point source at the centre of curvature of the meshed mirror images
    onto itself, so every hit on the plane at R/2 lies at the analytic ring
    radius (R/2) tan(theta), whatever the facet size.

The only departure from exactness is the FP32 rounding of the stored
vertices and normals: each vertex normal is within sqrt(3) 2^-25 = 5.2e-8
of the exact one and each vertex within sqrt(3) 1.22e-4 mm of its FP64
position (coordinates below 4096 mm), which moves (C - p)/R by at most
7.8e-8 at R = 2710 mm. So the smooth normal is within 1.3e-7 of (C - p)/|C - p|
(bound 2e-7 below), and a reflected ray turns by at most 2.6e-7 rad, which
over the ~1360 mm from the mirror to the plane moves a hit by at most
3.5e-4 mm (bound 5e-4 mm). A blend with two weights exchanged, a blend left
unnormalised, or the flat facet normal all miss these bounds by one to four
orders of magnitude: the mutation test compiles the oracle with each of
those mistakes and checks that the pins named for it fail.
"""
import math
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_2309_12496_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ETA_C4F10 = float(np.float32(0.0014))
R_MIRROR = 2710.0
NORMAL_BOUND = 2e-7        # |n_smooth - (C - p)/|C - p||, derived above
RING_BOUND_MM = 5e-4       # |ring radius - (R/2) tan(theta)|, derived above


def _sphere_mesh_rays(sc_, n, rng, bary):
    """Rays from the centre of curvature (the origin) through points with
    barycentrics `bary` of random triangles of the meshed mirror."""
    V = sc_.tri_vertices.astype(np.float64)
    k = rng.integers(0, sc_.n_triangles, n)
    p = np.einsum("ki,kij->kj", bary, V[k])
    d = p / np.linalg.norm(p, axis=1, keepdims=True)
    return k, np.zeros_like(d), d


def test_smooth_normal_points_at_centre_of_curvature(oracle_lib):
    """At random points of a smooth-normal sphere mesh the normal used for
    reflection is (C - p)/|C - p| within the FP32 input bound, of unit
    length to rounding, and differs from the flat facet normal (so the
    smooth branch is the one taken)."""
    sc_ = w.point_source_scene(meshed=True)
    sc = oracle_lib.Scene(sc_)
    rng = np.random.default_rng(0)
    k, o, d = _sphere_mesh_rays(sc_, 5000, rng, rng.dirichlet([1, 1, 1], 5000))
    # primitive 0 is the detector plane between the source and the mirror
    r = sc.probe(o, d, skip=np.zeros(len(d), np.int32))
    assert np.all(r["prim"] - 1 == k)
    p = r["t"][:, None] * d
    exact = -p / np.linalg.norm(p, axis=1, keepdims=True)
    ns = r["n_shade"]
    assert np.abs(np.linalg.norm(ns, axis=1) - 1.0).max() < 1e-12
    assert np.linalg.norm(ns - exact, axis=1).max() < NORMAL_BOUND
    # the facet normal is off by up to half the facet's angular size
    assert np.linalg.norm(r["n_geo"] - exact, axis=1).max() > 1e-3


@pytest.mark.parametrize("vertex", [0, 1, 2])
def test_smooth_normal_at_each_vertex_is_that_vertex_normal(oracle_lib, vertex):
    """Next to vertex i of a triangle (barycentric 1 - 2e-9 on it) the
    normal used for reflection is vertex i's own normal: each barycentric
    weight multiplies the normal of its own vertex."""
    sc_ = w.point_source_scene(meshed=True)
    sc = oracle_lib.Scene(sc_)
    rng = np.random.default_rng(1 + vertex)
    bary = np.full((3000, 3), 1e-9)
    bary[:, vertex] = 1.0 - 2e-9
    k, o, d = _sphere_mesh_rays(sc_, 3000, rng, bary)
    r = sc.probe(o, d, skip=np.zeros(len(d), np.int32))
    nv = sc_.tri_normals[k, vertex].astype(np.float64)
    nv /= np.linalg.norm(nv, axis=1, keepdims=True)
    assert np.linalg.norm(r["n_shade"] - nv, axis=1).max() < 1e-9
    # the other two vertex normals are far from it (facets ~15 mm, R 2710)
    other = sc_.tri_normals[k, (vertex + 1) % 3].astype(np.float64)
    assert np.linalg.norm(other - nv, axis=1).min() > 1e-3


_PIN_SCRIPT = r"""
import math, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2309_12496_gb300 import workloads as w
wl = w.point_source(20000, meshed=True)
sc = oracle.Scene(wl.scene)
out = sc.trace(wl.tracks, oracle.params(wl))
det = out["fate"] == 5
rect = wl.scene.rects[0]
hu = -float(np.dot(rect["origin"], rect["u_axis"]))
hv = -float(np.dot(rect["origin"], rect["v_axis"]))
rad = np.hypot(out["u"][det] - hu, out["v"][det] - hv)
n = 1.0 + float(np.float32(0.0014))
ring = float(np.abs(rad - 1355.0 * math.sqrt(n * n - 1)).max())
rng = np.random.default_rng(0)
V = wl.scene.tri_vertices.astype(np.float64)
k = rng.integers(0, wl.scene.n_triangles, 2000)
p = np.einsum("ki,kij->kj", rng.dirichlet([1, 1, 1], 2000), V[k])
d = p / np.linalg.norm(p, axis=1, keepdims=True)
r = sc.probe(np.zeros_like(d), d, skip=np.zeros(len(d), np.int32))
hit = r["t"][:, None] * d
exact = -hit / np.linalg.norm(hit, axis=1, keepdims=True)
ident = float(np.linalg.norm(r["n_shade"] - exact, axis=1).max())
unit = float(np.abs(np.linalg.norm(r["n_shade"], axis=1) - 1.0).max())
print(int(det.sum()), ring, ident, unit)
"""


def _pin_errors(lib_path=None):
    """(detected photons, ring radius error, normal identity error, unit
    length error) of an oracle build, run in a fresh process."""
    env = dict(os.environ)
    if lib_path:
        env["RICH_ORACLE_LIB"] = lib_path
    res = subprocess.run([sys.executable, "-c", _PIN_SCRIPT, ROOT], env=env,
                         capture_output=True, text=True, check=True)
    n_det, ring, ident, unit = res.stdout.split()
    return int(n_det), float(ring), float(ident), float(unit)


def test_meshed_point_source_ring_radius(oracle_lib):
    """A point source at the centre of curvature of the smooth-normal
    meshed mirror: every hit lies at (R/2) tan(theta) = 71.72495 mm within
    the FP32 input bound (5e-4 mm), as for the analytic sphere."""
    wl = w.point_source(20000, meshed=True)
    sc = oracle_lib.Scene(wl.scene)
    out = sc.trace(wl.tracks, oracle_lib.params(wl))
    det = out["fate"] == 5
    rect = wl.scene.rects[0]
    hu = -float(np.dot(rect["origin"], rect["u_axis"]))
    hv = -float(np.dot(rect["origin"], rect["v_axis"]))
    rad = np.hypot(out["u"][det] - hu, out["v"][det] - hv)
    n = 1.0 + ETA_C4F10
    assert det.sum() > 2000
    assert np.abs(rad - (R_MIRROR / 2) * math.sqrt(n * n - 1)).max() < RING_BOUND_MM
    assert set(np.unique(out["fate"])) <= {2, 4, 5}


# Each mutation replaces one exact piece of the smooth-normal blend in the
# oracle's source (the test fails loudly if the piece is no longer there),
# and names the pins that must catch it: the ring radius of the meshed
# point source, the normal identity n = (C - p)/|C - p|, the unit length.
_BLEND = ("*n_shade = unit(add(add(scl(t->n0, b0), scl(t->n1, h->b1)),\n"
          "                                scl(t->n2, h->b2)));")
_MUTANTS = {
    "weights_swapped": ("scl(t->n0, b0), scl(t->n1, h->b1)",
                        "scl(t->n0, h->b1), scl(t->n1, b0)", ("ring", "identity")),
    # a point source at the centre meets the mirror along the normal, so
    # only the unit-length pin sees a blend left unnormalised
    "not_renormalised": (_BLEND,
                         "*n_shade = add(add(scl(t->n0, b0), scl(t->n1, h->b1)),\n"
                         "                                scl(t->n2, h->b2));", ("unit",)),
    "facet_normal": (_BLEND, "*n_shade = t->ng;", ("ring", "identity")),
}


@pytest.mark.parametrize("mutant", sorted(_MUTANTS))
def test_pins_catch_smooth_normal_mistakes(oracle_lib, mutant):
    """The oracle compiled with one deliberate mistake in its smooth-normal
    blend (two barycentric weights exchanged; the blend not renormalised;
    the flat facet normal in place of the blend) fails the pins named for
    it, by at least tenfold their bounds, while the unmodified oracle passes
    every one."""
    src = open(os.path.join(ROOT, "oracle", "rich_oracle.c")).read()
    old, new, caught_by = _MUTANTS[mutant]
    assert src.count(old) == 1, "the mutated piece of the oracle has changed"
    with tempfile.TemporaryDirectory() as tmp:
        c_path = os.path.join(tmp, "mutant.c")
        so_path = os.path.join(tmp, "libmutant.so")
        open(c_path, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", so_path, c_path, "-lm"], check=True)
        n_det, ring, ident, unit = _pin_errors(so_path)
    bounds = {"ring": RING_BOUND_MM, "identity": NORMAL_BOUND, "unit": 1e-12}
    got = {"ring": ring, "identity": ident, "unit": unit}
    assert n_det > 2000
    for pin in caught_by:
        assert got[pin] > 10 * bounds[pin], (mutant, pin, got)
    n_ok, *good = _pin_errors()
    assert all(e < bounds[k] for k, e in zip(("ring", "identity", "unit"), good)), good


def test_replay_smooth_branch_reproduces_forward_hits(oracle_lib):
    """On the meshed RICH1 scene every reflection is off a smooth-normal
    triangle: the gradient replay (barycentrics from the hit point by
    Cramer's rule on the triangle's edge vectors) reproduces the forward
    trace's hits (Moeller-Trumbore barycentrics) to 1e-9 mm."""
    tr = w.pion_tracks(6, seed=2, n_fixed=300)
    wl = w.Workload("g", w.rich1_scene(meshed=True), tr, n_minus_1=0.0014)
    sc = oracle_lib.Scene(wl.scene)
    prm = oracle_lib.params(wl)
    th = w.nominal_theta(wl.scene, wl.n_minus_1)
    out = sc.trace(wl.tracks, prm)
    off = out["offsets"].astype(np.int64)
    checked = 0
    for g in np.nonzero(out["fate"] == 5)[0][::5]:
        t = int(np.searchsorted(off, g, side="right") - 1)
        fate, u, v, du, dv = sc.hit_jacobian(wl.tracks, prm, th, t, int(g - off[t]))
        assert fate == 5
        assert abs(u - out["u"][g]) < 1e-9 and abs(v - out["v"][g]) < 1e-9
        checked += 1
    assert checked > 20


def test_skip_rule_flags_a_chord_on_the_same_concave_segment(oracle_lib):
    """A photon leaving a concave mirror segment is not intersected with the
    same segment at its next step. For a sphere that is exact only away from
    the tangent plane: a ray leaving the sphere at angle a into its inside
    meets it again after the chord 2 R sin(a). Rays start on the meshed
    mirror near its pole (depth h below the sphere, known) at a = 0.04 rad
    to the sphere's tangent plane; the chord (~217 mm) ends on the same
    mesh. The oracle takes no hit from that surface, reports the skipped hit
    at the chord length from the start point to the true sphere within the
    far facet's sagitta over sin(a) (21.2 mm cell diagonals: sagitta
    <= 21.2^2 / (8 R) = 0.021 mm, so within 0.021/0.04 = 0.52 mm; bound
    0.6 mm) and flags the decision (graze bit 8). At a = 0.4 rad the chord
    (2110 mm) leaves the mesh and nothing is flagged."""
    sc_ = w.point_source_scene(meshed=True)
    sc = oracle_lib.Scene(sc_)
    rng = np.random.default_rng(5)
    n = 400
    xy = rng.uniform(-30.0, 30.0, (n, 2))
    zc = np.sqrt(R_MIRROR ** 2 - (xy ** 2).sum(axis=1))
    radial = np.column_stack([xy, zc]) / R_MIRROR        # outward unit normal
    tang = np.cross(radial, rng.normal(size=(n, 3)))
    tang /= np.linalg.norm(tang, axis=1, keepdims=True)
    first = sc.probe(np.zeros((n, 3)), radial, skip=np.zeros(n, np.int32))
    assert np.all(first["prim"] >= 1)
    # start on the facet, on the ray from the centre, 1e-9 mm inside it
    o = radial * (first["t"] - 1e-9)[:, None]
    h = R_MIRROR - np.linalg.norm(o, axis=1)
    assert np.all((h >= 0) & (h < 0.021))
    for a, expect_flag in ((0.04, True), (0.4, False)):
        d = math.cos(a) * tang - math.sin(a) * radial
        r = sc.probe(o, d, skip=first["prim"])
        if expect_flag:
            assert np.all(r["graze"] & 8)
            rs = R_MIRROR - h
            chord = rs * math.sin(a) + np.sqrt((rs * math.sin(a)) ** 2 + 2 * R_MIRROR * h - h * h)
            assert np.abs(r["skipped_t"] - chord).max() < 0.6
            # what the rule decides: the photon goes on to the detector plane
            # or escapes, past the skipped chord
            assert np.all((r["prim"] == -1) | (r["t"] > r["skipped_t"]))
        else:
            assert not np.any(r["graze"] & 8)
            assert np.all(np.isinf(r["skipped_t"]))
