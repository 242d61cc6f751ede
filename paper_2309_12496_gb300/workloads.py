"""Seeded synthetic inputs: detector scenes and charged tracks.

This module builds the *inputs* of the photon propagator -- geometry
descriptions and track lists -- and nothing of the propagation itself (no
emission, intersection, reflection or detection arithmetic lives here). Both
the CUDA path and the FP64 oracle read what it produces, so every floating
value it hands out is rounded to FP32 first: the two sides then start from
bit-identical inputs and differ only in their own arithmetic.

The paper's own inputs -- Geant4 photons from a 100 GeV muon and the
simplified LHCb RICH geometry translated to meshes (Sec. 4.1, Sec. 5.1) --
are not available, so the scenes below are synthetic stand-ins with the
stated shapes:

* ``point_source``: one spherical mirror (R = 2710 mm) with the source at
  its centre of curvature, a 256 x 256 plane of 2.88 mm pixels at R/2, a
  Gaussian quantum efficiency and reflectivity 0.9.
* ``rich1``: four spherical tiles (R = 2710 mm, two tilted up, two down),
  two flat mirrors and three 256 x 256 planes (upper, lower, and a monitor
  wall behind the mirror gaps, cf. the wall of Sec. 5.1); the mirrors as
  ~20k triangles (meshed) or as analytic surfaces.
* ``rich2``: 56 hexagonal tiles (R = 8600 mm), two flat mirrors, an
  absorbing support plate (~150k triangles) and two 512 x 512 planes.

Response tables follow Sec. 4.3: a quantum efficiency histogram in 33 nm
bins peaking at 35% near 450 nm, and reflectivity histograms in 25 nm bins
falling from 94% to 89% over 200-600 nm (the curves themselves are only in
a figure, so their shapes here are plausible synthetic ones).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------- layouts
# Binary layouts of the geometry records (little-endian, 4-byte fields).
TABLE_DTYPE = np.dtype([
    ("kind", "<i4"), ("nbins", "<i4"),
    ("p0", "<f4"), ("p1", "<f4"), ("p2", "<f4"), ("p3", "<f4"),
    ("values", "<f4", (64,)),
])
MATERIAL_DTYPE = np.dtype([
    ("kind", "<i4"), ("table", "<i4"), ("plane", "<i4"), ("flags", "<i4"),
])
SPHERE_DTYPE = np.dtype([
    ("center", "<f4", (3,)), ("radius", "<f4"),
    ("axis", "<f4", (3,)), ("cos_min", "<f4"),
    ("e1", "<f4", (3,)), ("n_edges", "<i4"),
    ("e2", "<f4", (3,)), ("material", "<i4"),
    ("edges", "<f4", (8, 3)),
])
RECT_DTYPE = np.dtype([
    ("origin", "<f4", (3,)), ("width", "<f4"),
    ("u_axis", "<f4", (3,)), ("height", "<f4"),
    ("v_axis", "<f4", (3,)), ("pitch", "<f4"),
    ("normal", "<f4", (3,)), ("material", "<i4"),
    ("nx", "<i4"), ("ny", "<i4"), ("reserved0", "<i4"), ("reserved1", "<i4"),
])
assert TABLE_DTYPE.itemsize == 280
assert MATERIAL_DTYPE.itemsize == 16
assert SPHERE_DTYPE.itemsize == 160
assert RECT_DTYPE.itemsize == 80

TABLE_CONST, TABLE_GAUSS, TABLE_HIST, TABLE_CDF = 0, 1, 2, 3
SOURCE_CHERENKOV, SOURCE_ISOTROPIC = 0, 1
MAT_MIRROR, MAT_ABSORBER, MAT_DETECTOR, MAT_DIELECTRIC = 0, 1, 2, 3
MAT_SMOOTH = 1

PION_MASS = 0.13957   # GeV/c^2
MUON_MASS = 0.10566   # GeV/c^2
PIXEL_PITCH = 2.88    # mm


def f32(x):
    """Round to FP32 (the precision every geometric input is stored in)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32)


# ------------------------------------------------------------------- scene
@dataclasses.dataclass
class Scene:
    name: str
    tables: np.ndarray
    materials: np.ndarray
    spheres: np.ndarray
    rects: np.ndarray
    tri_vertices: np.ndarray          # (n, 3, 3) float32
    tri_normals: np.ndarray | None    # (n, 3, 3) float32
    tri_material: np.ndarray          # (n,) int32
    tri_surface: np.ndarray | None = None   # (n,) int32 surface ids, or None

    @property
    def n_triangles(self) -> int:
        return int(self.tri_vertices.shape[0])

    @property
    def planes(self):
        """Detector planes as (plane index, nx, ny, pitch), sorted by index."""
        out = {}
        for r in self.rects:
            m = self.materials[r["material"]]
            if m["kind"] == MAT_DETECTOR:
                out[int(m["plane"])] = (int(r["nx"]), int(r["ny"]),
                                        float(r["pitch"]))
        return [(k,) + out[k] for k in sorted(out)]

    @property
    def pixels_per_event(self) -> int:
        return sum(nx * ny for _, nx, ny, _ in self.planes)


class _Builder:
    def __init__(self, name):
        self.name = name
        self.tables, self.materials, self.spheres, self.rects = [], [], [], []
        self.tris, self.tri_normals, self.tri_mat, self.tri_surf = [], [], [], []
        self.any_smooth = False

    def table_const(self, value):
        t = np.zeros((), TABLE_DTYPE)
        t["kind"], t["p0"] = TABLE_CONST, value
        self.tables.append(t)
        return len(self.tables) - 1

    def table_gauss(self, a, mu, sigma):
        t = np.zeros((), TABLE_DTYPE)
        t["kind"], t["p0"], t["p1"], t["p2"] = TABLE_GAUSS, a, mu, sigma
        self.tables.append(t)
        return len(self.tables) - 1

    def table_hist(self, lam0, width, values):
        t = np.zeros((), TABLE_DTYPE)
        t["kind"], t["p0"], t["p1"] = TABLE_HIST, lam0, width
        t["nbins"] = len(values)
        t["values"][: len(values)] = values
        self.tables.append(t)
        return len(self.tables) - 1

    def table_cdf(self, lam0, width, weights):
        """Binned emission spectrum as its CDF at the bin edges: c_0 = 0,
        c_n = 1, nondecreasing, rounded to FP32 (both sides invert the same
        FP32 table)."""
        w = np.asarray(weights, np.float64)
        c = np.concatenate([[0.0], np.cumsum(w) / w.sum()])
        c = f32(c)
        c[0], c[-1] = 0.0, 1.0
        c = np.maximum.accumulate(c)
        t = np.zeros((), TABLE_DTYPE)
        t["kind"], t["p0"], t["p1"] = TABLE_CDF, lam0, width
        t["nbins"] = len(w)
        t["values"][: len(c)] = c
        self.tables.append(t)
        return len(self.tables) - 1

    def material(self, kind, table=-1, plane=-1, flags=0):
        m = np.zeros((), MATERIAL_DTYPE)
        m["kind"], m["table"], m["plane"], m["flags"] = kind, table, plane, flags
        self.materials.append(m)
        return len(self.materials) - 1

    def sphere(self, center, radius, axis, e1, e2, material, cos_min=0.0,
               edges=()):
        s = np.zeros((), SPHERE_DTYPE)
        s["center"], s["radius"], s["axis"] = center, radius, axis
        s["e1"], s["e2"], s["cos_min"] = e1, e2, cos_min
        s["material"], s["n_edges"] = material, len(edges)
        for j, e in enumerate(edges):
            s["edges"][j] = e
        self.spheres.append(s)
        return len(self.spheres) - 1

    def rect(self, origin, u_axis, v_axis, width, height, material,
             nx=0, ny=0, pitch=0.0):
        r = np.zeros((), RECT_DTYPE)
        n = np.cross(u_axis, v_axis)
        n = n / np.linalg.norm(n)
        r["origin"], r["u_axis"], r["v_axis"], r["normal"] = (
            origin, u_axis, v_axis, n)
        r["width"], r["height"], r["material"] = width, height, material
        r["nx"], r["ny"], r["pitch"] = nx, ny, pitch
        self.rects.append(r)
        return len(self.rects) - 1

    def triangles(self, verts, normals, material, smooth):
        verts = np.asarray(verts, np.float64)
        self.tris.append(verts)
        if normals is None:
            g = np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0])
            g /= np.linalg.norm(g, axis=1, keepdims=True)
            normals = np.repeat(g[:, None, :], 3, axis=1)
        self.tri_normals.append(np.asarray(normals, np.float64))
        self.tri_mat.append(np.full(len(verts), material, np.int32))
        # one surface per call (a mirror segment, a flat mirror, a plate)
        self.tri_surf.append(np.full(len(verts), len(self.tri_surf), np.int32))
        self.any_smooth |= smooth

    def build(self) -> Scene:
        def arr(lst, dt):
            return np.array(lst, dtype=dt) if lst else np.zeros(0, dt)
        if self.tris:
            tv = f32(np.concatenate(self.tris))
            tn = f32(np.concatenate(self.tri_normals))
            tm = np.concatenate(self.tri_mat).astype(np.int32)
            ts = np.concatenate(self.tri_surf).astype(np.int32)
        else:
            tv = np.zeros((0, 3, 3), np.float32)
            tn = None
            tm = np.zeros(0, np.int32)
            ts = np.zeros(0, np.int32)
        return Scene(self.name, arr(self.tables, TABLE_DTYPE),
                     arr(self.materials, MATERIAL_DTYPE),
                     arr(self.spheres, SPHERE_DTYPE),
                     arr(self.rects, RECT_DTYPE), tv,
                     tn if self.any_smooth else None, tm, ts)


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


# ---------------------------------------------------- response tables (4.3)
# Quantum efficiency: 33 nm bins from 200 nm, peak 35% near 450 nm, falling
# towards both ends of the 200-1000 nm window (synthetic shape).
QE_LAMBDA0, QE_WIDTH = 200.0, 33.0
QE_BINS = [0.010, 0.070, 0.150, 0.220, 0.280, 0.320, 0.340, 0.350, 0.335,
           0.300, 0.255, 0.205, 0.160, 0.120, 0.085, 0.060, 0.040, 0.027,
           0.018, 0.011, 0.007, 0.004, 0.002, 0.001, 0.0]
# Mirror reflectivity: 25 nm bins over 200-600 nm, from 94% down to 89%, one
# table per mirror segment family (the two interpolated segments of Sec. 4.3).
R_LAMBDA0, R_WIDTH = 200.0, 25.0
R_BINS_A = [0.940, 0.938, 0.935, 0.932, 0.929, 0.926, 0.923, 0.920, 0.916,
            0.912, 0.909, 0.905, 0.902, 0.898, 0.895, 0.891]
R_BINS_B = [0.935, 0.934, 0.932, 0.930, 0.927, 0.924, 0.921, 0.917, 0.914,
            0.910, 0.906, 0.903, 0.899, 0.896, 0.893, 0.890]


# Refractive index of a fused-silica-like window, 25 nm bins over 200-600 nm
# (synthetic smooth shape: 1.551 at 200 nm falling to 1.458 at 600 nm).
QUARTZ_LAMBDA0, QUARTZ_WIDTH = 200.0, 25.0
QUARTZ_N = [1.5510, 1.5320, 1.5170, 1.5050, 1.4950, 1.4870, 1.4810, 1.4760, 1.4720,
            1.4690, 1.4660, 1.4640, 1.4620, 1.4610, 1.4595, 1.4580]


# ----------------------------------------------------------- point source
def point_source_scene(radius=2710.0, half_aperture=0.3, n_pix=256,
                       pitch=PIXEL_PITCH, meshed=False, mesh_half=300.0,
                       mesh_cells=40) -> Scene:
    """One spherical mirror with centre of curvature at the origin and its
    pole on +z; a detector plane at z = R/2 facing the mirror, n_pix x n_pix
    pixels centred on the axis. QE = 0.3 exp(-((l-400)/120)^2), R = 0.9
    (both analytic). meshed: the mirror is instead the patch of the sphere
    over the tangent square [-mesh_half, mesh_half]^2 as 2 x mesh_cells^2
    smooth-normal triangles (15 mm cells by default, vertex normals pointing
    at the centre), one surface."""
    b = _Builder("point_source_meshed" if meshed else "point_source")
    t_qe = b.table_gauss(0.3, 400.0, 120.0)
    t_r = b.table_const(0.9)
    m_mirror = b.material(MAT_MIRROR, t_r, flags=MAT_SMOOTH if meshed else 0)
    m_det = b.material(MAT_DETECTOR, t_qe, plane=0)
    c = np.zeros(3)
    axis, e1, e2 = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    if meshed:
        tris, nrm = _mesh_rect_tile(c, radius, axis, e1, e2, -mesh_half, mesh_half,
                                    -mesh_half, mesh_half, mesh_cells, mesh_cells)
        b.triangles(tris, nrm, m_mirror, smooth=True)
    else:
        b.sphere(center=c, radius=radius, axis=axis, e1=e1, e2=e2, material=m_mirror,
                 cos_min=math.cos(half_aperture))
    half = n_pix * pitch / 2.0
    b.rect(origin=(-half, -half, radius / 2.0), u_axis=(1.0, 0.0, 0.0),
           v_axis=(0.0, 1.0, 0.0), width=n_pix * pitch, height=n_pix * pitch,
           material=m_det, nx=n_pix, ny=n_pix, pitch=pitch)
    return b.build()


def two_mirror_scene(radius=20000.0, n_pix=256, pitch=PIXEL_PITCH) -> Scene:
    """A periscope of two analytic concave tiles: light from the origin along
    +z meets tile 0 (pole (0, 0, 1000) mm, turned 45 degrees so that it sends
    the light along +y), then tile 1 (pole (0, 1000, 1000), sending it along
    +z again), then a plane at z = 2000 facing it. Every detected photon's
    path meets both tilted tiles (the gradient's several-tile case); R = 0.9,
    QE = 0.3 exp(-((l-400)/120)^2)."""
    b = _Builder("two_mirror")
    t_qe = b.table_gauss(0.3, 400.0, 120.0)
    t_r = b.table_const(0.9)
    m_mirror = b.material(MAT_MIRROR, t_r)
    m_det = b.material(MAT_DETECTOR, t_qe, plane=0)
    s2 = 1.0 / math.sqrt(2.0)
    e1 = np.array([1.0, 0.0, 0.0])
    for pole, towards_centre in (((0.0, 0.0, 1000.0), (0.0, s2, -s2)),
                                 ((0.0, 1000.0, 1000.0), (0.0, -s2, s2))):
        n = np.asarray(towards_centre)
        centre = np.asarray(pole) + radius * n
        axis = -n                                  # centre -> pole
        b.sphere(center=centre, radius=radius, axis=axis, e1=e1, e2=np.cross(axis, e1),
                 material=m_mirror, cos_min=math.cos(0.02))
    half = n_pix * pitch / 2.0
    # u x v = -z: the plane faces the light arriving along +z
    b.rect(origin=(-half, 1000.0 - half, 2000.0), u_axis=(0.0, 1.0, 0.0),
           v_axis=(1.0, 0.0, 0.0), width=n_pix * pitch, height=n_pix * pitch,
           material=m_det, nx=n_pix, ny=n_pix, pitch=pitch)
    return b.build()


# ------------------------------------------------------- folded RICH layout
def _reflect_point(p, plane_point, plane_normal):
    p = np.asarray(p, np.float64)
    return p - 2.0 * np.dot(p - plane_point, plane_normal) * plane_normal


def _half_frame(tilt_dir, gamma):
    """Sphere frame of one mirror half tilted by gamma towards tilt_dir."""
    t = _unit(tilt_dir)
    z = np.array([0.0, 0.0, 1.0])
    axis = -math.sin(gamma) * t + math.cos(gamma) * z   # centre -> pole
    e2 = math.cos(gamma) * t + math.sin(gamma) * z      # outward on surface
    e1 = np.cross(e2, axis)
    return axis, _unit(e1), _unit(e2)


def _sphere_point(center, radius, axis, e1, e2, x, y):
    h = np.sqrt(radius * radius - x * x - y * y)
    return (center[None, :] + x[:, None] * e1[None, :] + y[:, None] * e2[None, :]
            + h[:, None] * axis[None, :])


def _mesh_rect_tile(center, radius, axis, e1, e2, x0, x1, y0, y1, nx, ny):
    """Triangles of the sphere patch over the tangent rectangle
    [x0,x1] x [y0,y1], wound so the geometric normal faces the centre."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    P = _sphere_point(center, radius, axis, e1, e2, X.ravel(), Y.ravel())
    P = P.reshape(nx + 1, ny + 1, 3)
    a, bq = P[:-1, :-1], P[1:, :-1]
    c, d = P[1:, 1:], P[:-1, 1:]
    t1 = np.stack([a, bq, c], axis=2).reshape(-1, 3, 3)
    t2 = np.stack([a, c, d], axis=2).reshape(-1, 3, 3)
    return _orient(np.concatenate([t1, t2]), center, radius)


def _orient(tris, center, radius):
    g = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    toward = center[None, :] - tris.mean(axis=1)
    flip = np.einsum("ij,ij->i", g, toward) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    normals = (center[None, None, :] - tris) / radius
    normals /= np.linalg.norm(normals, axis=2, keepdims=True)
    return tris, normals


def _mesh_rectangle(origin, u_axis, v_axis, width, height, nu, nv):
    """Flat rectangle as triangles, geometric normal = u x v."""
    us = np.linspace(0.0, width, nu + 1)
    vs = np.linspace(0.0, height, nv + 1)
    U, V = np.meshgrid(us, vs, indexing="ij")
    P = (np.asarray(origin)[None, None, :] + U[..., None] * u_axis
         + V[..., None] * v_axis)
    a, bq = P[:-1, :-1], P[1:, :-1]
    c, d = P[1:, 1:], P[:-1, 1:]
    t1 = np.stack([a, bq, c], axis=2).reshape(-1, 3, 3)
    t2 = np.stack([a, c, d], axis=2).reshape(-1, 3, 3)
    return np.concatenate([t1, t2])


@dataclasses.dataclass
class _Half:
    center: np.ndarray
    axis: np.ndarray
    e1: np.ndarray
    e2: np.ndarray
    flat_center: np.ndarray
    flat_normal: np.ndarray
    flat_u: np.ndarray
    flat_v: np.ndarray
    det_center: np.ndarray
    det_normal: np.ndarray
    det_u: np.ndarray
    det_v: np.ndarray


def _fold_half(tilt_dir, gamma, z_pole, radius, d1, image_angle, side_axis,
               y_mid):
    """One half of a folded RICH: a spherical mirror tilted by gamma towards
    tilt_dir, a flat mirror at distance d1 along the chief ray (from the
    mirror point at tangent height y_mid to the focus of light parallel to
    the beam) sending light along tilt_dir, and a detector plane through the
    folded focus of parallel light at image_angle (rad, towards tilt_dir)."""
    axis, e1, e2 = _half_frame(tilt_dir, gamma)
    pole = np.array([0.0, 0.0, z_pole])
    center = pole - radius * axis
    t = _unit(tilt_dir)
    zhat = np.array([0.0, 0.0, 1.0])
    focus0 = center + 0.5 * radius * zhat
    mid = _sphere_point(center, radius, axis, e1, e2, np.array([0.0]),
                        np.array([y_mid]))[0]
    chief = _unit(focus0 - mid)
    flat_center = mid + d1 * chief
    out_dir = t
    n_f = _unit(out_dir - chief)          # front normal (faces the light)
    f_u = _unit(np.asarray(side_axis, np.float64))
    f_v = _unit(np.cross(n_f, f_u))
    # folded focus of parallel light at image_angle towards the tilt side
    u_dir = math.sin(image_angle) * t + math.cos(image_angle) * zhat
    focus = center + 0.5 * radius * u_dir
    det_center = _reflect_point(focus, flat_center, n_f)
    det_normal = -out_dir
    d_u = f_u
    d_v = _unit(np.cross(det_normal, d_u))
    d_v = -d_v if np.dot(np.cross(d_u, d_v), det_normal) < 0 else d_v
    return _Half(center, axis, e1, e2, flat_center, n_f, f_u, f_v,
                 det_center, det_normal, d_u, d_v)


def _add_detector(b, h, material, n_pix, pitch):
    half = n_pix * pitch / 2.0
    origin = h.det_center - half * h.det_u - half * h.det_v
    b.rect(origin=origin, u_axis=h.det_u, v_axis=h.det_v,
           width=n_pix * pitch, height=n_pix * pitch, material=material,
           nx=n_pix, ny=n_pix, pitch=pitch)


def _add_window(b, h, material, n_pix, pitch, gap, thickness):
    """A flat window slab in front of a detector plane: the entry face at
    `gap` from the plane (normal towards the incoming light) and the exit
    face at gap - thickness (normal towards the plane), so the glass lies
    behind both faces."""
    half = n_pix * pitch / 2.0
    n = np.cross(h.det_u, h.det_v)
    n = n / np.linalg.norm(n)
    o = h.det_center - half * h.det_u - half * h.det_v
    b.rect(origin=o + gap * n, u_axis=h.det_u, v_axis=h.det_v, width=2 * half,
           height=2 * half, material=material)
    b.rect(origin=o + (gap - thickness) * n, u_axis=h.det_v, v_axis=h.det_u,
           width=2 * half, height=2 * half, material=material)


def rich1_scene(meshed=True, tiles_per_edge=45, flat_cells=(45, 32),
                gamma=0.30, d1=950.0, flat_size=(1000.0, 800.0),
                flat_shift=150.0, image_angle=0.12, windows=False) -> Scene:
    """RICH1-like folded geometry (synthetic, project-defined layout).

    Spherical mirror R = 2710 mm with its pole on the beam axis at
    z = 1900 mm, split into a 2 x 2 array of tiles 620 mm on a side with
    10 mm gaps; the upper pair is tilted up by gamma = 0.30 rad and the
    lower pair down, each pair focusing via a flat mirror (1000 x 800 mm,
    d1 = 950 mm from the tile centre along the chief ray) onto a 256 x 256
    plane of 2.88 mm pixels. A third 256 x 256 plane (a monitor wall at
    z = 2400 mm facing the radiator) records photons passing the tile gaps.
    Meshed: each tile as 2 x 45 x 45 smooth-normal triangles (~14 mm edges)
    and each flat mirror as 2 x 45 x 32 triangles, 21,960 triangles in
    total. Analytic: spheres and rectangles."""
    R, z_pole = 2710.0, 1900.0
    tile, gap = 620.0, 10.0
    b = _Builder("rich1_meshed" if meshed else "rich1_analytic")
    t_qe = b.table_hist(QE_LAMBDA0, QE_WIDTH, QE_BINS)
    t_ra = b.table_hist(R_LAMBDA0, R_WIDTH, R_BINS_A)
    t_rb = b.table_hist(R_LAMBDA0, R_WIDTH, R_BINS_B)
    m_sph = b.material(MAT_MIRROR, t_ra, flags=MAT_SMOOTH)
    m_flat = b.material(MAT_MIRROR, t_rb)
    m_det = [b.material(MAT_DETECTOR, t_qe, plane=i) for i in range(3)]
    halves = [
        _fold_half((0, 1, 0), gamma, z_pole, R, d1, image_angle, (1, 0, 0),
                   gap / 2 + tile / 2),
        _fold_half((0, -1, 0), gamma, z_pole, R, d1, image_angle, (1, 0, 0),
                   gap / 2 + tile / 2),
    ]
    g2 = gap / 2.0
    for h in halves:
        for xs in ((g2, g2 + tile), (-g2 - tile, -g2)):
            ys = (g2, g2 + tile)
            if meshed:
                tris, nrm = _mesh_rect_tile(h.center, R, h.axis, h.e1, h.e2,
                                            xs[0], xs[1], ys[0], ys[1],
                                            tiles_per_edge, tiles_per_edge)
                b.triangles(tris, nrm, m_sph, smooth=True)
            else:
                edges = [(1.0, 0.0, xs[1]), (-1.0, 0.0, -xs[0]),
                         (0.0, 1.0, ys[1]), (0.0, -1.0, -ys[0])]
                b.sphere(center=h.center, radius=R, axis=h.axis, e1=h.e1,
                         e2=h.e2, material=m_sph, cos_min=0.5, edges=edges)
        fw, fh = flat_size
        fu, fv, cells = h.flat_u, h.flat_v, flat_cells
        outward = 1.0 if np.dot(fv, h.det_normal) < 0 else -1.0
        f_origin = (h.flat_center + outward * flat_shift * fv - fw / 2 * fu
                    - fh / 2 * fv)
        if meshed:
            b.triangles(_mesh_rectangle(f_origin, fu, fv, fw, fh, *cells),
                        None, m_flat, smooth=False)
        else:
            b.rect(origin=f_origin, u_axis=fu, v_axis=fv, width=fw,
                   height=fh, material=m_flat)
    for i, h in enumerate(halves):
        _add_detector(b, h, m_det[i], 256, PIXEL_PITCH)
    if windows:
        # quartz windows, 6 mm thick, 20 mm in front of the two focal planes
        # (the detector windows the paper's simplified geometry removed, Sec. 4.1)
        t_quartz = b.table_hist(QUARTZ_LAMBDA0, QUARTZ_WIDTH, QUARTZ_N)
        m_quartz = b.material(MAT_DIELECTRIC, t_quartz)
        for h in halves:
            _add_window(b, h, m_quartz, 256, PIXEL_PITCH, gap=20.0, thickness=6.0)
    half = 256 * PIXEL_PITCH / 2.0
    b.rect(origin=(half, -half, 2400.0), u_axis=(-1.0, 0.0, 0.0),
           v_axis=(0.0, 1.0, 0.0), width=256 * PIXEL_PITCH,
           height=256 * PIXEL_PITCH, material=m_det[2], nx=256, ny=256,
           pitch=PIXEL_PITCH)
    return b.build()


def _hex_centers(radius_c, n_cols, n_rows):
    """Flat-topped hexagon centres in tangent coordinates (x', y'): columns
    march outward along y' >= 0, rows are centred on x' = 0."""
    out = []
    dx = math.sqrt(3.0) * radius_c
    for c in range(n_cols):
        y = radius_c + 1.5 * radius_c * c
        shift = 0.5 * dx if c % 2 else 0.0
        for r in range(n_rows):
            x = (r - (n_rows - 1) / 2.0) * dx + shift - 0.25 * dx
            out.append((x, y))
    return out


def _hex_edges(cx, cy, radius_c, gap):
    """Six half-planes a x + b y <= c of a pointy-in-x hexagon (flat edges
    facing +-x'), shrunk by gap/2."""
    inr = radius_c * math.sqrt(3.0) / 2.0 - gap / 2.0
    edges = []
    for j in range(6):
        ang = math.radians(60.0 * j)
        a, bb = math.cos(ang), math.sin(ang)
        edges.append((a, bb, inr + a * cx + bb * cy))
    return edges


def _mesh_hex(center, R, axis, e1, e2, cx, cy, radius_c, gap, k):
    inr = radius_c * math.sqrt(3.0) / 2.0 - gap / 2.0
    rc = inr * 2.0 / math.sqrt(3.0)
    corners = [(cx + rc * math.cos(math.radians(60 * j + 30)),
                cy + rc * math.sin(math.radians(60 * j + 30))) for j in range(6)]
    tris2d = []
    for j in range(6):
        A = np.array([cx, cy])
        B = np.array(corners[j])
        C = np.array(corners[(j + 1) % 6])
        for i in range(k):
            for jj in range(k - i):
                p00 = A + (B - A) * i / k + (C - A) * jj / k
                p10 = A + (B - A) * (i + 1) / k + (C - A) * jj / k
                p01 = A + (B - A) * i / k + (C - A) * (jj + 1) / k
                tris2d.append((p00, p10, p01))
                if jj < k - i - 1:
                    p11 = A + (B - A) * (i + 1) / k + (C - A) * (jj + 1) / k
                    tris2d.append((p10, p11, p01))
    t2 = np.array(tris2d)                                  # (m, 3, 2)
    pts = _sphere_point(center, R, axis, e1, e2, t2[..., 0].ravel(),
                        t2[..., 1].ravel()).reshape(-1, 3, 3)
    return _orient(pts, center, R)


def rich2_scene(meshed=True, hex_subdiv=18, gamma=0.15, d1=3200.0,
                flat_size=(2000.0, 1500.0), flat_shift=250.0,
                image_angle=0.07) -> Scene:
    """RICH2-like folded geometry (synthetic, project-defined layout).

    Spherical mirror R = 8600 mm with its pole at z = 5000 mm, two halves
    tilted left/right by 0.15 rad, each tiled by 28 hexagons (circumradius
    143 mm, 3 mm gaps) -> 56 tiles; flat mirrors (2000 x 1500 mm) fold the
    light sideways onto two 512 x 512 planes of 2.88 mm pixels; an absorbing
    support plate sits 300 mm behind the mirrors. Meshed: 56 x 1944
    smooth-normal tile triangles (~8 mm edges), 2 x 5120 flat-mirror
    triangles and a 29,768-triangle support plate (148,872 in total)."""
    R, z_pole = 8600.0, 5000.0
    rc, gap = 143.0, 3.0
    b = _Builder("rich2_meshed" if meshed else "rich2_analytic")
    t_qe = b.table_hist(QE_LAMBDA0, QE_WIDTH, QE_BINS)
    t_ra = b.table_hist(R_LAMBDA0, R_WIDTH, R_BINS_A)
    t_rb = b.table_hist(R_LAMBDA0, R_WIDTH, R_BINS_B)
    m_sph = b.material(MAT_MIRROR, t_ra, flags=MAT_SMOOTH)
    m_flat = b.material(MAT_MIRROR, t_rb)
    m_abs = b.material(MAT_ABSORBER)
    m_det = [b.material(MAT_DETECTOR, t_qe, plane=i) for i in range(2)]
    halves = [
        _fold_half((1, 0, 0), gamma, z_pole, R, d1, image_angle, (0, 1, 0),
                   3.25 * rc),
        _fold_half((-1, 0, 0), gamma, z_pole, R, d1, image_angle, (0, 1, 0),
                   3.25 * rc),
    ]
    for h in halves:
        for (cx, cy) in _hex_centers(rc, 4, 7):
            if meshed:
                tris, nrm = _mesh_hex(h.center, R, h.axis, h.e1, h.e2, cx, cy,
                                      rc, gap, hex_subdiv)
                b.triangles(tris, nrm, m_sph, smooth=True)
            else:
                b.sphere(center=h.center, radius=R, axis=h.axis, e1=h.e1,
                         e2=h.e2, material=m_sph, cos_min=0.5,
                         edges=_hex_edges(cx, cy, rc, gap))
        fw, fh = flat_size
        fu, fv, cells = h.flat_u, h.flat_v, (64, 40)
        outward = 1.0 if np.dot(fv, h.det_normal) < 0 else -1.0
        f_origin = (h.flat_center + outward * flat_shift * fv - fw / 2 * fu
                    - fh / 2 * fv)
        if meshed:
            b.triangles(_mesh_rectangle(f_origin, fu, fv, fw, fh, *cells),
                        None, m_flat, smooth=False)
        else:
            b.rect(origin=f_origin, u_axis=fu, v_axis=fv, width=fw,
                   height=fh, material=m_flat)
    # support plate behind the mirror, facing the radiator (normal -z)
    side = 2300.0
    origin = np.array([side / 2, -side / 2, z_pole + 300.0])
    u_ax, v_ax = np.array([-1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    if meshed:
        b.triangles(_mesh_rectangle(origin, u_ax, v_ax, side, side, 122, 122),
                    None, m_abs, smooth=False)
    else:
        b.rect(origin=origin, u_axis=u_ax, v_axis=v_ax, width=side,
               height=side, material=m_abs)
    for i, h in enumerate(halves):
        _add_detector(b, h, m_det[i], 512, PIXEL_PITCH)
    return b.build()


# ------------------------------------------------------------------ tracks
@dataclasses.dataclass
class Tracks:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    dz: np.ndarray
    p: np.ndarray
    mass: np.ndarray
    length: np.ndarray
    event: np.ndarray
    id: np.ndarray
    n_fixed: np.ndarray | None = None

    FIELDS = ("x", "y", "z", "dx", "dy", "dz", "p", "mass", "length")

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subset(self, sel) -> "Tracks":
        kw = {f: getattr(self, f)[sel] for f in self.FIELDS + ("event", "id")}
        kw["n_fixed"] = None if self.n_fixed is None else self.n_fixed[sel]
        return Tracks(**kw)

    def nbytes(self) -> int:
        n = 9 * 4 + 2 * 4 + (4 if self.n_fixed is not None else 0)
        return n * self.n


def _make_tracks(n, origin, dirs, p, mass, length, event, tid, n_fixed=None):
    o = np.broadcast_to(np.asarray(origin, np.float64), (n, 3))
    return Tracks(x=f32(o[:, 0]), y=f32(o[:, 1]), z=f32(o[:, 2]),
                  dx=f32(dirs[:, 0]), dy=f32(dirs[:, 1]), dz=f32(dirs[:, 2]),
                  p=f32(p), mass=f32(mass), length=f32(length),
                  event=np.asarray(event, np.uint32),
                  id=np.asarray(tid, np.uint32),
                  n_fixed=None if n_fixed is None
                  else np.asarray(n_fixed, np.uint32))


def point_source_tracks(n_photons=100_000) -> Tracks:
    """A single massless 'track' of zero length at the origin pointing along
    +z: a point source at the mirror's centre of curvature emitting
    n_photons photons on the beta = 1 Cherenkov cone."""
    return _make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]),
                        p=np.array([1.0e6]), mass=np.array([0.0]),
                        length=np.array([0.0]), event=[0], tid=[0],
                        n_fixed=[n_photons])


def muon_point_tracks(n_photons=600_000, p_gev=100.0) -> Tracks:
    """One muon of p_gev GeV/c (m = 105.66 MeV) of zero length at the origin
    pointing along +z, emitting a fixed n_photons on its Cherenkov cone: the
    paper-scale point source (one 100 GeV muon, ~6e5 photons)."""
    return _make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]),
                        p=np.array([p_gev]), mass=np.array([MUON_MASS]),
                        length=np.array([0.0]), event=[0], tid=[0],
                        n_fixed=[n_photons])


def _cone_dirs(rng, n, max_angle):
    """Directions uniform in solid angle within max_angle of +z."""
    cos_t = 1.0 - rng.random(n) * (1.0 - math.cos(max_angle))
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * rng.random(n)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def pion_tracks(n, seed=0, length=1000.0, max_angle=0.25, p_min=2.0,
                p_max=100.0, event=0, n_fixed=None) -> Tracks:
    """n pion tracks from the origin: momentum log-uniform in
    [p_min, p_max] GeV/c, direction uniform in solid angle within max_angle
    of +z, emitting along `length` mm of radiator."""
    rng = np.random.default_rng(seed)
    p = p_min * (p_max / p_min) ** rng.random(n)
    dirs = _cone_dirs(rng, n, max_angle)
    nf = None if n_fixed is None else np.full(n, n_fixed)
    return _make_tracks(n, (0.0, 0.0, 0.0), dirs, p, np.full(n, PION_MASS),
                        np.full(n, length), np.full(n, event), np.arange(n),
                        nf)


def batched_tracks(n_events=4096, mean_tracks=50.0, seed=0, length=1000.0,
                   max_angle=0.25) -> Tracks:
    """Events with Poisson(mean_tracks) pion tracks each (same spectrum as
    pion_tracks); track ids restart at 0 in every event."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(mean_tracks, n_events)
    n = int(counts.sum())
    p = 2.0 * 50.0 ** rng.random(n)
    dirs = _cone_dirs(rng, n, max_angle)
    event = np.repeat(np.arange(n_events), counts)
    starts = np.repeat(np.cumsum(counts) - counts, counts)
    tid = np.arange(n) - starts
    return _make_tracks(n, (0.0, 0.0, 0.0), dirs, p, np.full(n, PION_MASS),
                        np.full(n, length), event, tid)


# ---------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    tracks: Tracks
    n_minus_1: float
    lambda_min: float = 200.0
    lambda_max: float = 600.0
    seed: int = 0
    description: str = ""
    source: int = SOURCE_CHERENKOV
    yield_per_mm: float = 0.0         # isotropic source: mean photons per mm
    spectrum_table: int = -1          # isotropic source: CDF table index
    dispersion: tuple | None = None   # (a nm^-2, lambda0 nm): n - 1 = a/(1/l0^2 - 1/l^2)


def point_source(n_photons=100_000, meshed=False) -> Workload:
    return Workload("point_source_meshed" if meshed else "point_source",
                    point_source_scene(meshed=meshed),
                    point_source_tracks(n_photons), n_minus_1=0.0014,
                    description=f"{n_photons} photons from the centre of "
                    "curvature of an R=2710 mm sphere"
                    + (" (smooth-normal triangle mesh)" if meshed else "")
                    + ", n=1.0014, beta=1")


def point_source_muon(n_photons=600_000) -> Workload:
    return Workload("point_source_muon", point_source_scene(),
                    muon_point_tracks(n_photons), n_minus_1=0.0014,
                    description=f"{n_photons} photons from one 100 GeV/c muon at the "
                    "centre of curvature of an R=2710 mm sphere, n=1.0014")


def two_mirror(n_photons=20_000) -> Workload:
    return Workload("two_mirror", two_mirror_scene(), point_source_tracks(n_photons),
                    n_minus_1=0.0014, description=f"{n_photons} photons from a point "
                    "through a periscope of two tilted analytic tiles")


def rich1(n_tracks=1000, seed=0, meshed=True) -> Workload:
    return Workload("rich1", rich1_scene(meshed=meshed),
                    pion_tracks(n_tracks, seed=seed), n_minus_1=0.0014,
                    seed=seed, description=f"{n_tracks} pion tracks, 1000 mm "
                    "C4F10 (n=1.0014), 4-tile R=2710 mm mirror + 2 flats, "
                    "3 x 256^2 planes")


def batched(n_events=4096, seed=0) -> Workload:
    return Workload("batched", rich1_scene(meshed=True),
                    batched_tracks(n_events, seed=seed), n_minus_1=0.0014,
                    seed=seed, description=f"{n_events} events, Poisson(50) "
                    "pion tracks per event, RICH1-like meshed geometry")


def rich2(n_tracks=330_000, seed=0, meshed=True) -> Workload:
    return Workload("rich2", rich2_scene(meshed=meshed),
                    pion_tracks(n_tracks, seed=seed, length=2000.0,
                                max_angle=0.15),
                    n_minus_1=0.0005, seed=seed,
                    description=f"{n_tracks} pion tracks, 2000 mm CF4 "
                    "(n=1.0005), 56 hex tiles R=8600 mm + flats + support, "
                    "2 x 512^2 planes")


# ------------------------------------------------------------- ring targets
def ring_targets(n_tracks, n_planes, track_index, plane, u, v, min_hits=10):
    """Expected ring of every (track, plane) from a set of hits: the
    algebraic least-squares circle (Kasa's fit: u^2 + v^2 + D u + E v + F
    = 0 solved linearly, centre (-D/2, -E/2), radius sqrt(|c|^2 - F)),
    which recovers centre and radius from partial arcs; weight 1 when at
    least min_hits hits define it, else 0. Returns float32
    [n_tracks][n_planes][4] = (cu, cv, r, weight), the targets of the soft
    ring chi^2."""
    out = np.zeros((n_tracks, n_planes, 4), np.float64)
    key = np.asarray(track_index, np.int64) * n_planes + np.asarray(plane, np.int64)
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    order = np.argsort(key, kind="stable")
    ks, us, vs = key[order], u[order], v[order]
    bounds = np.flatnonzero(np.diff(ks)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [len(ks)]])
    flat = out.reshape(-1, 4)
    for a, b in zip(starts, ends):
        if b - a < min_hits:
            continue
        uu, vv = us[a:b], vs[a:b]
        mu, mv = uu.mean(), vv.mean()          # centre the fit for conditioning
        x, y = uu - mu, vv - mv
        A = np.stack([x, y, np.ones_like(x)], axis=1)
        rhs = -(x * x + y * y)
        (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
        cx, cy = -D / 2.0, -E / 2.0
        r2 = cx * cx + cy * cy - F
        if not (r2 > 0.0):
            continue
        flat[ks[a], :] = (cx + mu, cy + mv, np.sqrt(r2), 1.0)
    return out.astype(np.float32)


def adjoint_workload(n_tracks=200, photons_per_track=5000, seed=0) -> Workload:
    """The gradient configuration: the RICH1-like geometry with analytic
    tiles and flat mirrors, n_tracks pion tracks with a fixed photon count
    each (1e6 photons by default); momenta from 3 GeV/c so every track is
    above the 2.64 GeV/c Cherenkov threshold of C4F10."""
    return Workload("adjoint", rich1_scene(meshed=False),
                    pion_tracks(n_tracks, seed=seed, n_fixed=photons_per_track, p_min=3.0),
                    n_minus_1=0.0014, seed=seed,
                    description=f"{n_tracks} pion tracks x {photons_per_track} photons, "
                    "RICH1-like analytic geometry, 10 parameters")


def nominal_theta(scene, n_minus_1):
    """Parameters at the nominal geometry: tilts 0, the tiles' radius of
    curvature, n - 1 (as the FP32 inputs hold them)."""
    th = np.zeros(10)
    th[8] = float(scene.spheres[0]["radius"]) if len(scene.spheres) else 0.0
    th[9] = float(np.float32(n_minus_1))
    return th


# ------------------------------------------- other light sources (Sec. 6)
# Sec. 6 names water Cherenkov detectors and scintillation light in liquid
# noble-gas detectors as the next light sources. Two synthetic stand-ins:

# Wavelength-shifted scintillation light (TPB-like emission, peak near
# 425 nm), 20 bins of 15 nm from 350 nm (synthetic shape).
SCINT_LAMBDA0, SCINT_WIDTH = 350.0, 15.0
SCINT_WEIGHTS = [math.exp(-0.5 * ((350.0 + 15.0 * (k + 0.5) - 425.0) / 30.0) ** 2)
                 for k in range(20)]
# Specular wall reflectivity of the scintillator box, 25 nm bins over
# 300-700 nm (synthetic shape).
WALL_LAMBDA0, WALL_WIDTH = 300.0, 25.0
WALL_R = [0.97 - 0.0025 * k for k in range(16)]


def _box_walls(b, half, material_for_face, n_pix):
    """Six inward-facing faces of the cube [-half, half]^3; faces 0/1 are
    z = -half / z = +half (detector planes of n_pix^2 pixels when their
    material is a detector), 2..5 the side walls."""
    side = 2.0 * half
    pitch = side / n_pix
    faces = [
        ((-half, -half, -half), (1, 0, 0), (0, 1, 0)),    # z = -half, normal +z
        ((-half, half, half), (1, 0, 0), (0, -1, 0)),     # z = +half, normal -z
        ((-half, -half, -half), (0, 1, 0), (0, 0, 1)),    # x = -half, normal +x
        ((half, half, -half), (0, -1, 0), (0, 0, 1)),     # x = +half, normal -x
        ((half, -half, -half), (-1, 0, 0), (0, 0, 1)),    # y = -half, normal +y
        ((-half, half, -half), (1, 0, 0), (0, 0, 1)),     # y = +half, normal -y
    ]
    for k, (o, u, v) in enumerate(faces):
        m = material_for_face(k)
        det = b.materials[m]["kind"] == MAT_DETECTOR
        b.rect(origin=o, u_axis=u, v_axis=v, width=side, height=side, material=m,
               nx=n_pix if det else 0, ny=n_pix if det else 0, pitch=pitch if det else 0.0)


def scint_box_scene(half=500.0, n_pix=256) -> Scene:
    """Liquid-argon-like scintillator volume (synthetic): the cube
    [-500, 500]^3 mm with photodetector planes of 256^2 pixels
    (3.90625 mm) on the top and bottom faces and specular reflecting side
    walls, so photons reach the planes after up to several reflections.
    Tables: 0 QE, 1 wall reflectivity, 2 emission spectrum (CDF)."""
    b = _Builder("scint_box")
    t_qe = b.table_hist(QE_LAMBDA0, QE_WIDTH, QE_BINS)
    t_wall = b.table_hist(WALL_LAMBDA0, WALL_WIDTH, WALL_R)
    b.table_cdf(SCINT_LAMBDA0, SCINT_WIDTH, SCINT_WEIGHTS)
    m_wall = b.material(MAT_MIRROR, t_wall)
    m_det = [b.material(MAT_DETECTOR, t_qe, plane=i) for i in range(2)]
    _box_walls(b, half, lambda k: m_det[k] if k < 2 else m_wall, n_pix)
    return b.build()


def scint_tracks(n, seed=0, length=100.0, inner=350.0, event=0) -> Tracks:
    """n straight segments of `length` mm starting uniformly in the cube
    [-inner, inner]^3, isotropic directions (they stay inside the box for
    inner + length < 500)."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(-inner, inner, (n, 3))
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(1.0 - ct * ct)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    t = _make_tracks(n, (0.0, 0.0, 0.0), d, np.full(n, 1.0), np.full(n, MUON_MASS),
                     np.full(n, length), np.full(n, event), np.arange(n))
    t.x, t.y, t.z = f32(o[:, 0]), f32(o[:, 1]), f32(o[:, 2])
    return t


def scintillation(n_tracks=200, seed=0, yield_per_mm=20.0) -> Workload:
    """Isotropic scintillation light from n_tracks 100 mm segments inside
    the scintillator box, yield_per_mm photons per mm (Poisson), the
    binned emission spectrum of the scene (~4e5 photons for 200 tracks)."""
    return Workload("scintillation", scint_box_scene(), scint_tracks(n_tracks, seed=seed),
                    n_minus_1=0.0, lambda_min=SCINT_LAMBDA0,
                    lambda_max=SCINT_LAMBDA0 + SCINT_WIDTH * len(SCINT_WEIGHTS),
                    seed=seed, source=SOURCE_ISOTROPIC, yield_per_mm=yield_per_mm,
                    spectrum_table=2,
                    description=f"{n_tracks} x 100 mm segments, isotropic emission, "
                    f"{yield_per_mm} photons/mm, 1 m scintillator box, mirror side walls")


def water_tank_scene(half=2000.0, n_pix=256) -> Scene:
    """Water Cherenkov tank (synthetic): the cube [-2000, 2000]^3 mm with
    all six faces photodetector planes of 256^2 pixels (15.625 mm).
    Tables: 0 QE."""
    b = _Builder("water_tank")
    t_qe = b.table_hist(QE_LAMBDA0, QE_WIDTH, QE_BINS)
    m_det = [b.material(MAT_DETECTOR, t_qe, plane=i) for i in range(6)]
    _box_walls(b, half, lambda k: m_det[k], n_pix)
    return b.build()


def water_muons(n, seed=0, length=2000.0, max_angle=0.3, event=0) -> Tracks:
    """n through-going muons entering near the top of the tank and heading
    down within max_angle of -z, p log-uniform 1-20 GeV/c, emitting along
    `length` mm."""
    rng = np.random.default_rng(seed)
    p = 1.0 * 20.0 ** rng.random(n)
    d = _cone_dirs(rng, n, max_angle)
    d[:, 2] = -d[:, 2]
    o = np.stack([rng.uniform(-600, 600, n), rng.uniform(-600, 600, n),
                  np.full(n, 1500.0)], axis=1)
    t = _make_tracks(n, (0.0, 0.0, 0.0), d, p, np.full(n, MUON_MASS), np.full(n, length),
                     np.full(n, event), np.arange(n))
    t.x, t.y, t.z = f32(o[:, 0]), f32(o[:, 1]), f32(o[:, 2])
    return t


def water(n_tracks=10, seed=0) -> Workload:
    """Cherenkov light of muons in water (n = 1.33, theta ~ 41 degrees,
    ~33 photons/mm over 300-600 nm): ~6.6e5 photons for 10 tracks."""
    return Workload("water", water_tank_scene(), water_muons(n_tracks, seed=seed),
                    n_minus_1=0.33, lambda_min=300.0, lambda_max=600.0, seed=seed,
                    description=f"{n_tracks} muons, 2000 mm of water, 4 m tank of detector walls")


# ------------------------------------------------- dispersive radiator
# Single-resonance form n(lambda) - 1 = a / (1/lambda0^2 - 1/lambda^2)
# (lambda in nm) with parameters chosen for a C4F10-like gas: n - 1 =
# 1.59e-3 at 200 nm, 1.42e-3 at 400 nm, 1.40e-3 at 600 nm (synthetic).
C4F10_DISPERSION = (float(np.float32(2.5324e-7)), float(np.float32(73.7)))


def rich1_dispersive(n_tracks=1000, seed=0, meshed=True) -> Workload:
    """The RICH1-like workload with a dispersive radiator: each photon's
    Cherenkov angle follows n(lambda) of its own wavelength, the yield is
    the Frank-Tamm integral of sin^2 theta(lambda), and the wavelength law
    is sin^2 theta(lambda) / lambda^2."""
    wl = rich1(n_tracks, seed=seed, meshed=meshed)
    wl.name = "rich1_dispersive"
    wl.dispersion = C4F10_DISPERSION
    wl.description += ", dispersive n(lambda)"
    return wl


def rich1_windows(n_tracks=1000, seed=0, meshed=True) -> Workload:
    """The RICH1-like workload with 6 mm quartz windows 20 mm in front of the
    two focal planes: photons refract into and out of each window (Snell's
    law with the wavelength-dependent index of the window)."""
    wl = rich1(n_tracks, seed=seed, meshed=meshed)
    wl.scene = rich1_scene(meshed=meshed, windows=True)
    wl.name = "rich1_windows"
    wl.description += ", quartz windows"
    return wl


def _slab(b, z_lo, z_hi, half, material):
    """Slab z_lo <= z <= z_hi: two faces whose normals point away from the
    glass (the material's index applies behind each face)."""
    b.rect(origin=(-half, -half, z_hi), u_axis=(1, 0, 0), v_axis=(0, 1, 0), width=2 * half,
           height=2 * half, material=material)                      # normal +z
    b.rect(origin=(-half, half, z_lo), u_axis=(1, 0, 0), v_axis=(0, -1, 0), width=2 * half,
           height=2 * half, material=material)                      # normal -z


def slab_ring_scene() -> Scene:
    """A 30 mm quartz slab (900 < z < 930) before a plane at z = 1000 (256^2
    pixels of 10 mm, QE = 1): a point source at the origin along +z rings
    the plane at 970 tan(theta) + 30 tan(theta_r)."""
    b = _Builder("slab_ring")
    t_qe = b.table_const(1.0)
    t_n = b.table_hist(QUARTZ_LAMBDA0, QUARTZ_WIDTH, QUARTZ_N)
    m_det = b.material(MAT_DETECTOR, t_qe, plane=0)
    m_glass = b.material(MAT_DIELECTRIC, t_n)
    _slab(b, 900.0, 930.0, 2000.0, m_glass)
    b.rect(origin=(-1280.0, 1280.0, 1000.0), u_axis=(1, 0, 0), v_axis=(0, -1, 0), width=2560.0,
           height=2560.0, material=m_det, nx=256, ny=256, pitch=10.0)
    return b.build()


def slab_tir_scene(n_glass=1.5) -> Scene:
    """A 6 mm slab of index n_glass (-3 < z < 3, 4 m wide) between two
    photodetector planes at z = +-10 (256^2 pixels of 16 mm, QE = 1): an
    isotropic source inside escapes only below the critical angle."""
    b = _Builder("slab_tir")
    t_qe = b.table_const(1.0)
    t_n = b.table_const(n_glass)
    m_det = [b.material(MAT_DETECTOR, t_qe, plane=i) for i in range(2)]
    m_glass = b.material(MAT_DIELECTRIC, t_n)
    _slab(b, -3.0, 3.0, 2000.0, m_glass)
    b.rect(origin=(-2048.0, 2048.0, 10.0), u_axis=(1, 0, 0), v_axis=(0, -1, 0), width=4096.0,
           height=4096.0, material=m_det[0], nx=256, ny=256, pitch=16.0)
    b.rect(origin=(-2048.0, -2048.0, -10.0), u_axis=(1, 0, 0), v_axis=(0, 1, 0), width=4096.0,
           height=4096.0, material=m_det[1], nx=256, ny=256, pitch=16.0)
    return b.build()


def point_track(n_photons, p=1e6, mass=0.0) -> Tracks:
    """One zero-length track at the origin along +z with a fixed count."""
    return _make_tracks(1, (0.0, 0.0, 0.0), np.array([[0.0, 0.0, 1.0]]), p=[p], mass=[mass],
                        length=[0.0], event=[0], tid=[0], n_fixed=[n_photons])


def slab_ring(n_photons=5000) -> Workload:
    return Workload("slab_ring", slab_ring_scene(), point_track(n_photons), n_minus_1=0.33,
                    description="water-angle Cherenkov cone through a 30 mm quartz slab")


def slab_tir(n_photons=40000) -> Workload:
    return Workload("slab_tir", slab_tir_scene(), point_track(n_photons, p=1.0), n_minus_1=0.0,
                    source=SOURCE_ISOTROPIC,
                    description="isotropic source inside a 6 mm slab of index 1.5")
