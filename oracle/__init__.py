"""FP64 CPU oracle of the Cherenkov photon propagator -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the C-ABI library
and its Python binding) never does.

The oracle is a plain C program (``rich_oracle.c``) compiled on demand with
gcc; this module marshals the seeded synthetic inputs into its records and
returns its results as numpy arrays. What each oracle function follows in
the paper is stated in the C file's header.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rich_oracle.c")
_LIB = os.path.join(_HERE, "librich_oracle.so")
_lock = threading.Lock()
_lib = None

FATE_NAMES = ["none", "escaped", "mirror_absorbed", "absorbed", "qe_rejected",
              "detected", "max_bounces", "max_steps", "prefiltered"]
FATE_DETECTED = 5
FATE_PREFILTERED = 8


def build(force: bool = False) -> str:
    """Compile the oracle into librich_oracle.so (gcc, OpenMP, no FP
    contraction so FP32 decision arithmetic is one IEEE operation at a
    time)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The compiled oracle. RICH_ORACLE_LIB names another build of the same
    source to load instead (the mutation tests load a copy with one step
    deliberately broken, to show that a pin catches it)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(os.environ.get("RICH_ORACLE_LIB") or build())
            _declare(_lib)
        return _lib


# ------------------------------------------------------------------ records
class SceneIn(C.Structure):
    _fields_ = [("n_tables", C.c_int32), ("n_materials", C.c_int32),
                ("n_spheres", C.c_int32), ("n_rects", C.c_int32),
                ("n_triangles", C.c_int64),
                ("tables", C.c_void_p), ("materials", C.c_void_p),
                ("spheres", C.c_void_p), ("rects", C.c_void_p),
                ("tri_v", C.c_void_p), ("tri_n", C.c_void_p),
                ("tri_m", C.c_void_p), ("tri_s", C.c_void_p)]


class TracksIn(C.Structure):
    _fields_ = [("n", C.c_int64)] + [
        (f, C.c_void_p) for f in ("x", "y", "z", "dx", "dy", "dz", "p",
                                  "mass", "length", "event", "id", "n_fixed")]


class Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_minus_1", C.c_double),
                ("lambda_min", C.c_float), ("lambda_max", C.c_float),
                ("max_bounces", C.c_int32), ("max_steps", C.c_int32),
                ("t_min", C.c_double), ("eps", C.c_double),
                ("prob_eps", C.c_double), ("use_bvh", C.c_int32),
                ("n_threads", C.c_int32), ("n_prefilter", C.c_int32),
                ("prefilter_tables", C.c_int32 * 4), ("source", C.c_int32),
                ("yield_per_mm", C.c_float), ("spectrum", C.c_void_p),
                ("dispersion", C.c_int32), ("disp_a", C.c_float),
                ("disp_lambda0", C.c_float)]


class PhotonOut(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in (
        "fate", "plane", "ix", "iy", "u", "v", "lambda_", "n_refl", "graze",
        "path", "dir_out", "pos_out", "pixel_counts", "event_sums")] + [
        ("n_hist_events", C.c_int64)]


def _declare(L):
    vp, i64, u32 = C.c_void_p, C.c_int64, C.c_uint32
    L.oracle_philox.argtypes = [vp, vp, vp]
    L.oracle_philox_batch.argtypes = [i64, vp, vp, vp]
    L.oracle_yield_per_mm.argtypes = [C.c_double] * 4
    L.oracle_yield_per_mm.restype = C.c_double
    L.oracle_disp_yield_per_mm.argtypes = [vp, C.c_double, C.c_double]
    L.oracle_disp_yield_per_mm.restype = C.c_double
    L.oracle_poisson.argtypes = [C.c_double, C.c_uint64, u32, u32]
    L.oracle_poisson.restype = i64
    L.oracle_yield.argtypes = [vp, vp, vp, vp, vp]
    L.oracle_yield.restype = i64
    L.oracle_emit.argtypes = [vp, vp, i64, u32, vp, vp, vp]
    L.oracle_scene_create.argtypes = [vp, C.c_int]
    L.oracle_scene_create.restype = vp
    L.oracle_scene_destroy.argtypes = [vp]
    L.oracle_scene_n_nodes.argtypes = [vp]
    L.oracle_scene_n_nodes.restype = C.c_int
    L.oracle_scene_pixels_per_event.argtypes = [vp]
    L.oracle_scene_pixels_per_event.restype = i64
    L.oracle_raycast.argtypes = [vp, i64, vp, vp, vp, C.c_double, C.c_int,
                                 vp, vp]
    L.oracle_probe.argtypes = [vp, i64, vp, vp, vp, C.c_double, C.c_double, vp, vp,
                               vp, vp, vp, vp]
    L.oracle_trace_photons.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]
    L.oracle_trace_photons.restype = C.c_int
    L.oracle_table_eval.argtypes = [vp, C.c_int, C.c_float]
    L.oracle_table_eval.restype = C.c_float
    L.oracle_trace.argtypes = [vp, vp, vp, vp, i64, i64, vp]
    L.oracle_trace.restype = C.c_int
    L.oracle_max_threads.restype = C.c_int
    L.oracle_trace_grad.argtypes = [vp, vp, vp, vp, vp, C.c_int, C.c_double, C.c_double,
                                    C.c_double, vp, vp, vp]
    L.oracle_trace_grad.restype = i64
    L.oracle_trace_at.argtypes = [vp, vp, vp, vp, vp, vp]
    L.oracle_trace_at.restype = C.c_int
    L.oracle_hit_jacobian.argtypes = [vp, vp, vp, vp, i64, u32, vp, vp, vp, vp]
    L.oracle_hit_jacobian.restype = C.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data


# ------------------------------------------------------------------- API
def philox(counters, key):
    """Philox4x32-10 of an (n, 4) uint32 counter array under a 2-word key."""
    ctr = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().oracle_philox_batch(len(ctr), _ptr(ctr), _ptr(k), _ptr(out))
    return out


def yield_per_mm(n_minus_1, beta, lam_min=200.0, lam_max=600.0):
    return lib().oracle_yield_per_mm(n_minus_1, beta, lam_min, lam_max)


def disp_yield_per_mm(prm, p, m):
    """Frank-Tamm photons per mm of the dispersive radiator of prm for a
    particle of momentum p and mass m."""
    return lib().oracle_disp_yield_per_mm(C.byref(prm), p, m)


def poisson(mu, seed=0, event=0, track=0):
    return int(lib().oracle_poisson(mu, seed, event, track))


class _TracksHold:
    """Keeps contiguous copies of the track arrays alive for a call."""

    def __init__(self, tracks):
        self.arrs = {}
        for f in ("x", "y", "z", "dx", "dy", "dz", "p", "mass", "length"):
            self.arrs[f] = np.ascontiguousarray(getattr(tracks, f), np.float32)
        self.arrs["event"] = np.ascontiguousarray(tracks.event, np.uint32)
        self.arrs["id"] = np.ascontiguousarray(tracks.id, np.uint32)
        self.arrs["n_fixed"] = (None if tracks.n_fixed is None else
                                np.ascontiguousarray(tracks.n_fixed, np.uint32))
        self.rec = TracksIn(n=tracks.n, **{k: _ptr(v) for k, v in self.arrs.items()})


def params(workload=None, seed=None, n_minus_1=None, lambda_min=None,
           lambda_max=None, max_bounces=8, max_steps=16, t_min=1e-3,
           eps=1e-3, prob_eps=1e-6, use_bvh=True, n_threads=0, prefilter=()):
    """Oracle parameters; radiator and seed default to the workload's.
    prefilter: indices of the scene tables whose product is applied as one
    accept/reject before propagation (Sec. 4.3); empty: in flight."""
    w = workload
    # n - 1 and the band are FP32 inputs of the propagator: promote exactly
    nm1 = float(np.float32(n_minus_1 if n_minus_1 is not None else w.n_minus_1))
    # light source: Cherenkov, or isotropic with a yield per mm and a binned
    # spectrum taken from the scene's tables (a CDF table)
    source = int(getattr(w, "source", 0)) if w is not None else 0
    spec = None
    st = int(getattr(w, "spectrum_table", -1)) if w is not None else -1
    if source == 1 and st >= 0:
        spec = np.ascontiguousarray(w.scene.tables[st:st + 1])
    prm = Params(seed=int(seed if seed is not None else w.seed),
                  n_minus_1=nm1,
                  lambda_min=lambda_min if lambda_min is not None else w.lambda_min,
                  lambda_max=lambda_max if lambda_max is not None else w.lambda_max,
                  max_bounces=max_bounces, max_steps=max_steps, t_min=t_min,
                  eps=eps, prob_eps=prob_eps, use_bvh=int(use_bvh),
                  n_threads=n_threads, n_prefilter=len(prefilter),
                  prefilter_tables=(C.c_int32 * 4)(*(list(prefilter) + [0] * (4 - len(prefilter)))),
                  source=source,
                  yield_per_mm=float(getattr(w, "yield_per_mm", 0.0)) if w is not None else 0.0,
                  spectrum=None if spec is None else spec.ctypes.data,
                  dispersion=int(getattr(w, "dispersion", None) is not None) if w is not None else 0,
                  disp_a=float(w.dispersion[0]) if w is not None and getattr(w, "dispersion", None) else 0.0,
                  disp_lambda0=float(w.dispersion[1]) if w is not None and getattr(w, "dispersion", None) else 0.0)
    prm._keep = spec
    return prm


def track_yield(tracks, prm):
    """Per-track photon counts, Frank-Tamm means and photon offsets."""
    h = _TracksHold(tracks)
    n = np.empty(tracks.n, np.uint32)
    mu = np.empty(tracks.n, np.float64)
    off = np.empty(tracks.n + 1, np.uint64)
    lib().oracle_yield(C.byref(h.rec), C.byref(prm), _ptr(n), _ptr(mu),
                       _ptr(off))
    return n, mu, off


def emit(tracks, prm, track, photon):
    """Origin (mm), unit direction and wavelength (nm) of one photon."""
    h = _TracksHold(tracks)
    o = np.empty(3)
    d = np.empty(3)
    lam = np.empty(1, np.float32)
    lib().oracle_emit(C.byref(h.rec), C.byref(prm), track, photon, _ptr(o),
                      _ptr(d), _ptr(lam))
    return o, d, float(lam[0])


class Scene:
    """The oracle's FP64 copy of a scene plus its median-split BVH."""

    def __init__(self, scene, leaf_size=4):
        self.src = scene
        self._keep = [np.ascontiguousarray(scene.tables),
                      np.ascontiguousarray(scene.materials),
                      np.ascontiguousarray(scene.spheres),
                      np.ascontiguousarray(scene.rects),
                      np.ascontiguousarray(scene.tri_vertices, np.float32),
                      None if scene.tri_normals is None else
                      np.ascontiguousarray(scene.tri_normals, np.float32),
                      np.ascontiguousarray(scene.tri_material, np.int32),
                      None if scene.tri_surface is None else
                      np.ascontiguousarray(scene.tri_surface, np.int32)]
        k = self._keep
        rec = SceneIn(n_tables=len(k[0]), n_materials=len(k[1]),
                      n_spheres=len(k[2]), n_rects=len(k[3]),
                      n_triangles=scene.n_triangles, tables=_ptr(k[0]),
                      materials=_ptr(k[1]), spheres=_ptr(k[2]),
                      rects=_ptr(k[3]), tri_v=_ptr(k[4]), tri_n=_ptr(k[5]),
                      tri_m=_ptr(k[6]), tri_s=_ptr(k[7]))
        self.handle = lib().oracle_scene_create(C.byref(rec), leaf_size)
        self.n_planes = len(scene.planes)
        self.pixels_per_event = int(lib().oracle_scene_pixels_per_event(self.handle))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.oracle_scene_destroy(h)
            self.handle = None

    @property
    def n_nodes(self):
        return lib().oracle_scene_n_nodes(self.handle)

    def table(self, index, lam):
        return float(lib().oracle_table_eval(self.handle, index, lam))

    def raycast(self, origins, dirs, skip=None, t_min=1e-3, use_bvh=True):
        o = np.ascontiguousarray(origins, np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        t = np.empty(len(o))
        prim = np.empty(len(o), np.int32)
        lib().oracle_raycast(self.handle, len(o), _ptr(o), _ptr(d), _ptr(sk),
                             t_min, int(use_bvh), _ptr(t), _ptr(prim))
        return t, prim

    def probe(self, origins, dirs, skip=None, t_min=1e-3, eps=1e-3):
        """Nearest hit of each ray with the normals at the hit: returns a dict
        of prim (-1: none), t, n_geo, n_shade (the normal the reflection
        uses), graze (bits of the nearest-hit decision; 8: the skipped
        surface would have been nearer) and skipped_t (nearest hit on the
        skipped surface, inf if none)."""
        o = np.ascontiguousarray(origins, np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
        n = len(o)
        sk = None if skip is None else np.ascontiguousarray(skip, np.int32)
        out = {"prim": np.empty(n, np.int32), "t": np.empty(n), "n_geo": np.empty((n, 3)),
               "n_shade": np.empty((n, 3)), "graze": np.empty(n, np.int32),
               "skipped_t": np.empty(n)}
        lib().oracle_probe(self.handle, n, _ptr(o), _ptr(d), _ptr(sk), t_min, eps,
                           _ptr(out["prim"]), _ptr(out["t"]), _ptr(out["n_geo"]),
                           _ptr(out["n_shade"]), _ptr(out["graze"]), _ptr(out["skipped_t"]))
        return out

    def grad(self, tracks, prm, theta, targets, sigma=1.0, fd=False, h_angle=1e-6,
             h_rel=1e-6):
        """Soft ring chi^2 loss at theta (10 parameters: 8 tile tilts, the
        radius of curvature, n - 1), its dual-number gradient and, with fd,
        its central-difference gradient. targets: float32 [n_tracks][n_planes][4]
        = (cu, cv, r, weight). Returns (loss, grad, grad_fd or None, n_used)."""
        h = _TracksHold(tracks)
        th = np.ascontiguousarray(theta, np.float64).reshape(10)
        tg = np.ascontiguousarray(targets, np.float32)
        g = np.zeros(10)
        gfd = np.zeros(10) if fd else None
        loss = np.zeros(1)
        used = lib().oracle_trace_grad(self.handle, C.byref(h.rec), C.byref(prm), _ptr(th),
                                       _ptr(tg), self.n_planes, sigma, h_angle, h_rel,
                                       _ptr(loss), _ptr(g), _ptr(gfd))
        if used < 0:
            raise ValueError("oracle_trace_grad rejected its parameters")
        return float(loss[0]), g, gfd, int(used)

    def hit_jacobian(self, tracks, prm, theta, track, photon):
        """(fate, u, v, du/dtheta[10], dv/dtheta[10]) of one photon at theta."""
        h = _TracksHold(tracks)
        th = np.ascontiguousarray(theta, np.float64).reshape(10)
        u, v = np.zeros(1), np.zeros(1)
        du, dv = np.zeros(10), np.zeros(10)
        fate = lib().oracle_hit_jacobian(self.handle, C.byref(h.rec), C.byref(prm), _ptr(th),
                                         int(track), int(photon), _ptr(u), _ptr(v), _ptr(du),
                                         _ptr(dv))
        return int(fate), float(u[0]), float(v[0]), du, dv

    def trace_at(self, tracks, prm, theta, n_hist_events=None):
        """Per-photon results of the forward trace at theta."""
        th = np.ascontiguousarray(theta, np.float64).reshape(10)
        p2 = Params(**{f: getattr(prm, f) for f, _ in Params._fields_})
        p2.n_minus_1 = float(th[9])
        _, _, off = track_yield(tracks, p2)
        n = int(off[-1])
        h = _TracksHold(tracks)
        out = {k: np.zeros(n, dt) for k, dt in (("fate", np.uint8), ("ix", np.int32),
                                                ("iy", np.int32), ("u", np.float64),
                                                ("v", np.float64), ("lambda", np.float32),
                                                ("n_refl", np.uint8), ("graze", np.uint8))}
        out["plane"] = np.full(n, -1, np.int32)
        rec = PhotonOut(fate=_ptr(out["fate"]), plane=_ptr(out["plane"]), ix=_ptr(out["ix"]),
                        iy=_ptr(out["iy"]), u=_ptr(out["u"]), v=_ptr(out["v"]),
                        lambda_=_ptr(out["lambda"]), n_refl=_ptr(out["n_refl"]),
                        graze=_ptr(out["graze"]), n_hist_events=0)
        rc = lib().oracle_trace_at(self.handle, C.byref(h.rec), C.byref(p2), _ptr(th),
                                   _ptr(np.ascontiguousarray(off, np.uint64)), C.byref(rec))
        if rc != 0:
            raise ValueError("oracle_trace_at rejected its parameters")
        out["offsets"] = off
        return out

    def _outputs(self, n, prm, n_hist_events, want_path, want_final, want_hist):
        out = {
            "fate": np.zeros(n, np.uint8), "plane": np.full(n, -1, np.int32),
            "ix": np.zeros(n, np.int32), "iy": np.zeros(n, np.int32),
            "u": np.zeros(n), "v": np.zeros(n),
            "lambda": np.zeros(n, np.float32), "n_refl": np.zeros(n, np.uint8),
            "graze": np.zeros(n, np.uint8),
        }
        if want_path:
            out["path"] = np.full((n, prm.max_steps), -1, np.int32)
        if want_final:
            out["dir"] = np.zeros((n, 3))
            out["pos"] = np.zeros((n, 3))
        if want_hist:
            out["pixel_counts"] = np.zeros(
                (n_hist_events, self.pixels_per_event), np.uint32)
            out["event_sums"] = np.zeros((n_hist_events, self.n_planes, 4))
        rec = PhotonOut(fate=_ptr(out["fate"]), plane=_ptr(out["plane"]),
                        ix=_ptr(out["ix"]), iy=_ptr(out["iy"]),
                        u=_ptr(out["u"]), v=_ptr(out["v"]),
                        lambda_=_ptr(out["lambda"]),
                        n_refl=_ptr(out["n_refl"]), graze=_ptr(out["graze"]),
                        path=_ptr(out.get("path")),
                        dir_out=_ptr(out.get("dir")),
                        pos_out=_ptr(out.get("pos")),
                        pixel_counts=_ptr(out.get("pixel_counts")),
                        event_sums=_ptr(out.get("event_sums")),
                        n_hist_events=n_hist_events if want_hist else 0)
        return out, rec

    def trace(self, tracks, prm, offsets=None, track_range=None,
              n_hist_events=None, want_path=False, want_final=False,
              want_hist=True):
        """Trace every photon of tracks[track_range] and return per-photon
        arrays indexed by global photon index (offsets from track_yield)."""
        if offsets is None:
            _, _, offsets = track_yield(tracks, prm)
        offsets = np.ascontiguousarray(offsets, np.uint64)
        tb, te = track_range if track_range is not None else (0, tracks.n)
        n = int(offsets[-1])
        h = _TracksHold(tracks)
        if n_hist_events is None:
            n_hist_events = int(tracks.event.max()) + 1 if tracks.n else 0
        out, rec = self._outputs(n, prm, n_hist_events, want_path, want_final, want_hist)
        rc = lib().oracle_trace(self.handle, C.byref(h.rec), C.byref(prm),
                                _ptr(offsets), tb, te, C.byref(rec))
        if rc != 0:
            raise ValueError("oracle_trace rejected its parameters")
        out["offsets"] = offsets
        return out

    def trace_photons(self, origin, direction, lam, event, track, photon, prm,
                      n_hist_events=None, want_path=False, want_final=False,
                      want_hist=True):
        """Trace photons given by the caller (Sec. 4.2): FP32 origins and
        directions (n, 3), FP32 wavelengths and the (event, track, photon)
        keys of their draws under prm.seed. Per-photon arrays indexed by the
        photon's position."""
        o = np.ascontiguousarray(origin, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(direction, np.float32).reshape(-1, 3)
        n = len(o)
        lam = np.ascontiguousarray(lam, np.float32).reshape(n)
        ev = np.ascontiguousarray(event, np.uint32).reshape(n)
        tk = np.ascontiguousarray(track, np.uint32).reshape(n)
        ph = np.ascontiguousarray(photon, np.uint32).reshape(n)
        if n_hist_events is None:
            n_hist_events = int(ev.max()) + 1 if n else 0
        out, rec = self._outputs(n, prm, n_hist_events, want_path, want_final, want_hist)
        rc = lib().oracle_trace_photons(self.handle, n, _ptr(o), _ptr(d), _ptr(lam), _ptr(ev),
                                        _ptr(tk), _ptr(ph), C.byref(prm), C.byref(rec))
        if rc != 0:
            raise ValueError("oracle_trace_photons rejected its parameters")
        return out


def max_threads():
    return int(lib().oracle_max_threads())
