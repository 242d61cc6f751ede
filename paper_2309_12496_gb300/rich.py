"""Python binding of the C ABI in include/rich.h (argument marshalling only).

Every step of the photon path runs in the CUDA library ``librich.so``; this
module only passes pointers and sizes. PyTorch provides device memory and
streams. Importing the module does not need a GPU; creating a context does,
and fails loudly when the library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librich.so")

RICH_OK = 0
STATUS_NAMES = {0: "RICH_OK", 1: "RICH_ERR_ARG", 2: "RICH_ERR_CUDA", 3: "RICH_ERR_OOM",
                4: "RICH_ERR_OVERFLOW", 5: "RICH_ERR_TIMEOUT", 6: "RICH_ERR_GEOMETRY",
                7: "RICH_ERR_STATE"}
PREC_FP32, PREC_REFINE64 = 0, 1
FATE_NAMES = ["none", "escaped", "mirror_absorbed", "absorbed", "qe_rejected",
              "detected", "max_bounces", "max_steps", "prefiltered"]
FATE_DETECTED = 5
FATE_PREFILTERED = 8
N_FATES = 9

EXPORTED = ["rich_create", "rich_destroy", "rich_set_stream", "rich_init_geometry",
            "rich_emit", "rich_trace", "rich_hits", "rich_philox", "rich_last_error",
            "rich_version", "rich_photon_counts_static", "rich_trace_grad",
            "rich_graph_capture", "rich_graph_launch", "rich_run_host", "rich_run_host_async",
            "rich_run_wait", "rich_set_timing", "rich_kernel_times", "rich_trace_work"]
# include/rich_peaks.h (microbenchmarks of the roofline denominators)
EXPORTED_PEAKS = ["rich_measure_peaks", "rich_peaks_last_error"]

# bytes a counters' read (rich_hits) brings back: the device counters (96 B)
# and the photon total (8 B)
COUNTERS_BYTES = 104

# rich_hit, 40 bytes
HIT_DTYPE = np.dtype([("event", "<u4"), ("track", "<u4"), ("photon", "<u4"),
                      ("plane", "u1"), ("n_reflections", "u1"), ("reserved", "<u2"),
                      ("ix", "<u2"), ("iy", "<u2"), ("lambda", "<f4"),
                      ("u", "<f8"), ("v", "<f8")])
assert HIT_DTYPE.itemsize == 40


class RichError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


# --------------------------------------------------------------- structs
class GeometryDesc(C.Structure):
    _fields_ = [("n_tables", C.c_int32), ("n_materials", C.c_int32),
                ("n_spheres", C.c_int32), ("n_rects", C.c_int32),
                ("n_triangles", C.c_int64),
                ("tables", C.c_void_p), ("materials", C.c_void_p),
                ("spheres", C.c_void_p), ("rects", C.c_void_p),
                ("tri_vertices", C.c_void_p), ("tri_normals", C.c_void_p),
                ("tri_material", C.c_void_p), ("tri_surface", C.c_void_p)]


class TracksDesc(C.Structure):
    _fields_ = [("n", C.c_int64)] + [
        (f, C.c_void_p) for f in ("x", "y", "z", "dx", "dy", "dz", "p", "mass",
                                  "length", "event", "id", "n_fixed")]


SOURCE_CHERENKOV, SOURCE_ISOTROPIC = 0, 1


class EmitParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_minus_1", C.c_float),
                ("lambda_min", C.c_float), ("lambda_max", C.c_float),
                ("reserved", C.c_float), ("source", C.c_int32),
                ("yield_per_mm", C.c_float), ("spectrum_table", C.c_int32),
                ("dispersion", C.c_int32), ("disp_a", C.c_float),
                ("disp_lambda0", C.c_float)]


_OPTS_CACHE = {}


def _host_hits(hits_host):
    """(pointer, capacity in hit records) of a host hit buffer; None reads
    the counters only."""
    if hits_host is None:
        return None, 0
    return hits_host.data_ptr(), hits_host.numel() * hits_host.element_size() // HIT_DTYPE.itemsize


def _trace_opts(seed, precision, max_bounces, max_steps, t_min, block_threads, blocks_per_sm,
                refill_min, chunk, wide_regs, bvh_smem_nodes, prefilter, wait_limit=0):
    """rich_trace_opts, one struct per distinct set of values (the library
    only reads it)."""
    key = (int(seed), precision, max_bounces, max_steps, float(t_min), block_threads,
           blocks_per_sm, refill_min, chunk, wide_regs, bvh_smem_nodes, tuple(prefilter),
           int(wait_limit))
    o = _OPTS_CACHE.get(key)
    if o is None:
        if len(_OPTS_CACHE) > 256:
            _OPTS_CACHE.clear()
        o = _OPTS_CACHE[key] = TraceOpts(
            seed=int(seed), precision=precision, max_bounces=max_bounces, max_steps=max_steps,
            t_min=t_min, block_threads=block_threads, blocks_per_sm=blocks_per_sm,
            refill_min=refill_min, chunk=chunk, wide_regs=wide_regs,
            bvh_smem_nodes=bvh_smem_nodes, wait_limit=int(wait_limit),
            **_prefilter_fields(prefilter))
    return o


def _emit_params(seed, n_minus_1, lambda_min, lambda_max, source=SOURCE_CHERENKOV,
                 yield_per_mm=0.0, spectrum_table=-1, dispersion=None):
    """rich_emit_params; dispersion: None (constant index) or (a nm^-2,
    lambda0 nm) of n(lambda) - 1 = a / (1/lambda0^2 - 1/lambda^2)."""
    return EmitParams(seed=int(seed), n_minus_1=float(n_minus_1),
                      lambda_min=float(lambda_min), lambda_max=float(lambda_max),
                      source=int(source), yield_per_mm=float(yield_per_mm),
                      spectrum_table=int(spectrum_table),
                      dispersion=0 if dispersion is None else 1,
                      disp_a=0.0 if dispersion is None else float(dispersion[0]),
                      disp_lambda0=0.0 if dispersion is None else float(dispersion[1]))


class PhotonsDesc(C.Structure):
    _fields_ = [("n", C.c_uint64), ("capacity", C.c_uint64)] + [
        (f, C.c_void_p) for f in ("x", "y", "z", "dx", "dy", "dz", "lambda_",
                                  "event", "track", "photon")]


class TraceOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("precision", C.c_int32),
                ("max_bounces", C.c_int32), ("max_steps", C.c_int32),
                ("t_min", C.c_float), ("block_threads", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("refill_min", C.c_int32),
                ("chunk", C.c_int32), ("wide_regs", C.c_int32),
                ("bvh_smem_nodes", C.c_int32), ("n_prefilter", C.c_int32),
                ("prefilter_tables", C.c_int32 * 4), ("wait_limit", C.c_int32)]


def _prefilter_fields(prefilter):
    """TraceOpts fields of a prefilter table list (Sec. 4.3 efficiencies
    applied before propagation; empty: in flight)."""
    tabs = [int(x) for x in (prefilter or ())]
    if len(tabs) > 4:
        raise ValueError("at most 4 prefilter tables")
    return {"n_prefilter": len(tabs),
            "prefilter_tables": (C.c_int32 * 4)(*(tabs + [0] * (4 - len(tabs))))}


class Outputs(C.Structure):
    _fields_ = [("hits", C.c_void_p), ("hit_capacity", C.c_uint64),
                ("pixel_counts", C.c_void_p), ("event_sums", C.c_void_p),
                ("n_hist_events", C.c_uint32), ("reserved", C.c_uint32),
                ("fate", C.c_void_p), ("fate_capacity", C.c_uint64)]


class GradParams(C.Structure):
    _fields_ = [("tilt", C.c_float * 8), ("radius", C.c_float), ("n_minus_1", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("n_photons", C.c_uint64), ("n_hits", C.c_uint64),
                ("n_fate", C.c_uint64 * N_FATES), ("device_status", C.c_uint32),
                ("photon_order", C.c_uint32)]


class KernelMs(C.Structure):
    _fields_ = [("yield_", C.c_float), ("order", C.c_float), ("trace", C.c_float),
                ("refine", C.c_float)]


class Work(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("photons", "steps", "nodes_smem", "nodes_global",
                                          "tri_tests", "smooth_normals", "turns", "detected",
                                          "tracks")] + [
        ("sphere_groups", C.c_int32), ("rects", C.c_int32)]


class Peaks(C.Structure):
    _fields_ = [("fp32_fma_flops", C.c_double), ("fp32_minmax_ops", C.c_double),
                ("mufu_ops", C.c_double), ("l2_read_bytes", C.c_double),
                ("n_sm", C.c_int32), ("reserved", C.c_int32),
                ("sm_clock_mhz_max", C.c_double)]


# ------------------------------------------------------------------ library
_lib = None
_lock = threading.Lock()


def load():
    """Load librich.so (built by build.py / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.rich_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        L.rich_destroy.argtypes = [vp]
        L.rich_set_stream.argtypes = [vp, vp]
        L.rich_init_geometry.argtypes = [vp, C.POINTER(GeometryDesc)]
        L.rich_emit.argtypes = [vp, C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                C.POINTER(PhotonsDesc), C.POINTER(C.c_uint64)]
        L.rich_trace.argtypes = [vp, C.POINTER(PhotonsDesc), C.POINTER(TraceOpts),
                                 C.POINTER(Outputs)]
        L.rich_hits.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(Stats)]
        L.rich_philox.argtypes = [vp, vp, C.c_uint64, C.c_uint64, vp]
        L.rich_photon_counts_static.argtypes = [C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                                vp, vp, vp]
        L.rich_graph_capture.argtypes = [vp, C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                         C.POINTER(TraceOpts), C.POINTER(Outputs)]
        L.rich_graph_launch.argtypes = [vp]
        L.rich_trace_grad.argtypes = [vp, C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                      C.POINTER(GradParams), vp, C.c_float,
                                      C.POINTER(TraceOpts), C.POINTER(Outputs),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_uint64)]
        L.rich_run_host.argtypes = [vp, C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                    C.POINTER(TraceOpts), C.POINTER(Outputs), vp, C.c_uint64,
                                    C.POINTER(C.c_uint64), C.POINTER(Stats)]
        L.rich_run_host_async.argtypes = [vp, C.POINTER(TracksDesc), C.POINTER(EmitParams),
                                          C.POINTER(TraceOpts), C.POINTER(Outputs), vp,
                                          C.c_uint64, C.POINTER(C.c_uint64)]
        L.rich_run_wait.argtypes = [vp, C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(Stats)]
        L.rich_set_timing.argtypes = [vp, C.c_int]
        L.rich_kernel_times.argtypes = [vp, C.POINTER(KernelMs)]
        L.rich_trace_work.argtypes = [vp, C.POINTER(TraceOpts), C.POINTER(Outputs),
                                      C.POINTER(Work)]
        L.rich_measure_peaks.argtypes = [C.c_int, vp, C.POINTER(Peaks)]
        L.rich_measure_peaks.restype = C.c_int
        L.rich_peaks_last_error.restype = C.c_char_p
        L.rich_last_error.argtypes = [vp]
        L.rich_last_error.restype = C.c_char_p
        L.rich_version.restype = C.c_char_p
        for f in ("rich_create", "rich_destroy", "rich_set_stream", "rich_init_geometry",
                  "rich_emit", "rich_trace", "rich_hits", "rich_philox",
                  "rich_photon_counts_static", "rich_trace_grad", "rich_graph_capture",
                  "rich_graph_launch", "rich_run_host", "rich_run_host_async", "rich_run_wait",
                  "rich_set_timing", "rich_kernel_times", "rich_trace_work"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


def _check(ctx, st):
    if st != RICH_OK:
        msg = load().rich_last_error(ctx).decode(errors="replace")
        raise RichError(st, msg)


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def current_stream_handle():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


# ----------------------------------------------------------- device inputs
class DeviceTracks:
    """A Tracks set uploaded to device memory (torch tensors)."""

    def __init__(self, tracks: W.Tracks, device="cuda"):
        torch = _torch()
        self.n = tracks.n
        self.t = {}
        for f in W.Tracks.FIELDS:
            self.t[f] = torch.from_numpy(np.ascontiguousarray(getattr(tracks, f), np.float32)).to(device)
        self.t["event"] = torch.from_numpy(
            np.ascontiguousarray(tracks.event, np.uint32).view(np.int32)).to(device)
        self.t["id"] = torch.from_numpy(
            np.ascontiguousarray(tracks.id, np.uint32).view(np.int32)).to(device)
        self.t["n_fixed"] = (None if tracks.n_fixed is None else torch.from_numpy(
            np.ascontiguousarray(tracks.n_fixed, np.uint32).view(np.int32)).to(device))

    @classmethod
    def packed(cls, tracks: W.Tracks, device="cuda"):
        """Tracks whose device arrays are slices of one buffer, and a pinned
        host copy of that buffer: one host-to-device copy
        (`dt.upload(host)`) moves a whole track set."""
        torch = _torch()
        fields = list(W.Tracks.FIELDS) + ["event", "id"]
        n = tracks.n
        host = torch.empty(len(fields) * max(n, 1), dtype=torch.int32).pin_memory()
        hv = host.numpy()
        for k, f in enumerate(fields):
            a = getattr(tracks, f)
            dtp = np.float32 if f in W.Tracks.FIELDS else np.uint32
            hv[k * n:(k + 1) * n] = np.ascontiguousarray(a, dtp).view(np.int32)
        dev = host.to(device)
        self = cls.__new__(cls)
        self.n = n
        self.t = {}
        for k, f in enumerate(fields):
            v = dev[k * n:(k + 1) * n]
            self.t[f] = v.view(torch.float32) if f in W.Tracks.FIELDS else v
        self.t["n_fixed"] = (None if tracks.n_fixed is None else torch.from_numpy(
            np.ascontiguousarray(tracks.n_fixed, np.uint32).view(np.int32)).to(device))
        self._buf = dev
        return self, host

    def upload(self, host):
        """Copy a packed pinned host buffer (from `packed`) into the device
        arrays, asynchronously on the current stream."""
        self._buf.copy_(host, non_blocking=True)

    def desc(self) -> TracksDesc:
        """The rich_tracks descriptor (built once: the arrays are fixed)."""
        d = getattr(self, "_desc", None)
        if d is None:
            d = self._desc = TracksDesc(n=self.n, **{k: (None if v is None else v.data_ptr())
                                                     for k, v in self.t.items()})
        return d


class HostTracks:
    """A Tracks set in one pinned host buffer, the arrays back to back in
    rich_tracks order (so rich_run_host copies them with one transfer)."""

    def __init__(self, tracks: W.Tracks):
        torch = _torch()
        fields = list(W.Tracks.FIELDS) + ["event", "id"]
        if tracks.n_fixed is not None:
            fields.append("n_fixed")
        n = self.n = tracks.n
        self.buf = torch.empty(len(fields) * max(n, 1), dtype=torch.int32).pin_memory()
        hv = self.buf.numpy()
        for k, f in enumerate(fields):
            dtp = np.float32 if f in W.Tracks.FIELDS else np.uint32
            hv[k * n:(k + 1) * n] = np.ascontiguousarray(getattr(tracks, f), dtp).view(np.int32)
        base = self.buf.data_ptr()
        self.ptrs = {f: base + 4 * k * n for k, f in enumerate(fields)}

    def desc(self) -> TracksDesc:
        d = getattr(self, "_desc", None)
        if d is None:
            d = self._desc = TracksDesc(n=self.n, **{f: self.ptrs.get(f) for f in
                                                     list(W.Tracks.FIELDS) + ["event", "id",
                                                                              "n_fixed"]})
        return d


class PhotonBuffers:
    """Device structure-of-arrays photons (rich_photons)."""

    FIELDS = ("x", "y", "z", "dx", "dy", "dz", "lambda_")
    KEYS = ("event", "track", "photon")

    def __init__(self, capacity, device="cuda"):
        torch = _torch()
        self.capacity = int(capacity)
        self.n = 0
        self.t = {f: torch.empty(max(1, self.capacity), dtype=torch.float32, device=device)
                  for f in self.FIELDS}
        self.t.update({f: torch.empty(max(1, self.capacity), dtype=torch.int32, device=device)
                       for f in self.KEYS})

    @classmethod
    def from_arrays(cls, device="cuda", **arrays):
        n = len(arrays["x"])
        pb = cls(n, device)
        torch = _torch()
        for f in cls.FIELDS:
            src = arrays["lambda"] if f == "lambda_" else arrays[f]
            pb.t[f][:n].copy_(torch.from_numpy(np.ascontiguousarray(src, np.float32)))
        for f in cls.KEYS:
            pb.t[f][:n].copy_(torch.from_numpy(np.ascontiguousarray(arrays[f], np.uint32).view(np.int32)))
        pb.n = n
        return pb

    def desc(self) -> PhotonsDesc:
        return PhotonsDesc(n=self.n, capacity=self.capacity,
                           **{k: v.data_ptr() for k, v in self.t.items()})


class TraceOutputs:
    """Device output buffers of rich_trace (rich_outputs)."""

    def __init__(self, hit_capacity, pixels_per_event=0, n_planes=0,
                 n_hist_events=0, n_photons_fate=0, device="cuda"):
        torch = _torch()
        self.hit_capacity = int(hit_capacity)
        self.hits = torch.empty(max(1, self.hit_capacity) * HIT_DTYPE.itemsize,
                                dtype=torch.uint8, device=device)
        self.n_hist_events = int(n_hist_events)
        self.pixels_per_event = int(pixels_per_event)
        self.n_planes = int(n_planes)
        self.pixel_counts = (torch.zeros(n_hist_events * pixels_per_event, dtype=torch.int32,
                                         device=device) if n_hist_events and pixels_per_event
                             else None)
        self.event_sums = (torch.zeros(n_hist_events * n_planes * 4, dtype=torch.float64,
                                       device=device) if n_hist_events and n_planes else None)
        self.fate = (torch.zeros(n_photons_fate, dtype=torch.uint8, device=device)
                     if n_photons_fate else None)

    def clear(self):
        if self.pixel_counts is not None:
            self.pixel_counts.zero_()
        if self.event_sums is not None:
            self.event_sums.zero_()
        if self.fate is not None:
            self.fate.zero_()

    def desc(self) -> Outputs:
        """The rich_outputs descriptor (built once: the buffers are fixed)."""
        d = getattr(self, "_desc", None)
        if d is None:
            d = self._desc = self._make_desc()
        return d

    def _make_desc(self) -> Outputs:
        return Outputs(hits=self.hits.data_ptr(), hit_capacity=self.hit_capacity,
                       pixel_counts=None if self.pixel_counts is None else self.pixel_counts.data_ptr(),
                       event_sums=None if self.event_sums is None else self.event_sums.data_ptr(),
                       n_hist_events=self.n_hist_events if (self.pixel_counts is not None or
                                                            self.event_sums is not None) else 0,
                       fate=None if self.fate is None else self.fate.data_ptr(),
                       fate_capacity=0 if self.fate is None else self.fate.numel())

    def hits_numpy(self, n):
        n = min(int(n), self.hit_capacity)
        raw = self.hits[: n * HIT_DTYPE.itemsize].cpu().numpy()
        return raw.view(HIT_DTYPE).copy()

    def pixel_counts_numpy(self):
        return self.pixel_counts.cpu().numpy().view(np.uint32).reshape(
            self.n_hist_events, self.pixels_per_event)

    def event_sums_numpy(self):
        return self.event_sums.cpu().numpy().reshape(self.n_hist_events, self.n_planes, 4)


# ---------------------------------------------------------------- context
class Context:
    """Owns one rich_ctx. Methods mirror the C entry points."""

    def __init__(self, device=0, stream=None):
        L = load()
        h = C.c_void_p()
        s = current_stream_handle() if stream is None else stream
        st = L.rich_create(C.byref(h), int(device), C.c_void_p(s))
        if st != RICH_OK:
            raise RichError(st, L.rich_last_error(None).decode(errors="replace"))
        self.handle = h
        self.device = device
        self._geom_keep = None
        self.scene = None

    def close(self):
        if getattr(self, "handle", None):
            load().rich_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(self.handle, load().rich_set_stream(self.handle, C.c_void_p(stream)))

    def init_geometry(self, scene: W.Scene):
        keep = [np.ascontiguousarray(scene.tables), np.ascontiguousarray(scene.materials),
                np.ascontiguousarray(scene.spheres), np.ascontiguousarray(scene.rects),
                np.ascontiguousarray(scene.tri_vertices, np.float32),
                None if scene.tri_normals is None else
                np.ascontiguousarray(scene.tri_normals, np.float32),
                np.ascontiguousarray(scene.tri_material, np.int32),
                None if scene.tri_surface is None else
                np.ascontiguousarray(scene.tri_surface, np.int32)]
        p = lambda a: None if a is None or a.size == 0 else a.ctypes.data
        d = GeometryDesc(n_tables=len(keep[0]), n_materials=len(keep[1]),
                         n_spheres=len(keep[2]), n_rects=len(keep[3]),
                         n_triangles=scene.n_triangles, tables=p(keep[0]),
                         materials=p(keep[1]), spheres=p(keep[2]), rects=p(keep[3]),
                         tri_vertices=p(keep[4]), tri_normals=p(keep[5]),
                         tri_material=p(keep[6]), tri_surface=p(keep[7]))
        _check(self.handle, load().rich_init_geometry(self.handle, C.byref(d)))
        self.scene = scene

    def emit(self, tracks: DeviceTracks, n_minus_1, lambda_min=200.0, lambda_max=600.0,
             seed=0, photons: PhotonBuffers | None = None, sync=True,
             source=SOURCE_CHERENKOV, yield_per_mm=0.0, spectrum_table=-1, dispersion=None):
        """source: SOURCE_CHERENKOV, or SOURCE_ISOTROPIC with yield_per_mm
        photons per mm and the scene's CDF table spectrum_table (-1: the
        1/lambda^2 law on the band). dispersion: None or (a, lambda0) of
        the dispersive radiator (Cherenkov source)."""
        prm = _emit_params(seed, n_minus_1, lambda_min, lambda_max, source, yield_per_mm,
                           spectrum_table, dispersion)
        n = C.c_uint64(0)
        pd = photons.desc() if photons is not None else None
        st = load().rich_emit(self.handle, C.byref(tracks.desc()), C.byref(prm),
                              None if pd is None else C.byref(pd),
                              C.byref(n) if sync else None)
        _check(self.handle, st)
        if photons is not None:
            photons.n = int(pd.n)
        return int(n.value) if sync else None

    def trace(self, outputs: TraceOutputs, photons: PhotonBuffers | None = None,
              precision=PREC_REFINE64, max_bounces=8, max_steps=16, t_min=1e-3,
              seed=0, block_threads=0, blocks_per_sm=0, refill_min=0, chunk=0,
              wide_regs=0, bvh_smem_nodes=-1, prefilter=(), wait_limit=0):
        """prefilter: scene table indices whose product is applied as one
        accept/reject per photon before propagation (Sec. 4.3). wait_limit:
        iterations of the bounded wait for the shared-memory node copy (0:
        default; negative: the wait gives up at once, a test of that path)."""
        o = _trace_opts(seed, precision, max_bounces, max_steps, t_min, block_threads,
                        blocks_per_sm, refill_min, chunk, wide_regs, bvh_smem_nodes, prefilter,
                        wait_limit)
        pd = photons.desc() if photons is not None else None
        st = load().rich_trace(self.handle, None if pd is None else C.byref(pd),
                               C.byref(o), C.byref(outputs.desc()))
        _check(self.handle, st)

    def run_host(self, tracks: HostTracks, outputs: TraceOutputs, hits_host, n_minus_1,
                 lambda_min=200.0, lambda_max=600.0, seed=0, precision=PREC_REFINE64,
                 max_bounces=8, max_steps=16, t_min=1e-3, block_threads=0, blocks_per_sm=0,
                 refill_min=0, chunk=0, wide_regs=0, bvh_smem_nodes=-1, prefilter=(),
                 source=SOURCE_CHERENKOV, yield_per_mm=0.0, spectrum_table=-1,
                 dispersion=None):
        """One synchronous step from host memory (rich_run_host): host tracks
        in, the hit records copied into hits_host (a pinned uint8 tensor of
        n x 40 bytes; None reads the counters only). Emission arguments as
        for emit. Returns (n_hits, stats dict)."""
        # the call's argument objects are kept between steps (only the seed
        # changes in place): a step is dominated by the GPU, and the host
        # time before the first launch delays it
        key = (float(n_minus_1), float(lambda_min), float(lambda_max), source,
               float(yield_per_mm), spectrum_table, dispersion)
        rh = getattr(self, "_rh", None)
        if rh is None or rh[0] != key:
            prm = _emit_params(seed, n_minus_1, lambda_min, lambda_max, source, yield_per_mm,
                               spectrum_table, dispersion)
            rh = self._rh = (key, prm, C.c_uint64(0), Stats())
        _, prm, n, s = rh
        prm.seed = int(seed)
        o = _trace_opts(0, precision, max_bounces, max_steps, t_min, block_threads,
                        blocks_per_sm, refill_min, chunk, wide_regs, bvh_smem_nodes, prefilter)
        ptr, cap = _host_hits(hits_host)
        st = load().rich_run_host(self.handle, C.byref(tracks.desc()), C.byref(prm),
                                  C.byref(o), C.byref(outputs.desc()), ptr, cap, C.byref(n),
                                  C.byref(s))
        _check(self.handle, st)
        return n.value, {"n_photons": s.n_photons, "n_hits": s.n_hits, "fate": list(s.n_fate),
                         "device_status": s.device_status, "photon_order": s.photon_order}

    def run_host_async(self, tracks: HostTracks, outputs: TraceOutputs, hits_host, n_minus_1,
                       lambda_min=200.0, lambda_max=600.0, seed=0, precision=PREC_REFINE64,
                       max_bounces=8, max_steps=16, t_min=1e-3, block_threads=0,
                       blocks_per_sm=0, refill_min=0, chunk=0, wide_regs=0,
                       bvh_smem_nodes=-1, prefilter=(), source=SOURCE_CHERENKOV,
                       yield_per_mm=0.0, spectrum_table=-1, dispersion=None):
        """Pipelined step (rich_run_host_async): returns a ticket for
        run_wait. Two steps may be in flight, each with its own outputs and
        hits_host (None: counters only); the HostTracks must not change
        until waited for. Emission arguments as for emit."""
        prm = _emit_params(seed, n_minus_1, lambda_min, lambda_max, source, yield_per_mm,
                           spectrum_table, dispersion)
        o = _trace_opts(0, precision, max_bounces, max_steps, t_min, block_threads,
                        blocks_per_sm, refill_min, chunk, wide_regs, bvh_smem_nodes, prefilter)
        t = C.c_uint64(0)
        ptr, cap = _host_hits(hits_host)
        st = load().rich_run_host_async(self.handle, C.byref(tracks.desc()), C.byref(prm),
                                        C.byref(o), C.byref(outputs.desc()), ptr, cap,
                                        C.byref(t))
        _check(self.handle, st)
        return t.value

    def run_wait(self, ticket):
        """Completes a pipelined step: (n_hits, stats dict)."""
        n = C.c_uint64(0)
        s = Stats()
        st = load().rich_run_wait(self.handle, int(ticket), C.byref(n), C.byref(s))
        _check(self.handle, st)
        return n.value, {"n_photons": s.n_photons, "n_hits": s.n_hits, "fate": list(s.n_fate),
                         "device_status": s.device_status, "photon_order": s.photon_order}

    def philox(self, counters, seed):
        """Library Philox4x32-10 of an (n, 4) uint32 counter array."""
        torch = _torch()
        ctr = np.ascontiguousarray(counters, np.uint32).reshape(-1, 4)
        d_in = torch.from_numpy(ctr.view(np.int32).copy()).to(f"cuda:{self.device}")
        d_out = torch.empty_like(d_in)
        _check(self.handle, load().rich_philox(self.handle, C.c_void_p(d_in.data_ptr()),
                                               len(ctr), int(seed),
                                               C.c_void_p(d_out.data_ptr())))
        return d_out.cpu().numpy().view(np.uint32).reshape(-1, 4)

    def graph_capture(self, tracks: DeviceTracks, outputs: TraceOutputs, n_minus_1,
                      lambda_min=200.0, lambda_max=600.0, seed=0, precision=PREC_REFINE64,
                      max_bounces=8, max_steps=16, t_min=1e-3, block_threads=0,
                      blocks_per_sm=0, refill_min=0, chunk=0, wide_regs=0,
                      bvh_smem_nodes=-1, prefilter=()):
        """Capture emit + trace into a CUDA graph (after a warm-up pass)."""
        prm = EmitParams(seed=int(seed), n_minus_1=float(n_minus_1),
                         lambda_min=float(lambda_min), lambda_max=float(lambda_max))
        o = TraceOpts(seed=0, precision=precision, max_bounces=max_bounces,
                      max_steps=max_steps, t_min=t_min, block_threads=block_threads,
                      blocks_per_sm=blocks_per_sm, refill_min=refill_min, chunk=chunk,
                      wide_regs=wide_regs, bvh_smem_nodes=bvh_smem_nodes,
                      **_prefilter_fields(prefilter))
        self._graph_keep = (tracks, outputs)
        _check(self.handle, load().rich_graph_capture(self.handle, C.byref(tracks.desc()),
                                                      C.byref(prm), C.byref(o),
                                                      C.byref(outputs.desc())))

    def graph_launch(self):
        _check(self.handle, load().rich_graph_launch(self.handle))

    def set_timing(self, on=True):
        """Kernel timing on or off (rich_set_timing)."""
        _check(self.handle, load().rich_set_timing(self.handle, int(bool(on))))

    def kernel_times(self):
        """Durations (ms) of the kernels of the last timed emit and trace:
        dict of yield, order, trace, refine (-1: not timed)."""
        k = KernelMs()
        _check(self.handle, load().rich_kernel_times(self.handle, C.byref(k)))
        return {"yield": k.yield_, "order": k.order, "trace": k.trace, "refine": k.refine}

    def trace_work(self, outputs: TraceOutputs, max_bounces=8, max_steps=16, t_min=1e-3,
                   block_threads=0, blocks_per_sm=0, refill_min=0, chunk=0, wide_regs=0,
                   bvh_smem_nodes=-1):
        """rich_trace_work: the last emission traced by the counting build
        (refined precision); returns the work tallies as a dict."""
        o = _trace_opts(0, PREC_REFINE64, max_bounces, max_steps, t_min, block_threads,
                        blocks_per_sm, refill_min, chunk, wide_regs, bvh_smem_nodes, ())
        w = Work()
        st = load().rich_trace_work(self.handle, C.byref(o), C.byref(outputs.desc()),
                                    C.byref(w))
        if st not in (RICH_OK, 4):
            _check(self.handle, st)
        return {f: getattr(w, f) for f, _ in Work._fields_}

    def trace_grad(self, tracks: DeviceTracks, theta, targets, outputs: TraceOutputs,
                   sigma=1.0, seed=0, lambda_min=200.0, lambda_max=600.0, max_bounces=8,
                   max_steps=16, t_min=1e-3, **launch):
        """Soft ring chi^2 loss, its gradient (10) and the number of hits used
        at theta = (8 tile tilts, radius of curvature, n - 1). targets: device
        float32 tensor [n_tracks][n_planes][4]."""
        th = [float(x) for x in theta]
        gp = GradParams(tilt=(C.c_float * 8)(*th[:8]), radius=th[8], n_minus_1=th[9])
        prm = EmitParams(seed=int(seed), n_minus_1=th[9], lambda_min=float(lambda_min),
                         lambda_max=float(lambda_max))
        o = TraceOpts(seed=0, precision=PREC_REFINE64, max_bounces=max_bounces,
                      max_steps=max_steps, t_min=t_min,
                      block_threads=launch.get("block_threads", 0),
                      blocks_per_sm=launch.get("blocks_per_sm", 0),
                      refill_min=launch.get("refill_min", 0), chunk=launch.get("chunk", 0),
                      wide_regs=launch.get("wide_regs", 0),
                      bvh_smem_nodes=launch.get("bvh_smem_nodes", -1))
        g = (C.c_double * 10)()
        loss = C.c_double(0.0)
        used = C.c_uint64(0)
        st = load().rich_trace_grad(self.handle, C.byref(tracks.desc()), C.byref(prm),
                                    C.byref(gp), C.c_void_p(targets.data_ptr()),
                                    float(sigma), C.byref(o), C.byref(outputs.desc()), g,
                                    C.byref(loss), C.byref(used))
        _check(self.handle, st)
        return float(loss.value), np.array(g[:], np.float64), int(used.value)

    def hits(self, allow_overflow=False, allow=()):
        """Returns (n_hits, stats dict); synchronises the context stream.
        Raises RichError on a non-OK status, except overflow with
        allow_overflow and the statuses listed in `allow` (stats["status"]
        then holds it)."""
        n = C.c_uint64(0)
        s = Stats()
        st = load().rich_hits(self.handle, C.byref(n), C.byref(s))
        if not ((allow_overflow and st == 4) or st in allow):
            _check(self.handle, st)
        stats = {"n_photons": int(s.n_photons), "n_hits": int(s.n_hits),
                 "fate": [int(x) for x in s.n_fate], "device_status": int(s.device_status),
                 "photon_order": int(s.photon_order), "status": int(st)}
        return int(n.value), stats


def measure_peaks(device=0, stream=None):
    """rich_measure_peaks: measured FP32 FMA, FP32 min/max, MUFU and L2 read
    rates of the device (dict)."""
    pk = Peaks()
    s = current_stream_handle() if stream is None else stream
    rc = load().rich_measure_peaks(int(device), C.c_void_p(s), C.byref(pk))
    if rc != 0:
        raise RuntimeError(load().rich_peaks_last_error().decode(errors="replace"))
    return {f: getattr(pk, f) for f, _ in Peaks._fields_ if f != "reserved"}


# ------------------------------------------ C-ABI-named module functions
def rich_create(device=0, stream=None) -> Context:
    return Context(device, stream)


def rich_destroy(ctx: Context):
    ctx.close()


def rich_init_geometry(ctx: Context, scene):
    ctx.init_geometry(scene)


def rich_emit(ctx: Context, tracks, n_minus_1, **kw):
    return ctx.emit(tracks, n_minus_1, **kw)


def rich_trace(ctx: Context, outputs, **kw):
    ctx.trace(outputs, **kw)


def rich_hits(ctx: Context, **kw):
    return ctx.hits(**kw)


def rich_run_host(ctx: Context, tracks: HostTracks, outputs, hits_host, n_minus_1, **kw):
    return ctx.run_host(tracks, outputs, hits_host, n_minus_1, **kw)


def rich_run_host_async(ctx: Context, tracks: HostTracks, outputs, hits_host, n_minus_1, **kw):
    return ctx.run_host_async(tracks, outputs, hits_host, n_minus_1, **kw)


def rich_run_wait(ctx: Context, ticket):
    return ctx.run_wait(ticket)


def rich_photon_counts_static(tracks: DeviceTracks, n_minus_1, counts, offsets,
                              lambda_min=200.0, lambda_max=600.0, seed=0, stream=None,
                              n=None, source=SOURCE_CHERENKOV, yield_per_mm=0.0,
                              dispersion=None):
    """Per-track photon counts (int32 view of u32) and offsets (int64 view of
    u64, n + 1 entries) into caller device tensors, with no device
    allocation by the library. `n` overrides the track count passed."""
    L = load()
    d = TracksDesc.from_buffer_copy(tracks.desc())
    if n is not None:
        d.n = int(n)
    prm = _emit_params(seed, n_minus_1, lambda_min, lambda_max, source, yield_per_mm, -1,
                       dispersion)
    s = current_stream_handle() if stream is None else stream
    st = L.rich_photon_counts_static(C.byref(d), C.byref(prm), C.c_void_p(counts.data_ptr()),
                                     C.c_void_p(offsets.data_ptr()), C.c_void_p(s))
    _check(None, st)


def rich_version() -> str:
    return load().rich_version().decode()


def ring_chi2(ctx: Context, theta, tracks: DeviceTracks, targets, outputs: TraceOutputs,
              sigma=1.0, seed=0):
    """Differentiable soft ring chi^2: a torch.autograd.Function over the
    10 parameters (8 tile tilts, radius of curvature, n - 1); its backward
    is the gradient from rich_trace_grad's adjoint pass."""
    torch = _torch()

    class _RingChi2(torch.autograd.Function):
        @staticmethod
        def forward(fctx, th):
            loss, grad, used = ctx.trace_grad(tracks, th.detach().cpu().tolist(), targets,
                                              outputs, sigma=sigma, seed=seed)
            fctx.save_for_backward(torch.tensor(grad, dtype=th.dtype, device=th.device))
            fctx.n_used = used
            return th.new_tensor(loss)

        @staticmethod
        def backward(fctx, gout):
            (grad,) = fctx.saved_tensors
            return gout * grad

    return _RingChi2.apply(theta)


def rich_trace_grad(ctx: Context, tracks, theta, targets, outputs, **kw):
    return ctx.trace_grad(tracks, theta, targets, outputs, **kw)
