"""Autotuner of the trace launch knobs.

The persistent trace kernel's speed depends on the block shape (256 threads
capped at 64 registers, four blocks per SM; 256 uncapped; 512, 768 or 896
threads capped at 72 registers; 512 or 1024 threads capped at 64), on how many top BVH nodes each block stages in shared
memory, on the compaction interval (refill a warp once `refill_min` lanes
are idle) and on the photons a warp takes from the queue at a time. Which
combination wins depends on the scene and on the number of photons (a small
batch is dominated by the tail of the persistent grid). `tune` times every
candidate on the caller's own emitted photons with CUDA events and returns
the fastest; results are cached per (GPU, scene signature, photon-count
bucket, precision) in ~/.cache/rich_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rich_gb300", "tune.json")

# (knobs, error message) of the candidates the last tune() could not launch
failed = []


def candidates(n_triangles: int):
    """The search space (the BVH staging sizes only matter with meshes)."""
    nodes = (0, 256, 768) if n_triangles else (0,)      # 128-byte four-wide nodes
    out = []
    for threads, bps in ((1024, 0), (512, 0), (512, 1)):
        for n in nodes:
            for refill in (24, 32):
                for chunk in (32, 64):
                    out.append(dict(block_threads=threads, blocks_per_sm=bps,
                                    bvh_smem_nodes=n, refill_min=refill, chunk=chunk))
    for wide in (0, 1):
        for refill in (24, 32):
            out.append(dict(block_threads=256, bvh_smem_nodes=0, refill_min=refill,
                            chunk=32, wide_regs=wide))
    for threads in (896, 768, 512):       # 72-register variant
        for n in nodes:
            for refill in (24, 32):
                out.append(dict(block_threads=threads, blocks_per_sm=0, bvh_smem_nodes=n,
                                refill_min=refill, chunk=32, wide_regs=1))
    return out


def _key(ctx, scene, n_photons, precision):
    import torch
    name = torch.cuda.get_device_name(ctx.device)
    sig = (f"t{scene.n_triangles}-s{len(scene.spheres)}-r{len(scene.rects)}")
    bucket = int(round(math.log2(max(n_photons, 1))))
    return f"{name}|{sig}|p2^{bucket}|prec{precision}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def tune(ctx, outputs, n_photons, precision, reps=3, use_cache=True, space=None):
    """Fastest launch knobs for the photons of the last rich_emit on ctx.
    Returns (knobs dict, median ms, table of (knobs, ms))."""
    import torch
    key = _key(ctx, ctx.scene, n_photons, precision)
    db = _load() if use_cache else {}
    if use_cache and key in db:
        e = db[key]
        return e["knobs"], e["ms"], []
    stream = torch.cuda.current_stream()
    table = []
    failed.clear()
    for knobs in space or candidates(ctx.scene.n_triangles):
        try:
            ctx.trace(outputs, precision=precision, **knobs)     # warm-up
            ms = []
            for _ in range(reps):
                outputs.clear()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.trace(outputs, precision=precision, **knobs)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        except RuntimeError as e:
            failed.append((knobs, str(e)))    # a shape that does not fit this GPU
            continue
        table.append((knobs, statistics.median(ms)))
    best, best_ms = min(table, key=lambda kv: kv[1])
    if use_cache:
        db[key] = {"knobs": best, "ms": best_ms}
        _store(db)
    return best, best_ms, table
