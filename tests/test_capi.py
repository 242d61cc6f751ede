"""The C-ABI library without a GPU: it loads, exports every entry point
declared in include/rich.h, and reports errors instead of failing when no
device is present."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rich.h")
PEAKS_HEADER = os.path.join(ROOT, "include", "rich_peaks.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2309_12496_gb300 import build, rich
    build.build()
    return rich.load()


def declared_entry_points():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"RICH_API\s+[\w\s\*]+?\b(rich_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("rich_create", "rich_destroy", "rich_init_geometry", "rich_emit",
                     "rich_trace", "rich_hits", "rich_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2309_12496_gb300 import rich
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} declared in rich.h but not exported"
    assert sorted(rich.EXPORTED) == declared_entry_points()
    peaks = sorted(set(re.findall(r"RICH_PEAKS_API\s+[\w\s\*]+?\b(rich_\w+)\s*\(",
                                  open(PEAKS_HEADER).read())))
    assert peaks == sorted(rich.EXPORTED_PEAKS)
    for name in peaks:
        assert hasattr(lib, name), f"{name} declared in rich_peaks.h but not exported"
    # every header in include/ is one of the two checked here
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == [
        "rich.h", "rich_peaks.h"]


def test_version_and_null_handling(lib):
    from paper_2309_12496_gb300 import rich
    assert b"sm_103a" in lib.rich_version()
    assert lib.rich_destroy(None) == 0
    assert lib.rich_hits(None, None, None) == 1       # RICH_ERR_ARG
    assert lib.rich_create(None, 0, None) == 1
    assert lib.rich_measure_peaks(0, None, None) == 1
    assert lib.rich_set_timing(None, 1) == 1
    assert lib.rich_kernel_times(None, None) == 1
    assert lib.rich_trace_work(None, None, None, None) == 1


def test_struct_layouts_match_header():
    """The ctypes mirrors and numpy record layouts have the header's sizes."""
    from paper_2309_12496_gb300 import rich
    from paper_2309_12496_gb300 import workloads as W
    assert C.sizeof(rich.GeometryDesc) == 4 * 4 + 8 + 8 * 8
    assert C.sizeof(rich.TracksDesc) == 8 + 12 * 8
    assert C.sizeof(rich.PhotonsDesc) == 16 + 10 * 8
    assert C.sizeof(rich.TraceOpts) == 8 + 16 * 4
    assert C.sizeof(rich.EmitParams) == 8 + 10 * 4
    assert C.sizeof(rich.Outputs) == 8 * 4 + 8 + 8 + 8
    assert C.sizeof(rich.Stats) == 16 + 8 * rich.N_FATES + 8
    assert C.sizeof(rich.KernelMs) == 16
    assert C.sizeof(rich.Work) == 9 * 8 + 8
    assert C.sizeof(rich.Peaks) == 4 * 8 + 8 + 8
    assert rich.HIT_DTYPE.itemsize == 40
    assert W.TABLE_DTYPE.itemsize == 280 and W.SPHERE_DTYPE.itemsize == 160
    assert W.RECT_DTYPE.itemsize == 80 and W.MATERIAL_DTYPE.itemsize == 16


def test_create_without_gpu_fails_loudly(lib):
    """On a machine without a CUDA device, rich_create returns an error and
    a message; nothing falls back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2309_12496_gb300 import rich
    with pytest.raises(rich.RichError) as e:
        rich.Context(0, stream=0)
    assert "no CUDA device" in str(e.value)
