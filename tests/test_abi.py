"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gc.h declares.  No GPU needed: nothing here computes."""
import ctypes
import os
import re

import pytest

from gc_testutil import GOLDEN_DIR  # noqa: F401  (keeps the tests dir importable)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gc_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gc_open", "gc_count_static", "gc_apply_batch", "gc_close"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2308_14493_gb300 import gc as binding

    lib = binding.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding exposes the same names
    for name in declared_functions():
        assert hasattr(binding, name) or name == "gc_default_options", name


def test_library_is_built_for_sm103a():
    from paper_2308_14493_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.build())


def test_open_without_gpu_fails_loudly_or_runs():
    """Without a usable GPU, gc_open must return an error, never fall back."""
    import numpy as np

    from paper_2308_14493_gb300 import gc as binding

    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(binding.GCError) as ei:
        binding.gc_open(4, np.array([0, 1, 2, 3, 4], np.int32), np.array([1, 0, 3, 2], np.int32))
    assert ei.value.code in (binding.GC_ECUDA, binding.GC_ENOMEM)


def test_invalid_arguments_are_rejected_before_any_device_work():
    import numpy as np

    from paper_2308_14493_gb300 import gc as binding

    lib = binding.load()
    h = ctypes.c_void_p()
    rp = np.array([0, 2, 1], np.int32)  # decreasing
    col = np.array([1, 0], np.int32)
    rc = lib.gc_open(2, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, ctypes.byref(h))
    assert rc == binding.GC_EINVAL
    assert b"non-decreasing" in lib.gc_last_error(None)


def test_null_handles_are_rejected():
    """Every call that takes a handle refuses a null one without device work."""
    import numpy as np

    from paper_2308_14493_gb300 import gc as binding

    lib = binding.load()
    out = np.zeros(64, np.uint64)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    for name in ("gc_counts", "gc_counts3", "gc_counts_all", "gc_vertex_counts", "gc_vertex_orbits",
                 "gc_count_static"):
        assert getattr(lib, name)(None, p) == binding.GC_EINVAL, name
    e = np.zeros(8, np.int32)
    for name in ("gc_edge_counts", "gc_edge_orbits"):
        assert getattr(lib, name)(None, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), p) == binding.GC_EINVAL
    assert lib.gc_num_edges(None) == -1
