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


_CTYPES = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "float": ctypes.c_float, "double": ctypes.c_double}


def declared_structs():
    """{name: [(field, ctypes type)]} of every typedef struct in gc.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in (d.strip() for d in body.split(";")):
            if not decl:
                continue
            fp = re.match(r".*\(\s*\*\s*(\w+)\s*\)\s*\(", decl)   # function pointer
            if fp:
                fields.append((fp.group(1), ctypes.c_void_p))
                continue
            if decl.startswith("void *") or decl.startswith("void*"):
                fields.append((decl.split("*")[-1].strip(), ctypes.c_void_p))
                continue
            typ, rest = decl.split(None, 1)
            for item in (x.strip() for x in rest.split(",")):
                m = re.match(r"(\w+)(?:\[(\d+)\])?$", item)
                base = _CTYPES[typ]
                fields.append((m.group(1), base * int(m.group(2)) if m.group(2) else base))
        out[name] = fields
    return out


def test_binding_structs_match_the_header():
    """Every struct of the ABI has the same fields, in the same order, with
    the same types and the same size in the Python binding (a drift here
    would pass wrong values through every call that takes the struct)."""
    from paper_2308_14493_gb300 import gc as binding

    structs = declared_structs()
    assert set(structs) == {"gc_options", "gc_stats", "gc_tuning", "gc_server_options", "gc_result"}
    for name, fields in structs.items():
        cls = getattr(binding, name)
        got = [(f, t) for f, t in cls._fields_]
        assert [f for f, _ in got] == [f for f, _ in fields], name
        for (f, t_py), (_, t_h) in zip(got, fields):
            assert ctypes.sizeof(t_py) == ctypes.sizeof(t_h) and getattr(t_py, "_type_", None) == getattr(
                t_h, "_type_", None), (name, f)

        class Mirror(ctypes.Structure):
            _fields_ = fields

        assert ctypes.sizeof(cls) == ctypes.sizeof(Mirror), name


def _open_raw(n, rp, col, **opt_fields):
    import numpy as np

    from paper_2308_14493_gb300 import gc as binding

    lib = binding.load()
    opt = binding.gc_options()
    lib.gc_default_options(ctypes.byref(opt))
    for k, v in opt_fields.items():
        setattr(opt, k, v)
    h = ctypes.c_void_p()
    rpa = None if rp is None else np.ascontiguousarray(rp, dtype=np.int32)
    ca = None if col is None else np.ascontiguousarray(col, dtype=np.int32)
    ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    rc = lib.gc_open(n, ptr(rpa), ptr(ca), ctypes.byref(opt), ctypes.byref(h))
    return rc, lib.gc_last_error(None).decode()


@pytest.mark.parametrize("case,n,rp,col,opt,msg", [
    ("negative n", -1, [0], [0], {}, "n must be in"),
    ("n too large", 1 << 30, [0], [0], {}, "n must be in"),
    ("row_ptr NULL", 3, None, [0], {}, "row_ptr is NULL"),
    ("row_ptr[0] != 0", 2, [1, 2, 2], [0, 1], {}, "row_ptr[0] must be 0"),
    ("odd entries", 2, [0, 1, 1], [1], {}, "even number of entries"),
    ("col NULL", 2, [0, 1, 2], None, {}, "col is NULL"),
    ("hops 1", 2, [0, 1, 2], [1, 0], {"region_hops": 1}, "region_hops"),
    ("hops 9", 2, [0, 1, 2], [1, 0], {"region_hops": 9}, "region_hops"),
    ("cluster 4", 2, [0, 1, 2], [1, 0], {"dense_cluster": 4}, "dense_cluster"),
    ("alloc without free", 2, [0, 1, 2], [1, 0], {"alloc": 1}, "alloc and free"),
])
def test_open_rejects_bad_arguments_on_the_host(case, n, rp, col, opt, msg):
    """Argument errors of gc_open are found on the host, before any device
    call, each with its own message (so they hold without a GPU too)."""
    from paper_2308_14493_gb300 import gc as binding

    rc, err = _open_raw(n, rp, col, **opt)
    assert rc == binding.GC_EINVAL, case
    assert msg in err, (case, err)
