"""The C ABI library loads and exports every entry point that include/*.h declares.

No compute call is made, so this runs without a GPU; the checks a call makes
on the host before touching a device are exercised too.
"""
import glob
import os
import re

import numpy as np
import pytest

import paper_1702_04645_gb300 as slm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(slm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    slm.build()
    return slm.load()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("slm_create_graph", "slm_run", "slm_get_partition", "slm_modularity"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(set(slm.EXPORTS)) == declared_functions()


def test_host_only_entry_points(lib):
    o = slm.Options()
    lib.slm_default_options(o)
    assert (o.seed, o.accept_p32, o.max_sweeps, o.max_levels, o.flags) == (1, 1 << 31, 1000, 64, 0)
    assert lib.slm_status_string(2) == b"matrix not symmetric"
    # NULL handles are rejected without touching a device
    assert lib.slm_run(None, None, None) == 1
    assert lib.slm_num_levels(None, None) == 1


def test_server_host_entry_points(lib):
    # the admission estimate is a pure host function, growing with n and nnz
    f = [slm.footprint(n, e) for n, e in ((0, 0), (1000, 16000), (2000, 16000), (2000, 32000))]
    assert f[0] == 64 << 20
    assert f[0] < f[1] < f[2] < f[3]
    # arguments are checked before any device is touched
    h = slm.C.c_void_p()
    assert lib.slm_server_create(1 << 30, 0, slm.C.byref(h)) == 1
    assert lib.slm_server_create(0, 4, slm.C.byref(h)) == 1
    assert not h.value
    assert lib.slm_server_submit(None, None, None, None) == 1
    assert lib.slm_server_poll(None, 1, None) == 1
    lib.slm_server_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(slm, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(slm, "_lib", None)
    with pytest.raises(RuntimeError):
        slm.load()


def _create(lib, n, rp, col=None, w=None):
    h = slm.C.c_void_p()
    arr = [None if x is None else np.ascontiguousarray(x, np.int32) for x in (rp, col, w)]
    ptr = [None if a is None else a.ctypes.data_as(slm.C.c_void_p) for a in arr]
    st = lib.slm_create_graph(n, ptr[0], ptr[1], ptr[2], 0, None, slm.C.byref(h))
    return st, h


def test_csr_shape_is_checked_on_the_host(lib):
    # row_ptr must start at 0 and never decrease; n >= 0; col_idx present when
    # there are entries: all refused with INVALID_ARGUMENT before any device call
    assert _create(lib, 2, [1, 1, 2], [0, 1], [1, 1])[0] == 1
    assert _create(lib, 2, [0, 2, 1], [0, 1], [1, 1])[0] == 1
    assert _create(lib, -1, [0])[0] == 1
    assert _create(lib, 2, [0, 1, 2])[0] == 1
    st, h = _create(lib, 2, [0, 1, 2], [1, 0], [1, 1])
    # a valid graph needs a device: created where there is one, SLM_ERR_CUDA where not
    assert st in (0, 5)
    if st == 0:
        lib.slm_destroy_graph(h)
    else:
        assert not h.value


def test_forest_offsets_are_checked_on_the_host(lib):
    def create(goff, rp, col=(1, 0), w=(1, 1)):
        arr = [np.ascontiguousarray(x, np.int32) for x in (goff, rp, col, w)]
        p = [a.ctypes.data_as(slm.C.c_void_p) for a in arr]
        h = slm.C.c_void_p()
        st = lib.slm_batch_create(len(goff) - 1, p[0], p[1], p[2], p[3], None, 0, None,
                                  slm.C.byref(h))
        return st, h
    assert create([1, 2], [0, 1, 2])[0] == 1          # graph_off[0] != 0
    assert create([0, 2, 1], [0, 1, 2])[0] == 1       # decreasing graph_off
    assert create([0, 2], [1, 1, 2])[0] == 1          # row_ptr[0] != 0
    assert create([0, 2], [0, 2, 1])[0] == 1          # decreasing row_ptr
    st, h = create([0, 2], [0, 1, 2])
    assert st in (0, 5)
    if st == 0:
        lib.slm_batch_destroy(h)
    else:
        assert not h.value
