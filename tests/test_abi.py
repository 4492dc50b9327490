"""The C-ABI library loads and exports every entry point include/rqb.h declares
(no GPU needed: only symbol lookup, no compute call)."""
import ctypes
import os
import re

import pytest

from paper_1503_07157_gb300 import build
from paper_1503_07157_gb300 import rqb


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rqb.lib()


def test_library_exports_every_declared_symbol(lib):
    names = rqb.declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"librqb.so does not export {name}"


def test_header_status_codes_match_binding():
    text = open(rqb.HEADER).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"(RQB_[A-Z_]+)\s*=\s*(\d+)", text))
    for k, v in codes.items():
        if hasattr(rqb, k):
            assert getattr(rqb, k) == v, k


def test_status_strings(lib):
    assert rqb.status_string(0) == "ok"
    assert "invalid" in rqb.status_string(rqb.RQB_ERR_INVALID)
    assert rqb.status_string(999) == "unknown status"


def test_struct_layout_matches_header():
    # rqb_config: 2 x int32, int64, 2 x int32, pointer, 2 x int32
    assert ctypes.sizeof(rqb.rqb_config) == 40
    assert ctypes.sizeof(rqb.rqb_stats) == (8 * 2 + 4 * 2 + 8 * 2 + 8 * 2 * rqb.RQB_MAX_TRACKED_BLOCKS + 8
                                            + 8 * rqb.RQB_NUM_PHASES + 4 * rqb.RQB_NUM_PHASES + 4 * 6)


@pytest.mark.parametrize("sname", ["rqb_config", "rqb_stats"])
def test_struct_fields_match_header(sname):
    """The binding's ctypes fields name the header's struct members in the
    header's order (a member added on one side only, or out of order, would
    shift every field after it)."""
    text = re.sub(r"/\*.*?\*/", "", open(rqb.HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct\s*(?:\w+\s*)?\{([^{}]*)\}\s*" + sname + r"\s*;", text)
    assert m, sname
    body = m.group(1)
    members = re.findall(r"\b(?:u?int32_t|u?int64_t|double|float|void)\s*\**\s*(\w+)\s*(?:\[[^\]]*\])?\s*;", body)
    assert [f[0] for f in getattr(rqb, sname)._fields_] == members


def test_null_handle_rejected_without_gpu(lib):
    assert lib.rqb_destroy(None) == rqb.RQB_ERR_INVALID
    assert lib.rqb_get_stats(None, None) == rqb.RQB_ERR_INVALID
    assert lib.rqb_create(None, None) == rqb.RQB_ERR_INVALID


def test_library_is_in_tree():
    assert os.path.dirname(rqb.LIB_PATH) == os.path.dirname(os.path.abspath(rqb.__file__))


@pytest.mark.parametrize("dtype,ncols,m,want_norm,expect", [
    # FP64 products use 64-row tiles: 600000 rows are 9375 norm partials > 8192
    ("f64", 64, 600000, True, "RQB_ERR_SCRATCH_LIMIT"),
    # FP32 at 256 columns also uses 64-row tiles
    ("f32", 256, 600000, True, "RQB_ERR_SCRATCH_LIMIT"),
    # FP32 at 128 columns: 128-row tiles, 1048577 rows need 8193 partials
    ("f32", 128, 1048577, True, "RQB_ERR_SCRATCH_LIMIT"),
    # an Omega block beyond the array is rejected whether or not the norm is asked for
    ("f32", 128, 64, False, "RQB_ERR_SCRATCH_LIMIT"),
])
def test_noalloc_rejects_before_any_launch_without_gpu(lib, dtype, ncols, m, want_norm, expect):
    """The capacity checks run on the host before any CUDA call, so they need no
    GPU: the pointers below are never dereferenced."""
    fake = ctypes.c_void_p(0x10000)
    n = 1 << 20 if m == 64 else 16
    dt = rqb.RQB_F64 if dtype == "f64" else rqb.RQB_F32
    nrm = ctypes.c_double(0.0)
    rc = lib.rqb_sketch_noalloc(dt, fake, m, n, m, 0, ncols, 0, fake, m,
                                ctypes.byref(nrm) if want_norm else None, None)
    assert rc == getattr(rqb, expect), rqb.status_string(rc)


def test_alloc_failure_hook_arguments_without_gpu(lib):
    assert lib.rqb_inject_alloc_failure(-2) == rqb.RQB_ERR_INVALID
    assert lib.rqb_inject_alloc_failure(3) == rqb.RQB_OK
    assert lib.rqb_inject_alloc_failure(-1) == rqb.RQB_OK
