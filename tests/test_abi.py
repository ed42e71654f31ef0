"""The C-ABI library loads and exports every entry point include/mf.h declares.

CPU-only: no compute call is made (without a GPU only argument validation
and static queries run).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def mf():
    import __graft_entry__ as g
    g.build()
    import paper_2601_07154_gb300 as m
    return m


def test_every_declared_symbol_is_exported(mf):
    lib = ctypes.CDLL(mf._mf.LIB_PATH)
    names = _declared()
    assert "mf_push_frames" in names and "mf_get_maps" in names and "mf_open_stream" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/mf.h but not exported"
    assert set(mf._mf.EXPORTED) <= set(names)


def test_static_queries(mf):
    assert mf.mf_version() == 1
    assert mf.mf_status_string(mf.MF_ERR_TIMEOUT) == "timeout"
    assert mf.mf_status_string(12345) == "unknown status"
    d = mf.mf_stream_desc_init()
    assert (d.window, d.smooth_len, d.sigma_rel, d.s_lo, d.s_hi, d.depth_ref_m) == \
        (8, 15, 0.1, 0.25, 4.0, 1.0)


@pytest.mark.parametrize("fields", [
    dict(width=0, height=10), dict(width=10, height=10, window=0),
    dict(width=10, height=10, window=33), dict(width=10, height=10, smooth_len=2),
    dict(width=10, height=10, mode=1, smooth_len=1), dict(width=10, height=10, window=32, smooth_len=34),
    dict(width=10, height=10, overlap=2), dict(width=10, height=10, pose_frame=1, overlap=0),
    dict(width=10, height=10, depth_dtype=7), dict(width=10, height=10, sigma_rel=0.0),
    dict(width=10, height=10, s_lo=2.0, s_hi=1.0), dict(width=20000, height=10),
    dict(width=10, height=10, normalize=2), dict(width=10, height=10, normalize=-1),
    dict(width=10, height=10, flags=8 | 16),
])
def test_invalid_descriptors_rejected_before_any_device_work(mf, fields):
    d = mf.mf_stream_desc_init(**fields)
    with pytest.raises(mf.MFError) as e:
        mf.mf_open_stream(d)
    assert e.value.status == mf.MF_ERR_INVALID_ARG


def test_null_arguments(mf):
    assert mf._mf.lib.mf_push_frames(None, 1, None, None, None) == mf.MF_ERR_INVALID_ARG
    assert mf._mf.lib.mf_get_maps(None, 1, None, None, None, None, None, 0) == mf.MF_ERR_INVALID_ARG
    assert mf._mf.lib.mf_close_stream(None) == mf.MF_OK


def test_struct_layouts_match_the_header(mf):
    """ctypes mirrors of the C structs: sizes that the header fixes."""
    import ctypes
    assert ctypes.sizeof(mf._mf.MFStats) == 7 * 8 + 2 * 4
    assert mf._mf.FRAME_INFO_DTYPE.itemsize == 64
    assert mf._mf.MOTION_POINT_DTYPE.itemsize == 40
    assert mf._mf.PUSH_DTYPE.itemsize == 64
    assert mf._mf.MF_FLAG_MAP_CUDA_CORES & mf._mf.MF_FLAG_MAP_TENSOR_CORES == 0
    assert (mf._mf.MF_FLAG_MAP_CUDA_CORES | mf._mf.MF_FLAG_MAP_TENSOR_CORES) & mf._mf.MF_FLAG_TIME_KERNELS == 0


def test_fault_spec_parsing(mf):
    """mf_set_fault accepts rule lists and refuses malformed ones without
    changing the rules in force (host only: no rule fires here)."""
    for spec in ("alloc_fail", "alloc_fail@2", "bad_pose@5,drop_push@1", "admission_full,wait_timeout@3",
                 "", None):
        mf.mf_set_fault(spec)
    for spec in ("nope", "alloc_fail@0", "alloc_fail@", "alloc_fail@x", "bad_pose@-1", "@3"):
        with pytest.raises(mf.MFError) as e:
            mf.mf_set_fault(spec)
        assert e.value.status == mf.MF_ERR_INVALID_ARG, spec
    mf.mf_set_fault(None)
