"""The C-ABI library builds, loads and exports every entry point that
include/dgfs.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1903_04670_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    exp = B.exported_symbols()
    assert len(exp) >= 12
    missing = [k for k, v in exp.items() if not v]
    assert not missing, missing


def test_header_declarations_are_extern_c_and_plain():
    hdr = open(os.path.join(ROOT, "include", "dgfs.h")).read()
    assert 'extern "C"' in hdr
    assert "torch" not in hdr.replace("no torch", "")
    for name in re.findall(r"\b(dgfs_[a-z0-9_]+)\s*\(", hdr):
        assert hasattr(B.lib(), name)


def test_status_strings_and_version():
    assert B.dgfs_status_string(0) == "DGFS_OK"
    assert B.dgfs_status_string(4) == "DGFS_ETIMEOUT"
    assert "sm_103a" in B.dgfs_version()


def test_library_is_sm103a_only():
    # the fatbin of the in-tree library carries sm_103a code (checked through
    # the build flags, without reading the binary)
    from paper_1903_04670_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(B.library_path())


def test_argument_errors_without_gpu():
    # invalid arguments are rejected before any device work
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_plan_create(5, 1.0, 6, 4, [1.0], [dict(omega=0.8, alpha=1.0, d=1.0)])
    assert e.value.status in (1, 5)
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_plan_create(8, -1.0, 6, 4, [1.0], [dict(omega=0.8, alpha=1.0, d=1.0)])
    assert e.value.status == 1
    with pytest.raises(B.DgfsError) as e:
        B.dgfs_plan_create(8, 1.0, 7, 4, [1.0], [dict(omega=0.8, alpha=1.0, d=1.0)])
    assert e.value.status == 1
    for mp in (0, 65536):  # the points are one grid dimension of the per-point passes
        with pytest.raises(B.DgfsError) as e:
            B.dgfs_plan_create(8, 1.0, 6, 4, [1.0], [dict(omega=0.8, alpha=1.0, d=1.0)], max_points=mp)
        assert e.value.status == 1
    null = ctypes.c_void_p()
    assert B.lib().dgfs_collide(null, 1, None, None, None) == 1
    assert B.lib().dgfs_plan_destroy(null) == 0
    # schedules: NULL handles
    assert B.lib().dgfs_plan_set_schedule(null, 1) == 1
    assert B.lib().dgfs_plan_get_schedule(null, None) == 1
    assert B.lib().dgfs_batch_set_schedule(null, 0) == 1
    # batches: NULL handles and empty instance lists are argument errors
    out = ctypes.c_void_p()
    assert B.lib().dgfs_batch_create(0, None, None, None, None, 0.0, ctypes.byref(out)) == 1
    assert B.lib().dgfs_batch_launch(null, None) == 1
    assert B.lib().dgfs_batch_destroy(null) == 0
