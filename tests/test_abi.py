"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mpf.h.  Runs without a GPU: only calls that need no
device (status strings, limits, argument checks that fail before any CUDA
call) are made."""
import ctypes
import os
import re

import pytest

from paper_1707_09683_gb300 import build, mpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mpf.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpf_profile_create", "mpf_db_upload", "mpf_msv_scan", "mpf_ssv_scan",
                     "mpf_scan_batch", "mpf_ctx_create", "mpf_sync", "mpf_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(mpf.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    src = open(os.path.join(ROOT, "paper_1707_09683_gb300", "mpf.py")).read()
    for n in declared_functions():
        assert f'"{n}"' in src, f"binding lacks {n}"


def test_status_strings_and_limits(lib):
    assert mpf.strerror(mpf.MPF_OK) == "ok"
    assert mpf.strerror(mpf.MPF_EINVAL) == "invalid argument"
    assert mpf.strerror(99) == "unknown status"
    assert mpf.max_model_length() == 100000
    assert mpf.max_striped_length() == 3072


def test_null_arguments_are_rejected_without_a_device(lib):
    h = ctypes.c_void_p()
    assert lib.mpf_ctx_create(0, None, None) == mpf.MPF_EINVAL
    assert lib.mpf_profile_create(None, 10, 20, None, 0, 0, 0, 0, None, 0, 1.0, 190,
                                  ctypes.byref(h)) == mpf.MPF_EINVAL
    assert lib.mpf_db_upload(None, None, 0, None, None, 0, ctypes.byref(h)) == mpf.MPF_EINVAL
    assert lib.mpf_msv_scan(None, None, None, None, None, None) == mpf.MPF_EINVAL
    assert lib.mpf_plan_launch(None) == mpf.MPF_EINVAL
    assert lib.mpf_plan_group_count(None) == 0
    assert lib.mpf_plan_group_info(None, 0, None, None, None, None, None, None) == mpf.MPF_EINVAL
    assert lib.mpf_sync(None) == mpf.MPF_EINVAL
    lib.mpf_ctx_destroy(None)
    lib.mpf_profile_destroy(None)
    lib.mpf_db_destroy(None)
    lib.mpf_plan_destroy(None)


def test_stage_and_viterbi_calls_reject_null_arguments_without_a_device(lib):
    h = ctypes.c_void_p()
    i16 = (ctypes.c_int16 * 8)()
    assert lib.mpf_vit_profile_create(None, 10, 20, i16, i16, i16, 12000, 721.0,
                                      ctypes.byref(h)) == mpf.MPF_EINVAL
    assert lib.mpf_vit_profile_create(None, 10, 20, i16, i16, i16, 12000, 721.0, None) == mpf.MPF_EINVAL
    assert lib.mpf_viterbi_scan(None, None, 1, None, None, None, None) == mpf.MPF_EINVAL
    assert lib.mpf_viterbi_rescore(None, None, 1, None, None, None, 0.0, None, None, None,
                                   None) == mpf.MPF_EINVAL
    assert lib.mpf_pipeline_scan(None, None, 1, None, 0.0, None, None, None, None, None, None,
                                 None) == mpf.MPF_EINVAL
    assert lib.mpf_pvalues(None, None, 0, 0.0, 1.0, None) == mpf.MPF_EINVAL
    assert lib.mpf_scan_noalloc(None, 0, None, None, None, None, None) == mpf.MPF_EINVAL
    lib.mpf_vit_profile_destroy(None)
