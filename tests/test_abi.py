"""The C-ABI library: it loads, exports every symbol include/membrane.h declares, and rejects bad
arguments before touching the GPU. CPU only (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "membrane.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mb_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_02120_gb300 import build, membrane
    build.build()
    return membrane.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mb_net_create", "mb_load_weights", "mb_infer_volume", "mb_infer_batch", "mb_student_train",
                 "mb_infer_cascade", "mb_calibrate_fp8", "mb_net_destroy", "mb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1612_02120_gb300 import membrane
    so = membrane.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mb_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(membrane.EXPORTED) == set(declared_functions())


def test_status_strings(lib):
    from paper_1612_02120_gb300 import membrane as m
    assert m.status_name(m.MB_OK) == "MB_OK"
    assert m.status_name(m.MB_ERR_SHAPE) == "MB_ERR_SHAPE"
    assert m.status_name(99) == "MB_ERR_UNKNOWN"


def test_null_and_malformed_arguments_fail_before_cuda(lib):
    from paper_1612_02120_gb300 import membrane as m
    out = ctypes.c_void_p()
    assert lib.mb_net_create(None, 6, 0, 0, ctypes.byref(out)) == m.MB_ERR_INVALID_ARG
    bad = m.layer_array([(7, 5, 1, 32, 1)])
    assert lib.mb_net_create(bad, 1, 0, 0, ctypes.byref(out)) == m.MB_ERR_INVALID_ARG
    assert "malformed" in m.last_error()
    import synth
    good = m.layer_array(synth.TEACHER)
    assert lib.mb_net_create(good, 6, 9, 0, ctypes.byref(out)) == m.MB_ERR_INVALID_ARG
    odd = m.layer_array([(0, 7, 1, 8, 1), (2, 1, 8, 1, 0)])
    assert lib.mb_net_create(odd, 2, 0, 0, ctypes.byref(out)) == m.MB_ERR_UNSUPPORTED
    st = m.layer_array(synth.STUDENT)
    assert lib.mb_net_create(st, 3, 2, 0, ctypes.byref(out)) == m.MB_ERR_UNSUPPORTED
    assert lib.mb_net_destroy(None) == m.MB_OK
    assert lib.mb_infer_volume(None, None, 1, 64, 64, None, 0, None) == m.MB_ERR_INVALID_ARG
    n = ctypes.c_int64()
    assert lib.mb_net_param_count(None, ctypes.byref(n)) == m.MB_ERR_INVALID_ARG


def test_launch_counter_starts_at_zero_in_a_fresh_process():
    code = ("from paper_1612_02120_gb300 import membrane as m; print(m.launch_count())")
    r = subprocess.run(["python", "-c", code], capture_output=True, text=True, cwd=ROOT, check=True)
    assert r.stdout.strip() == "0"
