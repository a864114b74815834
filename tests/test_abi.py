"""The C-ABI boundary without a GPU: the library loads, exports every entry
point include/rdct.h declares, and rejects bad arguments before touching the
device."""
import ctypes
import os
import re

import pytest

from paper_1402_6034_gb300 import rdct

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rdct.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^RDCT_API[^(]*?\b(rdct_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rdct_forward", "rdct_compress", "rdct_inverse", "rdct_mse_psnr", "rdct_fused", "rdct_sweep",
                 "rdct_batch_plan_create", "rdct_batch_run", "rdct_autotune", "rdct_server_create",
                 "rdct_server_submit", "rdct_server_wait", "rdct_pipeline_run"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = rdct.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(rdct._SIGS)


def test_status_strings_and_version():
    lib = rdct.load()
    assert lib.rdct_status_string(0) == b"ok"
    assert lib.rdct_status_string(2) == b"invalid shape"
    assert lib.rdct_version() >= 10000


def _last_error():
    buf = ctypes.create_string_buffer(256)
    rdct.load().rdct_last_error(buf, 256)
    return buf.value.decode()


def test_validation_happens_before_any_launch():
    lib = rdct.load()
    bad = rdct.Plane(ctypes.c_void_p(16), 12, 12, 8)  # width not a multiple of 8
    assert lib.rdct_forward(ctypes.byref(bad), ctypes.c_void_p(16), None) == 2
    assert "multiples of 8" in _last_error()
    ok = rdct.Plane(ctypes.c_void_p(16), 16, 16, 8)
    assert lib.rdct_fused(ctypes.byref(ok), 0, 0, None, ctypes.c_void_p(16), None, None) == 1  # r = 0
    assert lib.rdct_fused(ctypes.byref(ok), 65, 0, None, ctypes.c_void_p(16), None, None) == 1  # r = 65
    assert lib.rdct_fused(ctypes.byref(ok), 10, 7, None, ctypes.c_void_p(16), None, None) == 1  # bad kind
    assert lib.rdct_fused(None, 10, 0, None, ctypes.c_void_p(16), None, None) == 1
    # the 8-bit error slot must be aligned and distinct from the SSE slot
    assert lib.rdct_fused(ctypes.byref(ok), 10, 0, None, ctypes.c_void_p(16), ctypes.c_void_p(20), None) == 1
    assert lib.rdct_fused(ctypes.byref(ok), 10, 0, None, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
    short = rdct.Plane(ctypes.c_void_p(16), 8, 16, 8)  # pitch < width
    assert lib.rdct_forward(ctypes.byref(short), ctypes.c_void_p(16), None) == 2
    assert lib.rdct_compress(None, 4, 10, ctypes.c_void_p(16), None) == 1
    assert lib.rdct_compress(ctypes.c_void_p(16), 4, 0, ctypes.c_void_p(16), None) == 1
    job = rdct.Job(ok, None, 0, 10, 5)  # image index out of range
    plan = ctypes.c_void_p()
    assert lib.rdct_batch_plan_create((rdct.Job * 1)(job), 1, 2, None, ctypes.byref(plan)) == 1
    tune = rdct.Tune(64, 0, 8, 2, 0)  # too many warps
    job = rdct.Job(ok, None, 0, 10, 0)
    assert lib.rdct_batch_plan_create((rdct.Job * 1)(job), 1, 1, ctypes.byref(tune), ctypes.byref(plan)) == 1
    tune = rdct.Tune(4, 0, 8, 2, 2)  # unknown staging
    job = rdct.Job(ok, None, 0, 10, 0)
    assert lib.rdct_batch_plan_create((rdct.Job * 1)(job), 1, 1, ctypes.byref(tune), ctypes.byref(plan)) == 1
    opts = rdct.ServerOpts(1024, 1, 1, 1, 0)  # budget below 1 MiB
    srv = ctypes.c_void_p()
    assert lib.rdct_server_create(ctypes.byref(opts), ctypes.byref(srv)) == 1


def test_noalloc_sweep_limits_are_checked_on_the_host():
    lib = rdct.load()
    ok = rdct.Plane(ctypes.c_void_p(16), 16, 16, 8)
    planes = (rdct.Plane * 2049)(*([ok] * 2049))
    assert lib.rdct_sweep_noalloc(planes, 2049, 0, ctypes.c_void_p(16), None) == 4
    assert "2048" in _last_error()


def test_batch_job_errors_name_the_job_and_keep_the_detail():
    lib = rdct.load()
    jobs = (rdct.Job * 2)()
    jobs[0].src = rdct.Plane(ctypes.c_void_p(16), 16, 16, 8)
    jobs[0].r, jobs[0].image = 10, 0
    jobs[1].src = rdct.Plane(ctypes.c_void_p(16), 12, 12, 8)  # width not a multiple of 8
    jobs[1].r, jobs[1].image = 10, 0
    h = ctypes.c_void_p()
    assert lib.rdct_batch_plan_create(jobs, 2, 1, None, ctypes.byref(h)) == 2
    msg = _last_error()
    assert "batch job 1" in msg and "multiples of 8" in msg, msg
    assert not h.value


def test_binding_has_sync():
    assert callable(rdct.sync)
    assert "rdct_sync" in rdct._SIGS


def test_batch_run_rejects_bad_error_slots():
    lib = rdct.load()
    assert lib.rdct_batch_run(None, ctypes.c_void_p(16), None, None) == 1
    assert lib.rdct_batch_run_per_plane(None, ctypes.c_void_p(16), None, None) == 1


def test_batch_plan_kernels_rejects_null():
    lib = rdct.load()
    k = ctypes.c_int32(-1)
    assert lib.rdct_batch_plan_kernels(None, ctypes.byref(k)) == 1
    assert k.value == -1
