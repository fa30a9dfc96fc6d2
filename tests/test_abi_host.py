"""Host-side checks of the C ABI: no GPU, no compute calls.

The library must load, export every entry point declared in include/*.h,
validate arguments before touching the device, and describe plans (lengths,
per-pass line counts, work and byte counts) as the paper's §3 does.
"""
import ctypes
import glob
import json
import os
import re

import pytest

from paper_1211_5244_gb300 import build as _build
from paper_1211_5244_gb300 import psolver as ps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ps.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(ps_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(lib, name), name


def _create(lib, n=(8, 8, 8), h=0.3, bc=(1, 1, 1), dtype=0):
    out = ctypes.c_void_p()
    rc = lib.ps_plan_create(n[0], n[1], n[2], h, bc[0], bc[1], bc[2], dtype, ctypes.byref(out))
    return rc, out


@pytest.mark.parametrize("kw", [dict(n=(0, 4, 4)), dict(n=(4, -1, 4)), dict(h=0.0), dict(h=-1.0),
                                dict(h=float("nan")), dict(h=float("inf")), dict(bc=(2, 1, 1)),
                                dict(dtype=3)])
def test_create_rejects_bad_arguments(lib, kw):
    rc, out = _create(lib, **kw)
    assert rc == 1 and not out.value
    assert lib.ps_last_error().decode()


def test_create_null_out_and_too_long(lib):
    assert lib.ps_plan_create(4, 4, 4, 0.3, 1, 1, 1, 0, None) == 1
    rc, out = _create(lib, n=(2049, 4, 4))  # free: L = 4098 > 4096
    assert rc == 2 and not out.value
    rc, out = _create(lib, n=(4096, 4, 4), bc=(0, 1, 1))  # periodic: L = 4096 is fine
    assert rc == 0
    lib.ps_plan_destroy(out)


def test_set_lengths_rules(lib):
    rc, p = _create(lib, n=(10, 12, 7), bc=(0, 1, 1))
    assert rc == 0
    assert lib.ps_plan_set_lengths(p, 11, 0, 0) == 1  # periodic axis must keep n
    assert lib.ps_plan_set_lengths(p, 0, 22, 0) == 1  # free axis needs >= 2n - 1 = 23
    assert lib.ps_plan_set_lengths(p, 0, 23, 15) == 0
    info = ps.PlanInfo()
    assert lib.ps_plan_query(p, ctypes.byref(info)) == 0
    assert list(info.L) == [10, 23, 15] and info.c == 6
    assert lib.ps_plan_set_math(p, 7) == 1
    assert lib.ps_plan_set_math(p, 0) == 0
    assert lib.ps_plan_set_math(p, 1) == 0  # tensor-core mode on an FP32 plan
    assert lib.ps_plan_set_math(p, 2) == 2  # split-BF16 stages: declared, not built
    assert b"BF16" in lib.ps_last_error()
    lib.ps_plan_destroy(p)
    rc, p = _create(lib, n=(10, 12, 7), bc=(0, 1, 1), dtype=1)
    assert rc == 0
    assert lib.ps_plan_set_math(p, 1) == 2  # FP64 plans stay on the CUDA cores
    assert lib.ps_plan_set_math(p, 0) == 0
    lib.ps_plan_destroy(p)


def test_set_schedule_rules(lib):
    rc, p = _create(lib, n=(10, 12, 7), bc=(0, 1, 1))
    assert rc == 0
    for bad in ((3, 0, 0, 0, 0, 0), (64, 0, 0, 0, 0, 0), (0, 2, 0, 0, 0, 0), (0, 0, 4, 0, 0, 0),
                (0, 0, 0, 3, 0, 0), (0, 0, 0, 0, 2, 0), (-1, 0, 0, 0, 0, 0), (0, 0, 0, 0, 0, 65)):
        assert lib.ps_plan_set_schedule(p, *bad) == 1, bad
    assert lib.ps_plan_set_schedule(p, 4, 1, 16, 2, 1, 8) == 0
    info = ps.PlanInfo()
    assert lib.ps_plan_query(p, ctypes.byref(info)) == 0
    assert list(info.schedule) == [4, 1, 16, 2, 1, 8] and info.fused == 0 and info.chunks == 0
    assert lib.ps_plan_set_schedule(None, 0, 0, 0, 0, 0, 0) == 1
    lib.ps_plan_destroy(p)


def test_set_axis_schedule_rules(lib):
    rc, p = _create(lib, n=(10, 12, 7), bc=(0, 1, 1))
    assert rc == 0
    info = ps.PlanInfo()
    assert lib.ps_plan_query(p, ctypes.byref(info)) == 0
    assert [list(a) for a in info.axis_schedule] == [[0, -1]] * 3  # plan-wide choices by default
    for bad in ((3, 0, 0), (-1, 0, 0), (0, 3, 0), (0, 64, 0), (0, -2, 0), (0, 0, 2), (0, 0, -2)):
        assert lib.ps_plan_set_axis_schedule(p, *bad) == 1, bad
    assert lib.ps_plan_set_axis_schedule(p, 1, 4, 1) == 0
    assert lib.ps_plan_set_axis_schedule(p, 2, 0, 0) == 0
    assert lib.ps_plan_query(p, ctypes.byref(info)) == 0
    assert [list(a) for a in info.axis_schedule] == [[0, -1], [4, 1], [0, 0]]
    assert lib.ps_plan_set_axis_schedule(None, 0, 0, 0) == 1
    lib.ps_plan_destroy(p)


def test_solve_on_unbuilt_plan_is_rejected_before_any_launch(lib):
    rc, p = _create(lib)
    fake_in, fake_out = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000)
    assert lib.ps_solve(p, fake_in, fake_out, None, None) == 3
    assert lib.ps_solve_adjoint(p, fake_in, fake_out, None) == 3
    assert lib.ps_kernel_get(p, fake_out, None) == 3
    assert lib.ps_kernel_set_real(p, fake_in, None) == 3
    assert lib.ps_kernel_set_real(None, fake_in, None) == 1
    assert lib.ps_plan_device_status(p, None) == 3
    assert lib.ps_solve(p, None, fake_out, None, None) == 1
    assert lib.ps_solve(None, fake_in, fake_out, None, None) == 1
    arr = ctypes.c_void_p * 1
    assert lib.ps_solve_batched(1, arr(p.value), arr(0x10000), arr(0x20000), None, None) == 3
    assert lib.ps_solve_batched(0, None, None, None, None, None) == 0
    assert lib.ps_solve_batched(-1, None, None, None, None, None) == 1
    assert lib.ps_plan_destroy(p) == 0
    assert lib.ps_plan_destroy(None) == 0


def test_strerror(lib):
    for code in range(7):
        assert lib.ps_strerror(code).decode()
    assert lib.ps_strerror(99).decode() == "unknown status"


GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "work_fractions.json")))


@pytest.mark.parametrize("bc", sorted(GOLDEN["fractions"]))
@pytest.mark.parametrize("n", [8, 64, 256])
def test_work_fraction_matches_section3(bc, n):
    p = ps.Plan((n, n, n), bc, 0.3, "f32", build=False)
    info = p.info()
    assert list(info.order) == GOLDEN["orders"][bc]
    num, den = GOLDEN["fractions"][bc]
    assert info.paper_points * den == info.paper_full_points * num


@pytest.mark.parametrize("bc", sorted(GOLDEN["orders"]))
def test_lines_per_pass_match_listing(bc):
    n = (12, 7, 9)
    p = ps.Plan(n, bc, 0.3, "f64", build=False)
    info = p.info()
    a, b, c = GOLDEN["orders"][bc]
    L = list(info.L)
    env = dict(Sa=L[a], Sb=L[b], Nb=n[b], Nc=n[c])
    rows = {k: eval(v, {}, env) for k, v in GOLDEN["listing_rows"].items()}
    assert list(info.lines) == [rows["first"], rows["second"], rows["third"], rows["second"], rows["first"]]
    assert list(info.line_len) == [L[a], L[b], L[c], L[b], L[a]]
    assert info.c == L[a] // 2 + 1
    for j, bj in enumerate(bc):
        assert info.L[j] == n[j] * (2 if bj == "f" else 1)


@pytest.mark.parametrize("bcs", [("pff", "fpf", "ffp"), ("ppf", "pfp", "fpp")])
def test_axis_assignments_of_one_class_move_the_same_bytes(bcs):
    # with the axis rule the work and the traffic depend on how many axes are
    # periodic, not on which: a cube of one BC class costs the same for each
    # assignment of the axes
    infos = [ps.Plan((64, 64, 64), bc, 0.3, "f32", build=False).info() for bc in bcs]
    assert len({i.alg_bytes for i in infos}) == 1
    assert len({i.paper_points for i in infos}) == 1
    assert len({i.fft_points for i in infos}) == 1


def test_set_order_rules():
    lib = ps.load_library()
    p = ps.Plan((10, 12, 7), "ffp", 0.3, "f32", build=False)
    assert list(p.info().order) == [2, 0, 1]
    for bad in ((0, 0, 1), (0, 1, 3), (-1, 1, 2)):
        assert lib.ps_plan_set_order(p.handle, *bad) == 1
    assert list(p.info().order) == [2, 0, 1]
    assert lib.ps_plan_set_order(p.handle, 0, 1, 2) == 0
    info = p.info()
    assert list(info.order) == [0, 1, 2] and info.c == 11
    assert lib.ps_plan_set_order(None, 0, 1, 2) == 1


def test_algorithmic_bytes_256_free_fp32():
    info = ps.Plan((256, 256, 256), "fff", 0.3, "f32", build=False).info()
    n, c, L = 256 ** 3, 257, 512
    expect = 2 * n * 4 + 8 * 4 * c * 256 * (256 + L) + 4 * c * 257 * 257
    assert info.alg_bytes == expect
    assert abs(info.alg_bytes / 1e9 - 1.819) < 1e-3


def test_autotune_rejects_null_plan(lib):
    assert lib.ps_plan_autotune(None, 5, None) == 1


def test_host_stream_and_vjp_argument_checks(lib):
    rc, p = _create(lib)
    arr = ctypes.c_void_p * 1
    buf = ctypes.create_string_buffer(8 * 8 * 8 * 4)
    assert lib.ps_solve_host_stream(None, 1, arr(ctypes.addressof(buf)), arr(ctypes.addressof(buf)), None, None) == 1
    assert lib.ps_solve_host_stream(p, -1, None, None, None, None) == 1
    assert lib.ps_solve_host_stream(p, 0, None, None, None, None) == 0
    assert lib.ps_solve_host_stream(p, 1, None, None, None, None) == 1
    assert lib.ps_solve_host_stream(p, 1, arr(ctypes.addressof(buf)), arr(None), None, None) == 1
    assert lib.ps_solve_host_stream(p, 1, arr(ctypes.addressof(buf)), arr(ctypes.addressof(buf)), None, None) == 3
    fake = ctypes.c_void_p(0x10000)
    assert lib.ps_solve_vjp(p, None, None, None, fake, None) == 1          # every term omitted
    assert lib.ps_solve_vjp(p, fake, ctypes.c_void_p(0x20000), None, ctypes.c_void_p(0x30000), None) == 1
    assert lib.ps_solve_vjp(p, fake, None, None, ctypes.c_void_p(0x30000), None) == 3  # not built
    lib.ps_plan_destroy(p)
