"""Host-side checks of the benchmark's byte and FLOP models (no GPU).

The per-pass algorithmic bytes must add up to the library's count for the
whole solve, and the paper's unfused byte count is recomputed here from the
§3 step list, one kernel at a time.
"""
import math
import os
import sys

import pytest

from paper_1211_5244_gb300 import build as _build
from paper_1211_5244_gb300 import psolver as ps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    _build.build()
    return ps.load_library()


CASES = [((256, 256, 256), "fff", "f32"), ((128, 128, 128), "pff", "f32"), ((96, 40, 70), "ppf", "f64"),
         ((33, 18, 21), "fpf", "f32"), ((16, 16, 16), "ppp", "f64")]


@pytest.mark.parametrize("n,bc,dt", CASES)
def test_pass_bytes_add_up_to_the_solve(n, bc, dt):
    info = ps.Plan(n, bc, 0.3, dt, build=False).info()
    esz = 4 if dt == "f32" else 8
    assert sum(bench._pass_bytes(info, esz)) == pytest.approx(info.alg_bytes, rel=1e-12)


def _paper_steps(n, bc, esz, order):
    """The §3 step list as separate kernels, each reading its input and writing
    its output once (written out step by step), with the axes taken in the
    processing order (first axis a, then b, then c3: x, y, z by default)."""
    a, b, c3 = order
    free = [f == "f" for f in bc]
    S = [2 * v if f else v for v, f in zip(n, free)]
    c = S[a] // 2 + 1
    r, cx = esz, 2 * esz
    N = n[0] * n[1] * n[2]
    steps = []
    if free[a]:
        steps.append(("spread first axis", N * r, S[a] * n[b] * n[c3] * r))
    steps.append(("1DFFT first axis R2C", S[a] * n[b] * n[c3] * r, c * n[b] * n[c3] * cx))
    steps.append(("transpose(+spread) second axis", c * n[b] * n[c3] * cx, c * S[b] * n[c3] * cx))
    steps.append(("1DFFT second axis", c * S[b] * n[c3] * cx, c * S[b] * n[c3] * cx))
    steps.append(("transpose(+spread) third axis", c * S[b] * n[c3] * cx, c * S[b] * S[c3] * cx))
    steps.append(("1DFFT third axis", c * S[b] * S[c3] * cx, c * S[b] * S[c3] * cx))
    steps.append(("kernel multiplication", c * S[b] * S[c3] * cx + c * S[b] * S[c3] * r, c * S[b] * S[c3] * cx))
    steps.append(("inverse 1DFFT third axis", c * S[b] * S[c3] * cx, c * S[b] * S[c3] * cx))
    steps.append(("compaction+transpose third axis", c * S[b] * S[c3] * cx, c * S[b] * n[c3] * cx))
    steps.append(("inverse 1DFFT second axis", c * S[b] * n[c3] * cx, c * S[b] * n[c3] * cx))
    steps.append(("compaction+transpose second axis", c * S[b] * n[c3] * cx, c * n[b] * n[c3] * cx))
    steps.append(("inverse 1DFFT first axis C2R", c * n[b] * n[c3] * cx, S[a] * n[b] * n[c3] * r))
    if free[a]:
        steps.append(("compaction first axis", S[a] * n[b] * n[c3] * r, N * r))
    return sum(rd + wr for _, rd, wr in steps)


@pytest.mark.parametrize("n,bc,dt", CASES)
def test_paper_unfused_bytes_follow_the_step_list(n, bc, dt):
    info = ps.Plan(n, bc, 0.3, dt, build=False).info()
    esz = 4 if dt == "f32" else 8
    assert bench._paper_unfused_bytes(info, esz) == _paper_steps(n, bc, esz, list(info.order))


def test_paper_unfused_bytes_256_free():
    info = ps.Plan((256, 256, 256), "fff", 0.3, "f32", build=False).info()
    assert bench._paper_unfused_bytes(info, 4) == 7947157504
    assert bench._paper_unfused_bytes(info, 4) / info.alg_bytes == pytest.approx(4.37, abs=0.01)


def test_nominal_flops_256_free():
    info = ps.Plan((256, 256, 256), "fff", 0.3, "f32", build=False).info()
    f = bench._pass_flops(info)
    lg = math.log2(512)
    assert f[0] == f[4] == 256 * 256 * 2.5 * 512 * lg
    assert f[1] == f[3] == 257 * 256 * 5 * 512 * lg
    assert f[2] == 257 * 512 * (2 * 5 * 512 * lg + 2 * 512)
