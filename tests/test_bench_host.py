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


def _paper_steps(n, bc, esz):
    """The §3 step list as separate kernels, each reading its input and writing
    its output once (written out step by step)."""
    n1, n2, n3 = n
    free = [b == "f" for b in bc]
    S1, S2, S3 = [2 * v if f else v for v, f in zip(n, free)]
    c = S1 // 2 + 1
    r, cx = esz, 2 * esz
    N = n1 * n2 * n3
    steps = []
    if free[0]:
        steps.append(("spread_X", N * r, S1 * n2 * n3 * r))
    steps.append(("1DFFT_X R2C", S1 * n2 * n3 * r, c * n2 * n3 * cx))
    steps.append(("transpose(+spread)_Y", c * n2 * n3 * cx, c * S2 * n3 * cx))
    steps.append(("1DFFT_Y", c * S2 * n3 * cx, c * S2 * n3 * cx))
    steps.append(("transpose(+spread)_Z", c * S2 * n3 * cx, c * S2 * S3 * cx))
    steps.append(("1DFFT_Z", c * S2 * S3 * cx, c * S2 * S3 * cx))
    steps.append(("kernel multiplication", c * S2 * S3 * cx + c * S2 * S3 * r, c * S2 * S3 * cx))
    steps.append(("inverse 1DFFT_Z", c * S2 * S3 * cx, c * S2 * S3 * cx))
    steps.append(("compaction_Z+transpose", c * S2 * S3 * cx, c * S2 * n3 * cx))
    steps.append(("inverse 1DFFT_Y", c * S2 * n3 * cx, c * S2 * n3 * cx))
    steps.append(("compaction_Y+transpose", c * S2 * n3 * cx, c * n2 * n3 * cx))
    steps.append(("inverse 1DFFT_X C2R", c * n2 * n3 * cx, S1 * n2 * n3 * r))
    if free[0]:
        steps.append(("compaction_X", S1 * n2 * n3 * r, N * r))
    return sum(rd + wr for _, rd, wr in steps)


@pytest.mark.parametrize("n,bc,dt", CASES)
def test_paper_unfused_bytes_follow_the_step_list(n, bc, dt):
    info = ps.Plan(n, bc, 0.3, dt, build=False).info()
    esz = 4 if dt == "f32" else 8
    assert bench._paper_unfused_bytes(info, esz) == _paper_steps(n, bc, esz)


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
