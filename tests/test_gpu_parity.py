"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 and relative max error of V over the physical grid,
and relative error of the energy): 1e-12 for FP64 plans, 1e-5 for FP32 plans.
Sizes span several CTA tiles with ragged tails; full-size cases compare
sampled points with the literal Eq. 2 sum and check properties that hold at
any size.
"""
import numpy as np
import pytest

from oracle import poisson as op
from paper_1211_5244_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
ALL_BCS = ["fff", "pff", "fpf", "ffp", "ppf", "pfp", "fpp", "ppp"]


@pytest.fixture(scope="module")
def torch_cuda(gpu_lib):
    import torch
    return torch


def _np_dtype(dtype):
    return np.float32 if dtype == "f32" else np.float64


XFIRST = (0, 1, 2)  # the processing order of the specialised FP32 kernels (x, then y, then z)


def _gpu_solve(torch, rho, bc, h, dtype, L=None, order=None):
    from paper_1211_5244_gb300 import psolver
    n = rho.shape[::-1]
    plan = psolver.Plan(n, bc, h, dtype, L=L, order=order)
    r = torch.from_numpy(np.ascontiguousarray(rho.astype(_np_dtype(dtype)))).cuda()
    V, E = plan.solve(r)
    torch.cuda.synchronize()
    return V.double().cpu().numpy(), float(E.item()), plan


def _errs(V, Vo):
    rel_l2 = np.linalg.norm(V - Vo) / np.linalg.norm(Vo)
    rel_max = np.abs(V - Vo).max() / np.abs(Vo).max()
    return rel_l2, rel_max


def _check(V, E, rho, bc, h, dtype, L=None):
    # the oracle sees the density the GPU saw (rounded to the plan dtype)
    rho_seen = rho.astype(_np_dtype(dtype)).astype(np.float64)
    Vo, Eo = op.solve(rho_seen, bc, h, L=L)
    l2, mx = _errs(V, Vo)
    eerr = abs(E - Eo) / abs(Eo)
    tol = TOL[dtype]
    assert l2 <= tol and mx <= tol and eerr <= tol, (bc, dtype, l2, mx, eerr)
    return l2, mx, eerr


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("n", [(37, 29, 23), (16, 40, 9), (1, 7, 5), (33, 1, 18)])
def test_parity_ragged(torch_cuda, n, bc, dtype):
    rho = synth.random_density(n, seed=sum(n) + ALL_BCS.index(bc), subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.37, dtype)
    _check(V, E, rho, bc, 0.37, dtype)


ORDERS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("order", ORDERS, ids=lambda o: "".join("xyz"[a] for a in o))
@pytest.mark.parametrize("n,bc", [((13, 10, 7), "fff"), ((12, 9, 15), "pfp"), ((11, 14, 8), "ffp"),
                                  ((16, 7, 10), "ppp"), ((9, 16, 12), "fpf")])
def test_parity_every_processing_order(torch_cuda, n, bc, order, dtype):
    """Every order of the three axis passes (the R2C along x, y or z with the
    pairing of real columns, strided line passes, the fused pass along any
    axis, odd and even lengths) against the FP64 oracle."""
    rho = synth.random_density(n, seed=sum(n) + sum(order), subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.33, dtype, order=order)
    assert tuple(plan.info().order) == order
    _check(V, E, rho, bc, 0.33, dtype)


# x first, then z, then y (the axis rule for pfp, or set by hand): the
# specialised FP32 kernels along z and y through strides, K^F read with its
# ky and kz strides swapped; packed, persistent and register kernels on both.
XZY_CASES = [
    ((64, 128, 64), "pfp", (0, 2, 1)),     # z L = 64 (register y-pass kernel), y L = 256 (persistent unpacked)
    ((128, 256, 256), "pfp", (0, 2, 1)),   # z L = 256 persistent, y L = 512 packed persistent
    ((64, 64, 128), "fff", (0, 2, 1)),     # z L = 256 half, y L = 128 packed
    ((32, 40, 512), "ppf", (0, 2, 1)),     # y periodic 40: generic strided passes, x on the register kernels
]


@pytest.mark.parametrize("n,bc,order", XZY_CASES)
def test_parity_fast_kernels_x_z_y(torch_cuda, n, bc, order):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=61 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", order=order)
    info = plan.info()
    assert tuple(info.order) == order
    pow2 = lambda v: v & (v - 1) == 0
    if pow2(info.L[1]) and pow2(info.L[2]):
        assert all(b > 0 for b in info.blocks), list(info.blocks)  # every pass on a specialised kernel
    _check(V, E, rho, bc, 0.25, "f32")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,bc", [((31, 17, 13), "ppp"), ((29, 23, 11), "pff"), ((157, 5, 6), "pfp"),
                                  ((24, 131, 7), "ppf")])
def test_parity_prime_lengths(torch_cuda, n, bc, dtype):
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=5, noise=1e-3, subtract_mean=True)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.3, dtype)
    _check(V, E, rho, bc, 0.3, dtype)


# Lengths with radix-7 stages (closed-form 7-point butterflies) and prime
# lengths whose Bluestein convolution length has a factor 7: 49 = 7 * 7,
# 343 = 7^3, L1 = 98 (the R2C runs as a 49-point complex transform),
# 11 -> M = 21 (3 * 7), 17 -> 35 (5 * 7), 23 -> 49, 137 -> 280 (8 * 5 * 7),
# 109 -> 224 (8 * 4 * 7); free axes padded to 7-smooth lengths.
RADIX7_CASES = [
    ((49, 21, 343), "ppp", None),
    ((98, 35, 56), "ppp", None),
    ((22, 17, 23), "ppp", None),
    ((137, 12, 10), "pff", None),
    ((8, 109, 6), "fpf", None),
    ((28, 45, 49), "fff", (56, 98, 98)),
    ((30, 7, 31), "fpf", (63, 7, 126)),
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,bc,L", RADIX7_CASES)
def test_parity_radix7_and_bluestein_lengths(torch_cuda, n, bc, L, dtype):
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=13 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.3, dtype, L=L)
    _check(V, E, rho, bc, 0.3, dtype, L=L)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,L", [("fff", (19, 25, 27)), ("pff", (10, 27, 45)), ("ppf", (10, 12, 27))])
def test_parity_other_padded_lengths(torch_cuda, bc, L, dtype):
    n = (10, 12, 14)
    L = tuple(n[j] if bc[j] == "p" else L[j] for j in range(3))
    rho = synth.random_density(n, seed=9, subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.3, dtype, L=L)
    # the physical result does not depend on the padded length (§2)
    _check(V, E, rho, bc, 0.3, dtype)


def test_free32_fp64_workload(torch_cuda):
    w = synth.WORKLOADS["free32_f64"]
    rho = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"])
    V, E, _ = _gpu_solve(torch_cuda, rho, "fff", w["h"], "f64")
    _check(V, E, rho, "fff", w["h"], "f64")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["ppp", "pff", "ppf", "fff"])
def test_bc128_workload(torch_cuda, bc, dtype):
    w = synth.WORKLOADS["bc128"]
    rho = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"],
                                 subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, w["h"], dtype)
    _check(V, E, rho, bc, w["h"], dtype)


@pytest.mark.parametrize("bc", ALL_BCS)
def test_kernel_octant_matches_oracle(torch_cuda, bc):
    from paper_1211_5244_gb300 import psolver
    n = (12, 9, 14)
    plan = psolver.Plan(n, bc, 0.3, "f64")
    K = plan.kernel_octant().cpu().numpy()
    L = op.padded_lengths(n, bc)
    Ko = op.kernel_fourier_octant(n, bc, 0.3) / (L[0] * L[1] * L[2])
    assert K.shape == Ko.shape
    assert np.abs(K - Ko).max() <= 1e-13 * np.abs(Ko).max()


def test_kernel_octant_wire_fine_grid(torch_cuda):
    # many wavenumbers, small h: exercises K0 over a wide argument range
    from paper_1211_5244_gb300 import psolver
    n, h = (64, 20, 20), 0.05
    plan = psolver.Plan(n, "pff", h, "f64")
    K = plan.kernel_octant().cpu().numpy()
    L = op.padded_lengths(n, "pff")
    Ko = op.kernel_fourier_octant(n, "pff", h) / (L[0] * L[1] * L[2])
    assert np.abs(K - Ko).max() <= 1e-13 * np.abs(Ko).max()


@pytest.mark.parametrize("bc", ["fff", "pff", "ppf", "ppp"])
def test_adjoint_is_the_symmetric_solve(torch_cuda, bc):
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    n = (21, 18, 15)
    plan = psolver.Plan(n, bc, 0.3, "f64")
    u = torch.from_numpy(synth.random_density(n, 1)).cuda()
    v = torch.from_numpy(synth.random_density(n, 2)).cuda()
    Ku, _ = plan.solve(u, energy=False)
    KTv = plan.solve_adjoint(v)
    lhs, rhs = float((v * Ku).sum()), float((KTv * u).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    Kv, _ = plan.solve(v, energy=False)
    assert torch.equal(Kv, KTv)


@pytest.mark.parametrize("order", ["lpt", "rr"])
def test_batched_mixed_dtypes_match_oracle(torch_cuda, monkeypatch, order):
    """Every item of a batched solve (FP32 and FP64 plans mixed, more items
    than side streams) against the FP64 oracle, with the items on the side
    streams longest first (the default) or round robin; each item also equals
    its single solve bit for bit."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    if order == "rr":
        monkeypatch.setenv("PS_BATCH_ORDER", "rr")
    shapes = synth.batched_shapes(36, 8, 40, seed=3)
    plans, rhos, dts = [], [], []
    for i, (n, bc) in enumerate(shapes):
        dtype = "f32" if i % 3 else "f64"
        plans.append(psolver.Plan(n, bc, 0.3, dtype))
        r = synth.gaussian_mixture(n, 0.3, 3, seed=i, noise=1e-3, subtract_mean="p" in bc)
        rhos.append(torch.from_numpy(r.astype(_np_dtype(dtype))).cuda())
        dts.append(dtype)
    Vs, Es = psolver.solve_batched(plans, rhos)
    torch.cuda.synchronize()
    for (n, bc), dt, r, V, E, p in zip(shapes, dts, rhos, Vs, Es, plans):
        _check(V.double().cpu().numpy(), float(E.item()), r.double().cpu().numpy(), bc, 0.3, dt)
        V1, E1 = p.solve(r)
        assert torch.equal(V, V1) and torch.equal(E, E1)


def test_batched_every_assignment_matches_oracle(torch_cuda):
    """A batch over all 8 free/periodic assignments (each plan in the axis
    rule's order, so generic strided passes, the specialised kernels and the
    x z y order share one graph), FP32 and FP64, against the oracle."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    plans, rhos, meta = [], [], []
    for i, bc in enumerate(ALL_BCS):
        for dtype, n in (("f32", (32, 64, 32)), ("f64", (14 + i, 11, 9 + i))):
            plans.append(psolver.Plan(n, bc, 0.3, dtype))
            r = synth.gaussian_mixture(n, 0.3, 3, seed=70 + i, noise=1e-3, subtract_mean="p" in bc)
            rhos.append(torch.from_numpy(r.astype(_np_dtype(dtype))).cuda())
            meta.append((bc, dtype))
    Vs, Es = psolver.solve_batched(plans, rhos)
    torch.cuda.synchronize()
    for (bc, dtype), r, V, E in zip(meta, rhos, Vs, Es):
        _check(V.double().cpu().numpy(), float(E.item()), r.double().cpu().numpy(), bc, 0.3, dtype)


@pytest.mark.parametrize("n,bc", [((64, 64, 32), "ffp"), ((32, 64, 64), "fpp")])
def test_autotuned_order_matches_oracle(torch_cuda, n, bc):
    """FP32 power-of-two shapes whose rule order starts with y or z: the
    autotuner may keep the rule's order or take x first (the specialised
    kernels); either way the result is the oracle's."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    rule = psolver.Plan(n, bc, 0.3, "f32", build=False).info().order
    plan = psolver.Plan(n, bc, 0.3, "f32", autotune=True)
    assert tuple(plan.info().order) in (tuple(rule), (0, 1, 2))
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=9, noise=1e-3, subtract_mean=True)
    V, E = plan.solve(torch.from_numpy(rho.astype(np.float32)).cuda())
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.3, "f32")


def test_batched_c4_workload_matches_oracle(torch_cuda):
    """The uneven batch of the benchmark recipe: 64 FP32 problems, n ~ U{24..160}
    per axis (primes such as 131, 137 and 157 among them), boundary conditions
    drawn over free, wire, surface and periodic, autotuned plans, one batched
    call; every item's V and E against the FP64 oracle."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    w = synth.WORKLOADS["batched64"]
    shapes = synth.batched_shapes(w["count"], w["nmin"], w["nmax"], w["seed"])
    assert {bc for _, bc in shapes} == {"fff", "pff", "ppf", "ppp"}
    assert {131, 137, 157} <= {v for n, _ in shapes for v in n}
    plans, rhos = [], []
    for i, (n, bc) in enumerate(shapes):
        plans.append(psolver.Plan(n, bc, w["h"], "f32", autotune=True))
        r = synth.gaussian_mixture(n, w["h"], w["n_gauss"], w["seed"] + i, noise=w["noise"],
                                   subtract_mean="p" in bc)
        rhos.append(torch.from_numpy(r.astype(np.float32)).cuda())
    Vs, Es = psolver.solve_batched(plans, rhos)
    torch.cuda.synchronize()
    worst = 0.0
    for (n, bc), r, V, E in zip(shapes, rhos, Vs, Es):
        l2, mx, ee = _check(V.double().cpu().numpy(), float(E.item()), r.double().cpu().numpy(), bc, w["h"], "f32")
        worst = max(worst, l2, mx, ee)
    assert worst <= TOL["f32"]


def test_host_path_matches_oracle(torch_cuda):
    """ps_solve_host (pinned host buffers in and out) against the FP64 oracle,
    and bit for bit against the device solve of the same plan."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    n = (40, 33, 27)
    plan = psolver.Plan(n, "fff", 0.3, "f32")
    rho_np = synth.gaussian_mixture(n, 0.3, 3, 4).astype(np.float32)
    rho = torch.from_numpy(rho_np)
    Vh, Eh = plan.solve_host(rho.pin_memory())
    _check(Vh.double().numpy(), Eh, rho_np, "fff", 0.3, "f32")
    Vd, Ed = plan.solve(rho.cuda())
    assert torch.equal(Vh, Vd.cpu()) and Eh == float(Ed.item())


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_host_path_full_size_matches_oracle(torch_cuda, dtype):
    """ps_solve_host on a 128^3 wire density (the specialised FP32 kernels, or
    the FP64 generic ones) against the FP64 oracle."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    w = synth.WORKLOADS["bc128"]
    rho_np = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"],
                                    subtract_mean=True).astype(_np_dtype(dtype))
    plan = psolver.Plan(w["n"], "pff", w["h"], dtype)
    Vh, Eh = plan.solve_host(torch.from_numpy(rho_np).pin_memory())
    _check(Vh.double().numpy(), Eh, rho_np, "pff", w["h"], dtype)


@pytest.mark.parametrize("name", ["free256_f32", "free512_f32"])
def test_full_size_free_sampled(torch_cuda, name):
    """Full-size free BCs in FP32, the benchmark's launch configuration:
    sampled points against the literal Eq. 2 sum in FP64, and the energy
    against 1/2 h^3 sum rho V formed in FP64 from the GPU's own V."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    w = synth.WORKLOADS[name]
    rho = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"])
    rho32 = rho.astype(np.float32)
    plan = psolver.Plan(w["n"], "fff", w["h"], "f32")
    V, E = plan.solve(torch.from_numpy(rho32).cuda())
    Vh = V.double().cpu().numpy()
    n3, n2, n1 = rho.shape
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (n3 - 1, n2 - 1, n1 - 1), (n3 // 2, n2 // 2, n1 // 2)]
    pts += [tuple(int(v) for v in rng.integers(0, [n3, n2, n1])) for _ in range(3 if n1 > 256 else 9)]
    ref = op.direct_at(rho32.astype(np.float64), w["h"], pts)
    got = np.array([Vh[p] for p in pts])
    scale = np.abs(Vh).max()
    assert np.abs(got - ref).max() <= TOL["f32"] * scale
    e_direct = 0.5 * w["h"] ** 3 * float(np.sum(rho32.astype(np.float64) * Vh))
    assert abs(float(E.item()) - e_direct) <= TOL["f32"] * abs(e_direct)


# Power-of-two padded lengths above 2n (any L >= 2n - 1 is exact, §2): the
# specialised kernels then see physical counts below L/2, inputs beyond them
# zero and outputs beyond them not stored.
PADDED_CASES = [
    ((42, 50, 100), "fff", (128, 128, 256)),  # x M=64 (n1=42), y L=128 (n2=50), z L=256 (n3=100)
    ((30, 45, 200), "pff", (30, 128, 512)),   # y odd n2=45, z persistent packed (n3=200)
    ((60, 33, 130), "fff", (128, 128, 512)),  # n3=130 with the persistent z kernel
    ((100, 64, 7), "fff", (256, 128, 14)),    # x M=128 (n1=100), z generic
    ((8, 300, 8), "ffp", (16, 1024, 8)),      # y L=1024 (n2=300)
    ((33, 5, 300), "fff", (66, 64, 1024)),    # z L=1024 (n3=300: physical rows end mid-sweep)
    ((16, 100, 16), "fff", (32, 256, 32)),    # y persistent L=256 (n2=100)
    ((24, 20, 60), "fff", (64, 64, 128)),     # z packed L=128 (n3=60), x M=32 (n1=24)
    ((18, 9, 31), "fff", (64, 64, 64)),       # odd n2, n3; L=64 y and z
]


@pytest.mark.parametrize("n,bc,L", PADDED_CASES)
def test_parity_padded_below_half(torch_cuda, n, bc, L):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=13 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", L=L, order=XFIRST)
    assert list(plan.info().L) == list(L)
    # the specialised kernels take the padded passes
    blocks = list(plan.info().blocks)
    assert blocks[1] > 0 and blocks[3] > 0, blocks
    _check(V, E, rho, bc, 0.25, "f32", L=L)


# Lengths 3 * 2^k with register kernels: 384 = 12 x 32 (the factor 3 of 2n at
# n = 192; the packed z kernel with 12-point steps 1 and 4, half and full
# inputs, a ragged last kx tile, an odd L2, the z-pass kernel along y), the
# packed y and the x kernels at 384, and the unpacked y / z kernels at 96 and
# 192 and x kernels at 96 and 192 (M = 48, 96), with masked counts.
LEN384_CASES = [
    ((40, 36, 192), "fff", (80, 72, 384), XFIRST),
    ((24, 20, 150), "fff", (48, 40, 384), XFIRST),   # n3 = 150 < L3/2: masked rows
    ((30, 17, 384), "ffp", (60, 34, 384), XFIRST),   # periodic z, all 384 rows
    ((12, 7, 192), "fpf", (24, 7, 384), XFIRST),     # odd L2 = 7
    ((20, 192, 64), "pfp", (20, 384, 64), (0, 2, 1)),  # z-pass kernel along the free y axis
    ((192, 10, 12), "fff", (384, 20, 24), XFIRST),     # x R2C / C2R at M = 192 = 24 x 8
    ((384, 6, 8), "pff", (384, 12, 16), XFIRST),       # periodic x, all 384 reals
    ((150, 6, 8), "fff", (384, 12, 16), XFIRST),       # n1 = 150 < L1/2
    ((191, 5, 6), "fff", (384, 10, 12), XFIRST),       # odd n1
    ((20, 192, 12), "fff", (40, 384, 24), XFIRST),     # packed y passes at L2 = 384
    ((20, 384, 10), "fpf", (40, 384, 20), XFIRST),     # periodic y, all 384 rows
    ((24, 150, 10), "fff", (48, 384, 20), XFIRST),     # n2 = 150 < L2/2: masked rows
    ((20, 32, 384), "pfp", (20, 64, 384), (0, 2, 1)),  # y-pass kernels along z
    ((192, 192, 48), "fff", (384, 384, 96), XFIRST),   # x and y at 384 together, z at 96
    ((20, 96, 96), "fff", (40, 192, 192), XFIRST),     # y and z at 192
    ((16, 12, 192), "ffp", (32, 24, 192), XFIRST),     # periodic z of 192
    ((20, 70, 80), "fff", (40, 192, 192), XFIRST),     # counts below L/2 at 192
    ((24, 48, 48), "fff", (48, 96, 96), XFIRST),       # y and z at 96
    ((10, 96, 30), "fpf", (20, 96, 60), XFIRST),       # periodic y of 96
    ((96, 10, 12), "fff", (192, 20, 24), XFIRST),      # x at M = 96
    ((192, 6, 8), "pff", (192, 12, 16), XFIRST),       # periodic x of 192
    ((70, 6, 8), "fff", (192, 12, 16), XFIRST),        # n1 = 70 < 96
    ((48, 10, 12), "fff", (96, 20, 24), XFIRST),       # x at M = 48
    ((41, 6, 8), "fff", (96, 12, 16), XFIRST),         # odd n1 at M = 48
    ((96, 96, 96), "fff", (192, 192, 192), XFIRST),    # every pass at 192
    ((20, 32, 96), "pfp", (20, 64, 96), (0, 2, 1)),    # y-pass kernels along the periodic z axis of 96
]


@pytest.mark.parametrize("n,bc,L,order", LEN384_CASES)
def test_parity_length_3x2k_kernels(torch_cuda, n, bc, L, order):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=41 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", L=L, order=order)
    info = plan.info()
    assert list(info.L) == list(L)
    # the specialised kernel of every pass along an axis of length 3 * 2^k ran
    along = [info.order[0], info.order[1], info.order[2]]  # axes of the x, y and z passes
    for passes, axis in (((0, 4), along[0]), ((1, 3), along[1]), ((2,), along[2])):
        if L[axis] in (96, 192, 384):
            assert all(info.blocks[k] > 0 for k in passes), (passes, list(info.blocks))
    _check(V, E, rho, bc, 0.25, "f32", L=L)


def test_hartree_shape_on_length_384(torch_cuda):
    """The 192^3 free grid of the Hartree workload at the paper's 2n = 384 on
    every axis (the specialised kernels of all five passes), full grid against
    the oracle."""
    n = (192, 192, 192)
    rho = synth.gaussian_mixture(n, 0.3, 8, seed=501, noise=1e-3)
    V, E, plan = _gpu_solve(torch_cuda, rho, "fff", 0.3, "f32")
    assert list(plan.info().L) == [384, 384, 384]
    assert all(b > 0 for b in plan.info().blocks), list(plan.info().blocks)
    _check(V, E, rho, "fff", 0.3, "f32")


# Periodic prime lengths whose Bluestein convolution takes the register form at
# 96, 192 and 384 (3 * 2^k, at least 2N) along each axis, FP32; FP64 plans keep
# the Stockham stages
BLUE3_CASES = [
    ((37, 89, 131), "ppp", "f32"),   # x M = 96, y M = 192, z M = 384
    ((157, 47, 179), "ppp", "f32"),  # 384, 96, 384
    ((89, 11, 12), "pff", "f32"),    # wire x of 89 (M = 192)
    ((37, 89, 131), "ppp", "f64"),
]


@pytest.mark.parametrize("n,bc,dtype", BLUE3_CASES)
def test_parity_bluestein_register_lengths(torch_cuda, n, bc, dtype):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=71 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.25, dtype)
    _check(V, E, rho, bc, 0.25, dtype)


# The unpacked L3 = 1024 z kernel (32 x 32) with counts below and at L3/2, an
# odd L2, a ragged kx tile, and all 1024 rows physical
SPLIT1024_CASES = [
    ((20, 12, 512), "fff", (40, 24, 1024)),    # n3 = L3/2
    ((9, 7, 400), "fpf", (18, 7, 1024)),       # n3 = 400 < 512, odd L2, a ragged kx tile
    ((6, 5, 1024), "ffp", (12, 10, 1024)),     # periodic z of 1024
]


@pytest.mark.parametrize("n,bc,L", SPLIT1024_CASES)
def test_parity_z_length_1024(torch_cuda, n, bc, L):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=61 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", L=L, order=XFIRST)
    assert plan.info().blocks[2] > 0
    _check(V, E, rho, bc, 0.25, "f32", L=L)


# Odd L2 (a periodic y axis of odd length) with the specialised z kernels:
# their tile order pairs ky with L2 - ky and must still visit every ky once.
ODD_L2_CASES = [
    ((12, 5, 64), "fpf"),     # z L=128 half (packed), L2 = 5
    ((8, 7, 256), "fpf"),     # z L=512 half (persistent packed), L2 = 7
    ((6, 9, 512), "fpp"),     # z L=512 full, L2 = 9
    ((10, 3, 32), "fpf"),     # z L=64 half (register kernel), L2 = 3
]


@pytest.mark.parametrize("n,bc", ODD_L2_CASES)
def test_parity_odd_y_length_fast_z(torch_cuda, n, bc):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=7 + sum(n), noise=1e-3, subtract_mean=True)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", order=XFIRST)
    assert plan.info().L[1] % 2 == 1
    _check(V, E, rho, bc, 0.25, "f32")


# odd n1 on the specialised x kernels (rows off the 8-byte grid: reals moved
# one at a time), each x shape (M = 32, 64, 128, 256, 512)
ODD_N1_CASES = [
    ((31, 6, 10), "fff", (64, 12, 20)),
    ((63, 20, 18), "fff", (128, 40, 36)),
    ((127, 9, 7), "fpf", (256, 9, 14)),
    ((255, 6, 5), "fff", (512, 12, 10)),
    ((511, 3, 4), "ffp", (1024, 6, 4)),
]


@pytest.mark.parametrize("n,bc,L", ODD_N1_CASES)
def test_parity_odd_n1_fast_x(torch_cuda, n, bc, L):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=37 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", L=L, order=XFIRST)
    assert plan.info().blocks[0] > 0 and plan.info().blocks[4] > 0  # the specialised x kernels ran
    _check(V, E, rho, bc, 0.25, "f32", L=L)


# The fused x/y kernels (thread-block clusters of 16 CTAs exchanging a z plane
# through distributed shared memory): L1 = 512 with n1 = 256 (free x) or 512
# (periodic x), L2 = 512 with n2 = 256 (free y); the z pass on every kind of
# kernel (generic, register, packed, persistent, tensor-core).
FUSED_CASES = [
    ((256, 256, 5), "fff", "cudacore"),    # z generic (L3 = 10)
    ((256, 256, 32), "fff", "cudacore"),   # z L3 = 64 register kernel
    ((512, 256, 7), "pff", "cudacore"),    # periodic x (n1 = 512), z generic
    ((256, 256, 24), "ffp", "cudacore"),   # periodic z
    ((256, 256, 64), "fff", "cudacore"),   # z packed L3 = 128
    ((256, 256, 256), "fff", "tf32x3"),    # the tensor-core z pass
]


@pytest.mark.parametrize("n,bc,math", FUSED_CASES)
def test_parity_fused_xy(torch_cuda, n, bc, math):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=43 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    # not the default schedule (the separate passes are faster)
    plan = psolver.Plan(n, bc, 0.25, "f32", math=math, schedule={"xy": 1}, order=XFIRST)
    info = plan.info()
    assert info.fused == (1 << 1) | (1 << 4) and info.launches == 3, (info.fused, info.launches)
    r = torch.from_numpy(rho.astype(np.float32)).cuda()
    V, E = plan.solve(r)
    if math == "tf32x3":
        plan.device_status()
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.25, "f32")
    # repeatable: every CTA computes the same values on every call
    V2 = torch.empty_like(V)
    plan.solve(r, V2)
    assert torch.equal(V, V2)


# The x and y passes chunk by chunk of z planes (x then y per chunk forward,
# y then x inverse, through one chunk of A): ragged last chunks, one plane per
# chunk, and the default count of the 256^3 workload.
CHUNK_CASES = [
    ((256, 256, 20), "fff", 3, 3),     # chunks of 7, 7, 6 planes (y packed persistent L = 512)
    ((64, 128, 40), "fff", 4, 4),      # y unpacked persistent L = 256, x M = 64
    ((128, 128, 17), "pff", 17, 17),   # one plane per chunk
    ((80, 256, 24), "ppf", 5, 1),      # x M = 40 on the generic kernels: chunks do not apply
    ((96, 256, 24), "ppf", 5, 5),      # x M = 48 (12 x 4 register kernels) in chunks
    ((256, 512, 12), "fpf", 2, 2),     # y packed full L = 512
]


@pytest.mark.parametrize("n,bc,chunks,used", CHUNK_CASES)
def test_parity_chunked_xy_passes(torch_cuda, n, bc, chunks, used):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=53 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    plan = psolver.Plan(n, bc, 0.25, "f32", schedule={"chunks": chunks}, order=XFIRST)
    info = plan.info()
    assert info.chunks == used, (info.chunks, list(info.blocks))
    V, E = plan.solve(torch.from_numpy(rho.astype(np.float32)).cuda())
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.25, "f32")


@pytest.mark.parametrize("n,bc,off", [((64, 48, 40), "fff", 1), ((128, 20, 18), "pff", 1), ((512, 6, 5), "fff", 1),
                                      ((256, 256, 6), "fff", 1), ((256, 256, 6), "fff", 2)])
def test_parity_rho_v_not_8_byte_aligned(torch_cuda, n, bc, off):
    """rho and V starting 4 bytes past an 8-byte boundary (valid FP32
    pointers): the x passes, whose specialised kernels move pairs of reals,
    run the generic kernels with their own launch configuration; 8 bytes past
    a 16-byte boundary: the separate specialised x and y kernels run where the
    fused ones (16-byte copies of rho) would."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=31 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    rho32 = rho.astype(np.float32)
    size = rho32.size
    rbuf = torch.zeros(size + off, dtype=torch.float32, device="cuda")
    vbuf = torch.zeros(size + off, dtype=torch.float32, device="cuda")
    r = rbuf[off:].view(rho32.shape)
    V = vbuf[off:].view(rho32.shape)
    r.copy_(torch.from_numpy(rho32))
    assert r.data_ptr() % 16 == 4 * off and V.data_ptr() % 16 == 4 * off
    plan = psolver.Plan(n, bc, 0.25, "f32", schedule={"xy": 1})  # fused kernels where they apply must step aside
    assert plan.info().blocks[0] > 0  # the plan has the specialised x kernels
    _, E = plan.solve(r, V)
    torch.cuda.synchronize()
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.25, "f32")


# c - 1 a multiple of the kx tile width: the last kx column (kx = L1/2) is the
# only valid line of its tile in the persistent packed y and z kernels; odd
# plane and ky-row counts.
LAST_COLUMN_CASES = [
    ((32, 256, 13), "fff"),   # y L=512 half, c = 33, 13 z planes in one last-column tile
    ((64, 512, 20), "fpf"),   # y L=512 full, c = 65, 20 z planes
    ((32, 13, 256), "fpf"),   # z L=512 half, c = 33, L2 = 13 ky rows
    ((64, 6, 512), "ffp"),    # z L=512 full, c = 65, L2 = 12
]


@pytest.mark.parametrize("n,bc", LAST_COLUMN_CASES)
def test_parity_last_column_tiles(torch_cuda, n, bc):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=29 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", order=XFIRST)
    _check(V, E, rho, bc, 0.25, "f32")


# The tensor-core z pass (PS_MATH_TF32X3, L3 = 512): n3 = 256 (free z) and
# n3 = 512 (periodic z); ragged kx tiles (c not a multiple of 8), odd L2, c = 1.
TC_CASES = [
    ((20, 12, 256), "fff"),   # c = 21
    ((20, 12, 256), "pff"),   # c = 11
    ((9, 5, 256), "fpf"),     # c = 10, L2 = 5
    ((1, 3, 256), "pff"),     # c = 1
    ((6, 7, 512), "ppp"),     # n3 = 512, L2 = 7
    ((16, 6, 512), "ffp"),    # n3 = 512, c = 17
    ((64, 40, 256), "fff"),   # c = 65, L2 = 80
]


def _tc_solve(torch, rho, bc, h):
    from paper_1211_5244_gb300 import psolver
    n = rho.shape[::-1]
    plan = psolver.Plan(n, bc, h, "f32", math="tf32x3", order=XFIRST)
    assert plan.info().tensor_passes == 1 << 2
    r = torch.from_numpy(np.ascontiguousarray(rho.astype(np.float32))).cuda()
    V, E = plan.solve(r)
    plan.device_status()
    return V.double().cpu().numpy(), float(E.item()), plan


@pytest.mark.parametrize("n,bc", TC_CASES)
def test_parity_tensor_core_z(torch_cuda, n, bc):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=11 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, _ = _tc_solve(torch_cuda, rho, bc, 0.25)
    _check(V, E, rho, bc, 0.25, "f32")


def test_tensor_core_mode_elsewhere_stays_on_cuda_cores(torch_cuda):
    """Where no tensor-core kernel exists (here L3 = 256) the mode changes nothing."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    n = (24, 20, 128)
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=3, noise=1e-3)
    r = torch.from_numpy(rho.astype(np.float32)).cuda()
    a = psolver.Plan(n, "fff", 0.3, "f32", math="tf32x3")
    b = psolver.Plan(n, "fff", 0.3, "f32")
    assert a.info().tensor_passes == 0
    Va, Ea = a.solve(r)
    Vb, Eb = b.solve(r)
    assert torch.equal(Va, Vb) and float(Ea.item()) == float(Eb.item())


def test_tensor_core_z_full_size_sampled(torch_cuda):
    """256^3 free FP32 with the tensor-core z pass, in the benchmark's launch
    configuration: sampled points against the literal Eq. 2 sum in FP64, the
    energy against 1/2 h^3 sum rho V from the GPU's own V, and the whole V
    against the CUDA-core solve."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    w = synth.WORKLOADS["free256_f32"]
    rho = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"])
    rho32 = rho.astype(np.float32)
    r = torch.from_numpy(rho32).cuda()
    plan = psolver.Plan(w["n"], "fff", w["h"], "f32", math="tf32x3")
    V, E = plan.solve(r)
    plan.device_status()
    Vh = V.double().cpu().numpy()
    n3, n2, n1 = rho.shape
    rng = np.random.default_rng(1)
    pts = [(0, 0, 0), (n3 - 1, n2 - 1, n1 - 1), (n3 // 2, n2 // 2, n1 // 2)]
    pts += [tuple(int(v) for v in rng.integers(0, [n3, n2, n1])) for _ in range(9)]
    ref = op.direct_at(rho32.astype(np.float64), w["h"], pts)
    got = np.array([Vh[p] for p in pts])
    scale = np.abs(Vh).max()
    assert np.abs(got - ref).max() <= TOL["f32"] * scale
    e_direct = 0.5 * w["h"] ** 3 * float(np.sum(rho32.astype(np.float64) * Vh))
    assert abs(float(E.item()) - e_direct) <= TOL["f32"] * abs(e_direct)
    Vc, _ = psolver.Plan(w["n"], "fff", w["h"], "f32").solve(r)
    l2, mx = _errs(Vh, Vc.double().cpu().numpy())
    assert l2 <= TOL["f32"] and mx <= TOL["f32"], (l2, mx)


# Shapes that select every specialised FP32 kernel: strided lengths 64..1024
# (half = zero-padded free axis, full = periodic axis) and x passes with
# M = L1/2 from 32 to 512.
FAST_CASES = [
    ((32, 32, 32), "fff"),     # x M=32 half, y/z L=64 half
    ((64, 64, 64), "ppp"),     # x M=32 full, y/z L=64 full
    ((128, 64, 32), "pff"),    # x M=64 full, y L=128 half, z L=64 half
    ((64, 128, 128), "fpp"),   # x M=64 half, y/z L=128 full
    ((128, 128, 8), "ffp"),    # x M=128 half, y L=256 half, z generic
    ((256, 8, 256), "ppp"),    # x M=128 full, z L=256 full
    ((512, 4, 128), "pff"),    # x M=256 full, z L=256 half
    ((8, 512, 16), "fpf"),     # y L=512 full
    ((8, 256, 16), "pff"),     # y L=512 half
    ((4, 4, 512), "ffp"),      # z L=512 full
    ((4, 4, 512), "fff"),      # z L=1024 half
    ((4, 3, 1024), "ffp"),     # z L=1024 full
    ((6, 1024, 4), "ppf"),     # y L=1024 full
    ((1024, 4, 6), "pff"),     # x M=512 full
    ((512, 6, 4), "fff"),      # x M=512 half
    ((16, 24, 64), "fff"),     # z L=128 half
    ((12, 10, 128), "ffp"),    # z L=128 full
    ((20, 12, 256), "pff"),    # z L=512 half
    ((10, 256, 6), "ppf"),     # y L=256 full
]


@pytest.mark.parametrize("n,bc", FAST_CASES)
def test_parity_fast_kernels_fp32(torch_cuda, n, bc):
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.25, "f32", order=XFIRST)
    _check(V, E, rho, bc, 0.25, "f32")


@pytest.mark.parametrize("n,bc,dtype", [((60, 37, 29), "fff", "f32"), ((50, 44, 70), "pff", "f32"),
                                        ((33, 40, 27), "ppf", "f64")])
def test_autotuned_plan_matches_oracle(torch_cuda, n, bc, dtype):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    plan = psolver.Plan(n, bc, 0.3, dtype, autotune=True)
    L = list(plan.info().L)
    for j in range(3):
        if bc[j] == "p":
            assert L[j] == n[j]
        else:
            assert L[j] >= 2 * n[j] - 1
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=3, noise=1e-3, subtract_mean="p" in bc)
    r = torch.from_numpy(rho.astype(_np_dtype(dtype))).cuda()
    V, E = plan.solve(r)
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.3, dtype)


@pytest.mark.parametrize("n,bc", [((256, 256, 16), "fff"), ((24, 40, 256), "pff"), ((50, 33, 20), "ppp")])
def test_autotuned_schedule_matches_oracle(torch_cuda, n, bc):
    """Plans whose autotuned schedule has choices to make: the fused x/y
    passes (256 x 256 planes), the tile width of the persistent packed z kernel
    and the y kernel form (L3 = 512), the generic tile width and radix split
    (periodic lengths 50, 33, 20); the chosen plan against the FP64 oracle."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    plan = psolver.Plan(n, bc, 0.3, "f32", autotune=True)
    sched = list(plan.info().schedule)
    assert sched[1] in (0, 1) and sched[2] in (0, 16) and sched[3] in (0, 1, 2) and sched[4] in (0, 1), sched
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=5, noise=1e-3, subtract_mean="p" in bc)
    V, E = plan.solve(torch.from_numpy(rho.astype(np.float32)).cuda())
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.3, "f32")


@pytest.mark.parametrize("radix", [1])
def test_radix4_schedule_matches_oracle(torch_cuda, monkeypatch, radix):
    """The radix-4 split of the generic Stockham stages, forced on plans of
    several generic lengths (powers of two with odd exponents, 2^k 3, a
    Bluestein length), against the FP64 oracle."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    for n, bc, dtype in (((40, 24, 20), "ppp", "f32"), ((17, 12, 24), "fpf", "f64"), ((96, 6, 10), "pff", "f32")):
        plan = psolver.Plan(n, bc, 0.3, dtype, schedule={"radix": radix})
        assert plan.info().schedule[1] == radix
        rho = synth.gaussian_mixture(n, 0.3, 3, seed=9, noise=1e-3, subtract_mean="p" in bc)
        V, E = plan.solve(torch.from_numpy(rho.astype(_np_dtype(dtype))).cuda())
        _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.3, dtype)


def test_host_stream_matches_oracle(torch_cuda):
    """ps_solve_host_stream (uploads, solves and downloads of neighbouring
    densities overlapped): every V and E against the FP64 oracle, and bit for
    bit against the device solves of the same plan."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    n = (48, 40, 36)
    plan = psolver.Plan(n, "pff", 0.3, "f32")
    rhos = [torch.from_numpy(synth.gaussian_mixture(n, 0.3, 3, 20 + i, subtract_mean=True).astype(np.float32))
            .pin_memory() for i in range(5)]
    Vh, Eh = plan.solve_host_stream(rhos)
    for r, v, e in zip(rhos, Vh, Eh):
        _check(v.double().numpy(), e, r.numpy(), "pff", 0.3, "f32")
        Vd, Ed = plan.solve(r.cuda())
        assert torch.equal(v, Vd.cpu()) and e == float(Ed.item())
    assert plan.solve_host_stream([]) == ([], [])


def test_full_grid_headline_matches_oracle(torch_cuda):
    """The benchmark workload itself (256^3 free FP32, padded 512^3, the launch
    configuration bench.py times): the whole V element by element and E
    against the FP64 oracle's full solve."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    w = synth.WORKLOADS["free256_f32"]
    rho32 = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"]).astype(np.float32)
    plan = psolver.Plan(w["n"], "fff", w["h"], "f32")
    V, E = plan.solve(torch.from_numpy(rho32).cuda())
    torch.cuda.synchronize()
    _check(V.double().cpu().numpy(), float(E.item()), rho32, "fff", w["h"], "f32")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,bc", [((1031, 2, 3), "ppp"), ((3, 509, 2), "fpf"), ((2, 3, 257), "ffp"),
                                  ((1571, 2, 3), "ppp"), ((2, 1579, 3), "fpf")])
def test_parity_long_prime_axes(torch_cuda, n, bc, dtype):
    # long prime periodic axes: chirp-z (Bluestein) transforms of length up to
    # 3584; for 1571 and 1579 the cheapest convolution length (3584) does not
    # fit the FP64 tiles' shared memory, and FP64 plans take one that does (3200)
    rho = synth.random_density(n, seed=sum(n), subtract_mean=True)
    V, E, _ = _gpu_solve(torch_cuda, rho, bc, 0.2, dtype)
    _check(V, E, rho, bc, 0.2, dtype)


# Maximum sizes: the longest transform (L = 4096 along y, the generic
# kernels at two lines per tile), and an FP64 x axis whose tile buffers fill
# the shared memory so the twiddles are read from global memory (odd
# L1 = 2625 = 3 * 5^3 * 7: 2626 rows of 16 bytes, two real rows per line).
@pytest.mark.parametrize("n,bc,dtype", [((4, 2048, 3), "ffp", "f32"), ((3, 2048, 2), "ffp", "f64"),
                                        ((2625, 2, 3), "ppp", "f64"), ((2625, 3, 2), "pff", "f32")])
def test_parity_maximum_lengths(torch_cuda, n, bc, dtype):
    rho = synth.gaussian_mixture(n, 0.2, 3, seed=41 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    V, E, plan = _gpu_solve(torch_cuda, rho, bc, 0.2, dtype)
    assert max(plan.info().L) >= 2625
    _check(V, E, rho, bc, 0.2, dtype)


# The schedule choices of ps_plan_set_schedule (which the autotuner picks
# among by timing) and the measurement switches, against the oracle.
SCHEDULES = [
    ({"ztk": 16}, {}),                   # 16 lines per z tile, separate input stage
    ({"ykind": 1}, {}),                  # unpacked persistent y kernels
    ({"ykind": 2}, {}),                  # non-persistent y kernels
    ({"tile": 32}, {}),                  # generic passes: up to 32 lines per tile
    ({"tile": 4}, {}),                   # generic passes: at most 4 lines per tile
    ({"tile": 1, "radix": 1}, {}),       # one line per tile, radix-4 stages
    ({"xy": 1}, {}),                     # fused x/y kernels where they apply (256 x 256 planes)
    ({}, {"PS_L2ORDER": "0"}),           # every pass in forward plane order
    ({}, {"PS_BLUE_M": "min"}),          # smallest 5-smooth Bluestein length (137: 288, not 280)
    ({}, {"PS_BLUE_REGS": "0"}),         # Bluestein on Stockham stages at the cheapest smooth length
]


@pytest.mark.parametrize("sched,env", SCHEDULES,
                         ids=lambda e: ",".join(f"{k}={v}" for k, v in e.items()) or "-")
@pytest.mark.parametrize("n,bc", [((64, 48, 256), "fff"), ((20, 17, 256), "pff"), ((30, 256, 40), "fff"),
                                  ((137, 12, 10), "pff"), ((256, 256, 16), "fff")])
def test_parity_schedules(torch_cuda, monkeypatch, sched, env, n, bc):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    rho = synth.gaussian_mixture(n, 0.25, 4, seed=17 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    plan = psolver.Plan(n, bc, 0.25, "f32", schedule=sched, order=XFIRST)
    V, E = plan.solve(torch.from_numpy(rho.astype(np.float32)).cuda())
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.25, "f32")


# Per-axis generic tiles and radix splits (ps_plan_set_axis_schedule) on
# shapes whose passes run the generic kernels along all three axes (smooth,
# Bluestein in register form and on Stockham stages), FP32 and FP64.
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n,bc,axis_sched", [
    ((45, 27, 35), "ppp", {0: dict(tile=4, radix=1), 1: dict(tile=1), 2: dict(radix=1)}),
    ((37, 61, 139), "ppp", {0: dict(tile=2), 1: dict(radix=1), 2: dict(tile=8, radix=0)}),
    ((29, 23, 11), "pff", {0: dict(tile=1, radix=1), 2: dict(tile=2)}),
    ((61, 50, 37), "ppp", {0: dict(tile=32), 1: dict(tile=32, radix=1), 2: dict(tile=32)}),
])
def test_parity_axis_schedules(torch_cuda, n, bc, axis_sched, dtype):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=23 + sum(n), noise=1e-3, subtract_mean="p" in bc)
    plan = psolver.Plan(n, bc, 0.3, dtype, axis_schedule=axis_sched, order=XFIRST)
    info = plan.info()
    for axis, sched in axis_sched.items():
        assert list(info.axis_schedule[axis]) == [sched.get("tile", 0), sched.get("radix", -1)]
    tdt = torch.float32 if dtype == "f32" else torch.float64
    V, E = plan.solve(torch.from_numpy(rho).to(tdt).cuda())
    _check(V.double().cpu().numpy(), float(E.item()), rho, bc, 0.3, dtype)
