"""GPU parity for a caller's convolution kernel (ps_kernel_set_real).

The same zero-padded convolution with another even kernel (§5: e.g. a local
potential applied to many wave functions): the CUDA path through the C ABI
against the FP64 oracle's convolve, with the tolerances of the solve (1e-12
FP64, 1e-5 FP32).
"""
import numpy as np
import pytest

from oracle import poisson as op
from paper_1211_5244_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def torch_cuda(gpu_lib):
    import torch
    return torch


def _octant(n, bc, seed, width=2.5):
    """An even kernel: a Gaussian of the offset plus a small random even part."""
    L = op.padded_lengths(n, bc)
    rng = np.random.default_rng(seed)
    d = [np.arange(Lj // 2 + 1, dtype=np.float64) for Lj in L]
    r2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
    return np.exp(-r2 / (2 * width ** 2)) + 0.05 * rng.standard_normal(r2.shape)


def _errs(V, Vo):
    return (np.linalg.norm(V - Vo) / np.linalg.norm(Vo), np.abs(V - Vo).max() / np.abs(Vo).max())


CASES = [
    ((37, 29, 23), "fff", "f64", None),
    ((20, 17, 12), "pfp", "f64", None),       # the axis rule's order x z y
    ((9, 14, 11), "ppp", "f64", None),
    ((16, 24, 9), "ppp", "f32", None),
    ((64, 40, 32), "fff", "f32", None),       # specialised FP32 kernels
    ((33, 18, 21), "fpf", "f32", None),       # order y x z: R2C along y, conv along z
    ((24, 16, 20), "ffp", "f64", None),       # order z x y: conv along y
    ((12, 5, 64), "fpf", "f32", (0, 1, 2)),   # x first: odd L2 with the packed z kernel
    ((64, 128, 64), "pfp", "f32", None),      # x z y on the specialised kernels
]


@pytest.mark.parametrize("n,bc,dtype,order", CASES)
def test_custom_kernel_matches_oracle(torch_cuda, n, bc, dtype, order):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    h = 0.3
    k = _octant(n, bc, seed=sum(n))
    rho = synth.gaussian_mixture(n, h, 4, seed=2 + sum(n), noise=1e-3)
    npdt = np.float32 if dtype == "f32" else np.float64
    plan = psolver.Plan(n, bc, h, dtype, order=order).set_kernel_real(k)
    V, E = plan.solve(torch.from_numpy(rho.astype(npdt)).cuda())
    rho_seen = rho.astype(npdt).astype(np.float64)
    Vo, Eo = op.convolve(rho_seen, bc, h, k)
    l2, mx = _errs(V.double().cpu().numpy(), Vo)
    eerr = abs(float(E.item()) - Eo) / abs(Eo)
    tol = TOL[dtype]
    assert l2 <= tol and mx <= tol and eerr <= tol, (l2, mx, eerr)


@pytest.mark.parametrize("n,bc", [((20, 17, 12), "fpf"), ((16, 16, 16), "ppp")])
def test_custom_kernel_octant_is_the_oracle_transform(torch_cuda, n, bc):
    from paper_1211_5244_gb300 import psolver
    k = _octant(n, bc, seed=9)
    plan = psolver.Plan(n, bc, 0.3, "f64").set_kernel_real(k)
    got = plan.kernel_octant().cpu().numpy()
    L = op.padded_lengths(n, bc)
    KF = op.kernel_fourier_from_real(k, n, bc)
    ref = KF.real[: L[2] // 2 + 1, : L[1] // 2 + 1, : L[0] // 2 + 1] / (L[0] * L[1] * L[2])
    assert np.abs(KF.imag).max() <= 1e-12 * np.abs(KF.real).max()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_custom_kernel_many_fields_through_host_stream(torch_cuda):
    """Several fields (wave functions) with one kernel, through the host-buffer
    stream entry point."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    n, bc, h = (40, 24, 32), "fff", 0.25
    k = _octant(n, bc, seed=5, width=1.5)
    plan = psolver.Plan(n, bc, h, "f32").set_kernel_real(k)
    fields = [synth.gaussian_mixture(n, h, 3, seed=40 + i, noise=1e-3).astype(np.float32) for i in range(3)]
    rh = [torch.from_numpy(f).pin_memory() for f in fields]
    Vh = [torch.empty_like(r).pin_memory() for r in rh]
    _, E = plan.solve_host_stream(rh, Vh)
    torch.cuda.synchronize()
    for i, f in enumerate(fields):
        Vo, Eo = op.convolve(f.astype(np.float64), bc, h, k)
        l2, mx = _errs(Vh[i].double().numpy(), Vo)
        assert l2 <= TOL["f32"] and mx <= TOL["f32"], (i, l2, mx)
        assert abs(float(E[i]) - Eo) <= TOL["f32"] * abs(Eo)


def test_custom_kernel_with_tensor_core_z(torch_cuda):
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    n, bc, h = (20, 12, 256), "pff", 0.25
    k = _octant(n, bc, seed=6)
    plan = psolver.Plan(n, bc, h, "f32", math="tf32x3").set_kernel_real(k)
    assert plan.info().tensor_passes == 1 << 2
    rho = synth.gaussian_mixture(n, h, 4, seed=8, noise=1e-3, subtract_mean=True).astype(np.float32)
    V, E = plan.solve(torch.from_numpy(rho).cuda())
    plan.device_status()
    Vo, Eo = op.convolve(rho.astype(np.float64), bc, h, k)
    l2, mx = _errs(V.double().cpu().numpy(), Vo)
    assert l2 <= TOL["f32"] and mx <= TOL["f32"] and abs(float(E.item()) - Eo) <= TOL["f32"] * abs(Eo)


def test_poisson_kernel_restored_by_rebuild_of_a_new_plan(torch_cuda):
    """A custom kernel belongs to its plan: a new plan of the same geometry
    solves Poisson's equation again."""
    from paper_1211_5244_gb300 import psolver
    torch = torch_cuda
    n, bc, h = (18, 14, 10), "fff", 0.3
    rho = synth.gaussian_mixture(n, h, 3, seed=1)
    r = torch.from_numpy(rho).cuda()
    psolver.Plan(n, bc, h, "f64").set_kernel_real(_octant(n, bc, seed=1))
    V, _ = psolver.Plan(n, bc, h, "f64").solve(r)
    Vo, _ = op.solve(rho, bc, h)
    assert _errs(V.cpu().numpy(), Vo)[0] <= TOL["f64"]
