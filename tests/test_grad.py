"""Gradients through the library's adjoint (ps_solve_vjp behind autograd).

E = 1/2 h^3 <rho, K rho> is exactly quadratic, so central differences in FP64
have no truncation error: they must match <dE/drho, u> to rounding. The
gradient must also equal the oracle's h^3 V, and the VJP through V must be
the symmetric solve of the incoming gradient.
"""
import numpy as np
import pytest

from oracle import poisson as op
from paper_1211_5244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda(gpu_lib):
    import torch
    return torch


@pytest.mark.parametrize("bc", ["fff", "ppf"])
def test_energy_gradient_finite_differences_fp64(torch_cuda, bc):
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    from paper_1211_5244_gb300.autograd import hartree
    n, h = (48, 48, 48), 0.3
    plan = psolver.Plan(n, bc, h, "f64")
    rho_np = synth.gaussian_mixture(n, h, 8, seed=501, noise=1e-3, subtract_mean="p" in bc)
    rho = torch.from_numpy(rho_np).cuda().requires_grad_(True)
    V, E = hartree(rho, plan)
    E.backward()
    grad = rho.grad.detach()
    u = torch.from_numpy(synth.random_density(n, seed=7)).cuda()
    eps = 1e-3
    with torch.no_grad():
        Ep = plan.solve(rho.detach() + eps * u)[1].item()
        Em = plan.solve(rho.detach() - eps * u)[1].item()
    fd = (Ep - Em) / (2 * eps)
    an = float((grad * u).sum())
    assert abs(fd - an) <= 1e-10 * max(abs(an), 1.0), (fd, an)
    # the oracle's gradient: h^3 V
    Vo, _ = op.solve(rho_np, bc, h)
    g_o = h ** 3 * Vo
    assert np.abs(grad.cpu().numpy() - g_o).max() <= 1e-12 * np.abs(g_o).max()


@pytest.mark.parametrize("bc", ["fff", "pff"])
def test_vjp_through_V_is_the_symmetric_solve(torch_cuda, bc):
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    from paper_1211_5244_gb300.autograd import hartree
    n, h = (20, 18, 16), 0.3
    plan = psolver.Plan(n, bc, h, "f64")
    rho = torch.from_numpy(synth.random_density(n, 3)).cuda().requires_grad_(True)
    w_np = synth.random_density(n, 4)
    V, E = hartree(rho, plan)
    (V * torch.from_numpy(w_np).cuda()).sum().backward()
    Kw, _ = op.solve(w_np, bc, h)
    assert np.abs(rho.grad.cpu().numpy() - Kw).max() <= 1e-12 * np.abs(Kw).max()


def test_both_outputs_and_gradcheck(torch_cuda):
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    from paper_1211_5244_gb300.autograd import hartree
    n, h = (5, 4, 3), 0.4
    plan = psolver.Plan(n, "fff", h, "f64")
    rho = torch.from_numpy(synth.random_density(n, 5)).cuda().requires_grad_(True)

    def f(r):
        V, E = hartree(r, plan)
        return V, E

    assert torch.autograd.gradcheck(f, (rho,), eps=1e-6, atol=1e-9, rtol=1e-7)


def test_hartree192_fp32_forward_backward(torch_cuda):
    """The 192^3 free-BC FP32 workload (padded 384 = 2^7 * 3): forward and
    backward; dE/drho must be h^3 V and E must match 1/2 h^3 <rho, V>."""
    torch = torch_cuda
    from paper_1211_5244_gb300 import psolver
    from paper_1211_5244_gb300.autograd import hartree
    w = synth.WORKLOADS["hartree192_f32"]
    plan = psolver.Plan(w["n"], "fff", w["h"], "f32")
    rho_np = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], w["seed"], noise=w["noise"]).astype(np.float32)
    rho = torch.from_numpy(rho_np).cuda().requires_grad_(True)
    V, E = hartree(rho, plan)
    E.backward()
    h3 = w["h"] ** 3
    assert torch.allclose(rho.grad, (h3 * V).float(), rtol=1e-6, atol=0)
    e_direct = 0.5 * h3 * float((rho.detach().double() * V.double()).sum())
    assert abs(E.detach().item() - e_direct) <= 1e-5 * abs(e_direct)
    # sampled points of V against the literal Eq. 2 sum
    pts = [(0, 0, 0), (96, 96, 96), (191, 5, 17)]
    ref = op.direct_at(rho_np.astype(np.float64), w["h"], pts)
    Vh = V.detach().double().cpu().numpy()
    got = np.array([Vh[p] for p in pts])
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(Vh).max()
