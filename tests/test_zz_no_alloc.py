"""The allocation-free energy entry point, through the C ABI.

ps_hartree_energy_noalloc serves callers that must not allocate device memory
(their memory belongs to their own arena or allocator, or an allocation or the
synchronisation of a free cannot be risked mid-run). Its scratch is a static
array inside the library, so these checks compare it with the energy that
ps_solve computes, on two calls in a row with different grids: the second call
must not see anything the first left in the shared scratch. This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1211_5244_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
MAX_POINTS = 65536 * 8192


def _solve(torch, n, bc, dtype, seed):
    from paper_1211_5244_gb300 import psolver
    rho = synth.gaussian_mixture(n, 0.3, 4, seed=seed, noise=1e-3, subtract_mean="p" in bc)
    rho_t = torch.from_numpy(rho.astype(np.float32 if dtype == "f32" else np.float64)).cuda()
    plan = psolver.Plan(n, bc, 0.3, dtype)
    V, E = plan.solve(rho_t)
    return rho_t, V, float(E.item())


def _noalloc(lib, torch, rho, V, h, E=None):
    if E is None:
        E = torch.full((), float("nan"), dtype=torch.float64, device=rho.device)
    dtype = 0 if rho.dtype == torch.float32 else 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ps_hartree_energy_noalloc(dtype, rho.numel(), h, ctypes.c_void_p(rho.data_ptr()),
                                       ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(E.data_ptr()), stream)
    assert rc == 0, lib.ps_last_error().decode()
    return float(E.item())


@pytest.mark.parametrize("dtype,first,second", [
    ("f64", ((40, 36, 28), "fff"), ((24, 30, 33), "pff")),
    ("f32", ((256, 256, 256), "fff"), ((64, 48, 40), "ppf")),
])
def test_noalloc_energy_matches_solve_on_two_calls(gpu_lib, dtype, first, second):
    import torch
    for k, (n, bc) in enumerate((first, second)):
        rho, V, E_solve = _solve(torch, n, bc, dtype, seed=11 + k)
        E = _noalloc(gpu_lib, torch, rho, V, 0.3)
        assert abs(E - E_solve) <= TOL[dtype] * abs(E_solve), (n, bc, E, E_solve)


def test_noalloc_rejects_grids_beyond_its_scratch(gpu_lib):
    import torch
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    E = torch.zeros((), dtype=torch.float64, device="cuda")
    rc = gpu_lib.ps_hartree_energy_noalloc(0, MAX_POINTS + 1, 0.3, ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                           None)
    assert rc == 2 and b"exceeds" in gpu_lib.ps_last_error()
    assert gpu_lib.ps_hartree_energy_noalloc(0, 0, 0.3, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                             None) == 1


def test_noalloc_call_leaves_device_memory_unchanged(gpu_lib):
    """The defining property: once the first call on the device has looked up
    the scratch address (and the kernel's module is loaded), a call takes no
    device memory. Free memory is read before and after a second call on the
    same, already allocated tensors."""
    import torch
    rho, V, E_solve = _solve(torch, (64, 48, 40), "fff", "f32", seed=5)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    _noalloc(gpu_lib, torch, rho, V, 0.3, E)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    e2 = _noalloc(gpu_lib, torch, rho, V, 0.3, E)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert abs(e2 - E_solve) <= TOL["f32"] * abs(E_solve)
