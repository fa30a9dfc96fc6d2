"""Seeded synthetic densities shaped like the paper's workloads.

This module only draws inputs. It holds none of the solver's arithmetic, so the
CUDA path and the FP64 oracle can both take their inputs from it without
sharing any of the method.

The paper (Dugan, Genovese, Goedecker, §4) benchmarks smooth molecular-style
densities on grids from a few tens to a few hundred points per axis but prints
neither the densities nor a dataset. The stand-in is a sum of Gaussians:

    rho(r) = sum_g A_g exp(-|r - c_g|^2 / (2 sigma_g^2))

with grid point (i, j, k) at r = h (i, j, k), centres drawn per axis in the
middle half of the box, sigma_g = h U[1.5, 4), A_g ~ N(0, 1), evaluated
without periodic images. Optional uniform noise and mean removal follow the
workload recipes below. All values are drawn in FP64 with numpy's PCG64.
Arrays are (n3, n2, n1) C-contiguous, i.e. x (axis of length n1) fastest.
"""
from __future__ import annotations

import numpy as np

__all__ = ["gaussian_mixture", "random_density", "WORKLOADS"]


def gaussian_mixture(n, h, n_gauss, seed, noise=0.0, subtract_mean=False,
                     sigma_range=(1.5, 4.0)):
    """Sum of ``n_gauss`` seeded Gaussians on an (n3, n2, n1) grid.

    n: (n1, n2, n3) physical grid; h: grid spacing; noise: amplitude of
    added U[-1, 1) noise; subtract_mean: remove the global mean (neutral
    density, needed when an axis is periodic).
    """
    n1, n2, n3 = (int(v) for v in n)
    rng = np.random.default_rng(seed)
    dims = np.array([n1, n2, n3], dtype=np.float64)
    centres = h * (dims / 4.0 + rng.uniform(0.0, 1.0, size=(n_gauss, 3)) * dims / 2.0)
    sigmas = h * rng.uniform(sigma_range[0], sigma_range[1], size=n_gauss)
    amps = rng.standard_normal(n_gauss)
    x = h * np.arange(n1, dtype=np.float64)
    y = h * np.arange(n2, dtype=np.float64)
    z = h * np.arange(n3, dtype=np.float64)
    rho = np.zeros((n3, n2, n1), dtype=np.float64)
    for c, s, a in zip(centres, sigmas, amps):
        gx = np.exp(-((x - c[0]) ** 2) / (2.0 * s * s))
        gy = np.exp(-((y - c[1]) ** 2) / (2.0 * s * s))
        gz = np.exp(-((z - c[2]) ** 2) / (2.0 * s * s))
        rho += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    if noise:
        rho += noise * rng.uniform(-1.0, 1.0, size=rho.shape)
    if subtract_mean:
        rho -= rho.mean()
    return rho


def random_density(n, seed, subtract_mean=False):
    """Unstructured N(0,1) density: exercises every Fourier mode."""
    n1, n2, n3 = (int(v) for v in n)
    rng = np.random.default_rng(seed)
    rho = rng.standard_normal((n3, n2, n1))
    if subtract_mean:
        rho -= rho.mean()
    return rho


# Workload recipes (sizes, boundary conditions, precision, seeds). BC strings
# name the x, y, z axes in order: "f" free, "p" periodic.
WORKLOADS = {
    # free BCs, 32^3, FP64, h = 0.3, 3 Gaussians
    "free32_f64": dict(n=(32, 32, 32), bc="fff", h=0.3, dtype="f64", n_gauss=3,
                       noise=0.0, seed=101),
    # 128^3, all four BC kinds, 8 Gaussians + 1e-3 noise, neutral when periodic
    "bc128": dict(n=(128, 128, 128), bcs=("ppp", "pff", "ppf", "fff"), h=0.3,
                  n_gauss=8, noise=1e-3, seed=201),
    # headline: free BCs 256^3 FP32 (padded FFT 512^3)
    "free256_f32": dict(n=(256, 256, 256), bc="fff", h=0.3, dtype="f32", n_gauss=8,
                        noise=1e-3, seed=301),
    "free512_f32": dict(n=(512, 512, 512), bc="fff", h=0.3, dtype="f32", n_gauss=8,
                        noise=1e-3, seed=302),
    # 64 uneven problems, n ~ U{24..160} per axis, BC uniform over 4 kinds
    "batched64": dict(count=64, nmin=24, nmax=160, h=0.3, dtype="f32", n_gauss=8,
                      noise=1e-3, seed=401),
    # differentiable Hartree energy, free 192^3 FP32; FD checks at 48^3
    "hartree192_f32": dict(n=(192, 192, 192), bc="fff", h=0.3, dtype="f32", n_gauss=8,
                           noise=1e-3, seed=501),
}


def batched_shapes(count, nmin, nmax, seed):
    """Shapes and BC strings of the uneven batch (one draw per problem)."""
    rng = np.random.default_rng(seed)
    kinds = ("fff", "pff", "ppf", "ppp")
    out = []
    for _ in range(count):
        n = tuple(int(v) for v in rng.integers(nmin, nmax + 1, size=3))
        bc = kinds[int(rng.integers(0, 4))]
        out.append((n, bc))
    return out
