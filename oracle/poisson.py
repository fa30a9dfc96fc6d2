"""FP64 CPU oracle for the FFT-convolution Poisson solve.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may. It shares no code with the CUDA library (different
language, different algorithm: full zero-padded transforms, no pruning,
no transposes, no octant storage).

What it computes (Dugan, Genovese, Goedecker, "A Customized 3D GPU Poisson
Solver for Free Boundary Conditions"):

* Eq. 1: the Poisson equation  laplacian(V) = rho, with the sign as printed
  (no -4*pi). The free-space Green's function is therefore
  G(r) = -1 / (4 pi |r|).
* Eq. 2: the discrete convolution V(r) = sum_r' K(r - r') rho(r'), with
  K = h^3 G sampled on the grid (the grid-point weight h^3 is part of K).
* Eq. 3: the same convolution as a product V^F = K^F rho^F in Fourier space.
* §2: free axes are zero padded to twice their length (Hockney-Eastwood), so
  the circular convolution of the padded arrays equals the aperiodic one on
  the physical points; periodic axes are transformed at their own length.
  The result is the plain definition: aperiodic along free axes, circular
  along periodic axes. Any padded length L >= 2n - 1 gives the same physical
  result; L = 2n is the paper's choice and the default here.
* Mixed boundary conditions (§2 cites Cerioni et al. for their Green's
  functions without giving them). The oracle uses the textbook kernels of
  the operator restricted to the free axes, written in the wavenumber k of
  the periodic axes:
    - 0 periodic axes (free):   K(d) = -h^2 / (4 pi |d|),  d != 0
                                K(0) = -h^2 C3 / (4 pi)  (cell average of G)
    - 1 periodic axis (wire):   K = h^2 G_k(r),  r = h |d_perp|
          G_0(r) = ln(r) / (2 pi),   G_k(r) = -K0(k r) / (2 pi)
          r = 0: cell average over the h x h square (see ``_wire_cell``)
    - 2 periodic axes (surface): K = h G_k(z),  z = h |d|
          G_0(z) = |z| / 2,   G_k(z) = -exp(-k |z|) / (2 k)
    - 3 periodic axes:          K^F(k) = -1 / |k|^2,  K^F(0) = 0
  with wavenumbers k_j = 2 pi m / (n_j h), m in (-n_j/2, n_j/2].
* The Hartree energy E = 1/2 h^3 sum_r rho(r) V(r).

Arrays are (n3, n2, n1) numpy arrays: x, the axis of length n1, is the last
(fastest) numpy axis. Boundary conditions are given per axis x, y, z as a
string such as "pff" (p = periodic, f = free) or a sequence of those letters.
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np
from scipy import integrate, special

__all__ = [
    "C2", "C3", "padded_lengths", "green_mixed", "kernel_fourier",
    "kernel_fourier_octant", "solve", "brute_force", "direct_at", "hartree_energy",
]

# Cell average of 1/|u| over the unit cube centred at the origin:
#   C3 = int_{[-1/2,1/2]^3} d^3u / |u| = 3 ln(2 + sqrt 3) - pi / 2
C3 = 3.0 * math.log(2.0 + math.sqrt(3.0)) - math.pi / 2.0
# Cell average of ln|u| over the unit square centred at the origin:
#   C2 = int_{[-1/2,1/2]^2} ln|u| d^2u = -3/2 + pi/4 - ln(2)/2
C2 = -1.5 + math.pi / 4.0 - 0.5 * math.log(2.0)


def _bc_tuple(bc):
    out = tuple(str(b).lower() for b in bc)
    if len(out) != 3 or any(b not in ("p", "f") for b in out):
        raise ValueError(f"bc must name 3 axes with 'p' or 'f', got {bc!r}")
    return out


def padded_lengths(n, bc, L=None):
    """FFT length per axis (§3: S_j = N_j B_j): 2 n_j on free axes, n_j on periodic
    ones. ``L`` overrides the free-axis lengths (any L_j >= 2 n_j - 1)."""
    bc = _bc_tuple(bc)
    out = []
    for j in range(3):
        if bc[j] == "p":
            out.append(int(n[j]))
        else:
            lj = 2 * int(n[j]) if L is None else int(L[j])
            if lj < 2 * int(n[j]) - 1:
                raise ValueError("free-axis padded length must be >= 2n-1")
            out.append(lj)
    return tuple(out)


@functools.lru_cache(maxsize=None)
def _wire_cell(k, h):
    """Cell integral  I(k) = int_{h x h cell} [K0(k|u|) + ln|u|] d^2u  for k > 0.

    The integrand is radial, so in polar coordinates over the eight triangles
    of the square, I = 8 int_0^{pi/4} F(h / (2 cos t)) dt with the exact radial
    antiderivative F(R) = int_0^R [K0(k r) + ln r] r dr
                        = 1/k^2 - R K1(k R)/k + R^2 ln(R)/2 - R^2/4.
    The remaining smooth angle integral is done by adaptive quadrature.
    """
    def F(t):
        R = 0.5 * h / math.cos(t)
        return (1.0 / (k * k) - R * special.k1(k * R) / k
                + 0.5 * R * R * math.log(R) - 0.25 * R * R)
    val, _ = integrate.quad(F, 0.0, math.pi / 4.0, epsabs=1e-15, epsrel=1e-13, limit=200)
    return 8.0 * val


def green_mixed(nper, kp, dfree, h):
    """Kernel in the mixed representation: spectral along periodic axes,
    real-space along free axes.

    nper:  number of periodic axes (0..3)
    kp:    |k| over the periodic axes (array, 1/length units)
    dfree: |d| over the free axes in grid units (array, any shape
           broadcastable with kp); ignored when nper == 3
    """
    kp = np.asarray(kp, dtype=np.float64)
    dfree = np.asarray(dfree, dtype=np.float64)
    kp, dfree = np.broadcast_arrays(kp, dfree)
    out = np.zeros(kp.shape, dtype=np.float64)
    if nper == 0:
        with np.errstate(divide="ignore"):
            out = -h * h / (4.0 * math.pi * dfree)
        out[dfree == 0] = -h * h * C3 / (4.0 * math.pi)
    elif nper == 1:
        r = h * dfree
        rpos = dfree > 0
        kzero = kp == 0
        m = kzero & rpos
        out[m] = h * h * np.log(r[m]) / (2.0 * math.pi)
        m = ~kzero & rpos
        out[m] = -h * h * special.k0(kp[m] * r[m]) / (2.0 * math.pi)
        m = ~rpos
        if np.any(m):
            base = (math.log(h) + C2) / (2.0 * math.pi)
            kk = kp[m]
            vals = np.empty(kk.shape)
            for i, k in enumerate(kk):
                v = base
                if k > 0:
                    v -= _wire_cell(float(k), h) / (2.0 * math.pi * h * h)
                vals[i] = h * h * v
            out[m] = vals
    elif nper == 2:
        z = h * dfree
        pos = kp > 0
        out[~pos] = h * 0.5 * z[~pos]
        kk = kp[pos]
        out[pos] = -h * np.exp(-kk * z[pos]) / (2.0 * kk)
    elif nper == 3:
        pos = kp > 0
        out[pos] = -1.0 / (kp[pos] ** 2)
    else:
        raise ValueError("nper must be 0..3")
    return out


def _axis_values(nj, Lj, periodic, h):
    """Periodic axis: signed wavenumbers 2 pi m / (n h), m in (-n/2, n/2].
    Free axis: wrapped offsets d in (-L/2, L/2] of the padded length L."""
    i = np.arange(Lj)
    if periodic:
        m = np.where(i <= nj // 2, i, i - nj)
        return 2.0 * math.pi * m / (nj * h)
    return np.where(i <= Lj // 2, i, i - Lj).astype(np.float64)


def kernel_fourier(n, bc, h, L=None):
    """Full K^F on the padded grid, shape (L3, L2, L1), complex.

    The mixed-representation kernel is sampled on the whole padded grid and
    transformed with a full FFT along every free axis (Eq. 3, §2). K is even,
    so K^F is real up to rounding; the imaginary part is kept so tests can
    check that.
    """
    bc = _bc_tuple(bc)
    Ls = padded_lengths(n, bc, L)
    vals = [_axis_values(int(n[j]), Ls[j], bc[j] == "p", h) for j in range(3)]
    # numpy axis order is (z, y, x)
    grids = (vals[0][None, None, :], vals[1][None, :, None], vals[2][:, None, None])
    kp2 = np.zeros((1, 1, 1))
    df2 = np.zeros((1, 1, 1))
    for j in range(3):
        if bc[j] == "p":
            kp2 = kp2 + grids[j] ** 2
        else:
            df2 = df2 + grids[j] ** 2
    nper = sum(1 for b in bc if b == "p")
    M = green_mixed(nper, np.sqrt(kp2), np.sqrt(df2), h)
    free_axes = [2 - j for j in range(3) if bc[j] == "f"]
    if free_axes:
        return np.fft.fftn(M, axes=free_axes)
    return M.astype(np.complex128)


def kernel_fourier_octant(n, bc, h, L=None):
    """Real part of K^F on the non-negative octant, shape
    (L3//2+1, L2//2+1, L1//2+1). K^F is even along every axis, so this
    octant determines it."""
    KF = kernel_fourier(n, bc, h, L)
    Ls = padded_lengths(n, bc, L)
    return np.ascontiguousarray(KF[: Ls[2] // 2 + 1, : Ls[1] // 2 + 1, : Ls[0] // 2 + 1].real)


def solve(rho, bc, h, L=None, KF=None):
    """V and E for density ``rho`` (n3, n2, n1).

    rho is placed at the low corner [0, n) of the padded grid, transformed with
    a full 3D FFT, multiplied by K^F, transformed back with the 1/(L1 L2 L3)
    normalisation, and V is read from the same corner (Eq. 3 with the zero
    padding of §2).
    """
    rho = np.asarray(rho, dtype=np.float64)
    n3, n2, n1 = rho.shape
    n = (n1, n2, n3)
    Ls = padded_lengths(n, bc, L)
    if KF is None:
        KF = kernel_fourier(n, bc, h, L)
    padded = np.zeros((Ls[2], Ls[1], Ls[0]), dtype=np.float64)
    padded[:n3, :n2, :n1] = rho
    VF = KF * np.fft.fftn(padded)
    V = np.fft.ifftn(VF)[:n3, :n2, :n1].real.copy()
    return V, hartree_energy(rho, V, h)


def hartree_energy(rho, V, h):
    """E = 1/2 h^3 sum_r rho(r) V(r)."""
    return 0.5 * h ** 3 * float(np.sum(np.asarray(rho, np.float64) * np.asarray(V, np.float64)))


def brute_force(rho, bc, h):
    """Direct O(N^2) evaluation of Eq. 2 along the free axes.

    Periodic axes are first transformed exactly (a DFT at their own length);
    then for every source point of the free-axis sub-grid the mixed kernel at
    the offset (target - source) is accumulated, and the periodic axes are
    transformed back. With no periodic axis this is the literal real-space
    double sum; with no free axis it is the plain Fourier multiply.
    """
    bc = _bc_tuple(bc)
    rho = np.asarray(rho, dtype=np.float64)
    n3, n2, n1 = rho.shape
    n = (n1, n2, n3)
    per = [j for j in range(3) if bc[j] == "p"]
    free = [j for j in range(3) if bc[j] == "f"]
    per_np_axes = [2 - j for j in per]
    rho_hat = np.fft.fftn(rho, axes=per_np_axes) if per else rho.astype(np.complex128)

    # |k| over the periodic axes, broadcast over the full (z, y, x) grid
    shape = (n3, n2, n1)
    kp2 = np.zeros(shape)
    for j in per:
        kj = _axis_values(n[j], n[j], True, h)
        kp2 = kp2 + (kj ** 2).reshape([-1 if (2 - a) == j else 1 for a in range(3)])
    kp = np.sqrt(kp2)
    if not free:
        Vhat = np.where(kp > 0, -1.0 / np.where(kp > 0, kp, 1.0) ** 2, 0.0) * rho_hat
        return np.fft.ifftn(Vhat, axes=per_np_axes).real

    idx = [np.arange(n[j]) for j in range(3)]
    Vhat = np.zeros(shape, dtype=np.complex128)
    for src in itertools.product(*[range(n[j]) for j in free]):
        d2 = np.zeros(shape)
        for j, s in zip(free, src):
            dj = (idx[j] - s).astype(np.float64)
            d2 = d2 + (dj ** 2).reshape([-1 if (2 - a) == j else 1 for a in range(3)])
        Kval = green_mixed(len(per), kp, np.sqrt(d2), h)
        sl = [slice(None)] * 3
        for j, s in zip(free, src):
            sl[2 - j] = slice(s, s + 1)
        Vhat += Kval * rho_hat[tuple(sl)]
    if per:
        return np.fft.ifftn(Vhat, axes=per_np_axes).real
    return Vhat.real


def kernel_fourier_from_real(kernel, n, bc, L=None):
    """K^F of a convolution kernel given in real space (§5: the same zero-padded
    convolution serves kernels other than the Poisson kernel, e.g. a local
    potential applied to wave functions).

    ``kernel`` has shape (L3//2 + 1, L2//2 + 1, L1//2 + 1): kernel[d3, d2, d1] is
    the value at the offset (d1, d2, d3), and the kernel is even in every offset,
    K(..., -d_j, ...) = K(..., d_j, ...). The full kernel on the padded grid takes
    at index i_j the value at offset min(i_j, L_j - i_j); its full FFT is K^F
    (real, since the kernel is even). Along a periodic axis (L_j = n_j) this is a
    kernel of period n_j; along a free axis the offsets |d_j| <= n_j - 1 couple
    physical points and the others are never used.
    """
    bc = _bc_tuple(bc)
    Ls = padded_lengths(n, bc, L)
    kernel = np.asarray(kernel, dtype=np.float64)
    want = (Ls[2] // 2 + 1, Ls[1] // 2 + 1, Ls[0] // 2 + 1)
    if kernel.shape != want:
        raise ValueError(f"kernel octant must have shape {want}, got {kernel.shape}")
    idx = [np.minimum(np.arange(Lj), Lj - np.arange(Lj)) for Lj in Ls]
    full = kernel[np.ix_(idx[2], idx[1], idx[0])]
    return np.fft.fftn(full)


def convolve(rho, bc, h, kernel, L=None):
    """V = K * rho (Eq. 2 with a caller's kernel, no h^3 factor added) and
    E = 1/2 h^3 sum rho V, by the zero-padded FFT of ``solve``."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[::-1]
    KF = kernel_fourier_from_real(kernel, n, bc, L)
    return solve(rho, bc, h, L=L, KF=KF)


def convolve_direct(rho, bc, kernel):
    """The literal sum V(r) = sum_r' K(r - r') rho(r') for tiny grids, with the
    kernel's octant values: along a free axis the offset is r_j - r'_j, along a
    periodic axis it is taken modulo n_j; either way the value used is the one at
    |offset| folded into [0, L_j // 2] (L_j = 2 n_j free, n_j periodic)."""
    bc = _bc_tuple(bc)
    rho = np.asarray(rho, dtype=np.float64)
    n3, n2, n1 = rho.shape
    n = (n1, n2, n3)
    Ls = padded_lengths(n, bc)
    kernel = np.asarray(kernel, dtype=np.float64)
    V = np.zeros_like(rho)
    tgt = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    for s3, s2, s1 in itertools.product(range(n3), range(n2), range(n1)):
        off = []
        for j, (t, sj) in enumerate(zip(tgt[::-1], (s1, s2, s3))):
            d = t - sj
            if bc[j] == "p":
                d = np.mod(d, n[j])
                d = np.minimum(d, n[j] - d)
            else:
                d = np.abs(d)
            off.append(d)
        V += rho[s3, s2, s1] * kernel[off[2], off[1], off[0]]
    return V


def direct_at(rho, h, points):
    """Eq. 2 evaluated literally at selected grid points, free BCs on all axes:
    V(t) = sum_r' K(t - r') rho(r') for each t = (k, j, i) in ``points``
    (numpy index order z, y, x). O(N) per point, summed slab by slab."""
    rho = np.asarray(rho, dtype=np.float64)
    n3, n2, n1 = rho.shape
    y = np.arange(n2, dtype=np.float64)[:, None]
    x = np.arange(n1, dtype=np.float64)[None, :]
    out = []
    for tz, ty, tx in points:
        dyx2 = (ty - y) ** 2 + (tx - x) ** 2
        acc = 0.0
        for k in range(n3):
            K = green_mixed(0, 0.0, np.sqrt((tz - k) ** 2 + dyx2), h)
            acc += float(np.sum(K * rho[k]))
        out.append(acc)
    return np.array(out)
