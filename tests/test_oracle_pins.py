"""Pins for the FP64 oracle: each test ties it to something other than itself.

* brute force: the literal O(N^2) sum of Eq. 2 (and an exact DFT along the
  periodic axes for mixed BCs) on tiny uneven grids;
* closed forms: periodic plane waves; Gaussian charge (free); Gaussian sheet
  and Fourier mode over a sheet (surface); Gaussian line charge and a Fourier
  mode along a Gaussian wire (wire) -- these are discretisation-accuracy
  checks, so they assert second-order convergence and a small error;
* the cell-average constants against independent quadratures;
* invariants: linearity, symmetry, reflection, periodic shifts, real K^F,
  independence of the padded length, and the exact quadratic energy.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import poisson as op

ALL_BCS = ["fff", "pff", "fpf", "ffp", "ppf", "pfp", "fpp", "ppp"]


def _grid(n, h):
    n1, n2, n3 = n
    z, y, x = np.meshgrid(np.arange(n3) * h, np.arange(n2) * h, np.arange(n1) * h,
                          indexing="ij")
    return x, y, z


# ---------------------------------------------------------------- constants

def test_c3_by_face_pyramids():
    # The unit cube is six pyramids with apex at the origin; integrating 1/|u|
    # radially leaves C3 = 3/2 * int_{[-1/2,1/2]^2} da db / sqrt(1/4 + a^2 + b^2).
    val, _ = integrate.dblquad(lambda b, a: 1.0 / math.sqrt(0.25 + a * a + b * b),
                               -0.5, 0.5, -0.5, 0.5, epsabs=1e-14, epsrel=1e-13)
    assert abs(1.5 * val - op.C3) < 1e-12
    assert abs(op.C3 - 2.380077363979553) < 1e-14


def test_c2_by_edge_triangles():
    # The unit square is four triangles with apex at the origin:
    # C2 = -1/2 + 1/2 int_{-1/2}^{1/2} ln(1/4 + a^2) da.
    val, _ = integrate.quad(lambda a: math.log(0.25 + a * a), -0.5, 0.5,
                            epsabs=1e-15, epsrel=1e-14)
    assert abs(-0.5 + 0.5 * val - op.C2) < 1e-13


@pytest.mark.parametrize("k,h", [(0.05, 0.3), (1.0, 0.3), (3.0, 0.25), (10.0, 0.3)])
def test_wire_cell_integral_by_2d_quadrature(k, h):
    # I(k) = int over the h x h cell of K0(k|u|) + ln|u|, by plain 2D quadrature
    # over one quadrant (the integrand is bounded at the origin).
    f = lambda y, x: special.k0(k * math.hypot(x, y)) + math.log(math.hypot(x, y))
    val, _ = integrate.dblquad(f, 0.0, h / 2, 0.0, h / 2, epsabs=1e-14, epsrel=1e-11)
    ref = 4.0 * val
    got = op._wire_cell(k, h)
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 2), (5, 4, 6), (7, 5, 3), (2, 7, 5)])
def test_free_matches_direct_sum(shape):
    rng = np.random.default_rng(11)
    rho = rng.standard_normal(shape[::-1])
    V, E = op.solve(rho, "fff", 0.37)
    Vb = op.brute_force(rho, "fff", 0.37)
    assert np.abs(V - Vb).max() <= 1e-13 * np.abs(Vb).max()


def test_direct_sum_is_literal_eq2():
    # brute_force must be the literal double sum: check one output point by hand.
    rng = np.random.default_rng(5)
    h = 0.3
    rho = rng.standard_normal((3, 4, 5))
    Vb = op.brute_force(rho, "fff", h)
    t = (2, 1, 3)  # (z, y, x)
    acc = 0.0
    for k in range(3):
        for j in range(4):
            for i in range(5):
                d = math.sqrt((t[0] - k) ** 2 + (t[1] - j) ** 2 + (t[2] - i) ** 2)
                K = -h * h * op.C3 / (4 * math.pi) if d == 0 else -h ** 3 / (4 * math.pi * h * d)
                acc += K * rho[k, j, i]
    assert abs(acc - Vb[t]) < 1e-13 * abs(acc)


@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("shape", [(4, 3, 5), (6, 5, 2)])
def test_mixed_matches_direct_sum(bc, shape):
    rng = np.random.default_rng(ALL_BCS.index(bc) * 100 + sum(shape))
    rho = rng.standard_normal(shape[::-1])
    V, _ = op.solve(rho, bc, 0.41)
    Vb = op.brute_force(rho, bc, 0.41)
    assert np.abs(V - Vb).max() <= 1e-13 * np.abs(Vb).max()


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,m", [((8, 6, 10), (1, 2, 3)), ((9, 7, 5), (4, -3, 2)),
                                 ((6, 6, 6), (3, 0, 0)), ((5, 8, 4), (0, 5, 1))])
def test_periodic_plane_wave(n, m):
    h = 0.4
    x, y, z = _grid(n, h)
    k = [2 * math.pi * m[j] / (n[j] * h) for j in range(3)]
    rho = np.cos(k[0] * x + k[1] * y + k[2] * z)
    V, _ = op.solve(rho, "ppp", h)
    # on the grid, index m is the same wave as its alias in (-n/2, n/2]
    ma = [((m[j] + n[j] // 2) % n[j]) - n[j] // 2 if n[j] % 2 else
          ((m[j] - 1 + n[j] // 2) % n[j]) - n[j] // 2 + 1 for j in range(3)]
    k2 = sum((2 * math.pi * ma[j] / (n[j] * h)) ** 2 for j in range(3))
    assert np.abs(V + rho / k2).max() < 1e-13


def test_periodic_drops_the_mean():
    rho = np.full((4, 5, 6), 2.5)
    V, E = op.solve(rho, "ppp", 0.3)
    assert np.abs(V).max() < 1e-14 and abs(E) < 1e-14


def _gauss_free_err(n):
    Lbox, sig = 9.6, 1.0
    h = Lbox / n
    x, y, z = _grid((n, n, n), h)
    c = 0.5 * Lbox + 0.13 * h
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    rho = np.exp(-r ** 2 / (2 * sig ** 2))
    Q = (2 * math.pi * sig ** 2) ** 1.5
    Va = -Q / (4 * math.pi * r) * special.erf(r / (math.sqrt(2) * sig))
    V, _ = op.solve(rho, "fff", h)
    return np.abs(V - Va).max() / np.abs(Va).max()


def test_free_gaussian_charge_second_order():
    # V = -Q erf(r / (sqrt2 sigma)) / (4 pi r): O(h^2) discretisation error
    e16, e32, e64 = (_gauss_free_err(n) for n in (16, 32, 64))
    assert e64 < 1e-3
    assert 3.3 < e16 / e32 < 4.7 and 3.3 < e32 / e64 < 4.7


def _surface_err(n, m):
    s, Lx = (0.6 if m == 0 else 0.8), 6.0
    h = Lx / n
    x, y, z = _grid((n, 4, n), h)
    z0 = 0.5 * n * h + 0.17 * h
    zz = z - z0
    g = np.exp(-zz ** 2 / (2 * s * s))
    if m == 0:
        f = 0.5 * (zz * s * math.sqrt(2 * math.pi) * special.erf(zz / (math.sqrt(2) * s))
                   + 2 * s * s * g)
        k = 0.0
    else:
        k = 2 * math.pi * m / (n * h)
        f = -(1 / (2 * k)) * s * math.sqrt(math.pi / 2) * np.exp(k * k * s * s / 2) * (
            np.exp(-k * zz) * special.erfc((k * s * s - zz) / (math.sqrt(2) * s))
            + np.exp(k * zz) * special.erfc((k * s * s + zz) / (math.sqrt(2) * s)))
    rho = np.cos(k * x) * g
    Va = np.cos(k * x) * f
    V, _ = op.solve(rho, "ppf", h)
    return np.abs(V - Va).max() / np.abs(Va).max()


@pytest.mark.parametrize("m", [0, 1, 2])
def test_surface_closed_form_second_order(m):
    e = [_surface_err(n, m) for n in (16, 32, 64)]
    assert e[2] < 5e-3
    assert 3.3 < e[0] / e[1] < 4.7 and 3.3 < e[1] / e[2] < 4.7


def _wire_line_err(n):
    sig, Lb = 0.7, 7.0
    h = Lb / n
    x, y, z = _grid((4, n, n), h)
    c = 0.5 * Lb + 0.11 * h
    r2 = (y - c) ** 2 + (z - c) ** 2
    rho = np.exp(-r2 / (2 * sig ** 2))
    lam = 2 * math.pi * sig ** 2
    Va = (lam / (4 * math.pi)) * (np.log(r2) + special.exp1(r2 / (2 * sig ** 2)))
    V, _ = op.solve(rho, "pff", h)
    return np.abs(V - Va).max() / np.abs(Va).max()


def test_wire_line_charge_second_order():
    # V = lambda / (4 pi) [ln r^2 + E1(r^2 / 2 sigma^2)]: fixes the ln convention
    e = [_wire_line_err(n) for n in (16, 32, 64)]
    assert e[2] < 1e-3
    assert 3.3 < e[0] / e[1] < 4.7 and 3.3 < e[1] / e[2] < 4.7


def _radial_mode(r, k, sig):
    # u(r) = -int_0^inf I0(k r_<) K0(k r_>) g(t) t dt  solves (lap_2D - k^2) u = g
    g = lambda t: math.exp(-t * t / (2 * sig * sig))
    f1 = lambda t: special.ive(0, k * t) * special.kve(0, k * r) * math.exp(k * t - k * r) * g(t) * t
    f2 = lambda t: special.ive(0, k * r) * special.kve(0, k * t) * math.exp(k * r - k * t) * g(t) * t
    a = integrate.quad(f1, 0, r, epsabs=1e-14, epsrel=1e-12)[0] if r > 0 else 0.0
    b = integrate.quad(f2, r, np.inf, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
    return -(a + b)


def _wire_mode_err(n):
    sig, Lb = 0.7, 7.0
    h = Lb / n
    n1 = n // 4
    x, y, z = _grid((n1, n, n), h)
    c = 0.5 * Lb + 0.11 * h
    k = 2 * math.pi / (n1 * h)
    r = np.sqrt((y - c) ** 2 + (z - c) ** 2)
    rho = np.cos(k * x) * np.exp(-r ** 2 / (2 * sig ** 2))
    V, _ = op.solve(rho, "pff", h)
    pts = [(n // 2, n // 2), (n // 2 + 1, n // 2), (n // 2 + 3, n // 2 + 2), (n // 4, n // 2)]
    got = np.array([V[kz, jy, 0] for jy, kz in pts])
    ref = np.array([_radial_mode(r[kz, jy, 0], k, sig) for jy, kz in pts])
    return np.abs(got - ref).max() / np.abs(ref).max()


def test_wire_fourier_mode_converges():
    # cos(k x) g(r_perp) -> cos(k x) u(r_perp); pins K0, its 1/(2 pi) and the
    # cell average at r_perp = 0 (dropping the latter gives ~4% at n = 64)
    e32, e64 = _wire_mode_err(32), _wire_mode_err(64)
    assert e64 < 1.2e-2
    assert e32 / e64 > 2.8


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("bc", ALL_BCS)
def test_linearity_and_symmetry(bc):
    rng = np.random.default_rng(3)
    shape = (6, 5, 7)
    r1, r2 = rng.standard_normal(shape), rng.standard_normal(shape)
    V1, _ = op.solve(r1, bc, 0.3)
    V2, _ = op.solve(r2, bc, 0.3)
    V12, _ = op.solve(2.0 * r1 - 3.0 * r2, bc, 0.3)
    assert np.abs(V12 - (2 * V1 - 3 * V2)).max() < 1e-12 * np.abs(V12).max()
    a, b = np.sum(r1 * V2), np.sum(r2 * V1)
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("bc", ["fff", "pff", "ppf", "fpp"])
def test_reflection(bc):
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((5, 6, 7))
    V, _ = op.solve(rho, bc, 0.3)
    for j in range(3):
        ax = 2 - j
        if bc[j] == "f":
            fl = lambda a: np.flip(a, axis=ax)
        else:
            fl = lambda a: np.roll(np.flip(a, axis=ax), 1, axis=ax)  # i -> -i mod n
        Vr, _ = op.solve(fl(rho), bc, 0.3)
        assert np.abs(Vr - fl(V)).max() < 1e-12 * np.abs(V).max()


@pytest.mark.parametrize("bc", ["pff", "ppf", "ppp", "fpf"])
def test_periodic_shift_equivariance(bc):
    rng = np.random.default_rng(6)
    rho = rng.standard_normal((5, 6, 7))
    V, _ = op.solve(rho, bc, 0.3)
    for j in range(3):
        if bc[j] == "p":
            ax = 2 - j
            Vs, _ = op.solve(np.roll(rho, 2, axis=ax), bc, 0.3)
            assert np.abs(Vs - np.roll(V, 2, axis=ax)).max() < 1e-12 * np.abs(V).max()


@pytest.mark.parametrize("bc", ALL_BCS)
def test_kernel_is_real_and_even(bc):
    KF = op.kernel_fourier((6, 5, 7), bc, 0.3)
    assert np.abs(KF.imag).max() <= 1e-14 * np.abs(KF.real).max()
    # even along each axis: K(k) = K(L - k)
    for ax in range(3):
        idx = (-np.arange(KF.shape[ax])) % KF.shape[ax]
        assert np.allclose(np.take(KF.real, idx, axis=ax), KF.real, rtol=0, atol=1e-14 * np.abs(KF).max())


@pytest.mark.parametrize("bc", ["fff", "pff", "ppf", "fpf"])
def test_padded_length_does_not_matter(bc):
    # any free-axis length L >= 2n - 1 gives the same physical result (§2)
    rng = np.random.default_rng(7)
    n = (5, 4, 6)
    rho = rng.standard_normal(n[::-1])
    V0, _ = op.solve(rho, bc, 0.3)
    for extra in (-1, 1, 3):
        L = tuple(2 * n[j] + extra for j in range(3))
        V1, _ = op.solve(rho, bc, 0.3, L=L)
        assert np.abs(V1 - V0).max() < 1e-13 * np.abs(V0).max()


@pytest.mark.parametrize("bc", ["fff", "ppf", "pff"])
def test_energy_is_exactly_quadratic(bc):
    # E(rho) = 1/2 h^3 <rho, K rho> with K symmetric: central differences are exact
    rng = np.random.default_rng(8)
    h = 0.3
    rho, u = rng.standard_normal((6, 5, 4)), rng.standard_normal((6, 5, 4))
    V, E = op.solve(rho, bc, h)
    eps = 0.37
    Ep = op.solve(rho + eps * u, bc, h)[1]
    Em = op.solve(rho - eps * u, bc, h)[1]
    fd = (Ep - Em) / (2 * eps)
    assert abs(fd - h ** 3 * np.sum(V * u)) < 1e-12 * max(1.0, abs(fd))


def test_direct_at_matches_brute_force():
    rng = np.random.default_rng(12)
    rho = rng.standard_normal((6, 5, 7))
    Vb = op.brute_force(rho, "fff", 0.3)
    pts = [(0, 0, 0), (5, 4, 6), (2, 3, 1)]
    got = op.direct_at(rho, 0.3, pts)
    assert np.abs(got - np.array([Vb[p] for p in pts])).max() < 1e-13 * np.abs(Vb).max()


# ---- convolution with a caller's kernel (§5: the same zero-padded convolution
# for other kernels, e.g. a local potential applied to wave functions)

def _kernel_octant(rng, n, bc):
    L = op.padded_lengths(n, bc)
    return rng.standard_normal((L[2] // 2 + 1, L[1] // 2 + 1, L[0] // 2 + 1))


@pytest.mark.parametrize("bc", ALL_BCS)
@pytest.mark.parametrize("n", [(5, 4, 3), (3, 6, 7), (1, 5, 4)])
def test_convolve_matches_literal_sum(bc, n):
    """FFT convolution with a random even kernel == the literal double sum
    (odd periodic lengths included: n = 5, 3, 7)."""
    rng = np.random.default_rng(sum(n) + ALL_BCS.index(bc))
    k = _kernel_octant(rng, n, bc)
    rho = rng.standard_normal(n[::-1])
    V, E = op.convolve(rho, bc, 0.3, k)
    Vd = op.convolve_direct(rho, bc, k)
    assert np.abs(V - Vd).max() <= 1e-13 * np.abs(Vd).max()
    assert abs(E - 0.5 * 0.3 ** 3 * np.sum(rho * Vd)) <= 1e-13 * abs(E)


@pytest.mark.parametrize("bc", ["fff", "pfp", "ppp"])
def test_convolve_delta_kernel_is_identity(bc):
    n = (6, 5, 4)
    L = op.padded_lengths(n, bc)
    k = np.zeros((L[2] // 2 + 1, L[1] // 2 + 1, L[0] // 2 + 1))
    k[0, 0, 0] = 1.0
    rho = np.random.default_rng(3).standard_normal(n[::-1])
    V, _ = op.convolve(rho, bc, 0.5, k)
    assert np.abs(V - rho).max() < 1e-14 * np.abs(rho).max()


def test_convolve_with_sampled_free_kernel_is_the_free_solve():
    """The free-space Poisson kernel sampled on the octant (Eq. 2 with K = h^3 G
    and the cell-averaged K(0)) reproduces the free-BC solve."""
    n = (6, 5, 7)
    h = 0.4
    L = op.padded_lengths(n, "fff")
    d = [np.arange(Lj // 2 + 1) for Lj in L]
    dist = np.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
    k = op.green_mixed(0, 0.0, dist, h)
    rho = np.random.default_rng(4).standard_normal(n[::-1])
    V, E = op.convolve(rho, "fff", h, k)
    Vs, Es = op.solve(rho, "fff", h)
    assert np.abs(V - Vs).max() < 1e-13 * np.abs(Vs).max()
    assert abs(E - Es) < 1e-13 * abs(Es)


def test_convolve_rejects_wrong_octant_shape():
    with pytest.raises(ValueError):
        op.convolve(np.zeros((3, 4, 5)), "fff", 0.3, np.zeros((4, 5, 5)))
