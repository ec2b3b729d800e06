"""Pins for the oracle's one-dimensional bases (Section 2.1, items 2-3).

Each check compares against something other than the oracle itself: a library
routine (scipy's DST, scipy's associated Legendre functions), an exact property
(quadrature exactness, orthogonality) or a closed form (sine eigenfunctions of
d^2/dx^2, derivatives of known sine series).
"""
import numpy as np
import pytest
import scipy.fft
import scipy.special

from oracle import basis


@pytest.mark.parametrize("N", [6, 24, 36, 48, 64])
def test_dst2_matrix_matches_scipy(N):
    S = basis.dst2_matrix(N)
    x = np.random.default_rng(N).standard_normal(N)
    ref = scipy.fft.dst(x, type=2, norm="ortho")
    np.testing.assert_allclose(S @ x, ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(S @ S.T, np.eye(N), atol=1e-13)


@pytest.mark.parametrize("N,mass", [(32, 1377.7), (48, 1224.5)])
def test_kinetic_sine_eigenfunctions(N, mass):
    """sin(j pi (x - xa)/L) sampled on the nodes is an eigenvector with k_j^2 / 2 mass."""
    xa, xb = 0.5, 10.0
    x, dx = basis.sine_dvr_nodes(xa, xb, N)
    T = basis.radial_kinetic_matrix(xa, xb, N, mass, tcut=1e9)
    L = xb - xa
    for j in (1, 2, 7, N // 2, N - 1, N):
        f = np.sin(j * np.pi * (x - xa) / L)
        k = j * np.pi / L
        np.testing.assert_allclose(T @ f, k * k / (2 * mass) * f, atol=1e-12 * k * k / mass)


def test_kinetic_cap_is_spectral():
    """The cap clips eigenvalues: T's spectrum is min(k_j^2/2m, tcut)."""
    N, mass, tcut = 40, 1000.0, 0.05
    T = basis.radial_kinetic_matrix(0.0, 8.0, N, mass, tcut)
    ev = np.sort(np.linalg.eigvalsh(T))
    k = np.arange(1, N + 1) * np.pi / 8.0
    np.testing.assert_allclose(ev, np.sort(np.minimum(k * k / (2 * mass), tcut)), atol=1e-14)


def test_kinetic_on_gaussian_matches_second_derivative():
    """-(1/2m) f'' for a Gaussian well inside the walls (spectral accuracy)."""
    N, mass = 96, 1.0
    xa, xb = 0.0, 20.0
    x, dx = basis.sine_dvr_nodes(xa, xb, N)
    f = np.exp(-(x - 10.0) ** 2)
    d2 = (4 * (x - 10.0) ** 2 - 2) * f
    T = basis.radial_kinetic_matrix(xa, xb, N, mass, tcut=1e9)
    np.testing.assert_allclose(T @ f, -d2 / (2 * mass), atol=1e-9)


def test_sine_interpolation_exact_for_sine_series():
    N = 36
    xa, xb = 0.5, 12.0
    L = xb - xa
    x, dx = basis.sine_dvr_nodes(xa, xb, N)
    c = np.random.default_rng(3).standard_normal(N)
    j = np.arange(1, N + 1)

    def f(y):
        return np.sum(c * np.sin(j * np.pi * (y - xa) / L))

    def df(y):
        return np.sum(c * j * np.pi / L * np.cos(j * np.pi * (y - xa) / L))

    q = np.array([f(xi) for xi in x]) * np.sqrt(dx)
    for xs in (1.0, 6.0, 6.37, 11.9):
        w, dw = basis.sine_interpolation_weights(xa, xb, N, xs)
        assert abs(w @ q - f(xs)) < 1e-11
        assert abs(dw @ q - df(xs)) < 1e-9


@pytest.mark.parametrize("n", [2, 12, 24, 96])
def test_gauss_legendre_exactness(n):
    x, w = basis.gauss_legendre(n)
    for d in range(0, 2 * n):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-12


def test_gauss_legendre_against_library_and_high_precision():
    """Nodes match numpy's leggauss; weights match 40-digit Newton values to 2e-13
    (the library routine's weights are only good to ~1e-12 at n = 96)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for n in (24, 96, 180):
        x, w = basis.gauss_legendre(n)
        xl, wl = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, xl, atol=1e-15)
        np.testing.assert_allclose(w, wl, rtol=1e-11)
        for i in (0, 1, n // 3, n // 2, n - 1):
            z = mpmath.mpf(x[i])
            for _ in range(6):
                z = z - mpmath.legendre(n, z) / mpmath.diff(lambda t: mpmath.legendre(n, t), z)
            dp = mpmath.diff(lambda t: mpmath.legendre(n, t), z)
            wz = 2 / ((1 - z ** 2) * dp ** 2)
            assert abs(float(z) - x[i]) < 1e-15
            assert abs(float((wz - w[i]) / wz)) < 2e-13


@pytest.mark.parametrize("omega", [0, 1, 2, 5, 10])
def test_norm_assoc_legendre_matches_scipy(omega):
    x = np.linspace(-0.97, 0.97, 13)
    jmax = omega + 25
    P = basis.norm_assoc_legendre(jmax, omega, x)
    for j in range(omega, jmax + 1):
        ref = scipy.special.lpmv(omega, j, x)   # includes the Condon-Shortley phase
        lnorm = 0.5 * (np.log((2 * j + 1) / 2.0) + scipy.special.gammaln(j - omega + 1)
                       - scipy.special.gammaln(j + omega + 1))
        np.testing.assert_allclose(P[j - omega], ref * np.exp(lnorm), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("omega,n", [(0, 24), (1, 12), (3, 20), (10, 96), (20, 96), (20, 180)])
def test_fbr_rows_orthonormal(omega, n):
    """Quadrature exactness makes the n - Omega rows orthonormal, even at large Omega."""
    T = basis.fbr_matrix(omega, n)
    assert T.shape == (n - omega, n)
    np.testing.assert_allclose(T @ T.T, np.eye(n - omega), atol=2e-14)


def test_fbr_rows_are_legendre_functions():
    n, om = 24, 4
    x, w = basis.gauss_legendre(n)
    T = basis.fbr_matrix(om, n, x, w)
    for i in (0, 5, n - om - 1):
        j = om + i
        ref = scipy.special.lpmv(om, j, x) * np.sqrt((2 * j + 1) / 2.0 * np.exp(
            scipy.special.gammaln(j - om + 1) - scipy.special.gammaln(j + om + 1)))
        np.testing.assert_allclose(T[i], ref * np.sqrt(w), atol=1e-13)
    # Omega = 0 is a square orthogonal matrix
    T0 = basis.fbr_matrix(0, n, x, w)
    np.testing.assert_allclose(T0.T @ T0, np.eye(n), atol=1e-14)
