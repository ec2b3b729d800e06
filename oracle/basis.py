"""Grids and one-dimensional bases for the oracle. Test infrastructure only.

Section 2.1: equidistant grids in r and R, Gauss-Legendre points in gamma; the
radial kinetic terms are applied with a real sine transform that imposes regular
boundary conditions (item 2); the angular terms j^2 and l^2 are applied in a finite
basis (FBR) where their matrix elements are analytic (item 3).

Reading of the silent points (the paper names only "real sine transform" and the
FBR): the radial grid is the midpoint sine DVR between walls at the interval ends,
transformed by the orthonormal DST-II; the FBR of helicity Omega uses normalised
associated Legendre functions j = Omega .. n - 1 on the shared n Gauss-Legendre
nodes, which that quadrature makes exactly orthonormal.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- radial

def sine_dvr_nodes(xa: float, xb: float, N: int):
    """Midpoint nodes x_i = xa + (i - 1/2) dx, i = 1..N, dx = (xb - xa)/N."""
    dx = (xb - xa) / N
    return xa + (np.arange(1, N + 1) - 0.5) * dx, dx


def dst2_matrix(N: int) -> np.ndarray:
    """Orthonormal DST-II: S[j-1, i-1] = sqrt(2/N) s_j sin(j pi (i - 1/2) / N).

    s_j = 1 for j < N and s_N = 1/sqrt(2), so that S S^T = 1.
    """
    j = np.arange(1, N + 1)[:, None]
    i = np.arange(1, N + 1)[None, :]
    S = np.sqrt(2.0 / N) * np.sin(j * np.pi * (i - 0.5) / N)
    S[N - 1, :] *= 1.0 / np.sqrt(2.0)
    return S


def sine_wavenumbers(xa: float, xb: float, N: int) -> np.ndarray:
    """k_j = j pi / L for j = 1..N: the sine functions vanish at both walls."""
    return np.arange(1, N + 1) * np.pi / (xb - xa)


def radial_kinetic_eigenvalues(xa, xb, N, mass, tcut):
    """Capped kinetic energies min(k_j^2 / 2 mass, tcut), j = 1..N (radcutmaxeV)."""
    k = sine_wavenumbers(xa, xb, N)
    return np.minimum(k * k / (2.0 * mass), tcut)


def radial_kinetic_matrix(xa, xb, N, mass, tcut) -> np.ndarray:
    """T = S^T diag(min(k_j^2/2 mass, tcut)) S: -(1/2 mass) d^2/dx^2 in the sine DVR."""
    S = dst2_matrix(N)
    lam = radial_kinetic_eigenvalues(xa, xb, N, mass, tcut)
    return S.T @ (lam[:, None] * S)


def sine_basis_at(xa, xb, N, x):
    """phi_j(x) = sqrt(2/L) sin(k_j (x - xa)) and d phi_j/dx, j = 1..N."""
    L = xb - xa
    k = sine_wavenumbers(xa, xb, N)
    ph = np.sqrt(2.0 / L) * np.sin(k * (x - xa))
    dph = np.sqrt(2.0 / L) * k * np.cos(k * (x - xa))
    return ph, dph


def sine_interpolation_weights(xa, xb, N, x):
    """Weights w, dw with f(x) = w . q and f'(x) = dw . q for a DVR vector q.

    If q_i = f(x_i) sqrt(dx) and f = sum_j alpha_j phi_j, then the DST-II
    coefficients a = S q satisfy alpha_j = s_j a_j, so
      f(x) = sum_j s_j a_j phi_j(x).
    """
    S = dst2_matrix(N)
    s = np.ones(N)
    s[N - 1] = 1.0 / np.sqrt(2.0)
    ph, dph = sine_basis_at(xa, xb, N, x)
    return S.T @ (s * ph), S.T @ (s * dph)


# ---------------------------------------------------------------------------- angular

def gauss_legendre(n: int):
    """Gauss-Legendre nodes x_k = cos(gamma_k) (ascending) and weights on [-1, 1].

    From the definition: the nodes are the roots of P_n, found by Newton's method
    from cos(pi (k + 3/4) / (n + 1/2)); the weights are w_k = 2 / ((1 - x_k^2) P_n'(x_k)^2).
    """
    def pn_dpn(z):
        p0, p1 = np.ones_like(z), z.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k
        if n == 1:
            p0 = np.ones_like(z)
        return p1, n * (z * p1 - p0) / (z * z - 1.0)

    z = np.cos(np.pi * (np.arange(n) + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = pn_dpn(z)
        dz = p / dp
        z = z - dz
        if np.max(np.abs(dz)) < 1e-16:
            break
    _, dp = pn_dpn(z)
    w = 2.0 / ((1.0 - z * z) * dp * dp)
    order = np.argsort(z)
    return z[order], w[order]


def norm_assoc_legendre(jmax: int, omega: int, x) -> np.ndarray:
    """P-bar_j^Omega(x) for j = Omega..jmax, normalised so that int P-bar^2 dx = 1.

    Condon-Shortley phase included. Recurrences (standard, in normalised form):
      P-bar_Omega^Omega = c_Omega (1 - x^2)^(Omega/2),  c_0 = 1/sqrt(2),
                          c_Omega = -sqrt((2 Omega + 1) / (2 Omega)) c_(Omega-1)
      P-bar_(Omega+1)^Omega = sqrt(2 Omega + 3) x P-bar_Omega^Omega
      P-bar_j^Omega = a_j (x P-bar_(j-1) - P-bar_(j-2) / a_(j-1)),
                      a_j = sqrt((4 j^2 - 1) / (j^2 - Omega^2))
    Returns an array of shape (jmax - omega + 1, len(x)).
    """
    x = np.asarray(x, dtype=float)
    out = np.zeros((jmax - omega + 1,) + x.shape)
    c = 1.0 / np.sqrt(2.0)
    for m in range(1, omega + 1):
        c *= -np.sqrt((2.0 * m + 1.0) / (2.0 * m))
    out[0] = c * (1.0 - x * x) ** (0.5 * omega)
    if jmax >= omega + 1:
        out[1] = np.sqrt(2.0 * omega + 3.0) * x * out[0]

    def a(j):
        return np.sqrt((4.0 * j * j - 1.0) / (j * j - omega * omega))

    for j in range(omega + 2, jmax + 1):
        out[j - omega] = a(j) * (x * out[j - omega - 1] - out[j - omega - 2] / a(j - 1))
    return out


def fbr_matrix(omega: int, n: int, x=None, w=None) -> np.ndarray:
    """Angular transform T^Omega ((n - Omega) x n) from the DVR points to the FBR.

    Rows T[i, k] = P-bar_j^Omega(x_k) sqrt(w_k) for j = Omega + i = Omega .. n - 1.
    Every product P-bar_j^Omega P-bar_j'^Omega is (1 - x^2)^Omega times a polynomial
    of degree j + j' - 2 Omega, so the whole integrand has degree j + j' <= 2n - 2
    and the n-point Gauss-Legendre rule integrates it exactly: the rows are
    orthonormal (T T^T = 1). For Omega = 0 the matrix is square and orthogonal.
    (Completing the Omega > 0 basis to n functions is ill-conditioned on the shared
    grid and is not done; block Omega carries n - Omega angular functions.)
    """
    if x is None:
        x, w = gauss_legendre(n)
    return norm_assoc_legendre(n - 1, omega, x) * np.sqrt(w)[None, :]
