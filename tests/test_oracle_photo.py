"""Pins for the photodissociation analysis of the oracle (Sections 2.3.2 and 2.5).

Autocorrelation against exact diagonalisation (undamped: C_k = sum_n |<phi_n|q_0>|^2
cos(k arccos lambda_n), lambda_n the eigenvalues of H_s); the spectrum's sum rule
(integral of a0(E) over the spectral range = C_0, exact for any number of terms) and its
line weights (undamped, the spectrum of a packet made of a few eigenstates carries each
state's population under its line).
"""
import copy

import numpy as np

import workloads as W
from oracle import photo
from oracle.hamiltonian import GridHamiltonian


def tiny(J, omega_max, NR=8, nr=6, ng=4):
    cfg = copy.deepcopy(W.C1)
    cfg["grid"] = dict(NR=NR, Rmin=0.8, Rmax=9.0, nr=nr, rmin=0.6, rmax=6.0, ngamma=ng)
    cfg["J"] = list(J)
    cfg["omega_max"] = omega_max
    return cfg


def dipole(r, R, x):
    """A smooth synthetic transition dipole (parallel-type: proportional to cos gamma)."""
    return (1.0 + 0.3 * (r - 1.4)) * np.exp(-0.05 * (R - 4.0) ** 2) * x


def bound_guess(H):
    """A normalised Gaussian standing in for the initial bound state."""
    n3, k3, m3 = np.meshgrid(H.x, H.r, H.R, indexing="ij")
    g = np.exp(-((k3 - 1.5) ** 2) - 0.2 * (m3 - 4.0) ** 2) * (1.0 + 0.5 * n3)
    return g / np.linalg.norm(g)


def per_J_spectral(H):
    """Eigen-decomposition of the dense H_s restricted to each J of the batch."""
    M = H.dense_H()
    bj = np.repeat(H.block_J_index(), np.prod(H.shape[1:]))
    out = []
    for iJ in range(len(H.Js)):
        idx = np.nonzero(bj == iJ)[0]
        Ms = (M[np.ix_(idx, idx)] - H.E0[iJ] * np.eye(len(idx))) / H.dE[iJ]
        lam, U = np.linalg.eigh(0.5 * (Ms + Ms.T))
        out.append((idx, lam, U))
    return out


def test_autocorrelation_matches_exact_diagonalisation():
    H = GridHamiltonian(tiny(J=(0, 2), omega_max=2))
    q0 = photo.photo_packet(H, bound_guess(H), dipole, block=0)
    q0 = q0 + photo.photo_packet(H, bound_guess(H), dipole, block=2)   # a block of J = 2
    assert np.linalg.norm(q0) > 0.1
    D = np.ones((1, 1) + H.shape[2:])
    N = 300
    C = photo.autocorrelation(H, q0, D, N)
    for iJ, (idx, lam, U) in enumerate(per_J_spectral(H)):
        c = U.T @ q0.ravel()[idx]
        th = np.arccos(np.clip(lam, -1, 1))
        exact = np.cos(np.outer(np.arange(N), th)) @ (c * c)
        assert np.max(np.abs(C[:, iJ] - exact)) < 1e-12 * max(1.0, abs(exact[0]))


def test_spectrum_sum_rule():
    """Substituting E = E0 + dE cos(theta) leaves (1/pi) int_0^pi sum_k (2 - delta_k0)
    cos(k theta) C_k d theta = C_0; the midpoint rule in theta with more nodes than terms
    integrates it exactly."""
    rng = W.rng(3)
    C = rng.standard_normal(40)
    E0, dE = 0.3, 0.7
    M = 400
    th = (np.arange(M) + 0.5) * np.pi / M
    E = E0 + dE * np.cos(th)
    a = photo.chebyshev_spectrum(C, E, E0, dE)
    integral = np.sum(a * dE * np.sin(th)) * np.pi / M
    assert abs(integral - C[0]) < 1e-12


def test_spectrum_line_weights():
    """Undamped, a packet of three eigenstates with populations w_n: the spectrum's integral
    over a window around each eigenvalue is w_n (the truncated sum is a Dirichlet kernel;
    its tails limit the agreement to about 1/(N * window))."""
    H = GridHamiltonian(tiny(J=(1,), omega_max=1))
    (idx, lam, U), = per_J_spectral(H)
    pick = [5, len(lam) // 2, len(lam) - 8]
    w = np.array([0.5, 0.3, 0.2])
    q0 = np.zeros(int(np.prod(H.shape)))
    q0[idx] = U[:, pick] @ np.sqrt(w)
    q0 = q0.reshape(H.shape)
    D = np.ones((1, 1) + H.shape[2:])
    N = 4000
    C = photo.autocorrelation(H, q0, D, N)[:, 0]
    assert abs(C[0] - 1.0) < 1e-12
    for n, wn in zip(pick, w):
        gap = min(abs(lam[n] - lam[m]) for m in pick if m != n)
        half = 0.4 * min(gap, 1.0 - abs(lam[n]))
        # integrate over theta in the window (E = E0 + dE cos theta), fine midpoint rule
        t_lo, t_hi = np.arccos(min(lam[n] + half, 1.0)), np.arccos(max(lam[n] - half, -1.0))
        M = 6000
        th = t_lo + (np.arange(M) + 0.5) * (t_hi - t_lo) / M
        E = H.E0[0] + H.dE[0] * np.cos(th)
        a = photo.chebyshev_spectrum(C, E, H.E0[0], H.dE[0])
        integral = np.sum(a * H.dE[0] * np.sin(th)) * (t_hi - t_lo) / M
        assert abs(integral - wn) < 1e-2, (n, integral, wn)
