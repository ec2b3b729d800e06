"""Pins for the oracle's non-orthogonal (Cullum-Willoughby) Lanczos (Section 2.3.2, the
bound-state program): on a tiny grid, with six times as many steps as the dimension
(so orthogonality is long lost), the accepted eigenvalues are exactly the distinct
eigenvalues of the dense Hamiltonian on the blocks' span, no spurious value survives the
identification test (and without it some would), and a Ritz vector solves the eigenvalue
equation. The recursion runs in the blocks' FBR coordinates (as the propagation does).
"""
import copy

import numpy as np

import workloads as W
from oracle import lanczos
from oracle.hamiltonian import GridHamiltonian


def tiny_cfg():
    cfg = copy.deepcopy(W.C1)
    cfg["grid"] = dict(NR=8, Rmin=0.8, Rmax=9.0, nr=6, rmin=0.6, rmax=6.0, ngamma=4)
    cfg["J"], cfg["omega_max"] = [1], 1
    return cfg


def span_spectrum(H):
    """Eigenvalues (hartree) of H on the span of the blocks' angular functions."""
    n = int(np.prod(H.shape))
    P = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0.0
        e[i] = 1.0
        P[:, i] = H.project(e).ravel()
    w, U = np.linalg.eigh(0.5 * (P + P.T))
    Q = U[:, w > 0.5]
    M = H.dense_H()
    return np.linalg.eigvalsh(Q.T @ (0.5 * (M + M.T)) @ Q)


def test_cullum_willoughby_finds_the_spectrum():
    H = GridHamiltonian(tiny_cfg())
    exact = span_spectrum(H)
    distinct = exact[np.concatenate(([True], np.diff(exact) > 1e-9 * H.dE[0]))]
    v1 = H.project(W.random_state(H.shape, 4))
    m = 6 * len(exact)
    E, alpha, beta = lanczos.bound_states(H, v1, m, -np.inf, np.inf)
    tol = 1e-8 * H.dE[0]
    # every accepted value is an eigenvalue, every distinct eigenvalue is found once
    assert len(E) == len(distinct)
    assert np.max(np.abs(np.sort(E) - distinct)) < tol
    # without the identification test, spurious values (or extra copies) remain
    lam_all = np.linalg.eigvalsh(np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1))
    E_all = H.E0[0] + H.dE[0] * lam_all
    far = [x for x in E_all if np.min(np.abs(exact - x)) > 1e3 * tol]
    assert len(far) > 0


def test_ritz_vector_solves_the_eigenvalue_equation():
    H = GridHamiltonian(tiny_cfg())
    v1 = H.project(W.random_state(H.shape, 4))
    m = 300
    E, alpha, beta = lanczos.bound_states(H, v1, m, -np.inf, np.inf)
    E0 = np.min(E)
    lam = (E0 - H.E0[0]) / H.dE[0]
    to_fbr, from_fbr = lanczos.fbr_maps(H)
    c = lanczos.ritz_vector(lambda c: to_fbr(H.apply_Hs(from_fbr(c))), to_fbr(v1), alpha, beta,
                            lam)
    x = from_fbr(c)
    res = np.linalg.norm(H.apply_H(x) - E0 * x)
    assert res < 1e-8 * H.dE[0]
