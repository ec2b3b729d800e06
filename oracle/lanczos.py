"""Bound states by the non-orthogonal (Cullum-Willoughby) Lanczos method. Test
infrastructure only.

Section 2.3.2 obtains the initial bound state of a photodissociation from a separate
program that applies the same grid Hamiltonian in an iterative non-orthogonal Lanczos
method (the paper cites Cullum and Willoughby and gives no further detail). The steps,
as that method defines them:
  * the plain three-term recursion without any reorthogonalisation,
      beta_1 v_0 = 0,  w = H v_i - beta_i v_(i-1),  alpha_i = <v_i|w>,
      w <- w - alpha_i v_i,  beta_(i+1) = ||w||,  v_(i+1) = w / beta_(i+1),
    for i = 1..m, from a normalised start vector v_1;
  * the eigenvalues of the m x m tridiagonal T_m (diagonal alpha, off-diagonal beta);
    lost orthogonality shows as repeated copies of converged eigenvalues and as spurious
    ones;
  * the identification test: an eigenvalue of T_m that is simple (no copy within the
    tolerance) and also an eigenvalue of T_m with its first row and column deleted is
    spurious; every other distinct eigenvalue (each cluster of copies counted once) is
    accepted;
  * an eigenvector x = sum_i s_i v_i from the eigenvector s of T_m, with the Lanczos
    vectors regenerated by a second run of the same recursion.
The recursion runs on H_s = (H - E0)/dE (the propagation's operator) in the coordinates of
each block's angular functions (the FBR coefficients c = T^Omega q that the propagation
holds), i.e. on the span of those functions only. On the full grid the complement of that
span would add spurious directions: rounding seeds them and the unreorthogonalised
recursion finds their eigenvalues (the radial kinetic spectrum of H_s, or 0 of P H_s P).
Eigenvalues are returned in hartree, E = E0 + dE lambda.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal


def lanczos_coefficients(apply, v1, m):
    """alpha[0..m-1], beta[1..m] of the recursion (beta[0] = 0 is not returned)."""
    v_prev = np.zeros_like(v1)
    v = v1 / np.linalg.norm(v1)
    alpha = np.zeros(m)
    beta = np.zeros(m)      # beta[i] couples v_i and v_(i+1)
    b = 0.0
    for i in range(m):
        w = apply(v) - b * v_prev
        a = float(np.sum(v * w))
        w = w - a * v
        b = float(np.linalg.norm(w))
        alpha[i], beta[i] = a, b
        v_prev, v = v, w / b
    return alpha, beta


def cw_eigenvalues(alpha, beta, tol=1e-10):
    """Accepted eigenvalues of T_m (scaled units) by the identification test above."""
    m = len(alpha)
    lam = eigh_tridiagonal(alpha, beta[:m - 1], eigvals_only=True)
    hat = eigh_tridiagonal(alpha[1:], beta[1:m - 1], eigvals_only=True)
    out = []
    i = 0
    while i < m:
        j = i
        while j + 1 < m and lam[j + 1] - lam[i] <= tol:
            j += 1
        cluster = lam[i:j + 1]
        value = float(np.mean(cluster))
        if j > i or np.min(np.abs(hat - value)) > tol:
            out.append(value)           # a multiple copy, or simple and not in T-hat
        i = j + 1
    return np.array(out)


def ritz_vector(apply, v1, alpha, beta, lam):
    """x = sum_i s_i v_i for the eigenvector s of T_m nearest to lam (second run)."""
    m = len(alpha)
    ev, S = eigh_tridiagonal(alpha, beta[:m - 1])
    s = S[:, int(np.argmin(np.abs(ev - lam)))]
    v_prev = np.zeros_like(v1)
    v = v1 / np.linalg.norm(v1)
    x = np.zeros_like(v1)
    for i in range(m):
        x += s[i] * v
        w = apply(v) - (beta[i - 1] if i > 0 else 0.0) * v_prev
        w = w - alpha[i] * v
        v_prev, v = v, w / beta[i]
    return x / np.linalg.norm(x)


def fbr_maps(H, iJ=0):
    """(to_fbr, from_fbr) between grid values of the J's blocks and the concatenated FBR
    coefficients c = T^Omega q of those blocks (rows j = Omega .. ngamma - 1)."""
    blocks = [(b, om) for b, (jJ, J, om, L) in enumerate(H.blocks) if jJ == iJ]
    flat = (H.ng, H.nr * H.NR)

    def to_fbr(q):
        q = np.asarray(q).reshape(H.shape)
        return np.concatenate([(H.T[om] @ q[b].reshape(flat)).ravel() for b, om in blocks])

    def from_fbr(c):
        q = np.zeros(H.shape)
        o = 0
        for b, om in blocks:
            n = (H.ng - om) * H.nr * H.NR
            q[b] = (H.T[om].T @ c[o:o + n].reshape(H.ng - om, -1)).reshape(H.shape[1:])
            o += n
        return q

    return to_fbr, from_fbr


def bound_states(H, v1, m, emin, emax, iJ=0, tol=1e-10):
    """Accepted eigenvalues of H (hartree) in [emin, emax] for the J with index iJ, from
    m Lanczos steps on the blocks of that J (v1 restricted to them), in FBR coordinates.
    Also returns alpha, beta and the start vector in FBR coordinates."""
    to_fbr, from_fbr = fbr_maps(H, iJ)

    def apply(c):
        return to_fbr(H.apply_Hs(from_fbr(c)))

    c1 = to_fbr(v1)
    alpha, beta = lanczos_coefficients(apply, c1, m)
    lam = cw_eigenvalues(alpha, beta, tol)
    E = H.E0[iJ] + H.dE[iJ] * lam
    return E[(E >= emin) & (E <= emax)], alpha, beta
