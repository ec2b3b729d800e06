"""Photodissociation analysis: autocorrelation and Chebyshev spectrum. Test infrastructure only.

Section 2.3.2, Eq. (initial-photo-wvp): the initial packet is the transition dipole
times the initial bound state, projected onto the body-fixed functions of the final
state; Eqs. (fourier-transform), (chebyshev-transform): its energy content follows from
the autocorrelation C_k = <Psi(k=0)|Psi(k)> of the Chebyshev iterates,
  a0(E) = (1/pi) sum_k (2 - delta_k0) cos(k arccos E_s) C_k / (dE sqrt(1 - E_s^2)),
  E_s = (E - E0)/dE;
Section 2.5, Eq. (spectrum): the total photodissociation cross section is proportional to
h nu times the same sum (the constant A/(2 pi hbar) is a unit factor and is left out).

Readings (the paper cites its reference for the angular algebra of the dipole and does
not give the dipole or the bound states of any example):
  * the synthetic dipole is one body-fixed component d(r, R, gamma) acting within one
    helicity block: Psi(0) = P_block [d * Psi_bound] (P the projection onto the block's
    angular functions), the rotational coupling coefficients of Eq. (initial-photo-wvp)
    being absorbed in d;
  * Psi(k) are the damped Chebyshev iterates of Eq. (wvp-k) started from Psi(0), and
    C_k is taken for k = 0..N-1 ("N iterations", as for the scattering sums);
  * cos(-k arccos E_s) = cos(k arccos E_s), evaluated directly from k * theta in FP64.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import GridHamiltonian
from .propagate import chebyshev_iterates


def autocorrelation(H: GridHamiltonian, q0, D, N):
    """C_k = <q_0|q_k> for k = 0..N-1, one value per J of the batch: [N, nJ].

    The blocks of different J are independent propagations, so each J has its own
    autocorrelation (the sum over its Omega and Lambda blocks)."""
    bj = H.block_J_index()
    nJ = len(H.Js)
    out = np.zeros((N, nJ))
    for k, q, _ in chebyshev_iterates(H, q0, D, N):
        per_block = np.sum(q0 * q, axis=(1, 2, 3))
        for iJ in range(nJ):
            out[k, iJ] = np.sum(per_block[bj == iJ])
    return out


def chebyshev_spectrum(C, E, E0, dE):
    """a0(E) of Eq. (chebyshev-transform) from the autocorrelation C[k] (k = 0..N-1) at
    total energies E (hartree) for the spectral centre E0 and half-width dE."""
    C = np.asarray(C, dtype=float)
    Es = (np.asarray(E, dtype=float) - E0) / dE
    theta = np.arccos(Es)
    k = np.arange(len(C))
    w = np.where(k == 0, 1.0, 2.0)
    s = np.cos(np.outer(theta, k)) @ (w * C)
    return s / (np.pi * dE * np.sqrt(1.0 - Es * Es))


def photo_packet(H: GridHamiltonian, bound, dipole, block=0):
    """Psi(0) = P_block [d Psi_bound] (the reading of Eq. initial-photo-wvp above).

    bound  grid values of the initial bound state on the (gamma, r, R) grid of one block
           (shape H.shape[1:]);
    dipole callable d(r, R, cos gamma) -> values (the synthetic transition dipole).
    The result has the full block shape, nonzero in `block` only."""
    n3, k3, m3 = np.meshgrid(H.x, H.r, H.R, indexing="ij")
    q = np.zeros(H.shape)
    q[block] = dipole(k3, m3, n3) * np.asarray(bound, dtype=float)
    return H.project(q)
