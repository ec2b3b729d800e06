"""Pins for the oracle's grid Hamiltonian and Chebyshev recursion (Sections 2.1-2.2).

P1 Hermiticity, P2 spectrum of H_s inside [-1, 1], closed-form spectra of the
radial and angular (J^2 + j^2 - 2 J.j) parts, P5 Chebyshev iterates against
exact diagonalisation, P6 time-domain norm conservation and the norm plateau.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import propagate
from oracle.hamiltonian import GridHamiltonian
from oracle.units import EV


def tiny(J=(0,), omega_max=0, nelec=1, NR=8, nr=6, ng=4, **kw):
    cfg = copy.deepcopy(W.C3 if nelec == 2 else W.C1)
    cfg["grid"] = dict(NR=NR, Rmin=0.8, Rmax=9.0, nr=nr, rmin=0.6, rmax=6.0, ngamma=ng)
    cfg["J"] = list(J)
    cfg["omega_max"] = omega_max
    cfg["nelec"] = nelec
    cfg.update(kw)
    return cfg


CASES = {
    "j0": tiny(),
    "j3_4omega": tiny(J=(3,), omega_max=3),
    "j5_trunc": tiny(J=(5,), omega_max=2),
    "two_state_batch": tiny(J=(0, 2), omega_max=2, nelec=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_hermiticity(name):
    """P1: <a | H b> = <H a | b> for seeded random vectors."""
    H = GridHamiltonian(CASES[name])
    a = W.random_state(H.shape, 2412)
    b = W.random_state(H.shape, 2413)
    lhs = np.vdot(a, H.apply_H(b))
    rhs = np.vdot(H.apply_H(a), b)
    scale = np.linalg.norm(a) * np.linalg.norm(H.apply_H(b))
    assert abs(lhs - rhs) <= 1e-13 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_scaled_spectrum_inside_unit_interval(name):
    """P2: the dense H_s (<= 2000 dims) has its spectrum inside [-1, 1]."""
    H = GridHamiltonian(CASES[name])
    M = H.dense_H()
    np.testing.assert_allclose(M, M.T, atol=1e-13 * np.abs(M).max())
    bj = np.repeat(H.block_J_index(), np.prod(H.shape[1:]))
    # H_s is block-diagonal in J: check each J separately
    for iJ in range(len(H.Js)):
        sel = bj == iJ
        ev = np.linalg.eigvalsh(M[np.ix_(sel, sel)])
        evs = (ev - H.E0[iJ]) / H.dE[iJ]
        assert evs.min() >= -1.0 and evs.max() <= 1.0
        emin, emax = H.spectral_bounds(iJ)
        assert emin <= ev.min() + 1e-12 and ev.max() <= emax + 1e-12


def test_radial_kinetic_closed_form_spectrum():
    """With V = 0 and one angular point (j = 0 only) H = T_R (+) T_r: eigenvalues add."""
    H = GridHamiltonian(tiny(ng=1, NR=10, nr=7))
    H.V[:] = 0.0
    ev = np.sort(np.linalg.eigvalsh(H.dense_H()))
    k_R = np.arange(1, 11) * np.pi / (9.0 - 0.8)
    k_r = np.arange(1, 8) * np.pi / (6.0 - 0.6)
    eR = np.minimum(k_R ** 2 / (2 * H.mu), H.tcut)
    er = np.minimum(k_r ** 2 / (2 * H.m), H.tcut)
    np.testing.assert_allclose(ev, np.sort((eR[:, None] + er[None, :]).ravel()), atol=1e-14)


@pytest.mark.parametrize("J,ng", [(0, 6), (1, 5), (3, 6), (4, 5)])
def test_angular_spectrum_is_rotor_l2(J, ng):
    """At one (r, R) point the angular operator has eigenvalues
    j(j+1)/(2 m r^2) + l(l+1)/(2 mu R^2) with l = |J-j|, |J-j|+2, ..., J+j
    (parity (-1)^J), for every j whose Omega blocks are all present.
    This pins the FBR transform, the Coriolis magnitudes and the sqrt(2)."""
    cfg = tiny(J=(J,), omega_max=J, NR=2, nr=2, ng=ng)
    cfg["caps"] = dict(vcut_eV=2.5, tcut_eV=2.5, erot_eV=1e6)
    H = GridHamiltonian(cfg)
    H.V[:] = 0.0
    H.TR[:] = 0.0
    H.Tr[:] = 0.0
    M = H.dense_H()
    k, m = 1, 0
    idx = [np.ravel_multi_index((b, n, k, m), H.shape)
           for b in range(H.nblk) for n in range(H.ng)]
    ev = np.sort(np.linalg.eigvalsh(M[np.ix_(idx, idx)]))
    fr, fR = H.fr[k], H.fR[m]
    expected = []
    for j in range(ng):           # j <= ng - 1 is present in every Omega block
        for l in range(abs(J - j), J + j + 1, 2):
            expected.append(fr * j * (j + 1) + fR * l * (l + 1))
    expected = np.sort(expected)
    # every expected eigenvalue appears in the spectrum
    for e in expected:
        assert np.min(np.abs(ev - e)) < 1e-12 * max(1.0, e / fr)


def _chebyshev_exact(H, q0, N):
    M = H.dense_H()
    bj = np.repeat(H.block_J_index(), np.prod(H.shape[1:]))
    E0 = H.E0[bj]
    dE = H.dE[bj]
    Ms = (M - np.diag(E0)) / dE[:, None]
    lam, U = np.linalg.eigh(Ms)
    c = U.T @ q0.ravel()
    th = np.arccos(np.clip(lam, -1, 1))
    return [U @ (np.cos(k * th) * c) for k in range(N)]


@pytest.mark.parametrize("name", ["j0", "j3_4omega"])
def test_chebyshev_matches_exact_diagonalisation(name):
    """P5: undamped q_k = T_k(H_s) q_0 = U cos(k arccos Lambda) U^T q_0."""
    H = GridHamiltonian(CASES[name])
    q0 = W.random_unit_state(H.shape, 2412)
    N = 200
    exact = _chebyshev_exact(H, q0, N + 1)
    D = np.ones((1, 1) + H.shape[2:])
    for k, q, qn in propagate.chebyshev_iterates(H, q0, D, N):
        assert np.linalg.norm(q.ravel() - exact[k]) < 1e-12
    assert np.linalg.norm(qn.ravel() - exact[N]) < 1e-12


def test_time_domain_norm_conserved():
    """P6: Psi(t) = sum_k f_k q_k (Bessel coefficients) equals exp(-iHt) Psi_0."""
    H = GridHamiltonian(CASES["j3_4omega"])
    q0 = W.random_unit_state(H.shape, 7)
    D = np.ones((1, 1) + H.shape[2:])
    t = 40.0 / H.dE[0]
    N = int(t * H.dE[0]) + 60
    states = [q0] + [qn for _, _, qn in propagate.chebyshev_iterates(H, q0, D, N)]
    psi_t = propagate.time_domain_packet(states, t, H.E0[0], H.dE[0])
    assert abs(np.linalg.norm(psi_t) - 1.0) < 1e-10
    lam, U = np.linalg.eigh(H.dense_H())
    exact = U @ (np.exp(-1j * lam * t) * (U.T @ q0.ravel()))
    assert np.linalg.norm(psi_t.ravel() - exact) < 1e-10


def test_undamped_norm_plateau_is_one_half():
    """Section 6: without absorption the Chebyshev norms oscillate about 1/2."""
    H = GridHamiltonian(CASES["j0"])
    q0 = W.random_unit_state(H.shape, 11)
    D = np.ones((1, 1) + H.shape[2:])
    norms = [np.sum(qn * qn) for _, _, qn in propagate.chebyshev_iterates(H, q0, D, 4000)]
    assert abs(np.mean(norms[1000:]) - 0.5) < 0.02
