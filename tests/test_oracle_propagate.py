"""Pins for the oracle's packet, damping, energy projection and flux (Sections 2.2-2.4).

P9 a(E) against the closed-form Gaussian integral; P7/P8 the separable Eckart
problem, whose transmission (flux) and reflection (channel projection) have a
textbook closed form; P10 r*-independence of the total flux and P11 unitarity
(flux + inelastic = 1), both paper invariants.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import propagate as P
from oracle.hamiltonian import GridHamiltonian
from oracle.units import EV


def test_damping_profile_definition():
    x = np.linspace(0.0, 10.0, 11)
    d = P.damping_profile(x, 6.0, 0.3, 2)
    assert np.all(d[x <= 6.0] == 1.0)
    np.testing.assert_allclose(d[x > 6.0], np.exp(-0.3 * (x[x > 6.0] - 6.0) ** 2))


def test_incoming_amplitude_closed_form():
    """P9: a(E) = N sqrt(mu/(2 pi K)) (sqrt(2 pi) Gamma / 2) sum_+- exp(i(K+-k0)R0 - Gamma^2 (K+-k0)^2 / 2)."""
    cfg = copy.deepcopy(W.C1)
    cfg["grid"].update(NR=320, Rmin=0.5, Rmax=20.0)
    cfg["packet"].update(Gamma=0.5, R0=10.0)
    H = GridHamiltonian(cfg)
    q0, info = P.initial_packet(H, cfg["packet"])
    assert abs(np.sum(q0 * q0) - 1.0) < 1e-14
    Ecol = np.linspace(0.2, 1.6, 15) * EV
    a = P.incoming_amplitude(H, info["g_tilde"], Ecol)
    G, R0, k0 = 0.5, 10.0, info["k0"]
    K = np.sqrt(2 * H.mu * Ecol)
    norm = 1.0 / np.sqrt(np.sqrt(np.pi) * G / 2 * (1 + np.exp(-k0 ** 2 * G ** 2) * np.cos(2 * k0 * R0)))
    s = sum(np.exp(1j * (K + sg * k0) * R0 - G ** 2 * (K + sg * k0) ** 2 / 2) for sg in (1, -1))
    exact = norm * np.sqrt(H.mu / (2 * np.pi * K)) * np.sqrt(2 * np.pi) * G / 2 * s
    np.testing.assert_allclose(a, exact, rtol=1e-10, atol=1e-12)


def eckart_cfg():
    cfg = copy.deepcopy(W.C1)
    cfg["grid"] = dict(NR=192, Rmin=0.5, Rmax=30.0, nr=16, rmin=0.5, rmax=4.0, ngamma=2)
    cfg["pes"] = dict(kind="separable_eckart", V0_eV=0.4, alpha=1.0, Rb=15.0, **W.LEPS_H3)
    # the cap is lifted so that V = Eckart(R) + Morse(r) stays separable where the
    # diatomic ground state has amplitude
    cfg["caps"] = dict(vcut_eV=6.0, tcut_eV=2.5, erot_eV=5.0)
    cfg["packet"] = dict(R0=22.0, Gamma=0.5, Ecol_eV=0.5, v0=0, j0=0, omega0=0, elec0=0)
    cfg["absorber"] = dict(RI=25.0, AR=0.5 / 25.0, nR=2, rI=3.9, Ar=0.0, nr=2,
                           RI_low=6.0, AR_low=0.5 / 5.5 ** 2)
    cfg["analysis"] = dict(rstar=2.0, E_lo_eV=0.15, E_hi_eV=1.0, nE=18, Rinf=23.5,
                           vmax=0, jmax=0, kmin=300)
    cfg["steps"] = 3500
    return cfg


def eckart_T(E, mu, V0, alpha):
    a = np.sinh(np.pi * np.sqrt(2 * mu * E) / alpha) ** 2
    return a / (a + np.cosh(0.5 * np.pi * np.sqrt(8 * mu * V0 / alpha ** 2 - 1)) ** 2)


def test_eckart_transmission_and_reflection():
    """P7 + P8: flux through R* = 8 on the far side gives T(E); the reactant
    channel projection at R_inf on the near side gives |S_00|^2 = 1 - T(E)."""
    cfg = eckart_cfg()
    res = P.propagate(cfg, flux_axis="R", flux_at=8.0, channels=True)
    H = res["H"]
    T = eckart_T(res["Ecol"], H.mu, 0.4 * EV, 1.0)
    # flux toward smaller R is negative in the r-convention; transmitted probability:
    Ptr = -res["P_total"][0]
    assert np.max(np.abs(Ptr - T)) < 1e-3
    refl = res["S2"][0]
    # below 0.25 eV the slow outgoing half of the packet, weakly reflected by the far
    # absorber, still crosses R_inf after k_min: a looser bound there
    hi = res["Ecol"] >= 0.25 * EV
    assert np.max(np.abs(refl - (1.0 - T))[hi]) < 1e-3
    assert np.max(np.abs(refl - (1.0 - T))) < 1e-2
    assert res["norms"][-1] < 1e-5


def physics_cfg():
    """J = 0 H + DH on the textbook H3 LEPS (beta = 1.9426 / Angstrom), converged in 3000 steps."""
    cfg = copy.deepcopy(W.C1)
    cfg["pes"]["beta"] = 1.9426 * 0.529177210903
    cfg["grid"] = dict(NR=72, Rmin=0.5, Rmax=14.0, nr=60, rmin=0.5, rmax=11.0, ngamma=12)
    cfg["absorber"] = W._absorber(14.0, 10.0, 11.0, 7.5, strength=0.5)
    cfg["packet"].update(R0=8.5, Gamma=0.4)
    cfg["analysis"].update(kmin=250, Rinf=9.0, rstar=5.0, nE=30, E_lo_eV=0.3, E_hi_eV=1.2,
                           vmax=2, jmax=11)
    cfg["steps"] = 3000
    return cfg


@pytest.mark.slow
def test_flux_surface_independence_and_unitarity():
    """P10: P(E) does not depend on r* (Section 2.4). P11: flux + inelastic = 1 (Section 6)."""
    cfg = physics_cfg()
    H = GridHamiltonian(cfg)
    an = cfg["analysis"]
    q0, info = P.initial_packet(H, cfg["packet"])
    D = P.damping_grid(H, cfg["absorber"])[None, None]
    Ecol, Etot, theta = P.energy_grid(H, an, info["E_v0j0"])
    rs = [4.5, 5.0, 5.5]
    A = [0j] * 3
    B = [0j] * 3
    chans, chis, eps = P.reactant_channels(H, an)
    m_inf = int(np.argmin(np.abs(H.R - an["Rinf"])))
    Cc = 0j
    for k, q, qn in P.chebyshev_iterates(H, q0, D, cfg["steps"]):
        ck = (1.0 if k == 0 else 2.0) * np.exp(-1j * k * theta[0])
        for i, rr in enumerate(rs):
            psi, dpsi = P.flux_cut(H, q, rr)
            A[i] = A[i] + ck[:, None, None] * psi[0][None]
            B[i] = B[i] + ck[:, None, None] * dpsi[0][None]
        if k >= an["kmin"]:
            Cc = Cc + ck[None, :] * P.channel_overlaps(H, q, chans, chis, m_inf)[:, None]
    a = P.incoming_amplitude(H, info["g_tilde"], Ecol)
    pref = 1 / (2 * np.pi * H.dE[0] * np.sin(theta[0]))
    Ps = [2 * np.pi / H.m * np.sum(np.imag(np.conj(A[i]) * B[i]), axis=(1, 2)) * pref ** 2
          / np.abs(a) ** 2 for i in range(3)]
    K2 = 2 * H.mu * (Etot[None] - eps[:, None])
    S2 = np.where(K2 > 0, 2 * np.pi * np.sqrt(np.maximum(K2, 0)) / H.mu
                  * np.abs(pref * Cc) ** 2 / np.abs(a) ** 2, 0)
    inel = S2.sum(0)
    assert np.all(Ps[1] > 0.2) and np.all(Ps[1] < 0.8)
    assert np.max(np.abs(Ps[0] - Ps[1])) < 1e-2
    assert np.max(np.abs(Ps[2] - Ps[1])) < 1e-2
    assert np.max(np.abs(Ps[1] + inel - 1.0)) < 3e-2
    assert np.mean(np.abs(Ps[1] + inel - 1.0)) < 1e-2


def test_propagate_bookkeeping_c1_short():
    """q_0..q_(N-1) enter the sums; the state after N steps is q_N (recursion of Eq. wvp-k)."""
    cfg = copy.deepcopy(W.C1)
    r3 = P.propagate(cfg, nsteps=3, channels=False)
    r2 = P.propagate(cfg, nsteps=2, channels=False)
    H = r3["H"]
    q0, _ = P.initial_packet(H, cfg["packet"])
    D = P.damping_grid(H, cfg["absorber"])[None, None]
    q1 = D * H.apply_Hs(q0)
    q2 = D * (2 * H.apply_Hs(q1) - D * q0)
    q3 = D * (2 * H.apply_Hs(q2) - D * q1)
    np.testing.assert_allclose(r3["q"], q3, atol=1e-15)
    np.testing.assert_allclose(r3["q_prev"], q2, atol=1e-15)
    np.testing.assert_allclose(r2["q"], q2, atol=1e-15)
    # sums: A(3 steps) - A(2 steps) = c_2 psi(q_2)
    psi2, _ = P.flux_cut(H, q2, cfg["analysis"]["rstar"])
    c2 = 2.0 * np.exp(-1j * 2 * r3["theta"][0])
    np.testing.assert_allclose(r3["A"] - r2["A"], c2[None, :, None, None] * psi2[:, None],
                               atol=1e-14)
