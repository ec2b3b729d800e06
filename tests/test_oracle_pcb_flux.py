"""Physics pin for the products-coordinate-based start (oracle/pcb.py; Section 2.4, the
first route; Eq. total-flux; Eq. initial-flux-collisions for a(E)).

The surface is an Eckart barrier in the PACKET's R_s plus a Morse curve in its r_s
(arrangement AC + B of the grid's labels), i.e. separable in the packet's own Jacobi
coordinates. At J = 0 a packet g(R_s) chi_(v0=0, j0=0)(r_s) keeps its diatomic state and
moves in R_s alone, so the probability transmitted through the barrier is the textbook Eckart
T(E_col) with the packet's reduced mass mu_s. The propagation, however, runs on the grid of
the other arrangement (A + BC): the packet is carried onto it once by the PCB start, and the
transmitted flux is measured there, through the grid's own surface r = r*. Atom C is heavy
(300 u), so the grid's r runs along the packet's R_s and its R along r_s; the surface
r = 5.5 lies between the barrier (R_s = 9) and the inner absorber, and every transmitted wave
crosses it toward smaller r: the flux probability (mass m of the grid's r) is -T.

This fixes, independently of the oracle's own formulas, the carried packet's normalisation,
the closed-form a(E) with mu_s and the energy reference e_(v0 j0) of the packet's diatom.
Plausible mistakes move the result well past the tolerance: the grid's mu in a(E) (mu is
twice mu_s here: |a|^2 off by sqrt 2) and the packet diatom's level solved with the grid's
r mass (an energy reference off by the zero-point difference) are planted below and must
fail.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import pcb, propagate as P
from oracle.hamiltonian import GridHamiltonian
from oracle.units import AMU, EV

V0_EV, ALPHA = 0.15, 1.0


def pcb_eckart_cfg():
    cfg = copy.deepcopy(W.C1)
    cfg["masses_u"] = (2.0, 1.0, 300.0)
    cfg["J"], cfg["omega_max"] = [0], 0
    # the grid's R ~ the packet's r_s (the bound A-C diatom), the grid's r ~ its R_s
    cfg["grid"] = dict(NR=24, Rmin=0.75, Rmax=2.6, nr=224, rmin=0.5, rmax=20.0, ngamma=12)
    cfg["pes"] = dict(kind="product_eckart", arrangement="AC+B", V0_eV=V0_EV, alpha=ALPHA,
                      Rb=9.0, D_eV=4.7466, beta=1.0, re=1.4014, delta=0.18)
    cfg["caps"] = dict(vcut_eV=5.0, tcut_eV=1.5, erot_eV=5.0)
    cfg["absorber"] = dict(RI=2.6, AR=0.0, nR=2, rI=16.5, Ar=0.5 / 3.5 ** 2, nr=2,
                           rI_low=4.0, Ar_low=0.5 / 3.5 ** 2)
    cfg["packet"] = dict(R0=13.5, Gamma=0.6, Ecol_eV=0.2, v0=0, j0=0, omega0=0, elec0=0)
    cfg["pcb"] = dict(arrangement="AC+B", rmin=0.5, rmax=4.5, nr=32)
    cfg["analysis"] = dict(rstar=5.5, E_lo_eV=0.08, E_hi_eV=0.34, nE=14, Rinf=2.0,
                           vmax=-1, jmax=0, kmin=0)
    cfg["steps"] = 1500
    return cfg


def eckart_T(E, mu, V0, alpha):
    a = np.sinh(np.pi * np.sqrt(2 * mu * E) / alpha) ** 2
    return a / (a + np.cosh(0.5 * np.pi * np.sqrt(8 * mu * V0 / alpha ** 2 - 1)) ** 2)


@pytest.mark.slow
def test_pcb_transmitted_flux_is_eckart_transmission(monkeypatch):
    cfg = pcb_eckart_cfg()
    H = GridHamiltonian(cfg)
    mA, mB, mC = (m * AMU for m in cfg["masses_u"])
    mu_s = mB * (mA + mC) / (mA + mB + mC)
    assert abs(H.mu / mu_s - 2.0) < 0.02              # the grid's mu is twice the packet's

    res = P.propagate(cfg, H=H, channels=False)
    pf = res["info"]["packet_function"]
    assert abs(pf.mu_s - mu_s) < 1e-9 * mu_s
    assert abs(res["norms"][0] - 1.0) < 1e-3          # the grid holds the carried packet
    Ecol = res["Ecol"]
    T = eckart_T(Ecol, mu_s, V0_EV * EV, ALPHA)
    assert T[0] < 1e-3 and T[-1] > 0.999              # the window spans the whole onset
    assert np.max(np.abs(-res["P_total"][0] - T)) < 1e-2

    # planted mistakes (on copies): the grid's mu in a(E); the packet diatom's level solved
    # with the grid's r mass m (an energy reference off by the zero-point difference)
    bad_pf = copy.copy(pf)
    bad_pf.mu_s = H.mu
    a_bad = pcb.incoming_amplitude(bad_pf, Ecol)
    _, Pbad = P.total_probability(H, res["A"], res["B"], res["theta"], a_bad)
    assert np.max(np.abs(-Pbad[0] - T)) > 0.1
    good_masses = pcb.packet_masses
    monkeypatch.setattr(pcb, "packet_masses", lambda m, a: (good_masses(m, a)[0], H.m))
    e_bad, _ = pcb.packet_diatom(H, cfg["pcb"], 0, 0, 1)
    de = (e_bad[0] - pf.e_v0j0) / EV
    assert abs(de) > 0.02
    shifted = copy.deepcopy(cfg)          # the sums taken at E_col + e_bad instead
    shifted["analysis"]["E_lo_eV"] += de
    shifted["analysis"]["E_hi_eV"] += de
    monkeypatch.setattr(pcb, "packet_masses", good_masses)
    res2 = P.propagate(shifted, H=H, channels=False)
    assert np.max(np.abs(-res2["P_total"][0] - T)) > 0.1
