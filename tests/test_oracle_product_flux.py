"""Pin for the product-channel |S|^2 assembly (Section 2.4, Eqs. final-states and
S-matrix-from-chebyshev): a product-arrangement Eckart problem with a closed form.

The surface is separable in PRODUCT Jacobi coordinates (arrangement AC + B): an Eckart
barrier in R' plus a Morse curve in r'. A packet g(R') chi_(v'=0, j'=1)(r') put in the
product frame keeps its diatomic state (V does not depend on gamma', so j' is conserved,
and the Morse part separates), so the probability transmitted through the barrier into
that product channel, summed over Omega', is the textbook Eckart transmission in R' with
the PRODUCT reduced mass mu', at the translational energy E - e_(v'j'). Atom C is heavy
(300 u), which makes R' run along the reactant r and r' along the reactant R, so the
product region is resolved by a modest reactant grid; A and B differ in mass so that the
reactant mu (about 2 u) and the product mu' (about 1 u) differ by a factor of two.

The packet carries equal Omega' = 0 and 1 components (J = 1), so the assembly is
checked in both helicities and in the sum over Omega'. The incoming amplitude a(E) of
the product packet is the closed-form Gaussian integral (the same closed form as the
reactant-packet pin), computed here with mu' and K' of the channel.

The same run pins the r branch of the total flux (Eq. total-flux): the surface r = r* = 5.5
lies between the barrier and the inner absorber, so every transmitted wave crosses it and
the flux probability, with the reduced mass m of r, is -T (the wave moves toward smaller r).

Plausible mistakes in the assembly each move the result by far more than the tolerance:
mu for mu' (x 0.71), a dropped K' (x 1/K' ~ 0.2), Omega' summed before squaring (x 2);
the first and the last are planted below and must fail.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import basis, products as PR, propagate as P
from oracle.hamiltonian import GridHamiltonian
from oracle.units import AMU, EV

V0_EV, ALPHA = 0.15, 1.0
PROD = dict(arrangement="AC+B", Rinf=5.0, rmin=0.5, rmax=4.5, nr=32, ngamma=12, vmax=1, jmax=2)


def product_eckart_cfg():
    cfg = copy.deepcopy(W.C1)
    cfg["masses_u"] = (2.0, 1.0, 300.0)
    cfg["J"], cfg["omega_max"] = [1], 1
    # reactant R ~ product r' (the bound A-C diatom), reactant r ~ product R'
    cfg["grid"] = dict(NR=24, Rmin=0.75, Rmax=2.6, nr=224, rmin=0.5, rmax=20.0, ngamma=12)
    cfg["pes"] = dict(kind="product_eckart", arrangement="AC+B", V0_eV=V0_EV, alpha=ALPHA,
                      Rb=9.0, D_eV=4.7466, beta=1.0, re=1.4014, delta=0.18)
    # the potential stays below the cap everywhere on this grid (max 4.46 eV), so the
    # surface is separable as written
    cfg["caps"] = dict(vcut_eV=5.0, tcut_eV=1.5, erot_eV=5.0)
    # absorbers at both ends of r (= R'): the transmitted wave (small R') and the
    # outgoing half of the real packet plus the reflected wave (large R')
    cfg["absorber"] = dict(RI=2.6, AR=0.0, nR=2, rI=16.5, Ar=0.5 / 3.5 ** 2, nr=2,
                           rI_low=4.0, Ar_low=0.5 / 3.5 ** 2)
    cfg["steps"] = 1500
    return cfg


def eckart_T(E, mu, V0, alpha):
    a = np.sinh(np.pi * np.sqrt(2 * mu * E) / alpha) ** 2
    return a / (a + np.cosh(0.5 * np.pi * np.sqrt(8 * mu * V0 / alpha ** 2 - 1)) ** 2)


def product_packet(H, pa, R0p, G, k0, Nn, jp, cop):
    """Phi'_(Omega') = g(R') chi_(0 jp)(r') P-bar_(jp)^(Omega')(cos gamma') cop[Omega'] in
    the product frame, put on the reactant grid: Phi_Omega = (r R / r' R') sum_Omega'
    T[Omega', Omega] Phi'_(Omega') (T orthogonal), q = Phi sqrt(dR dr w)."""
    M = PR.product_matrix(H.masses, PROD["arrangement"])
    n3, k3, m3 = np.meshgrid(np.arange(H.ng), np.arange(H.nr), np.arange(H.NR), indexing="ij")
    x, r, R = H.x[n3], H.r[k3], H.R[m3]
    r_vec = np.stack([r * np.sqrt(1 - x * x), 0 * r, r * x], axis=-1)
    R_vec = np.stack([0 * R, 0 * R, R], axis=-1)
    rp_vec = M[0, 0] * r_vec + M[0, 1] * R_vec
    Rp_vec = M[1, 0] * r_vec + M[1, 1] * R_vec
    rp, Rp = np.linalg.norm(rp_vec, axis=-1), np.linalg.norm(Rp_vec, axis=-1)
    nom = len(cop)
    flat_Rp, flat_rp = Rp_vec.reshape(-1, 3), rp_vec.reshape(-1, 3)
    Ts = np.array([PR.helicity_matrix(1, nom, PR.body_axes(a, b)) for a, b in zip(flat_Rp, flat_rp)])
    Ts = Ts.reshape(H.shape[1:] + (nom, nom))
    cgp = np.sum(rp_vec * Rp_vec, -1) / (rp * Rp)
    # the product diatomic state as a function: the sine-DVR interpolant of its vector
    Lp = PROD["rmax"] - PROD["rmin"]
    kk = np.arange(1, PROD["nr"] + 1) * np.pi / Lp
    sc = np.ones(PROD["nr"])
    sc[-1] = 1 / np.sqrt(2)
    coef = sc * (basis.dst2_matrix(PROD["nr"]) @ pa.states[(jp, 0)][1][:, 0])
    inside = (rp > PROD["rmin"]) & (rp < PROD["rmax"])
    chif = np.where(inside, np.sqrt(2 / Lp) * np.sin((rp[..., None] - PROD["rmin"]) * kk) @ coef, 0.0)
    g = Nn * np.exp(-(Rp - R0p) ** 2 / (2 * G * G)) * np.cos(k0 * Rp)
    jac = r * R / (rp * Rp)
    q = np.zeros(H.shape)
    for om in range(nom):
        ang = np.zeros(H.shape[1:])
        for op in range(nom):
            Pj = basis.norm_assoc_legendre(jp, op, cgp.ravel())[jp - op].reshape(cgp.shape)
            ang += Ts[..., op, om] * cop[op] * Pj
        q[H.block_index[(0, om, 0)]] = jac * g * chif * ang * np.sqrt(H.dR * H.dr * H.w[n3])
    return H.project(q)


@pytest.mark.slow
def test_product_channel_S2_is_eckart_transmission():
    cfg = product_eckart_cfg()
    H = GridHamiltonian(cfg)
    pa = PR.ProductAnalysis(H, PROD)
    mA, mB, mC = (m * AMU for m in cfg["masses_u"])
    mu_p = mB * (mA + mC) / (mA + mB + mC)          # B against the A-C diatom
    assert abs(H.mu / mu_p - 2.0) < 0.02             # the reactant mu is twice mu'

    # packet: Gaussian in R' (normalised in closed form), moving both ways; its inward
    # half meets the barrier at R' = 9, the projection surface is R'_inf = 5
    R0p, G, E0p = 13.5, 0.6, 0.2 * EV
    k0 = np.sqrt(2 * mu_p * E0p)
    Nn = 1.0 / np.sqrt(np.sqrt(np.pi) * G / 2 * (1 + np.exp(-k0 ** 2 * G ** 2) * np.cos(2 * k0 * R0p)))
    cop = np.array([1.0, 1.0]) / np.sqrt(2.0)        # Omega' = 0 and 1, equal weight
    q0 = product_packet(H, pa, R0p, G, k0, Nn, 1, cop)
    assert abs(np.sum(q0 * q0) - 1.0) < 1e-4         # the grid holds the normalised packet

    chans = pa.channels(0)
    e01 = [c[4] for c in chans if (c[0], c[1], c[2]) == (0, 0, 1)][0]
    Ep = np.linspace(0.08, 0.34, 14) * EV            # translational energy in R'
    Etot = e01 + Ep
    theta = np.arccos((Etot - H.E0[0]) / H.dE[0])
    D = P.damping_grid(H, cfg["absorber"])[None, None]
    Cp = np.zeros((len(chans), len(Ep)), dtype=complex)
    rstar = 5.5                                       # flux surface r = r*, also past the barrier
    psi0, _ = P.flux_cut(H, q0, rstar)
    A = np.zeros((H.nblk, len(Ep)) + psi0.shape[1:], dtype=complex)
    B = np.zeros_like(A)
    for k, q, _ in P.chebyshev_iterates(H, q0, D, cfg["steps"]):
        ck = (1.0 if k == 0 else 2.0) * np.exp(-1j * k * theta)
        Cp += ck[None, :] * pa.overlaps(q)[0][:, None]
        psi, dpsi = P.flux_cut(H, q, rstar)
        A += ck[None, :, None, None] * psi[:, None]
        B += ck[None, :, None, None] * dpsi[:, None]

    Kp = np.sqrt(2 * mu_p * Ep)
    a = np.sqrt(mu_p / (2 * np.pi * Kp)) * Nn * np.sqrt(2 * np.pi) * G / 2 * sum(
        np.exp(1j * (Kp + s * k0) * R0p - G ** 2 * (Kp + s * k0) ** 2 / 2) for s in (1, -1))
    T = eckart_T(Ep, mu_p, V0_EV * EV, ALPHA)
    assert T[0] < 1e-3 and T[-1] > 0.999              # the window spans the whole onset

    Pp = P.product_probabilities(H, pa, [Cp], theta[None, :], Etot, a)
    assert np.max(np.abs(Pp[(0, 0, 0, 1)] - T)) < 1e-2
    for key, val in Pp.items():                       # no other product channel is fed
        if key != (0, 0, 0, 1):
            assert np.max(val) < 1e-3, key

    # total flux through r = r* (the r branch of the total-flux reading, mass m of r):
    # every transmitted wave crosses that surface toward smaller r (negative flux), so
    # the flux probability is -T
    _, Ptot = P.total_probability(H, A, B, theta[None, :], a, flux_axis="r")
    assert np.max(np.abs(-Ptot[0] - T)) < 1e-2
    assert abs(H.mu / H.m - 2.0) < 0.02               # mu in place of m would halve it

    # planted mistakes (on copies, never in the oracle itself) must fail the same bound
    class MuSwapped:                                  # the reactant mu in place of mu'
        mu_p = H.mu
        channels = staticmethod(pa.channels)
    bad = P.product_probabilities(H, MuSwapped(), [Cp], theta[None, :], Etot, a)
    assert np.max(np.abs(bad[(0, 0, 0, 1)] - T)) > 0.2
    # Omega' summed before squaring: one channel carries the sum of both amplitudes
    Cs = Cp.copy()
    i0, i1 = [i for i, c in enumerate(chans) if (c[0], c[1], c[2]) == (0, 0, 1)]
    Cs[i0], Cs[i1] = Cp[i0] + Cp[i1], 0.0
    bad = P.product_probabilities(H, pa, [Cs], theta[None, :], Etot, a)
    assert np.max(np.abs(bad[(0, 0, 0, 1)] - T)) > 0.5
