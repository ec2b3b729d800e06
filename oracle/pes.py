"""Potential surfaces for the oracle. Test infrastructure only.

Geometry follows Section 2.1: r is the B->C vector, R joins the BC centre of mass
to A, and cos(gamma) = r.R / (rR). The user potential routine of Section 4
receives bond distances in bohr and returns the diabatic matrix in hartree; the
example routine clamps every distance to at least 0.25 bohr and references the
energy to the reactant asymptote (Section 6.1 listing). The surface itself is the
textbook Sato LEPS for H3 (the paper's BKMP2-like surface is not available).
"""
from __future__ import annotations

import numpy as np

from .units import EV

MIN_BOND = 0.25  # bohr, the clamp applied by the example potential routine


def bond_distances(r, R, cosg, mA, mB, mC):
    """Bond lengths (r_AB, r_BC, r_AC) from reactant Jacobi coordinates.

    With the BC centre of mass at B + (m_C/M_BC) r and A at that point plus R:
      A - B = R + (m_C/M_BC) r,   A - C = R - (m_B/M_BC) r,   C - B = r.
    """
    MBC = mB + mC
    sB = mC * r / MBC
    sC = mB * r / MBC
    rAB = np.sqrt(np.maximum(R * R + sB * sB + 2.0 * R * sB * cosg, 0.0))
    rAC = np.sqrt(np.maximum(R * R + sC * sC - 2.0 * R * sC * cosg, 0.0))
    rBC = np.asarray(r, dtype=float) * np.ones_like(rAB)
    return (np.maximum(rAB, MIN_BOND), np.maximum(rBC, MIN_BOND),
            np.maximum(rAC, MIN_BOND))


def leps(rAB, rBC, rAC, D_eV, beta, re, delta):
    """Sato LEPS energy in hartree, shifted so that A + BC(r = re) is zero.

    Singlet (Morse) and triplet (anti-Morse) curves per pair, x = r - re:
      1E = D (exp(-2 beta x) - 2 exp(-beta x))
      3E = (D/2) (exp(-2 beta x) + 2 exp(-beta x))
    Coulomb and exchange integrals with the Sato parameter Delta:
      Q = [1E (1 + Delta) + 3E (1 - Delta)] / (2 (1 + Delta))
      J = [1E (1 + Delta) - 3E (1 - Delta)] / (2 (1 + Delta))
    London equation:
      V = Q_AB + Q_BC + Q_AC - sqrt(((J_AB-J_BC)^2 + (J_BC-J_AC)^2 + (J_AC-J_AB)^2)/2)
    The returned value is V + D, which is zero at the reactant asymptote with BC at
    its equilibrium distance.
    """
    D = D_eV * EV

    def qj(rr):
        x = rr - re
        e1 = np.exp(-beta * x)
        singlet = D * (e1 * e1 - 2.0 * e1)
        triplet = 0.5 * D * (e1 * e1 + 2.0 * e1)
        den = 2.0 * (1.0 + delta)
        Q = (singlet * (1.0 + delta) + triplet * (1.0 - delta)) / den
        Jx = (singlet * (1.0 + delta) - triplet * (1.0 - delta)) / den
        return Q, Jx

    Qab, Jab = qj(rAB)
    Qbc, Jbc = qj(rBC)
    Qac, Jac = qj(rAC)
    exch = np.sqrt(0.5 * ((Jab - Jbc) ** 2 + (Jbc - Jac) ** 2 + (Jac - Jab) ** 2))
    return Qab + Qbc + Qac - exch + D


def morse(r, D_eV, beta, re):
    """Diatomic singlet curve shifted to zero at re (the LEPS limit for large R)."""
    D = D_eV * EV
    e1 = np.exp(-beta * (r - re))
    return D * (e1 * e1 - 2.0 * e1) + D


def potential_matrix(r, R, cosg, masses, pes):
    """Uncapped diabatic matrix V[..., L, L'] (hartree) at Jacobi points.

    ``pes`` is the workload's surface dictionary. With ``two_state`` set, state 2
    is the LEPS plus a bump in r, coupled to state 1 by a Gaussian in (R, r):
      V22 = V11 + b exp(-(r - r_b)^2 / w_b),  V12 = c exp(-((R-R_c)^2 + (r-r_c)^2)/w_c).
    Capping of the diagonal is applied later (it belongs to the Hamiltonian set-up,
    Section 2.1 item 5).
    """
    r, R, cosg = np.broadcast_arrays(np.asarray(r, float), np.asarray(R, float),
                                     np.asarray(cosg, float))
    if pes.get("kind") == "separable_eckart":
        return separable_eckart(r, R, pes)[..., None, None]
    if pes.get("kind") == "product_eckart":
        return product_eckart(r, R, cosg, masses, pes)[..., None, None]
    mA, mB, mC = masses
    rAB, rBC, rAC = bond_distances(r, R, cosg, mA, mB, mC)
    v11 = leps(rAB, rBC, rAC, pes["D_eV"], pes["beta"], pes["re"], pes["delta"])
    ts = pes.get("two_state")
    if not ts:
        return v11[..., None, None]
    v22 = v11 + ts["bump_eV"] * EV * np.exp(-(r - ts["bump_r0"]) ** 2 / ts["bump_w2"])
    v12 = ts["coup_eV"] * EV * np.exp(-((R - ts["coup_R0"]) ** 2 + (r - ts["coup_r0"]) ** 2)
                                      / ts["coup_w2"])
    out = np.empty(r.shape + (2, 2))
    out[..., 0, 0] = v11
    out[..., 1, 1] = v22
    out[..., 0, 1] = v12
    out[..., 1, 0] = v12
    return out


def eckart_barrier(R, V0_eV, alpha, Rb):
    """Symmetric Eckart barrier V0 sech^2(alpha (R - Rb)) in hartree."""
    return V0_eV * EV / np.cosh(alpha * (R - Rb)) ** 2


def product_jacobi_lengths(r, R, cosg, masses, arrangement):
    """(r', R'): lengths of the product Jacobi vectors at reactant Jacobi points.

    With B at the origin, C = r (along z) and A = (m_C/M_BC) r + R at angle gamma to r:
      "AC+B": r' = |C - A|, R' = |B - X_AC|;   "AB+C": r' = |B - A|, R' = |C - X_AB|,
    X_.. the centre of mass of the product diatom.
    """
    mA, mB, mC = masses
    r, R, cosg = np.broadcast_arrays(np.asarray(r, float), np.asarray(R, float),
                                     np.asarray(cosg, float))
    sing = np.sqrt(np.maximum(1.0 - cosg * cosg, 0.0))
    Ax, Az = R * sing, mC / (mB + mC) * r + R * cosg       # A; B = (0, 0); C = (0, r)
    if arrangement == "AC+B":
        rp = np.hypot(Ax, r - Az)
        Xx, Xz = mA * Ax / (mA + mC), (mA * Az + mC * r) / (mA + mC)
        Rp = np.hypot(Xx, Xz)
    elif arrangement == "AB+C":
        rp = np.hypot(Ax, Az)
        Xx, Xz = mA * Ax / (mA + mB), mA * Az / (mA + mB)
        Rp = np.hypot(Xx, r - Xz)
    else:
        raise ValueError("arrangement must be 'AC+B' or 'AB+C'")
    return rp, Rp


def product_eckart(r, R, cosg, masses, pes):
    """Test surface separable in PRODUCT Jacobi coordinates: an Eckart barrier in R' plus
    the diatomic Morse curve in r' (arrangement pes["arrangement"]).

    A product-arrangement packet in one diatomic state (v', j') keeps it, and its
    transmission through the barrier is the textbook Eckart closed form in R' with the
    product reduced mass mu' (the rotational terms conserve j' because V does not
    depend on gamma').
    """
    rp, Rp = product_jacobi_lengths(r, R, cosg, masses, pes["arrangement"])
    return (eckart_barrier(Rp, pes["V0_eV"], pes["alpha"], pes["Rb"])
            + morse(rp, pes["D_eV"], pes["beta"], pes["re"]))


def separable_eckart(r, R, pes):
    """Test surface: Eckart barrier in R plus the LEPS diatomic (Morse) curve in r.

    Separable, so a packet in the diatomic ground state keeps it and the
    transmission through the barrier has the textbook Eckart closed form.
    """
    return (eckart_barrier(R, pes["V0_eV"], pes["alpha"], pes["Rb"])
            + morse(r, pes["D_eV"], pes["beta"], pes["re"]))
