"""Pins for the oracle's potential surfaces and diatomic states (Section 4).

Checks against an independent Cartesian construction of the Jacobi geometry, the
closed-form limits of the LEPS surface, and the Morse closed-form eigenvalues.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import pes, propagate
from oracle.hamiltonian import GridHamiltonian
from oracle.units import AMU, EV


def test_bond_distances_match_cartesian_construction():
    mA, mB, mC = (m * AMU for m in W.MASSES_H_DH)
    rng = np.random.default_rng(7)
    for _ in range(50):
        r, R = rng.uniform(0.5, 6.0), rng.uniform(0.5, 8.0)
        g = rng.uniform(0, np.pi)
        B = np.zeros(3)
        C = np.array([0.0, 0.0, r])                       # r = B -> C
        com = (mB * B + mC * C) / (mB + mC)
        # body frame of Section 2.1 rotated so that r lies on z; R at angle gamma to r
        A = com + R * np.array([np.sin(g), 0.0, np.cos(g)])
        rab, rbc, rac = pes.bond_distances(r, R, np.cos(g), mA, mB, mC)
        assert abs(rab - max(np.linalg.norm(A - B), 0.25)) < 1e-12
        assert abs(rbc - max(np.linalg.norm(C - B), 0.25)) < 1e-12
        assert abs(rac - max(np.linalg.norm(A - C), 0.25)) < 1e-12


def test_leps_diatomic_limit_is_morse():
    p = W.LEPS_H3
    # the London exchange term selects the singlet (Morse) branch while J_BC < 0,
    # i.e. below about 40 eV; V is capped far below that
    r = np.linspace(0.8, 6.0, 40)
    v = pes.leps(np.full_like(r, 60.0), r, np.full_like(r, 61.0), **p)
    np.testing.assert_allclose(v, pes.morse(r, p["D_eV"], p["beta"], p["re"]), atol=1e-14)
    # Morse closed form: minimum 0 at re, dissociation at D
    assert abs(pes.morse(p["re"], p["D_eV"], p["beta"], p["re"])) < 1e-15
    assert abs(pes.morse(80.0, p["D_eV"], p["beta"], p["re"]) - p["D_eV"] * EV) < 1e-12


def test_leps_full_dissociation_and_symmetry():
    p = W.LEPS_H3
    # three atoms far apart: every pair energy vanishes, V + D = D
    assert abs(pes.leps(50.0, 60.0, 70.0, **p) - p["D_eV"] * EV) < 1e-14
    # identical pair curves: V is symmetric in the three distances
    rng = np.random.default_rng(1)
    d = rng.uniform(1.0, 4.0, size=(20, 3))
    for a, b, c in d:
        v = pes.leps(a, b, c, **p)
        for perm in [(b, a, c), (c, b, a), (a, c, b), (b, c, a)]:
            assert abs(pes.leps(*perm, **p) - v) < 1e-14


def test_two_state_matrix_definition():
    cfg = W.C3
    ts = cfg["pes"]["two_state"]
    r, R, cg = 1.7, 3.2, 0.3
    M = pes.potential_matrix(r, R, cg, [m * AMU for m in cfg["masses_u"]], cfg["pes"])
    v11 = M[0, 0]
    assert abs(M[0, 1] - M[1, 0]) == 0.0
    assert abs(M[1, 1] - v11 - 0.6 * EV * np.exp(-(r - 1.4) ** 2)) < 1e-15
    assert abs(M[0, 1] - 0.05 * EV * np.exp(-((R - 3) ** 2 + (r - 1.8) ** 2))) < 1e-16
    assert ts["bump_eV"] == 0.6


def _morse_cfg(nr=160, rmax=8.0):
    cfg = copy.deepcopy(W.C1)
    cfg["grid"] = dict(NR=4, Rmin=0.5, Rmax=14.0, nr=nr, rmin=0.3, rmax=rmax, ngamma=2)
    cfg["caps"] = dict(vcut_eV=1e4, tcut_eV=1e4, erot_eV=5.0)
    return cfg


def test_diatomic_morse_eigenvalues_closed_form():
    """P4: E_v = w (v + 1/2) - [w (v + 1/2)]^2 / (4 D), w = beta sqrt(2 D / m)."""
    cfg = _morse_cfg()
    H = GridHamiltonian(cfg)
    e, U = propagate.diatomic_states(H, 0, 0, 6)
    p = W.LEPS_H3
    D = p["D_eV"] * EV
    w = p["beta"] * np.sqrt(2 * D / H.m)
    v = np.arange(6)
    exact = w * (v + 0.5) - (w * (v + 0.5)) ** 2 / (4 * D)
    np.testing.assert_allclose(e, exact, rtol=1e-9)
    # eigenvectors are grid-normalised and sign-fixed
    np.testing.assert_allclose(np.sum(U * U, axis=0), 1.0, atol=1e-13)
    assert U[np.argmax(np.abs(U[:, 0])), 0] > 0


def test_diatomic_rotational_term():
    """For j > 0 the centrifugal term raises E_v0j by about B_e j(j+1), B_e = 1/(2 m re^2)."""
    cfg = _morse_cfg()
    H = GridHamiltonian(cfg)
    e0, _ = propagate.diatomic_states(H, 0, 0, 1)
    e1, _ = propagate.diatomic_states(H, 1, 0, 1)
    Be = 1.0 / (2 * H.m * W.LEPS_H3["re"] ** 2)
    assert 0.9 * 2 * Be < e1[0] - e0[0] < 1.1 * 2 * Be
