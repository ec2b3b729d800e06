"""Host side of the products-coordinate-based start (mw3_init_packet_pcb) on a set-up-only
context (device = -1): the packet diatom's level and the closed-form |a(E)|^2 against the
oracle (Section 2.4, iprod = 1; Eq. initial-flux-collisions), and the argument checks."""
import copy
import ctypes

import numpy as np

import workloads as W
from oracle import pcb
from oracle import propagate as P
from oracle.hamiltonian import GridHamiltonian
from oracle.units import EV


def test_reference_energy_and_amplitude_match_oracle():
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_PCB_SMALL
    pr = mw3.Propagator(cfg, device=-1)
    H = GridHamiltonian(cfg)
    pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    assert abs(pr.reference_energy() - pf.e_v0j0) < 1e-12
    an = cfg["analysis"]
    Ecol = np.linspace(an["E_lo_eV"] * EV, an["E_hi_eV"] * EV, an["nE"])
    a2 = np.abs(pcb.incoming_amplitude(pf, Ecol)) ** 2
    np.testing.assert_allclose(pr.incoming_amplitude(), a2, rtol=1e-11)
    pr.close()


def test_own_arrangement_level_is_the_ordinary_packet_level():
    from paper_2412_10167_gb300 import mw3
    cfg = copy.deepcopy(W.C2_PCB_SMALL)
    g = cfg["grid"]
    cfg["pcb"] = dict(arrangement="A+BC", rmin=g["rmin"], rmax=g["rmax"], nr=g["nr"])
    pr = mw3.Propagator(cfg, device=-1)
    H = GridHamiltonian(cfg)
    _, info = P.initial_packet(H, cfg["packet"])
    assert abs(pr.reference_energy() - info["E_v0j0"]) < 1e-12
    pr.close()


def test_pcb_argument_checks():
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_PCB_SMALL
    pr = mw3.Propagator(cfg, device=-1, analysis=False)
    lib = mw3.lib
    pk = cfg["packet"]
    d = mw3.mw3_packet_desc(pk["R0"], pk["Gamma"], pk["Ecol_eV"] / mw3.HARTREE_EV, 0, 2, 2, 0)
    s = mw3.mw3_pcb_desc(1, 0.5, 4.5, 48)
    assert lib.mw3_init_packet_pcb(pr.ctx, ctypes.byref(d), ctypes.byref(s)) == -1   # MW3_ERR_BAD_ARG: Omega0 > J
    d.j0, d.omega0 = 0, 0
    for bad in (mw3.mw3_pcb_desc(3, 0.5, 4.5, 48), mw3.mw3_pcb_desc(1, 4.5, 0.5, 48),
                mw3.mw3_pcb_desc(1, 0.5, 4.5, 2)):
        assert lib.mw3_init_packet_pcb(pr.ctx, ctypes.byref(d), ctypes.byref(bad)) == -1
    assert lib.mw3_init_packet_pcb(pr.ctx, ctypes.byref(d), ctypes.byref(s)) == 0
    pr.close()
