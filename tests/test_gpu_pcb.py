"""GPU parity of the products-coordinate-based start (mw3_init_packet_pcb; Section 2.4, the
first route, iprod = 1) against the oracle's pcb.py, through the C ABI.

  * the carried packet on the product grid: the device evaluates the packet at every node
    (Jacobi map, frame rotation with Wigner d^J in its Jacobi-polynomial form, Jacobian)
    and transforms it to each block's FBR; the oracle evaluates node by node with Wigner's
    explicit sum and projects. FP64: 1e-11 of the largest value (summation order and the
    two forms of d^J); mixed: the FP32 rounding of the FBR coefficients, 1e-6;
  * a propagation from it in FP64, probabilities to 1e-7 of their largest value (the
    grid's own channels are the product channels here; |a(E)|^2 is the closed form);
  * the packet's own arrangement ("A+BC") gives the ordinary initial packet up to the
    normalisation of g (closed form against the grid sum).
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import pcb
from oracle import propagate as P
from oracle.hamiltonian import GridHamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mw3():
    from paper_2412_10167_gb300 import mw3 as m
    return m


def heavy_cfg(J, j0, om0, arrangement, masses):
    """A heavy third atom puts the whole packet on a modest grid, with a large angle between
    the two body frames (every helicity populated)."""
    cfg = copy.deepcopy(W.C1)
    cfg["masses_u"] = masses
    cfg["J"], cfg["omega_max"] = [J], J
    cfg["grid"] = dict(NR=24, Rmin=0.6, Rmax=2.6, nr=60, rmin=2.5, rmax=9.5, ngamma=10)
    cfg["packet"] = dict(R0=6.0, Gamma=0.5, Ecol_eV=0.2, v0=0, j0=j0, omega0=om0, elec0=0)
    cfg["pcb"] = dict(arrangement=arrangement, rmin=0.6, rmax=2.6, nr=32)
    cfg["analysis"] = dict(cfg["analysis"], rstar=6.0, Rinf=2.0, kmin=0, nE=16, vmax=1, jmax=3)
    cfg["absorber"] = dict(RI=2.4, AR=0.5, nR=2, rI=8.5, Ar=0.3, nr=2)
    return cfg


def two_state_batch_cfg():
    """Several J in one batch (Omega blocks 0..min(J, 2)) and two diabatic states, the packet
    in the second one: the carry fills only that state's blocks, every J with its own d^J."""
    cfg = copy.deepcopy(W.C2_PCB_SMALL)
    cfg["J"], cfg["omega_max"], cfg["nelec"] = [0, 2, 3], 2, 2
    cfg["pes"] = dict(cfg["pes"], two_state=dict(W.TWO_STATE))
    cfg["packet"] = dict(cfg["packet"], omega0=0, elec0=1)
    cfg["grid"] = dict(cfg["grid"], ngamma=10)
    return cfg


CASES = {
    "h_dh_small": W.C2_PCB_SMALL,
    "two_states_J0_2_3": two_state_batch_cfg(),
    "heavyC_AC+B_J2": heavy_cfg(2, 2, 1, "AC+B", (2.0, 1.0, 300.0)),
    "heavyB_AB+C_J2": heavy_cfg(2, 2, 2, "AB+C", (2.0, 300.0, 1.0)),
    "generic_AC+B_J3": heavy_cfg(3, 1, 0, "AC+B", (2.0, 1.3, 30.0)),
}

_ORACLE = {}


def oracle_packet(name):
    if name not in _ORACLE:
        cfg = CASES[name]
        H = GridHamiltonian(cfg)
        _ORACLE[name] = pcb.pcb_packet(H, cfg["packet"], cfg["pcb"])[0]
    return _ORACLE[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pcb_packet_matches_oracle(name, prec):
    cfg = CASES[name]
    ref = oracle_packet(name)
    scale = np.max(np.abs(ref))
    assert scale > 1e-4                       # the packet is on the grid
    pr = mw3().Propagator(cfg, precision=prec)
    q, qp = pr.state()
    tol = 1e-11 if prec == "fp64" else 1e-6
    assert np.max(np.abs(q - ref)) <= tol * scale
    assert not np.any(qp)
    pr.close()


def test_pcb_propagation_matches_oracle():
    cfg = W.C2_PCB_SMALL
    N = cfg["steps"]
    ref = P.propagate(cfg, nsteps=N)
    pr = mw3().Propagator(cfg, precision="fp64")
    pr.propagate(N)
    q, _ = pr.state()
    assert np.linalg.norm(q - ref["q"]) / np.linalg.norm(ref["q"]) < 1e-10
    E, Pt, Pin = pr.probabilities()
    np.testing.assert_allclose(E, ref["Ecol"], rtol=1e-15)
    # the probabilities are still small this early: bound relative to their size
    assert np.max(np.abs(Pt - ref["P_total"])) <= 1e-7 * np.max(np.abs(ref["P_total"])) + 1e-15
    scale = max(np.max(np.abs(v)) for v in ref["P_inel"].values())
    assert scale > 0
    for (iJ, L, v, j), val in ref["P_inel"].items():
        assert np.max(np.abs(Pin[iJ, L, v, j] - val)) <= 1e-7 * scale + 1e-15, (iJ, L, v, j)
    pr.close()


def test_own_arrangement_equals_ordinary_packet():
    cfg = copy.deepcopy(W.C2_PCB_SMALL)
    g = cfg["grid"]
    cfg["pcb"] = dict(arrangement="A+BC", rmin=g["rmin"], rmax=g["rmax"], nr=g["nr"])
    cfg["packet"] = dict(cfg["packet"], Gamma=0.8, Ecol_eV=0.1)   # g^2 resolved by the grid
    a = mw3().Propagator(cfg, precision="fp64")
    qa, _ = a.state()
    plain = copy.deepcopy(cfg)
    del plain["pcb"]
    b = mw3().Propagator(plain, precision="fp64")
    qb, _ = b.state()
    assert np.max(np.abs(qa - qb)) <= 1e-7 * np.max(np.abs(qb))
    a.close()
    b.close()
