"""GPU parity of the photodissociation analysis (Sections 2.3.2 and 2.5): the per-step
autocorrelation C_k = <Psi(0)|Psi(k)> and the Chebyshev spectrum, through the C ABI,
against the FP64 oracle on damped propagations of a synthetic dipole packet.

Tolerances: FP64 path 1e-10 of C_0 (different summation orders only); mixed form (FP32
state, FP64 inner products) 2e-5 of C_0, the state's own rounding after a few hundred
iterations; the spectrum is a linear map of C and inherits the same bounds relative to
its largest value.
"""
import numpy as np
import pytest

import workloads as W
from oracle import photo
from oracle import propagate as P
from oracle.hamiltonian import GridHamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dipole(r, R, x):
    """Synthetic transition dipole (parallel type, proportional to cos gamma)."""
    return (1.0 + 0.3 * (r - 1.4)) * np.exp(-0.05 * (R - 5.0) ** 2) * x


def bound_guess(H):
    """A localised function standing in for the initial bound state."""
    n3, k3, m3 = np.meshgrid(H.x, H.r, H.R, indexing="ij")
    g = np.exp(-2.0 * (k3 - 1.45) ** 2 - 0.3 * (m3 - 5.0) ** 2)
    return g / np.linalg.norm(g)


def packet(H):
    q = np.zeros(H.shape)
    for b in range(H.nblk):    # the Omega = 0 block of every J
        if H.blocks[b][2] == 0 and H.blocks[b][3] == 0:
            q += photo.photo_packet(H, bound_guess(H), dipole, block=b)
    return q


@pytest.mark.parametrize("name", ["c2s", "c3s"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autocorrelation_and_spectrum_match_oracle(name, prec):
    from paper_2412_10167_gb300 import mw3
    cfg = W.SMALL[name]
    H = GridHamiltonian(cfg)
    q0 = packet(H)
    N = 200
    D = P.damping_grid(H, cfg["absorber"])[None, None]
    ref = photo.autocorrelation(H, q0, D, N)                       # [N, nJ]
    pr = mw3.Propagator(cfg, precision=prec, tuning={"kb": 32})
    pr.set_state(q0)
    pr.enable_autocorrelation()
    pr.propagate(N)
    C = pr.autocorrelation()
    assert C.shape == ref.shape
    scale = np.max(np.abs(ref[0]))
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.max(np.abs(C - ref)) <= tol * scale
    # spectrum at energies inside every J's spectral range (one call serves all J)
    lo = np.max(H.E0 - 0.9 * H.dE)
    hi = np.min(H.E0 + 0.9 * H.dE)
    E = np.linspace(lo, hi, 101)
    got = pr.photo_spectrum(E)
    for iJ in range(len(cfg["J"])):
        want = photo.chebyshev_spectrum(ref[:, iJ], E, H.E0[iJ], H.dE[iJ])
        assert np.max(np.abs(got[iJ] - want)) <= 10 * tol * np.max(np.abs(want))
    pr.close()


def test_autocorrelation_state_checks():
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    pr = mw3.Propagator(cfg, precision="fp64")
    pr.propagate(4)
    with pytest.raises(mw3.MW3Error) as e:      # the autocorrelation starts at k = 0
        pr.enable_autocorrelation()
    assert e.value.code == -7
    pr.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_time_packets_match_oracle(prec):
    """Time-domain packets (Eqs. wvf-chebyshev, chebyshev-expansion-constants) accumulated
    on the device against the oracle's Bessel sum of the same iterates, undamped: they also
    keep the norm of the initial packet (the reconstruction is exp(-iHt) Psi_0)."""
    import copy
    from paper_2412_10167_gb300 import mw3
    cfg = copy.deepcopy(W.C2_SMALL)
    cfg["absorber"] = dict(cfg["absorber"], AR=0.0, Ar=0.0)
    H = GridHamiltonian(cfg)
    q0 = H.project(W.random_unit_state(H.shape, 21))
    q0 /= np.linalg.norm(q0)                   # unit norm inside the blocks' span
    t = np.array([7.0, 35.0]) / H.dE[0]
    pr = mw3.Propagator(cfg, precision=prec)
    pr.set_state(q0)
    pr.enable_time_packets(t)
    pr.propagate(150)
    psi, K = pr.time_packets()
    assert 35 < K < 150
    D = np.ones((1, 1) + H.shape[2:])
    states = [q0] + [qn for _, _, qn in P.chebyshev_iterates(H, q0, D, K - 1)]
    tol = 1e-10 if prec == "fp64" else 2e-5
    for j, tj in enumerate(t):
        ref = P.time_domain_packet(states, tj, H.E0[0], H.dE[0])
        assert np.linalg.norm(psi[j] - ref) <= tol
        assert abs(np.linalg.norm(psi[j]) - 1.0) <= tol
    pr.close()
