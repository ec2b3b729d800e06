"""GPU parity of the non-orthogonal Lanczos bound states (Section 2.3.2) against the FP64
oracle, through the C ABI.

Tiny grid (full spectrum): after six times as many steps as the dimension the accepted
eigenvalues are the distinct eigenvalues of the dense Hamiltonian on the blocks' span, and
the first Lanczos coefficients equal the oracle's (the recursion is the same in exact
arithmetic; rounding differences grow only once orthogonality is lost). Config-2 copy
(J = 10, 11 coupled blocks): the lowest accepted eigenvalues after 300 steps equal the
oracle's, and the Ritz vector solves H x = E x.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lanczos
from oracle.hamiltonian import GridHamiltonian

from test_oracle_lanczos import span_spectrum, tiny_cfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gpu_tiny_cfg():
    """The oracle pin's tiny grid with an analysis surface and energy window inside it (the
    library sets up the analysis with every context; this grid's spectral range is narrow)."""
    cfg = tiny_cfg()
    cfg["analysis"] = dict(rstar=3.0, E_lo_eV=0.01, E_hi_eV=0.02, nE=4, Rinf=7.0, vmax=0, jmax=0,
                           kmin=0)
    return cfg


def test_lanczos_full_spectrum_tiny_grid():
    from paper_2412_10167_gb300 import mw3
    cfg = gpu_tiny_cfg()
    H = GridHamiltonian(cfg)
    exact = span_spectrum(H)
    distinct = exact[np.concatenate(([True], np.diff(exact) > 1e-9 * H.dE[0]))]
    v1 = H.project(W.random_state(H.shape, 4))
    m = 6 * len(exact)
    pr = mw3.Propagator(cfg, precision="fp64")
    a, b = pr.lanczos(v1, 40)
    to_fbr, _ = lanczos.fbr_maps(H)
    _, ra, rb = lanczos.bound_states(H, v1, 40, -np.inf, np.inf)
    np.testing.assert_allclose(a[:, 0], ra, rtol=0, atol=1e-12)
    np.testing.assert_allclose(b[:, 0], rb, rtol=0, atol=1e-12)
    E = pr.bound_states(v1, m)[0]
    assert len(E) == len(distinct)
    assert np.max(np.abs(np.sort(E) - distinct)) < 1e-8 * H.dE[0]
    pr.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lowest_bound_states_config2_copy(prec):
    from paper_2412_10167_gb300 import mw3
    cfg = W.C2_SMALL
    H = GridHamiltonian(cfg)
    v1 = H.project(W.random_state(H.shape, 8))
    m = 300
    ref, _, _ = lanczos.bound_states(H, v1, m, -np.inf, np.inf)
    pr = mw3.Propagator(cfg, precision=prec)
    E = pr.bound_states(v1, m)[0]
    tol = (1e-9 if prec == "fp64" else 2e-5) * H.dE[0]
    # FP32 recursion: its identification tolerance (1e-5 of the scaled range) can drop one
    # of a close pair (the 3rd and 4th levels here lie 1.3e-3 apart), so the lowest two
    nchk = 3 if prec == "fp64" else 2
    np.testing.assert_allclose(np.sort(E)[:nchk], np.sort(ref)[:nchk], rtol=0, atol=tol)
    if prec == "fp64":
        x = pr.bound_state_vector(v1, m, float(np.min(E)))
        res = np.linalg.norm(H.apply_H(x) - np.min(E) * x)
        assert abs(np.linalg.norm(x) - 1.0) < 1e-12
        assert res < 1e-7 * H.dE[0]
    pr.close()
