"""The fused radial kinetic kernel (both radial terms, the flux cut and the R_inf column in
one launch of thread-block clusters, one (block, i) plane per cluster) against the FP64
oracle's H_s, and bitwise against the two separate half-warp kernels it replaces: the same
pair transforms on the same values, added in the same order, so the propagated state, the
probabilities and the product channels agree to the bit.

Grids: the config-2 line lengths (NR = 256, nr = 192) with every cluster size, the config-3
ones (192 x 128), and 128 x 192 / 256 x 128 (other table pairs); three helicity blocks, so
planes of the Omega > 0 blocks are dead and skipped by whole clusters.
"""
import numpy as np
import pytest

import workloads as W
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


CASES = {
    "r256x192": (W.shrunk(W.C2, "r256x192", NR=256, nr=192, ngamma=6, J=[2], omega_max=2, nE=8),
                 [1, 2, 4, 8]),
    "r192x128": (W.shrunk(W.C3, "r192x128", NR=192, nr=128, ngamma=6, J=[1], omega_max=1, nE=8),
                 [1, 2]),
    "r128x192": (W.shrunk(W.C2, "r128x192", NR=128, nr=192, ngamma=6, J=[1], omega_max=1, nE=8),
                 [2, 4]),
    "r256x128": (W.shrunk(W.C2, "r256x128", NR=256, nr=128, ngamma=6, J=[2], omega_max=2, nE=8),
                 [2, 8]),
}
PARAMS = [(name, cs) for name, (_, css) in CASES.items() for cs in css]


@pytest.mark.parametrize("name,cs", PARAMS)
def test_fused_radial_matches_oracle(name, cs):
    cfg = CASES[name][0]
    pr = mw3().Propagator(cfg, precision="mixed", tuning={"kin_fused": cs})
    H = GridHamiltonian(cfg)
    q = H.project(W.random_state(H.shape, 78))
    ref = H.apply_Hs(q)
    got = pr.apply_hs(q)
    assert pr.get_tuning("kin_fused") == cs
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    pr.close()


def _run(cfg, tuning, n):
    pr = mw3().Propagator(cfg, precision="mixed", tuning=tuning)
    pr.kernel_times(enable=True)
    pr.propagate(n)
    kt = pr.kernel_times()
    q, qp = pr.state()
    _, Pt, Pin = pr.probabilities()
    Pp = pr.product_probabilities()
    pr.close()
    return (q, qp, Pt, Pin, Pp), kt


@pytest.mark.parametrize("name,cs", PARAMS)
def test_fused_radial_equals_separate_kernels_bitwise(name, cs):
    cfg = CASES[name][0]
    n = 40
    sep, kt0 = _run(cfg, {"kin_fused": 0, "kb": 16}, n)
    fus, kt1 = _run(cfg, {"kin_fused": cs, "kb": 16}, n)
    # the fused kernel ran in place of the two separate ones
    assert kt1["kinetic_radial"][1] == n and kt1["kinetic_rows"][1] == 0
    assert kt0["kinetic_radial"][1] == 0 and kt0["kinetic_rows"][1] == n
    for a, b in zip(sep, fus):
        assert np.array_equal(a, b)
