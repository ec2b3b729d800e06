"""Accuracy gate of the mixed form on a config-2-shaped grid, and CUDA-graph replay of the
tensor-core forms.

The mixed form (FP32 state and FFTs, split-TF32 tcgen05 gamma transforms, FP64 energy sums
and projections) is compared with the FP64 GPU path, which matches the FP64 oracle to
1e-10 on the state and 1e-8 on probabilities (test_gpu_parity.py). Gate: every
probability, total, reactant channel and product channel, within 1e-4 of the FP64 path
after 3000 iterations on the 256 x 192 x 96 grid of config 2 through the tile-major
tensor-core angular step (J = 2: three Coriolis-coupled helicity blocks, so the FP64
path finishes in about half a minute). The same run checks the probabilities against
the paper's bounds: 0 <= P <= 1 (to 1e-2) and the product channels (H2 + D only) not
above the total reaction probability.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mw3():
    from paper_2412_10167_gb300 import mw3 as m
    return m


C2_GRID_J2 = W.shrunk(W.C2, "h_dh_j2_256x192x96", J=[2], omega_max=2, steps=3000, nE=200)


def run(cfg, prec, n, tuning=None):
    pr = mw3().Propagator(cfg, precision=prec, tuning=tuning or {})
    pr.propagate(n)
    E, Pt, Pin = pr.probabilities()
    Pp = pr.product_probabilities()
    norm = pr.norm_trace()[-1]
    pr.close()
    return Pt, Pin, Pp, norm


def test_mixed_gate_on_config2_grid():
    cfg = C2_GRID_J2
    n = cfg["steps"]
    m_Pt, m_Pin, m_Pp, _ = run(cfg, "mixed", n)
    f_Pt, f_Pin, f_Pp, f_norm = run(cfg, "fp64", n)
    d_tot = np.max(np.abs(m_Pt - f_Pt))
    d_in = np.max(np.abs(m_Pin - f_Pin))
    d_pr = np.max(np.abs(m_Pp - f_Pp))
    print(f"max|dP| total {d_tot:.2e} reactant channels {d_in:.2e} product channels {d_pr:.2e}; "
          f"max P {f_Pt.max():.3f}, final norm {f_norm}")
    assert d_tot <= 1e-4 and d_in <= 1e-4 and d_pr <= 1e-4
    # the probabilities are meaningful, not only reproducible
    assert f_Pt.min() > -1e-2 and f_Pt.max() < 1 + 1e-2
    assert f_Pin.min() > -1e-12 and f_Pp.min() > -1e-12          # |S|^2 >= 0 by construction
    assert np.all(f_Pin.sum(axis=(1, 2, 3)) < 1 + 1e-2)
    assert np.all(f_Pp.sum(axis=(1, 2, 3)) <= f_Pt + 1e-2)


@pytest.mark.parametrize("name,cfg", [
    ("tile_major", W.shrunk(W.C2, "g96", NR=40, nr=36, ngamma=96, J=[4], omega_max=4, steps=64,
                            nE=16, kmin=10)),
    ("two_state", W.C3_SMALL),
])
def test_mixed_graph_replay_equals_eager_bitwise(name, cfg):
    """The tensor-core mixed path replayed from CUDA graphs (one graph per energy ring)
    gives the same bits as eager launches: state, probabilities and product channels."""
    runs = []
    for g in (0, 1):
        pr = mw3().Propagator(cfg, precision="mixed", tuning={"use_graph": g, "kb": 16})
        assert pr.get_tuning("use_tc") == 1
        pr.propagate(64)
        q, qp = pr.state()
        _, Pt, Pin = pr.probabilities()
        runs.append((q, qp, Pt, Pin, pr.product_probabilities()))
        pr.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,cfg", [
    ("ng96", W.shrunk(W.C2, "g96", NR=40, nr=36, ngamma=96, J=[4], omega_max=4, steps=40, nE=16,
                      kmin=10)),
    ("c2s", W.C2_SMALL),
])
def test_tma_tile_copies_equal_cp_async(name, cfg):
    """The tile-major angular step with its c, t and c_(k-1) tiles copied by the tensor memory
    accelerator (2-D tensor maps, ragged last tile filled with zeros) gives the same bits as
    the cp.async copies: the arithmetic is identical, only the copy engine differs."""
    runs = []
    for tma in (1, 0):
        pr = mw3().Propagator(cfg, precision="mixed", tuning={"tc_tma": tma, "tc_persist": 4})
        pr.propagate(40)
        runs.append(pr.state())
        pr.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
