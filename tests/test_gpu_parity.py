"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

States passed to the library are values on the grid; the library holds each block
in the span of its angular functions (j = Omega..ngamma-1), so random test vectors
are first projected onto that span.

Tolerances (written from the arithmetic):
  * FP64 path: the operator agrees with the oracle to 1e-12 of max|H_s q| (different
    summation orders only); after N iterations q_N agrees to 1e-10 relative (l2),
    and probabilities to 1e-8 absolute.
  * Mixed path (FP32 state): one H_s application to 2e-6 of max|H_s q| (FP32
    rounding of the FFT and gamma transforms, sum over ~log N + n_gamma terms).
"""
import copy
import os
import tempfile

import numpy as np
import pytest

import workloads as W
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


_ORACLE = {}


def oracle_run(name, cfg, nsteps):
    key = (name, nsteps)
    if key not in _ORACLE:
        _ORACLE[key] = P.propagate(cfg, nsteps=nsteps)
    return _ORACLE[key]


APPLY_CASES = dict(W.SMALL, odd=W.C_ODD)


@pytest.mark.parametrize("name", list(APPLY_CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_apply_hs_matches_oracle(name, prec):
    cfg = APPLY_CASES[name]
    pr = mw3().Propagator(cfg, precision=prec)
    H = GridHamiltonian(cfg)
    # the state of a block lies in the span of its angular functions
    q = H.project(W.random_state(H.shape, 2412))
    ref = H.apply_Hs(q)
    got = pr.apply_hs(q)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    pr.close()


# Line lengths 32 R for the warp-register FFT kinetic kernels (R up to 8 in FP64,
# up to 16 in the mixed path); NR = 72 leaves a ragged column tile in the r kernel.
WARP_CASES = {
    "w64x96": W.shrunk(W.C2, "w64x96", NR=64, nr=96, ngamma=8, J=[2], omega_max=2, nE=8),
    "w128x192": W.shrunk(W.C2, "w128x192", NR=128, nr=192, ngamma=6, J=[1], omega_max=1, nE=8),
    "w256x32": W.shrunk(W.C2, "w256x32", NR=256, nr=32, ngamma=6, J=[1], omega_max=1, nE=8),
    "w72x256": W.shrunk(W.C2, "w72x256", NR=72, nr=256, ngamma=5, J=[0], omega_max=0, nE=8),
    "w384x512": W.shrunk(W.C2, "w384x512", NR=384, nr=512, ngamma=4, J=[1], omega_max=1, nE=8),
    # half-warp form (FP32, N = 128, 192, 256): a partial last 32-row block (nrows = 432),
    # a column count that is not a multiple of 4 (scalar tile loads), dead rows of Omega > 0
    "h256x36": W.shrunk(W.C2, "h256x36", NR=256, nr=36, ngamma=6, J=[1], omega_max=1, nE=8),
    "h30x128": W.shrunk(W.C2, "h30x128", NR=30, nr=128, ngamma=6, J=[1], omega_max=1, nE=8),
    "h192x256": W.shrunk(W.C2, "h192x256", NR=192, nr=256, ngamma=5, J=[2], omega_max=2, nE=8),
}


@pytest.mark.parametrize("name", list(WARP_CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("warp", [3, 2, 1, 0])
def test_warp_fft_kinetic_matches_oracle(name, prec, warp):
    cfg = WARP_CASES[name]
    pr = mw3().Propagator(cfg, precision=prec, tuning={"kin_warp": warp, "kin_fused": 0})
    H = GridHamiltonian(cfg)
    q = H.project(W.random_state(H.shape, 77))
    ref = H.apply_Hs(q)
    got = pr.apply_hs(q)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    pr.close()


@pytest.mark.parametrize("name", list(W.SMALL))
def test_propagation_fp64_parity(name):
    cfg = W.SMALL[name]
    N = cfg["steps"]
    ref = oracle_run(name, cfg, N)
    pr = mw3().Propagator(cfg, precision="fp64")
    pr.propagate(N)
    q, qp = pr.state()
    rel = np.linalg.norm(q - ref["q"]) / np.linalg.norm(ref["q"])
    relp = np.linalg.norm(qp - ref["q_prev"]) / np.linalg.norm(ref["q_prev"])
    assert rel < 1e-10 and relp < 1e-10, (rel, relp)
    E, Pt, Pin = pr.probabilities()
    np.testing.assert_allclose(E, ref["Ecol"], rtol=1e-15)
    assert np.max(np.abs(Pt - ref["P_total"])) < 1e-8
    # channel probabilities, summed over Omega, per (J, Lambda, v, j)
    for (iJ, L, v, j), val in ref["P_inel"].items():
        assert np.max(np.abs(Pin[iJ, L, v, j] - val)) < 1e-8, (iJ, L, v, j)
    # norm trace ||q_k||^2, k = 1..N
    tr = pr.norm_trace()
    bj = ref["H"].block_J_index()
    assert tr.shape == (N, len(cfg["J"]))
    np.testing.assert_allclose(tr.sum(axis=1), ref["norms"][1:], rtol=1e-10)
    pr.close()


@pytest.mark.parametrize("name", ["c2s", "c3s", "c4s"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("gather", [1, 0])
def test_product_channels_match_oracle(name, prec, gather):
    """Product-channel probabilities (Eq. S-matrix-from-chebyshev) from a random first
    iterate that already overlaps the product surface: FP64 to 1e-9 of the largest
    value (summation order only), the mixed path to 1e-3 of it (FP32 state and sums
    within a flush block). Both forms of the node sums: stencil columns gathered
    plane-major first (gather 1) and stencils read from the state (gather 0)."""
    cfg = W.SMALL[name]
    H = GridHamiltonian(cfg)
    q0 = H.project(W.random_unit_state(H.shape, 31))
    N = 12
    ref = P.propagate(cfg, nsteps=N, H=H, q0=q0)
    pr = mw3().Propagator(cfg, precision=prec, tuning={"prod_gather": gather})
    assert pr.get_tuning("prod_gather") == gather
    pr.set_state(q0)
    pr.propagate(N)
    got = pr.product_probabilities()
    scale = max(np.max(np.abs(v)) for v in ref["P_prod"].values())
    assert scale > 0
    tol = 1e-9 if prec == "fp64" else 1e-3
    for (iJ, L, v, j), val in ref["P_prod"].items():
        assert np.max(np.abs(got[iJ, L, v, j] - val)) <= tol * scale, (iJ, L, v, j)
    pr.close()


def test_mixed_probabilities_close_to_fp64():
    """Mixed path on config 1: |dP| stays within 1e-4 of the FP64 oracle."""
    cfg = W.C1
    ref = oracle_run("c1", cfg, cfg["steps"])
    pr = mw3().Propagator(cfg, precision="mixed")
    pr.propagate(cfg["steps"])
    _, Pt, Pin = pr.probabilities()
    dP = np.max(np.abs(Pt - ref["P_total"]))
    assert dP < 1e-4, dP
    q, _ = pr.state()
    assert np.linalg.norm(q - ref["q"]) / np.linalg.norm(ref["q"]) < 1e-3
    pr.close()


def test_graph_replay_equals_eager_bitwise():
    cfg = W.C2_SMALL
    runs = []
    for g in (0, 1):
        pr = mw3().Propagator(cfg, precision="fp64", tuning={"use_graph": g, "kb": 16})
        pr.propagate(100)
        q, qp = pr.state()
        runs.append((q, qp, pr.probabilities()[1]))
        pr.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)


def test_batched_J_equals_single_J_bitwise():
    """A batch of uneven J stacks gives the same bits as each J run alone."""
    cfg = W.C3_SMALL
    pr = mw3().Propagator(cfg, precision="fp64")
    pr.propagate(60)
    qb, _ = pr.state()
    _, Pb, _ = pr.probabilities()
    H = GridHamiltonian(cfg)
    bj = H.block_J_index()
    pr.close()
    for iJ, J in enumerate(cfg["J"]):
        c1 = copy.deepcopy(cfg)
        c1["J"] = [J]
        p1 = mw3().Propagator(c1, precision="fp64")
        p1.propagate(60)
        q1, _ = p1.state()
        _, P1, _ = p1.probabilities()
        assert np.array_equal(q1, qb[bj == iJ])
        assert np.array_equal(P1[0], Pb[iJ])
        p1.close()


def test_deterministic_and_resumable():
    cfg = W.C2_SMALL
    a = mw3().Propagator(cfg, precision="fp64")
    a.propagate(70)
    b = mw3().Propagator(cfg, precision="fp64")
    b.propagate(25)
    b.propagate(45)
    qa, _ = a.state()
    qb, _ = b.state()
    assert np.array_equal(qa, qb)
    assert a.iteration == b.iteration == 70
    # the energy sums match to rounding (different flush grouping)
    np.testing.assert_allclose(a.probabilities()[1], b.probabilities()[1], rtol=0, atol=1e-12)
    a.close()
    b.close()


def test_checkpoint_roundtrip():
    cfg = W.C2_SMALL
    a = mw3().Propagator(cfg, precision="fp64")
    a.propagate(40)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.checkpoint_save(path)
        a.propagate(40)
        b = mw3().Propagator(cfg, precision="fp64")
        b.checkpoint_load(path)
        assert b.iteration == 40
        b.propagate(40)
    qa, _ = a.state()
    qb, _ = b.state()
    assert np.array_equal(qa, qb)
    np.testing.assert_allclose(a.probabilities()[1], b.probabilities()[1], atol=1e-13)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("pending", [1, 5, 8, 13])
def test_pending_ring_read_equals_flushed(prec, pending):
    """A propagation that stops inside an energy ring leaves the slots pending: a probability
    read adds up to eight (FP64) or sixteen (mixed) of them on the fly and flushes more.
    Either way the probabilities (total, reactant channels, product channels) equal those
    read after an explicit flush (a checkpoint save flushes); continuing afterwards gives the
    same state as one uninterrupted call.

    Tolerances. The total: the on-the-fly read must reproduce the pending slots' own
    contribution (the change from the last flushed read) to 1e-9 of it in FP64 and to 1e-4 in
    the mixed form, whose flush multiplies on the tensor cores (split-TF32 products summed in
    FP32 inside the MMA) while the read sums the FP32 products of the same values in FP32. The
    channel sums are FP64 in both forms (FP64 ring, phases and GEMM), so both use FP64 bounds."""
    cfg = W.C2_SMALL
    kb = 16
    n0 = 12 * kb
    drel, rel = (1e-9, 1e-10) if prec == "fp64" else (1e-4, 1e-6)

    a = mw3().Propagator(cfg, precision=prec, tuning={"kb": kb})
    a.propagate(n0)
    _, P0, _ = a.probabilities()               # ring empty: the flushed sums alone
    a.propagate(pending)
    E, Pt, Pin = a.probabilities()
    Pp = a.product_probabilities()
    E2, Pt2, Pin2 = a.probabilities()          # a second read sees the same sums
    assert np.array_equal(Pt, Pt2) and np.array_equal(Pin, Pin2)
    with tempfile.TemporaryDirectory() as d:
        a.checkpoint_save(os.path.join(d, "ck.bin"))
    _, Ft, Fin = a.probabilities()
    Fp = a.product_probabilities()
    step = np.max(np.abs(Ft - P0))             # what the pending slots add
    assert step > 0
    assert np.max(np.abs(Pt - Ft)) <= drel * step + rel * np.max(np.abs(Ft)) + 1e-15
    for x, y in ((Pin, Fin), (Pp, Fp)):
        assert np.max(np.abs(x - y)) <= 1e-9 * np.max(np.abs(y)) + 1e-14
    a.propagate(kb - pending + 3)
    b = mw3().Propagator(cfg, precision=prec, tuning={"kb": kb})
    b.propagate(n0 + kb + 3)
    assert np.array_equal(a.state()[0], b.state()[0])
    Fa, Fb = a.probabilities()[1], b.probabilities()[1]
    assert np.max(np.abs(Fa - Fb)) <= (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(Fb)) + 1e-15
    a.close()
    b.close()


def test_full_size_config2_operator_and_first_steps():
    """Config 2 at full size (256 x 192 x 96, 11 blocks): H_s on a seeded vector in
    both precisions, and the first two damped iterations plus their flux sums in FP64."""
    cfg = copy.deepcopy(W.C2)
    H = GridHamiltonian(cfg)
    q = H.project(W.random_state(H.shape, 2412))
    ref = H.apply_Hs(q)
    scale = np.max(np.abs(ref))
    for prec, tol in (("fp64", 1e-12), ("mixed", 2e-6)):
        pr = mw3().Propagator(cfg, precision=prec)
        got = pr.apply_hs(q)
        assert np.max(np.abs(got - ref)) <= tol * scale, prec
        pr.close()
    del q, ref
    cfg["analysis"]["vmax"] = 1
    cfg["analysis"]["jmax"] = 3
    cfg["analysis"]["nE"] = 20
    ref = P.propagate(cfg, nsteps=2, H=H)
    pr = mw3().Propagator(cfg, precision="fp64")
    pr.propagate(2)
    qg, qpg = pr.state()
    assert np.linalg.norm(qg - ref["q"]) / np.linalg.norm(ref["q"]) < 1e-12
    _, Pt, _ = pr.probabilities()
    assert np.max(np.abs(Pt - ref["P_total"])) < 1e-8 * max(1.0, np.max(np.abs(ref["P_total"])))
    pr.close()


def test_divergence_guard():
    """A state pair inconsistent with the recursion (q_(k-1) = -3 q_k) makes the norm
    jump far above ||q_0||^2: the library returns MW3_ERR_DIVERGED."""
    cfg = W.C2_SMALL
    pr = mw3().Propagator(cfg, precision="fp64")
    pr.propagate(10)
    q, _ = pr.state()
    pr.set_state(q, -3.0 * q)
    with pytest.raises(mw3().MW3Error) as e:
        pr.propagate(40)
    assert e.value.code == -4
    pr.close()


# n_gamma = 96 (kh = 48, the largest resident parity-split size, with a ragged last tile);
# n_gamma beyond the resident parity-split form (streamed operand matrices, kh = 64 and 96)
TC_CASES = dict(W.SMALL,
                ng96=W.shrunk(W.C2, "ng96", NR=40, nr=36, ngamma=96, J=[4], omega_max=4,
                              steps=40, nE=16, kmin=10),
                ng100=W.shrunk(W.C2, "ng100", NR=40, nr=36, ngamma=100, J=[2], omega_max=2,
                               steps=40, nE=16, kmin=10),
                ng180=W.shrunk(W.C4, "ng180", NR=24, nr=20, ngamma=180, J=[1], omega_max=1,
                               steps=40, nE=16, kmin=10))


@pytest.mark.parametrize("name", list(TC_CASES))
def test_tensor_core_step_matches_cuda_core_step(name):
    """Mixed precision: the fused tcgen05 angular step (split-TF32) in each of its forms —
    tile-major with on-chip Coriolis neighbours, persistent parity-split (resident or
    streamed operands), persistent tensor-memory-operand, one tile per CTA — agrees with
    the CUDA-core FP32 step to FP32 rounding after 40 iterations, and with the oracle."""
    cfg = TC_CASES[name]
    qs = []
    for tc, persist in ((1, 4), (1, 2), (1, 1), (1, 0), (0, 0)):
        pr = mw3().Propagator(cfg, precision="mixed", tuning={"use_tc": tc, "tc_persist": persist})
        assert pr.get_tuning("use_tc") == tc
        pr.propagate(40)
        qs.append(pr.state()[0])
        pr.close()
    ref = oracle_run(name, cfg, 40)
    for q in qs[:-1]:
        rel = np.linalg.norm(q - qs[-1]) / np.linalg.norm(qs[-1])
        assert rel < 2e-5, rel
        rel_o = np.linalg.norm(q - ref["q"]) / np.linalg.norm(ref["q"])
        assert rel_o < 2e-5, rel_o


def test_tensor_core_flush_matches_cuda_core_flush():
    """The energy-sum flush on the tensor cores (split-TF32, FP64 accumulators) gives the
    probabilities of the FP32 CUDA-core flush to FP32 rounding (and a partial last ring)."""
    cfg = W.C2_SMALL
    H = GridHamiltonian(cfg)
    q0 = H.project(W.random_unit_state(H.shape, 5))   # every sum generic and nonzero
    out = []
    for ftc in (1, 0):
        pr = mw3().Propagator(cfg, precision="mixed", tuning={"flush_tc": ftc, "kb": 32})
        pr.set_state(q0)
        pr.propagate(100)
        E, Pt, Pin = pr.probabilities()
        out.append((Pt, Pin, pr.product_probabilities()))
        pr.close()
    for a, b in zip(out[0], out[1]):
        assert np.max(np.abs(a - b)) <= 1e-5 * max(np.max(np.abs(b)), 1e-30)


def test_autotuner_picks_and_caches(tmp_path):
    """The tuner sweeps launch shapes with the library's own event timers, caches the
    winners per shape, and a tuned context reproduces the default results to FP32
    rounding (launch shapes change only the order of independent work)."""
    from paper_2412_10167_gb300 import tune
    cfg = W.C2_SMALL
    path = str(tmp_path / "tune.json")
    best = tune.tune(cfg, "mixed", steps=4, cache_path=path)
    assert set(best) == set(tune.SWEEP)
    assert tune.tune(cfg, "mixed", cache_path=path) == best          # cached
    a = mw3().Propagator(cfg, precision="mixed", tuning=best)
    b = mw3().Propagator(cfg, precision="mixed")
    a.propagate(40)
    b.propagate(40)
    qa, qb = a.state()[0], b.state()[0]
    assert np.linalg.norm(qa - qb) / np.linalg.norm(qb) < 1e-5
