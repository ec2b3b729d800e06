"""Host-side baselines of the surrogate pipeline (surrogate.py; no GPU): the J-shifting and
linear interpolations the trained networks are scored against, and the cumulative
probability of Eq. cumulative-probability.

J-shifting is checked against the oracle's own J-shifting (an independent restatement of
Eq. J-shifting-interpolation) and against an exactly J-shifted family, the linear baseline
against a family linear in J, and the cumulative sum against its definition written out."""
import numpy as np

from oracle import jshift
from paper_2412_10167_gb300 import surrogate as S


def _family(E, B, Js, nv=2, nj=3):
    """P[J][v][j](E): logistic steps at E = 0.5 + 0.1 v + 0.05 j + B J(J+1), exactly
    J-shifted with the rotational constant B; amplitudes differ per (v, j)."""
    out = np.zeros((len(Js), nv, nj, len(E)))
    for a, J in enumerate(Js):
        for v in range(nv):
            for j in range(nj):
                c = 0.5 + 0.1 * v + 0.05 * j + B * J * (J + 1)
                out[a, v, j] = (0.3 + 0.1 * v + 0.05 * j) / (1.0 + np.exp(-(E - c) / 0.05))
    return out


def test_jshift_baseline_recovers_shifted_family_and_matches_oracle():
    E = np.linspace(0.0, 3.0, 3001)
    Jtr = np.array([4, 8, 12])
    # B on the pipeline's search grid of the first interval (801 values over E range / dJ)
    dJ = 8 * 9 - 4 * 5
    B = np.linspace(0.0, (E[-1] - E[0]) / dJ, 801)[28]
    Ptr = _family(E, B, Jtr)
    Jte = [6, 10]
    got = S.jshift_baseline(E, Jtr, Ptr, Jte)
    ref = _family(E, B, Jte)
    inner = (E > 0.2) & (E < 2.2)
    assert np.max(np.abs(got[..., inner] - ref[..., inner])) < 2e-4
    # the oracle's interpolation with the same B on the bracketing pair, curve by curve
    for t, J in enumerate(Jte):
        k = 0 if J < 8 else 1
        Bk = B if k == 0 else jshift.fit_B(E, Ptr[k].sum(axis=(0, 1)), Ptr[k + 1].sum(axis=(0, 1)),
                                           Jtr[k], Jtr[k + 1],
                                           Bgrid=np.linspace(0.0, (E[-1] - E[0]) / (
                                               Jtr[k + 1] * (Jtr[k + 1] + 1) - Jtr[k] * (Jtr[k] + 1)), 801))
        for v in range(Ptr.shape[1]):
            for j in range(Ptr.shape[2]):
                o = jshift.interpolate(E, Ptr[k, v, j], Ptr[k + 1, v, j], Jtr[k], Jtr[k + 1], J, Bk)
                np.testing.assert_allclose(got[t, v, j], o, rtol=0, atol=1e-12)


def test_jshift_baseline_without_fit_is_linear_in_J():
    E = np.linspace(0.0, 3.0, 301)
    Jtr = np.array([0, 4, 8])
    Ptr = _family(E, 0.003, Jtr)
    np.testing.assert_allclose(S.jshift_baseline(E, Jtr, Ptr, [2, 5], fit=False),
                               S.linear_baseline(Jtr, Ptr, [2, 5]), rtol=0, atol=1e-15)


def test_linear_baseline_exact_for_linear_family():
    rng = np.random.default_rng(3)
    A, C = rng.uniform(0, 1, (2, 3, 40)), rng.uniform(-0.01, 0.01, (2, 3, 40))
    Jtr = np.array([0, 4, 8, 12])
    Ptr = np.stack([A + J * C for J in Jtr])
    Jte = [2, 6, 10, 12]
    got = S.linear_baseline(Jtr, Ptr, Jte)
    for t, J in enumerate(Jte):
        np.testing.assert_allclose(got[t], A + J * C, rtol=0, atol=1e-14)


def test_cumulative_probability_definition():
    rng = np.random.default_rng(4)
    Js = [0, 3, 7]
    P = rng.uniform(0, 1, (3, 2, 4, 11))
    want = np.zeros(11)
    for a, J in enumerate(Js):
        for v in range(2):
            for j in range(4):
                want += (2 * J + 1) * P[a, v, j]
    np.testing.assert_allclose(S.cumulative(Js, P), want, rtol=1e-14)
