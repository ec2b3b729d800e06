"""Pins for the surrogate's FP64 reference network and the J-shifting interpolation.

MLP: analytic gradients against central finite differences; the GELU derivative
against finite differences; one AdamW step against its closed form on a scalar.
J-shifting (Section 2.5): exact recovery of a shifted family, endpoint identities,
and the B fit on curves built with a known B.
"""
import numpy as np
import pytest

from oracle import jshift, mlp


def test_gelu_derivative_finite_difference():
    z = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-9)
    # limits: gelu(z) -> z for large z, -> 0 for very negative z
    assert abs(mlp.gelu(8.0) - 8.0) < 1e-12 and abs(mlp.gelu(-8.0)) < 1e-12


def test_mlp_gradients_finite_difference():
    params = mlp.init_params([4, 16, 16, 16, 1], seed=10167)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((32, 4))
    y = rng.standard_normal(32)
    loss, grads = mlp.loss_and_grads(params, X, y)
    h = 1e-6
    for li in range(len(params)):
        for pi in range(2):
            P = params[li][pi]
            flat = P.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = mlp.loss_and_grads(params, X, y)
                flat[idx] = old - h
                lm, _ = mlp.loss_and_grads(params, X, y)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][pi].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (li, pi, idx, fd, an)


def test_adamw_first_step_closed_form():
    """After one step, m/(1-b1) = g and v/(1-b2) = g^2, so the update is lr*sign(g) + decay."""
    W = np.array([[0.5, -2.0]])
    b = np.array([0.3])
    g = [[np.array([[0.1, -4.0]]), np.array([2.0])]]
    new = mlp.adamw_step([[W, b]], g, {}, {}, 1, lr=0.01, eps=0.0, wd=0.1)
    np.testing.assert_allclose(new[0][0], W - 0.01 * (np.sign(g[0][0]) + 0.1 * W), atol=1e-15)
    np.testing.assert_allclose(new[0][1], b - 0.01 * np.sign(g[0][1]), atol=1e-15)


def _family(E, B, Js):
    """P_J(E) = logistic((E - B J(J+1) - 0.5) / 0.05): an exactly J-shifted family."""
    return {J: 1.0 / (1.0 + np.exp(-(E - B * J * (J + 1) - 0.5) / 0.05)) for J in Js}


def test_jshift_recovers_exactly_shifted_family():
    E = np.linspace(0.0, 3.0, 3001)
    B = 0.002
    P = _family(E, B, [4, 6, 8])
    got = jshift.interpolate(E, P[4], P[8], 4, 8, 6, B)
    inner = (E > 0.3) & (E < 2.7)
    np.testing.assert_allclose(got[inner], P[6][inner], atol=1e-6)
    # endpoints reproduce the computed J
    np.testing.assert_allclose(jshift.interpolate(E, P[4], P[8], 4, 8, 4, B), P[4], atol=1e-15)
    np.testing.assert_allclose(jshift.interpolate(E, P[4], P[8], 4, 8, 8, B)[inner], P[8][inner],
                               atol=1e-12)
    # when the family is not exactly shifted (J-dependent width), the printed weight
    # order returns the shifted J2 curve at J = J1 instead of the computed J1 curve
    Q4 = 1.0 / (1.0 + np.exp(-(E - B * 20 - 0.5) / 0.05))
    Q8 = 1.0 / (1.0 + np.exp(-(E - B * 72 - 0.5) / 0.15))
    pr = jshift.interpolate(E, Q4, Q8, 4, 8, 4, B, printed=True)
    assert np.max(np.abs(pr - Q4)) > 0.1
    np.testing.assert_allclose(jshift.interpolate(E, Q4, Q8, 4, 8, 4, B), Q4, atol=1e-15)


def test_jshift_fit_recovers_B():
    E = np.linspace(0.0, 3.0, 3001)
    P = _family(E, 0.0017, [0, 10])
    B = jshift.fit_B(E, P[0], P[10], 0, 10, Bgrid=np.linspace(0, 0.004, 4001))
    assert abs(B - 0.0017) < 2e-6
