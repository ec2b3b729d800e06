"""Pins for the oracle's product-channel projector (Section 2.4, Eqs. final-states and
Chebyshev-products-overlaps, read as in oracle/products.py).

  * Wigner d: closed forms d^J_00 = P_J(cos b) and d^J_JJ = cos^(2J)(b/2), the J = 1
    table, orthogonality and the group law d(a) d(b) = d(a + b).
  * Jacobi maps: bond lengths from the product coordinates (built atom by atom)
    equal those from the reactant coordinates through the mapped point; the linear
    map has unit determinant.
  * Helicity transform: for any J, the rank-J tensor C^(J)_M of an in-plane vector
    (a J-state of parity (-1)^J) has body-fixed components C^(J)_Omega(v in that
    frame); the transform must carry the reactant-frame components into the
    product-frame ones. The spherical harmonics come from scipy, not from the
    Wigner formula.
  * Product states: Morse closed-form levels of the product diatom.
  * Projector: a synthetic product-channel function f(R') chi(r') P-bar(gamma') put
    on the reactant grid returns delta_(cc') f(R'_inf).
"""
import numpy as np
import pytest
from scipy.special import eval_legendre, lpmv

import workloads as W
from oracle import basis, products as PR
from oracle.hamiltonian import GridHamiltonian
from oracle.units import AMU, EV

MASSES = tuple(m * AMU for m in W.MASSES_H_DH)


def test_wigner_d_closed_forms():
    for J in range(0, 7):
        for b in (0.0, 0.3, 1.1, 2.0, np.pi):
            d = PR.wigner_d(J, b)
            assert abs(d[J, J] - eval_legendre(J, np.cos(b))) < 1e-12
            assert abs(d[2 * J, 2 * J] - np.cos(b / 2) ** (2 * J)) < 1e-12
            np.testing.assert_allclose(d @ d.T, np.eye(2 * J + 1), atol=1e-12)
    for a, b in ((0.4, 0.9), (1.3, -0.7)):
        for J in (1, 3, 5):
            np.testing.assert_allclose(PR.wigner_d(J, a) @ PR.wigner_d(J, b), PR.wigner_d(J, a + b),
                                       atol=1e-12)
    b = 0.8
    d1 = PR.wigner_d(1, b)            # rows m' = -1, 0, 1; columns m
    c, s = np.cos(b), np.sin(b)
    table = np.array([[(1 + c) / 2, s / np.sqrt(2), (1 - c) / 2],
                      [-s / np.sqrt(2), c, s / np.sqrt(2)],
                      [(1 - c) / 2, -s / np.sqrt(2), (1 + c) / 2]])
    np.testing.assert_allclose(d1, table, atol=1e-14)


@pytest.mark.parametrize("arr", ["AC+B", "AB+C"])
def test_jacobi_map_preserves_bond_lengths(arr):
    mA, mB, mC = MASSES
    M = PR.product_matrix(MASSES, arr)
    assert abs(abs(np.linalg.det(M)) - 1.0) < 1e-12
    rng = np.random.default_rng(3)
    for _ in range(20):
        Rp, rp, x = rng.uniform(2, 8), rng.uniform(0.5, 4), rng.uniform(-0.99, 0.99)
        # atoms from the product coordinates directly
        rpv = rp * np.array([np.sqrt(1 - x * x), 0, x])
        Rpv = np.array([0, 0, Rp])
        if arr == "AC+B":
            A = -mC / (mA + mC) * rpv
            C = mA / (mA + mC) * rpv
            B = Rpv
        else:
            A = -mB / (mA + mB) * rpv
            B = mA / (mA + mB) * rpv
            C = Rpv
        want = sorted([np.linalg.norm(A - B), np.linalg.norm(B - C), np.linalg.norm(A - C)])
        R, r, cosg, _ = PR.node_to_reactant(MASSES, arr, Rp, rp, x)
        from oracle import pes
        got = sorted(float(v) for v in pes.bond_distances(r, R, cosg, mA, mB, mC))
        np.testing.assert_allclose(got, want, rtol=1e-12)


def racah_components(J, v):
    """C^(J)_Omega(v) for Omega = 0..J of a vector v = (vx, 0, vz) in a body frame."""
    th = np.arctan2(abs(v[0]), v[2])
    phase = 1.0 if v[0] >= 0 else -1.0
    out = []
    for om in range(J + 1):
        norm = np.sqrt(np.exp(np.sum(np.log(np.arange(1, J - om + 1)))
                              - np.sum(np.log(np.arange(1, J + om + 1)))))
        out.append(norm * lpmv(om, J, np.cos(th)) * phase ** om)
    return np.array(out)


def adapted(C):
    s = np.ones(len(C))
    s[0] = np.sqrt(2.0)
    return C / s


@pytest.mark.parametrize("arr", ["AC+B", "AB+C"])
def test_helicity_transform_carries_tensor_components(arr):
    rng = np.random.default_rng(7)
    for _ in range(6):
        Rp, rp, x = rng.uniform(3, 8), rng.uniform(0.5, 4), rng.uniform(-0.95, 0.95)
        r_vec, R_vec = PR.product_to_reactant(MASSES, arr, Rp, rp, x)
        Rrc, rrc, cg, rho = PR.node_to_reactant(MASSES, arr, Rp, rp, x)
        axes_r = PR.body_axes(R_vec, r_vec)      # reactant axes in product coordinates
        rp_vec = rp * np.array([np.sqrt(1 - x * x), 0, x])
        for v in (R_vec, r_vec, rp_vec, np.array([0.0, 0.0, 1.0])):
            v = v / np.linalg.norm(v)
            v_react = axes_r.T @ v               # components in the reactant frame
            for J in range(0, 6):
                T = PR.helicity_matrix(J, J + 1, rho)
                a = adapted(racah_components(J, v_react))
                b = adapted(racah_components(J, v))
                np.testing.assert_allclose(T @ a, b, atol=1e-11, err_msg=f"J={J}")
                np.testing.assert_allclose(T @ T.T, np.eye(J + 1), atol=1e-11)


def test_lagrange4_exact_for_cubics():
    x0, dx, n = 0.5, 0.25, 40
    for x in (1.37, 3.01, 6.2):
        m0, w = PR.lagrange4(x0, dx, n, x)
        nodes = x0 + (m0 + np.arange(4)) * dx
        for p in (lambda t: 1 + 0 * t, lambda t: t, lambda t: t ** 2 - 3 * t, lambda t: t ** 3):
            assert abs(np.dot(w, p(nodes)) - p(x)) < 1e-11
        assert nodes[1] <= x < nodes[2]


def _prod():
    return dict(arrangement="AC+B", Rinf=6.0, rmin=0.5, rmax=4.5, nr=48, ngamma=16, vmax=2, jmax=4)


def test_product_states_morse_levels():
    cfg = W.shrunk(W.C1, "p", NR=16, nr=16, ngamma=4)
    cfg["caps"] = dict(vcut_eV=1e4, tcut_eV=1e4, erot_eV=5.0)   # no caps: pure Morse
    H = GridHamiltonian(cfg)
    prod = dict(_prod(), nr=160, rmin=0.3, rmax=8.0)
    pa = PR.ProductAnalysis(H, prod)
    e, _ = pa.states[(0, 0)]
    p = W.LEPS_H3
    D = p["D_eV"] * EV
    om = p["beta"] * np.sqrt(2 * D / pa.m_p)
    n = np.arange(len(e)) + 0.5
    np.testing.assert_allclose(e, om * n - (om * n) ** 2 / (4 * D), rtol=1e-9)


def test_projector_returns_synthetic_channel_amplitude():
    """f(R') chi_(v'j')(r') P-bar_(j')^(Omega')(cos gamma') in product coordinates, put on
    the reactant grid through the inverse maps, projects to delta_cc' f(R'_inf).

    The product quadrature is exact for these functions; what remains is the reactant
    grid's representation error (angular FBR truncation and 4-point interpolation),
    which falls as the grid is refined (max error 3.1e-2 at n_gamma = 40, 1.9e-3 /
    4.8e-3 for the two targets at n_gamma = 80). A wrong sign, index or Jacobian
    gives errors of order one."""
    cfg = W.shrunk(W.C2, "proj", NR=96, nr=96, ngamma=80, J=[1], omega_max=1,
                   Rmin=0.5, Rmax=12.0, rmin=0.5, rmax=12.0)
    H = GridHamiltonian(cfg)
    prod = _prod()
    pa = PR.ProductAnalysis(H, prod)
    chans = pa.channels(0)
    sig = 0.8
    f = lambda Rp: np.exp(-(Rp - prod["Rinf"]) ** 2 / (2 * sig ** 2))
    M = PR.product_matrix(H.masses, prod["arrangement"])
    # product coordinates of every reactant grid point (reactant body frame)
    n3, k3, m3 = np.meshgrid(np.arange(H.ng), np.arange(H.nr), np.arange(H.NR), indexing="ij")
    x, r, R = H.x[n3], H.r[k3], H.R[m3]
    r_vec = np.stack([r * np.sqrt(1 - x * x), 0 * r, r * x], axis=-1)
    R_vec = np.stack([0 * R, 0 * R, R], axis=-1)
    rp_vec = M[0, 0] * r_vec + M[0, 1] * R_vec
    Rp_vec = M[1, 0] * r_vec + M[1, 1] * R_vec
    rp, Rp = np.linalg.norm(rp_vec, axis=-1), np.linalg.norm(Rp_vec, axis=-1)
    live = (np.abs(Rp - prod["Rinf"]) < 5 * sig) & (rp > prod["rmin"]) & (rp < prod["rmax"])
    pts = np.argwhere(live)
    # rotation to the product frame at every live point (the transform is orthogonal)
    Ts = np.array([PR.helicity_matrix(1, 2, PR.body_axes(Rp_vec[tuple(p)], rp_vec[tuple(p)]))
                   for p in pts])
    cgp = np.array([np.dot(rp_vec[tuple(p)], Rp_vec[tuple(p)]) for p in pts]) / (rp[live] * Rp[live])
    # product diatomic state as a function: its sine-DVR interpolant
    Lp = prod["rmax"] - prod["rmin"]
    kk = np.arange(1, prod["nr"] + 1) * np.pi / Lp
    S = basis.dst2_matrix(prod["nr"])
    sc = np.ones(prod["nr"])
    sc[-1] = 1 / np.sqrt(2)
    phi_j = np.sqrt(2 / Lp) * np.sin(np.outer(rp[live] - prod["rmin"], kk))     # [pts, j]
    jac = (r * R)[live] / (rp * Rp)[live]
    for target in [(0, 0, 1, 0), (0, 1, 2, 1)]:
        L0, v0, j0, op0 = target
        chif = phi_j @ (sc * (S @ pa.states[(j0, L0)][1][:, v0]))
        Pj = basis.norm_assoc_legendre(j0, op0, cgp)[j0 - op0]
        amp = f(Rp[live]) * chif * Pj
        q = np.zeros(H.shape)
        for om in range(2):
            # Phi = T^T Phi', Phi' nonzero in helicity op0 only
            vals = jac * Ts[:, op0, om] * amp
            b = H.block_index[(0, om, 0)]
            q[b][live] = vals * np.sqrt(H.dR * H.dr * H.w[pts[:, 0]])
        q = H.project(q)
        C = pa.overlaps(q)[0]
        want = np.array([f(prod["Rinf"]) if (c[0], c[1], c[2], c[3]) == target else 0.0 for c in chans])
        assert np.max(np.abs(C - want)) < 6e-3, (target, np.max(np.abs(C - want)))
