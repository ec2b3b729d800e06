"""Pins for the products-coordinate-based (PCB) start of oracle/pcb.py (Section 2.4, the
first of its two routes; Section 2.3.1 for the packet).

  * the packet's arrangement equal to the grid's own ("A+BC") reduces the carried packet
    to the library's ordinary initial packet: identity rotation, unit Jacobian, the
    diatom's sine interpolant at its own nodes;
  * the carried packet keeps its norm (the normalisations of g and of the diatom's sine
    interpolant; with the heavy third atom used there the Jacobian is close to 1, so the
    Jacobian is pinned by the next check);
  * the space-fixed wave function is the same whichever body frame expresses it:
    sum_Omega conj(D^J_(M Omega)(grid frame)) f_Omega / (r R) equals the packet-frame sum
    with the packet's own components, for every M, at random points and orientations, with
    general (complex) Wigner D matrices and unadapted components f_(+-Omega) built from the
    parity-adapted blocks and generic masses. This fixes the Euler flips, the parity
    adaptation (the sqrt(2) of Omega = 0 and the sign of the -Omega term) and the Jacobian
    independently of the helicity matrix; planted mistakes in each fail it. (The rotation
    and its transpose give the same carried packet here: for these in-plane rotations the
    two differ by a sign pattern that the parity-adapted state absorbs.)
  * the closed-form a(E) equals a direct quadrature of its defining integral.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import basis, pcb, products as PR, propagate as P
from oracle.hamiltonian import GridHamiltonian
from oracle.units import EV


def identity_cfg():
    cfg = W.shrunk(W.C1, "pcb_identity", NR=96, nr=24, ngamma=8, J=[1], omega_max=1)
    cfg["packet"] = dict(cfg["packet"], R0=9.0, Gamma=0.6, Ecol_eV=0.3, j0=1, omega0=1)
    g = cfg["grid"]
    cfg["pcb"] = dict(arrangement="A+BC", rmin=g["rmin"], rmax=g["rmax"], nr=g["nr"])
    return cfg


def heavy_cfg(J=2, j0=2, om0=1, arrangement="AC+B"):
    """Atom C heavy (300 u): the packet's R_s runs along the grid's r and its r_s along the
    grid's R, so a modest grid holds the whole packet."""
    cfg = copy.deepcopy(W.C1)
    cfg["masses_u"] = (2.0, 1.0, 300.0)
    cfg["J"], cfg["omega_max"] = [J], J
    cfg["grid"] = dict(NR=24, Rmin=0.6, Rmax=2.6, nr=56, rmin=2.5, rmax=9.5, ngamma=10)
    cfg["packet"] = dict(R0=6.0, Gamma=0.5, Ecol_eV=0.2, v0=0, j0=j0, omega0=om0, elec0=0)
    cfg["pcb"] = dict(arrangement=arrangement, rmin=0.6, rmax=2.6, nr=32)
    return cfg


def test_identity_arrangement_gives_the_initial_packet():
    cfg = identity_cfg()
    H = GridHamiltonian(cfg)
    q_pcb, info = pcb.pcb_packet(H, cfg["packet"], cfg["pcb"])
    q_ref, info_ref = P.initial_packet(H, cfg["packet"])
    # the two differ only by the normalisation of g (closed form against the grid sum,
    # equal to rounding when the grid resolves g^2: here 2 k0 is half the Nyquist number)
    assert abs(info["E_v0j0"] - info_ref["E_v0j0"]) < 1e-12
    np.testing.assert_allclose(q_pcb, q_ref, rtol=0, atol=1e-9 * np.max(np.abs(q_ref)))
    assert np.max(np.abs(q_ref)) > 1e-3


@pytest.mark.parametrize("arrangement", ["AC+B", "AB+C"])
def test_carried_packet_keeps_its_norm(arrangement):
    if arrangement == "AB+C":
        # B heavy instead: the AB+C arrangement's R_s then runs along the grid's r
        cfg = heavy_cfg(J=1, j0=1, om0=1, arrangement=arrangement)
        cfg["masses_u"] = (2.0, 300.0, 1.0)
    else:
        cfg = heavy_cfg(J=1, j0=1, om0=1, arrangement=arrangement)
    H = GridHamiltonian(cfg)
    q, _ = pcb.pcb_packet(H, cfg["packet"], cfg["pcb"])
    assert abs(np.sum(q * q) - 1.0) < 2e-3
    # every helicity of the grid frame is populated (the frames differ by a large angle)
    for om in range(2):
        assert np.sum(q[H.block_index[(0, om, 0)]] ** 2) > 0.05


def _D(J, mp, m, Rot):
    """General Wigner D^J_(m'm) of the rotation matrix Rot (columns: body axes in space)."""
    a, b, c = PR.euler_zyz(Rot)
    return np.exp(-1j * mp * a) * PR.wigner_d_element(J, mp, m, b) * np.exp(-1j * m * c)


def _unadapted(phi):
    """f_Omega, Omega = -J..J (index Omega + J), from the parity-adapted blocks phi[0..J]
    (p = (-1)^J): f_0 = sqrt(2) phi_0, f_Omega = phi_Omega, f_(-Omega) = (-1)^Omega phi_Omega."""
    J = len(phi) - 1
    f = np.zeros(2 * J + 1)
    f[J] = np.sqrt(2.0) * phi[0]
    for om in range(1, J + 1):
        f[J + om] = phi[om]
        f[J - om] = (-1.0) ** om * phi[om]
    return f


def _space_fixed(J, M, Rot, f, r, R):
    return sum(np.conj(_D(J, M, om, Rot)) * f[om + J] for om in range(-J, J + 1)) / (r * R)


def _random_rotation(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def _grid_point_inside_packet(rng, masses, arrangement, pf):
    """A grid point (R, r, cos gamma) whose packet-frame image lies where the packet lives
    (R_s within a width of R0, r_s near the diatom's equilibrium)."""
    Rs = pf.R0 + rng.uniform(-1.0, 1.0) * pf.G
    rs = rng.uniform(1.2, 1.7)
    cs = rng.uniform(-0.95, 0.95)
    Minv = np.linalg.inv(pcb.packet_matrix(masses, arrangement))
    rs_vec, Rs_vec = rs * np.array([np.sqrt(1 - cs * cs), 0.0, cs]), np.array([0.0, 0.0, Rs])
    r_vec = Minv[0, 0] * rs_vec + Minv[0, 1] * Rs_vec
    R_vec = Minv[1, 0] * rs_vec + Minv[1, 1] * Rs_vec
    r, R = np.linalg.norm(r_vec), np.linalg.norm(R_vec)
    return R, r, np.dot(r_vec, R_vec) / (r * R)


@pytest.mark.parametrize("arrangement", ["AC+B", "AB+C"])
@pytest.mark.parametrize("om0", [0, 1, 2])
def test_space_fixed_wave_function_is_frame_independent(arrangement, om0):
    J = 2
    cfg = heavy_cfg(J=J, j0=2, om0=om0, arrangement=arrangement)
    cfg["masses_u"] = (2.0, 1.3, 3.1)          # generic masses: a generic frame angle
    H = GridHamiltonian(cfg)
    pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    rng = W.rng(20240)
    M = pcb.packet_matrix(H.masses, arrangement)
    checked = 0
    for _ in range(12):
        R, r, cosg = _grid_point_inside_packet(rng, H.masses, arrangement, pf)
        phi = pcb.grid_components(H, pf, J, J + 1, R, r, cosg)
        # the same configuration in space: grid body axes Q, Jacobi vectors from them
        Q = _random_rotation(rng)
        sg = np.sqrt(1 - cosg * cosg)
        r_sf, R_sf = Q @ (r * np.array([sg, 0.0, cosg])), Q @ np.array([0.0, 0.0, R])
        rs_sf, Rs_sf = M[0, 0] * r_sf + M[0, 1] * R_sf, M[1, 0] * r_sf + M[1, 1] * R_sf
        rs, Rs = np.linalg.norm(rs_sf), np.linalg.norm(Rs_sf)
        Qs = PR.body_axes(Rs_sf, rs_sf)          # packet body axes in space
        phis = np.zeros(J + 1)
        phis[om0] = pf.value(Rs, rs, np.dot(rs_sf, Rs_sf) / (rs * Rs))
        f_grid, f_pack = _unadapted(phi), _unadapted(phis)
        if np.max(np.abs(f_pack)) < 1e-6:
            continue
        checked += 1
        for Mz in range(-J, J + 1):
            a = _space_fixed(J, Mz, Q, f_grid, r, R)
            b = _space_fixed(J, Mz, Qs, f_pack, rs, Rs)
            assert abs(a - b) <= 1e-10 * max(abs(b), np.max(np.abs(f_pack)) / (rs * Rs))
    assert checked >= 10


def _sqrt2_dropped(J, n_omega, rho):
    """helicity_matrix without the sqrt(2) of the Omega = 0 blocks (a plausible mistake)."""
    eul = PR.euler_zyz(rho)
    T = np.zeros((n_omega, n_omega))
    for op in range(n_omega):
        for om in range(n_omega):
            v = PR.wigner_D_element(J, om, op, eul)
            if om > 0:
                v += (-1.0) ** om * PR.wigner_D_element(J, -om, op, eul)
            T[op, om] = v
    return T


@pytest.mark.parametrize("mistake", ["inverted_jacobian", "sqrt2_dropped", "parity_sign"])
def test_space_fixed_check_catches_planted_mistakes(monkeypatch, mistake):
    """Plausible mistakes planted in the oracle each break the frame independence."""
    J, om0 = 2, 0
    cfg = heavy_cfg(J=J, j0=2, om0=om0, arrangement="AC+B")
    cfg["masses_u"] = (2.0, 1.3, 3.1)
    H = GridHamiltonian(cfg)
    pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    good_components, good_T = pcb.grid_components, PR.helicity_matrix
    if mistake == "inverted_jacobian":
        def bad(H_, pf_, J_, nom, R, r, cosg):
            Rs, rs, _, _ = pcb.grid_to_packet(H_.masses, pf_.arr, R, r, cosg)
            return good_components(H_, pf_, J_, nom, R, r, cosg) * ((rs * Rs) / (r * R)) ** 2
        monkeypatch.setattr(pcb, "grid_components", bad)
    elif mistake == "sqrt2_dropped":
        monkeypatch.setattr(PR, "helicity_matrix", _sqrt2_dropped)
    else:
        def flipped(J_, n_omega, rho):     # (-1)^Omega dropped from the -Omega term
            eul = PR.euler_zyz(rho)
            T = good_T(J_, n_omega, rho)
            for op in range(n_omega):
                for om in range(1, n_omega):
                    T[op, om] -= 2 * (-1.0) ** om * PR.wigner_D_element(J_, -om, op, eul) / (
                        np.sqrt(2.0) if op == 0 else 1.0)
            return T
        monkeypatch.setattr(PR, "helicity_matrix", flipped)
        om0 = 1
        cfg["packet"]["omega0"] = om0
        pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    rng = W.rng(20241)
    M = pcb.packet_matrix(H.masses, "AC+B")
    worst = 0.0
    for _ in range(8):
        R, r, cosg = _grid_point_inside_packet(rng, H.masses, "AC+B", pf)
        phi = pcb.grid_components(H, pf, J, J + 1, R, r, cosg)
        Q = _random_rotation(rng)
        sg = np.sqrt(1 - cosg * cosg)
        r_sf, R_sf = Q @ (r * np.array([sg, 0.0, cosg])), Q @ np.array([0.0, 0.0, R])
        rs_sf, Rs_sf = M[0, 0] * r_sf + M[0, 1] * R_sf, M[1, 0] * r_sf + M[1, 1] * R_sf
        rs, Rs = np.linalg.norm(rs_sf), np.linalg.norm(Rs_sf)
        phis = np.zeros(J + 1)
        phis[om0] = pf.value(Rs, rs, np.dot(rs_sf, Rs_sf) / (rs * Rs))
        Qs = PR.body_axes(Rs_sf, rs_sf)
        for Mz in range(-J, J + 1):
            a = _space_fixed(J, Mz, Q, _unadapted(phi), r, R)
            b = _space_fixed(J, Mz, Qs, _unadapted(phis), rs, Rs)
            worst = max(worst, abs(a - b) / max(abs(phis[om0]) / (rs * Rs), 1e-30))
    assert worst > 1e-2


def test_closed_form_incoming_amplitude():
    cfg = heavy_cfg(J=1, j0=1, om0=1)
    H = GridHamiltonian(cfg)
    pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    Ecol = np.linspace(0.05, 0.6, 7) * EV
    a = pcb.incoming_amplitude(pf, Ecol)
    R = np.linspace(pf.R0 - 12 * pf.G, pf.R0 + 12 * pf.G, 40001)
    dR = R[1] - R[0]
    g = pf.g(R)
    assert abs(np.sum(g * g) * dR - 1.0) < 1e-10          # N normalises g
    K = np.sqrt(2 * pf.mu_s * Ecol)
    quad = np.sqrt(pf.mu_s / (2 * np.pi * K)) * (np.exp(1j * K[:, None] * R[None]) @ g) * dR
    np.testing.assert_allclose(a, quad, rtol=1e-9, atol=1e-12)


def test_packet_diatom_is_the_grid_diatom_for_the_own_arrangement():
    cfg = identity_cfg()
    H = GridHamiltonian(cfg)
    e, U = pcb.packet_diatom(H, cfg["pcb"], 1, 0, 2)
    e_ref, U_ref = P.diatomic_states(H, 1, 0, 2)
    np.testing.assert_allclose(e, e_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(U, U_ref, rtol=0, atol=1e-10)
    # the interpolant returns the grid function at the DVR nodes
    pf = pcb.PacketFunction(H, cfg["packet"], cfg["pcb"])
    for k in (3, 10, 17):
        assert abs(pf.chi(H.r[k]) - U_ref[k, 0] / np.sqrt(H.dr)) < 1e-10
