"""Products-coordinate-based (PCB) start of a propagation. Test infrastructure only.

Section 2.4 gives two routes to state-to-state probabilities when one set of Jacobi
coordinates serves the whole reaction (iprod = 1 and 2 of inputprod). In the first (PCB),
the initial packet, which is a product of one-dimensional functions in the reactant
Jacobi coordinates (Section 2.3.1, Eqs. initial-collision-wvp and initial-gaussian), is
carried once onto a grid in the PRODUCT Jacobi coordinates; the propagation then runs in
the product arrangement, where the overlaps of Eq. (Chebyshev-products-overlaps) are
plain projections on the grid's own channels at R_inf. The paper prints no formulas for
the carrying step; the reading used here:

  * the propagation grid's own labels (A + BC: r = C - B, R from the BC centre of mass
    to A) describe the product arrangement; the packet's arrangement s is named in the
    same labels: "AC+B" (r_s = C - A, R_s from the AC centre of mass to B), "AB+C"
    (r_s = B - A, R_s from the AB centre of mass to C) or "A+BC" (the grid's own, a
    test case);
  * in its own body-fixed frame (z along R_s, r_s in the x-z half plane x > 0) the packet
    has one parity-adapted helicity block Omega0:
      Phi^s_(Omega0)(R_s, r_s, gamma_s) = g(R_s) chi_(v0 j0)(r_s) P-bar_(j0)^(Omega0)(cos gamma_s),
      g(R) = N exp(-(R - R0)^2 / (2 Gamma^2)) cos(k0 R),  k0 = sqrt(2 mu_s E_col),
    with N fixing int g^2 dR = 1 in closed form and chi the packet diatom's state on a sine
    DVR of its own (the third atom 100 bohr away on the diatom axis, as for the product
    states), evaluated as its sine interpolant (zero outside the DVR interval), so that
    int |Phi^s|^2 dR_s dr_s dcos(gamma_s) = 1;
  * at a grid node (R, r, gamma) the packet's coordinates follow from the Jacobi
    transformation (r_s, R_s) = M (r, R); the helicity components follow from the rotation
    rho between the two body frames (the grid's axes written in the packet frame) through
    the parity-adapted matrix T of the product analysis (products.helicity_matrix:
    Phi_(Omega) = sum T[Omega, Omega_s] Phi^s_(Omega_s)); the scalar wave function is
    Phi / (r R) in either frame (the Jacobi transformation has unit Jacobian), so
      Phi_Omega(R, r, gamma) = (r R / (r_s R_s)) T[Omega, Omega0] Phi^s_(Omega0)(R_s, r_s, gamma_s);
  * q = Phi sqrt(dR dr w_n) on every helicity block of each J (electronic state Lambda0),
    projected onto each block's FBR span;
  * the incoming amplitude (Eq. initial-flux-collisions) is the closed-form Gaussian
    integral a(E) = sqrt(mu_s / (2 pi K)) int exp(i K R) g(R) dR with
    K = sqrt(2 mu_s (E - e_(v0 j0))), e_(v0 j0) the packet diatom's level;
  * the energy grid is E = E_col + e_(v0 j0).

The channel analysis at R_inf and the flux cut at r* of the propagation are those of
propagate.py on the product grid; |S_c|^2 takes K_c and the reduced mass of the grid's
arrangement, a(E) the packet's.
"""
from __future__ import annotations

import numpy as np

from . import basis, pes
from . import products as PR

ARRANGEMENTS = ("A+BC", "AC+B", "AB+C")
R_FAR = 100.0   # bohr: R_s at which the packet diatom's states are computed


def packet_matrix(masses, arrangement: str) -> np.ndarray:
    """M with (r_s, R_s) = M (r, R): the packet's Jacobi vectors from the grid's."""
    if arrangement == "A+BC":
        return np.eye(2)
    return PR.product_matrix(masses, arrangement)


def packet_masses(masses, arrangement: str):
    """(mu_s, m_s): reduced masses of R_s and r_s."""
    if arrangement == "A+BC":
        mA, mB, mC = masses
        return mA * (mB + mC) / (mA + mB + mC), mB * mC / (mB + mC)
    return PR.product_masses(masses, arrangement)


def grid_to_packet(masses, arrangement, R, r, cosg):
    """Packet-frame (R_s, r_s, cos gamma_s) of the grid point (R, r, cos gamma) and rho,
    the grid's body-fixed axes written in the packet's body-fixed coordinates (columns)."""
    M = packet_matrix(masses, arrangement)
    sg = np.sqrt(max(1.0 - cosg * cosg, 0.0))
    r_vec = r * np.array([sg, 0.0, cosg])
    R_vec = R * np.array([0.0, 0.0, 1.0])
    rs_vec = M[0, 0] * r_vec + M[0, 1] * R_vec
    Rs_vec = M[1, 0] * r_vec + M[1, 1] * R_vec
    Rs, rs = np.linalg.norm(Rs_vec), np.linalg.norm(rs_vec)
    cosgs = np.dot(rs_vec, Rs_vec) / (rs * Rs)
    axes_s = PR.body_axes(Rs_vec, rs_vec)            # packet axes, grid coordinates
    return Rs, rs, cosgs, axes_s.T


def packet_diatom(H, src: dict, j: int, L: int, nv: int):
    """Lowest nv levels of the packet diatom on its sine DVR (src: rmin, rmax, nr):
    T(m_s) + min(j(j+1)/(2 m_s r_s^2), E_rot) + min(V_LL, V_cut), the third atom R_FAR
    away on the diatom axis. Vectors grid-normalised, largest component positive."""
    arr = src["arrangement"]
    _, m_s = packet_masses(H.masses, arr)
    rs, _ = basis.sine_dvr_nodes(src["rmin"], src["rmax"], src["nr"])
    Minv = np.linalg.inv(packet_matrix(H.masses, arr))
    V = np.zeros(len(rs))
    for a, x in enumerate(rs):
        rs_vec, Rs_vec = x * np.array([0.0, 0.0, 1.0]), R_FAR * np.array([0.0, 0.0, 1.0])
        r_vec = Minv[0, 0] * rs_vec + Minv[0, 1] * Rs_vec
        R_vec = Minv[1, 0] * rs_vec + Minv[1, 1] * Rs_vec
        r, R = np.linalg.norm(r_vec), np.linalg.norm(R_vec)
        V[a] = pes.potential_matrix(r, R, np.dot(r_vec, R_vec) / (r * R), H.masses, H.pes)[L, L]
    V = np.minimum(V, H.vcut)
    T = basis.radial_kinetic_matrix(src["rmin"], src["rmax"], src["nr"], m_s, H.tcut)
    cent = np.minimum(j * (j + 1.0) / (2.0 * m_s * rs ** 2), H.erot)
    e, U = np.linalg.eigh(T + np.diag(V + cent))
    U = U[:, :nv].copy()
    for v in range(nv):
        if U[np.argmax(np.abs(U[:, v])), v] < 0:
            U[:, v] = -U[:, v]
    return e[:nv], U


class PacketFunction:
    """The packet of the module header in its own frame, as a function."""

    def __init__(self, H, packet: dict, src: dict):
        from .units import EV
        self.arr = src["arrangement"]
        if self.arr not in ARRANGEMENTS:
            raise ValueError(f"arrangement must be one of {ARRANGEMENTS}")
        self.mu_s, self.m_s = packet_masses(H.masses, self.arr)
        self.v0, self.j0, self.om0, self.L0 = (packet["v0"], packet["j0"], packet["omega0"],
                                                packet["elec0"])
        e, U = packet_diatom(H, src, self.j0, self.L0, self.v0 + 1)
        self.e_v0j0 = e[self.v0]
        self.rlim = (src["rmin"], src["rmax"])
        self.nr = src["nr"]
        self.vec = U[:, self.v0]
        # sine-series coefficients: with vec_i = chi(r_i) sqrt(dr) and a = S vec,
        # chi(r) = sum_j s_j a_j phi_j(r) (basis.sine_interpolation_weights)
        s = np.ones(self.nr)
        s[-1] = 1.0 / np.sqrt(2.0)
        self.coef = s * (basis.dst2_matrix(self.nr) @ self.vec)
        self.R0, self.G = packet["R0"], packet["Gamma"]
        self.k0 = np.sqrt(2.0 * self.mu_s * packet["Ecol_eV"] * EV)
        self.N = 1.0 / np.sqrt(np.sqrt(np.pi) * self.G / 2.0 *
                               (1.0 + np.exp(-(self.k0 * self.G) ** 2) * np.cos(2 * self.k0 * self.R0)))

    def g(self, R):
        return self.N * np.exp(-(R - self.R0) ** 2 / (2.0 * self.G ** 2)) * np.cos(self.k0 * R)

    def chi(self, r):
        """Sine interpolant of the DVR vector (a function: int chi^2 dr = 1)."""
        if not (self.rlim[0] < r < self.rlim[1]):
            return 0.0
        ph, _ = basis.sine_basis_at(*self.rlim, self.nr, r)
        return float(np.dot(ph, self.coef))

    def value(self, Rs, rs, cosgs):
        """Phi^s_(Omega0)(R_s, r_s, gamma_s)."""
        P = basis.norm_assoc_legendre(self.j0, self.om0, np.array([cosgs]))[self.j0 - self.om0][0]
        return self.g(Rs) * self.chi(rs) * P


def grid_components(H, pf: PacketFunction, J: int, nom: int, R, r, cosg):
    """Phi_Omega(R, r, gamma), Omega = 0..nom-1, of the packet at one grid point (the
    formula of the module header before the quadrature factor)."""
    Rs, rs, cosgs, rho = grid_to_packet(H.masses, pf.arr, R, r, cosg)
    T = PR.helicity_matrix(J, nom, rho)
    return (r * R / (rs * Rs)) * T[:, pf.om0] * pf.value(Rs, rs, cosgs)


def pcb_packet(H, packet: dict, src: dict):
    """q_0 of the PCB start on the grid of H (the product arrangement) and its info:
    E_v0j0 (the packet diatom's level) and the packet function (for a(E))."""
    pf = PacketFunction(H, packet, src)
    for J in H.Js:
        if pf.om0 > H.omega_top(J):
            raise ValueError("Omega0 must be a helicity block of every J")
    q = np.zeros(H.shape)
    for iJ, J in enumerate(H.Js):
        nom = H.omega_top(J) + 1
        for n in range(H.ng):
            for k in range(H.nr):
                for m in range(H.NR):
                    comp = grid_components(H, pf, J, nom, H.R[m], H.r[k], H.x[n])
                    qf = np.sqrt(H.dR * H.dr * H.w[n])
                    for om in range(nom):
                        q[H.block_index[(iJ, om, pf.L0)], n, k, m] = comp[om] * qf
    return H.project(q), dict(E_v0j0=pf.e_v0j0, packet_function=pf, k0=pf.k0)


def incoming_amplitude(pf: PacketFunction, Ecol):
    """a(E) = sqrt(mu_s / (2 pi K)) int exp(i K R) g(R) dR, K = sqrt(2 mu_s E_col): with
    g = N exp(-(R-R0)^2/(2 Gamma^2)) (exp(i k0 R) + exp(-i k0 R)) / 2 the integral is
    N sqrt(2 pi) Gamma / 2 sum_(s = +-1) exp(i (K + s k0) R0 - Gamma^2 (K + s k0)^2 / 2)."""
    K = np.sqrt(2.0 * pf.mu_s * np.asarray(Ecol, dtype=float))
    integral = pf.N * np.sqrt(2.0 * np.pi) * pf.G / 2.0 * sum(
        np.exp(1j * (K + s * pf.k0) * pf.R0 - pf.G ** 2 * (K + s * pf.k0) ** 2 / 2.0)
        for s in (1.0, -1.0))
    return np.sqrt(pf.mu_s / (2.0 * np.pi * K)) * integral
