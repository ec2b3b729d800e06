"""State-resolved product channels at R' = R'_inf. Test infrastructure only.

Section 2.4, Eqs. (final-states), (Chebyshev-products-overlaps) and
(S-matrix-from-chebyshev): the overlap of the wave packet with the product states
W Y_(j' Omega')(gamma', 0) chi_(v'j')(r') / (r' R') on the surface R' = R'_inf, for
a wave packet held in reactant Jacobi coordinates (the reactant-coordinates-based
route of that section). The paper cites the sequential transformation of its
reference for this step and prints no algorithm; the reading used here is:

  * products: arrangement "AC+B" (r' = C - A, R' from the AC centre of mass to B)
    or "AB+C" (r' = B - A, R' from the AB centre of mass to C);
  * a product quadrature on R' = R'_inf: the midpoint sine-DVR nodes r'_a of the
    product diatomic grid (weight dr') times n Gauss-Legendre nodes cos(gamma'_l)
    (weights w_l);
  * every node is mapped to reactant Jacobi coordinates (R, r, gamma) and to the
    rotation rho that takes the reactant body-fixed axes (z along R, r in the
    x-z half plane x > 0) to the product ones (z along R', r' in x > 0);
  * the reduced reactant function at the node is
      Phi^Omega(R, r, gamma) = sum_(a,b) L_a(R) L_b(r) sum_j c^Omega_j(r_b, R_a) P-bar_j^Omega(cos gamma)
                               / sqrt(dR dr)
    with 4-point Lagrange weights on the uniform R and r grids (grid values beyond
    the ends of the grid are zero) and the exact Legendre series in gamma;
  * helicities transform with the Wigner matrix of rho,
      Phi'_(Omega') = sum_Omega D^J_(Omega Omega')(rho) Phi_Omega,
    written for the parity-adapted blocks Omega >= 0 with parity p = (-1)^J, where
    Phi_(-Omega) = (-1)^Omega Phi_Omega and block Omega = 0 carries the factor
    sqrt(2); helicities above Omega_max are zero in both frames;
  * the scalar wave function is Phi / (r R) = Phi' / (r' R'), so
    Phi' = (r' R' / (r R)) Phi (the Jacobi transformation has unit Jacobian);
  * C_c(k) = sum_(a,l) dr' w_l chi_(v'j')(r'_a) P-bar_(j')^(Omega')(cos gamma'_l)
             Phi'^(Omega')(R'_inf, r'_a, gamma'_l)
    with chi the product diatomic state as a function (grid vector / sqrt(dr'));
  * |S_c|^2 = (2 pi K' / mu') |C_E(c)|^2 / |a(E)|^2, K' = sqrt(2 mu' (E - e_c)),
    zero for closed channels; product sums start at k = 0; each electronic state
    Lambda' has its own product states, from the diagonal V_(Lambda'Lambda') with
    the departing atom 100 bohr away.
"""
from __future__ import annotations

from math import factorial

import numpy as np

from . import basis, pes

R_FAR = 100.0   # bohr: R' at which the product diatomic states are computed


# ------------------------------------------------------------------------ Wigner d

def wigner_d_element(J: int, mp: int, m: int, beta: float) -> float:
    """d^J_(m'm)(beta) from Wigner's explicit sum

      d^J_(m'm) = sum_s (-1)^(m'-m+s) sqrt((J+m')!(J-m')!(J+m)!(J-m)!)
                  / ((J+m-s)! s! (m'-m+s)! (J-m'-s)!) cos(b/2)^(2J+m-m'-2s) sin(b/2)^(m'-m+2s).
    """
    c, s_ = np.cos(0.5 * beta), np.sin(0.5 * beta)
    pre = np.sqrt(float(factorial(J + mp) * factorial(J - mp) * factorial(J + m) * factorial(J - m)))
    tot = 0.0
    for s in range(max(0, m - mp), min(J + m, J - mp) + 1):
        den = factorial(J + m - s) * factorial(s) * factorial(mp - m + s) * factorial(J - mp - s)
        tot += ((-1.0) ** (mp - m + s) * c ** (2 * J + m - mp - 2 * s) * s_ ** (mp - m + 2 * s)
                / float(den))
    return pre * tot


def wigner_d(J: int, beta: float) -> np.ndarray:
    """The matrix d^J_(m'm)(beta), m', m = -J..J (index m + J)."""
    return np.array([[wigner_d_element(J, mp, m, beta) for m in range(-J, J + 1)]
                     for mp in range(-J, J + 1)])


def euler_zyz(Rot: np.ndarray):
    """Euler angles (a, b, c) with Rot = R_z(a) R_y(b) R_z(c) (active rotations)."""
    b = np.arccos(np.clip(Rot[2, 2], -1.0, 1.0))
    if abs(np.sin(b)) > 1e-12:
        a = np.arctan2(Rot[1, 2], Rot[0, 2])
        c = np.arctan2(Rot[2, 1], -Rot[2, 0])
    else:                                   # b = 0 or pi: only a + c (or a - c) matters
        a = np.arctan2(Rot[1, 0], Rot[0, 0]) if Rot[2, 2] > 0 else np.arctan2(-Rot[1, 0], -Rot[0, 0])
        c = 0.0
    return a, b, c


def wigner_D_element(J: int, mp: int, m: int, euler) -> float:
    """D^J_(m'm) = exp(-i m' a) d^J_(m'm)(b) exp(-i m c), real for the rotations used here
    (they keep the molecular plane, so a and c are 0 or pi)."""
    a, b, c = euler
    D = np.exp(-1j * mp * a) * wigner_d_element(J, mp, m, b) * np.exp(-1j * m * c)
    if abs(D.imag) > 1e-9:
        raise ValueError("rotation leaves the molecular plane")
    return D.real


# --------------------------------------------------------------- Jacobi coordinates

def atom_coefficients(masses):
    """Positions of A, B, C as x = alpha r + beta R (BC centre of mass at the origin,
    r = C - B, R = A - X_BC): rows (alpha, beta) for A, B, C."""
    mA, mB, mC = masses
    MBC = mB + mC
    return np.array([[0.0, 1.0], [-mC / MBC, 0.0], [mB / MBC, 0.0]])


def product_matrix(masses, arrangement: str) -> np.ndarray:
    """M with (r', R') = M (r, R) for the product arrangement."""
    X = atom_coefficients(masses)
    mA, mB, mC = masses
    A, B, C = X
    if arrangement == "AC+B":
        rp = C - A
        Rp = B - (mA * A + mC * C) / (mA + mC)
    elif arrangement == "AB+C":
        rp = B - A
        Rp = C - (mA * A + mB * B) / (mA + mB)
    else:
        raise ValueError("arrangement must be 'AC+B' or 'AB+C'")
    return np.array([rp, Rp])


def product_masses(masses, arrangement: str):
    """(mu', m'): reduced masses of R' and r'."""
    mA, mB, mC = masses
    M = mA + mB + mC
    if arrangement == "AC+B":
        return mB * (mA + mC) / M, mA * mC / (mA + mC)
    return mC * (mA + mB) / M, mA * mB / (mA + mB)


def body_axes(z_vec, x_ref):
    """Columns (x, y, z): z along z_vec, x in the plane of x_ref with x . x_ref > 0."""
    z = z_vec / np.linalg.norm(z_vec)
    x = x_ref - np.dot(x_ref, z) * z
    x = x / np.linalg.norm(x)
    return np.column_stack([x, np.cross(z, x), z])


def product_to_reactant(masses, arrangement, Rp, rp, cosgp):
    """Reactant Jacobi vectors (r, R) for the product point (R', r', cos gamma'), in
    product body-fixed coordinates (R' along z, r' in the x-z half plane x >= 0)."""
    Minv = np.linalg.inv(product_matrix(masses, arrangement))
    sg = np.sqrt(max(1.0 - cosgp * cosgp, 0.0))
    rp_vec = rp * np.array([sg, 0.0, cosgp])
    Rp_vec = Rp * np.array([0.0, 0.0, 1.0])
    r_vec = Minv[0, 0] * rp_vec + Minv[0, 1] * Rp_vec
    R_vec = Minv[1, 0] * rp_vec + Minv[1, 1] * Rp_vec
    return r_vec, R_vec


def node_to_reactant(masses, arrangement, Rp, rp, cosgp):
    """Reactant (R, r, cos gamma) and the rotation matrix rho (columns: product axes in
    reactant body-fixed coordinates) for the product point (R', r', cos gamma')."""
    r_vec, R_vec = product_to_reactant(masses, arrangement, Rp, rp, cosgp)
    R, r = np.linalg.norm(R_vec), np.linalg.norm(r_vec)
    cosg = np.dot(r_vec, R_vec) / (r * R)
    axes_r = body_axes(R_vec, r_vec)                  # reactant axes, product coordinates
    rho = axes_r.T                                    # product axes in reactant coordinates
    return R, r, cosg, rho


def helicity_matrix(J: int, n_omega: int, rho: np.ndarray) -> np.ndarray:
    """T[Omega', Omega] for parity-adapted blocks 0..n_omega-1 (p = (-1)^J):
      Phi'^p_(Omega') = sum_Omega T[Omega', Omega] Phi^p_Omega,
      T = [s_Omega D_(Omega Omega') + (Omega > 0) (-1)^Omega D_(-Omega, Omega')] / s_(Omega'),
    s_0 = sqrt(2), s_(Omega > 0) = 1 (see the module header)."""
    eul = euler_zyz(rho)
    T = np.zeros((n_omega, n_omega))
    s = lambda om: np.sqrt(2.0) if om == 0 else 1.0
    for op in range(n_omega):
        for om in range(n_omega):
            v = s(om) * wigner_D_element(J, om, op, eul)
            if om > 0:
                v += (-1.0) ** om * wigner_D_element(J, -om, op, eul)
            T[op, om] = v / s(op)
    return T


# -------------------------------------------------------------------- interpolation

def lagrange4(x0, dx, n, x):
    """Stencil start m0 and the 4 Lagrange weights of x on the uniform grid x0 + i dx,
    i = 0..n-1 (points m0..m0+3 with x in the middle interval)."""
    t = (x - x0) / dx
    m0 = int(np.floor(t)) - 1
    u = t - m0                                         # in [1, 2)
    w = np.array([-(u - 1) * (u - 2) * (u - 3) / 6.0, u * (u - 2) * (u - 3) / 2.0,
                  -u * (u - 1) * (u - 3) / 2.0, u * (u - 1) * (u - 2) / 6.0])
    return m0, w


# --------------------------------------------------------------------- the projector

class ProductAnalysis:
    """Product quadrature, product states and per-node maps for one configuration.

    The per-node evaluation below is the formula of the module header evaluated for
    all nodes at once (numpy gathers); nothing is reordered beyond that.
    """

    def __init__(self, H, prod: dict):
        self.H = H
        self.arr = prod["arrangement"]
        self.Rinf = prod["Rinf"]
        self.mu_p, self.m_p = product_masses(H.masses, self.arr)
        self.rlim = (prod["rmin"], prod["rmax"])
        self.rp, self.drp = basis.sine_dvr_nodes(prod["rmin"], prod["rmax"], prod["nr"])
        self.xg, self.wg = basis.gauss_legendre(prod["ngamma"])
        self.vmax, self.jmax = prod["vmax"], prod["jmax"]
        na, nl = len(self.rp), len(self.xg)
        self.node_a = np.repeat(np.arange(na), nl)
        self.node_l = np.tile(np.arange(nl), na)
        nn = na * nl
        self.R = np.zeros(nn)
        self.r = np.zeros(nn)
        self.cosg = np.zeros(nn)
        self.jac = np.zeros(nn)
        self.rho = np.zeros((nn, 3, 3))
        for n in range(nn):
            rp, x = self.rp[self.node_a[n]], self.xg[self.node_l[n]]
            R, r, cosg, rho = node_to_reactant(H.masses, self.arr, self.Rinf, rp, x)
            self.R[n], self.r[n], self.cosg[n], self.rho[n] = R, r, cosg, rho
            self.jac[n] = rp * self.Rinf / (r * R)
        # 4-point stencils; points beyond the grid carry zero weight
        self.midx, self.wR = self._stencils(H.R[0], H.dR, H.NR, self.R)
        self.kidx, self.wr = self._stencils(H.r[0], H.dr, H.nr, self.r)
        # Legendre rows of every helicity at the nodes' reactant angles
        top = max(H.omega_top(J) for J in H.Js)
        self.Pl = [basis.norm_assoc_legendre(H.ng - 1, om, self.cosg) for om in range(top + 1)]
        # helicity matrices per J and node
        self.T = [np.array([helicity_matrix(J, H.omega_top(J) + 1, self.rho[n]) for n in range(nn)])
                  for J in H.Js]
        # product states and channel weights per J
        self.states = {}
        for L in range(H.nelec):
            for j in range(self.jmax + 1):
                self.states[(j, L)] = self.diatomic_states(j, L, self.vmax + 1)
        self.W = []
        for iJ in range(len(H.Js)):
            chans = self.channels(iJ)
            W = np.zeros((len(chans), nn))
            for ic, (L, v, j, op, _) in enumerate(chans):
                chi = self.states[(j, L)][1][self.node_a, v] / np.sqrt(self.drp)
                Pj = basis.norm_assoc_legendre(j, op, self.xg)[j - op][self.node_l]
                W[ic] = self.drp * self.wg[self.node_l] * chi * Pj
            self.W.append(W)

    @staticmethod
    def _stencils(x0, dx, n, x):
        idx = np.zeros((len(x), 4), dtype=int)
        w = np.zeros((len(x), 4))
        for i, xi in enumerate(x):
            m0, wi = lagrange4(x0, dx, n, xi)
            for a in range(4):
                m = m0 + a
                if 0 <= m < n:
                    idx[i, a], w[i, a] = m, wi[a]
        return idx, w

    def diatomic_hamiltonian(self, j, L):
        """Product diatom on the r' sine DVR: T + min(j(j+1)/(2 m' r'^2), E_rot) +
        min(V_LL, V_cut) with the departing atom at R' = 100 bohr (collinear)."""
        H = self.H
        Tp = basis.radial_kinetic_matrix(*self.rlim, len(self.rp), self.m_p, H.tcut)
        V = np.zeros(len(self.rp))
        for a, rp in enumerate(self.rp):
            r_vec, R_vec = product_to_reactant(H.masses, self.arr, R_FAR, rp, 1.0)
            R, r = np.linalg.norm(R_vec), np.linalg.norm(r_vec)
            V[a] = pes.potential_matrix(r, R, np.dot(r_vec, R_vec) / (r * R), H.masses, H.pes)[L, L]
        V = np.minimum(V, H.vcut)
        cent = np.minimum(j * (j + 1.0) / (2.0 * self.m_p * self.rp ** 2), H.erot)
        return Tp + np.diag(V + cent)

    def diatomic_states(self, j, L, nv):
        """Lowest nv eigenpairs; grid-normalised vectors, largest component positive."""
        e, U = np.linalg.eigh(self.diatomic_hamiltonian(j, L))
        U = U[:, :nv].copy()
        for v in range(nv):
            if U[np.argmax(np.abs(U[:, v])), v] < 0:
                U[:, v] = -U[:, v]
        return e[:nv], U

    def channels(self, iJ):
        """Product channels (Lambda', v', j', Omega', e_c) of J index iJ."""
        J = self.H.Js[iJ]
        out = []
        for L in range(self.H.nelec):
            for j in range(self.jmax + 1):
                e, _ = self.states[(j, L)]
                for v in range(self.vmax + 1):
                    for op in range(0, min(j, J, self.H.omega_max) + 1):
                        out.append((L, v, j, op, e[v]))
        return out

    def reactant_values(self, q):
        """Phi^Omega(R, r, gamma) of every block at every node: [nblk, nnodes]."""
        H = self.H
        out = np.zeros((H.nblk, len(self.R)))
        for b, (iJ, J, om, L) in enumerate(H.blocks):
            c = np.einsum("in,nkm->ikm", H.T[om], q[b])            # FBR coefficients
            G = c[:, self.kidx[:, :, None], self.midx[:, None, :]]   # [i, node, b(r), a(R)]
            out[b] = np.einsum("ivba,iv,vb,va->v", G, self.Pl[om], self.wr, self.wR)
        return out / np.sqrt(H.dR * H.dr)

    def overlaps(self, q):
        """C_c(k) for every J index: list of arrays in the order of channels(iJ)."""
        H = self.H
        phi = self.reactant_values(q)
        out = []
        for iJ, J in enumerate(H.Js):
            nom = H.omega_top(J) + 1
            chans = self.channels(iJ)
            C = np.zeros(len(chans))
            for L in range(H.nelec):
                ph = np.array([phi[H.block_index[(iJ, om, L)]] for om in range(nom)])  # [Omega, node]
                php = self.jac[None, :] * np.einsum("vpo,ov->pv", self.T[iJ], ph)     # [Omega', node]
                for ic, (Lc, v, j, op, _) in enumerate(chans):
                    if Lc == L:
                        C[ic] = np.dot(self.W[iJ][ic], php[op])
            out.append(C)
        return out
