"""The grid Hamiltonian and its scaled form. Test infrastructure only.

Eq. (hamiltonian): H = T_R + T_r + l^2/(2 mu R^2) + j^2/(2 m r^2) + H_e with
mu = m_A (m_B + m_C)/M and m = m_B m_C/(m_B + m_C). In the body-fixed frame
l^2 = J^2 + j^2 - 2 J.j, so l^2 is non-diagonal in gamma and tridiagonal in the
helicity Omega (the coupled grid equations of Section 2.1 and item 4 of its list).

Coefficients: q[b, n, k, m] = Phi_b(R_m, r_k, gamma_n) sqrt(dR dr w_n) for block
b = (J, Omega, Lambda); the inner product is the plain dot product and every term
below is a real symmetric matrix in that basis.

Readings of silent points (each is restated where it is used):
  * parity p = (-1)^J, so Omega = 0 .. min(J, Omega_max) (Eq. angular-functions;
    the coupling to Omega_max + 1 is dropped);
  * Coriolis elements -lambda+_(J Omega) lambda+_(j Omega), with sqrt(2) for the
    Omega = 0 <-> 1 pair (from the (1 + delta_(Omega 0)) normalisation of W);
  * the rotational cap rotcutmaxeV is applied as min(j(j+1)/(2 m r^2), E_rot) and
    by replacing 1/(2 mu R^2) with g_j(R) = min(1/(2 mu R^2), E_rot / lmax2(j)),
    lmax2(j) = (sqrt(J(J+1)) + sqrt(j(j+1)))^2, a positive factor per j that keeps
    the operator symmetric and positive semidefinite;
  * the potential cap VcutmaxeV applies to the diagonal of H_e only;
  * block Omega carries the n - Omega angular functions j = Omega .. n - 1 (exactly
    orthonormal under the shared n-point Gauss-Legendre rule); the state of a block
    lies in their span and the potential enters through its quadrature matrix
    elements in that basis, i.e. as P V P with P = (T^Omega)^T T^Omega (P = 1 for
    Omega = 0);
  * E_min / E_max are rigorous bounds: the lowest / highest eigenvalue of H_e over
    the grid, plus the largest capped radial eigenvalues, plus the largest
    Gershgorin row sum of the angular FBR matrix.
"""
from __future__ import annotations

import numpy as np

from . import basis, pes
from .units import AMU, EV


def _lam(X, omega, sign):
    """lambda^(+/-)_(X Omega) = sqrt(X(X+1) - Omega(Omega +/- 1))."""
    return np.sqrt(max(X * (X + 1.0) - omega * (omega + sign), 0.0))


class GridHamiltonian:
    """H acting on a batch of J values, each with its Omega and electronic blocks."""

    def __init__(self, cfg: dict):
        g = cfg["grid"]
        mA, mB, mC = (m * AMU for m in cfg["masses_u"])
        self.masses = (mA, mB, mC)
        self.mu = mA * (mB + mC) / (mA + mB + mC)       # R reduced mass
        self.m = mB * mC / (mB + mC)                     # r reduced mass
        self.NR, self.nr, self.ng = g["NR"], g["nr"], g["ngamma"]
        self.Rlim = (g["Rmin"], g["Rmax"])
        self.rlim = (g["rmin"], g["rmax"])
        self.R, self.dR = basis.sine_dvr_nodes(g["Rmin"], g["Rmax"], self.NR)
        self.r, self.dr = basis.sine_dvr_nodes(g["rmin"], g["rmax"], self.nr)
        self.x, self.w = basis.gauss_legendre(self.ng)
        caps = cfg["caps"]
        self.vcut = caps["vcut_eV"] * EV
        self.tcut = caps["tcut_eV"] * EV
        self.erot = caps["erot_eV"] * EV
        self.nelec = cfg["nelec"]
        self.pes = cfg["pes"]
        self.Js = list(cfg["J"])
        self.omega_max = cfg["omega_max"]
        if min(max(self.Js), self.omega_max) >= self.ng:
            raise ValueError("every helicity block needs at least one angular function: "
                             "min(max J, omega_max) < ngamma")

        # radial kinetic operators (item 2): dense sine-DVR matrices
        self.TR = basis.radial_kinetic_matrix(*self.Rlim, self.NR, self.mu, self.tcut)
        self.Tr = basis.radial_kinetic_matrix(*self.rlim, self.nr, self.m, self.tcut)
        self.lamR = basis.radial_kinetic_eigenvalues(*self.Rlim, self.NR, self.mu, self.tcut)
        self.lamr = basis.radial_kinetic_eigenvalues(*self.rlim, self.nr, self.m, self.tcut)

        # blocks, J-major, then Omega, then electronic state
        self.blocks = []          # (iJ, J, Omega, Lambda)
        self.block_index = {}
        for iJ, J in enumerate(self.Js):
            for om in range(0, min(J, self.omega_max) + 1):
                for L in range(self.nelec):
                    self.block_index[(iJ, om, L)] = len(self.blocks)
                    self.blocks.append((iJ, J, om, L))
        self.nblk = len(self.blocks)
        self.shape = (self.nblk, self.ng, self.nr, self.NR)

        # angular FBR matrices per Omega (item 3)
        top = max(min(J, self.omega_max) for J in self.Js)
        self.T = [basis.fbr_matrix(om, self.ng, self.x, self.w) for om in range(top + 1)]

        # potential on the grid, diagonal capped (item 5)
        n3, k3, m3 = np.meshgrid(self.x, self.r, self.R, indexing="ij")
        V = pes.potential_matrix(k3, m3, n3, self.masses, cfg["pes"])   # [n,k,m,L,L']
        for L in range(self.nelec):
            V[..., L, L] = np.minimum(V[..., L, L], self.vcut)
        self.V = np.moveaxis(V, (3, 4), (0, 1)).copy()                  # [L,L',n,k,m]

        self.fR = 1.0 / (2.0 * self.mu * self.R ** 2)
        self.fr = 1.0 / (2.0 * self.m * self.r ** 2)
        self.E0 = np.zeros(len(self.Js))
        self.dE = np.zeros(len(self.Js))
        for iJ in range(len(self.Js)):
            emin, emax = self.spectral_bounds(iJ)
            self.E0[iJ] = 0.5 * (emax + emin)
            self.dE[iJ] = 1.0001 * 0.5 * (emax - emin)

    # ------------------------------------------------------------------ angular parts
    def omega_top(self, J):
        return min(J, self.omega_max)

    def g_j(self, J, j):
        """g_j(R) = min(1/(2 mu R^2), E_rot / lmax2(j)) on the R grid."""
        lmax2 = (np.sqrt(J * (J + 1.0)) + np.sqrt(j * (j + 1.0))) ** 2
        if lmax2 == 0.0:
            return self.fR.copy()
        return np.minimum(self.fR, self.erot / lmax2)

    def angular_coefficients(self, J, om):
        """a[i,k,m], bp[i,m], bm[i,m] of the FBR operator of block Omega = om.

        Rows i = 0 .. n - Omega - 1. For row i (j = Omega + i) at grid point (r_k, R_m):
          a  = min(j(j+1)/(2 m r^2), E_rot) + g_j(R) [J(J+1) + j(j+1) - 2 Omega^2]
          bp = -g_j(R) lambda+_(J Omega) lambda+_(j Omega) kappa   (couples to Omega+1, same j)
          bm = -g_j(R) lambda-_(J Omega) lambda-_(j Omega) kappa'  (couples to Omega-1, same j)
        kappa = sqrt(2) when the coupled pair is {0, 1}, otherwise 1.
        """
        n = self.ng - om
        a = np.zeros((n, self.nr, self.NR))
        bp = np.zeros((n, self.NR))
        bm = np.zeros((n, self.NR))
        top = self.omega_top(J)
        for i in range(n):
            j = om + i
            gj = self.g_j(J, j)
            jj = j * (j + 1.0)
            a[i] = (np.minimum(jj * self.fr, self.erot)[:, None]
                    + gj[None, :] * (J * (J + 1.0) + jj - 2.0 * om * om))
            if om + 1 <= top and i >= 1:
                kap = np.sqrt(2.0) if om == 0 else 1.0
                bp[i] = -gj * _lam(J, om, +1) * _lam(j, om, +1) * kap
            if om >= 1:
                kap = np.sqrt(2.0) if om == 1 else 1.0
                bm[i] = -gj * _lam(J, om, -1) * _lam(j, om, -1) * kap
        return a, bp, bm

    def apply_angular(self, q, out):
        """out += (T^Omega)^T [a c^Omega + bp c^(Omega+1) + bm c^(Omega-1) + T^Omega V P q],

        c^Omega = T^Omega q^Omega, for every block: the j^2 and l^2 terms in the FBR
        (Coriolis coupling between Omega and Omega +- 1 at equal j) and the diabatic
        potential through its FBR matrix elements (P V P, P = T^T T per block)."""
        blk = self.shape[1:]
        flat = (self.ng, self.nr * self.NR)
        for iJ, J in enumerate(self.Js):
            top = self.omega_top(J)
            c, pq = {}, {}
            for om in range(top + 1):
                for L in range(self.nelec):
                    b = self.block_index[(iJ, om, L)]
                    c[om, L] = (self.T[om] @ q[b].reshape(flat)).reshape((self.ng - om,) + blk[1:])
                    pq[om, L] = (self.T[om].T @ c[om, L].reshape(self.ng - om, -1)).reshape(blk)
            for om in range(top + 1):
                a, bp, bm = self.angular_coefficients(J, om)
                for L in range(self.nelec):
                    cp = a * c[om, L]
                    if om + 1 <= top:
                        # row i of block om meets row i-1 of block om+1 (same j)
                        cp[1:] += bp[1:, None, :] * c[om + 1, L]
                    if om >= 1:
                        # row i of block om meets row i+1 of block om-1 (same j)
                        cp += bm[:, None, :] * c[om - 1, L][1:]
                    vq = np.zeros(blk)
                    for Lp in range(self.nelec):
                        vq += self.V[L, Lp] * pq[om, Lp]
                    cp = cp.reshape(self.ng - om, -1) + self.T[om] @ vq.reshape(flat)
                    out[self.block_index[(iJ, om, L)]] += (self.T[om].T @ cp).reshape(blk)

    # ------------------------------------------------------------------ full operator
    def apply_H(self, q):
        """H q: radial kinetic (sine DVR), angular (FBR + Coriolis) and potential terms."""
        q = np.asarray(q, dtype=float).reshape(self.shape)
        out = q @ self.TR                                     # R kinetic (T_R symmetric)
        out += np.matmul(self.Tr, q)                          # r kinetic
        self.apply_angular(q, out)                            # j^2, l^2 and potential
        return out

    def project(self, q):
        """P q: each block's component in the span of its angular functions."""
        q = np.asarray(q, dtype=float).reshape(self.shape)
        out = np.empty_like(q)
        flat = (self.ng, self.nr * self.NR)
        for b, (iJ, J, om, L) in enumerate(self.blocks):
            out[b] = (self.T[om].T @ (self.T[om] @ q[b].reshape(flat))).reshape(self.shape[1:])
        return out

    def block_J_index(self):
        return np.array([iJ for (iJ, _, _, _) in self.blocks])

    def apply_Hs(self, q):
        """H_s q = (H - E0) q / dE with (E0, dE) of each block's J (Section 2.2)."""
        q = np.asarray(q, dtype=float).reshape(self.shape)
        bj = self.block_J_index()
        E0 = self.E0[bj][:, None, None, None]
        dE = self.dE[bj][:, None, None, None]
        return (self.apply_H(q) - E0 * q) / dE

    # ------------------------------------------------------------------ spectral bounds
    def spectral_bounds(self, iJ):
        """(E_min, E_max) bracketing the spectrum of H for the J with index iJ.

        E_min: lowest eigenvalue of the (capped) diabatic matrix over the grid;
        the kinetic and angular terms are positive semidefinite.
        E_max: highest eigenvalue of that matrix over the grid + largest capped
        R and r kinetic eigenvalues + the largest Gershgorin row sum |a|+|bp|+|bm|
        of the angular FBR matrix. f_r and g_j decrease with r and R, so that row
        sum is largest at the first nodes r_1, R_1.
        """
        J = self.Js[iJ]
        Vm = np.moveaxis(self.V, (0, 1), (-2, -1))           # [n,k,m,L,L']
        ev = np.linalg.eigvalsh(Vm)
        vmin, vmax = ev[..., 0].min(), ev[..., -1].max()
        ang = 0.0
        for om in range(self.omega_top(J) + 1):
            a, bp, bm = self.angular_coefficients(J, om)
            rows = a[:, 0, 0] + np.abs(bp[:, 0]) + np.abs(bm[:, 0])
            ang = max(ang, rows.max())
        return vmin, vmax + self.lamR.max() + self.lamr.max() + ang

    def dense_H(self, iJ=None):
        """Dense matrix of H by applying it to unit vectors (tiny grids only)."""
        N = int(np.prod(self.shape))
        M = np.zeros((N, N))
        e = np.zeros(N)
        for i in range(N):
            e[:] = 0.0
            e[i] = 1.0
            M[:, i] = self.apply_H(e).ravel()
        return M
