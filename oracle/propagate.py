"""Damped real Chebyshev propagation and its energy-resolved analysis. Test infrastructure only.

Section 2.2, Eq. (wvp-k):
  q_0 = Psi(t=0),  q_1 = D H_s q_0,  q_(k+1) = D (2 H_s q_k - D q_(k-1)),
with the damping D = exp(-phi) of Eq. (imaginary-potential).
Section 2.2, Eqs. (wvf-chebyshev), (chebyshev-expansion-constants): energy-domain
components from sum_k (2 - delta_k0) exp(-i k theta) q_k, cos(theta) = E_s.
Section 2.3.1: initial packet W chi_(v0 j0)(r) Y_(j0 Omega0)(gamma) g(R) with the real
g(R) of Eq. (initial-gaussian) and the incoming amplitude of Eq. (initial-flux-collisions).
Section 2.4: total reaction probability from the flux through r = r* (Eq. total-flux)
and state-resolved probabilities from projections at R_inf
(Eqs. Chebyshev-products-overlaps, S-matrix-from-chebyshev); product channels
through the projector of oracle/products.py.

Readings (the paper is silent, ambiguous or garbled at these points):
  * "N iterations" means q_0 .. q_(N-1) enter the energy sums;
  * the energy grid is an inclusive linspace of collision energies;
  * exp(-i k theta) is evaluated directly from k*theta in FP64 (no recurrence);
  * energy-resolved function: Psi_E = [1/(2 pi dE sin theta)] sum_k c_k q_k,
    which is (i/2pi) G+(E) Psi_0 by the Chebyshev expansion of the outgoing Green
    function; the printed prefactor of c_k (hbar / sqrt(dE^2 - (E-E0)^2)) is this
    1/(dE sin theta) up to the 2 pi, and the constant is fixed by the Eckart pin;
  * a(E) = sqrt(mu/(2 pi K)) sum_m dR exp(i K R_m) g~(R_m), with g~ the grid-normalised
    g; the 1/(2i) phase of the printed formula drops out of every |.|^2, and only
    the incoming half of the cosine contributes (Section 2.3.1);
  * the printed flux formula conjugates both factors; the reading used is
    P(E) = (2 pi / m) Im sum conj(Psi_E) dPsi_E/dr |_(r*) / |a(E)|^2, i.e. outgoing
    flux per unit incoming flux 1/(2 pi);
  * |S_c|^2 = (2 pi K_c / mu) |C_E(c)|^2 / |a(E)|^2 for an open reactant channel,
    0 for a closed one; channel sums start at k_min (kminelastic);
  * damping: phi = phi_R(R) + phi_r(r), phi_x = A_x (x - x_I)^n beyond x_I.
"""
from __future__ import annotations

import numpy as np

from . import basis, pes
from .hamiltonian import GridHamiltonian
from .products import ProductAnalysis
from .units import AMU, EV

R_DIATOM = 100.0   # bohr: R at which diatomic eigenfunctions are computed (Table 1)


# ------------------------------------------------------------------------------ damping

def damping_profile(x, xI, A, n):
    """exp(-phi(x)), phi = 0 for x < x_I and A (x - x_I)^n beyond (Eq. imaginary-potential)."""
    x = np.asarray(x, dtype=float)
    phi = np.where(x > xI, A * np.abs(x - xI) ** n, 0.0)
    return np.exp(-phi)


def damping_grid(H: GridHamiltonian, absorber: dict):
    """D[k, m] = exp(-phi_r(r_k)) exp(-phi_R(R_m)).

    Test options ``RI_low``/``AR_low`` and ``rI_low``/``Ar_low``: an extra absorber below
    R = RI_low (used only when the flux is taken in R, so that the transmitted part is
    absorbed too), or below r = rI_low (a product-arrangement packet whose R' runs
    along r).
    """
    DR = damping_profile(H.R, absorber["RI"], absorber["AR"], absorber["nR"])
    if absorber.get("RI_low") is not None:
        DR = DR * damping_profile(-H.R, -absorber["RI_low"], absorber["AR_low"], absorber["nR"])
    Dr = damping_profile(H.r, absorber["rI"], absorber["Ar"], absorber["nr"])
    if absorber.get("rI_low") is not None:
        Dr = Dr * damping_profile(-H.r, -absorber["rI_low"], absorber["Ar_low"], absorber["nr"])
    return Dr[:, None] * DR[None, :]


# --------------------------------------------------------------------- diatomic states

def diatomic_hamiltonian(H: GridHamiltonian, j: int, L: int):
    """T_r + min(j(j+1)/(2 m r^2), E_rot) + V_LL(r, R = 100 bohr) on the r sine DVR."""
    Vd = pes.potential_matrix(H.r, R_DIATOM, 0.0, H.masses, H.pes)[..., L, L]
    Vd = np.minimum(Vd, H.vcut)
    cent = np.minimum(j * (j + 1.0) * H.fr, H.erot)
    return H.Tr + np.diag(Vd + cent)


def diatomic_states(H: GridHamiltonian, j: int, L: int, nv: int):
    """Lowest nv eigenpairs (E_vj, chi_vj) of the diatomic Hamiltonian.

    chi is the grid-normalised DVR vector (sum chi^2 = 1); its sign is fixed so
    that its largest-magnitude component is positive.
    """
    e, U = np.linalg.eigh(diatomic_hamiltonian(H, j, L))
    U = U[:, :nv].copy()
    for v in range(nv):
        if U[np.argmax(np.abs(U[:, v])), v] < 0:
            U[:, v] = -U[:, v]
    return e[:nv], U


# ----------------------------------------------------------------------- initial packet

def packet_g(R, R0, Gamma, k0):
    """Real g(R) = exp(-(R - R0)^2 / (2 Gamma^2)) cos(k0 R) (Eq. initial-gaussian; constant dropped)."""
    return np.exp(-(R - R0) ** 2 / (2.0 * Gamma ** 2)) * np.cos(k0 * R)


def initial_packet(H: GridHamiltonian, packet: dict):
    """q_0 = N g(R_m) chi_(v0 j0)(r_k) y(gamma_n) in block (Omega0, elec0) of every J.

    y is the FBR basis row of T^Omega0 for j0 (for Omega0 = 0 this is
    P-bar_j0^0(x_n) sqrt(w_n)); ||q_0|| = 1. Returns (q0, info).
    """
    v0, j0, om0, L0 = packet["v0"], packet["j0"], packet["omega0"], packet["elec0"]
    Ev, chi = diatomic_states(H, j0, L0, v0 + 1)
    k0 = np.sqrt(2.0 * H.mu * packet["Ecol_eV"] * EV)
    g = packet_g(H.R, packet["R0"], packet["Gamma"], k0)
    gn = g / np.sqrt(np.sum(g * g))
    y = H.T[om0][j0 - om0]
    q0 = np.zeros(H.shape)
    for iJ in range(len(H.Js)):
        b = H.block_index[(iJ, om0, L0)]
        q0[b] = y[:, None, None] * chi[:, v0][None, :, None] * gn[None, None, :]
    info = dict(E_v0j0=Ev[v0], chi=chi[:, v0], g_tilde=gn / np.sqrt(H.dR), k0=k0)
    return q0, info


def incoming_amplitude(H: GridHamiltonian, g_tilde, Ecol):
    """a(E) = sqrt(mu / (2 pi K)) sum_m dR exp(i K R_m) g~(R_m), K = sqrt(2 mu E_col)."""
    K = np.sqrt(2.0 * H.mu * np.asarray(Ecol, dtype=float))
    ph = np.exp(1j * K[:, None] * H.R[None, :])
    return np.sqrt(H.mu / (2.0 * np.pi * K)) * (ph @ g_tilde) * H.dR


# ------------------------------------------------------------------------- flux cut

def flux_cut(H: GridHamiltonian, q, rstar):
    """psi(r*) and d psi/dr(r*) for every (block, gamma, R) from the sine interpolant.

    Along each r line: a = S_r q (DST-II coefficients) and
      psi(r*) = sum_j s_j a_j phi_j(r*),  psi'(r*) = sum_j s_j a_j phi_j'(r*).
    """
    S = basis.dst2_matrix(H.nr)
    s = np.ones(H.nr)
    s[-1] = 1.0 / np.sqrt(2.0)
    ph, dph = basis.sine_basis_at(*H.rlim, H.nr, rstar)
    a = np.einsum("jk,bnkm->bnjm", S, q)
    psi = np.einsum("j,bnjm->bnm", s * ph, a)
    dpsi = np.einsum("j,bnjm->bnm", s * dph, a)
    return psi, dpsi


def flux_cut_R(H: GridHamiltonian, q, Rstar):
    """Test option: the same cut taken along R at R = R* (flux in the R coordinate)."""
    S = basis.dst2_matrix(H.NR)
    s = np.ones(H.NR)
    s[-1] = 1.0 / np.sqrt(2.0)
    ph, dph = basis.sine_basis_at(*H.Rlim, H.NR, Rstar)
    a = np.einsum("jm,bnkm->bnkj", S, q)
    return np.einsum("j,bnkj->bnk", s * ph, a), np.einsum("j,bnkj->bnk", s * dph, a)


# ------------------------------------------------------------------ reactant channels

def reactant_channels(H: GridHamiltonian, analysis: dict):
    """Channels (J index, Omega, Lambda, v, j) with their DVR vectors and energies.

    Every block (J, Omega, Lambda) contributes the channels v = 0..vmax,
    j = Omega..min(jmax, n_gamma - 1) (the angular functions of the block).
    """
    vmax, jmax = analysis["vmax"], analysis["jmax"]
    chans, chis, eps = [], [], []
    cache = {}
    for (iJ, J, om, L) in H.blocks:
        for j in range(om, min(jmax, H.ng - 1) + 1):
            if (j, L) not in cache:
                cache[(j, L)] = diatomic_states(H, j, L, vmax + 1)
            e, U = cache[(j, L)]
            for v in range(vmax + 1):
                chans.append((iJ, om, L, v, j))
                chis.append(U[:, v])
                eps.append(e[v])
    return chans, np.array(chis), np.array(eps)


def channel_overlaps(H: GridHamiltonian, q, chans, chis, m_inf):
    """C_c(k) = (1/sqrt(dR)) sum_k chi_vj(r_k) c^Omega_j(r_k, R_inf), c^Omega = T^Omega q."""
    out = np.zeros(len(chans))
    for c, ((iJ, om, L, v, j), chi) in enumerate(zip(chans, chis)):
        b = H.block_index[(iJ, om, L)]
        col = q[b][:, :, m_inf]                       # [n, k]
        cj = H.T[om][j - om] @ col                    # FBR coefficient over r
        out[c] = np.dot(chi, cj) / np.sqrt(H.dR)
    return out


# --------------------------------------------------------------------------- propagate

class Result(dict):
    """Raw energy sums and derived probabilities of one propagation."""


def energy_grid(H: GridHamiltonian, analysis: dict, E_v0j0):
    Ecol = np.linspace(analysis["E_lo_eV"] * EV, analysis["E_hi_eV"] * EV, analysis["nE"])
    Etot = Ecol + E_v0j0
    theta = np.zeros((len(H.Js), len(Ecol)))
    for iJ in range(len(H.Js)):
        Es = (Etot - H.E0[iJ]) / H.dE[iJ]
        theta[iJ] = np.arccos(Es)
    return Ecol, Etot, theta


def chebyshev_iterates(H: GridHamiltonian, q0, D, N):
    """Yield (k, q_k, q_(k+1)) for k = 0..N-1 of the damped recursion of Eq. (wvp-k).

      q_1 = D H_s q_0,   q_(k+1) = D (2 H_s q_k - D q_(k-1)).
    """
    q_prev = np.zeros(H.shape)
    q = q0
    for k in range(N):
        Hs_q = H.apply_Hs(q)
        if k == 0:
            q_next = D * Hs_q
        else:
            q_next = D * (2.0 * Hs_q - D * q_prev)
        yield k, q, q_next
        q_prev, q = q, q_next


def propagate(cfg: dict, nsteps=None, H: GridHamiltonian = None, flux_axis="r",
              flux_at=None, keep_states=False, channels=True, q0=None):
    """Run the modified real Chebyshev recursion and accumulate the energy sums.

    Returns a Result with q_N, q_(N-1), the raw sums A (psi) and B (dpsi) per
    energy and cut point, the channel sums, the norm trace ||q_k||^2 (k = 0..N),
    and the derived probabilities. ``q0`` replaces the initial packet as the first
    iterate (the packet still defines a(E) and the energy grid). ``cfg["pcb"]`` (the
    packet's arrangement and its diatom's sine DVR) starts from the products-coordinate
    packet of pcb.py instead, with its closed-form a(E).
    """
    if H is None:
        H = GridHamiltonian(cfg)
    N = cfg["steps"] if nsteps is None else int(nsteps)
    an = cfg["analysis"]
    pcb_src = cfg.get("pcb")
    if pcb_src:     # products-coordinate-based start (pcb.py): the grid is the product arrangement
        from . import pcb
        qp, info = pcb.pcb_packet(H, cfg["packet"], pcb_src)
    else:
        qp, info = initial_packet(H, cfg["packet"])
    q0 = qp if q0 is None else np.asarray(q0, dtype=float)
    D = damping_grid(H, cfg["absorber"])[None, None, :, :]
    Ecol, Etot, theta = energy_grid(H, an, info["E_v0j0"])
    bj = H.block_J_index()
    th_blk = theta[bj]                                 # [nblk, nE]

    cut_at = an["rstar"] if flux_at is None else flux_at
    cutfn = flux_cut if flux_axis == "r" else flux_cut_R
    psi0, _ = cutfn(H, q0, cut_at)
    A = np.zeros((H.nblk, len(Ecol)) + psi0.shape[1:], dtype=complex)
    B = np.zeros_like(A)

    if channels:
        chans, chis, eps = reactant_channels(H, an)
        m_inf = int(np.argmin(np.abs(H.R - an["Rinf"])))
        chan_J = np.array([c[0] for c in chans], dtype=int)
        Cc = np.zeros((len(chans), len(Ecol)), dtype=complex)
    kmin = an.get("kmin", 0)
    prod = an.get("products") if channels else None
    if prod:
        pa = ProductAnalysis(H, prod)
        Cp = [np.zeros((len(pa.channels(iJ)), len(Ecol)), dtype=complex) for iJ in range(len(H.Js))]

    norms = [float(np.sum(q0 * q0))]
    states = [q0.copy()] if keep_states else []
    q, q_next = np.zeros(H.shape), q0
    for k, q, q_next in chebyshev_iterates(H, q0, D, N):
        ck = (1.0 if k == 0 else 2.0) * np.exp(-1j * k * th_blk)      # [nblk, nE]
        psi, dpsi = cutfn(H, q, cut_at)
        A += ck[:, :, None, None] * psi[:, None]
        B += ck[:, :, None, None] * dpsi[:, None]
        if channels and k >= kmin:
            ov = channel_overlaps(H, q, chans, chis, m_inf)
            ckc = (1.0 if k == 0 else 2.0) * np.exp(-1j * k * theta[chan_J])
            Cc += ckc * ov[:, None]
        if prod:
            ovp = pa.overlaps(q)
            for iJ in range(len(H.Js)):
                Cp[iJ] += ((1.0 if k == 0 else 2.0) * np.exp(-1j * k * theta[iJ]))[None, :] * ovp[iJ][:, None]
        norms.append(float(np.sum(q_next * q_next)))
        if keep_states:
            states.append(q_next.copy())
    q, q_prev = q_next, q
    res = Result(q=q, q_prev=q_prev, A=A, B=B, norms=np.array(norms), Ecol=Ecol, Etot=Etot,
                 theta=theta, info=info, H=H, states=states)
    if pcb_src:
        a = pcb.incoming_amplitude(info["packet_function"], Ecol)
    else:
        a = incoming_amplitude(H, info["g_tilde"], Ecol)
    res["a"] = a
    res["flux_sum"], res["P_total"] = total_probability(H, A, B, theta, a, flux_axis)
    if channels:
        pref_c = 1.0 / (2.0 * np.pi * H.dE[chan_J][:, None] * np.sin(theta[chan_J]))
        CE = pref_c * Cc
        Kc2 = 2.0 * H.mu * (Etot[None, :] - eps[:, None])
        open_ = Kc2 > 0
        Kc = np.sqrt(np.where(open_, Kc2, 0.0))
        S2 = np.where(open_, 2.0 * np.pi * Kc / H.mu * np.abs(CE) ** 2 / np.abs(a)[None, :] ** 2, 0.0)
        res.update(channels=chans, chan_energy=eps, C_raw=Cc, S2=S2)
        # inelastic probability per (J, Lambda, v, j), summed over Omega
        res["P_inel"] = {}
        for (iJ, om, L, v, j), s2 in zip(chans, S2):
            key = (iJ, L, v, j)
            res["P_inel"][key] = res["P_inel"].get(key, 0.0) + s2
    if prod:
        res["prod_channels"] = [pa.channels(iJ) for iJ in range(len(H.Js))]
        res["C_prod_raw"] = Cp
        res["P_prod"] = product_probabilities(H, pa, Cp, theta, Etot, a)
    return res


def total_probability(H: GridHamiltonian, A, B, theta, a, flux_axis="r"):
    """Total reaction probability from the flux through the cut (Section 2.4,
    Eq. total-flux, with the reading of the module header).

    A[b, E, ...], B[b, E, ...] are the Chebyshev sums sum_k (2 - delta_k0) exp(-i k theta)
    of psi_k and d psi_k / dx on the cut of every block b (x = r, or R for the test
    option), theta[iJ, E] the Chebyshev angles, a[E] the incoming amplitude:
      Psi_E = A / (2 pi dE sin theta),  dPsi_E = B / (2 pi dE sin theta),
      P(E) = (2 pi / m_x) Im sum_(b, cut) conj(Psi_E) dPsi_E / |a|^2,
    m_x the reduced mass of the cut's coordinate (m for r, mu for R). Returns the raw
    flux sum [nJ, nE] and P [nJ, nE].
    """
    bj = H.block_J_index()
    nE = theta.shape[1]
    pref = 1.0 / (2.0 * np.pi * H.dE[bj][:, None] * np.sin(theta[bj]))   # [nblk, nE]
    flux = np.zeros((len(H.Js), nE))
    for b in range(H.nblk):
        PsiE = pref[b][:, None, None] * A[b]
        dPsiE = pref[b][:, None, None] * B[b]
        flux[bj[b]] += np.sum(np.imag(np.conj(PsiE) * dPsiE), axis=(1, 2))
    mass = H.m if flux_axis == "r" else H.mu
    return flux, (2.0 * np.pi / mass) * flux / np.abs(a)[None, :] ** 2


def product_probabilities(H: GridHamiltonian, pa: ProductAnalysis, Cp, theta, Etot, a):
    """State-resolved product probabilities (Section 2.4, Eq. S-matrix-from-chebyshev).

    Cp[iJ][c, E] are the Chebyshev sums sum_k (2 - delta_k0) exp(-i k theta) C_c(k) of
    the product-channel overlaps, theta[iJ, E] the Chebyshev angles, Etot[E] the total
    energies and a[E] the incoming amplitude. Per channel c = (Lambda', v', j', Omega'):
      C_E(c) = C_c / (2 pi dE sin theta),  K' = sqrt(2 mu' (E - e_c)),
      |S_c|^2 = (2 pi K' / mu') |C_E(c)|^2 / |a|^2  (0 for a closed channel),
    and the result per (iJ, Lambda', v', j') is the sum of |S_c|^2 over Omega'.
    """
    out = {}
    for iJ in range(len(H.Js)):
        pref_p = 1.0 / (2.0 * np.pi * H.dE[iJ] * np.sin(theta[iJ]))
        for ic, (L, v, j, op, e) in enumerate(pa.channels(iJ)):
            K2 = 2.0 * pa.mu_p * (Etot - e)
            Kp = np.sqrt(np.where(K2 > 0, K2, 0.0))
            s2 = np.where(K2 > 0, 2.0 * np.pi * Kp / pa.mu_p * np.abs(pref_p * Cp[iJ][ic]) ** 2
                          / np.abs(a) ** 2, 0.0)
            key = (iJ, L, v, j)
            out[key] = out.get(key, 0.0) + s2
    return out


def time_domain_packet(states, t, E0, dE):
    """Psi(t) = sum_k f_k q_k, f_k = (2 - delta_k0) exp(-i E0 t) (-i)^k J_k(t dE).

    Eqs. (wvf-chebyshev), (chebyshev-expansion-constants) with hbar = 1; states is
    the list q_0, q_1, ... of an undamped propagation.
    """
    from scipy.special import jv
    out = np.zeros_like(states[0], dtype=complex)
    for k, qk in enumerate(states):
        fk = (1.0 if k == 0 else 2.0) * np.exp(-1j * E0 * t) * (-1j) ** k * jv(k, t * dE)
        out += fk * qk
    return out
