// Products-coordinate-based (PCB) start of a propagation (Section 2.4, the first of its two
// routes to state-to-state probabilities; the packet of Section 2.3.1, Eqs.
// initial-collision-wvp and initial-gaussian).
//
// The packet is a product of one-dimensional functions in its own (reactant) Jacobi frame,
//   Phi^s_(Omega0)(R_s, r_s, gamma_s) = g(R_s) chi(r_s) P-bar_(j0)^(Omega0)(cos gamma_s),
// and the propagation grid is the product arrangement. One launch evaluates it at every
// grid node (R_m, r_k, gamma_n): the packet's coordinates (r_s, R_s) = M (r, R), the angle and
// flips of the rotation between the two body frames, and for every (J, Omega) block
//   q[(J, Omega, Lambda0)][n][k][m] = (r R / (r_s R_s)) T^J[Omega][Omega0] Phi^s sqrt(dR dr w_n)
// with T the parity-adapted helicity transform (the same one the product projection uses).
// The gamma transform to the FBR follows on the library's stream.
//
// Work per node: the geometry, one sine series of the packet diatom (the three-term sine
// recurrence over its n_s coefficients), one Legendre recurrence, and per (J, Omega) two
// Jacobi-polynomial recurrences of length <= J: FP64 throughout (a one-off transform).
#include <cuda_runtime.h>

#include <algorithm>

#include "mw3_internal.h"
#include "mw3_wigner.h"

namespace mw3 {

__global__ void __launch_bounds__(256) k_pcb_packet(PcbParams p, const double* __restrict__ xw,
                                                    const double* __restrict__ coef,
                                                    const PcbTerm* __restrict__ terms,
                                                    int nterms, double* __restrict__ out) {
  extern __shared__ double scoef[];
  for (int j = threadIdx.x; j < p.nrs; j += blockDim.x) scoef[j] = coef[j];
  __syncthreads();
  const long npts = (long)p.ng * p.nr * p.NR;
  const double Ls = p.rsmax - p.rsmin;
  for (long v = (long)blockIdx.x * blockDim.x + threadIdx.x; v < npts;
       v += (long)gridDim.x * blockDim.x) {
    const int m = (int)(v % p.NR);
    const int k = (int)((v / p.NR) % p.nr);
    const int n = (int)(v / ((long)p.NR * p.nr));
    const double R = p.Rmin + (m + 0.5) * p.dR;
    const double r = p.rmin + (k + 0.5) * p.dr;
    const double x = xw[n], w = xw[p.ng + n];
    const double sg = sqrt(fmax(1.0 - x * x, 0.0));
    // plane vectors (x, z) of the grid's body frame: r = r (sin g, cos g), R = (0, R)
    const double rvx = r * sg, rvz = r * x;
    const double rsx = p.M00 * rvx, rsz = p.M00 * rvz + p.M01 * R;
    const double Rsx = p.M10 * rvx, Rsz = p.M10 * rvz + p.M11 * R;
    const double Rs = hypot(Rsx, Rsz), rs = hypot(rsx, rsz);
    if (!(Rs > 0.0 && rs > 0.0)) {   // a degenerate packet frame: the packet vanishes there
      for (int t = 0; t < nterms; ++t) out[(long)terms[t].blk * npts + v] = 0.0;
      continue;
    }
    const double cs = (rsx * Rsx + rsz * Rsz) / (rs * Rs);
    // the packet in its own frame
    const double dRs = Rs - p.R0;
    const double g = p.N * exp(-dRs * dRs / (2.0 * p.G * p.G)) * cos(p.k0 * Rs);
    double chi = 0.0;
    if (rs > p.rsmin && rs < p.rsmax) {
      const double th = M_PI * (rs - p.rsmin) / Ls;
      const double c2 = 2.0 * cos(th);
      double s0 = 0.0, s1 = sin(th);
      for (int j = 0; j < p.nrs; ++j) {   // sin((j + 1) th) by the three-term recurrence
        chi += scoef[j] * s1;
        const double s2 = c2 * s1 - s0;
        s0 = s1;
        s1 = s2;
      }
    }
    // normalised associated Legendre P-bar_(j0)^(Omega0)(cs)
    double pl = p.plc * pow(fmax(1.0 - cs * cs, 0.0), 0.5 * p.om0);
    if (p.j0 > p.om0) {
      double pm2 = pl, pm1 = sqrt(2.0 * p.om0 + 3.0) * cs * pl;
      double a_prev = sqrt((4.0 * (p.om0 + 1.0) * (p.om0 + 1.0) - 1.0) /
                           ((p.om0 + 1.0) * (p.om0 + 1.0) - (double)p.om0 * p.om0));
      for (int j = p.om0 + 2; j <= p.j0; ++j) {
        const double a = sqrt((4.0 * j * j - 1.0) / ((double)j * j - (double)p.om0 * p.om0));
        const double pj = a * (cs * pm1 - pm2 / a_prev);
        pm2 = pm1;
        pm1 = pj;
        a_prev = a;
      }
      pl = pm1;
    }
    const double base = (r * R / (rs * Rs)) * g * chi * pl * sqrt(p.dR * p.dr * w);
    // rotation between the frames: the packet's axes in grid coordinates, z_s along R_s and
    // x_s the unit part of r_s normal to it; rho (grid axes in the packet frame) is
    // R_z(a) R_y(beta) R_z(c) with a, c in {0, pi}
    const double zx = Rsx / Rs, zz = Rsz / Rs;
    const double rz = rsx * zx + rsz * zz;
    double xx = rsx - rz * zx, xz = rsz - rz * zz;
    const double nx = hypot(xx, xz);
    if (nx > 0) {
      xx /= nx;
      xz /= nx;
    }
    const double beta = acos(fmin(1.0, fmax(-1.0, zz)));
    int sa, sc;
    if (sin(beta) > 1e-12) {
      sa = xz >= 0 ? 1 : -1;
      sc = zx <= 0 ? 1 : -1;
    } else {
      sa = 1;
      sc = (zz * xx - zx * xz) >= 0 ? 1 : -1;
    }
    const double sh = sin(0.5 * beta), ch = cos(0.5 * beta), cb = cos(beta);
    const double fa = (sa < 0 && (p.om0 & 1)) ? -1.0 : 1.0;
    for (int t = 0; t < nterms; ++t) {
      const PcbTerm tm = terms[t];
      double T = tm.p1 * wigner_d_eval(tm.w1, 1.0, sh, ch, cb);
      if (tm.p2 != 0.0) T += tm.p2 * wigner_d_eval(tm.w2, 1.0, sh, ch, cb);
      if (sc < 0 && (tm.om & 1)) T = -T;
      out[(long)tm.blk * npts + v] = fa * T * base;
    }
  }
}

cudaError_t launch_pcb_packet(const PcbParams& p, const double* xw, const double* coef,
                              const PcbTerm* terms, int nterms, double* out, int nsm,
                              cudaStream_t st) {
  const long npts = (long)p.ng * p.nr * p.NR;
  const long blocks = std::max<long>(1, std::min<long>((long)nsm * 8, (npts + 255) / 256));
  k_pcb_packet<<<(unsigned)blocks, 256, (size_t)p.nrs * sizeof(double), st>>>(p, xw, coef, terms,
                                                                             nterms, out);
  return cudaGetLastError();
}

}  // namespace mw3
