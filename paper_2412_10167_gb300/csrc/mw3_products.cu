// Product-channel overlaps of q_k on the surface R' = R'_inf (Section 2.4,
// Eq. Chebyshev-products-overlaps), per Chebyshev iteration, into the cut ring.
//
// Two launches per step:
//   k_prod_eval     u[b][v] = sum_(a,c) wR_a wr_c sum_i P-bar_(Omega_b + i)^(Omega_b)(cos gamma_v)
//                             c^b_i(r_(k_c), R_(m_a))
//                   the reactant function of block b at product node v (4-point Lagrange
//                   stencils in R and r, Legendre series in gamma; 1/sqrt(dR dr) folded
//                   into wR). One warp per (node, block), lanes over the 16 stencil
//                   points and two interleaved halves of the FBR rows.
//   k_prod_project  per (J, Lambda', Omega') group: the rotated, Jacobian-weighted node
//                   values v'[v] = jac_v sum_Omega T_v[Omega'][Omega] u[b(J, Omega, Lambda')][v]
//                   in shared memory, then one warp per channel dots them with the
//                   channel's quadrature weights W[c][v] and writes the overlap into its
//                   cut-ring column.
#include <cuda_runtime.h>

#include "mw3_internal.h"

namespace mw3 {
namespace {

template <typename real>
__device__ __forceinline__ real warp_sum(real s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Lane l of the warp of node v takes stencil point (a, c) = (l & 3, (l >> 2) & 3) of the
// rows i = l >> 4, l >> 4 + 2, ...: one load instruction covers two rows of the 4 x 4
// stencil (8 short segments of 4 consecutive R values).
template <typename real>
__global__ void __launch_bounds__(256) k_prod_eval(const real* __restrict__ q,
                                                   const DevBlock* __restrict__ blocks, int ng,
                                                   int nr, int NR, int nn,
                                                   const int* __restrict__ idx,
                                                   const real* __restrict__ w,
                                                   const real* __restrict__ pl, int ltop,
                                                   real* __restrict__ u) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * 8 + warp;
  const int b = blockIdx.y;
  if (v >= nn) return;   // warp-uniform; the kernel has no block-wide barrier
  const DevBlock B = blocks[b];
  const int a = lane & 3, c = (lane >> 2) & 3, sub = lane >> 4;
  const long plane = (long)nr * NR;
  const real* src = q + (long)b * ng * plane + (long)idx[v * 8 + 4 + c] * NR + idx[v * 8 + a];
  const real* P = pl + ((long)v * ltop + B.omega) * ng;
  real s = 0;
  for (int i = sub; i < B.nrow; i += 2) s += P[i] * src[(long)i * plane];
  s *= w[v * 8 + a] * w[v * 8 + 4 + c];
  s = warp_sum(s);
  if (lane == 0) u[(long)b * nn + v] = s;
}

template <typename real>
__global__ void __launch_bounds__(256) k_prod_project(const real* __restrict__ u, int nn,
                                                      const real* __restrict__ T,
                                                      const real* __restrict__ jac,
                                                      const real* __restrict__ W,
                                                      const ProdGroup* __restrict__ groups,
                                                      real* __restrict__ cut) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* vp = reinterpret_cast<real*>(smem_raw);
  const ProdGroup g = groups[blockIdx.x];
  for (int n = threadIdx.x; n < nn; n += blockDim.x) {
    const real* Tn = T + g.toff + ((long)n * g.nom + g.op) * g.nom;
    real s = 0;
    for (int om = 0; om < g.nom; ++om) s += Tn[om] * u[(long)(g.b0 + om * g.bstride) * nn + n];
    vp[n] = jac[n] * s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < g.nc; c += blockDim.x / 32) {
    const real* Wc = W + (long)(g.c0 + c) * nn;
    real s = 0;
    for (int n = lane; n < nn; n += 32) s += Wc[n] * vp[n];
    s = warp_sum(s);
    if (lane == 0) cut[g.col0 + c] = s;
  }
}

}  // namespace

template <typename real>
cudaError_t launch_prod_eval(const real* q, const DevBlock* blocks, int nblk, int ng, int nr,
                             int NR, int nn, const int* idx, const real* w, const real* pl,
                             int ltop, real* u, cudaStream_t st) {
  dim3 grid((unsigned)((nn + 7) / 8), (unsigned)nblk);
  k_prod_eval<real><<<grid, 256, 0, st>>>(q, blocks, ng, nr, NR, nn, idx, w, pl, ltop, u);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_prod_project(const real* u, int nn, const real* T, const real* jac,
                                const real* W, const ProdGroup* groups, int ngroups,
                                real* cut_slot, cudaStream_t st) {
  if (ngroups == 0) return cudaSuccess;
  k_prod_project<real><<<ngroups, 256, sizeof(real) * (size_t)nn, st>>>(u, nn, T, jac, W, groups,
                                                                         cut_slot);
  return cudaGetLastError();
}

template cudaError_t launch_prod_eval<float>(const float*, const DevBlock*, int, int, int, int,
                                             int, const int*, const float*, const float*, int,
                                             float*, cudaStream_t);
template cudaError_t launch_prod_eval<double>(const double*, const DevBlock*, int, int, int, int,
                                              int, const int*, const double*, const double*, int,
                                              double*, cudaStream_t);
template cudaError_t launch_prod_project<float>(const float*, int, const float*, const float*,
                                                const float*, const ProdGroup*, int, float*,
                                                cudaStream_t);
template cudaError_t launch_prod_project<double>(const double*, int, const double*,
                                                 const double*, const double*, const ProdGroup*,
                                                 int, double*, cudaStream_t);

}  // namespace mw3
