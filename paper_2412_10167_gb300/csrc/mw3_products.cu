// Product-channel overlaps of q_k on the surface R' = R'_inf (Section 2.4,
// Eq. Chebyshev-products-overlaps), per Chebyshev iteration, into the cut ring.
//
// The projection is kept in FP64 whatever the state's precision (the asymptotic
// projections of the mixed form): the state times the Legendre rows in partial sums of
// eight rows (each product and partial sum in the state's precision), FP64 across the
// partials, the stencil weights, the helicity rotation, the Jacobian and the channel dots,
// and an FP64 overlap into the FP64 channel ring.
//
// Two launches per step (three in the plane-major form):
//   k_prod_nodes  u_Omega = sum_(a,c) wR_a wr_c sum_i P-bar_(Omega + i)^Omega(cos gamma_v)
//                           c^(J,Omega,Lambda')_i(r_(k_c), R_(m_a))
//                 the reactant function of every helicity block of (J, Lambda') at product
//                 node v (4-point Lagrange stencils in R and r, Legendre series in gamma;
//                 1/sqrt(dR dr) folded into wR), then the rotated, Jacobian-weighted node
//                 values v'[Omega'][v] = jac_v sum_Omega T_v[Omega'][Omega] u_Omega.
//   k_prod_dots   four warps per channel dot v'[Omega'(c)] with the channel's quadrature
//                 weights W[c][v] and write the overlap into its cut-ring column.
// Plane-major form (k_prod_gather + k_prod_nodes_g): the stencil reads of k_prod_nodes touch
// one 16-byte segment per (row, r) line, a cache line each, and the same grid columns are read
// again for every node whose stencil shares them. The gather kernel first copies the distinct
// stencil columns of every block, once, into rows that hold all FBR rows i of one column
// contiguously; the node sums then read 32 consecutive rows per load (one line in FP32).
#include <cuda_runtime.h>

#include "mw3_internal.h"

namespace mw3 {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Thread Omega' of the CTA rotates the helicities at node v (the node values u_Omega of every
// helicity block in us):
//   v[g(J, Lambda', Omega')][v] = jac_v sum_Omega T_v[Omega'][Omega] u_Omega.
__device__ __forceinline__ void rotate_node(const double* us, int v, int g0, const ProdGroup& G,
                                            int nn, const double* __restrict__ T,
                                            const double* __restrict__ jac,
                                            const ProdGroup* __restrict__ groups,
                                            double* __restrict__ vout) {
  const int nom = G.nom;
  const int op = threadIdx.x;
  if (op < nom && groups[g0 + op].op == op) {
    const double* Tv = T + G.toff + ((long)v * nom + op) * nom;
    double s = 0;
    for (int om = 0; om < nom; ++om) s += Tv[om] * us[om];
    vout[(long)(g0 + op) * nn + v] = jac[v] * s;
  }
}

// One CTA per (node v, J, Lambda'): warp w evaluates the reactant function of the block
// (J, Omega = w, Lambda') at the node. Lane l takes stencil point (a, c) =
// (l & 3, (l >> 2) & 3) of the rows i = l >> 4, l >> 4 + 2, ...: one load instruction
// covers two rows of the 4 x 4 stencil (8 short segments of 4 consecutive R values).
// A lane's rows are summed eight at a time (eight loads in flight, one partial in the
// state's precision) and the partials in FP64.
// Then thread Omega' of the CTA rotates the helicities at the node:
//   v[g(J, Lambda', Omega')][v] = jac_v sum_Omega T_v[Omega'][Omega] u_Omega.
template <typename real>
__global__ void __launch_bounds__(1024) k_prod_nodes(const real* __restrict__ q, int ng, int nr,
                                                     int NR, int nn,
                                                     const int* __restrict__ idx,
                                                     const double* __restrict__ w,
                                                     const real* __restrict__ pl, int ltop,
                                                     const double* __restrict__ T,
                                                     const double* __restrict__ jac,
                                                     const ProdGroup* __restrict__ groups,
                                                     const int* __restrict__ jl_group,
                                                     double* __restrict__ vout) {
  __shared__ double us[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x;
  const int g0 = jl_group[blockIdx.y];
  const ProdGroup G = groups[g0];          // Omega' = 0 group of this (J, Lambda')
  const int nom = G.nom;
  if (warp < nom) {
    const int b = G.b0 + warp * G.bstride;
    const int a = lane & 3, c = (lane >> 2) & 3, sub = lane >> 4;
    const long plane = (long)nr * NR;
    const real* src = q + (long)b * ng * plane + (long)idx[v * 8 + 4 + c] * NR + idx[v * 8 + a];
    const real* P = pl + ((long)v * ltop + warp) * ng;
    const int nrow = ng - warp;            // angular functions of helicity Omega = warp
    double acc = 0.0;
    int i = sub;
    for (; i + 14 < nrow; i += 16) {
      real x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = src[(long)(i + 2 * u) * plane];
      real part = P[i] * x[0];
#pragma unroll
      for (int u = 1; u < 8; ++u) part += P[i + 2 * u] * x[u];
      acc += (double)part;
    }
    real part = 0;
    for (; i < nrow; i += 2) part += P[i] * src[(long)i * plane];
    acc += (double)part;
    double s = acc * (w[v * 8 + a] * w[v * 8 + 4 + c]);
    s = warp_sum(s);
    if (lane == 0) us[warp] = s;
  }
  __syncthreads();
  rotate_node(us, v, g0, G, nn, T, jac, groups, vout);
}

// Plane-major gather: one CTA per (32 stencil columns, block b). Each warp reads rows of the
// block's (i, r, R) planes at the 32 columns (sorted, so neighbouring lanes mostly read
// neighbouring addresses), and the CTA writes them transposed through shared memory:
// G[b][s][i] for 32 rows i at a time, rows nrow.. of the block as zeros. The loads of the next
// 32 rows are issued before the transpose of the current ones. 256 threads: 8 warps x 4 rows
// (or 4 columns) per 32 x 32 chunk.
template <typename real>
__global__ void __launch_bounds__(256) k_prod_gather(const real* __restrict__ q, int ng, long plane,
                                                     const int* __restrict__ pts, int spad, int ngp,
                                                     const DevBlock* __restrict__ blocks,
                                                     real* __restrict__ G) {
  __shared__ real tile[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = blockIdx.x * 32;
  const int b = blockIdx.y;
  const int nrow = blocks[b].nrow;
  const real* qb = q + (long)b * ng * plane + pts[p0 + lane];
  real* Gb = G + ((long)b * spad + p0) * ngp;
  real x[4];
  auto load = [&](int i0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + warp + 8 * u;
      x[u] = i < nrow ? qb[(long)i * plane] : (real)0;
    }
  };
  load(0);
  for (int i0 = 0; i0 < ngp; i0 += 32) {
#pragma unroll
    for (int u = 0; u < 4; ++u) tile[warp + 8 * u][lane] = x[u];
    if (i0 + 32 < ngp) load(i0 + 32);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = warp + 8 * u;
      Gb[(long)s * ngp + i0 + lane] = tile[lane][s];
    }
    __syncthreads();
  }
}

// Node sums from the gathered rows: CTA (node v, (J, Lambda')), warp Omega; lane l takes the
// rows i = l, l + 32, ...: per row the stencil combination sum_s wst_s G[b][pix_s][i] in the
// state's precision (sixteen terms), times P-bar_(Omega+i)^Omega(cos gamma_v), the product
// and the sums over rows and lanes in FP64. Then the same helicity rotation. NCH = ngp / 32
// row chunks at compile time (all of them in flight per stencil point); NCH = 0: any ngp.
template <typename real, int NCH>
__global__ void __launch_bounds__(1024) k_prod_nodes_g(const real* __restrict__ Gs, int ng, int ngp,
                                                       int spad, int nn,
                                                       const int* __restrict__ pix,
                                                       const real* __restrict__ wst,
                                                       const real* __restrict__ pl, int ltop,
                                                       const double* __restrict__ T,
                                                       const double* __restrict__ jac,
                                                       const ProdGroup* __restrict__ groups,
                                                       const int* __restrict__ jl_group,
                                                       double* __restrict__ vout) {
  __shared__ double us[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x;
  const int g0 = jl_group[blockIdx.y];
  const ProdGroup G = groups[g0];          // Omega' = 0 group of this (J, Lambda')
  const int nom = G.nom;
  if (warp < nom) {
    const int b = G.b0 + warp * G.bstride;
    const real* gb = Gs + (long)b * spad * ngp + lane;
    const real* P = pl + ((long)v * ltop + warp) * ng;
    double acc = 0.0;
    if constexpr (NCH > 0) {
      real ts[NCH];
#pragma unroll
      for (int k = 0; k < NCH; ++k) ts[k] = 0;
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        const real* src = gb + pix[v * 16 + s] * ngp;
        const real w = wst[v * 16 + s];
#pragma unroll
        for (int k = 0; k < NCH; ++k) ts[k] += w * src[32 * k];
      }
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        const int i = 32 * k + lane;
        const real p = i < ng ? P[i] : (real)0;
        acc = fma((double)p, (double)ts[k], acc);
      }
    } else {
      for (int i0 = 0; i0 < ngp; i0 += 32) {
        real ts = 0;
#pragma unroll
        for (int s = 0; s < 16; ++s) ts += wst[v * 16 + s] * gb[pix[v * 16 + s] * ngp + i0];
        const int i = i0 + lane;
        const real p = i < ng ? P[i] : (real)0;
        acc = fma((double)p, (double)ts, acc);
      }
    }
    const double s = warp_sum(acc);
    if (lane == 0) us[warp] = s;
  }
  __syncthreads();
  rotate_node(us, v, g0, G, nn, T, jac, groups, vout);
}

// C_c = sum_v W[c][v] v'[group(c)][v], written to its cut column: four warps per channel
// (two channels per CTA), each warp a quarter of the nodes with two independent partial sums
// (the FP64 chain is the latency), then a fixed-order sum of the four warps (deterministic).
constexpr int kDotWarps = 4;
__global__ void __launch_bounds__(256) k_prod_dots(const double* __restrict__ vin, int nn,
                                                   const double* __restrict__ W,
                                                   const int2* __restrict__ chan, int nchan,
                                                   double* __restrict__ cut) {
  __shared__ double part[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int local = warp / kDotWarps, sub = warp % kDotWarps;
  const int c = blockIdx.x * (8 / kDotWarps) + local;
  double s = 0.0;
  if (c < nchan) {
    const int2 gc = chan[c];   // (group, cut column)
    const double* Wc = W + (long)c * nn;
    const double* vg = vin + (long)gc.x * nn;
    double s0 = 0.0, s1 = 0.0;
    int n = sub * 32 + lane;
    for (; n + 32 * kDotWarps < nn; n += 64 * kDotWarps) {
      s0 += Wc[n] * vg[n];
      s1 += Wc[n + 32 * kDotWarps] * vg[n + 32 * kDotWarps];
    }
    if (n < nn) s0 += Wc[n] * vg[n];
    s = warp_sum(s0 + s1);
  }
  if (lane == 0) part[warp] = s;
  __syncthreads();
  if (threadIdx.x < 8 / kDotWarps) {
    const int cc = blockIdx.x * (8 / kDotWarps) + threadIdx.x;
    if (cc < nchan) {
      double t = 0.0;
      for (int w = 0; w < kDotWarps; ++w) t += part[threadIdx.x * kDotWarps + w];
      cut[chan[cc].y] = t;
    }
  }
}

}  // namespace

template <typename real>
cudaError_t launch_products(const real* q, int ng, int nr, int NR, int nn, const int* idx,
                            const double* w, const real* pl, int ltop, const double* T,
                            const double* jac, const ProdGroup* groups, const int* jl_group,
                            int njl, int max_nom, double* vbuf, const double* W, const int2* chan,
                            int nchan, double* cut_slot, const ProdGather<real>* gather,
                            cudaStream_t st) {
  if (nchan == 0) return cudaSuccess;
  dim3 g1((unsigned)nn, (unsigned)njl);
  if (gather != nullptr) {
    const ProdGather<real>& pg = *gather;
    dim3 g0((unsigned)(pg.spad / 32), (unsigned)pg.nblk);
    k_prod_gather<real><<<g0, 256, 0, st>>>(q, ng, (long)nr * NR, pg.pts, pg.spad, pg.ngp,
                                            pg.blocks, pg.G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
#define NODES_G(nch)                                                                         \
  k_prod_nodes_g<real, nch><<<g1, 32 * max_nom, 0, st>>>(pg.G, ng, pg.ngp, pg.spad, nn, pg.pix, \
                                                         pg.wst, pl, ltop, T, jac, groups,     \
                                                         jl_group, vbuf)
    switch (pg.ngp / 32) {
      case 1: NODES_G(1); break;
      case 2: NODES_G(2); break;
      case 3: NODES_G(3); break;
      case 4: NODES_G(4); break;
      case 5: NODES_G(5); break;
      case 6: NODES_G(6); break;
      default: NODES_G(0); break;
    }
#undef NODES_G
  } else {
    k_prod_nodes<real><<<g1, 32 * max_nom, 0, st>>>(q, ng, nr, NR, nn, idx, w, pl, ltop, T, jac,
                                                    groups, jl_group, vbuf);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_prod_dots<<<(nchan + 1) / 2, 256, 0, st>>>(vbuf, nn, W, chan, nchan, cut_slot);
  return cudaGetLastError();
}

template cudaError_t launch_products<float>(const float*, int, int, int, int, const int*,
                                            const double*, const float*, int, const double*,
                                            const double*, const ProdGroup*, const int*, int, int,
                                            double*, const double*, const int2*, int, double*,
                                            const ProdGather<float>*, cudaStream_t);
template cudaError_t launch_products<double>(const double*, int, int, int, int, const int*,
                                             const double*, const double*, int, const double*,
                                             const double*, const ProdGroup*, const int*, int,
                                             int, double*, const double*, const int2*, int,
                                             double*, const ProdGather<double>*, cudaStream_t);

}  // namespace mw3
