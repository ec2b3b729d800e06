// Fused radial kinetic term of the mixed form: t = K_R c + K_r c for every live (block, i)
// plane in one launch (Section 2.2, the Hamiltonian's radial kinetic operators in the sine
// DVR; each applied as a DST-II, a diagonal scale and the inverse, as in mw3_kinetic_w.cu).
//
// The separate kernels move five state vectors per step (R pass: read c, write t; r pass:
// read c, read and write t). Here one thread-block cluster of CS CTAs owns one plane
// (nr x NR, R fastest) and moves two: c is read from HBM once per element (the second copy
// comes from L2, read by the partner CTA at the same time) and t is written once.
//   CTA q holds  A_q = all nr rows x the columns [q W, (q + 1) W)   (W = NR / CS), and
//                B_q = the rows [q H, (q + 1) H) x all NR columns    (H = nr / CS).
// The r-direction transforms run on the columns of A_q, the R-direction transforms on the
// rows of B_q, both in place and concurrently (one job list over the CTA's half-warps).
// After a cluster barrier CTA q writes t for its columns: t = B' + A', with A' from its own
// shared memory and B' from the CTA that owns each row, read through distributed shared
// memory. The flux cut psi(r*), d psi(r*) / dr and the R_inf column come from A_q before
// the transforms. Results are bitwise those of the separate half-warp kernels: the same
// pair transform on the same values, and t = K_R c + K_r c added in the same order.
//
// Shared memory: A pitch W + 1 (odd: the rows read by the 16 lanes of a column exchange
// fall in 16 banks, and the column pairs of a warp's two half-warps start 16 banks apart);
// B pitch NR + 8 (rows of a warp's two half-warps 16 banks apart; 16-byte aligned rows for
// cp.async). No spin-wait: the only waits are cp.async groups and hardware barriers, and a
// cluster leaves a dead plane (i >= rows of its block) as a whole before the first barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mw3_wdft.cuh"

namespace mw3 {
namespace {

__device__ __forceinline__ uint32_t cta_rank_in_cluster() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// every thread of every CTA of the cluster; release/acquire orders the shared-memory
// writes before the barrier with the distributed reads after it
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t dsmem_addr(const void* local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
  return r;
}

__device__ __forceinline__ float4 ld_dsmem4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

template <int N1R, int N1r, int CS>
struct RadialShape {
  static constexpr int NR = 16 * N1R;
  static constexpr int nr = 16 * N1r;
  static constexpr int W = NR / CS;
  static constexpr int H = nr / CS;
  static constexpr int PA = W + 1;
  static constexpr int PB = NR + 8;
  static constexpr size_t tabR = ((sizeof(HwTables<N1R>) + 15) / 16) * 16;
  static constexpr size_t tabr = ((sizeof(HwTables<N1r>) + 15) / 16) * 16;
  static constexpr size_t offA = tabR + tabr;
  static constexpr size_t offB = ((offA + sizeof(float) * (size_t)nr * PA + 15) / 16) * 16;
  static constexpr size_t offP = offB + sizeof(float) * (size_t)H * PB;
  static constexpr size_t smem = offP + sizeof(float) * 4 * 2 * (size_t)W;
  static constexpr bool valid = NR % CS == 0 && nr % CS == 0 && W % 32 == 0 && H % 2 == 0 &&
                                smem <= 227 * 1024;
};

template <int N1R, int N1r, int CS>
__global__ void __launch_bounds__(256) k_radial_hw(
    const float* __restrict__ q, float* __restrict__ t, int ng,
    const cpx<float>* __restrict__ twR, const cpx<float>* __restrict__ phR,
    const float* __restrict__ lamR, const cpx<float>* __restrict__ twr,
    const cpx<float>* __restrict__ phr, const float* __restrict__ lamr,
    const float* __restrict__ wpsi, const float* __restrict__ wdpsi, float* __restrict__ cut,
    const DevBlock* __restrict__ blocks, const int* __restrict__ ncut_J, int m_inf,
    float* __restrict__ qcol) {
  using S = RadialShape<N1R, N1r, CS>;
  constexpr int NR = S::NR, nr = S::nr, W = S::W, H = S::H, PA = S::PA, PB = S::PB;
  constexpr int NOUT = 2 * W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HwTables<N1R>& tbR = *reinterpret_cast<HwTables<N1R>*>(smem_raw);
  HwTables<N1r>& tbr = *reinterpret_cast<HwTables<N1r>*>(smem_raw + S::tabR);
  float* A = reinterpret_cast<float*>(smem_raw + S::offA);   // [nr][PA]
  float* B = reinterpret_cast<float*>(smem_raw + S::offB);   // [H][PB]
  float* part = reinterpret_cast<float*>(smem_raw + S::offP);   // [4][2W]
  const long plane = blockIdx.y;
  const int b = (int)(plane / ng);
  const int n = (int)(plane - (long)b * ng);
  if (n >= blocks[b].nrow) return;   // the whole cluster: every CTA sees the same plane
  const int qr = (int)cta_rank_in_cluster();
  const int c0 = qr * W, r0 = qr * H;
  const float* qp = q + plane * (long)nr * NR;
  float* tp = t + plane * (long)nr * NR;

  // B: H whole rows, contiguous in HBM, copied asynchronously while A is gathered
  {
    constexpr int NV = H * NR / 4;
    const float* src = qp + (long)r0 * NR;
    for (int e = threadIdx.x; e < NV; e += blockDim.x) {
      const int r = e / (NR / 4), c4 = (e - r * (NR / 4)) * 4;
      cp_async16_ca<float>(B + r * PB + c4, src + (long)r * NR + c4);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  hw_load_tables<N1R>(tbR, twR, phR, lamR);
  hw_load_tables<N1r>(tbr, twr, phr, lamr);
  // A: all rows, W columns (16-byte loads, odd pitch in shared memory)
  {
    constexpr int NV = nr * W / 4;
    constexpr int PERV = (NV + 255) / 256;
    constexpr int CHV = PERV < 8 ? PERV : 8;
    for (int u0 = 0; u0 < PERV; u0 += CHV) {
      float4 z[CHV];
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / (W / 4), m = (e % (W / 4)) * 4;
        z[u] = e < NV ? *reinterpret_cast<const float4*>(qp + (long)kr * NR + c0 + m)
                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        if (e < NV) {
          float* dst = A + (e / (W / 4)) * PA + (e % (W / 4)) * 4;
          dst[0] = z[u].x;
          dst[1] = z[u].y;
          dst[2] = z[u].z;
          dst[3] = z[u].w;
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // flux cut on the untransformed columns (4-way split over r, summed in a fixed order)
  if (cut != nullptr) {
    constexpr int SEG = (nr + 3) / 4;
    for (int o = threadIdx.x; o < 4 * NOUT; o += blockDim.x) {
      const int seg = o / NOUT, oc = o % NOUT, c = oc >> 1;
      const float* w = (oc & 1) ? wdpsi : wpsi;
      float s = 0;
      const int k0 = seg * SEG, k1 = min(nr, k0 + SEG);
      for (int kr = k0; kr < k1; ++kr) s += w[kr] * A[kr * PA + c];
      part[seg * NOUT + oc] = s;
    }
  }
  if (qcol != nullptr && m_inf >= c0 && m_inf < c0 + W) {
    for (int kr = threadIdx.x; kr < nr; kr += blockDim.x) qcol[plane * nr + kr] = A[kr * PA + (m_inf - c0)];
  }
  __syncthreads();
  if (cut != nullptr) {
    const DevBlock Bk = blocks[b];
    const long ncut = ncut_J[Bk.iJ];
    for (int oc = threadIdx.x; oc < NOUT; oc += blockDim.x) {
      const int m = c0 + (oc >> 1);
      const float s = ((part[oc] + part[NOUT + oc]) + part[2 * NOUT + oc]) + part[3 * NOUT + oc];
      cut[Bk.cutcol + (long)(oc & 1) * ncut + (long)n * NR + m] = s;
    }
  }
  // one job list over the half-warps: W / 2 column pairs of A (length nr), then H / 2 row
  // pairs of B (length NR). Column pair j = 16 g + 2 c + s: columns 32 g + c + 16 s and
  // that + 8, so the two half-warps of a warp start 16 banks apart.
  {
    constexpr int NJC = W / 2, NJ = W / 2 + H / 2;
    const int nh = blockDim.x >> 4, h = threadIdx.x >> 4, lane = threadIdx.x & 15;
    for (int j = h; j < NJ; j += nh) {
      if (j < NJC) {
        const int g = j >> 4, c = (j >> 1) & 7, s = j & 1;
        const int ca = 32 * g + c + 16 * s;
        hw_pair_kinetic<N1r, false>(A + ca, A + ca + 8, PA, lane, tbr.tw16, tbr.sig, tbr.fk);
      } else {
        const int p = j - NJC;
        hw_pair_kinetic<N1R, false>(B + 2 * p * PB, B + (2 * p + 1) * PB, 1, lane, tbR.tw16,
                                    tbR.sig, tbR.fk);
      }
    }
  }
  cluster_barrier();   // every CTA's K_R rows and K_r columns are complete
  // t[r][c0 + m] = B'_(owner of r)[r][c0 + m] + A'[r][m]; CTAs start at different owners
  {
    constexpr int NV = nr * W / 4;
    uint32_t Bremote[CS];
#pragma unroll
    for (int p = 0; p < CS; ++p) Bremote[p] = dsmem_addr(B, (uint32_t)p);
    for (int e0 = threadIdx.x; e0 < NV; e0 += blockDim.x) {
      int e = e0 + qr * (H * W / 4);
      if (e >= NV) e -= NV;
      const int r = e / (W / 4), m = (e - r * (W / 4)) * 4;
      const int owner = r / H;
      uint32_t base = Bremote[0];
#pragma unroll
      for (int p = 1; p < CS; ++p)
        if (owner == p) base = Bremote[p];
      const float4 bv = ld_dsmem4(base + (uint32_t)(((r - owner * H) * PB + c0 + m) * 4));
      const float* a = A + r * PA + m;
      float4 o;
      o.x = bv.x + a[0];
      o.y = bv.y + a[1];
      o.z = bv.z + a[2];
      o.w = bv.w + a[3];
      *reinterpret_cast<float4*>(tp + (long)r * NR + c0 + m) = o;
    }
  }
  cluster_barrier();   // no CTA leaves while a partner may still read its rows
}

template <int N1R, int N1r, int CS>
bool radial_launch(const float* q, float* t, long nplanes, const void* twR, const void* phR,
                   const float* lamR, const void* twr, const void* phr, const float* lamr,
                   int ng, const float* wpsi, const float* wdpsi, float* cut,
                   const DevBlock* blocks, const int* ncut_J, int m_inf, float* qcol,
                   cudaStream_t st, cudaError_t* err) {
  using S = RadialShape<N1R, N1r, CS>;
  if constexpr (!S::valid) {
    return false;
  } else {
    static int ok = -1;   // the cluster shape fits on this device
    if (ok < 0) {
      cudaFuncSetAttribute(k_radial_hw<N1R, N1r, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)S::smem);
      cudaLaunchConfig_t cfg{};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = CS;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(CS, 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = S::smem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      const cudaError_t e =
          cudaOccupancyMaxActiveClusters(&nclusters, k_radial_hw<N1R, N1r, CS>, &cfg);
      ok = (e == cudaSuccess && nclusters > 0) ? 1 : 0;
      (void)cudaGetLastError();
    }
    if (!ok) return false;
    if (q == nullptr) return true;   // query: the shape is built and fits on this device
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CS, (unsigned)nplanes, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = S::smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    *err = cudaLaunchKernelEx(&cfg, k_radial_hw<N1R, N1r, CS>, q, t, ng,
                              static_cast<const cpx<float>*>(twR),
                              static_cast<const cpx<float>*>(phR), lamR,
                              static_cast<const cpx<float>*>(twr),
                              static_cast<const cpx<float>*>(phr), lamr, wpsi, wdpsi, cut, blocks,
                              ncut_J, m_inf, qcol);
    return true;
  }
}

template <int N1R, int N1r>
bool radial_cs(int cs, const float* q, float* t, long nplanes, const void* twR, const void* phR,
               const float* lamR, const void* twr, const void* phr, const float* lamr, int ng,
               const float* wpsi, const float* wdpsi, float* cut, const DevBlock* blocks,
               const int* ncut_J, int m_inf, float* qcol, cudaStream_t st, cudaError_t* err) {
#define RL(c)                                                                                  \
  radial_launch<N1R, N1r, c>(q, t, nplanes, twR, phR, lamR, twr, phr, lamr, ng, wpsi, wdpsi, \
                             cut, blocks, ncut_J, m_inf, qcol, st, err)
  switch (cs) {
    case 2: return RL(2);
    case 4: return RL(4);
    case 8: return RL(8);
    default: return false;
  }
#undef RL
}

}  // namespace

// Cluster size for the grid when the caller asks for the automatic choice (cs = 1): the
// smallest of 2, 4, 8 whose shape is valid and leaves room for two CTAs per SM.
int radial_fused_default_cs(int NR, int nr) {
  for (int cs : {2, 4, 8}) {
    if (NR % cs || nr % cs) continue;
    const int W = NR / cs, H = nr / cs;
    if (W % 32 || H % 2) continue;
    // tables (<= 2 x 5 KB) + A + B + cut partials
    const size_t sm = 10240 + 4 * ((size_t)nr * (W + 1) + (size_t)H * (NR + 8) + 8 * (size_t)W);
    if (2 * (sm + 1024) <= 228 * 1024) return cs;
  }
  return 0;
}

// q == nullptr: only report whether a launch would happen (nothing is enqueued).
bool kinetic_radial_fused(int NR, int nr, int cs, const float* q, float* t, long nplanes,
                          const void* twR, const void* phR, const float* lamR, const void* twr,
                          const void* phr, const float* lamr, int ng, const float* wpsi,
                          const float* wdpsi, float* cut, const DevBlock* blocks,
                          const int* ncut_J, int m_inf, float* qcol, cudaStream_t st,
                          cudaError_t* err) {
  if (cs == 1) cs = radial_fused_default_cs(NR, nr);
  if (cs <= 0) return false;
#define RC(a, b)                                                                             \
  if (NR == 16 * a && nr == 16 * b)                                                          \
    return radial_cs<a, b>(cs, q, t, nplanes, twR, phR, lamR, twr, phr, lamr, ng, wpsi, wdpsi, \
                           cut, blocks, ncut_J, m_inf, qcol, st, err);
  RC(16, 12) RC(16, 16) RC(16, 8) RC(12, 8) RC(12, 12) RC(8, 8) RC(8, 12)
#undef RC
  return false;
}

}  // namespace mw3
