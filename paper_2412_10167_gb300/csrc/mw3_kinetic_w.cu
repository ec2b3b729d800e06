// Warp-level radial kinetic kernels for line lengths N = R * 32 (R = 1, 2, 3, 4, 6, 8, 12, 16).
//
// Same operator as mw3_kinetic.cu (DST-II kinetic of the sine DVR through a length-N
// complex FFT carrying two real lines), but each line pair is transformed by one warp
// entirely in registers: lane t holds elements n = t + 32 s (s < R); a forward FFT is
//   (1) an R-point DFT over s in registers, (2) twiddles w_N^(t k2), (3) a 32-point DFT
//   across the lanes by decimation in frequency with __shfl_xor_sync butterflies,
// leaving X[k2 + R bitrev5(t)] in lane t, slot k2; the inverse runs the three steps
// backwards (decimation in time across lanes first). No block-wide barrier is taken
// inside a transform. Tiles are staged through shared memory so that global loads and
// stores stay coalesced (row tiles for R, [nr x C] column tiles for r).
#include <cuda_runtime.h>

#include <algorithm>

#include "mw3_internal.h"
#include "mw3_wdft.cuh"

namespace mw3 {
namespace {


__device__ __forceinline__ int bitrev5(int t) { return (int)(__brev((unsigned)t) >> 27); }

template <typename T>
__device__ __forceinline__ cpx<T> shfl_xor(cpx<T> v, int d) {
  return {__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d)};
}
template <typename T>
__device__ __forceinline__ cpx<T> shfl_from(cpx<T> v, int src) {
  return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// Per-CTA shared tables laid out so that the 32 lanes of a warp read 32 consecutive
// entries (no bank conflicts): for slot k2 and lane t, w = exp(-2 pi i / N),
//   twk[k2][t] = w^(t k2)                           twiddles between the DFT levels
//   tws[i][t]  = w^((t mod d) N / 2d) on lanes with bit d set, 1 elsewhere (d = 16 >> i)
//   fk[k2][k1], sk[k2][k1]   spectral scale of index k = k2 + R k1 (see wscale)
template <typename T, int R>
struct WTables {
  cpx<T> twk[R][32];
  cpx<T> tws[5][32];
  cpx<T> fk[R][32];
  T sk[R][32];
};

template <typename T, int R>
__device__ __forceinline__ void load_tables(WTables<T, R>& tb, const cpx<T>* __restrict__ twg,
                                            const cpx<T>* __restrict__ phg,
                                            const T* __restrict__ lamg) {
  constexpr int N = 32 * R;
  for (int e = threadIdx.x; e < R * 32; e += blockDim.x) {
    const int k2 = e >> 5, t = e & 31;
    tb.twk[k2][t] = twg[t * k2];
    // sigma_k = (lambda_(N-k) + lambda_k) / 2, f_k = (lambda_(N-k) - lambda_k) / 2 exp(i pi k / N),
    // exp(i pi k / N) = conj(ph_k)^2 with ph_k = exp(-i pi k / 2N)
    const int k = k2 + R * t;
    const T lr = lamg[N - k], li = lamg[k];
    const cpx<T> e1 = phg[k];
    const cpx<T> e2 = {e1.x * e1.x - e1.y * e1.y, -(T)2 * e1.x * e1.y};
    const T dl = (T)0.5 * (lr - li);
    tb.sk[k2][t] = (T)0.5 * (lr + li);
    tb.fk[k2][t] = cpx<T>{dl * e2.x, dl * e2.y};
  }
  for (int e = threadIdx.x; e < 5 * 32; e += blockDim.x) {
    const int i = e >> 5, t = e & 31, d = 16 >> i;
    tb.tws[i][t] = (t & d) ? twg[(t & (d - 1)) * (N / (2 * d))] : cpx<T>{(T)1, (T)0};
  }
}

// Forward FFT of the distributed sequence (lane t, slot s) = z[t + 32 s];
// out: lane t, slot k2 = Z[k2 + R bitrev5(t)]. Cross-lane decimation in frequency:
// the lane without bit d keeps v + p, the lane with it (p - v) w; both as (p + s v) w
// with s = -1 on the lane with bit d and w = 1 on the other.
template <typename T, int R>
__device__ __forceinline__ void wfft_fwd(cpx<T>* v, int t, const WTables<T, R>& tb) {
  dftR<T, R>(v, (T)-1);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cm(v[k2], tb.twk[k2][t]);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int d = 16 >> i;
    const T sg = (t & d) ? (T)-1 : (T)1;
    const cpx<T> w = tb.tws[i][t];
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const cpx<T> p = shfl_xor(v[k2], d);
      const cpx<T> r = {p.x + sg * v[k2].x, p.y + sg * v[k2].y};
      v[k2] = (d > 1) ? cm(r, w) : r;   // w = 1 in the last stage
    }
  }
}

// Unnormalised inverse of wfft_fwd: in lane t, slot k2 = W[k2 + R bitrev5(t)];
// out lane t, slot s = N * IDFT(W)[t + 32 s]. Cross-lane decimation in time: the lane
// with bit d first multiplies by conj(w); then both take p + s v.
template <typename T, int R>
__device__ __forceinline__ void wfft_inv(cpx<T>* v, int t, const WTables<T, R>& tb) {
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    const int d = 16 >> i;
    const T sg = (t & d) ? (T)-1 : (T)1;
    const cpx<T> w = tb.tws[i][t];
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const cpx<T> u = (d > 1) ? cmc(v[k2], w) : v[k2];
      const cpx<T> p = shfl_xor(u, d);
      v[k2] = {p.x + sg * u.x, p.y + sg * u.y};
    }
  }
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmc(v[k2], tb.twk[k2][t]);
  dftR<T, R>(v, (T)1);
}

// Spectral scaling between the transforms. For the pair spectrum Z (two real lines
// a + i b), the DST-kinetic of mw3_kinetic.cu (split Z into the line spectra, twiddle
// by exp(-i pi k / 2N), scale real and imaginary parts by lambda_(N-k) and lambda_k,
// twiddle back, recombine) reduces to
//   W_k = sigma_k Z_k + f_k Z_(N-k),  sigma_k = (lambda_(N-k) + lambda_k) / 2,
//   f_k = (lambda_(N-k) - lambda_k) / 2 exp(i pi k / N).
template <typename T, int R>
__device__ __forceinline__ void wscale(cpx<T>* v, int t, const WTables<T, R>& tb) {
  const int k1 = bitrev5(t);
  cpx<T> o[R];
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) {
    // partner index N - k: slot (R - k2) % R, k1' = k2 ? 31 - k1 : (32 - k1) % 32
    const int k1p = k2 ? 31 - k1 : ((32 - k1) & 31);
    o[k2] = shfl_from(v[(R - k2) % R], bitrev5(k1p));
  }
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) {
    const T sgm = tb.sk[k2][k1];
    const cpx<T> f = tb.fk[k2][k1];
    const cpx<T> fz = cm(f, o[k2]);
    v[k2] = {sgm * v[k2].x + fz.x, sgm * v[k2].y + fz.y};
  }
}

__device__ __forceinline__ int iperm(int n, int N) { return n < N / 2 ? 2 * n : 2 * (N - 1 - n) + 1; }

// One line pair through forward FFT, spectral scale and inverse FFT. Element i of
// line a sits at xa[i * stride], of line b at xb[i * stride]; the result
// overwrites them (sign (-1)^i and the permutation of the DST-via-FFT on both
// sides).
template <typename T, int R>
__device__ __forceinline__ void pair_kinetic(T* xa, T* xb, int stride, int lane,
                                             const WTables<T, R>& tb) {
  constexpr int N = 32 * R;
  cpx<T> v[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int i = iperm(lane + 32 * s, N);
    const T sg = (i & 1) ? (T)-1 : (T)1;
    v[s] = {sg * xa[i * stride], sg * xb[i * stride]};
  }
  wfft_fwd<T, R>(v, lane, tb);
  wscale<T, R>(v, lane, tb);
  wfft_inv<T, R>(v, lane, tb);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int i = iperm(lane + 32 * s, N);
    const T sg = (i & 1) ? (T)-1 : (T)1;
    xa[i * stride] = sg * v[s].x;
    xb[i * stride] = sg * v[s].y;
  }
}

// Resident CTAs per SM asked of the register allocator (8 warps each).
template <typename T, int R>
constexpr int kMinBlocks = (sizeof(T) == 4 && R <= 8) ? 4 : (R <= 4 ? 3 : 1);

// 16-byte vector of T (float4 / double2).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};

// R direction, persistent: each CTA loads the FFT tables once and walks blocks of 16
// consecutive rows of length N (8 warps, one line pair each) with stride gridDim.x. The next
// block's rows are copied into the second shared buffer with cp.async while this block's
// transforms run; results leave with 16-byte vector stores (live rows only).
template <typename T, int R>
__global__ void __launch_bounds__(256, kMinBlocks<T, R>) k_rows_w(const T* __restrict__ q, T* __restrict__ t,
                                                long nrows, const cpx<T>* __restrict__ twg,
                                                const cpx<T>* __restrict__ phg,
                                                const T* __restrict__ lamg,
                                                const DevBlock* __restrict__ blocks, int ng,
                                                int nr) {
  constexpr int N = 32 * R;
  constexpr int ROWS = 16;
  using V = typename Vec16<T>::type;
  constexpr int VE = 16 / sizeof(T);          // elements per vector
  constexpr int NV = ROWS * N / VE;           // vectors per block of rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WTables<T, R>& tb = *reinterpret_cast<WTables<T, R>*>(smem_raw);
  T* tiles = reinterpret_cast<T*>(smem_raw + ((sizeof(WTables<T, R>) + 15) / 16) * 16);  // [2][ROWS * N]
  __shared__ int live[ROWS];
  load_tables<T, R>(tb, twg, phg, lamg);
  const long nrb = (nrows + ROWS - 1) / ROWS;
  auto prefetch = [&](long rb, int buf) {
    if (rb < nrb) {
      const long row0 = rb * ROWS;
      const long nvalid = min((long)ROWS, nrows - row0) * N / VE;
      const T* src = q + row0 * N;
      T* dst = tiles + buf * ROWS * N;
      for (int e = threadIdx.x; e < nvalid; e += blockDim.x)
        cp_async16_ca<T>(dst + (long)e * VE, src + (long)e * VE);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int buf = 0;
  prefetch(blockIdx.x, 0);
  for (long rb = blockIdx.x; rb < nrb; rb += gridDim.x, buf ^= 1) {
    __syncthreads();                              // the other buffer's last readers are done
    prefetch(rb + gridDim.x, buf ^ 1);
    const long row0 = rb * ROWS;
    if (threadIdx.x < ROWS) {
      const long row = row0 + threadIdx.x;
      const long plane = row / nr;
      live[threadIdx.x] = row < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // this block's rows
    __syncthreads();
    T* tile = tiles + buf * ROWS * N;
    // a pair never straddles planes (nr is even), so one flag covers both rows
    if (live[2 * warp]) pair_kinetic<T, R>(tile + 2 * warp * N, tile + (2 * warp + 1) * N, 1, lane, tb);
    __syncthreads();
    const long nvalid = min((long)ROWS, nrows - row0) * N / VE;
    const V* sv = reinterpret_cast<const V*>(tile);
    V* tv = reinterpret_cast<V*>(t + row0 * N);
    for (int e = threadIdx.x; e < NV; e += blockDim.x)
      if (e < nvalid && live[(e * VE) / N]) tv[e] = sv[e];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// r direction: one CTA = one (block, gamma) plane, columns [c0, c0 + C); N = nr.
template <typename T, int R, int C>
__global__ void __launch_bounds__(256, kMinBlocks<T, R>) k_cols_w(
    const T* __restrict__ q, T* __restrict__ t, int NR, const cpx<T>* __restrict__ twg,
    const cpx<T>* __restrict__ phg, const T* __restrict__ lamg, int ng,
    const T* __restrict__ wpsi, const T* __restrict__ wdpsi, T* __restrict__ cut,
    const DevBlock* __restrict__ blocks, const int* __restrict__ ncut_J, int m_inf,
    T* __restrict__ qcol) {
  constexpr int N = 32 * R;
  constexpr int LD = C + 1;
  constexpr int NOUT = 2 * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WTables<T, R>& tb = *reinterpret_cast<WTables<T, R>*>(smem_raw);
  T* tile = reinterpret_cast<T*>(smem_raw + sizeof(WTables<T, R>));   // [N][C + 1]
  T* part = tile + N * LD;                                            // [4][2C]
  const long plane = blockIdx.y;
  const int b = (int)(plane / ng);
  const int n = (int)(plane - (long)b * ng);
  if (n >= blocks[b].nrow) return;
  load_tables<T, R>(tb, twg, phg, lamg);
  const int c0 = blockIdx.x * C;
  const T* qp = q + plane * (long)N * NR;
  T* tp = t + plane * (long)N * NR;
  constexpr int PER = (N * C + 255) / 256;
  constexpr int CH = PER < 8 ? PER : 8;                         // loads in flight per thread
  using V = typename Vec16<T>::type;
  constexpr int VE = 16 / sizeof(T);
  constexpr int NV = N * C / VE;                                // 16-byte vectors per tile
  constexpr int PERV = (NV + 255) / 256;
  constexpr int CHV = PERV < 8 ? PERV : 8;
  // 16-byte vector loads when rows are vector-aligned (C is a multiple of VE; a vector
  // is then entirely inside or outside the grid)
  const bool vec = (NR % VE) == 0;
  if (vec) {
    for (int u0 = 0; u0 < PERV; u0 += CHV) {
      V z[CHV];
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / (C / VE), m = c0 + (e % (C / VE)) * VE;
        z[u] = (e < NV && m < NR) ? *reinterpret_cast<const V*>(qp + (long)kr * NR + m) : V{};
      }
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        if (e < NV) {
          T* dst = tile + (e / (C / VE)) * LD + (e % (C / VE)) * VE;
          const T* zs = reinterpret_cast<const T*>(&z[u]);
#pragma unroll
          for (int v = 0; v < VE; ++v) dst[v] = zs[v];
        }
      }
    }
  } else {
    for (int u0 = 0; u0 < PER; u0 += CH) {
      T z[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / C, m = c0 + e % C;
        z[u] = (e < N * C && m < NR) ? qp[(long)kr * NR + m] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        if (e < N * C) tile[(e / C) * LD + e % C] = z[u];
      }
    }
  }
  __syncthreads();
  if (cut != nullptr) {
    constexpr int SEG = (N + 3) / 4;
    for (int o = threadIdx.x; o < 4 * NOUT; o += blockDim.x) {
      const int seg = o / NOUT, oc = o % NOUT, c = oc >> 1;
      const T* w = (oc & 1) ? wdpsi : wpsi;
      T s = 0;
      const int k0 = seg * SEG, k1 = min(N, k0 + SEG);
      for (int kr = k0; kr < k1; ++kr) s += w[kr] * tile[kr * LD + c];
      part[seg * NOUT + oc] = s;
    }
  }
  if (qcol != nullptr && m_inf >= c0 && m_inf < c0 + C) {
    for (int kr = threadIdx.x; kr < N; kr += blockDim.x) qcol[plane * N + kr] = tile[kr * LD + (m_inf - c0)];
  }
  __syncthreads();
  if (cut != nullptr) {
    const DevBlock B = blocks[b];
    const long ncut = ncut_J[B.iJ];
    for (int oc = threadIdx.x; oc < NOUT; oc += blockDim.x) {
      const int m = c0 + (oc >> 1);
      if (m >= NR) continue;
      const T s = ((part[oc] + part[NOUT + oc]) + part[2 * NOUT + oc]) + part[3 * NOUT + oc];
      cut[B.cutcol + (long)(oc & 1) * ncut + (long)n * NR + m] = s;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < C / 2; p += blockDim.x / 32)
    pair_kinetic<T, R>(tile + 2 * p, tile + 2 * p + 1, LD, lane, tb);
  __syncthreads();
  if (vec) {
    for (int u0 = 0; u0 < PERV; u0 += CHV) {
      V z[CHV];
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / (C / VE), m = c0 + (e % (C / VE)) * VE;
        z[u] = (e < NV && m < NR) ? *reinterpret_cast<const V*>(tp + (long)kr * NR + m) : V{};
      }
#pragma unroll
      for (int u = 0; u < CHV; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / (C / VE), m = c0 + (e % (C / VE)) * VE;
        if (e < NV && m < NR) {
          T* zs = reinterpret_cast<T*>(&z[u]);
          const T* src = tile + kr * LD + (e % (C / VE)) * VE;
#pragma unroll
          for (int v = 0; v < VE; ++v) zs[v] += src[v];
          *reinterpret_cast<V*>(tp + (long)kr * NR + m) = z[u];
        }
      }
    }
  } else {
    for (int u0 = 0; u0 < PER; u0 += CH) {
      T z[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / C, m = c0 + e % C;
        z[u] = (e < N * C && m < NR) ? tp[(long)kr * NR + m] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int e = threadIdx.x + 256 * (u0 + u);
        const int kr = e / C, m = c0 + e % C;
        if (e < N * C && m < NR) tp[(long)kr * NR + m] = z[u] + tile[kr * LD + e % C];
      }
    }
  }
}


// FP64 lines stop at R = 8: beyond that a thread's registers would spill.
template <typename T, int R>
constexpr bool kWarpSupported = sizeof(T) == 4 || R <= 8;

template <typename T, int R>
bool rows_w(const T* q, T* t, long nrows, const void* tw, const void* ph, const T* lam,
            const DevBlock* blocks, int ng, int nr, cudaStream_t st, cudaError_t* err) {
  if constexpr (!kWarpSupported<T, R>) {
    return false;
  } else {
    constexpr int N = 32 * R;
    const size_t sm = ((sizeof(WTables<T, R>) + 15) / 16) * 16 + 2 * 16 * (size_t)N * sizeof(T);
    static bool attr = false;
    static int nsm = 0;
    if (!attr) {
      cudaFuncSetAttribute(k_rows_w<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      attr = true;
    }
    const long nrb = (nrows + 15) / 16;
    const unsigned grid = (unsigned)std::min<long>(nrb, (long)std::max(nsm, 1) * kMinBlocks<T, R>);
    k_rows_w<T, R><<<grid, 256, sm, st>>>(q, t, nrows, static_cast<const cpx<T>*>(tw),
                                          static_cast<const cpx<T>*>(ph), lam, blocks, ng, nr);
    *err = cudaGetLastError();
    return true;
  }
}

template <typename T, int R, int C>
bool cols_wc(const T* q, T* t, long nplanes, int NR, const void* tw, const void* ph,
             const T* lam, int ng, const T* wpsi, const T* wdpsi, T* cut,
             const DevBlock* blocks, const int* ncut_J, int m_inf, T* qcol, cudaStream_t st,
             cudaError_t* err) {
  constexpr int N = 32 * R;
  const size_t sm = sizeof(WTables<T, R>) + sizeof(T) * ((size_t)N * (C + 1) + 8 * (size_t)C);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cols_w<T, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  dim3 grid((unsigned)((NR + C - 1) / C), (unsigned)nplanes);
  k_cols_w<T, R, C><<<grid, 256, sm, st>>>(q, t, NR, static_cast<const cpx<T>*>(tw),
                                           static_cast<const cpx<T>*>(ph), lam, ng, wpsi, wdpsi,
                                           cut, blocks, ncut_J, m_inf, qcol);
  *err = cudaGetLastError();
  return true;
}

template <typename T, int R>
bool cols_w(const T* q, T* t, long nplanes, int NR, const void* tw, const void* ph,
            const T* lam, int C, int ng, const T* wpsi, const T* wdpsi, T* cut,
            const DevBlock* blocks, const int* ncut_J, int m_inf, T* qcol, cudaStream_t st,
            cudaError_t* err) {
  if constexpr (!kWarpSupported<T, R>) {
    return false;
  } else {
    switch (C) {
#define CC(c)                                                                                 \
  case c:                                                                                     \
    return cols_wc<T, R, c>(q, t, nplanes, NR, tw, ph, lam, ng, wpsi, wdpsi, cut, blocks,     \
                            ncut_J, m_inf, qcol, st, err);
      CC(8) CC(16) CC(32)
#undef CC
      default: return false;   // other column tiles: the shared-memory FFT kernels
    }
  }
}

// Half-warp form (FP32, N = 16 N1): the pair transform and its tables are in mw3_wdft.cuh.

// R direction, persistent: blocks of 32 rows (16 line pairs, one per half-warp of the 256
// threads), the next block copied into the second buffer with cp.async while this one
// transforms. Row pitch N + 8 floats: the rows of the two half-warps of a warp start 16
// banks apart, so their exchanges do not collide.
template <int N1, bool SHFL>
__global__ void __launch_bounds__(256, 3) k_rows_hw(const float* __restrict__ q, float* __restrict__ t,
                                                 long nrows, const cpx<float>* __restrict__ twg,
                                                 const cpx<float>* __restrict__ phg,
                                                 const float* __restrict__ lamg,
                                                 const DevBlock* __restrict__ blocks, int ng,
                                                 int nr) {
  constexpr int N = 16 * N1;
  constexpr int ROWS = 32;
  constexpr int P = N + 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HwTables<N1>& tb = *reinterpret_cast<HwTables<N1>*>(smem_raw);
  float* tiles = reinterpret_cast<float*>(smem_raw + ((sizeof(HwTables<N1>) + 15) / 16) * 16);
  __shared__ int live[ROWS];
  hw_load_tables<N1>(tb, twg, phg, lamg);
  const long nrb = (nrows + ROWS - 1) / ROWS;
  auto prefetch = [&](long rb, int buf) {
    if (rb < nrb) {
      const long row0 = rb * ROWS;
      const int nv = (int)min((long)ROWS, nrows - row0) * (N / 4);
      const float* src = q + row0 * N;
      float* dst = tiles + buf * ROWS * P;
      for (int e = threadIdx.x; e < nv; e += blockDim.x) {
        const int r = e / (N / 4), c4 = (e - r * (N / 4)) * 4;
        cp_async16_ca<float>(dst + r * P + c4, src + (long)r * N + c4);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int hw = threadIdx.x >> 4, lane = threadIdx.x & 15;
  int buf = 0;
  prefetch(blockIdx.x, 0);
  for (long rb = blockIdx.x; rb < nrb; rb += gridDim.x, buf ^= 1) {
    __syncthreads();                              // the other buffer's last readers are done
    prefetch(rb + gridDim.x, buf ^ 1);
    const long row0 = rb * ROWS;
    if (threadIdx.x < ROWS) {
      const long row = row0 + threadIdx.x;
      const long plane = row / nr;
      live[threadIdx.x] = row < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // this block's rows
    __syncthreads();
    float* tile = tiles + buf * ROWS * P;
    // a pair never straddles planes (nr is even), so one flag covers both rows
    if (live[2 * hw]) hw_pair_kinetic<N1, SHFL>(tile + 2 * hw * P, tile + (2 * hw + 1) * P, 1, lane,
                                                tb.tw16, tb.sig, tb.fk);
    __syncthreads();
    const int nv = (int)min((long)ROWS, nrows - row0) * (N / 4);
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
      const int r = e / (N / 4), c4 = (e - r * (N / 4)) * 4;
      if (live[r])
        *reinterpret_cast<float4*>(t + (row0 + r) * N + c4) =
            *reinterpret_cast<const float4*>(tile + r * P + c4);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// r direction: one CTA = one (block, gamma) plane and 32 columns [c0, c0 + 32); N = nr.
// Tile [N][33]: with the odd pitch, the 16 rows of an exchange fall in 16 banks, and the
// column pairs of a warp's two half-warps, (w, w + 8) and (w + 16, w + 24), start 16 banks
// apart. Flux cut (4-way split over r) and the R_inf column come from the tile first.
template <int N1, bool SHFL>
__global__ void __launch_bounds__(256) k_cols_hw(
    const float* __restrict__ q, float* __restrict__ t, int NR, const cpx<float>* __restrict__ twg,
    const cpx<float>* __restrict__ phg, const float* __restrict__ lamg, int ng,
    const float* __restrict__ wpsi, const float* __restrict__ wdpsi, float* __restrict__ cut,
    const DevBlock* __restrict__ blocks, const int* __restrict__ ncut_J, int m_inf,
    float* __restrict__ qcol) {
  constexpr int N = 16 * N1;
  constexpr int C = 32;
  constexpr int LD = C + 1;
  constexpr int NOUT = 2 * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HwTables<N1>& tb = *reinterpret_cast<HwTables<N1>*>(smem_raw);
  float* tile = reinterpret_cast<float*>(smem_raw + sizeof(HwTables<N1>));   // [N][C + 1]
  float* part = tile + N * LD;                                               // [4][2C]
  const long plane = blockIdx.y;
  const int b = (int)(plane / ng);
  const int n = (int)(plane - (long)b * ng);
  if (n >= blocks[b].nrow) return;
  hw_load_tables<N1>(tb, twg, phg, lamg);
  const int c0 = blockIdx.x * C;
  const float* qp = q + plane * (long)N * NR;
  float* tp = t + plane * (long)N * NR;
  constexpr int NV = N * C / 4;                                 // 16-byte vectors per tile
  constexpr int PERV = (NV + 255) / 256;
  constexpr int CHV = PERV < 8 ? PERV : 8;                      // loads in flight per thread
  const bool vec = (NR % 4) == 0;
  for (int u0 = 0; u0 < PERV; u0 += CHV) {
    float4 z[CHV];
#pragma unroll
    for (int u = 0; u < CHV; ++u) {
      const int e = threadIdx.x + 256 * (u0 + u);
      const int kr = e / (C / 4), m = c0 + (e % (C / 4)) * 4;
      if (e < NV && m < NR) {
        if (vec) {
          z[u] = *reinterpret_cast<const float4*>(qp + (long)kr * NR + m);
        } else {
          const float* s = qp + (long)kr * NR + m;
          z[u] = make_float4(s[0], m + 1 < NR ? s[1] : 0.0f, m + 2 < NR ? s[2] : 0.0f,
                             m + 3 < NR ? s[3] : 0.0f);
        }
      } else {
        z[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
    }
#pragma unroll
    for (int u = 0; u < CHV; ++u) {
      const int e = threadIdx.x + 256 * (u0 + u);
      if (e < NV) {
        float* dst = tile + (e / (C / 4)) * LD + (e % (C / 4)) * 4;
        dst[0] = z[u].x;
        dst[1] = z[u].y;
        dst[2] = z[u].z;
        dst[3] = z[u].w;
      }
    }
  }
  __syncthreads();
  if (cut != nullptr) {
    constexpr int SEG = (N + 3) / 4;
    for (int o = threadIdx.x; o < 4 * NOUT; o += blockDim.x) {
      const int seg = o / NOUT, oc = o % NOUT, c = oc >> 1;
      const float* w = (oc & 1) ? wdpsi : wpsi;
      float s = 0;
      const int k0 = seg * SEG, k1 = min(N, k0 + SEG);
      for (int kr = k0; kr < k1; ++kr) s += w[kr] * tile[kr * LD + c];
      part[seg * NOUT + oc] = s;
    }
  }
  if (qcol != nullptr && m_inf >= c0 && m_inf < c0 + C) {
    for (int kr = threadIdx.x; kr < N; kr += blockDim.x) qcol[plane * N + kr] = tile[kr * LD + (m_inf - c0)];
  }
  __syncthreads();
  if (cut != nullptr) {
    const DevBlock B = blocks[b];
    const long ncut = ncut_J[B.iJ];
    for (int oc = threadIdx.x; oc < NOUT; oc += blockDim.x) {
      const int m = c0 + (oc >> 1);
      if (m >= NR) continue;
      const float s = ((part[oc] + part[NOUT + oc]) + part[2 * NOUT + oc]) + part[3 * NOUT + oc];
      cut[B.cutcol + (long)(oc & 1) * ncut + (long)n * NR + m] = s;
    }
  }
  {
    const int h = threadIdx.x >> 4, lane = threadIdx.x & 15;
    const int ca = (h >> 1) + 16 * (h & 1);
    hw_pair_kinetic<N1, SHFL>(tile + ca, tile + ca + 8, LD, lane, tb.tw16, tb.sig, tb.fk);
  }
  __syncthreads();
  for (int u0 = 0; u0 < PERV; u0 += CHV) {
    float4 z[CHV];
#pragma unroll
    for (int u = 0; u < CHV; ++u) {
      const int e = threadIdx.x + 256 * (u0 + u);
      const int kr = e / (C / 4), m = c0 + (e % (C / 4)) * 4;
      z[u] = (vec && e < NV && m < NR) ? *reinterpret_cast<const float4*>(tp + (long)kr * NR + m)
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < CHV; ++u) {
      const int e = threadIdx.x + 256 * (u0 + u);
      const int kr = e / (C / 4), m = c0 + (e % (C / 4)) * 4;
      if (e < NV && m < NR) {
        const float* src = tile + kr * LD + (e % (C / 4)) * 4;
        if (vec) {
          float4 o = z[u];
          o.x += src[0];
          o.y += src[1];
          o.z += src[2];
          o.w += src[3];
          *reinterpret_cast<float4*>(tp + (long)kr * NR + m) = o;
        } else {
          for (int v = 0; v < 4 && m + v < NR; ++v) tp[(long)kr * NR + m + v] += src[v];
        }
      }
    }
  }
}

template <int N1, bool SHFL>
bool rows_hw(const float* q, float* t, long nrows, const void* tw, const void* ph,
             const float* lam, const DevBlock* blocks, int ng, int nr, cudaStream_t st,
             cudaError_t* err) {
  constexpr int N = 16 * N1;
  const size_t sm = ((sizeof(HwTables<N1>) + 15) / 16) * 16 + 2 * 32 * (size_t)(N + 8) * sizeof(float);
  static bool attr = false;
  static int nsm = 0, per_sm = 1;
  if (!attr) {
    cudaFuncSetAttribute(k_rows_hw<N1, SHFL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_hw<N1, SHFL>, 256, sm);
    per_sm = std::max(per_sm, 1);
    attr = true;
  }
  const long nrb = (nrows + 31) / 32;
  const unsigned grid = (unsigned)std::min<long>(nrb, (long)std::max(nsm, 1) * per_sm);
  k_rows_hw<N1, SHFL><<<grid, 256, sm, st>>>(q, t, nrows, static_cast<const cpx<float>*>(tw),
                                       static_cast<const cpx<float>*>(ph), lam, blocks, ng, nr);
  *err = cudaGetLastError();
  return true;
}

template <int N1, bool SHFL>
bool cols_hw(const float* q, float* t, long nplanes, int NR, const void* tw, const void* ph,
             const float* lam, int ng, const float* wpsi, const float* wdpsi, float* cut,
             const DevBlock* blocks, const int* ncut_J, int m_inf, float* qcol, cudaStream_t st,
             cudaError_t* err) {
  constexpr int N = 16 * N1;
  const size_t sm = sizeof(HwTables<N1>) + sizeof(float) * ((size_t)N * 33 + 8 * 32);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cols_hw<N1, SHFL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  dim3 grid((unsigned)((NR + 31) / 32), (unsigned)nplanes);
  k_cols_hw<N1, SHFL><<<grid, 256, sm, st>>>(q, t, NR, static_cast<const cpx<float>*>(tw),
                                       static_cast<const cpx<float>*>(ph), lam, ng, wpsi, wdpsi,
                                       cut, blocks, ncut_J, m_inf, qcol);
  *err = cudaGetLastError();
  return true;
}

}  // namespace

template <typename T>
bool kinetic_rows_warp(int N, const T* q, T* t, long nrows, const void* tw, const void* ph,
                       const T* lam, const DevBlock* blocks, int ng, int nr, cudaStream_t st,
                       cudaError_t* err, int form) {
  if constexpr (sizeof(T) == 4) {
    if (form >= 2) {
      const bool sh = form == 3;
      switch (N) {
#define HW(n1)                                                                               \
  case 16 * n1:                                                                              \
    return sh ? rows_hw<n1, true>(q, t, nrows, tw, ph, lam, blocks, ng, nr, st, err)         \
              : rows_hw<n1, false>(q, t, nrows, tw, ph, lam, blocks, ng, nr, st, err);
        HW(8) HW(12) HW(16)
#undef HW
        default: break;
      }
    }
  }
  switch (N) {
#define CASE(R) \
  case 32 * R: return rows_w<T, R>(q, t, nrows, tw, ph, lam, blocks, ng, nr, st, err);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(6) CASE(8) CASE(12) CASE(16)
#undef CASE
    default: return false;
  }
}

template <typename T>
bool kinetic_cols_warp(int N, const T* q, T* t, long nplanes, int NR, const void* tw,
                       const void* ph, const T* lam, int C, int ng, const T* wpsi,
                       const T* wdpsi, T* cut, const DevBlock* blocks, const int* ncut_J,
                       int m_inf, T* qcol, cudaStream_t st, cudaError_t* err, int form) {
  if constexpr (sizeof(T) == 4) {
    if (form >= 2) {
      const bool sh = form == 3;
      switch (N) {
#define HW(n1)                                                                                \
  case 16 * n1:                                                                               \
    return sh ? cols_hw<n1, true>(q, t, nplanes, NR, tw, ph, lam, ng, wpsi, wdpsi, cut, blocks, \
                                  ncut_J, m_inf, qcol, st, err)                               \
              : cols_hw<n1, false>(q, t, nplanes, NR, tw, ph, lam, ng, wpsi, wdpsi, cut,      \
                                   blocks, ncut_J, m_inf, qcol, st, err);
        HW(8) HW(12) HW(16)
#undef HW
        default: break;
      }
    }
  }
  switch (N) {
#define CASE(R)                                                                              \
  case 32 * R:                                                                               \
    return cols_w<T, R>(q, t, nplanes, NR, tw, ph, lam, C, ng, wpsi, wdpsi, cut, blocks,     \
                        ncut_J, m_inf, qcol, st, err);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(6) CASE(8) CASE(12) CASE(16)
#undef CASE
    default: return false;
  }
}

template bool kinetic_rows_warp<float>(int, const float*, float*, long, const void*, const void*,
                                       const float*, const DevBlock*, int, int, cudaStream_t,
                                       cudaError_t*, int);
template bool kinetic_rows_warp<double>(int, const double*, double*, long, const void*,
                                        const void*, const double*, const DevBlock*, int, int,
                                        cudaStream_t, cudaError_t*, int);
template bool kinetic_cols_warp<float>(int, const float*, float*, long, int, const void*,
                                       const void*, const float*, int, int, const float*,
                                       const float*, float*, const DevBlock*, const int*, int,
                                       float*, cudaStream_t, cudaError_t*, int);
template bool kinetic_cols_warp<double>(int, const double*, double*, long, int, const void*,
                                        const void*, const double*, int, int, const double*,
                                        const double*, double*, const DevBlock*, const int*, int,
                                        double*, cudaStream_t, cudaError_t*, int);

}  // namespace mw3
