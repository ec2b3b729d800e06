// Compile-time-sized versions of the radial kinetic kernels (same mathematics as
// mw3_kinetic.cu: DST-II kinetic through a length-N complex FFT carrying two real
// lines, spectral scaling by lambda_(N-k) / lambda_k, inverse FFT), for the line
// lengths of the configured grids. Other lengths use the runtime-plan kernels.
#include <cuda_runtime.h>

#include "mw3_fft.cuh"
#include "mw3_internal.h"

namespace mw3 {

namespace {

template <int N>
__device__ __forceinline__ int ppos(int i) { return (i & 1) ? N - 1 - (i >> 1) : (i >> 1); }

template <typename T, int N>
__device__ __forceinline__ void scale(const cpx<T>* __restrict__ z, cpx<T>* __restrict__ w, int P,
                                      const cpx<T>* __restrict__ ph, const T* __restrict__ lam) {
  for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
    const int p = idx / N;
    const int k = idx - p * N;
    const cpx<T> Zk = z[p * N + k];
    const cpx<T> Zn = z[p * N + (k == 0 ? 0 : N - k)];
    const cpx<T> Va = {(T)0.5 * (Zk.x + Zn.x), (T)0.5 * (Zk.y - Zn.y)};
    const cpx<T> Vb = {(T)0.5 * (Zk.y + Zn.y), (T)0.5 * (Zn.x - Zk.x)};
    const cpx<T> e = ph[k];
    const cpx<T> ec = {e.x, -e.y};
    const T lr = lam[N - k], li = lam[k];
    cpx<T> Pa = fftc::mul(e, Va), Pb = fftc::mul(e, Vb);
    cpx<T> Wa = fftc::mul(ec, cpx<T>{lr * Pa.x, li * Pa.y});
    cpx<T> Wb = fftc::mul(ec, cpx<T>{lr * Pb.x, li * Pb.y});
    w[p * N + k] = {Wa.x - Wb.y, Wa.y + Wb.x};
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_rows_t(const T* __restrict__ q, T* __restrict__ t,
                                                long nrows, const cpx<T>* __restrict__ twg,
                                                const cpx<T>* __restrict__ phg,
                                                const T* __restrict__ lamg, int P,
                                                const DevBlock* __restrict__ blocks, int ng,
                                                int nr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* ph = tw + N;
  T* lam = reinterpret_cast<T*>(ph + N);
  cpx<T>* za = reinterpret_cast<cpx<T>*>(lam + ((N + 2) & ~1));
  cpx<T>* zb = za + P * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twg[i];
    ph[i] = phg[i];
  }
  for (int i = threadIdx.x; i <= N; i += blockDim.x) lam[i] = lamg[i];
  const long row0 = 2L * blockIdx.x * P;
  for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
    const int p = idx / N;
    const int i = idx - p * N;
    const long ra = row0 + 2L * p;
    const long plane = ra / nr;
    const bool live = ra < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    T xa = 0, xb = 0;
    if (live) xa = q[ra * N + i];
    if (live && ra + 1 < nrows) xb = q[(ra + 1) * N + i];
    const T sg = (i & 1) ? (T)-1 : (T)1;
    za[p * N + ppos<N>(i)] = {sg * xa, sg * xb};
  }
  __syncthreads();
  cpx<T>* Z = fftc::fft<T, N>(za, zb, P, tw, (T)-1);
  cpx<T>* W = (Z == za) ? zb : za;
  scale<T, N>(Z, W, P, ph, lam);
  __syncthreads();
  cpx<T>* other = (W == za) ? zb : za;
  cpx<T>* Y = fftc::fft<T, N>(W, other, P, tw, (T)1);
  for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
    const int p = idx / N;
    const int i = idx - p * N;
    const long ra = row0 + 2L * p;
    const long plane = ra / nr;
    const bool live = ra < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    const T sg = (i & 1) ? (T)-1 : (T)1;
    const cpx<T> y = Y[p * N + ppos<N>(i)];
    if (live) t[ra * N + i] = sg * y.x;
    if (live && ra + 1 < nrows) t[(ra + 1) * N + i] = sg * y.y;
  }
}

// r direction: one CTA = one (block, gamma) plane, columns [c0, c0 + C), all N = nr rows.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_cols_t(
    const T* __restrict__ q, T* __restrict__ t, int NR, const cpx<T>* __restrict__ twg,
    const cpx<T>* __restrict__ phg, const T* __restrict__ lamg, int C, int ng,
    const T* __restrict__ wpsi, const T* __restrict__ wdpsi, T* __restrict__ cut,
    const DevBlock* __restrict__ blocks, const int* __restrict__ ncut_J, int m_inf,
    T* __restrict__ qcol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = C / 2;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* ph = tw + N;
  T* lam = reinterpret_cast<T*>(ph + N);
  cpx<T>* za = reinterpret_cast<cpx<T>*>(lam + ((N + 2) & ~1));
  cpx<T>* zb = za + P * N;
  T* part = reinterpret_cast<T*>(zb + P * N);  // [4][2C] partial cut sums
  const long plane = blockIdx.y;
  if ((int)(plane % ng) >= blocks[plane / ng].nrow) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twg[i];
    ph[i] = phg[i];
  }
  for (int i = threadIdx.x; i <= N; i += blockDim.x) lam[i] = lamg[i];
  const int c0 = blockIdx.x * C;
  const T* qp = q + plane * (long)N * NR;
  T* tp = t + plane * (long)N * NR;
  T* zar = reinterpret_cast<T*>(za);
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int kr = idx / C;
    const int c = idx - kr * C;
    const int m = c0 + c;
    T x = (m < NR) ? qp[(long)kr * NR + m] : (T)0;
    const T sg = (kr & 1) ? (T)-1 : (T)1;
    zar[2 * ((c >> 1) * N + ppos<N>(kr)) + (c & 1)] = sg * x;
  }
  __syncthreads();
  const int b = (int)(plane / ng);
  const int n = (int)(plane - (long)b * ng);
  if (cut != nullptr) {
    // 2C dot products of length N, split over 4 segments of kr, then summed in order
    const int nout = 2 * C;
    for (int o = threadIdx.x; o < 4 * nout; o += blockDim.x) {
      const int seg = o / nout;
      const int oc = o - seg * nout;
      const int c = oc >> 1;
      const T* w = (oc & 1) ? wdpsi : wpsi;
      T s = 0;
      const int k0 = seg * ((N + 3) / 4), k1 = min(N, k0 + (N + 3) / 4);
      for (int kr = k0; kr < k1; ++kr) {
        const T sg = (kr & 1) ? (T)-1 : (T)1;
        s += w[kr] * sg * zar[2 * ((c >> 1) * N + ppos<N>(kr)) + (c & 1)];
      }
      part[seg * nout + oc] = s;
    }
  }
  if (qcol != nullptr && m_inf >= c0 && m_inf < c0 + C) {
    const int c = m_inf - c0;
    for (int kr = threadIdx.x; kr < N; kr += blockDim.x) {
      const T sg = (kr & 1) ? (T)-1 : (T)1;
      qcol[plane * N + kr] = sg * zar[2 * ((c >> 1) * N + ppos<N>(kr)) + (c & 1)];
    }
  }
  __syncthreads();
  if (cut != nullptr) {
    const DevBlock B = blocks[b];
    const long ncut = ncut_J[B.iJ];
    for (int oc = threadIdx.x; oc < 2 * C; oc += blockDim.x) {
      const int m = c0 + (oc >> 1);
      if (m >= NR) continue;
      const int nout = 2 * C;
      const T s = ((part[oc] + part[nout + oc]) + part[2 * nout + oc]) + part[3 * nout + oc];
      cut[B.cutcol + (long)(oc & 1) * ncut + (long)n * NR + m] = s;
    }
  }
  cpx<T>* Z = fftc::fft<T, N>(za, zb, P, tw, (T)-1);
  cpx<T>* W = (Z == za) ? zb : za;
  scale<T, N>(Z, W, P, ph, lam);
  __syncthreads();
  cpx<T>* other = (W == za) ? zb : za;
  cpx<T>* Y = fftc::fft<T, N>(W, other, P, tw, (T)1);
  const T* yr = reinterpret_cast<const T*>(Y);
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int kr = idx / C;
    const int c = idx - kr * C;
    const int m = c0 + c;
    if (m >= NR) continue;
    const T sg = (kr & 1) ? (T)-1 : (T)1;
    tp[(long)kr * NR + m] += sg * yr[2 * ((c >> 1) * N + ppos<N>(kr)) + (c & 1)];
  }
}

template <typename T>
size_t smem_rows(int N, int P) {
  return sizeof(cpx<T>) * 2 * (size_t)N + sizeof(T) * (size_t)((N + 2) & ~1) +
         sizeof(cpx<T>) * 2 * (size_t)P * N;
}

template <typename T, int N>
cudaError_t rows_inst(const T* q, T* t, long nrows, const void* tw, const void* ph, const T* lam,
                      int P, const DevBlock* blocks, int ng, int nr, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rows_t<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  const long npairs = (nrows + 1) / 2;
  const unsigned grid = (unsigned)((npairs + P - 1) / P);
  k_rows_t<T, N><<<grid, 256, smem_rows<T>(N, P), st>>>(
      q, t, nrows, static_cast<const cpx<T>*>(tw), static_cast<const cpx<T>*>(ph), lam, P,
      blocks, ng, nr);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t cols_inst(const T* q, T* t, long nplanes, int NR, const void* tw, const void* ph,
                      const T* lam, int C, int ng, const T* wpsi, const T* wdpsi, T* cut,
                      const DevBlock* blocks, const int* ncut_J, int m_inf, T* qcol,
                      cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cols_t<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  const size_t sm = smem_rows<T>(N, C / 2) + sizeof(T) * 8 * (size_t)C;
  dim3 grid((unsigned)((NR + C - 1) / C), (unsigned)nplanes);
  k_cols_t<T, N><<<grid, 256, sm, st>>>(q, t, NR, static_cast<const cpx<T>*>(tw),
                                        static_cast<const cpx<T>*>(ph), lam, C, ng, wpsi, wdpsi,
                                        cut, blocks, ncut_J, m_inf, qcol);
  return cudaGetLastError();
}

}  // namespace

#define MW3_SIZES(X) X(20) X(24) X(36) X(40) X(48) X(60) X(64) X(128) X(192) X(256) X(384) X(512)

template <typename T>
bool kinetic_rows_fixed(int N, const T* q, T* t, long nrows, const void* tw, const void* ph,
                        const T* lam, int P, const DevBlock* blocks, int ng, int nr,
                        cudaStream_t st, cudaError_t* err) {
  switch (N) {
#define CASE(n) \
  case n: *err = rows_inst<T, n>(q, t, nrows, tw, ph, lam, P, blocks, ng, nr, st); return true;
    MW3_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

template <typename T>
bool kinetic_cols_fixed(int N, const T* q, T* t, long nplanes, int NR, const void* tw,
                        const void* ph, const T* lam, int C, int ng, const T* wpsi,
                        const T* wdpsi, T* cut, const DevBlock* blocks, const int* ncut_J,
                        int m_inf, T* qcol, cudaStream_t st, cudaError_t* err) {
  switch (N) {
#define CASE(n)                                                                               \
  case n:                                                                                     \
    *err = cols_inst<T, n>(q, t, nplanes, NR, tw, ph, lam, C, ng, wpsi, wdpsi, cut, blocks, \
                           ncut_J, m_inf, qcol, st);                                          \
    return true;
    MW3_SIZES(CASE)
#undef CASE
    default: return false;
  }
}

template bool kinetic_rows_fixed<float>(int, const float*, float*, long, const void*, const void*,
                                        const float*, int, const DevBlock*, int, int,
                                        cudaStream_t, cudaError_t*);
template bool kinetic_rows_fixed<double>(int, const double*, double*, long, const void*,
                                         const void*, const double*, int, const DevBlock*, int,
                                         int, cudaStream_t, cudaError_t*);
template bool kinetic_cols_fixed<float>(int, const float*, float*, long, int, const void*,
                                        const void*, const float*, int, int, const float*,
                                        const float*, float*, const DevBlock*, const int*, int,
                                        float*, cudaStream_t, cudaError_t*);
template bool kinetic_cols_fixed<double>(int, const double*, double*, long, int, const void*,
                                         const void*, const double*, int, int, const double*,
                                         const double*, double*, const DevBlock*, const int*,
                                         int, double*, cudaStream_t, cudaError_t*);

}  // namespace mw3
