// Radial kinetic terms of the grid Hamiltonian (Section 2.1, item 2): on every
// R line and every r line, t = S^T diag(lambda) S x with S the orthonormal DST-II
// of the midpoint sine DVR and lambda_j = min(k_j^2 / 2 mass, cap).
//
// GPU formulation (our design, not the paper's FFTW call): the DST-II of a real
// line is the reversed DCT-II of (-1)^n x, and a DCT-II of length N is one
// complex FFT of length N of the permuted sequence v_n = x_2n, v_(N-1-n) = x_(2n+1)
// followed by a twiddle exp(-i pi k / 2N). Two real lines share one complex FFT
// (real part / imaginary part). Between the forward and inverse FFT the spectrum
// is scaled per DCT index k by lambda_(N-k) (real part of the twiddled value) and
// lambda_k (imaginary part), which is T = S^T diag(lambda) S written in that basis.
// The FFT is a shared-memory Stockham autosort transform with radices 4, 2, 3, 5.
//
// Loads and stores are coalesced along R; the r-direction kernel reads a tile of
// [nr x C] values of one (block, gamma) plane, so consecutive threads read
// consecutive R. The r kernel also evaluates the flux cut psi(r*), dpsi/dr(r*)
// (dot products of each r line with fixed weights) and copies the column at R_inf
// used by the channel projections.
#include <cuda_runtime.h>

#include "mw3_internal.h"

namespace mw3 {

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
// multiply by i*s (s = +-1)
template <typename T>
__device__ __forceinline__ cpx<T> cmuli(cpx<T> a, T s) { return {-a.y * s, a.x * s}; }

// In-register DFT of size R with exp(sign * 2 pi i r k / R).
template <typename T, int R>
__device__ __forceinline__ void small_dft(cpx<T>* v, T sign) {
  if constexpr (R == 2) {
    cpx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    const T h = (T)0.86602540378443864676;  // sqrt(3)/2
    cpx<T> a = v[0], b = v[1], c = v[2];
    cpx<T> t1 = cadd(b, c);
    cpx<T> t2 = {a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y};
    cpx<T> t3 = cmuli(cscale(csub(b, c), h), sign);
    v[0] = cadd(a, t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  } else if constexpr (R == 4) {
    cpx<T> a = v[0], b = v[1], c = v[2], d = v[3];
    cpx<T> s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = cmuli(csub(b, d), sign);
    v[0] = cadd(s0, s2);
    v[1] = cadd(s1, s3);
    v[2] = csub(s0, s2);
    v[3] = csub(s1, s3);
  } else {  // R == 5
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212;   // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312917;   // sin(4 pi / 5)
    cpx<T> a = v[0];
    cpx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    cpx<T> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    cpx<T> m1 = {a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
    cpx<T> m2 = {a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
    cpx<T> n1 = cmuli(cpx<T>{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y}, sign);
    cpx<T> n2 = cmuli(cpx<T>{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y}, sign);
    v[0] = cadd(a, cadd(t1, t2));
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
  }
}

// One Stockham stage on P lines of length N held contiguously (line stride N).
// tw[t] = exp(-2 pi i t / N); the inverse uses the conjugate.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const cpx<T>* __restrict__ in,
                                               cpx<T>* __restrict__ out, int P, int N, int Ns,
                                               const cpx<T>* __restrict__ tw, T sign) {
  const int nb = N / R;
  const int total = P * nb;
  const int tstride = N / (Ns * R);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int p = idx / nb;
    const int j = idx - p * nb;
    const int k = j % Ns;
    const cpx<T>* src = in + (long)p * N;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T> x = src[j + r * nb];
      if (r > 0) {
        cpx<T> w = tw[r * k * tstride];
        if (sign > 0) w.y = -w.y;  // inverse transform: conjugate twiddle
        x = cmul(x, w);
      }
      v[r] = x;
    }
    small_dft<T, R>(v, sign);
    cpx<T>* dst = out + (long)p * N + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns] = v[r];
  }
}

// Full transform; returns the buffer holding the result (a or b).
template <typename T>
__device__ cpx<T>* stockham(cpx<T>* a, cpx<T>* b, int P, const FFTPlan& plan,
                            const cpx<T>* tw, T sign) {
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    switch (R) {
      case 4: stockham_stage<T, 4>(a, b, P, plan.N, Ns, tw, sign); break;
      case 2: stockham_stage<T, 2>(a, b, P, plan.N, Ns, tw, sign); break;
      case 3: stockham_stage<T, 3>(a, b, P, plan.N, Ns, tw, sign); break;
      default: stockham_stage<T, 5>(a, b, P, plan.N, Ns, tw, sign); break;
    }
    __syncthreads();
    cpx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Spectral scaling between the two FFTs (see file header). z holds Z = FFT(va + i vb)
// for P pairs; writes W (whose inverse FFT gives the permuted, scaled result).
template <typename T>
__device__ void kinetic_scale(const cpx<T>* __restrict__ z, cpx<T>* __restrict__ w, int P,
                              int N, const cpx<T>* __restrict__ ph,
                              const T* __restrict__ lam) {
  for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
    const int p = idx / N;
    const int k = idx - p * N;
    const cpx<T> Zk = z[(long)p * N + k];
    const cpx<T> Zn = z[(long)p * N + (k == 0 ? 0 : N - k)];
    // spectra of the two real sequences
    const cpx<T> Va = {(T)0.5 * (Zk.x + Zn.x), (T)0.5 * (Zk.y - Zn.y)};
    const cpx<T> Vb = {(T)0.5 * (Zk.y + Zn.y), (T)0.5 * (Zn.x - Zk.x)};
    const cpx<T> e = ph[k];                 // exp(-i pi k / 2N)
    const cpx<T> ec = {e.x, -e.y};
    const T lr = lam[N - k], li = lam[k];   // lam[0] = 0
    cpx<T> Pa = cmul(e, Va), Pb = cmul(e, Vb);
    cpx<T> Wa = cmul(ec, cpx<T>{lr * Pa.x, li * Pa.y});
    cpx<T> Wb = cmul(ec, cpx<T>{lr * Pb.x, li * Pb.y});
    w[(long)p * N + k] = {Wa.x - Wb.y, Wa.y + Wb.x};
  }
}

__device__ __forceinline__ int perm_pos(int i, int N) { return (i & 1) ? N - 1 - (i >> 1) : (i >> 1); }

// ----------------------------------------------------------------- R direction
template <typename T>
__global__ void __launch_bounds__(256) k_kinetic_rows(const T* __restrict__ q, T* __restrict__ t,
                                                      long nrows, FFTPlan plan,
                                                      const cpx<T>* __restrict__ twg,
                                                      const cpx<T>* __restrict__ phg,
                                                      const T* __restrict__ lamg, int P,
                                                      const DevBlock* __restrict__ blocks,
                                                      int ng, int nr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = plan.N;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* ph = tw + N;
  T* lam = reinterpret_cast<T*>(ph + N);
  cpx<T>* za = reinterpret_cast<cpx<T>*>(lam + ((N + 2) & ~1));
  cpx<T>* zb = za + (long)P * N;
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
    T xa = 0, xb = 0;
    // a pair never straddles planes (nr is even); rows beyond a block's angular
    // functions are zero and are neither read nor written
    const long plane = ra / nr;
    const bool live = ra < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    if (live) xa = q[ra * N + i];
    if (live && ra + 1 < nrows) xb = q[(ra + 1) * N + i];
    const T sg = (i & 1) ? (T)-1 : (T)1;
    za[(long)p * N + perm_pos(i, N)] = {sg * xa, sg * xb};
  }
  __syncthreads();
  cpx<T>* Z = stockham<T>(za, zb, P, plan, tw, (T)-1);
  cpx<T>* W = (Z == za) ? zb : za;
  kinetic_scale<T>(Z, W, P, N, ph, lam);
  __syncthreads();
  cpx<T>* other = (W == za) ? zb : za;
  cpx<T>* Y = stockham<T>(W, other, P, plan, tw, (T)1);
  for (int idx = threadIdx.x; idx < P * N; idx += blockDim.x) {
    const int p = idx / N;
    const int i = idx - p * N;
    const long ra = row0 + 2L * p;
    const T sg = (i & 1) ? (T)-1 : (T)1;
    const cpx<T> y = Y[(long)p * N + perm_pos(i, N)];
    const long plane = ra / nr;
    const bool live = ra < nrows && (int)(plane % ng) < blocks[plane / ng].nrow;
    if (live) t[ra * N + i] = sg * y.x;
    if (live && ra + 1 < nrows) t[(ra + 1) * N + i] = sg * y.y;
  }
}

// ----------------------------------------------------------------- r direction
// One CTA: one (block, gamma) plane, columns [c0, c0 + C) of R, all nr rows.
template <typename T>
__global__ void __launch_bounds__(256) k_kinetic_cols(
    const T* __restrict__ q, T* __restrict__ t, int nr, int NR, FFTPlan plan,
    const cpx<T>* __restrict__ twg, const cpx<T>* __restrict__ phg, const T* __restrict__ lamg,
    int C, int ng, const T* __restrict__ wpsi, const T* __restrict__ wdpsi,
    T* __restrict__ cut, const DevBlock* __restrict__ blocks, const int* __restrict__ ncut_J,
    int m_inf, T* __restrict__ qcol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = plan.N;  // == nr
  const int P = C / 2;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* ph = tw + N;
  T* lam = reinterpret_cast<T*>(ph + N);
  cpx<T>* za = reinterpret_cast<cpx<T>*>(lam + ((N + 2) & ~1));
  cpx<T>* zb = za + (long)P * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twg[i];
    ph[i] = phg[i];
  }
  for (int i = threadIdx.x; i <= N; i += blockDim.x) lam[i] = lamg[i];

  const long plane = blockIdx.y;                  // = b * ng + n
  if ((int)(plane % ng) >= blocks[plane / ng].nrow) return;  // beyond the angular functions
  const int c0 = blockIdx.x * C;
  const T* qp = q + plane * (long)nr * NR;
  T* tp = t + plane * (long)nr * NR;
  T* zar = reinterpret_cast<T*>(za);
  for (int idx = threadIdx.x; idx < nr * C; idx += blockDim.x) {
    const int kr = idx / C;
    const int c = idx - kr * C;
    const int m = c0 + c;
    T x = (m < NR) ? qp[(long)kr * NR + m] : (T)0;
    const T sg = (kr & 1) ? (T)-1 : (T)1;
    zar[2 * ((long)(c >> 1) * N + perm_pos(kr, N)) + (c & 1)] = sg * x;
  }
  __syncthreads();

  // flux cut and the R_inf column, from the unmodified tile
  const int b = (int)(plane / ng);
  const int n = (int)(plane - (long)b * ng);
  if (cut != nullptr) {
    const DevBlock B = blocks[b];
    const long ncut = ncut_J[B.iJ];
    for (int o = threadIdx.x; o < 2 * C; o += blockDim.x) {
      const int c = o >> 1;
      const int which = o & 1;
      const int m = c0 + c;
      if (m >= NR) continue;
      const T* w = which ? wdpsi : wpsi;
      T s = 0;
      for (int kr = 0; kr < nr; ++kr) {
        const T sg = (kr & 1) ? (T)-1 : (T)1;
        s += w[kr] * sg * zar[2 * ((long)(c >> 1) * N + perm_pos(kr, N)) + (c & 1)];
      }
      cut[B.cutcol + (long)which * ncut + (long)n * NR + m] = s;
    }
  }
  if (qcol != nullptr && m_inf >= c0 && m_inf < c0 + C) {
    const int c = m_inf - c0;
    for (int kr = threadIdx.x; kr < nr; kr += blockDim.x) {
      const T sg = (kr & 1) ? (T)-1 : (T)1;
      qcol[plane * nr + kr] = sg * zar[2 * ((long)(c >> 1) * N + perm_pos(kr, N)) + (c & 1)];
    }
  }

  cpx<T>* Z = stockham<T>(za, zb, P, plan, tw, (T)-1);
  cpx<T>* W = (Z == za) ? zb : za;
  kinetic_scale<T>(Z, W, P, N, ph, lam);
  __syncthreads();
  cpx<T>* other = (W == za) ? zb : za;
  cpx<T>* Y = stockham<T>(W, other, P, plan, tw, (T)1);
  const T* yr = reinterpret_cast<const T*>(Y);
  for (int idx = threadIdx.x; idx < nr * C; idx += blockDim.x) {
    const int kr = idx / C;
    const int c = idx - kr * C;
    const int m = c0 + c;
    if (m >= NR) continue;
    const T sg = (kr & 1) ? (T)-1 : (T)1;
    tp[(long)kr * NR + m] += sg * yr[2 * ((long)(c >> 1) * N + perm_pos(kr, N)) + (c & 1)];
  }
}

template <typename T>
static size_t kinetic_smem(int N, int P) {
  return sizeof(cpx<T>) * 2 * (size_t)N + sizeof(T) * (size_t)((N + 2) & ~1) +
         sizeof(cpx<T>) * 2 * (size_t)P * N;
}

template <typename T>
bool kinetic_rows_fixed(int N, const T* q, T* t, long nrows, const void* tw, const void* ph,
                        const T* lam, int P, const DevBlock* blocks, int ng, int nr,
                        cudaStream_t st, cudaError_t* err);
template <typename T>
bool kinetic_rows_warp(int N, const T* q, T* t, long nrows, const void* tw, const void* ph,
                       const T* lam, const DevBlock* blocks, int ng, int nr, cudaStream_t st,
                       cudaError_t* err, int form);
template <typename T>
bool kinetic_cols_warp(int N, const T* q, T* t, long nplanes, int NR, const void* tw,
                       const void* ph, const T* lam, int C, int ng, const T* wpsi,
                       const T* wdpsi, T* cut, const DevBlock* blocks, const int* ncut_J,
                       int m_inf, T* qcol, cudaStream_t st, cudaError_t* err, int form);
template <typename T>
bool kinetic_cols_fixed(int N, const T* q, T* t, long nplanes, int NR, const void* tw,
                        const void* ph, const T* lam, int C, int ng, const T* wpsi,
                        const T* wdpsi, T* cut, const DevBlock* blocks, const int* ncut_J,
                        int m_inf, T* qcol, cudaStream_t st, cudaError_t* err);

template <typename real>
cudaError_t launch_kinetic_rows(const real* q, real* t, long nrows, const FFTPlan& plan,
                                const void* tw, const void* ph, const real* lam, int pairs,
                                const DevBlock* blocks, int ng, int nr, int warp_fft,
                                cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  if (warp_fft &&
      kinetic_rows_warp<real>(plan.N, q, t, nrows, tw, ph, lam, blocks, ng, nr, st, &err,
                              warp_fft))
    return err;
  if (kinetic_rows_fixed<real>(plan.N, q, t, nrows, tw, ph, lam, pairs, blocks, ng, nr, st, &err))
    return err;
  const size_t sm = kinetic_smem<real>(plan.N, pairs);
  static bool attr_set[2] = {false, false};
  const int slot = sizeof(real) == 8 ? 1 : 0;
  if (!attr_set[slot]) {
    cudaFuncSetAttribute(k_kinetic_rows<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set[slot] = true;
  }
  const long npairs = (nrows + 1) / 2;
  const unsigned grid = (unsigned)((npairs + pairs - 1) / pairs);
  k_kinetic_rows<real><<<grid, 256, sm, st>>>(q, t, nrows, plan,
                                              static_cast<const cpx<real>*>(tw),
                                              static_cast<const cpx<real>*>(ph), lam, pairs,
                                              blocks, ng, nr);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_kinetic_cols(const real* q, real* t, long nplanes, int nr, int NR,
                                const FFTPlan& plan, const void* tw, const void* ph,
                                const real* lam, int ctile, int ng, const real* wpsi,
                                const real* wdpsi, real* cut_slot, const DevBlock* blocks,
                                const int* ncut_J, int m_inf, real* qcol, int warp_fft,
                                cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  if (warp_fft && kinetic_cols_warp<real>(plan.N, q, t, nplanes, NR, tw, ph, lam, ctile, ng, wpsi,
                                          wdpsi, cut_slot, blocks, ncut_J, m_inf, qcol, st, &err,
                                          warp_fft))
    return err;
  if (kinetic_cols_fixed<real>(plan.N, q, t, nplanes, NR, tw, ph, lam, ctile, ng, wpsi, wdpsi,
                               cut_slot, blocks, ncut_J, m_inf, qcol, st, &err))
    return err;
  const size_t sm = kinetic_smem<real>(plan.N, ctile / 2);
  static bool attr_set[2] = {false, false};
  const int slot = sizeof(real) == 8 ? 1 : 0;
  if (!attr_set[slot]) {
    cudaFuncSetAttribute(k_kinetic_cols<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_set[slot] = true;
  }
  dim3 grid((unsigned)((NR + ctile - 1) / ctile), (unsigned)nplanes);
  k_kinetic_cols<real><<<grid, 256, sm, st>>>(q, t, nr, NR, plan,
                                              static_cast<const cpx<real>*>(tw),
                                              static_cast<const cpx<real>*>(ph), lam, ctile, ng,
                                              wpsi, wdpsi, cut_slot, blocks, ncut_J, m_inf,
                                              qcol);
  return cudaGetLastError();
}

template cudaError_t launch_kinetic_rows<double>(const double*, double*, long, const FFTPlan&,
                                                 const void*, const void*, const double*, int,
                                                 const DevBlock*, int, int, int, cudaStream_t);
template cudaError_t launch_kinetic_rows<float>(const float*, float*, long, const FFTPlan&,
                                                const void*, const void*, const float*, int,
                                                const DevBlock*, int, int, int, cudaStream_t);
template cudaError_t launch_kinetic_cols<double>(const double*, double*, long, int, int,
                                                 const FFTPlan&, const void*, const void*,
                                                 const double*, int, int, const double*,
                                                 const double*, double*, const DevBlock*,
                                                 const int*, int, double*, int, cudaStream_t);
template cudaError_t launch_kinetic_cols<float>(const float*, float*, long, int, int,
                                                const FFTPlan&, const void*, const void*,
                                                const float*, int, int, const float*,
                                                const float*, float*, const DevBlock*,
                                                const int*, int, float*, int, cudaStream_t);

}  // namespace mw3
