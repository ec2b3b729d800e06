// Angular (gamma) part of the Hamiltonian, the potential and the Chebyshev update
// (Section 2.1 items 3-5 and Section 2.2, Eq. wvp-k), CUDA-core path (FP64, and
// FP32 when the tensor-core path is off).
//
// The state of block (J, Omega, Lambda) is held in its FBR: rows i = 0..ng-Omega-1
// are the coefficients of the normalised associated Legendre functions j = Omega + i
// (rows beyond are zero). Per iteration:
//   GEMM 1  u = (T^Omega)^T c_k                      FBR -> DVR values on the grid
//   GEMM 2  w = T^Omega (V u),  (V u)_L = sum_L' V_LL' u_L'  (potential in the DVR)
//   epilogue, per FBR coefficient:
//     h = w + a_j c^Omega_j + bp_j c^(Omega+1)_j + bm_j c^(Omega-1)_j + t
//     (j^2/(2 m r^2) + l^2/(2 mu R^2) with the Coriolis coupling tridiagonal in Omega,
//     neighbour rows shifted by one because block Omega starts at j = Omega; t is the
//     radial kinetic term), H_s c = h / dE - (E0 / dE) c, and the damped recursion
//     c_(k+1) = D (alpha H_s c_k - beta D c_(k-1)) written over c_(k-1).
#include <cuda_runtime.h>

#include <algorithm>

#include "mw3_internal.h"

namespace mw3 {

constexpr int GBM = 64, GBN = 64, GBK = 16, GTM = 4, GTN = 4, GTHREADS = 256;

// Generic SIMT tile: C[m, n] (+)= sum_k A(b, m, k) B(b, k, n), tiles 64 x 64 x 16,
// 256 threads with 4 x 4 outputs each. Loaders return 0 outside the matrices.
template <typename TA, typename TB, typename TC, class ALoad, class BLoad, class Epi>
__global__ void __launch_bounds__(GTHREADS) k_gemm(int M, long N, int K, ALoad al, BLoad bl,
                                                   Epi ep) {
  __shared__ TA As[GBK][GBM + 1];
  __shared__ TB Bs[GBK][GBN];
  const int b = blockIdx.z;
  if (!ep.active(b, blockIdx.x * (long)GBN)) return;
  const int m0 = blockIdx.y * GBM;
  const long n0 = (long)blockIdx.x * GBN;
  const int tx = threadIdx.x % (GBN / GTN);   // 16
  const int ty = threadIdx.x / (GBN / GTN);   // 16
  TC acc[GTM][GTN];
#pragma unroll
  for (int i = 0; i < GTM; ++i)
#pragma unroll
    for (int j = 0; j < GTN; ++j) acc[i][j] = (TC)0;

  for (int k0 = 0; k0 < K; k0 += GBK) {
    // A tile: 64 x 16, k fastest across threads
    for (int e = threadIdx.x; e < GBM * GBK; e += GTHREADS) {
      const int mm = e / GBK, kk = e - mm * GBK;
      As[kk][mm] = (m0 + mm < M && k0 + kk < K) ? al(b, m0 + mm, k0 + kk) : (TA)0;
    }
    // B tile: 16 x 64, n fastest across threads (coalesced)
    for (int e = threadIdx.x; e < GBK * GBN; e += GTHREADS) {
      const int kk = e / GBN, nn = e - kk * GBN;
      Bs[kk][nn] = (k0 + kk < K && n0 + nn < N) ? bl(b, k0 + kk, n0 + nn) : (TB)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      TC a[GTM], bb[GTN];
#pragma unroll
      for (int i = 0; i < GTM; ++i) a[i] = (TC)As[kk][ty + i * (GBM / GTM)];
#pragma unroll
      for (int j = 0; j < GTN; ++j) bb[j] = (TC)Bs[kk][tx + j * (GBN / GTN)];
#pragma unroll
      for (int i = 0; i < GTM; ++i)
#pragma unroll
        for (int j = 0; j < GTN; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < GTM; ++i) {
    const int m = m0 + ty + i * (GBM / GTM);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < GTN; ++j) {
      const long n = n0 + tx + j * (GBN / GTN);
      if (n < N) ep(b, m, n, acc[i][j]);
    }
  }
}

// ------------------------------------------------------------------ loaders
template <typename T>
struct LoadT {   // A(b, m, k) = Tmat[omega(b)][m][k]
  const T* T_;
  const DevBlock* blk;
  int ng;
  __device__ T operator()(int b, int m, int k) const {
    return T_[((long)blk[b].omega * ng + m) * ng + k];
  }
};

template <typename T>
struct LoadQ {   // B(b, k, n) = q[b][k][n]
  const T* q;
  long npts, ncol;
  __device__ T operator()(int b, int k, long n) const { return q[b * npts + k * ncol + n]; }
};

template <typename T>
struct LoadVu {   // B(b, n, col) = sum_L' V_(L L')(n, col) u_(b with L')(n, col)
  const T* u;
  const T* V;
  const DevBlock* blk;
  long npts, ncol;
  int nelec;
  __device__ T operator()(int b, int n, long col) const {
    const DevBlock B = blk[b];
    const long off = (long)n * ncol + col;
    T v = 0;
    for (int lp = 0; lp < nelec; ++lp)
      v += V[(long)(B.lam * nelec + lp) * npts + off] * u[(long)(B.base + lp) * npts + off];
    return v;
  }
};

// ---------------------------------------------------------------- epilogues
template <typename T>
struct EpiStore {
  T* out;
  long npts, ncol;
  __device__ bool active(int, long) const { return true; }
  __device__ void operator()(int b, int m, long n, T v) const { out[b * npts + m * ncol + n] = v; }
};

// mode 0: damped recursion in place into ckm1; mode 1: write H_s c into out.
template <typename T>
struct EpiUpdate {
  const T* ck;
  T* ckm1;
  const T* t;
  const DevBlock* blk;
  const T* coef;
  const T* fr;
  const T* fR;
  T erot;
  const T* DR;
  const T* Dr;
  const DevJ* dj;
  T alpha, beta;
  long npts, ncol;
  int NR, ng, mode;
  T* out;
  __device__ bool active(int, long) const { return true; }
  __device__ void operator()(int b, int i, long col, T w) const {
    const DevBlock B = blk[b];
    const long idx = b * npts + (long)i * ncol + col;
    if (i >= B.nrow) {  // beyond the block's angular functions: stays zero
      if (mode == 1) out[idx] = 0; else ckm1[idx] = 0;
      return;
    }
    const int kr = (int)(col / NR);
    const int m = (int)(col - (long)kr * NR);
    const T* cf = coef + (long)B.coef * kCoefRows * ng;
    const T g = fmin(fR[m], cf[4 * ng + i]);
    const T a = fmin(cf[i] * fr[kr], erot) + g * cf[ng + i];
    const T cv = ck[idx];
    T h = w + a * cv + t[idx];
    if (B.up >= 0 && i >= 1) h += g * cf[2 * ng + i] * ck[B.up * npts + (long)(i - 1) * ncol + col];
    if (B.dn >= 0) h += g * cf[3 * ng + i] * ck[B.dn * npts + (long)(i + 1) * ncol + col];
    const DevJ J = dj[B.iJ];
    const T hs = h * (T)J.invdE - (T)J.e0s * cv;
    if (mode == 1) {
      out[idx] = hs;
      return;
    }
    const T D = DR[m] * Dr[kr];
    ckm1[idx] = D * (alpha * hs - beta * D * ckm1[idx]);
  }
};

template <typename real>
cudaError_t launch_gamma_forward(const real* q, real* c, const real* T, const DevBlock* blocks,
                                 int nblk, int ng, long ncol, cudaStream_t st) {
  const long npts = (long)ng * ncol;
  dim3 grid((unsigned)((ncol + GBN - 1) / GBN), (unsigned)((ng + GBM - 1) / GBM), (unsigned)nblk);
  k_gemm<real, real, real><<<grid, GTHREADS, 0, st>>>(
      ng, ncol, ng, LoadT<real>{T, blocks, ng}, LoadQ<real>{q, npts, ncol},
      EpiStore<real>{c, npts, ncol});
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gamma_update(const real* u, const real* T, const DevBlock* blocks, int nblk,
                                int ng, long ncol, int NR, const real* coef, const real* fr,
                                const real* fR, real erot, const real* ck, real* ckm1,
                                const real* t, const real* V, int nelec, const real* DR,
                                const real* Dr, const DevJ* dj, real alpha, real beta, int mode,
                                real* out, cudaStream_t st) {
  const long npts = (long)ng * ncol;
  dim3 grid((unsigned)((ncol + GBN - 1) / GBN), (unsigned)((ng + GBM - 1) / GBM), (unsigned)nblk);
  k_gemm<real, real, real><<<grid, GTHREADS, 0, st>>>(
      ng, ncol, ng, LoadT<real>{T, blocks, ng}, LoadVu<real>{u, V, blocks, npts, ncol, nelec},
      EpiUpdate<real>{ck, ckm1, t, blocks, coef, fr, fR, erot, DR, Dr, dj, alpha, beta, npts,
                      ncol, NR, ng, mode, out});
  return cudaGetLastError();
}

// ------------------------------------------------------------ energy sums
// Ph[iJ][row][s]: rows 0..nE-1 hold (2 - delta_k0) cos(k theta), rows nE..2nE-1
// hold -(2 - delta_k0) sin(k theta), k = iteration of ring slot s (c_k = (2 -
// delta_k0) exp(-i k theta)); slots s >= nvalid are zero.
template <typename real>
__global__ void k_phases(const double* __restrict__ theta, int nJ, int nE, int kb, int nvalid,
                         const long* __restrict__ d_iter, real* __restrict__ ph) {
  const long total = (long)nJ * nE * kb;
  const long k0 = *d_iter;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const int s = (int)(e % kb);
    const long je = e / kb;
    const int iJ = (int)(je / nE);
    const int ie = (int)(je - (long)iJ * nE);
    real cr = 0, ci = 0;
    if (s < nvalid) {
      const long k = k0 + s;
      const double w = (k == 0) ? 1.0 : 2.0;
      double sn, cs;
      sincos((double)k * theta[je], &sn, &cs);
      cr = (real)(w * cs);
      ci = (real)(-w * sn);
    }
    real* P = ph + (long)iJ * 2 * nE * kb;
    P[(long)ie * kb + s] = cr;
    P[(long)(nE + ie) * kb + s] = ci;
  }
}

template <typename real>
struct LoadPh {
  const real* ph;
  int nE2, kb;
  __device__ real operator()(int iJ, int m, int k) const { return ph[((long)iJ * nE2 + m) * kb + k]; }
};

template <typename real>
struct LoadCut {   // columns beyond J's own range read as zero (never past the ring)
  const real* cut;
  long ncut_total;
  const long* colbase;
  const long* ncols;
  __device__ real operator()(int iJ, int k, long n) const {
    return n < ncols[iJ] ? cut[(long)k * ncut_total + colbase[iJ] + n] : (real)0;
  }
};

template <typename TC>
struct EpiAcc {
  double* acc;
  const long* accoff;
  const long* ncols;
  __device__ bool active(int iJ, long n0) const { return n0 < ncols[iJ]; }
  __device__ void operator()(int iJ, int m, long n, TC v) const {
    if (n < ncols[iJ]) acc[accoff[iJ] + (long)m * ncols[iJ] + n] += (double)v;
  }
};

template <typename real>
cudaError_t launch_phases(const double* theta, int nJ, int nE, int kb, int nvalid,
                          const long* d_iter, real* ph, cudaStream_t st) {
  const long total = (long)nJ * nE * kb;
  const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_phases<real><<<grid, 256, 0, st>>>(theta, nJ, nE, kb, nvalid, d_iter, ph);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_sums_flush(const real* ph, const real* cut, long ncut_total, int kb, int nvalid,
                              int nJ, int nE, const long* colbase, const long* ncols,
                              const long* accoff, long max_cols, double* acc,
                              cudaStream_t st) {
  if (nvalid < 1 || nvalid > kb) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((max_cols + GBN - 1) / GBN), (unsigned)((2 * nE + GBM - 1) / GBM),
            (unsigned)nJ);
  // M = 2 nE rows, K = the nvalid filled ring slots (the phases of the others are zero; ph
  // rows keep their stride kb), N = columns of each J (checked by the epilogue)
  k_gemm<real, real, real><<<grid, GTHREADS, 0, st>>>(
      2 * nE, max_cols, nvalid, LoadPh<real>{ph, 2 * nE, kb},
      LoadCut<real>{cut, ncut_total, colbase, ncols}, EpiAcc<real>{acc, accoff, ncols});
  return cudaGetLastError();
}

__global__ void k_advance(long* d_iter, long n) { *d_iter += n; }

// Precision conversion of a state vector on the device (host copies stay FP64).
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

cudaError_t launch_convert_d2f(const double* in, float* out, long n, cudaStream_t st) {
  k_convert<double, float><<<1216, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_f2d(const float* in, double* out, long n, cudaStream_t st) {
  k_convert<float, double><<<1216, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

// A state vector read straight from page-locked host memory through its device alias: 16-byte
// loads, four in flight per thread (the host link has a long latency), converted to the
// state's precision on the way. `in` is 16-byte aligned; an odd last element is read alone.
template <typename B>
__global__ void __launch_bounds__(256) k_host_read(const double* __restrict__ in,
                                                   B* __restrict__ out, long n) {
  const long n2 = n >> 1;
  const double2* in2 = reinterpret_cast<const double2*>(in);
  const long stride = (long)gridDim.x * blockDim.x;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n2; i += 4 * stride) {
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = in2[i + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      out[2 * (i + u * stride)] = (B)v[u].x;
      out[2 * (i + u * stride) + 1] = (B)v[u].y;
    }
  }
  for (; i < n2; i += stride) {
    const double2 v = in2[i];
    out[2 * i] = (B)v.x;
    out[2 * i + 1] = (B)v.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) out[n - 1] = (B)in[n - 1];
}

template <typename B>
cudaError_t launch_host_read(const double* host_alias, B* out, long n, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long blocks = std::min<long>((long)std::max(nsm, 1) * 8, (n / 2 + 255) / 256 + 1);
  k_host_read<B><<<(unsigned)blocks, 256, 0, st>>>(host_alias, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_host_read<float>(const double*, float*, long, cudaStream_t);
template cudaError_t launch_host_read<double>(const double*, double*, long, cudaStream_t);

cudaError_t launch_advance(long* d_iter, long n, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(d_iter, n);
  return cudaGetLastError();
}

// ------------------------------------------------------- channel projections
// cut_slot[chan_col[c]] = (k >= kmin) ? sum_kr chi[c][kr] qcol[block(c)][row(c)][kr] : 0,
// chi already divided by sqrt(dR); qcol holds the FBR coefficients at R_inf.
template <typename real>
__global__ void __launch_bounds__(128) k_channels(const real* __restrict__ qcol,
                                                  const double* __restrict__ chi,
                                                  const int* __restrict__ chan_block,
                                                  const int* __restrict__ chan_row,
                                                  const int* __restrict__ chan_col, int ng, int nr,
                                                  const long* __restrict__ d_iter, int slot,
                                                  long kmin, double* __restrict__ cut) {
  __shared__ double red[128];
  const int c = blockIdx.x;
  const double* p = chi + (long)c * nr;
  const real* x = qcol + ((long)chan_block[c] * ng + chan_row[c]) * nr;
  double s = 0;
  for (int i = threadIdx.x; i < nr; i += blockDim.x) s += p[i] * (double)x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long k = *d_iter + slot;
    cut[chan_col[c]] = (k >= kmin) ? red[0] : 0.0;
  }
}

template <typename real>
cudaError_t launch_channels(const real* qcol, const double* chi, const int* chan_block,
                            const int* chan_row, const int* chan_col, int nchan, int ng, int nr,
                            const long* d_iter, int slot, long kmin, double* cut_slot,
                            cudaStream_t st) {
  if (nchan <= 0) return cudaSuccess;
  k_channels<real><<<nchan, 128, 0, st>>>(qcol, chi, chan_block, chan_row, chan_col, ng, nr,
                                          d_iter, slot, kmin, cut_slot);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- norms
// partial[iJ][chunk] = sum of squares over a fixed contiguous chunk of J's range;
// out[iJ] = ordered sum of the partials (deterministic).
template <typename real>
__global__ void __launch_bounds__(256) k_norm_partial(const real* __restrict__ q,
                                                      const long* __restrict__ J_begin,
                                                      int nchunk, double* __restrict__ partial) {
  __shared__ double red[256];
  const int iJ = blockIdx.y;
  const long beg = J_begin[iJ], end = J_begin[iJ + 1];
  const long len = end - beg;
  const long per = (len + nchunk - 1) / nchunk;
  const long a = beg + per * blockIdx.x;
  const long z = (a + per < end) ? a + per : end;
  double s = 0;
  for (long i = a + threadIdx.x; i < z; i += blockDim.x) {
    const double v = (double)q[i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long)iJ * nchunk + blockIdx.x] = red[0];
}

// partial[iJ][chunk] = sum of a*b over a fixed contiguous chunk of J's range, in FP64
// whatever the precision of a and b (the autocorrelation of the photodissociation analysis).
template <typename real>
__global__ void __launch_bounds__(256) k_dot_partial(const real* __restrict__ a,
                                                     const real* __restrict__ b,
                                                     const long* __restrict__ J_begin,
                                                     int nchunk, double* __restrict__ partial) {
  __shared__ double red[256];
  const int iJ = blockIdx.y;
  const long beg = J_begin[iJ], end = J_begin[iJ + 1];
  const long len = end - beg;
  const long per = (len + nchunk - 1) / nchunk;
  const long lo = beg + per * blockIdx.x;
  const long hi = (lo + per < end) ? lo + per : end;
  double s = 0;
  for (long i = lo + threadIdx.x; i < hi; i += blockDim.x) s += (double)a[i] * (double)b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long)iJ * nchunk + blockIdx.x] = red[0];
}

// Time-domain packets (Eqs. wvf-chebyshev, chebyshev-expansion-constants): for iteration
// k = *d_iter + slot < K, acc[j][0 or 1][e] += Re or Im f_k(t_j) q_k[e], with f[k][iJ][j]
// (complex FP64) the coefficient of element e's J; the sums are FP64 whatever the state's
// precision. One thread per element, grid-stride.
template <typename real>
__global__ void __launch_bounds__(256) k_time_accum(const real* __restrict__ q, long n, long npts,
                                                    const DevBlock* __restrict__ blocks,
                                                    const double* __restrict__ f, int nJ, int nt,
                                                    long K, const long* __restrict__ d_iter,
                                                    int slot, double* __restrict__ acc) {
  const long k = *d_iter + slot;
  if (k >= K) return;
  const double* fk = f + (size_t)k * nJ * nt * 2;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const double x = (double)q[e];
    const int iJ = blocks[e / npts].iJ;
    for (int j = 0; j < nt; ++j) {
      const double fr = fk[((size_t)iJ * nt + j) * 2], fi = fk[((size_t)iJ * nt + j) * 2 + 1];
      acc[((size_t)j * 2) * n + e] += fr * x;
      acc[((size_t)j * 2 + 1) * n + e] += fi * x;
    }
  }
}

// Lanczos helpers on J segments (every element's scalar is that of its block's J):
//   k_axpy_seg:   y[e] += s * c[iJ(e)] * x[e]
//   k_rscale_seg: y[e] /= sqrt(c2[iJ(e)])  (c2 = 0 leaves y unchanged)
//   k_sqrt:       b[i] = sqrt(b2[i])
template <typename real>
__global__ void k_axpy_seg(real* __restrict__ y, const real* __restrict__ x,
                           const double* __restrict__ c, double s, long n, long npts,
                           const DevBlock* __restrict__ blocks) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    y[e] = (real)((double)y[e] + s * c[blocks[e / npts].iJ] * (double)x[e]);
}

template <typename real>
__global__ void k_rscale_seg(real* __restrict__ y, const double* __restrict__ c2, long n, long npts,
                             const DevBlock* __restrict__ blocks) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double v = c2[blocks[e / npts].iJ];
    if (v > 0.0) y[e] = (real)((double)y[e] / sqrt(v));
  }
}

__global__ void k_sqrt(const double* __restrict__ b2, double* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = sqrt(b2[i]);
}

__global__ void k_norm_final(const double* __restrict__ partial, int nchunk, double* out) {
  const int iJ = blockIdx.x;
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < nchunk; ++i) s += partial[(long)iJ * nchunk + i];
    out[iJ] = s;
  }
}

template <typename real>
cudaError_t launch_norms(const real* q, const long* J_begin, int nJ, double* partial,
                         int nchunk, double* out, cudaStream_t st) {
  k_norm_partial<real><<<dim3(nchunk, nJ), 256, 0, st>>>(q, J_begin, nchunk, partial);
  k_norm_final<<<nJ, 32, 0, st>>>(partial, nchunk, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_axpy_seg(real* y, const real* x, const double* c, double s, long n, long npts,
                            const DevBlock* blocks, cudaStream_t st) {
  const long nb = (n + 255) / 256;
  k_axpy_seg<real><<<(unsigned)(nb < 8192 ? nb : 8192), 256, 0, st>>>(y, x, c, s, n, npts, blocks);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_rscale_seg(real* y, const double* c2, long n, long npts, const DevBlock* blocks,
                              cudaStream_t st) {
  const long nb = (n + 255) / 256;
  k_rscale_seg<real><<<(unsigned)(nb < 8192 ? nb : 8192), 256, 0, st>>>(y, c2, n, npts, blocks);
  return cudaGetLastError();
}

cudaError_t launch_sqrt(const double* b2, double* b, int n, cudaStream_t st) {
  k_sqrt<<<(n + 127) / 128, 128, 0, st>>>(b2, b, n);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_time_accum(const real* q, long n, long npts, const DevBlock* blocks,
                              const double* f, int nJ, int nt, long K, const long* d_iter,
                              int slot, double* acc, cudaStream_t st) {
  const long nb = (n + 255) / 256;
  k_time_accum<real><<<(unsigned)(nb < 8192 ? nb : 8192), 256, 0, st>>>(q, n, npts, blocks, f, nJ,
                                                                         nt, K, d_iter, slot, acc);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_dots(const real* a, const real* b, const long* J_begin, int nJ,
                        double* partial, int nchunk, double* out, cudaStream_t st) {
  k_dot_partial<real><<<dim3(nchunk, nJ), 256, 0, st>>>(a, b, J_begin, nchunk, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_norm_final<<<nJ, 32, 0, st>>>(partial, nchunk, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------- flux reduce
// out[iJ][e] = sum_p Re A_psi Im A_dpsi - Im A_psi Re A_dpsi over J's cut points,
// with A rows e (real part) and nE + e (imaginary part).
// The flux sum of Eq. total-flux per (J, E): F = sum_p Re A(p) Im B(p) - Im A(p) Re B(p) over
// the J's cut points p (A the psi columns, B the dpsi columns of the accumulators), split over
// chunks of kFluxChunk points so that every SM takes part (the accumulators are GBs: the
// reduction is one read of them), with partial sums per chunk summed in chunk order by
// k_flux_final. PEEK: the accumulators are A + Ph Cut with the ring slots that have not been
// flushed yet (npend <= kPeekMax) added on the fly (the products summed in the ring's
// precision, then added to the FP64 accumulator values); A itself is only read, so a
// probability read between flushes moves the accumulators once instead of three times (read
// and write of a flush, then the read of the reduction).
constexpr int kFluxE = 8;          // energies per CTA (the ring values of a point read once)
constexpr long kFluxChunk = 4096;  // cut points per CTA

template <bool PEEK, typename real>
__global__ void __launch_bounds__(256) k_flux_partial(
    const double* __restrict__ acc, int nJ, int nE, const long* __restrict__ accoff,
    const long* __restrict__ ncols, const long* __restrict__ ncut, const real* __restrict__ ph,
    int kb, int npend, const real* __restrict__ cut, long ncut_total,
    const long* __restrict__ colbase, double* __restrict__ part, float* __restrict__ acc32) {
  // phase factors (real, imaginary row) per pending slot, in the ring's precision: the pending
  // terms are summed like the flush sums them (FP32 products in the mixed form; FP64 arithmetic
  // runs at 1/64 of the FP32 rate here) and added to the FP64 accumulators once
  __shared__ real sph[kFluxE][2][kPeekMax];
  __shared__ double red[kFluxE][256];
  const int e0 = blockIdx.x * kFluxE;
  const int iJ = blockIdx.y;
  const int ne = min(kFluxE, nE - e0);
  const long nc = ncols[iJ], np = ncut[iJ];
  const long p0 = (long)blockIdx.z * kFluxChunk, p1 = min(np, p0 + kFluxChunk);
  const double* A = acc + accoff[iJ];
  if constexpr (PEEK) {
    for (int x = threadIdx.x; x < kFluxE * 2 * kPeekMax; x += blockDim.x) {
      const int q = x / (2 * kPeekMax), prt = (x / kPeekMax) & 1, sl = x % kPeekMax;
      const int row = (prt ? nE : 0) + e0 + q;
      sph[q][prt][sl] = (q < ne && sl < npend) ? ph[((long)iJ * 2 * nE + row) * kb + sl] : (real)0;
    }
  }
  // the reduction keeps all energies of a point in registers (the loads of a point in flight
  // together); with pending slots the energies go two at a time and the sums live in shared
  // memory (a thread owns its column), which keeps the register count, and the occupancy, up
  double acc_q[PEEK ? 1 : kFluxE];
#pragma unroll
  for (int q = 0; q < (PEEK ? 1 : kFluxE); ++q) acc_q[q] = 0.0;
#pragma unroll
  for (int q = 0; q < kFluxE; ++q) red[q][threadIdx.x] = 0.0;
  __syncthreads();
  for (long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    real cp[kPeekMax], cq[kPeekMax];
    if constexpr (PEEK) {
      const real* cj = cut + colbase[iJ];
#pragma unroll
      for (int sl = 0; sl < kPeekMax; ++sl) {
        cp[sl] = sl < npend ? cj[(long)sl * ncut_total + p] : (real)0;
        cq[sl] = sl < npend ? cj[(long)sl * ncut_total + np + p] : (real)0;
      }
    }
#pragma unroll(PEEK ? 2 : kFluxE)
    for (int q = 0; q < kFluxE; ++q) {
      if (q < ne) {
        const double* re = A + (long)(e0 + q) * nc;
        const double* im = A + (long)(nE + e0 + q) * nc;
        double rp = re[p], ip = im[p], rq = re[np + p], iq = im[np + p];
        if (acc32) {   // an FP32 copy of the values read, for later reads with pending slots
          float* r32 = acc32 + accoff[iJ] + (long)(e0 + q) * nc;
          float* i32 = acc32 + accoff[iJ] + (long)(nE + e0 + q) * nc;
          r32[p] = (float)rp;
          i32[p] = (float)ip;
          r32[np + p] = (float)rq;
          i32[np + p] = (float)iq;
        }
        if constexpr (PEEK) {
          real drp = 0, dip = 0, drq = 0, diq = 0;
#pragma unroll
          for (int sl = 0; sl < kPeekMax; ++sl) {
            if (sl < npend) {
              drp += sph[q][0][sl] * cp[sl];
              dip += sph[q][1][sl] * cp[sl];
              drq += sph[q][0][sl] * cq[sl];
              diq += sph[q][1][sl] * cq[sl];
            }
          }
          rp += (double)drp;
          ip += (double)dip;
          rq += (double)drq;
          iq += (double)diq;
          red[q][threadIdx.x] += rp * iq - ip * rq;
        } else {
          acc_q[q] += rp * iq - ip * rq;
        }
      }
    }
  }
  if constexpr (!PEEK) {
#pragma unroll
    for (int q = 0; q < kFluxE; ++q) red[q][threadIdx.x] = acc_q[q];
  }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < kFluxE; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < ne)
    part[((long)blockIdx.z * nJ + iJ) * nE + e0 + threadIdx.x] = red[threadIdx.x][0];
}

// Mixed form, reads with pending ring slots: with A the flushed accumulators (their flux F_A
// already known, FP32 copy A32) and D = Ph Cut the pending terms,
//   flux(A + D) - F_A = sum_p Re A Im D_B + Re D_A Im B - Im A Re D_B - Im D_A Re B
//                              + Re D_A Im D_B - Im D_A Re D_B
// (A = psi column p, B = dpsi column np + p). The pending terms and their products with A
// are FP32 values like the flush's own products; each thread sums its points in FP32 and the
// CTA in FP64, so the FP64 accumulators are not read at all.
// A thread takes two neighbouring points at a time (8-byte loads: cut columns start at
// multiples of 4, the accumulator rows and np are even because NR is) and keeps their pending
// ring values in registers for all of the CTA's energies; each phase value read from shared
// memory then serves four products.
__global__ void __launch_bounds__(256) k_flux_cross(
    const float* __restrict__ acc32, int nJ, int nE, const long* __restrict__ accoff,
    const long* __restrict__ ncols, const long* __restrict__ ncut, const float* __restrict__ ph,
    int kb, int npend, const float* __restrict__ cut, long ncut_total,
    const long* __restrict__ colbase, double* __restrict__ part) {
  __shared__ __align__(16) float sph[kFluxE][2][kPeekMaxX];
  __shared__ double red[kFluxE][256];
  const int e0 = blockIdx.x * kFluxE;
  const int iJ = blockIdx.y;
  const int ne = min(kFluxE, nE - e0);
  const long nc = ncols[iJ], np = ncut[iJ];
  const long p0 = (long)blockIdx.z * kFluxChunk, p1 = min(np, p0 + kFluxChunk);
  const float* A = acc32 + accoff[iJ];
  const float* cj = cut + colbase[iJ];
  for (int x = threadIdx.x; x < kFluxE * 2 * kPeekMaxX; x += blockDim.x) {
    const int q = x / (2 * kPeekMaxX), prt = (x / kPeekMaxX) & 1, sl = x % kPeekMaxX;
    const int row = (prt ? nE : 0) + e0 + q;
    sph[q][prt][sl] = (q < ne && sl < npend) ? ph[((long)iJ * 2 * nE + row) * kb + sl] : 0.0f;
  }
  // a thread's FP32 sums in shared memory (it owns its column): the energy loop stays rolled,
  // so that the phases are read per energy instead of being held in registers across points
  __shared__ float accs[kFluxE][256];
#pragma unroll
  for (int q = 0; q < kFluxE; ++q) accs[q][threadIdx.x] = 0.0f;
  __syncthreads();
  for (long p = p0 + 2 * threadIdx.x; p < p1; p += 2 * blockDim.x) {
    float2 cp[kPeekMaxX], cq[kPeekMaxX];
#pragma unroll
    for (int sl = 0; sl < kPeekMaxX; ++sl) {
      const float* c = cj + (long)sl * ncut_total + p;
      cp[sl] = sl < npend ? *reinterpret_cast<const float2*>(c) : make_float2(0.0f, 0.0f);
      cq[sl] = sl < npend ? *reinterpret_cast<const float2*>(c + np) : make_float2(0.0f, 0.0f);
    }
#pragma unroll 1
    for (int q = 0; q < ne; ++q) {
      {
        const float* re = A + (long)(e0 + q) * nc + p;
        const float* im = A + (long)(nE + e0 + q) * nc + p;
        const float2 ra = *reinterpret_cast<const float2*>(re);
        const float2 ia = *reinterpret_cast<const float2*>(im);
        const float2 rb = *reinterpret_cast<const float2*>(re + np);
        const float2 ib = *reinterpret_cast<const float2*>(im + np);
        float2 dra = make_float2(0.0f, 0.0f), dia = dra, drb = dra, dib = dra;
#pragma unroll
        for (int sl = 0; sl < kPeekMaxX; ++sl) {
          if (sl < npend) {
            const float pr = sph[q][0][sl], pi = sph[q][1][sl];
            dra.x += pr * cp[sl].x;
            dra.y += pr * cp[sl].y;
            dia.x += pi * cp[sl].x;
            dia.y += pi * cp[sl].y;
            drb.x += pr * cq[sl].x;
            drb.y += pr * cq[sl].y;
            dib.x += pi * cq[sl].x;
            dib.y += pi * cq[sl].y;
          }
        }
        accs[q][threadIdx.x] += (ra.x * dib.x + dra.x * ib.x - ia.x * drb.x - dia.x * rb.x +
                                 dra.x * dib.x - dia.x * drb.x) +
                                (ra.y * dib.y + dra.y * ib.y - ia.y * drb.y - dia.y * rb.y +
                                 dra.y * dib.y - dia.y * drb.y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kFluxE; ++q) red[q][threadIdx.x] = (double)accs[q][threadIdx.x];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < kFluxE; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < ne)
    part[((long)blockIdx.z * nJ + iJ) * nE + e0 + threadIdx.x] = red[threadIdx.x][0];
}

// out[iJ][e] = base[iJ][e] (if given) + the sum over the chunks z (in order) of part[z][iJ][e].
__global__ void k_flux_final(const double* __restrict__ part, int nz, long n,
                             const double* __restrict__ base, double* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += part[(long)z * n + i];
  out[i] = base ? base[i] + s : s;
}

long flux_partial_size(int nJ, int nE, long max_ncut) {
  return std::max<long>(1, (max_ncut + kFluxChunk - 1) / kFluxChunk) * nJ * nE;
}

cudaError_t launch_flux_reduce(const double* acc, int nJ, int nE, const long* accoff,
                               const long* ncols, const long* ncut, long max_ncut, double* part,
                               double* out, float* acc32, cudaStream_t st) {
  const int nz = (int)std::max<long>(1, (max_ncut + kFluxChunk - 1) / kFluxChunk);
  k_flux_partial<false, double><<<dim3((nE + kFluxE - 1) / kFluxE, nJ, nz), 256, 0, st>>>(
      acc, nJ, nE, accoff, ncols, ncut, nullptr, 0, 0, nullptr, 0, nullptr, part, acc32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long n = (long)nJ * nE;
  k_flux_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nz, n, nullptr, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_flux_reduce_peek(const double* acc, int nJ, int nE, const long* accoff,
                                    const long* ncols, const long* ncut, long max_ncut,
                                    const real* ph, int kb, int npend, const real* cut,
                                    long ncut_total, const long* colbase, double* part,
                                    double* out, cudaStream_t st) {
  if (npend < 0 || npend > kPeekMax) return cudaErrorInvalidValue;
  const int nz = (int)std::max<long>(1, (max_ncut + kFluxChunk - 1) / kFluxChunk);
  k_flux_partial<true, real><<<dim3((nE + kFluxE - 1) / kFluxE, nJ, nz), 256, 0, st>>>(
      acc, nJ, nE, accoff, ncols, ncut, ph, kb, npend, cut, ncut_total, colbase, part, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long n = (long)nJ * nE;
  k_flux_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nz, n, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_flux_cross(const float* acc32, int nJ, int nE, const long* accoff,
                              const long* ncols, const long* ncut, long max_ncut, const float* ph,
                              int kb, int npend, const float* cut, long ncut_total,
                              const long* colbase, double* part, const double* fluxA, double* out,
                              cudaStream_t st) {
  if (npend < 0 || npend > kPeekMaxX || npend > kb) return cudaErrorInvalidValue;
  const int nz = (int)std::max<long>(1, (max_ncut + kFluxChunk - 1) / kFluxChunk);
  k_flux_cross<<<dim3((nE + kFluxE - 1) / kFluxE, nJ, nz), 256, 0, st>>>(
      acc32, nJ, nE, accoff, ncols, ncut, ph, kb, npend, cut, ncut_total, colbase, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long n = (long)nJ * nE;
  k_flux_final<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, nz, n, fluxA, out);
  return cudaGetLastError();
}

// State-resolved probabilities from the channel accumulators (Eq. S-matrix-from-chebyshev),
// one thread per (output key, energy), energies fastest: for the key's channels c (in channel
// order) with K_c^2 = 2 mu (E_col + E_ref - eps_c) > 0,
//   P[key][e] += (2 pi K_c / mu) |pref A_c(E)|^2 / |a(E)|^2,  pref = 1 / (2 pi dE_J sin theta_JE),
// A_c(E) = acc[col_c + e ld_c] + i acc[col_c + (nE + e) ld_c]. Keys without channels get 0.
__global__ void __launch_bounds__(256) k_channel_probs(const double* __restrict__ acc,
                                                       ChanTable t, const double* __restrict__ Ecol,
                                                       double Eref,
                                                       const double* __restrict__ theta,
                                                       const double* __restrict__ dE,
                                                       const double* __restrict__ a2, int nE,
                                                       double* __restrict__ out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)t.nkeys * nE) return;
  const int key = (int)(idx / nE), e = (int)(idx - (long)key * nE);
  const double Etot = Ecol[e] + Eref;
  double sum = 0.0;
  for (long q = t.key_first[key]; q < t.key_first[key + 1]; ++q) {
    const int c = t.key_chan[q];
    const double K2 = 2.0 * t.mu * (Etot - t.eps[c]);
    if (K2 <= 0.0) continue;
    const int iJ = t.chJ[c];
    const double pref = 1.0 / (2.0 * M_PI * dE[iJ] * sin(theta[(long)iJ * nE + e]));
    const double re = acc[t.col[c] + (long)e * t.ld[c]] * pref;
    const double im = acc[t.col[c] + (long)(nE + e) * t.ld[c]] * pref;
    sum += 2.0 * M_PI * sqrt(K2) / t.mu * (re * re + im * im) / a2[e];
  }
  out[idx] = sum;
}

cudaError_t launch_channel_probs(const double* acc, const ChanTable& t, const double* Ecol,
                                 double Eref, const double* theta, const double* dE,
                                 const double* a2, int nE, double* out, cudaStream_t st) {
  const long n = (long)t.nkeys * nE;
  if (n == 0) return cudaSuccess;
  k_channel_probs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, t, Ecol, Eref, theta, dE, a2,
                                                               nE, out);
  return cudaGetLastError();
}

#define MW3_INST(real)                                                                        \
  template cudaError_t launch_flux_reduce_peek<real>(const double*, int, int, const long*,      \
                                                     const long*, const long*, long, const real*, \
                                                     int, int, const real*, long, const long*,   \
                                                     double*, double*, cudaStream_t);            \
  template cudaError_t launch_gamma_forward<real>(const real*, real*, const real*,            \
                                                  const DevBlock*, int, int, long,            \
                                                  cudaStream_t);                              \
  template cudaError_t launch_gamma_update<real>(                                             \
      const real*, const real*, const DevBlock*, int, int, long, int, const real*,            \
      const real*, const real*, real, const real*, real*, const real*, const real*, int,      \
      const real*, const real*, const DevJ*, real, real, int, real*, cudaStream_t);           \
  template cudaError_t launch_phases<real>(const double*, int, int, int, int, const long*,    \
                                           real*, cudaStream_t);                              \
  template cudaError_t launch_sums_flush<real>(const real*, const real*, long, int, int, int, \
                                               int, const long*, const long*, const long*,    \
                                               long, double*, cudaStream_t);                  \
  template cudaError_t launch_channels<real>(const real*, const double*, const int*,          \
                                             const int*, const int*, int, int, int,           \
                                             const long*, int, long, double*, cudaStream_t);  \
  template cudaError_t launch_norms<real>(const real*, const long*, int, double*, int,        \
                                          double*, cudaStream_t);                             \
  template cudaError_t launch_dots<real>(const real*, const real*, const long*, int, double*, \
                                         int, double*, cudaStream_t);                         \
  template cudaError_t launch_time_accum<real>(const real*, long, long, const DevBlock*,      \
                                               const double*, int, int, long, const long*,    \
                                               int, double*, cudaStream_t);                   \
  template cudaError_t launch_axpy_seg<real>(real*, const real*, const double*, double, long, \
                                             long, const DevBlock*, cudaStream_t);            \
  template cudaError_t launch_rscale_seg<real>(real*, const double*, long, long,              \
                                               const DevBlock*, cudaStream_t);

MW3_INST(double)
MW3_INST(float)

}  // namespace mw3
