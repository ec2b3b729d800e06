// Compile-time-sized Stockham FFT building blocks (shared memory, one CTA works on
// P independent lines of length N). Radix-16 and radix-8 butterflies are composed in
// registers from radix-4/2 passes with constant inner twiddles, so a 256-point
// transform takes two shared-memory passes. All index arithmetic is by constants.
#pragma once

#include "mw3_internal.h"

namespace mw3 {
namespace fftc {

template <typename T>
__device__ __forceinline__ cpx<T> mul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> add(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> sub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> muli(cpx<T> a, T s) { return {-a.y * s, a.x * s}; }  // a * (i s)

// exp(sign * 2 pi i e / 16) for e = 0..15
template <typename T>
__device__ __forceinline__ cpx<T> w16(int e, T sign) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173,
          c2 = (T)0.70710678118654752440;
  T cr, ci;
  switch (e & 15) {
    case 0: cr = 1; ci = 0; break;
    case 1: cr = c1; ci = s1; break;
    case 2: cr = c2; ci = c2; break;
    case 3: cr = s1; ci = c1; break;
    case 4: cr = 0; ci = 1; break;
    case 5: cr = -s1; ci = c1; break;
    case 6: cr = -c2; ci = c2; break;
    case 7: cr = -c1; ci = s1; break;
    case 8: cr = -1; ci = 0; break;
    case 9: cr = -c1; ci = -s1; break;
    case 10: cr = -c2; ci = -c2; break;
    case 11: cr = -s1; ci = -c1; break;
    case 12: cr = 0; ci = -1; break;
    case 13: cr = s1; ci = -c1; break;
    case 14: cr = c2; ci = -c2; break;
    default: cr = c1; ci = -s1; break;
  }
  return {cr, sign * ci};
}

template <typename T>
__device__ __forceinline__ void dft2(cpx<T>& a, cpx<T>& b) {
  cpx<T> t = a;
  a = add(t, b);
  b = sub(t, b);
}

template <typename T>
__device__ __forceinline__ void dft4(cpx<T>* v, T sign) {
  cpx<T> s0 = add(v[0], v[2]), s1 = sub(v[0], v[2]), s2 = add(v[1], v[3]),
         s3 = muli(sub(v[1], v[3]), sign);
  v[0] = add(s0, s2);
  v[1] = add(s1, s3);
  v[2] = sub(s0, s2);
  v[3] = sub(s1, s3);
}

template <typename T>
__device__ __forceinline__ void dft3(cpx<T>* v, T sign) {
  const T h = (T)0.86602540378443864676;
  cpx<T> a = v[0], t1 = add(v[1], v[2]);
  cpx<T> t2 = {a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y};
  cpx<T> d = sub(v[1], v[2]);
  cpx<T> t3 = muli(cpx<T>{d.x * h, d.y * h}, sign);
  v[0] = add(a, t1);
  v[1] = add(t2, t3);
  v[2] = sub(t2, t3);
}

template <typename T>
__device__ __forceinline__ void dft5(cpx<T>* v, T sign) {
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410,
          s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
  cpx<T> a = v[0];
  cpx<T> t1 = add(v[1], v[4]), t2 = add(v[2], v[3]), t3 = sub(v[1], v[4]), t4 = sub(v[2], v[3]);
  cpx<T> m1 = {a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
  cpx<T> m2 = {a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
  cpx<T> n1 = muli(cpx<T>{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y}, sign);
  cpx<T> n2 = muli(cpx<T>{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y}, sign);
  v[0] = add(a, add(t1, t2));
  v[1] = add(m1, n1);
  v[4] = sub(m1, n1);
  v[2] = add(m2, n2);
  v[3] = sub(m2, n2);
}

// R-point DFT, R = R1 * R2 composed in registers: X[k1 + R1 k2] =
// sum_n2 w_R^(n2 k1) w_R2^(n2 k2) sum_n1 v[R2 n1 + n2] w_R1^(n1 k1).
template <typename T, int R>
__device__ __forceinline__ void dft(cpx<T>* v, T sign) {
  if constexpr (R == 2) {
    dft2(v[0], v[1]);
  } else if constexpr (R == 3) {
    dft3(v, sign);
  } else if constexpr (R == 4) {
    dft4(v, sign);
  } else if constexpr (R == 5) {
    dft5(v, sign);
  } else {
    constexpr int R1 = (R == 8) ? 2 : 4;
    constexpr int R2 = R / R1;  // 4
    cpx<T> y[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      cpx<T> u[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) u[n1] = v[R2 * n1 + n2];
      dft<T, R1>(u, sign);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int e = (16 / R) * n2 * k1;  // exponent in units of 2 pi / 16
        y[n2 * R1 + k1] = (n2 * k1 == 0) ? u[k1] : mul(u[k1], w16<T>(e, sign));
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cpx<T> z[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) z[n2] = y[n2 * R1 + k1];
      dft4(z, sign);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = z[k2];
    }
  }
}

template <int Rem, int MaxR>
struct pick_radix {
  static constexpr int value = (MaxR >= 16 && Rem % 16 == 0 && Rem != 32) ? 16
                               : (MaxR >= 8 && Rem % 8 == 0)               ? 8
                               : (Rem % 4 == 0)             ? 4
                               : (Rem % 2 == 0)             ? 2
                               : (Rem % 3 == 0)             ? 3
                                                            : 5;
};

// One Stockham stage: P lines of length N, contiguous, tw[t] = exp(-2 pi i t / N).
template <typename T, int N, int R, int Ns>
__device__ __forceinline__ void stage(const cpx<T>* __restrict__ in, cpx<T>* __restrict__ out,
                                     int P, const cpx<T>* __restrict__ tw, T sign) {
  constexpr int nb = N / R;
  constexpr int tstride = N / (Ns * R);
  const int total = P * nb;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int p = idx / nb;
    const int j = idx - p * nb;
    const int k = j % Ns;
    const cpx<T>* src = in + p * N;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cpx<T> x = src[j + r * nb];
      if (r > 0 && Ns > 1) {
        cpx<T> w = tw[r * k * tstride];
        if (sign > 0) w.y = -w.y;
        x = mul(x, w);
      }
      v[r] = x;
    }
    dft<T, R>(v, sign);
    cpx<T>* dst = out + p * N + (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns] = v[r];
  }
}

// Full transform; returns the buffer that holds the result.
template <typename T, int N, int Ns = 1>
__device__ __forceinline__ cpx<T>* fft(cpx<T>* a, cpx<T>* b, int P, const cpx<T>* tw, T sign) {
  if constexpr (Ns >= N) {
    return a;
  } else {
    constexpr int R = pick_radix<N / Ns, sizeof(T) == 8 ? 8 : 16>::value;
    stage<T, N, R, Ns>(a, b, P, tw, sign);
    __syncthreads();
    return fft<T, N, Ns * R>(b, a, P, tw, sign);
  }
}

}  // namespace fftc
}  // namespace mw3
