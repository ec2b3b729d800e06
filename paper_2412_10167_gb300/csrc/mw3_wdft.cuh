// Register DFT building blocks and the half-warp kinetic transform of one line pair, shared
// by the warp-level radial kernels (mw3_kinetic_w.cu) and the fused radial kernel
// (mw3_radial.cu). Device code only; every definition sits in an unnamed namespace, so each
// translation unit that includes this header owns its copy.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mw3_internal.h"

namespace mw3 {
namespace {

__device__ constexpr double kCos48[48] = {1.00000000000000000000,0.99144486137381038215,0.96592582628906831221,0.92387953251128673848,0.86602540378443870761,0.79335334029123516508,0.70710678118654757274,0.60876142900872065589,0.50000000000000011102,0.38268343236508983729,0.25881904510252073948,0.13052619222005171218,0.00000000000000006123,-0.13052619222005160116,-0.25881904510252062845,-0.38268343236508950422,-0.49999999999999977796,-0.60876142900872065589,-0.70710678118654746172,-0.79335334029123505406,-0.86602540378443870761,-0.92387953251128673848,-0.96592582628906820119,-0.99144486137381038215,-1.00000000000000000000,-0.99144486137381038215,-0.96592582628906831221,-0.92387953251128684951,-0.86602540378443881863,-0.79335334029123516508,-0.70710678118654790580,-0.60876142900872087793,-0.50000000000000044409,-0.38268343236508950422,-0.25881904510252062845,-0.13052619222005162891,-0.00000000000000018370,0.13052619222005126809,0.25881904510252029539,0.38268343236508917116,0.50000000000000011102,0.60876142900871987873,0.70710678118654735069,0.79335334029123494304,0.86602540378443837454,0.92387953251128684951,0.96592582628906809017,0.99144486137381038215};
__device__ constexpr double kSin48[48] = {0.00000000000000000000,0.13052619222005157340,0.25881904510252073948,0.38268343236508978178,0.49999999999999994449,0.60876142900872065589,0.70710678118654746172,0.79335334029123516508,0.86602540378443859659,0.92387953251128673848,0.96592582628906831221,0.99144486137381038215,1.00000000000000000000,0.99144486137381038215,0.96592582628906831221,0.92387953251128684951,0.86602540378443870761,0.79335334029123516508,0.70710678118654757274,0.60876142900872087793,0.49999999999999994449,0.38268343236508989280,0.25881904510252101703,0.13052619222005198973,0.00000000000000012246,-0.13052619222005176769,-0.25881904510252079499,-0.38268343236508967076,-0.49999999999999972244,-0.60876142900872065589,-0.70710678118654712865,-0.79335334029123494304,-0.86602540378443837454,-0.92387953251128684951,-0.96592582628906831221,-0.99144486137381038215,-1.00000000000000000000,-0.99144486137381049318,-0.96592582628906842324,-0.92387953251128696053,-0.86602540378443859659,-0.79335334029123572019,-0.70710678118654768376,-0.60876142900872087793,-0.50000000000000044409,-0.38268343236508955973,-0.25881904510252157214,-0.13052619222005168442};

template <typename T>
__device__ __forceinline__ cpx<T> cm(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cmc(cpx<T> a, cpx<T> b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> ca(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cs(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }

// exp(sign 2 pi i e / R), e in [0, R), R dividing 48
template <typename T, int R>
__device__ __forceinline__ cpx<T> wR(int e, T sign) {
  const int m = (e % R) * (48 / R);
  return {(T)kCos48[m], sign * (T)kSin48[m]};
}

template <typename T>
__device__ __forceinline__ void d2(cpx<T>* v) {
  cpx<T> a = v[0];
  v[0] = ca(a, v[1]);
  v[1] = cs(a, v[1]);
}
template <typename T>
__device__ __forceinline__ void d3(cpx<T>* v, T sign) {
  const T h = (T)0.86602540378443864676;
  cpx<T> a = v[0], t1 = ca(v[1], v[2]);
  cpx<T> t2 = {a.x - (T)0.5 * t1.x, a.y - (T)0.5 * t1.y};
  cpx<T> d = cs(v[1], v[2]);
  cpx<T> t3 = {-d.y * h * sign, d.x * h * sign};
  v[0] = ca(a, t1);
  v[1] = ca(t2, t3);
  v[2] = cs(t2, t3);
}
template <typename T>
__device__ __forceinline__ void d4(cpx<T>* v, T sign) {
  cpx<T> s0 = ca(v[0], v[2]), s1 = cs(v[0], v[2]), s2 = ca(v[1], v[3]), e = cs(v[1], v[3]);
  cpx<T> s3 = {-e.y * sign, e.x * sign};
  v[0] = ca(s0, s2);
  v[1] = ca(s1, s3);
  v[2] = cs(s0, s2);
  v[3] = cs(s1, s3);
}

template <typename T, int R>
__device__ __forceinline__ void dftR(cpx<T>* v, T sign);

// R = R1 R2: X[k1 + R1 k2] = sum_n2 w_R^(n2 k1) w_R2^(n2 k2) sum_n1 v[R2 n1 + n2] w_R1^(n1 k1)
template <typename T, int R1, int R2>
__device__ __forceinline__ void dft_composite(cpx<T>* v, T sign) {
  constexpr int R = R1 * R2;
  cpx<T> y[R];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    cpx<T> u[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) u[n1] = v[R2 * n1 + n2];
    dftR<T, R1>(u, sign);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
      y[n2 * R1 + k1] = (n2 * k1 == 0) ? u[k1] : cm(u[k1], wR<T, R>(n2 * k1, sign));
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cpx<T> z[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) z[n2] = y[n2 * R1 + k1];
    dftR<T, R2>(z, sign);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = z[k2];
  }
}

template <typename T, int R>
__device__ __forceinline__ void dftR(cpx<T>* v, T sign) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    d2(v);
  } else if constexpr (R == 3) {
    d3(v, sign);
  } else if constexpr (R == 4) {
    d4(v, sign);
  } else if constexpr (R == 6) {
    dft_composite<T, 2, 3>(v, sign);
  } else if constexpr (R == 8) {
    dft_composite<T, 2, 4>(v, sign);
  } else if constexpr (R == 12) {
    dft_composite<T, 4, 3>(v, sign);
  } else {
    dft_composite<T, 4, 4>(v, sign);  // 16
  }
}

// 16-byte asynchronous global -> shared copy (L2 only).
template <typename T>
__device__ __forceinline__ void cp_async16_ca(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}

// ===================================================================== half-warp form
// FP32 lines of length N = 16 * N1 (N1 = 8, 12, 16). One line pair per half-warp: lane t
// (t < 16) holds the elements n = 16 n1 + t (n1 < N1) of the packed sequence z = a + i b
// (after the sign and permutation of the DST-via-FFT). With n = 16 n1 + n2 and
// k = k1 + N1 k2 the forward transform is
//   Z[k1 + N1 k2] = sum_n2 w_16^(n2 k2) [ w_N^(n2 k1) sum_n1 z[16 n1 + n2] w_N1^(n1 k1) ]:
// an N1-point DFT over n1 in registers on lane n2, the twiddle, an exchange through the
// pair's own shared-memory storage, and a 16-point DFT over n2 on lane k1 < N1, which then
// holds Z[k1 + N1 k2] in slot k2. After the spectral scale W_k = sigma_k Z_k + f_k Z_(N-k)
// (the partner read back from shared memory) the inverse runs the same steps mirrored
// (16-point DFT over k2 on lane k1, twiddle w_N^(-n2 k1), exchange, N1-point DFT over k1
// on lane n2), so lane t ends with element 16 n1 + t and every value returns to the
// location it was read from. Exchange slot of (lane a, index b): (a xor b) + 16 b, so the
// 16 lanes of an exchange access 16 different banks. The partner values of the spectral
// scale come by shuffles within the half-warp. Lane synchronisation is per
// half-warp (the two halves of a warp may run different pairs, or one of them none), so
// the caller's blockDim.x is a multiple of 32 and each pair's 16 lanes are one half-warp.
template <int N1>
__device__ __forceinline__ int hw_xj(int a, int b) {
  return (a ^ b) + 16 * b;
}

// tw16[j * 16 + t] = w_N^(t j) (j < 16), sig[k] = sigma_k, fk[k] = f_k (shared memory).
// Element n = 16 n1 + t of the packed sequence sits at i = 2n for n1 < N1/2 (sign +) and
// at i = 2N - 1 - 2n for n1 >= N1/2 (sign -), so its address is lane-base + constant.
template <int N1, bool SHFL>
__device__ __forceinline__ void hw_pair_kinetic(float* __restrict__ xa, float* __restrict__ xb,
                                                int st, int t, const cpx<float>* tw16,
                                                const float* sig, const cpx<float>* fk) {
  constexpr int N = 16 * N1;
  // the 16 lanes of this half-warp only: the other half may work on another pair or none
  const unsigned hm = 0xffffu << (threadIdx.x & 16);
  float* const pa_lo = xa + 2 * t * st;                 // i = 32 n1 + 2t
  float* const pb_lo = xb + 2 * t * st;
  float* const pa_hi = xa + (2 * N - 1 - 2 * t) * st;   // i = 2N - 1 - 32 n1 - 2t
  float* const pb_hi = xb + (2 * N - 1 - 2 * t) * st;
  cpx<float> v[16];
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    if (n1 < N1 / 2) v[n1] = {pa_lo[32 * n1 * st], pb_lo[32 * n1 * st]};
    else v[n1] = {-pa_hi[-32 * n1 * st], -pb_hi[-32 * n1 * st]};
  }
  dftR<float, N1>(v, -1.0f);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) v[k1] = cm(v[k1], tw16[k1 * 16 + t]);
  __syncwarp(hm);                      // every lane's loads precede the exchange writes
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    const int j = hw_xj<N1>(t, k1);
    xa[j * st] = v[k1].x;
    xb[j * st] = v[k1].y;
  }
  __syncwarp(hm);
  if (t < N1) {
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      const int j = hw_xj<N1>(n2, t);
      v[n2] = {xa[j * st], xb[j * st]};
    }
    dftR<float, 16>(v, -1.0f);         // v[k2] = Z[t + N1 k2]
  }
  // spectral scale; the partner Z[N - k] of lane t, slot k2 is slot 15 - k2 of lane N1 - t
  // (lane 0: its own slot (16 - k2) mod 16), fetched by shuffles (SHFL) or written to and
  // read back from the pair's storage
  if constexpr (!SHFL) {
    __syncwarp(hm);
    if (t < N1) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int k = t + N1 * k2;
        xa[k * st] = v[k2].x;
        xb[k * st] = v[k2].y;
      }
    }
    __syncwarp(hm);
    if (t < N1) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const int k = t + N1 * k2;
        const int p = k == 0 ? 0 : N - k;
        const cpx<float> fz = cm(fk[k], cpx<float>{xa[p * st], xb[p * st]});
        const float sg = sig[k];
        v[k2] = {sg * v[k2].x + fz.x, sg * v[k2].y + fz.y};
      }
    }
  } else {
    // every partner is read from the unscaled values z (a register copy), never from a slot
    // that this loop has already overwritten
    cpx<float> z[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) z[k2] = v[k2];
    const int src = ((t == 0 || t >= N1) ? t : N1 - t) | (threadIdx.x & 16);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      const cpx<float> far = {__shfl_sync(hm, z[15 - k2].x, src), __shfl_sync(hm, z[15 - k2].y, src)};
      const cpx<float> zp = t == 0 ? z[(16 - k2) & 15] : far;
      if (t < N1) {
        const int k = t + N1 * k2;
        const cpx<float> fz = cm(fk[k], zp);
        const float sg = sig[k];
        v[k2] = {sg * z[k2].x + fz.x, sg * z[k2].y + fz.y};
      }
    }
  }
  if (t < N1) {
    dftR<float, 16>(v, 1.0f);          // over k2: v[n2]
#pragma unroll
    for (int n2 = 1; n2 < 16; ++n2) v[n2] = cmc(v[n2], tw16[n2 * 16 + t]);   // w_N^(-n2 t)
  }
  __syncwarp(hm);                      // every exchange read precedes the exchange writes
  if (t < N1) {
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      const int j = hw_xj<N1>(n2, t);
      xa[j * st] = v[n2].x;
      xb[j * st] = v[n2].y;
    }
  }
  __syncwarp(hm);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    const int j = hw_xj<N1>(t, k1);
    v[k1] = {xa[j * st], xb[j * st]};
  }
  dftR<float, N1>(v, 1.0f);            // v[n1] = element 16 n1 + t
  __syncwarp(hm);                      // every exchange read precedes the result writes
#pragma unroll
  for (int n1 = 0; n1 < N1; ++n1) {
    if (n1 < N1 / 2) {
      pa_lo[32 * n1 * st] = v[n1].x;
      pb_lo[32 * n1 * st] = v[n1].y;
    } else {
      pa_hi[-32 * n1 * st] = -v[n1].x;
      pb_hi[-32 * n1 * st] = -v[n1].y;
    }
  }
}

// Per-CTA tables of the half-warp form (FP32): twiddles w_N^(t j) for t, j < 16 and the
// spectral scale of every natural index k (sigma_k, f_k as in the warp-register form).
template <int N1>
struct HwTables {
  cpx<float> tw16[256];
  cpx<float> fk[16 * N1];
  float sig[16 * N1];
};

template <int N1>
__device__ __forceinline__ void hw_load_tables(HwTables<N1>& tb, const cpx<float>* __restrict__ twg,
                                               const cpx<float>* __restrict__ phg,
                                               const float* __restrict__ lamg) {
  constexpr int N = 16 * N1;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    const int j = e >> 4, t = e & 15;
    tb.tw16[e] = twg[(t * j) % N];
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const float lr = lamg[N - k], li = lamg[k];
    const cpx<float> e1 = phg[k];
    const cpx<float> e2 = {e1.x * e1.x - e1.y * e1.y, -2.0f * e1.x * e1.y};
    const float dl = 0.5f * (lr - li);
    tb.sig[k] = 0.5f * (lr + li);
    tb.fk[k] = {dl * e2.x, dl * e2.y};
  }
}

}  // namespace
}  // namespace mw3
