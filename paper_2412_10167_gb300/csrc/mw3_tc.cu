// Fused angular step on the 5th-generation tensor cores (mixed precision).
//
// One CTA handles 128 grid columns (r, R) of one (J, Omega) group (all its
// electronic states) and performs, per state L (Section 2.1 items 3-5, Eq. wvp-k):
//   GEMM 1   u_L^T[col][n] = sum_i c_L^T[col][i] T^Omega[i][n]          (FBR -> DVR)
//   potential (V u)_L[col][n] = sum_L' V_LL'[n][col] u_L'[col][n]
//   GEMM 2   w_L^T[col][i] = sum_n (V u)_L^T[col][n] T^Omega[i][n]     (DVR -> FBR)
//   epilogue h = w + a_j c + bp_j c^(Omega+1)_(j) + bm_j c^(Omega-1)_(j) + t,
//            c_(k+1) = D (alpha (h/dE - (E0/dE) c) - beta D c_(k-1)), norm partials.
// M = 128 grid columns (TMEM lanes), N = K = ngamma padded to a multiple of 16.
// FP32 accuracy from TF32 tensor cores by splitting every operand x = hi + lo
// (hi = x rounded to TF32, lo = x - hi exactly) and accumulating hi*hi + hi*lo + lo*hi
// in FP32 (the dropped lo*lo term is ~2^-22 relative).
//
// Operands are staged in shared memory in the canonical no-swizzle K-major layout:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (leading
// byte offset), 8-row groups K*4*8/... (stride byte offset = K * 32 B). One elected
// thread issues tcgen05.mma; completion is signalled through an mbarrier by
// tcgen05.commit; every wait is bounded and reports through an error word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mw3_internal.h"

namespace mw3 {

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 512;
constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) of a K-major core-matrix tile whose K extent is kp
__device__ __forceinline__ uint32_t cm_off(int row, int k, int kp) {
  return (uint32_t)((row >> 3) * (kp * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version (tcgen05); base offset 0; no swizzle
  return d;
}

// instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
               "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D (+)= A B with A (M x K, K-major) read from tensor memory
__device__ __forceinline__ void mma_tf32_ta(uint32_t dtmem, uint32_t atmem, uint64_t bd,
                                            uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "r"(atmem), "l"(bd), "r"(idesc), "r"(accum));
}

// Copy a padded kp x kp FP32 matrix pair (hi, lo), row-major, into core-matrix layout.
__device__ void load_b(const float* __restrict__ hi, const float* __restrict__ lo,
                       unsigned char* Bhi, unsigned char* Blo, int kp) {
  const int nq = kp * kp / 4;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int row = e / (kp / 4);
    const int k4 = (e - row * (kp / 4)) * 4;
    const float4 h = *reinterpret_cast<const float4*>(hi + (long)row * kp + k4);
    const float4 l = *reinterpret_cast<const float4*>(lo + (long)row * kp + k4);
    const uint32_t off = cm_off(row, k4, kp);
    *reinterpret_cast<float4*>(Bhi + off) = h;
    *reinterpret_cast<float4*>(Blo + off) = l;
  }
}

// 3 x (kp / 8) MMAs: D (+)= Ahi Bhi + Ahi Blo + Alo Bhi over K = kp.
__device__ void issue_split_gemm(uint32_t dtmem, const unsigned char* Ahi, const unsigned char* Alo,
                                 const unsigned char* Bhi, const unsigned char* Blo, int kp,
                                 uint32_t idesc) {
  const uint32_t sbo = (uint32_t)kp * 32, lbo = 128;
  const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
  for (int ks = 0; ks < kp / 8; ++ks) {
    const uint32_t o = (uint32_t)ks * 256;  // two core matrices along K per K-step of 8
    mma_tf32(dtmem, smem_desc(ah + o, lbo, sbo), smem_desc(bh + o, lbo, sbo), idesc, ks > 0);
    mma_tf32(dtmem, smem_desc(ah + o, lbo, sbo), smem_desc(bl + o, lbo, sbo), idesc, 1);
    mma_tf32(dtmem, smem_desc(al + o, lbo, sbo), smem_desc(bh + o, lbo, sbo), idesc, 1);
  }
}

// As issue_split_gemm, with A (hi, lo) in tensor-memory columns [ahi, ahi + kp) and
// [alo, alo + kp): one K-step of 8 TF32 values is 8 columns.
__device__ void issue_split_gemm_ta(uint32_t dtmem, uint32_t ahi, uint32_t alo,
                                    const unsigned char* Bhi, const unsigned char* Blo, int kp,
                                    uint32_t idesc) {
  const uint32_t sbo = (uint32_t)kp * 32, lbo = 128;
  const uint32_t bh = smem_u32(Bhi), bl = smem_u32(Blo);
  for (int ks = 0; ks < kp / 8; ++ks) {
    const uint32_t o = (uint32_t)ks * 256, ta = (uint32_t)ks * 8;
    mma_tf32_ta(dtmem, ahi + ta, smem_desc(bh + o, lbo, sbo), idesc, ks > 0);
    mma_tf32_ta(dtmem, ahi + ta, smem_desc(bl + o, lbo, sbo), idesc, 1);
    mma_tf32_ta(dtmem, alo + ta, smem_desc(bh + o, lbo, sbo), idesc, 1);
  }
}

}  // namespace



template <int KP, int NE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_angular_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int kp = KP;
  const size_t abytes = (size_t)TC_M * kp * 4, bbytes = (size_t)kp * kp * 4;
  unsigned char* Ahi = sm;
  unsigned char* Alo = Ahi + abytes;
  unsigned char* Bhi = Alo + abytes;
  unsigned char* Blo = Bhi + bbytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + bbytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  double* red = reinterpret_cast<double*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;          // TMEM lane quarter
  const int half = warp >> 2;      // which quarter of the N columns this warp reads
  const int m = q * 32 + lane;     // tile row = grid column within the tile
  // grid (group, tile): the helicity groups of one tile run side by side, so the
  // Coriolis neighbours' tiles (Omega +- 1) are read from L2
  const int g = blockIdx.x;
  const int tile = blockIdx.y;
  const long col = (long)tile * TC_M + m;
  const bool live = col < a.ncol;
  const int b0 = g * NE;
  const DevBlock B0 = a.blocks[b0];
  const int om = B0.omega;
  const int nrow = B0.nrow;
  const uint32_t mb = smem_u32(mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  bool ok = true;
  const uint32_t idesc = idesc_tf32(TC_M, kp);
  constexpr int ncb = kp / 4;       // columns per quarter (a multiple of 4)
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;

  // ---------------------------------------------------------- GEMM 1 (per state)
  load_b(a.Tt_hi + (long)om * kp * kp, a.Tt_lo + (long)om * kp * kp, Bhi, Blo, kp);
  for (int L = 0; L < NE && ok; ++L) {
    const float* c = a.ck + (long)(b0 + L) * a.npts;
    // A[m][i] = c[i][col0 + m], split; rows beyond the block's functions or the grid are 0.
    // All of a thread's global loads are issued before any is used.
    constexpr int nq = TC_M * (kp / 4);
    constexpr int kMaxItems = (nq + TC_THREADS - 1) / TC_THREADS;
    float x[kMaxItems][4];
#pragma unroll
    for (int it = 0; it < kMaxItems; ++it) {
      const int e = tid + it * TC_THREADS;
      const int i4 = (e / TC_M) * 4;
      const int mm = e - (e / TC_M) * TC_M;
      const long cc = (long)tile * TC_M + mm;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        x[it][u] = (e < nq && cc < a.ncol && i4 + u < nrow) ? __ldg(c + (long)(i4 + u) * a.ncol + cc) : 0.0f;
    }
#pragma unroll
    for (int it = 0; it < kMaxItems; ++it) {
      const int e = tid + it * TC_THREADS;
      if (e >= nq) break;
      const int i4 = (e / TC_M) * 4;
      const int mm = e - (e / TC_M) * TC_M;
      float4 h, l;
      h.x = tf32_hi(x[it][0]); l.x = x[it][0] - h.x;
      h.y = tf32_hi(x[it][1]); l.y = x[it][1] - h.y;
      h.z = tf32_hi(x[it][2]); l.z = x[it][2] - h.z;
      h.w = tf32_hi(x[it][3]); l.w = x[it][3] - h.w;
      const uint32_t off = cm_off(mm, i4, kp);
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_split_gemm(tmem + (uint32_t)(L * kp), Ahi, Alo, Bhi, Blo, kp, idesc);
      mma_commit(mb);
    }
    ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;  // CTA-uniform
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
  }

  // ---------------------------------------------------------- potential + GEMM 2
  if (ok) {
    __syncthreads();
    load_b(a.T_hi + (long)om * kp * kp, a.T_lo + (long)om * kp * kp, Bhi, Blo, kp);
  }
  const int kr = live ? (int)(col / a.NR) : 0;
  const int mR = live ? (int)(col - (long)kr * a.NR) : 0;
  for (int L = 0; L < NE && ok; ++L) {
    // (V u)_L[m][n] for this thread's quarter of n: V loads first, then TMEM
    float vv[NE][ncb];
#pragma unroll
    for (int Lp = 0; Lp < NE; ++Lp) {
      const float* V = a.V + (long)(L * NE + Lp) * a.npts;
#pragma unroll
      for (int s2 = 0; s2 < ncb; ++s2) {
        const int n = half * ncb + s2;
        vv[Lp][s2] = (live && n < a.ng) ? __ldg(V + (long)n * a.ncol + col) : 0.0f;
      }
    }
#pragma unroll
    for (int s0 = 0; s0 < ncb; s0 += 4) {
      float vu[4] = {0, 0, 0, 0};
#pragma unroll
      for (int Lp = 0; Lp < NE; ++Lp) {
        float u[4];
        tmem_ld4(tmem + lane_base + (uint32_t)(Lp * kp + half * ncb + s0), u);
#pragma unroll
        for (int s = 0; s < 4; ++s) vu[s] += vv[Lp][s0 + s] * u[s];
      }
      float4 h, l;
      h.x = tf32_hi(vu[0]); l.x = vu[0] - h.x;
      h.y = tf32_hi(vu[1]); l.y = vu[1] - h.y;
      h.z = tf32_hi(vu[2]); l.z = vu[2] - h.z;
      h.w = tf32_hi(vu[3]); l.w = vu[3] - h.w;
      const uint32_t off = cm_off(m, half * ncb + s0, kp);
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_split_gemm(tmem + (uint32_t)((NE + L) * kp), Ahi, Alo, Bhi, Blo, kp, idesc);
      mma_commit(mb);
    }
    ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;  // CTA-uniform
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
  }

  // ---------------------------------------------------------- epilogue
  double ss = 0.0;
  if (ok) {
    const DevJ J = a.dj[B0.iJ];
    const float* cf = a.coef + (long)B0.coef * kCoefRows * a.ng;
    const float D = live ? a.DR[mR] * a.Dr[kr] : 0.0f;
    const float frk = live ? a.fr[kr] : 0.0f;
    const float fRm = live ? a.fR[mR] : 0.0f;
    float* ts = reinterpret_cast<float*>(Ahi);              // [kp][TC_M] t tile
    float* ps = reinterpret_cast<float*>(Ahi) + kp * TC_M;  // [kp][TC_M] c_(k-1) tile
    const long col0 = (long)tile * TC_M;
    for (int L = 0; L < NE; ++L) {
      const int b = b0 + L;
      const DevBlock Bb = a.blocks[b];
      const float* c = a.ck + (long)b * a.npts;
      // one round trip: 16-byte asynchronous copies of this block's t and c_(k-1)
      // rows [0, nrow) x [col0, col0 + 128) (ncol is a multiple of 4, so a 4-float chunk
      // is entirely inside or outside the grid)
      __syncthreads();
      {
        const int nch = nrow * (TC_M / 4);
        for (int e = tid; e < nch; e += TC_THREADS) {
          const int i = e / (TC_M / 4);
          const int c4 = (e - i * (TC_M / 4)) * 4;
          if (col0 + c4 >= a.ncol) continue;
          const long go = (long)b * a.npts + (long)i * a.ncol + col0 + c4;
          cp_async16(ts + i * TC_M + c4, a.t + go);
          if (a.mode == 0) cp_async16(ps + i * TC_M + c4, a.ckm1 + go);
        }
        cp_async_wait_all();
      }
      __syncthreads();
      for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 4) {
        float w[4];
        tmem_ld4(tmem + lane_base + (uint32_t)((NE + L) * kp + i0), w);
        if (!live) continue;
        // issue every global load of the chunk before using any
        float cv[4], cu[4], cd[4], tv[4], pv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int i = i0 + s;
          const bool in = i < nrow;
          const long off = (long)i * a.ncol + col;
          cv[s] = in ? __ldg(c + off) : 0.0f;
          tv[s] = in ? ts[i * TC_M + m] : 0.0f;
          pv[s] = (in && a.mode == 0) ? ps[i * TC_M + m] : 0.0f;
          cu[s] = (in && Bb.up >= 0 && i >= 1) ? __ldg(a.ck + (long)Bb.up * a.npts + off - a.ncol) : 0.0f;
          cd[s] = (in && Bb.dn >= 0) ? __ldg(a.ck + (long)Bb.dn * a.npts + off + a.ncol) : 0.0f;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int i = i0 + s;
          if (i >= a.ng) break;
          const long idx = (long)b * a.npts + (long)i * a.ncol + col;
          if (i >= nrow) {
            if (a.mode == 1) a.out[idx] = 0.0f; else a.ckm1[idx] = 0.0f;
            continue;
          }
          const float g = fminf(fRm, cf[4 * a.ng + i]);
          const float aa = fminf(cf[i] * frk, a.erot) + g * cf[a.ng + i];
          float h = w[s] + aa * cv[s] + tv[s];
          h += g * cf[2 * a.ng + i] * cu[s];
          h += g * cf[3 * a.ng + i] * cd[s];
          const float hs = h * (float)J.invdE - (float)J.e0s * cv[s];
          if (a.mode == 1) {
            a.out[idx] = hs;
          } else {
            const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
            a.ckm1[idx] = nv;
            ss += (double)nv * (double)nv;
          }
        }
      }
    }
  }
  // norm partial of this CTA (fixed-order reduction)
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0) {
    double s = 0;
    for (int w2 = 0; w2 < TC_THREADS / 32; ++w2) s += red[w2];
    if (a.npart) a.npart[(long)g * a.ntiles + tile] = s;
    if (!ok) atomicExch(a.err, 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}


// ===================================================================== persistent form
// One CTA per SM walks a contiguous range of the (group, tile) list, group-major, so
// it keeps T^Omega and its transpose (hi and lo parts) resident in shared memory
// until the helicity changes; the data operand of both GEMMs goes to tensor memory
// with tcgen05.st (no shared-memory staging, no operand reload per tile). Sibling
// CTAs sit ntiles / (tiles per CTA) apart in the list, so the helicity groups of one
// tile are processed at about the same time and the Coriolis neighbours come from L2.
// Tensor-memory columns: A hi [0, kp), A lo [kp, 2kp), u_L at (2 + L) kp; w_0 at
// (2 + NE) kp when NE = 2 (else it reuses u_0), w_1 reuses u_0.
template <int KP>
constexpr size_t tc2_bbytes() { return (size_t)KP * KP * 4; }
template <int KP>
constexpr bool tc2_stage_t() { return 4 * tc2_bbytes<KP>() + (size_t)KP * TC_M * 4 + 1024 <= 227 * 1024; }
template <int KP>
constexpr size_t tc2_smem() {
  return 4 * tc2_bbytes<KP>() + (tc2_stage_t<KP>() ? (size_t)KP * TC_M * 4 : 0) + 16 +
         16 * sizeof(double) + 64;
}

template <int KP, int NE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_angular_tc2(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int kp = KP;
  constexpr size_t bbytes = tc2_bbytes<KP>();
  constexpr bool stage_t = tc2_stage_t<KP>();
  unsigned char* B1hi = sm;              // (T^Omega)^T: GEMM 1
  unsigned char* B1lo = B1hi + bbytes;
  unsigned char* B2hi = B1lo + bbytes;   // T^Omega: GEMM 2
  unsigned char* B2lo = B2hi + bbytes;
  float* ts = reinterpret_cast<float*>(B2lo + bbytes);                 // [kp][TC_M] t tile
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ts + (stage_t ? kp * TC_M : 0));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  double* red = reinterpret_cast<double*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;
  const int half = warp >> 2;
  const int m = q * 32 + lane;
  constexpr int ncb = kp / 4;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t idesc = idesc_tf32(TC_M, kp);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t tA_hi = tmem, tA_lo = tmem + kp;
  auto t_u = [&](int L) { return tmem + (uint32_t)((2 + L) * kp); };
  auto t_w = [&](int L) {
    return (NE == 1) ? tmem + (uint32_t)(2 * kp)
                     : (L == 0 ? tmem + (uint32_t)((2 + NE) * kp) : tmem + (uint32_t)(2 * kp));
  };
  uint32_t phase = 0;
  bool ok = true;
  int om_cur = -1;

  const long total = (long)a.ngroups * a.ntiles;
  const long f0 = (long)blockIdx.x * total / gridDim.x;
  const long f1 = (long)(blockIdx.x + 1) * total / gridDim.x;
  for (long f = f0; f < f1 && ok; ++f) {
    const int g = (int)(f / a.ntiles);
    const int tile = (int)(f - (long)g * a.ntiles);
    const int b0 = g * NE;
    const DevBlock B0 = a.blocks[b0];
    const int om = B0.omega;
    const int nrow = B0.nrow;
    const long col0 = (long)tile * TC_M;
    const long col = col0 + m;
    const bool live = col < a.ncol;
    const int kr = live ? (int)(col / a.NR) : 0;
    const int mR = live ? (int)(col - (long)kr * a.NR) : 0;

    __syncthreads();   // every thread is done with the shared buffers of the last tile
    if (om != om_cur) {
      load_b(a.Tt_hi + (long)om * kp * kp, a.Tt_lo + (long)om * kp * kp, B1hi, B1lo, kp);
      load_b(a.T_hi + (long)om * kp * kp, a.T_lo + (long)om * kp * kp, B2hi, B2lo, kp);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      om_cur = om;
    }
    // t rows of state 0 into shared memory while the GEMMs run
    if (stage_t) {
      const int nch = nrow * (TC_M / 4);
      for (int e = tid; e < nch; e += TC_THREADS) {
        const int i = e / (TC_M / 4);
        const int c4 = (e - i * (TC_M / 4)) * 4;
        if (col0 + c4 >= a.ncol) continue;
        cp_async16(ts + i * TC_M + c4, a.t + (long)b0 * a.npts + (long)i * a.ncol + col0 + c4);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // ------------------------------------------------------------ GEMM 1 per state
    for (int L = 0; L < NE && ok; ++L) {
      const float* c = a.ck + (long)(b0 + L) * a.npts;
      float x[ncb];
#pragma unroll
      for (int s2 = 0; s2 < ncb; ++s2) {
        const int i = half * ncb + s2;
        x[s2] = (live && i < nrow) ? __ldg(c + (long)i * a.ncol + col) : 0.0f;
      }
#pragma unroll
      for (int s0 = 0; s0 < ncb; s0 += 4) {
        float h[4], l[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          h[s] = tf32_hi(x[s0 + s]);
          l[s] = x[s0 + s] - h[s];
        }
        tmem_st4(tA_hi + lane_base + (uint32_t)(half * ncb + s0), h);
        tmem_st4(tA_lo + lane_base + (uint32_t)(half * ncb + s0), l);
      }
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue_split_gemm_ta(t_u(L), tA_hi, tA_lo, B1hi, B1lo, kp, idesc);
        mma_commit(mb);
      }
      ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }

    // ------------------------------------------------------------ potential + GEMM 2
    for (int L = 0; L < NE && ok; ++L) {
      float vv[NE][ncb];
#pragma unroll
      for (int Lp = 0; Lp < NE; ++Lp) {
        const float* V = a.V + (long)(L * NE + Lp) * a.npts;
#pragma unroll
        for (int s2 = 0; s2 < ncb; ++s2) {
          const int n = half * ncb + s2;
          vv[Lp][s2] = (live && n < a.ng) ? __ldg(V + (long)n * a.ncol + col) : 0.0f;
        }
      }
#pragma unroll
      for (int s0 = 0; s0 < ncb; s0 += 4) {
        float vu[4] = {0, 0, 0, 0};
#pragma unroll
        for (int Lp = 0; Lp < NE; ++Lp) {
          float u[4];
          tmem_ld4(t_u(Lp) + lane_base + (uint32_t)(half * ncb + s0), u);
#pragma unroll
          for (int s = 0; s < 4; ++s) vu[s] += vv[Lp][s0 + s] * u[s];
        }
        float h[4], l[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          h[s] = tf32_hi(vu[s]);
          l[s] = vu[s] - h[s];
        }
        tmem_st4(tA_hi + lane_base + (uint32_t)(half * ncb + s0), h);
        tmem_st4(tA_lo + lane_base + (uint32_t)(half * ncb + s0), l);
      }
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue_split_gemm_ta(t_w(L), tA_hi, tA_lo, B2hi, B2lo, kp, idesc);
        mma_commit(mb);
      }
      ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (stage_t) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
    }

    // ------------------------------------------------------------ epilogue
    double ss = 0.0;
    if (ok) {
      const DevJ J = a.dj[B0.iJ];
      const float* cf = a.coef + (long)B0.coef * kCoefRows * a.ng;
      const float D = live ? a.DR[mR] * a.Dr[kr] : 0.0f;
      const float frk = live ? a.fr[kr] : 0.0f;
      const float fRm = live ? a.fR[mR] : 0.0f;
      for (int L = 0; L < NE; ++L) {
        const int b = b0 + L;
        const DevBlock Bb = a.blocks[b];
        const float* c = a.ck + (long)b * a.npts;
        const bool tsm = stage_t && L == 0;
        for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 4) {
          float w[4];
          tmem_ld4(t_w(L) + lane_base + (uint32_t)i0, w);
          if (!live) continue;
          float cv[4], cu[4], cd[4], tv[4], pv[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int i = i0 + s;
            const bool in = i < nrow;
            const long off = (long)i * a.ncol + col;
            cv[s] = in ? __ldg(c + off) : 0.0f;
            tv[s] = in ? (tsm ? ts[i * TC_M + m] : __ldg(a.t + (long)b * a.npts + off)) : 0.0f;
            pv[s] = (in && a.mode == 0) ? __ldg(a.ckm1 + (long)b * a.npts + off) : 0.0f;
            cu[s] = (in && Bb.up >= 0 && i >= 1) ? __ldg(a.ck + (long)Bb.up * a.npts + off - a.ncol) : 0.0f;
            cd[s] = (in && Bb.dn >= 0) ? __ldg(a.ck + (long)Bb.dn * a.npts + off + a.ncol) : 0.0f;
          }
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int i = i0 + s;
            if (i >= a.ng) break;
            const long idx = (long)b * a.npts + (long)i * a.ncol + col;
            if (i >= nrow) {
              if (a.mode == 1) a.out[idx] = 0.0f; else a.ckm1[idx] = 0.0f;
              continue;
            }
            const float gg = fminf(fRm, cf[4 * a.ng + i]);
            const float aa = fminf(cf[i] * frk, a.erot) + gg * cf[a.ng + i];
            float h = w[s] + aa * cv[s] + tv[s];
            h += gg * cf[2 * a.ng + i] * cu[s];
            h += gg * cf[3 * a.ng + i] * cd[s];
            const float hs = h * (float)J.invdE - (float)J.e0s * cv[s];
            if (a.mode == 1) {
              a.out[idx] = hs;
            } else {
              const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
              a.ckm1[idx] = nv;
              ss += (double)nv * (double)nv;
            }
          }
        }
      }
    }
    // norm partial of this tile (the same fixed-order reduction as the one-tile form)
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if (lane == 0) red[warp] = ss;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      double s2 = 0;
      for (int w2 = 0; w2 < TC_THREADS / 32; ++w2) s2 += red[w2];
      if (a.npart) a.npart[(long)g * a.ntiles + tile] = s2;
    }
  }
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}

// out[iJ] = sum over the (J, Omega) groups of J and their tiles, in order.
__global__ void k_tc_norm_final(const double* __restrict__ npart, const int* __restrict__ g_begin,
                                int ntiles, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const int iJ = blockIdx.x;
  double s = 0;
  for (int g = g_begin[iJ]; g < g_begin[iJ + 1]; ++g)
    for (int t = 0; t < ntiles; ++t) s += npart[(long)g * ntiles + t];
  out[iJ] = s;
}

size_t angular_tc_smem(int kp) {
  return (size_t)2 * TC_M * kp * 4 + (size_t)2 * kp * kp * 4 + 16 + 8 * sizeof(double) + 64;
}

template <int KP, int NE>
static cudaError_t launch_tc_inst(const TcArgs& args, dim3 grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_angular_tc<KP, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  k_angular_tc<KP, NE><<<grid, TC_THREADS, angular_tc_smem(KP), st>>>(args);
  return cudaGetLastError();
}

template <int KP, int NE>
static cudaError_t launch_tc2_inst(const TcArgs& args, cudaStream_t st) {
  if constexpr (NE == 2 && (2 + 2 + 1) * KP > 512) {
    return cudaErrorInvalidValue;   // tensor-memory columns: 5 kp for two states
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_angular_tc2<KP, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           227 * 1024);
      attr = true;
    }
    const long total = (long)args.ngroups * args.ntiles;
    const unsigned grid = (unsigned)std::min<long>(total, args.nsm);
    k_angular_tc2<KP, NE><<<grid, TC_THREADS, tc2_smem<KP>(), st>>>(args);
    return cudaGetLastError();
  }
}

template <int NE>
static cudaError_t launch_tc2_ne(const TcArgs& a, cudaStream_t st) {
  switch (a.kp) {
    case 16: return launch_tc2_inst<16, NE>(a, st);
    case 32: return launch_tc2_inst<32, NE>(a, st);
    case 48: return launch_tc2_inst<48, NE>(a, st);
    case 64: return launch_tc2_inst<64, NE>(a, st);
    case 80: return launch_tc2_inst<80, NE>(a, st);
    case 96: return launch_tc2_inst<96, NE>(a, st);
    case 112: return launch_tc2_inst<112, NE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

bool angular_tc2_supported(int kp, int nelec) {
  return kp % 16 == 0 && kp <= kTcMaxKp && (nelec == 1 || 5 * kp <= 512);
}

template <int NE>
static cudaError_t launch_tc_ne(const TcArgs& a, dim3 grid, cudaStream_t st) {
  switch (a.kp) {
    case 16: return launch_tc_inst<16, NE>(a, grid, st);
    case 32: return launch_tc_inst<32, NE>(a, grid, st);
    case 48: return launch_tc_inst<48, NE>(a, grid, st);
    case 64: return launch_tc_inst<64, NE>(a, grid, st);
    case 80: return launch_tc_inst<80, NE>(a, grid, st);
    case 96: return launch_tc_inst<96, NE>(a, grid, st);
    case 112: return launch_tc_inst<112, NE>(a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_angular_tc(const TcArgs& args, int ngroups, const int* g_begin, int nJ,
                              double* norm_out, cudaStream_t st) {
  cudaError_t e;
  if (args.persistent) {
    e = (args.nelec == 1) ? launch_tc2_ne<1>(args, st) : launch_tc2_ne<2>(args, st);
  } else {
    if (args.ntiles > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)ngroups, (unsigned)args.ntiles);
    e = (args.nelec == 1) ? launch_tc_ne<1>(args, grid, st) : launch_tc_ne<2>(args, grid, st);
  }
  if (e != cudaSuccess) return e;
  if (norm_out && args.npart) {
    k_tc_norm_final<<<nJ, 32, 0, st>>>(args.npart, g_begin, args.ntiles, norm_out);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace mw3
