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
#include <type_traits>

#include "mw3_internal.h"

namespace mw3 {

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 512;
static_assert(TC_THREADS / 32 <= 16, "warp sums reduced by one warp in 4 shuffle levels");
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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long limit = kWaitLimit) {
  for (long it = 0; it < limit; ++it) {
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

// After a bounded wait expired, the MMAs committed to that barrier phase may still be
// running and writing tensor memory. Before a CTA releases its tensor memory it waits for
// that same phase once more, again bounded: the columns are freed only after the MMAs that
// write them have completed (or after a second expiry, when the tensor core is taken to
// have stopped answering).
__device__ __forceinline__ void drain_expired(bool ok, uint32_t mbar, uint32_t expired_parity) {
  if (!ok) (void)mbar_wait(mbar, expired_parity);
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

// Loads without their wait: several tensor-memory loads share one tcgen05.wait::ld, which
// takes the destination registers as operands so that no use moves above it.
__device__ __forceinline__ void tmem_ld4_issue(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld2_issue(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait8(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
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

// issue_split_gemm_ta for a compile-time K (= KP): the loop unrolls and the B descriptors are
// formed once; a K-step of 8 values advances the start-address field (16-byte units) by 16.
template <int KP>
__device__ __forceinline__ void issue_split_gemm_tk(uint32_t dtmem, uint32_t ahi, uint32_t alo,
                                                    const unsigned char* Bhi,
                                                    const unsigned char* Blo, uint32_t idesc) {
  constexpr uint32_t sbo = (uint32_t)KP * 32, lbo = 128;
  const uint64_t dh = smem_desc(smem_u32(Bhi), lbo, sbo), dl = smem_desc(smem_u32(Blo), lbo, sbo);
#pragma unroll
  for (int ks = 0; ks < KP / 8; ++ks) {
    const uint64_t o = (uint64_t)ks * 16;
    mma_tf32_ta(dtmem, ahi + ks * 8, dh + o, idesc, ks > 0);
    mma_tf32_ta(dtmem, ahi + ks * 8, dl + o, idesc, 1);
    mma_tf32_ta(dtmem, alo + ks * 8, dh + o, idesc, 1);
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
  float ssf = 0.0f;   // a thread's sum of squares (FP32: FP64 arithmetic is slow here)
  if (ok) {
    const DevJ J = a.dj[B0.iJ];
    const float invdE = (float)J.invdE, e0s = (float)J.e0s;   // once, not per row
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
          const float hs = h * invdE - e0s * cv[s];
          if (a.mode == 1) {
            a.out[idx] = hs;
          } else {
            const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
            a.ckm1[idx] = nv;
            ssf = fmaf(nv, nv, ssf);
          }
        }
      }
    }
  }
  // norm partial of this CTA (fixed-order reduction)
  double ss = (double)ssf;
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
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
    float ssf = 0.0f;   // a thread's sum of squares (FP32: FP64 arithmetic is slow here)
    if (ok) {
      const DevJ J = a.dj[B0.iJ];
      const float invdE = (float)J.invdE, e0s = (float)J.e0s;   // once, not per row
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
            const float hs = h * invdE - e0s * cv[s];
            if (a.mode == 1) {
              a.out[idx] = hs;
            } else {
              const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
              a.ckm1[idx] = nv;
              ssf = fmaf(nv, nv, ssf);
            }
          }
        }
      }
    }
    // norm partial of this tile (the same fixed-order reduction as the one-tile form)
    double ss = (double)ssf;
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
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}


// ============================================================ parity-split persistent form
// The Gauss-Legendre nodes are symmetric (x_(n') = -x_n, n' = n_gamma - 1 - n) and
// P-bar_j^Omega(-x) = (-1)^(j + Omega) P-bar_j^Omega(x), so T^Omega[i][n'] = (-1)^i T^Omega[i][n]
// (i = j - Omega). With h = n_gamma / 2 (n_gamma even) and n < h:
//   GEMM 1  u[n] = E[n] + O[n],  u[n'] = E[n] - O[n],
//           E[n] = sum_(i even) c_i T[i][n],  O[n] = sum_(i odd) c_i T[i][n]
//   GEMM 2  w_i = sum_(n < h) T[i][n] (y[n] + (-1)^i y[n']),  y = V u
// Four kh x kh operand matrices (kh = h rounded up to 16) replace two kp x kp ones: half
// the tensor work and half the shared memory, which then holds the c, t and c_(k-1) tiles
// copied in asynchronously (c of the next tile while this tile computes).
// Tensor-memory columns (units of kh): A even hi/lo [0, 2), A odd hi/lo [2, 4); per state
// E_L, O_L at 4 + 2L, 5 + 2L; w (even, odd) of state 0 at 4 + 2 NE when NE = 2 (else in
// E_0, O_0); w of state 1 in E_0, O_0; with one state the c tile itself (even, odd rows)
// at 6, 7 for the epilogue.
template <int KH>
constexpr size_t tc3_bbytes() { return (size_t)KH * KH * 4; }
template <int KH>
constexpr size_t tc3_tile() { return (size_t)2 * KH * TC_M * 4; }   // rows [0, 2 kh) x 128
template <int KH>
constexpr size_t tc3_smem() { return 8 * tc3_bbytes<KH>() + 3 * tc3_tile<KH>() + 16 + 16 * sizeof(double) + 64; }

template <int KH, int NE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_angular_tc3(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int kh = KH;
  constexpr size_t bb = tc3_bbytes<KH>();
  unsigned char* G = sm;                                   // 8 matrices: G1e, G1o, G2e, G2o (hi, lo)
  float* cs = reinterpret_cast<float*>(sm + 8 * bb);      // [2 kh][TC_M] c tile (state 0)
  float* ts = cs + 2 * kh * TC_M;                          // t tile (state 0)
  float* ps = ts + 2 * kh * TC_M;                          // c_(k-1) tile (state 0)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ps + 2 * kh * TC_M);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  double* red = reinterpret_cast<double*>(mbar + 2);
  auto Gm = [&](int k, int lo) { return G + (size_t)(2 * k + lo) * bb; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;
  const int half = warp >> 2;
  const int m = q * 32 + lane;
  constexpr int nq = kh / 4;         // parity rows / half-nodes per thread
  constexpr int ncb = kh / 2;        // rows per thread in the epilogue (2 kh / 4)
  const uint32_t mb = smem_u32(mbar);
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t idesc = idesc_tf32(TC_M, kh);
  const int ng = a.ng, h = ng / 2;

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
  auto col_of = [&](int unit) { return tmem + (uint32_t)(unit * kh); };
  const uint32_t tAe_hi = col_of(0), tAe_lo = col_of(1), tAo_hi = col_of(2), tAo_lo = col_of(3);
  auto tE = [&](int L) { return col_of(4 + 2 * L); };
  auto tO = [&](int L) { return col_of(5 + 2 * L); };
  auto tWe = [&](int L) { return (NE == 2 && L == 0) ? col_of(4 + 2 * NE) : col_of(4); };
  auto tWo = [&](int L) { return (NE == 2 && L == 0) ? col_of(5 + 2 * NE) : col_of(5); };
  // one state: the raw c tile (even rows, odd rows) stays in tensor memory for the epilogue
  const uint32_t tCe = col_of(6), tCo = col_of(7);

  const long total = (long)a.ngroups * a.ntiles;
  const long f0 = (long)blockIdx.x * total / gridDim.x;
  const long f1 = (long)(blockIdx.x + 1) * total / gridDim.x;
  // 16-byte asynchronous copy of rows [0, nrow) x [col0, col0 + 128) of plane src into dst
  auto stage = [&](float* dst, const float* src, int nrow, long col0) {
    const int nch = nrow * (TC_M / 4);
    for (int e = tid; e < nch; e += TC_THREADS) {
      const int i = e / (TC_M / 4);
      const int c4 = (e - i * (TC_M / 4)) * 4;
      if (col0 + c4 < a.ncol) cp_async16(dst + i * TC_M + c4, src + (long)i * a.ncol + col0 + c4);
    }
  };
  auto tile_of = [&](long f, int& g, int& tile) {
    g = (int)(f / a.ntiles);
    tile = (int)(f - (long)g * a.ntiles);
  };
  if (f0 < f1) {
    int g, tile;
    tile_of(f0, g, tile);
    stage(cs, a.ck + (long)(g * NE) * a.npts, a.blocks[g * NE].nrow, (long)tile * TC_M);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");

  uint32_t phase = 0;
  bool ok = true;
  int om_cur = -1;
  for (long f = f0; f < f1 && ok; ++f) {
    int g, tile;
    tile_of(f, g, tile);
    const int b0 = g * NE;
    const DevBlock B0 = a.blocks[b0];
    const int om = B0.omega;
    const int nrow = B0.nrow;
    const long col0 = (long)tile * TC_M;
    const long col = col0 + m;
    const bool live = col < a.ncol;
    const int kr = live ? (int)(col / a.NR) : 0;
    const int mR = live ? (int)(col - (long)kr * a.NR) : 0;

    __syncthreads();   // the previous tile's readers of ts / ps / tensor memory are done
    if (om != om_cur) {
      for (int k = 0; k < 4; ++k)
        load_b(a.Tp_hi + ((long)om * 4 + k) * kh * kh, a.Tp_lo + ((long)om * 4 + k) * kh * kh,
               Gm(k, 0), Gm(k, 1), kh);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      om_cur = om;
    }
    stage(ts, a.t + (long)b0 * a.npts, nrow, col0);
    if (a.mode == 0) stage(ps, a.ckm1 + (long)b0 * a.npts, nrow, col0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // c of this tile has landed
    __syncthreads();

    // ------------------------------------------------------------ GEMM 1 per state
    float v1a[nq], v1b[nq];   // one state: V(n), V(n') prefetched during GEMM 1
    for (int L = 0; L < NE && ok; ++L) {
      const float* c = a.ck + (long)(b0 + L) * a.npts;
#pragma unroll
      for (int s0 = 0; s0 < nq; s0 += 4) {
        float he[4], le[4], ho[4], lo[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int e = half * nq + s0 + s;
          const int ie = 2 * e, io = 2 * e + 1;
          float xe = 0.0f, xo = 0.0f;
          if (live) {
            if (L == 0) {
              xe = ie < nrow ? cs[ie * TC_M + m] : 0.0f;
              xo = io < nrow ? cs[io * TC_M + m] : 0.0f;
            } else {
              xe = ie < nrow ? __ldg(c + (long)ie * a.ncol + col) : 0.0f;
              xo = io < nrow ? __ldg(c + (long)io * a.ncol + col) : 0.0f;
            }
          }
          he[s] = tf32_hi(xe);
          le[s] = xe - he[s];
          ho[s] = tf32_hi(xo);
          lo[s] = xo - ho[s];
        }
        const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
        tmem_st4(tAe_hi + cc, he);
        tmem_st4(tAe_lo + cc, le);
        tmem_st4(tAo_hi + cc, ho);
        tmem_st4(tAo_lo + cc, lo);
        if (NE == 1) {
          float re[4], ro[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            re[s] = he[s] + le[s];   // exact: hi + lo reproduces the FP32 value
            ro[s] = ho[s] + lo[s];
          }
          tmem_st4(tCe + cc, re);
          tmem_st4(tCo + cc, ro);
        }
      }
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (L == 0) {
        // the c tile is in tensor memory now: bring in the next tile's (its own group)
        if (f + 1 < f1) {
          int g2, t2;
          tile_of(f + 1, g2, t2);
          stage(cs, a.ck + (long)(g2 * NE) * a.npts, a.blocks[g2 * NE].nrow, (long)t2 * TC_M);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue_split_gemm_ta(tE(L), tAe_hi, tAe_lo, Gm(0, 0), Gm(0, 1), kh, idesc);
        issue_split_gemm_ta(tO(L), tAo_hi, tAo_lo, Gm(1, 0), Gm(1, 1), kh, idesc);
        mma_commit(mb);
      }
      if (NE == 1) {
        // the potential at this thread's node pairs, loaded while the MMAs run
#pragma unroll
        for (int s2 = 0; s2 < nq; ++s2) {
          const int n = half * nq + s2;
          const bool in = live && n < h;
          v1a[s2] = in ? __ldg(a.V + (long)n * a.ncol + col) : 0.0f;
          v1b[s2] = in ? __ldg(a.V + (long)(ng - 1 - n) * a.ncol + col) : 0.0f;
        }
      }
      ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }

    // ------------------------------------------------------------ potential + GEMM 2
    for (int L = 0; L < NE && ok; ++L) {
      // V at the node pairs (n, n') of this thread's quarter, loads first
      float va[NE][nq], vb[NE][nq];
#pragma unroll
      for (int Lp = 0; Lp < NE; ++Lp) {
        const float* V = a.V + (long)(L * NE + Lp) * a.npts;
#pragma unroll
        for (int s2 = 0; s2 < nq; ++s2) {
          const int n = half * nq + s2;
          const bool in = live && n < h;
          if (NE == 1) {
            va[Lp][s2] = v1a[s2];
            vb[Lp][s2] = v1b[s2];
          } else {
            va[Lp][s2] = in ? __ldg(V + (long)n * a.ncol + col) : 0.0f;
            vb[Lp][s2] = in ? __ldg(V + (long)(ng - 1 - n) * a.ncol + col) : 0.0f;
          }
        }
      }
#pragma unroll
      for (int s0 = 0; s0 < nq; s0 += 4) {
        float ya[4] = {0, 0, 0, 0}, yb[4] = {0, 0, 0, 0};
#pragma unroll
        for (int Lp = 0; Lp < NE; ++Lp) {
          uint32_t r[8];   // E (4), O (4)
          tmem_ld4_issue(tE(Lp) + lane_base + (uint32_t)(half * nq + s0), r);
          tmem_ld4_issue(tO(Lp) + lane_base + (uint32_t)(half * nq + s0), r + 4);
          tmem_wait8(r);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const float E = __uint_as_float(r[s]), O = __uint_as_float(r[4 + s]);
            ya[s] += va[Lp][s0 + s] * (E + O);   // y[n]
            yb[s] += vb[Lp][s0 + s] * (E - O);   // y[n']
          }
        }
        float hs[4], ls[4], hd[4], ld[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const float S = ya[s] + yb[s], Dd = ya[s] - yb[s];
          hs[s] = tf32_hi(S);
          ls[s] = S - hs[s];
          hd[s] = tf32_hi(Dd);
          ld[s] = Dd - hd[s];
        }
        const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
        tmem_st4(tAe_hi + cc, hs);
        tmem_st4(tAe_lo + cc, ls);
        tmem_st4(tAo_hi + cc, hd);
        tmem_st4(tAo_lo + cc, ld);
      }
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue_split_gemm_ta(tWe(L), tAe_hi, tAe_lo, Gm(2, 0), Gm(2, 1), kh, idesc);
        issue_split_gemm_ta(tWo(L), tAo_hi, tAo_lo, Gm(3, 0), Gm(3, 1), kh, idesc);
        mma_commit(mb);
      }
      ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // t and c_(k-1) of this tile
    __syncthreads();

    // ------------------------------------------------------------ epilogue
    float ssf = 0.0f;   // a thread's sum of squares (FP32: FP64 arithmetic is slow here)
    if (ok) {
      const DevJ J = a.dj[B0.iJ];
      const float invdE = (float)J.invdE, e0s = (float)J.e0s;   // once, not per row
      const float* cf = a.coef + (long)B0.coef * kCoefRows * a.ng;
      const float D = live ? a.DR[mR] * a.Dr[kr] : 0.0f;
      const float frk = live ? a.fr[kr] : 0.0f;
      const float fRm = live ? a.fR[mR] : 0.0f;
      for (int L = 0; L < NE; ++L) {
        const int b = b0 + L;
        const DevBlock Bb = a.blocks[b];
        const float* c = a.ck + (long)b * a.npts;
        for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 4) {
          // global and shared loads first, then the tensor-memory loads under one wait
          float cv[4], cu[4], cd[4], tv[4], pv[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int i = i0 + s;
            const bool in = live && i < nrow;
            const long off = (long)i * a.ncol + col;
            cv[s] = (in && NE != 1) ? __ldg(c + off) : 0.0f;
            tv[s] = in ? (L == 0 ? ts[i * TC_M + m] : __ldg(a.t + (long)b * a.npts + off)) : 0.0f;
            pv[s] = (in && a.mode == 0) ? (L == 0 ? ps[i * TC_M + m] : __ldg(a.ckm1 + (long)b * a.npts + off)) : 0.0f;
            cu[s] = (in && Bb.up >= 0 && i >= 1) ? __ldg(a.ck + (long)Bb.up * a.npts + off - a.ncol) : 0.0f;
            cd[s] = (in && Bb.dn >= 0) ? __ldg(a.ck + (long)Bb.dn * a.npts + off + a.ncol) : 0.0f;
          }
          uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // w even, w odd, c even, c odd
          tmem_ld2_issue(tWe(L) + lane_base + (uint32_t)(i0 / 2), r);
          tmem_ld2_issue(tWo(L) + lane_base + (uint32_t)(i0 / 2), r + 2);
          if (NE == 1) {
            tmem_ld2_issue(tCe + lane_base + (uint32_t)(i0 / 2), r + 4);
            tmem_ld2_issue(tCo + lane_base + (uint32_t)(i0 / 2), r + 6);
          }
          tmem_wait8(r);
          if (!live) continue;
          const float w[4] = {__uint_as_float(r[0]), __uint_as_float(r[2]), __uint_as_float(r[1]),
                              __uint_as_float(r[3])};
          if (NE == 1) {
            cv[0] = __uint_as_float(r[4]);
            cv[1] = __uint_as_float(r[6]);
            cv[2] = __uint_as_float(r[5]);
            cv[3] = __uint_as_float(r[7]);
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
            float hh = w[s] + aa * cv[s] + tv[s];
            hh += gg * cf[2 * a.ng + i] * cu[s];
            hh += gg * cf[3 * a.ng + i] * cd[s];
            const float hs = hh * invdE - e0s * cv[s];
            if (a.mode == 1) {
              a.out[idx] = hs;
            } else {
              const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
              a.ckm1[idx] = nv;
              ssf = fmaf(nv, nv, ssf);
            }
          }
        }
      }
    }
    double ss = (double)ssf;
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
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && tid == 0) atomicExch(a.err, 1);
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}


// ============================================================ streamed parity-split form
// For n_gamma from 98 to 192 (kh = 64..96) the four half matrices do not fit in shared
// memory together: they stream through two buffers in the order G1e, G1o, G2e, G2o, each
// copied with cp.async while the MMAs of the previous one run, and the even and odd
// operand halves pass through tensor memory one after the other. One electronic state.
// Tensor-memory columns (units of kh): A hi/lo [0, 2), E 2, O 3, w_even 4; the potential
// step leaves S in A and D in O's columns; w_odd goes to E's columns.
template <int KH>
constexpr size_t tc4_smem() { return 4 * (size_t)KH * KH * 4 + 16 + 16 * sizeof(double) + 64; }

// 16-byte asynchronous copy of a kh x kh (hi, lo) pair, row-major, into core-matrix layout
__device__ __forceinline__ void load_b_async(const float* __restrict__ hi,
                                             const float* __restrict__ lo, unsigned char* Bhi,
                                             unsigned char* Blo, int kh) {
  const int nq = kh * kh / 4;
  for (int e = threadIdx.x; e < nq; e += blockDim.x) {
    const int row = e / (kh / 4);
    const int k4 = (e - row * (kh / 4)) * 4;
    const uint32_t off = cm_off(row, k4, kh);
    cp_async16(Bhi + off, hi + (long)row * kh + k4);
    cp_async16(Blo + off, lo + (long)row * kh + k4);
  }
}

template <int KH>
__global__ void __launch_bounds__(TC_THREADS, 1) k_angular_tc4(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int kh = KH;
  constexpr size_t bb = (size_t)KH * KH * 4;
  auto Bbuf = [&](int buf, int lo) { return sm + (size_t)(2 * buf + lo) * bb; };
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 4 * bb);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  double* red = reinterpret_cast<double*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;
  const int half = warp >> 2;
  const int m = q * 32 + lane;
  constexpr int nq = kh / 4;
  constexpr int ncb = kh / 2;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t idesc = idesc_tf32(TC_M, kh);
  const int ng = a.ng, h = ng / 2;

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
  const uint32_t tA_hi = tmem, tA_lo = tmem + kh, tE = tmem + 2 * kh, tO = tmem + 3 * kh,
                 tWe = tmem + 4 * kh, tWo = tE;

  const long total = (long)a.ngroups * a.ntiles;
  const long f0 = (long)blockIdx.x * total / gridDim.x;
  const long f1 = (long)(blockIdx.x + 1) * total / gridDim.x;
  auto omega_of = [&](long f) { return a.blocks[(int)(f / a.ntiles)].omega; };
  auto issue_b = [&](long f, int k) {   // matrix k (G1e, G1o, G2e, G2o) of tile f -> buffer k & 1
    if (f < f1) {
      const long base = ((long)omega_of(f) * 4 + k) * kh * kh;
      load_b_async(a.Tp_hi + base, a.Tp_lo + base, Bbuf(k & 1, 0), Bbuf(k & 1, 1), kh);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // MMA of matrix k of the current tile: its copy landed in every thread, visible to the
  // tensor core, and every operand store to tensor memory is complete
  uint32_t phase = 0;
  bool ok = true;
  auto run_mma = [&](uint32_t dtmem, int k) {
    tmem_st_wait();
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_split_gemm_ta(dtmem, tA_hi, tA_lo, Bbuf(k & 1, 0), Bbuf(k & 1, 1), kh, idesc);
      mma_commit(mb);
    }
    ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
  };
  issue_b(f0, 0);
  issue_b(f0, 1);

  for (long f = f0; f < f1 && ok; ++f) {
    const int g = (int)(f / a.ntiles);
    const int tile = (int)(f - (long)g * a.ntiles);
    const DevBlock B0 = a.blocks[g];
    const int nrow = B0.nrow;
    const long col = (long)tile * TC_M + m;
    const bool live = col < a.ncol;
    const int kr = live ? (int)(col / a.NR) : 0;
    const int mR = live ? (int)(col - (long)kr * a.NR) : 0;
    const float* c = a.ck + (long)g * a.npts;

    // ---- GEMM 1: E = c_even G1e, O = c_odd G1o (the operand halves in turn)
    for (int par = 0; par < 2 && ok; ++par) {
#pragma unroll 2
      for (int s0 = 0; s0 < nq; s0 += 4) {
        float hh[4], ll[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int i = 2 * (half * nq + s0 + s) + par;
          const float x = (live && i < nrow) ? __ldg(c + (long)i * a.ncol + col) : 0.0f;
          hh[s] = tf32_hi(x);
          ll[s] = x - hh[s];
        }
        const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
        tmem_st4(tA_hi + cc, hh);
        tmem_st4(tA_lo + cc, ll);
      }
      run_mma(par == 0 ? tE : tO, par);
      issue_b(f, 2 + par);                       // the buffer just used takes G2e / G2o
    }
    if (!ok) break;

    // ---- potential: y = V u at the node pairs; S = y(n) + y(n') into A, D = y(n) - y(n')
    // into O's columns
#pragma unroll 2
    for (int s0 = 0; s0 < nq; s0 += 4) {
      float va[4], vb[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int n = half * nq + s0 + s;
        const bool in = live && n < h;
        va[s] = in ? __ldg(a.V + (long)n * a.ncol + col) : 0.0f;
        vb[s] = in ? __ldg(a.V + (long)(ng - 1 - n) * a.ncol + col) : 0.0f;
      }
      uint32_t r[8];
      tmem_ld4_issue(tE + lane_base + (uint32_t)(half * nq + s0), r);
      tmem_ld4_issue(tO + lane_base + (uint32_t)(half * nq + s0), r + 4);
      tmem_wait8(r);
      float hs[4], ls[4], dd[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float E = __uint_as_float(r[s]), O = __uint_as_float(r[4 + s]);
        const float ya = va[s] * (E + O), yb = vb[s] * (E - O);
        const float S = ya + yb;
        dd[s] = ya - yb;
        hs[s] = tf32_hi(S);
        ls[s] = S - hs[s];
      }
      const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
      tmem_st4(tA_hi + cc, hs);
      tmem_st4(tA_lo + cc, ls);
      tmem_st4(tO + cc, dd);
    }
    run_mma(tWe, 2);
    issue_b(f + 1, 0);                           // next tile's G1e
    if (!ok) break;
#pragma unroll 2
    for (int s0 = 0; s0 < nq; s0 += 4) {
      uint32_t r[4];
      tmem_ld4_issue(tO + lane_base + (uint32_t)(half * nq + s0), r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
      float hd[4], ld[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float Dd = __uint_as_float(r[s]);
        hd[s] = tf32_hi(Dd);
        ld[s] = Dd - hd[s];
      }
      const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
      tmem_st4(tA_hi + cc, hd);
      tmem_st4(tA_lo + cc, ld);
    }
    run_mma(tWo, 3);
    issue_b(f + 1, 1);                           // next tile's G1o
    if (!ok) break;

    // ---- epilogue
    float ssf = 0.0f;   // a thread's sum of squares (FP32: FP64 arithmetic is slow here)
    {
      const DevJ J = a.dj[B0.iJ];
      const float invdE = (float)J.invdE, e0s = (float)J.e0s;   // once, not per row
      const float* cf = a.coef + (long)B0.coef * kCoefRows * a.ng;
      const float D = live ? a.DR[mR] * a.Dr[kr] : 0.0f;
      const float frk = live ? a.fr[kr] : 0.0f;
      const float fRm = live ? a.fR[mR] : 0.0f;
      const int b = g;
      for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 4) {
        float cv[4], cu[4], cd[4], tv[4], pv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int i = i0 + s;
          const bool in = live && i < nrow;
          const long off = (long)i * a.ncol + col;
          cv[s] = in ? __ldg(c + off) : 0.0f;
          tv[s] = in ? __ldg(a.t + (long)b * a.npts + off) : 0.0f;
          pv[s] = (in && a.mode == 0) ? __ldg(a.ckm1 + (long)b * a.npts + off) : 0.0f;
          cu[s] = (in && B0.up >= 0 && i >= 1) ? __ldg(a.ck + (long)B0.up * a.npts + off - a.ncol) : 0.0f;
          cd[s] = (in && B0.dn >= 0) ? __ldg(a.ck + (long)B0.dn * a.npts + off + a.ncol) : 0.0f;
        }
        uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        tmem_ld2_issue(tWe + lane_base + (uint32_t)(i0 / 2), r);
        tmem_ld2_issue(tWo + lane_base + (uint32_t)(i0 / 2), r + 2);
        tmem_wait8(r);
        if (!live) continue;
        const float w[4] = {__uint_as_float(r[0]), __uint_as_float(r[2]), __uint_as_float(r[1]),
                            __uint_as_float(r[3])};
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
          float hh = w[s] + aa * cv[s] + tv[s];
          hh += gg * cf[2 * a.ng + i] * cu[s];
          hh += gg * cf[3 * a.ng + i] * cd[s];
          const float hs = hh * invdE - e0s * cv[s];
          if (a.mode == 1) {
            a.out[idx] = hs;
          } else {
            const float nv = D * (a.alpha * hs - a.beta * D * pv[s]);
            a.ckm1[idx] = nv;
            ssf = fmaf(nv, nv, ssf);
          }
        }
      }
    }
    double ss = (double)ssf;
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
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && tid == 0) atomicExch(a.err, 1);
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}


// ================================================================ tile-major form
// One electronic state, kh <= 48. Each CTA walks a contiguous range of (tile, block) units
// in tile-major order, so consecutive units are the helicities Omega, Omega + 1, ... of one
// (r, R) tile. The Coriolis neighbours then come from on-chip copies: c^(Omega-1) is the
// raw c tile the previous unit left in tensor memory, c^(Omega+1) is the next unit's c tile,
// already copied into shared memory for its GEMM 1. The potential of the tile stays in
// registers across its units. The four half matrices change with Omega and stream through
// two shared-memory buffers (G1e, G1o, G2e, G2o), each copy overlapping earlier MMAs.
// Tensor-memory columns (units of kh): A even hi/lo 0, 1, A odd hi/lo 2, 3, E 4, O 5 (w even,
// w odd after GEMM 2), raw c tiles (even rows, odd rows) in two slots at 6, 7 and 8, 9.
template <int KH>
constexpr size_t tc5_smem() {
  return 4 * (size_t)KH * KH * 4 + 3 * (size_t)2 * KH * TC_M * 4 + 16 + 16 * sizeof(double) +
         (size_t)2 * KH * 8 * 4 + 64;
}

template <int KH, bool TMA>
__global__ void __launch_bounds__(TC_THREADS, 1) k_angular_tc5(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int kh = KH;
  constexpr size_t bb = (size_t)KH * KH * 4;
  auto Bbuf = [&](int buf, int lo) { return sm + (size_t)(2 * buf + lo) * bb; };
  float* cs = reinterpret_cast<float*>(sm + 4 * bb);   // [2 kh][TC_M] c of the next unit
  float* ts = cs + 2 * kh * TC_M;                       // t of this unit
  float* ps = ts + 2 * kh * TC_M;                       // c_(k-1) of this unit
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ps + 2 * kh * TC_M);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  double* red = reinterpret_cast<double*>(mbar + 2);
  float* cfs = reinterpret_cast<float*>(red + 16);           // [2 kh][8] coefficients
  float* redf = reinterpret_cast<float*>(red);                // per-warp sums of squares
  // TMA form: one barrier per tile buffer (0 cs, 1 ts, 2 ps), each completing once per copy
  uint64_t* tbar = reinterpret_cast<uint64_t*>(cfs + 2 * kh * 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3;
  const int half = warp >> 2;
  const int m = q * 32 + lane;
  constexpr int nq = kh / 4;
  constexpr int ncb = kh / 2;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t idesc = idesc_tf32(TC_M, kh);
  const int ng = a.ng, h = ng / 2;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(mb));
    if constexpr (TMA) {
      for (int w = 0; w < 3; ++w)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(tbar + w)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  auto col_of = [&](int unit) { return tmem + (uint32_t)(unit * kh); };
  const uint32_t tAe_hi = col_of(0), tAe_lo = col_of(1), tAo_hi = col_of(2), tAo_lo = col_of(3);
  const uint32_t tE = col_of(4), tO = col_of(5);

  const int ngr = a.ngroups;
  const long total = (long)ngr * a.ntiles;
  const long u0 = (long)blockIdx.x * total / gridDim.x;
  const long u1 = (long)(blockIdx.x + 1) * total / gridDim.x;
  auto unit_tile = [&](long u) { return (int)(u / ngr); };
  auto unit_block = [&](long u) { return (int)(u - (long)(u / ngr) * ngr); };
  // tile copies: rows [0, nrow) of block b's plane, columns [col0, col0 + 128). TMA form:
  // thread 64 issues ceil(nrow / 8) boxes of 8 x 128 into dst and arms the buffer's barrier
  // with their bytes (columns past the grid arrive as zeros; rows past nrow are not read)
  bool ok = true;                          // no bounded wait has expired
  bool tpend[3] = {false, false, false};   // a copy into buffer w is in flight
  uint32_t tph[3] = {0u, 0u, 0u};
  auto stage = [&](int which, float* dst, const float* src, int b, int nrow, long col0) {
    if constexpr (TMA) {
      const CUtensorMap* map = which == 0 ? &a.tm_ck : (which == 1 ? &a.tm_t : &a.tm_ckm1);
      const int nbox = (nrow + 7) / 8;
      if (tid == 64) {   // a thread of its own: threads 0 and 32 issue the MMAs
        const uint32_t bar = smem_u32(tbar + which);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)(nbox * 8 * TC_M * 4))
                     : "memory");
        for (int x = 0; x < nbox; ++x) {
          const int row = b * a.ng + 8 * x;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst + 8 * x * TC_M)),
              "l"(reinterpret_cast<uint64_t>(map)), "r"((int)col0), "r"(row), "r"(bar)
              : "memory");
        }
      }
      tpend[which] = true;
    } else {
      (void)which;
      (void)b;
      // 16-byte chunk (i, c4) of the tile goes to thread i * (TC_M / 4) + c4 / 4 modulo
      // TC_THREADS: a thread keeps its column c4 and walks rows i, i + TC_THREADS / 32, ...
      static_assert(TC_M / 4 == 32 && TC_THREADS % 32 == 0, "one warp per tile row");
      constexpr int kRowStep = TC_THREADS / 32;
      const int c4 = lane * 4;
      if (col0 + c4 < a.ncol) {
        const long gstep = (long)kRowStep * a.ncol;
        const float* s = src + (long)warp * a.ncol + col0 + c4;
        float* d = dst + warp * TC_M + c4;
        for (int i = warp; i < nrow; i += kRowStep, s += gstep, d += kRowStep * TC_M)
          cp_async16(d, s);
      }
    }
  };
  // TMA form: every thread waits (bounded) for the copies of the buffers in `mask` that are in
  // flight; the completed barrier phase makes the copied bytes visible to each waiting thread,
  // so no CTA barrier is needed here. The result is folded into the next CTA-wide vote, which
  // keeps ok uniform.
  auto wait_tiles_local = [&](int mask) -> bool {
    bool good = true;
    if constexpr (TMA) {
      for (int w = 0; w < 3; ++w)
        if ((mask >> w & 1) && tpend[w]) {
          if (mbar_wait(smem_u32(tbar + w), tph[w], a.wait_limit)) {
            tph[w] ^= 1u;
            tpend[w] = false;
          } else {
            good = false;   // still pending: the exit path waits for this copy once more
          }
        }
    }
    return good;
  };
  // matrices k0 (buffer 0) and k0 + 1 (buffer 1) of unit u, as one copy group
  auto issue_b2 = [&](long u, int k0) {
    if (u < u1) {
      const long om = a.blocks[unit_block(u)].omega;
      for (int k = k0; k < k0 + 2; ++k) {
        const long base = (om * 4 + k) * kh * kh;
        load_b_async(a.Tp_hi + base, a.Tp_lo + base, Bbuf(k & 1, 0), Bbuf(k & 1, 1), kh);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  uint32_t phase = 0;
  // both parities' MMAs of one GEMM (even: A even x buffer 0, odd: A odd x buffer 1), issued
  // once the copy groups it needs have landed (all, or all but the newest: visible to the tensor
  // core) and the operand stores to tensor memory are complete; the wait comes later, so that
  // CUDA-core work overlaps the MMAs
  auto issue_mma2 = [&](uint32_t de, uint32_t dodd, bool gemm1) {
    tmem_st_wait();
    // GEMM 1 of unit u: the groups [t(u)] and [c_(k-1)(u)] may still be in flight (the
    // remainder reads them after GEMM 2 is issued). TMA form: the only cp.async groups are
    // half matrices, all of which this GEMM needs.
    if (gemm1 && !TMA) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // two issuing threads in different warps (one parity each); each commit arrives once on
    // the barrier, which completes on the second
    if (tid == 0) {
      issue_split_gemm_tk<KH>(de, tAe_hi, tAe_lo, Bbuf(0, 0), Bbuf(0, 1), idesc);
      mma_commit(mb);
    } else if (tid == 32) {
      issue_split_gemm_tk<KH>(dodd, tAo_hi, tAo_lo, Bbuf(1, 0), Bbuf(1, 1), idesc);
      mma_commit(mb);
    }
  };
  auto wait_mma = [&](bool also = true) {
    ok = __syncthreads_and((mbar_wait(mb, phase, a.wait_limit) && also) ? 1 : 0) != 0;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
  };

  // Copy groups, in commit order: [c(u)] during GEMM 1 of unit u-1, [G1e G1o(u)] and then
  // [t(u)] after GEMM 2 of unit u-1, [c_(k-1)(u)] after the result of unit u-1 is written,
  // [G2e G2o(u)] after GEMM 1 of unit u; the first unit's four come from here. GEMM 1 of unit
  // u waits for [G1e G1o(u)] only, so the t tile's DRAM latency overlaps GEMM 1 and the
  // potential; GEMM 2's wait (all groups) covers everything the remainder reads.
  // (TMA form: the tile copies complete on their own barriers; only the half-matrix groups
  // remain cp.async groups.)
  const int b00 = u0 < u1 ? unit_block(u0) : 0;
  const long c00 = u0 < u1 ? (long)unit_tile(u0) * TC_M : 0;
  if (u0 < u1) stage(0, cs, a.ck + (long)b00 * a.npts, b00, a.blocks[b00].nrow, c00);
  asm volatile("cp.async.commit_group;" ::: "memory");
  issue_b2(u0, 0);
  if (u0 < u1) stage(1, ts, a.t + (long)b00 * a.npts, b00, a.blocks[b00].nrow, c00);
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (u0 < u1 && a.mode == 0)
    stage(2, ps, a.ckm1 + (long)b00 * a.npts, b00, a.blocks[b00].nrow, c00);
  asm volatile("cp.async.commit_group;" ::: "memory");

  float va[nq], vb[nq];
  int vtile = -1;
  int slot = 0;             // tensor-memory slot of this unit's raw c
  long prev_u = -2;         // last unit processed by this CTA
  for (long u = u0; u < u1 && ok; ++u) {
    const int tile = unit_tile(u);
    const int b = unit_block(u);
    const DevBlock B0 = a.blocks[b];
    const int nrow = B0.nrow;
    const long col0 = (long)tile * TC_M;
    const long col = col0 + m;
    const bool live = col < a.ncol;
    const int kr = live ? (int)(col / a.NR) : 0;
    const int mR = live ? (int)(col - (long)kr * a.NR) : 0;
    const uint32_t tC = col_of(6 + 2 * slot), tCp = col_of(6 + 2 * (slot ^ 1));
    // c^(Omega-1) in tensor memory when the previous unit was that block of this tile
    const bool dn_chip = B0.dn >= 0 && prev_u == u - 1 && B0.dn == b - 1 && tile == unit_tile(u - 1);
    // c^(Omega+1) in shared memory when the next unit is that block of this tile
    const bool up_chip = B0.up >= 0 && B0.up == b + 1 && u + 1 < u1 && unit_tile(u + 1) == tile;

    if constexpr (TMA) {
      // this unit's c tile has landed and the previous unit's readers of ts, ps, cs and
      // tensor memory are done: one barrier
      ok = __syncthreads_and(wait_tiles_local(1) ? 1 : 0) != 0;
      if (!ok) break;
    } else if (u == u0) {
      // the first unit's c tile: groups [c], [G1e G1o], [t], [c_(k-1)] are in flight. Later
      // units need no wait here: their c tile was part of the previous unit's GEMM 2 wait,
      // whose CTA barrier made it visible, and the previous unit's closing barrier orders
      // every reader of ts, ps, cs and tensor memory before this unit's writes.
      asm volatile("cp.async.wait_group 3;" ::: "memory");
      __syncthreads();
    }
    // ---- GEMM 1 operands (both parities) and the raw c tile, from shared memory
#pragma unroll
    for (int s0 = 0; s0 < nq; s0 += 4) {
      float he[4], le[4], ho[4], lo[4], re[4], ro[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int e = half * nq + s0 + s;
        const int ie = 2 * e, io = 2 * e + 1;
        const float xe = (live && ie < nrow) ? cs[ie * TC_M + m] : 0.0f;
        const float xo = (live && io < nrow) ? cs[io * TC_M + m] : 0.0f;
        re[s] = xe;
        ro[s] = xo;
        he[s] = tf32_hi(xe);
        le[s] = xe - he[s];
        ho[s] = tf32_hi(xo);
        lo[s] = xo - ho[s];
      }
      const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
      tmem_st4(tAe_hi + cc, he);
      tmem_st4(tAe_lo + cc, le);
      tmem_st4(tAo_hi + cc, ho);
      tmem_st4(tAo_lo + cc, lo);
      tmem_st4(tC + cc, re);
      tmem_st4(tC + kh + cc, ro);
    }
    // ---- GEMM 1: E = c_even G1e, O = c_odd G1o. While it runs: stage the next unit's c tile
    // (this unit's upper neighbour), and on a new tile load the potential
    issue_mma2(tE, tO, true);                     // [G1e G1o](u) landed; [t], [c_(k-1)](u) may not
    if (u + 1 < u1) {
      const int bn = unit_block(u + 1);
      stage(0, cs, a.ck + (long)bn * a.npts, bn, a.blocks[bn].nrow, (long)unit_tile(u + 1) * TC_M);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (tid < ng) {   // the block's five coefficient rows, interleaved per row i
      const float* cf = a.coef + (long)B0.coef * kCoefRows * a.ng;
      *reinterpret_cast<float4*>(cfs + tid * 8) =
          make_float4(cf[tid], cf[ng + tid], cf[2 * ng + tid], cf[3 * ng + tid]);
      cfs[tid * 8 + 4] = cf[4 * ng + tid];
    }
    if (tile != vtile) {
#pragma unroll
      for (int s2 = 0; s2 < nq; ++s2) {
        const int n = half * nq + s2;
        const bool in = live && n < h;
        va[s2] = in ? __ldg(a.V + (long)n * a.ncol + col) : 0.0f;
        vb[s2] = in ? __ldg(a.V + (long)(ng - 1 - n) * a.ncol + col) : 0.0f;
      }
      vtile = tile;
    }
    wait_mma();
    if (!ok) break;
    issue_b2(u, 2);                               // pending: [c_(k-1)(u)], [c(u+1)], [G2e G2o(u)]

    // ---- potential: S = y(n) + y(n') into A even, D = y(n) - y(n') into A odd
#pragma unroll
    for (int s0 = 0; s0 < nq; s0 += 4) {
      uint32_t r[8];
      tmem_ld4_issue(tE + lane_base + (uint32_t)(half * nq + s0), r);
      tmem_ld4_issue(tO + lane_base + (uint32_t)(half * nq + s0), r + 4);
      tmem_wait8(r);
      float hs[4], ls[4], hd[4], ld[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float E = __uint_as_float(r[s]), O = __uint_as_float(r[4 + s]);
        const float ya = va[s0 + s] * (E + O), yb = vb[s0 + s] * (E - O);
        const float S = ya + yb, Dd = ya - yb;
        hs[s] = tf32_hi(S);
        ls[s] = S - hs[s];
        hd[s] = tf32_hi(Dd);
        ld[s] = Dd - hd[s];
      }
      const uint32_t cc = lane_base + (uint32_t)(half * nq + s0);
      tmem_st4(tAe_hi + cc, hs);
      tmem_st4(tAe_lo + cc, ls);
      tmem_st4(tAo_hi + cc, hd);
      tmem_st4(tAo_lo + cc, ld);
    }

    // ---- GEMM 2: w_even = S G2e, w_odd = D G2o. While it runs, every term of the result
    // but w: with r = a c + b+ c^(Omega+1) + b- c^(Omega-1) + t,
    //   H_s c = invdE (w + r) - e0s c,  c_(k+1) = D (alpha H_s c - beta D c_(k-1)),
    // so the result is k1 w + r2 with r2 written over c_(k-1) in shared memory.
    issue_mma2(tE, tO, false);                    // c(u+1), c_(k-1)(u), G2e G2o(u) landed
    // TMA form: the tiles the remainder reads, t(u), c_(k-1)(u) and c(u+1) if on chip; the
    // outcome joins the vote after GEMM 2
    const bool tiles_ok = wait_tiles_local(2 | (a.mode == 0 ? 4 : 0) | (up_chip ? 1 : 0));
    const float invdE = a.dj[B0.iJ].invdE_f, e0s = a.dj[B0.iJ].e0s_f;
    const float D = live ? a.DR[mR] * a.Dr[kr] : 0.0f;
    const float k1 = a.mode == 1 ? invdE : D * a.alpha * invdE;
    {
      const float kc = a.mode == 1 ? 1.0f : D * a.alpha;
      const float kq = a.mode == 1 ? 0.0f : a.beta * D * D;
      const float frk = live ? a.fr[kr] : 0.0f;
      const float fRm = live ? a.fR[mR] : 0.0f;
      const float erot = a.erot;
      const bool has_up = B0.up >= 0, has_dn = B0.dn >= 0, use_pv = a.mode == 0;
      // neighbours that are not on chip come from global memory (rows i + 1 of block
      // Omega - 1 and i - 1 of block Omega + 1 share the (r, R) column of row i)
      const float* dn_g = a.ck + (long)(has_dn ? B0.dn : 0) * a.npts + a.ncol + col;
      const float* up_g = a.ck + (long)(has_up ? B0.up : 0) * a.npts - a.ncol + col;
      // The remainder of rows i0 .. i0 + 7, specialised on which neighbours are on chip
      // (uniform over the unit) and on whether all eight rows are live (every group but the
      // last ones of the high-Omega blocks). With c^(Omega-1) on chip, row i + 1 of the
      // previous unit's tile exists for every live row i (its block has one row more).
      auto remainder = [&](auto dn_tag, auto up_tag) {
        constexpr bool DNC = decltype(dn_tag)::value, UPC = decltype(up_tag)::value;
        for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 8) {
          // c of this unit: even columns i0/2.. = rows i0, i0+2, i0+4, i0+6, odd columns =
          // rows i0+1, ...; with c^(Omega-1) on chip, its rows i0+1.. = odd columns i0/2..
          // (rows i0+1, i0+3, ...) and even columns i0/2+1.. (rows i0+2, i0+4, ...) of the
          // previous unit's raw tile (row i of block Omega-1 is its row i + 1)
          uint32_t r[16];
          tmem_ld4_issue(tC + lane_base + (uint32_t)(i0 / 2), r);
          tmem_ld4_issue(tC + kh + lane_base + (uint32_t)(i0 / 2), r + 4);
          if constexpr (DNC) {
            tmem_ld4_issue(tCp + kh + lane_base + (uint32_t)(i0 / 2), r + 8);
            tmem_ld4_issue(tCp + lane_base + (uint32_t)(i0 / 2 + 1), r + 12);
            tmem_wait16(r);
          } else {
            tmem_wait8(r);
          }
          if (!live) continue;
          const int nv = nrow - i0;   // live rows from i0 on (may be <= 0)
          float* psr = ps + i0 * TC_M + m;
          const float* tsr = ts + i0 * TC_M + m;
          const float* csr = cs + (i0 - 1) * TC_M + m;   // row i - 1 of the next unit's tile
          const float* cfr = cfs + i0 * 8;
          const long goff = (long)i0 * a.ncol;
          auto row = [&](int s) {
            const float cv = __uint_as_float(r[(s & 1) * 4 + (s >> 1)]);
            float cd = 0.0f;
            if constexpr (DNC) cd = __uint_as_float(r[8 + (s & 1) * 4 + (s >> 1)]);
            else if (has_dn) cd = __ldg(dn_g + goff + (long)s * a.ncol);
            // row i of block Omega+1 is its row i - 1 (j = Omega + i); none for i = 0
            float cu = 0.0f;
            if (has_up && (s > 0 || i0 > 0)) {
              if constexpr (UPC) cu = csr[s * TC_M];
              else cu = __ldg(up_g + goff + (long)s * a.ncol);
            }
            const float tv = tsr[s * TC_M];
            const float pv = use_pv ? psr[s * TC_M] : 0.0f;
            const float4 c4 = *reinterpret_cast<const float4*>(cfr + s * 8);
            const float gg = fminf(fRm, cfr[s * 8 + 4]);
            const float aa = fminf(c4.x * frk, erot) + gg * c4.y;
            float rr = aa * cv + tv;
            rr += gg * c4.z * cu;
            rr += gg * c4.w * cd;
            psr[s * TC_M] = kc * (rr * invdE - e0s * cv) - kq * pv;
          };
          if (nv >= 8) {
#pragma unroll
            for (int s2 = 0; s2 < 8; ++s2) row(s2);
          } else {
#pragma unroll
            for (int s2 = 0; s2 < 8; ++s2)
              if (s2 < nv) row(s2);
          }
        }
      };
      if (dn_chip) {
        if (up_chip) remainder(std::true_type{}, std::true_type{});
        else remainder(std::true_type{}, std::false_type{});
      } else {
        if (up_chip) remainder(std::false_type{}, std::true_type{});
        else remainder(std::false_type{}, std::false_type{});
      }
    }
    wait_mma(tiles_ok);
    if (!ok) break;
    // t is free: the next unit's G1e G1o, then its t, one group each
    issue_b2(u + 1, 0);
    if (u + 1 < u1) {
      const int bn = unit_block(u + 1);
      stage(1, ts, a.t + (long)bn * a.npts, bn, a.blocks[bn].nrow, (long)unit_tile(u + 1) * TC_M);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");

    // ---- result = k1 w + r2, eight rows per tensor-memory wait (w even: rows i0, i0 + 2, ...;
    // w odd: rows i0 + 1, i0 + 3, ...); rows nrow..ng-1 of the block are zero
    float ssf = 0.0f;   // a thread's sum of squares (FP32: FP64 arithmetic is slow here)
    {
      const bool hs_out = a.mode == 1;
      float* outb = (hs_out ? a.out : a.ckm1) + (long)b * a.npts + col;
      for (int i0 = half * ncb; i0 < (half + 1) * ncb; i0 += 8) {
        uint32_t r[8];
        tmem_ld4_issue(tE + lane_base + (uint32_t)(i0 / 2), r);
        tmem_ld4_issue(tO + lane_base + (uint32_t)(i0 / 2), r + 4);
        tmem_wait8(r);
        if (!live) continue;
        const float* psr = ps + i0 * TC_M + m;
        float* o = outb + (long)i0 * a.ncol;
        const int nv = nrow - i0, nall = ng - i0;
        if (nv >= 8) {   // eight live rows
#pragma unroll
          for (int s2 = 0; s2 < 8; ++s2) {
            const float v = fmaf(k1, __uint_as_float(r[(s2 & 1) * 4 + (s2 >> 1)]), psr[s2 * TC_M]);
            o[(long)s2 * a.ncol] = v;
            ssf = fmaf(v, v, ssf);
          }
        } else {
#pragma unroll
          for (int s2 = 0; s2 < 8; ++s2) {
            if (s2 >= nall) break;
            float v = 0.0f;
            if (s2 < nv) {
              v = fmaf(k1, __uint_as_float(r[(s2 & 1) * 4 + (s2 >> 1)]), psr[s2 * TC_M]);
              ssf = fmaf(v, v, ssf);
            }
            o[(long)s2 * a.ncol] = v;
          }
        }
      }
      if (hs_out) ssf = 0.0f;   // H_s q: no norm
    }
    // the sum of squares reduced in FP32 (across the warp, then across the 16 warps by warp 0):
    // one FP64 value per (block, tile)
    float ws = ssf;
    for (int o = 16; o > 0; o >>= 1) ws += __shfl_down_sync(0xffffffffu, ws, o);
    if (lane == 0) redf[warp] = ws;
    // the remainder written into ps by these threads precedes the copy engine's next write
    if constexpr (TMA) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // c_(k-1) is free: the next unit's
    if (u + 1 < u1 && a.mode == 0) {
      const int bn = unit_block(u + 1);
      stage(2, ps, a.ckm1 + (long)bn * a.npts, bn, a.blocks[bn].nrow, (long)unit_tile(u + 1) * TC_M);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0) {
      float v = lane < TC_THREADS / 32 ? redf[lane] : 0.0f;
      for (int o = 8; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0 && a.npart) a.npart[(long)b * a.ntiles + tile] = (double)v;
    }
    prev_u = u;
    slot ^= 1;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (!ok && tid == 0) atomicExch(a.err, 1);
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
  if constexpr (TMA) {   // no tile copy may still be writing shared memory when the CTA ends
    for (int w = 0; w < 3; ++w)
      if (tpend[w]) (void)mbar_wait(smem_u32(tbar + w), tph[w]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
  }
}

// out[iJ] = sum over the (J, Omega) groups of J and their tiles: 256 threads per J take
// strided partial sums of the contiguous range, then a fixed-order tree (deterministic).
__global__ void __launch_bounds__(256) k_tc_norm_final(const double* __restrict__ npart,
                                                       const int* __restrict__ g_begin,
                                                       int ntiles, double* __restrict__ out) {
  __shared__ double red[256];
  const int iJ = blockIdx.x;
  const long e0 = (long)g_begin[iJ] * ntiles, e1 = (long)g_begin[iJ + 1] * ntiles;
  double s = 0;
  for (long e = e0 + threadIdx.x; e < e1; e += 256) s += npart[e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[iJ] = red[0];
}


// ================================================================== energy-sum flush
// Mixed precision: for J index iJ (blockIdx.z), a tile of 128 cut-ring columns (blockIdx.y)
// and 128 phase rows (blockIdx.x, fastest, so the tiles that share columns run together):
//   D[col][p] = sum_(k < kb) cut[k][colbase + col] ph[iJ][p][k]   (M = columns, N = phases)
//   acc[accoff + p ncols + col] += D  (FP64)
// on the tensor cores in split-TF32 (FP32 products within a flush, FP64 across flushes),
// K in chunks of FL_KC ring slots. Column j of the tile is tensor-memory lane j, so the FP64
// read-modify-write of one phase row is 128 consecutive doubles.
// FL_KC = 16 keeps shared memory at 32 KB per CTA, so tensor memory (128 columns per CTA)
// sets the residency: 4 CTAs per SM (3 with 32-wide chunks; 4.35 against 3.37 ms per flush)
constexpr int FL_M = 128, FL_N = 128, FL_KC = 16, FL_THREADS = 128;

__global__ void __launch_bounds__(FL_THREADS) k_flush_tc(const float* __restrict__ ph,
                                                         const float* __restrict__ cut,
                                                         long ncut_total, int kb, int kn, int nE2,
                                                         const long* __restrict__ colbase,
                                                         const long* __restrict__ ncols,
                                                         const long* __restrict__ accoff,
                                                         double* __restrict__ acc,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr uint32_t abytes = FL_M * FL_KC * 4, bbytes = FL_N * FL_KC * 4;
  unsigned char* Ahi = sm;
  unsigned char* Alo = Ahi + abytes;
  unsigned char* Bhi = Alo + abytes;
  unsigned char* Blo = Bhi + bbytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + bbytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int iJ = blockIdx.z;
  const long nc = ncols[iJ];
  const long c0 = (long)blockIdx.y * FL_M;
  const int p0 = blockIdx.x * FL_N;
  if (c0 >= nc) return;   // CTA-uniform, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5;
  const long col = c0 + tid;
  const bool live = col < nc;
  const uint32_t mb = smem_u32(mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(FL_N));
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
  const uint32_t idesc = idesc_tf32(FL_M, FL_N);
  const float* cutc = cut + colbase[iJ] + col;
  const float* phr = ph + ((long)iJ * nE2 + p0 + tid) * kb;
  const bool prow = p0 + tid < nE2;
  uint32_t phase = 0;
  bool ok = true;
  for (int kc = 0; kc < kn && ok; kc += FL_KC) {
    if (kc > 0) __syncthreads();   // the previous chunk's MMAs have completed (waited below)
    // A: row = column of the tile, K = ring slot; B: row = phase row, K = ring slot
    float x[FL_KC];
#pragma unroll
    for (int k = 0; k < FL_KC; ++k)
      x[k] = (live && kc + k < kn) ? __ldg(cutc + (long)(kc + k) * ncut_total) : 0.0f;
    float y[FL_KC];
#pragma unroll
    for (int k = 0; k < FL_KC; ++k) y[k] = (prow && kc + k < kn) ? __ldg(phr + kc + k) : 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < FL_KC; k4 += 4) {
      float4 h, l;
      h.x = tf32_hi(x[k4]); l.x = x[k4] - h.x;
      h.y = tf32_hi(x[k4 + 1]); l.y = x[k4 + 1] - h.y;
      h.z = tf32_hi(x[k4 + 2]); l.z = x[k4 + 2] - h.z;
      h.w = tf32_hi(x[k4 + 3]); l.w = x[k4 + 3] - h.w;
      const uint32_t off = cm_off(tid, k4, FL_KC);
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
      h.x = tf32_hi(y[k4]); l.x = y[k4] - h.x;
      h.y = tf32_hi(y[k4 + 1]); l.y = y[k4 + 1] - h.y;
      h.z = tf32_hi(y[k4 + 2]); l.z = y[k4 + 2] - h.z;
      h.w = tf32_hi(y[k4 + 3]); l.w = y[k4 + 3] - h.w;
      *reinterpret_cast<float4*>(Bhi + off) = h;
      *reinterpret_cast<float4*>(Blo + off) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sbo = FL_KC * 32, lbo = 128;
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
      for (int ks = 0; ks < FL_KC / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256;
        mma_tf32(tmem, smem_desc(ah + o, lbo, sbo), smem_desc(bh + o, lbo, sbo), idesc,
                 (kc > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + o, lbo, sbo), smem_desc(bl + o, lbo, sbo), idesc, 1);
        mma_tf32(tmem, smem_desc(al + o, lbo, sbo), smem_desc(bh + o, lbo, sbo), idesc, 1);
      }
      mma_commit(mb);
    }
    ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (ok) {
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    double* accJ = acc + accoff[iJ] + col;
    for (int j0 = 0; j0 < FL_N; j0 += 16) {   // 16 read-modify-writes in flight per thread
      float v[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) tmem_ld4(tmem + lane_base + (uint32_t)(j0 + 4 * u), v + 4 * u);
      if (!live) continue;
      double o[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int p = p0 + j0 + j;
        o[j] = p < nE2 ? accJ[(long)p * nc] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int p = p0 + j0 + j;
        if (p < nE2) accJ[(long)p * nc] = o[j] + (double)v[j];
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  drain_expired(ok, mb, phase ^ 1u);   // ok is CTA-uniform; the failed wait toggled phase
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(FL_N));
  }
}

cudaError_t launch_flush_tc(const float* ph, const float* cut, long ncut_total, int kb, int nvalid, int nJ,
                            int nE, const long* colbase, const long* ncols, const long* accoff,
                            long max_cols, double* acc, int* err, cudaStream_t st) {
  const long ytiles = (max_cols + FL_M - 1) / FL_M;
  if (ytiles > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)((2 * nE + FL_N - 1) / FL_N), (unsigned)ytiles, (unsigned)nJ);
  const size_t smem = 2 * (size_t)FL_M * FL_KC * 4 + 2 * (size_t)FL_N * FL_KC * 4 + 64;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_flush_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  // ring slots past the valid ones carry zero phases: multiply the valid ones only (K rounded up
  // to the chunk FL_KC); ph rows keep the stride kb
  const int kn = std::min(kb, ((nvalid + FL_KC - 1) / FL_KC) * FL_KC);
  if (kn <= 0) return cudaSuccess;
  k_flush_tc<<<grid, FL_THREADS, smem, st>>>(ph, cut, ncut_total, kb, kn, 2 * nE, colbase, ncols,
                                             accoff, acc, err);
  return cudaGetLastError();
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

template <int KH, int NE>
static cudaError_t launch_tc3_inst(const TcArgs& args, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_angular_tc3<KH, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  const long total = (long)args.ngroups * args.ntiles;
  const unsigned grid = (unsigned)std::min<long>(total, args.nsm);
  k_angular_tc3<KH, NE><<<grid, TC_THREADS, tc3_smem<KH>(), st>>>(args);
  return cudaGetLastError();
}

template <int NE>
static cudaError_t launch_tc3_ne(const TcArgs& a, cudaStream_t st) {
  switch (a.kh) {
    case 16: return launch_tc3_inst<16, NE>(a, st);
    case 32: return launch_tc3_inst<32, NE>(a, st);
    case 48: return launch_tc3_inst<48, NE>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int KH>
static cudaError_t launch_tc4_inst(const TcArgs& args, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_angular_tc4<KH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  const long total = (long)args.ngroups * args.ntiles;
  const unsigned grid = (unsigned)std::min<long>(total, args.nsm);
  k_angular_tc4<KH><<<grid, TC_THREADS, tc4_smem<KH>(), st>>>(args);
  return cudaGetLastError();
}

static cudaError_t launch_tc4(const TcArgs& a, cudaStream_t st) {
  switch (a.kh) {
    case 64: return launch_tc4_inst<64>(a, st);
    case 80: return launch_tc4_inst<80>(a, st);
    case 96: return launch_tc4_inst<96>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int KH, bool TMA>
static cudaError_t launch_tc5_tma(const TcArgs& args, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_angular_tc5<KH, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr = true;
  }
  const long total = (long)args.ngroups * args.ntiles;
  const unsigned grid = (unsigned)std::min<long>(total, args.nsm);
  k_angular_tc5<KH, TMA><<<grid, TC_THREADS, tc5_smem<KH>(), st>>>(args);
  return cudaGetLastError();
}

template <int KH>
static cudaError_t launch_tc5_inst(const TcArgs& args, cudaStream_t st) {
  return args.tma ? launch_tc5_tma<KH, true>(args, st) : launch_tc5_tma<KH, false>(args, st);
}

static cudaError_t launch_tc5(const TcArgs& a, cudaStream_t st) {
  switch (a.kh) {
    case 16: return launch_tc5_inst<16>(a, st);
    case 32: return launch_tc5_inst<32>(a, st);
    case 48: return launch_tc5_inst<48>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

int angular_tc4_kh(int ng, int nelec) {
  if (ng % 2 || nelec != 1) return 0;
  const int kh = ((ng / 2 + 15) / 16) * 16;
  return (kh > 48 && kh <= 96) ? kh : 0;
}

int angular_tc3_kh(int ng, int nelec) {
  if (ng % 2) return 0;
  const int kh = ((ng / 2 + 15) / 16) * 16;
  if (kh > 48 || (nelec == 2 && 10 * kh > 512) || nelec > 2) return 0;
  return kh;
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

// cuTensorMapEncodeTiled through the driver's entry point (the library does not link libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                        &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// A [rows x ncol] FP32 matrix (row stride ncol) as a 2-D tensor map with 128 x 8 boxes,
// no swizzle (shared-memory layout [8][128], the tile layout of the angular step), zero fill
// beyond the edges.
static bool tile_map(CUtensorMap* map, const float* base, long ncol, long rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || !base || (ncol * 4) % 16 != 0) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)ncol, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)ncol * 4};
  const cuuint32_t box[2] = {(cuuint32_t)TC_M, 8u};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_angular_tc(const TcArgs& args, int ngroups, const int* g_begin, int nJ,
                              double* norm_out, cudaStream_t st) {
  cudaError_t e;
  if (args.persistent == 4) {
    if (args.tma) {   // tile copies by the tensor memory accelerator when the maps encode
      TcArgs a = args;
      const long rows = (long)ngroups * args.ng;   // one electronic state: one block per group
      a.tma = tile_map(&a.tm_ck, a.ck, a.ncol, rows) && tile_map(&a.tm_t, a.t, a.ncol, rows) &&
              (a.mode != 0 || tile_map(&a.tm_ckm1, a.ckm1, a.ncol, rows));
      e = launch_tc5(a, st);
    } else {
      e = launch_tc5(args, st);
    }
  } else if (args.persistent == 3) {
    e = launch_tc4(args, st);
  } else if (args.persistent == 2) {
    e = (args.nelec == 1) ? launch_tc3_ne<1>(args, st) : launch_tc3_ne<2>(args, st);
  } else if (args.persistent) {
    e = (args.nelec == 1) ? launch_tc2_ne<1>(args, st) : launch_tc2_ne<2>(args, st);
  } else {
    if (args.ntiles > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)ngroups, (unsigned)args.ntiles);
    e = (args.nelec == 1) ? launch_tc_ne<1>(args, grid, st) : launch_tc_ne<2>(args, grid, st);
  }
  if (e != cudaSuccess) return e;
  if (norm_out && args.npart) {
    k_tc_norm_final<<<nJ, 256, 0, st>>>(args.npart, g_begin, args.ntiles, norm_out);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace mw3
