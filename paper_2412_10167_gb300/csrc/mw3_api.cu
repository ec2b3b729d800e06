// libmw3: context, set-up and the propagation driver behind include/mw3.h.
//
// The state of every block is held in its angular FBR (coefficients of the
// normalised associated Legendre functions j = Omega..ngamma-1 on each (r, R) point;
// mw3_get_state / mw3_set_state convert to and from values on the Gauss-Legendre
// grid). One propagation step (Eq. wvp-k) is the launch sequence
//   1. kinetic_rows   t = T_R c_k                          (R lines, DST-II kinetic)
//   2. kinetic_cols   t += T_r c_k; flux cut of c_k; c_k column at R_inf
//   3. gamma_to_dvr   u = (T^Omega)^T c_k                  (per block)
//   4. gamma_update   w = T^Omega V u; h = w + angular/Coriolis + t;
//                     c_(k+1) = D (alpha H_s c_k - beta D c_(k-1)), over c_(k-1)
//   5. channels       reactant-channel overlaps of c_k
//   6. norms          ||c_(k+1)||^2 per J
// The flux cut and overlaps of kb consecutive iterations are kept in a ring; every
// kb iterations (a "chunk") the energy sums are updated by one GEMM
//   A[J][2nE x cols] += Ph[J][2nE x kb] Cut[kb x cols],  Ph = Re/Im of c_k(E),
// so the FP64 accumulators are read and written once per chunk instead of once
// per iteration. Full chunks after the first are captured once as a CUDA graph and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "mw3_host.h"
#include "mw3_internal.h"

using namespace mw3;

namespace {

const char* kKernelNames[] = {"kinetic_rows", "kinetic_cols", "gamma_to_dvr", "gamma_update",
                              "channels",     "norms",        "sums_flush",   "angular_tc",
                              "products",     "autocorrelation", "time_packets", "kinetic_radial",
                              "pcb_packet"};
constexpr int kNumKernels = 13;
constexpr int kPcbKernel = 12;   // the one-off products-coordinate transform (not a step kernel)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

bool is_235(int n) {
  if (n <= 0) return false;
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

FFTPlan make_plan(int N) {
  FFTPlan p{};
  p.N = N;
  int n = N, s = 0;
  for (int r : {4, 2, 3, 5}) {
    while (n % r == 0 && s < 16) {
      p.radix[s++] = r;
      n /= r;
    }
  }
  p.nstages = s;
  return p;
}

}  // namespace

struct mw3_ctx {
  int device = -1;
  int precision = MW3_FP64;
  bool host_only = false;
  cudaStream_t stream = nullptr;
  // host-to-device state uploads: a copy stream and one event per block group, so that a
  // group's conversion and gamma transform overlap the next group's copy
  cudaStream_t up_stream = nullptr;
  bool up_direct_last = false;   // the last state upload read mapped host memory directly
  cudaEvent_t up_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool own_stream = false;
  mw3_alloc_fn alloc = nullptr;
  mw3_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::string err;
  int stage = 0;  // 1 grid, 2 potential, 3 packet, 4 absorber, 5 analysis
  Tuning tune{4, 32, 32, 1, 0, 2, 4, 1, 0, 0, 0, 1, 1L << 22};
  int nsm = 152;       // streaming multiprocessors of the device
  int kp = 0;          // ngamma padded to a multiple of 16 (tensor-core path)
  int kh = 0;          // parity-split operand size, resident form (0: not applicable)
  int kh4 = 0;         // parity-split operand size, streamed form (0: not applicable)
  bool tc_ok = false;  // the tensor-core angular step supports this grid
  // |a(E)|^2 of the incoming packet on the energy grid, kept until the packet or the grid changes
  std::vector<double> a2_cache;
  int tc_user = -1;    // explicit "use_tc" setting (-1: default = on when supported)

  // grid and blocks
  int NR = 0, nr = 0, ng = 0, nelec = 1, nJ = 0, omega_max = 0;
  double Rmin = 0, Rmax = 0, rmin = 0, rmax = 0, dR = 0, dr = 0;
  double mA = 0, mB = 0, mC = 0, mu = 0, m = 0;
  std::vector<int> J, omtop;
  std::vector<double> R, r, x, w, fR, fr;
  std::vector<DevBlock> blocks;
  int nblk = 0;
  long ncol = 0, npts = 0;
  std::vector<long> J_first_block;        // nJ + 1
  std::vector<int> coef_of;               // (iJ, om) -> coef index
  std::vector<std::vector<double>> T;     // T^Omega, Omega = 0..max top
  std::vector<double> coef;               // [ncoef][5][ng]
  int ncoef = 0;
  FFTPlan planR{}, planr{};

  // potential and caps
  double vcut = 0, tcut = 0, erot = 0;
  std::vector<double> V;                  // [L][L'][npts]
  std::vector<double> lamR, lamr;         // lambda_j, j = 0..N (lambda_0 = 0)
  std::vector<double> E0, dE;
  mw3_pot_fn pot_fn = nullptr;
  void* pot_user = nullptr;

  // packet
  mw3_packet_desc packet{};
  double Ev0j0 = 0;
  std::vector<double> q0;
  std::vector<double> g_tilde;
  // device tables of the channel-probability kernel (built by mw3_set_analysis)
  ChanTable chan_tab_r{}, chan_tab_p{};
  // products-coordinate-based start (mw3_init_packet_pcb): a(E) in closed form from the
  // packet's g(R_s) = N exp(-(R_s - R0)^2 / (2 G^2)) cos(k0 R_s) and reduced mass mu_s
  bool pcb_on = false;
  double pcb_mu = 0, pcb_N = 0, pcb_R0 = 0, pcb_G = 0, pcb_k0 = 0;

  // absorber
  std::vector<double> DR, Dr;

  // analysis
  mw3_analysis_desc an{};
  std::vector<double> Ecol, theta;        // theta[iJ * nE + e]
  std::vector<double> wpsi, wdpsi;
  int m_inf = 0;
  int nchan = 0;
  std::vector<int> chan_block, chan_row, chan_col, chan_v, chan_j, chan_om, chan_lam, chan_iJ;
  std::vector<double> chan_eps;
  // flux-cut ring (the context's precision): per J 2 ncut columns (psi, dpsi)
  std::vector<long> colbase, ncols, ncut, accoff;
  long NC = 0, max_cols = 0, acc_size = 0;
  // channel ring (FP64 in both precisions): per J the reactant, then the product channels
  std::vector<long> colbase_c, ncols_c, accoff_c;
  long NCc = 0, max_cols_c = 0, accc_size = 0;

  // product channels (mw3_set_products)
  bool prod_on = false;
  mw3_products_desc prod{};
  double mu_p = 0, m_p = 0;
  int prod_nn = 0, prod_ltop = 0;
  std::vector<int> prod_idx;               // [node][8]: R stencil, then r stencil
  std::vector<double> prod_w;              // [node][8] Lagrange weights (R ones / sqrt(dR dr))
  // plane-major form: distinct stencil columns r * NR + R, sorted and padded to a multiple of
  // 32 (prod_spad) with copies of the last one; per node and stencil point s = 4 c + a its
  // row in that list and the weight wR_a wr_c; FBR rows padded to prod_ngp
  std::vector<int> prod_pts, prod_pix;
  std::vector<double> prod_wst;
  int prod_npts = 0, prod_spad = 0, prod_ngp = 0;
  std::vector<double> prod_pl;             // [node][ltop][ng] P-bar_(Omega+i)^Omega(cos gamma)
  std::vector<double> prod_T;              // per J: [node][nom][nom] helicity transforms
  std::vector<double> prod_jac;            // [node] r'R'/(rR)
  std::vector<double> prod_W;              // [channel][node] quadrature weights
  std::vector<ProdGroup> prod_groups;      // col0 set by mw3_set_analysis
  std::vector<int> prod_jl;                // [iJ * nelec + L]: its Omega' = 0 group
  std::vector<int> prod_chan;              // [channel][2]: group, cut column
  int prod_max_nom = 0;
  std::vector<long> prod_first;            // nJ + 1: first channel of each J
  std::vector<int> pch_L, pch_v, pch_j, pch_op;
  std::vector<double> pch_eps;

  // propagation state
  long iter = 0;       // k of q_k
  int ring_n = 0;      // ring slots 0 .. ring_n - 1 hold iterations not yet flushed into the sums
  // the flux accumulators change with every flush, reset and load; a probability read keeps
  // their flux ("fluxA") and, in the mixed form, an FP32 copy ("acc32") for the reads that
  // follow while only ring slots are added
  long acc_version = 0;
  long fluxA_version = -1;
  int cur = 0;         // d_q[cur] holds q_k
  std::vector<double> norm_trace;  // [iter][nJ], ||q_k||^2 for k = 1..iter
  double norm0 = 1.0;
  // photodissociation analysis: C_k = <q_0|q_k> per J, k = 0..iter-1, after
  // mw3_enable_autocorrelation stored q_0
  bool ac_on = false;
  std::vector<double> ac_trace;    // [k][nJ]
  // time-domain packets: Psi(t_j) = sum_(k < tp_K) f_k(t_j) q_k accumulated in FP64 (FBR)
  bool tp_on = false;
  int tp_nt = 0;
  long tp_K = 0;

  // graphs
  cudaGraphExec_t graph[2] = {nullptr, nullptr};

  // timing: events recorded around launches, read back at chunk boundaries
  bool timing = false;
  cudaEvent_t ev[2 * kNumKernels] = {};
  std::vector<cudaEvent_t> evpool;
  std::vector<std::pair<int, int>> evrec;  // (kernel id, index of the start event)
  double kms[kNumKernels] = {};
  long klaunch[kNumKernels] = {};

  // device buffers
  std::map<std::string, DevBuf> buf;

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  size_t rs() const { return precision == MW3_FP64 ? 8 : 4; }
};

// ------------------------------------------------------------------ helpers
namespace {

thread_local std::string g_create_err;

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ctx->fail(MW3_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void* dptr(mw3_ctx* ctx, const char* name) {
  auto it = ctx->buf.find(name);
  return it == ctx->buf.end() ? nullptr : it->second.p;
}

int dfree(mw3_ctx* ctx, const char* name) {
  auto it = ctx->buf.find(name);
  if (it == ctx->buf.end()) return MW3_OK;
  if (it->second.p) {
    if (ctx->free_fn)
      ctx->free_fn(it->second.p, ctx->alloc_user);
    else
      cudaFree(it->second.p);
  }
  ctx->buf.erase(it);
  return MW3_OK;
}

// (Re)allocate a named device buffer; contents undefined.
int dalloc(mw3_ctx* ctx, const char* name, size_t bytes) {
  if (ctx->host_only) return MW3_OK;
  auto it = ctx->buf.find(name);
  if (it != ctx->buf.end() && it->second.bytes == bytes) return MW3_OK;
  dfree(ctx, name);
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->alloc_user);
    if (!p) return ctx->fail(MW3_ERR_OOM, std::string("allocator hook failed for ") + name);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess)
      return ctx->fail(MW3_ERR_OOM, std::string("cudaMalloc ") + name + ": " + cudaGetErrorString(e));
  }
  ctx->buf[name] = DevBuf{p, bytes};
  return MW3_OK;
}

int dzero(mw3_ctx* ctx, const char* name) {
  if (ctx->host_only) return MW3_OK;
  auto it = ctx->buf.find(name);
  if (it == ctx->buf.end()) return MW3_OK;
  CK(cudaMemsetAsync(it->second.p, 0, it->second.bytes, ctx->stream));
  return MW3_OK;
}

// Upload host doubles as the context's real type (or as doubles with as_double).
int upload_real(mw3_ctx* ctx, const char* name, const std::vector<double>& h, bool as_double = false) {
  const size_t es = as_double ? 8 : ctx->rs();
  int st = dalloc(ctx, name, h.size() * es);
  if (st) return st;
  if (ctx->host_only) return MW3_OK;
  if (es == 8) {
    CK(cudaMemcpyAsync(dptr(ctx, name), h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    std::vector<float> f(h.begin(), h.end());
    CK(cudaMemcpyAsync(dptr(ctx, name), f.data(), f.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

template <typename Tv>
int upload_raw(mw3_ctx* ctx, const char* name, const std::vector<Tv>& h) {
  int st = dalloc(ctx, name, h.size() * sizeof(Tv));
  if (st) return st;
  if (ctx->host_only) return MW3_OK;
  CK(cudaMemcpyAsync(dptr(ctx, name), h.data(), h.size() * sizeof(Tv), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// Complex tables for the FFT: twiddles exp(-2 pi i t/N) and exp(-i pi k / 2N).
int upload_fft_tables(mw3_ctx* ctx, const char* twn, const char* phn, int N) {
  std::vector<double> tw(2 * N), ph(2 * N);
  for (int t = 0; t < N; ++t) {
    tw[2 * t] = std::cos(2.0 * M_PI * t / N);
    tw[2 * t + 1] = -std::sin(2.0 * M_PI * t / N);
    ph[2 * t] = std::cos(M_PI * t / (2.0 * N));
    ph[2 * t + 1] = -std::sin(M_PI * t / (2.0 * N));
  }
  int st = upload_real(ctx, twn, tw);
  if (st) return st;
  return upload_real(ctx, phn, ph);
}

double lam_pm(double X, int om, int sign) {
  return std::sqrt(std::max(X * (X + 1.0) - (double)om * (om + sign), 0.0));
}

// diatomic Hamiltonian T_r + min(j(j+1) f_r, E_rot) + min(V_LL(r, R=100), vcut)
int diatomic(mw3_ctx* ctx, int j, int lam, int nv, std::vector<double>& E, std::vector<double>& chi) {
  const int n = ctx->nr;
  std::vector<double> H((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double s = 0;
      for (int jj = 1; jj <= n; ++jj) s += dst2(n, jj, a + 1) * ctx->lamr[jj] * dst2(n, jj, b + 1);
      H[(size_t)a * n + b] = s;
    }
  std::vector<double> pm((size_t)ctx->nelec * ctx->nelec);
  for (int a = 0; a < n; ++a) {
    double v;
    if (ctx->pot_fn) {
      if (ctx->pot_fn(ctx->r[a], 100.0, 0.0, pm.data(), ctx->pot_user) != 0)
        return ctx->fail(MW3_ERR_BAD_ARG, "potential callback failed");
      v = pm[(size_t)lam * ctx->nelec + lam];
    } else {
      // grid potential: the diatomic curve is taken at the last R node
      v = ctx->V[(size_t)(lam * ctx->nelec + lam) * ctx->npts + (size_t)0 * ctx->ncol +
                 (size_t)a * ctx->NR + (ctx->NR - 1)];
    }
    v = std::min(v, ctx->vcut);
    H[(size_t)a * n + a] += v + std::min(j * (j + 1.0) * ctx->fr[a], ctx->erot);
  }
  std::vector<double> ev, Z;
  symmetric_eigen(n, H, ev, Z);
  E.assign(ev.begin(), ev.begin() + nv);
  chi.assign((size_t)nv * n, 0.0);
  for (int v = 0; v < nv; ++v) {
    int imax = 0;
    for (int a = 0; a < n; ++a)
      if (std::fabs(Z[(size_t)a * n + v]) > std::fabs(Z[(size_t)imax * n + v])) imax = a;
    const double sg = Z[(size_t)imax * n + v] < 0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) chi[(size_t)v * n + a] = sg * Z[(size_t)a * n + v];
  }
  return MW3_OK;
}

#define LK(expr)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ctx->fail(MW3_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Transform `n` host FP64 values between the grid (DVR) and the FBR of every block
// on the device: to_fbr = 1 computes T^Omega x into dst_name, 0 computes (T^Omega)^T x.
// Device address of the `bytes` of caller memory at `p` when the whole range lies inside one
// page-locked host allocation that is mapped into the device's address space at the same
// address (cudaHostAlloc, cudaHostRegister); nullptr otherwise (the caller then copies with
// the DMA engines). The allocation's extent comes from the driver, so a kernel reading the
// alias never leaves the allocation.
const double* mapped_host_alias(const double* p, size_t bytes) {
  if (reinterpret_cast<uintptr_t>(p) % 16) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || at.devicePointer != static_cast<const void*>(p))
    return nullptr;
  using AttrFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static AttrFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<AttrFn>(f);
  }();
  if (!fn) return nullptr;
  CUdeviceptr start = 0;
  size_t size = 0;
  const CUdeviceptr a = (CUdeviceptr)reinterpret_cast<uintptr_t>(p);
  if (fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, a) != CUDA_SUCCESS ||
      fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, a) != CUDA_SUCCESS)
    return nullptr;
  if (start > a || a + bytes > start + size) return nullptr;
  return p;
}

// Host state values (FP64, or FP32 for mw3_set_state_f32) -> the FBR coefficients of
// buffer `dst_name` in the context's precision. The values cross in four block groups on the
// copy stream; each group's conversion and gamma transform on the library's stream overlap
// the next group's transfer.
template <typename Th>
int transform_upload(mw3_ctx* ctx, const Th* src, const char* dst_name, bool to_fbr) {
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  int st = dalloc(ctx, "xfer", n * ctx->rs());
  if (st) return st;
  const bool mixed = ctx->precision != MW3_FP64;
  // host values land in a staging buffer of their own type unless it is the state's type
  const bool same = mixed ? sizeof(Th) == 4 : sizeof(Th) == 8;
  const char* stage_name = sizeof(Th) == 8 ? "xfer64" : "xfer32";
  if (!same && (st = dalloc(ctx, stage_name, n * sizeof(Th)))) return st;
  Th* stg = (Th*)dptr(ctx, same ? "xfer" : stage_name);
  if (!ctx->up_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    for (auto& e : ctx->up_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  // page-locked, mapped FP64 caller memory may be read by a kernel over the host link and
  // converted on the way (no staging copy); everything else goes through the DMA engines
  const double* alias = nullptr;
  if constexpr (sizeof(Th) == 8)
    alias = ctx->tune.up_direct ? mapped_host_alias(src, n * 8) : nullptr;
  ctx->up_direct_last = alias != nullptr;
  // the copies start after earlier work on the library's stream (which may still read xfer)
  CK(cudaEventRecord(ctx->up_ev[4], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->up_stream, ctx->up_ev[4], 0));
  // every return from here on, an error return included, first waits for the copies queued
  // on the copy stream: they read the caller's host buffer, which is free once we return
  struct CopyDrain {
    cudaStream_t s;
    ~CopyDrain() { cudaStreamSynchronize(s); }
  } drain{ctx->up_stream};
  const int G = std::min(ctx->nblk, 4);
  auto group = [&](int g, long& b0, long& nb) {
    b0 = (long)g * ctx->nblk / G;
    nb = (long)(g + 1) * ctx->nblk / G - b0;
  };
  for (int g = 0; g < G; ++g) {
    long b0, nb;
    group(g, b0, nb);
    const long off = b0 * ctx->npts, cnt = nb * ctx->npts;
    if (alias && mixed) {   // narrowed on the way in
      LK(launch_host_read<float>(alias + off, (float*)dptr(ctx, "xfer") + off, cnt, ctx->up_stream));
    } else if (alias) {
      LK(launch_host_read<double>(alias + off, (double*)dptr(ctx, "xfer") + off, cnt,
                                  ctx->up_stream));
    } else {
      CK(cudaMemcpyAsync(stg + off, src + off, (size_t)cnt * sizeof(Th), cudaMemcpyHostToDevice,
                         ctx->up_stream));
    }
    CK(cudaEventRecord(ctx->up_ev[g], ctx->up_stream));
  }
  const DevBlock* blk = (const DevBlock*)dptr(ctx, "blocks");
  for (int g = 0; g < G; ++g) {
    long b0, nb;
    group(g, b0, nb);
    const long off = b0 * ctx->npts, cnt = nb * ctx->npts;
    CK(cudaStreamWaitEvent(ctx->stream, ctx->up_ev[g], 0));
    if (mixed) {
      float* x = (float*)dptr(ctx, "xfer");
      if constexpr (sizeof(Th) == 8) {
        if (!alias) LK(launch_convert_d2f((const double*)stg + off, x + off, cnt, ctx->stream));
      }
      LK(launch_gamma_forward<float>(x + off, (float*)dptr(ctx, dst_name) + off,
                                     (const float*)dptr(ctx, to_fbr ? "T" : "Tt"), blk + b0,
                                     (int)nb, ctx->ng, ctx->ncol, ctx->stream));
    } else {
      double* x = (double*)dptr(ctx, "xfer");
      if constexpr (sizeof(Th) == 4)
        LK(launch_convert_f2d((const float*)stg + off, x + off, cnt, ctx->stream));
      LK(launch_gamma_forward<double>(x + off, (double*)dptr(ctx, dst_name) + off,
                                      (const double*)dptr(ctx, to_fbr ? "T" : "Tt"), blk + b0,
                                      (int)nb, ctx->ng, ctx->ncol, ctx->stream));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

int transform_download(mw3_ctx* ctx, const char* src_name, double* dst) {
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  int st = dalloc(ctx, "xfer", n * ctx->rs());
  if (st) return st;
  if (ctx->precision == MW3_FP64) {
    LK(launch_gamma_forward<double>((const double*)dptr(ctx, src_name), (double*)dptr(ctx, "xfer"),
                                    (const double*)dptr(ctx, "Tt"),
                                    (const DevBlock*)dptr(ctx, "blocks"), ctx->nblk, ctx->ng,
                                    ctx->ncol, ctx->stream));
    CK(cudaMemcpyAsync(dst, dptr(ctx, "xfer"), n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    LK(launch_gamma_forward<float>((const float*)dptr(ctx, src_name), (float*)dptr(ctx, "xfer"),
                                   (const float*)dptr(ctx, "Tt"),
                                   (const DevBlock*)dptr(ctx, "blocks"), ctx->nblk, ctx->ng,
                                   ctx->ncol, ctx->stream));
    if ((st = dalloc(ctx, "xfer64", n * 8))) return st;
    LK(launch_convert_f2d((const float*)dptr(ctx, "xfer"), (double*)dptr(ctx, "xfer64"), (long)n,
                          ctx->stream));
    CK(cudaMemcpyAsync(dst, dptr(ctx, "xfer64"), n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return MW3_OK;
}

const char* state_name(const mw3_ctx* ctx, bool current) {
  return (current == (ctx->cur == 0)) ? "q0" : "q1";
}

// Upload FBR coefficients as q_k (q_(k-1) = 0).
int upload_state_fbr(mw3_ctx* ctx, const double* c) {
  if (ctx->host_only) return MW3_OK;
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  if (ctx->precision == MW3_FP64) {
    CK(cudaMemcpyAsync(dptr(ctx, state_name(ctx, true)), c, n * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    std::vector<float> f(c, c + n);
    CK(cudaMemcpyAsync(dptr(ctx, state_name(ctx, true)), f.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  CK(cudaMemsetAsync(dptr(ctx, state_name(ctx, false)), 0, n * ctx->rs(), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// Device table of one channel set for k_channel_probs: keys ((iJ ne + L) nv + v) nj + j, each
// key's channels in channel order. Buffers are named with `pfx`.
int build_chan_table(mw3_ctx* ctx, const std::string& pfx, int nv, int nj, double mu,
                     const std::vector<int>& cJ, const std::vector<int>& cL,
                     const std::vector<int>& cv, const std::vector<int>& cj,
                     const std::vector<long>& ccol, const std::vector<double>& ceps,
                     ChanTable& t) {
  const int nkeys = ctx->nJ * ctx->nelec * nv * nj;
  const size_t nc = cJ.size();
  std::vector<std::vector<int>> per(nkeys);
  for (size_t c = 0; c < nc; ++c)
    per[((cJ[c] * ctx->nelec + cL[c]) * nv + cv[c]) * nj + cj[c]].push_back((int)c);
  std::vector<long> first(nkeys + 1, 0), ld(nc);
  std::vector<int> chans;
  for (int k = 0; k < nkeys; ++k) {
    first[k] = (long)chans.size();
    chans.insert(chans.end(), per[k].begin(), per[k].end());
  }
  first[nkeys] = (long)chans.size();
  for (size_t c = 0; c < nc; ++c) ld[c] = ctx->ncols_c[cJ[c]];
  if (chans.empty()) chans.push_back(0);   // keep the buffers non-empty
  int st;
  if ((st = upload_raw(ctx, (pfx + "_first").c_str(), first)) ||
      (st = upload_raw(ctx, (pfx + "_chan").c_str(), chans)) ||
      (st = upload_raw(ctx, (pfx + "_J").c_str(), nc ? cJ : std::vector<int>{0})) ||
      (st = upload_raw(ctx, (pfx + "_col").c_str(), nc ? ccol : std::vector<long>{0})) ||
      (st = upload_raw(ctx, (pfx + "_ld").c_str(), nc ? ld : std::vector<long>{0})) ||
      (st = upload_raw(ctx, (pfx + "_eps").c_str(), nc ? ceps : std::vector<double>{0.0})))
    return st;
  t.key_first = (const long*)dptr(ctx, (pfx + "_first").c_str());
  t.key_chan = (const int*)dptr(ctx, (pfx + "_chan").c_str());
  t.chJ = (const int*)dptr(ctx, (pfx + "_J").c_str());
  t.col = (const long*)dptr(ctx, (pfx + "_col").c_str());
  t.ld = (const long*)dptr(ctx, (pfx + "_ld").c_str());
  t.eps = (const double*)dptr(ctx, (pfx + "_eps").c_str());
  t.mu = mu;
  t.nkeys = nkeys;
  return MW3_OK;
}

// A new q_0 is in place: the iteration counter, traces and energy sums start over.
int reset_after_packet(mw3_ctx* ctx) {
  ctx->iter = 0;
  ctx->norm_trace.clear();
  ctx->ac_on = false;
  ctx->ac_trace.clear();
  ctx->tp_on = false;
  if (ctx->stage < 3) ctx->stage = 3;
  if (ctx->stage >= 5) {
    int st;
    if ((st = dzero(ctx, "acc")) || (st = dzero(ctx, "cut")) || (st = dzero(ctx, "accc")) ||
        (st = dzero(ctx, "cutc")) || (st = dzero(ctx, "d_iter")))
      return st;
    ctx->ring_n = 0;
    ++ctx->acc_version;
    if (!ctx->host_only) CK(cudaStreamSynchronize(ctx->stream));
  }
  return MW3_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

const char* mw3_status_string(int s) {
  switch (s) {
    case MW3_OK: return "ok";
    case MW3_ERR_BAD_ARG: return "bad argument";
    case MW3_ERR_OOM: return "out of memory";
    case MW3_ERR_CUDA: return "CUDA error";
    case MW3_ERR_DIVERGED: return "propagation diverged";
    case MW3_ERR_SPECTRUM: return "energy outside the spectral range";
    case MW3_ERR_TIMEOUT: return "device wait timed out";
    case MW3_ERR_STATE: return "call out of order";
    case MW3_ERR_IO: return "file error";
    case MW3_ERR_NAN: return "NaN or Inf in input";
    default: return "unknown status";
  }
}

const char* mw3_last_error(const mw3_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

int mw3_create(mw3_ctx** out, int device, int precision) {
  if (!out) return MW3_ERR_BAD_ARG;
  *out = nullptr;
  if (precision != MW3_FP64 && precision != MW3_MIXED) {
    g_create_err = "precision must be MW3_FP64 or MW3_MIXED";
    return MW3_ERR_BAD_ARG;
  }
  mw3_ctx* ctx = new (std::nothrow) mw3_ctx();
  if (!ctx) return MW3_ERR_OOM;
  ctx->precision = precision;
  ctx->device = device;
  ctx->tune.kb = (precision == MW3_FP64) ? 32 : 128;
  ctx->tune.cols_tile = 16;
  ctx->tune.rows_pairs = (precision == MW3_FP64) ? 4 : 8;
  if (device < 0) {
    ctx->host_only = true;  // set-up mathematics only (no device work)
  } else {
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
      g_create_err = std::string("CUDA device ") + std::to_string(device) + ": " + cudaGetErrorString(e);
      delete ctx;
      return MW3_ERR_CUDA;
    }
    ctx->own_stream = true;
    for (int i = 0; i < 2 * kNumKernels; ++i) cudaEventCreate(&ctx->ev[i]);
  }
  *out = ctx;
  return MW3_OK;
}

void mw3_destroy(mw3_ctx* ctx) {
  if (!ctx) return;
  if (!ctx->host_only) {
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& g : ctx->graph)
      if (g) cudaGraphExecDestroy(g);
    std::vector<std::string> names;
    for (auto& kv : ctx->buf) names.push_back(kv.first);
    for (auto& n : names) dfree(ctx, n.c_str());
    for (int i = 0; i < 2 * kNumKernels; ++i)
      if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (auto e : ctx->evpool) cudaEventDestroy(e);
    for (auto e : ctx->up_ev)
      if (e) cudaEventDestroy(e);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

int mw3_set_stream(mw3_ctx* ctx, void* stream) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (ctx->host_only) return MW3_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  ctx->own_stream = false;
  ctx->stream = static_cast<cudaStream_t>(stream);
  for (auto& g : ctx->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return MW3_OK;
}

int mw3_set_allocator(mw3_ctx* ctx, mw3_alloc_fn alloc, mw3_free_fn free_fn, void* user) {
  if (!ctx || (alloc == nullptr) != (free_fn == nullptr)) return MW3_ERR_BAD_ARG;
  if (!ctx->buf.empty()) return ctx->fail(MW3_ERR_STATE, "mw3_set_allocator must precede mw3_grid");
  ctx->alloc = alloc;
  ctx->free_fn = free_fn;
  ctx->alloc_user = user;
  return MW3_OK;
}

int mw3_grid(mw3_ctx* ctx, const mw3_grid_desc* d) {
  if (!ctx || !d) return MW3_ERR_BAD_ARG;
  if (d->NR < 2 || d->nr < 2 || d->NR % 2 || d->nr % 2 || !is_235(d->NR) || !is_235(d->nr) ||
      d->NR > 1024 || d->nr > 1024)
    return ctx->fail(MW3_ERR_BAD_ARG, "NR and nr must be even, 2^a 3^b 5^c and <= 1024");
  if (d->ngamma < 1 || d->ngamma > 256) return ctx->fail(MW3_ERR_BAD_ARG, "ngamma must be in 1..256");
  if (!(d->Rmax > d->Rmin) || !(d->rmax > d->rmin) || d->Rmin < 0 || d->rmin < 0)
    return ctx->fail(MW3_ERR_BAD_ARG, "grid intervals must be increasing and non-negative");
  if (d->nJ < 1 || !d->J || d->omega_max < 0 || d->nelec < 1 || d->nelec > 2)
    return ctx->fail(MW3_ERR_BAD_ARG, "need nJ >= 1, omega_max >= 0 and nelec in {1, 2}");
  for (int i = 0; i < 3; ++i)
    if (!(d->masses[i] > 0)) return ctx->fail(MW3_ERR_BAD_ARG, "masses must be positive");
  int jtop = 0;
  for (int i = 0; i < d->nJ; ++i) {
    if (d->J[i] < 0) return ctx->fail(MW3_ERR_BAD_ARG, "J must be >= 0");
    jtop = std::max(jtop, std::min(d->J[i], d->omega_max));
  }
  if (jtop >= d->ngamma)
    return ctx->fail(MW3_ERR_BAD_ARG, "min(J, omega_max) must be < ngamma (angular functions per block)");
  ctx->NR = d->NR;
  ctx->nr = d->nr;
  ctx->ng = d->ngamma;
  ctx->Rmin = d->Rmin;
  ctx->Rmax = d->Rmax;
  ctx->rmin = d->rmin;
  ctx->rmax = d->rmax;
  ctx->nelec = d->nelec;
  ctx->nJ = d->nJ;
  ctx->omega_max = d->omega_max;
  ctx->J.assign(d->J, d->J + d->nJ);
  ctx->mA = d->masses[0];
  ctx->mB = d->masses[1];
  ctx->mC = d->masses[2];
  ctx->mu = ctx->mA * (ctx->mB + ctx->mC) / (ctx->mA + ctx->mB + ctx->mC);
  ctx->m = ctx->mB * ctx->mC / (ctx->mB + ctx->mC);
  ctx->dR = (ctx->Rmax - ctx->Rmin) / ctx->NR;
  ctx->dr = (ctx->rmax - ctx->rmin) / ctx->nr;
  ctx->R.resize(ctx->NR);
  ctx->r.resize(ctx->nr);
  ctx->fR.resize(ctx->NR);
  ctx->fr.resize(ctx->nr);
  for (int i = 0; i < ctx->NR; ++i) {
    ctx->R[i] = ctx->Rmin + (i + 0.5) * ctx->dR;
    ctx->fR[i] = 1.0 / (2.0 * ctx->mu * ctx->R[i] * ctx->R[i]);
  }
  for (int i = 0; i < ctx->nr; ++i) {
    ctx->r[i] = ctx->rmin + (i + 0.5) * ctx->dr;
    ctx->fr[i] = 1.0 / (2.0 * ctx->m * ctx->r[i] * ctx->r[i]);
  }
  gauss_legendre(ctx->ng, ctx->x, ctx->w);
  ctx->ncol = (long)ctx->nr * ctx->NR;
  ctx->npts = (long)ctx->ng * ctx->ncol;

  // blocks: J-major, Omega, Lambda
  ctx->blocks.clear();
  ctx->omtop.assign(ctx->nJ, 0);
  ctx->J_first_block.assign(ctx->nJ + 1, 0);
  ctx->coef_of.clear();
  int maxtop = 0;
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    const int top = std::min(ctx->J[iJ], ctx->omega_max);
    ctx->omtop[iJ] = top;
    maxtop = std::max(maxtop, top);
    ctx->J_first_block[iJ] = (long)ctx->blocks.size();
    for (int om = 0; om <= top; ++om) {
      const int ci = (int)ctx->coef_of.size();
      ctx->coef_of.push_back(iJ * 4096 + om);
      for (int L = 0; L < ctx->nelec; ++L) {
        DevBlock b{};
        b.iJ = iJ;
        b.omega = om;
        b.lam = L;
        b.coef = ci;
        b.base = (int)ctx->blocks.size() - L;
        b.nrow = ctx->ng - om;
        ctx->blocks.push_back(b);
      }
    }
  }
  ctx->J_first_block[ctx->nJ] = (long)ctx->blocks.size();
  ctx->nblk = (int)ctx->blocks.size();
  ctx->ncoef = (int)ctx->coef_of.size();
  for (auto& b : ctx->blocks) {
    const int top = ctx->omtop[b.iJ];
    const int per_om = ctx->nelec;
    const int idx = (int)(&b - &ctx->blocks[0]);
    b.up = (b.omega + 1 <= top) ? idx + per_om : -1;
    b.dn = (b.omega >= 1) ? idx - per_om : -1;
  }
  ctx->T.assign(maxtop + 1, {});
  for (int om = 0; om <= maxtop; ++om) fbr_matrix(om, ctx->ng, ctx->x, ctx->w, ctx->T[om]);
  ctx->planR = make_plan(ctx->NR);
  ctx->planr = make_plan(ctx->nr);
  ctx->stage = 1;
  ctx->iter = 0;
  return MW3_OK;
}

static int finish_potential(mw3_ctx* ctx, double vcut, double tcut, double erot) {
  ctx->vcut = vcut;
  ctx->tcut = tcut;
  ctx->erot = erot;
  const long np = ctx->npts;
  const int ne = ctx->nelec;
  for (double v : ctx->V)
    if (!std::isfinite(v)) return ctx->fail(MW3_ERR_NAN, "potential contains NaN or Inf");
  for (int L = 0; L < ne; ++L)
    for (long i = 0; i < np; ++i) {
      double& v = ctx->V[(size_t)(L * ne + L) * np + i];
      v = std::min(v, vcut);
    }
  // radial kinetic eigenvalues lambda_j = min(k_j^2 / 2 mass, tcut), lambda_0 = 0
  ctx->lamR.assign(ctx->NR + 1, 0.0);
  ctx->lamr.assign(ctx->nr + 1, 0.0);
  for (int j = 1; j <= ctx->NR; ++j) {
    const double k = j * M_PI / (ctx->Rmax - ctx->Rmin);
    ctx->lamR[j] = std::min(k * k / (2.0 * ctx->mu), tcut);
  }
  for (int j = 1; j <= ctx->nr; ++j) {
    const double k = j * M_PI / (ctx->rmax - ctx->rmin);
    ctx->lamr[j] = std::min(k * k / (2.0 * ctx->m), tcut);
  }
  // angular coefficient sets
  const int ng = ctx->ng;
  ctx->coef.assign((size_t)ctx->ncoef * kCoefRows * ng, 0.0);
  for (int ci = 0; ci < ctx->ncoef; ++ci) {
    const int iJ = ctx->coef_of[ci] / 4096, om = ctx->coef_of[ci] % 4096;
    const double Jv = ctx->J[iJ];
    const int top = ctx->omtop[iJ];
    double* cf = &ctx->coef[(size_t)ci * kCoefRows * ng];
    for (int i = 0; i < ng; ++i) {
      if (i >= ng - om) {  // beyond the block's angular functions
        cf[4 * ng + i] = 1e300;
        continue;
      }
      const double j = om + i;
      const double jj = j * (j + 1.0);
      cf[i] = jj;
      cf[ng + i] = Jv * (Jv + 1.0) + jj - 2.0 * om * om;
      cf[2 * ng + i] = (om + 1 <= top && i >= 1)
                           ? -lam_pm(Jv, om, +1) * lam_pm(j, om, +1) * (om == 0 ? std::sqrt(2.0) : 1.0)
                           : 0.0;
      cf[3 * ng + i] = (om >= 1)
                           ? -lam_pm(Jv, om, -1) * lam_pm(j, om, -1) * (om == 1 ? std::sqrt(2.0) : 1.0)
                           : 0.0;
      const double lmax2 = std::pow(std::sqrt(Jv * (Jv + 1.0)) + std::sqrt(jj), 2);
      cf[4 * ng + i] = (lmax2 == 0.0) ? 1e300 : erot / lmax2;
    }
  }
  // spectral bounds per J
  double vmin = 1e300, vmax = -1e300;
  for (long i = 0; i < np; ++i) {
    if (ne == 1) {
      vmin = std::min(vmin, ctx->V[i]);
      vmax = std::max(vmax, ctx->V[i]);
    } else {
      const double a = ctx->V[i], b = ctx->V[(size_t)np + i], dd = ctx->V[(size_t)3 * np + i];
      const double h = 0.5 * (a + dd), s = std::sqrt(0.25 * (a - dd) * (a - dd) + b * b);
      vmin = std::min(vmin, h - s);
      vmax = std::max(vmax, h + s);
    }
  }
  const double radmax = ctx->lamR[ctx->NR] + ctx->lamr[ctx->nr];
  ctx->E0.assign(ctx->nJ, 0.0);
  ctx->dE.assign(ctx->nJ, 0.0);
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    double ang = 0;
    for (int ci = 0; ci < ctx->ncoef; ++ci) {
      if (ctx->coef_of[ci] / 4096 != iJ) continue;
      const double* cf = &ctx->coef[(size_t)ci * kCoefRows * ng];
      const int om = ctx->coef_of[ci] % 4096;
      for (int i = 0; i < ng - om; ++i) {
        const double g = std::min(ctx->fR[0], cf[4 * ng + i]);
        const double a = std::min(cf[i] * ctx->fr[0], erot) + g * cf[ng + i];
        ang = std::max(ang, a + std::fabs(g * cf[2 * ng + i]) + std::fabs(g * cf[3 * ng + i]));
      }
    }
    const double emax = vmax + radmax + ang, emin = vmin;
    ctx->E0[iJ] = 0.5 * (emax + emin);
    ctx->dE[iJ] = 1.0001 * 0.5 * (emax - emin);
  }
  // device tables
  int st;
  std::vector<double> Tall, Ttall;
  for (auto& Tm : ctx->T) {
    Tall.insert(Tall.end(), Tm.begin(), Tm.end());
    for (int a = 0; a < ng; ++a)
      for (int b = 0; b < ng; ++b) Ttall.push_back(Tm[(size_t)b * ng + a]);
  }
  if ((st = upload_real(ctx, "T", Tall))) return st;
  if ((st = upload_real(ctx, "Tt", Ttall))) return st;
  // tensor-core operands: T^Omega and its transpose, padded to kp x kp, split into a
  // TF32-rounded high part and the exact FP32 remainder
  ctx->kp = ((ng + 15) / 16) * 16;
  ctx->kh = angular_tc3_kh(ng, ctx->nelec);
  ctx->kh4 = angular_tc4_kh(ng, ctx->nelec);
  // (16-byte asynchronous copies of tile rows need ncol % 4 == 0)
  ctx->tc_ok = (ctx->precision == MW3_MIXED) && (ctx->kp <= kTcMaxKp || ctx->kh4 > 0) &&
               (ctx->ncol + 127) / 128 <= 65535 && ctx->ncol % 4 == 0;
  ctx->tune.use_tc = (ctx->tc_ok && ctx->tc_user != 0) ? 1 : 0;
  if (ctx->tc_ok) {
    const int kp = ctx->kp;
    const size_t nom = ctx->T.size();
    std::vector<float> th(nom * kp * kp, 0.f), tl(th.size(), 0.f), tth(th.size(), 0.f),
        ttl(th.size(), 0.f);
    auto split = [](double v, float& hi, float& lo) {
      const float x = (float)v;
      uint32_t u;
      std::memcpy(&u, &x, 4);
      u = (u + 0x1000u) & 0xFFFFE000u;  // round to nearest (ties away) at 10 mantissa bits
      std::memcpy(&hi, &u, 4);
      lo = x - hi;
    };
    for (size_t om = 0; om < nom; ++om)
      for (int i = 0; i < ng; ++i)
        for (int n = 0; n < ng; ++n) {
          const double v = ctx->T[om][(size_t)i * ng + n];
          split(v, th[(om * kp + i) * kp + n], tl[(om * kp + i) * kp + n]);
          split(v, tth[(om * kp + n) * kp + i], ttl[(om * kp + n) * kp + i]);
        }
    if ((st = upload_raw(ctx, "T_hi", th)) || (st = upload_raw(ctx, "T_lo", tl)) ||
        (st = upload_raw(ctx, "Tt_hi", tth)) || (st = upload_raw(ctx, "Tt_lo", ttl)))
      return st;
    // parity-split operands (n_gamma even): with h = n_gamma / 2, n < h, e/o = even/odd row
    //   G1e[n][e] = T[2e][n], G1o[n][o] = T[2o+1][n], G2e[e][n] = T[2e][n], G2o[o][n] = T[2o+1][n]
    const int khp = ctx->kh > 0 ? ctx->kh : ctx->kh4;
    if (khp > 0) {
      const int kh = khp, h = ng / 2;
      std::vector<float> ph(nom * 4 * kh * kh, 0.f), pl(ph.size(), 0.f);
      for (size_t om = 0; om < nom; ++om)
        for (int r = 0; r < kh; ++r)
          for (int n = 0; n < h; ++n)
            for (int par = 0; par < 2; ++par) {
              const int i = 2 * r + par;
              if (i >= ng) continue;
              const double v = ctx->T[om][(size_t)i * ng + n];
              const size_t g1 = ((om * 4 + par) * kh + n) * kh + r;       // G1e / G1o
              const size_t g2 = ((om * 4 + 2 + par) * kh + r) * kh + n;   // G2e / G2o
              split(v, ph[g1], pl[g1]);
              split(v, ph[g2], pl[g2]);
            }
      if ((st = upload_raw(ctx, "Tp_hi", ph)) || (st = upload_raw(ctx, "Tp_lo", pl))) return st;
    }
    std::vector<int> gb(ctx->nJ + 1);
    for (int iJ = 0; iJ <= ctx->nJ; ++iJ) gb[iJ] = (int)(ctx->J_first_block[iJ] / ctx->nelec);
    if ((st = upload_raw(ctx, "g_begin", gb))) return st;
    const long ntiles = (ctx->ncol + 127) / 128;
    if ((st = dalloc(ctx, "npart", (size_t)(ctx->nblk / ctx->nelec) * ntiles * 8))) return st;
    if ((st = dalloc(ctx, "tc_err", 16)) || (st = dzero(ctx, "tc_err"))) return st;
  }
  if ((st = upload_real(ctx, "coef", ctx->coef))) return st;
  if ((st = upload_real(ctx, "fR", ctx->fR))) return st;
  if ((st = upload_real(ctx, "fr", ctx->fr))) return st;
  if ((st = upload_real(ctx, "V", ctx->V))) return st;
  {
    std::vector<double> lr(ctx->NR + 1), lrr(ctx->nr + 1);
    for (int j = 0; j <= ctx->NR; ++j) lr[j] = ctx->lamR[j] / ctx->NR;   // 1/N of the inverse FFT
    for (int j = 0; j <= ctx->nr; ++j) lrr[j] = ctx->lamr[j] / ctx->nr;
    if ((st = upload_real(ctx, "lamR", lr))) return st;
    if ((st = upload_real(ctx, "lamr", lrr))) return st;
  }
  if ((st = upload_fft_tables(ctx, "twR", "phR", ctx->NR))) return st;
  if ((st = upload_fft_tables(ctx, "twr", "phr", ctx->nr))) return st;
  std::vector<DevJ> dj(ctx->nJ);
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    const double e0s = ctx->E0[iJ] / ctx->dE[iJ], invdE = 1.0 / ctx->dE[iJ];
    dj[iJ] = DevJ{e0s, invdE, (float)e0s, (float)invdE};
  }
  if ((st = upload_raw(ctx, "dj", dj))) return st;
  if ((st = upload_raw(ctx, "blocks", ctx->blocks))) return st;
  std::vector<long> jb(ctx->nJ + 1);
  for (int iJ = 0; iJ <= ctx->nJ; ++iJ) jb[iJ] = ctx->J_first_block[iJ] * ctx->npts;
  if ((st = upload_raw(ctx, "J_begin", jb))) return st;
  // default: no absorption
  ctx->DR.assign(ctx->NR, 1.0);
  ctx->Dr.assign(ctx->nr, 1.0);
  if ((st = upload_real(ctx, "DR", ctx->DR))) return st;
  if ((st = upload_real(ctx, "Dr", ctx->Dr))) return st;
  // state buffers
  const size_t vb = (size_t)ctx->nblk * ctx->npts * ctx->rs();
  if ((st = dalloc(ctx, "q0", vb)) || (st = dalloc(ctx, "q1", vb)) || (st = dalloc(ctx, "t", vb)) ||
      (st = dalloc(ctx, "u", vb)))
    return st;
  if ((st = dzero(ctx, "q0")) || (st = dzero(ctx, "q1"))) return st;
  ctx->stage = 2;
  return MW3_OK;
}

int mw3_load_potential(mw3_ctx* ctx, mw3_pot_fn fn, void* user, double vcut, double tcut,
                       double erot) {
  if (!ctx || !fn) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 1) return ctx->fail(MW3_ERR_STATE, "mw3_grid first");
  if (!(vcut > 0) || !(tcut > 0) || !(erot > 0))
    return ctx->fail(MW3_ERR_BAD_ARG, "caps must be positive");
  const int ne = ctx->nelec;
  const long np = ctx->npts;
  ctx->V.assign((size_t)ne * ne * np, 0.0);
  ctx->pot_fn = fn;
  ctx->pot_user = user;
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<int> bad(nth, 0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t) {
    th.emplace_back([&, t]() {
      std::vector<double> pm((size_t)ne * ne);
      for (int n = (int)t; n < ctx->ng; n += (int)nth)
        for (int kr = 0; kr < ctx->nr; ++kr)
          for (int mm = 0; mm < ctx->NR; ++mm) {
            if (fn(ctx->r[kr], ctx->R[mm], ctx->x[n], pm.data(), user) != 0) {
              bad[t] = 1;
              return;
            }
            const long off = (long)n * ctx->ncol + (long)kr * ctx->NR + mm;
            for (int a = 0; a < ne * ne; ++a) ctx->V[(size_t)a * np + off] = pm[a];
          }
    });
  }
  for (auto& tt : th) tt.join();
  for (int b : bad)
    if (b) return ctx->fail(MW3_ERR_BAD_ARG, "potential callback returned an error");
  return finish_potential(ctx, vcut, tcut, erot);
}

int mw3_load_potential_grid(mw3_ctx* ctx, const double* V, double vcut, double tcut, double erot) {
  if (!ctx || !V) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 1) return ctx->fail(MW3_ERR_STATE, "mw3_grid first");
  const size_t n = (size_t)ctx->nelec * ctx->nelec * ctx->npts;
  ctx->V.assign(V, V + n);
  ctx->pot_fn = nullptr;
  ctx->pot_user = nullptr;
  return finish_potential(ctx, vcut, tcut, erot);
}

int mw3_init_packet(mw3_ctx* ctx, const mw3_packet_desc* d) {
  if (ctx) ctx->a2_cache.clear();
  if (!ctx || !d) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (d->v0 < 0 || d->j0 < d->omega0 || d->omega0 < 0 || d->elec0 < 0 || d->elec0 >= ctx->nelec ||
      !(d->Gamma > 0) || !(d->Ecol > 0) || d->j0 >= ctx->ng || d->v0 >= ctx->nr)
    return ctx->fail(MW3_ERR_BAD_ARG, "invalid packet description");
  ctx->packet = *d;
  std::vector<double> E, chi;
  int st = diatomic(ctx, d->j0, d->elec0, d->v0 + 1, E, chi);
  if (st) return st;
  ctx->Ev0j0 = E[d->v0];
  const double k0 = std::sqrt(2.0 * ctx->mu * d->Ecol);
  std::vector<double> g(ctx->NR);
  double gn = 0;
  for (int i = 0; i < ctx->NR; ++i) {
    const double dx = ctx->R[i] - d->R0;
    g[i] = std::exp(-dx * dx / (2.0 * d->Gamma * d->Gamma)) * std::cos(k0 * ctx->R[i]);
    gn += g[i] * g[i];
  }
  gn = 1.0 / std::sqrt(gn);
  ctx->g_tilde.resize(ctx->NR);
  for (int i = 0; i < ctx->NR; ++i) {
    g[i] *= gn;
    ctx->g_tilde[i] = g[i] / std::sqrt(ctx->dR);
  }
  // FBR coefficients of q_0: one angular function (j0, Omega0) times chi g
  ctx->q0.assign((size_t)ctx->nblk * ctx->npts, 0.0);
  for (int bi = 0; bi < ctx->nblk; ++bi) {
    const DevBlock& b = ctx->blocks[bi];
    if (b.omega != d->omega0 || b.lam != d->elec0) continue;
    const int i0 = d->j0 - d->omega0;
    for (int kr = 0; kr < ctx->nr; ++kr)
      for (int mm = 0; mm < ctx->NR; ++mm)
        ctx->q0[(size_t)bi * ctx->npts + (size_t)i0 * ctx->ncol + (size_t)kr * ctx->NR + mm] =
            chi[(size_t)d->v0 * ctx->nr + kr] * g[mm];
  }
  ctx->norm0 = 1.0;
  ctx->pcb_on = false;
  if ((st = upload_state_fbr(ctx, ctx->q0.data()))) return st;
  return reset_after_packet(ctx);
}

int mw3_init_packet_pcb(mw3_ctx* ctx, const mw3_packet_desc* d, const mw3_pcb_desc* s) {
  if (ctx) ctx->a2_cache.clear();
  if (!ctx || !d || !s) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (s->arrangement < 0 || s->arrangement > 2 || s->nr < 4 || s->nr > 4096 || !(s->rmin > 0) ||
      !(s->rmax > s->rmin))
    return ctx->fail(MW3_ERR_BAD_ARG, "invalid PCB description");
  if (d->v0 < 0 || d->j0 < d->omega0 || d->omega0 < 0 || d->elec0 < 0 || d->elec0 >= ctx->nelec ||
      !(d->Gamma > 0) || !(d->Ecol > 0) || d->v0 >= s->nr)
    return ctx->fail(MW3_ERR_BAD_ARG, "invalid packet description");
  for (int iJ = 0; iJ < ctx->nJ; ++iJ)
    if (d->omega0 > ctx->omtop[iJ])
      return ctx->fail(MW3_ERR_BAD_ARG, "Omega0 must be a helicity block of every J");
  if (!ctx->pot_fn) return ctx->fail(MW3_ERR_BAD_ARG, "the packet diatom needs a potential callback");
  const double masses[3] = {ctx->mA, ctx->mB, ctx->mC};
  double M[2][2] = {{1.0, 0.0}, {0.0, 1.0}};
  double mu_s = ctx->mu, m_s = ctx->m;
  if (s->arrangement > 0) {
    product_jacobi_matrix(masses, s->arrangement, M);
    product_masses(masses, s->arrangement, &mu_s, &m_s);
  }
  const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  const double Mi[2][2] = {{M[1][1] / det, -M[0][1] / det}, {-M[1][0] / det, M[0][0] / det}};
  // the packet diatom on its sine DVR, the third atom 100 bohr away on its axis
  const int ns = s->nr;
  const double Ls = s->rmax - s->rmin, drs = Ls / ns;
  std::vector<double> Hd((size_t)ns * ns, 0.0), lam(ns + 1, 0.0), pm((size_t)ctx->nelec * ctx->nelec);
  for (int j = 1; j <= ns; ++j) {
    const double k = j * M_PI / Ls;
    lam[j] = std::min(k * k / (2.0 * m_s), ctx->tcut);
  }
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      double t = 0;
      for (int j = 1; j <= ns; ++j) t += dst2(ns, j, a + 1) * lam[j] * dst2(ns, j, b + 1);
      Hd[(size_t)a * ns + b] = t;
    }
  const int L0 = d->elec0, j0 = d->j0;
  for (int a = 0; a < ns; ++a) {
    const double x = s->rmin + (a + 0.5) * drs;
    // packet vectors (r_s, R_s) along z -> the grid's (r, R)
    const double rz = Mi[0][0] * x + Mi[0][1] * 100.0, Rz = Mi[1][0] * x + Mi[1][1] * 100.0;
    const double r = std::fabs(rz), R = std::fabs(Rz), cg = (rz * Rz) / (r * R);
    if (ctx->pot_fn(r, R, cg, pm.data(), ctx->pot_user) != 0)
      return ctx->fail(MW3_ERR_BAD_ARG, "potential callback failed");
    Hd[(size_t)a * ns + a] += std::min(pm[(size_t)L0 * ctx->nelec + L0], ctx->vcut) +
                              std::min(j0 * (j0 + 1.0) / (2.0 * m_s * x * x), ctx->erot);
  }
  std::vector<double> ev, Z;
  symmetric_eigen(ns, Hd, ev, Z);
  std::vector<double> vec(ns);
  int imax = 0;
  for (int a = 0; a < ns; ++a) {
    vec[a] = Z[(size_t)a * ns + d->v0];
    if (std::fabs(vec[a]) > std::fabs(vec[imax])) imax = a;
  }
  if (vec[imax] < 0)
    for (double& v : vec) v = -v;
  // chi(r_s) = sum_j s_j (S vec)_j sqrt(2/L) sin(j pi (r_s - rmin) / L), s_N = 1/sqrt(2)
  std::vector<double> coef(ns);
  for (int j = 1; j <= ns; ++j) {
    double a = 0;
    for (int i = 1; i <= ns; ++i) a += dst2(ns, j, i) * vec[i - 1];
    coef[j - 1] = a * (j == ns ? 1.0 / std::sqrt(2.0) : 1.0) * std::sqrt(2.0 / Ls);
  }
  ctx->packet = *d;
  ctx->Ev0j0 = ev[d->v0];
  const double k0 = std::sqrt(2.0 * mu_s * d->Ecol);
  const double G = d->Gamma;
  ctx->pcb_on = true;
  ctx->pcb_mu = mu_s;
  ctx->pcb_R0 = d->R0;
  ctx->pcb_G = G;
  ctx->pcb_k0 = k0;
  ctx->pcb_N = 1.0 / std::sqrt(std::sqrt(M_PI) * G / 2.0 *
                               (1.0 + std::exp(-k0 * k0 * G * G) * std::cos(2.0 * k0 * d->R0)));
  ctx->q0.clear();
  ctx->norm0 = 1.0;
  if (ctx->host_only) return reset_after_packet(ctx);
  // output blocks (J, Omega, Lambda0) and their helicity-transform terms
  std::vector<PcbTerm> terms;
  const int om0 = d->omega0;
  const double s0 = std::sqrt(2.0);
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    const int J = ctx->J[iJ];
    for (int om = 0; om <= ctx->omtop[iJ]; ++om) {
      PcbTerm t{};
      t.blk = (int)(ctx->J_first_block[iJ] + (long)om * ctx->nelec + L0);
      t.om = om;
      // T[Omega][Omega0] = [s(Omega0) d(Omega0, Omega) + (Omega0 > 0)(-1)^Omega0 d(-Omega0, Omega)]
      //                    / s(Omega), s(0) = sqrt(2), s(>0) = 1
      const double so = om == 0 ? s0 : 1.0;
      t.w1 = wigner_index(J, om0, om);
      t.p1 = (om0 == 0 ? s0 : 1.0) / so * wigner_prefactor(J, t.w1);
      t.w2 = wigner_index(J, -om0, om);
      t.p2 = om0 > 0 ? ((om0 & 1) ? -1.0 : 1.0) / so * wigner_prefactor(J, t.w2) : 0.0;
      terms.push_back(t);
    }
  }
  PcbParams p{};
  p.M00 = M[0][0];
  p.M01 = M[0][1];
  p.M10 = M[1][0];
  p.M11 = M[1][1];
  p.R0 = d->R0;
  p.G = G;
  p.k0 = k0;
  p.N = ctx->pcb_N;
  p.rsmin = s->rmin;
  p.rsmax = s->rmax;
  p.nrs = ns;
  p.j0 = j0;
  p.om0 = om0;
  p.NR = ctx->NR;
  p.nr = ctx->nr;
  p.ng = ctx->ng;
  p.Rmin = ctx->Rmin;
  p.dR = ctx->dR;
  p.rmin = ctx->rmin;
  p.dr = ctx->dr;
  p.plc = 1.0 / std::sqrt(2.0);
  for (int mm = 1; mm <= om0; ++mm) p.plc *= -std::sqrt((2.0 * mm + 1.0) / (2.0 * mm));
  std::vector<double> xw(ctx->x);
  xw.insert(xw.end(), ctx->w.begin(), ctx->w.end());
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  const bool mixed = ctx->precision != MW3_FP64;
  int st;
  if ((st = upload_raw(ctx, "pcb_xw", xw)) || (st = upload_raw(ctx, "pcb_coef", coef)) ||
      (st = upload_raw(ctx, "pcb_terms", terms)) || (st = dalloc(ctx, "pcb_dvr", n * 8)) ||
      (st = dzero(ctx, "pcb_dvr")))
    return st;
  // with the kernel timers on, CUDA events on the library's stream bracket the launch
  cudaEvent_t te[2] = {nullptr, nullptr};
  if (ctx->timing) {
    CK(cudaEventCreate(&te[0]));
    CK(cudaEventCreate(&te[1]));
    CK(cudaEventRecord(te[0], ctx->stream));
  }
  LK(launch_pcb_packet(p, (const double*)dptr(ctx, "pcb_xw"), (const double*)dptr(ctx, "pcb_coef"),
                       (const PcbTerm*)dptr(ctx, "pcb_terms"), (int)terms.size(),
                       (double*)dptr(ctx, "pcb_dvr"), ctx->nsm, ctx->stream));
  if (ctx->timing) {
    CK(cudaEventRecord(te[1], ctx->stream));
    CK(cudaEventSynchronize(te[1]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, te[0], te[1]));
    ctx->kms[kPcbKernel] += ms;
    ctx->klaunch[kPcbKernel] += 1;
    cudaEventDestroy(te[0]);
    cudaEventDestroy(te[1]);
  }
  const DevBlock* blk = (const DevBlock*)dptr(ctx, "blocks");
  if (!mixed) {
    LK(launch_gamma_forward<double>((const double*)dptr(ctx, "pcb_dvr"),
                                    (double*)dptr(ctx, state_name(ctx, true)),
                                    (const double*)dptr(ctx, "T"), blk, ctx->nblk, ctx->ng,
                                    ctx->ncol, ctx->stream));
  } else {
    // the FP64 FBR coefficients, rounded once to the FP32 state
    std::vector<double> Tall;
    for (auto& Tm : ctx->T) Tall.insert(Tall.end(), Tm.begin(), Tm.end());
    if ((st = upload_real(ctx, "pcb_T64", Tall, true)) || (st = dalloc(ctx, "pcb_fbr", n * 8)))
      return st;
    LK(launch_gamma_forward<double>((const double*)dptr(ctx, "pcb_dvr"),
                                    (double*)dptr(ctx, "pcb_fbr"),
                                    (const double*)dptr(ctx, "pcb_T64"), blk, ctx->nblk, ctx->ng,
                                    ctx->ncol, ctx->stream));
    LK(launch_convert_d2f((const double*)dptr(ctx, "pcb_fbr"),
                          (float*)dptr(ctx, state_name(ctx, true)), (long)n, ctx->stream));
  }
  CK(cudaMemsetAsync(dptr(ctx, state_name(ctx, false)), 0, n * ctx->rs(), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (const char* b : {"pcb_dvr", "pcb_fbr", "pcb_T64", "pcb_xw", "pcb_coef", "pcb_terms"})
    dfree(ctx, b);
  return reset_after_packet(ctx);
}

int mw3_set_absorber(mw3_ctx* ctx, double RI, double AR, int nR, double rI, double Ar, int nrx) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (AR < 0 || Ar < 0 || nR < 1 || nrx < 1) return ctx->fail(MW3_ERR_BAD_ARG, "invalid absorber");
  for (int i = 0; i < ctx->NR; ++i)
    ctx->DR[i] = ctx->R[i] > RI ? std::exp(-AR * std::pow(ctx->R[i] - RI, nR)) : 1.0;
  for (int i = 0; i < ctx->nr; ++i)
    ctx->Dr[i] = ctx->r[i] > rI ? std::exp(-Ar * std::pow(ctx->r[i] - rI, nrx)) : 1.0;
  int st;
  if ((st = upload_real(ctx, "DR", ctx->DR)) || (st = upload_real(ctx, "Dr", ctx->Dr))) return st;
  if (ctx->stage == 3) ctx->stage = 4;
  return MW3_OK;
}

int mw3_set_products(mw3_ctx* ctx, const mw3_products_desc* d) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 3) return ctx->fail(MW3_ERR_STATE, "mw3_init_packet first");
  if (ctx->stage >= 5) return ctx->fail(MW3_ERR_STATE, "set products before mw3_set_analysis");
  ctx->prod_on = false;
  if (!d) return MW3_OK;
  if ((d->arrangement != 1 && d->arrangement != 2) || !(d->Rinf > 0) || d->nr < 4 ||
      !(d->rmin > 0) || !(d->rmax > d->rmin) || d->ngamma < 1 || d->vmax < 0 || d->jmax < 0 ||
      d->vmax >= d->nr)
    return ctx->fail(MW3_ERR_BAD_ARG, "invalid products description");
  if (!ctx->pot_fn)
    return ctx->fail(MW3_ERR_BAD_ARG, "product channels need a potential callback");
  const double masses[3] = {ctx->mA, ctx->mB, ctx->mC};
  product_masses(masses, d->arrangement, &ctx->mu_p, &ctx->m_p);
  const int nrp = d->nr, ngp = d->ngamma, nn = nrp * ngp, ng = ctx->ng;
  const double drp = (d->rmax - d->rmin) / nrp;
  std::vector<double> rp(nrp), xg, wg;
  for (int a = 0; a < nrp; ++a) rp[a] = d->rmin + (a + 0.5) * drp;
  gauss_legendre(ngp, xg, wg);
  // nodes: reactant point, 4-point stencils, Jacobian, frame rotation
  std::vector<double> cosg(nn), beta(nn);
  std::vector<int> sa(nn), sc(nn);
  ctx->prod_idx.assign((size_t)nn * 8, 0);
  ctx->prod_w.assign((size_t)nn * 8, 0.0);
  ctx->prod_jac.assign(nn, 0.0);
  auto stencil = [](double x0, double dx, int n, double x, int* id, double* w, double scale) {
    const double t = (x - x0) / dx;
    const int m0 = (int)std::floor(t) - 1;
    const double u = t - m0;
    const double L[4] = {-(u - 1) * (u - 2) * (u - 3) / 6.0, u * (u - 2) * (u - 3) / 2.0,
                         -u * (u - 1) * (u - 3) / 2.0, u * (u - 1) * (u - 2) / 6.0};
    for (int a = 0; a < 4; ++a) {
      const int m = m0 + a;
      const bool in = m >= 0 && m < n;
      id[a] = in ? m : 0;
      w[a] = in ? L[a] * scale : 0.0;
    }
  };
  for (int a = 0; a < nrp; ++a)
    for (int l = 0; l < ngp; ++l) {
      const int v = a * ngp + l;
      double R, r;
      product_point(masses, d->arrangement, d->Rinf, rp[a], xg[l], &R, &r, &cosg[v], &beta[v],
                    &sa[v], &sc[v]);
      if (!(R >= ctx->Rmin && R <= ctx->Rmax && r >= ctx->rmin && r <= ctx->rmax))
        return ctx->fail(MW3_ERR_BAD_ARG, "a product quadrature node lies outside the grid");
      stencil(ctx->R[0], ctx->dR, ctx->NR, R, &ctx->prod_idx[(size_t)v * 8],
              &ctx->prod_w[(size_t)v * 8], 1.0 / std::sqrt(ctx->dR * ctx->dr));
      stencil(ctx->r[0], ctx->dr, ctx->nr, r, &ctx->prod_idx[(size_t)v * 8 + 4],
              &ctx->prod_w[(size_t)v * 8 + 4], 1.0);
      ctx->prod_jac[v] = rp[a] * d->Rinf / (r * R);
    }
  {   // plane-major form: the distinct stencil columns, sorted, and each node's rows in them
    std::vector<int> cols((size_t)nn * 16);
    for (int v = 0; v < nn; ++v)
      for (int c = 0; c < 4; ++c)
        for (int a = 0; a < 4; ++a)
          cols[(size_t)v * 16 + 4 * c + a] =
              ctx->prod_idx[(size_t)v * 8 + 4 + c] * ctx->NR + ctx->prod_idx[(size_t)v * 8 + a];
    std::vector<int> u(cols);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    ctx->prod_npts = (int)u.size();
    ctx->prod_spad = (ctx->prod_npts + 31) / 32 * 32;
    ctx->prod_ngp = (ng + 31) / 32 * 32;
    ctx->prod_pts = u;
    ctx->prod_pts.resize(ctx->prod_spad, u.back());
    ctx->prod_pix.resize((size_t)nn * 16);
    ctx->prod_wst.resize((size_t)nn * 16);
    for (int v = 0; v < nn; ++v)
      for (int c = 0; c < 4; ++c)
        for (int a = 0; a < 4; ++a) {
          const size_t k = (size_t)v * 16 + 4 * c + a;
          ctx->prod_pix[k] = (int)(std::lower_bound(u.begin(), u.end(), cols[k]) - u.begin());
          ctx->prod_wst[k] = ctx->prod_w[(size_t)v * 8 + a] * ctx->prod_w[(size_t)v * 8 + 4 + c];
        }
  }
  // Legendre rows of every helicity at the nodes' reactant angles
  int ltop = 0;
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) ltop = std::max(ltop, ctx->omtop[iJ] + 1);
  ctx->prod_ltop = ltop;
  ctx->prod_pl.assign((size_t)nn * ltop * ng, 0.0);
  for (int om = 0; om < ltop && om < ng; ++om) {
    std::vector<double> P;
    norm_assoc_legendre(ng - 1, om, cosg, P);
    for (int v = 0; v < nn; ++v)
      for (int i = 0; i < ng - om; ++i)
        ctx->prod_pl[((size_t)v * ltop + om) * ng + i] = P[(size_t)i * nn + v];
  }
  // helicity transforms per J and node
  ctx->prod_T.clear();
  std::vector<long> toff(ctx->nJ);
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    toff[iJ] = (long)ctx->prod_T.size();
    const int nom = ctx->omtop[iJ] + 1;
    std::vector<double> Tm;
    for (int v = 0; v < nn; ++v) {
      helicity_transform(ctx->J[iJ], nom, beta[v], sa[v], sc[v], Tm);
      ctx->prod_T.insert(ctx->prod_T.end(), Tm.begin(), Tm.end());
    }
  }
  // product diatomic states on the r' sine DVR (departing atom 100 bohr away, collinear)
  const int nv = d->vmax + 1, ne = ctx->nelec;
  std::vector<double> lam(nrp + 1, 0.0);
  for (int jj = 1; jj <= nrp; ++jj) {
    const double k = jj * M_PI / (d->rmax - d->rmin);
    lam[jj] = std::min(k * k / (2.0 * ctx->m_p), ctx->tcut);
  }
  std::vector<double> Tk((size_t)nrp * nrp, 0.0), Vd((size_t)ne * nrp), pm((size_t)ne * ne);
  for (int a = 0; a < nrp; ++a)
    for (int b = 0; b < nrp; ++b) {
      double s = 0;
      for (int jj = 1; jj <= nrp; ++jj) s += dst2(nrp, jj, a + 1) * lam[jj] * dst2(nrp, jj, b + 1);
      Tk[(size_t)a * nrp + b] = s;
    }
  for (int a = 0; a < nrp; ++a) {
    double R, r, cg, bb;
    int s1, s2;
    product_point(masses, d->arrangement, 100.0, rp[a], 1.0, &R, &r, &cg, &bb, &s1, &s2);
    if (ctx->pot_fn(r, R, cg, pm.data(), ctx->pot_user) != 0)
      return ctx->fail(MW3_ERR_BAD_ARG, "potential callback failed");
    for (int L = 0; L < ne; ++L) Vd[(size_t)L * nrp + a] = std::min(pm[(size_t)L * ne + L], ctx->vcut);
  }
  std::vector<std::vector<double>> chi((size_t)ne * (d->jmax + 1)), eps((size_t)ne * (d->jmax + 1));
  for (int L = 0; L < ne; ++L)
    for (int j = 0; j <= d->jmax; ++j) {
      std::vector<double> H = Tk, ev, Z;
      for (int a = 0; a < nrp; ++a)
        H[(size_t)a * nrp + a] += Vd[(size_t)L * nrp + a] +
                                  std::min(j * (j + 1.0) / (2.0 * ctx->m_p * rp[a] * rp[a]), ctx->erot);
      symmetric_eigen(nrp, H, ev, Z);
      auto& c = chi[(size_t)L * (d->jmax + 1) + j];
      c.assign((size_t)nv * nrp, 0.0);
      for (int v = 0; v < nv; ++v) {
        int imax = 0;
        for (int a = 0; a < nrp; ++a)
          if (std::fabs(Z[(size_t)a * nrp + v]) > std::fabs(Z[(size_t)imax * nrp + v])) imax = a;
        const double sg = Z[(size_t)imax * nrp + v] < 0 ? -1.0 : 1.0;
        for (int a = 0; a < nrp; ++a) c[(size_t)v * nrp + a] = sg * Z[(size_t)a * nrp + v];
      }
      eps[(size_t)L * (d->jmax + 1) + j].assign(ev.begin(), ev.begin() + nv);
    }
  // channels, grouped by (J, Lambda', Omega'), and their quadrature weights
  ctx->prod_groups.clear();
  ctx->prod_W.clear();
  ctx->pch_L.clear();
  ctx->pch_v.clear();
  ctx->pch_j.clear();
  ctx->pch_op.clear();
  ctx->pch_eps.clear();
  ctx->prod_first.assign(ctx->nJ + 1, 0);
  ctx->prod_jl.assign((size_t)ctx->nJ * ne, 0);
  ctx->prod_max_nom = 0;
  long nch = 0;
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    ctx->prod_first[iJ] = nch;
    const int nom = ctx->omtop[iJ] + 1;
    if (nom > 32) return ctx->fail(MW3_ERR_BAD_ARG, "product channels support at most 32 helicities");
    ctx->prod_max_nom = std::max(ctx->prod_max_nom, nom);
    for (int L = 0; L < ne; ++L) {
      ctx->prod_jl[(size_t)iJ * ne + L] = (int)ctx->prod_groups.size();
      for (int op = 0; op < nom; ++op) {
        std::vector<double> Pp;
        if (op <= d->jmax) norm_assoc_legendre(d->jmax, op, xg, Pp);   // (no channels above jmax)
        ProdGroup g{};
        g.b0 = (int)ctx->J_first_block[iJ] + L;
        g.bstride = ne;
        g.nom = nom;
        g.op = op;
        g.toff = toff[iJ];
        g.c0 = (int)nch;
        for (int j = op; j <= d->jmax; ++j)
          for (int v = 0; v < nv; ++v) {
            const auto& c = chi[(size_t)L * (d->jmax + 1) + j];
            for (int a = 0; a < nrp; ++a)
              for (int l = 0; l < ngp; ++l)
                ctx->prod_W.push_back(drp * wg[l] * c[(size_t)v * nrp + a] / std::sqrt(drp) *
                                      Pp[(size_t)(j - op) * ngp + l]);
            ctx->pch_L.push_back(L);
            ctx->pch_v.push_back(v);
            ctx->pch_j.push_back(j);
            ctx->pch_op.push_back(op);
            ctx->pch_eps.push_back(eps[(size_t)L * (d->jmax + 1) + j][v]);
            ++nch;
          }
        g.nc = (int)(nch - g.c0);
        ctx->prod_groups.push_back(g);
      }
    }
  }
  ctx->prod_first[ctx->nJ] = nch;
  ctx->prod_nn = nn;
  ctx->prod = *d;
  ctx->prod_on = true;
  return MW3_OK;
}

int mw3_set_analysis(mw3_ctx* ctx, const mw3_analysis_desc* d) {
  if (ctx) ctx->a2_cache.clear();
  if (!ctx || !d) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 3) return ctx->fail(MW3_ERR_STATE, "mw3_init_packet first");
  if (d->nE < 1 || !(d->E_hi >= d->E_lo) || !(d->E_lo > 0) || d->rstar <= ctx->rmin ||
      d->rstar >= ctx->rmax || d->kmin < 0)
    return ctx->fail(MW3_ERR_BAD_ARG, "invalid analysis description");
  ctx->an = *d;
  const int nE = d->nE;
  ctx->Ecol.resize(nE);
  for (int e = 0; e < nE; ++e)
    ctx->Ecol[e] = (nE == 1) ? d->E_lo : d->E_lo + (d->E_hi - d->E_lo) * e / (nE - 1.0);
  ctx->theta.assign((size_t)ctx->nJ * nE, 0.0);
  for (int iJ = 0; iJ < ctx->nJ; ++iJ)
    for (int e = 0; e < nE; ++e) {
      const double Es = (ctx->Ecol[e] + ctx->Ev0j0 - ctx->E0[iJ]) / ctx->dE[iJ];
      if (!(Es > -1.0 && Es < 1.0)) return ctx->fail(MW3_ERR_SPECTRUM, "energy outside (E_min, E_max)");
      ctx->theta[(size_t)iJ * nE + e] = std::acos(Es);
    }
  sine_interpolation_weights(ctx->rmin, ctx->rmax, ctx->nr, d->rstar, ctx->wpsi, ctx->wdpsi);
  int mi = 0;
  for (int i = 0; i < ctx->NR; ++i)
    if (std::fabs(ctx->R[i] - d->Rinf) < std::fabs(ctx->R[mi] - d->Rinf)) mi = i;
  ctx->m_inf = mi;

  // channels and the column layout of the cut ring, per J
  ctx->chan_block.clear();
  ctx->chan_row.clear();
  ctx->chan_col.clear();
  ctx->chan_v.clear();
  ctx->chan_j.clear();
  ctx->chan_om.clear();
  ctx->chan_lam.clear();
  ctx->chan_iJ.clear();
  ctx->chan_eps.clear();
  std::vector<double> P;
  std::map<std::pair<int, int>, std::pair<std::vector<double>, std::vector<double>>> cache;
  const int ng = ctx->ng, nr = ctx->nr;
  ctx->colbase.assign(ctx->nJ, 0);
  ctx->ncols.assign(ctx->nJ, 0);
  ctx->ncut.assign(ctx->nJ, 0);
  ctx->accoff.assign(ctx->nJ, 0);
  ctx->colbase_c.assign(ctx->nJ, 0);
  ctx->ncols_c.assign(ctx->nJ, 0);
  ctx->accoff_c.assign(ctx->nJ, 0);
  long col = 0, acc = 0, maxc = 0, colc = 0, accc = 0, maxcc = 0;
  for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
    const long b0 = ctx->J_first_block[iJ], b1 = ctx->J_first_block[iJ + 1];
    const long nc = (b1 - b0) * ng * ctx->NR;
    ctx->colbase[iJ] = col;
    ctx->colbase_c[iJ] = colc;
    ctx->ncut[iJ] = nc;
    for (long b = b0; b < b1; ++b) ctx->blocks[b].cutcol = (int)(col + (b - b0) * ng * ctx->NR);
    long nch = 0;
    if (d->vmax >= 0) {
      for (long b = b0; b < b1; ++b) {
        const DevBlock& B = ctx->blocks[b];
        for (int j = B.omega; j <= std::min(d->jmax, ng - 1); ++j) {
          auto key = std::make_pair(j, B.lam);
          if (!cache.count(key)) {
            std::vector<double> E, chi;
            int st = diatomic(ctx, j, B.lam, d->vmax + 1, E, chi);
            if (st) return st;
            cache[key] = {E, chi};
          }
          auto& ec = cache[key];
          for (int v = 0; v <= d->vmax; ++v) {
            ctx->chan_block.push_back((int)b);
            ctx->chan_col.push_back((int)(colc + nch));
            ctx->chan_v.push_back(v);
            ctx->chan_j.push_back(j);
            ctx->chan_om.push_back(B.omega);
            ctx->chan_lam.push_back(B.lam);
            ctx->chan_iJ.push_back(iJ);
            ctx->chan_eps.push_back(ec.first[v]);
            ctx->chan_row.push_back(j - B.omega);
            for (int kr = 0; kr < nr; ++kr)
              P.push_back(ec.second[(size_t)v * nr + kr] / std::sqrt(ctx->dR));
            ++nch;
          }
        }
      }
    }
    long nchp = 0;
    if (ctx->prod_on) {
      const long p0 = ctx->prod_first[iJ];
      nchp = ctx->prod_first[iJ + 1] - p0;
      for (auto& g : ctx->prod_groups)
        if (g.c0 >= p0 && g.c0 < p0 + nchp) g.col0 = (int)(colc + nch + (g.c0 - p0));
    }
    ctx->ncols[iJ] = 2 * nc;
    ctx->accoff[iJ] = acc;
    acc += 2L * nE * ctx->ncols[iJ];
    maxc = std::max(maxc, ctx->ncols[iJ]);
    col += ((ctx->ncols[iJ] + 3) / 4) * 4;
    ctx->ncols_c[iJ] = nch + nchp;
    ctx->accoff_c[iJ] = accc;
    accc += 2L * nE * ctx->ncols_c[iJ];
    maxcc = std::max(maxcc, ctx->ncols_c[iJ]);
    colc += ((ctx->ncols_c[iJ] + 3) / 4) * 4;
  }
  ctx->nchan = (int)ctx->chan_block.size();
  ctx->NC = col;
  ctx->max_cols = maxc;
  ctx->acc_size = acc;
  ctx->NCc = colc;
  ctx->max_cols_c = maxcc;
  ctx->accc_size = accc;
  int st;
  const int kb = ctx->tune.kb;
  if ((st = upload_raw(ctx, "blocks", ctx->blocks))) return st;
  if ((st = dalloc(ctx, "cut", (size_t)kb * ctx->NC * ctx->rs())) || (st = dzero(ctx, "cut"))) return st;
  if ((st = dalloc(ctx, "acc", (size_t)acc * 8)) || (st = dzero(ctx, "acc"))) return st;
  ctx->ring_n = 0;
  ++ctx->acc_version;
  if ((st = dalloc(ctx, "ph", (size_t)ctx->nJ * 2 * nE * kb * ctx->rs()))) return st;
  // channel ring, its FP64 accumulators and (mixed form) its FP64 phase matrix
  if ((st = dalloc(ctx, "cutc", (size_t)kb * std::max(ctx->NCc, 4L) * 8)) || (st = dzero(ctx, "cutc")))
    return st;
  if ((st = dalloc(ctx, "accc", (size_t)std::max(accc, 1L) * 8)) || (st = dzero(ctx, "accc"))) return st;
  if (ctx->precision != MW3_FP64 &&
      (st = dalloc(ctx, "ph64", (size_t)ctx->nJ * 2 * nE * kb * 8)))
    return st;
  if ((st = upload_real(ctx, "theta", ctx->theta, true))) return st;
  if ((st = upload_real(ctx, "wpsi", ctx->wpsi)) || (st = upload_real(ctx, "wdpsi", ctx->wdpsi))) return st;
  if ((st = upload_raw(ctx, "colbase", ctx->colbase)) || (st = upload_raw(ctx, "ncols", ctx->ncols)) ||
      (st = upload_raw(ctx, "ncut", ctx->ncut)) || (st = upload_raw(ctx, "accoff", ctx->accoff)))
    return st;
  if ((st = upload_raw(ctx, "colbase_c", ctx->colbase_c)) ||
      (st = upload_raw(ctx, "ncols_c", ctx->ncols_c)) || (st = upload_raw(ctx, "accoff_c", ctx->accoff_c)))
    return st;
  {
    std::vector<int> nci(ctx->nJ);
    for (int i = 0; i < ctx->nJ; ++i) nci[i] = (int)ctx->ncut[i];
    if ((st = upload_raw(ctx, "ncut_i", nci))) return st;
  }
  if ((st = dalloc(ctx, "qcol", (size_t)ctx->nblk * ng * nr * ctx->rs()))) return st;
  if (ctx->nchan > 0) {
    if ((st = upload_real(ctx, "P", P, true)) || (st = upload_raw(ctx, "chan_block", ctx->chan_block)) ||
        (st = upload_raw(ctx, "chan_row", ctx->chan_row)) ||
        (st = upload_raw(ctx, "chan_col", ctx->chan_col)))
      return st;
  }
  if (ctx->prod_on) {
    ctx->prod_chan.assign(2 * (size_t)ctx->prod_first[ctx->nJ], 0);
    for (size_t gi = 0; gi < ctx->prod_groups.size(); ++gi) {
      const ProdGroup& g = ctx->prod_groups[gi];
      for (int c = 0; c < g.nc; ++c) {
        ctx->prod_chan[2 * (size_t)(g.c0 + c)] = (int)gi;
        ctx->prod_chan[2 * (size_t)(g.c0 + c) + 1] = g.col0 + c;
      }
    }
    if ((st = upload_raw(ctx, "p_jl", ctx->prod_jl)) || (st = upload_raw(ctx, "p_chan", ctx->prod_chan)))
      return st;
    // the projection runs in FP64 in both precisions: only the Legendre rows, which multiply
    // the state inside the blocked partial sums, take the state's precision
    if ((st = upload_raw(ctx, "p_idx", ctx->prod_idx)) ||
        (st = upload_real(ctx, "p_w", ctx->prod_w, true)) ||
        (st = upload_real(ctx, "p_pl", ctx->prod_pl)) || (st = upload_real(ctx, "p_T", ctx->prod_T, true)) ||
        (st = upload_real(ctx, "p_jac", ctx->prod_jac, true)) ||
        (st = upload_real(ctx, "p_W", ctx->prod_W, true)) ||
        (st = upload_raw(ctx, "p_groups", ctx->prod_groups)) ||
        (st = dalloc(ctx, "p_v", ctx->prod_groups.size() * (size_t)ctx->prod_nn * 8)))
      return st;
    // plane-major form: the stencil weights wR_a wr_c in the state's precision (they multiply
    // the state in the sixteen-term stencil sums), the gathered rows of every block
    if ((st = upload_raw(ctx, "p_pts", ctx->prod_pts)) ||
        (st = upload_raw(ctx, "p_pix", ctx->prod_pix)) ||
        (st = upload_real(ctx, "p_wst", ctx->prod_wst)) ||
        (st = dalloc(ctx, "p_G", (size_t)ctx->nblk * ctx->prod_spad * ctx->prod_ngp * ctx->rs())))
      return st;
  }
  if ((st = dalloc(ctx, "d_iter", 8))) return st;
  if (!ctx->host_only) {
    long it = ctx->iter;
    CK(cudaMemcpyAsync(dptr(ctx, "d_iter"), &it, 8, cudaMemcpyHostToDevice, ctx->stream));
  }
  if ((st = dalloc(ctx, "normbuf", (size_t)kb * ctx->nJ * 8))) return st;
  if ((st = dalloc(ctx, "npartial", (size_t)ctx->nJ * 256 * 8))) return st;
  // channel-probability tables, the energy grid and dE for the device assembly
  if ((st = upload_raw(ctx, "Ecol", ctx->Ecol)) || (st = upload_raw(ctx, "dE", ctx->dE)) ||
      (st = dalloc(ctx, "a2", (size_t)nE * 8)) || (st = dalloc(ctx, "pout", 8)))
    return st;
  ctx->chan_tab_r = ChanTable{};
  ctx->chan_tab_p = ChanTable{};
  if (d->vmax >= 0) {
    std::vector<long> ccol(ctx->nchan);
    for (int c = 0; c < ctx->nchan; ++c) {
      const int iJ = ctx->chan_iJ[c];
      ccol[c] = ctx->accoff_c[iJ] + (ctx->chan_col[c] - ctx->colbase_c[iJ]);
    }
    if ((st = build_chan_table(ctx, "cr", d->vmax + 1, d->jmax + 1, ctx->mu, ctx->chan_iJ,
                               ctx->chan_lam, ctx->chan_v, ctx->chan_j, ccol, ctx->chan_eps,
                               ctx->chan_tab_r)))
      return st;
  }
  if (ctx->prod_on) {
    const long nchp = ctx->prod_first[ctx->nJ];
    std::vector<int> cJ(nchp);
    std::vector<long> ccol(nchp);
    for (int iJ = 0; iJ < ctx->nJ; ++iJ) {
      const long p0 = ctx->prod_first[iJ], np = ctx->prod_first[iJ + 1] - p0;
      const long first = ctx->ncols_c[iJ] - np;   // local column of the J's first product channel
      for (long c = 0; c < np; ++c) {
        cJ[p0 + c] = iJ;
        ccol[p0 + c] = ctx->accoff_c[iJ] + first + c;
      }
    }
    if ((st = build_chan_table(ctx, "cp", ctx->prod.vmax + 1, ctx->prod.jmax + 1, ctx->mu_p, cJ,
                               ctx->pch_L, ctx->pch_v, ctx->pch_j, ccol, ctx->pch_eps,
                               ctx->chan_tab_p)))
      return st;
  }
  for (auto& g : ctx->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (!ctx->host_only) CK(cudaStreamSynchronize(ctx->stream));
  ctx->stage = 5;
  return MW3_OK;
}

}  // extern "C"

// ============================================================ propagation
namespace {

template <typename real>
struct Bufs {
  real *q[2], *t, *u, *V, *T, *Tt, *coef, *fR, *fr, *DR, *Dr, *lamR, *lamr, *wpsi, *wdpsi, *cut,
      *qcol, *ph;
  double *P, *cutc, *ph64, *accc;
  long *colbase_c, *ncols_c, *accoff_c;
  void *twR, *phR, *twr, *phr;
  DevBlock* blocks;
  DevJ* dj;
  int *ncut_i, *chan_block, *chan_row, *chan_col;
  long *colbase, *ncols, *ncut, *accoff, *d_iter, *J_begin;
  double *acc, *theta, *normbuf, *npartial;
};

template <typename real>
Bufs<real> bufs(mw3_ctx* ctx) {
  Bufs<real> b;
  b.q[0] = (real*)dptr(ctx, "q0");
  b.q[1] = (real*)dptr(ctx, "q1");
  b.t = (real*)dptr(ctx, "t");
  b.u = (real*)dptr(ctx, "u");
  b.V = (real*)dptr(ctx, "V");
  b.T = (real*)dptr(ctx, "T");
  b.Tt = (real*)dptr(ctx, "Tt");
  b.coef = (real*)dptr(ctx, "coef");
  b.fR = (real*)dptr(ctx, "fR");
  b.fr = (real*)dptr(ctx, "fr");
  b.DR = (real*)dptr(ctx, "DR");
  b.Dr = (real*)dptr(ctx, "Dr");
  b.lamR = (real*)dptr(ctx, "lamR");
  b.lamr = (real*)dptr(ctx, "lamr");
  b.wpsi = (real*)dptr(ctx, "wpsi");
  b.wdpsi = (real*)dptr(ctx, "wdpsi");
  b.cut = (real*)dptr(ctx, "cut");
  b.qcol = (real*)dptr(ctx, "qcol");
  b.P = (double*)dptr(ctx, "P");
  b.ph = (real*)dptr(ctx, "ph");
  b.cutc = (double*)dptr(ctx, "cutc");
  // FP64 phases of the channel ring: the flux ring's own in the FP64 form
  b.ph64 = std::is_same<real, double>::value ? (double*)b.ph : (double*)dptr(ctx, "ph64");
  b.accc = (double*)dptr(ctx, "accc");
  b.colbase_c = (long*)dptr(ctx, "colbase_c");
  b.ncols_c = (long*)dptr(ctx, "ncols_c");
  b.accoff_c = (long*)dptr(ctx, "accoff_c");
  b.twR = dptr(ctx, "twR");
  b.phR = dptr(ctx, "phR");
  b.twr = dptr(ctx, "twr");
  b.phr = dptr(ctx, "phr");
  b.blocks = (DevBlock*)dptr(ctx, "blocks");
  b.dj = (DevJ*)dptr(ctx, "dj");
  b.ncut_i = (int*)dptr(ctx, "ncut_i");
  b.chan_block = (int*)dptr(ctx, "chan_block");
  b.chan_row = (int*)dptr(ctx, "chan_row");
  b.chan_col = (int*)dptr(ctx, "chan_col");
  b.colbase = (long*)dptr(ctx, "colbase");
  b.ncols = (long*)dptr(ctx, "ncols");
  b.ncut = (long*)dptr(ctx, "ncut");
  b.accoff = (long*)dptr(ctx, "accoff");
  b.d_iter = (long*)dptr(ctx, "d_iter");
  b.J_begin = (long*)dptr(ctx, "J_begin");
  b.acc = (double*)dptr(ctx, "acc");
  b.theta = (double*)dptr(ctx, "theta");
  b.normbuf = (double*)dptr(ctx, "normbuf");
  b.npartial = (double*)dptr(ctx, "npartial");
  return b;
}

struct Timer {
  mw3_ctx* ctx;
  int k;
  int idx = -1;
  Timer(mw3_ctx* c, int kk, bool enable) : ctx(c), k(kk) {
    if (!(enable && c->timing)) return;
    idx = (int)ctx->evrec.size() * 2;
    while ((int)ctx->evpool.size() < idx + 2) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ctx->evpool.push_back(e);
    }
    cudaEventRecord(ctx->evpool[idx], ctx->stream);
  }
  void stop() {
    if (idx < 0) return;
    cudaEventRecord(ctx->evpool[idx + 1], ctx->stream);
    ctx->evrec.push_back({k, idx});
    idx = -1;
  }
};

// Accumulate the recorded launch times (call after the stream is synchronised).
void collect_times(mw3_ctx* ctx) {
  for (auto& r : ctx->evrec) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->evpool[r.second], ctx->evpool[r.second + 1]);
    ctx->kms[r.first] += ms;
    ctx->klaunch[r.first] += 1;
  }
  ctx->evrec.clear();
}



// One Chebyshev iteration; cut data into ring slot `slot`. mode 1 computes H_s q
// into `hs_out` instead (no damping, no analysis).
template <typename real>
int step(mw3_ctx* ctx, int slot, bool first, bool timed, int mode = 0, real* hs_out = nullptr) {
  Bufs<real> B = bufs<real>(ctx);
  cudaStream_t st = ctx->stream;
  real* qk = B.q[ctx->cur];
  real* qkm1 = B.q[1 - ctx->cur];
  const long nrows = (long)ctx->nblk * ctx->ng * ctx->nr;
  const bool analysis = (mode == 0) && ctx->stage >= 5;
  real* cut_slot = analysis ? B.cut + (long)slot * ctx->NC : nullptr;
  double* cutc_slot = analysis ? B.cutc + (long)slot * ctx->NCc : nullptr;
  // both radial terms in one launch where a fused shape applies (FP32, half-warp form with
  // the spectral partners through shared memory)
  bool fused = false;
  if constexpr (std::is_same<real, float>::value) {
    if (ctx->tune.kin_warp == 2 && ctx->tune.kin_fused) {
      const long nplanes = (long)ctx->nblk * ctx->ng;
      auto radial = [&](const float* qin, cudaError_t* e) {
        return kinetic_radial_fused(ctx->NR, ctx->nr, ctx->tune.kin_fused, qin, B.t, nplanes,
                                    B.twR, B.phR, B.lamR, B.twr, B.phr, B.lamr, ctx->ng, B.wpsi,
                                    B.wdpsi, cut_slot, B.blocks, B.ncut_i,
                                    analysis ? ctx->m_inf : -1, analysis ? B.qcol : nullptr, st,
                                    e);
      };
      cudaError_t e = cudaSuccess;
      if (radial(nullptr, &e)) {
        Timer tm(ctx, 11, timed);
        radial(qk, &e);
        LK(e);
        tm.stop();
        fused = true;
      }
    }
  }
  if (!fused) {
    {
      Timer tm(ctx, 0, timed);
      LK(launch_kinetic_rows<real>(qk, B.t, nrows, ctx->planR, B.twR, B.phR, B.lamR,
                                   ctx->tune.rows_pairs, B.blocks, ctx->ng, ctx->nr,
                                   ctx->tune.kin_warp, st));
      tm.stop();
    }
    {
      Timer tm(ctx, 1, timed);
      LK(launch_kinetic_cols<real>(qk, B.t, (long)ctx->nblk * ctx->ng, ctx->nr, ctx->NR,
                                   ctx->planr, B.twr, B.phr, B.lamr, ctx->tune.cols_tile, ctx->ng,
                                   B.wpsi, B.wdpsi, cut_slot, B.blocks, B.ncut_i,
                                   analysis ? ctx->m_inf : -1, analysis ? B.qcol : nullptr,
                                   ctx->tune.kin_warp, st));
      tm.stop();
    }
  }
  const bool tc = std::is_same<real, float>::value && ctx->tc_ok && ctx->tune.use_tc;
  if (tc) {
    Timer tm(ctx, 7, timed);
    TcArgs a{};
    a.ck = (const float*)qk;
    a.ckm1 = (float*)qkm1;
    a.t = (const float*)B.t;
    a.V = (const float*)B.V;
    a.T_hi = (const float*)dptr(ctx, "T_hi");
    a.T_lo = (const float*)dptr(ctx, "T_lo");
    a.Tt_hi = (const float*)dptr(ctx, "Tt_hi");
    a.Tt_lo = (const float*)dptr(ctx, "Tt_lo");
    a.blocks = B.blocks;
    a.coef = (const float*)B.coef;
    a.fr = (const float*)B.fr;
    a.fR = (const float*)B.fR;
    a.DR = (const float*)B.DR;
    a.Dr = (const float*)B.Dr;
    a.dj = B.dj;
    a.out = (float*)hs_out;
    a.npart = mode == 0 ? (double*)dptr(ctx, "npart") : nullptr;
    a.err = (int*)dptr(ctx, "tc_err");
    a.wait_limit = ctx->tune.tc_wait_limit;
    a.erot = (float)ctx->erot;
    a.alpha = first ? 1.0f : 2.0f;
    a.beta = first ? 0.0f : 1.0f;
    a.ncol = ctx->ncol;
    a.npts = ctx->npts;
    a.ng = ctx->ng;
    a.kp = ctx->kp;
    a.NR = ctx->NR;
    a.nelec = ctx->nelec;
    a.mode = mode;
    a.ntiles = (int)((ctx->ncol + 127) / 128);
    a.ngroups = ctx->nblk / ctx->nelec;
    a.kh = ctx->kh;
    a.Tp_hi = (const float*)dptr(ctx, "Tp_hi");
    a.Tp_lo = (const float*)dptr(ctx, "Tp_lo");
    a.persistent = 0;
    if (ctx->tune.tc_persist >= 4 && ctx->kh > 0 && ctx->nelec == 1) {
      a.persistent = 4;
    } else if (ctx->tune.tc_persist >= 2 && ctx->kh > 0) {
      a.persistent = 2;
    } else if (ctx->kh4 > 0 && (ctx->kp > kTcMaxKp || ctx->tune.tc_persist >= 2)) {
      a.persistent = 3;   // the only tensor-core form beyond kTcMaxKp
      a.kh = ctx->kh4;
    } else if (ctx->tune.tc_persist >= 1 && angular_tc2_supported(ctx->kp, ctx->nelec)) {
      a.persistent = 1;
    }
    a.nsm = ctx->nsm;
    a.tma = ctx->tune.tc_tma;
    int tc = 32;
    while (tc < 2 * ctx->nelec * ctx->kp) tc *= 2;
    a.tmem_cols = a.persistent ? 512 : tc;
    LK(launch_angular_tc(a, ctx->nblk / ctx->nelec, (const int*)dptr(ctx, "g_begin"), ctx->nJ,
                         mode == 0 ? B.normbuf + (long)slot * ctx->nJ : nullptr, st));
    tm.stop();
  } else {
    Timer tm(ctx, 2, timed);
    LK(launch_gamma_forward<real>(qk, B.u, B.Tt, B.blocks, ctx->nblk, ctx->ng, ctx->ncol, st));
    tm.stop();
  }
  if (!tc) {
    Timer tm(ctx, 3, timed);
    const real alpha = first ? (real)1 : (real)2;
    const real beta = first ? (real)0 : (real)1;
    LK(launch_gamma_update<real>(B.u, B.T, B.blocks, ctx->nblk, ctx->ng, ctx->ncol, ctx->NR,
                                 B.coef, B.fr, B.fR, (real)ctx->erot, qk, qkm1, B.t, B.V,
                                 ctx->nelec, B.DR, B.Dr, B.dj, alpha, beta, mode, hs_out, st));
    tm.stop();
  }
  if (mode == 1) return MW3_OK;
  if (analysis && ctx->nchan > 0) {
    Timer tm(ctx, 4, timed);
    LK(launch_channels<real>(B.qcol, B.P, B.chan_block, B.chan_row, B.chan_col, ctx->nchan,
                             ctx->ng, ctx->nr, B.d_iter, slot, ctx->an.kmin, cutc_slot, st));
    tm.stop();
  }
  if (analysis && ctx->prod_on) {
    Timer tm(ctx, 8, timed);
    ProdGather<real> pg{(const int*)dptr(ctx, "p_pts"), (const int*)dptr(ctx, "p_pix"),
                        (const real*)dptr(ctx, "p_wst"), (real*)dptr(ctx, "p_G"), ctx->prod_spad,
                        ctx->prod_ngp, B.blocks, ctx->nblk};
    LK(launch_products<real>(qk, ctx->ng, ctx->nr, ctx->NR, ctx->prod_nn,
                             (const int*)dptr(ctx, "p_idx"), (const double*)dptr(ctx, "p_w"),
                             (const real*)dptr(ctx, "p_pl"), ctx->prod_ltop,
                             (const double*)dptr(ctx, "p_T"), (const double*)dptr(ctx, "p_jac"),
                             (const ProdGroup*)dptr(ctx, "p_groups"), (const int*)dptr(ctx, "p_jl"),
                             (int)ctx->prod_jl.size(), ctx->prod_max_nom, (double*)dptr(ctx, "p_v"),
                             (const double*)dptr(ctx, "p_W"), (const int2*)dptr(ctx, "p_chan"),
                             (int)ctx->prod_first[ctx->nJ], cutc_slot,
                             ctx->tune.prod_gather ? &pg : nullptr, st));
    tm.stop();
  }
  if (!tc) {
    Timer tm(ctx, 5, timed);
    LK(launch_norms<real>(qkm1, B.J_begin, ctx->nJ, B.npartial, 256, B.normbuf + (long)slot * ctx->nJ, st));
    tm.stop();
  }
  if (ctx->tp_on) {   // Psi(t_j) += f_k(t_j) q_k, k = iter + slot
    Timer tm(ctx, 10, timed);
    LK(launch_time_accum<real>(qk, (long)ctx->nblk * ctx->npts, ctx->npts, B.blocks,
                               (const double*)dptr(ctx, "tp_f"), ctx->nJ, ctx->tp_nt, ctx->tp_K,
                               B.d_iter, slot, (double*)dptr(ctx, "tp_acc"), st));
    tm.stop();
  }
  if (ctx->ac_on) {   // C_k = <q_0|q_k> of each J, FP64, for k = iter + slot
    Timer tm(ctx, 9, timed);
    LK(launch_dots<real>(qk, (const real*)dptr(ctx, "ac0"), B.J_begin, ctx->nJ,
                         (double*)dptr(ctx, "acpart"), 64,
                         (double*)dptr(ctx, "acbuf") + (long)slot * ctx->nJ, st));
    tm.stop();
  }
  ctx->cur = 1 - ctx->cur;
  return MW3_OK;
}

template <typename real>
int flush(mw3_ctx* ctx, int nvalid, bool timed) {
  ++ctx->acc_version;
  Bufs<real> B = bufs<real>(ctx);
  cudaStream_t st = ctx->stream;
  Timer tm(ctx, 6, timed);
  LK(launch_phases<real>(B.theta, ctx->nJ, ctx->an.nE, ctx->tune.kb, nvalid, B.d_iter, B.ph, st));
  if (std::is_same<real, float>::value && ctx->tc_ok && ctx->tune.flush_tc) {
    LK(launch_flush_tc((const float*)B.ph, (const float*)B.cut, ctx->NC, ctx->tune.kb, nvalid, ctx->nJ,
                       ctx->an.nE, B.colbase, B.ncols, B.accoff, ctx->max_cols, B.acc,
                       (int*)dptr(ctx, "tc_err"), st));
  } else {
    LK(launch_sums_flush<real>(B.ph, B.cut, ctx->NC, ctx->tune.kb, nvalid, ctx->nJ, ctx->an.nE,
                               B.colbase, B.ncols, B.accoff, ctx->max_cols, B.acc, st));
  }
  // channel overlaps: FP64 ring, FP64 phases, FP64 GEMM into their own accumulators
  if (ctx->max_cols_c > 0) {
    if (!std::is_same<real, double>::value)
      LK(launch_phases<double>(B.theta, ctx->nJ, ctx->an.nE, ctx->tune.kb, nvalid, B.d_iter,
                               B.ph64, st));
    LK(launch_sums_flush<double>(B.ph64, B.cutc, ctx->NCc, ctx->tune.kb, nvalid, ctx->nJ, ctx->an.nE,
                                 B.colbase_c, B.ncols_c, B.accoff_c, ctx->max_cols_c, B.accc, st));
  }
  LK(launch_advance(B.d_iter, nvalid, st));
  tm.stop();
  return MW3_OK;
}

// Run `n` iterations starting at ring slot 0 (n <= kb), then flush.
template <typename real>
int chunk(mw3_ctx* ctx, int n, bool timed) {
  for (int s = 0; s < n; ++s) {
    const bool first = (ctx->iter + s == 0);
    int st = step<real>(ctx, s, first, timed);
    if (st) return st;
  }
  return flush<real>(ctx, n, timed);
}

// Norms (and autocorrelations) of the n iterations just run, ring slots slot0 .. slot0 + n - 1.
int check_norms(mw3_ctx* ctx, int slot0, int n) {
  std::vector<double> h((size_t)n * ctx->nJ), ac;
  CK(cudaMemcpyAsync(h.data(), (const double*)dptr(ctx, "normbuf") + (size_t)slot0 * ctx->nJ,
                     h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->ac_on) {
    ac.resize((size_t)n * ctx->nJ);
    CK(cudaMemcpyAsync(ac.data(), (const double*)dptr(ctx, "acbuf") + (size_t)slot0 * ctx->nJ,
                       ac.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  }
  int tc_err = 0;
  if (dptr(ctx, "tc_err"))
    CK(cudaMemcpyAsync(&tc_err, dptr(ctx, "tc_err"), 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  collect_times(ctx);
  if (tc_err) return ctx->fail(MW3_ERR_TIMEOUT, "tensor-core step: an mbarrier wait timed out");
  ctx->norm_trace.insert(ctx->norm_trace.end(), h.begin(), h.end());
  ctx->ac_trace.insert(ctx->ac_trace.end(), ac.begin(), ac.end());
  for (double v : h)
    if (!(v <= 1.5 * ctx->norm0)) return ctx->fail(MW3_ERR_DIVERGED, "||q_k||^2 > 1.5 ||q_0||^2");
  return MW3_OK;
}

template <typename real>
int propagate_impl(mw3_ctx* ctx, long nsteps) {
  const int kb = ctx->tune.kb;
  long done = 0;
  while (done < nsteps) {
    // fill the ring from its first free slot; a full ring is flushed into the sums, a partly
    // filled one stays pending (a probability read adds it on the fly or flushes it)
    const int slot0 = ctx->ring_n;
    const int n = (int)std::min<long>(kb - slot0, nsteps - done);
    const bool can_graph =
        ctx->tune.use_graph && !ctx->timing && slot0 == 0 && n == kb && ctx->iter > 0;
    int st;
    if (can_graph) {
      cudaGraphExec_t& ge = ctx->graph[ctx->cur];
      if (!ge) {
        const int cur0 = ctx->cur;
        const long it0 = ctx->iter;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        st = chunk<real>(ctx, n, false);
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
        if (st) return st;
        if (e2 != cudaSuccess) return ctx->fail(MW3_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e2));
        CK(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        ctx->cur = cur0;   // capture did not execute anything
        ctx->iter = it0;
      }
      CK(cudaGraphLaunch(ge, ctx->stream));
      ++ctx->acc_version;   // the ring's flush is part of the graph
      ctx->cur = (kb % 2) ? 1 - ctx->cur : ctx->cur;
    } else {
      for (int s = 0; s < n; ++s) {
        const bool first = (ctx->iter + s == 0);
        if ((st = step<real>(ctx, slot0 + s, first, true))) return st;
      }
      ctx->ring_n = slot0 + n;
      if (ctx->ring_n == kb) {
        if ((st = flush<real>(ctx, kb, true))) return st;
        ctx->ring_n = 0;
      }
    }
    ctx->iter += n;
    done += n;
    if ((st = check_norms(ctx, slot0, n))) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// Flush the pending ring slots into the sums (readers that need the accumulators themselves).
int flush_pending(mw3_ctx* ctx) {
  if (ctx->ring_n == 0 || ctx->host_only) return MW3_OK;
  const int n = ctx->ring_n;
  const int st = ctx->precision == MW3_FP64 ? flush<double>(ctx, n, false) : flush<float>(ctx, n, false);
  if (st) return st;
  ctx->ring_n = 0;
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// The channel accumulators as a reader sees them: "accc" itself when no ring slot is pending,
// else a device copy with the pending slots added by the same FP64 GEMM a flush uses (their
// FP64 phases first; phases of the slots beyond ring_n are zero). The copy is a few MB.
int channel_accumulators(mw3_ctx* ctx, const double** out) {
  *out = (const double*)dptr(ctx, "accc");
  if (ctx->ring_n == 0 || ctx->max_cols_c <= 0) return MW3_OK;
  int st;
  if ((st = dalloc(ctx, "accc_peek", (size_t)ctx->accc_size * 8))) return st;
  double* pk = (double*)dptr(ctx, "accc_peek");
  CK(cudaMemcpyAsync(pk, dptr(ctx, "accc"), (size_t)ctx->accc_size * 8, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  double* ph64 = (double*)dptr(ctx, ctx->precision == MW3_FP64 ? "ph" : "ph64");
  LK(launch_phases<double>((const double*)dptr(ctx, "theta"), ctx->nJ, ctx->an.nE, ctx->tune.kb,
                           ctx->ring_n, (const long*)dptr(ctx, "d_iter"), ph64, ctx->stream));
  LK(launch_sums_flush<double>(ph64, (const double*)dptr(ctx, "cutc"), ctx->NCc, ctx->tune.kb,
                               ctx->ring_n,
                               ctx->nJ, ctx->an.nE, (const long*)dptr(ctx, "colbase_c"),
                               (const long*)dptr(ctx, "ncols_c"), (const long*)dptr(ctx, "accoff_c"),
                               ctx->max_cols_c, pk, ctx->stream));
  *out = pk;
  return MW3_OK;
}

void incoming_a2(mw3_ctx* ctx, std::vector<double>& a2);

// |S|^2 per (J, Lambda, v, j) summed over the helicities, assembled on the device from the
// channel accumulators `accc` and copied into the caller's array out[nkeys][nE].
int channel_probabilities(mw3_ctx* ctx, const double* accc, const ChanTable& t, double* out) {
  const int nE = ctx->an.nE;
  std::vector<double> a2;
  incoming_a2(ctx, a2);
  const size_t n = (size_t)t.nkeys * nE;
  int st;
  if ((st = dalloc(ctx, "pout", std::max<size_t>(n, 1) * 8))) return st;
  CK(cudaMemcpyAsync(dptr(ctx, "a2"), a2.data(), (size_t)nE * 8, cudaMemcpyHostToDevice, ctx->stream));
  LK(launch_channel_probs(accc, t, (const double*)dptr(ctx, "Ecol"), ctx->Ev0j0,
                          (const double*)dptr(ctx, "theta"), (const double*)dptr(ctx, "dE"),
                          (const double*)dptr(ctx, "a2"), nE, (double*)dptr(ctx, "pout"),
                          ctx->stream));
  CK(cudaMemcpyAsync(out, dptr(ctx, "pout"), n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// Pending ring slots a probability read adds on the fly (more are flushed first).
int peek_max(const mw3_ctx* ctx) { return ctx->precision == MW3_FP64 ? kPeekMax : kPeekMaxX; }

// The flux of the flushed accumulators alone into "fluxA" (and, in the mixed form, their FP32
// copy "acc32"), unless the accumulators are unchanged since the last time.
int flux_flushed(mw3_ctx* ctx) {
  const int nJ = ctx->nJ, nE = ctx->an.nE;
  if (ctx->fluxA_version == ctx->acc_version && dptr(ctx, "fluxA")) return MW3_OK;
  const long max_ncut = *std::max_element(ctx->ncut.begin(), ctx->ncut.end());
  const bool mixed = ctx->precision != MW3_FP64;
  int st;
  if ((st = dalloc(ctx, "flux_part", (size_t)flux_partial_size(nJ, nE, max_ncut) * 8)) ||
      (st = dalloc(ctx, "fluxA", (size_t)nJ * nE * 8)) ||
      (mixed && (st = dalloc(ctx, "acc32", (size_t)ctx->acc_size * 4))))
    return st;
  LK(launch_flux_reduce((const double*)dptr(ctx, "acc"), nJ, nE, (const long*)dptr(ctx, "accoff"),
                        (const long*)dptr(ctx, "ncols"), (const long*)dptr(ctx, "ncut"), max_ncut,
                        (double*)dptr(ctx, "flux_part"), (double*)dptr(ctx, "fluxA"),
                        mixed ? (float*)dptr(ctx, "acc32") : nullptr, ctx->stream));
  ctx->fluxA_version = ctx->acc_version;
  return MW3_OK;
}

// Flux sums over A + Ph Cut for the pending ring slots (phases of those slots first): in FP64
// from the FP64 accumulators; in the mixed form as the flushed flux plus the change that the
// pending slots make, from the FP32 copy of the accumulators (the FP64 ones are not read).
template <typename real>
int flux_peek(mw3_ctx* ctx) {
  Bufs<real> B = bufs<real>(ctx);
  const int nJ = ctx->nJ, nE = ctx->an.nE, kb = ctx->tune.kb;
  LK(launch_phases<real>(B.theta, nJ, nE, kb, ctx->ring_n, B.d_iter, B.ph, ctx->stream));
  const long max_ncut = *std::max_element(ctx->ncut.begin(), ctx->ncut.end());
  int st;
  if ((st = dalloc(ctx, "flux_part", (size_t)flux_partial_size(nJ, nE, max_ncut) * 8))) return st;
  if constexpr (std::is_same<real, float>::value) {
    if ((st = flux_flushed(ctx))) return st;
    LK(launch_flux_cross((const float*)dptr(ctx, "acc32"), nJ, nE, B.accoff, B.ncols, B.ncut,
                         max_ncut, B.ph, kb, ctx->ring_n, B.cut, ctx->NC, B.colbase,
                         (double*)dptr(ctx, "flux_part"), (const double*)dptr(ctx, "fluxA"),
                         (double*)dptr(ctx, "flux"), ctx->stream));
  } else {
    LK(launch_flux_reduce_peek<real>(B.acc, nJ, nE, B.accoff, B.ncols, B.ncut, max_ncut, B.ph, kb,
                                     ctx->ring_n, B.cut, ctx->NC, B.colbase,
                                     (double*)dptr(ctx, "flux_part"), (double*)dptr(ctx, "flux"),
                                     ctx->stream));
  }
  return MW3_OK;
}

// Non-orthogonal Lanczos on H_s in the FBR coordinates of the state (Section 2.3.2, the
// bound-state program): m steps per J from the start vector already in "lz_v" (normalised
// per J here), without reorthogonalisation. alpha/beta (device [m][nJ]) hold
// alpha_i = <v_i|H_s v_i - beta_(i-1) v_(i-1)> and beta_i = ||w_i||, w_i the residual that
// becomes v_(i+1) (beta_i couples v_i and v_(i+1)). With accumulate, x += s[i][iJ] v_i
// each step ("lz_s" device [m][nJ]) into "lz_x" (the second run of a Ritz vector).
template <typename real>
int lanczos_run(mw3_ctx* ctx, int m, bool accumulate) {
  cudaStream_t st = ctx->stream;
  const long n = (long)ctx->nblk * ctx->npts;
  const int nJ = ctx->nJ;
  const DevBlock* blk = (const DevBlock*)dptr(ctx, "blocks");
  const long* Jb = (const long*)dptr(ctx, "J_begin");
  double* part = (double*)dptr(ctx, "lz_part");
  double* a = (double*)dptr(ctx, "lz_a");
  double* b = (double*)dptr(ctx, "lz_b");
  double* b2 = (double*)dptr(ctx, "lz_b2");
  double* nrm = (double*)dptr(ctx, "lz_nrm");
  real* v = (real*)dptr(ctx, "lz_v");
  real* vp = (real*)dptr(ctx, "lz_vp");
  real* w = (real*)dptr(ctx, "lz_w");
  real* x = accumulate ? (real*)dptr(ctx, "lz_x") : nullptr;
  const double* S = accumulate ? (const double*)dptr(ctx, "lz_s") : nullptr;
  LK(launch_dots<real>(v, v, Jb, nJ, part, 64, nrm, st));
  LK(launch_rscale_seg<real>(v, nrm, n, ctx->npts, blk, st));
  CK(cudaMemsetAsync(vp, 0, n * sizeof(real), st));
  if (accumulate) CK(cudaMemsetAsync(x, 0, n * sizeof(real), st));
  const char* qname = state_name(ctx, true);
  void* saved = ctx->buf[qname].p;
  const int cur0 = ctx->cur;
  int status = MW3_OK;
  for (int i = 0; i < m && status == MW3_OK; ++i) {
    if (accumulate) LK(launch_axpy_seg<real>(x, v, S + (size_t)i * nJ, 1.0, n, ctx->npts, blk, st));
    ctx->buf[qname].p = v;   // H_s v through the step's own kernels (mode 1)
    status = step<real>(ctx, 0, true, false, 1, w);
    ctx->buf[qname].p = saved;
    ctx->cur = cur0;
    if (status) break;
    if (i > 0) LK(launch_axpy_seg<real>(w, vp, b + (size_t)(i - 1) * nJ, -1.0, n, ctx->npts, blk, st));
    LK(launch_dots<real>(v, w, Jb, nJ, part, 64, a + (size_t)i * nJ, st));
    LK(launch_axpy_seg<real>(w, v, a + (size_t)i * nJ, -1.0, n, ctx->npts, blk, st));
    LK(launch_dots<real>(w, w, Jb, nJ, part, 64, b2 + (size_t)i * nJ, st));
    LK(launch_sqrt(b2 + (size_t)i * nJ, b + (size_t)i * nJ, nJ, st));
    LK(launch_rscale_seg<real>(w, b2 + (size_t)i * nJ, n, ctx->npts, blk, st));
    real* t = vp;   // (v_(i-1), v_i, w) <- (v_i, v_(i+1), free)
    vp = v;
    v = w;
    w = t;
  }
  ctx->buf[qname].p = saved;
  CK(cudaStreamSynchronize(st));
  return status;
}

// Lanczos coefficients of m steps from the host start vector v0 (grid values), per J.
int lanczos_coefficients(mw3_ctx* ctx, const double* v0, int m, std::vector<double>& alpha,
                         std::vector<double>& beta, bool accumulate = false) {
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  const int nJ = ctx->nJ;
  int st;
  if ((st = dalloc(ctx, "lz_v", n * ctx->rs())) || (st = dalloc(ctx, "lz_vp", n * ctx->rs())) ||
      (st = dalloc(ctx, "lz_w", n * ctx->rs())) ||
      (st = dalloc(ctx, "lz_part", (size_t)nJ * 64 * 8)) ||
      (st = dalloc(ctx, "lz_a", (size_t)m * nJ * 8)) || (st = dalloc(ctx, "lz_b", (size_t)m * nJ * 8)) ||
      (st = dalloc(ctx, "lz_b2", (size_t)m * nJ * 8)) || (st = dalloc(ctx, "lz_nrm", (size_t)nJ * 8)))
    return st;
  if (accumulate && (st = dalloc(ctx, "lz_x", n * ctx->rs()))) return st;
  if ((st = transform_upload(ctx, v0, "lz_v", true))) return st;
  st = ctx->precision == MW3_FP64 ? lanczos_run<double>(ctx, m, accumulate)
                                  : lanczos_run<float>(ctx, m, accumulate);
  if (st) return st;
  alpha.resize((size_t)m * nJ);
  beta.resize((size_t)m * nJ);
  CK(cudaMemcpyAsync(alpha.data(), dptr(ctx, "lz_a"), alpha.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(beta.data(), dptr(ctx, "lz_b"), beta.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

// Cullum-Willoughby identification for one J: accepted eigenvalues of T_m (scaled units).
void cw_accept(const std::vector<double>& al, const std::vector<double>& be, double tol,
               std::vector<double>& out) {
  const int m = (int)al.size();
  std::vector<double> lam, hat;
  tridiagonal_eigenvalues(al, std::vector<double>(be.begin(), be.begin() + std::max(m - 1, 0)), lam);
  if (m > 1) {
    std::vector<double> ah(al.begin() + 1, al.end()), bh(be.begin() + 1, be.begin() + (m - 1));
    tridiagonal_eigenvalues(ah, bh, hat);
  }
  out.clear();
  for (int i = 0; i < m;) {
    int j = i;
    while (j + 1 < m && lam[j + 1] - lam[i] <= tol) ++j;
    double mean = 0;
    for (int k = i; k <= j; ++k) mean += lam[k];
    mean /= (j - i + 1);
    double dh = 1e300;
    for (double h : hat) dh = std::min(dh, std::fabs(h - mean));
    if (j > i || dh > tol) out.push_back(mean);   // copies, or simple and not in T-hat
    i = j + 1;
  }
}

// |a(E)|^2 of the incoming packet, a(E) = sqrt(mu/(2 pi K)) sum_m dR exp(i K R_m) g~(R_m).
void incoming_a2(mw3_ctx* ctx, std::vector<double>& a2) {
  const int nE = ctx->an.nE;
  if ((int)ctx->a2_cache.size() == nE) {
    a2 = ctx->a2_cache;
    return;
  }
  a2.assign(nE, 0.0);
  if (ctx->pcb_on) {
    // products-coordinate-based start: a(E) = sqrt(mu_s/(2 pi K)) int exp(i K R) g(R) dR
    // = sqrt(mu_s/(2 pi K)) N sqrt(2 pi) G / 2 sum_(s = +-1) exp(i (K + s k0) R0 - G^2 (K + s k0)^2 / 2)
    for (int e = 0; e < nE; ++e) {
      const double K = std::sqrt(2.0 * ctx->pcb_mu * ctx->Ecol[e]);
      double re = 0, im = 0;
      for (double sgn : {1.0, -1.0}) {
        const double q = K + sgn * ctx->pcb_k0;
        const double mag = std::exp(-ctx->pcb_G * ctx->pcb_G * q * q / 2.0);
        re += mag * std::cos(q * ctx->pcb_R0);
        im += mag * std::sin(q * ctx->pcb_R0);
      }
      const double sc = std::sqrt(ctx->pcb_mu / (2.0 * M_PI * K)) * ctx->pcb_N *
                        std::sqrt(2.0 * M_PI) * ctx->pcb_G / 2.0;
      a2[e] = sc * sc * (re * re + im * im);
    }
    ctx->a2_cache = a2;
    return;
  }
  for (int e = 0; e < nE; ++e) {
    const double K = std::sqrt(2.0 * ctx->mu * ctx->Ecol[e]);
    double re = 0, im = 0;
    for (int i = 0; i < ctx->NR; ++i) {
      re += std::cos(K * ctx->R[i]) * ctx->g_tilde[i];
      im += std::sin(K * ctx->R[i]) * ctx->g_tilde[i];
    }
    const double s = std::sqrt(ctx->mu / (2.0 * M_PI * K)) * ctx->dR;
    a2[e] = s * s * (re * re + im * im);
  }
  ctx->a2_cache = a2;
}

}  // namespace

extern "C" {

int mw3_propagate(mw3_ctx* ctx, long nsteps) {
  if (!ctx || nsteps < 0) return MW3_ERR_BAD_ARG;
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context cannot propagate");
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  cudaSetDevice(ctx->device);
  return ctx->precision == MW3_FP64 ? propagate_impl<double>(ctx, nsteps)
                                    : propagate_impl<float>(ctx, nsteps);
}

long mw3_iteration(const mw3_ctx* ctx) { return ctx ? ctx->iter : -1; }

int mw3_sizes(const mw3_ctx* ctx, long* nblocks, long* ppb) {
  if (!ctx || ctx->stage < 1) return MW3_ERR_STATE;
  if (nblocks) *nblocks = ctx->nblk;
  if (ppb) *ppb = ctx->npts;
  return MW3_OK;
}

int mw3_spectral_range(const mw3_ctx* ctx, double* E0, double* dE) {
  if (!ctx || ctx->stage < 2) return MW3_ERR_STATE;
  for (int i = 0; i < ctx->nJ; ++i) {
    if (E0) E0[i] = ctx->E0[i];
    if (dE) dE[i] = ctx->dE[i];
  }
  return MW3_OK;
}

int mw3_reference_energy(const mw3_ctx* ctx, double* e) {
  if (!ctx || ctx->stage < 3 || !e) return MW3_ERR_STATE;
  *e = ctx->Ev0j0;
  return MW3_OK;
}

int mw3_set_state(mw3_ctx* ctx, const double* q, const double* qprev) {
  if (!ctx || !q) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return MW3_OK;
  cudaSetDevice(ctx->device);
  int st = transform_upload(ctx, q, state_name(ctx, true), true);
  if (st) return st;
  if (qprev) return transform_upload(ctx, qprev, state_name(ctx, false), true);
  CK(cudaMemsetAsync(dptr(ctx, state_name(ctx, false)), 0,
                     (size_t)ctx->nblk * ctx->npts * ctx->rs(), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

int mw3_set_state_f32(mw3_ctx* ctx, const float* q, const float* qprev) {
  if (!ctx || !q) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return MW3_OK;
  cudaSetDevice(ctx->device);
  int st = transform_upload(ctx, q, state_name(ctx, true), true);
  if (st) return st;
  if (qprev) return transform_upload(ctx, qprev, state_name(ctx, false), true);
  CK(cudaMemsetAsync(dptr(ctx, state_name(ctx, false)), 0,
                     (size_t)ctx->nblk * ctx->npts * ctx->rs(), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MW3_OK;
}

int mw3_get_state(mw3_ctx* ctx, double* q, double* qprev) {
  if (!ctx || !q) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  cudaSetDevice(ctx->device);
  int st = transform_download(ctx, state_name(ctx, true), q);
  if (st) return st;
  if (qprev) return transform_download(ctx, state_name(ctx, false), qprev);
  return MW3_OK;
}

int mw3_enable_autocorrelation(mw3_ctx* ctx) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  if (ctx->iter != 0) return ctx->fail(MW3_ERR_STATE, "the autocorrelation starts at k = 0");
  cudaSetDevice(ctx->device);
  const size_t bytes = (size_t)ctx->nblk * ctx->npts * ctx->rs();
  int st;
  if ((st = dalloc(ctx, "ac0", bytes)) || (st = dalloc(ctx, "acpart", (size_t)ctx->nJ * 64 * 8)) ||
      (st = dalloc(ctx, "acbuf", (size_t)ctx->tune.kb * ctx->nJ * 8)))
    return st;
  CK(cudaMemcpyAsync(dptr(ctx, "ac0"), dptr(ctx, state_name(ctx, true)), bytes,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& g : ctx->graph)   // the captured steps do not contain the extra dot
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ctx->ac_on = true;
  ctx->ac_trace.clear();
  return MW3_OK;
}

int mw3_enable_time_packets(mw3_ctx* ctx, int nt, const double* t) {
  if (!ctx || nt < 1 || !t) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  if (ctx->iter != 0) return ctx->fail(MW3_ERR_STATE, "the time-domain sums start at k = 0");
  for (int j = 0; j < nt; ++j)
    if (!(t[j] >= 0.0 && t[j] < 1e12)) return ctx->fail(MW3_ERR_BAD_ARG, "times must be >= 0");
  cudaSetDevice(ctx->device);
  // f_k(t) = (2 - delta_k0) exp(-i E0 t) (-i)^k J_k(t dE) per (J, t_j), up to the last k
  // at which some |J_k| is above 1e-17 (beyond it the terms are below FP64 resolution)
  const int nJ = ctx->nJ;
  std::vector<std::vector<double>> Js((size_t)nJ * nt);
  long K = 1;
  for (int iJ = 0; iJ < nJ; ++iJ)
    for (int j = 0; j < nt; ++j) {
      const double x = t[j] * ctx->dE[iJ];
      std::vector<double>& b = Js[(size_t)iJ * nt + j];
      bessel_j_sequence(x, (int)(x + 60.0 + 15.0 * std::cbrt(x)), b);
      for (long k = (long)b.size() - 1; k >= 0; --k)
        if (std::fabs(b[k]) > 1e-17) {
          K = std::max(K, k + 1);
          break;
        }
    }
  std::vector<double> f((size_t)K * nJ * nt * 2, 0.0);
  for (long k = 0; k < K; ++k)
    for (int iJ = 0; iJ < nJ; ++iJ)
      for (int j = 0; j < nt; ++j) {
        const std::vector<double>& b = Js[(size_t)iJ * nt + j];
        const double jk = k < (long)b.size() ? b[k] : 0.0;
        const double w = (k == 0 ? 1.0 : 2.0) * jk;
        const double ph = -ctx->E0[iJ] * t[j];
        const double c = std::cos(ph), sn = std::sin(ph);
        // (-i)^k: 1, -i, -1, i
        const double pr = (k % 4 == 0) ? 1.0 : (k % 4 == 2 ? -1.0 : 0.0);
        const double pi_ = (k % 4 == 1) ? -1.0 : (k % 4 == 3 ? 1.0 : 0.0);
        const size_t o = (((size_t)k * nJ + iJ) * nt + j) * 2;
        f[o] = w * (c * pr - sn * pi_);
        f[o + 1] = w * (c * pi_ + sn * pr);
      }
  int st;
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  if ((st = upload_real(ctx, "tp_f", f, true))) return st;
  if ((st = dalloc(ctx, "tp_acc", (size_t)nt * 2 * n * 8)) || (st = dzero(ctx, "tp_acc"))) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& g : ctx->graph)   // the captured steps do not contain the accumulation
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ctx->tp_nt = nt;
  ctx->tp_K = K;
  ctx->tp_on = true;
  return MW3_OK;
}

int mw3_time_packets(mw3_ctx* ctx, double* out, long* kmax) {
  if (!ctx || !out) return MW3_ERR_BAD_ARG;
  if (!ctx->tp_on) return ctx->fail(MW3_ERR_STATE, "mw3_enable_time_packets first");
  cudaSetDevice(ctx->device);
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  const int ng = ctx->ng;
  int st;
  if (!ctx->buf.count("Tt64")) {   // FP64 (T^Omega)^T for the FBR -> grid transform
    std::vector<double> Ttall;
    for (auto& Tm : ctx->T)
      for (int a = 0; a < ng; ++a)
        for (int b = 0; b < ng; ++b) Ttall.push_back(Tm[(size_t)b * ng + a]);
    if ((st = upload_real(ctx, "Tt64", Ttall, true))) return st;
  }
  if ((st = dalloc(ctx, "tp_tmp", n * 8))) return st;
  for (int c = 0; c < 2 * ctx->tp_nt; ++c) {
    LK(launch_gamma_forward<double>((const double*)dptr(ctx, "tp_acc") + (size_t)c * n,
                                    (double*)dptr(ctx, "tp_tmp"), (const double*)dptr(ctx, "Tt64"),
                                    (const DevBlock*)dptr(ctx, "blocks"), ctx->nblk, ng, ctx->ncol,
                                    ctx->stream));
    CK(cudaMemcpyAsync(out + (size_t)c * n, dptr(ctx, "tp_tmp"), n * 8, cudaMemcpyDeviceToHost,
                       ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (kmax) *kmax = ctx->tp_K;
  return MW3_OK;
}

long mw3_autocorrelation(mw3_ctx* ctx, double* C, long n) {
  if (!ctx || !C || n < 0) return MW3_ERR_BAD_ARG;
  const long have = (long)ctx->ac_trace.size() / std::max(1, ctx->nJ);
  const long cnt = std::min(n, have);
  std::copy(ctx->ac_trace.begin(), ctx->ac_trace.begin() + cnt * ctx->nJ, C);
  return cnt;
}

int mw3_photo_spectrum(mw3_ctx* ctx, const double* E, int nE, double* a0) {
  if (!ctx || !E || !a0 || nE < 0) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  const int nJ = ctx->nJ;
  const long N = (long)ctx->ac_trace.size() / std::max(1, nJ);
  for (int iJ = 0; iJ < nJ; ++iJ)
    for (int e = 0; e < nE; ++e) {
      const double Es = (E[e] - ctx->E0[iJ]) / ctx->dE[iJ];
      if (!(Es > -1.0 && Es < 1.0))
        return ctx->fail(MW3_ERR_BAD_ARG, "energy outside the spectral range of H");
      const double th = std::acos(Es);
      double s = 0;
      for (long k = 0; k < N; ++k)   // (2 - delta_k0) cos(k theta) C_k, k theta formed in FP64
        s += (k == 0 ? 1.0 : 2.0) * std::cos((double)k * th) * ctx->ac_trace[(size_t)k * nJ + iJ];
      a0[(size_t)iJ * nE + e] = s / (M_PI * ctx->dE[iJ] * std::sqrt(1.0 - Es * Es));
    }
  return MW3_OK;
}

int mw3_apply_hs(mw3_ctx* ctx, const double* q, double* out) {
  if (!ctx || !q || !out) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  cudaSetDevice(ctx->device);
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  int st;
  if ((st = dalloc(ctx, "hs_in", n * ctx->rs())) || (st = dalloc(ctx, "hs_out", n * ctx->rs()))) return st;
  if ((st = transform_upload(ctx, q, "hs_in", true))) return st;
  // route the input through the q_k slot temporarily
  const int cur0 = ctx->cur;
  const char* qname = state_name(ctx, true);
  void* saved = ctx->buf[qname].p;
  ctx->buf[qname].p = dptr(ctx, "hs_in");
  if (ctx->precision == MW3_FP64)
    st = step<double>(ctx, 0, true, false, 1, (double*)dptr(ctx, "hs_out"));
  else
    st = step<float>(ctx, 0, true, false, 1, (float*)dptr(ctx, "hs_out"));
  ctx->buf[qname].p = saved;
  ctx->cur = cur0;
  if (st) return st;
  return transform_download(ctx, "hs_out", out);
}

long mw3_norm_trace(mw3_ctx* ctx, double* out, long n) {
  if (!ctx || !out || n < 0) return MW3_ERR_BAD_ARG;
  const long have = (long)ctx->norm_trace.size() / std::max(1, ctx->nJ);
  const long cnt = std::min(n, have);
  std::copy(ctx->norm_trace.end() - cnt * ctx->nJ, ctx->norm_trace.end(), out);
  return cnt;
}

int mw3_lanczos(mw3_ctx* ctx, const double* v0, int m, double* alpha, double* beta) {
  if (!ctx || !v0 || m < 1 || !alpha || !beta) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  cudaSetDevice(ctx->device);
  std::vector<double> a, b;
  int st = lanczos_coefficients(ctx, v0, m, a, b);
  if (st) return st;
  std::copy(a.begin(), a.end(), alpha);
  std::copy(b.begin(), b.end(), beta);
  return MW3_OK;
}

int mw3_bound_states(mw3_ctx* ctx, const double* v0, int m, double emin, double emax, int maxev,
                     double* E, int* count) {
  if (!ctx || !v0 || m < 2 || maxev < 1 || !E || !count) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  cudaSetDevice(ctx->device);
  std::vector<double> a, b;
  int st = lanczos_coefficients(ctx, v0, m, a, b);
  if (st) return st;
  const int nJ = ctx->nJ;
  const double tol = ctx->precision == MW3_FP64 ? 1e-10 : 1e-5;
  for (int iJ = 0; iJ < nJ; ++iJ) {
    std::vector<double> al(m), be(m), acc;
    for (int i = 0; i < m; ++i) {
      al[i] = a[(size_t)i * nJ + iJ];
      be[i] = b[(size_t)i * nJ + iJ];
    }
    cw_accept(al, be, tol, acc);
    int c = 0;
    for (double lam : acc) {
      const double e = ctx->E0[iJ] + ctx->dE[iJ] * lam;
      if (e >= emin && e <= emax && c < maxev) E[(size_t)iJ * maxev + c++] = e;
    }
    count[iJ] = c;
  }
  return MW3_OK;
}

int mw3_bound_state_vector(mw3_ctx* ctx, const double* v0, int m, int iJ, double E, double* out) {
  if (!ctx || !v0 || m < 2 || !out) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 2) return ctx->fail(MW3_ERR_STATE, "mw3_load_potential first");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  if (iJ < 0 || iJ >= ctx->nJ) return ctx->fail(MW3_ERR_BAD_ARG, "J index out of range");
  cudaSetDevice(ctx->device);
  std::vector<double> a, b;
  int st = lanczos_coefficients(ctx, v0, m, a, b);
  if (st) return st;
  const int nJ = ctx->nJ;
  std::vector<double> al(m), be(m - 1), s;
  for (int i = 0; i < m; ++i) al[i] = a[(size_t)i * nJ + iJ];
  for (int i = 0; i + 1 < m; ++i) be[i] = b[(size_t)i * nJ + iJ];
  tridiagonal_eigenvector(al, be, (E - ctx->E0[iJ]) / ctx->dE[iJ], s);
  std::vector<double> S((size_t)m * nJ, 0.0);
  for (int i = 0; i < m; ++i) S[(size_t)i * nJ + iJ] = s[i];
  if ((st = upload_raw(ctx, "lz_s", S))) return st;
  if ((st = lanczos_coefficients(ctx, v0, m, a, b, true))) return st;   // second run
  // normalise the J's part on the host after the transform (an orthogonal map per block)
  if ((st = transform_download(ctx, "lz_x", out))) return st;
  double nrm = 0;
  const size_t n = (size_t)ctx->nblk * ctx->npts;
  for (size_t e = 0; e < n; ++e) nrm += out[e] * out[e];
  nrm = std::sqrt(nrm);
  if (nrm > 0)
    for (size_t e = 0; e < n; ++e) out[e] /= nrm;
  return MW3_OK;
}

int mw3_incoming_amplitude(mw3_ctx* ctx, double* a2) {
  if (!ctx || !a2) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  std::vector<double> v;
  incoming_a2(ctx, v);
  std::copy(v.begin(), v.end(), a2);
  return MW3_OK;
}

int mw3_product_probabilities(mw3_ctx* ctx, double* P) {
  if (!ctx || !P) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  if (!ctx->prod_on) return ctx->fail(MW3_ERR_STATE, "product channels are not enabled");
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  int st;
  if (ctx->ring_n > peek_max(ctx) && (st = flush_pending(ctx))) return st;
  const double* accc = nullptr;   // with the pending ring slots added
  if ((st = channel_accumulators(ctx, &accc))) return st;
  return channel_probabilities(ctx, accc, ctx->chan_tab_p, P);
}

int mw3_flux_probabilities(mw3_ctx* ctx, double* E, double* Ptot, double* Pinel) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5) return ctx->fail(MW3_ERR_STATE, "mw3_set_analysis first");
  const int nE = ctx->an.nE, nJ = ctx->nJ;
  if (E)
    for (int e = 0; e < nE; ++e) E[e] = ctx->Ecol[e];
  if (ctx->host_only) return ctx->fail(MW3_ERR_STATE, "host-only context");
  std::vector<double> a2;
  incoming_a2(ctx, a2);
  int st;
  if ((st = dalloc(ctx, "flux", (size_t)nJ * nE * 8))) return st;
  // a few pending ring slots are added on the fly (the accumulators are only read); more are
  // flushed first
  if (ctx->ring_n > peek_max(ctx) && (st = flush_pending(ctx))) return st;
  if (ctx->ring_n > 0) {
    st = ctx->precision == MW3_FP64 ? flux_peek<double>(ctx) : flux_peek<float>(ctx);
    if (st) return st;
  } else {
    if ((st = flux_flushed(ctx))) return st;
    CK(cudaMemcpyAsync(dptr(ctx, "flux"), dptr(ctx, "fluxA"), (size_t)nJ * nE * 8,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  }
  std::vector<double> F((size_t)nJ * nE);
  CK(cudaMemcpyAsync(F.data(), dptr(ctx, "flux"), F.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (Ptot) {
    for (int iJ = 0; iJ < nJ; ++iJ)
      for (int e = 0; e < nE; ++e) {
        const double th = ctx->theta[(size_t)iJ * nE + e];
        const double pref = 1.0 / (2.0 * M_PI * ctx->dE[iJ] * std::sin(th));
        Ptot[(size_t)iJ * nE + e] = (2.0 * M_PI / ctx->m) * F[(size_t)iJ * nE + e] * pref * pref / a2[e];
      }
  }
  if (Pinel && ctx->an.vmax >= 0) {
    const double* accc = nullptr;   // with the pending ring slots added
    if ((st = channel_accumulators(ctx, &accc))) return st;
    if ((st = channel_probabilities(ctx, accc, ctx->chan_tab_r, Pinel))) return st;
  }
  return MW3_OK;
}

int mw3_set_tuning(mw3_ctx* ctx, const char* key, long v) {
  if (!ctx || !key) return MW3_ERR_BAD_ARG;
  const std::string k(key);
  auto drop_graphs = [&]() {
    for (auto& g : ctx->graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  };
  if (k == "kb") {
    if (v < 1 || v > 1024) return ctx->fail(MW3_ERR_BAD_ARG, "kb must be in 1..1024");
    if (ctx->stage >= 5) return ctx->fail(MW3_ERR_STATE, "set kb before mw3_set_analysis");
    ctx->tune.kb = (int)v;
  } else if (k == "rows_pairs") {
    if (v < 1 || v > 16) return ctx->fail(MW3_ERR_BAD_ARG, "rows_pairs must be in 1..16");
    ctx->tune.rows_pairs = (int)v;
  } else if (k == "cols_tile") {
    if (v < 2 || v > 64 || v % 2) return ctx->fail(MW3_ERR_BAD_ARG, "cols_tile must be even, 2..64");
    ctx->tune.cols_tile = (int)v;
  } else if (k == "use_graph") {
    ctx->tune.use_graph = v != 0;
  } else if (k == "kin_warp") {
    if (v < 0 || v > 3) return ctx->fail(MW3_ERR_BAD_ARG, "kin_warp is 0, 1, 2 or 3");
    ctx->tune.kin_warp = (int)v;
  } else if (k == "kin_fused") {
    if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8)
      return ctx->fail(MW3_ERR_BAD_ARG, "kin_fused is 0, 1 (automatic), 2, 4 or 8");
    ctx->tune.kin_fused = (int)v;
  } else if (k == "up_direct") {
    ctx->tune.up_direct = v != 0;
  } else if (k == "flush_tc") {
    ctx->tune.flush_tc = v != 0;
  } else if (k == "tc_tma") {
    ctx->tune.tc_tma = v != 0;
    drop_graphs();
  } else if (k == "prod_gather") {
    ctx->tune.prod_gather = v != 0;
  } else if (k == "tc_wait_limit") {
    if (v < 0 || v > (1L << 22)) return ctx->fail(MW3_ERR_BAD_ARG, "tc_wait_limit must be in 0..2^22");
    ctx->tune.tc_wait_limit = v;
  } else if (k == "tc_persist") {
    if (v < 0 || v > 4) return ctx->fail(MW3_ERR_BAD_ARG, "tc_persist must be in 0..4");
    ctx->tune.tc_persist = (int)v;
  } else if (k == "use_tc") {
    if (v != 0 && ctx->precision != MW3_MIXED)
      return ctx->fail(MW3_ERR_BAD_ARG, "use_tc needs MW3_MIXED");
    ctx->tc_user = v != 0;
    ctx->tune.use_tc = (v != 0) && (ctx->stage < 2 || ctx->tc_ok);
  } else {
    return ctx->fail(MW3_ERR_BAD_ARG, "unknown tuning key " + k);
  }
  drop_graphs();
  return MW3_OK;
}

long mw3_get_tuning(const mw3_ctx* ctx, const char* key) {
  if (!ctx || !key) return MW3_ERR_BAD_ARG;
  const std::string k(key);
  if (k == "kb") return ctx->tune.kb;
  if (k == "rows_pairs") return ctx->tune.rows_pairs;
  if (k == "cols_tile") return ctx->tune.cols_tile;
  if (k == "use_graph") return ctx->tune.use_graph;
  if (k == "kin_warp") return ctx->tune.kin_warp;
  if (k == "tc_persist") return ctx->tune.tc_persist;
  if (k == "tc_tma") return ctx->tune.tc_tma;
  if (k == "prod_gather") return ctx->tune.prod_gather;
  if (k == "tc_wait_limit") return ctx->tune.tc_wait_limit;
  if (k == "prod_points") return ctx->prod_npts;
  if (k == "kin_fused") return ctx->tune.kin_fused;
  if (k == "up_direct") return ctx->tune.up_direct;
  if (k == "up_direct_last") return ctx->up_direct_last ? 1 : 0;
  if (k == "flush_tc") return ctx->tune.flush_tc;
  if (k == "use_tc") return ctx->stage >= 2 ? ctx->tune.use_tc : (ctx->tc_user != 0);
  return MW3_ERR_BAD_ARG;
}

int mw3_kernel_times(mw3_ctx* ctx, int enable, const char** names, double* ms, long* launches,
                     int* count) {
  if (!ctx) return MW3_ERR_BAD_ARG;
  if (enable >= 0) {
    ctx->timing = enable != 0;
    std::fill(ctx->kms, ctx->kms + kNumKernels, 0.0);
    std::fill(ctx->klaunch, ctx->klaunch + kNumKernels, 0L);
  }
  if (count) {
    const int n = std::min(*count, kNumKernels);
    for (int i = 0; i < n; ++i) {
      if (names) names[i] = kKernelNames[i];
      if (ms) ms[i] = ctx->kms[i];
      if (launches) launches[i] = ctx->klaunch[i];
    }
    *count = n;
  }
  return MW3_OK;
}

int mw3_checkpoint_save(mw3_ctx* ctx, const char* path) {
  if (!ctx || !path) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5 || ctx->host_only) return ctx->fail(MW3_ERR_STATE, "nothing to save");
  cudaSetDevice(ctx->device);
  int fst = flush_pending(ctx);   // the saved sums hold every iteration run so far
  if (fst) return fst;
  // raw device state (FBR coefficients in the context's precision), no conversion
  const size_t nb = (size_t)ctx->nblk * ctx->npts * ctx->rs();
  std::vector<char> q(nb), qp(nb);
  std::vector<double> acc(ctx->acc_size), accc(ctx->accc_size);
  CK(cudaMemcpyAsync(q.data(), dptr(ctx, state_name(ctx, true)), nb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(qp.data(), dptr(ctx, state_name(ctx, false)), nb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(acc.data(), dptr(ctx, "acc"), acc.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (!accc.empty())
    CK(cudaMemcpyAsync(accc.data(), dptr(ctx, "accc"), accc.size() * 8, cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::ofstream f(path, std::ios::binary);
  if (!f) return ctx->fail(MW3_ERR_IO, std::string("cannot open ") + path);
  const uint64_t magic = 0x4d57334350543033ULL;  // "MW3CPT03"
  const uint64_t hdr[7] = {magic, (uint64_t)ctx->nblk, (uint64_t)ctx->npts, (uint64_t)ctx->acc_size,
                           (uint64_t)ctx->iter, (uint64_t)ctx->precision, (uint64_t)ctx->accc_size};
  f.write((const char*)hdr, sizeof(hdr));
  f.write(q.data(), nb);
  f.write(qp.data(), nb);
  f.write((const char*)acc.data(), acc.size() * 8);
  f.write((const char*)accc.data(), accc.size() * 8);
  const uint64_t nt = ctx->norm_trace.size();
  f.write((const char*)&nt, 8);
  f.write((const char*)ctx->norm_trace.data(), nt * 8);
  if (!f) return ctx->fail(MW3_ERR_IO, "write failed");
  return MW3_OK;
}

int mw3_checkpoint_load(mw3_ctx* ctx, const char* path) {
  if (!ctx || !path) return MW3_ERR_BAD_ARG;
  if (ctx->stage < 5 || ctx->host_only) return ctx->fail(MW3_ERR_STATE, "set up the context first");
  std::ifstream f(path, std::ios::binary);
  if (!f) return ctx->fail(MW3_ERR_IO, std::string("cannot open ") + path);
  uint64_t hdr[7];
  f.read((char*)hdr, sizeof(hdr));
  if (!f || hdr[0] != 0x4d57334350543033ULL || hdr[1] != (uint64_t)ctx->nblk ||
      hdr[2] != (uint64_t)ctx->npts || hdr[3] != (uint64_t)ctx->acc_size ||
      hdr[5] != (uint64_t)ctx->precision || hdr[6] != (uint64_t)ctx->accc_size)
    return ctx->fail(MW3_ERR_IO, "checkpoint does not match this configuration");
  ctx->ring_n = 0;   // the saved sums hold every saved iteration
  ++ctx->acc_version;
  const size_t nb = (size_t)ctx->nblk * ctx->npts * ctx->rs();
  std::vector<char> q(nb), qp(nb);
  std::vector<double> acc(ctx->acc_size), accc(ctx->accc_size);
  f.read(q.data(), nb);
  f.read(qp.data(), nb);
  f.read((char*)acc.data(), acc.size() * 8);
  f.read((char*)accc.data(), accc.size() * 8);
  uint64_t nt = 0;
  f.read((char*)&nt, 8);
  std::vector<double> tr(nt);
  f.read((char*)tr.data(), nt * 8);
  if (!f) return ctx->fail(MW3_ERR_IO, "truncated checkpoint");
  CK(cudaMemcpyAsync(dptr(ctx, state_name(ctx, true)), q.data(), nb, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dptr(ctx, state_name(ctx, false)), qp.data(), nb, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dptr(ctx, "acc"), acc.data(), acc.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  if (!accc.empty())
    CK(cudaMemcpyAsync(dptr(ctx, "accc"), accc.data(), accc.size() * 8, cudaMemcpyHostToDevice,
                       ctx->stream));
  ctx->iter = (long)hdr[4];
  long it = ctx->iter;
  CK(cudaMemcpyAsync(dptr(ctx, "d_iter"), &it, 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->norm_trace = tr;
  return MW3_OK;
}

}  // extern "C"

// ------------------------------------------------------- FMA-chain peak probe
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)12345.678) out[threadIdx.x] = s;  // keeps the chains live
}
}  // namespace

extern "C" int mw3_measure_peak(int device, int kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return MW3_ERR_BAD_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MW3_ERR_CUDA;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  void* out = nullptr;
  if (cudaMalloc(&out, 1024 * 8) != cudaSuccess) return MW3_ERR_OOM;
  const int blocks = prop.multiProcessorCount * 8;
  const int iters = kind == 0 ? 1 << 12 : 1 << 16;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (kind == 0)
      k_fma_chain<double><<<blocks, 256>>>((double*)out, iters, 0.999999, 1e-7);
    else
      k_fma_chain<float><<<blocks, 256>>>((float*)out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8.0 * iters * (double)blocks * 256.0;
    if (rep > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return MW3_ERR_CUDA;
  *tflops = best;
  return MW3_OK;
}
