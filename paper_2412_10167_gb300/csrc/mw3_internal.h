// Internal declarations of libmw3: device-side tables, kernel launchers and the
// context. Everything here is private to the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mw3.h"
#include "mw3_wigner.h"

namespace mw3 {

// ---------------------------------------------------------------- small complex
template <typename T>
struct cpx {
  T x, y;
};

// ------------------------------------------------------------------ FFT plan
// Mixed-radix Stockham plan for a complex transform of length N = 2^a 3^b 5^c.
struct FFTPlan {
  int N;
  int nstages;
  int radix[16];
};

// One block (J, Omega, Lambda) of the state, as seen by the kernels.
struct DevBlock {
  int iJ;      // index of J in the batch
  int omega;   // helicity
  int lam;     // electronic state
  int up;      // block index of (J, Omega+1, Lambda), -1 if absent
  int dn;      // block index of (J, Omega-1, Lambda), -1 if absent
  int base;    // block index of (J, Omega, Lambda = 0)
  int coef;    // index of the (J, Omega) angular coefficient set
  int cutcol;  // first column of this block's psi(r*) values in the cut ring
  int nrow;    // angular functions of the block: ngamma - Omega (rows beyond are zero)
  int pad;
};

// Angular coefficient set of one (J, Omega): five rows of ngamma values, for
// row i (j = Omega + i):
//   [0] j(j+1)          [1] J(J+1) + j(j+1) - 2 Omega^2
//   [2] -lambda+_(J Omega) lambda+_(j Omega) kappa  (0 if no Omega+1 partner)
//   [3] -lambda-_(J Omega) lambda-_(j Omega) kappa  (0 if no Omega-1 partner)
//   [4] E_rot / lmax2(j)  (the g_j cap; 1e300 when lmax2 = 0)
constexpr int kCoefRows = 5;

// Per-J scalars used in the update epilogue.
struct DevJ {
  double e0s;     // E0 / dE
  double invdE;   // 1 / dE
  float e0s_f;    // the same rounded to FP32 (FP64 arithmetic is slow on this part)
  float invdE_f;
};

// Launch shapes chosen by the tuner (defaults in the context).
struct Tuning {
  int rows_pairs;   // line pairs per CTA of the R-direction kinetic kernel
  int cols_tile;    // columns per CTA of the r-direction kinetic kernel (even)
  int kb;           // Chebyshev iterations per energy-sum flush (ring depth)
  int use_graph;    // capture full chunks as CUDA graphs
  int use_tc;       // tensor-core gamma transform (mixed precision only)
  int kin_warp;     // kinetic kernels where the line length allows: 2 and 3 half-warp form
                    // (FP32, N = 128, 192, 256; else as 1; 3 exchanges the spectral partners
                    // by shuffles, 2 through shared memory), 1 warp-register FFT, 0
                    // shared-memory FFT
  int tc_persist;   // persistent tensor-core angular step (operands in tensor memory)
  int flush_tc;     // energy-sum flush on the tensor cores (mixed precision)
  int kin_fused;    // both radial kinetic terms in one launch (FP32, kin_warp = 2, half-warp
                    // line lengths in both directions): 0 separate kernels (the default:
                    // 0.302 against 0.310 ms per step on config 2, where both forms are
                    // bound by instruction issue), 1 automatic cluster size, 2/4/8 that many
                    // CTAs per (block, i) plane
  int up_direct;    // FP64 state uploads from page-locked, mapped host memory read by a kernel
                    // over the host link (1) or copied by the DMA engines (0, the default:
                    // 4.49 against 5.05 ms for both state vectors of config 2)
  int tc_tma;       // tile-major angular step: tile copies by TMA (1) or cp.async (0, the
                    // default: 0.380 against 0.399 ms per step on config 2)
  int prod_gather;  // product-channel node sums: stencil columns gathered plane-major first
                    // (1) or read as 4 x 4 stencils straight from the state (0)
  long tc_wait_limit;   // polls of the tile-major angular step's bounded waits (2^22; smaller
                        // values serve the failure-detection test)
};

// --------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError().
template <typename real>
cudaError_t launch_kinetic_rows(const real* q, real* t, long nrows, const FFTPlan& plan,
                                const void* tw, const void* ph, const real* lam, int pairs,
                                const DevBlock* blocks, int ng, int nr, int warp_fft,
                                cudaStream_t st);

template <typename real>
cudaError_t launch_kinetic_cols(const real* q, real* t, long nplanes, int nr, int NR,
                                const FFTPlan& plan, const void* tw, const void* ph,
                                const real* lam, int ctile, int ng,
                                // flux cut
                                const real* wpsi, const real* wdpsi, real* cut_slot,
                                const DevBlock* blocks, const int* ncut_J,
                                // column at R_inf for channel projections
                                int m_inf, real* qcol, int warp_fft, cudaStream_t st);

// t = K_R c + K_r c for every live plane in one launch of CS-CTA clusters, with the flux cut
// and the R_inf column (mw3_radial.cu). Returns false (nothing enqueued) where no fused
// shape applies; q == nullptr only asks. cs = 1 picks the cluster size.
bool kinetic_radial_fused(int NR, int nr, int cs, const float* q, float* t, long nplanes,
                          const void* twR, const void* phR, const float* lamR, const void* twr,
                          const void* phr, const float* lamr, int ng, const float* wpsi,
                          const float* wdpsi, float* cut, const DevBlock* blocks,
                          const int* ncut_J, int m_inf, float* qcol, cudaStream_t st,
                          cudaError_t* err);
int radial_fused_default_cs(int NR, int nr);

// out[b] = Tmat[omega(b)] in[b] (per block [ng x ng] x [ng x ncol]); Tmat is T (DVR ->
// FBR) or its transpose (FBR -> DVR), zero-padded to ng x ng.
template <typename real>
cudaError_t launch_gamma_forward(const real* q, real* c, const real* T, const DevBlock* blocks,
                                 int nblk, int ng, long ncol, cudaStream_t st);

// w = T^Omega (V u) per block, then the FBR combination and the damped update:
// u holds the DVR values of every block (u = (T^Omega)^T c_k), c = c_k.
template <typename real>
cudaError_t launch_gamma_update(const real* u, const real* T, const DevBlock* blocks, int nblk,
                                int ng, long ncol, int NR, const real* coef, const real* fr,
                                const real* fR, real erot, const real* ck, real* ckm1,
                                const real* t, const real* V, int nelec, const real* DR,
                                const real* Dr, const DevJ* dj, real alpha, real beta, int mode,
                                real* out, cudaStream_t st);

// cut[chan_col[c]] = sum_kr chi[c][kr] qcol[block(c)][row(c)][kr]  (0 before kmin), in FP64
// (products and sum) whatever the state's precision; cut is the FP64 channel ring.
template <typename real>
cudaError_t launch_channels(const real* qcol, const double* chi, const int* chan_block,
                            const int* chan_row, const int* chan_col, int nchan, int ng, int nr,
                            const long* d_iter, int slot, long kmin, double* cut_slot,
                            cudaStream_t st);

template <typename real>
cudaError_t launch_norms(const real* q, const long* J_begin, int nJ, double* partial,
                         int nchunk, double* out, cudaStream_t st);

// acc[j][0/1][e] += Re/Im f[k][iJ(e)][j] q[e] for k = *d_iter + slot < K (time-domain
// packets; FP64 sums and coefficients)
template <typename real>
cudaError_t launch_time_accum(const real* q, long n, long npts, const DevBlock* blocks,
                              const double* f, int nJ, int nt, long K, const long* d_iter,
                              int slot, double* acc, cudaStream_t st);

// Lanczos helpers on J segments: y += s c[iJ] x; y /= sqrt(c2[iJ]); b = sqrt(b2)
template <typename real>
cudaError_t launch_axpy_seg(real* y, const real* x, const double* c, double s, long n, long npts,
                            const DevBlock* blocks, cudaStream_t st);
template <typename real>
cudaError_t launch_rscale_seg(real* y, const double* c2, long n, long npts, const DevBlock* blocks,
                              cudaStream_t st);
cudaError_t launch_sqrt(const double* b2, double* b, int n, cudaStream_t st);

// out[iJ] = sum over J's element range of a * b, in FP64 (partial: [nJ][nchunk])
template <typename real>
cudaError_t launch_dots(const real* a, const real* b, const long* J_begin, int nJ,
                        double* partial, int nchunk, double* out, cudaStream_t st);

template <typename real>
cudaError_t launch_phases(const double* theta, int nJ, int nE, int kb, int nvalid,
                          const long* d_iter, real* ph, cudaStream_t st);

template <typename real>
cudaError_t launch_sums_flush(const real* ph, const real* cut, long ncut_total, int kb, int nvalid,
                              int nJ, int nE, const long* colbase, const long* ncols,
                              const long* accoff, long max_cols, double* acc, cudaStream_t st);

cudaError_t launch_advance(long* d_iter, long n, cudaStream_t st);
// Ring slots a probability read adds on the fly instead of flushing them first.
constexpr int kPeekMax = 8;
// The same for the mixed form's reads, which add only the change of the pending slots from an
// FP32 copy of the flushed accumulators (launch_flux_cross).
constexpr int kPeekMaxX = 16;
// out[iJ][e] = the same flux sum over A + Ph Cut for the npend pending ring slots (phases
// ph[iJ][2 nE][kb] of those slots already computed), A read only.
template <typename real>
cudaError_t launch_flux_reduce_peek(const double* acc, int nJ, int nE, const long* accoff,
                                    const long* ncols, const long* ncut, long max_ncut,
                                    const real* ph, int kb, int npend, const real* cut,
                                    long ncut_total, const long* colbase, double* part,
                                    double* out, cudaStream_t st);
cudaError_t launch_convert_d2f(const double* in, float* out, long n, cudaStream_t st);
// out[0, n) = (B) host[0, n), read by the device through the device alias of page-locked,
// mapped host memory (16-byte aligned).
template <typename B>
cudaError_t launch_host_read(const double* host_alias, B* out, long n, cudaStream_t st);
cudaError_t launch_convert_f2d(const float* in, double* out, long n, cudaStream_t st);

// Channel probabilities on the device (mw3_gamma.cu): output keys (J, Lambda, v, j) in
// CSR form over their channels; channel c reads the accumulator pair at col[c] (real row e,
// imaginary row nE + e, row stride ld[c]) with its energy eps[c] and J index chJ[c].
struct ChanTable {
  const long* key_first;   // nkeys + 1
  const int* key_chan;
  const int* chJ;
  const long* col;
  const long* ld;
  const double* eps;
  double mu;
  int nkeys;
};
cudaError_t launch_channel_probs(const double* acc, const ChanTable& t, const double* Ecol,
                                 double Eref, const double* theta, const double* dE,
                                 const double* a2, int nE, double* out, cudaStream_t st);

// Products-coordinate-based start (mw3_pcb.cu). The packet frame's Jacobi vectors are
// (r_s, R_s) = M (r, R); its diatom is a sine series sum_j coef[j] sin((j+1) pi (r_s - rsmin) / L)
// on (rsmin, rsmax); g(R_s) = N exp(-(R_s - R0)^2 / (2 G^2)) cos(k0 R_s); plc is the
// normalisation of P-bar_(om0)^(om0).
struct PcbParams {
  double M00, M01, M10, M11;
  double R0, G, k0, N;
  double rsmin, rsmax;
  int nrs;
  int j0, om0;
  int NR, nr, ng;
  double Rmin, dR, rmin, dr;
  double plc;
};
// One output block (J, Omega, Lambda0): T^J[Omega][Omega0] = (sign flips of the frame
// rotation) x (p1 d^J_(Omega0, Omega) + p2 d^J_(-Omega0, Omega)), the prefactors of the
// Jacobi form and the parity-adapted weights folded into p1, p2.
struct PcbTerm {
  int blk;
  int om;
  WignerIdx w1, w2;
  double p1, p2;
};
cudaError_t launch_pcb_packet(const PcbParams& p, const double* xw, const double* coef,
                              const PcbTerm* terms, int nterms, double* out, int nsm,
                              cudaStream_t st);

// Product-channel projection (mw3_products.cu): channels of one (J, Lambda', Omega').
struct ProdGroup {
  int b0;        // block index of (J, Omega = 0, Lambda')
  int bstride;   // block index step per Omega (= nelec)
  int nom;       // helicities of this J
  int op;        // Omega'
  long toff;     // offset of this J's helicity matrices [node][nom][nom]
  int c0, nc;    // rows [c0, c0 + nc) of the channel weight table
  int col0;      // cut-ring column of channel c0 (the group's channels are consecutive)
  int pad;
};

// jl_group[iJ * nelec + L] = index of the Omega' = 0 group of (J, Lambda'); chan[c] =
// (group, cut column) of product channel c; vbuf holds [groups][nn]. The projection is
// accumulated in FP64 whatever the state's precision: the state (real) times the Legendre
// rows (real) in partial sums of eight rows, FP64 across them and in every later stage
// (stencil weights, helicity rotation, Jacobian, channel dots); cut is the FP64 channel ring.
// Plane-major form of the node sums (tuning key "prod_gather"): the distinct (r, R) grid
// columns of all stencils, sorted (pts, padded to spad, a multiple of 32, with copies of the
// last column), are first gathered per block into G[b][s][i] (rows padded to ngp, a multiple
// of 32); node v then takes stencil point s (= 4 c + a) from row pix[v][s] of G with the
// weight wst[v][s] = wR_a wr_c. Unset (gather == nullptr): the stencils are read from q.
template <typename real>
struct ProdGather {
  const int* pts;
  const int* pix;
  const real* wst;
  real* G;
  int spad, ngp;
  const DevBlock* blocks;
  int nblk;
};

template <typename real>
cudaError_t launch_products(const real* q, int ng, int nr, int NR, int nn, const int* idx,
                            const double* w, const real* pl, int ltop, const double* T,
                            const double* jac, const ProdGroup* groups, const int* jl_group,
                            int njl, int max_nom, double* vbuf, const double* W, const int2* chan,
                            int nchan, double* cut_slot, const ProdGather<real>* gather,
                            cudaStream_t st);

// Fused tensor-core angular step (mw3_tc.cu), FP32 state, ngamma padded to kp <= 112.
struct TcArgs {
  const float* ck;
  float* ckm1;
  const float* t;
  const float* V;
  const float* T_hi;    // [omega][kp][kp]  T^Omega[i][n]       (GEMM 2 B: N = i, K = n)
  const float* T_lo;
  const float* Tt_hi;   // [omega][kp][kp]  T^Omega[i][n] at [n][i] (GEMM 1 B: N = n, K = i)
  const float* Tt_lo;
  const DevBlock* blocks;
  const float* coef;
  const float* fr;
  const float* fR;
  const float* DR;
  const float* Dr;
  const DevJ* dj;
  float* out;           // mode 1: H_s c
  double* npart;        // [group][tile] sums of squares of c_(k+1)
  int* err;             // set on a wait that timed out
  long wait_limit;      // polls of a bounded wait in the tile-major form (the wait for the MMAs
                        // of an expired phase before tensor memory is freed keeps 2^22)
  float erot, alpha, beta;
  long ncol, npts;
  int ng, kp, NR, nelec, mode, ntiles, tmem_cols;
  int ngroups;          // (J, Omega) groups
  int persistent;       // 1: one CTA per SM over a range of (group, tile) pairs;
                        // 2: the same with the parity-split operands (Tp_*);
                        // 3: parity-split with the operand matrices streamed (kh 64..96)
  int nsm;              // CTAs of the persistent forms
  int kh;               // parity-split operand size: n_gamma / 2 rounded up to 16
  const float* Tp_hi;   // [omega][4][kh][kh]: G1e, G1o, G2e, G2o (see mw3_tc.cu)
  const float* Tp_lo;
  // 2-D tensor maps (columns x rows = ncol x nblk ng, FP32, boxes of 128 x 8) of c_k, t
  // and c_(k-1) for the tensor-memory-accelerator tile copies of the tile-major form; set
  // by launch_angular_tc (tma = 1) when the driver provides the encoder
  int tma;
  CUtensorMap tm_ck;
  CUtensorMap tm_t;
  CUtensorMap tm_ckm1;
};
bool angular_tc2_supported(int kp, int nelec);
// Energy-sum flush on the tensor cores (FP32 ring, split-TF32, FP64 accumulators).
cudaError_t launch_flush_tc(const float* ph, const float* cut, long ncut_total, int kb, int nvalid, int nJ,
                            int nE, const long* colbase, const long* ncols, const long* accoff,
                            long max_cols, double* acc, int* err, cudaStream_t st);
int angular_tc3_kh(int ng, int nelec);   // 0 when the parity-split form does not apply
int angular_tc4_kh(int ng, int nelec);   // 0 when the streamed parity-split form does not apply
size_t angular_tc_smem(int kp);
cudaError_t launch_angular_tc(const TcArgs& args, int ngroups, const int* g_begin, int nJ,
                              double* norm_out, cudaStream_t st);
constexpr int kTcMaxKp = 112;

// out[iJ][e] = the flux sum of the J's cut columns (psi, dpsi) at energy e; `part` holds
// flux_partial_size(nJ, nE, max_ncut) doubles of per-chunk partial sums.
long flux_partial_size(int nJ, int nE, long max_ncut);
// acc32 (may be null): an FP32 copy of every accumulator value the reduction reads, written on
// the way (for launch_flux_cross).
cudaError_t launch_flux_reduce(const double* acc, int nJ, int nE, const long* accoff,
                               const long* ncols, const long* ncut, long max_ncut, double* part,
                               double* out, float* acc32, cudaStream_t st);
// Mixed form: out = fluxA + the flux change that the npend pending ring slots make, from the
// FP32 copy acc32 of the flushed accumulators (whose flux is fluxA) and the FP32 ring.
cudaError_t launch_flux_cross(const float* acc32, int nJ, int nE, const long* accoff,
                              const long* ncols, const long* ncut, long max_ncut, const float* ph,
                              int kb, int npend, const float* cut, long ncut_total,
                              const long* colbase, double* part, const double* fluxA, double* out,
                              cudaStream_t st);

}  // namespace mw3
