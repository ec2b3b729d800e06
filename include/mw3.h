/*
 * mw3.h - C ABI of libmw3, a GB300 (sm_103a) implementation of the damped real
 * Chebyshev wave-packet propagation of MADWAVE3 (Roncero & del Mazo-Sevillano,
 * arXiv 2412.10167) for A + BC collisions in reactant Jacobi coordinates.
 *
 * Conventions
 *   - Atomic units everywhere: bohr, hartree, electron masses (1 u = 1822.888486 m_e).
 *   - Every call returns MW3_OK (0) or a negative MW3_ERR_* code; no C++ exception
 *     crosses this boundary. mw3_last_error() gives a message for the last failure.
 *   - Host arrays passed in are caller-owned and copied before the call returns;
 *     host arrays passed out are caller-owned and must hold the stated number of
 *     elements. Device memory is owned by the context (allocated through the hook of
 *     mw3_set_allocator, else cudaMalloc) and released by mw3_destroy.
 *   - Call order: mw3_create -> [mw3_set_stream, mw3_set_allocator] -> mw3_grid ->
 *     mw3_load_potential | mw3_load_potential_grid -> mw3_init_packet ->
 *     mw3_set_absorber -> mw3_set_analysis -> mw3_propagate (any number of times;
 *     each call continues from the current iteration) -> mw3_flux_probabilities.
 *     A call out of order returns MW3_ERR_STATE.
 *   - Not thread-safe per context; distinct contexts are independent.
 *
 * State layout (device): q[block][gamma][r][R], R fastest. Blocks are ordered by
 * total angular momentum J (in the order given), then helicity Omega = 0..
 * min(J, omega_max) (parity p = (-1)^J), then electronic state Lambda.
 */
#ifndef MW3_H
#define MW3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  MW3_OK = 0,
  MW3_ERR_BAD_ARG = -1,   /* invalid argument (sizes, NULL, out of range)      */
  MW3_ERR_OOM = -2,       /* device or host allocation failed                  */
  MW3_ERR_CUDA = -3,      /* a CUDA runtime call or kernel launch failed        */
  MW3_ERR_DIVERGED = -4,  /* ||q_k||^2 exceeded 1.5 ||q_0||^2 (bad E_min/E_max) */
  MW3_ERR_SPECTRUM = -5,  /* grid energy range invalid (E_s outside (-1, 1))    */
  MW3_ERR_TIMEOUT = -6,   /* a bounded device wait gave up                     */
  MW3_ERR_STATE = -7,     /* call made out of order                            */
  MW3_ERR_IO = -8,        /* checkpoint file error                             */
  MW3_ERR_NAN = -9        /* NaN or Inf in user input                          */
};

/* Arithmetic of the propagation. MW3_FP64: FP64 state, transforms and sums.
 * MW3_MIXED: FP32 state, FP32 radial transforms, gamma transform on tensor cores
 * (FP32 accumulation), FP64 spectral scaling constants, FP64 energy sums. */
enum { MW3_FP64 = 0, MW3_MIXED = 1 };

typedef struct mw3_ctx mw3_ctx;

/* Grid, basis and block structure (Section 2.1 and the inputgridbase namelist of
 * Table 1). Radial grids: NR (nr) midpoint nodes R_m = Rmin + (m + 1/2) dR between
 * walls at Rmin and Rmax (sine DVR, regular at both walls); NR and nr must be even,
 * of the form 2^a 3^b 5^c and at most 1024. ngamma Gauss-Legendre points in
 * cos(gamma), 1 <= ngamma <= 256. J[0..nJ-1] is the batch of total angular
 * momenta, each with helicities 0..min(J, omega_max). nelec diabatic states
 * (1 or 2). masses = (m_A, m_B, m_C) for A + BC, r = B->C, R = c.o.m.(BC)->A. */
typedef struct {
  int NR;
  double Rmin, Rmax;
  int nr;
  double rmin, rmax;
  int ngamma;
  double masses[3];
  int nJ;
  const int* J;
  int omega_max;
  int nelec;
} mw3_grid_desc;

/* Initial collision packet (Section 2.3.1, Eqs. initial-collision-wvp and
 * initial-gaussian): N g(R) chi_{v0 j0}(r) y_{j0 Omega0}(gamma) in the block
 * (Omega0, elec0) of every J, g(R) = exp(-(R-R0)^2/(2 Gamma^2)) cos(k0 R),
 * k0 = sqrt(2 mu Ecol). chi from the diatomic Hamiltonian at R = 100 bohr. */
typedef struct {
  double R0, Gamma, Ecol;
  int v0, j0, omega0, elec0;
} mw3_packet_desc;

/* Products-coordinate-based (PCB) start (Section 2.4, the first of its two routes to
 * state-to-state probabilities, iprod = 1): the grid of the context is the PRODUCT
 * arrangement and the packet of mw3_packet_desc lives in another arrangement, named in the
 * grid's atom labels (grid: A + BC, r = C - B, R from the BC centre of mass to A):
 *   arrangement  1: the packet's diatom is A-C (r_s = C - A, R_s from the AC centre of mass
 *                to B); 2: A-B (r_s = B - A, R_s to C); 0: the grid's own (a test case)
 *   rmin, rmax, nr  the sine DVR (midpoint nodes) of the packet's diatom, 4 <= nr <= 4096 */
typedef struct {
  int arrangement;
  double rmin, rmax;
  int nr;
} mw3_pcb_desc;

/* Energy analysis (Section 2.4 and the inputflux/inputtime namelists):
 * nE collision energies E_i = linspace(E_lo, E_hi, nE) (inclusive), flux through
 * r = rstar (Eq. total-flux), reactant channels (Lambda, v <= vmax, j <= jmax,
 * Omega) projected at the R node nearest Rinf, counted from iteration kmin
 * (kminelastic). Set vmax < 0 for no channel analysis. */
typedef struct {
  double rstar;
  double E_lo, E_hi;
  int nE;
  double Rinf;
  int vmax, jmax;
  long kmin;
} mw3_analysis_desc;

/* Product channels (Section 2.4, Eqs. final-states, Chebyshev-products-overlaps and
 * S-matrix-from-chebyshev; the inputprod namelist): overlaps of q_k with the
 * product states chi_(v'j')(r') P-bar_(j')^(Omega')(cos gamma') on the surface
 * R' = Rinf, for the wave packet held in reactant Jacobi coordinates. The surface
 * integral uses a product quadrature (the nr midpoint sine-DVR nodes of
 * [rmin, rmax] times ngamma Gauss-Legendre nodes); at each node the reactant
 * function is interpolated (4-point Lagrange in R and r, its Legendre series in
 * gamma) and its helicity components rotated into the product frame with the
 * Wigner matrix d^J of the angle between R and R' (parity (-1)^J; helicities
 * above omega_max are zero in both frames), times the Jacobian r'R'/(rR).
 *   arrangement  1: products AC + B (r' = C - A); 2: products AB + C (r' = B - A)
 *   vmax, jmax   channels v' <= vmax, j' <= jmax, Omega' <= min(j', J, omega_max),
 *                for every electronic state (product states from V_LL with the
 *                departing atom 100 bohr away; needs a potential callback)
 * Every node's reactant point must lie inside the grid; stencil points beyond the
 * ends of the grid count as zero. */
typedef struct {
  int arrangement;
  double Rinf;
  int nr;
  double rmin, rmax;
  int ngamma;
  int vmax, jmax;
} mw3_products_desc;

/* Potential callback (the potelebond routine of Section 4, in Jacobi form):
 * given r, R (bohr) and cos(gamma) write the nelec x nelec diabatic matrix
 * (hartree, row-major, symmetric) into potmat; return 0 on success. */
typedef int (*mw3_pot_fn)(double r, double R, double cosg, double* potmat, void* user);

/* Device allocator hook: alloc returns a device pointer (256-byte aligned) or NULL. */
typedef void* (*mw3_alloc_fn)(size_t bytes, void* user);
typedef void (*mw3_free_fn)(void* ptr, void* user);

/* Sato LEPS surface parameters (hartree, bohr) for the built-in mw3_pes_leps. */
typedef struct {
  double D, beta, re, delta;   /* shared pair curve and Sato parameter           */
  double masses[3];            /* m_A, m_B, m_C (m_e) to map Jacobi -> bonds     */
  int two_state;               /* 0: one surface; 1: diabatic pair (below)       */
  double bump, bump_r0, bump_w2;           /* V22 = V11 + bump exp(-(r-r0)^2/w2) */
  double coup, coup_R0, coup_r0, coup_w2;  /* V12 = coup exp(-((R-R0)^2+(r-r0)^2)/w2) */
} mw3_leps_params;

/* ------------------------------------------------------------------ lifecycle */

/* Create a context on CUDA device `device` with precision MW3_FP64 or MW3_MIXED.
 * *out receives the handle (NULL on failure). */
int mw3_create(mw3_ctx** out, int device, int precision);

/* Release every device and host resource of the context. NULL is ignored. */
void mw3_destroy(mw3_ctx* ctx);

/* Message for the last failing call on ctx (or of mw3_create when ctx is NULL). */
const char* mw3_last_error(const mw3_ctx* ctx);

/* Text for a status code. */
const char* mw3_status_string(int status);

/* Launch every kernel on `stream` (a cudaStream_t; NULL = legacy default stream). */
int mw3_set_stream(mw3_ctx* ctx, void* stream);

/* Route device allocations through alloc/free (must precede mw3_grid). */
int mw3_set_allocator(mw3_ctx* ctx, mw3_alloc_fn alloc, mw3_free_fn free_fn, void* user);

/* -------------------------------------------------------------------- set-up */

/* Build grids, bases and the block table (Section 2.1). Copies desc->J. */
int mw3_grid(mw3_ctx* ctx, const mw3_grid_desc* desc);

/* Evaluate the potential on the grid through fn (Section 4, potelebond), cap the
 * diagonal at vcut (VcutmaxeV), and set the radial kinetic cap tcut_rad
 * (radcutmaxeV) and the rotational cap ecut_rot (rotcutmaxeV); then compute the
 * spectral bounds E_min, E_max of each J (Section 2.2, H_s). */
int mw3_load_potential(mw3_ctx* ctx, mw3_pot_fn fn, void* user, double vcut, double tcut_rad,
                       double ecut_rot);

/* Same with a caller-owned host grid V[nelec][nelec][ngamma][nr][NR] (hartree,
 * uncapped; symmetric in the state indices), copied in. */
int mw3_load_potential_grid(mw3_ctx* ctx, const double* V, double vcut, double tcut_rad,
                            double ecut_rot);

/* Built-in Sato LEPS (+ optional two-state extension); user = mw3_leps_params*.
 * Energies are shifted by +D so that A + BC(re) is zero; bond lengths are
 * clamped to >= 0.25 bohr as in the example potential routine of Section 6.1. */
int mw3_pes_leps(double r, double R, double cosg, double* potmat, void* user);

/* Solve the diatomic states and write q_0 (Section 2.3.1); resets the iteration
 * counter and every energy sum. */
int mw3_init_packet(mw3_ctx* ctx, const mw3_packet_desc* desc);

/* PCB start (Section 2.4, iprod = 1; packet of Section 2.3.1): the packet
 * g(R_s) chi_(v0 j0)(r_s) P-bar_(j0)^(Omega0)(cos gamma_s) of `desc`, in its own arrangement
 * `src` (mw3_pcb_desc), is evaluated once at every node of the context's grid (the product
 * arrangement) on the device: the packet's Jacobi coordinates from the grid's, every helicity
 * Omega = 0..min(J, omega_max) of every J from the rotation between the two body frames
 * (parity-adapted Wigner d^J; Omega0 must be a block of every J), the Jacobian
 * r R / (r_s R_s), then the gamma transform to each block's FBR. g is normalised in closed
 * form (int g^2 dR = 1, k0 = sqrt(2 mu_s Ecol), mu_s the packet's reduced mass of R_s); chi
 * is the packet diatom's state (departing atom 100 bohr away on its axis; needs a potential
 * callback) as its sine interpolant. E_(v0 j0) is that diatom's level, so the energy grid of
 * mw3_set_analysis is E_col + E_(v0 j0), and |a(E)|^2 becomes the closed-form Gaussian
 * integral with mu_s. The grid's own channel analysis (mw3_set_analysis: vmax, jmax at Rinf)
 * then gives the state-to-state probabilities of the product arrangement; set kmin = 0.
 * Resets the iteration counter and every energy sum. Device scratch: two FP64 state-sized
 * buffers (one in the FP64 form), freed before the return. Synchronous.
 * MW3_ERR_BAD_ARG for an invalid description, MW3_ERR_STATE before mw3_load_potential. */
int mw3_init_packet_pcb(mw3_ctx* ctx, const mw3_packet_desc* desc, const mw3_pcb_desc* src);

/* Damping exp(-phi), phi = A_R (R-RI)^nR for R > RI plus A_r (r-rI)^nr for r > rI
 * (Eq. imaginary-potential, inputabsorcion namelist). */
int mw3_set_absorber(mw3_ctx* ctx, double RI, double AR, int nR, double rI, double Ar, int nr);

/* Energy grid, flux surface and reactant channels (Section 2.4); allocates the
 * energy-sum accumulators. Must follow mw3_init_packet (needs E_{v0 j0}). */
int mw3_set_analysis(mw3_ctx* ctx, const mw3_analysis_desc* desc);

/* Enable product channels (call after mw3_init_packet and before mw3_set_analysis;
 * NULL disables them). MW3_ERR_BAD_ARG for an invalid description, a grid potential
 * without a callback, or a node outside the grid. */
int mw3_set_products(mw3_ctx* ctx, const mw3_products_desc* desc);

/* --------------------------------------------------------------- propagation */

/* Advance nsteps Chebyshev iterations of Eq. (wvp-k):
 *   q_1 = D H_s q_0,  q_{k+1} = D (2 H_s q_k - D q_{k-1}),
 * accumulating c_k(E) = (2 - delta_k0) exp(-i k theta_E) times the flux cut and
 * the channel overlaps of q_k into the energy sums (Eqs. wvf-chebyshev and
 * chebyshev-expansion-constants). Returns MW3_ERR_DIVERGED if a norm exceeds
 * 1.5 ||q_0||^2. Synchronous: returns after the work is complete. */
int mw3_propagate(mw3_ctx* ctx, long nsteps);

/* Number of iterations done so far (k of the current q_k). */
long mw3_iteration(const mw3_ctx* ctx);

/* ------------------------------------------------------------------- results */

/* Probabilities from the sums so far (Eqs. total-flux, S-matrix-from-chebyshev):
 *   E[nE]            collision energies (hartree);
 *   Ptot[nJ * nE]    total reaction probability through r* per J;
 *   Pinel[nJ * nelec * (vmax+1) * (jmax+1) * nE] or NULL: reactant-channel
 *                    probabilities summed over Omega, zero for closed channels.
 * Every iteration run so far counts. Iterations still in the energy ring (a propagation that
 * stopped between flushes) are added on the fly when there are at most eight (MW3_FP64) or
 * sixteen (MW3_MIXED) of them, else flushed first; the |S|^2 assembly runs on the device and
 * only the results are copied back. The flux of the flushed sums is kept until the next flush; in MW3_MIXED the first
 * read after a flush also keeps an FP32 copy of the flux accumulators (half their size) from
 * which later reads add the pending iterations. Synchronous. */
int mw3_flux_probabilities(mw3_ctx* ctx, double* E, double* Ptot, double* Pinel);

/* Copy q_k (and q_{k-1} if qprev != NULL) to host FP64 arrays of
 * nblocks * ngamma * nr * NR elements. */
int mw3_get_state(mw3_ctx* ctx, double* q, double* qprev);

/* Overwrite q_k and q_{k-1} (host FP64, same size; qprev == NULL sets q_{k-1} = 0) without
 * touching the sums. Synchronous; the caller's arrays are not read after the return. The
 * values cross to the device in four block groups on a library-owned stream, each group's
 * DVR -> FBR transform overlapping the next group's transfer. An array that lies wholly
 * inside one page-locked host allocation mapped into the device's address space
 * (cudaHostAlloc, cudaHostRegister; 16-byte aligned) is read by a kernel over the host link
 * and narrowed to the state's precision on the way (tuning key "up_direct"); any other
 * array is copied by the DMA engines into a staging buffer first. Both give the same bits. */
int mw3_set_state(mw3_ctx* ctx, const double* q, const double* qprev);

/* mw3_set_state for FP32 host arrays (same sizes and layout): half the bytes over the host
 * link. In MW3_MIXED the values are the FP32 state itself (the FP64 form of mw3_set_state
 * rounds to them on the device, so both give the same state for FP32-representable input);
 * in MW3_FP64 they are widened exactly. Synchronous; always copied by the DMA engines. */
int mw3_set_state_f32(mw3_ctx* ctx, const float* q, const float* qprev);

/* out[i] = (H_s q)[i] for a host FP64 vector q (one application of the scaled
 * Hamiltonian through the same kernels as a propagation step). */
int mw3_apply_hs(mw3_ctx* ctx, const double* q, double* out);

/* ||q_k||^2 per J after each iteration: out[nJ * n] for the last n iterations
 * (n <= mw3_iteration); returns the count written. */
long mw3_norm_trace(mw3_ctx* ctx, double* out, long n);

/* Photodissociation analysis (Section 2.3.2, Eqs. initial-photo-wvp, fourier-transform and
 * chebyshev-transform; Section 2.5, Eq. spectrum). The initial packet d.e |Psi_bound>,
 * projected onto the final state's body-fixed functions, is supplied by the caller as the
 * state (mw3_set_state at k = 0). mw3_enable_autocorrelation then keeps a device copy of
 * that state as Psi(k=0) and makes every later iteration add one FP64 inner product per J,
 * C_k = <Psi(0)|Psi(k)> (k = 0, 1, ...; read back at each ring boundary). It returns
 * MW3_ERR_STATE unless the analysis is set and the context is at k = 0; mw3_init_packet
 * switches it off. The autocorrelation is not part of checkpoints.
 *   mw3_autocorrelation: C[k * nJ + iJ] for k < min(n, recorded); returns the count.
 *   mw3_photo_spectrum:  a0[iJ * nE + e] = (1/pi) sum_k (2 - delta_k0) cos(k arccos E_s)
 *                        C_k / (dE sqrt(1 - E_s^2)), E_s = (E[e] - E0_J)/dE_J, for total
 *                        energies E (hartree) inside each J's spectral range (else
 *                        MW3_ERR_BAD_ARG); host FP64, caller-owned arrays. The cross
 *                        section of Eq. spectrum is proportional to h nu times a0. */
int mw3_enable_autocorrelation(mw3_ctx* ctx);
long mw3_autocorrelation(mw3_ctx* ctx, double* C, long n);
int mw3_photo_spectrum(mw3_ctx* ctx, const double* E, int nE, double* a0);

/* Time-domain packets (Section 2.2, Eqs. wvf-chebyshev and chebyshev-expansion-constants):
 * Psi(t_j) = sum_k f_k(t_j) Psi(k), f_k(t) = (2 - delta_k0) exp(-i E0 t) (-i)^k J_k(t dE)
 * (hbar = 1, E0 and dE of each J), for nt times t[j] >= 0 (atomic units). Enabled at k = 0
 * (MW3_ERR_STATE otherwise, or before mw3_set_analysis); every later iteration k < K adds
 * its term to FP64 accumulators on the device (2 nt state vectors of FP64), where K is the
 * first index beyond which every |J_k(t_j dE)| < 1e-17 (Bessel functions by Miller's
 * backward recurrence). The packets are exact for the undamped recursion once K
 * iterations have run. mw3_init_packet switches the accumulation off.
 *   mw3_time_packets: out[(j * 2 + c) * nblocks * ppb + ...] grid values (c = 0 real,
 *                     1 imaginary part), host FP64, caller-owned; *kmax = K (may be NULL). */
int mw3_enable_time_packets(mw3_ctx* ctx, int nt, const double* t);
int mw3_time_packets(mw3_ctx* ctx, double* out, long* kmax);

/* Bound states by non-orthogonal Lanczos (Section 2.3.2: the bound-state program that
 * supplies photodissociation initial states applies the same grid Hamiltonian in the
 * iterative non-orthogonal Lanczos method of Cullum and Willoughby). m steps of the plain
 * three-term recursion on H_s, on the device in the FBR coordinates of the state, without
 * reorthogonalisation, from the start vector v0 (host FP64 grid values of every block,
 * normalised per J; the blocks of different J are independent). FP64 contexts give the
 * eigenvalues to ~1e-10 dE, mixed contexts to the FP32 rounding of the recursion.
 *   mw3_lanczos:       alpha[i * nJ + iJ], beta[i * nJ + iJ] (i < m; beta_i couples
 *                      v_i and v_(i+1)), caller-owned.
 *   mw3_bound_states:  eigenvalues (hartree) of each J accepted by the Cullum-Willoughby
 *                      test (a cluster of numerically equal copies counts once; a simple
 *                      eigenvalue of T_m that is also one of T_m without its first row and
 *                      column is spurious) inside [emin, emax]: E[iJ * maxev + k],
 *                      k < count[iJ] <= maxev.
 *   mw3_bound_state_vector: the Ritz vector of J index iJ nearest the eigenvalue E, from a
 *                      second run of the recursion: out = grid values (every block; zero
 *                      outside J), normalised.
 * All three allocate work vectors on the device and leave the propagation state alone. */
int mw3_lanczos(mw3_ctx* ctx, const double* v0, int m, double* alpha, double* beta);
int mw3_bound_states(mw3_ctx* ctx, const double* v0, int m, double emin, double emax, int maxev,
                     double* E, int* count);
int mw3_bound_state_vector(mw3_ctx* ctx, const double* v0, int m, int iJ, double E, double* out);

/* Sizes and scaling constants: nblocks, points per block, E0 and dE per J. */
int mw3_sizes(const mw3_ctx* ctx, long* nblocks, long* points_per_block);
int mw3_spectral_range(const mw3_ctx* ctx, double* E0, double* dE);

/* Energy of the initial diatomic state E_{v0 j0} (hartree). */
int mw3_reference_energy(const mw3_ctx* ctx, double* Ev0j0);

/* Write / read a restart file: q_k, q_{k-1}, k, the energy sums and a hash of the
 * configuration (the ncontfile option of Table 1). */
int mw3_checkpoint_save(mw3_ctx* ctx, const char* path);
int mw3_checkpoint_load(mw3_ctx* ctx, const char* path);

/* |a(E)|^2 of the initial packet's incoming part at the analysis energies (Eq.
 * initial-flux-collisions; the denominator of every probability): a2[nE], caller-owned. */
int mw3_incoming_amplitude(mw3_ctx* ctx, double* a2);

/* State-resolved product probabilities |S|^2 (Eq. S-matrix-from-chebyshev, with the
 * flux normalisation of the reactant channels: (2 pi K'/mu') |C_E|^2 / |a(E)|^2,
 * K' = sqrt(2 mu' (E - e_(v'j'))), closed channels 0), summed over Omega':
 * P[((iJ * nelec + L) * (vmax + 1) + v) * (jmax + 1) + j][e], caller-owned host
 * array. MW3_ERR_STATE if product channels are not enabled. */
int mw3_product_probabilities(mw3_ctx* ctx, double* P);

/* Launch-shape and scheduling knobs (the autotuner's hook). Keys:
 *   "kb"         Chebyshev iterations per energy-sum flush (1..1024; before mw3_set_analysis)
 *   "rows_pairs" line pairs per CTA of the R-direction kinetic kernel (1..16)
 *   "cols_tile"  R columns per CTA of the r-direction kinetic kernel (even, 2..64)
 *   "use_graph"  0/1: replay full chunks as CUDA graphs
 *   "use_tc"     0/1: tensor-core gamma transform in MW3_MIXED
 *   "tc_persist" form of the tensor-core angular step: 0 one tile per CTA; 1 persistent
 *                (one CTA per SM, T^Omega resident in shared memory, operands in tensor
 *                memory); 2 persistent with the Gauss-Legendre parity split (even
 *                ngamma <= 96); 4 (default) the parity split walked tile-major with the
 *                Coriolis neighbours kept on chip (one electronic state); each falls back
 *                to the next lower form that applies. Even ngamma 98..192 always use the
 *                streamed parity split.
 *   "flush_tc"   0/1: energy-sum flush on the tensor cores in MW3_MIXED (split-TF32 within
 *                a flush, FP64 accumulators); default 1
 *   "kin_warp"   radial kinetic kernels: 2 (default) and 3 the half-warp FFT form in
 *                MW3_MIXED for line lengths 128, 192, 256 (spectral partners through
 *                shared memory, or by shuffles), else as 1; 1 warp-register FFT kernels for
 *                line lengths 32 R (R = 1, 2, 3, 4, 6, 8, 12, 16; FP64 up to R = 8); 0 the
 *                shared-memory FFT kernels
 *   "kin_fused"  with kin_warp 2 in MW3_MIXED, both radial kinetic terms, the flux cut and
 *                the R_inf column in one launch of thread-block clusters, each cluster one
 *                (block, i) plane (NR and nr in {128, 192, 256}): 1 cluster size chosen by
 *                the library, 2, 4 or 8 that size, 0 (default) the two separate kernels;
 *                shapes without a fused form use the separate kernels
 *   "up_direct"  0/1: mw3_set_state reads page-locked, mapped host arrays with a kernel
 *                (default 0: the DMA engines were faster over this host link);
 *                "up_direct_last" (read only) is 1 when the last upload did
 *   "tc_tma"     0/1: tile copies of the tile-major angular step by the tensor memory
 *                accelerator (2-D tensor maps) instead of cp.async; default 0
 *   "prod_gather" 0/1: product-channel node sums (Section 2.4) in the plane-major form: the
 *                distinct grid columns of all interpolation stencils are first copied, per
 *                block, into rows that hold all FBR rows of a column contiguously (1, the
 *                default), or the stencils are read from the state directly (0); both sum
 *                the stencil terms in the state's precision and the rest in FP64;
 *                "prod_points" (read only) is the number of distinct stencil columns
 *   "tc_wait_limit" 0..2^22: polls of each bounded mbarrier wait of the tile-major angular
 *                step (default 2^22). A wait that runs out makes its CTA stop, wait (with the
 *                full 2^22 bound) for the tensor-core work already committed, free its tensor
 *                memory and set the error word that mw3_propagate returns as
 *                MW3_ERR_TIMEOUT; 0 makes every wait run out (the failure-detection test).
 *                The context is not usable for propagation after a timeout; the device is.
 * Values outside a key's range return MW3_ERR_BAD_ARG. mw3_get_tuning reads a key. */
int mw3_set_tuning(mw3_ctx* ctx, const char* key, long value);
long mw3_get_tuning(const mw3_ctx* ctx, const char* key);

/* Per-kernel CUDA-event timing of the last mw3_propagate call, summed:
 * names[i] (static strings), ms[i], launches[i] for i < *count (in/out capacity).
 * "pcb_packet" times the one-off transform of mw3_init_packet_pcb while the timers are on. */
int mw3_kernel_times(mw3_ctx* ctx, int enable, const char** names, double* ms, long* launches,
                     int* count);

/* ------------------------------------------------- J-interpolation surrogate
 * A small fully connected network (n_in -> depth x width, GELU -> 1) trained with
 * hand-written kernels on probabilities P_J(E, v', j') that the propagation produced
 * at a coarse set of J, to predict intermediate J for the partial-wave sums of
 * Eqs. collisional-xsection and cumulative-probability (the paper interpolates
 * with J-shifting, Eq. J-shifting-interpolation; the network is this library's
 * extension). Weights in BF16 for the products, FP32 master weights, AdamW
 * moments, activations and accumulation. Flat parameter order: for each layer
 * W (row-major [out][in]) then b. Host arrays are caller-owned and copied. */
typedef struct mw3_mlp mw3_mlp;

/* He-normal initialisation from `seed` (zero biases). */
int mw3_mlp_create(mw3_mlp** out, int device, int n_in, int width, int depth,
                   unsigned long long seed);
void mw3_mlp_destroy(mw3_mlp* net);
const char* mw3_mlp_last_error(const mw3_mlp* net);
long mw3_mlp_num_params(const mw3_mlp* net);

/* Replace / read the FP32 master parameters (flat[mw3_mlp_num_params]); setting
 * them resets the optimiser state. */
int mw3_mlp_set_params(mw3_mlp* net, const double* flat);
int mw3_mlp_get_params(mw3_mlp* net, double* flat);

/* y[i] = network(X[i][0..n_in-1]) for i < n (X row-major FP32). */
int mw3_mlp_forward(mw3_mlp* net, const float* X, long n, float* y);

/* Mean-squared error over the n samples and its gradient (flat, may be NULL). */
int mw3_mlp_loss_grad(mw3_mlp* net, const float* X, const float* y, long n, double* loss,
                      double* grad);

/* `epochs` passes of minibatch AdamW (beta1 0.9, beta2 0.999, eps 1e-8; decoupled
 * weight decay `wd` on weights), shuffled by `seed`; *final_loss = mean batch loss of
 * the last epoch. */
int mw3_mlp_train(mw3_mlp* net, const float* X, const float* y, long n, int epochs, int batch,
                  double lr, double wd, unsigned long long seed, double* final_loss);

/* Allocation-free sums of squares, for callers that cannot call cudaMalloc (a fixed
 * memory arena, a region where allocating would stall other streams). The paper has
 * no counterpart: this is the per-J norm reduction of the propagation (its divergence
 * check, ||q_k||^2) with the partial-sum scratch in a 128 KB file-scope device array
 * instead of context memory. out[s] = sum_i x[s * seg_len + i]^2 for s < nseg.
 *   x    device FP64 [nseg * seg_len], caller-owned;  out  device FP64 [nseg].
 *   nseg 1..64 (the array's capacity); other values return MW3_ERR_BAD_ARG.
 * Enqueued on `stream` (a cudaStream_t, NULL = legacy default); returns without
 * synchronising. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it with the current
 * CUDA context; a call under a different context (after cudaDeviceReset, say) looks
 * it up again. Make the first call of each context before any stream capture.
 * Returns MW3_ERR_CUDA when one of its own two launches fails (an error left pending
 * by earlier work is not reported or cleared). All calls share the array; calls that
 * overlap on the GPU race. */
int mw3_norms_noalloc(const double* x, long seg_len, int nseg, double* out, void* stream);

/* Diagnostic: achieved FMA throughput of this GPU in TFLOP/s from an FMA-chain
 * kernel (kind 0 = FP64, 1 = FP32), the ALU roofline of the CUDA-core kernels.
 * Allocates 8 KB of device memory for the duration of the call. */
int mw3_measure_peak(int device, int kind, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* MW3_H */
