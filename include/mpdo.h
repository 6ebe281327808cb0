/*
 * mpdo.h -- C ABI of the GB300 noisy neutral-atom MPDO library (libmpdo.so).
 *
 * Method: arXiv:2309.08572 ("Simulating Large One-Dimensional Neutral Atom Quantum
 * Systems").  The state is a matrix product density operator (Sec. III.C, Fig. 3a):
 * rho = sum_k X_k X_k^+, stored as site tensors A_n[l][s][k][r] (left bond l, atom
 * level s in {0:|0>, 1:|1>, 2:|r>}, inner/Kraus index k, right bond r; r fastest).
 * A two-site channel is applied by contracting the two site tensors with the channel
 * and splitting back by a truncated SVD (Sec. III.A, Fig. 2c, Fig. 6a); the inner
 * index of the new orthogonality centre is truncated with the purity-preserving
 * scheme (Sec. III.D, Eqs. xiformula and ppt, App. B).  Energies, success probability
 * and samples come from transfer-matrix contractions (Sec. IV, Eq. tfim_hamiltonian,
 * qubit trace in Sec. IV.A).
 *
 * Conventions for every entry point:
 *  - Returns MPDO_OK (0) or a negative MPDO_ERR_* code; no C++ exception crosses the ABI.
 *  - Host pointers passed in are borrowed for the duration of the call only.
 *  - "host" arrays are ordinary CPU memory; "device" arrays live in GPU memory.
 *  - complex numbers are (re, im) pairs of doubles, interleaved, row-major.
 *  - All work is enqueued on the handle's CUDA stream; calls that return host
 *    results synchronise that stream before returning.
 *  - mpdo_last_error(h) describes the last failure on handle h (valid until the next
 *    call on h); mpdo_last_error(NULL) describes the last handle-less failure.
 */
#ifndef MPDO_H
#define MPDO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MPDO_OK = 0,
  MPDO_ERR_ARG = -1,      /* invalid argument (sizes, sites, null pointers, layout)   */
  MPDO_ERR_OOM = -2,      /* device allocation failed                                  */
  MPDO_ERR_CUDA = -3,     /* a CUDA call failed (message in mpdo_last_error)           */
  MPDO_ERR_NUMERIC = -4,  /* NaN/Inf in inputs or state, zero state, non-PSD Gram     */
  MPDO_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up                        */
  MPDO_ERR_STATE = -6     /* op does not touch the orthogonality centre, etc.          */
};

/* Arithmetic of the hot path.
 *  MPDO_FP64 : complex128 state, FP64 GEMMs and FP64 Jacobi eigensolves.
 *  MPDO_C64  : complex64 state, FP32 GEMMs (FP32 accumulation), FP32 Jacobi;
 *              cutoff, PPT and trace renormalisation in FP64 scalars.  With
 *              mpdo_config.gram_fp64 = 1 the Grams and the small matrices are FP64.
 *  MPDO_TF32X3, MPDO_BF16X3 : complex64 state as MPDO_C64, with every complex64 product
 *              of at least 2^21 complex multiply-adds run on the tensor cores (tcgen05.mma,
 *              TMA-fed) in split precision: operands x = hi + lo in TF32 (resp. BF16),
 *              hi*hi + hi*lo + lo*hi accumulated in FP32 (~2^-22 resp. ~2^-16 relative per
 *              product).  gram_fp64 = 0: the Grams are such products too, and the numerical
 *              floor of the cuts is 10 x 2.4e-7 (TF32X3) resp. 10 x 1.5e-5 (BF16X3) of the
 *              largest weight.  gram_fp64 = 1: the mixed form (FP64 Grams and small
 *              matrices) with its FP32 products -- the new centre B_j, the inner isometry,
 *              sampling -- on the tensor cores.
 *              The routing threshold can be changed with the environment variable
 *              MPDO_TC_MIN_MACS (read at create; 0 routes every product). */
typedef enum { MPDO_FP64 = 0, MPDO_C64 = 1, MPDO_TF32X3 = 2, MPDO_BF16X3 = 3 } mpdo_prec;

typedef struct mpdo_ctx* mpdo_t;   /* opaque; the handle owns its device memory (allocated
                                      through the config's hooks when given)              */

typedef struct {
  int n_sites;          /* N >= 2                                                       */
  int d;                /* local dimension; must be 3 (|0>,|1>,|r>)                    */
  int chi_max;          /* bond dimension cap chi (1..1024)                             */
  int k_max;            /* inner (Kraus) dimension cap K (1..1024)                      */
  int m_max;            /* largest Kraus count of any two-site op that will be applied */
  mpdo_prec prec;
  double sv_cutoff;     /* bond values with s <= sv_cutoff*s_max are dropped (<=0: default) */
  double kraus_cutoff;  /* inner values with sqrt(w) <= kraus_cutoff*sqrt(w_max) dropped   */
  int use_ppt;          /* 1: purity-preserving inner truncation; 0: plain + trace renorm  */
  void* cuda_stream;    /* cudaStream_t to use; NULL = a non-blocking stream the handle owns
                           (pass cudaStreamLegacy to run on the legacy default stream)   */
  int gram_fp64;        /* MPDO_C64, MPDO_TF32X3, MPDO_BF16X3.  1 = mixed precision: the Gram matrices (a2, a8)
                           are formed from the FP32 tensors with FP64 products and sums, and
                           everything derived from them (Jacobi eigenpairs, bond factors,
                           Phi and H, the cuts, PPT) is FP64; site tensors and the large
                           contractions stay FP32.  The numerical floor of the cuts drops
                           from ~6e-7 to ~1e-13 of the largest weight.  Ignored otherwise. */
  int order;            /* sweep order of the layers (reading of Sec. IV, blocks "applied
                           sequentially"): 0 = left to right -- when a layer's first two-site op
                           is on bond (0,1) and the orthogonality centre is elsewhere, the centre
                           is first moved to site 0 by identity two-site updates (truncated
                           with the handle's cuts), so every layer can run left to right;
                           1 = snake -- ops must touch the centre, layers alternate direction
                           (as the QAOA layer builder orders them).  Both give the same result
                           for snake-ordered layers.                                        */
  /* Device-memory hooks.  When alloc is non-NULL every device buffer the handle owns is
   * obtained as alloc(bytes, alloc_ctx) and returned with free(ptr, alloc_ctx) (free must
   * then be non-NULL too), so an outside allocator (e.g. a framework's caching allocator)
   * owns the memory; alloc returns NULL when it cannot serve the request, which the call
   * reports as MPDO_ERR_OOM.  NULL hooks: cudaMalloc / cudaFree. */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
} mpdo_config;

/* One op of a layer.  kind 2: two-site channel on (site, site+1) with n_kraus Kraus
 * operators E_m, each 9x9 on the index s_site*3 + s_{site+1}; kind 1: one-site unitary
 * (n_kraus must be 1) on `site`, 3x3.  ops points to n_kraus*(d^k)^2 complex numbers
 * (host, complex128 interleaved, row-major per operator). */
typedef struct {
  int kind;
  int site;
  int n_kraus;
  const double* ops;
} mpdo_op;

typedef struct {
  int n_ops;
  const mpdo_op* ops;   /* applied in array order */
} mpdo_layer;

/* Per-call truncation statistics (accumulated over the call's updates). */
typedef struct {
  double disc_bond_w;     /* sum over updates of discarded bond weight / total         */
  double disc_kraus_w;    /* sum over updates of discarded inner weight / total        */
  double ppt_theta_min;   /* smallest PPT cone angle used (rad)                          */
  int ppt_infeasible;     /* updates where PPT had no solution and used theta = 0       */
  int ppt_clamped;        /* negative PPT values clamped to zero                         */
  int chi_used_max;       /* largest bond dimension kept                                 */
  int k_used_max;         /* largest inner dimension kept                                */
  int n_updates;          /* two-site updates performed                                  */
} mpdo_trunc_stats;

/* Create a handle.  init_site_vec: host, d complex numbers (interleaved) giving the
 * product state (x)_n |v>, or NULL for |+_X> = (|0>+|1>)/sqrt(2) (Sec. IV initial state).
 * The orthogonality centre starts at site 0.  *out is set only on success. */
int mpdo_create(const mpdo_config* cfg, const double* init_site_vec, mpdo_t* out);

/* Reset the state of an existing handle to the product state (no reallocation). */
int mpdo_reset(mpdo_t h, const double* init_site_vec);

/* Apply the ops of `layer` in order (Sec. III.A two-site update; Sec. IV layers).
 * Each two-site op must be on a bond that contains the current orthogonality centre;
 * the centre moves to the other site of the bond, whose inner index receives the
 * op's Kraus index and is then truncated (PPT when enabled).  stats may be NULL. */
int mpdo_apply_layer(mpdo_t h, const mpdo_layer* layer, mpdo_trunc_stats* stats);

/* Device-resident layer: upload once, apply many times (inputs resident in HBM). */
typedef struct mpdo_dlayer_s* mpdo_dlayer;
int mpdo_layer_upload(mpdo_t h, const mpdo_layer* layer, mpdo_dlayer* out);
int mpdo_apply_dlayer(mpdo_t h, mpdo_dlayer dl, mpdo_trunc_stats* stats);
int mpdo_layer_free(mpdo_t h, mpdo_dlayer dl);

/* Re-truncate the whole chain to (chi_max, k_max): identity two-site updates swept from
 * the centre to the right end and back to site 0, so every bond and inner index is
 * truncated with the centre on it.  The centre ends at site 0. */
int mpdo_truncate(mpdo_t h, int chi_max, int k_max, int use_ppt, mpdo_trunc_stats* stats);

/* TFIM energies (Eq. tfim_hamiltonian, S = Pauli on the qubit levels, 0 on |r>):
 * H = -J sum Z_i Z_{i+1} - h sum X_i - b J sum Z_i.
 *   e_raw        = tr(H rho)/tr(rho)
 *   e_success    = tr(Pi_q H Pi_q rho)/success_prob,  Pi_q = (x)(|0><0|+|1><1|)
 *   success_prob = tr(Pi_q rho) (qubit trace, Sec. IV.A), trace = tr(rho)
 * Output pointers are host doubles; any of them may be NULL. */
int mpdo_expect_energy(mpdo_t h, double J, double hx, double b, double* e_raw,
                       double* e_success, double* success_prob, double* trace);

/* Second-order observables (quadratic in rho; Sec. III.E, costs of Fig. 6c-d), from
 * environments of two copies of rho contracted site by site in the sites' precision with
 * FP64 final sums:
 *   xi        = tr(rho^2) / tr(rho)^2            (the purity PPT preserves, Sec. III.D)
 *   collision = sum_x <x|rho|x>^2 / tr(rho)^2   (anticoncentration of the outcomes)
 *   s2_left, s2_right = -log(tr(rho_A^2) / tr(rho)^2) for A = sites < cut resp. >= cut
 *   i2        = s2_left + s2_right + log(xi)    (Renyi-2 mutual information across the cut)
 * The environments have D^4 entries (D the largest bond dimension): the call allocates
 * ~50 D^4 complex numbers for its duration (through the handle's hooks) and refuses more than
 * 32 GB with MPDO_ERR_ARG.  cut in 1..N-1; outputs are host doubles, any may be NULL. */
int mpdo_expect_second_order(mpdo_t h, int cut, double* xi, double* collision, double* s2_left,
                             double* s2_right, double* i2);

/* Draw n_samples configurations x in {0,1,2}^N from <x|rho|x>/tr(rho) by sequential
 * conditional sampling with Philox4x32-10 uniforms (counter (site, sample, 0, 0), key
 * = seed).  bits: host uint8 [n_samples][N]; probs: host double [n_samples] receives
 * <x|rho|x>.  Either output may be NULL. */
int mpdo_sample_probs(mpdo_t h, int n_samples, uint64_t seed, uint8_t* bits, double* probs);

/* Change the active limits of a handle (each at most what it was created with) and reset
 * its state to the product state; lets one handle serve circuits of different sizes. */
int mpdo_reconfigure(mpdo_t h, int n_sites, int chi_max, int k_max, int use_ppt,
                     const double* init_site_vec);

/* Batched form: many independent circuits advanced concurrently.  Each pool handle runs on
 * its own CUDA stream, driven by its own host thread, so the kernels of different circuits
 * overlap on the GPU; circuits are taken from a shared queue in index order.  For circuit i
 * the worker reconfigures its handle to (n_sites, chi_max, k_max, use_ppt), applies the
 * device-resident layers in order (each must have been uploaded by a handle of the same
 * precision on the same device) and evaluates the TFIM energy; out[4i..4i+3] = e_raw,
 * e_success, success_prob, trace; status[i] (may be NULL) = its return code.  The pool
 * handles must be distinct and not used by other threads during the call.  The driver
 * maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (default 8); with more
 * handles than queues, streams that share a queue wait on each other's launches, so set
 * it (up to 32) in the environment before the process creates its CUDA context. */
typedef struct {
  int n_sites, chi_max, k_max, use_ppt;
  int n_layers;
  const mpdo_dlayer* layers;
  double J, hx, b;
} mpdo_circuit;
int mpdo_batch_run(int n_handles, mpdo_t* handles, int n_circuits, const mpdo_circuit* circuits,
                   double* out, int* status);

/* The same executor for circuits given as host layers (as for mpdo_apply_layer): each
 * worker converts its circuit's layers and copies them into its handle's staging buffer
 * on the handle's stream, layer by layer, so one circuit's uploads overlap the other
 * circuits' kernels.  Inputs are read only during the call; errors as for
 * mpdo_batch_run (an invalid or non-finite op fails its circuit with MPDO_ERR_ARG or
 * MPDO_ERR_NUMERIC). */
typedef struct {
  int n_sites, chi_max, k_max, use_ppt;
  int n_layers;
  const mpdo_layer* layers;   /* host layers, n_layers of them */
  double J, hx, b;
} mpdo_circuit_host;
int mpdo_batch_run_host(int n_handles, mpdo_t* handles, int n_circuits,
                        const mpdo_circuit_host* circuits, double* out, int* status);

/* Current bond dimensions (host int[N-1]), inner dimensions (host int[N]) and centre. */
int mpdo_get_dims(mpdo_t h, int* bond_dims, int* kraus_dims, int* centre);

/* Copy site tensor n to the host as complex128 [Dl][d][K][Dr] (capacity in complex
 * numbers given by cap; the dims are written to dims[4]). */
int mpdo_get_site(mpdo_t h, int n, double* out, size_t cap, int* dims);

int mpdo_destroy(mpdo_t h);
const char* mpdo_last_error(mpdo_t h);

/* Channel builder (host, FP64, off the hot path).  Builds the Kraus set of one noisy
 * ZZ block on a bond in the gate-level model: crosstalk phase exp(-i phi n_r n_r)
 * (Sec. III.B, active pair), the ideal block CNOT (I (x) exp(-i a Z)) CNOT with
 * CNOT = (I (x) Had) CZ (I (x) Had) (Eq. HZ_block_representation), post-promotion
 * exp(-i dPP (|1><r| + h.c.)) on both atoms (Sec. IV.A), one unit of Rydberg decay
 * (branching b0, b1, bd; Sec. II jump operators) and dephasing (linear rate) on both
 * atoms, then the one-site unitaries post_left / post_right (3x3 complex128, may be
 * NULL).  The Kraus set is the Choi eigendecomposition, eigenvalues below
 * eta*lambda_max dropped (eta >= 0; the layer builders below reject a negative eta with
 * MPDO_ERR_ARG too).  out: host complex128 [cap][9][9]; *n_kraus receives M.
 * Returns MPDO_ERR_ARG if cap < M. */
int mpdo_build_block_channel(double angle_zz, double gamma_diss, double gamma_deph,
                             double xtalk_phase, double delta_pp, double b0, double b1,
                             double bd, const double* post_left, const double* post_right,
                             double eta, double* out, int cap, int* n_kraus);

/* QAOA layer builder: the ordered two-site ops of layer k (0-based) of the TFIM QAOA
 * (Sec. IV, Eqs. tfim_model, HZ_block_representation, HZ_representation): blocks with
 * ZZ angle J*alpha, left->right for even k and right->left for odd k; the one-site gate
 * exp(-i beta S^x) exp(-i b J alpha S^z) of each site folded into the last block that
 * touches it.  Writes n_sites-1 ops: sites[i], kraus counts ms[i], and the Kraus data
 * into out (host complex128, capacity cap complex numbers). */
int mpdo_build_qaoa_layer(int n_sites, int k, double alpha, double beta, double J,
                          double bz, double gamma_diss, double gamma_deph,
                          double xtalk_phase, double delta_pp, double b0, double b1,
                          double bd, double eta, int* sites, int* ms, double* out,
                          size_t cap);

/* The same QAOA layer split by the coherent part of Rydberg dissipation (App. E): the
 * dissipation gamma_diss (per pulse) damps the gate's two-atom coherences by
 * alpha = e^{-0.012291 gamma_diss} and beta = e^{-0.0185454 gamma_diss}, which act on the
 * Ising phase gate as the extra phases d1 = ((1-alpha)/(1+alpha))^2 on S^z_i + S^z_j and
 * d2 = ((alpha-beta)/(alpha+beta))^2 on S^z_i S^z_j.  part 0: the coherent part alone -- every
 * block without dissipation (the other noise kept), followed by the diagonal shift
 * exp(-i J alpha (d2 z_i z_j + d1 (z_i + z_j))), z = (1, -1, 0) on (|0>, |1>, |r>); part 1:
 * the incoherent part -- the full block followed by the inverse shift.  Outputs, capacity
 * and the other arguments as for mpdo_build_qaoa_layer; MPDO_ERR_ARG for part not 0 or 1 or
 * a negative or non-finite gamma_diss. */
int mpdo_build_qaoa_layer_appe(int n_sites, int k, double alpha, double beta, double J,
                               double bz, double gamma_diss, double gamma_deph,
                               double xtalk_phase, double delta_pp, double b0, double b1,
                               double bd, int part, double eta, int* sites, int* ms,
                               double* out, size_t cap);

/* Random-circuit layer k (0-based) of the paper's RCS workload (Sec. IV, Figs. 4 and 5 a-c):
 * a Haar one-qubit gate on every atom, then a noisy CZ on the bonds (i, i+1) with
 * i = k mod 2 (brickwork), written as one sweep of n_sites-1 two-site ops (left to right for
 * even k, right to left for odd k): CZ bonds get the G0 channel (crosstalk phase
 * exp(-i xtalk_phase n_r n_r), ideal CZ |11> -> -|11>, post-promotion, one unit of decay and
 * dephasing on both atoms), the other bonds a one-Kraus unitary; each atom's gate is folded
 * into the first op that touches it.  haar: host complex128 [n_sites][2][2] (qubit levels;
 * |r> is left alone).  Outputs as for mpdo_build_qaoa_layer. */
int mpdo_build_rcs_layer(int n_sites, int k, const double* haar, double gamma_diss,
                         double gamma_deph, double xtalk_phase, double delta_pp, double b0,
                         double b1, double bd, double eta, int* sites, int* ms, double* out,
                         size_t cap);

/* Gate model G1: the pulse-level CZ channel (Sec. II, Eqs. LME_Hamiltonian,
 * LME_Single_Site, LME; Fig. 1 caption; integrated into one channel as in Sec. III.A).
 * Two atoms under H_p = H_1 (x) I + I (x) H_2 + B|rr><rr|, H_i = Omega(t)/2 (|r><1| + h.c.)
 * + Delta|r><r|, Omega(t) = omega_max [exp(-(t - T/2)^2/u^2) - a]/(1 - a), u = width*T,
 * a = exp(-(T/2u)^2); times in us, frequencies angular (rad/us).  The one-atom dissipators
 * (decay with branching b0, b1 into the qubit levels, the rest to dark states; dephasing,
 * linear-rate reading) run at gamma/T, i.e. gamma is per pulse.  n_steps equal steps,
 * each N(tau/2) U_k N(tau/2) with U_k = exp(-i tau H_p(midpoint)) and N the closed-form
 * noise of both atoms; then each atom gets diag(1, e^{-i phi_1}, 1), phi_1 the |01> phase
 * of the noiseless pulse.  superop: host complex128 [81][81] on the two-atom row-major
 * vec((a,b),(a',b')); *phi1, *infidelity (may be NULL): phi_1 and 1 - the average gate
 * fidelity of the corrected noiseless pulse against CZ on the qubit subspace.  Host only
 * (no GPU); cost ~n_steps * 4e5 complex multiply-adds.  MPDO_ERR_ARG for n_steps outside
 * 1..1e6, T or width <= 0 or negative rates; MPDO_ERR_NUMERIC for non-finite input. */
typedef struct {
  double T, omega_max, delta, blockade, width;
} mpdo_pulse;
int mpdo_build_cz_pulse(const mpdo_pulse* pulse, double gamma_diss, double gamma_deph,
                        double b0, double b1, int n_steps, double* superop, double* phi1,
                        double* infidelity);

/* Crosstalk CZ (Sec. III.B, noiseless): a Rydberg atom next to an active atom shifts that
 * atom's detuning by the neighbour blockade b_x, so the gate on (i, i+1) with its non-active
 * neighbours i-1 and i+2 is  sum_{a,b} P_a (x) C(delta + a b_x, delta + b b_x) (x) P_b,
 * P_1 = |r><r|, P_0 = 1 - P_1, C the pulse of `pulse` with those detunings followed by the
 * one-atom phase correction of the unshifted pulse (as mpdo_build_cz_pulse).  out: host
 * complex128 [81][81], index ((s_{i-1} 3 + s_i) 3 + s_{i+1}) 3 + s_{i+2}.  n_steps midpoint
 * exponentials.  A four-site unitary: the two-site update of the engine does not apply it
 * (it serves the host and the tests). */
int mpdo_build_crosstalk_cz(const mpdo_pulse* pulse, double b_x, int n_steps, double* out);

/* The QAOA layer of mpdo_build_qaoa_layer with every CZ of the ZZ blocks replaced by the
 * channel cz_superop (host complex128 [81][81], e.g. from mpdo_build_cz_pulse): block =
 * (I(x)Had) CZ (I(x)Had Rz(J alpha) Had) CZ (I(x)Had) as superoperators, the crosstalk phase
 * exp(-i xtalk_phase n_r(x)n_r) first; no post-promotion and no separate noise unit (the
 * pulse carries both).  Outputs as for mpdo_build_qaoa_layer. */
int mpdo_build_qaoa_layer_cz(int n_sites, int k, double alpha, double beta, double J,
                             double bz, const double* cz_superop, double xtalk_phase,
                             double eta, int* sites, int* ms, double* out, size_t cap);

/* Vectorized MPO engine (the paper's main engine, Sec. III.A "vectorized MPO", with the
 * purity-preserving truncation on the bond, Sec. III.D Eqs. xiformula and ppt, App. B):
 * rho as an MPS over the doubled index (s, s') (local dimension 9), complex128, mixed-canonical
 * in the Frobenius inner product.  Each two-site op (kind 2, its Kraus set as for mpdo_op) acts
 * as its superoperator on the pair; the pair is split by an SVD (eigenpairs of the Gram of the
 * updated pair, FP64 Jacobi) and cut to at most chi_max values above sv_cutoff (Schmidt values
 * below sqrt(1e-15) of the largest are numerical zeros in any case).  use_ppt = 0 keeps the
 * largest values unchanged ("naive"); 1 replaces them by PPT's values with the trace
 * environment T_k of each Schmidt pair (from the trace contractions of the two sides), which
 * keeps tr rho and tr rho^2 / tr rho^2 of the cut.  The op order rules are those of
 * mpdo_apply_layer (ops must touch the centre; the centre moves to the other site).
 * stats: disc_bond_w (sum over updates of the discarded sum of Lambda^2, fractions),
 * PPT theta/infeasible/clamped, chi_used_max, n_updates.  mpdo_vmpo_purity: tr rho^2 (the
 * centre's squared Frobenius norm in the canonical gauge).  mpdo_vmpo_collision: the
 * collision probability sum_x <x|rho|x>^2 / (tr rho)^2 (Sec. III.E, the anticoncentration of
 * Fig. 7), from the diagonal entries (s, s) of each site contracted over two copies; O(D^3)
 * per site, FP64; MPDO_ERR_NUMERIC for a zero trace.  chi_max in 1..256; init_site_vec
 * as for mpdo_create; cuda_stream NULL = an own non-blocking stream. */
typedef struct mpdo_vmpo_s* mpdo_vmpo;
int mpdo_vmpo_create(int n_sites, int chi_max, int use_ppt, double sv_cutoff,
                     const double* init_site_vec, void* cuda_stream, mpdo_vmpo* out);
int mpdo_vmpo_apply_layer(mpdo_vmpo h, const mpdo_layer* layer, mpdo_trunc_stats* stats);
int mpdo_vmpo_expect_energy(mpdo_vmpo h, double J, double hx, double b, double* e_raw,
                            double* e_success, double* success_prob, double* trace);
int mpdo_vmpo_purity(mpdo_vmpo h, double* purity);
int mpdo_vmpo_collision(mpdo_vmpo h, double* collision);
/* Arithmetic of the vMPO updates.  mode 0 (default): FP64 products on the CUDA cores and
 * the FP64 Jacobi eigensolver.  mode 1 (the tensor-core form): products of at least 2^21
 * complex multiply-adds as error-free BF16 slice products on the tensor cores summed in
 * FP64 (carried to ~2^-48 of each operand row's largest entry), and the Gram's eigenpairs
 * from the mixed-precision solver (FP32 Jacobi levels with FP64 refinement); its
 * resolution raises the numerical-zero floor of the Schmidt values from sqrt(1e-15) to
 * sqrt(1e-13) of the largest.  The first switch to mode 1 allocates ~0.3 GB plus the
 * solver's workspace (~1 GB at chi 256).  MPDO_ERR_TIMEOUT from a later update when a
 * tensor-core pipeline wait gave up. */
int mpdo_vmpo_set_precision(mpdo_vmpo h, int mode);
int mpdo_vmpo_get_dims(mpdo_vmpo h, int* bond_dims, int* centre);
int mpdo_vmpo_destroy(mpdo_vmpo h);

/* Instrumentation.
 * mpdo_kernel_launches: number of CUDA kernels this library has launched in the process.
 * mpdo_profile: time kernel launches of the selected classes on handle h with CUDA events
 *   recorded on its stream (bit 0: complex GEMMs, bit 1: eigensolver calls, bit 2: all
 *   other kernels); 0 switches timing off.  Resets the accumulators.
 * mpdo_profile_read: accumulated device milliseconds, launch count and algorithmic FLOPs
 *   (8 m n k per complex GEMM; for the eigensolver 8 x 3 x 16 x 16 x padded n per active
 *   block-pair rotation round, the multiply-adds its block Jacobi executes; 0 for other
 *   kernels) of class cls since mpdo_profile. */
long long mpdo_kernel_launches(void);
int mpdo_profile(mpdo_t h, int class_mask);
int mpdo_profile_read(mpdo_t h, int cls, double* ms, long long* launches, double* flops);

/* Kernel-level entry points used by the unit tests (device pointers). */
/* Tile-shape autotuner of the complex GEMMs (all handles of the process).  For precision
 * prec (0: FP64 products, including FP32 x FP32 -> FP64; 1: FP32) and each bucket of
 * (number of 16 x 16 output tiles: 1 .. 1024 in powers of 2) x (K: 16 .. 4096 in powers of
 * 2), times on `stream` (cudaStream_t; reps runs after one warm-up, minimum taken, CUDA
 * events) the 64 x 64 tile kernel, the 16 x 16 tile kernel and the 16 x 16 kernel with K
 * split over a thread-block cluster of 2, 4 or 8, on a representative shape of the
 * bucket, and makes the fastest the choice for every product of that bucket.  Untuned
 * buckets, and all of them after a call with reps <= 0, follow the built-in size rules.
 * The choice changes the summation order of products, not their precision: call it
 * before running circuits, not while another thread runs them.  Allocates ~70 MB of
 * device scratch for the call; synchronises the stream.  *n_tuned (may be NULL) receives
 * the number of buckets set.  MPDO_ERR_ARG for prec outside {0, 1}; MPDO_ERR_OOM;
 * MPDO_ERR_CUDA (the table is then reset to the size rules). */
int mpdo_autotune_gemm(int prec, void* stream, int reps, int* n_tuned);

/* C[b] = op(A[b]) op(B[b]) for complex matrices; prec 0 = complex128, 1 = complex64.
 * opa/opb: 0 = N, 1 = T, 2 = C (conjugate transpose).  A is m x k after op, etc.;
 * leading dimensions in complex elements (row-major), batch strides in elements. */
int mpdo_kernel_cgemm(int prec, int opa, int opb, int m, int n, int k, const void* a,
                      long lda, long sa, const void* b, long ldb, long sb, void* c,
                      long ldc, long sc, int batch, void* stream);
/* Hermitian eigendecomposition of a (n x n, row-major complex, overwritten): eigenvalues
 * descending into w (double, host-visible device array of n), eigenvectors as the
 * columns of v (n x n row-major complex of the same precision).  prec 0: complex128 Jacobi;
 * 1: complex64 Jacobi; 2: complex128 matrix through the mixed-precision solver (FP32
 * Jacobi levels with FP64 refinement, resolved down to 1e-14 of the largest eigenvalue);
 * 3: as 2 with the solver's FP64 products formed as error-free BF16 slice products on the
 * tensor cores (allocates a 256 MiB workspace for the call).  Returns the sweeps (0, 1) or
 * levels (2, 3) used in *sweeps (host).  n in 1..4096; MPDO_ERR_TIMEOUT when a tensor-core
 * pipeline wait gave up. */
int mpdo_kernel_heig(int prec, int n, void* a, void* v, double* w, int* sweeps, void* stream);

/* Tensor-core GEMMs (tcgen05.mma, TMEM accumulators, TMA-fed shared-memory pipeline) on
 * which the contractions of the two-site update run in the split-precision modes (Sec.
 * III.A: contracting the site tensors and the gate, Fig. 6a; the Gram products of the
 * truncation).  Device pointers; stream = cudaStream_t (NULL = legacy default stream);
 * both calls synchronise the stream and allocate their own scratch (test entry points).
 * mpdo_kernel_tcgemm_real: d (m x n FP32, row stride ldd) = a b^T with a (m x k) and b
 *   (n x k) K-major, elements FP32 read as TF32 (elt 4) or BF16 (elt 2); lda, ldb in
 *   elements, >= k and multiples of 16 bytes.
 * mpdo_kernel_tcgemm: complex64 c[b] = op(a[b]) op(b[b]) (ops and layouts as in
 *   mpdo_kernel_cgemm) in mode 0 TF32, 1 TF32x3 (hi/lo split, FP32-level accuracy),
 *   2 BF16, 3 BF16x3, FP32 accumulation.
 * MPDO_ERR_ARG for bad sizes or layouts, MPDO_ERR_OOM, MPDO_ERR_CUDA, MPDO_ERR_TIMEOUT when a
 * pipeline wait inside the kernel gave up (the output is then undefined). */
/* Number of tensor-core GEMM kernels (tcgen05) this library has launched in the process. */
long long mpdo_tc_gemm_launches(void);
int mpdo_kernel_tcgemm_real(int elt, int m, int n, int k, const void* a, long lda, const void* b,
                            long ldb, float* d, long ldd, void* stream);
int mpdo_kernel_tcgemm(int mode, int opa, int opb, int m, int n, int k, const void* a, long lda,
                       long sa, const void* b, long ldb, long sb, void* c, long ldc, long sc,
                       int batch, void* stream);
/* FP64-accurate product of complex64 operands on the BF16 tensor cores: complex128
 * c[b] = op(a[b]) op(b[b]), each operand row scaled by a power of two and split into six
 * integer slices (exact in BF16), the 21 slice products of weight above 2^-48 accumulated
 * exactly in FP32 over chunks of 1024 real terms and summed in FP64, so the result carries
 * the product of the FP32 inputs to ~2^-48 of the rows' largest entries (error-free
 * transformation of matrix products; Ozaki, Ogita, Oishi, Rump 2012).  This is what gives the
 * Gram matrices of FP32 site tensors their FP64 eigenvalue floor in the mixed form (Sec.
 * III.A truncation "removing the least significant diagonal elements" down to ~1e-13 of the
 * largest).  Layouts as mpdo_kernel_cgemm; c has leading dimension ldc (complex128). */
int mpdo_kernel_tcgemm_exact(int opa, int opb, int m, int n, int k, const void* a, long lda,
                             long sa, const void* b, long ldb, long sb, void* c, long ldc,
                             long sc, int batch, void* stream);

/* MLP surrogate (no counterpart in the paper; the workload's learned part).  A fully
 * connected network with tanh hidden layers and a linear output maps a circuit description
 * (chain length, noise rates, QAOA angles; scaled by the caller) to (energy per site,
 * success probability).  Trained on the GPU on samples the MPDO engine produced; its input
 * gradient proposes angles that the engine then re-scores.  FP32 parameters and
 * arithmetic.  Parameters are one flat array W_0 b_0 W_1 b_1 ... with W_l stored
 * [fan_in][fan_out] row-major.  x, t, y, gx are device arrays [batch][width], row-major;
 * batch <= max_batch.  stream NULL = the network owns a non-blocking stream (inputs written
 * by other streams must then be synchronised first; cudaStreamLegacy is accepted).
 *   mpdo_mlp_loss_grad: forward, mean-squared loss (host *loss), backward into the
 *     network's gradient buffer (copied to grad_host when not NULL, n_params floats)
 *   mpdo_mlp_adam_step: one Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) with the last
 *     gradient
 *   mpdo_mlp_input_grad: gx = d(sum_j wout_j y_j)/dx, wout host [n_out] */
typedef struct mpdo_mlp_s* mpdo_mlp;
int mpdo_mlp_create(int n_layers, const int* widths, int max_batch, void* stream, mpdo_mlp* out);
long long mpdo_mlp_n_params(mpdo_mlp m);
int mpdo_mlp_set_params(mpdo_mlp m, const float* host_params);
int mpdo_mlp_get_params(mpdo_mlp m, float* host_params);
int mpdo_mlp_forward(mpdo_mlp m, int batch, const float* x, float* y);
int mpdo_mlp_loss_grad(mpdo_mlp m, int batch, const float* x, const float* t, float* loss,
                       float* grad_host);
int mpdo_mlp_adam_step(mpdo_mlp m, float lr);
int mpdo_mlp_input_grad(mpdo_mlp m, int batch, const float* x, const float* wout_host, float* gx);
/* Precision of the network's products: 0 = FP32 on the CUDA cores (default); 1 = BF16
 * operands on the tensor cores (tcgen05, TMA-fed) with FP32 accumulation, parameters,
 * gradients and Adam moments kept in FP32 (mixed-precision training).  Allocates the packed
 * operand buffers on first use; MPDO_ERR_ARG for another mode. */
int mpdo_mlp_set_precision(mpdo_mlp m, int mode);
int mpdo_mlp_destroy(mpdo_mlp m);

/* Allocation-free variant of mpdo_kernel_heig.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- processes where every
 * byte of device memory is owned by an outside allocator or budget (a framework's caching
 * allocator, a serving process with a fixed memory pool), where a stray cudaMalloc would
 * fragment or overrun that budget, and latency-critical loops, where cudaMalloc and
 * cudaFree can synchronise the whole device.  Arguments are those of mpdo_kernel_heig
 * (a, v, w are caller-owned device arrays; sweeps is an optional host int).
 * Its scratch is one file-scope device array sized for n <= MPDO_HEIG_NOALLOC_NMAX; larger
 * n returns MPDO_ERR_ARG with a message in mpdo_last_error(NULL).  No call allocates.
 * The array's device address is looked up on the first call made on each device (with
 * that device current), and again on the first call after the device's context changed (a
 * device reset loads the library's device code anew); make such first calls outside any
 * stream capture.  Every GPU that
 * loads the library holds the array (~1.2 MB) until the process exits.  All calls share
 * the one array, and each call re-initialises the part it uses (padded matrix, identity
 * accumulator, zeroed counters); calls that overlap on the GPU -- on different streams
 * or from different host threads -- race on it and must be serialised by the caller. */
#define MPDO_HEIG_NOALLOC_NMAX 192
int mpdo_heig_noalloc(int prec, int n, void* a, void* v, double* w, int* sweeps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPDO_H */
