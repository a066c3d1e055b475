/*
 * chi0.h -- C ABI of the GB300 (sm_103a) library that computes the RPA
 * independent-particle polarizability chi0_{GG'}(q, w) and the inverse
 * symmetric dielectric matrix eps~^-1(q, w) of the GW/BSE method described in
 * Sangalli et al., "Many-body perturbation theory calculations using the yambo
 * code", J. Phys.: Condens. Matter 31, 325902 (2019), arXiv:1902.03837.
 *
 * The operations (paper sections / equations):
 *   - oscillator strengths  rho_{nmk}(q,G) = <n k| e^{i(q+G).r} |m k-q>,
 *     Linear Response section, Eq. (rhotw), evaluated through the
 *     real-space product of the two states and a Fourier transform;
 *   - chi0_{GG'}(q,w) = f_s/(N_k Omega) sum_{nmk} rho rho^* x (two-pole
 *     frequency factor), Eq. (X_IP), organised as in Appendix B, Eqs.
 *     (X_IP_split), (X_IP_split1), (X_IP_split2): frequency-independent
 *     rho rho^* products weighted by per-transition frequency factors;
 *   - the Dyson step of the Linear Algebra subsection, Eqs. (X_rpa) and
 *     (X_rpa_inv), written for the symmetric matrix
 *     eps~ = 1 - v^1/2 chi0 v^1/2, v(q+G) = 4 pi / |q+G|^2 (Coulomb
 *     interaction subsection), whose inverse gives W through Eq. (W_def).
 *
 * Units: Hartree atomic units (Ha, bohr).  Complex numbers are interleaved
 * (re, im).  All arrays are row-major (C order).
 *
 * Conventions fixed by this library (readings of the paper):
 *   - n is the band at k and m the band at k - q (as in Eq. rhotw); k - q is
 *     folded to the grid as k - q = k' + G0 with the periodic gauge
 *     psi_{k'+G0} = psi_{k'};
 *   - time-reversal two-pole form: transitions t = (k, n, m) with weight
 *     w_t(w) = f_s/(N_k Omega) (f_{m,k-q} - f_{n,k})
 *              [1/(w + D_t + i eta) - 1/(w - D_t + i eta)],
 *     D_t = eps_{m,k-q} - eps_{n,k}; chi0(w) = sum_t w_t rho_t rho_t^H.  Pairs
 *     with f_{m,k-q} - f_{n,k} <= occ_drop_tol carry zero weight;
 *   - the response G set is the ng vectors of smallest |q+G|, ties broken by
 *     ascending (Gx, Gy, Gz), |q+G|^2 compared exactly;
 *   - time-reversal-symmetric inputs only; frequencies on the imaginary axis
 *     (real weights, Hermitian chi0) or on the real axis with eta > 0
 *     (complex weights; chi0 and eps~ general complex matrices); other
 *     frequencies return CHI0_EUNSUPPORTED.
 *
 * Asynchrony: every call that launches work is asynchronous on
 * config.cuda_stream (NULL = the legacy default stream).  The returned status
 * covers argument checks and launch errors; errors raised on the device are
 * reported by the next call that synchronises (chi0_synchronize, or a call
 * that copies results to the host).
 *
 * Errors never abort the process: every call returns a chi0_status and
 * chi0_last_error() describes the most recent failure on that context.
 */
#ifndef CHI0_H_
#define CHI0_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chi0_ctx chi0_ctx; /* opaque */

typedef enum {
  CHI0_OK = 0,
  CHI0_EINVAL = -1,       /* bad argument (NULL pointer, size out of range, ...) */
  CHI0_ENOMEM = -2,       /* device or host allocation failed */
  CHI0_ECUDA = -3,        /* a CUDA runtime/driver call failed */
  CHI0_ESTATE = -4,       /* call out of order (see "Ordering" below) */
  CHI0_ENOTPD = -5,       /* a pivot of the Dyson elimination vanished or eps~ not positive */
  CHI0_ESINGULAR = -6,    /* reserved: singular matrix in a general solve */
  CHI0_ETIMEOUT = -7,     /* a bounded device-side wait gave up (error flag set by a kernel) */
  CHI0_EUNSUPPORTED = -8  /* valid request outside what this build implements */
} chi0_status;

typedef enum {
  CHI0_FP64 = 0,          /* FP64 end to end (rho, contraction, Dyson) */
  CHI0_MIXED_BF16X3 = 1   /* FP32 rho, split-precision BF16x3 tensor-core contraction
                             accumulated in FP32 over bounded transition chunks and
                             summed in FP64, FP64 Dyson */
} chi0_precision;

typedef struct {
  double lattice[3][3];   /* bohr, rows a1, a2, a3; this build needs a cubic cell a*I */
  int kgrid[3];           /* Gamma-centred grid, k = (i/N1, j/N2, l/N3), k index = (i*N2+j)*N3+l */
  int nbands;             /* bands per k */
  int npw_max;            /* largest plane-wave sphere over all k */
  int fft[3];             /* real-space grid (N1, N2, N3) used for rho; must be alias free */
  int ng;                 /* number of response G vectors */
  int nq;                 /* number of q points */
  const double* q_frac;   /* [nq][3] reduced coordinates; each q must be a vector of the k grid;
                             copied at chi0_create */
  int nw;                 /* number of frequencies */
  const double* omega;    /* [nw][2] complex frequencies (re, im) in Ha; copied at chi0_create.
                             Either imaginary-axis (re = 0: chi0 Hermitian) or real-axis (im = 0,
                             re > 0, and eta > 0: complex weights, chi0 = H_r + i H_i: one
                             complex-weight contraction in the mixed form, two Hermitian ones
                             combined in the FP64 form; eps~ inverted by general Gauss-Jordan);
                             other forms give CHI0_EUNSUPPORTED at chi0_build_chi0 */
  double eta;             /* Ha; +i*eta on both poles (retarded); 0 on the imaginary axis */
  double spin_factor;     /* f_s: 2 without spin polarisation, 1 with it */
  int precision;          /* chi0_precision */
  int time_reversal;      /* must be 1: inputs obey psi_{-k} = psi_k^*, eps_{-k} = eps_k */
  double occ_drop_tol;    /* transitions with f_m - f_n <= tol get zero weight (>= 0) */
  void* cuda_stream;      /* cudaStream_t for all work; NULL = default stream */
} chi0_config;

/* Create a context.  Validates the configuration and copies q_frac and omega.
 * Allocates nothing on the device yet.  *out receives the handle (NULL on
 * failure).  Errors: CHI0_EINVAL, CHI0_EUNSUPPORTED (non-cubic cell,
 * time_reversal != 1), CHI0_ENOMEM. */
chi0_status chi0_create(const chi0_config* cfg, chi0_ctx** out);

/* Plane-wave sphere and coefficients of every band at k point ik
 * (the states of the paper's wavefunction databases, k-centred spheres).
 *   gvec: [npw][3] int32 Miller indices of G with |k+G| < k_c (any order);
 *   coef: [nbands][npw] complex coefficients c_{n,k}(G), interleaved, complex64
 *         when coef_is_c64 = 1, else complex128;
 *   on_device: 1 if gvec and coef are device pointers (copied device to device),
 *              0 if host pointers (copied; pinned host memory makes the copy async).
 * The data are copied (converted to the working precision when needed); the
 * caller keeps ownership of its buffers.  Pageable host buffers may be reused
 * once the call has returned.  Pinned host coefficients are copied
 * asynchronously: on an unchanged sphere the copy runs on an internal upload
 * stream that chi0_compute_rho overlaps with its transforms and rho; the
 * buffer may be reused after chi0_synchronize, or after any call that
 * returns results to the host and follows the next chi0_compute_rho.  Device
 * buffers may be reused once the context's stream has passed this point.
 * Errors: CHI0_EINVAL (ik or npw out of range, NULL), CHI0_ENOMEM, CHI0_ECUDA. */
chi0_status chi0_set_wavefunctions(chi0_ctx* ctx, int ik, int npw, const int32_t* gvec,
                                   const void* coef, int coef_is_c64, int on_device);

/* Band energies eps[nk][nbands] (Ha) and occupations occ[nk][nbands] in [0,1]
 * per spin channel (host pointers, copied).  Errors: CHI0_EINVAL. */
chi0_status chi0_set_energies(chi0_ctx* ctx, const double* eps, const double* occ);

/* Oscillator strengths rho_t(G_i), Eq. (rhotw), for every transition of the
 * time-reversal form at q index iq; kept on the device as R[nt][ng] (G fastest;
 * complex128 in FP64 mode, complex64 in mixed mode).  Requires all
 * wavefunctions and energies.  Errors: CHI0_ESTATE, CHI0_EINVAL, CHI0_ENOMEM,
 * CHI0_ECUDA. */
chi0_status chi0_compute_rho(chi0_ctx* ctx, int iq);

/* chi0(q_iq, w) for every configured frequency, Eq. (X_IP) in the App. B
 * organisation.  out: [nw][ng][ng] complex128, row index G, column index G'.
 * out_on_device = 1: out is a device pointer (written asynchronously);
 * 0: host pointer (this call synchronises); out may be NULL to keep chi0 on
 * the device only (the Dyson step reads it from there).  Requires
 * chi0_compute_rho(iq).  Errors: CHI0_ESTATE, CHI0_EUNSUPPORTED (non-real
 * weights), CHI0_ENOMEM, CHI0_ECUDA, CHI0_ETIMEOUT (host copies only). */
chi0_status chi0_build_chi0(chi0_ctx* ctx, int iq, void* out, int out_on_device);

/* eps~^-1(q_iq, w) = (1 - v^1/2 chi0 v^1/2)^-1 for every frequency, Eqs.
 * (X_rpa), (X_rpa_inv) in the symmetric form of Eq. (W_def), by FP64
 * Gauss-Jordan elimination without pivoting: on the imaginary axis eps~ is
 * Hermitian positive definite (lower tiles only, Hermitian sweep rule); on
 * the real axis (w > 0, eta > 0) eps~ has a positive semidefinite imaginary
 * part, inherited by every Schur complement, and the elimination runs over
 * every tile.
 * out: [nw][ng][ng] complex128 as for chi0_build_chi0 (NULL not allowed).
 * Requires chi0_build_chi0(iq).  A vanishing pivot is reported as CHI0_ENOTPD
 * by the next synchronising call.  Errors: CHI0_ESTATE, CHI0_EINVAL,
 * CHI0_ENOTPD, CHI0_ENOMEM, CHI0_ECUDA. */
chi0_status chi0_invert_eps(chi0_ctx* ctx, int iq, void* out, int out_on_device);

/* chi0_build_chi0 followed by chi0_invert_eps (Eqs. chi0_def, X_rpa_inv, in
 * the symmetric form of Eq. W_def) as one pipelined call: in the mixed form
 * the Dyson step of frequency w runs on the FP64 units while the tensor-core
 * contraction of the later frequencies proceeds (two internal streams forked
 * from and joined back into the context's stream, the Dyson step at the
 * higher priority).  In FP64 mode, or with a terminator set, the two steps run
 * one after the other.  The results equal those of the two separate calls.
 *   eps_out: [nw][ng][ng] complex128, receives eps~^-1 (NULL not allowed);
 *   chi_out: NULL, or [nw][ng][ng] complex128 receiving chi0 (it also stays
 *            on the device for a later chi0_invert_eps);
 *   out_on_device: both outputs are device (1) or host (0) buffers; with host
 *            buffers the call synchronises.
 * Requires chi0_compute_rho(iq).  Errors: as chi0_build_chi0 and
 * chi0_invert_eps. */
chi0_status chi0_build_invert(chi0_ctx* ctx, int iq, void* chi_out, void* eps_out, int out_on_device);

/* The response G vectors used at q index iq, out: [ng][3] int32 (host).
 * Errors: CHI0_EINVAL. */
chi0_status chi0_get_response_gvectors(chi0_ctx* ctx, int iq, int32_t* out);

/* The transition list of the last chi0_compute_rho: *nt receives the count;
 * if out is not NULL it receives [nt][3] int32 triples (ik, n, m), in the row
 * order of R.  Errors: CHI0_ESTATE. */
chi0_status chi0_get_transitions(chi0_ctx* ctx, int64_t* nt, int32_t* out);

/* Copy R = rho (the last chi0_compute_rho) to a host buffer out [nt][ng]
 * complex128 (converted from complex64 in mixed mode).  Synchronises.
 * Errors: CHI0_ESTATE, CHI0_ECUDA. */
chi0_status chi0_get_rho(chi0_ctx* ctx, void* out);

/* Copy selected rows of R (the last chi0_compute_rho) to a host buffer:
 * rows[nrows] transition indices (0 <= row < nt), out [nrows][ng] complex128.
 * Synchronises.  Errors: CHI0_ESTATE, CHI0_EINVAL (row out of range), CHI0_ECUDA. */
chi0_status chi0_get_rho_rows(chi0_ctx* ctx, const int64_t* rows, int64_t nrows, void* out);

/* Band-block streaming for problems whose oscillator strengths do not fit in
 * device memory (the paper distributes the response function's memory over
 * the band indices: Parallelism section, linear response).  With
 * bands_per_block > 0, chi0_compute_rho keeps only the mixed grids of the
 * occupied-side bands m (at every k) and chi0_build_chi0 / chi0_build_invert
 * take the transitions in blocks of k_per_block k points (0: all) times
 * bands_per_block bands n: for each block the n grids, rho, the weights and
 * the contraction, whose results are summed into chi0 (Eq. X_IP is a sum
 * over transitions; only the order of the additions changes).  Device
 * memory then holds one block's grids and rho instead of all of them.
 * bands_per_block = 0 switches streaming off.  Takes effect at the next
 * chi0_compute_rho.  While on, chi0_get_rho / chi0_get_rho_rows return
 * CHI0_ESTATE and chi0_build_sigma_i CHI0_EUNSUPPORTED; chi0_compute_rho
 * returns CHI0_EUNSUPPORTED with the extrapolar correction, the learned
 * terminator or pole grouping set.  Errors: CHI0_EINVAL. */
chi0_status chi0_set_band_blocks(chi0_ctx* ctx, int bands_per_block, int k_per_block);

/* Wait for all work queued by this context and report device-side errors
 * (CHI0_ETIMEOUT, CHI0_ENOTPD, CHI0_ECUDA).  Reading an error clears the
 * device flag, so the context stays usable. */
chi0_status chi0_synchronize(chi0_ctx* ctx);

/* Failure detection check (no counterpart in the paper): queue one kernel
 * whose single thread waits, through the bounded wait every spin-wait of the
 * contraction uses, on a barrier that nothing completes.  The wait gives up
 * after about two seconds, raises the device error flag and the kernel
 * returns; the next chi0_synchronize reports CHI0_ETIMEOUT and clears the
 * flag.  While it runs, other contraction launches of any context sharing
 * the flag would stop early, so call it with nothing else queued.
 * Errors: CHI0_EINVAL, CHI0_ENOMEM, CHI0_ECUDA. */
chi0_status chi0_check_bounded_wait(chi0_ctx* ctx);

/* Stages of the path, for chi0_get_stats. */
enum {
  CHI0_STAGE_WF_GRID = 0,    /* wavefunctions to the mixed real/reciprocal grid */
  CHI0_STAGE_RHO = 1,        /* pair products, pruned transforms -> rho */
  CHI0_STAGE_WEIGHTS = 2,    /* transition weights (+ operand split in mixed mode) */
  CHI0_STAGE_CONTRACT = 3,   /* chi0 contraction (FP64 tiles or tensor cores) */
  CHI0_STAGE_REDUCE = 4,     /* chunk sums, Hermitian completion */
  CHI0_STAGE_DYSON = 5,      /* eps~ and its inverse */
  CHI0_NSTAGES = 6
};

/* Device time of every stage summed over the launches since the previous
 * chi0_get_stats (ms, CUDA events on the context's stream), the algorithmic
 * bytes and flops of the most recent instance of each stage, and the number
 * of kernels this context has launched since chi0_create.  Any pointer may
 * be NULL; arrays have CHI0_NSTAGES entries.  Synchronises. */
chi0_status chi0_get_stats(chi0_ctx* ctx, double* ms, double* bytes, double* flops,
                           int64_t* launches);

/* Allocation-free eps~^-1 for callers that cannot allocate device memory.
 * The paper has no counterpart: this exists for code whose device memory is
 * owned by another allocator (which must account for every byte), or that
 * must keep a fixed device footprint once running (so that no later
 * allocation can fail or take memory from another tenant of the GPU).
 * It computes the same result as chi0_invert_eps from a chi0 the caller holds:
 *   chi0:   device pointer, [nw][ng][ng] complex128 (input, not modified);
 *   v_sqrt: host pointer, [ng] doubles, V_i = sqrt(4 pi) / |q + G_i| (> 0);
 *   out:    device pointer, [nw][ng][ng] complex128, receives eps~^-1;
 *   cuda_stream: cudaStream_t (NULL = default stream).
 * It calls no allocating routine: its scratch (about 2.1 MB: panels for
 * ng <= 2048, the pivot-block inverse, V and an error flag) is one static
 * device array that every GPU loading this library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (once per device, with the device current); make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (the error flag is cleared at the start of each call), so calls
 * whose work overlaps on the GPU -- from two streams or two threads -- race
 * and must not be issued.  The call synchronises the stream before returning.
 * Errors: CHI0_EINVAL (NULL pointer, ng or nw < 1, V not finite and positive),
 * CHI0_EUNSUPPORTED (ng > 2048, beyond the static scratch), CHI0_ENOTPD (a
 * Gauss-Jordan pivot was not positive: eps~ is not Hermitian positive
 * definite), CHI0_ECUDA. */
chi0_status chi0_invert_eps_noalloc(const void* chi0, const double* v_sqrt, int ng, int nw,
                                    void* out, void* cuda_stream);

/* ---- Batched problems -------------------------------------------------------
 * The paper spreads the response function over q points and transitions
 * (Parallelism section, linear response) and notes that q points are uneven
 * because the number of transitions varies.  A batch runs many independent
 * problems -- problem i is context ctxs[i] at q index iqs[i] -- as one unit.
 * A context may appear several times with different q indices (every q point
 * of one system): its problems share its coefficients and its mixed grids,
 * which are computed once per replay.  At creation: all host set-up; the
 * problems' remaining work is assigned to `nstreams` helper streams, longest
 * first, each to the stream with the least estimated work, and the problems
 * of one stream share one set of scratch buffers (operands, partials, chi0,
 * Dyson panels) sized for the largest of them; the rho tile width and every
 * contraction's transition split are timed on the batch's own data and the
 * fastest kept.  Every replay runs the oscillator strengths of all problems
 * in ONE persistent launch over a device task table, the rest on the helper
 * streams, all captured once into a CUDA graph.
 *   chi_out: NULL, or n device pointers to [nw_i][ng_i][ng_i] complex128
 *            receiving chi0 of each problem (NULL entries: not returned);
 *   eps_out: NULL, or n device pointers to [nw_i][ng_i][ng_i] complex128
 *            receiving eps~^-1 of each problem (NULL entries skip the Dyson
 *            step of that problem).  Each problem needs at least one output.
 * The batch keeps its own q-point state and scratch: the contexts are read
 * (inputs only) and may be used for other calls, but their wavefunctions and
 * energies must not change, and the contexts must not be destroyed, while
 * the batch exists (it reads their input buffers in place).  All contexts must share
 * one precision.  The output pointers are captured into the graph: they must
 * stay valid while the batch exists.
 * Errors: CHI0_EINVAL (NULL, a repeated (context, q) pair, a problem with no
 * output, iq out of range), CHI0_ESTATE (inputs not set), CHI0_EUNSUPPORTED
 * (mixed precisions, or a problem too large for one persistent launch),
 * CHI0_ENOMEM, CHI0_ECUDA. */
typedef struct chi0_batch chi0_batch;

chi0_status chi0_batch_create(chi0_ctx* const* ctxs, const int* iqs, void* const* chi_out, void* const* eps_out,
                              int n, int nstreams, chi0_batch** out);

/* Replay the batch on `stream` (asynchronous; the first call captures the
 * graph).  Device-side errors are read with chi0_batch_synchronize. */
chi0_status chi0_batch_run(chi0_batch* b, void* stream);

/* Wait for the batch's work on every helper stream and report device-side
 * errors of any problem (CHI0_ETIMEOUT, CHI0_ENOTPD, CHI0_ECUDA). */
chi0_status chi0_batch_synchronize(chi0_batch* b);

/* The schedule chosen at creation: stream_of (NULL or [n]) receives the
 * helper stream of each problem; tuned_split_ms (NULL or one double) the
 * summed time of the fastest split of each contraction during the tuning. */
chi0_status chi0_batch_info(const chi0_batch* b, int* stream_of, double* tuned_split_ms);

/* m bands per block chosen for the persistent rho launch (1, 2 or 4). */
int chi0_batch_rho_width(const chi0_batch* b);

void chi0_batch_destroy(chi0_batch* b);

/* ---- Learned band-sum terminator -------------------------------------------
 * The paper's X-terminator (Linear Response section, Eq. X_term_def; its
 * expressions in Appendix C) corrects a band-truncated chi0 by an extra term
 * Delta chi.  Here Delta chi_GG'(w) is predicted entry by entry by a small
 * network trained on pairs of truncated and full-band chi0 of the same
 * systems; the full-band sum stays the reference that judges it.
 *   features x = (|q+G|/Kn, |q+G'|/Kn, |Im w|/Wn, Re chi0_trunc/c, Im chi0_trunc/c),
 *   Kn = largest |q+G| of the response set, Wn = largest |Im w|,
 *   c = mean_G |chi0_trunc,GG(w_0)|; the prediction y (2 values) means
 *   Delta chi = c (y0 + i y1), Hermitised before it is added.
 * Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3 with
 * 5 -> 128 -> 128 -> 2; parameters are one FP32 vector [W1(128x5) b1(128)
 * W2(128x128) b2(128) W3(2x128) b3(2)] (chi0_mlp_nparams() entries, device
 * memory, row-major).  bf16 = 1 rounds every operand of a matrix product to
 * BF16 (FP32 accumulation); bf16 = 0 keeps FP32 operands.  All pointers of
 * the chi0_mlp_* calls are device pointers; the calls are asynchronous on
 * `stream`.  Errors: CHI0_EINVAL (NULL pointer, non-positive size),
 * CHI0_ECUDA. */
int chi0_mlp_nparams(void);

/* Floats of device workspace that chi0_mlp_loss_grad needs for `batch` samples. */
int64_t chi0_mlp_workspace_floats(int64_t batch);

/* loss = 1/(2 batch) sum_b sum_o (y_bo - t_bo)^2 and grad = d loss / d params
 * (backpropagation; block partials summed in a fixed order, so repeatable).
 * x: [batch][5], t: [batch][2], grad: [nparams], loss: one float (may be NULL),
 * work: chi0_mlp_workspace_floats(batch) floats. */
chi0_status chi0_mlp_loss_grad(const float* params, const float* x, const float* t, int64_t batch,
                               int bf16, float* grad, float* loss, float* work, void* stream);

/* One Adam update (step >= 1, bias-corrected moments m, v of n entries). */
chi0_status chi0_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n, float lr,
                          float beta1, float beta2, float eps, int step, void* stream);

/* y[batch][2] = network(x[batch][5]). */
chi0_status chi0_mlp_predict(const float* params, const float* x, int64_t batch, int bf16, float* y,
                             void* stream);

/* Features x [nw*ng*ng][5] of a truncated chi0 (device [nw][ng][ng] c128) at
 * q index iq, and, when chi_full is not NULL, the targets t [nw*ng*ng][2] =
 * (chi_full - chi_trunc)/c; *scale receives c (host, may be NULL; reading it
 * synchronises).  Requires chi0_compute_rho(iq) on ctx (the response set).
 * Errors: CHI0_EINVAL, CHI0_ESTATE, CHI0_ENOMEM, CHI0_ECUDA. */
chi0_status chi0_term_features(chi0_ctx* ctx, int iq, const void* chi_trunc, const void* chi_full,
                               float* x, float* t, double* scale);

/* Use the network `params` (device, nparams floats, kept alive by the caller)
 * to correct every following chi0_build_chi0 on ctx; NULL switches it off. */
chi0_status chi0_set_terminator(chi0_ctx* ctx, const float* params, int bf16);

/* ---- Bruneval-Gonze extrapolar correction (X-terminator) --------------------
 * Eq. (X_term_def) with Appendix C (Eqs. rhotw-term, F-term, X-term): the
 * bands that the sum leaves out (band index >= nbands) are given one energy
 * eps_bar (Ha, absolute) and no occupation.  By the closure relation over the
 * bands at k their contribution is
 *   sum_{k,m} wbar_m(w) [ <m k-q| e^{i(G-G').r} |m k-q> - sum_{n<nbands} rho_nm(G) conj(rho_nm(G')) ],
 * wbar_m(w) the frequency factor of a transition from m into a state at
 * eps_bar, in the form of the other weights.  on = 1 applies it to every
 * following chi0_build_chi0 / chi0_build_invert / batch run; on = 0 switches
 * it off.  Either change requires chi0_compute_rho again (the transition
 * block then covers every band n < nbands at k, occupied ones included).  The
 * diagonal densities are taken on the difference vectors G - G' of the
 * response set; the FFT grid must be alias-free for them
 * (fft[a] > 2 max|G_a| of the spheres + max|G_a - G'_a|), checked at
 * chi0_build_chi0.  Excludes the learned terminator (chi0_set_terminator).
 * Errors: CHI0_EINVAL (eps_bar not finite, learned terminator set). */
chi0_status chi0_set_bg_terminator(chi0_ctx* ctx, int on, double eps_bar);

/* ---- Degenerate-pole grouping and the double grid ------------------------------
 * Appendix B (Eqs. X_IP_split, split1, split2): chi0 is a sum of frequency
 * factors F(w) of the pole energies d_t = eps_{m,k-q} - eps_{n,k} times
 * frequency-independent rho rho^* terms, and poles closer than eps_thresh
 * share one factor.  With eps_thresh > 0 the poles of the transitions that
 * carry weight are sorted by energy (ties in transition order); a group
 * opens at the smallest pole not yet taken (its representative) and takes
 * every following pole with d_t - d_rep < eps_thresh; every member uses the
 * representative's factor.  eps_thresh = 0 (the default) switches it off.
 * The paper's input CGrdSpXd = 100 means eps_thresh = 1e-5 Ha.
 * The double grid (the dense-grid paragraph of the Bethe-Salpeter section)
 * replaces the factor of each transition by its mean over nd transitions of
 * a dense grid: eps_dense is a host array [nk][nd][nbands] (Ha) holding the
 * energies of nd dense points around each coarse k (point j of k and point j
 * of k - q form one dense transition); the occupation factor stays that of
 * the coarse grid.  nd = 0 switches it off; the two options exclude each
 * other.  Both act on the weights of every following chi0_build_chi0 /
 * chi0_build_invert (and batch creation); the tensor-core contraction is
 * unchanged (it sums over every transition either way).
 * Errors: CHI0_EINVAL (threshold negative or not finite; nd out of
 * [0, 4096]; NULL or non-finite energies; both options set), CHI0_ENOMEM,
 * CHI0_ECUDA. */
chi0_status chi0_set_pole_grouping(chi0_ctx* ctx, double eps_thresh);

/* The grouping of the last planned chi0 (chi0_build_chi0 / chi0_build_invert
 * plan it): *ngroups receives the number of pole groups (0 with grouping
 * off), *grouped_contraction 1 when the groups were large enough for the
 * grouped contraction.  In the mixed form on the imaginary axis, with neither
 * correction nor band-block streaming, and when the groups average at least
 * 32 transitions (padding to 64 at most doubles them) and their sums fit in
 * 30% of the free device memory, chi0 is built as Appendix B writes it: one
 * contraction over the transitions in group order gives every group's
 * frequency-independent sum M_g = sum_{t in g} f_s/(N_k Omega)
 * (f_m - f_n) rho_t rho_t^H, and each frequency is then
 * chi0(w) = sum_g F(w, d_g) M_g with the representative's factor, so the
 * tensor-core work no longer grows with the number of frequencies.  Either
 * way chi0 is the same sum.  Errors: CHI0_EINVAL, CHI0_ESTATE (nothing
 * planned). */
chi0_status chi0_get_pole_groups(chi0_ctx* ctx, int64_t* ngroups, int* grouped_contraction);
chi0_status chi0_set_double_grid(chi0_ctx* ctx, int nd, const double* eps_dense);

/* ---- Self-energy kernel I (full-frequency GW) --------------------------------
 * Full frequency GW subsection, Eqs. (W_def), (W_delta), (I_c):
 *   I^{ab k}_{m q}(w) = -1/(N_k Omega) sum_{G,G'} W^d_GG'(q,w) rho_{amk}(q,G) conj(rho_{bmk}(q,G')),
 * W = V eps~^-1 V (Eq. W_def in the symmetric form, V_i = sqrt(4 pi)/|q+G_i|),
 *   W^d_GG' = 1/2 Im(W_GG' + W_G'G) - i/2 Re(W_GG' - W_G'G)   (Eq. W_delta),
 * a, b bands of the quasiparticle window [qp_lo, qp_hi) at k, m every band
 * (0 .. nbands-1) at k - q, rho of Eq. (rhotw) as for chi0, for every k of
 * the grid.  W^d vanishes where eps~^-1 is Hermitian (imaginary axis); it is
 * the spectral part of W on the real axis.
 *   eps_inv: DEVICE pointer, [nw][ng][ng] complex128: eps~^-1 of the response
 *            set of q index iq at nw frequencies (as written by
 *            chi0_invert_eps / chi0_build_invert with out_on_device = 1, or
 *            by chi0_ppa_eval); read only.
 *   out:     [nw][nk][nbands][nqp][nqp] complex128, nqp = qp_hi - qp_lo,
 *            entry [w][k][m][a - qp_lo][b - qp_lo]; device (out_on_device = 1,
 *            asynchronous on the context's stream) or host (synchronises).
 * The contraction sum_j W^d_ij conj(rho(j)) runs on the tensor cores in the
 * mixed form (BF16x3 products, FP32 accumulation in 128-term pieces, FP64
 * sums), in plain FP64 in the FP64 form.  Requires chi0_compute_rho(iq)
 * (mixed-grid wavefunctions and the response set).  Device memory: rho of
 * the window (nk nbands nqp ng complex) and an N_G x nk nbands nqp FP64
 * complex work array.
 * Errors: CHI0_EINVAL (window empty or outside [0, nbands), NULL pointer,
 * nw < 1, |q+G| = 0), CHI0_EUNSUPPORTED (more than 64 bands in the window,
 * or too many transitions for one contraction), CHI0_ESTATE, CHI0_ENOMEM,
 * CHI0_ECUDA, CHI0_ETIMEOUT. */
chi0_status chi0_build_sigma_i(chi0_ctx* ctx, int iq, int qp_lo, int qp_hi, const void* eps_inv, int nw,
                               void* out, int out_on_device);

/* ---- Godby-Needs plasmon-pole model ------------------------------------------
 * Full frequency GW subsection: eps^-1_GG'(w) is modelled by one pole pair per
 * element, its two parameters chosen so that the model reproduces eps^-1 at
 * w = 0 and at w = i omega_p (PPAPntXp, default 1 Ha).  With
 * x(w) = eps^-1_GG'(w) - delta_GG' the model is, in the retarded form of the
 * chi0 weights,
 *   x(w) = R [1/(w - wt + i eta) - 1/(w + wt + i eta)],
 * so that wt^2 = omega_p^2 x(i omega_p) / (x(0) - x(i omega_p)) and
 * R = -x(0) wt / 2 (wt the principal square root).  An element with
 * Re wt^2 <= 0, or with x(0) = x(i omega_p), has no real pole and keeps its
 * static value: wt = 0 and R = x(0) mark it.
 * All matrices are device pointers, [ng][ng] complex128 (row-major, the
 * layout of chi0_invert_eps's output for one frequency), owned by the caller;
 * the calls are asynchronous on cuda_stream (NULL = default stream) and
 * allocate nothing.
 * Errors: CHI0_EINVAL (NULL pointer, ng < 1, omega_p not finite and > 0),
 * CHI0_ECUDA. */
chi0_status chi0_ppa_fit(const void* eps_inv_0, const void* eps_inv_p, int ng, double omega_p,
                         void* omega_t, void* R, void* cuda_stream);

/* eps^-1 of the model at nf complex frequencies: freqs is a host array of nf
 * (re, im) pairs (copied; may be NULL when nf = 0), eta >= 0 the broadening,
 * out a device pointer to [nf][ng][ng] complex128.  A frequency on a pole
 * (w + i eta = +-wt exactly) gives an infinite entry.  Errors: CHI0_EINVAL
 * (NULL pointer, ng < 1, nf < 0, eta or a frequency not finite, eta < 0),
 * CHI0_ECUDA. */
chi0_status chi0_ppa_eval(const void* omega_t, const void* R, int ng, const double* freqs, int nf,
                          double eta, void* out, void* cuda_stream);

/* Text of the last error on ctx (static storage inside ctx; never NULL). */
const char* chi0_last_error(const chi0_ctx* ctx);

/* Release all device and host memory of ctx (synchronises its stream). */
void chi0_destroy(chi0_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CHI0_H_ */
