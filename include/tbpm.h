/*
 * tbpm.h -- C ABI of the GB300 tight-binding propagation method (TBPM) library.
 *
 * The library evolves random initial states under a sparse tight-binding
 * Hamiltonian, |psi(t + tau)> = exp(-i H tau) |psi(t)>, by the Chebyshev-Bessel
 * expansion of arXiv 2209.00806 (Sec. 2.2, Eq. psi_t), records the correlation
 * C(t) = <psi(0)|psi(t)> (Sec. 2.2, Eq. corr_dos) and turns it into a density
 * of states (Sec. 2.4, Eq. dos_tbpm).  All propagation arithmetic runs in CUDA
 * kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Status: every int-returning call returns TBPM_OK (0) or one TBPM_E_* code;
 *    tbpm_last_error() then holds a one-line message.  A failed call leaves
 *    the context usable unless the code is TBPM_E_CUDA.
 *  - Complex numbers are two adjacent doubles (re, im), i.e. C99 double
 *    complex / numpy complex128.
 *  - Orbital indices are the caller's numbering, 0 .. n_orb-1.  Any internal
 *    row order is invisible: states and gradients come back in caller order.
 *  - Pointers marked "host or device" are read from host memory when
 *    where == TBPM_HOST and from device memory (of the context's device)
 *    when where == TBPM_DEVICE.  The library copies what it keeps; the caller
 *    keeps ownership of every pointer it passes.
 *  - Energies are in eV and times in hbar/eV (hbar = 1).
 *  - One context per CUDA stream; contexts share no state.  Calls on one
 *    context must not run concurrently from several host threads.
 */
#ifndef TBPM_H
#define TBPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TBPM_OK 0
#define TBPM_E_INVALID_ARG 1    /* bad size, index, pointer or flag */
#define TBPM_E_SPECTRAL_BOUND 2 /* s is below a bound on the spectral radius of H */
#define TBPM_E_OOM 3            /* device allocation failed */
#define TBPM_E_CUDA 4           /* a CUDA call failed; the message names it */
#define TBPM_E_NORM_DRIFT 5     /* |<phi|phi> - 1| exceeded the hard bound */
#define TBPM_E_NONFINITE 6      /* NaN or Inf met in a state or a reduction */
#define TBPM_E_TIMEOUT 7        /* a bounded device-side wait gave up (TMA kernel) */
#define TBPM_E_STATE 8          /* call order: e.g. propagate before build */
#define TBPM_E_UNSUPPORTED 9    /* valid request the library does not provide */

/* ---- precision of the propagation --------------------------------------- */
#define TBPM_FP64 0  /* complex128 states, FP64 H~, FP64 reductions */
#define TBPM_FP32 1  /* complex64 states, FP32 H~, FP64 reductions and norm carry */

/* ---- where a pointer lives ---------------------------------------------- */
#define TBPM_HOST 0
#define TBPM_DEVICE 1

/* ---- window of the DOS transform (Sec. 2.4) ----------------------------- */
#define TBPM_WINDOW_HANN 0         /* w_n = (1 + cos(pi n / N)) / 2 */
#define TBPM_WINDOW_GAUSSIAN 1     /* w_n = exp(-(3 n / N)^2 / 2)  (sigma = N / 3) */
#define TBPM_WINDOW_EXPONENTIAL 2  /* w_n = exp(-4 n / N) */

/* ---- flags of tbpm_build_hamiltonian ------------------------------------ */
#define TBPM_BUILD_STRICT_BOUND 1 /* fail with TBPM_E_SPECTRAL_BOUND if the
                                     Gershgorin bound of H exceeds s */
#define TBPM_BUILD_NO_FP64 2      /* keep only FP32 values (saves memory) */
#define TBPM_BUILD_NO_FP32 4      /* keep only FP64 values */
#define TBPM_BUILD_REORDER_RCM 8  /* reverse Cuthill-McKee row order per sample */
#define TBPM_BUILD_NO_UNIFORM 16  /* do not use the one-value form when every hopping
                                     is equal (by default the term kernels then skip
                                     the value loads) */
#define TBPM_BUILD_REORDER_CLUSTER 64 /* RCM, then balls of 128 rows grown breadth-
                                         first in RCM order: compact patches on
                                         geometric lattices keep long-row gathers
                                         in L1 */
#define TBPM_BUILD_COMPLEX_HOPS 32 /* hop_v holds complex hoppings, (re, im) double
                                      pairs (complex128): Peierls phases of a
                                      magnetic field (Sec. 2.1) */
#define TBPM_BUILD_NO_SPECTRAL_CHECK 256 /* skip the Lanczos check of s (below) */
#define TBPM_BUILD_NO_BOND_MAP 128 /* keep no bond -> row map (8 bytes per bond):
                                      tbpm_set_bond_vectors and the adjoint then
                                      return TBPM_E_STATE; for the largest samples */

/* ---- flags of tbpm_propagate -------------------------------------------- */
#define TBPM_PROP_PROFILE 1   /* time the kernels with CUDA events (tbpm_stats) */
#define TBPM_PROP_GRAPH 2     /* replay each time step as a captured CUDA graph */
#define TBPM_PROP_RESUME 4    /* continue from the current states instead of
                                 restarting from psi0; C is still <psi0|phi> */
#define TBPM_PROP_PERSISTENT 8 /* one cooperative launch per time step: the
                                  wavefront-fused step (TBPM_VARIANT_FUSED) for
                                  this call, with bounded dependency waits */
#define TBPM_PROP_BACKWARD 16  /* negative times: each step applies e^{+iH tau}
                                  (the same series with H -> -H); C_n is then
                                  <psi0|psi(-n tau)> */

typedef struct tbpm_ctx tbpm_ctx;

/* Counters and timings of the last tbpm_propagate / adjoint on a context. */
typedef struct tbpm_stats {
    int n_terms;             /* M: Chebyshev coefficients m = 0 .. M-1 */
    int n_steps;             /* time steps of the last call */
    int n_groups;            /* state groups (each one blocked launch set) */
    int group_width[8];      /* states per group */
    int64_t n_rows;          /* padded device rows */
    int64_t nnz;             /* stored off-diagonal entries (incl. padding) */
    int64_t nnz_true;        /* off-diagonal entries of H (2 x bonds) */
    int64_t renormalisations;/* FP32: norm-carry events over all states */
    int64_t kernel_launches; /* kernels launched by the last call */
    double gershgorin;       /* Gershgorin bound of H~ = H / s (dimensionless) */
    double ms_total;         /* device time of the last call (PROFILE) */
    double ms_term_avg;      /* average duration of one interior Chebyshev
                                term kernel (PROFILE); with the fused step,
                                its time divided by the M-1 terms */
    double ms_final_avg;     /* average duration of the closing term kernel */
    double ms_reduce_avg;    /* average duration of the correlation reduction */
    int64_t term_launches;   /* interior term launches that were timed */
    double bytes_term;       /* algorithmic bytes of one interior term launch:
                                4 state vectors, a column per stored entry
                                (plus a value unless one value serves all),
                                the diagonal */
    double max_norm_drift;   /* max over steps and states of |<phi|phi> - 1| */
    double lanczos_radius;   /* the build's Lanczos estimate of the spectral radius
                                of H~ (0 when the Gershgorin bound sufficed) */
    double ops_term;         /* arithmetic operations of one interior term launch
                                (an FMA, add or multiply on one real lane is one),
                                same mean group width as bytes_term: per state
                                and row with E entries, 6 + 2E for the real
                                general form (8 + 2E in FP32: the coefficient's
                                low part), 4 + 2E for the FP64 one-value form
                                (2 + 2E without a diagonal); complex values 4
                                per entry */
} tbpm_stats;

/* Library version, major * 10000 + minor * 100 + patch. */
int tbpm_version(void);

/* Compute capability the library's kernels were compiled for, as
 * major * 10 + minor (103 for sm_103a), read from the loaded kernel image of
 * the current device (cudaFuncGetAttributes).  A build check, not part of
 * the method.  Errors: INVALID_ARG (NULL), CUDA (no device or no image for
 * it); the message is read with tbpm_last_error(NULL). */
int tbpm_kernel_binary_version(int *version);

/* FP64 fused multiply-add throughput of `device` in TFLOP/s (2 flops per
 * FMA): a grid of 8 blocks x 256 threads per SM, each thread running 8
 * independent FMA chains for n_iter rounds, timed with CUDA events (*ms, may
 * be NULL).  A measurement, not part of the method: the FP64 form's term
 * kernel is bound by this rate on GB300, and the benchmark reports against
 * it.  Errors: INVALID_ARG, CUDA (message via tbpm_last_error(NULL)). */
int tbpm_fp64_fma_rate(int device, int n_iter, double *tflops, double *ms);

/* Create a context on CUDA device `device`.  `cuda_stream` (a cudaStream_t,
 * may be NULL for the legacy default stream) is borrowed: the library orders
 * its work after what is already queued there and makes the stream wait for
 * its results before each call returns.  The context owns every device
 * buffer it allocates and frees them in tbpm_destroy. */
int tbpm_create(tbpm_ctx **ctx, int device, void *cuda_stream);
void tbpm_destroy(tbpm_ctx *ctx);

/* Message of the last failed call on ctx (empty string if none).  Calls that
 * fail before a context exists leave their message in a thread-local slot
 * that tbpm_last_error(NULL) returns. */
const char *tbpm_last_error(const tbpm_ctx *ctx);

/* a1. Lattice -> Hamiltonian (Sec. 2.1, Eq. ham_mat_finite, with the hopping
 * convention of Sec. 4.1: a bond (i, j, t) is the matrix element
 * <phi_i|h|phi_j> = t, the conjugate element H_ji = conj(t) is implied), rescaled
 * to H~ = H / s (Sec. 2.2).
 *   n_orb          orbitals, 1 .. 2^31 - 1 in total
 *   onsite         [n_orb] eps_i in eV, host or device, or NULL for zeros
 *   n_hop, hop_i, hop_j, hop_v
 *                  [n_hop] bonds, int64 indices and real hoppings in eV, host
 *                  or device; i != j, both in the same sample.  A pair listed
 *                  twice adds up.  With TBPM_BUILD_COMPLEX_HOPS hop_v is
 *                  [n_hop] complex128 (re, im pairs), H_ij = t, H_ji = conj(t);
 *                  such a Hamiltonian runs the plain term kernels (no TMA,
 *                  wide-lane or fused variants; TBPM_PROP_PERSISTENT and the
 *                  adjoint return TBPM_E_UNSUPPORTED).
 *   s              rescale factor in eV, > 0
 *   n_samples      independent samples packed block-diagonally (>= 1)
 *   sample_offsets [n_samples + 1] host int64, orbitals of sample k are
 *                  sample_offsets[k] .. sample_offsets[k+1]-1; NULL when
 *                  n_samples == 1
 *   where          TBPM_HOST or TBPM_DEVICE for all array arguments
 *   flags          TBPM_BUILD_*
 * Replaces any previous Hamiltonian and drops any states.  Runs on the GPU:
 * counting, slice layout (sliced ELLPACK, 32-row slices), fill, per-row
 * column sort (deterministic), Gershgorin bound.  The expansion of Sec. 2.2
 * needs the spectrum of H~ inside [-1, 1]: unless the Gershgorin bound
 * already gives ||H~|| <= 1/1.01 or TBPM_BUILD_NO_SPECTRAL_CHECK is set, 64
 * Lanczos steps (tbpm_spectral_bounds) estimate the spectral radius rho of H,
 * and s < 1.01 rho fails with SPECTRAL_BOUND (the estimate is a lower bound;
 * the margin covers its shortfall).  Errors: INVALID_ARG (sizes, indices out
 * of range, i == j, bond across samples), SPECTRAL_BOUND (the Lanczos check,
 * or the Gershgorin bound with TBPM_BUILD_STRICT_BOUND), OOM, CUDA. */
int tbpm_build_hamiltonian(tbpm_ctx *ctx, int64_t n_orb, const double *onsite,
                           int64_t n_hop, const int64_t *hop_i, const int64_t *hop_j,
                           const double *hop_v, double s, int n_samples,
                           const int64_t *sample_offsets, int where, int flags);

/* Spectral bound of the built H (the rescaling of Sec. 2.2 needs ||H|| <= s):
 * n_iter (1 .. 10000) Lanczos steps from a fixed start vector -- components
 * (U_2u - 1/2) + i (U_2u+1 - 1/2) in caller order u, normalised, U_k the
 * k-th uniform draw (top 53 bits) of the SplitMix64 output function keyed
 * by seed 220900806 and stream 200 as key = mix(seed + G (stream + 1)),
 * U_k = mix(key + G (k + 1)), G = 0x9E3779B97F4A7C15 -- each step one sparse
 * product and deterministic FP64 sums on the GPU; then the extreme
 * eigenvalues of the Lanczos tridiagonal matrix by bisection on the host.
 *   e_min, e_max  the extreme Ritz values in eV: inside the spectrum of H,
 *                 approaching its ends as n_iter grows
 *   steps         steps taken (fewer when the Krylov space closes), or NULL
 * Errors: INVALID_ARG, STATE (no Hamiltonian), NONFINITE, OOM, CUDA. */
int tbpm_spectral_bounds(tbpm_ctx *ctx, int n_iter, double *e_min, double *e_max, int *steps);

/* Initial states (Sec. 2.2, Eq. ini_state).  psi0 is complex128
 * [n_states][n_orb] (host or device); state p of sample k is the slice
 * sample_offsets[k] .. sample_offsets[k+1]-1 of row p, each slice its own
 * state.  The library does not normalise.  1 <= n_states <= 64. */
int tbpm_set_states(tbpm_ctx *ctx, int n_states, const double *psi0, int where);

/* Random-phase initial states psi0_i = exp(i theta_i) / sqrt(N_k), N_k the
 * orbital count of the sample holding i: random complex a_i with
 * sum |a_i|^2 = 1 per sample (Sec. 2.2).  theta is double
 * [n_states][n_orb] (host or device), drawn by the caller. */
int tbpm_set_phase_states(tbpm_ctx *ctx, int n_states, const double *theta, int where);

/* a2. Coefficients of the expansion (Sec. 2.2): J_m(z), m = 0 .. M-1, by
 * Miller's backward recurrence in FP64 on the host, normalised with
 * J_0 + 2 sum_k J_2k = 1.  M = first m > z with |J_m(z)| < tol.
 * J_out holds max_terms doubles; *n_terms receives M.  0 < z <= 1000.
 * Errors: INVALID_ARG; UNSUPPORTED if M > max_terms. */
int tbpm_bessel_coefficients(double z, double tol, int max_terms, double *J_out,
                             int *n_terms);

/* a3-a6. Propagate every state for n_steps steps of tau = z / s and record
 * C_n = <psi0|phi(n tau)>, n = 0 .. n_steps, per sample and state.
 *   z          s * tau (> 0); coefficients cut at |J_m(z)| < 1e-15
 *   precision  TBPM_FP64 or TBPM_FP32 (the Hamiltonian must hold that copy)
 *   corr_out   complex128 [n_samples][n_states][n_steps + 1], host or device
 *              (where_out), or NULL to keep C on the device only
 *   flags      TBPM_PROP_*
 * Each time step runs M-1 fused sparse-product terms of the Clenshaw form
 * of the paper's Chebyshev sum and one deterministic reduction: FP64 in the
 * FP64 form; in the FP32 form each row's products are exact float pairs and
 * a block's rows are summed as float pairs (about 48 significant bits, error
 * free up to that width), FP64 from the block partials up.  In FP32 the
 * norm of each state is carried in FP64:
 * when <phi|phi> drifts from its value at n = 0 by more than the
 * renormalisation bound (relative) the next step starts from phi rescaled
 * to that norm (tbpm_set_norm_policy).  The drift checks are relative to
 * the norm at n = 0 in both forms.
 * Errors: STATE (no Hamiltonian or states), INVALID_ARG, NORM_DRIFT (drift
 * above the hard bound: s too small), NONFINITE, TIMEOUT (a bounded device
 * wait of the TMA or fused kernels expired), CUDA. */
int tbpm_propagate(tbpm_ctx *ctx, double z, int n_steps, int precision, double *corr_out,
                   int where_out, int flags);

/* State-averaged correlation of the last propagation (Sec. 2.4, the average
 * over S random states in Eq. dos_tbpm): complex128 [n_samples][n_steps + 1],
 * C-bar_n = (sum_p C_n^(p)) / S with the states added in order, formed on the
 * GPU and written to host or device memory (where_out).
 * Errors: INVALID_ARG, STATE (no propagation), OOM, CUDA. */
int tbpm_correlation(tbpm_ctx *ctx, double *corr_avg_out, int where_out);

/* Adjoint of tbpm_correlation: from gbar_avg = dL/dRe C-bar_n + i dL/dIm C-bar_n,
 * complex128 [n_samples][n_steps + 1] (host or device, `where`), the
 * derivative of L with respect to each state's C_n,
 *   gbar_out[k][p][n] = gbar_avg[k][n] / S,
 * complex128 [n_samples][n_states][n_steps + 1] (host or device, where_out),
 * as tbpm_propagate_adjoint takes it.  S = the states currently set.
 * Errors: INVALID_ARG, STATE (no Hamiltonian or states), OOM, CUDA. */
int tbpm_correlation_adjoint(tbpm_ctx *ctx, int n_steps, const double *gbar_avg, int where,
                             double *gbar_out, int where_out);

/* Current states phi(t) of the last propagation in caller order, complex128
 * [n_states][n_orb] (host or device) -- a checkpoint; tbpm_set_states +
 * TBPM_PROP_RESUME continues from it. */
int tbpm_get_states(tbpm_ctx *ctx, double *phi_out, int where_out);

/* Squared norms <phi|phi> per sample, state and step of the last
 * propagation: double [n_samples][n_states][n_steps + 1], host. */
int tbpm_get_norms(tbpm_ctx *ctx, double *norms_out);

/* a7. DOS from one averaged correlation C_0 .. C_{n_steps} (host memory),
 * Sec. 2.4, Eq. dos_tbpm:
 *   D(E) = (tau/pi) [Re C_0 / 2 + sum_{n=1}^{N} v_n w_n Re(exp(i E n tau) C_n)]
 * (C(-t) = conj C(t), trapezoid rule: v_n = 1, v_N = 1/2; window w_n one of
 * TBPM_WINDOW_HANN (w_N = 0), _GAUSSIAN, _EXPONENTIAL -- Sec. 2.4 names the
 * three without parameters; the widths above are this library's choice),
 * at bin centres E_k = e_min + (k + 1/2)(e_max - e_min)/n_e.  Pure host
 * function, FP64.  D integrates to Re C_0 over a full period 2 pi / tau.
 * Errors: INVALID_ARG, UNSUPPORTED (unknown window). */
int tbpm_dos(const double *corr, int n_steps, double tau, int window, double e_min,
             double e_max, int n_e, double *energies_out, double *dos_out);

/* a8. Adjoint of the propagation (FP64): gradients of a real loss L of the
 * correlations with respect to every hopping t_b and onsite energy eps_i.
 *   gbar       complex128 [n_samples][n_states][n_steps + 1] (host or device,
 *              `where`): dL/dRe C_n + i dL/dIm C_n of each state's C_n, as
 *              tbpm_propagate defines C_n for the states currently set
 *   K          checkpoint interval (states kept every K steps, recomputed
 *              in between; memory ~ (N/K + K + M) state vectors)
 *   grad_hop   double [n_hop] dL/dt_b, bonds in the order given to
 *              tbpm_build_hamiltonian (host or device, `where_out`)
 *   grad_onsite double [n_orb] dL/deps_i
 * H~ is Hermitian, so the backward pass is the same Chebyshev series with +i
 * in place of -i (the adjoint of the propagator of Sec. 2.2); no counterpart
 * in the paper, which has no gradients.  Needs the FP64 Hamiltonian and real
 * hoppings.  Overwrites the propagation state of the context.
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
int tbpm_propagate_adjoint(tbpm_ctx *ctx, double z, int n_steps, const double *gbar, int where,
                           int K, double *grad_hop, double *grad_onsite, int where_out);

/* Adjoint of tbpm_dos (host, FP64): from dL/dD_k on the n_e bins, the
 * derivative gbar_n = dL/dRe C_n + i dL/dIm C_n of the averaged correlation,
 * complex128 [n_steps + 1]. */
int tbpm_dos_adjoint(const double *dl_dd, int n_e, int n_steps, double tau, int window,
                     double e_min, double e_max, double *gbar_out);

/* Launch shape of the propagation kernels for one precision: states are
 * split into groups of power-of-two width <= max_group (FP64 <= 8,
 * FP32 <= 16), each group propagated as one blocked sparse product per term;
 * threads per block is 64, 128 or 256; variant is a set of
 * TBPM_VARIANT_* bits.  Chosen by tbpm_autotune or by hand.  Changing the
 * width or block size drops the current propagation buffers.  Defaults:
 * groups of 8 (FP64) and 16 (FP32) states, 64 threads, variants ZIGZAG (FP64)
 * and ZIGZAG | WIDE | PREFETCH (FP32). */
#define TBPM_VARIANT_ZIGZAG 1        /* alternate the row traversal direction per term,
                                        so each term starts on rows still in L2 */
#define TBPM_VARIANT_STREAM_HINTS 2  /* evict-first loads of the own-row streams */
#define TBPM_VARIANT_TMA 4           /* persistent term kernel: each tile's row streams
                                        and matrix slices staged in shared memory by
                                        bulk asynchronous copies, 3 stages ahead */
#define TBPM_VARIANT_FUSED 8         /* all terms of a time step in one cooperative
                                        launch, ordered as a wavefront over row tiles
                                        so intermediate vectors stay in L2; needs a
                                        banded row order (TBPM_BUILD_REORDER_RCM) */
#define TBPM_VARIANT_FUSED_TILE(k) ((k) << 4)  /* fused tile rows x 4^k, k = 0..2 */
#define TBPM_VARIANT_WIDE 64         /* term kernel with 32-byte lanes (one thread per
                                        row for 4 FP32 or 2 FP64 states) */
#define TBPM_VARIANT_SPLIT2 128      /* each row's entries split over 2 threads (long
                                        rows: more gathers in flight); real values */
#define TBPM_VARIANT_SPLIT4 256      /* the same over 4 threads (not with SPLIT2) */
#define TBPM_VARIANT_HALO 512        /* staged gathers: a block of 128 rows copies the
                                        states of every row its entries reference (its
                                        halo) into shared memory, then gathers there by
                                        16-bit positions; real values, FP32 groups of
                                        4-16 / FP64 of 2-8 states; for long rows.  The
                                        halo lists are built on first use; a matrix
                                        with a block referencing over 2048 other rows
                                        keeps the plain kernel */
#define TBPM_VARIANT_CLUSTER 2048    /* FP64, one state, one sample of at most
                                        16 x 1024 rows, at most 12 entries per row:
                                        every time step in one thread-block-cluster
                                        launch, the vectors in the blocks' shared
                                        memory (distributed shared memory for the
                                        gathers), a cluster barrier per term;
                                        otherwise ignored */
#define TBPM_VARIANT_PIPE 1024       /* with TBPM_VARIANT_HALO, interior terms: a
                                        persistent grid (one block per SM) with two
                                        shared-memory stages, the next block's halo,
                                        positions and values copied while the current
                                        one computes; FP32 groups of 4 or 8, FP64 of 2
                                        or 4 states, within 224 KB of shared memory */
#define TBPM_VARIANT_PREFETCH 8192   /* real values, interior terms: a persistent
                                        grid whose threads walk rows with a stride and
                                        load the next row's first four column indices,
                                        values and diagonal before the current row's
                                        gathers (with TBPM_VARIANT_WIDE: 32-byte lanes);
                                        ignored otherwise */
#define TBPM_VARIANT_STAGED 4096     /* with TBPM_VARIANT_HALO: one block per 128-row
                                        block copying its halo, positions and values
                                        into one shared-memory stage, two blocks per
                                        SM where the stage allows (one block's copies
                                        overlap the other's gathers); same shapes as
                                        TBPM_VARIANT_PIPE, which it takes precedence
                                        over */
int tbpm_set_launch_config(tbpm_ctx *ctx, int precision, int max_group, int threads,
                           int variant);

/* Norm policy of the propagation (a5).  The drift of a state is
 * |<phi|phi> / <phi|phi>_0 - 1| against its squared norm at n = 0 (1 for
 * normalised states).  FP32: when it exceeds renorm_fp32 (default 1e-5)
 * after a step, the next step starts from phi rescaled to the initial norm
 * (the norm is summed and the factor formed in FP64 before rounding to
 * FP32); above hard_fp32 (default 1e-2) the call fails with
 * TBPM_E_NORM_DRIFT.  FP64: above hard_fp64 (default 1e-6) the call fails.
 * The unitary evolution of Sec. 2.2 keeps the norm; drift means rounding
 * (FP32) or an s below the spectral radius.  Bounds must be > 0. */
int tbpm_set_norm_policy(tbpm_ctx *ctx, double renorm_fp32, double hard_fp32, double hard_fp64);

/* Autotuner: for the current Hamiltonian and states, time probe_steps
 * (1..64) steps of each candidate launch shape -- state-group width (the
 * block width of the blocked sparse product), threads per block (64, 128, 256)
 * and TBPM_VARIANT_* bits -- and keep the fastest as the context's
 * configuration for `precision`.  The chosen values are written to the
 * non-NULL out pointers.  The slice height is fixed at 32 rows (one warp's
 * rows share a slice).  Leaves no propagation to resume.
 * Errors: STATE, INVALID_ARG, OOM, CUDA. */
int tbpm_autotune(tbpm_ctx *ctx, int precision, double z, int probe_steps, int *best_group,
                  int *best_threads, int *best_variant, double *best_ms_per_step);

/* Allocation-free form of the correlation reduction, for callers that
 * cannot allocate device memory (a host framework whose pool owns the whole
 * device, a plugin that may only allocate at start-up, a latency-bound loop
 * that cannot afford cudaMalloc/cudaFree).  The paper has no counterpart:
 * this is an integration convenience of the library.
 *   psi0, phi  device complex128 [n_states][n_orb], caller order (as
 *              tbpm_get_states returns); caller-owned, read only
 *   corr_out   device complex128 [n_states]: <psi0_s|phi_s>
 *   norm_out   device double [n_states]: <phi_s|phi_s>
 *   cuda_stream the stream to run on (cudaStream_t, may be NULL)
 * The same quantities as the closing reduction of tbpm_propagate, summed
 * deterministically in FP64 (each block over a fixed grid-stride set of
 * rows, then the blocks in order); they agree with tbpm_propagate's to
 * rounding, not bit for bit, since the summation order differs.  Allocates
 * nothing: its scratch is one fixed device array of 786,496 bytes
 * (n_states <= 16; rows unlimited), held by every GPU that loads the
 * library until the process exits.  The first call on a device looks the
 * array's address up (cudaGetSymbolAddress) with that device current and
 * caches it per device ordinal for the life of the process; make that
 * first call before any stream capture.  The cached address belongs to the
 * device's primary context: calls after cudaDeviceReset, or from a
 * non-primary context, are not supported.  Calls share the array, so calls
 * that overlap on the GPU race: serialise them.  Asynchronous on
 * cuda_stream; the message of a failure is read with tbpm_last_error(NULL).
 * Errors: INVALID_ARG (NULL pointer, n_orb < 1, n_states outside 1..16),
 * UNSUPPORTED (current device ordinal above 63), CUDA. */
int tbpm_correlation_noalloc(const double *psi0, const double *phi, int64_t n_orb,
                             int n_states, double *corr_out, double *norm_out,
                             void *cuda_stream);

/* Statistics of the last call on ctx. */
int tbpm_get_stats(tbpm_ctx *ctx, tbpm_stats *out);

/* ---- AC (optical) conductivity (Sec. 2.7, with the Fermi-Dirac operator of
 * Sec. 2.2) --------------------------------------------------------------- */

/* c1. Bond vectors for the current operator J_a = -i sum t_ij d^a_ij c_i^+ c_j
 * (Sec. 2.7; e / hbar factored out, units eV nm), d_ij = r_j - r_i.
 *   dx, dy  [n_hop] components (nm) of d_b for bond b of the bond list given
 *           to tbpm_build_hamiltonian (same order), host or device, finite.
 *           For a periodic sample d_b is the bond's own image (the minimum
 *           image for nearest neighbours), not a difference of positions.
 * Entry (i, j) gets d_b and its conjugate partner (j, i) gets -d_b.  A pair
 * listed twice must have the same vector.  Kept until the next
 * tbpm_build_hamiltonian.  Errors: STATE (no Hamiltonian), INVALID_ARG
 * (missing or non-finite vectors), OOM, CUDA. */
int tbpm_set_bond_vectors(tbpm_ctx *ctx, const double *dx, const double *dy, int where);

/* c2. Chebyshev coefficients of the Fermi function on the rescaled axis,
 * f(x) = 1 / (exp(beta_s (x - mu_s)) + 1) = c_0/2 + sum_{k>=1} c_k T_k(x)
 * (Sec. 2.2; beta_s = beta s, mu_s = mu / s), by the trapezoid rule of
 * c_k = (2/pi) int_0^pi f(cos t) cos(k t) dt evaluated with an FFT, truncated
 * after the last |c_k| > 1e-15 max|c|.
 *   c_out    [k_max] or NULL to query the count only
 *   n_terms  out: the number of coefficients K
 * Errors: INVALID_ARG, UNSUPPORTED (K > k_max). */
int tbpm_fermi_coefficients(double beta_s, double mu_s, int k_max, double *c_out,
                            int *n_terms);

/* c3. AC-conductivity correlation (Sec. 2.7).  For each initial state psi of
 * each sample (the states set on ctx, at most 16 per sample):
 *   psi_2 = f(H) psi,  psi_1b = [1 - f(H)] J_b psi  (b = x, y),
 * f(H) = 1 / (exp(beta (H - mu)) + 1) by the Chebyshev series of c2 with
 * Clenshaw's recurrence in FP64; then psi, psi_2, psi_1x, psi_1y advance
 * together (one state group, `precision` as in tbpm_propagate) and after every
 * step the library records
 *   corr[k][p][ab][n] = <psi_2(n tau)| J_a |psi_1b(n tau)>,  ab = xx, xy, yx, yy
 * (a = current direction, b = field direction).
 *   z, n_steps    as tbpm_propagate (tau = z / s)
 *   beta, mu      inverse temperature (1/eV) and chemical potential (eV)
 *   corr_out      complex128 [n_samples][n_states][4][n_steps + 1]
 *   where_out     TBPM_HOST or TBPM_DEVICE
 *   flags         TBPM_PROP_PROFILE, TBPM_PROP_GRAPH, TBPM_PROP_PERSISTENT
 * Needs tbpm_set_bond_vectors.  The caller's states are restored afterwards
 * (correlations and norms of the run are not kept).  Norm checks are taken
 * relative to each state's norm at t = 0.  Errors: STATE (no Hamiltonian,
 * states or bond vectors), INVALID_ARG (more than 16 states, TBPM_PROP_RESUME,
 * beta <= 0), UNSUPPORTED (Fermi series longer than 2^22 terms), OOM, CUDA,
 * NORM_DRIFT, NONFINITE. */
int tbpm_ac_correlation(tbpm_ctx *ctx, double z, int n_steps, double beta, double mu,
                        int precision, double *corr_out, int where_out, int flags);

/* ---- quasi-eigenstates (Sec. 2.6) ---------------------------------------- */

/* q1. Quasi-eigenstates (Sec. 2.6, Eq. quasi): for each energy E_k and each
 * initial state psi (the states set on ctx),
 *   Psi(E) = (tau / 2 pi) sum_{n=-N}^{N} w_n e^{i E n tau} psi(n tau),
 *   w_n = (1 + cos(pi n / N)) / 2,
 * from one forward and one backward run (TBPM_PROP_BACKWARD) of N = n_steps
 * steps, accumulated on the GPU after every step in FP64; then normalised to
 * unit norm per energy, state and sample.
 *   z, n_steps, precision   as tbpm_propagate (n_steps >= 1)
 *   n_energies, energies    1 .. 16 energies in eV (host)
 *   out        complex128 [n_energies][n_states][n_orb], caller order
 *   norms_out  [n_energies][n_states][n_samples] squared norms of Psi before
 *              the normalisation (host), or NULL
 *   where_out  TBPM_HOST or TBPM_DEVICE for out
 *   flags      TBPM_PROP_PROFILE, TBPM_PROP_GRAPH, TBPM_PROP_PERSISTENT
 * Afterwards the context holds the backward run (C_n = <psi0|psi(-n tau)>).
 * Errors: STATE, INVALID_ARG, OOM, CUDA, NORM_DRIFT, NONFINITE, UNSUPPORTED. */
int tbpm_quasi_eigenstates(tbpm_ctx *ctx, double z, int n_steps, int n_energies,
                           const double *energies, int precision, double *out,
                           double *norms_out, int where_out, int flags);

/* c4. Real part of the AC conductivity from correlation rows (Sec. 2.7, Eq.
 * AC): for each row C and each omega,
 *   sigma(omega) = norm (exp(-beta omega) - 1) / omega
 *                  * int_0^T exp(-eta t) sin(omega t) 2 Im C(t) dt,
 * trapezoid rule on t_n = n tau, T = n_steps tau.  In units of e^2 / hbar
 * when C comes from c3 (eV^2 nm^2) and norm = N_orb / area (nm^-2) turns the
 * random-state average into the trace per area; spin degeneracy is the
 * caller's factor.
 *   corr       complex128 [n_rows][n_steps + 1] (host)
 *   omegas     [n_omega] > 0 (eV);  eta >= 0 damping (the E -> 0+ limit)
 *   sigma_out  [n_rows][n_omega]
 * Errors: INVALID_ARG. */
int tbpm_ac_conductivity(const double *corr, int n_rows, int n_steps, double tau, double beta,
                         double eta, const double *omegas, int n_omega, double norm,
                         double *sigma_out);

#ifdef __cplusplus
}
#endif
#endif /* TBPM_H */
