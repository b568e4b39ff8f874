// Internal declarations of the TBPM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tbpm.h"

namespace tbpm {

// Rows of one sliced-ELLPACK slice.  Entry k of local row r of slice q sits
// at slice_ptr[q] + k * kSliceRows + r, so the rows of a warp read
// consecutive words for each k.
constexpr int kSliceRows = 32;
// Samples are padded to a multiple of this many rows; it is also the row
// chunk that one partial of the correlation reduction covers.
constexpr int kChunkRows = 1024;
constexpr int kMaxStates = 64;
constexpr int kMaxTerms = 128;
constexpr int kMaxGroups = 64;

// Error-free FP32 transformations for the reductions of the FP32 form.  A
// float pair (hi, lo) with |lo| <= ulp(hi) / 2 carries about 48 significant
// bits: the product of two floats is exactly hi + lo (TwoProduct by FMA),
// and two pairs add with Knuth's TwoSum of the high parts, the low parts
// and the sum's error folded in, then renormalised (Fast2Sum).  Sums of
// FP32 products thus accumulate at FP64-grade accuracy on the FP32 pipe;
// GB300 issues FP64 instructions at a small fraction of the FP32 rate.  The
// _rn intrinsics keep the compiler from contracting or reassociating them.
#ifdef __CUDACC__
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return FF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return FF{h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }
// <a|o> = conj(a) o and |o|^2 of one complex pair, each as an exact pair sum.
__device__ __forceinline__ void ff_dot3(float are, float aim, float ore, float oim, FF &re,
                                        FF &im, FF &nr)
{
    re = ff_add(ff_prod(are, ore), ff_prod(aim, oim));
    im = ff_add(ff_prod(are, oim), ff_neg(ff_prod(aim, ore)));
    nr = ff_add(ff_prod(ore, ore), ff_prod(oim, oim));
}
#endif

// Launch variants of the term kernels (bits of TermArgs::variant).
constexpr int kVariantZigZag = 1;       // alternate the traversal direction per launch
constexpr int kVariantStreamHints = 2;  // evict-first loads of the own-row streams
constexpr int kVariantTma = 4;          // persistent TMA-staged term kernel
constexpr int kVariantFused = 8;        // all terms of a step in one wavefront launch
constexpr int kVariantFusedTileShift = 4;  // bits 4-5: fused tile rows x 4^k
constexpr int kVariantWide = 64;        // term kernel with 32-byte lanes
constexpr int kVariantSplit2 = 128;     // each row's entries over 2 threads
constexpr int kVariantSplit4 = 256;     // each row's entries over 4 threads
constexpr int kVariantHalo = 512;       // gathers from a shared-memory copy of the block's halo
constexpr int kVariantPipe = 1024;      // with kVariantHalo: persistent, two stages in flight
constexpr int kVariantCluster = 2048;   // small FP64 samples: all steps in one cluster launch
constexpr int kVariantStaged = 4096;    // with kVariantHalo: one stage, two blocks per SM
constexpr int kVariantPrefetch = 8192;  // FP32: persistent term kernel, next row's indices loaded ahead

// Staged-gather term kernel: rows per block, and the most other rows one
// block may reference (16-bit positions; the shared copy is sized by the
// longest list of the matrix).
constexpr int kHaloRows = 128;
constexpr int kHaloMaxExt = 2048;
constexpr int kHaloSmemMax = 160 * 1024;   // largest shared copy of a halo (bytes)
constexpr int kPipeSmemMax = 224 * 1024;   // two stages of the pipelined form (bytes)

// Device-side sliced-ELLPACK matrix of H~ (off-diagonal part) plus its
// diagonal, one copy per value precision.
struct SellView {
    const int64_t *slice_ptr;  // [n_slices + 1]
    const int32_t *col;        // [nnz_pad]
    const void *val;           // double or float [nnz_pad], pairs (re, im) if complex
    const void *diag;          // double or float [n_rows]
};

// One Clenshaw term: out = c * psi + gamma * (-i) * H~ x + z, optionally
// with psi scaled per state (FP32 norm carry).
struct TermArgs {
    SellView H;
    const void *x;        // gathered vector
    const void *psi;      // current state (own row only)
    const void *z;        // b_{m+2} (own row) or nullptr
    void *out;            // may alias z
    double c_hi, c_lo;    // coefficient of psi as an unevaluated sum (FP32)
    double gamma;
    float c_hi_f, c_lo_f, gamma_f;  // the same in FP32 (no conversions on the device)
    int x_is_psi;         // apply the state scale to x as well
    const double *scale;  // [n_samples * B] or nullptr
    const float *scale_f; // FP32 copy of scale (read by the FP32 kernels)
    const int32_t *chunk_sample;  // [n_rows / kChunkRows]
    int64_t n_rows;
    int variant;          // kVariant* bits
    int reverse;          // walk the blocks from the end (zig-zag order)
    int uniform;          // every off-diagonal value equals h_uniform (no value loads)
    int cplx;             // complex matrix values (re, im) per entry
    int fixed_width;      // slices all this wide: base = 32 q w, no slice_ptr loads
    double h_uniform;
    float h_uniform_f;
    // FP64 one-value form: out = z + (-i)(gd x + gh s) + c psi with s the sum of
    // the neighbours, gd = gamma d, gh = gamma h_uniform (rounded once, here)
    double gh;
    const double *gdiag;  // gamma d already formed (d or 2d) when |gamma| is 1 or 2, else nullptr
    unsigned long long gdiag_sign;  // sign bit applied to gdiag (gamma < 0)
    int zero_diag;        // every onsite energy is zero: no diagonal term
    // staged-gather variant: halo lists and 16-bit column positions
    const int64_t *halo_ptr;
    const int32_t *halo_rows;
    const uint16_t *lcol;             // packed: entry k of row lr of slice q at
                                      // pslice[q] + (k/4)*128 + lr*4 + k%4
    const int64_t *pslice;
    const void *vpack;                // packed values (pipelined kernel), or nullptr
    int halo_max;
    int halo_ent_max;     // most stored entries of one halo block (pipelined form)
    int num_sms;          // grid of the persistent pipelined form
    // closing term only (H.col == nullptr: reduce `out` without computing it)
    const void *psi0;
    double *partial;        // [n_chunks][B][3]
    double *block_partial;  // [n_blocks][B][3]
    int *chunk_count;       // [n_chunks], zero between launches
};

struct ReduceArgs {
    const double *partial;           // [n_chunks][B][3]
    double *partial2;                // [n_samples][64][B][3]
    unsigned int *sample_ticket;     // [n_samples], zero between launches
    const int64_t *sample_chunk_off; // [n_samples + 1]
    int n_samples;
    int B;
    int group_state0;                // first state of this group
    int n_states;
    int n_steps;
    int *step;                       // device step counter (index of the new C)
    double2 *corr;                   // [n_samples][n_states][n_steps + 1]
    double *norms;                   // [n_samples][n_states][n_steps + 1]
    double *scale;                   // [n_samples * B] next-step scale (FP32) or nullptr
    float *scale_f;                  // its FP32 copy
    double renorm_bound;             // |<phi|phi>/ref - 1| above which to renormalise
    double hard_bound;               // above which to flag NORM_DRIFT
    unsigned long long *renorm_count;
    int *error_flags;                // bit 0 drift, bit 1 non-finite
    double *norm_ref;                // [n_samples][n_states] squared norm at t = 0
    int set_ref;                     // this pass records norm_ref (the C_0 pass)
};

// AC-conductivity correlation (Sec. 2.7).  States of one random state p sit
// in four adjacent lanes 4q .. 4q+3 of a group: psi(t), psi_2(t) = e^{-iHt} f psi,
// psi_1x(t), psi_1y(t) with psi_1b = e^{-iHt} (1 - f) J_b psi.  After each time
// step the observer forms, per row, g_a = sum_c H~_rc d^a_rc psi_2,c and
// conj(g_a) psi_1b,r; the reduction multiplies by i s, so that the entry is
// <J_a psi_2|psi_1b> = <psi_2|J_a|psi_1b> with (J_a)_rc = -i s H~_rc d^a_rc and
// d_rc = r_c - r_r the bond vector of the stored entry (nm).
constexpr int kAcRows = 128;         // rows per observer block
struct AcArgs {
    SellView H;                      // values of the group precision
    const double *dx, *dy;           // [nnz_pad] bond vector of each stored entry (nm)
    const float *dx32, *dy32;        // their FP32 copies (FP32 form)
    const void *psi;                 // current buffer of the group, [row][B]
    const double *scale;             // FP32 norm carry [n_samples][B] or nullptr
    const float *scale_f;            // its FP32 copy
    const int32_t *chunk_sample;
    int64_t n_rows;
    int B;                           // multiple of 4
    double *block_partial;           // [n_rows / kAcRows][B / 4][8]
};
struct AcReduceArgs {
    const double *block_partial;
    const int64_t *sample_chunk_off; // [n_samples + 1] in 1024-row chunks
    int n_samples, B, group_state0, n_states, n_steps;
    const int *step;                 // per sample, already advanced by k_reduce
    double s;
    double2 *corr_ac;                // [n_samples][n_states / 4][4][n_steps + 1]
};
// Quasi-eigenstate accumulation (Sec. 2.6): acc[k][r][s0 + l] += coef[n][k] psi[r][l].
struct QeArgs {
    const void *psi;                 // current buffer of the group, [row][B]
    const double *scale;             // FP32 norm carry [n_samples][B] or nullptr
    const float *scale_f;            // its FP32 copy
    const int32_t *chunk_sample;
    const int *step;                 // per sample, already advanced by k_reduce
    const double2 *coef;             // [n_steps + 1][K] (tau / 2 pi) w_n e^{i E_k t_n}
    const float2 *coef_f;            // its FP32 copy
    void *acc;                       // [K][n_rows][S], complex in the group's precision
    int64_t n_rows;
    int B, s0, S, K;
};
cudaError_t launch_qe_acc(const QeArgs &a, int fp32, cudaStream_t st);
cudaError_t launch_qe_finish(const void *acc, int fp32, int K, int S, int64_t n_rows, int64_t n_orb,
                             int n_samples, const int32_t *user_to_row, const int32_t *orb_sample,
                             const int64_t *orb_off, double2 *out, double *norms, cudaStream_t st);
cudaError_t launch_ac_observe(const AcArgs &a, int fp32, int cplx, cudaStream_t st);
cudaError_t launch_ac_reduce(const AcReduceArgs &a, cudaStream_t st);
cudaError_t launch_vec_to_f32(int64_t n, const double *src, float *dst, cudaStream_t st);
// Preparation of the AC states, FP64, four lanes per row ([n_rows][4] complex):
// lanes 0 and 1 <- psi_p; lanes 2, 3 <- J_x psi_p, J_y psi_p; Fermi Clenshaw
// terms out = c v + gamma H~ x + zeta z on lanes 1 .. 3; the result goes
// back to the caller's layout as the four states of p.
cudaError_t launch_ac_load(const double2 *psi_user, int p, int64_t n_orb,
                           const int32_t *user_to_row, double2 *v4, cudaStream_t st);
cudaError_t launch_current4(SellView H, int fp32_vals, int cplx, int64_t n_rows,
                            const double *dxe, const double *dye, double s, double2 *v4,
                            cudaStream_t st);
cudaError_t launch_cheb_real4(SellView H, int fp32_vals, int cplx, int64_t n_rows, double c,
                              double gamma, double zeta, const double2 *v, const double2 *x,
                              const double2 *z, double2 *out, cudaStream_t st);
cudaError_t launch_ac_store(const double2 *v4, const double2 *f4, int p, int64_t n_orb,
                            const int32_t *user_to_row, double2 *out_user, cudaStream_t st);
cudaError_t launch_bond_vectors(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                                const int32_t *col, const double *dx, const double *dy,
                                int *claim, double *dxe, double *dye, int *err, cudaStream_t st);

// One backward (adjoint) term with gradient accumulation, FP64:
//   out = c psi + gamma (-i) (H~ x) + z [+ gbar_step psi0],
//   G_rc += gfac Im(conj(x_c) T_r) for every stored entry, Gdiag_r likewise.
struct AdjArgs {
    SellView H;
    const void *x, *psi, *z, *T_own;
    void *out;
    double c, gamma, gfac;
    double *G, *Gdiag;
    const double2 *gbar;   // [n_samples][n_states][n_steps + 1] or nullptr
    const void *psi0;
    int n_states, state0, n_steps, step;
    const int32_t *chunk_sample;
    int64_t n_rows;
};

// Kernel launchers (cheb_kernels.cu).  `fp32` selects the value precision,
// B the states per row (a group).  Return cudaError_t of the launch.
cudaError_t launch_term(const TermArgs &a, int fp32, int B, int threads, cudaStream_t st);
// The staged-gather kernel serves this group width in this precision with
// halo lists of at most halo_max rows.
bool halo_launchable(int fp32, int B, bool final_term, int halo_max);
// The pipelined form serves this shape within the shared-memory budget.
bool pipe_launchable(int fp32, int B, int halo_max, int ent_max, int uniform);
// The one-stage staged-gather kernel (kVariantStaged) for that shape.
bool staged_launchable(int fp32, int B, int halo_max, int ent_max, int uniform);
cudaError_t launch_final(const TermArgs &a, int fp32, int B, int threads, cudaStream_t st,
                         int *n_launch = nullptr);   // kernels it launched (1 or 2)
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st);
// State average of the correlations (and its adjoint, a broadcast of
// dL/dC-bar / S), complex128 [n_samples][S][n1] <-> [n_samples][n1].
// Compute capability (major * 10 + minor) the library's kernels were built for.
cudaError_t kernel_binary_version(int *version);
cudaError_t launch_corr_mean(const double2 *corr, int n_samples, int S, int n1, double2 *avg,
                             cudaStream_t st);
cudaError_t launch_corr_mean_adjoint(const double2 *gavg, int n_samples, int S, int n1,
                                     double2 *g, cudaStream_t st);
cudaError_t launch_phase_user(const double *theta, int64_t n_orb, int n_states,
                              const double *inv_sqrt_n, const int32_t *orb_sample,
                              double2 *psi_user, cudaStream_t st);
cudaError_t launch_set_states(const double2 *psi_user, int64_t n_orb, int n_states,
                              const int32_t *user_to_row, int group_state0, int B,
                              int fp32, void *psi, cudaStream_t st);
cudaError_t launch_get_states(const void *psi, int64_t n_orb, int n_states,
                              const int32_t *user_to_row, int group_state0, int B,
                              int fp32, double2 *out_user, cudaStream_t st);

// One term of the fused step (fused_kernels.cu): buffer indices 0..2 of the
// group (x < 0: x is psi; z < 0: none) and the coefficients.
struct FusedTerm {
    int x, z, out, final_term;
    double c_hi, c_lo, gamma;
    float c_hi_f, c_lo_f, gamma_f;
    // FP64 one-value form (cluster stepping): gh = gamma h_uniform; gamma d
    // is d (gd_sel 1) or 2d (gd_sel 2) with the sign bit gd_sign when
    // |gamma| is 1 or 2, else gamma * d (gd_sel 0)
    double gh;
    int gd_sel;
    unsigned long long gd_sign;
};

#ifdef __CUDACC__
// v with its sign bit flipped by sgn (0 or 1 << 63): an integer operation,
// off the FP64 pipe
__device__ __forceinline__ double xor_sign(double v, unsigned long long sgn)
{
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)sgn);
}
#endif

struct FusedArgs {
    SellView H;
    int uniform;                // FP64 one-value form (terms' gh, gd_sel)
    int zero_diag;
    const double *diag2;        // 2 d (FP64 one-value form) or nullptr
    const void *psi;            // current state (read only during the step)
    const void *psi0;
    void *bufs[3];
    const FusedTerm *terms;     // [J]
    const int32_t *items;       // [J * n_tiles] (j << 25 | t) in wavefront order
    int64_t n_items;
    int64_t n_tiles;
    int tile_rows, radius;
    int *done;                  // [J][n_tiles] epoch flags
    unsigned long long *counter;
    const int *epoch_ptr;       // epoch = *epoch_ptr + 1
    int *err;
    const double *scale;
    const float *scale_f;
    const int32_t *chunk_sample;
    double *tile_partial;       // [n_tiles][B][3]
    double *partial;            // [n_chunks][B][3]
    int *chunk_count;
};

cudaError_t launch_step_fused(const FusedArgs &f, int fp32, int B, int num_sms, cudaStream_t st);

// Cluster-resident time stepping (cluster_kernels.cu): all steps of one FP64
// state of a sample of up to 16 x 1024 rows in one cluster launch.
constexpr int kClusterMaxW = 12;           // entries per row it takes
constexpr int kClusterMaxTerms = 40;       // Chebyshev terms per step it takes (z <= ~25)
struct ClusterArgs {
    const int32_t *col;
    const double *val;
    const double *diag;
    const int64_t *slice_ptr;
    int fixed_width, uniform, max_w, rows_per_cta;
    int zero_diag;              // every onsite energy is zero
    double h_uniform;
    const double2 *psi0;
    double2 *bufs[3];
    int cur0;
    const FusedTerm *terms;     // [3][kMaxTerms] schedules by the buffer holding psi
    int J;                      // terms per step
    int next_cur[3];
    int n_steps;
    double2 *corr;              // C_n, n = 1 .. n_steps (state 0 of sample 0)
    double *norms;
    const double *norm_ref;
    double hard_bound;
    int *err;
};
// Blocks of the cluster for n_rows rows (16 where the device runs such a
// cluster, else 8), or 0 when the sample does not fit.
int cluster_blocks_for(int64_t n_rows, int max_w, int uniform);
cudaError_t launch_cluster_steps(const ClusterArgs &a, int K, cudaStream_t st);
int fused_tile_rows(int fp32, int B, int log4_mult);
int fused_grid(int fp32, int B, int num_sms);

// Persistent TMA-staged term kernel (tma_kernels.cu); err bit 4 = bounded
// wait expired.
cudaError_t launch_term_tma(const TermArgs &a, int fp32, int B, int max_width, int *err,
                            int num_sms, cudaStream_t st);

// Adjoint kernels (adjoint_kernels.cu).
cudaError_t launch_adj_term(const AdjArgs &a, int B, int threads, cudaStream_t st);
cudaError_t launch_source_init(int64_t n_rows, int B, const int32_t *chunk_sample,
                               const double2 *gbar, int n_states, int state0, int n_steps,
                               int step, const void *psi0, void *out, cudaStream_t st);
cudaError_t launch_param_grads(int64_t n_hop, const int32_t *bond_rows, const int64_t *slice_ptr,
                               const int32_t *col, const double *G, const double *Gd,
                               int64_t n_orb, const int32_t *user_to_row, double inv_s,
                               double *grad_hop, double *grad_onsite, cudaStream_t st);

// Builder (build_kernels.cu).
struct BuildInput {
    int64_t n_orb;
    const double *onsite;   // device or nullptr
    int64_t n_hop;
    const int64_t *hop_i, *hop_j;
    const double *hop_v;    // device
    double inv_s;
    int n_samples;
    const int64_t *d_sample_off;      // device [n_samples + 1] (caller order)
    const int64_t *d_sample_row_off;  // device [n_samples + 1] (padded rows)
    const int32_t *d_perm;            // device [n_orb] caller -> position in sample, or nullptr
    int cplx;                         // hop_v holds (re, im) per bond
};

struct BuildOutput {
    int64_t n_rows = 0, n_slices = 0, nnz_pad = 0, nnz_true = 0;
    int64_t n_orb_user = 0;          // caller orbitals (n_rows counts padding too)
    int32_t *user_to_row = nullptr;  // [n_orb]
    int32_t *orb_sample = nullptr;   // [n_orb]
    int64_t *slice_ptr = nullptr;    // [n_slices + 1]
    int32_t *col = nullptr;
    double *val64 = nullptr;
    float *val32 = nullptr;
    double *diag64 = nullptr;
    float *diag32 = nullptr;
    int32_t *chunk_sample = nullptr; // [n_rows / kChunkRows]
    int32_t *bond_rows = nullptr;    // [2 n_hop] rows of each bond
    int64_t n_hop = 0;
    double gershgorin = 0.0;
    int max_width = 0;
    int fixed_width = 0;             // every slice has this width (0: widths vary)
    int64_t bandwidth = 0;           // max |col - row| over the stored entries
    int uniform = 0;                 // all off-diagonal values are equal
    int zero_diag = 0;               // no onsite energies were given (H_ii = 0)
    int cplx = 0;                    // values are complex (re, im) per entry
    double h_uniform = 0.0;          // that value (H~ units)
    // halo lists of the staged-gather term kernel (built on first use)
    int64_t *halo_ptr = nullptr;     // [n_rows / kHaloRows + 1]
    int32_t *halo_rows = nullptr;    // own rows, then the other referenced rows
    uint16_t *lcol = nullptr;        // [n_packed] halo position of each entry's column, packed
    int64_t *pslice = nullptr;       // [n_slices + 1] packed offset of each slice
    int64_t n_packed = 0;            // packed entries (widths rounded up to 4)
    void *vpack[2] = {nullptr, nullptr}; // packed values, FP64 / FP32 (pipelined kernel)
    int halo_max = 0;                // longest list
    int halo_ent_max = 0;            // most packed entries of one block
    int64_t halo_total = 0;          // entries of all lists
    double *diag2_64 = nullptr;      // 2 d (FP64 one-value form; built on first use)
};

// 2 d for the FP64 one-value form's interior terms (gamma = +-2), exact.
int build_diag2(BuildOutput &b, cudaStream_t st, std::string &msg);

// Packed copy of the values of one precision for the pipelined kernel
// (built on first use).
int build_packed_values(BuildOutput &b, int fp32, cudaStream_t st, std::string &msg);

// Lanczos estimate of the extreme eigenvalues of H~ (lanczos.cu): n_iter
// steps from the SplitMix64 start vector of (kLanczosSeed, kLanczosStream);
// lo, hi are the extreme Ritz values (inside the spectrum), steps the
// steps taken (fewer at an invariant subspace).
constexpr uint64_t kLanczosSeed = 220900806ull;
constexpr int kLanczosStream = 200;
constexpr int kLanczosSteps = 64;          // the build's check
int lanczos_extremes(const BuildOutput &H, int n_iter, cudaStream_t st, double *lo, double *hi,
                     int *steps, std::string &msg);

// Halo lists for TBPM_VARIANT_HALO (build_kernels.cu); TBPM_E_UNSUPPORTED
// when a block references more than kHaloMaxExt other rows.
int build_halo(BuildOutput &b, cudaStream_t st, std::string &msg);

// Returns TBPM status; fills msg on failure.  Allocations in `out` are owned
// by the caller afterwards (freed with free_build).
int build_sell(const BuildInput &in, int keep64, int keep32, int detect_uniform,
               int keep_bond_map, BuildOutput &out, cudaStream_t st, std::string &msg);
void free_build(BuildOutput &b);

// Thread-local message returned by tbpm_last_error(NULL) (api.cu).
void set_thread_error(const std::string &m);

// Host math (host_math.cpp).
int bessel_miller(double z, double tol, int max_terms, double *J, int *n_terms);
// Chebyshev coefficients of the Fermi function on the rescaled axis (Sec. 2.2).
int fermi_coefficients(double beta_s, double mu_s, double tol, int k_max, std::vector<double> &c);
int ac_conductivity(const double *corr, int n_rows, int n_steps, double tau, double beta,
                    double eta, const double *omegas, int n_omega, double norm, double *sigma);
double window_weight(int window, int n, int n_steps);
int dos_adjoint(const double *dl_dd, int n_e, int n_steps, double tau, double e_min,
                double e_max, int window, double *gbar_out);

}  // namespace tbpm
