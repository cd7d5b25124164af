/*
 * xx.h -- C ABI of the GB300 plane-wave Fock exchange library (libxx.so).
 *
 * The library applies the exact-exchange (Fock) operator V_x of a block of
 * occupied orbitals to a block of target orbitals in a plane-wave basis, and
 * reduces the exchange energy E_x, following Hutchinson & Widom, "VASP on a
 * GPU" (Sec. "Our Implementation", Eq. 2: the four nested loops over k, q and
 * two band indices, whose inner band loops run on the GPU).  One GPU, one
 * process; every call is asynchronous on the caller's CUDA stream.
 *
 * Units and conventions (Hartree atomic units, lengths in bohr):
 *   - lattice: 9 doubles, rows a1, a2, a3.  Reciprocal rows b_i with
 *     a_i . b_j = 2 pi delta_ij.  Omega = |a1 . (a2 x a3)|.
 *   - k-points: fractional coordinates kfrac[k][3] (reciprocal basis).  The
 *     same mesh serves as target k and occupied q; weights are 1/N_k.
 *   - basis of k: Miller indices miller[k][g][3], g < npw[k], of plane waves
 *     exp(i (G + k).r); rows g >= npw[k] are padding and ignored.
 *   - orbitals: complex128 coefficients c[k][b][g] (interleaved re, im) of the
 *     cell-periodic part u_kb(r) = Omega^(-1/2) sum_G c_kb(G) exp(i G.r).
 *   - occupations w[k][b]: per spin, in [0, 1]; spin-paired (s = 2).
 *   - FFT grid N1 x N2 x N3, index p = i1 + N1 (i2 + N2 i3).
 *
 * Operator (per target (k, a)), exactly as the paper's loops state it:
 *   rho_aj(r) = conj(u_qj(r)) u_ka(r)
 *   W_aj(r)   = sum_G v(k - q + G) rhohat_aj(G) exp(i G.r),
 *               rhohat(G) = (1/N) sum_p rho(r_p) exp(-i G.r_p)
 *   (V_x u_ka)(r) = -sum_{q,j} (w_qj / N_k) u_qj(r) W_aj(r)
 *   (V_x c)_ka(G) = (sqrt(Omega)/N) sum_p exp(-i G.r_p) (V_x u_ka)(r_p), G in the basis of k
 *   E_x = (s/2) (1/N_k) sum_{k,a} w_ka Re <c_ka | V_x c_ka>
 * Kernels: XX_KERNEL_HSE is the screened (erfc(mu r)/r, HSE-type) interaction
 *   v(g) = 4 pi / |g|^2 (1 - exp(-|g|^2 / (4 mu^2))), v(0) = pi / mu^2;
 * XX_KERNEL_COULOMB_G0_DROPPED is 4 pi / |g|^2 with the g = 0 term dropped.
 * The library returns pure exchange: a hybrid functional's mixing fraction is
 * the caller's to apply.
 *
 * Grids: every axis must hold the codensity without aliasing, i.e.
 * N_i >= 4 n_i + 1 where n_i is the largest |Miller index| along axis i over
 * all basis sets (the paper sizes its FFT grids so that no aliasing occurs);
 * otherwise xx_create returns XX_ERR_GRID_ALIASING.  Supported axis lengths:
 * 24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96, 108 on each axis.  The transforms
 * run on an N x N x M grid: with two lengths equal (any axis order) the plan
 * relabels the axes internally so the equal pair spans its planes, which changes
 * nothing in the results or in the layout of any argument.  With three different
 * lengths the plan raises the shorter of two axes to the longer, choosing the
 * pair that gives the fewest points; since the caller's grid is free of
 * wrap-around, so is the raised one, and V_x c, E_x and the derivatives are those
 * of the caller's grid up to rounding (the cost is that of the raised grid).
 * xx_plan_info reports the grid the transforms run on.
 *
 * Ownership: the caller owns every input and output buffer (device memory
 * unless stated otherwise).  The plan owns its derived tables and workspace,
 * allocated with cudaMalloc on the current device at first use and released
 * by xx_destroy.  A plan may be used from one host thread at a time.
 *
 * Errors: every entry point returns an int status (XX_OK = 0, negative on
 * failure) and never throws.  Argument checks happen before any GPU work.
 * Device-side problems (an inconsistent Miller index, say) set a flag in the
 * plan that xx_sync reports.
 */
#ifndef XX_H
#define XX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XX_OK 0
#define XX_ERR_INVALID_ARGUMENT (-1)
#define XX_ERR_UNSUPPORTED_GRID (-2)
#define XX_ERR_GRID_ALIASING (-3)
#define XX_ERR_OUT_OF_MEMORY (-4)
#define XX_ERR_CUDA (-5)
#define XX_ERR_DEVICE_FLAG (-6)
#define XX_ERR_TIMEOUT (-7)
#define XX_ERR_NO_DEVICE (-8)
#define XX_ERR_SIZE_LIMIT (-9)

#define XX_FP32_MIXED 0   /* FFTs and pointwise products in FP32, sums in FP64 */
#define XX_FP64 1         /* every step in FP64 */

#define XX_KERNEL_HSE 0
#define XX_KERNEL_COULOMB_G0_DROPPED 1

typedef struct xx_plan_s *xx_plan;

/* Plan facts, filled by xx_plan_info. */
typedef struct {
  int grid[3];              /* FFT grid the transforms run on (caller's axis order) */
  int n_max[3];             /* largest |Miller index| per axis */
  int pruned[3];            /* kept codensity frequencies per axis, 4 n_max + 1 */
  int nk;                   /* k-points */
  int npw_max;
  int precision;            /* XX_FP32_MIXED or XX_FP64 */
  int targets_per_batch;    /* band-pair batch shape (NSIM analogue) */
  int occupied_per_batch;
  double omega;             /* cell volume, bohr^3 */
  size_t workspace_bytes;   /* device workspace held now */
  size_t peak_workspace_bytes;
  long long kernel_launches; /* kernels launched by this plan so far */
  long long pairs_transformed; /* band pairs (or packed slots) that went through the
                                  codensity transform so far; below the logical pair
                                  count when the pair symmetry is used */
  int q_per_batch;          /* k-points whose whole occupied sets share one band-pair batch
                               in the last xx_apply / xx_energy (1 unless a k-point has at
                               most half as many occupied bands as the default batch width) */
} xx_info;

/*
 * Create a plan (the paper's per-run library context, created at the start of
 * the run).  lattice[9], grid[3], kfrac[nk*3], npw[nk] and
 * miller[nk*npw_max*3] are HOST arrays, copied into the plan.  kernel_type is
 * XX_KERNEL_HSE (mu > 0, bohr^-1) or XX_KERNEL_COULOMB_G0_DROPPED (mu
 * ignored).  precision is XX_FP32_MIXED or XX_FP64.  workspace_cap bounds the
 * band-pair intermediate in bytes (0 = 16 GiB); it sets how many band pairs are
 * processed per batch (the paper's NSIM control of GPU memory): the default
 * batch of 64 targets x 80 occupied bands is halved (occupied first) until its
 * intermediate fits.  When a k-point has at most half as many occupied bands as
 * the batch is wide, the occupied sets of consecutive k-points share a batch.
 * Returns XX_ERR_INVALID_ARGUMENT, XX_ERR_UNSUPPORTED_GRID (also when a row of
 * z-planes of the pruned codensity does not fit one CTA's shared memory:
 * (N3 + N3 P1 + P3 P1) complex values, P_i = 4 n_max,i + 1, in the plan's
 * precision; e.g. FP64 with P1 = P3 = N3 = 96), XX_ERR_GRID_ALIASING,
 * XX_ERR_NO_DEVICE, XX_ERR_OUT_OF_MEMORY or XX_OK; *out is NULL on failure.
 */
int xx_create(xx_plan *out, const double *lattice, const int *grid, int nk, const double *kfrac,
              const int *npw, int npw_max, const int *miller, int kernel_type, double mu,
              int precision, size_t workspace_cap);

/* Release the plan and its device memory (the paper's context destruction).
 * Synchronises the device first.  NULL is accepted. */
int xx_destroy(xx_plan plan);

/*
 * vx_out[k][a][g] = (V_x c_tgt)_ka(G) for every k and target a: the operator
 * the paper's FOCK_ACC applies (Sec. "CPU Performance Analysis"), evaluated by
 * the k, q, band, band loops of Sec. "Our Implementation" (Eq. 2) as stated at
 * the top of this file.
 *   c_occ: device complex128 [nk][ld_occ][npw_max]; the occupied orbitals are
 *          bands 0..n_occ-1 of each k (ld_occ >= n_occ band slots per k; 0
 *          means n_occ).  When c_occ == c_tgt and ld_occ == n_tgt the
 *          occupied grids are taken from the target grids (computed once).
 *   w_occ: device double [nk][n_occ] per-spin occupations.
 *   c_tgt: device complex128 [nk][n_tgt][npw_max].
 *   vx_out: device complex128 [nk][n_tgt][npw_max], caller-allocated, must not
 *          alias an input; padding rows are written as zero.
 *   stream: a cudaStream_t (NULL = legacy default stream).
 */
int xx_apply(xx_plan plan, const void *c_occ, int ld_occ, const double *w_occ, int n_occ,
             const void *c_tgt, int n_tgt, void *vx_out, void *stream);

/*
 * Same as xx_apply for the target k-points k_first .. k_first + k_count - 1
 * only (the occupied orbitals still span every q of the mesh): c_tgt and
 * vx_out hold [k_count][n_tgt][npw_max].  Target k-points are independent, so
 * disjoint ranges may run on different GPUs (each needs every occupied orbital).
 */
int xx_apply_range(xx_plan plan, int k_first, int k_count, const void *c_occ, int ld_occ,
                   const double *w_occ, int n_occ, const void *c_tgt, int n_tgt, void *vx_out,
                   void *stream);

/*
 * E_x of the targets (Eq. 2, with the sign and spin readings stated at the top
 * of this file): runs xx_apply into vx_out (device, required) and then the
 * deterministic FP64 reduction of (s/2)(1/N_k) sum w_tgt <c_tgt|V_x c_tgt>.
 *   w_tgt: device double [nk][n_tgt].
 *   ex_out: device double[2] = {Re E_x, Im E_x}; the imaginary part is a
 *          diagnostic that vanishes for a Hermitian V_x.
 */
int xx_energy(xx_plan plan, const void *c_occ, int ld_occ, const double *w_occ, int n_occ,
              const void *c_tgt, const double *w_tgt, int n_tgt, void *vx_out, double *ex_out,
              void *stream);

/* The share of E_x from target k-points k_first .. k_first + k_count - 1 (the
 * 1/N_k of the full mesh is kept, so the shares of disjoint ranges add up to
 * E_x); c_tgt, w_tgt and vx_out hold those k-points only. */
int xx_energy_range(xx_plan plan, int k_first, int k_count, const void *c_occ, int ld_occ,
                    const double *w_occ, int n_occ, const void *c_tgt, const double *w_tgt,
                    int n_tgt, void *vx_out, double *ex_out, void *stream);

/* The reduction alone: ex_out[2] from a V_x c already in vx (device). */
int xx_energy_from_vx(xx_plan plan, const void *c_tgt, const double *w_tgt, int n_tgt,
                      const void *vx, double *ex_out, void *stream);

/* The reduction alone over target k-points k_first .. k_first + k_count - 1. */
int xx_energy_from_vx_range(xx_plan plan, int k_first, int k_count, const void *c_tgt,
                            const double *w_tgt, int n_tgt, const void *vx, double *ex_out,
                            void *stream);

/*
 * Gradients of E_x[c] (the paper computes none; these are derivatives of Eq. 2)
 * where the same orbitals c (device complex128
 * [nk][n_b][npw_max]) with occupations w (device double [nk][n_b]) are both the
 * occupied set and the targets.
 *   vx: V_x c from a previous xx_apply/xx_energy with these inputs (device), or
 *       NULL to recompute it inside this call.
 *   grad_ex: upstream scalar dL/dE_x.
 *   dc_out (device complex128 [nk][n_b][npw_max], or NULL): the Wirtinger
 *       derivative grad_ex * dE_x/dc* = grad_ex * (s w_kb / N_k) (V_x c)_kb.
 *   dmu_out (device double[1], or NULL): grad_ex * dE_x/dmu, with
 *       dv/dmu = -(2 pi / mu^3) exp(-|g|^2 / (4 mu^2)); it recomputes every pair
 *       codensity (forward transforms only) and stores no pair grid.
 *       Requires XX_KERNEL_HSE.
 */
int xx_apply_backward(xx_plan plan, const void *c, const double *w, int n_b, const void *vx,
                      double grad_ex, void *dc_out, double *dmu_out, void *stream);

/*
 * Strain derivative of E_x[c] (c both occupied and targets, as in
 * xx_apply_backward): the analogue, for a cell without ions, of the paper's
 * FOCK_FORCE derivative routine (Sec. "CPU Performance Analysis").  Under a
 * homogeneous strain the lattice rows become a_i (I + eps) with the plane-wave
 * coefficients held fixed, so g = (m + k - q).B becomes g (I - eps^T) and
 * Omega becomes Omega det(I + eps):
 *   dE_x/deps_ab = -delta_ab E_x
 *                  + (s Omega / N_k^2) sum w_ka w_qj sum_G v'(|g|^2) g_a g_b |rhohat(G)|^2.
 * (Stress = dE_x/deps / Omega in the convention sigma = (1/Omega) dE/deps.)
 *   dex_deps: device double[9], row-major 3x3 (symmetric).
 *   ex_out: device double[1] or NULL: E_x from the pair sum (Parseval form).
 * Recomputes every codensity (forward transforms only).
 */
int xx_strain_derivative(xx_plan plan, const void *c, const double *w, int n_b, double *dex_deps,
                         double *ex_out, void *stream);

/* One independent exchange job for xx_run_many. */
typedef struct {
  xx_plan plan;             /* each job needs its own plan (workspace) */
  const void *c_occ;        /* as xx_energy */
  int ld_occ;
  const double *w_occ;
  int n_occ;
  const void *c_tgt;
  const double *w_tgt;      /* may be NULL when ex_out is NULL */
  int n_tgt;
  void *vx_out;
  double *ex_out;           /* device double[2], or NULL for V_x c only */
} xx_job;

/*
 * Run independent jobs (different cells, grids or k-meshes, one plan each)
 * concurrently, as the paper does with CUDA streams for small structures:
 * each job runs on its plan's own stream, which first waits for the work
 * already queued on `stream`; `stream` then waits for every job.  Results are
 * identical to running the jobs one after another.  Returns the first failing
 * job's status (XX_ERR_INVALID_ARGUMENT if two jobs share a plan).
 */
int xx_run_many(int n_jobs, const xx_job *jobs, void *stream);

/*
 * Run independent Gamma-only jobs (one plan each, one k-point per plan, e.g.
 * cells with different FFT grid lengths) with ONE launch per band-pair pass
 * covering every band-pair batch of every job: a table of batches (grid
 * pointers, grid length, pruned box, batch shape) goes to each launch, and
 * every CTA runs the pass of its batch's grid length.  This replaces the
 * paper's streams for small structures (xx_run_many) by a single work list.
 * Per job, on the plan's own stream (which first waits for the work queued
 * on `stream`): sphere -> grid and the kernel table; then, on `stream`, per
 * round the passes A, B, C and, for mirrored k = q tiles, the role-swapped
 * pass C (one launch each for all jobs; batches that add into the same
 * targets add into private accumulator planes, summed per target in batch
 * order afterwards); then per job on its own stream the sums, grid -> sphere
 * and, when ex_out is set, E_x; `stream` finally waits for every job.
 * A round holds as many of each job's batches as its plan's workspace cap
 * allows; with enough workspace (the caller's workspace_cap) there is one
 * round.  Results equal xx_energy / xx_apply on each job up to the order of
 * FP32 summation within a batch (the batches are the same as theirs, so the
 * results are identical when the batch shapes are).  All plans must share one
 * precision, be unsharded and have nk = 1; a plan may appear once.  Returns
 * XX_ERR_INVALID_ARGUMENT for a violated requirement, else the first error.
 */
int xx_run_batched(int n_jobs, const xx_job *jobs, void *stream);

/*
 * Vector-Jacobian product (the paper has none; the derivative of the Eq. 2
 * loops' output) of y = V_x[c_occ] c_tgt (xx_apply's output) for a
 * real loss L with cotangent ybar = dL/dy* (Wirtinger; device complex128
 * [nk][n_tgt][npw_max]).  Inputs as xx_apply.
 *   grad_tgt_out (device complex128 [nk][n_tgt][npw_max], or NULL):
 *       dL/dc_tgt* = V_x ybar (V_x is Hermitian; one more operator application).
 *   grad_occ_out (device complex128 [nk][n_occ][npw_max], or NULL):
 *       dL/dc_occ* through both places the occupied orbitals enter the loops
 *       (the codensity conj(u_qj) u_ka and the multiplication by u_qj):
 *       dL/dc_qj* = P_q[ -(w_qj/N_k) sum_{k,a} (ubar_ka conj(W_aj) + u_ka conj(Wbar_aj)) ]
 *       with ubar the grids of ybar, W_aj the pair potential of (u_ka, u_qj) and
 *       Wbar_aj that of (ubar_ka, u_qj).  With both outputs requested the two
 *       cost two transforms per band pair (XX_OPT_FUSED_VJP), else one (target
 *       part) and two (occupied part); pair potentials are recomputed, never
 *       stored beyond one batch.
 * When the same orbitals are both occupied and targets, the total gradient
 * is the sum of the two outputs.  Occupations are treated as constants.
 */
int xx_apply_vjp(xx_plan plan, const void *c_occ, int ld_occ, const double *w_occ, int n_occ,
                 const void *c_tgt, int n_tgt, const void *ybar, void *grad_tgt_out,
                 void *grad_occ_out, void *stream);

/*
 * Wait for the plan's work on stream with a time limit (seconds, <= 0 waits
 * without limit), then report the device error flag.  Returns XX_OK,
 * XX_ERR_TIMEOUT (the stream is still busy; nothing was cancelled),
 * XX_ERR_DEVICE_FLAG (and clears the flag) or XX_ERR_CUDA.
 */
int xx_sync(xx_plan plan, void *stream, double timeout_s);

/* Plan options for xx_set_option. */
#define XX_OPT_PAIR_SYMMETRY 0  /* value != 0 (default): when the occupied grids are the
                                   leading target grids, transform each occupied band pair
                                   of a pair of k-points (k, q) once and use W_qj,ka =
                                   conj(W_ka,qj) for the other target (v depends on |g| only,
                                   so v(q - k + G) = v(k - q - G)); results differ only by
                                   rounding order.  On k = q blocks the occupied square is
                                   cut into tiles and tiles I <= J are transformed.  Of the
                                   k != q blocks only q > k are transformed: always in the
                                   pair sums of dE_x/dmu and the strain derivative; in
                                   xx_apply / xx_energy over all k-points when FP64
                                   accumulators of every target of every k-point
                                   (nk * n_tgt * N^3 * 16 bytes) fit in XX_OPT_ACC_LIMIT_MB
                                   (64 GiB) and can be allocated, else both orders are
                                   transformed */
#define XX_OPT_REAL_GAMMA 1     /* value != 0: the orbitals passed to later calls are real in
                                   real space (c(-G) = conj c(G) for every G of the basis), so
                                   every codensity is real and, at k = q = Gamma, so is every
                                   W_aj.  Two occupied bands then share one transform: the
                                   codensity of u_2p - i u_2p+1 with u_a is rho_a,2p +
                                   i rho_a,2p+1, and the real and imaginary parts of its W are
                                   the two bands' potentials.  Halves the transforms of
                                   xx_apply, xx_energy, xx_apply_backward and
                                   xx_strain_derivative (with XX_OPT_PAIR_SYMMETRY as well,
                                   the k = q square is halved again); xx_apply_vjp keeps the
                                   general path.  Allowed only on a plan with one k-point at
                                   Gamma whose basis holds -G for every G (else
                                   XX_ERR_INVALID_ARGUMENT); with complex orbitals the results
                                   are wrong.  Default 0. */

#define XX_OPT_TMA_PASS_B 2     /* FP32 pass B (the z transforms and kernel multiply of the
                                   band-pair intermediates): 1 (default) runs the
                                   persistent kernel whose rows arrive by bulk tensor copies,
                                   two rows ahead, when the z length is at least 80 and the
                                   kept f_x of a row are at most 3/4 of the x length, else
                                   the one-row-per-block kernel; 2 always the tensor-copy
                                   kernel; 0 never.  Both
                                   run the same arithmetic in the same order.  Other values
                                   give XX_ERR_INVALID_ARGUMENT. */

#define XX_OPT_STAGE_PASS_A 3   /* FP32 pass A: 2 runs one CTA per SM with the occupied
                                   orbital's plane staged in shared memory by one bulk copy
                                   per band, issued while the previous band's plane is being
                                   transformed; 0 runs two CTAs per SM reading both planes
                                   with global loads; 1 (default) stages for grid lengths up
                                   to 48.  Same arithmetic in the same order.  Other values
                                   give XX_ERR_INVALID_ARGUMENT. */

#define XX_OPT_TEST_WAIT_EXPIRY 4 /* tests of the failure path only: value != 0 announces the
                                   first tensor copy of every pass-B CTA as 16 bytes longer
                                   than it is, so the bounded wait on it (2 s) runs out; the
                                   CTA then sets the device flag and returns.  Results of
                                   such a call are invalid; xx_sync reports
                                   XX_ERR_DEVICE_FLAG and the context stays usable.  Takes
                                   effect only where the tensor-copy pass B runs.  Default 0. */

#define XX_OPT_FUSED_VJP 5      /* value != 0 (default): xx_apply_vjp asked for both gradients
                                   transforms each band pair twice instead of three times: the
                                   pair potential of (ubar_ka, u_qj) feeds both V_x ybar and the
                                   u_ka conj(Wbar) term of the occupied gradient.  Needs FP64
                                   accumulators of every occupied band of every k-point
                                   (nk * n_occ * N^3 * 16 bytes, within XX_OPT_ACC_LIMIT_MB);
                                   otherwise,
                                   or with 0, the two gradients are computed one after the
                                   other.  Results differ only by rounding order. */

#define XX_OPT_ACC_LIMIT_MB 6   /* value >= 0: MiB of FP64 accumulators the plan may hold for
                                   every k-point at once (the k != q pair symmetry of xx_apply
                                   and xx_energy, the fused VJP); default 65536 (64 GiB).  Above
                                   it those calls use per-k accumulators (k = q symmetry only,
                                   VJP parts one after the other).  Negative values give
                                   XX_ERR_INVALID_ARGUMENT. */

#define XX_OPT_TABLE_CACHE 7    /* value != 0 (default): the kernel tables v(k - q + G)/N of
                                   every (k, q) are built in one launch at the first call that
                                   needs them and kept for the plan's life, when they fit in
                                   min(1 GiB, workspace_cap / 8) and nk^2 <= 65535; otherwise,
                                   or with 0, each band-pair batch builds its tables.  The
                                   values are the same either way.  0 frees the kept tables. */

/* Set a plan option; XX_ERR_INVALID_ARGUMENT for an unknown option. */
int xx_set_option(xx_plan plan, int option, long long value);

/* Override the band-pair batch shape (targets x occupied per batch); 0 keeps
 * the automatic choice.  Takes effect at the next call. */
int xx_set_batch(xx_plan plan, int targets_per_batch, int occupied_per_batch);

/*
 * Sharding over GPUs (one process per GPU), after the paper's distribution of
 * the exchange loops over k-points and bands across MPI ranks (Sec. "Our
 * Implementation").  The unit is the unordered k-point block {k, q}: every
 * band pair of targets at k with occupied bands at q, and (the pair symmetry
 * W_qj,ka = conj W_ka,qj) of targets at q with occupied bands at k.  A block's
 * contributions add into V_x c of k and of q, so a plan set to shard s of n
 * computes, in xx_apply / xx_apply_range / xx_energy / xx_energy_range and the
 * dE/dc* of xx_apply_backward, the partial V_x c and partial E_x of the blocks
 * assigned to s; summing the n partial results (an all-reduce of V_x c, a sum
 * of the n E_x shares) gives the full operator, because every block is
 * assigned to exactly one shard.  Every shard needs every occupied orbital
 * (the caller distributes them, e.g. a broadcast) and writes V_x c for every
 * target.  The assignment balances the band-pair transforms of the blocks
 * (greedy, largest block first, deterministic: the same on every rank).
 * xx_set_shard(plan, 0, 1) (the default) computes every block.  While n > 1,
 * dE/dmu (xx_apply_backward with dmu_out), xx_strain_derivative and
 * xx_apply_vjp return XX_ERR_INVALID_ARGUMENT.
 */
int xx_set_shard(xx_plan plan, int shard, int n_shards);

/* The block assignment itself, host only: owner_out[b] (host int array of
 * nk (nk + 1) / 2) = shard of block b, with b = k nk - k (k - 1) / 2 + (q - k)
 * for k <= q.  Returns XX_ERR_INVALID_ARGUMENT for nk < 1, negative band
 * counts, n_shards < 1 or a NULL owner_out. */
int xx_shard_blocks(int nk, int n_occ, int n_tgt, int n_shards, int *owner_out);

/* Kernel classes of the per-kernel timing (xx_profile_read). */
#define XX_PROF_PASS_A 0          /* codensity + forward xy FFT */
#define XX_PROF_PASS_B 1          /* z FFT, kernel multiply, inverse z FFT */
#define XX_PROF_PASS_C 2          /* inverse xy FFT, multiply by u_j, accumulate */
#define XX_PROF_SPHERE_TO_GRID 3  /* scatter + inverse 3D FFT of orbitals */
#define XX_PROF_GRID_TO_SPHERE 4  /* forward 3D FFT + gather of V_x u */
#define XX_PROF_KERNEL_TABLE 5    /* v(k - q + G) table */
#define XX_PROF_REDUCE 6          /* E_x reduction */
#define XX_PROF_PASS_B_DMU 7      /* forward z FFT x dv/dmu reduction */
#define XX_PROF_CLASSES 8

/* Turn per-kernel-class timing on or off: when on, every launch group of the
 * plan is bracketed by CUDA events on its stream (measurement use; adds two
 * event records per group). */
int xx_profile_enable(xx_plan plan, int enable);

/* Device time in ms and number of timed launch groups per kernel class since
 * the last reset, for classes 0 .. n_classes-1 (host arrays).  Waits for the
 * recorded events.  reset != 0 discards the records. */
int xx_profile_read(xx_plan plan, double *ms, long long *launches, int n_classes, int reset);

/* Fill *info with the plan's facts. */
int xx_plan_info(xx_plan plan, xx_info *info);

/*
 * Smallest FFT grid length this library supports on which the operator is
 * exact (the no-wrap-around condition of the setup section, read as
 * N >= 4 n_max + 1 on every axis): n_max[3] is the largest |Miller index| of
 * the basis sets per axis (host array), *n_out receives the cubic length.  On
 * such a grid every codensity transform is exact on its support |f| <= 2 n_max
 * and the sphere projection of u_j W sees no alias, so V_x c, E_x and the
 * gradients equal those computed on any larger admissible grid up to rounding.
 * Host only (no GPU work).  Returns XX_ERR_INVALID_ARGUMENT (NULL pointer,
 * negative n_max), XX_ERR_UNSUPPORTED_GRID (no supported length is large
 * enough) or XX_OK.
 */
int xx_exact_grid(const int *n_max, int *n_out);

/*
 * The same per axis: the supported grid N1 x N2 x N3 with N_i >= 4 n_max,i + 1
 * and two lengths equal (the shape the transforms run on) that has the fewest
 * points; grid_out[3] (host) in the caller's axis order.  Ties go to the first
 * candidate in the order: axes (1, 2) equal, (1, 3) equal, (2, 3) equal, as in
 * xx_create's raising of three different lengths, so a plan created on the
 * smallest admissible length per axis runs on this grid.
 * Host only.  Errors as xx_exact_grid.
 */
int xx_exact_grid3(const int *n_max, int *grid_out);

/*
 * E_x reduction for callers that cannot allocate device memory.  The paper has
 * no counterpart: this entry point exists for callers whose device memory is
 * already reserved by their own memory manager (a framework's caching
 * allocator, a fixed per-process budget), or that must not hit the
 * device-wide synchronisation cudaFree implies.  It computes the same
 * fixed-order FP64 reduction as xx_energy_from_vx, needs no plan, and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   nk, n_tgt, npw_max: sizes of c_tgt and vx ([nk][n_tgt][npw_max] complex128,
 *       device); npw: device int [nk] basis sizes, each required to satisfy
 *       1 <= npw[k] <= npw_max (the kernel clamps a value outside [0, npw_max]
 *       to that range, so a bad size never reads past a row, but the result is
 *       then that of the clamped size); w_tgt: device double [nk][n_tgt];
 *       ex_out: device double[2] = {Re E_x, Im E_x}.
 * Its per-target partial sums live in one fixed device array of
 * XX_NOALLOC_MAX_ROWS complex128 entries (256 KiB) that every GPU loading the
 * library holds until the process exits; nk * n_tgt above that limit returns
 * XX_ERR_SIZE_LIMIT.  The first call on a device looks up the array's device
 * address (with that device current), so make that first call before any
 * stream capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that destroys the device's primary
 * context) the module may load elsewhere, so a reset after the first call on a
 * device is not supported.  All calls on a device share the array: calls whose work
 * overlaps on the GPU (different streams, concurrent threads) race and must be
 * serialised by the caller.  Every entry is written before it is read, so no
 * clearing is needed between calls.
 */
#define XX_NOALLOC_MAX_ROWS 16384
int xx_energy_from_vx_noalloc(int nk, int n_tgt, int npw_max, const int *npw, const void *c_tgt,
                              const double *w_tgt, const void *vx, double *ex_out, void *stream);

/*
 * Measured CUDA-core fused-multiply-add rate of the current device, in TFLOP/s
 * (two flops per FMA): the denominator of the ALU rooflines of the benchmark
 * (FP32 for the mixed-precision passes, FP64 for the all-FP64 path).  The
 * paper has no counterpart; this is a measurement helper, not part of the
 * exchange method.  Launches 6 short kernels (8 x SMs CTAs of 256 threads, 8
 * independent FMA chains of 4096 steps per thread) on stream, times the last 5
 * with CUDA events and waits for them (blocking).  Allocates no device memory.
 *   precision: XX_FP32_MIXED (FP32 FMA) or XX_FP64 (FP64 FMA);
 *   tflops_out: host double.
 * Returns XX_ERR_INVALID_ARGUMENT, XX_ERR_NO_DEVICE, XX_ERR_CUDA or XX_OK.
 */
int xx_measure_fma_rate(int precision, double *tflops_out, void *stream);

/* Static description of a status code. */
const char *xx_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* XX_H */
