/*
 * rbe2d.h — C ABI of the GB300 (sm_103a) random-batch Ewald k-space force for
 * dielectrically confined quasi-2D Coulomb systems (RBE2D; Gan, Gao, Liang, Xu,
 * arXiv 2405.06333).
 *
 * Problem (Sec. 2.1 and Sec. 3.1): N point charges q_i at r_i = (x_i, y_i, z_i) in a
 * cell periodic in x (period Lx) and y (period Ly), confined to the slab 0 <= z <= H
 * between two dielectric interfaces with contrasts gamma_top (at z = H) and
 * gamma_bot (at z = 0), |gamma| <= 1 (Eq. 3.1).  The image series is truncated at M
 * reflection levels (Eq. 3.2, Theorem 3.2) and the k-space sum is taken on the
 * lattice of the period-Lz extension, Lz >= (M+1) H (Theorem 3.3, Eq. 3.23).  The
 * total charge must vanish (Eq. 2.2).  Units are Gaussian (energy q q'/r), scaled by
 * coulomb_k; forces are F = -grad U.
 *
 * Memory and threading conventions, for every entry point below:
 *  - Array arguments are caller-owned, contiguous, row-major DEVICE pointers on the
 *    device that was current at rbe2d_init, unless RBE2D_HOST_BUFFERS is set for a
 *    call that accepts it; then they are host pointers and the call returns after the
 *    results have arrived.  Pinned (page-locked or registered) host buffers are read
 *    and written in place by the kernels over the host link (NVLink-C2C on Grace
 *    hosts), so the transfers overlap the computation; other host memory is copied
 *    in and out on the context's stream.
 *  - pos is N x 3 (x, y, z) and q is N, both float64, or both float32 with
 *    RBE2D_INPUT_F32.  x and y are wrapped periodically (never an error); z must lie
 *    in [0, H].
 *  - Outputs are float64 in RBE2D_FP64 mode and float32 in RBE2D_FP32_MIXED mode
 *    (force N x 3, phi and dq N, dpos N x 3).  energy_out, rho_out and dgamma are
 *    always float64.
 *  - All work is enqueued on the stream given to rbe2d_init; calls without
 *    RBE2D_HOST_BUFFERS or RBE2D_VALIDATE never synchronise and never allocate, so a
 *    sequence of them can be captured in a CUDA graph.  A context is not thread-safe.
 *  - Every call returns RBE2D_OK (0) or a negative status; rbe2d_last_error gives the
 *    message of the last failure on that context.  A failed call leaves the outputs
 *    unspecified.
 */
#ifndef RBE2D_H
#define RBE2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define RBE2D_OK 0
#define RBE2D_EINVAL (-1)      /* bad argument: sizes, |gamma| > 1, alpha <= 0, P <= 0, Lz < (M+1)H, N > n_max, NULL */
#define RBE2D_ENONNEUTRAL (-2) /* |sum q| > 1e-10 sum |q| (Eq. 2.2), reported with RBE2D_VALIDATE */
#define RBE2D_ERANGE (-3)      /* some z outside [0, H], reported with RBE2D_VALIDATE */
#define RBE2D_ECUDA (-4)       /* a CUDA runtime call or kernel launch failed */
#define RBE2D_ETIMEOUT (-5)    /* a bounded device-side wait gave up */
#define RBE2D_ESAMPLER (-6)    /* a k-sample was rejected 64 times in a row */
#define RBE2D_ENOMEM (-7)      /* device or host allocation failed in rbe2d_init */

/* Arithmetic modes. */
#define RBE2D_FP64 0        /* every step in float64, 64-bit fixed-point phases */
#define RBE2D_FP32_MIXED 1  /* float32 phases and products, float64 reductions and coefficients */

/* Flags for rbe2d_force. */
#define RBE2D_KSPACE 1         /* random-batch k-space force (Eq. 3.26) */
#define RBE2D_REAL 2           /* erfc real-space force with near-slab images (Eq. 3.12) */
#define RBE2D_IBC 4            /* include F_IBC^M / U_IBC^M (Eq. 3.18) */
#define RBE2D_ENERGY 8         /* write energy_out */
#define RBE2D_POTENTIAL 16     /* write phi_out = dU/dq_i (k-space + self + IBC) */
#define RBE2D_HOST_BUFFERS 32  /* pos, q, force_out, phi_out, energy_out are host pointers */
#define RBE2D_VALIDATE 64      /* check neutrality and the z range on the device (synchronises) */
#define RBE2D_INPUT_F32 128    /* pos and q are float32 instead of float64 */
#define RBE2D_REUSE_SF 256     /* reuse the structure factors of the previous call (same batch, same input) */
#define RBE2D_ACCUMULATE 512   /* add the result to force_out / phi_out instead of overwriting them */

typedef struct rbe2d_ctx rbe2d_ctx;

typedef struct {
    double Lx, Ly, H;            /* cell; the slab is 0 <= z <= H (Sec. 2.1) */
    double Lz;                   /* extended z period; <= 0: Eq. 3.23 at eps, rounded up */
    double gamma_top, gamma_bot; /* dielectric contrasts at z = H and z = 0 (Eq. 3.1) */
    int M;                       /* image levels; < 0: Eq. 3.10 at eps (capped at 64); 0 = homogeneous */
    double alpha;                /* Ewald parameter; <= 0: (N/(Lx Ly H))^(1/3) with N = n_max (Sec. 2.3) */
    double r_c;                  /* real-space cutoff; <= 0: 3 / alpha */
    int P;                       /* batch size (number of sampled k per step), 1 <= P <= 65536 */
    uint64_t seed;               /* Philox4x64-10 key word 0 of the k sampler */
    double eps;                  /* tolerance of the automatic rules; <= 0: 1e-4 */
    int precision;               /* RBE2D_FP64 or RBE2D_FP32_MIXED */
    double coulomb_k;            /* energy prefactor; <= 0: 1 */
    int real_space;              /* 1: build the real-space cell list buffers at init (needed by RBE2D_REAL) */
    double skin;                 /* > 0 with real_space = 1 in RBE2D_FP32_MIXED mode: Verlet pair lists of
                                    width r_c + skin for rbe2d_md_step (see there); <= 0: none */
} rbe2d_params;

/*
 * Create a context for up to n_max particles on the current CUDA device, with all
 * scratch memory, the k-sampler tables (the 1-D factors of w(k) = exp(-k^2/4alpha^2),
 * Sec. 2.3) and the image-series constants allocated and computed once.  stream is a
 * cudaStream_t (NULL: the legacy default stream) and is used by every later call.
 * Returns RBE2D_EINVAL for inconsistent parameters (with the message), RBE2D_ENOMEM
 * or RBE2D_ECUDA; *out is set only on success.  The caller owns the context.
 */
int rbe2d_init(const rbe2d_params* params, int64_t n_max, void* stream, rbe2d_ctx** out);

/* Release every resource of the context (synchronises its stream).  NULL is allowed. */
int rbe2d_destroy(rbe2d_ctx* ctx);

/* Message of the last failed call on ctx ("" if none); valid until the next call.
 * With ctx == NULL: the message of the last failed rbe2d_init on the calling thread. */
const char* rbe2d_last_error(const rbe2d_ctx* ctx);

/*
 * The parameters actually in use after the automatic rules: S = sum_{k != 0} w(k)
 * (Eq. 2.21), Lz, M, alpha, r_c.  Any pointer may be NULL.  Host pointers.
 */
int rbe2d_get_derived(const rbe2d_ctx* ctx, double* S, double* Lz, int* M, double* alpha,
                      double* r_c);

/*
 * Draw the batch for MD step `step`: P i.i.d. wave vectors k = 2 pi (nx/Lx, ny/Ly, nz/Lz),
 * k != 0, with probability w(k)/S (Sec. 2.3; Algorithm 2, first step of the loop),
 * and precompute per k the coefficient -(2 pi/V)(S/P)/k^2 and the image-series factors
 * E(kz) = Y_even and O(kz) = conj(Y_odd) of the re-calibration (Sec. 3.4).
 * Sample l, attempt a uses Philox4x64-10 with counter (l, a, step, 0) and key
 * (seed, 0); u_d = (word_d >> 11) 2^-53; index n_d is the first entry of the
 * normalised cumulative table of the 1-D factor that exceeds u_d; (0,0,0) is rejected.
 * k_idx_out (device, P x 3 int32, may be NULL) receives (nx, ny, nz).  An exhausted
 * sample sets a device flag reported as RBE2D_ESAMPLER by rbe2d_sync_status.
 */
int rbe2d_sample_k(rbe2d_ctx* ctx, uint64_t step, int32_t* k_idx_out);

/*
 * Metropolis variant of the sampler (Sec. 2.3 draws the batch by a Metropolis procedure
 * whose proposal the paper does not fix; rbe2d_sample_k draws the same distribution
 * exactly and i.i.d.).  One chain per batch slot l, a random walk on the lattice inside
 * the sampler's table box without k = 0: proposal n' = n + delta, delta_d uniform on
 * {-s_d, ..., s_d} with s_d = max(1, ceil(alpha L_d / (pi sqrt 2))), accepted when
 * u w(n) < w(n') (w the product of the three tabulated 1-D factors).  Update `it` of
 * step `step` uses Philox4x64-10 with counter (l, it, step, 1) and key (seed, 0):
 * delta_d = ((word_d >> 32) (2 s_d + 1)) >> 32 minus s_d, u = (word_3 >> 11) 2^-53.
 *  - rbe2d_metropolis_reset: k_start (device, P x 3 int32) sets every chain's state; NULL
 *    starts each chain at the i.i.d. draw of step 0 (a stationary start).  Also clears
 *    the acceptance count.  Must precede the first rbe2d_sample_k_metropolis.
 *  - rbe2d_sample_k_metropolis: applies `sweeps` (1..2^20) updates to every chain and
 *    makes the chain states the batch (coefficients as for rbe2d_sample_k).
 *    k_idx_out (device, P x 3 int32, may be NULL) receives the states.
 *  - rbe2d_metropolis_accepted: accepted moves since the reset (host out; synchronises).
 * Successive batches are correlated; the estimator stays unbiased once the chains are
 * stationary.
 */
int rbe2d_metropolis_reset(rbe2d_ctx* ctx, const int32_t* k_start);
int rbe2d_sample_k_metropolis(rbe2d_ctx* ctx, uint64_t step, int sweeps, int32_t* k_idx_out);
int rbe2d_metropolis_accepted(rbe2d_ctx* ctx, uint64_t* accepted_out);

/*
 * Use an explicit batch instead of a sampled one: k_idx (device, P x 3 int32, no
 * (0,0,0) row) with the same per-k coefficients as rbe2d_sample_k.  The batch size
 * must equal the context's P.  Lets a caller supply its own random numbers.
 */
int rbe2d_set_k(rbe2d_ctx* ctx, const int32_t* k_idx);

/*
 * Structure factors of the current batch (Theorem 3.3, Eq. 3.17; Sec. 3.4):
 *   rho_l   = sum_j q_j exp(i k_l . r_j)
 *   sigma_l = sum_j q_j exp(i khat_l . r_j),  khat = (kx, ky, -kz)
 * reduced over all N charges in float64 (float32 short runs in FP32_MIXED mode).
 * rho_out (device, P x 4 float64: Re rho, Im rho, Re sigma, Im sigma) may be NULL;
 * the values stay in the context for a following rbe2d_force / rbe2d_energy_backward
 * with RBE2D_REUSE_SF on the same input.
 */
int rbe2d_structure_factor(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                           double* rho_out);

/*
 * One force evaluation.  With RBE2D_KSPACE: the random-batch estimate of the k-space
 * force with the image series folded into per-k coefficients (Eq. 3.26, gradient
 * Eq. 3.25 in the re-calibrated form of Sec. 3.4):
 *   F_i = q_i sum_l c_l [ k_l Im(e^{-i k_l.r_i} A_l) + khat_l Im(e^{-i khat_l.r_i} B_l) ]
 *   A_l = (2 + 2E) rho_l + conj(O) sigma_l,  B_l = O rho_l,  c_l = -(2 pi/V)(S/P)/k_l^2;
 * with RBE2D_IBC: + F_IBC = -dU_IBC^M/dz_i (Eq. 3.18, general non-neutral form);
 * with RBE2D_REAL: + the erfc real-space force of real and image charges within r_c
 * (Eq. 3.12; the context must have been created with real_space = 1).  force_out
 * (N x 3) is overwritten, or added to with RBE2D_ACCUMULATE (device buffers only; the
 * same holds for phi_out).  phi_out (N, may be NULL) receives
 * dU/dq_i with RBE2D_POTENTIAL.  energy_out (4 float64, may be NULL) receives
 * {U_k, U_self, U_IBC, U_real} with RBE2D_ENERGY: U_k = (2 pi/V)(S/P) sum_l
 * [(1+E)|rho|^2 + Re(O rho conj(sigma))]/k^2, U_self = -alpha/sqrt(pi) sum q^2.
 * The batch is the last one drawn or set; a call before any batch returns
 * RBE2D_EINVAL.
 */
int rbe2d_force(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                void* force_out, void* phi_out, double* energy_out);

/*
 * Adjoint of the k-space energy U = U_k + U_self + U_IBC for the current batch:
 *   dpos = grad_energy * dU/dr_i   (= -grad_energy * F_i, N x 3)
 *   dq   = grad_energy * dU/dq_i   (N)
 *   dgamma[0..1] = grad_energy * dU/dgamma_top, dU/dgamma_bot  (device float64)
 * The N x P phase table is never stored: the phases are recomputed.  Any output may
 * be NULL.  flags: RBE2D_INPUT_F32, RBE2D_REUSE_SF.
 */
int rbe2d_energy_backward(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                          double grad_energy, void* dpos, void* dq, double* dgamma);

/*
 * Structure factors rho_l, sigma_l (as rbe2d_structure_factor, float32 phases and
 * float64 sums) for callers that cannot allocate device memory on their call path:
 * code running inside a stream capture in global mode, where cudaMalloc is refused,
 * and hosts whose device memory is owned by their own pool.  The paper has no
 * counterpart; this is a deployment variant of the structure-factor step.
 *  - No context and no allocation: the scratch (512 x 256 x 4 float64 partial sums,
 *    4 MiB) is a fixed array inside the library, held by every GPU that loads it
 *    until the process exits.
 *  - pos (N x 3), q (N) float64, k_idx (P x 3 int32) and rho_out (P x 4 float64:
 *    Re rho, Im rho, Re sigma, Im sigma) are caller-owned device pointers on the
 *    current device; stream is a cudaStream_t (NULL: the legacy default stream).
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call shares the one array, and each call writes every slot it reads, so
 *    nothing needs clearing; calls that overlap on the GPU race on it and must be
 *    serialised by the caller.
 *  - Returns RBE2D_EINVAL, launching nothing, for P outside [1, 512], N < 0,
 *    non-positive Lx, Ly, Lz or a NULL pointer; RBE2D_ECUDA if the address lookup or
 *    a launch fails.
 */
int rbe2d_structure_factor_noalloc(double Lx, double Ly, double Lz, int64_t N, const double* pos,
                                   const double* q, int P, const int32_t* k_idx, double* rho_out,
                                   void* stream);

/*
 * As rbe2d_sample_k, with the step number read from device memory (*step_dev, one
 * uint64) when the kernel runs, so a captured CUDA graph draws a new batch on every
 * replay once the counter advances.
 */
int rbe2d_sample_k_dev(rbe2d_ctx* ctx, const uint64_t* step_dev, int32_t* k_idx_out);

/* Langevin molecular dynamics (Eq. 2.27; Algorithm 2's loop). */
typedef struct {
    double dt;                   /* time step */
    double gamma;                /* friction coefficient of the Langevin thermostat */
    double kT;                   /* thermal energy k_B T */
    double mass;                 /* mass of every particle */
    double sigma_lj, eps_lj;     /* WCA repulsion between charges (Sec. 4.1); sigma <= 0: none */
    double sigma_wall, eps_wall; /* WCA walls at z = 0 and z = H (Sec. 4.1); sigma <= 0: none */
    uint64_t noise_seed;         /* Philox4x32-10 key of the thermostat noise */
    int force_flags;             /* subset of RBE2D_KSPACE | RBE2D_IBC | RBE2D_REAL */
} rbe2d_md_params;

#define RBE2D_MD_FORCE 1  /* compute force_inout at pos (before the first step) */
#define RBE2D_MD_STEP 2   /* one BAOAB step; force_inout must hold the force at pos */

/*
 * One Langevin step in the BAOAB splitting (Leimkuhler and Matthews): half kick with
 * force_inout (+ walls), half drift, Ornstein-Uhlenbeck velocity update with Philox
 * normals (counter = particle, *step_dev; key = noise_seed), half drift, a new batch for
 * step *step_dev (rbe2d_sample_k_dev), the force at the new positions (flags of
 * md->force_flags, plus WCA pairs through the real-space cell list when sigma_lj > 0),
 * half kick; then *step_dev += 1 on the device.
 *  - pos, vel: N x 3 float64 device arrays, updated in place (x, y wrapped into the cell).
 *  - q: N float64 device array.
 *  - force_inout: N x 3 in the context's output precision (float64 in FP64 mode, else
 *    float32), device; holds the force (without walls) at pos on entry (mode
 *    RBE2D_MD_FORCE computes it) and at the new positions on exit.
 *  - step_dev: device uint64 step counter.  stats_dev (device, may be NULL) receives the
 *    kinetic energy after the step.
 *  - No allocation and no synchronisation: a step can be captured in a CUDA graph.
 *  - Real space and WCA pairs: with the pair lists of a context created with skin > 0
 *    (FP32-mixed mode, real_space = 1, Lx and Ly at least 2 (r_c + 2 skin), n_max below
 *    2^25), every charge keeps the list of sources (charges and images) within r_c + skin
 *    and each step evaluates the listed pairs within r_c.  The lists are rebuilt on the
 *    device, inside the same step, whenever some charge has moved more than skin / 2
 *    since the last build (so they hold every pair within r_c), and whenever N changes.
 *    The result equals the cell scan's up to float32 summation order.  Without lists the
 *    cell scan runs every step.  A list that would exceed its capacity is reported as
 *    RBE2D_ERANGE by rbe2d_sync_status.
 *  - RBE2D_EINVAL for non-positive dt, mass or kT < 0, WCA cutoffs beyond r_c, or
 *    RBE2D_REAL / sigma_lj > 0 without the real-space buffers (real_space = 1 at init).
 */
int rbe2d_md_step(rbe2d_ctx* ctx, int64_t N, double* pos, double* vel, const double* q, void* force_inout,
                  uint64_t* step_dev, const rbe2d_md_params* md, int mode, double* stats_dev);

/* Pair-list state of rbe2d_md_step (no counterpart in the paper): *enabled_out (host, may
 * be NULL) = 1 if the context has pair lists; *builds_out (host, may be NULL) = the
 * number of list builds so far.  Synchronises the context's stream. */
int rbe2d_md_list_stats(rbe2d_ctx* ctx, int* enabled_out, uint64_t* builds_out);

/*
 * Batched systems: many independent slabs, each with its own rbe2d_params (geometry,
 * contrasts, M, alpha, P <= 512, seed; precision must be RBE2D_FP32_MIXED), evaluated
 * by one sampling launch and one persistent launch (the batched form of rbe2d_sample_k +
 * rbe2d_force with RBE2D_KSPACE [| RBE2D_IBC]).  Particles of system s are the rows
 * offsets[s] .. offsets[s+1]-1 of the concatenated arrays (offsets: host, n_sys + 1
 * entries, non-decreasing).  Automatic rules apply per system, alpha from its own N.
 */
typedef struct rbe2d_batch rbe2d_batch;
int rbe2d_batch_init(const rbe2d_params* per_sys, int n_sys, const int64_t* offsets, void* stream,
                     rbe2d_batch** out);
int rbe2d_batch_destroy(rbe2d_batch* batch);
const char* rbe2d_batch_last_error(const rbe2d_batch* batch);
/*
 * Forces of every system for MD step `step`: pos (sum N x 3) and q (sum N) float64
 * device arrays, force_out (sum N x 3) float32 device array; energy_out (device,
 * n_sys x 4 float64 {U_k, U_self, U_IBC, F_IBC factor}, may be NULL) with RBE2D_ENERGY.
 * A force item that waits longer than the limit of rbe2d_batch_set_wait (2 s by
 * default) for its system raises a flag reported as RBE2D_ETIMEOUT by
 * rbe2d_batch_sync_status (its chunk is then left unwritten).
 */
int rbe2d_batch_force(rbe2d_batch* batch, uint64_t step, const double* pos, const double* q, int flags,
                      float* force_out, double* energy_out);
/* Synchronise and report device flags (RBE2D_ESAMPLER, RBE2D_ETIMEOUT); clears them. */
int rbe2d_batch_sync_status(rbe2d_batch* batch);
/*
 * Failure detection of the persistent launch (no counterpart in the paper).  seconds in
 * (0, 10] bounds every force item's wait for its system's fold (default 2 s).
 * withhold_sys >= 0 is host-side fault injection for tests of that path: from the next
 * rbe2d_batch_force on, the fold of system withhold_sys completes but never publishes
 * its ready flag, so each of that system's force items waits out the limit, leaves its
 * rows of force_out unwritten and raises RBE2D_ETIMEOUT (rbe2d_batch_sync_status); every
 * other system is evaluated as usual and the launch returns.  -1 (the default) injects
 * nothing.  RBE2D_EINVAL for a limit or a system index out of range.
 */
int rbe2d_batch_set_wait(rbe2d_batch* batch, double seconds, int withhold_sys);
/*
 * Time the persistent launch for structure-factor chunks {256, 512, 1024, 2048}
 * particles, force chunks {256, 512, 1024}, 1 or 2 resident CTAs' worth of grid and four
 * kernel variants -- bit 0: registers capped for 8 resident CTAs per SM (P <= 256 only),
 * bit 1: one angle of each group of the structure-factor items on the FMA-pipe
 * polynomial -- on the given inputs (overwriting force_out) and keep the fastest; choice
 * (host, 4 ints, may be NULL) receives {sf_chunk, f_chunk, grid, variant}.  Synchronises;
 * not for use inside a capture.
 */
int rbe2d_batch_autotune(rbe2d_batch* batch, const double* pos, const double* q, float* force_out, int* choice);
/* Set the batched launch's choice directly (host, 4 ints as rbe2d_batch_autotune writes
 * them: chunk sizes of at least 256, grid >= 1, variant 0-3).  RBE2D_EINVAL when out of
 * range.  Synchronises (uploads the work items). */
int rbe2d_batch_set_tuning(rbe2d_batch* batch, const int* choice);

/*
 * Autotuner of the FP32-mixed kernels (no counterpart in the paper): times the
 * structure-factor and force kernels on the given inputs and the current batch and keeps
 * the fastest variant of each.  The variants are
 *  - the share of sin/cos evaluated on the FMA pipe by a full-circle polynomial instead of
 *    MUFU (which bounds both kernels): level 0-3 = 0, 1, 2 or 4 angles in each group of 8
 *    (structure factor: wave vectors of a thread with their k-hat angle moved; force: the
 *    (particle, wave vector) terms of a record with their second angle moved, a pair of
 *    them evaluated with paired instructions);
 *  - the structure factor's shape: wave vectors per thread x particles per shared-memory
 *    tile x resident CTAs per SM = {4 x 224 x 8, 4 x 448 x 5, 2 x 224 x 8} (shapes 0-2;
 *    float64 device inputs; other inputs run shape 0);
 *  - the force kernel's round: threads per CTA x particles per thread =
 *    {256 x 2, 128 x 2, 256 x 1, 512 x 2, 256 x 2 with registers cut for 5 resident CTAs
 *    per SM, 256 x 1 with each particle's k-sum split over 2 and over 4 threads} (shapes
 *    0-6; the split shapes serve systems too small to fill the GPU; the potential variant
 *    has its own choice, rbe2d_autotune_potential).
 * Every variant computes the same sums; they differ in rounding only where an angle moves
 * to the polynomial.  flags: RBE2D_IBC, RBE2D_INPUT_F32.  force_scratch (device, N x 3
 * float32) is overwritten.  choice (host, 4 ints, may be NULL) receives {structure-factor
 * share, force share, structure-factor shape, force shape}.  Synchronises; a no-op in
 * RBE2D_FP64 mode.
 */
int rbe2d_autotune(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                   void* force_scratch, int* choice);
/* Set the tuner's choice directly (host, 4 ints as rbe2d_autotune writes them), e.g. one
 * saved earlier.  RBE2D_EINVAL for a value out of range. */
int rbe2d_set_tuning(rbe2d_ctx* ctx, const int* choice);
/*
 * Autotuner of the force kernel's potential variant (no counterpart in the paper): the
 * launch that computes dU/dq_i beside the force (RBE2D_POTENTIAL, and dq of
 * rbe2d_energy_backward, the gradient of Eq. 3.16 through Sec. 3.4's recalibrated form).
 * Times it on the given inputs and the current batch, after one structure factor, and
 * keeps the fastest of
 *  - the FMA-pipe share of its sin/cos, levels 0-3 as in rbe2d_autotune;
 *  - its round: threads per CTA x particles per thread = {256 x 2 with registers cut for
 *    4 resident CTAs per SM and each particle's k-sum in 1, 2 or 4 threads, 256 x 1 cut
 *    for 6 resident CTAs per SM} (shapes 0-3).
 * flags: RBE2D_IBC, RBE2D_INPUT_F32.  force_scratch (device, N x 3 float32) and
 * phi_scratch (device, N float32) are overwritten.  choice (host, 2 ints, may be NULL)
 * receives {share, shape}.  Synchronises; a no-op in RBE2D_FP64 mode.  Until it runs
 * (or rbe2d_set_tuning_potential) the potential variant takes {0, 0}.
 */
int rbe2d_autotune_potential(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                             void* force_scratch, void* phi_scratch, int* choice);
/* Set the potential variant's choice directly (host, 2 ints as rbe2d_autotune_potential
 * writes them).  RBE2D_EINVAL for a value out of range. */
int rbe2d_set_tuning_potential(rbe2d_ctx* ctx, const int* choice);

/*
 * Particle-sharded evaluation (the exchange behind the paper's O(1) communication,
 * Sec. 2.4): every shard draws the same batch (same seed and step), evaluates
 * rbe2d_structure_factor on its own particles, adds rho_out and the charge sums of all
 * shards (one allreduce of P x 4 + 4 float64), hands the totals back with
 * rbe2d_set_structure_factor, and calls rbe2d_force with RBE2D_REUSE_SF on its own
 * particles.  The per-shard energies then refer to the whole system.
 *  - rbe2d_charge_sums: sums_out (device, 4 float64) = {sum q, sum q^2, sum q z, sum |q|}
 *    of the last rbe2d_structure_factor call.
 *  - rbe2d_set_structure_factor: rho (device, P x 4) and sums (device, 4) are the totals;
 *    N must be the local particle count of the preceding rbe2d_structure_factor.
 */
int rbe2d_charge_sums(rbe2d_ctx* ctx, double* sums_out);
int rbe2d_set_structure_factor(rbe2d_ctx* ctx, int64_t N, const double* rho, const double* sums);

/*
 * Synchronise the context's stream and report device-side status flags
 * (RBE2D_ESAMPLER, RBE2D_ETIMEOUT) raised since the previous call; clears them.
 */
int rbe2d_sync_status(rbe2d_ctx* ctx);

/*
 * Deterministic lattice sum (no random batch): the k-space part of Eq. 3.16 with the
 * re-calibrated images (Sec. 3.4) summed over every k != 0 of the box |n_d| <= nmax[d]
 * with its Gaussian weight w(k) = exp(-k^2/4alpha^2) (Eq. 2.21), which is the sum the
 * random batch estimates without bias (Theorem 2.3); with nmax large enough that the
 * weights left out are negligible it is the Ewald sum of the extended system, the
 * quasi-2D reference that the random batch converges to (Theorem 3.3).  The lattice is
 * processed as chunks of P wave vectors of the half space {(nz, ny, nx) > 0 in
 * lexicographic order}, each counted twice (the terms of k and -k are equal), through
 * the same structure-factor, fold and force kernels as rbe2d_force; the chunks' energies
 * and forces are summed on the device in chunk order.
 *   nmax: host, 3 int32 in [0, 2^20], not all 0; cost is (number of k / 2) x N pairs.
 *   flags: RBE2D_IBC, RBE2D_ENERGY, RBE2D_POTENTIAL, RBE2D_INPUT_F32, RBE2D_ACCUMULATE
 *   (RBE2D_KSPACE is implied; others are EINVAL).  Outputs as for rbe2d_force; energy_out
 *   = {U_k over the lattice, U_self, U_IBC, 0}.
 * Afterwards the context's current batch is the last chunk (weights included); call
 * rbe2d_sample_k or rbe2d_set_k before the next random-batch evaluation.
 */
int rbe2d_force_lattice(rbe2d_ctx* ctx, int64_t N, const void* pos, const void* q, int flags,
                        const int32_t* nmax, void* force_out, void* phi_out, double* energy_out);

/*
 * Per-kernel timer (no counterpart in the paper; a measurement aid).  While enabled,
 * every launch of a class selected by class_mask (bit k = class k below) made by this
 * context records a pair of CUDA events on the context's stream around it, up to
 * `capacity` launches per class; launches past that, and launches made while the stream
 * is being captured into a graph, are not recorded.  Each recorded pair adds a few
 * microseconds of stream time, so time only the classes you need.
 * rbe2d_timer_enable(ctx, 0, 0) disables the timer and frees the events; a new call
 * discards earlier records.  EINVAL for capacity outside [0, 2^20] or unknown mask bits.
 * rbe2d_timer_read synchronises the stream, writes for each class the summed device time
 * in ms (total_ms, host, RBE2D_TIMER_COUNT doubles) and the number of recorded launches
 * (launches, host, RBE2D_TIMER_COUNT int64, may be NULL), then clears the records.
 * RBE2D_TIMER_REAL covers the whole cell-list build plus pair kernel of one call;
 * RBE2D_TIMER_PACK only the FP64 mode's separate packing kernel (FP32 mode packs inside
 * the structure-factor kernel).
 */
enum {
    RBE2D_TIMER_SAMPLE = 0,
    RBE2D_TIMER_PACK = 1,
    RBE2D_TIMER_SF = 2,
    RBE2D_TIMER_FOLD = 3,
    RBE2D_TIMER_FORCE = 4,
    RBE2D_TIMER_REAL = 5,
    RBE2D_TIMER_MD = 6,
    RBE2D_TIMER_COUNT = 7
};
#define RBE2D_TIMER_ALL 0x7Fu
int rbe2d_timer_enable(rbe2d_ctx* ctx, int capacity, unsigned class_mask);
/*
 * Number of CUDA kernels this library has enqueued in this process, over all contexts
 * and devices (host counter, no synchronisation; count_out is a host pointer).  The
 * difference of two readings counts the kernels of the calls in between.
 */
int rbe2d_kernel_launches(uint64_t* count_out);
/*
 * Measured throughput of the pipes that bound this library's kernels, on the current
 * device (no counterpart in the paper; the denominators of the roofline fractions):
 * out (host, 4 doubles) = {sin/cos results (MUFU), float32 FMAs, float64 FMAs} per clock
 * per SM, and the SM clock in MHz over the sin/cos probe (its cycles over its event
 * time).  Each probe runs 32 warps per SM with eight independent chains per thread,
 * three times; the best rate is kept.  Allocates and synchronises (about 10 ms);
 * RBE2D_EINVAL for a NULL out, RBE2D_ECUDA if a launch fails.
 */
int rbe2d_pipe_probe(double* out);
int rbe2d_timer_read(rbe2d_ctx* ctx, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* RBE2D_H */
