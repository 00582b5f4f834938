/*
 * ac.h -- C ABI of the GB300 (sm_103a) Allen-Cahn stepper.
 *
 * The library advances the explicit finite-difference Allen-Cahn scheme of
 * Kim, "Fast Numerical Simulation of Allen-Cahn Equation" (arXiv 2105.09671):
 *
 *   phi_t = -F'(phi)/eps^2 + Lap phi,  F(phi) = (phi^2 - 1)^2 / 4  (Eq. oriACeq)
 *   phi^{n+1} = phi^n + dt ((phi^n - (phi^n)^3)/eps^2 + Lap_h phi^n)  (Eq. pytorchACeq)
 *
 * on a cell-centred grid with h = 1/Nx, zero-Neumann boundaries realised by
 * replicating the boundary cell into a ghost layer (Section 2), a 5-point
 * (2D) or 7-point (3D) Laplacian and forward Euler with dt = 0.1 h^2.
 *
 * Conventions for every entry point:
 *   - All functions return an int status: AC_OK (0) or one of AC_ERR_*.
 *     No C++ exception crosses this boundary.  ac_last_error() gives a
 *     thread-local message for the last failure on the calling thread.
 *   - Device pointers are plain CUDA global-memory addresses owned by the
 *     caller; the library never frees them.  The library allocates only
 *     small internal reduction/status buffers in ac_create and releases them
 *     in ac_destroy.
 *   - Work is stream-ordered on the caller's CUDA stream (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).  Only the functions
 *     documented as synchronising wait for the stream.
 *   - Not thread-safe per context: one host thread drives one context at a
 *     time.  Different contexts are independent.
 */
#ifndef AC_H_
#define AC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status ---- */
enum {
  AC_OK = 0,
  AC_ERR_INVALID = 1,     /* bad descriptor, pointer, alignment or argument */
  AC_ERR_CUDA = 2,        /* a CUDA runtime / driver call failed            */
  AC_ERR_NONFINITE = 3,   /* the field holds NaN or Inf                     */
  AC_ERR_TIMEOUT = 4,     /* a bounded device-side wait expired             */
  AC_ERR_UNSUPPORTED = 5, /* valid request this build cannot serve          */
  AC_ERR_NOMEM = 6        /* internal allocation failed                     */
};

/* ------------------------------------------------------ storage types ---- */
typedef enum {
  AC_F64 = 0,  /* FP64 storage, FP64 arithmetic                        */
  AC_F32 = 1,  /* FP32 storage, FP32 arithmetic                        */
  AC_F16S = 2  /* FP16 storage (IEEE binary16), FP32 arithmetic; values
                  are rounded to nearest-even only when written to memory */
} ac_dtype;

/* -------------------------------------------------------- descriptor ---- */
/* One simulation grid (Section 2): Nx x Ny (x Nz) cells of size h.
 *
 * Layout of phi in device memory: row-major, x fastest.  Cell (i, j, k),
 * 0-based, lives at element  (k * ny + j) * pitch_x + i.
 *
 *   ndim     2 or 3.  For ndim == 2, nz must be 1.
 *   dtype    an ac_dtype.
 *   nx,ny,nz number of cells per axis, each >= 1.
 *   pitch_x  elements between consecutive rows; pitch_x >= nx and
 *            pitch_x * element_size is a multiple of 16 bytes.
 *   h        cell size (the paper uses h = 1/Nx).
 *   eps      interface-thickness parameter epsilon > 0 (Eq. emvalue gives
 *            the paper's choice eps_m = h m / (2 sqrt(2) atanh(0.9))).
 *            eps = +INFINITY drops the reaction term (alpha = 0): the same
 *            kernels then advance the heat equation phi_t = Lap phi with
 *            explicit Euler, the kind of other explicit finite-difference
 *            PDE the paper's conclusion names for its scheme (the energy
 *            reduces to the Dirichlet term).
 *   dt       time step > 0.  The paper uses dt = 0.1 h^2.  The library
 *            requires dt <= h^2 / (2 ndim) (stability of the explicit
 *            Laplacian) and dt <= eps^2 (reaction step alpha = dt/eps^2
 *            at most 1); anything else is AC_ERR_INVALID.  Within those
 *            limits the scheme keeps |phi| <= 1 (a discrete maximum
 *            principle, and with it the monotone energy decrease) only
 *            while the centre coefficient 1 + alpha - 3 alpha phi^2 -
 *            2 ndim dt/h^2 stays positive, i.e. alpha < (1 - 2 ndim dt/h^2)/2
 *            (0.2 in 3D and 0.3 in 2D at dt = 0.1 h^2); beyond that (eps
 *            well below h) a run can overshoot +-1, as the same scheme does
 *            in FP64.
 */
typedef struct {
  int32_t ndim;
  int32_t dtype;
  int64_t nx, ny, nz;
  int64_t pitch_x;
  double h, eps, dt;
} ac_grid_desc;

typedef struct ac_ctx ac_ctx; /* opaque */

/* Bytes of device workspace ac_create needs: one more field of the same
 * layout (the ping-pong partner of phi).  Writes the count to *out. */
int ac_workspace_bytes(const ac_grid_desc *desc, size_t *out);

/* Create a stepping context for the field phi_dev (laid out as described
 * by desc) with workspace_dev of at least ac_workspace_bytes() bytes.
 * Both pointers must be 16-byte aligned device addresses and must not
 * overlap.  cuda_stream is the cudaStream_t all later work is ordered on.
 * The context keeps the pointers; the caller keeps ownership and must keep
 * them alive until ac_destroy.  The device current at this call is used. */
int ac_create(const ac_grid_desc *desc, void *phi_dev, void *workspace_dev,
              void *cuda_stream, ac_ctx **out);

/* Advance phi by n >= 0 explicit Euler steps of Eq. (pytorchACeq) with the
 * zero-Neumann ghosts of Section 2.  Asynchronous on the context's stream;
 * when the work completes the result is in phi_dev (the workspace holds
 * intermediate states).  The schedule (kernel variant and temporal-block
 * depth k: steps advanced per HBM round trip) is the one chosen by
 * ac_set_schedule / ac_autotune, else a built-in default. */
int ac_step(ac_ctx *ctx, int64_t n);

/* Discrete Ginzburg-Landau energy of the current phi, summed in FP64:
 *   E_h = h^d [ sum_cells F(phi)/eps^2 + 1/2 sum_interior faces ((phi_a - phi_b)/h)^2 ]
 * (not defined in the paper; its gradient is -h^d times the right-hand side
 * of Eq. pytorchACeq, so the scheme decreases it).  The per-cell terms are
 * formed in FP64 for FP64 storage and in float-float arithmetic (~46 bits;
 * the stored values are exact in FP32) for FP32 / FP16 storage, so the
 * result is within ~1e-15 relative of FP64 terms.  Synchronises the stream.
 * Returns AC_ERR_NONFINITE (and still writes *out) if phi holds NaN/Inf. */
int ac_energy(ac_ctx *ctx, double *out);

/* Phase volume V = h^d sum (1 + phi)/2 in FP64 (area in 2D).  The
 * equivalent radius sqrt(V/pi) (2D) or (3V/(4 pi))^(1/3) (3D) is compared
 * with the shrinking law r(t)^2 = r0^2 + 2(1 - d) t (Eq. exactradiusEQ).
 * Synchronises the stream. */
int ac_phase_volume(ac_ctx *ctx, double *out);

/* Energy, volume and the count of non-finite cells from one pass over phi,
 * written to out[0], out[1], out[2] (the count as a double).  Synchronises. */
int ac_observe(ac_ctx *ctx, double out[3]);

/* Initial conditions of Section 3.1, generated on the device into phi.
 * ac_init_sphere: phi = tanh((r0 - |x - c|)/(sqrt(2) eps)) at cell centres
 *   x_i = lower + (i + 0.5) h (circle in 2D; cz is ignored), evaluated in
 *   FP64 and rounded once to the storage type.
 * ac_init_random: phi = amplitude * (2 u - 1), u = (z >> 11) 2^-53, where z
 *   is output number (c + 1) of the SplitMix64 sequence seeded with `seed`
 *   (Steele, Lea, Flood 2014) and c is the cell's linear index x + nx (y +
 *   ny z) (pitch excluded).  The paper's random state is amplitude 0.1.
 * Both are asynchronous on the context's stream. */
int ac_init_sphere(ac_ctx *ctx, double lower_x, double lower_y, double lower_z,
                   double cx, double cy, double cz, double r0);
int ac_init_random(ac_ctx *ctx, uint64_t seed, double amplitude);

/* The further initial shapes of Section 3.1 (Eqs. 2Ddumbellini,
 * 3Ddumbellini, 2Dstarini, 3Dstarini, 2Dtorusini, 3Dtorusini), generated on
 * the device at the cell centres lower + (i + 0.5) h, in FP64 with
 * w = sqrt(2) eps, rounded once to the storage type:
 *   AC_SHAPE_DUMBBELL (p0 = R0; domain (0,2) x (0,1) [x (0,1)]): 1 inside the
 *     bar 0.4 < x < 1.6, 0.4 < y [, z] < 0.6, else 1 + tanh((R0 - d_l)/w)
 *     + tanh((R0 - d_r)/w), d_l, d_r the distances to (0.3, 0.5 [, 0.5]) and
 *     (1.7, 0.5 [, 0.5]);
 *   AC_SHAPE_STAR (no parameters): 2D tanh((0.25 + 0.1 cos 6t - r)/w) about
 *     (0.5, 0.5) (unit square); 3D tanh((0.7 + 0.2 cos 6t - |p|)/w) on
 *     (-1,1)^3 with t the polar angle of (x, z) about the origin (the
 *     printed test "x > 0.5" read as the 2D form's);
 *   AC_SHAPE_TORUS (p0 = R1, p1 = R2): 2D annulus -1 + tanh((R1 - r)/w)
 *     - tanh((R2 - r)/w) about (0.5, 0.5); 3D the printed signed distance
 *     d = sqrt(z^2 + (sqrt(x^2 + y^2) - R1)^2) - R2 to a ring about the z
 *     axis, used as tanh(-d/w) (phase +1 inside the tube).
 * Unused parameters are ignored.  AC_ERR_INVALID for an unknown kind or a
 * non-finite value.  Asynchronous on the context's stream. */
enum { AC_SHAPE_DUMBBELL = 1, AC_SHAPE_STAR = 2, AC_SHAPE_TORUS = 3 };
int ac_init_shape(ac_ctx *ctx, int32_t kind, double lower_x, double lower_y, double lower_z,
                  double p0, double p1);

/* ------------------------------------------------------- scheduling ---- */
/* Kernel variants selectable with ac_set_schedule. */
enum {
  AC_VARIANT_AUTO = 0,    /* autotuned choice if ac_autotune ran, else default */
  AC_VARIANT_DIRECT = 1,  /* one step per launch, neighbours read from global
                             memory with clamped indices (k must be 1)         */
  AC_VARIANT_STREAM = 2   /* TMA-staged streaming kernel with temporal blocking:
                             2D warp strips streaming along y with warp-shuffle
                             x neighbours; 3D xy tiles streaming along z with
                             shared-memory x/y neighbours; k steps per pass    */
};

/* Force the kernel variant and temporal-block depth k (1..AC_MAX_K) used by
 * ac_step.  variant = AC_VARIANT_AUTO with k = 0 restores the default. */
#define AC_MAX_K 8
int ac_set_schedule(ac_ctx *ctx, int32_t variant, int32_t k);
int ac_get_schedule(ac_ctx *ctx, int32_t *variant, int32_t *k);

/* Tile shape of the streaming kernel.  3D: the xy block each CTA streams
 * along z (temporal blocking recomputes a halo of k cells around it),
 * tiles 0..AC_NUM_TILES_3D-1 (FP32 / FP16 storage; FP64 tiles are half as
 * wide in x):
 *   0: 128 x 32 outputs, two rows per thread
 *   1: 128 x 16 outputs, two rows per thread, several CTAs per SM
 *   2: 128 x 32 outputs, four rows per thread (FP16 storage: one)
 * 2D: the width of the column strip each warp streams along y, tiles
 * 0..AC_NUM_TILES_2D-1:
 *   0: one 16-byte vector per lane (FP32 / FP16 storage: 4 / 8 cells;
 *      FP64: two vectors, 4 cells), depths up to 8 (FP16 storage: 6)
 *   1: FP32 only, two vectors per lane (8 cells, 256-cell strips; half
 *      the shuffles and the strip-halo share per cell), depths up to 6
 * AC_TILE_AUTO (-1) restores the autotuned or default choice; a tile the
 * grid kind does not offer is AC_ERR_UNSUPPORTED.  The result of a step
 * does not depend on the tile. */
#define AC_TILE_AUTO (-1)
#define AC_NUM_TILES_3D 3
#define AC_NUM_TILES_2D 2
int ac_set_tile(ac_ctx *ctx, int32_t tile);
int ac_get_tile(ac_ctx *ctx, int32_t *tile);

/* Time the candidate (variant, k, tile) schedules on the context's own buffers
 * with CUDA events (about steps_per_trial steps each) and keep the fastest;
 * a context with graph replay on (ac_set_graph) has each candidate timed as
 * a replayed graph, the way its steps will run.
 * phi is saved to a temporary device buffer that this call allocates and
 * frees, and restored after every trial, so the field is unchanged.  The
 * choice is cached per (ndim, dtype, log2 of the cell count, device model,
 * graph replay on or off) for the process lifetime (and in a file, see ac_set_tune_cache); later
 * contexts of the same class reuse it without timing.  Synchronises the
 * stream. */
int ac_autotune(ac_ctx *ctx, int64_t steps_per_trial);

/* Keep autotuning results in a text file as well (one line per choice:
 * "ac-tune-v2 ndim dtype size_class device graph variant k tile", device =
 * the model name and SM count, graph = 1 for choices timed as graph
 * replays; lines of the earlier v1 form, without the graph field, are read
 * as graph = 0), so that later processes skip the timing:
 * ac_autotune first looks in the process cache, then in the file, and
 * appends what it measures.  NULL or "" stops using a file.  Also empties
 * the process cache.  An unreadable file is treated as empty and a failed
 * append is ignored (the choice is still used in this process).  Entries
 * for a schedule this library does not offer are ignored. */
int ac_set_tune_cache(const char *path);

/* Replay ac_step through a CUDA graph: the first ac_step(n) after enabling
 * (or after the schedule or n changes) captures the whole launch sequence
 * for n steps into a graph; later calls with the same n launch the graph
 * (one launch instead of one per pass).  Needs a non-default stream
 * (AC_ERR_UNSUPPORTED otherwise).  enable = 0 drops the graph. */
int ac_set_graph(ac_ctx *ctx, int32_t enable);

/* Device-side error word of the context (bounded waits that expired set
 * it).  Synchronises, returns AC_ERR_TIMEOUT if set and clears it. */
int ac_status(ac_ctx *ctx);

/* Number of CUDA kernels this context has enqueued on its stream since
 * ac_create (stencil passes, reductions, initial conditions; a graph replay
 * counts the kernels it contains).  The ws -> phi copy that ends an odd
 * number of single-step passes is a copy, not a kernel, and is not counted. */
int ac_launch_count(ac_ctx *ctx, int64_t *out);

/* ------------------------------------------------ tensor-core building block */
/* D[m x 32] = A[m x k] * B[32 x k]^T with BF16 operands (row-major, k
 * contiguous) and FP32 accumulation on the 5th-generation tensor cores
 * (tcgen05, accumulator in tensor memory).  m a multiple of 128, k a multiple
 * of 16 in [16, 512]; all pointers device memory, 16-byte aligned.  The
 * learned stepper's convolutions are built from the same primitive (their
 * reduction dimension is 9 or 27 taps x 32 channels); exposed so the operand
 * layout can be verified on its own.  Asynchronous on cuda_stream. */
int ac_tc_gemm_bf16_n32(const void *a_dev, const void *b_dev, float *d_dev, int64_t m,
                        int32_t k, void *cuda_stream);

/* --------------------------------------------------- learned stepper ---- */
/* A small convolutional network that jumps n (default 16) explicit Euler
 * steps at once, trained on trajectories of the plain stepper, with the
 * plain stepper as its fallback (not in the paper; its building block is the
 * paper's replicate padding + convolution of Section 2.2).  Definition:
 *   z1 = conv(phi, W1) + b1, a1 = gelu(z1)            1 -> 32 channels
 *   zl = conv(a_{l-1}, Wl) + bl, al = gelu(zl)         32 -> 32, l = 2..5
 *   z6 = conv(a5, W6) + b6                             32 -> 1
 *   phi_hat = phi + s * z6,   s = n dt / eps^2
 * conv = 3x3 (2D) or 3x3x3 (3D) cross-correlation with replicate padding;
 * gelu(x) = x/2 (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3))).  Activations are
 * BF16, accumulation FP32; the 32 -> 32 layers (forward, data and weight
 * gradients) run as implicit GEMMs on the tcgen05 tensor cores.
 * Parameters: one flat FP32 vector, per layer W[t][ci][co] then b[co],
 * taps t over offsets (-1, 0, 1)^d with x fastest.
 * Fields: FP32, contiguous [batch][nz][ny][nx] device arrays. */
typedef struct ac_net ac_net; /* opaque */

/* The guard every learned jump phi -> phi_hat must pass; a rejected jump is
 * replaced by n plain steps.  Checks, all on the device:
 *   energy    E(phi_hat) <= E(phi) (1 + energy_rtol)  (the scheme decreases
 *             the discrete energy; FP64 reduction);
 *   max-norm  max |phi_hat| <= max_abs (the scheme keeps |phi| <= 1);
 *   residual  max |phi_hat - phi - n dt RHS(phi)| <= residual_tol, RHS the
 *             bracket of Eq. (pytorchACeq): a one-shot Euler estimate of the
 *             jump, a coarse consistency check (ac_net_calibrate_guard sets
 *             residual_tol from the plain stepper's own residual);
 *   spot      the local error against the plain stepper itself: on
 *             spot_samples boxes of spot_size^d cells (plus an n-cell margin)
 *             at pseudo-random places (spot_seed, advanced every jump) the
 *             plain stepper's n-step result is computed exactly (the n-step
 *             domain of dependence fits in the box) and compared with
 *             phi_hat: accept if sqrt(sum (phi_hat - ref)^2 / sum ref^2)
 *             <= spot_rtol over the checked cells.
 * A tolerance <= 0 disables its check.  spot_samples / spot_size = 0 take
 * the defaults 64 / 32 (2D) and 16 / 8 (3D). */
typedef struct {
  int32_t steps_per_jump; /* n: Euler steps one learned jump stands for            */
  double energy_rtol;     /* accept if E(phi_hat) <= E(phi) (1 + energy_rtol)       */
  double max_abs;         /* accept if max |phi_hat| <= max_abs                     */
  double residual_tol;    /* accept if max |phi_hat - phi - n dt RHS(phi)| <= this  */
  double spot_rtol;       /* accept if the spot-checked relative L2 error <= this   */
  int32_t spot_samples;   /* boxes checked per jump (0 = default)                   */
  int32_t spot_size;      /* checked cells per box side (0 = default)               */
  uint64_t spot_seed;     /* places of the boxes (jump j uses spot_seed + j)        */
} ac_guard;

/* What ac_learned_advance saw: jumps tried, rejections by cause (a jump can
 * fail several checks; each failed check is counted), and the largest
 * values of the checked quantities over all jumps (accepted or not). */
typedef struct {
  int64_t jumps, fallbacks;
  int64_t rejected_nonfinite, rejected_energy, rejected_max_abs, rejected_residual, rejected_spot;
  double max_residual;      /* largest max |phi_hat - phi - n dt RHS(phi)|      */
  double max_spot_rel;      /* largest spot-checked relative L2 error           */
  double max_spot_abs;      /* largest spot-checked max |phi_hat - ref|         */
} ac_learned_report;

int ac_net_param_count(int32_t ndim, int64_t *out);
/* ndim 2 or 3; weights start He-normal (std sqrt(2 / fan_in), seed 0) with
 * the last layer and all biases zero, i.e. the identity jump.
 * Allocates parameter, gradient and optimiser buffers; per-shape activation
 * buffers are allocated on first use of a shape and kept until destroy. */
int ac_net_create(int32_t ndim, void *cuda_stream, ac_net **out);
/* Copy count (= ac_net_param_count) FP32 parameters from / to host memory;
 * setting them also resets the Adam moments.  Synchronise. */
int ac_net_set_params(ac_net *net, const float *host_params, int64_t count);
int ac_net_get_params(ac_net *net, float *host_params, int64_t count);
/* Re-draw the initial weights as ac_net_create does, from another seed. */
int ac_net_init_params(ac_net *net, uint64_t seed);
/* out = phi + scale * NN(phi) for batch fields of nx x ny x nz (nz = 1 in
 * 2D).  phi and out must not overlap.  Asynchronous. */
int ac_net_forward(ac_net *net, const float *phi_dev, float *out_dev, int32_t batch, int64_t nx,
                   int64_t ny, int64_t nz, double scale);
/* Mean over cells of ((phi + scale NN(phi) - target) / scale)^2 and its
 * gradient wrt every parameter (kept for ac_net_adam; copied to grads_host
 * when non-NULL).  Synchronises; *loss is the mean. */
int ac_net_loss_grads(ac_net *net, const float *phi_dev, const float *target_dev, int32_t batch,
                      int64_t nx, int64_t ny, int64_t nz, double scale, double *loss,
                      float *grads_host);
/* One Adam step (Kingma & Ba 2015, bias-corrected) with the last gradients. */
int ac_net_adam(ac_net *net, double lr, double beta1, double beta2, double eps);
/* ac_net_loss_grads + ac_net_adam(lr, 0.9, 0.999, 1e-8). */
int ac_net_train_step(ac_net *net, const float *phi_dev, const float *target_dev, int32_t batch,
                      int64_t nx, int64_t ny, int64_t nz, double scale, double lr, double *loss);
int ac_net_launch_count(ac_net *net, int64_t *out);
int ac_net_destroy(ac_net *net);

/* Training on trajectories of the plain stepper (the network's only data). */
typedef struct {
  int32_t n;                /* training grid: n x n (2D) or n^3 (3D), h = 1/n, n % 4 == 0 */
  double eps_cells;         /* eps = eps_cells * h (dt = 0.1 h^2)                       */
  int32_t pool;             /* trajectories advanced together = the batch size           */
  int32_t trajectory_jumps; /* jumps after which a trajectory is replaced by a new one   */
  int32_t iterations;       /* Adam steps                                                */
  int32_t steps_per_jump;   /* Euler steps per jump                                      */
  double lr, lr_final;      /* cosine learning-rate schedule from lr to lr_final         */
  uint64_t seed;
} ac_train_config;

/* Train `net` (its ndim) on the fly: a pool of trajectories of the plain
 * stepper, started staggered in age, each replaced after trajectory_jumps
 * jumps by a new initial state (alternately random with amplitude 0.1 and a
 * tanh circle / sphere of radius uniform in [0.1, 0.4], Section 3.1).  Each
 * iteration takes the pool as inputs, its steps_per_jump-step advance by
 * the plain stepper (the batched persistent stepper in 2D) as targets, and
 * one Adam step.  loss_history (length iterations, may be NULL) receives
 * each iteration's loss; *trajectories_used the number of trajectories
 * started.  Allocates its pool for the duration of the call.  Synchronises. */
int ac_net_train(ac_net *net, const ac_train_config *cfg, double *loss_history,
                 int64_t *trajectories_used);

/* Guard quantities of a candidate jump phat_dev (FP32 field of the context's
 * layout, pitch_x == nx) from the context's current phi over `steps` steps:
 * out[0] = max |phat|, out[1] = max |phat - phi - steps dt RHS(phi)| with
 * RHS the bracket of Eq. (pytorchACeq).  Used to calibrate the residual
 * threshold on jumps of the plain stepper.  Synchronises. */
int ac_jump_residual(ac_ctx *ctx, const float *phat_dev, int32_t steps, double out[2]);

/* The guard's spot check on its own (FP32 context, phat_dev laid out as
 * the context's field, any pitch): compares phat_dev with the plain
 * stepper's `steps`-step result from the context's phi on `samples` boxes
 * of size^d checked cells (0 = the ac_guard defaults) placed by `seed`.
 * out[0] = max |phat - ref|, out[1] = relative L2 error over the checked
 * cells, out[2] = cells checked.  The reference values are the plain
 * stepper's own FP32 results bit for bit, so a jump made by ac_step gives 0.
 * Allocates and frees a scratch buffer; synchronises. */
int ac_jump_spot_check(ac_ctx *ctx, const float *phat_dev, int32_t steps, int32_t samples,
                       int32_t size, uint64_t seed, double out[3]);

/* Advance the context's field (FP32, pitch_x == nx, same stream as the net)
 * by `jumps` learned jumps of guard->steps_per_jump steps each.  Every jump
 * is checked as ac_guard describes (and for non-finite values); a rejected
 * jump is replaced by that many plain steps (ac_step), so the result is
 * then bit for bit the plain stepper's.  *fallbacks (if non-NULL) receives
 * the number of rejected jumps and *report (if non-NULL) the statistics.
 * Uses the context's workspace for phi_hat and keeps the spot check's
 * scratch in the network (allocated on first use, kept until
 * ac_net_destroy); synchronises once per jump. */
int ac_learned_advance(ac_ctx *ctx, ac_net *net, int64_t jumps, const ac_guard *guard,
                       int64_t *fallbacks, ac_learned_report *report);

/* Calibration of the guard on held-out jumps of the plain stepper, drawn as
 * ac_net_train draws its data (cfg: grid n, eps_cells, steps_per_jump,
 * trajectory_jumps = the age range, pool = the number of held-out states,
 * seed: use one that training did not):  for each state phi the plain
 * n-step result P(phi) and the network's jump phi_hat are formed; the
 * residual threshold is set to residual_factor times the largest residual
 * max |P(phi) - phi - n dt RHS(phi)| of the plain stepper itself (the
 * network must be about as consistent as the method it stands for), i.e.
 * guard->residual_tol is written; the other fields of *guard are kept.
 * *report (if non-NULL) receives the plain and network residuals and the
 * network's relative L2 error against P over whole fields next to the spot
 * check's estimate of it (which uses guard's spot settings).  Allocates its
 * fields for the duration of the call; synchronises. */
typedef struct {
  int32_t states;
  double plain_residual_max;  /* max over states of the plain jump's residual       */
  double net_residual_max;    /* the same for the network's jumps                   */
  double net_rel_err_median;  /* whole-field relative L2 of phi_hat - P(phi)        */
  double net_rel_err_max;
  double spot_rel_err_max;    /* the spot check's estimate of the same, max         */
} ac_guard_calibration;
int ac_net_calibrate_guard(ac_net *net, const ac_train_config *cfg, double residual_factor,
                           ac_guard *guard, ac_guard_calibration *report);

/* ------------------------------------------------------ batched mode ---- */
/* Many independent 2D grids (each its own size, eps, dt and state) advanced
 * together by ONE persistent kernel launch (the paper runs one grid at a
 * time).  Work items are the warp strips x row chunks of the 2D
 * streaming stencil of every instance; a step-block of an item starts once
 * its 3 x 3 neighbourhood has finished the previous one (bounded waits on
 * per-item progress counters), so no grid-wide barrier is needed.  */
typedef struct ac_batch ac_batch; /* opaque */

/* Bytes of device workspace for count instances: the sum over instances of
 * one field of the same layout, each rounded up to 256 bytes. */
int ac_batch_workspace_bytes(const ac_grid_desc *descs, int32_t count, size_t *out);

/* descs[i] / phi_devs[i]: instance i (ndim must be 2, all with one dtype;
 * phi 16-byte aligned).  workspace_dev: 256-byte aligned, at least
 * ac_batch_workspace_bytes() bytes, carved into one ping-pong partner per
 * instance in index order.  The caller owns all buffers.  Allocates small
 * internal tables (per-instance TMA descriptors, work items, progress
 * counters, reduction buffers). */
int ac_batch_create(const ac_grid_desc *descs, void *const *phi_devs, int32_t count,
                    void *workspace_dev, void *cuda_stream, ac_batch **out);

/* Advance instance i by n_per_instance[i] >= 0 steps of Eq. (pytorchACeq)
 * (the same scheme and results as ac_step on that grid with the same depth
 * k).  One kernel launch (plus a ws -> phi copy for an instance whose plan
 * is an odd number of single steps).  Asynchronous; results in phi_devs.
 * Re-planning (new n values or k) synchronises the stream once. */
int ac_batch_step(ac_batch *batch, const int64_t *n_per_instance);

/* Temporal-block depth k of every instance: 1..4 with tile 0, 1..6 with
 * tile 1; 0 = default (4 for FP32/FP16 storage, 1 for FP64). */
int ac_batch_set_schedule(ac_batch *batch, int32_t k);
int ac_batch_get_schedule(ac_batch *batch, int32_t *k);

/* Strip width of every instance's work items (as the 2D tiles of
 * ac_set_tile): 0 = the storage type's default strips, 1 = FP32 strips of
 * 8 cells per lane (AC_ERR_UNSUPPORTED for other storage types, or while
 * the depth exceeds what the tile offers).  Results do not depend on it. */
int ac_batch_set_tile(ac_batch *batch, int32_t tile);
int ac_batch_get_tile(ac_batch *batch, int32_t *tile);

/* Time every (tile, k) the storage type offers on the batch's own fields
 * (steps_per_trial steps each, fields saved to a temporary device buffer
 * this call allocates and restored after each trial) and keep the fastest.
 * Synchronises. */
int ac_batch_autotune(ac_batch *batch, int64_t steps_per_trial);

/* Replay ac_batch_step through a CUDA graph (captured on the first call per
 * plan; needs a non-default stream). */
int ac_batch_set_graph(ac_batch *batch, int32_t enable);

/* ac_observe for instance i (energy, volume, non-finite count).  Synchronises. */
int ac_batch_observe(ac_batch *batch, int32_t i, double out[3]);

/* Synchronises; AC_ERR_TIMEOUT if a bounded wait in the batched kernel
 * expired since the last call (then the results are not valid). */
int ac_batch_status(ac_batch *batch);

/* Poll limit of each bounded wait in the batched kernel (0 = default,
 * about a second).  Lowering it makes waits give up early; used to test
 * the timeout path. */
int ac_batch_set_wait_limit(ac_batch *batch, uint32_t polls);

/* Kernels enqueued by this batch since creation (graph replays count the
 * kernels they contain). */
int ac_batch_launch_count(ac_batch *batch, int64_t *out);

/* Release internal tables (not the caller's buffers).  Synchronises. */
int ac_batch_destroy(ac_batch *batch);

/* ------------------------------------------------ slab decomposition ---- */
/* Domain decomposition of one grid along its slowest axis (z in 3D, y in
 * 2D) into slabs, for grids split over several devices or processes (the
 * paper's conclusion points at larger simulations; the scheme itself is
 * Eq. (pytorchACeq) unchanged).  A step of a cell reads its neighbours
 * only, so n steps of a slab's own planes need the n planes beyond each of
 * its faces: every part holds `halo` extra planes on each side that faces
 * another part, advances its extended slab by at most `halo` steps with
 * the ordinary stepper (the zero-Neumann clamp at an extended slab's
 * artificial faces corrupts only its halo planes, one plane per step), and
 * then refreshes its halos from its neighbours' owned planes.  Owned planes
 * are therefore bit for bit those of the undivided grid (FP16 storage: when
 * both round at the same pass boundaries; a slab's blocks of `halo` steps
 * may place them elsewhere, and then the two agree to the storage rounding). */
typedef struct {
  int64_t own_lo, own_hi; /* planes this part owns: [own_lo, own_hi)              */
  int64_t ext_lo, ext_hi; /* planes it holds, owned plus halos: [ext_lo, ext_hi)  */
} ac_slab_part;

/* Host-only plan, no CUDA call: `extent` planes split into `parts` slabs
 * of extent / parts planes, the first extent % parts of them one plane
 * larger; ext_lo = max(0, own_lo - halo), ext_hi = min(extent, own_hi +
 * halo).  Part p's lower halo [ext_lo, own_lo) is owned by part p - 1 and
 * its upper halo [own_hi, ext_hi) by part p + 1.  AC_ERR_INVALID unless
 * 1 <= parts <= extent, halo >= 1 and every part owns >= halo planes (so
 * each halo comes from one neighbour).  out: parts entries. */
int ac_slab_plan(int64_t extent, int32_t parts, int32_t halo, ac_slab_part *out);

/* In-process slabs on the current device: `parts` contexts over extended
 * slabs that this call allocates (field and workspace each; freed by
 * ac_slab_destroy).  halo = 0 takes twice the default temporal-block depth
 * of the grid (3D: 4; 2D: 8, 10 for FP32 grids of at least 1024^2 cells,
 * 12 for FP32 and FP16-storage grids of at least 4096^2 cells; FP64: 2), so
 * that a block is two passes.  All work is ordered on
 * cuda_stream: with several parts each part steps on a stream of its own
 * (created here), forked from cuda_stream before every block of steps and
 * joined back after it, so the parts' launches may run concurrently; halo
 * exchanges, scatter and gather are device-to-device copies of contiguous
 * plane blocks on cuda_stream. */
typedef struct ac_slab ac_slab; /* opaque */
int ac_slab_create(const ac_grid_desc *desc, int32_t parts, int32_t halo, void *cuda_stream,
                   ac_slab **out);
/* Copy a whole field (desc's layout, device memory) into the parts, halos
 * included / the parts' owned planes back into a whole field.  Async. */
int ac_slab_scatter(ac_slab *slab, const void *phi_dev);
int ac_slab_gather(ac_slab *slab, void *phi_dev);
/* n steps: blocks of at most `halo` steps, each part stepped by ac_step,
 * halos refreshed between blocks.  Async on the stream. */
int ac_slab_step(ac_slab *slab, int64_t n);
/* Schedule of every part (as ac_set_schedule). */
int ac_slab_set_schedule(ac_slab *slab, int32_t variant, int32_t k);
/* Replay ac_slab_step through a CUDA graph: the whole sequence for n steps
 * (every part's launches and the halo copies) is captured on the first call
 * with that n (and halo state) and replayed afterwards.  Needs a
 * non-default stream (AC_ERR_UNSUPPORTED otherwise); enable = 0 drops it. */
int ac_slab_set_graph(ac_slab *slab, int32_t enable);
/* Plan entry, halo depth and field of one part (its layout: desc with the
 * slow axis extent ext_hi - ext_lo). */
int ac_slab_get_part(ac_slab *slab, int32_t part, ac_slab_part *plan, int32_t *halo, void **phi_dev);
/* Kernels and halo copies issued so far (all parts). */
int ac_slab_launch_count(ac_slab *slab, int64_t *kernels, int64_t *copies);
int ac_slab_destroy(ac_slab *slab);

/* Allocation-free variant of ac_observe, for callers that cannot allocate
 * device or host memory at the point of the call: code running under a
 * memory budget owned by someone else (a framework's caching allocator, a
 * serving process with a fixed pool), and latency-critical loops where the
 * device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.
 * It needs no context (ac_create allocates) and calls no cudaMalloc,
 * cudaFree or allocating routine: the per-block partial sums go to a fixed
 * 512 KiB array compiled into the library, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart; it
 * computes the same observables as ac_observe.
 *
 *   desc     the grid descriptor (validated as for ac_create).
 *   phi_dev  the field in device memory (16-byte aligned), laid out as desc says.
 *   cuda_stream  the cudaStream_t to run on (NULL = legacy default stream).
 *   out_dev  caller-owned device memory for 3 doubles (8-byte aligned):
 *            out_dev[0] = E_h, out_dev[1] = V, out_dev[2] = non-finite count.
 *
 * Asynchronous: nothing is copied to the host and the stream is not
 * synchronised.  Grids with ny * nz above 1048576 rows (the fixed scratch
 * holds 16384 blocks of 64 rows) are rejected with AC_ERR_INVALID and a
 * message naming the limit.  The first call on each device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture on the device.  All calls on a device share the
 * array: calls whose kernels overlap on the GPU (for example, issued on two
 * streams without ordering between them) race and give wrong sums.  Each
 * call writes every partial it reads, so no state carries over between calls. */
int ac_observe_noalloc(const ac_grid_desc *desc, const void *phi_dev, void *cuda_stream,
                       double *out_dev);

/* Release the context's internal buffers.  Does not touch phi/workspace.
 * Synchronises the stream first.  NULL is accepted. */
int ac_destroy(ac_ctx *ctx);

/* Message for the last failure on this thread ("" if none). */
const char *ac_last_error(void);

/* Library version string, e.g. "1.0.0 sm_103a". */
const char *ac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AC_H_ */
