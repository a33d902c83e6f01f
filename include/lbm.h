/*
 * lbm.h - C ABI of the GB300 D3Q19-MRT lattice Boltzmann permeability solver.
 *
 * Method: Rao & Schaefer, "Lattice Boltzmann Models for Micro-tomographic
 * Pore-spaces" (arXiv:1902.11193).  Stokes flow through a binary voxel image
 * is time-stepped with the D3Q19 MRT lattice Boltzmann equation with Guo
 * forcing (eqs. MRT Collision, LBE-MRT, MRT-LBE, Guo_Forcing; Sec. 2.2.1),
 * equilibrium moments of eq. (MRT Equi), relaxation rates of Table 2 (Sets
 * A-E as functions of tau and the magic parameter Lambda, eq. Magic param),
 * a uniform body force with periodic boundaries (Sec. 2.4), bounceback on the
 * solid mask applied at the half-link, and the permeability of eq. (perm_calc)
 * from the mean velocity, with the stopping rule of eq. (convergence).
 *
 * Conventions shared by every call:
 *  - The voxel image ("mask") is uint8 [Lz][Ly][Lx], x fastest, 1 = solid,
 *    0 = fluid.  dims = {Lx, Ly, Lz}.  Node index n = x + Lx*(y + Ly*z).
 *  - D3Q19 velocity order: i = 0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 *    7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
 *    (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
 *  - Populations exchanged through this ABI are unshifted f_i in FP64,
 *    laid out [19][N], holding the post-collision state after the last step
 *    (solid nodes hold the rest value w_i).  Internally they are stored as
 *    shifted deviations f_i - w_i (rho0 = 1).
 *  - Velocities are u = (sum_i c_i f_i + F/2) / rho0 of the streamed state
 *    (the shifted velocity of Sec. 2.2.1), 0 at solid voxels.  Mean values are
 *    over all N voxels (superficial velocity).
 *  - Every pointer argument is a HOST pointer unless the name says _dev.
 *    The caller owns all buffers it passes; the context owns its device memory.
 *  - Return value 0 = success, a negative LBM_E* code on failure; a failed
 *    call leaves the context usable unless it returned LBM_ECUDA.
 *  - One context is used by one host thread at a time.  All device work runs
 *    on the context's CUDA stream; calls that return host data synchronise it.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,      /* bad argument: tau <= 1/2, rate outside (0,2), dims, mask */
    LBM_ENOMEM = -2,      /* device or host allocation failed */
    LBM_ECUDA = -3,       /* CUDA runtime error (see lbm_last_cuda_error) */
    LBM_ENOTCONV = -4,    /* max_steps reached before the stopping rule held */
    LBM_EUNSTABLE = -5,   /* non-finite density or velocity detected */
    LBM_ETIMEOUT = -6,    /* a bounded device wait expired */
    LBM_ENOSTATE = -7,    /* operation needs a state the context does not have */
    LBM_EIO = -8          /* checkpoint file could not be read or written */
};

/* Relaxation-rate sets of Table 2; SRT sets every rate to 1/tau. */
typedef enum { LBM_SET_A = 0, LBM_SET_B, LBM_SET_C, LBM_SET_D, LBM_SET_E, LBM_SET_SRT } lbm_set;

/* Storage precision of the populations.  FP64 stores and computes in double;
 * FP32_SHIFTED stores f_i - w_i in float and computes in float;
 * FP16_SHIFTED stores 2^S (f_i - w_i) in half and computes in float.  Mean
 * velocities and residuals are accumulated in double across warps.  Within a
 * warp, float values are added in float with the exact rounding error of
 * every addition carried along (a compensated sum, off by at most about
 * 2^-43 of the sum of magnitudes); double values are added in double.  The
 * order is fixed, so results are reproducible. */
typedef enum { LBM_FP64 = 0, LBM_FP32_SHIFTED = 1, LBM_FP16_SHIFTED = 2 } lbm_precision;

/* AB: two population arrays, pull stream.  AA: one array, in-place AA
 * pattern (even steps read and write a node's own slots swapped, odd steps
 * read and write neighbour slots).  SPARSE: AA pattern over the list of fluid
 * nodes with a neighbour table; solid voxels take no storage. */
typedef enum { LBM_LAYOUT_AB = 0, LBM_LAYOUT_AA = 1, LBM_LAYOUT_SPARSE = 2 } lbm_layout;

typedef struct {
    int32_t precision;        /* lbm_precision, default LBM_FP32_SHIFTED */
    int32_t layout;           /* lbm_layout, default LBM_LAYOUT_AA */
    int32_t check_interval;   /* K: stopping rule evaluated every K steps, default 100 */
    int32_t linear_eq;        /* 1: drop the quadratic equilibrium and forcing terms
                                 (Stokes simplification, Sec. 2.2.1); default 0 */
    int64_t max_steps;        /* lbm_run_to_convergence limit, default 1000000 */
    void *cuda_stream;        /* cudaStream_t to run on; NULL: the context makes one */
    int32_t fp16_scale_log2;  /* S for FP16 storage; 0 selects it from the drive */
    int32_t block_size;       /* threads per block of the stream-collide kernel;
                                 0 = default (256) */
    int32_t stop_rule;        /* 0 (default): eq. (convergence) on the per-step value;
                                 1: on the mean over two consecutive steps, measured
                                 in the last three steps of a chunk (K >= 3).  Halfway
                                 bounceback in gaps one or two voxels wide supports
                                 modes of eigenvalue near -1 that keep the per-step
                                 value alternating around the fixed point; the
                                 two-step mean cancels them. */
    int32_t bounceback;       /* 0 (default): halfway bounceback, the wall at the
                                 half-link, applied in the pull of each fluid node.
                                 1: full-way bounceback (Sec. 3): solid voxels with a
                                 fluid link neighbour (flag 1 of the image analysis)
                                 hold the populations streamed into them and return
                                 each along the opposite link in the next step,
                                 without collision or force.  Same steady state as
                                 halfway bounceback, one step more per reflection.
                                 LBM_LAYOUT_AB only (LBM_EINVAL otherwise); its
                                 bounceback voxels are internal state: velocity 0,
                                 rest populations in lbm_get_populations, untouched
                                 by lbm_set_populations; no adjoint (LBM_ENOSTATE). */
    int32_t pressure_x;       /* 1: the x faces are density boundaries (Zou-He, Sec. 2.4):
                                 inlet x = 0 at rho_in, outlet x = Lx-1 at rho_out;
                                 needs force = 0 and Lx >= 2.  k along x then takes
                                 the pressure gradient c_s^2 (rho_in - rho_out)/(Lx - 1)
                                 in place of F_x (eq. perm_calc with grad p); k_y, k_z
                                 are NaN.  0 (default): periodic in x. */
    int32_t symmetry;         /* bit 0: the y faces, bit 1: the z faces are symmetry
                                 (mirror) planes half a link outside the outer nodes
                                 (Sec. 2.4); unset bits stay periodic.  Default 0.
                                 pressure_x and symmetry need LBM_LAYOUT_AB and
                                 halfway bounceback; link counts stay those of the
                                 periodic image; no adjoint (LBM_ENOSTATE). */
    double rho_in, rho_out;   /* prescribed densities (rho0 = 1), default 1 */
    int32_t collision;        /* 0 (default): the link-basis TRT form where the rates
                                 have one even and one odd value (Sets B, E, SRT;
                                 the same collision as the MRT, fewer operations),
                                 the moment-space MRT otherwise.  1: always MRT. */
    int32_t index_width;      /* 0 (default) or 32: flat population offsets in 32 bits
                                 whenever 19 * (stored units) < 2^32, in 64 bits
                                 beyond; 64: always in 64 bits (the path of very
                                 large lattices, selectable on small ones for
                                 testing).  The results are bitwise the same. */
} lbm_options;

typedef struct lbm_ctx lbm_ctx;

/* Fills *opt with the defaults listed above. */
void lbm_default_options(lbm_options *opt);

/* Relaxation rates s[19] (diagonal of S, eq. MRT params) of Table 2 for
 * (set, tau, Lambda).  Lambda is used by Set E only.  Returns LBM_EINVAL for
 * tau <= 1/2, Lambda <= 0 with Set E, or an unknown set. */
int lbm_rates(int32_t set, double tau, double Lambda, double s[19]);

/* Creates a solver for the voxel image `mask` (host, Lz*Ly*Lx bytes, copied;
 * the caller keeps ownership).  force = body force density F = rho0 a
 * (Sec. 2.4), applied at every fluid node.  opt may be NULL (defaults).
 * The state starts at rest (f_i = w_i).  On success *out owns all device
 * memory until lbm_destroy.  Errors: LBM_EINVAL (dims <= 0, N >= 2^31, mask
 * entries other than 0/1, bad rates), LBM_ENOMEM, LBM_ECUDA. */
int lbm_create(lbm_ctx **out, const uint8_t *mask, const int32_t dims[3], int32_t set,
               double tau, double Lambda, const double force[3], const lbm_options *opt);

/* Like lbm_create, with the 19 relaxation rates given directly (s[0], s[3],
 * s[5], s[7] must be 0; the others in (0, 2); s[9] = 1/tau sets the
 * viscosity nu = (1/s[9] - 1/2)/3). */
int lbm_create_rates(lbm_ctx **out, const uint8_t *mask, const int32_t dims[3],
                     const double s[19], const double force[3], const lbm_options *opt);

void lbm_destroy(lbm_ctx *ctx);

/* Advances n >= 0 time steps (eq. LBE with the MRT collision, pull stream,
 * halfway bounceback).  Asynchronous on the context stream. */
int lbm_step(lbm_ctx *ctx, int64_t n);

/* Steps in chunks of check_interval until the stopping rule of eq.
 * (convergence) holds: |U_b - U_a| <= tol |U_b| for the mean velocity along the
 * drive (the largest |F_j|) measured in the last two steps of a chunk.
 * *steps_taken (nullable) receives the steps run by this call.  Returns 0,
 * LBM_ENOTCONV after max_steps (state kept), LBM_EUNSTABLE on non-finite
 * values.  Each chunk shape is captured once as a CUDA graph on the context
 * stream and replayed (the context keeps up to four); where the stream is
 * already being captured by the caller, chunks are launched directly.  Either
 * way the results and the kernel-launch count are those of direct launches. */
int lbm_run_to_convergence(lbm_ctx *ctx, double tol, int64_t *steps_taken);

/* One evaluation of the stopping rule: the step count after the chunk, the
 * measured mean velocity along the drive (U_b; under stop_rule 1 the mean of
 * the chunk's last two steps) and the relative change |U_b - U_a| / |U_b|
 * the rule compares with tol (NaN where no earlier value exists). */
typedef struct {
    int64_t step;
    double U;
    double change;
} lbm_check;

/* The checks of the last lbm_run_to_convergence, in order: copies up to cap
 * records to out (nullable) and the total number to *count.  The record of a
 * run: how the convergence measure of eq. (convergence) evolved. */
int lbm_convergence_history(lbm_ctx *ctx, lbm_check *out, int64_t cap, int64_t *count);

/* Mean velocity U[3] of the current state after streaming (not advanced). */
int lbm_mean_velocity(lbm_ctx *ctx, double U[3]);

/* The mean velocity the last lbm_run_to_convergence stopped on (the last
 * measured step under stop_rule 0, the two-step mean under stop_rule 1) and
 * the permeability from it (eq. perm_calc).  LBM_ENOSTATE before a run. */
int lbm_converged_velocity(lbm_ctx *ctx, double U[3]);
int lbm_converged_permeability(lbm_ctx *ctx, double k[3]);

/* eq. (perm_calc) with body forcing: k_j = nu <u_j> / F_j, nu = (tau-1/2)/3,
 * NaN where F_j == 0 (lattice units). */
int lbm_permeability(lbm_ctx *ctx, double k[3]);

/* Velocity field u[3][N] (host, caller buffer) of the streamed state. */
int lbm_velocity(lbm_ctx *ctx, double *u);

/* Post-collision populations f[19][N] (host, unshifted FP64) of the current
 * state, and the inverse.  Sizes are 19*N doubles. */
int lbm_get_populations(lbm_ctx *ctx, double *f);
int lbm_set_populations(lbm_ctx *ctx, const double *f);

/* Post-collision populations at selected nodes: nodes[count] are node
 * indices n = x + Lx*(y + Ly*z) (host); f[count][19] (host) receives the
 * unshifted FP64 values of each node (w_i at solid nodes).  Sized for
 * sampled checks of lattices too large to copy whole.  LBM_EINVAL for an
 * index outside [0, N). */
int lbm_get_populations_at(lbm_ctx *ctx, const int64_t *nodes, int64_t count, double *f);

/* Largest lattice (nodes) lbm_mean_velocity_noalloc accepts: 2^24, e.g. 256^3. */
#define LBM_NOALLOC_MAX_NODES 16777216

/* Mean velocity of a caller-held population array, without allocating any
 * device memory.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc where they need the measurement (device memory
 * owned by another allocator that must not be bypassed, or a loop that must
 * not take cudaMalloc's implicit device synchronisation).
 *   f_dev    device, FP64 [19][N]: post-collision populations of the last
 *            step minus w_i (two-array layout: population i of node n at
 *            i*N + n), as the FP64 AB layout keeps them
 *   mask_dev device, uint8 [N], 1 = solid
 *   U_dev    device, double[3]: receives the streamed-state mean velocity
 *            (as lbm_mean_velocity: halfway bounceback, F/2 shift, over all N)
 * The lattice is taken as periodic with halfway bounceback at every nonzero
 * mask byte: the result equals lbm_mean_velocity only for contexts built
 * with those boundaries (not with full-way bounceback, pressure faces or
 * symmetry planes).
 *   cuda_stream  stream to run on (NULL: the legacy default stream)
 * Asynchronous on the stream.  Its scratch is a file-scope device array that
 * every GPU loading the library keeps until exit (1.5 MiB); the first call
 * on a device looks up the array's address (cudaGetSymbolAddress) with that
 * device current, so make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU race.  LBM_EINVAL for
 * a NULL pointer, dims <= 0, or more than LBM_NOALLOC_MAX_NODES nodes (each
 * edge is checked before the node count is formed). */
int lbm_mean_velocity_noalloc(const double *f_dev, const uint8_t *mask_dev, const int32_t dims[3],
                              const double force[3], double *U_dev, void *cuda_stream);

/* Fluid-node count and per-direction bounceback link counts (links[i] =
 * number of fluid nodes x whose upstream neighbour x - c_i is solid). */
int lbm_link_counts(lbm_ctx *ctx, int64_t *n_fluid, int64_t links[19]);

/* Sparse layout only: copies the fluid list fluid_idx[Nf] (node indices),
 * the pull-neighbour table nbr[18][Nf] (fluid index of x - c_i, -1 where
 * solid; direction i at row i-1) and the bounceback bits bbmask[Nf] (bit i
 * set iff x - c_i is solid).  Any pointer may be NULL. */
int lbm_sparse_tables(lbm_ctx *ctx, int32_t *fluid_idx, int32_t *nbr, uint32_t *bbmask);

/* Reads and clears the context's device flags (synchronises its stream):
 * bit 0 (1): a measuring launch met a non-finite density or momentum (the
 * convergence loop reports it as LBM_EUNSTABLE); bit 1 (2): in a library
 * built with -DLBM_BOUNDS_CHECK, a kernel formed an index outside the array
 * it was about to access and skipped that access (never set otherwise).
 * The checked build is a debugging aid for the streaming of eq. (LBE)
 * over a voxel image (Sec. 2.1): every computed offset into the population,
 * index-record, row-word and row-start arrays is range-checked first. */
int lbm_device_flags(lbm_ctx *ctx, int32_t *flags);

/* Number of time steps taken since creation (or since the loaded checkpoint). */
int64_t lbm_steps_done(const lbm_ctx *ctx);

/* Checkpoint: writes dims, mask, rates, force, options, step count and the
 * stored populations to a file; lbm_load recreates an identical context
 * (same stream if opt is NULL: a fresh one).  Resuming continues bit-identically. */
int lbm_save(lbm_ctx *ctx, const char *path);
int lbm_load(lbm_ctx **out, const char *path, const lbm_options *opt);

/* Gradient of the converged permeability k along the drive direction d (the
 * largest |F_j|), from lbm_adjoint. */
typedef struct {
    double dk_dtau;      /* total derivative in tau under the set's rate rules
                            (rates given directly: through s_nu = 1/tau only) */
    double dk_dLambda;   /* Sets B, D, E: both odd rates through their magic
                            parameters moved together (eq. Magic param); NaN otherwise */
    double dk_dLambda_q; /* Sets B, D, E: through s_q alone; NaN otherwise */
    double dk_dLambda_m; /* Sets B, D, E: through s_m alone; NaN otherwise */
    double dk_dF[3];     /* with respect to the body-force components */
    double dk_ds[6];     /* partial derivatives with respect to the grouped rates
                            (s_e, s_eps, s_q, s_nu, s_pi, s_m), tau fixed in nu */
    double k;            /* k_d at the state the adjoint was taken */
    int64_t iterations;  /* adjoint iterations run */
    double residual;     /* final ||psi_{n+1} - psi_n|| / ||psi_{n+1}|| */
} lbm_grad;

/* Steady fixed-point adjoint of k_d (no counterpart in the paper: the
 * derivative of eq. (perm_calc) at a converged state).  Solves
 * psi = J_C^T S^T psi + dk/dh in the context's precision (FP64 for FP64
 * storage, FP32 otherwise) with the residual checked every check_interval
 * iterations until <= tol or max_iter, then reduces the gradient (per-node
 * terms in that precision, sums as for the mean velocity).  The iterations
 * between two checks are replayed from a CUDA graph on the context stream.
 * The state must be the converged one: LBM_ENOSTATE unless the last
 * lbm_run_to_convergence succeeded and nothing stepped or set the state
 * since.  The linearisation point is the mean of the streamed states of the
 * current and the next step (the context advances one step), the residual
 * compares iterates two apart and the gradient uses the mean of the last two
 * iterates, so a period-2 component of either iteration drops out.
 * LBM_EINVAL if every force component is zero.  Allocates four
 * population-sized work arrays for the duration of the call. */
int lbm_adjoint(lbm_ctx *ctx, double tol, int64_t max_iter, lbm_grad *out);

/* Transient adjoint: the gradient of k_d after n more steps (the value
 * lbm_permeability returns once the context has taken them), by reverse
 * accumulation through the n steps (no counterpart in the paper; the
 * transient k(n) is what its convergence rule watches).  The context
 * advances n steps.  The forward states are recomputed from checkpoints of
 * the population array taken every ceil(sqrt(n)) steps, so the call holds
 * about 2 sqrt(n) population-sized arrays; LBM_ENOMEM if they do not fit.
 * Arithmetic as lbm_adjoint; iterations = n, residual = NaN.  Halfway
 * bounceback on a periodic domain (LBM_ENOSTATE otherwise); LBM_EINVAL for
 * n < 1 or a zero force. */
int lbm_adjoint_transient(lbm_ctx *ctx, int64_t n, lbm_grad *out);

/* ------------------------------------------------------------------------
 * Batched sweep: many lattices of uneven sizes stepped together, as in the
 * paper's parameter study (Sets A-E x tau x geometry x resolution, Secs.
 * 4.1-4.3).  One persistent cooperative kernel per chunk of check_interval
 * steps walks a tile table of every active lattice, with a bounded-wait grid
 * barrier between steps; each lattice measures its mean velocity in the
 * chunk's last two steps and retires when its own stopping rule holds.  The
 * chunk (kernel, per-lattice reductions, result copy) is replayed from a
 * CUDA graph.  Each lattice's layout (dense AA or sparse) and nodes per
 * thread are chosen by timing candidates per distinct image (autotuner), or
 * fixed by the options. */

typedef struct {
    const uint8_t *mask;  /* host, Lz*Ly*Lx, 1 = solid (copied at create) */
    int32_t dims[3];
    int32_t set;          /* lbm_set; -1: rates from s[] */
    double tau, Lambda;
    double s[19];         /* used when set == -1 */
    double force[3];
} lbm_lattice_desc;

typedef struct {
    int32_t precision;          /* LBM_FP32_SHIFTED (default) or LBM_FP64 */
    int32_t layout;             /* -1 (default): autotune; LBM_LAYOUT_AA or LBM_LAYOUT_SPARSE */
    int32_t nodes_per_thread;   /* 0 (default): autotune; 1 or 2 */
    int32_t check_interval;     /* K >= 2, default 100 */
    int32_t linear_eq;
    int64_t max_steps;          /* per lattice, default 1000000 */
    void *cuda_stream;          /* NULL: the batch makes one */
    int32_t use_graph;          /* 1 (default): replay chunks from a CUDA graph */
    int32_t barrier_timeout_ms; /* bounded grid-barrier wait, default 2000 */
    int32_t test_skip_block;    /* test hook, default -1: block that skips its first barrier
                                   arrival, so the others' waits run out (LBM_ETIMEOUT) */
    int32_t stop_rule;          /* as lbm_options.stop_rule */
    int32_t solo;               /* lattices whose layout and nodes per thread are
                                   autotuned, and that fill the GPU by themselves (at
                                   least four waves of the batched kernel's threads),
                                   may run alone with the single-lattice kernels where
                                   the autotuner times that faster than the batched
                                   kernel: 1 (default) let it choose, 0 never, 2 always
                                   (every autotuned lattice runs alone, whatever its
                                   size).  The stepwise schedule needs no lone runs, so
                                   with it the default offers none. */
    int32_t schedule;           /* 0 (default): per chunk, each lattice of at least 10^5
                                   units (fluid nodes or voxels) runs the chunk with its
                                   own single-lattice kernels, replayed from its own CUDA
                                   graph, and all others share one persistent launch;
                                   1: every lattice in the persistent kernel; 2: grouped
                                   stepwise (FP32 only): per step, one launch per class
                                   of lattices (layout x collision form x parity) of the
                                   multi-lattice twins of the single-lattice kernels,
                                   lattices packed into groups that fit L2, each group
                                   run through the whole chunk in turn; lattices of at
                                   least 10^5 units on their own kernels.  Results are
                                   bitwise the same under every schedule. */
} lbm_batch_options;

typedef struct lbm_batch lbm_batch;

void lbm_batch_default_options(lbm_batch_options *opt);
/* Creates n lattices (each validated like lbm_create).  Errors as lbm_create. */
int lbm_batch_create(lbm_batch **out, int32_t n, const lbm_lattice_desc *lattices,
                     const lbm_batch_options *opt);
/* Runs every lattice until its stopping rule (as lbm_run_to_convergence, with
 * the batch's check_interval) holds or it reaches max_steps.  steps[n] and
 * status[n] (nullable) receive each lattice's step count and result
 * (0, LBM_ENOTCONV or LBM_EUNSTABLE).  Returns LBM_ETIMEOUT if a grid-barrier
 * wait expired (the batch is then unusable), else 0. */
int lbm_batch_run(lbm_batch *b, double tol, int64_t *steps, int32_t *status);
/* Per-lattice results: k[n][3] (eq. perm_calc) from the mean velocity each
 * lattice's stopping rule stopped on (the current state's before a run), and
 * the current states' mean velocities U[n][3]. */
int lbm_batch_permeability(lbm_batch *b, double *k);
int lbm_batch_mean_velocity(lbm_batch *b, double *U);
/* Layout and nodes per thread chosen for each lattice (nullable outputs);
 * nodes_per_thread 0 marks a lattice that runs alone (see solo) or, under the
 * automatic and grouped stepwise schedules, one of at least 1e5 units that
 * runs its chunks on its own single-lattice kernels. */
int lbm_batch_config(lbm_batch *b, int32_t *layout, int32_t *nodes_per_thread);
/* The context of lattice i (owned by the batch; valid until lbm_batch_destroy),
 * for the single-lattice readers (populations, velocity, checkpoint). */
lbm_ctx *lbm_batch_lattice(lbm_batch *b, int32_t i);
/* Kernel launches and graph replays so far (launch accounting). */
int64_t lbm_batch_kernel_launches(const lbm_batch *b);
/* Chunks so far that ran lattices with their own kernels or grouped stepwise
 * launches (stepwise), and chunks with a persistent launch (nullable). */
int lbm_batch_schedule_counts(const lbm_batch *b, int64_t *stepwise, int64_t *persistent);
void lbm_batch_destroy(lbm_batch *b);

/* Number of CUDA kernels this context has launched (for launch accounting). */
int64_t lbm_kernel_launches(const lbm_ctx *ctx);

const char *lbm_strerror(int code);
/* Text of the last CUDA runtime error seen by this library (thread-local). */
const char *lbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
