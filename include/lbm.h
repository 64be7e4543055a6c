/*
 * C ABI of the B300-native coupled lattice Boltzmann + conservative Allen–Cahn solver
 * (arXiv 2501.00846, "Thread-safe multiphase lattice Boltzmann model for droplet and bubble
 * dynamics at high density and viscosity contrasts").
 *
 * One context owns one box of nx*ny*nz nodes on the current CUDA device.  Every entry point
 * takes plain pointers and sizes; no C++ or PyTorch type crosses this boundary.  All device
 * work is enqueued on the context's stream (lbm_params.stream; NULL is the legacy default
 * stream, as everywhere in CUDA).
 *
 * Lattice: D3Q27, cs^2 = 1/3, dx = dt = 1.  Velocity index i = 9 (cz+1) + 3 (cy+1) + (cx+1)
 * for c_i = (cx, cy, cz) in {-1,0,1}^3; the opposite of i is 26 - i; the rest velocity is 13.
 *
 * Array layouts (all FP32, structure of arrays, x fastest):
 *   scalar field   s[(z*ny + y)*nx + x]                     N = nx*ny*nz floats
 *   vector field   v[a*N + (z*ny + y)*nx + x], a = 0,1,2   3N floats
 *   populations    g[i*N + (z*ny + y)*nx + x], i = 0..26   27N floats
 *
 * Phase convention: phi = 1 is the heavy (liquid) phase of density rho_l, phi = 0 the light
 * (gas) phase of density rho_g; rho = rho_l phi + (1 - phi) rho_g (paper Section "Model
 * extension for high-density and viscosity contrasts").
 *
 * State after step n: (g^n, phi^n, ubar^n).  g^n_i(x) is the post-collision population at its
 * origin node, phi^n the phase field that collision used, ubar^n the velocity it produced.
 * p* = sum_i g_i and p = p* rho cs^2 (Eq. eqts and the relation that follows Eq. press_corr).
 *
 * Errors: every function returns LBM_OK or a negative lbm_status; lbm_last_error() gives a
 * one-line message for the calling thread's last failure.  On error no output is written
 * except where stated.  Functions never abort the process and never trap the GPU.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,        /* invalid argument or parameter set */
    LBM_ERR_OOM = -2,        /* device allocation failed; nothing leaked */
    LBM_ERR_CUDA = -3,       /* a CUDA call failed; see lbm_last_error() */
    LBM_ERR_NONFINITE = -4,  /* the state holds NaN/Inf (observables still filled) */
    LBM_ERR_TIMEOUT = -5,    /* a bounded device wait expired */
    LBM_ERR_STATE = -6       /* call out of order (e.g. lbm_step before lbm_init_fields) */
} lbm_status;

typedef enum {
    LBM_FP32 = 0,            /* populations stored as FP32 */
    LBM_BF16 = 1,            /* populations stored as BF16 deviations (see below) */
    LBM_FP16 = 2,            /* populations stored as FP16 deviations (see below) */
    LBM_MOM = 3,             /* moment-only storage: 13 FP32 moments per node (see below) */
    LBM_MOM_BF16 = 4,        /* moment-only storage, the 9 deviation moments in BF16 (see below) */
    LBM_MOM_FP16 = 5         /* moment-only storage, the 9 deviation moments in FP16 (see below) */
} lbm_storage;

/*
 * Moment-only storage (LBM_MOM).  The paper's collision forms every post-collision population
 * from macroscopic fields alone (Section "Thread-safe lattice Boltzmann": Eq. LBexp with
 * Eqs. eqts and noneqts and the forcing), so the populations leaving a node are a fixed
 * polynomial in c_i of its p*, u, a = F / rho and B = 4.5 (1 - omega) A (A: the regularised
 * second-order non-equilibrium moment).  This storage keeps those 13 FP32 numbers per node
 * (u in the velocity arrays, the other 10 as m[q N + node], q = 0 p*, 1..3 a, 4..9 B xx yy zz
 * xy xz yz) and rebuilds g_i(x - c_i) from the moments of x - c_i when it streams: 104 bytes
 * per node and step move instead of 248, for more arithmetic.  Path 0 runs a tiled kernel
 * (populations staged in shared memory), path 1 a one-thread-per-node kernel that rebuilds
 * every population from global memory (the cross-check; the two agree to FP32 rounding); path 2
 * is rejected.  lbm_get_state expands the moments to FP32 g; lbm_set_state projects g onto the
 * moments (p* = sum g, a = 2 (sum g c - u), B from sum g c c), which is exact up to rounding
 * for any state this library produced and the Hermite projection of any other.
 *
 * LBM_MOM_BF16 / LBM_MOM_FP16 keep p* and u in FP32 and store the 9 moments a and B, which vanish
 * at equilibrium (deviations by construction), in BF16 or in FP16 as 2^12 times the value, packed
 * per node in five 32-bit words (p*[N] FP32, then words[5 N]): 36 bytes of moments per node
 * instead of 52.  Arithmetic stays FP32, and sum_i g_i = p* holds for
 * any rounded a and B, so sum p* does not drift from the rounding.  lbm_set_state allocates a
 * temporary FP32 buffer of 10 N floats for the projection with these two storages.
 */

/*
 * 16-bit population storage (LBM_BF16, LBM_FP16).  The paper stores FP32 populations; this is a
 * bandwidth option of the library.  Per node it stores, instead of g_i, the deviation from the
 * equilibrium of the node's own p* and velocity u (Eq. eqts), per unit weight,
 *     h_i = (g_i - f^eq_i(p*, u)) / w_i       (27 x 16 bit; FP16 holds 2^12 h_i),
 * and P = p* - sum_i w_i h_i(rounded) in FP32; u is the velocity stored with the node anyway.
 * The populations that streaming rebuilds, w_i P + f^eq_i(0, u) + w_i h_i, then sum to the
 * collision's p* exactly (no drift of sum p* from rounding), and only the non-equilibrium part,
 * orders of magnitude below p* and u, is rounded to 16 bits.  Arithmetic stays FP32.
 * 148 bytes move per node and step instead of 248.  Paths 0 and 1 (lbm_set_path) run it;
 * lbm_get_state / lbm_set_state convert to and from FP32 g; lbm_read_fields and
 * lbm_observables report p* = P + sum_i w_i h_i.
 */

/*
 * Parameters, lattice units.  Plain old data; set struct_size = sizeof(lbm_params).
 * Validation in lbm_create (LBM_ERR_ARG on failure):
 *   nx, ny, nz >= 4, ny, nz <= 65535 and nx*ny*nz < 2^31;
 *   rho_l, rho_g, mu_l, mu_g, width > 0; sigma >= 0; 0 <= mobility < 9/26 (FTCS limit of the
 *   27-point Laplacian: mobility * 52/9 < 2); forces finite.
 */
typedef struct {
    size_t struct_size;
    int nx, ny, nz;
    int wall_z;           /* 0: periodic in z.  1: no-slip walls at z = -1/2 and z = nz - 1/2
                             (halfway bounce-back; phase field mirrored, neutral wetting) */
    double rho_l, rho_g;  /* densities of the phi = 1 and phi = 0 phases */
    double mu_l, mu_g;    /* dynamic viscosities; mu(phi) = mu_g + phi (mu_l - mu_g),
                             nu = mu / rho, tau = nu / cs^2 + 1/2 (the paper gives no
                             interpolation law; this linear law in phi is the one applied) */
    double sigma;         /* surface tension: beta = 12 sigma/width, kappa = 3 sigma width/2 */
    double width;         /* interface width delta (W) */
    double mobility;      /* Allen–Cahn diffusivity D; sharpening kappa_AC = 4 D / width */
    double gravity[3];    /* gravitational acceleration; buoyancy force (rho - rho_ref) g */
    double rho_ref;       /* reference density; rho_l applies gravity to the light phase only */
    double body[3];       /* uniform body-force density (e.g. a driven channel) */
    int storage;          /* lbm_storage */
    void *stream;         /* cudaStream_t to enqueue on; NULL: the legacy default stream */
} lbm_params;

/* Integral diagnostics, accumulated in FP64 on the device (all doubles). */
typedef struct {
    double step;              /* steps taken since lbm_init_fields / lbm_set_state */
    double sum_phi;           /* sum phi */
    double mass;              /* sum rho */
    double sum_pstar;         /* sum p* */
    double momentum[3];       /* sum rho ubar */
    double centroid_liq[3];   /* sum phi x / sum phi */
    double centroid_gas[3];   /* sum (1-phi) x / sum (1-phi) */
    double vel_liq[3];        /* sum phi ubar / sum phi */
    double vel_gas[3];        /* sum (1-phi) ubar / sum (1-phi) */
    double p_liq, p_gas;      /* mean p over nodes with phi > 0.999 / phi < 0.001 (NaN if none) */
    double n_liq, n_gas;      /* node counts of those two sets */
    double umax;              /* max |ubar| */
    double phi_min, phi_max;  /* extrema of phi (overshoot outside [0,1] is not clamped) */
    double n_nonfinite;       /* count of nodes with a non-finite phi, ubar or p* */
} lbm_obs;

/* Create a context: validates *params, allocates every device buffer (two copies of g, phi,
 * ubar: 2 x 31 floats per node with FP32 storage, 2 x (27 halves + 5 floats) with 16-bit
 * storage, 2 x 14 floats with moment storage, plus scratch).  The caller owns *out and releases it
 * with lbm_destroy.  On error *out = NULL and nothing is leaked. */
lbm_status lbm_create(const lbm_params *params, lbm_ctx **out);

/* Set the initial state (the paper's loop starts from equilibrium populations):
 *   g = f^eq(p*0, u0) (Eq. eqts), phi = phi0, ubar = u0, step counter = 0.
 * phi: N floats; u: 3N floats; pstar: N floats or NULL for p*0 = 0.
 * on_device = 0: host pointers (copied, then the stream is synchronised); 1: device pointers
 * on the context's device (copied on the context's stream).  The library never keeps the
 * caller's pointers. */
lbm_status lbm_init_fields(lbm_ctx *ctx, const float *phi, const float *u, const float *pstar,
                           int on_device);

/* Advance nsteps >= 0 time steps.  One step is the coupled update of the paper's step list
 * (Section "Implementation of the hybrid LB-finite difference implementation"): Allen–Cahn
 * FTCS update of phi, pull streaming (each node writes only itself), moments, surface-tension /
 * pressure / viscous / body forces, velocity, pre-regularisation and the third-order
 * regularised collision (Eqs. lbe to guoforce, press_corr, visc_corr).
 * Asynchronous on the context's stream; no host synchronisation.  LBM_ERR_STATE before
 * lbm_init_fields.  No NaN check (lbm_observables reports non-finite values). */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* FP64 reductions over the current state into *out (see lbm_obs).  Synchronises the stream.
 * Returns LBM_ERR_NONFINITE when out->n_nonfinite > 0; *out is filled in that case too. */
lbm_status lbm_observables(lbm_ctx *ctx, lbm_obs *out);

/* Diagnostics of a state the caller owns, without allocating any device memory.  The paper has
 * no counterpart: this is a library convenience.  It is for callers that cannot allocate device
 * memory: code embedded in an application that owns the whole device heap (a fixed arena handed
 * out at start-up, or a framework allocator that must account for every byte), and code that
 * must not call cudaMalloc because it would synchronise the device and stall queued work.
 *   g, phi, u   device pointers to populations (27N floats), phi (N) and ubar (3N) in the
 *               layouts above; nx, ny, nz the box; rho_l, rho_g the phase densities
 *   stream      cudaStream_t to run on (NULL: the legacy default stream).  Every call ends by
 *               copying its result to the host and synchronising this stream.
 *   out         filled as by lbm_observables, except out->step = 0
 * The reduction's scratch is a fixed array of 1185 x 32 doubles (303,360 bytes) inside the
 * library, held by every GPU that loads the library until the process exits.  Boxes of up to
 * 2^31 - 1 nodes fit; larger boxes return LBM_ERR_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture.  A process that resets
 * the device (cudaDeviceReset) afterwards must not call this entry point again: the kept
 * address belongs to the context that the reset destroyed.  All calls share the array and
 * nothing in it carries over between calls, but calls whose work overlaps on the GPU (e.g. on
 * two streams) race on it.
 * Returns LBM_ERR_NONFINITE when out->n_nonfinite > 0 (out filled), LBM_ERR_ARG for bad
 * arguments, LBM_ERR_CUDA if a CUDA call fails.  Calls no allocating routine. */
lbm_status lbm_observables_noalloc(const float *g, const float *phi, const float *u, int nx, int ny,
                                   int nz, double rho_l, double rho_g, void *stream, lbm_obs *out);

/* Copy out phi (N floats), ubar (3N floats) and p = p* rho cs^2 (N floats).  Any of the three
 * pointers may be NULL.  on_device as in lbm_init_fields.  Synchronises the stream. */
lbm_status lbm_read_fields(lbm_ctx *ctx, float *phi, float *u, float *p, int on_device);

/* Checkpoint / resume of the raw state: g (27N floats), phi (N), ubar (3N).  A state written
 * by lbm_get_state and restored by lbm_set_state continues bit-identically with FP32 storage.
 * With 16-bit storage g is exchanged as FP32 g_i = w_i (h_i + p*): lbm_get_state expands it and
 * lbm_set_state rounds it back (a round trip is not guaranteed to reproduce the stored h bit
 * for bit).  With moment storage g is the expansion of the moments, and lbm_set_state projects
 * it back (exact up to rounding for a state of this library).  lbm_set_state sets the step counter to `step`.  Both synchronise the stream. */
lbm_status lbm_get_state(lbm_ctx *ctx, float *g, float *phi, float *u, int on_device);
lbm_status lbm_set_state(lbm_ctx *ctx, const float *g, const float *phi, const float *u,
                         long long step, int on_device);

/* Block the host until the context's stream is idle. */
lbm_status lbm_synchronize(lbm_ctx *ctx);

/* Number of nodes N and steps taken; 0 for NULL. */
long long lbm_num_nodes(const lbm_ctx *ctx);
long long lbm_step_count(const lbm_ctx *ctx);

/* Select how a step is launched (all three compute the same step; they differ in data movement):
 *   0  two kernels (default, fastest): a z-marching Allen–Cahn kernel with separable stencils
 *      writes phi^{n+1}, then the one-thread-per-node lattice Boltzmann kernel
 *   1  three kernels: Allen–Cahn flux, Allen–Cahn update, lattice Boltzmann (plain 27-point
 *      stencils from global memory; the simplest form, kept as a cross-check)
 *   2  one fused kernel: the Allen–Cahn stencils of a z-marching shared-memory window and the
 *      lattice Boltzmann update of each plane in the same kernel
 * LBM_ERR_ARG for other values, and for path 2 with any storage but LBM_FP32. */
lbm_status lbm_set_path(lbm_ctx *ctx, int path);

/* Advection term of the Allen–Cahn update.  0 (default): flux form div(ubar phi), which conserves
 * sum phi to rounding (the reading the library applies everywhere; it equals ubar . grad(phi) when
 * div ubar = 0).  1: the paper's literal form ubar . G[phi] (Section "Model extension": the
 * advection term of the phase-field equation and its FTCS update), whose sum phi drifts by
 * -sum ubar . G[phi] per step; for studying that drift.  Form 1 runs on path 1 only: LBM_ERR_ARG
 * unless the path is 1, and lbm_set_path rejects paths 0 and 2 while form 1 is set. */
lbm_status lbm_set_advection(lbm_ctx *ctx, int form);

/* Work split of the z-marching kernels (paths 0 and 2): the number of z chunks each 32 x 8
 * column tile is cut into.  0 restores the library's default.
 * Results are bit-identical for every value:
 * the halo points each CTA recomputes use the same arithmetic as their owners.  LBM_ERR_ARG
 * for negative values. */
lbm_status lbm_set_split(lbm_ctx *ctx, int split);

/* Profiling aid: launch one kernel of the two-kernel step nrep times on the context's stream
 * without advancing the state (phase 0: the Allen–Cahn kernel, reading phi^n and ubar^n and
 * writing the idle phi buffer; phase 1: the lattice Boltzmann kernel, reading g^n, that phi buffer
 * and ubar^n and writing the idle g and ubar buffers).  The next lbm_step overwrites those idle
 * buffers.  Asynchronous.  LBM_ERR_STATE before lbm_init_fields. */
lbm_status lbm_run_phase(lbm_ctx *ctx, int phase, int nrep);

/* Free every resource of ctx; NULL-safe.  Waits for the context's stream first. */
void lbm_destroy(lbm_ctx *ctx);

/* Static description of a status code; never NULL. */
const char *lbm_status_string(lbm_status s);

/* Message of the calling thread's last failure ("" if none). */
const char *lbm_last_error(void);

/* ABI version of this header (incremented on incompatible changes). */
int lbm_abi_version(void);

/* ---------------------------------------------------------------------------------------------
 * Batched ensemble: many independent boxes advanced together.  The paper has no counterpart (it
 * runs one box); this is the library's batching of its step for ensembles of small boxes, which
 * one at a time cannot fill the GPU.  Every box has its own lbm_params (size, walls, densities,
 * viscosities, surface tension, mobility, forces; the storage, LBM_FP32 or one of the moment
 * storages, is the same for every box) and its own state; the boxes never interact.  A step
 * advances every box by one time step with two launches for the whole ensemble: the Allen–Cahn
 * kernel over the (column tile, z chunk) tasks of all boxes, then the lattice Boltzmann kernel
 * over the node blocks of all boxes (moment storage: over the (32 x 8 column tile, 32-plane
 * chunk) tasks of all boxes, each running the one-box tiled kernel's code).  Each box's arithmetic is
 * exactly that of lbm_step on a context with the same parameters (bit-identical results), for
 * every tuning.  Steps are replayed from a captured CUDA graph of graph_steps steps.
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_ens lbm_ens;

/* Launch configuration of the ensemble kernels (lbm_ens_autotune chooses one). */
typedef struct {
    int lbm_block;       /* threads per block of the lattice Boltzmann kernel: 64, 128 or 256
                            (FP32 populations; kept but unused with moment storage) */
    int ac_rows;         /* output rows per warp of the Allen–Cahn kernel: 2 or 4 */
    int ac_zlen;         /* planes per Allen–Cahn task (z-march depth), >= 1 */
    int graph_steps;     /* steps per captured CUDA graph: even and >= 2, or 0 for direct launches */
    double lbm_us;       /* output of lbm_ens_autotune: mean launch time of each kernel with the */
    double ac_us;        /* chosen configuration, microseconds (0 when not measured) */
} lbm_tuning;

/* Create an ensemble of nboxes >= 1 boxes; params[b] is validated as in lbm_create (its stream
 * field is ignored).  stream: the cudaStream_t every ensemble call enqueues on (NULL: the legacy
 * default stream).  Allocates the packed state of all boxes (two copies of g, phi, ubar and one
 * flux W: 272 B per node) plus scratch.  The caller owns *out (lbm_ens_destroy).  On error
 * *out = NULL and nothing is leaked: LBM_ERR_ARG (bad count or box parameters, message names the
 * box), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_ens_create(const lbm_params *params, int nboxes, void *stream, lbm_ens **out);
void lbm_ens_destroy(lbm_ens *ens);

/* Initial state of box b, as lbm_init_fields (phi: N_b floats, u: 3 N_b, pstar: N_b or NULL). */
lbm_status lbm_ens_init_fields(lbm_ens *ens, int box, const float *phi, const float *u, const float *pstar,
                               int on_device);

/* Advance every box by nsteps >= 0 steps (asynchronous on the ensemble's stream).  LBM_ERR_STATE
 * if any box has not been initialised. */
lbm_status lbm_ens_step(lbm_ens *ens, int nsteps);

/* Diagnostics and fields of box b, as lbm_observables / lbm_read_fields (synchronising). */
lbm_status lbm_ens_observables(lbm_ens *ens, int box, lbm_obs *out);
lbm_status lbm_ens_read_fields(lbm_ens *ens, int box, float *phi, float *u, float *p, int on_device);

/* Launch configuration: get, set (validated; LBM_ERR_ARG for values outside the documented
 * sets), and autotune: time each candidate (lbm_block in {64, 128, 256}; ac_rows in {2, 4} x
 * ac_zlen in {8, 16, 32, 64}) over reps >= 1 launches of each kernel on the current state,
 * without advancing it, keep the fastest, and report it in *out (may be NULL).  The state is
 * unchanged by autotuning. */
lbm_status lbm_ens_get_tuning(const lbm_ens *ens, lbm_tuning *out);
lbm_status lbm_ens_set_tuning(lbm_ens *ens, const lbm_tuning *t);
lbm_status lbm_ens_autotune(lbm_ens *ens, int reps, lbm_tuning *out);

/* Launch form of lbm_ens_step.  on = 0 (default): two launches per step, replayed from the CUDA
 * graph.  on = 1: one persistent cooperative launch per step (as many 256-thread CTAs as the GPU
 * holds at once): every warp takes Allen–Cahn tasks, the CTAs meet at a grid barrier, then take
 * the lattice Boltzmann work; results are bit-identical to the two-launch form.  Each wait at the
 * barrier is bounded (100 ms of the GPU's global timer); when one expires, that launch and every
 * later one of the same lbm_ens_step call do nothing further, and lbm_ens_step returns
 * LBM_ERR_TIMEOUT with the state of the last completed step (its step count, fields and flux), so
 * the ensemble stays usable.  In this form lbm_ens_step synchronises the stream before it returns.
 * Synchronises the stream.  LBM_ERR_ARG for other values of on. */
lbm_status lbm_ens_set_persistent(lbm_ens *ens, int on);

/* Test hook of the bounded barrier: with on = 1, CTA 0 of every persistent launch skips its arrival
 * at the grid barrier and the wait limit drops to 2 ms, so every wait expires and lbm_ens_step
 * returns LBM_ERR_TIMEOUT without advancing the state.  on = 0 restores normal operation
 * (100 ms).  Synchronises the stream. */
lbm_status lbm_ens_test_stall_barrier(lbm_ens *ens, int on);

/* Set the state of a coarse context (FP32 storage, half the box's size in every direction, same
 * parameters rescaled by the caller) to the 2x restriction of box b's state: the populations, phi
 * and ubar of each coarse cell are the means over its 8 fine nodes.  Enqueued on the coarse
 * context's stream after the ensemble's pending work.  The library's own addition (data for the
 * learned closure), not in the paper.  LBM_ERR_ARG for an ensemble that does not store FP32
 * populations. */
lbm_status lbm_ens_restrict_state(lbm_ens *ens, int box, lbm_ctx *coarse);

/* Number of boxes, total nodes, nodes of box b, steps taken; 0 for NULL or a bad index. */
int lbm_ens_num_boxes(const lbm_ens *ens);
long long lbm_ens_num_nodes(const lbm_ens *ens);
long long lbm_ens_box_nodes(const lbm_ens *ens, int box);
long long lbm_ens_step_count(const lbm_ens *ens);

/* ---------------------------------------------------------------------------------------------
 * Learned closure.  The paper has no learned component; this is the library's coarse-grid
 * correction.  A 4-layer network of periodic 3x3x3 convolutions (channels 5 -> 32 -> 32 -> 32 ->
 * 4, SiLU after the first three layers, biases on all four) maps the normalised state of a box,
 * x = ((phi, ubar_x, ubar_y, ubar_z, p) - in_shift) / in_scale, to a correction y; the correction
 * applied is dphi = out_scale[0] y_0 (minus its mean, so sum phi is unchanged) and
 * dubar_a = out_scale[a+1] y_{a+1}.  Convolutions run on the tensor cores (BF16 weights and
 * activations, FP32 accumulation); master weights, gradients and Adam moments are FP32.
 * Parameter order (lbm_cnn_get_params / set_params / get_grads): W1, b1, W2, b2, W3, b3, W4, b4
 * with W_l[o][i][k] (output channel, input channel, offset k = 9 (dz+1) + 3 (dy+1) + (dx+1)).
 * Grids: periodic, nx a multiple of 32, ny, nz >= 1.
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_cnn lbm_cnn;

typedef struct {
    float in_shift[5], in_scale[5];   /* input normalisation of (phi, ubar_x, ubar_y, ubar_z, p) */
    float out_scale[4];               /* correction scale of (phi, ubar_x, ubar_y, ubar_z) */
} lbm_closure_norm;

/* Network for nx x ny x nz grids; weights drawn from a seeded Glorot-uniform distribution, biases
 * zero, Adam moments zero.  stream: the cudaStream_t all calls enqueue on (NULL: legacy default).
 * LBM_ERR_ARG for nx % 32 != 0 or non-positive sizes. */
lbm_status lbm_cnn_create(int nx, int ny, int nz, unsigned long long seed, void *stream, lbm_cnn **out);
void lbm_cnn_destroy(lbm_cnn *cnn);
int lbm_cnn_num_params(void);
lbm_status lbm_cnn_get_params(lbm_cnn *cnn, float *params);        /* host, lbm_cnn_num_params() floats */
lbm_status lbm_cnn_set_params(lbm_cnn *cnn, const float *params);  /* host; resets nothing else */
lbm_status lbm_cnn_get_grads(lbm_cnn *cnn, float *grads);          /* host, the kept gradients */

/* Convolution kernel: 0 (default, the fastest measured) tcgen05.mma with TMEM accumulators
 * (shared-memory descriptors; each input plane read once for its three z offsets, N = 3 x the
 * output channels; the activation fused into its epilogue; launched with programmatic dependent
 * launch); 1 mma.sync from shared-memory tiles; 2 mma.sync with fragments straight from global
 * memory.  All three add the same BF16 products in the same FP32 order per output and give
 * identical results.  Training is deterministic: no reduction uses atomics.  lbm_cnn_forward and
 * lbm_cnn_grad return LBM_ERR_TIMEOUT if a tensor-core kernel gave up waiting for its MMAs.
 * LBM_ERR_ARG for other values. */
lbm_status lbm_cnn_set_conv_kernel(lbm_cnn *cnn, int kernel);

/* Test hook of the bounded waits.  Every mbarrier wait of the tensor-core convolution is bounded
 * in time (20 ms of the GPU's global timer; a plane's MMAs take about a microsecond).  With
 * on = 1, every tensor-core convolution (kernel 0) first waits, with a 20 us limit, on an
 * mbarrier that no MMA is committed to, so the wait expires
 * before the kernel issues any MMA; the kernel then records the expiry, waits for its own copies,
 * frees its TMEM and returns, and lbm_cnn_forward / lbm_cnn_grad return LBM_ERR_TIMEOUT (the
 * record is cleared once reported, so the network stays usable).  on = 0 restores normal
 * operation.  LBM_ERR_ARG for other values. */
lbm_status lbm_cnn_test_expire_wait(lbm_cnn *cnn, int on);

/* y = network(x): x [5][N] and y [4][N] FP32 channel-first device arrays (N = nx ny nz). */
lbm_status lbm_cnn_forward(lbm_cnn *cnn, const float *x, float *y);

/* Forward and backward pass for one sample with the mean-squared loss against t [4][N] (device):
 * loss (may be NULL) = mean over 4 N values of (y - t)^2; the gradients are kept (added to the
 * kept ones when accumulate != 0, else replacing them).  Synchronises the stream. */
lbm_status lbm_cnn_grad(lbm_cnn *cnn, const float *x, const float *t, int accumulate, double *loss);

/* Inspection of one layer l = 0..3 (host arrays, channel-first, any pointer may be NULL):
 *   a_in  the layer's input as the tensor cores read it, BF16 widened exactly to FP32 [CIN_l][N]
 *         (layer 0: the rounded network input x; layers 1..3: silu(z_{l-1}) rounded to BF16)
 *   z     the layer's FP32 pre-activation from the last lbm_cnn_grad [COUT_l][N] (layer 3: also
 *         from lbm_cnn_forward; a forward pass without gradients keeps only the output layer's)
 *   dz    d loss / d z_l in FP32 from the last lbm_cnn_grad [COUT_l][N]
 * with CIN = 5, 32, 32, 32 and COUT = 32, 32, 32, 4.  For testing the convolutions one at a time
 * against their definition; synchronises the stream.  LBM_ERR_ARG for a bad layer. */
lbm_status lbm_cnn_get_layer(lbm_cnn *cnn, int layer, float *a_in, float *z, float *dz);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) with the kept gradients
 * multiplied by grad_scale (e.g. 1 / samples accumulated). */
lbm_status lbm_cnn_adam_step(lbm_cnn *cnn, float lr, float grad_scale);

/* Network input of a context's current state (FP32 storage): x [5][N] device array. */
lbm_status lbm_closure_features(lbm_ctx *ctx, const lbm_closure_norm *norm, float *x);
/* Training target against a reference state: t = ((phi, u)_ref - (phi, ubar)_ctx) / out_scale,
 * ref: device [>= 4][N] channel-first (phi, u_x, u_y, u_z), t: device [4][N]. */
lbm_status lbm_closure_target(lbm_ctx *ctx, const float *ref, const lbm_closure_norm *norm, float *t);
/* Correct a context's state in place with the network (periodic boxes, FP32 storage, grid equal to
 * the network's): phi += dphi - w c with w = max(4 phi (1 - phi), 0) and c chosen so that sum phi
 * is unchanged (the compensation sits in the interfaces, the bulk phases stay untouched), ubar +=
 * du - sum(rho du) / sum(rho) with rho = rho(phi) before the correction (the correction adds no
 * momentum), populations shifted by f^eq(p*, ubar + du') - f^eq(p*, ubar) for that du'.
 * Asynchronous on the context's stream. */
lbm_status lbm_closure_apply(lbm_ctx *ctx, lbm_cnn *cnn, const lbm_closure_norm *norm);

/* Set the state of a fine context to the 2x prolongation of a coarse context's state: the
 * fallback of a corrected coarse run to the fine solver (the library's own addition for the
 * learned closure; the paper has no counterpart).  Both contexts: initialised, FP32 populations;
 * the fine box is twice the coarse box in every direction with the same walls (its parameters,
 * rescaled for the fine grid, are the caller's).  Cell-centred trilinear interpolation: fine node X
 * of coarse cell X / 2 takes 3/4 of that cell and 1/4 of the neighbour it lies towards along each
 * axis (periodic axes wrap; beyond a z wall the wall cell itself), applied to the 27 populations,
 * phi and ubar alike: the fine sums of phi, ubar and every population (so of p* and of the
 * populations' first moment) are 8 times the coarse ones.
 * Enqueued on the fine context's stream after the coarse context's pending work; the fine
 * context's step count is not changed.  LBM_ERR_ARG for mismatched boxes or storages,
 * LBM_ERR_STATE for an uninitialised context. */
lbm_status lbm_prolong2_state(lbm_ctx *coarse, lbm_ctx *fine);

/* 2x restriction of a fine state to the coarse grid (device arrays, channel-first): phi and p
 * averaged over the 8 fine nodes of a coarse cell, u averaged with weight rho(phi), and
 * p* = 3 p / rho(phi).  phi, p: N floats; u: 3N; out: 6 N/8 floats (phi, u_x, u_y, u_z, p, p*).
 * nx, ny, nz even.  rho_l, rho_g: the densities of the phases. */
lbm_status lbm_restrict2(const float *phi, const float *u, const float *p, int nx, int ny, int nz, double rho_l,
                         double rho_g, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
