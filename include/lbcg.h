/*
 * lbcg.h -- C ABI of the GB300 (sm_103a) library for the regularized
 * colour-gradient lattice Boltzmann method for two immiscible components
 * (Montessori, Lauricella, La Rocca, Succi, Stolovicki, Ziblat, Weitz,
 * arXiv:1711.02003).
 *
 * The library advances the populations f_i^k (k = red, blue) of Eq. 1 with the
 * fused per-site update:
 *   streaming (Eq. 1) with halfway bounce-back walls and ghost-site ports,
 *   densities rho^k and momentum (Eqs. 2-3), the phase field
 *   psi = (rho_R - rho_B)/rho and its isotropic gradient F (Sec. II, colour
 *   gradient), relaxation at the mixture relaxation time regularized by the
 *   second-order Hermite projection (Eqs. 5, 6, 11), the surface-tension
 *   perturbation with parameter A (Eq. 9) and recolouring with beta (Eq. 10).
 * The composition of Eq. 4 is applied as relax -> perturb -> recolour on the
 * total f = f^R + f^B; only recolouring separates the components.
 *
 * Conventions for every entry point:
 *   - Return LBCG_OK (0) on success or a negative LBCG_ERR_* code; nothing is
 *     thrown across the ABI.  lbcg_last_error() gives a message for the calling
 *     thread's last failure.
 *   - All GPU work is enqueued on the CUDA stream given to lbcg_create (NULL is
 *     the legacy default stream).  Calls taking HOST pointers copy synchronously
 *     and return after the copy; calls taking DEVICE pointers are asynchronous
 *     on that stream.
 *   - The two population buffers are owned by the caller (e.g. torch tensors)
 *     and bound with lbcg_bind_state.  The library allocates device tables
 *     (per-site link flags, port ghost lists, reduction partials) at
 *     lbcg_set_geometry, and a staging / read-back scratch on the first call that
 *     needs one (kept until lbcg_destroy).  Both state buffers hold a defined value
 *     at every site: initialisation writes both, steps write fluid sites and refill
 *     port ghosts, wall sites stay zero.
 *   - Per-site arrays are indexed site = x + nx*(y + ny*z), x fastest.
 *   - Population layout seen through lbcg_get_populations/lbcg_set_populations:
 *     FP64 [k][i][site], k = 0 red, 1 blue, directions 0-based with 0 = rest:
 *       D2Q9 : (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *       D3Q19: (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1)
 *              (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1)
 *              (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *     The stored state is post-collision (what Eq. 1 streams next).
 *   - A context is used by one host thread at a time.
 */
#ifndef LBCG_H
#define LBCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBCG_ABI_VERSION 2
#define LBCG_MAX_PORTS 8

enum lbcg_status {
    LBCG_OK = 0,
    LBCG_ERR_ARG = -1,       /* invalid argument: null pointer, size, parameter out of range */
    LBCG_ERR_STATE = -2,     /* call out of order: no state bound, no geometry, no fields */
    LBCG_ERR_CUDA = -3,      /* CUDA runtime failure (message in lbcg_last_error) */
    LBCG_ERR_NOMEM = -4,     /* a library-internal device allocation failed */
    LBCG_ERR_DIVERGED = -5,  /* non-finite or non-positive density found */
    LBCG_ERR_GEOMETRY = -6,  /* invalid mask / port table */
    LBCG_ERR_CAPACITY = -7,  /* caller buffer too small */
    LBCG_ERR_UNSUPPORTED = -8,
    LBCG_ERR_TIMEOUT = -9,     /* a bounded device-side wait or iteration ran out (state invalid) */
    LBCG_ERR_BOUNDS = -10      /* bounds-checked build: a step kernel met an index outside its array */
};

enum lbcg_lattice { LBCG_D2Q9 = 0, LBCG_D3Q19 = 1 };

/* Storage precision of the populations.  Arithmetic is FP64 for LBCG_FP64 and
 * FP32 for the others.
 *   LBCG_FP64        f^R_i, f^B_i in double
 *   LBCG_FP32        f^R_i, f^B_i in float
 *   LBCG_FP32_DEV    red f^R_i and total deviation g_i = f^R_i + f^B_i - w_i rho0 in float
 *   LBCG_FP16_SCALED red deviation and total deviation in binary16 with fixed scale factors */
enum lbcg_precision { LBCG_FP64 = 0, LBCG_FP32 = 1, LBCG_FP32_DEV = 2, LBCG_FP16_SCALED = 3 };

/* Eq. 11 regularized relaxation, or the plain BGK relaxation of Eq. 5 */
enum lbcg_collision { LBCG_REG = 0, LBCG_BGK = 1 };

/* Mask codes: fluid, wall (halfway bounce-back), or a ghost site of port m (code 2 + m). */
enum lbcg_mask { LBCG_MASK_FLUID = 0, LBCG_MASK_WALL = 1, LBCG_MASK_PORT0 = 2 };

/* Port kinds.  Ghost sites are refilled before each streaming step from their inward
 * neighbour x' = ghost + normal:
 *   VELOCITY       f^k = f^{k,eq}(chi^k rho(x'), u_port) + chi^k (f(x') - f^eq(x')),
 *                  chi^R = (1+psi)/2, chi^B = (1-psi)/2 of the port's colour psi;
 *   PRESSURE       f^k = f^{k,eq}(rho_port rho^k(x')/rho(x'), u(x')) + f^k(x') - f^{k,eq}(x');
 *   ZERO_GRADIENT  f^k = f^k(x').
 * The paper prints no boundary rule; these are the library's definitions. */
enum lbcg_port_kind { LBCG_PORT_VELOCITY = 0, LBCG_PORT_PRESSURE = 1, LBCG_PORT_ZERO_GRADIENT = 2 };
/* Velocity profile over the port's bounding box in the transverse axes; the walls sit
 * halfway beyond the first and last port sites: u = u_max * prod 4 s (W - s) / W^2. */
enum lbcg_profile { LBCG_PROFILE_PARABOLIC = 0, LBCG_PROFILE_FLAT = 1 };

typedef struct {
    int lattice;        /* lbcg_lattice */
    int nx, ny, nz;     /* box; nz is ignored (1) for D2Q9 */
    int periodic[3];    /* per axis; a closed axis acts as a wall outside the box */
    int collision;      /* lbcg_collision */
    int precision;      /* lbcg_precision */
    double tau_r, tau_b;     /* relaxation times of red and blue, > 1/2 (Eq. 5) */
    double alpha_r, alpha_b; /* Eq. 7 free parameters in (0,1); alpha = w_0 gives density ratio 1 */
    double A;           /* surface-tension parameter of Eq. 9, >= 0 */
    double beta;        /* recolouring parameter of Eq. 10, in [0,1] */
    double rho0;        /* reference density of the deviation storage (and default port density) */
    double psi_wall;    /* phase field seen at wall sites by the colour gradient, in [-1,1] */
} lbcg_params;

typedef struct {
    int kind;           /* lbcg_port_kind */
    int normal_axis;    /* 0,1,2: axis of the inward normal */
    int normal_sign;    /* +1 or -1 */
    int profile;        /* lbcg_profile (velocity ports) */
    double u_max;       /* peak inflow speed along the inward normal (velocity ports) */
    double rho;         /* imposed density (pressure ports) */
    double psi;         /* colour of the injected fluid, +1 red .. -1 blue (velocity ports) */
} lbcg_port;

/* Observables of the stored state over fluid sites (FP64 reductions on the GPU):
 * component masses (Eq. 2), momentum (Eq. 3), pressure p = sum_k c_p(alpha_k) rho^k
 * (Eq. 8: c_p = 3(1-alpha)/5 in D2Q9; (1-alpha)/2 in D3Q19) averaged inside r < r_in
 * and outside r > r_out of a centre (minimum-image distance on periodic axes), their
 * difference dp (Laplace pressure), the equivalent radius from the red amount
 * sum (1+psi)/2, and max |u| (spurious currents). */
typedef struct {
    double mass_r, mass_b;
    double mom[3];
    double p_in, p_out, dp;
    double r_eff;
    double umax;
    double amount;      /* sum over fluid sites of (1+psi)/2 */
    double n_in, n_out; /* sites in the two pressure windows */
    long long step;
    int nonfinite;      /* fluid sites with non-finite or non-positive density */
    int pad_;
} lbcg_obs;

typedef struct lbcg_ctx lbcg_ctx;

/* Human-readable name of a status code (static string). */
const char* lbcg_strerror(int status);
/* Message of the calling thread's last failed call (static per thread, never NULL). */
const char* lbcg_last_error(void);
/* LBCG_ABI_VERSION of the loaded library. */
int lbcg_abi_version(void);
/* 1 if the loaded library is the bounds-checked debug build (compiled with
 * -DLBCG_CHECK_BOUNDS: every population, link-word and psi-ring index of the step kernels
 * is checked, an index outside its array is skipped and reported as LBCG_ERR_BOUNDS by
 * lbcg_synchronize and the read-backs), 0 for the normal build.  Not part of the method. */
int lbcg_bounds_checked(void);

/* Bytes of ONE population buffer for these parameters (0 if they are invalid).
 * Layout: 2*Q planes of npad values of the storage type, npad = nsites rounded up to
 * a multiple of 128, each plane 256-byte aligned relative to the buffer start. */
size_t lbcg_state_bytes(const lbcg_params* p);

/* Validate parameters and create a context on the current CUDA device.
 * stream: a cudaStream_t (NULL = legacy default stream) on which all work runs.
 * Errors: LBCG_ERR_ARG for an invalid parameter (tau <= 1/2, beta outside [0,1],
 * A < 0, alpha outside (0,1), non-positive size, unknown lattice/precision). */
int lbcg_create(const lbcg_params* p, void* stream, lbcg_ctx** out);
void lbcg_destroy(lbcg_ctx* ctx);

/* Bind caller-owned device buffers (each >= lbcg_state_bytes, 256-byte aligned).
 * The library never frees them; they must outlive the context's use of them. */
int lbcg_bind_state(lbcg_ctx* ctx, void* dev_a, void* dev_b, size_t bytes_each);

/* Geometry: host mask of nsites codes (lbcg_mask) and the port table.  Every port
 * ghost's inward neighbour must be a fluid site, and every port index used by the
 * mask must be < nports (else LBCG_ERR_GEOMETRY).  Allocates the library's device
 * tables (replacing earlier ones).  Synchronous. */
int lbcg_set_geometry(lbcg_ctx* ctx, const uint8_t* host_mask, const lbcg_port* ports, int nports);

/* Initial state f^k = f^{k,eq}(rho^k, u) (Eq. 6) on fluid sites, zero elsewhere.
 * rho_r, rho_b: nsites doubles; u: dim*nsites doubles ([axis][site]) or NULL (rest).
 * Host pointers (synchronous) or device pointers (_device, asynchronous). Resets the step counter. */
int lbcg_init_fields(lbcg_ctx* ctx, const double* rho_r, const double* rho_b, const double* u);
int lbcg_init_fields_device(lbcg_ctx* ctx, const double* rho_r, const double* rho_b, const double* u);

/* Advance n >= 0 steps, asynchronously on the context's stream. */
int lbcg_step(lbcg_ctx* ctx, long long n);
long long lbcg_step_count(const lbcg_ctx* ctx);
int lbcg_synchronize(lbcg_ctx* ctx);

/* Macroscopic fields of the stored state (Eqs. 2-3): rho_r, rho_b (nsites) and
 * u (dim*nsites, [axis][site]); zeros at non-fluid sites.  Host (synchronous) or
 * device (asynchronous) destinations. */
int lbcg_get_fields(lbcg_ctx* ctx, double* rho_r, double* rho_b, double* u);
int lbcg_get_fields_device(lbcg_ctx* ctx, double* rho_r, double* rho_b, double* u);

/* Populations of the stored state as FP64 f^k_i in the layout above (2*Q*nsites
 * doubles, host), converted from the storage precision; and the reverse. */
int lbcg_get_populations(lbcg_ctx* ctx, double* host_f);
int lbcg_set_populations(lbcg_ctx* ctx, const double* host_f);

/* Raw stored state (the current population buffer, lbcg_state_bytes long, in the
 * storage format) to / from host memory: lossless checkpoint and restore in every
 * precision.  lbcg_set_state writes both buffers.  Synchronous. */
int lbcg_get_state(lbcg_ctx* ctx, void* host, size_t bytes);
int lbcg_set_state(lbcg_ctx* ctx, const void* host, size_t bytes);

/* The bound device buffer that holds the current (post-collision) state, in the layout of
 * lbcg_state_bytes; the two bound buffers swap roles as steps run, so the answer is valid
 * until the next lbcg_step.  NULL without a context or bound buffers.  Not part of the
 * method; the paper has no counterpart. */
void* lbcg_current_state(lbcg_ctx* ctx);

/* Checkpoint file of the stored state: parameters, step count and raw state.  lbcg_load
 * requires the same lattice, box and precision (LBCG_ERR_ARG otherwise), restores the
 * step count and writes both buffers.  Synchronous. */
int lbcg_save(lbcg_ctx* ctx, const char* path);
int lbcg_load(lbcg_ctx* ctx, const char* path);

/* Observables (see lbcg_obs).  centre[3] in lattice units; r_in < 0 selects
 * r_eff/2 and r_out < 0 selects r_eff + 5 (the paper's interface width of about
 * 5 lattice units, Sec. III).  Synchronous.  Returns LBCG_ERR_DIVERGED (with *out
 * filled) when nonfinite > 0. */
int lbcg_observables(lbcg_ctx* ctx, const double centre[3], double r_in, double r_out, lbcg_obs* out);

/* Allocation-free observables.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory, e.g. plug-ins whose host application
 * owns every device allocation through its own pool, loops that forbid allocation after
 * start-up, or code running with the device memory budget fully committed.  It needs no
 * context and allocates nothing: the caller passes the inputs and receives the result;
 * the reduction's scratch is a file-scope device array of 131,328 bytes (1024 partial
 * rows of 16 doubles plus 2 result rows) that every GPU loading the library holds until
 * the process exits.
 *   p        lattice, box and storage precision of the state (validated as by
 *            lbcg_create; LBCG_ERR_ARG otherwise)
 *   dev_state device buffer holding one population state in the layout of
 *            lbcg_state_bytes(p) (e.g. lbcg_current_state of a context); read only
 *   dev_mask device array of nsites mask codes (only code 0 = fluid is counted), or
 *            NULL when every site is fluid
 *   centre, r_in, r_out   as for lbcg_observables
 *   stream   CUDA stream of the kernels (NULL = legacy default); the call waits for it
 *   out      host result; out->step = -1 (no context)
 * Results equal those of lbcg_observables for the same state.  The reduction launches at
 * most 1024 blocks, each striding over the sites, so every lattice the library accepts
 * fits the array.  The call is synchronous (it copies the result to the host and waits),
 * so it cannot be recorded into a CUDA graph: on a stream that is being captured it
 * returns LBCG_ERR_STATE without touching the stream.  The first call on each device looks
 * up the array's device address with cudaGetSymbolAddress (with that device current).
 * All calls share the one array and it keeps the last call's contents (every row a call
 * reads is written by that call first): calls whose GPU work overlaps, on different
 * streams or host threads, race and must be ordered by the caller.  Returns
 * LBCG_ERR_DIVERGED (out filled) when a fluid site has a non-finite or non-positive
 * density. */
int lbcg_observables_noalloc(const lbcg_params* p, const void* dev_state, const uint8_t* dev_mask,
                             const double centre[3], double r_in, double r_out, void* stream, lbcg_obs* out);

/* Droplet labelling: connected components of {fluid sites with rho_R > rho_B}
 * (psi > 0), face-connected, wrapping periodic axes.  labels[nsites] receives the
 * smallest linear site index of the site's component, or -1.  counts/volumes (may be
 * NULL) receive, in increasing label order, each droplet's site count and its
 * sum of (1+psi)/2, for at most cap droplets; *n_drops receives the total number.
 * Synchronous.  The union-find passes are bounded: LBCG_ERR_TIMEOUT if the bound is
 * reached (labels then invalid). */
int lbcg_label(lbcg_ctx* ctx, int32_t* labels, int64_t* counts, double* volumes, int cap, int* n_drops);

/* ------------------------------------------------------------------ batches
 * Many independent instances (contexts of one lattice and storage precision) advanced
 * together: each chunk of up to 32 steps replays one captured CUDA graph whose nodes run
 * the port refill and the fused step for all instances at once (a persistent grid
 * striding over every instance's tiles).  Admission and retirement only rewrite a device
 * table, never the graph.  Every instance's result is bit-identical to running it alone
 * with lbcg_step (same per-site code).  The batch works on the stream given at creation;
 * the instances' own streams are not used while they are in the batch.  A context must
 * not be stepped by itself while it is in a batch.  The batch owns small device tables
 * (slot table, work lists) and a pinned host copy of the slot table. */
typedef struct lbcg_batch lbcg_batch;

/* max_instances in 1..4096. */
int lbcg_batch_create(int lattice, int precision, int max_instances, void* stream, lbcg_batch** out);
void lbcg_batch_destroy(lbcg_batch* batch);
/* Add a ready context (bound state, geometry, fields) that is to run `steps` more steps;
 * *slot receives its slot.  LBCG_ERR_CAPACITY when the batch is full. */
int lbcg_batch_add(lbcg_batch* batch, lbcg_ctx* ctx, long long steps, int* slot);
/* Remove an instance (finished or not); waits for the batch's stream first. */
int lbcg_batch_remove(lbcg_batch* batch, int slot);
/* Steps an instance still has to run, or -1 for an empty slot. */
long long lbcg_batch_remaining(const lbcg_batch* batch, int slot);
/* Advance every instance by min(max_steps, its remaining steps); asynchronous. */
int lbcg_batch_step(lbcg_batch* batch, long long max_steps);
/* Wait for the batch's work, then report (once each) the slots that have no steps left. */
int lbcg_batch_poll(lbcg_batch* batch, int* done_slots, int cap, int* ndone);

/* Launch shape of a batch (0 in a field = default).  Not part of the method; the paper has
 * no counterpart: it sets how the batched kernels cut the instances into work items and how
 * many steps one captured graph replays, and is chosen by measurement (autotune.py).
 *   rows             D2Q9: rows per warp strip (default 16); D3Q19: z-planes per tile (8)
 *   block_rows       D3Q19: warps per block along y, 3..8 (8); 0 for D2Q9
 *   strips_per_item  D2Q9: warp strips per work item (one block), 1..8 (8); 0 for D3Q19
 *   blocks_per_sm    resident blocks per SM of the persistent grid (0 or more than fit: as
 *                    many as fit, by the occupancy of the batched kernel on this device)
 *   graph_steps      steps per captured graph, even, 2..256 (32)
 *   sms              read back only: the device's SM count (grid = sms x blocks_per_sm)
 * lbcg_batch_set_shape waits for the batch's stream, re-cuts every instance in the batch and
 * drops the captured graph; results are bit-identical across shapes (the cut into work
 * items changes nothing in the per-site arithmetic).
 * lbcg_batch_get_shape returns the shape after defaults. */
typedef struct {
    int rows, block_rows, strips_per_item, blocks_per_sm, graph_steps, sms;
} lbcg_batch_shape;
int lbcg_batch_set_shape(lbcg_batch* batch, const lbcg_batch_shape* shape);
int lbcg_batch_get_shape(const lbcg_batch* batch, lbcg_batch_shape* shape);
/* Multiply-add throughput of the current device in GFLOP/s (2 flops per FMA), measured by
 * a kernel of independent FMA chains timed with CUDA events on `stream` (synchronises):
 * precision LBCG_FP64 for FP64, anything else for FP32.  The ALU roofline of the FP64 step
 * (bound by the FP64 rate, not by HBM) and of the FP32 arithmetic.  Not part of the
 * method; the paper has no counterpart. */
int lbcg_fma_peak(int precision, void* stream, double* gflops);

/* Message of the calling thread's last failed batch call. */
const char* lbcg_batch_last_error(void);

/* Kernel timing: when enabled, CUDA events bracket every fused step kernel that
 * lbcg_step launches on its own, on the context's stream: the n mod 32 steps left after
 * the 32-step CUDA graphs that lbcg_step replays (so every step when n < 32; graph
 * replays stay untimed and unchanged).  lbcg_kernel_time returns the summed duration in
 * milliseconds and the number of timed launches since the last reset (synchronises). */
int lbcg_set_kernel_timing(lbcg_ctx* ctx, int enable);
int lbcg_kernel_time(lbcg_ctx* ctx, double* total_ms, long long* launches);

/* Launch shape of the fused step kernel (0 = library default):
 * rows: sites per warp along the marching axis (D2Q9: y rows per warp strip;
 * D3Q19: z planes per block); block_rows: D3Q19 warps per block along y (3..8; up to
 * 16 with variant 7 and the regularized collision).
 * variant: 0 default, 1 keep the next row/plane's populations in registers,
 * 2 re-read them when colliding, 5 (D3Q19) re-read compiled for three resident blocks per
 * SM, 6 (D3Q19, regularized) moment march: the waiting plane is held as the 11 moments the
 * regularized collision needs (Eq. 11 rebuilds every population from them), so nothing
 * is read twice, 7 the same with those moments in shared memory (64 registers),
 * 8 (D3Q19, regularized, FP32 or FP32-dev storage, nx a multiple of 4, block_rows 6 or
 * 8) the moment march with every plane's pulled populations staged in shared memory by
 * the tensor memory accelerator (two-stage pipeline of Q boxes per plane, bounded
 * waits); where its conditions do not hold it runs as 7 (FP64: 6), 9 (D3Q19, regularized,
 * block_rows 3..8) variant 6 with each warp waiting per plane only for the two warps whose
 * psi rows it reads (named barriers) instead of the whole block: identical results, warps
 * up to one plane apart.  The D3Q19 moment marches (6, 7, 9) and both D2Q9 strip marches
 * refill the port ghosts of the state they write themselves (each block or warp after its
 * tile or strip, from the populations it has just written), so a step with ports is one
 * launch; the other variants run the separate refill kernel before each step.
 * Variants 6, 7 and 9 fall back to 5 (FP64: 2) for the BGK collision.  A context created while
 * the environment variable LBCG_TEST_PIPELINE_STALL=1 is set makes every pipeline wait of
 * variant 8 run out (failure-path test): the step then leaves the state invalid and
 * lbcg_synchronize and the read-back calls report LBCG_ERR_TIMEOUT once.  The default is the
 * moment march for the regularized collision on either lattice (D3Q19 boxes with walls or
 * ports: 9, up to 8 warps per block; otherwise 6); with BGK the plain march for D2Q9 and
 * variant 5 (FP64: 2) for D3Q19.  D2Q9 takes 6 (moment march,
 * regularized only) and treats every other value as the plain march.  Values 3, 4 and
 * above 9 are rejected (LBCG_ERR_ARG).
 * Within one variant results are bit-identical across shapes; variants may contract
 * multiply-adds and order sums differently and agree to
 * rounding.  Drops captured step graphs. */
int lbcg_set_launch(lbcg_ctx* ctx, int rows, int block_rows, int variant);

/* The launch shape the next step uses, after defaults: rows, block_rows (0 for D2Q9) and
 * the kernel variant actually run (never 0; see lbcg_set_launch).  Null outputs are
 * skipped. */
int lbcg_get_launch(lbcg_ctx* ctx, int* rows, int* block_rows, int* variant);

/* Grid of the next fused step launch: the number of thread blocks and threads per block,
 * and the kernels one step launches (the fused step, plus the port refill unless the step
 * kernel refills the port ghosts itself, as the D3Q19 moment marches do).  Not part of the
 * method; the paper has no counterpart.  Null outputs are skipped. */
int lbcg_get_grid(lbcg_ctx* ctx, long long* blocks, int* threads, int* kernels_per_step);

#ifdef __cplusplus
}
#endif

#endif /* LBCG_H */
