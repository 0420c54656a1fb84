/*
 * lbm.h — C ABI of the GB300 entropic multi-relaxation-time two-phase lattice
 * Boltzmann library (liblbm.so).
 *
 * The method is that of Hosseini, Dorschner & Karlin, "Entropic
 * multi-relaxation-time lattice Boltzmann model for large density ratio
 * two-phase flows" (arXiv:2201.12404).  One call of lbm_step advances the
 * populations f_i of a D2Q9 or D3Q27 lattice by whole time steps of Eq. (LBGK):
 *
 *   f_i(r + c_i dt, t + dt) = (1 - w/2) f_i + (w/2) f_i^mirr + (f_i^* - f_i^eq)
 *
 * with the product-form equilibria of Sec. 2.2 (Eqs. LBMeq, LBMstar), the
 * Peng-Robinson pressure of Sec. 3.1 (Eq. PREoS) entering through the
 * pseudo-potential force of Sec. 2.3 (Eq. Kforce_final), the diagonal
 * correction Phi (Eq. correction, with the sign that cancels the lattice's
 * third-moment defect, the job Sec. 2.2 gives it; the printed sign doubles the
 * defect), and the entropic mirror state of Sec. 2.4
 * (k/s/h split in the central Hermite basis of Appendix A, gamma from the
 * entropic scalar products).
 *
 * Conventions shared by every call:
 *  - Lattice units: dt = dr = 1, cs^2 = 1/3, P0 = rho cs^2 (Sec. 2.3).
 *  - Host field arrays are float64, node index x + nx*(y + ny*z), x fastest
 *    (nz = 1 in 2-D).  The caller owns every host buffer; the library copies.
 *  - Populations are exchanged in "canonical" order: float64 array of Q*N
 *    values, element [i*N + node], velocity index i = (cx+1) + 3(cy+1) +
 *    9(cz+1), holding the post-streaming, pre-collision state.  The opposite
 *    direction of i is Q-1-i.
 *  - The library owns all device memory of a domain (allocated in
 *    lbm_create_domain, freed in lbm_destroy).  Calls that take host buffers
 *    stage them in scratch device memory from a pool of the library's own,
 *    which keeps up to 4 GiB per device between calls.
 *  - Every call that launches GPU work enqueues it on the domain's stream and
 *    returns without waiting, except those documented as synchronising.
 *  - Handles are not thread-safe: use one handle per host thread or lock.
 *  - After an error other than LBM_ERR_INVALID_ARG the handle refuses further
 *    work with LBM_ERR_STATE until destroyed; lbm_last_error() says why.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain* lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID_ARG = 1, /* bad argument; the handle stays usable */
  LBM_ERR_OOM = 2,         /* device allocation failed */
  LBM_ERR_CUDA = 3,        /* a CUDA call failed */
  LBM_ERR_UNSTABLE = 4,    /* a non-finite or non-positive density appeared */
  LBM_ERR_TIMEOUT = 5,     /* a bounded device-side wait (a shared-memory tile copy) gave up */
  LBM_ERR_STATE = 6,       /* the handle is poisoned by an earlier error */
  LBM_ERR_BOUNDS = 7       /* only in a library built with -DLBM_BOUNDS_CHECK: a kernel computed
                            * a population address or auxiliary-field index outside its buffer
                            * (the access was redirected to the buffer's first element) */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q27 = 1 } lbm_lattice;

/* Storage and arithmetic of the populations.
 * LBM_FP64: stored and computed in float64 (the GPU reference path).
 * LBM_FP32: stored and computed in float32; float64 only in the Peng-Robinson
 *           pressure inside the interface band and in the gamma ratio.
 * LBM_FP16DEV: stored as float16 deviations f_i/(w_i rho_w) - 1, rho_w the
 *           density of the node that wrote the slot (kept per node, one float32
 *           per node and parity); computed in float32 like LBM_FP32. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16DEV = 2 } lbm_precision;

/* Boundary of each face (-x,+x,-y,+y,-z,+z).  Periodic needs both faces of an
 * axis periodic.  Bounce-back is half-way: the wall sits half a node outside
 * the first and last node, populations reverse there, and the auxiliary
 * density/pseudo-potential fields are mirrored across it. */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_BOUNCEBACK = 1 } lbm_bc;

/* LBM_GAMMA_ENTROPIC: gamma per node from Sec. 2.4.
 * LBM_GAMMA_FIXED: gamma = gamma_value everywhere (2 reproduces LBGK; 2/omega
 * relaxes the higher-order moments fully onto f*). */
typedef enum { LBM_GAMMA_ENTROPIC = 0, LBM_GAMMA_FIXED = 1 } lbm_gamma_mode;


typedef struct {
  int32_t lattice;     /* lbm_lattice */
  int32_t precision;   /* lbm_precision */
  int32_t nx, ny, nz;  /* nodes per axis, each >= 5; nz must be 1 for D2Q9 */
  /* Peng-Robinson EOS, Sec. 3.1: a, b, gas constant R, reduced temperature
   * T/Tc and acentric factor w'.  Tc = 0.0778 a/(0.45724 b R). */
  double a, b, R, T_over_Tc, acentric;
  double kappa;        /* capillary coefficient kappa~ = kappa dr^2 of Eq. (Kforce_final), >= 0 */
  /* Kinematic viscosity: nu(rho) = nu_vapour + phi (nu_liquid - nu_vapour),
   * phi = clamp((rho - rho_vapour)/(rho_liquid - rho_vapour), 0, 1); local
   * omega = 1/(3 nu + 1/2) (Sec. 2.1 with P0 = rho cs^2).  Equal viscosities
   * give a uniform omega.  rho_liquid > rho_vapour > 0 is required. */
  double nu_liquid, nu_vapour, rho_liquid, rho_vapour;
  double body_force[3]; /* uniform acceleration g: adds rho*g to the force */
  int32_t bc[6];        /* lbm_bc per face -x,+x,-y,+y,-z,+z (z faces ignored in 2-D) */
  int32_t gamma_mode;   /* lbm_gamma_mode */
  double gamma_value;   /* used when gamma_mode == LBM_GAMMA_FIXED */
  /* FP32 path only: 0 = Peng-Robinson pressure in float32 everywhere,
   * 1 = in float64 where rho lies inside the interface band (default),
   * 2 = float64 everywhere. */
  int32_t eos_fp64;
  void* stream;         /* cudaStream_t to run on; NULL = a stream the library creates */
  /* Optional device allocator for the buffers a domain keeps for its lifetime
   * (populations, auxiliary fields, error words, the gamma record), for example
   * a framework's caching allocator; NULL dev_alloc = cudaMalloc/cudaFree.  Set
   * both or neither.  dev_alloc(bytes, alloc_ctx) returns memory of the current
   * device aligned to 256 bytes, or NULL when it cannot (lbm_create_domain then
   * fails with LBM_ERR_OOM); dev_free(ptr, alloc_ctx) releases it and is called
   * from lbm_destroy after the domain's stream has been synchronised, on the
   * same host thread as other calls on the handle.  Scratch memory of the calls
   * that take host buffers still comes from the library's own pool. */
  void* (*dev_alloc)(size_t bytes, void* alloc_ctx);
  void (*dev_free)(void* ptr, void* alloc_ctx);
  void* alloc_ctx;
} lbm_params;

/* Fill p with defaults: D2Q9 FP32 64x64, the paper's EOS constants
 * (a = 0.003, b = 0.095, R = 1, w' = 0.344, Sec. 3.1), T/Tc = 0.8, kappa = 0,
 * nu = 0.1, rho_liquid = 1, rho_vapour = 0.5, periodic, entropic gamma,
 * eos_fp64 = 1, NULL stream, no allocator. */
lbm_status lbm_default_params(lbm_params* p);

/* Validate p, allocate the domain's device memory and create its handle.
 * *out receives the handle (NULL on failure).  Errors (message via
 * lbm_last_error(NULL)): INVALID_ARG; OOM when lbm_footprint_bytes(p) exceeds
 * the device's free memory (checked before anything is allocated) or an
 * allocation fails; CUDA. */
lbm_status lbm_create_domain(const lbm_params* p, lbm_handle* out);

/* Initial state from host arrays of N values each (uz is NULL in 2-D): the
 * equilibrium f^eq(rho, u_b) of Eq. (LBMeq) at the bare velocity
 * u_b = u - F dt/(2 rho), F the force of the density field rho (Eq.
 * Kforce_final plus rho g), so that the reported velocity of the initial state
 * (see lbm_read_macroscopic) is u.  Starting from u_b = u instead leaves an
 * impulse of F/(2 rho) at every interface, which destabilises runs at large
 * density ratios.  Resets the step counter and the streaming parity.
 * Synchronising. */
lbm_status lbm_init_fields(lbm_handle h, const double* rho, const double* ux, const double* uy,
                           const double* uz);

/* Advance nsteps >= 0 time steps of Eq. (LBGK) (asynchronous).  A step is three
 * kernels: moments and the Peng-Robinson pseudo-potential (Sec. 2.3); the force
 * of Eq. (Kforce_final) and the flux q of Eq. (correction); the collision of
 * Sec. 2.4 with the A-A stream.  With timing off, once the domain has run two
 * steps, pairs of steps are replayed as a captured CUDA graph of those kernels
 * (same kernels and arguments, bit-identical results; recaptured when the gamma
 * record is switched on).  An instability detected by an earlier call surfaces
 * here or in any later synchronising call as LBM_ERR_UNSTABLE. */
lbm_status lbm_step(lbm_handle h, int64_t nsteps);

/* Wait for the domain's stream; report LBM_ERR_UNSTABLE if a non-finite or
 * non-positive density has appeared.  Synchronising. */
lbm_status lbm_synchronize(lbm_handle h);

/* Density and velocity of the current state into host arrays of N values each
 * (uz ignored/NULL in 2-D).  The velocity is the exact-difference-method
 * velocity u + F dt/(2 rho).  Synchronising. */
lbm_status lbm_read_macroscopic(lbm_handle h, double* rho, double* ux, double* uy, double* uz);

/* Release the domain.  NULL-safe. */
lbm_status lbm_destroy(lbm_handle h);

/* Canonical populations (see conventions) as float64, count = Q*N.
 * Synchronising. */
lbm_status lbm_read_populations(lbm_handle h, double* host, size_t count);

/* Canonical populations of a box of nodes, for checking or probing a part of a
 * large domain without copying all of it.  Window node (i, j, k), 0 <= i <
 * extent[0] and so on, is the domain node ((origin[0] + i) mod nx, (origin[1] +
 * j) mod ny, (origin[2] + k) mod nz): a window may wrap across any face.  host
 * receives count = Q*extent[0]*extent[1]*extent[2] float64 values in the order
 * [i_pop][k][j][i] (x fastest), the same per-node values lbm_read_populations
 * gives.  Needs 0 <= origin[a] < n_a and 1 <= extent[a] <= n_a on every axis
 * (in 2-D origin[2] = 0, extent[2] = 1), else LBM_ERR_INVALID_ARG with the
 * handle left usable.  The caller owns both arrays.  Synchronising. */
lbm_status lbm_read_populations_window(lbm_handle h, const int64_t origin[3], const int64_t extent[3],
                                       double* host, size_t count);

/* Replace the state with canonical populations (float64, count = Q*N; rounded
 * to the storage precision).  Resets the streaming parity.  Synchronising. */
lbm_status lbm_write_populations(lbm_handle h, const double* host, size_t count);

/* Totals of the current state: mass sum rho, momentum sum_i c_i f_i (3 values,
 * bare), max |u| of the bare velocity.  gamma_field (nullable) receives, per
 * node (N values), the gamma of the last step run while gamma recording was on
 * (lbm_record_gamma), zeros otherwise.  Deterministic.  Synchronising. */
lbm_status lbm_read_diag(lbm_handle h, double* mass, double* momentum3, double* max_u,
                         double* gamma_field);

/* A drop falling onto a liquid film (the impact of Secs. 3.2 and 3.3), built on
 * the GPU for domains whose fields are too large to pass from the host.  With
 * the last axis vertical (y in 2-D, z in 3-D; the film on its low face) and the
 * drop centred at x = (nx-1)/2 [, y = (ny-1)/2], height film + radius + gap:
 * rho = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 d / width), d the smaller of
 * the distance to the drop surface and the height above the film surface
 * (film - 1/2), with rho_l, rho_v those of the domain's parameters; the velocity
 * is -speed along the last axis times the drop's liquid fraction
 * 1/2 - 1/2 tanh(2 d_drop / width), plus, where noise > 0, normal white noise of
 * standard deviation noise * speed in every component, also weighted by that
 * fraction (the perturbation of Sec. 3.3), drawn from SplitMix64 keyed by
 * (seed, node, component).  film <= 0: no film.  Then, as lbm_init_fields, the
 * populations start at rest in the reported sense.  LBM_ERR_INVALID_ARG for a
 * NULL geometry or radius/width not positive.  Synchronising. */
typedef struct {
  double radius, film, gap, speed, width, noise;
  uint64_t seed;
} lbm_drop_on_film;
lbm_status lbm_init_drop_on_film(lbm_handle h, const lbm_drop_on_film* g);

/* Largest speed over the domain of the reported velocity u + F dt/(2 rho)
 * (the exact-difference-method velocity that lbm_read_macroscopic returns,
 * the velocity whose maximum the paper reports as the spurious current,
 * Sec. 3.1.2), reduced on the GPU: one pass-1 launch for the current state,
 * one reduction.  A state with a non-finite speed gives +inf.  Synchronising. */
lbm_status lbm_max_speed(lbm_handle h, double* max_u);

/* Interface thickness W = (rho_liquid - rho_vapour) / max |grad rho| of the
 * current state (Sec. 3.1.1), rho_liquid and rho_vapour those of the domain's
 * parameters, the gradient by second-order central differences (across periodic
 * wraps and mirrored at walls), the maximum reduced on the GPU; +inf for a uniform
 * state.  max_grad (nullable) receives max |grad rho|.  Synchronising. */
lbm_status lbm_interface_width(lbm_handle h, double* width, double* max_grad);

/* Crown (spreading) radius of a drop impact (Sec. 3.2): over the nodes of layer
 * `layer` (index along the last axis: y in 2-D, z in 3-D), the largest distance
 * from the vertical axis through the domain centre (x = (nx-1)/2 [, y = (ny-1)/2])
 * of a node whose density exceeds (rho_liquid + rho_vapour)/2; 0 when none does.
 * Reduced on the GPU.  LBM_ERR_INVALID_ARG for a layer outside the domain.
 * Synchronising. */
lbm_status lbm_crown_radius(lbm_handle h, int32_t layer, double* radius);

/* 2/(omega gamma) per node (N values, x fastest) of the last step run with gamma
 * recording on, omega the node's relaxation rate in that step: about 1 where the
 * entropic stabiliser is idle, away from the interfaces (Sec. 3.3).
 * LBM_ERR_INVALID_ARG when no step has been recorded.  Synchronising. */
lbm_status lbm_read_relaxation(lbm_handle h, double* two_over_omega_gamma);

/* Turn per-node gamma recording on (enable != 0) or off for later lbm_step
 * calls.  Recording adds a float32 store per node and step (the 2/(omega gamma)
 * field of Sec. 3.3 is derived from it). */
lbm_status lbm_record_gamma(lbm_handle h, int enable);

/* Number of nodes where the f*_i <= 0 guard set gamma = 2, summed over all
 * steps since creation.  Synchronising. */
lbm_status lbm_guard_count(lbm_handle h, uint64_t* count);

/* Device bytes lbm_create_domain would allocate for p (0 if p is invalid). */
size_t lbm_footprint_bytes(const lbm_params* p);

/* Maxwell equal-area coexistence of the Peng-Robinson EOS (Sec. 3.1.1,
 * Eq. Maxwell_equal_area) for the EOS fields of p: densities of the vapour and
 * liquid and the saturation pressure.  Host-only. */
lbm_status lbm_coexistence(const lbm_params* p, double* rho_vapour, double* rho_liquid, double* p_sat);

/* Densities on (0, 1/b) where P(rho) - rho cs^2 changes sign for the EOS fields
 * of p: the sign s of the pseudo-potential (Sec. 2.3; s = +1 where P > rho cs^2,
 * -1 otherwise, including equality) flips there.  Writes them ascending into
 * changes[0..n-1] (n <= 3, the rest +inf), each the first float64 density with
 * the new sign, and the sign below changes[0] into *s0; the kernels decide s
 * this way.  Host-only; LBM_ERR_INVALID_ARG for NULL pointers or a, b, R,
 * T/Tc not positive. */
lbm_status lbm_psi_sign_changes(const lbm_params* p, double changes[3], int* n, double* s0);

/* Kernel timing on the domain's stream with CUDA events.  When enabled, every
 * launch made by lbm_step is bracketed by events; lbm_kernel_times then
 * synchronises and returns, per kernel kind, the summed milliseconds and the
 * launch count: ms[0]/count[0] the moments+EOS kernel and the force+q kernel that
 * follows it (timed together; two launches a step), ms[1]/count[1] the
 * collide+stream kernel.  Enabling resets the sums; while enabled, lbm_step
 * launches kernel by kernel (no graph replay). */
lbm_status lbm_set_timing(lbm_handle h, int enable);
lbm_status lbm_kernel_times(lbm_handle h, double ms[2], int64_t count[2]);

/* Kernels this handle has launched since creation (all kinds). */
int64_t lbm_launch_count(lbm_handle h);

/* Message of the last error on h, or of the last failed lbm_create_domain /
 * lbm_coexistence on this thread when h is NULL.  Never NULL. */
const char* lbm_last_error(lbm_handle h);

/* ---- Batches: many D2Q9 domains advanced by one persistent launch ----
 *
 * A batch holds D2Q9 domains of one precision and any sizes and parameters.
 * lbm_batch_step advances all of them by nsteps time steps with a single
 * cooperative (all blocks resident) kernel launch: the blocks walk a work list of
 * (domain, tile) items for pass 1 (moments, EOS), meet at a grid barrier, walk it
 * for pass 1b (force, q), meet again, walk it for pass 2 (collide, stream), and
 * repeat per step.  Every grid-barrier wait is bounded; a wait that gives up
 * stops the kernel and surfaces as LBM_ERR_TIMEOUT.  The launch is captured in a
 * CUDA graph per distinct nsteps (replayed afterwards) when the driver accepts
 * capturing a cooperative launch, and launched directly otherwise.  Work runs on
 * the stream of the first domain.  While a domain belongs to a batch, advance it
 * only through the batch.  The results are the same as stepping each domain alone
 * (same kernels' per-tile arithmetic). */
typedef struct lbm_batch* lbm_batch_handle;

/* Create a batch over `count` >= 1 distinct domains (the caller keeps owning
 * them; destroy the batch before them).  Synchronising. */
lbm_status lbm_batch_create(const lbm_handle* domains, int32_t count, lbm_batch_handle* out);

/* Advance every domain of the batch by nsteps >= 0 time steps (asynchronous). */
lbm_status lbm_batch_step(lbm_batch_handle b, int64_t nsteps);

/* Wait for the batch; LBM_ERR_TIMEOUT if a grid-barrier wait gave up, otherwise the
 * first error of lbm_synchronize over the domains.  Synchronising. */
lbm_status lbm_batch_synchronize(lbm_batch_handle b);

/* Tile-shape autotuner: time every compiled tile shape of the persistent kernel for
 * trial_steps steps on copies of the batch's domains (the domains themselves do not
 * advance) and keep the fastest.  cache_path (nullable) names a file of JSON lines
 * {"key": ..., "block": [bx, by], "ms_per_step": ...}; a line whose key matches this
 * batch's size class (precision, total nodes rounded down to a power of two, domain
 * count) is used without timing, and a new choice is appended.  Synchronising. */
lbm_status lbm_batch_tune(lbm_batch_handle b, int32_t trial_steps, const char* cache_path);

/* Test and diagnostic extension (the paper has no counterpart): bound the
 * grid-barrier waits of later lbm_batch_step calls to poll_limit polls of about
 * 0.1 us each (0 restores the default, about 3 s), and with skip_arrival != 0 make
 * block 0 pass the barriers without arriving, so that every other block's wait
 * runs out.  This exercises the timeout path without any GPU fault: the kernel
 * stops, lbm_batch_synchronize returns LBM_ERR_TIMEOUT and the batch is poisoned;
 * the domains' states are then not valid.  LBM_ERR_INVALID_ARG for a NULL batch. */
lbm_status lbm_batch_set_wait(lbm_batch_handle b, uint32_t poll_limit, int32_t skip_arrival);

/* Chosen tile shape, grid size (blocks) and whether launches go through a CUDA graph. */
lbm_status lbm_batch_info(lbm_batch_handle b, int32_t* block_x, int32_t* block_y, int32_t* grid_blocks,
                          int32_t* graph_captured);

/* Release the batch (not its domains).  NULL-safe. */
lbm_status lbm_batch_destroy(lbm_batch_handle b);

/* Message of the last error on b, or of the last failed lbm_batch_create on this
 * thread when b is NULL. */
const char* lbm_batch_last_error(lbm_batch_handle b);

/* Library build string (lattices, precisions, target architecture). */
const char* lbm_version(void);

/* Allocation-free stepping.  The paper has no counterpart: this call exists for
 * callers that cannot allocate device memory (a host framework that owns the
 * whole device pool, a memory-capped process, code that must not enter the
 * allocator while other work runs).  It advances caller-owned populations by
 * nsteps time steps exactly as lbm_step does, without any handle and without
 * any cudaMalloc/cudaFree or allocating library call.
 *
 *   p            domain parameters, validated as by lbm_create_domain; p->stream
 *                is the stream to run on (NULL = the legacy default stream).
 *   populations  device pointer to Q*N values of the storage type (float32 for
 *                LBM_FP32, float64 for LBM_FP64; LBM_FP16DEV is not accepted
 *                here) in canonical order (see the
 *                conventions above); read and overwritten in place.  The caller
 *                owns it.
 *   nsteps       even and >= 0, so that the state is in canonical order again on
 *                return.
 *
 * The auxiliary fields between the passes live in a 16 MiB scratch array
 * compiled into the library (every GPU that loads the library holds it until
 * the process exits).  Domains whose 2 + 2D padded auxiliary fields, ((rho,
 * psi) pairs, q and j), px(ny+4)(nz+4) values each in the storage type with
 * px = nx+4 rounded up to a multiple of 4, need more than 16 MiB - 256 B are
 * rejected: for example 64x64x96 D3Q27 in float32 fits, 64x64x128 does not;
 * 800x800 D2Q9 in float32 fits, 1000x1000 does not.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call shares the one array: calls that overlap on
 * the GPU (two streams, or two host threads) race and corrupt each other.
 * Asynchronous: returns once the work is enqueued.  Instabilities (a
 * non-finite or non-positive density) and bounded device waits that gave up
 * are not reported here: read them with lbm_noalloc_status once the stream's
 * work has completed.
 * Returns LBM_ERR_INVALID_ARG for NULL pointers, invalid parameters, LBM_FP16DEV,
 * odd or negative nsteps, populations not aligned to their storage type, or a
 * domain beyond the scratch maximum; LBM_ERR_CUDA if a CUDA error was already
 * pending when the call began (it is left pending for the caller) or if the
 * symbol lookup or a launch fails. */
lbm_status lbm_step_noalloc(const lbm_params* p, void* populations, int64_t nsteps);

/* Outcome of the last lbm_step_noalloc call on the current device, for the same
 * callers (the paper has no counterpart): LBM_ERR_BOUNDS (bounds-checked builds
 * only) if a kernel computed an index outside its buffer, else LBM_ERR_TIMEOUT if
 * one of its bounded device-side waits gave up (those tiles were left unwritten),
 * else LBM_ERR_UNSTABLE if a non-finite or non-positive density appeared, else LBM_OK;
 * LBM_ERR_CUDA if the flag word cannot be read.  Reads the flag word at the start
 * of the shared scratch array into a host variable (no allocation); call it after
 * the stream that ran the steps has completed, before the next call clears it. */
lbm_status lbm_noalloc_status(void);

/* Host buffers for the calls that take host arrays (lbm_init_fields,
 * lbm_read_macroscopic, lbm_read/write_populations and their windows).  The
 * paper has no counterpart: these exist for the host-to-device path on Grace
 * hosts, where a pageable or small-page pinned buffer that the GPU has not
 * touched for a while copies several times slower than the NVLink-C2C link
 * (the copy engines' address translation, not the bandwidth, sets the pace).
 *
 * lbm_host_alloc maps at least `bytes` bytes of zero-filled host memory and
 * registers it with the CUDA runtime (page-locked), so that copies from and to it
 * run as direct transfers.  A request of at least half a transparent huge page
 * is mapped at a huge-page boundary, rounded up to whole huge pages, and the
 * kernel is asked for huge pages (advice: small pages where it has none); a
 * smaller one, or any request where transparent huge pages are off, uses the
 * system page size.  *out receives the start (aligned to the huge page or page
 * size it was mapped with); the caller owns the buffer until
 * lbm_host_free.  Returns LBM_ERR_INVALID_ARG for bytes == 0 or out == NULL,
 * LBM_ERR_OOM if the mapping fails, LBM_ERR_CUDA if the registration fails (no
 * CUDA device, for one); *out is NULL on any error.  Not synchronising; costs
 * one pass of zero-filling over the memory.
 *
 * lbm_host_free unregisters and unmaps a buffer that lbm_host_alloc returned.
 * NULL-safe; LBM_ERR_INVALID_ARG for any other pointer (nothing is released),
 * LBM_ERR_CUDA if the unregistration fails (the memory is unmapped anyway).
 * Thread-safe.  No copy or kernel may still be using the buffer. */
lbm_status lbm_host_alloc(size_t bytes, void** out);
lbm_status lbm_host_free(void* p);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
