/*
 * alb — adaptive-lattice Boltzmann on one GPU.
 *
 * C ABI of the interpolation-free, state-adaptive compressible lattice
 * Boltzmann method of Coreixas & Latt (arXiv:2009.13426): a D2Q21 double
 * distribution (f for the monatomic part, g for internal degrees of freedom)
 * whose velocities c_i = xi_i + U are shifted per node by an integer vector U
 * (Fig. 1, Eq. discrete_norm_peculiar with theta = 1).
 *
 * One time step (Sec. IV.A.3, "Algorithm overview") is, per node x:
 *   - pull streaming h_i(x, t+1) = h_i*(x - c_i, t) (Eq. stream) in the lattice
 *     U'(x) selected from the node's own velocity by Eq. criterion; a pull
 *     whose sender collided in another lattice is missing and is rebuilt by
 *     Grad's approximation (Eqs. GradGeneral, GradGeneral_f, GradGeneral_g)
 *     from the sender's moments and their second-order central differences;
 *   - moments rho, u, T (Eq. polyTemp);
 *   - the 8-moment exponential numerical equilibrium (Eq. feqNum_8Mom, with
 *     the constraints of Eqs. G0_8mom..G3yaa_8mom), its multipliers found by
 *     FP64 Newton iterations; g^eq = (2 Cv - D) T f^eq (Eq. gEq);
 *   - optional kinetic sensor tau <- tau * alpha(eps_Kn) (Eq. DeltaAvg);
 *   - BGK relaxation h* = h - (h - h^eq)/tau, tau = 1/2 + nu/T (Eq. coll,
 *     App. E).
 *
 * Conventions for every call:
 *   - Return value: ALB_OK (0) or a negative ALB_E* code; alb_last_error()
 *     then gives a message for the calling thread.
 *   - Fields are arrays of nx*ny doubles, x fastest (index y*nx + x), owned by
 *     the caller. where = ALB_HOST: host memory, the call copies synchronously.
 *     where = ALB_DEVICE: device memory of the current CUDA device, the copy
 *     is ordered on the handle's stream and the call returns after enqueueing.
 *   - The library owns all state it allocates; alb_destroy frees it.
 *   - Lattice units: unit time step and spacing, p = rho T, gamma given,
 *     Cv = 1/(gamma - 1), total polyatomic energy rho E = rho |u|^2 / 2 + rho Cv T.
 *   - Numerical failures never trap: a node whose root finder fails is left
 *     uncollided and counted; a failed rebuild falls back to the exponential
 *     of the Maxwellian guess and is counted; the step returns ALB_ENEWTON
 *     only from alb_sync/alb_stats once the counters show failures.
 */
#ifndef ALB_H
#define ALB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALB_VERSION 1

/* return codes */
#define ALB_OK 0
#define ALB_EINVAL (-1)         /* bad argument or configuration */
#define ALB_ENOMEM (-2)         /* device or host allocation failed, or over budget */
#define ALB_EUNSUPPORTED (-3)   /* stencil / option not supported */
#define ALB_ENEWTON (-4)        /* >= 1 node failed to converge; state valid, flagged */
#define ALB_EUNREALIZABLE (-5)  /* rho <= 0 or T <= 0 in initial fields */
#define ALB_ETIMEDOUT (-6)      /* bounded wait expired */
#define ALB_EBUSY (-7)          /* resource in use */
#define ALB_ECUDA (-8)          /* CUDA runtime error (message in alb_last_error) */
#define ALB_ENOTFOUND (-9)      /* unknown request id */

enum { ALB_D2Q21 = 21, ALB_D2Q49 = 49 };
enum { ALB_FP64_PLAIN = 0, ALB_FP32_FORM = 1 };
enum { ALB_PERIODIC = 0, ALB_ZERO_GRADIENT = 1 };
enum { ALB_HOST = 0, ALB_DEVICE = 1 };
enum { ALB_START_AUTO = 0, ALB_START_MAXWELLIAN = 1, ALB_START_PREVIOUS = 2 };
enum { ALB_RULE_HISTORY = 0, ALB_RULE_NEIGHBOURS = 1 };

typedef struct alb_handle alb_handle; /* opaque */

/* Configuration of one flow.
 *   nx, ny       grid size (>= 1 each).
 *   stencil      ALB_D2Q21, the adaptive lattice of the paper; or ALB_D2Q49,
 *                the lattice {-3..3}^2 of its reference solver (App. C.1,
 *                Sec. IV.B) with moments = 13, ALB_FP64_PLAIN, Maxwellian
 *                starts, one flow per handle (no batches, no server); the
 *                step is the same adaptive algorithm. D2Q49 velocity
 *                (x, y) has index (x + 3) + 7 (y + 3).
 *   u_max        shift set {-u_max..u_max}^2, 0 <= u_max <= 3.
 *   nu           kinematic viscosity (>= 0); tau = 1/2 + nu/T.
 *   gamma        specific heat ratio gamma_r (> 1).
 *   n0           criterion offset: U = n iff n - n0 < u <= n + 1 - n0
 *                (0.5 gives Eq. criterion as printed).
 *   precision    ALB_FP64_PLAIN: populations, moments and arithmetic in FP64.
 *                ALB_FP32_FORM: populations and moment sums in FP32
 *                (compensated summation), FP64 only in the Newton solve.
 *   bc_x, bc_y   ALB_PERIODIC, or ALB_ZERO_GRADIENT (ghost nodes carry the
 *                nearest interior node's moments; pulls from them are rebuilt).
 *   sensor       1 enables tau <- tau * alpha(eps_Kn) (Eq. DeltaAvg). alpha is
 *                1 for eps <= sensor_eps[0], then continuous and piecewise
 *                linear in log10(eps) through (sensor_eps[1], sensor_alpha[0]),
 *                (sensor_eps[2], sensor_alpha[1]), (10 sensor_eps[2],
 *                sensor_alpha[2]), constant beyond (sensor_eps increasing).
 *   newton_tol   stop when max_k |G_k| / rho <= newton_tol (paper: 1e-12).
 *   newton_maxit iteration cap.
 *   newton_start starting point of each equilibrium solve: ALB_START_AUTO
 *                (the node's multipliers of the previous step in the FP32
 *                form, the Maxwellian in FP64 plain), ALB_START_MAXWELLIAN,
 *                or ALB_START_PREVIOUS (the node's, or for a rebuilt pull the
 *                sender's, multipliers of the previous step moved to the
 *                lattice of the solve; 8 more planes per buffer). The root is
 *                unique, so the start changes only the path and round-off;
 *                ALB_START_MAXWELLIAN follows the oracle's iteration.
 *   shift_overlap w in [0, 1]: each shift's range widened by w on both
 *                sides, U - n0 - w < u <= U + 1 - n0 + w, so that the ranges
 *                of neighbouring shifts overlap (Sec. III.A.2); 0 (the
 *                default) is Eq. criterion.
 *   moments      constraint set of the numerical equilibrium: 8 (Eqs.
 *                G0_8mom..G3yaa_8mom, the default) or 4 (the reduced model
 *                of App. C.2, Eq. feqNum_4Mom: mass, momentum and the energy
 *                trace; a 4x4 FP64 Newton in both precisions) on D2Q21; 13
 *                (Eqs. G0..G4yyaa: moments up to third order and the trace
 *                of the fourth, Eq. feqNum_13Mom with the x^3 monomial the
 *                printed exponent omits) on D2Q49.
 *   shift_rule   where ranges overlap: ALB_RULE_HISTORY keeps the node's
 *                current shift while its widened range holds u (else the
 *                criterion's shift); ALB_RULE_NEIGHBOURS takes, among the
 *                shifts whose widened range holds u, the one most of the
 *                eight surrounding nodes currently use (the criterion's
 *                shift unless another is used by strictly more).
 *   prandtl      Prandtl number Pr > 0. 1 (the default) is the BGK collision
 *                of Eq. coll. Otherwise the collision of App. E (Eqs. Shakhov,
 *                prandtlPoly) adds (1/tau - 1/tau_Pr) times a heat-flux term,
 *                tau_Pr = 1/2 + (nu/Pr)/T, q = 1/2 sum cbar (|cbar|^2 f + g)
 *                of the pre-collision populations; Grad's heat flux (Eq.
 *                GradGeneral_f) takes kappa = rho Cp nu / Pr, and a rebuilt
 *                pull is that collision applied to the Grad population. The
 *                sensor factor scales tau and tau_Pr alike.
 *   stream       cudaStream_t to work on; NULL: the library creates one. */
typedef struct {
  int nx, ny;
  int stencil;
  int u_max;
  double nu;
  double gamma;
  double n0;
  int precision;
  int bc_x, bc_y;
  int sensor;
  double sensor_eps[3];
  double sensor_alpha[3];
  double newton_tol;
  int newton_maxit;
  int newton_start;
  double shift_overlap;
  int shift_rule;
  int moments;
  double prandtl;
  void* stream;
} alb_config;

/* Counters accumulated since alb_init. */
typedef struct {
  uint64_t steps;
  uint64_t node_updates;
  uint64_t newton_iterations;       /* FP64 Newton steps, node and rebuild equilibria */
  uint64_t newton_failures;         /* node equilibria that failed */
  uint64_t reconstructions;         /* missing pulls rebuilt (Grad) */
  uint64_t reconstruction_failures; /* rebuilds that fell back */
  uint64_t newton_calls;            /* equilibrium solves, node and rebuild */
  uint64_t fp64_evaluations;        /* FP64 evaluations of the 21 exponentials */
  uint64_t fp32_iterations;         /* FP32 Newton steps (FP32 form) */
  uint64_t fp64_updates;            /* FP32 form: residual evaluations that updated
                                       the 21 FP64 populations multiplicatively
                                       after a small step instead of evaluating
                                       the exponentials (not in fp64_evaluations) */
} alb_stats;

/* Fill *cfg with defaults: 64x64, D2Q21, u_max 2, nu 1e-3, gamma 1.4,
 * n0 0.5, FP64 plain, periodic, sensor off (eps 0.01/0.1/1, alpha
 * 1.05/1.35/1.6), tol 1e-12, 50 iterations, ALB_START_AUTO, no range
 * overlap, 8 moments, Pr 1, library stream. */
int alb_config_default(alb_config* cfg);

/* Create a flow: validates cfg and allocates two buffers of 42 population
 * planes, lattice planes and moment planes on the current device. */
int alb_create(const alb_config* cfg, alb_handle** out);

/* Grad-regularised initial state h = h^eq (1 + phi_h) (Sec. IV.A.1, IV.C)
 * from conserved fields rho, rho ux, rho uy, rho E; the lattice of each node
 * is chosen by Eq. criterion from the initial velocity, gradients by central
 * differences. The first collision is applied, so the state is ready to pull.
 * ALB_EUNREALIZABLE if some rho <= 0 or T <= 0 (checked on the device). */
int alb_init(alb_handle* h, const double* rho, const double* rhoux, const double* rhouy,
             const double* rhoE, int where);

/* Enqueue nsteps time iterations on the handle's stream; returns after
 * enqueueing (nsteps >= 0). */
int alb_step(alb_handle* h, int nsteps);

/* Wait for the handle's stream, at most timeout_ms milliseconds (< 0: no
 * limit). ALB_ETIMEDOUT if the work is still running; ALB_ENEWTON if failure
 * counters are non-zero. */
int alb_sync(alb_handle* h, int timeout_ms);

/* Conserved moments (rho, rho ux, rho uy, rho E) of the current populations. */
int alb_moments(alb_handle* h, double* rho, double* rhoux, double* rhouy, double* rhoE,
                int where);

/* Lattice shift (U_x, U_y) of the current populations, one byte each per node. */
int alb_shifts(alb_handle* h, signed char* ux, signed char* uy, int where);

/* Lattice shift selected for the next pull (Eq. criterion applied at the
 * last collision), one byte each per node. */
int alb_next_shifts(alb_handle* h, signed char* ux, signed char* uy, int where);

/* Post-collision populations of the current state as FP64 planes:
 * f[i * n + k], g[i * n + k] for velocity i (order of
 * alb_stencil_velocities) and node k = y * nx + x, n = nx * ny; 21 planes
 * each (49 on D2Q49). They live in the lattice of alb_shifts. */
int alb_populations(alb_handle* h, double* f, double* g, int where);

/* Primitive moments stored with the current state (rho, u_x, u_y, T; the
 * values the next step's rebuilds read), as FP64 arrays of n. */
int alb_primitives(alb_handle* h, double* rho, double* ux, double* uy, double* T, int where);

/* Checkpoint / restart. alb_checkpoint_size gives the bytes of an image of
 * the whole flow state (populations, moments, lattices, stored multipliers,
 * counters, step count, and a header naming the configuration);
 * alb_checkpoint_save writes it to host memory buf (synchronises);
 * alb_checkpoint_load restores it into a flow of the same grid, precision,
 * start option, u_max and boundaries (ALB_EINVAL otherwise). Continuing
 * from a loaded image gives the same results bit for bit as continuing
 * the saved flow. The paper has no counterpart. */
int alb_checkpoint_size(alb_handle* h, size_t* bytes);
int alb_checkpoint_save(alb_handle* h, void* buf);
int alb_checkpoint_load(alb_handle* h, const void* buf);

/* Global totals of the current state: out[0..3] = sum over nodes of rho,
 * rho ux, rho uy, rho E (host memory, 4 doubles). Mass, momentum and total
 * energy are the invariants of the collision (Eqs. G0_8mom..G2yy_8mom with
 * Eq. polyTemp); streaming preserves them except where pulls are rebuilt
 * (Sec. III.B). Deterministic: a fixed chunking of the nodes and a fixed
 * summation order, independent of the launch configuration. Synchronises the
 * handle's stream. */
int alb_totals(alb_handle* h, double* out);

/* Global totals without any allocation, for callers that cannot allocate
 * device memory (for example code that runs while another component owns
 * every allocation, or a context where cudaMalloc is not allowed). The paper
 * has no counterpart: this is a service of the library, not a step of the
 * method.
 *   rho, rhoux, rhouy, rhoE: device arrays of n doubles each (conserved
 *       fields, e.g. from alb_moments(..., ALB_DEVICE)), read only.
 *   n:   number of nodes, 0 <= n <= 268,435,456 (4096 chunks of 65536);
 *        larger n returns ALB_EINVAL and launches nothing.
 *   out: device array of 4 doubles, receives the sums of the four fields.
 *   stream: cudaStream_t (NULL: the legacy default stream); asynchronous.
 * The partial sums live in a 128 KB static device array that every GPU that
 * loads the library holds until the process exits; nothing is allocated or
 * freed. Every call looks up the array's device address on the current
 * device (a host-side query, so a device reset between calls is harmless); the
 * first call on a device may load the library's device code there: make that
 * first call before any stream capture.
 * Calls share the array: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong sums; serialise them. Each call writes every
 * partial it reads, so no state carries over between calls. Same chunking
 * and summation order as alb_totals. */
int alb_totals_noalloc(const double* rho, const double* rhoux, const double* rhouy,
                       const double* rhoE, long long n, double* out, void* stream);

/* Counters (synchronises the handle's stream). */
int alb_stats_get(alb_handle* h, alb_stats* out);

/* Free everything the handle owns (synchronises first). */
int alb_destroy(alb_handle* h);

/* Message of the last error on the calling thread ("" if none). */
const char* alb_last_error(void);

/* ------------------------------------------------------------------------
 * Stateless device entry points (device pointers, current device, stream
 * may be NULL for the legacy default stream). */

/* Numerical equilibrium (Eqs. exponential, feqNum_8Mom, constraints
 * G0_8mom..G3yaa_8mom) of n states given in the lattice frame: rho[k],
 * relative velocity (ubx[k], uby[k]) and T[k]; stop at max|G|/rho <= tol.
 * precision selects the solver of the step kernels: ALB_FP64_PLAIN, damped
 * Newton in FP64; ALB_FP32_FORM, Newton in FP32 refined with FP64 residuals
 * (full FP64 Newton if that fails). Writes feq[k*21 + i] (velocity order of
 * alb_velocities), lambda[k*8 + j] if lambda != NULL (order 0, x, y, xx, xy,
 * yy, x|xi|^2, y|xi|^2), iters[k] (FP64 Newton steps, or FP64 residual
 * evaluations, full and multiplicative, for ALB_FP32_FORM; the latter's
 * populations are exponential-family members to about 1e-10 relative, their
 * constraint residuals exact FP64 sums) and status[k] (0 converged, 1 not
 * converged, 2 singular / non-finite, 3 unrealizable input) if non-NULL. */
int alb_equilibrium(const double* rho, const double* ubx, const double* uby, const double* T,
                    int n, double tol, int maxit, int precision, double* feq, double* lambda,
                    int* iters, int* status, void* stream);

/* out[k] = exp(-s[k]) by the table-driven FP64 exponential of the FP64
 * Newton (Tang's method: 256-entry table of 2^(j/256), two-part reduction,
 * degree-4 polynomial on |r| <= ln2/512). 0 below 2^-1022, +inf from 2^1024
 * on. Device arrays of n doubles. Exposed so that its accuracy can be
 * checked. */
int alb_exp_neg(const double* s, int n, double* out, void* stream);

/* The same with the cheaper variant of the FP32 form's FP64 residual
 * evaluations: table index from an FP32 copy of s, one-step reduction and
 * degree-2 polynomial, relative error below 5e-10 for |s| <= 700 (the
 * residuals are summed over the values it returns, so the 1e-12 criterion
 * does not depend on it). Same arguments and limits. */
int alb_exp_neg_refine(const double* s, int n, double* out, void* stream);

/* Shift criterion (Eq. criterion with offset n0, clamped to +-u_max) applied
 * to u[k] = rhou[k] / rho[k] in FP64 for n values; writes out[k]. */
int alb_select_shift(const double* rho, const double* rhou, int n, double n0, int u_max,
                     signed char* out, void* stream);

/* D2Q21 velocity table used by every entry point (host memory, 21 each). */
int alb_velocities(int* xi_x, int* xi_y);

/* Velocity table of a stencil (ALB_D2Q21: 21 entries, ALB_D2Q49: 49) into
 * host arrays; ALB_EUNSUPPORTED for another stencil. */
int alb_stencil_velocities(int stencil, int* xi_x, int* xi_y);

/* The reference solver's equilibrium (App. C.1) on D2Q49 for n states in the
 * lattice frame, FP64 damped Newton on the 13 multipliers (order 1, x, y,
 * xx, xy, yy, xxx, xxy, xyy, yyy, xx|xi|^2, xy|xi|^2, yy|xi|^2), stop at
 * max|G|/rho <= tol. Device arrays: feq[k*49 + i], lambda[k*13 + j],
 * iters[k], status[k] (codes of alb_equilibrium); all required. */
int alb_equilibrium13(const double* rho, const double* ubx, const double* uby, const double* T,
                      int n, double tol, int maxit, double* feq, double* lambda, int* iters,
                      int* status, void* stream);

/* ------------------------------------------------------------------------
 * Batched flows. Many independent flows, each with its own grid size and
 * parameters, advance together: one persistent kernel launch per time step
 * and precision walks a table of work items (a tile of one flow each), and
 * two steps are replayed as one CUDA graph. A node's update is the same code
 * as in alb_step and reads only its own flow's state, so a flow's results
 * do not depend on the batch it runs in, on the tile shape or on the kernel
 * variant. The paper has no counterpart: it describes one flow at a time. */
typedef struct alb_batch alb_batch; /* opaque */

/* Launch shape of the batched kernel for one precision.
 *   variant        compiled kernel variant: index into alb_batch_variants
 *                  (block size and minimum resident blocks per SM, which
 *                  bounds the registers per thread).
 *   tile_w[3]      tile width in nodes for flows with nx < 128, with
 *                  nx < 512, and wider; the tile height is block / tile_w.
 *                  Powers of two in [8, block].
 *   dynamic        1: blocks fetch work items from an atomic counter;
 *                  0: block b takes items b, b + grid, b + 2 grid, ...
 *   blocks_per_sm  resident blocks per SM of the persistent grid (0: the
 *                  occupancy maximum; larger values are capped by it). */
typedef struct {
  int variant;
  int tile_w[3];
  int dynamic;
  int blocks_per_sm;
} alb_batch_tuning;

/* Compiled variants of a precision: *count (at most 8) and, if non-NULL,
 * block[v] and min_blocks[v] for each. */
int alb_batch_variants(int precision, int* count, int* block, int* min_blocks);

/* Create nflows (>= 1) flows from cfgs[0..nflows-1] (any mix of sizes,
 * parameters and precisions; each cfg's stream is ignored). All work runs on
 * `stream` (cudaStream_t; NULL: the batch creates one; not the legacy
 * default stream, which cannot be captured). Default launch shape: variant
 * 0, tiles of 64 / 128 / 128 nodes (at most the block), dynamic items. */
int alb_batch_create(const alb_config* cfgs, int nflows, void* stream, alb_batch** out);

/* Handle of flow i (0 <= i < nflows), owned by the batch: use it with
 * alb_init (required before the first alb_batch_step), alb_moments,
 * alb_shifts, alb_totals, alb_stats_get, alb_sync and alb_step (which steps
 * that flow alone); alb_destroy refuses it (ALB_EINVAL). */
int alb_batch_flow(alb_batch* b, int i, alb_handle** out);

/* Enqueue nsteps time steps of every flow (all must be initialised) on the
 * batch's stream: nsteps / 2 replays of a two-step CUDA graph, then one more
 * step if nsteps is odd. Returns after enqueueing. The first call after
 * creation or a tuning change captures the graph. */
int alb_batch_step(alb_batch* b, int nsteps);

/* Wait for the batch's stream (alb_sync on every flow; timeout_ms as there). */
int alb_batch_sync(alb_batch* b, int timeout_ms);

/* Autotuner: for each precision present, time the kernel variants, then the
 * tile width of each size class of flows present (timing that class's items
 * alone), then static against dynamic work distribution, with `trials`
 * timed launches (>= 1) per candidate, and keep the fastest. Every timed
 * launch reads the current state and writes only the spare buffers, and the
 * flows' counters are restored, so the flows do not advance. Flows must be
 * initialised. Synchronises the stream. */
int alb_batch_tune(alb_batch* b, int trials);

/* Read or set the launch shape of one precision (set: ALB_EINVAL if the
 * shape is invalid; synchronises the stream). */
int alb_batch_get_tuning(alb_batch* b, int precision, alb_batch_tuning* t);
int alb_batch_set_tuning(alb_batch* b, int precision, const alb_batch_tuning* t);

/* Free the batch and all its flows (synchronises first). */
int alb_batch_destroy(alb_batch* b);

/* ------------------------------------------------------------------------
 * Serving loop. A server owns two threads and two streams. Requests (a
 * flow configuration, its initial fields and a step count) queue as they
 * are submitted. The admission thread takes the queued request of least
 * estimated work (nodes x steps x the measured time of a node update of its
 * precision) that fits the device-memory budget, while the resident flows
 * hold fewer than 2 batch_nodes nodes, and creates and Grad-initialises its
 * flow on its own stream, overlapping the stepping. The worker thread
 * advances the resident flows in chunks of steps with the batched kernel of
 * alb_batch_step (least remaining work first, up to batch_nodes nodes per
 * chunk; each flow for exactly its remaining steps), so requests that
 * arrive while others run join at the next chunk. A finished flow's moments
 * go to host memory and its device memory is freed. Results are identical to
 * those of the same request run alone through alb_step. Under sustained
 * overload, requests of large work wait for as long as smaller ones keep
 * arriving. The paper has no counterpart: this is a service of the library.
 */
typedef struct alb_server alb_server; /* opaque */

/* Server settings.
 *   hbm_fraction  admission budget as a fraction of the device's total
 *                 memory (0 < f <= 1; 0.8 by default), capped by the memory
 *                 free at creation minus 1 GiB.
 *   chunk_ms      target duration of a chunk of steps (> 0; 100 by
 *                 default); the worker sizes chunks from the previous one.
 *   max_chunk     most steps in one chunk (>= 1; 256 by default).
 *   max_flows     most resident flows (0: no limit).
 *   batch_nodes   nodes stepped per chunk at most (0: every resident flow
 *                 steps in every chunk; 2^22 by default). Resident flows are
 *                 ranked by remaining work (nodes x steps left x the measured
 *                 time of a node update of their precision), least first,
 *                 and taken in that order until their nodes reach
 *                 batch_nodes (at least one flow per chunk).
 *   tune          1: run alb_batch_tune's search once on the first chunk
 *                 that holds flows of a precision (0 by default). */
typedef struct {
  double hbm_fraction;
  double chunk_ms;
  int max_chunk;
  int max_flows;
  long long batch_nodes;
  int tune;
} alb_server_config;

/* Producer of a request's initial fields, called on the worker thread when
 * the request is admitted: fill rho, rho ux, rho uy, rho E (host arrays of
 * nx*ny doubles, x fastest) and return 0, or non-zero to fail the request. */
typedef int (*alb_fill_fn)(void* user, double* rho, double* rhoux, double* rhouy, double* rhoE);

/* A request. cfg: the flow (its stream is ignored). nsteps >= 0.
 * Initial fields: either host arrays rho..rhoE (copied by alb_submit), or,
 * with those NULL, fill(user, ...) at admission (user must stay valid until
 * then). keep_result: 1 keeps the final moments in host memory until
 * alb_poll collects them; 0 keeps only the status and times. */
typedef struct {
  alb_config cfg;
  int nsteps;
  const double* rho;
  const double* rhoux;
  const double* rhouy;
  const double* rhoE;
  alb_fill_fn fill;
  void* user;
  int keep_result;
} alb_request;

enum { ALB_QUEUED = 0, ALB_RUNNING = 1, ALB_DONE = 2, ALB_FAILED = 3 };

/* Outcome of a request. The caller sets rho..rhoE to host arrays of nx*ny
 * doubles to receive the final moments (NULL: not copied; ignored unless
 * keep_result was 1). Times are seconds since the server's creation. */
typedef struct {
  double* rho;
  double* rhoux;
  double* rhouy;
  double* rhoE;
  int status;         /* ALB_OK, or the error that failed or flagged the request */
  uint64_t steps;     /* steps taken */
  alb_stats stats;    /* the flow's counters at completion */
  double t_submit, t_admit, t_done;
} alb_result;

/* Aggregate counters of a server. */
typedef struct {
  uint64_t submitted, admitted, completed, failed;
  uint64_t queued, running;
  uint64_t node_updates;       /* node updates of all chunks so far */
  uint64_t chunks, steps;      /* chunks run, and batched steps within them */
  uint64_t resident_bytes;     /* device memory of the resident flows */
  uint64_t budget_bytes;       /* admission budget */
  double busy_seconds;         /* wall time spent running chunks */
  double elapsed_seconds;      /* since creation */
  double ns_per_update[2];     /* measured time of one node update, [0] FP64
                                  plain, [1] FP32 form (smoothed over chunks) */
} alb_server_stats;

/* Fill *c with the defaults above. */
int alb_server_config_default(alb_server_config* c);
/* Create a server on the current device (starts its worker thread). */
int alb_server_create(const alb_server_config* c, alb_server** out);
/* Queue a request; *id identifies it. ALB_EINVAL for a bad request,
 * ALB_ENOMEM if the flow alone exceeds the budget (nothing queued). */
int alb_submit(alb_server* s, const alb_request* r, uint64_t* id);
/* Non-blocking state of request id (*state one of ALB_QUEUED .. ALB_FAILED).
 * Once it is DONE or FAILED the call fills *res (if non-NULL) and forgets
 * the request: a later poll of that id gives ALB_ENOTFOUND. */
int alb_poll(alb_server* s, uint64_t id, int* state, alb_result* res);
/* Block until no request is queued or running, at most timeout_ms (< 0: no
 * limit); ALB_ETIMEDOUT otherwise. */
int alb_server_drain(alb_server* s, int timeout_ms);
int alb_server_stats_get(alb_server* s, alb_server_stats* out);
/* Stop the worker after its current chunk and free everything; requests
 * still queued or running are dropped. */
int alb_server_destroy(alb_server* s);

#ifdef __cplusplus
}
#endif
#endif /* ALB_H */
