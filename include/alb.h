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

enum { ALB_D2Q21 = 21 };
enum { ALB_FP64_PLAIN = 0, ALB_FP32_FORM = 1 };
enum { ALB_PERIODIC = 0, ALB_ZERO_GRADIENT = 1 };
enum { ALB_HOST = 0, ALB_DEVICE = 1 };

typedef struct alb_handle alb_handle; /* opaque */

/* Configuration of one flow.
 *   nx, ny       grid size (>= 1 each).
 *   stencil      ALB_D2Q21 (only one supported).
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
} alb_stats;

/* Fill *cfg with defaults: 64x64, D2Q21, u_max 2, nu 1e-3, gamma 1.4,
 * n0 0.5, FP64 plain, periodic, sensor off (eps 0.01/0.1/1, alpha
 * 1.05/1.35/1.6), tol 1e-12, 50 iterations, library stream. */
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
 * freed. The first call on a device looks up the array's device address with
 * that device current: make that first call before any stream capture.
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
 * evaluations for ALB_FP32_FORM) and status[k] (0 converged, 1 not
 * converged, 2 singular / non-finite, 3 unrealizable input) if non-NULL. */
int alb_equilibrium(const double* rho, const double* ubx, const double* uby, const double* T,
                    int n, double tol, int maxit, int precision, double* feq, double* lambda,
                    int* iters, int* status, void* stream);

/* out[k] = exp(-s[k]) by the table-driven FP64 exponential that the FP32
 * form's equilibrium uses (Tang's method: 32-entry table of 2^(j/32), degree-6
 * polynomial on |r| <= ln2/64). 0 below 2^-1022, +inf from 2^1024 on. Device
 * arrays of n doubles. Exposed so that its accuracy can be checked. */
int alb_exp_neg(const double* s, int n, double* out, void* stream);

/* Shift criterion (Eq. criterion with offset n0, clamped to +-u_max) applied
 * to u[k] = rhou[k] / rho[k] in FP64 for n values; writes out[k]. */
int alb_select_shift(const double* rho, const double* rhou, int n, double n0, int u_max,
                     signed char* out, void* stream);

/* D2Q21 velocity table used by every entry point (host memory, 21 each). */
int alb_velocities(int* xi_x, int* xi_y);

#ifdef __cplusplus
}
#endif
#endif /* ALB_H */
