/*
 * Plain FP64 CPU oracle of the interpolation-free state-adaptive D2Q21 lattice
 * Boltzmann method (Coreixas & Latt, arXiv:2009.13426).
 *
 * TEST INFRASTRUCTURE ONLY. This code is the slow, obviously-correct reference
 * that the CUDA path is checked against. Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it. The product library never
 * links, loads or calls it, and it shares no code with the CUDA path.
 *
 * Everything is double precision. One time step is two full passes over the
 * grid, in the order of the algorithm overview of Sec. IV.A.3:
 *   (i)  per node: moments (Eq. polyTemp), numerical equilibrium (Eq. feqNum_8Mom
 *        with the 8 constraints G0_8mom..G3yaa_8mom), g^eq (Eq. gEq), optional
 *        kinetic sensor (Eq. DeltaAvg), BGK collision (Eq. coll), and the shift
 *        U' for the next pull (Eq. criterion);
 *   (ii) per node and velocity: pull streaming (Eq. stream) from x - (xi_i + U'(x));
 *        a pull whose sender lives in another lattice is rebuilt by Grad's
 *        reconstruction (Eqs. GradGeneral, GradGeneral_f, GradGeneral_g) with
 *        second-order central differences of u and T at the sender.
 *
 * Every function here is pinned by tests/test_oracle_*.py against what the
 * paper and the mathematics fix (closed forms, exact rational arithmetic,
 * Gauss-Hermite moments, the paper's printed values, an exact Riemann
 * solver); none is unpinned.
 */
#ifndef ALB_ORACLE_H
#define ALB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_Q 21    /* D2Q21 */
#define ORA_M 8     /* 8-moment constraint set */
#define ORA_Q49 49  /* D2Q49, the reference solver's lattice (App. C.1) */
#define ORA_M13 13  /* its 13-moment constraint set */
#define ORA_QMAX 49

/* Stencils (ora_config.stencil): the adaptive D2Q21 lattice, or the D2Q49
 * lattice {-3..3}^2 with the 13-moment equilibrium of App. C.1 (Eqs. G0..G4yyaa,
 * feqNum_13Mom) that the paper uses for its reference data. D2Q49 velocity
 * i = (x, y) has index i = (x + 3) + 7 (y + 3). */
enum { ORA_D2Q21 = 21, ORA_D2Q49 = 49 };

enum { ORA_PERIODIC = 0, ORA_ZERO_GRADIENT = 1 };

enum {
  ORA_OK = 0,
  ORA_ENEWTON = 1,       /* root finder did not reach the tolerance */
  ORA_ESINGULAR = 2,     /* Jacobian not positive definite / non-finite values */
  ORA_EUNREALIZABLE = 3, /* rho <= 0 or T <= 0 */
  ORA_EINVAL = 4
};

typedef struct {
  int nx, ny;
  int umax;            /* shift set {-umax..umax}^2 */
  double nu;           /* kinematic viscosity (lattice units) */
  double gamma;        /* specific heat ratio gamma_r */
  double n0;           /* criterion offset: U = n iff n - n0 < u <= n + 1 - n0 */
  int bc_x, bc_y;      /* ORA_PERIODIC | ORA_ZERO_GRADIENT */
  int sensor;          /* 1: tau <- tau * alpha(eps_Kn) (Eq. DeltaAvg) */
  double sensor_eps[3];   /* increasing knots e0 < e1 < e2 of eps_Kn */
  double sensor_alpha[3]; /* alpha at e1, e2 and 10 e2 (alpha = 1 up to e0) */
  double newton_tol;   /* max_k |G_k| / rho */
  int newton_maxit;
  double overlap;      /* w in [0, 1]: each shift's range widened by w on both sides,
                          so that ranges overlap (Sec. III.A.2); 0 = Eq. criterion */
  int overlap_rule;    /* where ranges overlap: ORA_RULE_HISTORY keeps the node's shift,
                          ORA_RULE_NEIGHBOURS takes the one most neighbours use */
  int moments;         /* constraint set of the equilibrium: 8 (Eqs. G0_8mom..G3yaa_8mom,
                          the default) or 4 (the reduced model, App. C.2) */
  double prandtl;      /* Pr > 0. 1: BGK (Eq. coll). Otherwise the heat-flux
                          corrected collision of App. E (Eqs. Shakhov, prandtlPoly)
                          with tau_Pr = 1/2 + (nu/Pr)/T, and kappa = rho Cp nu / Pr in
                          Grad's heat flux (Eq. GradGeneral_f) */
  int stencil;         /* ORA_D2Q21, or ORA_D2Q49 with moments = 13 */
} ora_config;

enum { ORA_RULE_HISTORY = 0, ORA_RULE_NEIGHBOURS = 1 };

typedef struct {
  long long newton_calls;
  long long newton_iters;
  long long newton_failures;      /* node equilibria that failed (node not collided) */
  long long reconstructions;      /* missing pulls rebuilt by Grad's formula */
  long long reconstruction_failures;
} ora_stats;

typedef struct ora_state ora_state;

/* Velocity table of a stencil (ORA_D2Q21 or ORA_D2Q49), in the index order used
 * everywhere in the oracle. */
void ora_velocities(int stencil, int* xi_x, int* xi_y);

/* Numerical equilibrium (Eqs. exponential, feqNum_8Mom) in a lattice whose
 * populations move with xi_i + U: (rho, ubx, uby) is the velocity relative to U.
 * Writes the 8 multipliers (order: 0, x, y, xx, xy, yy, x|xi|^2, y|xi|^2) and
 * f^eq_i. Returns ORA_OK or an error code; *iters receives the Newton count. */
int ora_equilibrium(double rho, double ubx, double uby, double T, double tol,
                    int maxit, double lambda[ORA_M], double feq[ORA_Q], int* iters);

/* Reduced model (App. C.2, Eq. feqNum_4Mom): the numerical equilibrium
 * f_i = rho exp[-(1 + l0 + l1x xi_x + l1y xi_y + l2 |xi|^2)] whose mass,
 * momentum and energy trace sum_i f xi_a xi_a = 2 rho E = rho (|ubar|^2 + D T)
 * (monatomic energy, D = 2) match the state; lambda order (0, x, y, |xi|^2).
 * Same damped Newton and stopping rule as ora_equilibrium. */
int ora_equilibrium4(double rho, double ubx, double uby, double T, double tol, int maxit,
                     double lambda[4], double feq[ORA_Q], int* iters);

/* Constraint targets M_k(rho, ubar, T) of Eqs. G0_8mom..G3yaa_8mom. */
void ora_targets(double rho, double ubx, double uby, double T, double m[ORA_M]);

/* Reference solver's equilibrium on D2Q49 (App. C.1): the 13 constraints of
 * Eqs. G0..G4yyaa (moments up to third order and the trace of the fourth,
 * 2E = |ubar|^2 + D T) and the exponential family of Eq. feqNum_13Mom with the
 * monomials (1, x, y, x^2, xy, y^2, x^3, x^2 y, x y^2, y^3, x^2 r^2, x y r^2,
 * y^2 r^2), r^2 = x^2 + y^2, in that order for lambda. Same iteration and
 * stopping rule as ora_equilibrium. */
int ora_equilibrium13(double rho, double ubx, double uby, double T, double tol, int maxit,
                      double lambda[ORA_M13], double feq[ORA_Q49], int* iters);

/* Targets of Eqs. G0..G4yyaa in the monomial order of ora_equilibrium13. */
void ora_targets13(double rho, double ubx, double uby, double T, double m[ORA_M13]);

/* Shift criterion (Eq. criterion, with the n0 offset reading). */
int ora_select_shift(double u, double n0, int umax);

/* Shift selection with overlapping ranges (Sec. III.A.2, ranges wider than 1
 * chosen by the node's history): keep `current` while
 * current - n0 - w < u <= current + 1 - n0 + w, else Eq. criterion. */
int ora_select_shift_kept(double u, double n0, int umax, int current, double w);

/* Shift selection with overlapping ranges chosen by the neighbourhood (Sec.
 * III.A.2, to reduce interface cells): among the shifts n in [-umax, umax]
 * whose widened range n - n0 - w < u <= n + 1 - n0 + w holds u, the one that
 * most of the nb[0..nnb-1] neighbour shifts equal; Eq. criterion's shift
 * unless another candidate is used by strictly more neighbours (candidates
 * examined in increasing n). */
int ora_select_shift_neighbours(double u, double n0, int umax, double w, const int* nb, int nnb);

/* Macroscopic moments of one node (Eq. polyTemp), Q = 21 or 49 populations in
 * lattice U. out = {rho, ux, uy, T} with u absolute (lattice-frame sums plus U). */
void ora_node_moments(int Q, const double* f, const double* g, int Ux, int Uy, double gamma,
                      double out[4]);

/* Collision of one node in its own lattice: BGK (Eqs. coll, gEq; optional
 * sensor) and, for Pr != 1, the heat-flux term of Eqs. Shakhov / prandtlPoly
 * with q the heat flux of the pre-collision populations (ora_heat_flux).
 * Arrays hold cfg->stencil populations. Returns ORA_OK or a Newton error
 * (then fs, gs = f, g). */
int ora_collide_node(const ora_config* cfg, const double* f, const double* g, int Ux, int Uy,
                     double* fs, double* gs);

/* Grad populations h = h^eq (1 + omega * phi_h + w_pr * phi_h,q) in lattice
 * (Ux, Uy) for the macroscopic state (rho, ux, uy, T) with velocity gradients
 * du[a][b] = d_a u_b and temperature gradient dT[a] (Eqs. GradGeneral,
 * GradGeneral_f, _g); phi_h,q is the heat-flux part of phi_h (all of phi_g).
 * omega = 1, w_pr = 0 for initial conditions; omega = 1 - 1/tau and
 * w_pr = 1/tau - 1/tau_Pr for post-collision rebuilds, which is the collision
 * of App. E applied to the Grad population with q its Fourier heat flux. */
int ora_grad_populations(const ora_config* cfg, int Ux, int Uy, double rho, double ux,
                         double uy, double T, const double du[2][2], const double dT[2],
                         double omega, double w_pr, double* f, double* g);

/* Heat flux of one node's Q = 21 or 49 populations in lattice U (the flux of
 * Eqs. Shakhov / prandtlPoly): q_a = 1/2 sum_i cbar_ia (|cbar_i|^2 f_i + g_i),
 * cbar_i = xi_i + U - u, with u the node's velocity (absolute). */
void ora_heat_flux(int Q, const double* f, const double* g, int Ux, int Uy, double ux,
                   double uy, double q[2]);

ora_state* ora_create(const ora_config* cfg);
void ora_destroy(ora_state* s);

/* Grad-regularised initial state from conserved fields (x fastest, nx*ny each):
 * rho, rho*ux, rho*uy, rho*E with rho*E = rho|u|^2/2 + rho*Cv*T. */
int ora_init(ora_state* s, const double* rho, const double* rhoux, const double* rhouy,
             const double* rhoE);

/* Advance nsteps time iterations. Returns ORA_OK, or ORA_ENEWTON if any node
 * failed (state stays valid, failures are counted). */
int ora_step(ora_state* s, int nsteps);

/* One time iteration in which the lattice each node pulls into is given
 * (ux, uy: nx*ny shifts within +-umax) instead of chosen by Eq. criterion;
 * everything else as ora_step. Replays lattice decisions recorded from
 * another implementation, so that arithmetic differences can be compared
 * without the discontinuity of a threshold decision taken differently. */
int ora_step_forced(ora_state* s, const signed char* ux, const signed char* uy);

/* Conserved moments of the current (pre-collision) populations. */
void ora_get_moments(const ora_state* s, double* rho, double* rhoux, double* rhouy,
                     double* rhoE);
/* Primitive moments (rho, ux, uy, T) of the current populations. */
void ora_get_primitives(const ora_state* s, double* rho, double* ux, double* uy, double* T);
/* Lattice of the current populations. */
void ora_get_shifts(const ora_state* s, signed char* ux, signed char* uy);
/* Populations, layout [node][i]. */
void ora_get_populations(const ora_state* s, double* f, double* g);
void ora_set_state(ora_state* s, const double* f, const double* g, const signed char* ux,
                   const signed char* uy);
void ora_get_stats(const ora_state* s, ora_stats* out);

#ifdef __cplusplus
}
#endif
#endif
