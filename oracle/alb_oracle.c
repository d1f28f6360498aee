/*
 * Plain FP64 CPU oracle of the interpolation-free state-adaptive D2Q21 LBM
 * (Coreixas & Latt, arXiv:2009.13426). TEST INFRASTRUCTURE ONLY: see the header.
 *
 * Written for readability against the paper, not for speed: populations are
 * stored node-major ([node][i]), every step makes two full passes, and nothing
 * is fused, blocked or reordered beyond the algorithm overview of Sec. IV.A.3.
 */
#include "alb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* D2Q21 velocity set. The paper takes it from Zhang et al. (Fig. 1, Fig. 11,
 * Tab. 3) without printing it; the reading used here is the rest velocity, the
 * 4 unit axis, 4 unit diagonal, 4 axis-2, 4 diagonal-2 and 4 axis-3 velocities. */
static const int XI[ORA_Q][2] = {
    {0, 0},
    {1, 0},  {0, 1},  {-1, 0},  {0, -1},
    {1, 1},  {-1, 1}, {-1, -1}, {1, -1},
    {2, 0},  {0, 2},  {-2, 0},  {0, -2},
    {2, 2},  {-2, 2}, {-2, -2}, {2, -2},
    {3, 0},  {0, 3},  {-3, 0},  {0, -3},
};

/* D2Q49: every integer velocity in {-3..3}^2, index (x + 3) + 7 (y + 3); the
 * lattice of the paper's reference solver (Sec. IV.B, App. C.1). */
#define ROW49(y) {-3, y}, {-2, y}, {-1, y}, {0, y}, {1, y}, {2, y}, {3, y}
static const int XI49[ORA_Q49][2] = {ROW49(-3), ROW49(-2), ROW49(-1), ROW49(0),
                                     ROW49(1),  ROW49(2),  ROW49(3)};
#undef ROW49

/* Velocity table of a stencil (Q = 21 or 49). */
static const int (*stencil_xi(int Q))[2] { return Q == ORA_Q49 ? XI49 : XI; }

static const double D_SPACE = 2.0; /* D = 2 spatial dimensions (Sec. C.1) */

struct ora_state {
  ora_config cfg;
  int n;
  int Q;                /* populations per node: 21 or 49 */
  const int (*xi)[2];   /* their velocities */
  double *f, *g;        /* pre-collision populations [node][i] */
  double *fs, *gs;      /* post-collision populations [node][i] */
  signed char *Ux, *Uy; /* lattice of f, g */
  signed char *Unx, *Uny; /* lattice selected for the next pull */
  double *rho, *ux, *uy, *T; /* moments of f, g at the current step */
  ora_stats stats;
};

void ora_velocities(int stencil, int* xi_x, int* xi_y) {
  const int Q = stencil == ORA_D2Q49 ? ORA_Q49 : ORA_Q;
  const int(*xi)[2] = stencil_xi(Q);
  for (int i = 0; i < Q; ++i) {
    xi_x[i] = xi[i][0];
    xi_y[i] = xi[i][1];
  }
}

/* Monomials of the 8-moment set (Eq. 8moments): 1, xi_a, xi_a xi_b, xi_a |xi|^2. */
static void monomials(int i, double P[ORA_M]) {
  const double x = XI[i][0], y = XI[i][1];
  const double r2 = x * x + y * y;
  P[0] = 1.0;
  P[1] = x;
  P[2] = y;
  P[3] = x * x;
  P[4] = x * y;
  P[5] = y * y;
  P[6] = x * r2;
  P[7] = y * r2;
}

/* Targets of Eqs. G0_8mom..G3yaa_8mom, written in the lattice frame: the
 * velocity is the one relative to the lattice shift, and 2E = |u|^2 + D T with
 * D = 2 (Sec. C.1), so 2 rho u_a (E + T) = rho u_a (|u|^2 + 4T). */
void ora_targets(double rho, double ubx, double uby, double T, double m[ORA_M]) {
  const double E = 0.5 * (ubx * ubx + uby * uby + D_SPACE * T);
  m[0] = rho;
  m[1] = rho * ubx;
  m[2] = rho * uby;
  m[3] = rho * (ubx * ubx + T);
  m[4] = rho * ubx * uby;
  m[5] = rho * (uby * uby + T);
  m[6] = 2.0 * rho * ubx * (E + T);
  m[7] = 2.0 * rho * uby * (E + T);
}

/* p_i = exp(-(1 + lambda . P(xi_i))), the equilibrium divided by rho (Eq. exponential, a = rho). */
static void exp_family(const double lambda[ORA_M], double p[ORA_Q]) {
  for (int i = 0; i < ORA_Q; ++i) {
    double P[ORA_M];
    monomials(i, P);
    double s = 1.0;
    for (int k = 0; k < ORA_M; ++k) s += lambda[k] * P[k];
    p[i] = exp(-s);
  }
}

/* Dual objective F(lambda) = sum_i p_i + lambda . m (per unit density). Its
 * gradient is -(G / rho) and its Hessian sum_i p_i P P^T, so Newton on G = 0 is
 * Newton on this strictly convex function. */
static double dual_value(const double lambda[ORA_M], const double p[ORA_Q], const double m[ORA_M]) {
  double F = 0.0;
  for (int i = 0; i < ORA_Q; ++i) F += p[i];
  for (int k = 0; k < ORA_M; ++k) F += lambda[k] * m[k];
  return F;
}

/* Cholesky solve of the symmetric positive definite system A x = b (A is 8x8). */
static int cholesky_solve(const double A[ORA_M][ORA_M], const double b[ORA_M], double x[ORA_M]) {
  double L[ORA_M][ORA_M];
  memset(L, 0, sizeof(L));
  for (int j = 0; j < ORA_M; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !isfinite(d)) return ORA_ESINGULAR;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < ORA_M; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  double y[ORA_M];
  for (int i = 0; i < ORA_M; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = ORA_M - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < ORA_M; ++k) s -= L[k][i] * x[k];
    x[i] = s / L[i][i];
  }
  return ORA_OK;
}

/* Maxwellian starting point: lambda_1 = -u/T, lambda_2aa = 1/(2T), the rest 0,
 * and lambda_0 fixed by the normalisation sum_i p_i = 1. */
static void maxwellian_guess(double ubx, double uby, double T, double lambda[ORA_M]) {
  for (int k = 0; k < ORA_M; ++k) lambda[k] = 0.0;
  lambda[1] = -ubx / T;
  lambda[2] = -uby / T;
  lambda[3] = 0.5 / T;
  lambda[5] = 0.5 / T;
  double p[ORA_Q];
  exp_family(lambda, p); /* with lambda_0 = 0: p_i = exp(-1 - ...) */
  double Z = 0.0;
  for (int i = 0; i < ORA_Q; ++i) Z += p[i];
  /* exp(-1 - lambda0 - rest) summed = 1  <=>  lambda0 = ln(Z) */
  lambda[0] = log(Z);
}

/* Root of G(lambda) = 0 (Sec. II.C.2, App. C): Newton's method on the
 * multipliers with the exact Jacobian, damped by backtracking on the convex
 * dual. The paper uses Powell's hybrid method; the root is unique, so any
 * convergent method yields the same equilibrium up to the tolerance. Stop when
 * max_k |G_k| / rho <= tol (the paper's criterion 1e-12). */
int ora_equilibrium(double rho, double ubx, double uby, double T, double tol, int maxit,
                    double lambda[ORA_M], double feq[ORA_Q], int* iters) {
  *iters = 0;
  if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ubx) ||
      !isfinite(uby))
    return ORA_EUNREALIZABLE;
  double m[ORA_M], mt[ORA_M];
  ora_targets(rho, ubx, uby, T, mt);
  for (int k = 0; k < ORA_M; ++k) m[k] = mt[k] / rho;

  maxwellian_guess(ubx, uby, T, lambda);
  double p[ORA_Q];
  exp_family(lambda, p);
  double F = dual_value(lambda, p, m);
  int status = ORA_ENEWTON;
  int it = 0;
  for (;;) {
    /* residual G / rho */
    double G[ORA_M];
    for (int k = 0; k < ORA_M; ++k) G[k] = -m[k];
    for (int i = 0; i < ORA_Q; ++i) {
      double P[ORA_M];
      monomials(i, P);
      for (int k = 0; k < ORA_M; ++k) G[k] += p[i] * P[k];
    }
    double gmax = 0.0;
    for (int k = 0; k < ORA_M; ++k) gmax = fmax(gmax, fabs(G[k]));
    if (!isfinite(gmax)) { status = ORA_ESINGULAR; break; }
    if (gmax <= tol) { status = ORA_OK; break; }
    if (it >= maxit) { status = ORA_ENEWTON; break; }
    /* Jacobian dG/d(-lambda) = sum_i p_i P P^T */
    double H[ORA_M][ORA_M];
    memset(H, 0, sizeof(H));
    for (int i = 0; i < ORA_Q; ++i) {
      double P[ORA_M];
      monomials(i, P);
      for (int a = 0; a < ORA_M; ++a)
        for (int b = 0; b < ORA_M; ++b) H[a][b] += p[i] * P[a] * P[b];
    }
    double d[ORA_M];
    if (cholesky_solve((const double(*)[ORA_M])H, G, d) != ORA_OK) { status = ORA_ESINGULAR; break; }
    double gd = 0.0;
    for (int k = 0; k < ORA_M; ++k) gd += G[k] * d[k];
    /* backtracking (Armijo) on F along lambda + t d */
    double t = 1.0, lam_c[ORA_M], p_c[ORA_Q], F_c = 0.0;
    int accepted = 0;
    for (int ls = 0; ls < 40; ++ls) {
      for (int k = 0; k < ORA_M; ++k) lam_c[k] = lambda[k] + t * d[k];
      exp_family(lam_c, p_c);
      F_c = dual_value(lam_c, p_c, m);
      if (isfinite(F_c) && F_c <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) { accepted = 1; break; }
      t *= 0.5;
    }
    ++it;
    if (!accepted) { status = ORA_ENEWTON; break; }
    for (int k = 0; k < ORA_M; ++k) lambda[k] = lam_c[k];
    for (int i = 0; i < ORA_Q; ++i) p[i] = p_c[i];
    F = F_c;
  }
  *iters = it;
  for (int i = 0; i < ORA_Q; ++i) feq[i] = rho * p[i];
  return status;
}

/* Reduced model (App. C.2): four constraints - mass, momentum and the
 * trace of the energy, sum_i f xi_a xi_a = 2 rho E with the monatomic energy
 * 2E = |ubar|^2 + D T - and the exponential family of Eq. feqNum_4Mom. The
 * iteration is ora_equilibrium's (Maxwellian start with lambda_0 from the
 * normalisation, Newton on the convex dual with Armijo backtracking, stop at
 * max_k |G_k| / rho <= tol) on four multipliers. */
static void exp_family4(const double l[4], double p[ORA_Q]) {
  for (int i = 0; i < ORA_Q; ++i) {
    const double x = XI[i][0], y = XI[i][1];
    p[i] = exp(-(1.0 + l[0] + l[1] * x + l[2] * y + l[3] * (x * x + y * y)));
  }
}

static double dual_value4(const double l[4], const double p[ORA_Q], const double m[4]) {
  double F = 0.0;
  for (int i = 0; i < ORA_Q; ++i) F += p[i];
  for (int k = 0; k < 4; ++k) F += l[k] * m[k];
  return F;
}

int ora_equilibrium4(double rho, double ubx, double uby, double T, double tol, int maxit,
                     double lambda[4], double feq[ORA_Q], int* iters) {
  *iters = 0;
  if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ubx) ||
      !isfinite(uby))
    return ORA_EUNREALIZABLE;
  const double m[4] = {1.0, ubx, uby, ubx * ubx + uby * uby + D_SPACE * T};
  /* Maxwellian start: l1 = -ubar/T, l2 = 1/(2T), l0 from sum p = 1 */
  lambda[0] = 0.0;
  lambda[1] = -ubx / T;
  lambda[2] = -uby / T;
  lambda[3] = 0.5 / T;
  double p[ORA_Q];
  exp_family4(lambda, p);
  double Z = 0.0;
  for (int i = 0; i < ORA_Q; ++i) Z += p[i];
  lambda[0] = log(Z);
  exp_family4(lambda, p);
  double F = dual_value4(lambda, p, m);
  int status = ORA_ENEWTON;
  int it = 0;
  for (;;) {
    double G[4] = {-m[0], -m[1], -m[2], -m[3]};
    double H[4][4];
    memset(H, 0, sizeof(H));
    for (int i = 0; i < ORA_Q; ++i) {
      const double x = XI[i][0], y = XI[i][1];
      const double P[4] = {1.0, x, y, x * x + y * y};
      for (int a = 0; a < 4; ++a) {
        G[a] += p[i] * P[a];
        for (int b = 0; b < 4; ++b) H[a][b] += p[i] * P[a] * P[b];
      }
    }
    double gmax = 0.0;
    for (int k = 0; k < 4; ++k) gmax = fmax(gmax, fabs(G[k]));
    if (!isfinite(gmax)) { status = ORA_ESINGULAR; break; }
    if (gmax <= tol) { status = ORA_OK; break; }
    if (it >= maxit) { status = ORA_ENEWTON; break; }
    /* Cholesky solve H d = G */
    double L[4][4], y[4], d[4];
    memset(L, 0, sizeof(L));
    int ok = 1;
    for (int j = 0; j < 4 && ok; ++j) {
      double s = H[j][j];
      for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
      if (!(s > 0.0) || !isfinite(s)) { ok = 0; break; }
      L[j][j] = sqrt(s);
      for (int i = j + 1; i < 4; ++i) {
        double t = H[i][j];
        for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
        L[i][j] = t / L[j][j];
      }
    }
    if (!ok) { status = ORA_ESINGULAR; break; }
    for (int i = 0; i < 4; ++i) {
      double s = G[i];
      for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
      y[i] = s / L[i][i];
    }
    for (int i = 3; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < 4; ++k) s -= L[k][i] * d[k];
      d[i] = s / L[i][i];
    }
    double gd = 0.0;
    for (int k = 0; k < 4; ++k) gd += G[k] * d[k];
    double t = 1.0, lam_c[4], p_c[ORA_Q], F_c = 0.0;
    int accepted = 0;
    for (int ls = 0; ls < 40; ++ls) {
      for (int k = 0; k < 4; ++k) lam_c[k] = lambda[k] + t * d[k];
      exp_family4(lam_c, p_c);
      F_c = dual_value4(lam_c, p_c, m);
      if (isfinite(F_c) && F_c <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) { accepted = 1; break; }
      t *= 0.5;
    }
    ++it;
    if (!accepted) { status = ORA_ENEWTON; break; }
    for (int k = 0; k < 4; ++k) lambda[k] = lam_c[k];
    for (int i = 0; i < ORA_Q; ++i) p[i] = p_c[i];
    F = F_c;
  }
  *iters = it;
  for (int i = 0; i < ORA_Q; ++i) feq[i] = rho * p[i];
  return status;
}

/* ------------------------------------------------------------------------- */
/* The reference solver's equilibrium (App. C.1) on D2Q49. */

/* Monomials of Eq. feqNum_13Mom. The printed exponent lists nine of the ten
 * monomials up to third order (lambda_3,xxx x^3 is missing) for thirteen
 * constraints; the square system needs all of them, so x^3 is included. */
static void monomials13(double x, double y, double P[ORA_M13]) {
  const double r2 = x * x + y * y;
  P[0] = 1.0;
  P[1] = x;
  P[2] = y;
  P[3] = x * x;
  P[4] = x * y;
  P[5] = y * y;
  P[6] = x * x * x;
  P[7] = x * x * y;
  P[8] = x * y * y;
  P[9] = y * y * y;
  P[10] = x * x * r2;
  P[11] = x * y * r2;
  P[12] = y * y * r2;
}

/* Eqs. G0..G4yyaa in the lattice frame, 2E = |u|^2 + D T. */
void ora_targets13(double rho, double ubx, double uby, double T, double m[ORA_M13]) {
  const double E = 0.5 * (ubx * ubx + uby * uby + D_SPACE * T);
  m[0] = rho;
  m[1] = rho * ubx;
  m[2] = rho * uby;
  m[3] = rho * (ubx * ubx + T);
  m[4] = rho * ubx * uby;
  m[5] = rho * (uby * uby + T);
  m[6] = rho * ubx * (ubx * ubx + 3.0 * T);
  m[7] = rho * (ubx * ubx + T) * uby;
  m[8] = rho * ubx * (uby * uby + T);
  m[9] = rho * uby * (uby * uby + 3.0 * T);
  m[10] = 2.0 * rho * ((E + 2.0 * T) * ubx * ubx + (E + T) * T);
  m[11] = 2.0 * rho * ((E + 2.0 * T) * ubx * uby);
  m[12] = 2.0 * rho * ((E + 2.0 * T) * uby * uby + (E + T) * T);
}

static void exp_family13(const double l[ORA_M13], double p[ORA_Q49]) {
  for (int i = 0; i < ORA_Q49; ++i) {
    double P[ORA_M13];
    monomials13(XI49[i][0], XI49[i][1], P);
    double s = 1.0;
    for (int k = 0; k < ORA_M13; ++k) s += l[k] * P[k];
    p[i] = exp(-s);
  }
}

static double dual_value13(const double l[ORA_M13], const double p[ORA_Q49],
                           const double m[ORA_M13]) {
  double F = 0.0;
  for (int i = 0; i < ORA_Q49; ++i) F += p[i];
  for (int k = 0; k < ORA_M13; ++k) F += l[k] * m[k];
  return F;
}

/* Cholesky solve of an n x n symmetric positive definite system (row-major A). */
static int cholesky_solve_n(int n, const double* A, const double* b, double* x) {
  double L[ORA_M13 * ORA_M13], y[ORA_M13];
  memset(L, 0, sizeof(L));
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0) || !isfinite(d)) return ORA_ESINGULAR;
    L[j * n + j] = sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
    y[i] = t / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * x[k];
    x[i] = t / L[i * n + i];
  }
  return ORA_OK;
}

int ora_equilibrium13(double rho, double ubx, double uby, double T, double tol, int maxit,
                      double lambda[ORA_M13], double feq[ORA_Q49], int* iters) {
  *iters = 0;
  if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ubx) ||
      !isfinite(uby))
    return ORA_EUNREALIZABLE;
  double m[ORA_M13];
  ora_targets13(rho, ubx, uby, T, m);
  for (int k = 0; k < ORA_M13; ++k) m[k] /= rho;
  /* Maxwellian start: lambda_1 = -ubar/T, lambda_2aa = 1/(2T), lambda_0 from
   * the normalisation, the rest 0 */
  for (int k = 0; k < ORA_M13; ++k) lambda[k] = 0.0;
  lambda[1] = -ubx / T;
  lambda[2] = -uby / T;
  lambda[3] = 0.5 / T;
  lambda[5] = 0.5 / T;
  double p[ORA_Q49];
  exp_family13(lambda, p);
  double Z = 0.0;
  for (int i = 0; i < ORA_Q49; ++i) Z += p[i];
  lambda[0] = log(Z);
  exp_family13(lambda, p);
  double F = dual_value13(lambda, p, m);
  int status = ORA_ENEWTON;
  int it = 0;
  for (;;) {
    double G[ORA_M13], H[ORA_M13 * ORA_M13];
    for (int k = 0; k < ORA_M13; ++k) G[k] = -m[k];
    memset(H, 0, sizeof(H));
    for (int i = 0; i < ORA_Q49; ++i) {
      double P[ORA_M13];
      monomials13(XI49[i][0], XI49[i][1], P);
      for (int a = 0; a < ORA_M13; ++a) {
        G[a] += p[i] * P[a];
        for (int b = 0; b < ORA_M13; ++b) H[a * ORA_M13 + b] += p[i] * P[a] * P[b];
      }
    }
    double gmax = 0.0;
    for (int k = 0; k < ORA_M13; ++k) gmax = fmax(gmax, fabs(G[k]));
    if (!isfinite(gmax)) { status = ORA_ESINGULAR; break; }
    if (gmax <= tol) { status = ORA_OK; break; }
    if (it >= maxit) { status = ORA_ENEWTON; break; }
    double d[ORA_M13];
    if (cholesky_solve_n(ORA_M13, H, G, d) != ORA_OK) { status = ORA_ESINGULAR; break; }
    double gd = 0.0;
    for (int k = 0; k < ORA_M13; ++k) gd += G[k] * d[k];
    double t = 1.0, lam_c[ORA_M13], p_c[ORA_Q49], F_c = 0.0;
    int accepted = 0;
    for (int ls = 0; ls < 40; ++ls) {
      for (int k = 0; k < ORA_M13; ++k) lam_c[k] = lambda[k] + t * d[k];
      exp_family13(lam_c, p_c);
      F_c = dual_value13(lam_c, p_c, m);
      if (isfinite(F_c) && F_c <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) { accepted = 1; break; }
      t *= 0.5;
    }
    ++it;
    if (!accepted) { status = ORA_ENEWTON; break; }
    for (int k = 0; k < ORA_M13; ++k) lambda[k] = lam_c[k];
    for (int i = 0; i < ORA_Q49; ++i) p[i] = p_c[i];
    F = F_c;
  }
  *iters = it;
  for (int i = 0; i < ORA_Q49; ++i) feq[i] = rho * p[i];
  return status;
}

/* Eq. criterion: U_a = n iff n - 0.5 < u_a <= n + 0.5. With an offset n0 the
 * interval is read as (n - n0, n + 1 - n0]; shifts are clamped to [-umax, umax]. */
int ora_select_shift(double u, double n0, int umax) {
  for (int n = -umax; n <= umax; ++n) {
    const double lo = (double)n - n0;
    const double hi = (double)(n + 1) - n0;
    if (lo < u && u <= hi) return n;
  }
  return u > 0.0 ? umax : -umax;
}

/* Overlapping ranges (Sec. III.A.2): the paper allows the range of a shift to
 * be wider than 1, so that ranges of neighbouring shifts overlap; where they
 * do, the shift a node already has is kept (its history). Here the range of
 * the current shift is the criterion's interval widened by w on each side;
 * outside it the node takes the criterion's shift. */
int ora_select_shift_kept(double u, double n0, int umax, int current, double w) {
  if (w > 0.0) {
    const double lo = ((double)current - n0) - w;
    const double hi = ((double)(current + 1) - n0) + w;
    if (lo < u && u <= hi) return current;
  }
  return ora_select_shift(u, n0, umax);
}

/* Overlapping ranges chosen by the neighbourhood (Sec. III.A.2): where the
 * widened ranges of several shifts hold u, prefer the shift most of the eight
 * surrounding nodes use, so that neighbours share a lattice and fewer nodes
 * sit at an interface. The criterion's shift stays unless another candidate
 * is used by strictly more neighbours. */
int ora_select_shift_neighbours(double u, double n0, int umax, double w, const int* nb,
                                int nnb) {
  const int c = ora_select_shift(u, n0, umax);
  if (!(w > 0.0)) return c;
  int best = c, best_count = 0;
  for (int j = 0; j < nnb; ++j) best_count += nb[j] == c;
  for (int n = -umax; n <= umax; ++n) {
    if (n == c) continue;
    const double lo = ((double)n - n0) - w;
    const double hi = ((double)(n + 1) - n0) + w;
    if (!(lo < u && u <= hi)) continue;
    int count = 0;
    for (int j = 0; j < nnb; ++j) count += nb[j] == n;
    if (count > best_count) {
      best = n;
      best_count = count;
    }
  }
  return best;
}

/* Eq. polyTemp, evaluated with the populations' own velocities c_i = xi_i + U:
 * rho = sum f, rho u = sum f c, and T = [sum(|c|^2 f + g) - rho |u|^2] / (2 rho Cv).
 * Summing in the lattice frame (xi instead of c) gives the same T exactly in
 * exact arithmetic; the lattice frame is used so that results do not depend on U. */
void ora_node_moments(int Q, const double* f, const double* g, int Ux, int Uy, double gamma,
                      double out[4]) {
  const int(*xi)[2] = stencil_xi(Q);
  const double Cv = 1.0 / (gamma - 1.0);
  double rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
  for (int i = 0; i < Q; ++i) {
    const double x = xi[i][0], y = xi[i][1];
    rho += f[i];
    jx += f[i] * x;
    jy += f[i] * y;
    e += (x * x + y * y) * f[i] + g[i];
  }
  const double ubx = jx / rho, uby = jy / rho;
  const double T = (e - rho * (ubx * ubx + uby * uby)) / (2.0 * rho * Cv);
  out[0] = rho;
  out[1] = ubx + (double)Ux;
  out[2] = uby + (double)Uy;
  out[3] = T;
}

/* alpha(eps_Kn) of Sec. IV.A.2. The paper gives only its onset (alpha = 1 for
 * eps_Kn <= 0.01); the function itself comes from another work. Reading used
 * here: continuous and piecewise linear in log10(eps) through the knots
 * (e0, 1), (e1, a0), (e2, a1), (10 e2, a2), constant beyond, so that the
 * relaxation time is a continuous function of the populations. */
static double sensor_alpha(const ora_config* c, double eps) {
  const double* e = c->sensor_eps;
  const double* a = c->sensor_alpha;
  if (!(eps > e[0])) return 1.0;
  const double kx[4] = {log10(e[0]), log10(e[1]), log10(e[2]), log10(e[2]) + 1.0};
  const double ky[4] = {1.0, a[0], a[1], a[2]};
  const double l = log10(eps);
  for (int k = 0; k < 3; ++k)
    if (l <= kx[k + 1]) return ky[k] + (ky[k + 1] - ky[k]) * (l - kx[k]) / (kx[k + 1] - kx[k]);
  return a[2];
}

/* Numerical equilibrium of the configured constraint set (8 or 4 moments). */
static int equilibrium_cfg(const ora_config* c, double rho, double ubx, double uby, double T,
                           double* feq) {
  int iters;
  if (c->stencil == ORA_D2Q49) {
    double l13[ORA_M13];
    return ora_equilibrium13(rho, ubx, uby, T, c->newton_tol, c->newton_maxit, l13, feq, &iters);
  }
  if (c->moments == 4) {
    double l4[4];
    return ora_equilibrium4(rho, ubx, uby, T, c->newton_tol, c->newton_maxit, l4, feq, &iters);
  }
  double lambda[ORA_M];
  return ora_equilibrium(rho, ubx, uby, T, c->newton_tol, c->newton_maxit, lambda, feq, &iters);
}

void ora_heat_flux(int Q, const double* f, const double* g, int Ux, int Uy, double ux,
                   double uy, double q[2]) {
  const int(*xi)[2] = stencil_xi(Q);
  q[0] = q[1] = 0.0;
  for (int i = 0; i < Q; ++i) {
    const double cx = (double)(xi[i][0] + Ux) - ux;
    const double cy = (double)(xi[i][1] + Uy) - uy;
    const double e = (cx * cx + cy * cy) * f[i] + g[i];
    q[0] += 0.5 * cx * e;
    q[1] += 0.5 * cy * e;
  }
}

/* Collision of one node (Eqs. coll, gEq, DeltaAvg) in its own lattice U; for
 * Pr != 1 the heat-flux term of Eqs. Shakhov / prandtlPoly is added:
 *   f* += (1/tau - 1/tau_Pr) q.cbar / (rho Cp T^2) (|cbar|^2 / (2T) - Cp) f^eq,
 *   g* += (1/tau - 1/tau_Pr) 2 q.cbar / (rho Cp) g^eq,
 * with tau_Pr = 1/2 + (nu/Pr)/T; the sensor factor scales tau and tau_Pr alike. */
int ora_collide_node(const ora_config* cfg, const double* f, const double* g, int Ux, int Uy,
                     double* fs, double* gs) {
  const int Q = cfg->stencil == ORA_D2Q49 ? ORA_Q49 : ORA_Q;
  const int(*xi)[2] = stencil_xi(Q);
  double mom[4];
  ora_node_moments(Q, f, g, Ux, Uy, cfg->gamma, mom);
  const double rho = mom[0], T = mom[3];
  double feq[ORA_QMAX];
  int st = equilibrium_cfg(cfg, rho, mom[1] - Ux, mom[2] - Uy, T, feq);
  if (st != ORA_OK) {
    /* failure policy: the node is left uncollided */
    for (int i = 0; i < Q; ++i) { fs[i] = f[i]; gs[i] = g[i]; }
    return st;
  }
  const double Cv = 1.0 / (cfg->gamma - 1.0);
  const double Cp = cfg->gamma * Cv;
  double tau = 0.5 + cfg->nu / T;
  double tau_pr = 0.5 + (cfg->nu / cfg->prandtl) / T;
  if (cfg->sensor) {
    double eps = 0.0;
    for (int i = 0; i < Q; ++i) eps += fabs(f[i] - feq[i]) / feq[i];
    eps /= (double)Q;
    const double a = sensor_alpha(cfg, eps);
    tau *= a;
    tau_pr *= a;
  }
  for (int i = 0; i < Q; ++i) {
    const double geq = (2.0 * Cv - D_SPACE) * T * feq[i];
    fs[i] = f[i] - (f[i] - feq[i]) / tau;
    gs[i] = g[i] - (g[i] - geq) / tau;
  }
  if (cfg->prandtl != 1.0) {
    double q[2];
    ora_heat_flux(Q, f, g, Ux, Uy, mom[1], mom[2], q);
    const double w = 1.0 / tau - 1.0 / tau_pr;
    for (int i = 0; i < Q; ++i) {
      const double cx = (double)(xi[i][0] + Ux) - mom[1];
      const double cy = (double)(xi[i][1] + Uy) - mom[2];
      const double c2 = cx * cx + cy * cy;
      const double qc = q[0] * cx + q[1] * cy;
      const double geq = (2.0 * Cv - D_SPACE) * T * feq[i];
      fs[i] += w * qc / (rho * Cp * T * T) * (c2 / (2.0 * T) - Cp) * feq[i];
      gs[i] += w * 2.0 * qc / (rho * Cp) * geq;
    }
  }
  return ORA_OK;
}

/* Grad's approximation h = h^eq (1 + omega phi_h): Eq. GradGeneral with phi_f
 * from Eq. GradGeneral_f (traceless viscous stress, Fourier heat flux, mu = rho nu,
 * kappa = rho Cp nu / Pr, Pr = 1 for BGK) and phi_g from Eq. GradGeneral_g, both
 * as printed. cbar = c_i - u with c_i = xi_i + U. The heat-flux part of phi_f
 * has the shape of the App. E term, so the collision of App. E applied to the
 * Grad population (with q its Fourier flux) adds w_pr times that part. */
int ora_grad_populations(const ora_config* cfg, int Ux, int Uy, double rho, double ux,
                         double uy, double T, const double du[2][2], const double dT[2],
                         double omega, double w_pr, double* f, double* g) {
  const int Q = cfg->stencil == ORA_D2Q49 ? ORA_Q49 : ORA_Q;
  const int(*xi)[2] = stencil_xi(Q);
  const double Cv = 1.0 / (cfg->gamma - 1.0);
  const double Cp = cfg->gamma * Cv;
  double feq[ORA_QMAX];
  int st = equilibrium_cfg(cfg, rho, ux - Ux, uy - Uy, T, feq);
  if (st != ORA_OK) return st;
  const double mu = rho * cfg->nu;
  const double kappa = rho * Cp * cfg->nu / cfg->prandtl;
  /* -sigma_ab = mu [d_a u_b + d_b u_a - (2/D) d_c u_c delta_ab] */
  const double div = du[0][0] + du[1][1];
  const double sxx = -mu * (2.0 * du[0][0] - (2.0 / D_SPACE) * div);
  const double syy = -mu * (2.0 * du[1][1] - (2.0 / D_SPACE) * div);
  const double sxy = -mu * (du[0][1] + du[1][0]);
  const double qx = -kappa * dT[0];
  const double qy = -kappa * dT[1];
  for (int i = 0; i < Q; ++i) {
    const double cx = (double)(xi[i][0] + Ux) - ux;
    const double cy = (double)(xi[i][1] + Uy) - uy;
    const double c2 = cx * cx + cy * cy;
    const double qc = qx * cx + qy * cy;
    const double phi_s = (sxx * cx * cx + 2.0 * sxy * cx * cy + syy * cy * cy) / (2.0 * rho * T * T);
    const double phi_q = qc / (rho * Cp * T * T) * (c2 / (2.0 * T) - Cp);
    const double phi_f = phi_s + phi_q;
    const double phi_g = 2.0 * qc / (rho * Cp);
    const double geq = (2.0 * Cv - D_SPACE) * T * feq[i];
    f[i] = feq[i] * (1.0 + omega * phi_f + w_pr * phi_q);
    g[i] = geq * (1.0 + omega * phi_g + w_pr * phi_g);
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------------- */
/* Grid helpers */

/* Resolve a coordinate along one axis: periodic wrap, or, for zero-gradient
 * ends, clamp into the domain (ghost nodes carry the nearest interior moments).
 * *ghost is set when the coordinate was outside the domain. */
static int resolve(int x, int n, int bc, int* ghost) {
  if (bc == ORA_PERIODIC) {
    int r = x % n;
    if (r < 0) r += n;
    *ghost = 0;
    return r;
  }
  if (x < 0) { *ghost = 1; return 0; }
  if (x >= n) { *ghost = 1; return n - 1; }
  *ghost = 0;
  return x;
}

/* Second-order central differences of a node field at (x, y), x and y possibly
 * ghost coordinates (Sec. IV.A.1: gradients by second-order FD). Neighbours are
 * resolved with the boundary rule, so a gradient across a zero-gradient end is 0. */
static void central_diff(const ora_state* s, const double* F, int x, int y, double d[2]) {
  const int nx = s->cfg.nx, ny = s->cfg.ny;
  int gh;
  const int ry = resolve(y, ny, s->cfg.bc_y, &gh);
  const int rx = resolve(x, nx, s->cfg.bc_x, &gh);
  const int xp = resolve(x + 1, nx, s->cfg.bc_x, &gh);
  const int xm = resolve(x - 1, nx, s->cfg.bc_x, &gh);
  const int yp = resolve(y + 1, ny, s->cfg.bc_y, &gh);
  const int ym = resolve(y - 1, ny, s->cfg.bc_y, &gh);
  d[0] = 0.5 * (F[ry * nx + xp] - F[ry * nx + xm]);
  d[1] = 0.5 * (F[yp * nx + rx] - F[ym * nx + rx]);
}

ora_state* ora_create(const ora_config* cfg) {
  if (cfg->nx <= 0 || cfg->ny <= 0 || cfg->umax < 0 || cfg->umax > 3) return NULL;
  if (!(cfg->overlap >= 0.0 && cfg->overlap <= 1.0)) return NULL;
  if (cfg->overlap_rule != ORA_RULE_HISTORY && cfg->overlap_rule != ORA_RULE_NEIGHBOURS)
    return NULL;
  if (!(cfg->prandtl > 0.0)) return NULL;
  if (cfg->stencil == ORA_D2Q21) {
    if (cfg->moments != 8 && cfg->moments != 4) return NULL;
  } else if (cfg->stencil == ORA_D2Q49) {
    if (cfg->moments != 13) return NULL;
  } else {
    return NULL;
  }
  ora_state* s = (ora_state*)calloc(1, sizeof(ora_state));
  if (!s) return NULL;
  s->cfg = *cfg;
  s->n = cfg->nx * cfg->ny;
  s->Q = cfg->stencil == ORA_D2Q49 ? ORA_Q49 : ORA_Q;
  s->xi = stencil_xi(s->Q);
  const size_t nq = (size_t)s->n * s->Q;
  s->f = (double*)calloc(nq, sizeof(double));
  s->g = (double*)calloc(nq, sizeof(double));
  s->fs = (double*)calloc(nq, sizeof(double));
  s->gs = (double*)calloc(nq, sizeof(double));
  s->Ux = (signed char*)calloc(s->n, 1);
  s->Uy = (signed char*)calloc(s->n, 1);
  s->Unx = (signed char*)calloc(s->n, 1);
  s->Uny = (signed char*)calloc(s->n, 1);
  s->rho = (double*)calloc(s->n, sizeof(double));
  s->ux = (double*)calloc(s->n, sizeof(double));
  s->uy = (double*)calloc(s->n, sizeof(double));
  s->T = (double*)calloc(s->n, sizeof(double));
  if (!s->f || !s->g || !s->fs || !s->gs || !s->Ux || !s->Uy || !s->Unx || !s->Uny || !s->rho ||
      !s->ux || !s->uy || !s->T) {
    ora_destroy(s);
    return NULL;
  }
  return s;
}

void ora_destroy(ora_state* s) {
  if (!s) return;
  free(s->f); free(s->g); free(s->fs); free(s->gs);
  free(s->Ux); free(s->Uy); free(s->Unx); free(s->Uny);
  free(s->rho); free(s->ux); free(s->uy); free(s->T);
  free(s);
}

/* Initial condition (Sec. IV.A.1, IV.B): populations h = h^eq (1 + phi_h) from
 * the given fields, in the lattice chosen by the criterion for the initial
 * velocity, with FD gradients of the initial u and T. */
int ora_init(ora_state* s, const double* rho, const double* rhoux, const double* rhouy,
             const double* rhoE) {
  const ora_config* c = &s->cfg;
  const int nx = c->nx, ny = c->ny;
  const double Cv = 1.0 / (c->gamma - 1.0);
  for (int k = 0; k < s->n; ++k) {
    const double r = rho[k];
    if (!(r > 0.0)) return ORA_EUNREALIZABLE;
    const double ux = rhoux[k] / r, uy = rhouy[k] / r;
    const double T = (rhoE[k] - 0.5 * r * (ux * ux + uy * uy)) / (r * Cv);
    if (!(T > 0.0)) return ORA_EUNREALIZABLE;
    s->rho[k] = r; s->ux[k] = ux; s->uy[k] = uy; s->T[k] = T;
  }
  memset(&s->stats, 0, sizeof(s->stats));
  int status = ORA_OK;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const int k = y * nx + x;
      const int Ux = ora_select_shift(s->ux[k], c->n0, c->umax);
      const int Uy = ora_select_shift(s->uy[k], c->n0, c->umax);
      double du[2][2], dT[2], dux[2], duy[2];
      central_diff(s, s->ux, x, y, dux);
      central_diff(s, s->uy, x, y, duy);
      central_diff(s, s->T, x, y, dT);
      du[0][0] = dux[0]; du[1][0] = dux[1]; /* du[a][b] = d_a u_b */
      du[0][1] = duy[0]; du[1][1] = duy[1];
      int st = ora_grad_populations(c, Ux, Uy, s->rho[k], s->ux[k], s->uy[k], s->T[k], du, dT,
                                    1.0, 0.0, &s->f[(size_t)k * s->Q], &s->g[(size_t)k * s->Q]);
      if (st != ORA_OK) status = st;
      s->Ux[k] = (signed char)Ux;
      s->Uy[k] = (signed char)Uy;
    }
  }
  return status;
}

/* Post-collision population of velocity i pulled by the receiver (x, y) in
 * lattice (Upx, Upy) from the (possibly ghost) sender (sx, sy) = (x, y) -
 * (xi_i + U') whose lattice differs: Grad rebuild with the sender's moments
 * and gradients and the sender's relaxation time (Sec. III.B.2: the rebuilt
 * population is the sender's post-collision one). */
static int rebuild_pull(ora_state* s, int i, int Upx, int Upy, int x, int y, double* fi,
                        double* gi) {
  const ora_config* c = &s->cfg;
  const int sx = x - (s->xi[i][0] + Upx);
  const int sy = y - (s->xi[i][1] + Upy);
  int gx, gy;
  const int rx = resolve(sx, c->nx, c->bc_x, &gx);
  const int ry = resolve(sy, c->ny, c->bc_y, &gy);
  const int k = ry * c->nx + rx;
  double dux[2], duy[2], dT[2], du[2][2];
  central_diff(s, s->ux, sx, sy, dux);
  central_diff(s, s->uy, sx, sy, duy);
  central_diff(s, s->T, sx, sy, dT);
  du[0][0] = dux[0]; du[1][0] = dux[1];
  du[0][1] = duy[0]; du[1][1] = duy[1];
  const double tau = 0.5 + c->nu / s->T[k];
  const double tau_pr = 0.5 + (c->nu / c->prandtl) / s->T[k];
  double f[ORA_QMAX], g[ORA_QMAX];
  int st = ora_grad_populations(c, Upx, Upy, s->rho[k], s->ux[k], s->uy[k], s->T[k], du, dT,
                                1.0 - 1.0 / tau, 1.0 / tau - 1.0 / tau_pr, f, g);
  if (st != ORA_OK) return st;
  *fi = f[i];
  *gi = g[i];
  return ORA_OK;
}

/* Fallback for a rebuild whose root finder failed: the Maxwellian-guess
 * exponential (always positive) of the sender's state in the receiver's lattice,
 * rho exp(-|xi - ubar|^2 / (2T)) normalised over the lattice. */
static void rebuild_fallback(ora_state* s, int i, int Upx, int Upy, int sx, int sy, double* fi,
                             double* gi) {
  const ora_config* c = &s->cfg;
  int gx, gy;
  const int k = resolve(sy, c->ny, c->bc_y, &gy) * c->nx + resolve(sx, c->nx, c->bc_x, &gx);
  const double Cv = 1.0 / (c->gamma - 1.0);
  const double ubx = s->ux[k] - Upx, uby = s->uy[k] - Upy, T = s->T[k];
  if (s->Q == ORA_Q) {
    double lambda[ORA_M], p[ORA_Q];
    maxwellian_guess(ubx, uby, T, lambda);
    exp_family(lambda, p);
    *fi = s->rho[k] * p[i];
  } else {
    double Z = 0.0, pi = 0.0;
    for (int j = 0; j < s->Q; ++j) {
      const double dx = s->xi[j][0] - ubx, dy = s->xi[j][1] - uby;
      const double e = exp(-(dx * dx + dy * dy) / (2.0 * T));
      Z += e;
      if (j == i) pi = e;
    }
    *fi = s->rho[k] * pi / Z;
  }
  *gi = (2.0 * Cv - D_SPACE) * T * (*fi);
}

/* One time iteration; if forced_x / forced_y are given they replace the
 * criterion's choice of the next lattice (replay of recorded decisions). */
static int step_once(ora_state* s, const signed char* forced_x, const signed char* forced_y) {
  const ora_config* c = &s->cfg;
  const int nx = c->nx, ny = c->ny;
  const int Q = s->Q;
  const int(*xi)[2] = s->xi;
  int status = ORA_OK;
  {
    /* (i) moments, equilibrium, collision, next shift: every node in its own lattice */
    long long fails = 0, calls = 0;
#pragma omp parallel for reduction(+ : fails, calls) schedule(static)
    for (int k = 0; k < s->n; ++k) {
      const double* f = &s->f[(size_t)k * Q];
      const double* g = &s->g[(size_t)k * Q];
      double mom[4];
      ora_node_moments(Q, f, g, s->Ux[k], s->Uy[k], c->gamma, mom);
      s->rho[k] = mom[0]; s->ux[k] = mom[1]; s->uy[k] = mom[2]; s->T[k] = mom[3];
      int st = ora_collide_node(c, f, g, s->Ux[k], s->Uy[k], &s->fs[(size_t)k * Q],
                                &s->gs[(size_t)k * Q]);
      calls += 1;
      if (st != ORA_OK) fails += 1;
      if (forced_x) {
        s->Unx[k] = forced_x[k];
        s->Uny[k] = forced_y[k];
      } else if (c->overlap > 0.0 && c->overlap_rule == ORA_RULE_NEIGHBOURS) {
        /* the current shifts of the eight surrounding nodes (boundary rule) */
        const int x = k % nx, y = k / nx;
        int nbx[8], nby[8], m = 0;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int gx, gy;
            const int kk = resolve(y + dy, ny, c->bc_y, &gy) * nx + resolve(x + dx, nx, c->bc_x, &gx);
            nbx[m] = s->Ux[kk];
            nby[m] = s->Uy[kk];
            ++m;
          }
        s->Unx[k] = (signed char)ora_select_shift_neighbours(mom[1], c->n0, c->umax, c->overlap,
                                                             nbx, 8);
        s->Uny[k] = (signed char)ora_select_shift_neighbours(mom[2], c->n0, c->umax, c->overlap,
                                                             nby, 8);
      } else {
        s->Unx[k] = (signed char)ora_select_shift_kept(mom[1], c->n0, c->umax, s->Ux[k],
                                                       c->overlap);
        s->Uny[k] = (signed char)ora_select_shift_kept(mom[2], c->n0, c->umax, s->Uy[k],
                                                       c->overlap);
      }
    }
    s->stats.newton_calls += calls;
    s->stats.newton_failures += fails;
    if (fails) status = ORA_ENEWTON;

    /* (ii) pull streaming in the receiver's new lattice, Grad rebuild of missing pulls */
    long long rec = 0, rec_fail = 0;
#pragma omp parallel for reduction(+ : rec, rec_fail) schedule(static)
    for (int k = 0; k < s->n; ++k) {
      const int x = k % nx, y = k / nx;
      const int Upx = s->Unx[k], Upy = s->Uny[k];
      for (int i = 0; i < Q; ++i) {
        const int sx = x - (xi[i][0] + Upx);
        const int sy = y - (xi[i][1] + Upy);
        int gx, gy;
        const int rx = resolve(sx, nx, c->bc_x, &gx);
        const int ry = resolve(sy, ny, c->bc_y, &gy);
        const int ks = ry * nx + rx;
        double fi, gi;
        if (!gx && !gy && s->Ux[ks] == Upx && s->Uy[ks] == Upy) {
          fi = s->fs[(size_t)ks * Q + i];
          gi = s->gs[(size_t)ks * Q + i];
        } else {
          rec += 1;
          if (rebuild_pull(s, i, Upx, Upy, x, y, &fi, &gi) != ORA_OK) {
            rec_fail += 1;
            rebuild_fallback(s, i, Upx, Upy, sx, sy, &fi, &gi);
          }
        }
        s->f[(size_t)k * Q + i] = fi;
        s->g[(size_t)k * Q + i] = gi;
      }
    }
    s->stats.reconstructions += rec;
    s->stats.reconstruction_failures += rec_fail;
    if (rec_fail) status = ORA_ENEWTON;

    /* (iii) the received populations now live in the new lattice */
    memcpy(s->Ux, s->Unx, (size_t)s->n);
    memcpy(s->Uy, s->Uny, (size_t)s->n);
  }
  return status;
}

int ora_step(ora_state* s, int nsteps) {
  int status = ORA_OK;
  for (int step = 0; step < nsteps; ++step) {
    const int st = step_once(s, NULL, NULL);
    if (st != ORA_OK) status = st;
  }
  return status;
}

int ora_step_forced(ora_state* s, const signed char* ux, const signed char* uy) {
  for (int k = 0; k < s->n; ++k)
    if (ux[k] < -s->cfg.umax || ux[k] > s->cfg.umax || uy[k] < -s->cfg.umax ||
        uy[k] > s->cfg.umax)
      return ORA_EINVAL;
  return step_once(s, ux, uy);
}

void ora_get_primitives(const ora_state* s, double* rho, double* ux, double* uy, double* T) {
  for (int k = 0; k < s->n; ++k) {
    double mom[4];
    ora_node_moments(s->Q, &s->f[(size_t)k * s->Q], &s->g[(size_t)k * s->Q], s->Ux[k],
                     s->Uy[k], s->cfg.gamma, mom);
    rho[k] = mom[0]; ux[k] = mom[1]; uy[k] = mom[2]; T[k] = mom[3];
  }
}

void ora_get_moments(const ora_state* s, double* rho, double* rhoux, double* rhouy,
                     double* rhoE) {
  const double Cv = 1.0 / (s->cfg.gamma - 1.0);
  for (int k = 0; k < s->n; ++k) {
    double mom[4];
    ora_node_moments(s->Q, &s->f[(size_t)k * s->Q], &s->g[(size_t)k * s->Q], s->Ux[k],
                     s->Uy[k], s->cfg.gamma, mom);
    const double r = mom[0], ux = mom[1], uy = mom[2], T = mom[3];
    rho[k] = r;
    rhoux[k] = r * ux;
    rhouy[k] = r * uy;
    rhoE[k] = 0.5 * r * (ux * ux + uy * uy) + r * Cv * T;
  }
}

void ora_get_shifts(const ora_state* s, signed char* ux, signed char* uy) {
  memcpy(ux, s->Ux, (size_t)s->n);
  memcpy(uy, s->Uy, (size_t)s->n);
}

void ora_get_populations(const ora_state* s, double* f, double* g) {
  memcpy(f, s->f, sizeof(double) * (size_t)s->n * s->Q);
  memcpy(g, s->g, sizeof(double) * (size_t)s->n * s->Q);
}

void ora_set_state(ora_state* s, const double* f, const double* g, const signed char* ux,
                   const signed char* uy) {
  memcpy(s->f, f, sizeof(double) * (size_t)s->n * s->Q);
  memcpy(s->g, g, sizeof(double) * (size_t)s->n * s->Q);
  memcpy(s->Ux, ux, (size_t)s->n);
  memcpy(s->Uy, uy, (size_t)s->n);
}

void ora_get_stats(const ora_state* s, ora_stats* out) { *out = s->stats; }
