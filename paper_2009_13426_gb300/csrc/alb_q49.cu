// The paper's reference solver (App. C.1, used for its reference data in
// Sec. IV.B): the same adaptive step - pull in the receiver's lattice, Grad
// rebuild of missing pulls, moments, next lattice, numerical equilibrium, BGK
// (or the App. E collision) - on the D2Q49 lattice {-3..3}^2 with the
// 13-moment equilibrium of Eqs. G0..G4yyaa / feqNum_13Mom. FP64 throughout.
//
// Velocity i = (x, y) has index i = (x + 3) + 7 (y + 3). One thread per node;
// a block is a row segment of B nodes. Each thread owns two columns of the
// block's dynamic shared memory (stride B): its 98 pulled populations and the
// 49 equilibrium values per unit density of its latest solve. A missing pull
// needs the equilibrium of its sender's state in the receiver's lattice; the
// block solves each distinct (sender, lattice) once, round-robin over its
// threads, and forms the pulls from the multipliers (see step_kernel).
// Exponentials use the table-driven FP64 exp of the D2Q21 kernels.
//
// Newton on the 13 multipliers follows the 8-moment solver's iteration
// (Maxwellian start with lambda_0 from the normalisation, exact Jacobian,
// Armijo backtracking on the convex dual, stop at max|G|/rho <= tol). The
// Jacobian entries are moments sum_i p_i x^a y^b with a + b <= 8; the lattice
// is a tensor product, so they come from per-row sums S_a(y) = sum_x p x^a
// (756 multiply-adds instead of 49 x 91).
#include "alb_internal.h"
#include "alb_mixed.cuh"

namespace alb {
namespace q49 {

constexpr int Q = 49;      // velocities
constexpr int M = 13;      // constraints
constexpr int NP = 2 * Q;  // f and g planes
constexpr int B = 64;      // nodes per block
constexpr size_t SMEM = (size_t)(NP + Q) * B * sizeof(double);

__host__ __device__ constexpr int vx(int i) { return i % 7 - 3; }
__host__ __device__ constexpr int vy(int i) { return i / 7 - 3; }
__host__ __device__ constexpr int ipow(int v, int e) { return e == 0 ? 1 : v * ipow(v, e - 1); }

// s + v * c for a compile-time integer c, with the 0 and +-1 cases folded.
__device__ __forceinline__ double madd(double s, double v, int c) {
  if (c == 0) return s;
  if (c == 1) return s + v;
  if (c == -1) return s - v;
  return fma(v, (double)c, s);
}

// Monomial k of Eq. feqNum_13Mom as at most two terms c x^a y^b:
// 1, x, y, x^2, xy, y^2, x^3, x^2 y, x y^2, y^3, x^2 r^2, x y r^2, y^2 r^2.
// (The printed exponent omits lambda_3,xxx x^3; thirteen constraints need
// thirteen multipliers, so it is included.)
struct Term {
  int a, b;
};
__host__ __device__ constexpr int nterms(int k) { return k >= 10 ? 2 : 1; }
__host__ __device__ constexpr Term term(int k, int t) {
  return k == 0 ? Term{0, 0} : k == 1 ? Term{1, 0} : k == 2 ? Term{0, 1}
       : k == 3 ? Term{2, 0} : k == 4 ? Term{1, 1} : k == 5 ? Term{0, 2}
       : k == 6 ? Term{3, 0} : k == 7 ? Term{2, 1} : k == 8 ? Term{1, 2}
       : k == 9 ? Term{0, 3}
       : k == 10 ? (t == 0 ? Term{4, 0} : Term{2, 2})
       : k == 11 ? (t == 0 ? Term{3, 1} : Term{1, 3})
                 : (t == 0 ? Term{2, 2} : Term{0, 4});
}

// Targets of Eqs. G0..G4yyaa per unit density, lattice frame, 2E = |u|^2 + D T.
__device__ __forceinline__ void targets13(double ubx, double uby, double T, double m[M]) {
  const double E = 0.5 * (ubx * ubx + uby * uby + 2.0 * T);
  m[0] = 1.0;
  m[1] = ubx;
  m[2] = uby;
  m[3] = ubx * ubx + T;
  m[4] = ubx * uby;
  m[5] = uby * uby + T;
  m[6] = ubx * (ubx * ubx + 3.0 * T);
  m[7] = (ubx * ubx + T) * uby;
  m[8] = ubx * (uby * uby + T);
  m[9] = uby * (uby * uby + 3.0 * T);
  m[10] = 2.0 * ((E + 2.0 * T) * ubx * ubx + (E + T) * T);
  m[11] = 2.0 * ((E + 2.0 * T) * ubx * uby);
  m[12] = 2.0 * ((E + 2.0 * T) * uby * uby + (E + T) * T);
}

// lambda . P(xi_i) for velocity i (compile-time after unrolling).
__device__ __forceinline__ double lam_dot(const double l[M], int i) {
  const int x = vx(i), y = vy(i), r2 = x * x + y * y;
  double s = l[0];
  s = madd(s, l[1], x);
  s = madd(s, l[2], y);
  s = madd(s, l[3], x * x);
  s = madd(s, l[4], x * y);
  s = madd(s, l[5], y * y);
  s = madd(s, l[6], x * x * x);
  s = madd(s, l[7], x * x * y);
  s = madd(s, l[8], x * y * y);
  s = madd(s, l[9], y * y * y);
  s = madd(s, l[10], x * x * r2);
  s = madd(s, l[11], x * y * r2);
  s = madd(s, l[12], y * y * r2);
  return s;
}

// p_i = exp(-(1 + lambda . P_i)) into eq (stride B); returns sum_i p_i.
__device__ __forceinline__ double eval_p(const double l[M], double* eq, const double* tab) {
  double z = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double p = exp_neg(1.0 + lam_dot(l, i), tab);
    eq[i * B] = p;
    z += p;
  }
  return z;
}

// Moments Mab[a][b] = sum_i p_i x^a y^b, a + b <= 8, from the row sums.
__device__ __forceinline__ void moments(const double* eq, double Mab[9][9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a)
#pragma unroll
    for (int b = 0; b < 9; ++b) Mab[a][b] = 0.0;
#pragma unroll
  for (int yy = 0; yy < 7; ++yy) {
    const int y = yy - 3;
    double S[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) S[a] = 0.0;
#pragma unroll
    for (int xx = 0; xx < 7; ++xx) {
      const double p = eq[(xx + 7 * yy) * B];
#pragma unroll
      for (int a = 0; a < 9; ++a) S[a] = madd(S[a], p, ipow(xx - 3, a));
    }
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
      for (int b = 0; a + b < 9; ++b) Mab[a][b] = madd(Mab[a][b], S[a], ipow(y, b));
  }
}

enum { OK = NEWTON_OK, MAXIT = NEWTON_MAXIT, SINGULAR = NEWTON_SINGULAR };

// Newton on the 13 multipliers for (ubx, uby, T) in the lattice frame; the
// equilibrium per unit density is left in eq (stride B).
__device__ __noinline__ int newton13(double ubx, double uby, double T, double tol, int maxit,
                                     double* eq, const double* tab, double lam[M], int* iters) {
  *iters = 0;
  if (!(T > 0.0) || !isfinite(T) || !isfinite(ubx) || !isfinite(uby)) return NEWTON_UNREALIZABLE;
  double m[M];
  targets13(ubx, uby, T, m);
  double l[M];
#pragma unroll
  for (int k = 0; k < M; ++k) l[k] = 0.0;
  l[1] = -ubx / T;
  l[2] = -uby / T;
  l[3] = 0.5 / T;
  l[5] = 0.5 / T;
  // lambda_0 = ln Z normalises the start; p = exp(-(1 + rest)) / Z
  const double Z = eval_p(l, eq, tab);
  l[0] = log(Z);
  const double iz = 1.0 / Z;
  double F = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    eq[i * B] *= iz;
    F += eq[i * B];
  }
#pragma unroll
  for (int k = 0; k < M; ++k) F += l[k] * m[k];
  int status = MAXIT, it = 0;
  for (;;) {
    double Mab[9][9];
    moments(eq, Mab);
    double G[M];
    double gmax = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      double s = -m[k];
#pragma unroll
      for (int t = 0; t < nterms(k); ++t) s += Mab[term(k, t).a][term(k, t).b];
      G[k] = s;
      gmax = fmax(gmax, fabs(s));
    }
    if (!isfinite(gmax)) { status = SINGULAR; break; }
    if (gmax <= tol) { status = OK; break; }
    if (it >= maxit) { status = MAXIT; break; }
    // Jacobian sum_i p_i P_k P_j, factored in place (lower triangle, packed)
    double H[M * (M + 1) / 2];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) {
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < nterms(r); ++t)
#pragma unroll
          for (int u = 0; u < nterms(c); ++u)
            s += Mab[term(r, t).a + term(c, u).a][term(r, t).b + term(c, u).b];
        H[r * (r + 1) / 2 + c] = s;
      }
    // Cholesky H = L L^T in place; the diagonal keeps 1 / L_jj
    bool spd = true;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      double d = H[j * (j + 1) / 2 + j];
#pragma unroll
      for (int k = 0; k < j; ++k) d -= H[j * (j + 1) / 2 + k] * H[j * (j + 1) / 2 + k];
      if (!(d > 0.0) || !isfinite(d)) spd = false;
      const double inv = 1.0 / sqrt(d);
      H[j * (j + 1) / 2 + j] = inv;
#pragma unroll
      for (int i = j + 1; i < M; ++i) {
        double t = H[i * (i + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) t -= H[i * (i + 1) / 2 + k] * H[j * (j + 1) / 2 + k];
        H[i * (i + 1) / 2 + j] = t * inv;
      }
    }
    if (!spd) { status = SINGULAR; break; }
    double d[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      double t = G[i];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= H[i * (i + 1) / 2 + k] * d[k];
      d[i] = t * H[i * (i + 1) / 2 + i];
    }
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
      double t = d[i];
#pragma unroll
      for (int k = i + 1; k < M; ++k) t -= H[k * (k + 1) / 2 + i] * d[k];
      d[i] = t * H[i * (i + 1) / 2 + i];
    }
    double gd = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) gd += G[k] * d[k];
    // backtracking on the dual F = sum p + lambda . m along lambda + t d
    double t = 1.0, lc[M], Fc = 0.0;
    bool accepted = false;
    for (int ls = 0; ls < 40; ++ls) {
#pragma unroll
      for (int k = 0; k < M; ++k) lc[k] = l[k] + t * d[k];
      Fc = eval_p(lc, eq, tab);
#pragma unroll
      for (int k = 0; k < M; ++k) Fc += lc[k] * m[k];
      if (isfinite(Fc) && Fc <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    ++it;
    if (!accepted) { status = MAXIT; break; }
#pragma unroll
    for (int k = 0; k < M; ++k) l[k] = lc[k];
    F = Fc;
  }
  *iters = it;
#pragma unroll
  for (int k = 0; k < M; ++k) lam[k] = l[k];
  return status;
}

struct Count {
  unsigned iters = 0, calls = 0, fail = 0, rec = 0, rec_fail = 0;
};

// The sender of a rebuilt pull: its stored moments at the (possibly ghost)
// position (sx, sy) and the central differences of u and T around it.
struct Sender {
  double rho, ux, uy, T, du[2][2], dT[2];
};

__device__ __forceinline__ Sender sender_state(const Params& pr, const double* __restrict__ mom,
                                               size_t ps, int sx, int sy) {
  bool gh = false;
  const int rx = resolve(sx, pr.nx, pr.bcx, &gh), ry = resolve(sy, pr.ny, pr.bcy, &gh);
  const int xp = resolve(sx + 1, pr.nx, pr.bcx, &gh), xm = resolve(sx - 1, pr.nx, pr.bcx, &gh);
  const int yp = resolve(sy + 1, pr.ny, pr.bcy, &gh), ym = resolve(sy - 1, pr.ny, pr.bcy, &gh);
  const size_t nx = (size_t)pr.nx;
  const size_t ks = ry * nx + rx;
  const size_t kxp = ry * nx + xp, kxm = ry * nx + xm, kyp = yp * nx + rx, kym = ym * nx + rx;
  const double* mux = mom + ps;
  const double* muy = mom + 2 * ps;
  const double* mT = mom + 3 * ps;
  Sender s;
  s.rho = mom[ks];
  s.ux = mux[ks];
  s.uy = muy[ks];
  s.T = mT[ks];
  s.du[0][0] = 0.5 * (mux[kxp] - mux[kxm]);
  s.du[1][0] = 0.5 * (mux[kyp] - mux[kym]);
  s.du[0][1] = 0.5 * (muy[kxp] - muy[kxm]);
  s.du[1][1] = 0.5 * (muy[kyp] - muy[kym]);
  s.dT[0] = 0.5 * (mT[kxp] - mT[kxm]);
  s.dT[1] = 0.5 * (mT[kyp] - mT[kym]);
  return s;
}

// Grad value of pull i in lattice (Upx, Upy) from the sender's equilibrium
// multipliers lam in that lattice: h* = h^eq (1 + (1 - 1/tau) phi_h +
// (1/tau - 1/tau_Pr) phi_h,q), tau of the sender without the sensor.
__device__ __forceinline__ void grad_value(const Params& pr, const Sender& s, int i, int Upx,
                                           int Upy, const double* lam, const double* tab,
                                           double* fi, double* gi) {
  const double gfac = (2.0 * pr.cv - 2.0) * s.T;
  const double tau = 0.5 + pr.nu / s.T;
  const double omega = 1.0 - 1.0 / tau;
  double l[M];
#pragma unroll
  for (int k = 0; k < M; ++k) l[k] = lam[k];
  const double feq = s.rho * exp_neg(1.0 + lam_dot(l, i), tab);
  const double cbx = (double)(vx(i) + Upx) - s.ux;
  const double cby = (double)(vy(i) + Upy) - s.uy;
  double phf, phg, phq;
  grad_phi(pr, s.rho, s.T, cbx, cby, s.du, s.dT, &phf, &phg, &phq);
  const double w = pr.shakhov ? 1.0 / tau - 1.0 / (0.5 + (pr.nu / pr.prandtl) / s.T) : 0.0;
  *fi = feq * (1.0 + omega * phf + w * phq);
  *gi = gfac * feq * (1.0 + omega * phg + w * phg);
}

// Fallback of a rebuild whose solve failed: the Maxwellian exponential of the
// sender's state normalised over the lattice.
__device__ __forceinline__ void fallback_value(const Params& pr, const Sender& s, int i, int Upx,
                                               int Upy, double* fi, double* gi) {
  const double ubx = s.ux - Upx, uby = s.uy - Upy;
  double z = 0.0, pi = 0.0;
  if (s.T > 0.0) {
    for (int j = 0; j < Q; ++j) {
      const double dx = vx(j) - ubx, dy = vy(j) - uby;
      const double e = exp(-(dx * dx + dy * dy) / (2.0 * s.T));
      z += e;
      if (j == i) pi = e;
    }
    *fi = s.rho * pi / z;
  } else {
    *fi = 0.0;
  }
  *gi = (2.0 * pr.cv - 2.0) * s.T * (*fi);
}

// Equilibrium multipliers of the sender's state in lattice (Upx, Upy); the
// thread's equilibrium column is scratch. Returns the solve's status.
__device__ __noinline__ int sender_solve(const Params pr, const Sender s, int Upx, int Upy,
                                         double* eq, const double* tab, double lam[M],
                                         Count* cnt) {
  int it = 0;
  const int st = s.rho > 0.0 ? newton13(s.ux - Upx, s.uy - Upy, s.T, pr.tol, pr.maxit, eq, tab,
                                        lam, &it)
                             : NEWTON_UNREALIZABLE;
  cnt->iters += it;
  cnt->calls += 1;
  return st;
}

// A rebuild done in full by one thread (pulls that did not fit the block's
// table of distinct senders): returns 1 if the fallback was used.
__device__ __noinline__ int rebuild(const Params pr, const double* __restrict__ mom, size_t ps,
                                    int i, int Upx, int Upy, int sx, int sy, double* fi,
                                    double* gi, double* eq, const double* tab, Count* cnt) {
  const Sender s = sender_state(pr, mom, ps, sx, sy);
  double lam[M];
  if (sender_solve(pr, s, Upx, Upy, eq, tab, lam, cnt) != NEWTON_OK) {
    fallback_value(pr, s, i, Upx, Upy, fi, gi);
    return 1;
  }
  grad_value(pr, s, i, Upx, Upy, lam, tab, fi, gi);
  return 0;
}

// Lattice codes of the eight nodes around (x, y) (boundary rule outside).
__device__ __forceinline__ void neighbours(const Params& pr, const uint8_t* cur, int x, int y,
                                           uint8_t nb[8]) {
  int m = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      bool gh = false;
      const int rx = resolve(x + dx, pr.nx, pr.bcx, &gh), ry = resolve(y + dy, pr.ny, pr.bcy, &gh);
      nb[m++] = cur[(size_t)ry * pr.nx + rx];
    }
}

// Moments, next lattice, equilibrium and collision of the node whose 98
// pre-collision populations (lattice `code`) sit in col; stores the result.
__device__ __forceinline__ void collide(const Params& pr, const double* col, double* eq, int code,
                                        size_t k, size_t ps, double* __restrict__ pop_out,
                                        double* __restrict__ mom_out, uint8_t* lat_out,
                                        uint8_t* nxt_out, const uint8_t* nb, const double* tab,
                                        Count* cnt) {
  const int Ux = lat_ux(code), Uy = lat_uy(code);
  double rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double f = col[i * B], g = col[(Q + i) * B];
    rho += f;
    jx = madd(jx, f, vx(i));
    jy = madd(jy, f, vy(i));
    e += (double)(vx(i) * vx(i) + vy(i) * vy(i)) * f + g;
  }
  const double ubx = jx / rho, uby = jy / rho;
  const double T = (e - rho * (ubx * ubx + uby * uby)) / (2.0 * rho * pr.cv);
  const double ux = ubx + (double)Ux, uy = uby + (double)Uy;
  const bool by_nb = pr.overlap > 0.0 && pr.rule == 1 && nb;
  const int code2 = by_nb ? lat_code(select_shift_neighbours(ux, 0, nb, pr),
                                     select_shift_neighbours(uy, 1, nb, pr))
                          : lat_code(select_shift_kept(ux, Ux, pr), select_shift_kept(uy, Uy, pr));
  double lam[M];
  int it = 0;
  const int ns = rho > 0.0 ? newton13(ubx, uby, T, pr.tol, pr.maxit, eq, tab, lam, &it)
                           : NEWTON_UNREALIZABLE;
  cnt->iters += it;
  cnt->calls += 1;
  if (ns == NEWTON_OK) {
    const double gp = (2.0 * pr.cv - 2.0) * T;
    double tau = 0.5 + pr.nu / T, alpha = 1.0;
    if (pr.sensor) {
      double eps = 0.0;
      for (int i = 0; i < Q; ++i) {
        const double fe = eq[i * B] * rho;
        eps += fabs(col[i * B] - fe) / fe;
      }
      alpha = sensor_alpha<double>(pr, eps / (double)Q);
      tau *= alpha;
    }
    const double om = 1.0 / tau;
    double w = 0.0, qx = 0.0, qy = 0.0;
    if (pr.shakhov) {
      // App. E: q of the pre-collision populations, cbar = xi - ubar
      for (int i = 0; i < Q; ++i) {
        const double cx = (double)vx(i) - ubx, cy = (double)vy(i) - uby;
        const double en = (cx * cx + cy * cy) * col[i * B] + col[(Q + i) * B];
        qx += 0.5 * cx * en;
        qy += 0.5 * cy * en;
      }
      w = om - 1.0 / ((0.5 + (pr.nu / pr.prandtl) / T) * alpha);
    }
    const double af = w / (rho * pr.cp * T * T), ag = 2.0 * w / (rho * pr.cp);
#pragma unroll 7
    for (int i = 0; i < Q; ++i) {
      const double fe = eq[i * B] * rho, ge = gp * fe;
      const double f = col[i * B], g = col[(Q + i) * B];
      double fs = fma(om, fe - f, f), gs = fma(om, ge - g, g);
      if (pr.shakhov) {
        const double cx = (double)vx(i) - ubx, cy = (double)vy(i) - uby;
        const double qc = qx * cx + qy * cy;
        fs += af * qc * ((cx * cx + cy * cy) / (2.0 * T) - pr.cp) * fe;
        gs += ag * qc * ge;
      }
      pop_out[i * ps + k] = fs;
      pop_out[(Q + i) * ps + k] = gs;
    }
  } else {
    cnt->fail += 1;
    for (int i = 0; i < NP; ++i) pop_out[i * ps + k] = col[i * B];
  }
  mom_out[k] = rho;
  mom_out[ps + k] = ux;
  mom_out[2 * ps + k] = uy;
  mom_out[3 * ps + k] = T;
  lat_out[k] = (uint8_t)code;
  nxt_out[k] = (uint8_t)code2;
}

__device__ __forceinline__ void flush(unsigned long long* ctr, const Count& c) {
  warp_count(ctr + CTR_NEWTON_ITERS, c.iters);
  warp_count(ctr + CTR_NEWTON_CALLS, c.calls);
  warp_count(ctr + CTR_NEWTON_FAIL, c.fail);
  warp_count(ctr + CTR_REC, c.rec);
  warp_count(ctr + CTR_REC_FAIL, c.rec_fail);
}

// Distinct rebuild solves of a block: every missing pull (owner, i) needs the
// equilibrium of its sender's state in the owner's lattice, and the pulls of
// neighbouring owners often share the sender and the lattice. Phase 1 enters
// each (sender position, lattice) key into a hash table in shared memory;
// phase 2 solves each distinct key once (round-robin over the block) and keeps
// its multipliers; phase 3 forms every missing pull from them (one exponential
// and the Grad factors). Keys beyond the table's capacity are rebuilt in full
// by their owner. A pull's value is a function of its key and velocity only,
// so neither the order of insertion nor the solving thread changes it.
constexpr int HCAP = 512;        // hash positions per block (power of two)
constexpr int SCAP = 192;        // distinct solves kept per block
constexpr int KW = B + 12;       // sender x offsets: x0 - 6 .. x0 + B + 5
constexpr unsigned EMPTY = 0xffffffffu;
constexpr unsigned short NOSLOT = 0xffff;

__device__ __forceinline__ unsigned rebuild_key(int sx, int sy, int x0, int y, int code) {
  return (unsigned)(((sy - y + 6) * KW + (sx - x0 + 6)) * 49 + code);
}

__global__ void __launch_bounds__(B) step_kernel(StepArgs<double> a) {
  extern __shared__ __align__(16) double smem49[];
  __shared__ double s_tab[EXPT_N];
  __shared__ double s_lam[SCAP * M];      // multipliers of the distinct solves
  __shared__ unsigned s_hkey[HCAP];       // hash table: key or EMPTY
  __shared__ unsigned short s_hslot[HCAP];  // solve slot of a key, or NOSLOT
  __shared__ unsigned s_skey[SCAP];       // key of each solve slot
  __shared__ unsigned char s_sok[SCAP];   // 1 if the slot's solve converged
  __shared__ unsigned short s_pos[Q * B];  // hash position of each missing pull
  __shared__ int s_nslots;
  const int t = threadIdx.x;
  for (int j = t; j < HCAP; j += B) s_hkey[j] = EMPTY;
  if (t == 0) s_nslots = 0;
  load_exptab(s_tab);  // includes a barrier
  double* col = smem49 + t;
  double* eq = smem49 + NP * B + t;
  const Params& pr = a.prm;
  const size_t ps = a.ps;
  const int x0 = blockIdx.x * B, y = blockIdx.y;
  const int x = x0 + t;
  const bool active = x < pr.nx;
  Count cnt;
  size_t k = 0;
  int code = 0;
  unsigned long long missing = 0;
  if (active) {
    k = (size_t)y * pr.nx + x;
    code = a.nxt_in[k];
    const int Upx = lat_ux(code), Upy = lat_uy(code);
    for (int i = 0; i < Q; ++i) {
      const int sx = x - vx(i) - Upx, sy = y - vy(i) - Upy;
      bool gh = false;
      const int rx = resolve(sx, pr.nx, pr.bcx, &gh), ry = resolve(sy, pr.ny, pr.bcy, &gh);
      const size_t ks = (size_t)ry * pr.nx + rx;
      if (!gh && a.lat_in[ks] == code) {
        col[i * B] = a.pop_in[i * ps + ks];
        col[(Q + i) * B] = a.pop_in[(Q + i) * ps + ks];
        continue;
      }
      missing |= 1ull << i;
      const unsigned key = rebuild_key(sx, sy, x0, y, code);
      unsigned short pos = NOSLOT;
      unsigned h = (key * 2654435761u) >> 23;  // 9 bits: HCAP = 512
      for (int probe = 0; probe < HCAP; ++probe, h = (h + 1) & (HCAP - 1)) {
        const unsigned old = atomicCAS(&s_hkey[h], EMPTY, key);
        if (old == EMPTY) {
          const int slot = atomicAdd(&s_nslots, 1);
          s_hslot[h] = slot < SCAP ? (unsigned short)slot : NOSLOT;
          if (slot < SCAP) s_skey[slot] = key;
          pos = (unsigned short)h;
          break;
        }
        if (old == key) {
          pos = (unsigned short)h;
          break;
        }
      }
      s_pos[i * B + t] = pos;
    }
  }
  __syncthreads();
  // phase 2: one solve per distinct (sender, lattice), round-robin
  const int ns = s_nslots < SCAP ? s_nslots : SCAP;
  for (int e = t; e < ns; e += B) {
    const unsigned key = s_skey[e];
    const int c = (int)(key % 49u), off = (int)(key / 49u);
    const int sx = x0 + off % KW - 6, sy = y + off / KW - 6;
    const Sender snd = sender_state(pr, a.mom_in, ps, sx, sy);
    double lam[M];
    const int st = sender_solve(pr, snd, lat_ux(c), lat_uy(c), eq, s_tab, lam, &cnt);
    s_sok[e] = st == NEWTON_OK ? 1 : 0;
#pragma unroll
    for (int j = 0; j < M; ++j) s_lam[e * M + j] = lam[j];
  }
  __syncthreads();
  if (active) {
    // phase 3: the node's missing pulls from the solves, then its collision
    const int Upx = lat_ux(code), Upy = lat_uy(code);
    for (int i = 0; i < Q; ++i) {
      if (!((missing >> i) & 1ull)) continue;
      const int sx = x - vx(i) - Upx, sy = y - vy(i) - Upy;
      const unsigned short pos = s_pos[i * B + t];
      const unsigned short slot = pos == NOSLOT ? NOSLOT : s_hslot[pos];
      double fd, gd;
      cnt.rec += 1;
      if (slot == NOSLOT) {
        cnt.rec_fail += rebuild(pr, a.mom_in, ps, i, Upx, Upy, sx, sy, &fd, &gd, eq, s_tab, &cnt);
      } else {
        const Sender snd = sender_state(pr, a.mom_in, ps, sx, sy);
        if (s_sok[slot]) {
          grad_value(pr, snd, i, Upx, Upy, s_lam + slot * M, s_tab, &fd, &gd);
        } else {
          fallback_value(pr, snd, i, Upx, Upy, &fd, &gd);
          cnt.rec_fail += 1;
        }
      }
      col[i * B] = fd;
      col[(Q + i) * B] = gd;
    }
    uint8_t nb[8];
    if (pr.overlap > 0.0 && pr.rule == 1) neighbours(pr, a.nxt_in, x, y, nb);
    collide(pr, col, eq, code, k, ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out, nb, s_tab,
            &cnt);
  }
  flush(a.ctr, cnt);
}

struct InitArgs49 {
  const double *rho, *rhoux, *rhouy, *rhoE;
  double* pop_out;
  double* mom_out;
  uint8_t* lat_out;
  uint8_t* nxt_out;
  size_t ps;
  Params prm;
  unsigned long long* ctr;
};

__device__ __forceinline__ void prim(const InitArgs49& a, size_t k, double* r, double* ux,
                                     double* uy, double* T) {
  *r = a.rho[k];
  *ux = a.rhoux[k] / *r;
  *uy = a.rhouy[k] / *r;
  *T = (a.rhoE[k] - 0.5 * (*r) * ((*ux) * (*ux) + (*uy) * (*uy))) / ((*r) * a.prm.cv);
}

// Initial state (Sec. IV.A.1): h = h^eq (1 + phi_h) in the lattice of Eq.
// criterion for the initial velocity, gradients by central differences of the
// initial fields, then the first collision.
__global__ void __launch_bounds__(B) init_kernel(InitArgs49 a) {
  extern __shared__ __align__(16) double smem49[];
  __shared__ double s_tab[EXPT_N];
  load_exptab(s_tab);
  double* col = smem49 + threadIdx.x;
  double* eq = smem49 + NP * B + threadIdx.x;
  const Params& pr = a.prm;
  const int x = blockIdx.x * B + threadIdx.x, y = blockIdx.y;
  Count cnt;
  unsigned bad = 0;
  if (x < pr.nx) {
    const size_t nx = (size_t)pr.nx;
    const size_t k = (size_t)y * nx + x;
    bool gh = false;
    const int xp = resolve(x + 1, pr.nx, pr.bcx, &gh), xm = resolve(x - 1, pr.nx, pr.bcx, &gh);
    const int yp = resolve(y + 1, pr.ny, pr.bcy, &gh), ym = resolve(y - 1, pr.ny, pr.bcy, &gh);
    double r, ux, uy, T, r1, ux1, uy1, T1, r2, ux2, uy2, T2;
    prim(a, k, &r, &ux, &uy, &T);
    double du[2][2], dT[2];
    prim(a, y * nx + xp, &r1, &ux1, &uy1, &T1);
    prim(a, y * nx + xm, &r2, &ux2, &uy2, &T2);
    du[0][0] = 0.5 * (ux1 - ux2);
    du[0][1] = 0.5 * (uy1 - uy2);
    dT[0] = 0.5 * (T1 - T2);
    prim(a, yp * nx + x, &r1, &ux1, &uy1, &T1);
    prim(a, ym * nx + x, &r2, &ux2, &uy2, &T2);
    du[1][0] = 0.5 * (ux1 - ux2);
    du[1][1] = 0.5 * (uy1 - uy2);
    dT[1] = 0.5 * (T1 - T2);
    const int U0x = select_shift(ux, pr.n0, pr.umax), U0y = select_shift(uy, pr.n0, pr.umax);
    const int code = lat_code(U0x, U0y);
    const bool ok = (r > 0.0) && (T > 0.0) && isfinite(r) && isfinite(T);
    double lam[M];
    int it = 0;
    const int ns = ok ? newton13(ux - U0x, uy - U0y, T, pr.tol, pr.maxit, eq, s_tab, lam, &it)
                      : NEWTON_UNREALIZABLE;
    if (!ok) bad += 1;
    if (ok && ns != NEWTON_OK) cnt.fail += 1;
    if (ns == NEWTON_OK) {
      const double gfac = (2.0 * pr.cv - 2.0) * T;
      for (int i = 0; i < Q; ++i) {
        const double cbx = (double)(vx(i) + U0x) - ux, cby = (double)(vy(i) + U0y) - uy;
        double phf, phg, phq;
        grad_phi(pr, r, T, cbx, cby, du, dT, &phf, &phg, &phq);
        const double feq = r * eq[i * B];
        col[i * B] = feq * (1.0 + phf);
        col[(Q + i) * B] = gfac * feq * (1.0 + phg);
      }
      uint8_t nb[8];
      if (pr.overlap > 0.0 && pr.rule == 1) {
        int m = 0;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            bool g2 = false;
            const size_t kk = (size_t)resolve(y + dy, pr.ny, pr.bcy, &g2) * nx +
                              resolve(x + dx, pr.nx, pr.bcx, &g2);
            const double rr = a.rho[kk];
            nb[m++] = (uint8_t)lat_code(select_shift(a.rhoux[kk] / rr, pr.n0, pr.umax),
                                        select_shift(a.rhouy[kk] / rr, pr.n0, pr.umax));
          }
      }
      collide(pr, col, eq, code, k, a.ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out, nb, s_tab,
              &cnt);
    } else {
      for (int i = 0; i < NP; ++i) a.pop_out[i * a.ps + k] = 0.0;
      a.mom_out[k] = r;
      a.mom_out[a.ps + k] = ux;
      a.mom_out[2 * a.ps + k] = uy;
      a.mom_out[3 * a.ps + k] = T;
      a.lat_out[k] = (uint8_t)code;
      a.nxt_out[k] = (uint8_t)code;
    }
  }
  // the initial solves are not step work: only failures are counted
  warp_count(a.ctr + CTR_UNREALIZABLE, bad);
  warp_count(a.ctr + CTR_NEWTON_FAIL, cnt.fail);
}

// Stateless equilibria for the C ABI: one node per thread.
__global__ void __launch_bounds__(B)
    equilibrium_kernel(const double* rho, const double* ubx, const double* uby, const double* T,
                       int n, double tol, int maxit, double* feq, double* lambda, int* iters,
                       int* status) {
  __shared__ double s_eq[Q * B];
  __shared__ double s_tab[EXPT_N];
  load_exptab(s_tab);
  const int k = blockIdx.x * B + threadIdx.x;
  if (k >= n) return;
  double* eq = s_eq + threadIdx.x;
  double lam[M];
  int it = 0;
  const double r = rho[k];
  const int st = (r > 0.0 && isfinite(r))
                     ? newton13(ubx[k], uby[k], T[k], tol, maxit, eq, s_tab, lam, &it)
                     : NEWTON_UNREALIZABLE;
  for (int i = 0; i < Q; ++i) feq[(size_t)k * Q + i] = st == NEWTON_OK ? r * eq[i * B] : 0.0;
  for (int j = 0; j < M; ++j) lambda[(size_t)k * M + j] = st == NEWTON_OK ? lam[j] : 0.0;
  iters[k] = it;
  status[k] = st;
}

static dim3 grid_of(const Params& p) { return dim3((p.nx + B - 1) / B, p.ny); }

}  // namespace q49

cudaError_t launch_init_q49(FlowDev& f, const double* rho, const double* rhoux,
                            const double* rhouy, const double* rhoE, cudaStream_t s) {
  const int out = f.cur;
  q49::InitArgs49 a{rho, rhoux, rhouy, rhoE, (double*)f.pop[out], (double*)f.mom[out],
                    f.lat[out], f.nxt[out], f.ps, f.prm, f.ctr};
  cudaError_t e = cudaFuncSetAttribute(q49::init_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)q49::SMEM);
  if (e != cudaSuccess) return e;
  q49::init_kernel<<<q49::grid_of(f.prm), q49::B, q49::SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_step_q49(FlowDev& f, cudaStream_t s) {
  const int in = f.cur, out = f.cur ^ 1;
  const StepArgs<double> a = step_args<double>(f, in);
  cudaError_t e = cudaFuncSetAttribute(q49::step_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)q49::SMEM);
  if (e != cudaSuccess) return e;
  q49::step_kernel<<<q49::grid_of(f.prm), q49::B, q49::SMEM, s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) f.cur = out;
  return e;
}

cudaError_t launch_equilibrium13(const double* rho, const double* ubx, const double* uby,
                                 const double* T, int n, double tol, int maxit, double* feq,
                                 double* lambda, int* iters, int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  q49::equilibrium_kernel<<<(n + q49::B - 1) / q49::B, q49::B, 0, s>>>(
      rho, ubx, uby, T, n, tol, maxit, feq, lambda, iters, status);
  return cudaGetLastError();
}

}  // namespace alb
