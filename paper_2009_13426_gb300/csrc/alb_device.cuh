// Device-side building blocks of the adaptive D2Q21 LBM step (sm_103a).
//
// The lattice, the 8-moment numerical equilibrium and its FP64 Newton solve,
// the shift criterion and Grad's reconstruction, written for one node per
// thread. Loops over velocities are fully unrolled with compile-time velocity
// components, so every multiplication by a zero component disappears and the
// sums below touch only the velocities that contribute.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "alb_cvt.cuh"

namespace alb {

constexpr int Q = 21;   // D2Q21
constexpr int NM = 8;   // 8-moment constraint set (Eq. 8moments)
constexpr int NPLANES = 2 * Q;  // f and g planes

// D2Q21 velocity set (Fig. 1 / Tab. 3 reading): rest, axis 1, diagonal 1,
// axis 2, diagonal 2, axis 3. The index order is part of the C ABI
// (alb_velocities, alb_equilibrium).
__host__ __device__ __forceinline__ constexpr int XI_X(int i) {
  return i == 1 ? 1 : i == 3 ? -1 : i == 5 ? 1 : i == 6 ? -1 : i == 7 ? -1 : i == 8 ? 1
       : i == 9 ? 2 : i == 11 ? -2 : i == 13 ? 2 : i == 14 ? -2 : i == 15 ? -2 : i == 16 ? 2
       : i == 17 ? 3 : i == 19 ? -3 : 0;
}
__host__ __device__ __forceinline__ constexpr int XI_Y(int i) {
  return i == 2 ? 1 : i == 4 ? -1 : i == 5 ? 1 : i == 6 ? 1 : i == 7 ? -1 : i == 8 ? -1
       : i == 10 ? 2 : i == 12 ? -2 : i == 13 ? 2 : i == 14 ? 2 : i == 15 ? -2 : i == 16 ? -2
       : i == 18 ? 3 : i == 20 ? -3 : 0;
}
// Monomial k of the 8-moment set at velocity i: 1, x, y, x^2, xy, y^2, x|xi|^2, y|xi|^2.
__host__ __device__ __forceinline__ constexpr int PM(int k, int i) {
  return k == 0 ? 1 : k == 1 ? XI_X(i) : k == 2 ? XI_Y(i) : k == 3 ? XI_X(i) * XI_X(i)
       : k == 4 ? XI_X(i) * XI_Y(i) : k == 5 ? XI_Y(i) * XI_Y(i)
       : k == 6 ? XI_X(i) * (XI_X(i) * XI_X(i) + XI_Y(i) * XI_Y(i))
       : XI_Y(i) * (XI_X(i) * XI_X(i) + XI_Y(i) * XI_Y(i));
}

// Lattice code of a shift U in [-3, 3]^2: one byte per node.
__host__ __device__ __forceinline__ int lat_code(int ux, int uy) { return (ux + 3) + 7 * (uy + 3); }
__host__ __device__ __forceinline__ int lat_ux(int c) { return c % 7 - 3; }
__host__ __device__ __forceinline__ int lat_uy(int c) { return c / 7 - 3; }

// A double in the population precision P: FP32 rounded on the integer pipe
// (cvt_f32_rn, the hardware rounding for every value of FP32's normal range),
// FP64 unchanged.
template <typename P>
__device__ __forceinline__ P to_p(double v);
template <>
__device__ __forceinline__ float to_p<float>(double v) { return cvt_f32_rn(v); }
template <>
__device__ __forceinline__ double to_p<double>(double v) { return v; }

// Physical and numerical parameters of one flow, passed by value.
struct Params {
  int nx, ny;
  int umax;
  int bcx, bcy;      // 0 periodic, 1 zero-gradient
  int sensor;
  int maxit;
  int warm;          // 1: solves start from the previous step's multipliers
  int rule;          // where ranges overlap: 0 history, 1 neighbourhood
  int moments;       // constraint set: 8, or 4 (reduced model)
  int shakhov;       // 1: Pr != 1, heat-flux term of App. E in the collision
  double nu, gamma, n0, tol;
  double prandtl;    // Pr: tau_Pr = 1/2 + (nu/Pr)/T, kappa = rho Cp nu / Pr
  double overlap;    // widening of the current shift's range (0: Eq. criterion)
  double cv, cp;     // Cv = 1/(gamma-1), Cp = gamma Cv
  double half_gm1;   // (gamma - 1) / 2 = 1 / (2 Cv)
  double seps[3], salpha[3];
  double skx[4], sky[4];  // sensor knots: log10(eps) and alpha (host-computed)
  double thr[6];          // criterion thresholds (t + 1) - n0, t = -umax .. umax - 1
  double wlo[7], whi[7];  // widened range of shift n = j - 3: ((n - n0) - w, ((n + 1) - n0) + w]
};

// Comparisons of the criterion on the integer pipe: the FP64 pipe bounds the
// step, and an FP64 compare takes one of its slots. order_key maps a double's
// bits to a signed integer in IEEE order (negative values have their
// magnitude bits flipped). Integer order then equals IEEE order for all
// non-NaN values except +0 against -0, which cannot meet here: the host's
// thresholds are differences of distinct values, never -0, and a velocity
// ubar + U with an integer U is never -0. A NaN u compares false both ways,
// as in IEEE.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool not_nan(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool gt_order(double u, double v) {  // u > v
  return not_nan(u) && order_key(u) > order_key(v);
}
__device__ __forceinline__ bool le_order(double u, double v) {  // u <= v
  return not_nan(u) && order_key(u) <= order_key(v);
}

// Eq. criterion with the host-computed thresholds of Params (the same IEEE
// values as select_shift computes).
__device__ __forceinline__ int select_shift_thr(double u, const Params& pr) {
  int n = -pr.umax;
#pragma unroll
  for (int t = 0; t < 6; ++t)
    if (t < 2 * pr.umax && gt_order(u, pr.thr[t])) ++n;
  return n;
}

// Overlapping ranges chosen by history (Sec. III.A.2): keep the current shift
// while current - n0 - w < u <= current + 1 - n0 + w, else Eq. criterion.
// The widened bounds come from the host (same IEEE operations as the oracle).
__device__ __forceinline__ int select_shift_kept(double u, int current, const Params& pr) {
  if (order_key(pr.overlap) > 0 && gt_order(u, pr.wlo[current + 3]) &&
      le_order(u, pr.whi[current + 3]))
    return current;
  return select_shift_thr(u, pr);
}

// Overlapping ranges chosen by the neighbourhood (Sec. III.A.2): among the
// shifts whose widened range holds u, the one most of the eight surrounding
// nodes use (component `axis` of their lattice codes nb[0..7]); the
// criterion's shift unless another candidate is used by strictly more.
__device__ __forceinline__ int select_shift_neighbours(double u, int axis, const uint8_t nb[8],
                                                       const Params& pr) {
  const int c = select_shift_thr(u, pr);
  int cnt[7] = {0, 0, 0, 0, 0, 0, 0};  // neighbours per shift n = j - 3
#pragma unroll
  for (int j = 0; j < 8; ++j) cnt[(axis ? lat_uy(nb[j]) : lat_ux(nb[j])) + 3] += 1;
  int best = c, best_count = cnt[c + 3];
  // with w <= 1 only the criterion's neighbours c - 1 and c + 1 can also hold u
#pragma unroll
  for (int d = -1; d <= 1; d += 2) {
    const int n = c + d;
    if (n < -pr.umax || n > pr.umax) continue;
    if (!(gt_order(u, pr.wlo[n + 3]) && le_order(u, pr.whi[n + 3]))) continue;
    if (cnt[n + 3] > best_count) {
      best = n;
      best_count = cnt[n + 3];
    }
  }
  return best;
}

// s + c * v with c a compile-time integer after unrolling: the zero and unit
// cases fold away, keeping IEEE semantics for the rest.
template <typename R>
__device__ __forceinline__ R madd(R s, R v, int c) {
  if (c == 0) return s;
  if (c == 1) return s + v;
  if (c == -1) return s - v;
  return fma(v, (R)c, s);
}

// Eq. criterion with offset n0: U = n iff n - n0 < u <= n + 1 - n0, clamped.
__device__ __forceinline__ int select_shift(double u, double n0, int umax) {
  int n = -umax;
  // count the thresholds n + 1 - n0 (n = -umax .. umax-1) that u lies above
  for (int t = -umax; t < umax; ++t) {
    const double hi = (double)(t + 1) - n0;
    if (u > hi) n = t + 1;
  }
  return n;
}

// alpha(eps_Kn) of the kinetic sensor (Sec. IV.A.2): 1 up to seps[0], then
// continuous and piecewise linear in log10(eps) through (seps[1], salpha[0]),
// (seps[2], salpha[1]), (10 seps[2], salpha[2]), constant beyond. Evaluated
// in the population precision P.
template <typename P>
__device__ __forceinline__ P sensor_alpha(const Params& pr, P eps) {
  if (!(eps > to_p<P>(pr.seps[0]))) return (P)1;
  const P l = log10(eps);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (l <= (P)pr.skx[k + 1])
      return (P)pr.sky[k] + ((P)pr.sky[k + 1] - (P)pr.sky[k]) * (l - (P)pr.skx[k]) /
                                ((P)pr.skx[k + 1] - (P)pr.skx[k]);
  return (P)pr.sky[3];
}

// Targets of Eqs. G0_8mom..G3yaa_8mom per unit density, lattice frame.
__device__ __forceinline__ void targets(double ubx, double uby, double T, double m[NM]) {
  const double u2 = ubx * ubx + uby * uby;
  m[0] = 1.0;
  m[1] = ubx;
  m[2] = uby;
  m[3] = ubx * ubx + T;
  m[4] = ubx * uby;
  m[5] = uby * uby + T;
  m[6] = ubx * (u2 + 4.0 * T);
  m[7] = uby * (u2 + 4.0 * T);
}

// p_i = exp(-(1 + lambda . P(xi_i))) for all 21 velocities (Eq. exponential / rho).
__device__ __forceinline__ void exp_family(const double lam[NM], double p[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double s = 1.0 + lam[0];
#pragma unroll
    for (int k = 1; k < NM; ++k) s = madd(s, lam[k], PM(k, i));
    p[i] = exp(-s);
  }
}

enum { NEWTON_OK = 0, NEWTON_MAXIT = 1, NEWTON_SINGULAR = 2, NEWTON_UNREALIZABLE = 3 };

// Maxwellian starting multipliers, lambda_0 from the normalisation sum p = 1.
__device__ __forceinline__ void maxwellian_guess(double ubx, double uby, double T, double lam[NM]) {
  const double iT = 1.0 / T;
#pragma unroll
  for (int k = 0; k < NM; ++k) lam[k] = 0.0;
  lam[1] = -ubx * iT;
  lam[2] = -uby * iT;
  lam[3] = 0.5 * iT;
  lam[5] = 0.5 * iT;
  double p[Q];
  exp_family(lam, p);
  double Z = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) Z += p[i];
  lam[0] = log(Z);
}

// exp(-(1 + lambda . P(xi_i))) for one velocity given at run time.
__device__ __forceinline__ double exp_family_one(const double lam[NM], int cx, int cy) {
  const double x = cx, y = cy, r2 = x * x + y * y;
  double s = 1.0 + lam[0];
  s = fma(lam[1], x, s);
  s = fma(lam[2], y, s);
  s = fma(lam[3], x * x, s);
  s = fma(lam[4], x * y, s);
  s = fma(lam[5], y * y, s);
  s = fma(lam[6], x * r2, s);
  s = fma(lam[7], y * r2, s);
  return exp(-s);
}

// Grad's factors (Eqs. GradGeneral_f, GradGeneral_g) for cbar = c_i - u:
// phi_f = phi_s + phi_q with phi_s the traceless viscous stress part (mu =
// rho nu) and phi_q the Fourier heat-flux part (kappa = rho Cp nu / Pr), and
// phi_g. phi_q has the shape of the heat-flux term of App. E.
__device__ __forceinline__ void grad_phi(const Params& pr, double rho, double T, double cbx,
                                         double cby, const double du[2][2], const double dT[2],
                                         double* phi_f, double* phi_g, double* phi_q) {
  const double mu = rho * pr.nu;
  const double kappa = rho * pr.cp * pr.nu / pr.prandtl;
  const double div = du[0][0] + du[1][1];
  const double sxx = -mu * (2.0 * du[0][0] - div);
  const double syy = -mu * (2.0 * du[1][1] - div);
  const double sxy = -mu * (du[0][1] + du[1][0]);
  const double qx = -kappa * dT[0];
  const double qy = -kappa * dT[1];
  const double c2 = cbx * cbx + cby * cby;
  const double qc = qx * cbx + qy * cby;
  const double iT = 1.0 / T;
  const double ps = (sxx * cbx * cbx + 2.0 * sxy * cbx * cby + syy * cby * cby) *
                    (0.5 * iT * iT / rho);
  const double pq = qc * (iT * iT / (rho * pr.cp)) * (0.5 * c2 * iT - pr.cp);
  *phi_f = ps + pq;
  *phi_q = pq;
  *phi_g = 2.0 * qc / (rho * pr.cp);
}

// Resolve a coordinate along one axis: periodic wrap or zero-gradient clamp.
__device__ __forceinline__ int resolve(int x, int n, int bc, bool* ghost) {
  if (bc == 0) {
    if ((unsigned)x < (unsigned)n) return x;  // inside: no remainder needed
    int r = x % n;
    if (r < 0) r += n;
    return r;
  }
  if (x < 0) { *ghost = true; return 0; }
  if (x >= n) { *ghost = true; return n - 1; }
  return x;
}

// Warp-aggregated counter increment (all lanes of the warp must call it).
__device__ __forceinline__ void warp_count(unsigned long long* ctr, unsigned v) {
  const unsigned s = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

}  // namespace alb
