// Mixed-precision solver of the 8-moment numerical equilibrium, FP32 form.
//
// The multipliers of Eq. feqNum_8Mom solve G(lambda) = 0 (Eqs. G0_8mom..
// G3yaa_8mom). On GB300 the FP64 pipe runs at 1/62 of the FP32 rate, so the
// Newton iterations run in FP32 (exponentials, exact Jacobian, Jacobi-scaled
// Cholesky), and FP64 is used only where the accuracy of the result comes
// from: the residual. The FP64 refinement evaluates the 21 exponentials and
// the 8 constraint residuals in FP64 and corrects lambda with the FP32
// Cholesky factor (iterative refinement of the Newton step) until
// max_k |G_k| / rho <= tol, the same criterion as the full FP64 Newton. If the
// FP32 phase or the refinement fails, the full FP64 Newton takes over.
//
// The FP64 exponential is table-driven (Tang, ACM TOMS 15(2), 1989):
// exp(-s) = 2^(n/32) exp(r), n = round(-32 s / ln 2), |r| <= ln2/64, with
// 2^(j/32) from a 32-entry table and exp(r) by its degree-6 Taylor polynomial
// (constants in exp_table.h, generated by gen_exp_table.py).
//
// Exponents and constraint sums use the symmetry of the velocity set: for each
// pair (or quadruple) of velocities related by a sign change, the sum and
// difference (butterfly) are formed once and shared by all moments.
#pragma once

#include "alb_device.cuh"
#include "exp_table.h"

namespace alb {

// Exponents s_i = 1 + lambda . P(xi_i) for the 21 velocities (index order of
// XI_X / XI_Y), built from the even and odd parts of each symmetric group.
template <typename R>
__device__ __forceinline__ void exponents(const R l[NM], R s[Q]) {
  const R c = (R)1 + l[0];
  s[0] = c;
  {  // axis, |xi| = 1
    const R ex = c + l[3], ox = l[1] + l[6];
    s[1] = ex + ox;
    s[3] = ex - ox;
    const R ey = c + l[5], oy = l[2] + l[7];
    s[2] = ey + oy;
    s[4] = ey - oy;
  }
  {  // axis, |xi| = 2
    const R ex = fma((R)4, l[3], c), ox = fma((R)8, l[6], (R)2 * l[1]);
    s[9] = ex + ox;
    s[11] = ex - ox;
    const R ey = fma((R)4, l[5], c), oy = fma((R)8, l[7], (R)2 * l[2]);
    s[10] = ey + oy;
    s[12] = ey - oy;
  }
  {  // axis, |xi| = 3
    const R ex = fma((R)9, l[3], c), ox = fma((R)27, l[6], (R)3 * l[1]);
    s[17] = ex + ox;
    s[19] = ex - ox;
    const R ey = fma((R)9, l[5], c), oy = fma((R)27, l[7], (R)3 * l[2]);
    s[18] = ey + oy;
    s[20] = ey - oy;
  }
  const R l35 = l[3] + l[5];
  {  // diagonal (+-1, +-1): s = E + sx sy Z + sx X + sy Y
    const R E = c + l35;
    const R X = fma((R)2, l[6], l[1]), Y = fma((R)2, l[7], l[2]);
    const R Ep = E + l[4], Em = E - l[4];
    const R XpY = X + Y, XmY = X - Y;
    s[5] = Ep + XpY;  // ( 1, 1)
    s[7] = Ep - XpY;  // (-1,-1)
    s[8] = Em + XmY;  // ( 1,-1)
    s[6] = Em - XmY;  // (-1, 1)
  }
  {  // diagonal (+-2, +-2)
    const R E = fma((R)4, l35, c);
    const R X = fma((R)16, l[6], (R)2 * l[1]), Y = fma((R)16, l[7], (R)2 * l[2]);
    const R Z = (R)4 * l[4];
    const R Ep = E + Z, Em = E - Z;
    const R XpY = X + Y, XmY = X - Y;
    s[13] = Ep + XpY;  // ( 2, 2)
    s[15] = Ep - XpY;  // (-2,-2)
    s[16] = Em + XmY;  // ( 2,-2)
    s[14] = Em - XmY;  // (-2, 2)
  }
}

// The 8 constraint moments M_k = sum_i p_i P_k(xi_i) (Eq. 8moments order).
template <typename R>
__device__ __forceinline__ void moments8(const R p[Q], R M[NM]) {
  R m0 = p[0], m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0, m6 = 0, m7 = 0;
  // axis pairs (+a, -a) along x and y, a = 1, 2, 3
  const int ax[3][2] = {{1, 3}, {9, 11}, {17, 19}};
  const int ay[3][2] = {{2, 4}, {10, 12}, {18, 20}};
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    const R Sx = p[ax[a - 1][0]] + p[ax[a - 1][1]], Dx = p[ax[a - 1][0]] - p[ax[a - 1][1]];
    const R Sy = p[ay[a - 1][0]] + p[ay[a - 1][1]], Dy = p[ay[a - 1][0]] - p[ay[a - 1][1]];
    m0 += Sx + Sy;
    m1 = madd(m1, Dx, a);
    m2 = madd(m2, Dy, a);
    m3 = madd(m3, Sx, a * a);
    m5 = madd(m5, Sy, a * a);
    m6 = madd(m6, Dx, a * a * a);
    m7 = madd(m7, Dy, a * a * a);
  }
  // diagonal quadruples (a,a), (a,-a), (-a,a), (-a,-a), a = 1, 2
  const int dg[2][4] = {{5, 8, 6, 7}, {13, 16, 14, 15}};  // (++), (+-), (-+), (--)
#pragma unroll
  for (int a = 1; a <= 2; ++a) {
    const R A = p[dg[a - 1][0]] + p[dg[a - 1][1]];  // sx = +1
    const R B = p[dg[a - 1][2]] + p[dg[a - 1][3]];  // sx = -1
    const R C = p[dg[a - 1][0]] - p[dg[a - 1][1]];
    const R D = p[dg[a - 1][2]] - p[dg[a - 1][3]];
    const R sum = A + B, xs = A - B, ys = C + D, xys = C - D;
    m0 += sum;
    m1 = madd(m1, xs, a);
    m2 = madd(m2, ys, a);
    m3 = madd(m3, sum, a * a);
    m4 = madd(m4, xys, a * a);
    m5 = madd(m5, sum, a * a);
    m6 = madd(m6, xs, 2 * a * a * a);
    m7 = madd(m7, ys, 2 * a * a * a);
  }
  M[0] = m0; M[1] = m1; M[2] = m2; M[3] = m3; M[4] = m4; M[5] = m5; M[6] = m6; M[7] = m7;
}

// 2^(j/32), j = 0..31; kernels copy it to shared memory (lanes index it freely).
static __constant__ double c_exptab[32] = {ALB_EXPT_TABLE_VALUES};

// Copy the table into a block's shared array (all threads; includes a barrier).
__device__ __forceinline__ void load_exptab(double* s_tab) {
  if (threadIdx.x < 32) s_tab[threadIdx.x] = c_exptab[threadIdx.x];
  __syncthreads();
}

// Table-driven FP64 exp(-s); tab = 2^(j/32), j = 0..31 (in shared memory).
// Returns 0 below 2^-1022 (no subnormal results) and +inf from 2^1024 on.
__device__ __forceinline__ double exp_neg(double s, const double* tab) {
  const double shifter = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer
  const double t = fma(-s, EXPT_INV_L, shifter);
  const int n = (int)(unsigned)__double2loint(t);
  const double nd = t - shifter;
  double r = fma(nd, -EXPT_L_HI, -s);
  r = fma(nd, -EXPT_L_LO, r);
  double q = fma(r, EXPT_C6, EXPT_C5);
  q = fma(q, r, EXPT_C4);
  q = fma(q, r, EXPT_C3);
  q = fma(q, r, EXPT_C2);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  const int e = n >> 5;
  const long long bits = __double_as_longlong(tab[n & 31]) + ((long long)e << 52);
  double sc = __longlong_as_double(bits);
  sc = e < -1022 ? 0.0 : (e > 1023 ? __longlong_as_double(0x7ff0000000000000LL) : sc);
  return q * sc;
}

// exp(-s) for the 21 velocities in FP32 (CUDA expf).
__device__ __forceinline__ void exp_family32(const float l[NM], float p[Q]) {
  float s[Q];
  exponents<float>(l, s);
#pragma unroll
  for (int i = 0; i < Q; ++i) p[i] = expf(-s[i]);
}

// Jacobi-scaled Cholesky factor of the Jacobian sum_i p_i P P^T, FP32.
struct Fact32 {
  float d[NM];       // scaling 1/sqrt(H_kk)
  float L[NM][NM];   // lower factor of D H D
};

__device__ __forceinline__ bool factor32(const float p[Q], Fact32& fc) {
  float H[NM][NM];
#pragma unroll
  for (int a = 0; a < NM; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      float s = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i) s = madd(s, p[i], PM(a, i) * PM(b, i));
      H[a][b] = s;
    }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    ok = ok && (H[k][k] > 0.0f);
    fc.d[k] = rsqrtf(fmaxf(H[k][k], 1e-30f));
  }
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    float dj = H[j][j] * fc.d[j] * fc.d[j];
#pragma unroll
    for (int k = 0; k < j; ++k) dj = fmaf(-fc.L[j][k], fc.L[j][k], dj);
    ok = ok && (dj > 0.0f);
    const float il = rsqrtf(fmaxf(dj, 1e-30f));
    fc.L[j][j] = dj * il;
#pragma unroll
    for (int i = j + 1; i < NM; ++i) {
      float s = H[i][j] * fc.d[i] * fc.d[j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = fmaf(-fc.L[i][k], fc.L[j][k], s);
      fc.L[i][j] = s * il;
    }
  }
  return ok;
}

// delta = H^-1 g with the scaled factor.
__device__ __forceinline__ void solve32(const Fact32& fc, const float g[NM], float dl[NM]) {
  float y[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    float s = g[i] * fc.d[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = fmaf(-fc.L[i][k], y[k], s);
    y[i] = s / fc.L[i][i];
  }
#pragma unroll
  for (int i = NM - 1; i >= 0; --i) {
    float s = y[i];
#pragma unroll
    for (int k = i + 1; k < NM; ++k) s = fmaf(-fc.L[k][i], y[k], s);
    y[i] = s / fc.L[i][i];
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) dl[i] = y[i] * fc.d[i];
}

// Multipliers in the frame of another lattice: lam'.P(u) = lam.P(u - d) for
// every velocity u, where d = U - U' (a velocity xi relative to lattice U is
// xi - d relative to U'). Exact for the exponential; it serves as the starting
// point of the Newton iteration after a change of lattice.
__device__ __forceinline__ void shift_multipliers(const float l[NM], float dx, float dy,
                                                  float o[NM]) {
  const float d2 = dx * dx + dy * dy;
  o[0] = l[0] - l[1] * dx - l[2] * dy + l[3] * dx * dx + l[4] * dx * dy + l[5] * dy * dy -
         l[6] * dx * d2 - l[7] * dy * d2;
  o[1] = l[1] - 2.0f * l[3] * dx - l[4] * dy + l[6] * (3.0f * dx * dx + dy * dy) +
         2.0f * l[7] * dx * dy;
  o[2] = l[2] - l[4] * dx - 2.0f * l[5] * dy + 2.0f * l[6] * dx * dy +
         l[7] * (dx * dx + 3.0f * dy * dy);
  o[3] = l[3] - 3.0f * l[6] * dx - l[7] * dy;
  o[4] = l[4] - 2.0f * l[6] * dy - 2.0f * l[7] * dx;
  o[5] = l[5] - l[6] * dx - 3.0f * l[7] * dy;
  o[6] = l[6];
  o[7] = l[7];
}

// FP32 phase: damped Newton from lam (warm start) or, if warm is false, from
// the Maxwellian; on success fc holds the factor of the Jacobian at the
// returned multipliers. Returns NEWTON_OK or NEWTON_SINGULAR (non-finite
// values or a non-positive pivot).
static __device__ __noinline__ int newton_fp32(float ubx, float uby, float T, int maxit, bool warm,
                                               float lam[NM], Fact32& fc, int* iters) {
  *iters = 0;
  float m[NM];
  {
    const float u2 = ubx * ubx + uby * uby;
    m[0] = 1.0f; m[1] = ubx; m[2] = uby;
    m[3] = fmaf(ubx, ubx, T); m[4] = ubx * uby; m[5] = fmaf(uby, uby, T);
    m[6] = ubx * fmaf(4.0f, T, u2); m[7] = uby * fmaf(4.0f, T, u2);
  }
  float p[Q];
  if (warm) {
    exp_family32(lam, p);
    float Z = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) Z += p[i];
    warm = isfinite(Z) && Z > 0.0f;
  }
  if (!warm) {
    const float iT = 1.0f / T;
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = 0.0f;
    lam[1] = -ubx * iT;
    lam[2] = -uby * iT;
    lam[3] = 0.5f * iT;
    lam[5] = 0.5f * iT;
    exp_family32(lam, p);
    float Z = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) Z += p[i];
    const float l0 = logf(Z);
    const float iz = 1.0f / Z;
    lam[0] = l0;
#pragma unroll
    for (int i = 0; i < Q; ++i) p[i] *= iz;
  }
  auto dual = [&](const float* l, const float* pp) {
    float F = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) F += pp[i];
#pragma unroll
    for (int k = 0; k < NM; ++k) F = fmaf(l[k], m[k], F);
    return F;
  };
  float F = dual(lam, p);
  int it = 0;
  for (; it < maxit; ++it) {
    float G[NM];
    moments8<float>(p, G);
    float gmax = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      G[k] -= m[k];
      gmax = fmaxf(gmax, fabsf(G[k]));
    }
    if (!isfinite(gmax)) return NEWTON_SINGULAR;
    if (gmax <= 2e-7f) break;
    if (!factor32(p, fc)) return NEWTON_SINGULAR;
    float dl[NM];
    solve32(fc, G, dl);
    float gd = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) gd = fmaf(G[k], dl[k], gd);
    if (!(gd > 1e-14f)) break;  // no further progress is measurable in FP32
    float t = 1.0f, lc[NM], pc[Q], Fc = 0.0f;
    bool acc = false;
    for (int ls = 0; ls < 24; ++ls) {
#pragma unroll
      for (int k = 0; k < NM; ++k) lc[k] = fmaf(t, dl[k], lam[k]);
      exp_family32(lc, pc);
      Fc = dual(lc, pc);
      if (isfinite(Fc) && Fc <= F - 1e-4f * t * gd + 4e-7f * fabsf(F)) {
        acc = true;
        break;
      }
      t *= 0.5f;
    }
    if (!acc) break;
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = lc[k];
#pragma unroll
    for (int i = 0; i < Q; ++i) p[i] = pc[i];
    F = Fc;
  }
  *iters = it;
  return factor32(p, fc) ? NEWTON_OK : NEWTON_SINGULAR;
}

// FP64 refinement: lambda <- lambda + H32^-1 G64(lambda) until max|G|/rho <= tol.
// On NEWTON_OK, p holds exp(-s) in FP64 at the returned lambda.
static __device__ __noinline__ int refine_fp64(double ubx, double uby, double T, double tol,
                                               int maxr, const float lam32[NM], const Fact32& fc,
                                               const double* tab, double lam[NM], double p[Q],
                                               int* evals) {
  double m[NM];
  targets(ubx, uby, T, m);
#pragma unroll
  for (int k = 0; k < NM; ++k) lam[k] = (double)lam32[k];
  *evals = 0;
  for (int r = 0;; ++r) {
    double s[Q];
    exponents<double>(lam, s);
#pragma unroll
    for (int i = 0; i < Q; ++i) p[i] = exp_neg(s[i], tab);
    double G[NM];
    moments8<double>(p, G);
    ++*evals;
    double gmax = 0.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      G[k] -= m[k];
      gmax = fmax(gmax, fabs(G[k]));
    }
    if (!isfinite(gmax)) return NEWTON_SINGULAR;
    if (gmax <= tol) return NEWTON_OK;
    if (r >= maxr) return NEWTON_MAXIT;
    float g32[NM], dl[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) g32[k] = (float)G[k];
    solve32(fc, g32, dl);
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] += (double)dl[k];
  }
}

// Work counts of one equilibrium solve.
struct SolveCount {
  unsigned fp32_iters = 0, fp64_evals = 0, fp64_iters = 0;
};

// Equilibrium of the FP32 form: FP32 Newton (from the warm start if given,
// else from the Maxwellian; again from the Maxwellian if the warm start
// fails), FP64 refinement, full FP64 Newton as the last fallback. p receives
// exp(-(1 + lambda . P)) in FP64.
__device__ __forceinline__ int equilibrium_mixed(double ubx, double uby, double T, double tol,
                                                 int maxit, const double* tab, const float* warm,
                                                 double lam[NM], double p[Q], SolveCount* cnt) {
  if (!(T > 0.0) || !isfinite(T) || !isfinite(ubx) || !isfinite(uby)) return NEWTON_UNREALIZABLE;
  float lam32[NM];
  Fact32 fc;
  int it32 = 0, ev = 0;
  int st = NEWTON_SINGULAR;
  if (warm) {
#pragma unroll
    for (int k = 0; k < NM; ++k) lam32[k] = warm[k];
    st = newton_fp32((float)ubx, (float)uby, (float)T, 30, true, lam32, fc, &it32);
    cnt->fp32_iters += it32;
  }
  if (st != NEWTON_OK) {
    st = newton_fp32((float)ubx, (float)uby, (float)T, 30, false, lam32, fc, &it32);
    cnt->fp32_iters += it32;
  }
  if (st == NEWTON_OK) {
    st = refine_fp64(ubx, uby, T, tol, 6, lam32, fc, tab, lam, p, &ev);
    cnt->fp64_evals += ev;
  }
  if (st != NEWTON_OK) {
    int it = 0;
    st = newton_fp64(ubx, uby, T, tol, maxit, lam, p, &it, &ev);
    cnt->fp64_iters += it;
    cnt->fp64_evals += ev;
  }
  return st;
}

}  // namespace alb
