// Mixed-precision solver of the 8-moment numerical equilibrium, FP32 form.
//
// The multipliers of Eq. feqNum_8Mom solve G(lambda) = 0 (Eqs. G0_8mom..
// G3yaa_8mom). On GB300 the FP64 pipe runs at 1/62 of the FP32 rate, so the
// Newton iterations run in FP32 (exponentials, exact Jacobian, Cholesky
// factor), and FP64 is used only where the accuracy of the result comes
// from: the residual. The FP64 refinement evaluates the 21 exponentials and
// the 8 constraint residuals in FP64 and corrects lambda with the FP32
// Cholesky factor (iterative refinement of the Newton step) until
// max_k |G_k| / rho <= tol, the same criterion as the full FP64 Newton. If the
// FP32 phase or the refinement fails, the full FP64 Newton takes over.
//
// The FP64 exponential is table-driven (Tang, ACM TOMS 15(2), 1989):
// exp(-s) = 2^(n/256) exp(r), n = round(-256 s / ln 2), |r| <= ln2/512, with
// 2^(j/256) from a 256-entry table and exp(r) by its degree-4 Taylor
// polynomial (constants in exp_table.h, generated by gen_exp_table.py).
//
// Every pass over the velocities streams through the symmetric groups of the
// D2Q21 set (the rest velocity, the axis pairs +-a, the diagonal quadruples):
// a group's exponents are built from shared even and odd parts, exponentiated
// and folded into the sums at once, so no per-velocity array stays live. The
// FP64 constraint sums use the butterfly of each group (sums and differences
// formed once for all moments).
#pragma once

#include <type_traits>

#include "alb_device.cuh"
#include "exp_table.h"

namespace alb {

// Calls v.rest(s_0), v.pair<a, axis, i+, i->(s_+, s_-) and
// v.quad<a, i++, i-+, i--, i+->(...) with the exponents
// s_i = base + lambda . P(xi_i) of every group (index order of XI_X / XI_Y);
// base is 1 for the exponents of Eq. exponential, 0 for the change of the
// exponents under a step of the multipliers.
template <typename R, typename V>
__device__ __forceinline__ void visit_groups(const R l[NM], V& v, R base = (R)1) {
  const R c = base + l[0];
  v.rest(c);
  {  // axis, |xi| = 1
    const R ex = c + l[3], ox = l[1] + l[6];
    v.template pair<1, 0, 1, 3>(ex + ox, ex - ox);
    const R ey = c + l[5], oy = l[2] + l[7];
    v.template pair<1, 1, 2, 4>(ey + oy, ey - oy);
  }
  {  // axis, |xi| = 2
    const R ex = fma((R)4, l[3], c), ox = fma((R)8, l[6], (R)2 * l[1]);
    v.template pair<2, 0, 9, 11>(ex + ox, ex - ox);
    const R ey = fma((R)4, l[5], c), oy = fma((R)8, l[7], (R)2 * l[2]);
    v.template pair<2, 1, 10, 12>(ey + oy, ey - oy);
  }
  {  // axis, |xi| = 3
    const R ex = fma((R)9, l[3], c), ox = fma((R)27, l[6], (R)3 * l[1]);
    v.template pair<3, 0, 17, 19>(ex + ox, ex - ox);
    const R ey = fma((R)9, l[5], c), oy = fma((R)27, l[7], (R)3 * l[2]);
    v.template pair<3, 1, 18, 20>(ey + oy, ey - oy);
  }
  const R l35 = l[3] + l[5];
  {  // diagonal (+-1, +-1): s = E + sx sy Z + sx X + sy Y
    const R E = c + l35;
    const R X = fma((R)2, l[6], l[1]), Y = fma((R)2, l[7], l[2]);
    const R Ep = E + l[4], Em = E - l[4];
    const R XpY = X + Y, XmY = X - Y;
    v.template quad<1, 5, 6, 7, 8>(Ep + XpY, Em - XmY, Ep - XpY, Em + XmY);
  }
  {  // diagonal (+-2, +-2)
    const R E = fma((R)4, l35, c);
    const R X = fma((R)16, l[6], (R)2 * l[1]), Y = fma((R)16, l[7], (R)2 * l[2]);
    const R Z = (R)4 * l[4];
    const R Ep = E + Z, Em = E - Z;
    const R XpY = X + Y, XmY = X - Y;
    v.template quad<2, 13, 14, 15, 16>(Ep + XpY, Em - XmY, Ep - XpY, Em + XmY);
  }
}

// 2^(j/N), j = 0..N-1 (N = EXPT_N); kernels copy it to shared memory (lanes
// index it freely).
static __constant__ double c_exptab[EXPT_N] = {ALB_EXPT_TABLE_VALUES};

// Copy the table into a block's shared array of EXPT_N doubles (all threads;
// includes a barrier).
__device__ __forceinline__ void load_exptab(double* s_tab) {
  for (int j = threadIdx.x; j < EXPT_N; j += blockDim.x) s_tab[j] = c_exptab[j];
  __syncthreads();
}

// Exponent e = n >> 8 of the scale 2^(n/N) of the table exponentials below.
// t = 1.5 * 2^52 + n holds n exactly while |n| < 2^51, and its low word holds n
// only while |n| < 2^31 (|s| below about 5.8e6); past that the low word wraps,
// so e is saturated from the high word: 0x43380000 for 0 <= n < 2^32,
// 0x4337ffff for -2^32 <= n < 0, larger or smaller beyond (also when the
// rounding trick itself no longer applies). A non-finite t (s NaN or
// infinite) keeps e in range, so that the NaN of the polynomial comes
// through. Integer operations only.
__device__ __forceinline__ int exp_scale_exponent(double t, int n) {
  const int hi = __double2hiint(t);
  const bool finite = (hi & 0x7ff00000) != 0x7ff00000;
  const bool over = hi > 0x43380000 || (hi == 0x43380000 && n < 0);
  const bool under = hi < 0x4337ffff || (hi == 0x4337ffff && n >= 0);
  return !finite ? 0 : (over ? 4096 : (under ? -4096 : (n >> EXPT_BITS)));
}

// Table-driven FP64 exp(-s) (Tang's method with an N = 256 table): n nearest
// to -s N / ln2, r = -s - n ln2/N in two parts (|r| <= ln2/512), exp(r) by its
// degree-4 Taylor polynomial, times 2^(n/N) = 2^(n >> 8) tab[n & 255].
// 9 FP64 operations. Returns 0 below 2^-1022 (no subnormal results) and +inf
// from 2^1024 on, for any finite s.
__device__ __forceinline__ double exp_neg(double s, const double* tab) {
  const double shifter = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer
  const double t = fma(-s, EXPT_INV_L, shifter);
  const int n = (int)(unsigned)__double2loint(t);
  const double nd = t - shifter;
  double r = fma(nd, -EXPT_L_HI, -s);
  r = fma(nd, -EXPT_L_LO, r);
  double q = fma(r, EXPT_C4, EXPT_C3);
  q = fma(q, r, EXPT_C2);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  const int e = exp_scale_exponent(t, n);
  const long long bits =
      __double_as_longlong(tab[n & (EXPT_N - 1)]) + ((long long)e << 52);
  const double v = q * __longlong_as_double(bits);
  // out of range: the limits themselves (q need not be finite there)
  return e < -1022 ? 0.0 : (e > 1023 ? __longlong_as_double(0x7ff0000000000000LL) : v);
}

// exp(-s) for the FP32 form's refinement: the same table, the reduction in
// one step with ln2/N rounded, and the degree-2 Taylor polynomial. Its
// accuracy does not enter the convergence test: each residual is summed
// exactly (in FP64) over the column of values this function fills, so
// max|G|/rho <= 1e-12 holds for the populations returned. It only sets how
// closely those populations follow the exponential family of the returned
// multipliers: to 5e-10 relative here, next to the ~1e-10 the multiplicative
// updates leave, both far below the FP32 storage of the populations.
// The table index n nearest to -s N / ln2 comes from s32, an FP32 value of
// the same exponent: within |s| <= 745 (past which the result is 0 or +inf
// anyway) FP32 holds s to 5e-5, a fiftieth of ln2/N, so n is the nearest
// integer or its neighbour at a tie and |r| stays below 0.52 ln2/N
// (truncation r^3/3! below 4.7e-10). 4 FP64 operations: the reduction, the
// polynomial and the scaling (n reaches FP64 exactly on the integer pipe).
// For |s32 N / ln2| >= 2^31 the float-to-int rounding saturates and e takes
// the limits; a NaN gives n = 0 and passes through the polynomial.
__device__ __forceinline__ double exp_neg_refine(double s, float s32, const double* tab) {
  const int n = __float2int_rn(-s32 * (float)EXPT_INV_L);
  const double r = fma(cvt_f64(n), -EXPT_L, -s);
  double q = fma(r, EXPT_C2, 1.0);
  q = fma(q, r, 1.0);
  const int e = n >> EXPT_BITS;
  const int ec = e < -1100 ? -1100 : (e > 1100 ? 1100 : e);  // keeps the shift defined
  const long long bits = __double_as_longlong(tab[n & (EXPT_N - 1)]) + ((long long)ec << 52);
  const double v = q * __longlong_as_double(bits);
  // out of range: the limits themselves (q need not be finite there)
  return e < -1022 ? 0.0 : (e > 1023 ? __longlong_as_double(0x7ff0000000000000LL) : v);
}

// An exponent held twice: in FP64 and in FP32 (the FP32 copy picks the
// table index of exp_neg_refine). visit_groups runs on it unchanged; its
// operators live in a namespace of their own, found by argument-dependent
// lookup, so that they hide no FP64 fma.
namespace dual {
struct Exp2 {
  double d;
  float f;
  Exp2() = default;
  __device__ __forceinline__ Exp2(double d_, float f_) : d(d_), f(f_) {}
  __device__ __forceinline__ explicit Exp2(double c) : d(c), f((float)c) {}
};
__device__ __forceinline__ Exp2 operator+(Exp2 a, Exp2 b) { return Exp2(a.d + b.d, a.f + b.f); }
__device__ __forceinline__ Exp2 operator-(Exp2 a, Exp2 b) { return Exp2(a.d - b.d, a.f - b.f); }
__device__ __forceinline__ Exp2 operator*(Exp2 a, Exp2 b) { return Exp2(a.d * b.d, a.f * b.f); }
__device__ __forceinline__ Exp2 fma(Exp2 a, Exp2 b, Exp2 c) {
  return Exp2(::fma(a.d, b.d, c.d), fmaf(a.f, b.f, c.f));
}
}  // namespace dual
using dual::Exp2;

// Packed lower triangle of the 8x8 Jacobian: entry (a, b), b <= a.
__host__ __device__ constexpr int tri(int a, int b) { return a * (a + 1) / 2 + b; }

// FP32 pass: F = sum p, G = sum p P and H = sum p P P^T at the visited
// multipliers, accumulated group by group of the velocity set (compile-time
// monomials).
struct PassGH32 {
  float Fs, Gs[NM], Hs[36];
  __device__ __forceinline__ PassGH32() {
    Fs = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) Gs[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 36; ++k) Hs[k] = 0.0f;
  }
  template <int I>
  __device__ __forceinline__ void point(float p) {
    Fs += p;
#pragma unroll
    for (int a = 0; a < NM; ++a) {
      Gs[a] = madd(Gs[a], p, PM(a, I));
#pragma unroll
      for (int b = 0; b <= a; ++b) Hs[tri(a, b)] = madd(Hs[tri(a, b)], p, PM(a, I) * PM(b, I));
    }
  }
  __device__ __forceinline__ void rest(float s) { point<0>(expf(-s)); }
  // A symmetric pair enters through the sum S and difference D of its two
  // points: every sum takes c S or c D, with c the compile-time value of the
  // monomial (product) at the first point and D where the second point flips
  // its sign (the grouping of the FP64 Jacobian, jac_pair).
  template <int A, int AX, int IP, int IM>
  __device__ __forceinline__ void pair(float sp, float sm) {
    const float pp = expf(-sp), pm = expf(-sm);
    const float S = pp + pm, D = pp - pm;
    Fs += S;
#pragma unroll
    for (int a = 0; a < NM; ++a) {
      const int ca = PM(a, IP);
      if (ca != 0) Gs[a] = madd(Gs[a], PM(a, IM) == ca ? S : D, ca);
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        const int c = PM(a, IP) * PM(b, IP);
        if (c != 0) Hs[tri(a, b)] = madd(Hs[tri(a, b)], PM(a, IM) * PM(b, IM) == c ? S : D, c);
      }
    }
  }
  // A diagonal quadruple enters through its four parity combinations (even
  // or odd in x, even or odd in y), as in jac_quad.
  template <int A, int IPP, int IMP, int IMM, int IPM>
  __device__ __forceinline__ void quad(float spp, float smp, float smm, float spm) {
    const float ppp = expf(-spp), pmp = expf(-smp), pmm = expf(-smm), ppm = expf(-spm);
    const float Ap = ppp + ppm, Bm = pmp + pmm, Cp = ppp - ppm, Dm = pmp - pmm;
    const float ee = Ap + Bm, oe = Ap - Bm, eo = Cp + Dm, oo = Cp - Dm;
    Fs += ee;
#pragma unroll
    for (int a = 0; a < NM; ++a) {
      const int ca = PM(a, IPP);
      if (ca != 0) {
        const bool xo = PM(a, IMP) == -ca, yo = PM(a, IPM) == -ca;
        Gs[a] = madd(Gs[a], xo ? (yo ? oo : oe) : (yo ? eo : ee), ca);
      }
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        const int c = PM(a, IPP) * PM(b, IPP);
        if (c == 0) continue;
        const bool xo = PM(a, IMP) * PM(b, IMP) == -c;  // x -> -x flips the sign
        const bool yo = PM(a, IPM) * PM(b, IPM) == -c;  // y -> -y flips the sign
        Hs[tri(a, b)] = madd(Hs[tri(a, b)], xo ? (yo ? oo : oe) : (yo ? eo : ee), c);
      }
    }
  }
  __device__ __forceinline__ float F() const { return Fs; }
  __device__ __forceinline__ void scale(float z) {
    Fs *= z;
#pragma unroll
    for (int k = 0; k < NM; ++k) Gs[k] *= z;
#pragma unroll
    for (int k = 0; k < 36; ++k) Hs[k] *= z;
  }
  __device__ __forceinline__ void assemble(float G[NM], float H[36]) const {
#pragma unroll
    for (int k = 0; k < NM; ++k) G[k] = Gs[k];
#pragma unroll
    for (int k = 0; k < 36; ++k) H[k] = Hs[k];
  }
};

// FP64 constraint sums M = sum p P over the groups of the velocity set, the
// grouping of PassG64: a symmetric pair enters through its sum and
// difference, a diagonal quadruple through its four parity combinations.
struct SumsG64 {
  double M[NM];
  // The sums start at -m (the targets), so that they end as the residual
  // G = sum p P - m without a separate subtraction.
  __device__ __forceinline__ explicit SumsG64(const double m[NM]) {
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] = -m[k];
  }
  __device__ __forceinline__ void add_rest(double p) { M[0] += p; }
  template <int A, int AX>
  __device__ __forceinline__ void add_pair(double pp, double pm) {
    const double S = pp + pm, D = pp - pm;
    M[0] += S;
    if (AX == 0) {
      M[1] = madd(M[1], D, A);
      M[3] = madd(M[3], S, A * A);
      M[6] = madd(M[6], D, A * A * A);
    } else {
      M[2] = madd(M[2], D, A);
      M[5] = madd(M[5], S, A * A);
      M[7] = madd(M[7], D, A * A * A);
    }
  }
  template <int A>
  __device__ __forceinline__ void add_quad(double ppp, double pmp, double pmm, double ppm) {
    const double Ap = ppp + ppm, Bm = pmp + pmm;  // sx = +1, sx = -1
    const double Cp = ppp - ppm, Dm = pmp - pmm;
    const double sum = Ap + Bm, xs = Ap - Bm, ys = Cp + Dm, xys = Cp - Dm;
    M[0] += sum;
    M[1] = madd(M[1], xs, A);
    M[2] = madd(M[2], ys, A);
    M[3] = madd(M[3], sum, A * A);
    M[4] = madd(M[4], xys, A * A);
    M[5] = madd(M[5], sum, A * A);
    M[6] = madd(M[6], xs, 2 * A * A * A);
    M[7] = madd(M[7], ys, 2 * A * A * A);
  }
};

// FP64 pass: the constraint sums M = sum p P with p = exp(-s) in FP64, each p
// also written to the caller's shared column (p_i at col[i * stride]);
// REFINE selects the cheaper exponential of the FP32 form's refinement.
template <bool REFINE>
struct PassG64 {
  double M[NM];
  const double* tab;
  double* col;
  int stride;
  __device__ __forceinline__ PassG64(const double* t, double* c, int s) : tab(t), col(c), stride(s) {
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] = 0.0;
  }
  // sums started at -m: they end as the residual G = sum p P - m
  __device__ __forceinline__ PassG64(const double* t, double* c, int s, const double m[NM])
      : tab(t), col(c), stride(s) {
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] = -m[k];
  }
  // exponents: double, or Exp2 (FP64 with an FP32 copy) in the refinement
  using S = typename std::conditional<REFINE, Exp2, double>::type;
  __device__ __forceinline__ double ex(double s) const { return exp_neg(s, tab); }
  __device__ __forceinline__ double ex(Exp2 s) const { return exp_neg_refine(s.d, s.f, tab); }
  __device__ __forceinline__ void rest(S s) {
    const double p = ex(s);
    col[0] = p;
    M[0] += p;
  }
  template <int A, int AX, int IP, int IM>
  __device__ __forceinline__ void pair(S sp, S sm) {
    const double pp = ex(sp), pm = ex(sm);
    col[IP * stride] = pp;
    col[IM * stride] = pm;
    const double S = pp + pm, D = pp - pm;
    M[0] += S;
    if (AX == 0) {
      M[1] = madd(M[1], D, A);
      M[3] = madd(M[3], S, A * A);
      M[6] = madd(M[6], D, A * A * A);
    } else {
      M[2] = madd(M[2], D, A);
      M[5] = madd(M[5], S, A * A);
      M[7] = madd(M[7], D, A * A * A);
    }
  }
  template <int A, int IPP, int IMP, int IMM, int IPM>
  __device__ __forceinline__ void quad(S spp, S smp, S smm, S spm) {
    const double ppp = ex(spp), pmp = ex(smp);
    const double pmm = ex(smm), ppm = ex(spm);
    col[IPP * stride] = ppp;
    col[IMP * stride] = pmp;
    col[IMM * stride] = pmm;
    col[IPM * stride] = ppm;
    const double Ap = ppp + ppm, Bm = pmp + pmm;  // sx = +1, sx = -1
    const double Cp = ppp - ppm, Dm = pmp - pmm;
    const double sum = Ap + Bm, xs = Ap - Bm, ys = Cp + Dm, xys = Cp - Dm;
    M[0] += sum;
    M[1] = madd(M[1], xs, A);
    M[2] = madd(M[2], ys, A);
    M[3] = madd(M[3], sum, A * A);
    M[4] = madd(M[4], xys, A * A);
    M[5] = madd(M[5], sum, A * A);
    M[6] = madd(M[6], xs, 2 * A * A * A);
    M[7] = madd(M[7], ys, 2 * A * A * A);
  }
};

// Multiplicative pass of the FP32 form's refinement: after a step dl of the
// multipliers, p_i(lambda + dl) = p_i(lambda) exp(-d_i) with d_i = dl . P(xi_i)
// (Eq. exponential), so the populations in the column are updated in place,
// p_i <- p_i + p_i (exp(-d_i) - 1), and the FP64 sums taken again. d_i and
// exp(-d_i) - 1 = -d (1 - d/2 + d^2/6) are formed in FP32 (the step is an FP32
// vector); for |d_i| <= 1e-3 (checked by the caller) the update's factor has
// a relative error of about 1e-10, so the column stays an exponential-family
// member to that level, while the sums that decide convergence are exact FP64
// sums of the column. One FP64 operation per velocity (the factor reaches
// FP64 exactly on the integer pipe) instead of an exponent and an
// exponential.
struct PassMul64 : SumsG64 {
  double* col;
  int stride;
  __device__ __forceinline__ PassMul64(double* c, int s, const double m[NM])
      : SumsG64(m), col(c), stride(s) {}
  __device__ __forceinline__ double upd(int i, float d) const {
    const float e = d * fmaf(d, fmaf(d, -1.0f / 6.0f, 0.5f), -1.0f);
    double* q = col + (size_t)i * stride;
    const double p = fma(*q, cvt_f64(e), *q);
    *q = p;
    return p;
  }
  __device__ __forceinline__ void rest(float d) { add_rest(upd(0, d)); }
  template <int A, int AX, int IP, int IM>
  __device__ __forceinline__ void pair(float dp, float dm) {
    add_pair<A, AX>(upd(IP, dp), upd(IM, dm));
  }
  template <int A, int IPP, int IMP, int IMM, int IPM>
  __device__ __forceinline__ void quad(float dpp, float dmp, float dmm, float dpm) {
    add_quad<A>(upd(IPP, dpp), upd(IMP, dmp), upd(IMM, dmm), upd(IPM, dpm));
  }
};

// Cholesky factor of the Jacobian, FP32: the packed lower triangle L with the
// reciprocals of its diagonal entries in the diagonal slots, so that the
// solves multiply. No diagonal (Jacobi) scaling: the backward error of the
// Cholesky factorisation does not depend on it, and on the 4096^2 layer the
// unscaled factor gave the same iteration counts (and 1 % more MLUPS).
struct Fact32 {
  float L[36];
};

__device__ __forceinline__ bool factor32(const float H[36], Fact32& fc) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    float dj = H[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) dj = fmaf(-fc.L[tri(j, k)], fc.L[tri(j, k)], dj);
    ok = ok && (dj > 0.0f);
    const float il = rsqrtf(fmaxf(dj, 1e-30f));
    fc.L[tri(j, j)] = il;
#pragma unroll
    for (int i = j + 1; i < NM; ++i) {
      float s = H[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s = fmaf(-fc.L[tri(i, k)], fc.L[tri(j, k)], s);
      fc.L[tri(i, j)] = s * il;
    }
  }
  return ok;
}

// delta = H^-1 g with the factor (forward and backward substitution).
__device__ __forceinline__ void solve32(const Fact32& fc, const float g[NM], float dl[NM]) {
  float y[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    float s = g[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = fmaf(-fc.L[tri(i, k)], y[k], s);
    y[i] = s * fc.L[tri(i, i)];
  }
#pragma unroll
  for (int i = NM - 1; i >= 0; --i) {
    float s = y[i];
#pragma unroll
    for (int k = i + 1; k < NM; ++k) s = fmaf(-fc.L[tri(k, i)], y[k], s);
    y[i] = s * fc.L[tri(i, i)];
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) dl[i] = y[i];
}

// Multipliers in the frame of another lattice: lam'.P(u) = lam.P(u - d) for
// every velocity u, where d = U - U' (a velocity xi relative to lattice U is
// xi - d relative to U'). Exact for the exponential; it serves as the starting
// point of the Newton iteration after a change of lattice.
template <typename R>
__device__ __forceinline__ void shift_multipliers(const R l[NM], R dx, R dy, R o[NM]) {
  const R d2 = dx * dx + dy * dy;
  o[0] = l[0] - l[1] * dx - l[2] * dy + l[3] * dx * dx + l[4] * dx * dy + l[5] * dy * dy -
         l[6] * dx * d2 - l[7] * dy * d2;
  o[1] = l[1] - (R)2 * l[3] * dx - l[4] * dy + l[6] * ((R)3 * dx * dx + dy * dy) +
         (R)2 * l[7] * dx * dy;
  o[2] = l[2] - l[4] * dx - (R)2 * l[5] * dy + (R)2 * l[6] * dx * dy +
         l[7] * (dx * dx + (R)3 * dy * dy);
  o[3] = l[3] - (R)3 * l[6] * dx - l[7] * dy;
  o[4] = l[4] - (R)2 * l[6] * dy - (R)2 * l[7] * dx;
  o[5] = l[5] - l[6] * dx - (R)3 * l[7] * dy;
  o[6] = l[6];
  o[7] = l[7];
}

// FP32 phase: damped Newton from lam (warm start) or, if warm is false, from
// the Maxwellian; on success fc holds the factor of the Jacobian at the
// returned multipliers. Returns NEWTON_OK or NEWTON_SINGULAR (non-finite
// values or a non-positive pivot).
//
// Written as one loop with a single evaluation pass and a single
// factorisation, so that the unrolled pass (21 exponentials and the 44 sums)
// exists once in the code: each turn evaluates the point `lc` and then acts
// on it according to why it was evaluated (a start, a line-search trial, the
// full step taken near the root). The points evaluated and the steps
// accepted are those of the plain formulation: start, then per Newton step
// the factor and direction at the accepted point and an Armijo line search.
static __device__ __noinline__ int newton_fp32(float ubx, float uby, float T, int maxit, bool warm,
                                               float lam[NM], Fact32& fc, int* iters) {
  enum { START_WARM, START_MAXWELL, TRIAL, FULL_STEP };
  *iters = 0;
  float m[NM];
  {
    const float u2 = ubx * ubx + uby * uby;
    m[0] = 1.0f; m[1] = ubx; m[2] = uby;
    m[3] = fmaf(ubx, ubx, T); m[4] = ubx * uby; m[5] = fmaf(uby, uby, T);
    m[6] = ubx * fmaf(4.0f, T, u2); m[7] = uby * fmaf(4.0f, T, u2);
  }
  auto dual = [&](const float* l, float F) {
#pragma unroll
    for (int k = 0; k < NM; ++k) F = fmaf(l[k], m[k], F);
    return F;
  };
  // Maxwellian multipliers with lambda_0 = 0 (fixed from the normalisation
  // once evaluated)
  auto maxwell = [&](float* l) {
    const float iT = 1.0f / T;
#pragma unroll
    for (int k = 0; k < NM; ++k) l[k] = 0.0f;
    l[1] = -ubx * iT;
    l[2] = -uby * iT;
    l[3] = 0.5f * iT;
    l[5] = 0.5f * iT;
  };
  float lc[NM], dl[NM];
  int mode = START_WARM;
  if (warm) {
#pragma unroll
    for (int k = 0; k < NM; ++k) lc[k] = lam[k];
  } else {
    maxwell(lc);
    mode = START_MAXWELL;
  }
  float Fd = 0.0f, gd = 0.0f, t = 1.0f;
  int it = 0, ls = 0;
  for (;;) {
    PassGH32 pc;
    visit_groups<float>(lc, pc);
    float F = pc.F();
    if (mode == START_WARM) {
      if (!(isfinite(F) && F > 0.0f)) {
        maxwell(lc);
        mode = START_MAXWELL;
        continue;
      }
    } else if (mode == START_MAXWELL) {
      // the pass at lambda_0 = 0 gives Z = F; all its sums scale by 1/Z
      const float iz = 1.0f / F;
      lc[0] = logf(F);
      pc.scale(iz);
      F = pc.F();
    } else if (mode == TRIAL) {
      const float Fc = dual(lc, F);
      if (!(isfinite(Fc) && Fc <= Fd - 1e-4f * t * gd + 4e-7f * fabsf(Fd))) {
        t *= 0.5f;
        if (++ls >= 12) break;  // no acceptable step: fc is the factor at lam
#pragma unroll
        for (int k = 0; k < NM; ++k) lc[k] = fmaf(t, dl[k], lam[k]);
        continue;
      }
      ++it;
    } else if (!isfinite(F)) {  // FULL_STEP
      return NEWTON_SINGULAR;
    }
    // accepted point: the Newton step there
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = lc[k];
    Fd = dual(lam, F);
    float G[NM], H[36];
    pc.assemble(G, H);
    float gmax = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      G[k] -= m[k];
      gmax = fmaxf(gmax, fabsf(G[k]));
    }
    if (!isfinite(gmax) || !factor32(H, fc)) return NEWTON_SINGULAR;
    // FP32 exit at 1e-6, five times the FP32 residual's own noise (about
    // 2e-7): below that the FP32 steps only chase rounding, and the FP64
    // refinement contracts by about 1e-4 per residual from either level
    if (mode == FULL_STEP || gmax <= 1e-6f || it >= maxit) break;
    solve32(fc, G, dl);
    gd = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) gd = fmaf(G[k], dl[k], gd);
    if (!(gd > 0.0f)) break;
#pragma unroll
    for (int k = 0; k < NM; ++k) lc[k] = lam[k] + dl[k];
    if (gd <= 2e-6f * fmaxf(1.0f, fabsf(Fd))) {
      // The predicted decrease gd/2 of the dual lies below its FP32 resolution:
      // a line search would only compare rounding noise. This close to the root
      // the full Newton step is safe; take it and leave the rest to the FP64
      // refinement. The refinement contracts by about |I - H32^-1 H| per
      // residual, so it gets the factor of the Jacobian at the new multipliers
      // (one more FP32 pass): a factor one step old costs about one more FP64
      // residual per solve.
      mode = FULL_STEP;
      ++it;
    } else {
      mode = TRIAL;
      t = 1.0f;
      ls = 0;
    }
  }
  *iters = it;
  return NEWTON_OK;
}

// max_i |P_k(xi_i)| over the velocity set (compile time).
__host__ __device__ constexpr int pm_max(int k) {
  int m = 0;
  for (int i = 0; i < Q; ++i) m = PM(k, i) > m ? PM(k, i) : (-PM(k, i) > m ? -PM(k, i) : m);
  return m;
}

// Largest |dl . P(xi_i)| over the velocities is at most this bound (FP32);
// the weights are max_i |P_k(xi_i)|, checked at compile time.
static_assert(pm_max(0) == 1 && pm_max(1) == 3 && pm_max(2) == 3 && pm_max(3) == 9 &&
                  pm_max(4) == 4 && pm_max(5) == 9 && pm_max(6) == 27 && pm_max(7) == 27,
              "monomial bounds of the D2Q21 set");
__device__ __forceinline__ float step_exponent_bound(const float dl[NM]) {
  return fabsf(dl[0]) + 3.0f * (fabsf(dl[1]) + fabsf(dl[2])) + 4.0f * fabsf(dl[4]) +
         9.0f * (fabsf(dl[3]) + fabsf(dl[5])) + 27.0f * (fabsf(dl[6]) + fabsf(dl[7]));
}

// FP64 refinement: lambda <- lambda + H32^-1 G64(lambda) until max|G|/rho <= tol.
// The first residual evaluates the 21 exponentials in FP64; after a step whose
// exponent changes are all below 1e-3 in magnitude, the next one updates the
// column multiplicatively instead (PassMul64), else it evaluates them again.
// On NEWTON_OK the FP64 equilibrium per unit density at the returned lambda
// is in col[i * stride] (a shared-memory column of the calling thread).
// The residual is formed in FP64 and its maximum taken on its FP32 copy (the
// one the correction is solved with; FP32 resolves 1e-12 to 6e-8 of itself).
// The corrections are summed in FP32 for lam_out32 (lam32 plus every step:
// the multipliers the warm start stores in FP32) and join the FP64
// multipliers only before a full evaluation and, if lam_out64 is given, at
// the end. *evals counts the full evaluations, *updates the multiplicative
// ones.
static __device__ __noinline__ int refine_fp64(double ubx, double uby, double T, double tol,
                                               int maxr, const float lam32[NM], const Fact32& fc,
                                               const double* tab, double* col, int stride,
                                               float lam_out32[NM], double* lam_out64,
                                               int* evals, int* updates) {
  double m[NM];
  targets(ubx, uby, T, m);
  double lam[NM];  // FP64 multipliers of the last full evaluation
  float acc[NM];   // corrections since then
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    lam[k] = cvt_f64(lam32[k]);
    acc[k] = 0.0f;
    lam_out32[k] = lam32[k];
  }
  const float tolf = (float)tol;
  *evals = 0;
  *updates = 0;
  float dl[NM];
  bool small_step = false;
  for (int r = 0;; ++r) {
    double G[NM];  // residual sum p P - m
    if (small_step) {
      PassMul64 pu(col, stride, m);
      visit_groups<float>(dl, pu, 0.0f);
      ++*updates;
#pragma unroll
      for (int k = 0; k < NM; ++k) G[k] = pu.M[k];
    } else {
      if (r > 0) {
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          lam[k] += cvt_f64(acc[k]);
          acc[k] = 0.0f;
        }
      }
      PassG64<true> ps(tab, col, stride, m);
      Exp2 l2[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) l2[k] = Exp2(lam[k], lam_out32[k]);
      visit_groups<Exp2>(l2, ps, Exp2(1.0));
      ++*evals;
#pragma unroll
      for (int k = 0; k < NM; ++k) G[k] = ps.M[k];
    }
    float gmax = 0.0f;
    bool finite = true;
    float g32[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      g32[k] = cvt_f32_rn(G[k]);
      finite = finite && isfinite(g32[k]);
      gmax = fmaxf(gmax, fabsf(g32[k]));
    }
    if (!finite) return NEWTON_SINGULAR;
    if (gmax <= tolf) {
      if (lam_out64)
#pragma unroll
        for (int k = 0; k < NM; ++k) lam_out64[k] = lam[k] + (double)acc[k];
      return NEWTON_OK;
    }
    if (r >= maxr) return NEWTON_MAXIT;
    solve32(fc, g32, dl);
    small_step = step_exponent_bound(dl) <= 1e-3f;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      acc[k] += dl[k];
      lam_out32[k] += dl[k];
    }
  }
}

// Work counts of one equilibrium solve.
struct SolveCount {
  unsigned fp32_iters = 0, fp64_evals = 0, fp64_iters = 0, fp64_updates = 0;
};

// Jacobian H = sum_i p_i P(xi_i) P(xi_i)^T (packed lower triangle) from the
// populations per unit density in col[i * stride], group by group: a
// symmetric pair contributes its sum or difference, a diagonal quadruple one
// of its four parity combinations, with the compile-time value of P_a P_b at
// the group's first point as coefficient.
template <int IP, int IM>
__device__ __forceinline__ void jac_pair(const double* col, int stride, double H[36]) {
  const double pp = col[IP * stride], pm = col[IM * stride];
  const double S = pp + pm, D = pp - pm;
#pragma unroll
  for (int a = 0; a < NM; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int c = PM(a, IP) * PM(b, IP);
      if (c != 0) H[tri(a, b)] = madd(H[tri(a, b)], PM(a, IM) * PM(b, IM) == c ? S : D, c);
    }
}

template <int IPP, int IMP, int IMM, int IPM>
__device__ __forceinline__ void jac_quad(const double* col, int stride, double H[36]) {
  const double ppp = col[IPP * stride], pmp = col[IMP * stride];
  const double pmm = col[IMM * stride], ppm = col[IPM * stride];
  const double Ap = ppp + ppm, Bm = pmp + pmm, Cp = ppp - ppm, Dm = pmp - pmm;
  const double ee = Ap + Bm, oe = Ap - Bm, eo = Cp + Dm, oo = Cp - Dm;
#pragma unroll
  for (int a = 0; a < NM; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int c = PM(a, IPP) * PM(b, IPP);
      const bool xodd = PM(a, IMP) * PM(b, IMP) == -c;  // x -> -x flips the sign
      const bool yodd = PM(a, IPM) * PM(b, IPM) == -c;  // y -> -y flips the sign
      if (c != 0)
        H[tri(a, b)] = madd(H[tri(a, b)], xodd ? (yodd ? oo : oe) : (yodd ? eo : ee), c);
    }
}

__device__ __forceinline__ void jacobian_grouped(const double* col, int stride, double H[36]) {
#pragma unroll
  for (int k = 0; k < 36; ++k) H[k] = 0.0;
  H[0] = col[0];  // rest velocity: only P_0 = 1 is non-zero
  jac_pair<1, 3>(col, stride, H);
  jac_pair<2, 4>(col, stride, H);
  jac_pair<9, 11>(col, stride, H);
  jac_pair<10, 12>(col, stride, H);
  jac_pair<17, 19>(col, stride, H);
  jac_pair<18, 20>(col, stride, H);
  jac_quad<5, 6, 7, 8>(col, stride, H);
  jac_quad<13, 14, 15, 16>(col, stride, H);
}

// Evaluation of the exponential family at l: p_i = exp(-(1 + l . P(xi_i)))
// into col, and the moments M_k = sum_i p_i P_k(xi_i) (table-driven FP64
// exponential, grouped exponents and sums).
__device__ __forceinline__ void eval_fp64(const double l[NM], const double* tab, double* col,
                                          int stride, double M[NM]) {
  PassG64<false> pg(tab, col, stride);
  visit_groups<double>(l, pg);
#pragma unroll
  for (int k = 0; k < NM; ++k) M[k] = pg.M[k];
}

// FP64 Newton on the multipliers of the 8-moment equilibrium (Sec. II.C.2,
// App. C): damped by backtracking (Armijo) on the strictly convex dual
// F(lambda) = sum_i p_i + lambda . m, whose gradient is -G/rho and Hessian the
// exact Jacobian sum_i p_i P P^T; stops at max_k |G_k|/rho <= tol. Starts from
// `warm` if given, else (or if warm gives a non-finite dual) from the
// Maxwellian with lambda_0 from the normalisation. The iteration is the
// oracle's; its arithmetic is grouped by the symmetry of the velocity set and
// uses the table-driven exponential. On return col[i * stride] holds the
// equilibrium per unit density at lam; *iters counts Newton steps, *evals
// evaluations of the 21 exponentials.
static __device__ __noinline__ int newton_fp64g(double ubx, double uby, double T, double tol,
                                                int maxit, const double* tab, double* col,
                                                int stride, double lam[NM], int* iters,
                                                int* evals, const double* warm) {
  *iters = 0;
  *evals = 0;
  if (!(T > 0.0) || !isfinite(T) || !isfinite(ubx) || !isfinite(uby)) return NEWTON_UNREALIZABLE;
  double m[NM];
  targets(ubx, uby, T, m);
  double M[NM];
  int ev = 0;
  double F = 0.0;
  if (warm) {
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = warm[k];
    eval_fp64(lam, tab, col, stride, M);
    ev = 1;
    F = M[0];
#pragma unroll
    for (int k = 0; k < NM; ++k) F = fma(lam[k], m[k], F);
  }
  if (!warm || !isfinite(F)) {
    // Maxwellian: lambda_1 = -u/T, lambda_xx = lambda_yy = 1/(2T), lambda_0
    // from sum p = 1 (the exponentials at lambda_0 = 0 divided by their sum)
    const double iT = 1.0 / T;
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = 0.0;
    lam[1] = -ubx * iT;
    lam[2] = -uby * iT;
    lam[3] = 0.5 * iT;
    lam[5] = 0.5 * iT;
    eval_fp64(lam, tab, col, stride, M);
    ev += 1;
    const double Z = M[0];
    lam[0] = log(Z);
    const double iZ = 1.0 / Z;
#pragma unroll
    for (int i = 0; i < Q; ++i) col[i * stride] *= iZ;
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] *= iZ;
    F = M[0];
#pragma unroll
    for (int k = 0; k < NM; ++k) F = fma(lam[k], m[k], F);
  }
  int it = 0;
  for (;;) {
    double G[NM];
    double gmax = 0.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      G[k] = M[k] - m[k];
      gmax = fmax(gmax, fabs(G[k]));
    }
    if (!isfinite(gmax)) { *iters = it; *evals = ev; return NEWTON_SINGULAR; }
    if (gmax <= tol) { *iters = it; *evals = ev; return NEWTON_OK; }
    if (it >= maxit) { *iters = it; *evals = ev; return NEWTON_MAXIT; }
    // Jacobian, then its Cholesky factor in place (reciprocal pivots kept)
    double H[36], il[NM];
    jacobian_grouped(col, stride, H);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < NM; ++j) {
      double d = H[tri(j, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) d = fma(-H[tri(j, k)], H[tri(j, k)], d);
      ok = ok && (d > 0.0);
      const double l = sqrt(fmax(d, 1e-300));
      il[j] = 1.0 / l;
      H[tri(j, j)] = l;
#pragma unroll
      for (int i = j + 1; i < NM; ++i) {
        double s = H[tri(i, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fma(-H[tri(i, k)], H[tri(j, k)], s);
        H[tri(i, j)] = s * il[j];
      }
    }
    if (!ok) { *iters = it; *evals = ev; return NEWTON_SINGULAR; }
    double d[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      double s = G[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s = fma(-H[tri(i, k)], d[k], s);
      d[i] = s * il[i];
    }
#pragma unroll
    for (int i = NM - 1; i >= 0; --i) {
      double s = d[i];
#pragma unroll
      for (int k = i + 1; k < NM; ++k) s = fma(-H[tri(k, i)], d[k], s);
      d[i] = s * il[i];
    }
    double gd = 0.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) gd = fma(G[k], d[k], gd);
    // backtracking (Armijo) along lam + t d
    double t = 1.0, Fc = 0.0;
    bool accepted = false;
    double lc[NM];
    for (int ls = 0; ls < 40; ++ls) {
#pragma unroll
      for (int k = 0; k < NM; ++k) lc[k] = fma(t, d[k], lam[k]);
      eval_fp64(lc, tab, col, stride, M);
      ++ev;
      Fc = M[0];
#pragma unroll
      for (int k = 0; k < NM; ++k) Fc = fma(lc[k], m[k], Fc);
      if (isfinite(Fc) && Fc <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) { accepted = true; break; }
      t *= 0.5;
    }
    ++it;
    if (!accepted) {
      eval_fp64(lam, tab, col, stride, M);
      *iters = it;
      *evals = ev + 1;
      return NEWTON_MAXIT;
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = lc[k];
    F = Fc;
  }
}

// Reduced model (App. C.2, Eq. feqNum_4Mom): four constraints - mass,
// momentum and the energy trace sum f xi_a xi_a = rho (|ubar|^2 + D T) - and
// the exponential family in (1, xi_x, xi_y, |xi|^2). The multipliers are kept
// in the 8-slot layout of the full set (lambda_xx = lambda_yy = l2, the rest
// 0), so the grouped evaluation, the warm-start planes and the lattice shift
// of the multipliers are shared. The iteration is the oracle's: Maxwellian
// start with lambda_0 from the normalisation (or the warm multipliers),
// Newton on the dual with Armijo backtracking, stop at max|G|/rho <= tol; the
// 4x4 Jacobian takes its entries from the constraint sums of the evaluation
// plus sum p |xi|^4.
__device__ __forceinline__ void expand4(const double l4[4], double l8[NM]) {
  l8[0] = l4[0]; l8[1] = l4[1]; l8[2] = l4[2];
  l8[3] = l4[3]; l8[4] = 0.0; l8[5] = l4[3]; l8[6] = 0.0; l8[7] = 0.0;
}

static __device__ __noinline__ int newton4_fp64g(double ubx, double uby, double T, double tol,
                                                 int maxit, const double* tab, double* col,
                                                 int stride, double lam[NM], int* iters,
                                                 int* evals, const double* warm) {
  *iters = 0;
  *evals = 0;
  if (!(T > 0.0) || !isfinite(T) || !isfinite(ubx) || !isfinite(uby)) return NEWTON_UNREALIZABLE;
  const double m[4] = {1.0, ubx, uby, ubx * ubx + uby * uby + 2.0 * T};
  double l4[4], M[NM];
  int ev = 0;
  double F = 0.0;
  if (warm) {
    l4[0] = warm[0]; l4[1] = warm[1]; l4[2] = warm[2]; l4[3] = warm[3];
    expand4(l4, lam);
    eval_fp64(lam, tab, col, stride, M);
    ev = 1;
    F = M[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) F = fma(l4[k], m[k], F);
  }
  if (!warm || !isfinite(F)) {
    const double iT = 1.0 / T;
    l4[0] = 0.0; l4[1] = -ubx * iT; l4[2] = -uby * iT; l4[3] = 0.5 * iT;
    expand4(l4, lam);
    eval_fp64(lam, tab, col, stride, M);
    ev += 1;
    const double Z = M[0];
    l4[0] = log(Z);
    const double iZ = 1.0 / Z;
#pragma unroll
    for (int i = 0; i < Q; ++i) col[i * stride] *= iZ;
#pragma unroll
    for (int k = 0; k < NM; ++k) M[k] *= iZ;
    F = M[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) F = fma(l4[k], m[k], F);
  }
  int it = 0;
  for (;;) {
    const double G[4] = {M[0] - m[0], M[1] - m[1], M[2] - m[2], (M[3] + M[5]) - m[3]};
    double gmax = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) gmax = fmax(gmax, fabs(G[k]));
    if (!isfinite(gmax)) { expand4(l4, lam); *iters = it; *evals = ev; return NEWTON_SINGULAR; }
    if (gmax <= tol) { expand4(l4, lam); *iters = it; *evals = ev; return NEWTON_OK; }
    if (it >= maxit) { expand4(l4, lam); *iters = it; *evals = ev; return NEWTON_MAXIT; }
    // Jacobian sum p P4 P4^T: all but sum p |xi|^4 are the sums of the last
    // evaluation (P4 = (1, x, y, x^2 + y^2)); |xi|^4 is a^4 on an axis pair and
    // 4 a^4 on a diagonal quadruple of the velocity set
    const double sr4 =
        (col[1 * stride] + col[3 * stride]) + (col[2 * stride] + col[4 * stride]) +
        16.0 * ((col[9 * stride] + col[11 * stride]) + (col[10 * stride] + col[12 * stride])) +
        81.0 * ((col[17 * stride] + col[19 * stride]) + (col[18 * stride] + col[20 * stride])) +
        4.0 * ((col[5 * stride] + col[6 * stride]) + (col[7 * stride] + col[8 * stride])) +
        64.0 * ((col[13 * stride] + col[14 * stride]) + (col[15 * stride] + col[16 * stride]));
    double H[10];
    H[tri(0, 0)] = M[0];
    H[tri(1, 0)] = M[1];
    H[tri(1, 1)] = M[3];
    H[tri(2, 0)] = M[2];
    H[tri(2, 1)] = M[4];
    H[tri(2, 2)] = M[5];
    H[tri(3, 0)] = M[3] + M[5];
    H[tri(3, 1)] = M[6];
    H[tri(3, 2)] = M[7];
    H[tri(3, 3)] = sr4;
    bool ok = true;
    double il[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double d = H[tri(j, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) d = fma(-H[tri(j, k)], H[tri(j, k)], d);
      ok = ok && (d > 0.0);
      const double l = sqrt(fmax(d, 1e-300));
      il[j] = 1.0 / l;
      H[tri(j, j)] = l;
#pragma unroll
      for (int i = j + 1; i < 4; ++i) {
        double s = H[tri(i, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fma(-H[tri(i, k)], H[tri(j, k)], s);
        H[tri(i, j)] = s * il[j];
      }
    }
    if (!ok) { expand4(l4, lam); *iters = it; *evals = ev; return NEWTON_SINGULAR; }
    double d[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double s = G[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s = fma(-H[tri(i, k)], d[k], s);
      d[i] = s * il[i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
      double s = d[i];
#pragma unroll
      for (int k = i + 1; k < 4; ++k) s = fma(-H[tri(k, i)], d[k], s);
      d[i] = s * il[i];
    }
    double gd = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) gd = fma(G[k], d[k], gd);
    double t = 1.0, Fc = 0.0, lc[4];
    bool accepted = false;
    for (int ls = 0; ls < 40; ++ls) {
#pragma unroll
      for (int k = 0; k < 4; ++k) lc[k] = fma(t, d[k], l4[k]);
      expand4(lc, lam);
      eval_fp64(lam, tab, col, stride, M);
      ++ev;
      Fc = M[0];
#pragma unroll
      for (int k = 0; k < 4; ++k) Fc = fma(lc[k], m[k], Fc);
      if (isfinite(Fc) && Fc <= F - 1e-4 * t * gd + 1e-15 * fabs(F)) { accepted = true; break; }
      t *= 0.5;
    }
    ++it;
    if (!accepted) {
      expand4(l4, lam);
      eval_fp64(lam, tab, col, stride, M);
      *iters = it;
      *evals = ev + 1;
      return NEWTON_MAXIT;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) l4[k] = lc[k];
    F = Fc;
  }
}

// Equilibrium of the FP32 form: FP32 Newton (from the warm start if given,
// else from the Maxwellian; again from the Maxwellian if the warm start
// fails), FP64 refinement, full FP64 Newton as the last fallback. The FP64
// equilibrium per unit density lands in col[i * stride]; the multipliers in
// lam32 (FP32, as the warm start keeps them) and, if lam64 is given, in FP64.
__device__ __forceinline__ int equilibrium_mixed(double ubx, double uby, double T, double tol,
                                                 int maxit, const double* tab, const float* warm,
                                                 double* col, int stride, float lam32[NM],
                                                 double* lam64, SolveCount* cnt) {
  if (!(T > 0.0) || !isfinite(T) || !isfinite(ubx) || !isfinite(uby)) return NEWTON_UNREALIZABLE;
  float l32[NM];
  Fact32 fc;
  int it32 = 0, ev = 0;
  int st = NEWTON_SINGULAR;
  const float ubx32 = cvt_f32_rn(ubx), uby32 = cvt_f32_rn(uby), T32 = cvt_f32_rn(T);
  if (warm) {
#pragma unroll
    for (int k = 0; k < NM; ++k) l32[k] = warm[k];
    st = newton_fp32(ubx32, uby32, T32, 30, true, l32, fc, &it32);
    cnt->fp32_iters += it32;
  }
  if (st != NEWTON_OK) {
    st = newton_fp32(ubx32, uby32, T32, 30, false, l32, fc, &it32);
    cnt->fp32_iters += it32;
  }
  if (st == NEWTON_OK) {
    int up = 0;
    st = refine_fp64(ubx, uby, T, tol, 6, l32, fc, tab, col, stride, lam32, lam64, &ev, &up);
    cnt->fp64_evals += ev;
    cnt->fp64_updates += up;
  }
  if (st != NEWTON_OK) {
    int it = 0;
    double ld[NM];
    st = newton_fp64g(ubx, uby, T, tol, maxit, tab, col, stride, ld, &it, &ev, nullptr);
    cnt->fp64_iters += it;
    cnt->fp64_evals += ev;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      lam32[k] = (float)ld[k];
      if (lam64) lam64[k] = ld[k];
    }
  }
  return st;
}

}  // namespace alb
