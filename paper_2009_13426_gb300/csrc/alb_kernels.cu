// Kernels of the adaptive D2Q21 LBM step (one node per thread).
//
//  step_kernel   pull (Eq. stream) in the receiver's lattice with Grad rebuild
//                of missing pulls (Eqs. GradGeneral*), moments (Eq. polyTemp),
//                shift for the next pull (Eq. criterion), FP64 Newton for the
//                numerical equilibrium (Eq. feqNum_8Mom), g^eq (Eq. gEq),
//                optional sensor (Eq. DeltaAvg), BGK (Eq. coll), store.
//  init_kernel   Grad-regularised initial populations, then the same collision.
//  export / equilibrium / select kernels for the C ABI.
//
// Layout: structure of arrays. Plane p (f_0..f_20, g_0..g_20) of a buffer is
// a contiguous nx*ny array, x fastest; lattice codes and moments likewise.
#include <type_traits>

#include "alb_internal.h"
#include "alb_mixed.cuh"

namespace alb {

constexpr int BLOCK = 128;

// Equilibrium of one node in the storage precision P: the full FP64 Newton for
// the FP64 plain path, the mixed FP32/FP64 solver for the FP32 form.
template <typename P>
__device__ __forceinline__ int node_equilibrium(const Params& pr, double ubx, double uby,
                                                double T, const double* tab, const float* warm,
                                                double lam[NM], double p[Q], SolveCount* cnt) {
  if constexpr (std::is_same<P, float>::value) {
    return equilibrium_mixed(ubx, uby, T, pr.tol, pr.maxit, tab, warm, lam, p, cnt);
  } else {
    int it = 0, ev = 0;
    const int st = newton_fp64(ubx, uby, T, pr.tol, pr.maxit, lam, p, &it, &ev);
    cnt->fp64_iters += it;
    cnt->fp64_evals += ev;
    return st;
  }
}

// exp(-(1 + lambda . P(xi))) for one velocity (cx, cy) given at run time.
template <typename P>
__device__ __forceinline__ double p_one(const double lam[NM], int cx, int cy, const double* tab) {
  if constexpr (std::is_same<P, float>::value) {
    const double x = cx, y = cy, r2 = x * x + y * y;
    double s = 1.0 + lam[0];
    s = fma(lam[1], x, s);
    s = fma(lam[2], y, s);
    s = fma(lam[3], x * x, s);
    s = fma(lam[4], x * y, s);
    s = fma(lam[5], y * y, s);
    s = fma(lam[6], x * r2, s);
    s = fma(lam[7], y * r2, s);
    return exp_neg(s, tab);
  } else {
    return exp_family_one(lam, cx, cy);
  }
}

// Moment accumulation: plain in FP64; Neumaier-compensated in FP32.
template <typename P>
struct Acc {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double val() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    if (fabsf(s) >= fabsf(v))
      c += (s - t) + v;
    else
      c += (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double val() const { return (double)(s + c); }
};

template <typename P>
struct StepArgs {
  const P* pop_in;
  P* pop_out;
  const P* mom_in;
  P* mom_out;
  const uint8_t* lat_in;
  const uint8_t* nxt_in;
  uint8_t* lat_out;
  uint8_t* nxt_out;
  const float* lam_in;  // FP32 form: multipliers of the previous step (8 planes)
  float* lam_out;
  size_t ps;
  Params prm;
  unsigned long long* ctr;
};

// Multipliers stored for node k (8 planes), moved into the frame of lattice
// (Ux, Uy) from the lattice code they were computed in.
__device__ __forceinline__ void load_warm(const float* lam, size_t ps, size_t k, int code_from,
                                          int Ux, int Uy, float w[NM]) {
  float l[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) l[j] = lam[j * ps + k];
  const int dx = lat_ux(code_from) - Ux, dy = lat_uy(code_from) - Uy;
  if (dx == 0 && dy == 0) {
#pragma unroll
    for (int j = 0; j < NM; ++j) w[j] = l[j];
  } else {
    shift_multipliers(l, (float)dx, (float)dy, w);
  }
}

// Grad rebuild of a missing pull (Sec. III.B.2, IV.A.3): the post-collision
// population of velocity (cx, cy) in the receiver's lattice (Upx, Upy), built
// from the sender's moments at (sx, sy) (possibly a ghost), their central
// differences and the sender's relaxation time: h* = h^eq (1 + (1 - 1/tau) phi_h).
// Returns 1 if the root finder failed and the Maxwellian-guess fallback was used.
template <typename P>
__device__ __noinline__ int rebuild_pull(const Params pr, const P* __restrict__ mom, size_t ps,
                                         int cx, int cy, int Upx, int Upy, int sx, int sy,
                                         double* fi, double* gi, const double* tab,
                                         const float* lam_in, const uint8_t* lat_in,
                                         SolveCount* cnt) {
  bool gh = false;
  const int rx = resolve(sx, pr.nx, pr.bcx, &gh);
  const int ry = resolve(sy, pr.ny, pr.bcy, &gh);
  const int xp = resolve(sx + 1, pr.nx, pr.bcx, &gh);
  const int xm = resolve(sx - 1, pr.nx, pr.bcx, &gh);
  const int yp = resolve(sy + 1, pr.ny, pr.bcy, &gh);
  const int ym = resolve(sy - 1, pr.ny, pr.bcy, &gh);
  const size_t nx = (size_t)pr.nx;
  const size_t ks = ry * nx + rx;
  const size_t kxp = ry * nx + xp, kxm = ry * nx + xm, kyp = yp * nx + rx, kym = ym * nx + rx;
  const P* mr = mom;
  const P* mux = mom + ps;
  const P* muy = mom + 2 * ps;
  const P* mT = mom + 3 * ps;
  const double rho = (double)mr[ks], ux = (double)mux[ks], uy = (double)muy[ks],
               T = (double)mT[ks];
  double du[2][2], dT[2];
  du[0][0] = 0.5 * ((double)mux[kxp] - (double)mux[kxm]);
  du[1][0] = 0.5 * ((double)mux[kyp] - (double)mux[kym]);
  du[0][1] = 0.5 * ((double)muy[kxp] - (double)muy[kxm]);
  du[1][1] = 0.5 * ((double)muy[kyp] - (double)muy[kym]);
  dT[0] = 0.5 * ((double)mT[kxp] - (double)mT[kxm]);
  dT[1] = 0.5 * ((double)mT[kyp] - (double)mT[kym]);
  const double ubx = ux - Upx, uby = uy - Upy;
  double lam[NM], p[Q];
  float wbuf[NM];
  const float* warm = nullptr;
  if constexpr (std::is_same<P, float>::value) {
    load_warm(lam_in, ps, ks, lat_in[ks], Upx, Upy, wbuf);
    warm = wbuf;
  }
  const int st = (rho > 0.0) ? node_equilibrium<P>(pr, ubx, uby, T, tab, warm, lam, p, cnt)
                             : NEWTON_UNREALIZABLE;
  const double gfac = (2.0 * pr.cv - 2.0) * T;
  if (st != NEWTON_OK) {
    if (T > 0.0) {
      maxwellian_guess(ubx, uby, T, lam);
      *fi = rho * exp_family_one(lam, cx, cy);
    } else {
      *fi = 0.0;
    }
    *gi = gfac * (*fi);
    return 1;
  }
  const double tau = 0.5 + pr.nu / T;
  const double omega = 1.0 - 1.0 / tau;
  const double feq = rho * p_one<P>(lam, cx, cy, tab);
  const double cbx = (double)(cx + Upx) - ux;
  const double cby = (double)(cy + Upy) - uy;
  double phf, phg;
  grad_phi(pr, rho, T, cbx, cby, du, dT, &phf, &phg);
  *fi = feq * (1.0 + omega * phf);
  *gi = gfac * feq * (1.0 + omega * phg);
  return 0;
}

// Moments, next shift, equilibrium and BGK of one node whose 42 pre-collision
// populations sit in the shared stash (column of this thread), then store.
template <typename P>
__device__ __forceinline__ void collide_store(const Params& pr, const P* st, int code, size_t k,
                                              size_t ps, P* __restrict__ pop_out,
                                              P* __restrict__ mom_out, uint8_t* lat_out,
                                              uint8_t* nxt_out, const double* tab,
                                              const float* warm, float* lam_out,
                                              SolveCount* cnt, unsigned* n_fail) {
  const int Ux = lat_ux(code), Uy = lat_uy(code);
  Acc<P> ar, ajx, ajy, ae;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const P f = st[i * BLOCK];
    const P g = st[(Q + i) * BLOCK];
    constexpr int dummy = 0;
    (void)dummy;
    ar.add(f);
    if (XI_X(i) != 0) ajx.add(XI_X(i) == 1 ? f : XI_X(i) == -1 ? -f : (P)XI_X(i) * f);
    if (XI_Y(i) != 0) ajy.add(XI_Y(i) == 1 ? f : XI_Y(i) == -1 ? -f : (P)XI_Y(i) * f);
    const int c2 = XI_X(i) * XI_X(i) + XI_Y(i) * XI_Y(i);
    if (c2 != 0) ae.add(c2 == 1 ? f : (P)c2 * f);
    ae.add(g);
  }
  const double rho = ar.val();
  const double ubx = ajx.val() / rho, uby = ajy.val() / rho;
  const double T = (ae.val() - rho * (ubx * ubx + uby * uby)) / (2.0 * rho * pr.cv);
  const double ux = ubx + (double)Ux, uy = uby + (double)Uy;
  const int code2 = lat_code(select_shift(ux, pr.n0, pr.umax), select_shift(uy, pr.n0, pr.umax));

  double lam[NM], p[Q];
  const int ns = (rho > 0.0) ? node_equilibrium<P>(pr, ubx, uby, T, tab, warm, lam, p, cnt)
                             : NEWTON_UNREALIZABLE;
  if constexpr (std::is_same<P, float>::value) {
    // multipliers for the next step's warm start (lattice `code`)
    if (ns == NEWTON_OK) {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = (float)lam[j];
    } else if (warm) {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = warm[j];
    } else {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = j == 3 || j == 5 ? 0.5f : 0.0f;
    }
  }
  if (ns == NEWTON_OK) {
    const double gfac = (2.0 * pr.cv - 2.0) * T;
    double tau = 0.5 + pr.nu / T;
    if (pr.sensor) {
      P eps = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const P fe = (P)(rho * p[i]);
        eps += fabs(st[i * BLOCK] - fe) / fe;
      }
      eps /= (P)Q;
      tau *= (double)sensor_alpha<P>(pr, eps);
    }
    const P om = (P)(1.0 / tau);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const P fe = (P)(rho * p[i]);
      const P ge = (P)(gfac * rho * p[i]);
      const P f = st[i * BLOCK];
      const P g = st[(Q + i) * BLOCK];
      pop_out[i * ps + k] = fma(om, fe - f, f);
      pop_out[(Q + i) * ps + k] = fma(om, ge - g, g);
    }
  } else {
    *n_fail += 1;
#pragma unroll
    for (int i = 0; i < NPLANES; ++i) pop_out[i * ps + k] = st[i * BLOCK];
  }
  mom_out[k] = (P)rho;
  mom_out[ps + k] = (P)ux;
  mom_out[2 * ps + k] = (P)uy;
  mom_out[3 * ps + k] = (P)T;
  lat_out[k] = (uint8_t)code;
  nxt_out[k] = (uint8_t)code2;
}

template <typename P>
__global__ void __launch_bounds__(BLOCK, (std::is_same<P, float>::value ? 4 : 1))
    step_kernel(StepArgs<P> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_tab[32];
  load_exptab(s_tab);
  P* st = reinterpret_cast<P*>(smem_raw) + threadIdx.x;
  const Params& pr = a.prm;
  const int x = blockIdx.x * BLOCK + threadIdx.x;
  const int y = blockIdx.y;
  unsigned n_rec = 0, n_rec_fail = 0, n_fail = 0, n_calls = 0;
  SolveCount cnt;
  if (x < pr.nx) {
    const size_t k = (size_t)y * pr.nx + x;
    const size_t ps = a.ps;
    const int code = a.nxt_in[k];
    const int Upx = lat_ux(code), Upy = lat_uy(code);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int sx = x - XI_X(i) - Upx;
      const int sy = y - XI_Y(i) - Upy;
      bool gh = false;
      const int rx = resolve(sx, pr.nx, pr.bcx, &gh);
      const int ry = resolve(sy, pr.ny, pr.bcy, &gh);
      const size_t ks = (size_t)ry * pr.nx + rx;
      P fi, gi;
      if (!gh && a.lat_in[ks] == code) {
        fi = a.pop_in[i * ps + ks];
        gi = a.pop_in[(Q + i) * ps + ks];
      } else {
        double fd, gd;
        n_rec += 1;
        n_rec_fail += rebuild_pull<P>(pr, a.mom_in, ps, XI_X(i), XI_Y(i), Upx, Upy, sx, sy, &fd,
                                      &gd, s_tab, a.lam_in, a.lat_in, &cnt);
        fi = (P)fd;
        gi = (P)gd;
      }
      st[i * BLOCK] = fi;
      st[(Q + i) * BLOCK] = gi;
    }
    float wbuf[NM];
    const float* warm = nullptr;
    if constexpr (std::is_same<P, float>::value) {
      load_warm(a.lam_in, ps, k, a.lat_in[k], Upx, Upy, wbuf);
      warm = wbuf;
    }
    collide_store<P>(pr, st, code, k, ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out, s_tab,
                     warm, a.lam_out, &cnt, &n_fail);
    n_calls = 1 + n_rec;
  }
  warp_count(a.ctr + CTR_NEWTON_ITERS, cnt.fp64_iters);
  warp_count(a.ctr + CTR_FP64_EVALS, cnt.fp64_evals);
  warp_count(a.ctr + CTR_FP32_ITERS, cnt.fp32_iters);
  warp_count(a.ctr + CTR_NEWTON_CALLS, n_calls);
  warp_count(a.ctr + CTR_NEWTON_FAIL, n_fail);
  warp_count(a.ctr + CTR_REC, n_rec);
  warp_count(a.ctr + CTR_REC_FAIL, n_rec_fail);
}

template <typename P>
struct InitArgs {
  const double *rho, *rhoux, *rhouy, *rhoE;
  P* pop_out;
  P* mom_out;
  uint8_t* lat_out;
  uint8_t* nxt_out;
  float* lam_out;
  size_t ps;
  Params prm;
  unsigned long long* ctr;
};

__device__ __forceinline__ void init_prim(const double* rho, const double* rhoux,
                                          const double* rhouy, const double* rhoE, double cv,
                                          size_t k, double* r, double* ux, double* uy,
                                          double* T) {
  *r = rho[k];
  *ux = rhoux[k] / *r;
  *uy = rhouy[k] / *r;
  *T = (rhoE[k] - 0.5 * (*r) * ((*ux) * (*ux) + (*uy) * (*uy))) / ((*r) * cv);
}

// Grad-regularised initial condition (Sec. IV.A.1): h = h^eq (1 + phi_h) in the
// lattice chosen from the initial velocity, then the first collision.
template <typename P>
__global__ void __launch_bounds__(BLOCK) init_kernel(InitArgs<P> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_tab[32];
  load_exptab(s_tab);
  P* st = reinterpret_cast<P*>(smem_raw) + threadIdx.x;
  const Params& pr = a.prm;
  const int x = blockIdx.x * BLOCK + threadIdx.x;
  const int y = blockIdx.y;
  unsigned n_bad = 0, n_fail = 0;
  SolveCount cnt;
  if (x < pr.nx) {
    const size_t nx = (size_t)pr.nx;
    const size_t k = (size_t)y * nx + x;
    bool gh = false;
    const int xp = resolve(x + 1, pr.nx, pr.bcx, &gh), xm = resolve(x - 1, pr.nx, pr.bcx, &gh);
    const int yp = resolve(y + 1, pr.ny, pr.bcy, &gh), ym = resolve(y - 1, pr.ny, pr.bcy, &gh);
    double r, ux, uy, T, r1, ux1, uy1, T1, r2, ux2, uy2, T2;
    init_prim(a.rho, a.rhoux, a.rhouy, a.rhoE, pr.cv, k, &r, &ux, &uy, &T);
    double du[2][2], dT[2];
    init_prim(a.rho, a.rhoux, a.rhouy, a.rhoE, pr.cv, y * nx + xp, &r1, &ux1, &uy1, &T1);
    init_prim(a.rho, a.rhoux, a.rhouy, a.rhoE, pr.cv, y * nx + xm, &r2, &ux2, &uy2, &T2);
    du[0][0] = 0.5 * (ux1 - ux2);
    du[0][1] = 0.5 * (uy1 - uy2);
    dT[0] = 0.5 * (T1 - T2);
    init_prim(a.rho, a.rhoux, a.rhouy, a.rhoE, pr.cv, yp * nx + x, &r1, &ux1, &uy1, &T1);
    init_prim(a.rho, a.rhoux, a.rhouy, a.rhoE, pr.cv, ym * nx + x, &r2, &ux2, &uy2, &T2);
    du[1][0] = 0.5 * (ux1 - ux2);
    du[1][1] = 0.5 * (uy1 - uy2);
    dT[1] = 0.5 * (T1 - T2);
    const int U0x = select_shift(ux, pr.n0, pr.umax), U0y = select_shift(uy, pr.n0, pr.umax);
    const int code = lat_code(U0x, U0y);
    double lam[NM], p[Q];
    const bool realizable = (r > 0.0) && (T > 0.0) && isfinite(r) && isfinite(T);
    const int ns = realizable
                       ? node_equilibrium<P>(pr, ux - U0x, uy - U0y, T, s_tab, nullptr, lam, p, &cnt)
                       : NEWTON_UNREALIZABLE;
    if (!realizable) n_bad += 1;
    if (ns != NEWTON_OK && realizable) n_fail += 1;
    const double gfac = (2.0 * pr.cv - 2.0) * T;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double cbx = (double)(XI_X(i) + U0x) - ux;
      const double cby = (double)(XI_Y(i) + U0y) - uy;
      double phf = 0.0, phg = 0.0;
      double feq = 0.0;
      if (ns == NEWTON_OK) {
        grad_phi(pr, r, T, cbx, cby, du, dT, &phf, &phg);
        feq = r * p[i];
      }
      st[i * BLOCK] = (P)(feq * (1.0 + phf));
      st[(Q + i) * BLOCK] = (P)(gfac * feq * (1.0 + phg));
    }
    if (ns == NEWTON_OK) {
      float wbuf[NM];
      const float* warm = nullptr;
      if constexpr (std::is_same<P, float>::value) {
#pragma unroll
        for (int j = 0; j < NM; ++j) wbuf[j] = (float)lam[j];
        warm = wbuf;
      }
      collide_store<P>(pr, st, code, k, a.ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out,
                       s_tab, warm, a.lam_out, &cnt, &n_fail);
    } else {
      for (int i = 0; i < NPLANES; ++i) a.pop_out[i * a.ps + k] = (P)0;
      a.mom_out[k] = (P)r;
      a.mom_out[a.ps + k] = (P)ux;
      a.mom_out[2 * a.ps + k] = (P)uy;
      a.mom_out[3 * a.ps + k] = (P)T;
      a.lat_out[k] = (uint8_t)code;
      a.nxt_out[k] = (uint8_t)code;
      if constexpr (std::is_same<P, float>::value)
#pragma unroll
        for (int j = 0; j < NM; ++j) a.lam_out[j * a.ps + k] = j == 3 || j == 5 ? 0.5f : 0.0f;
    }
  }
  warp_count(a.ctr + CTR_UNREALIZABLE, n_bad);
  warp_count(a.ctr + CTR_NEWTON_FAIL, n_fail);
}

template <typename P>
__global__ void export_moments_kernel(const P* mom, size_t ps, size_t n, double cv, double* rho,
                                      double* rhoux, double* rhouy, double* rhoE) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const double r = (double)mom[k], ux = (double)mom[ps + k], uy = (double)mom[2 * ps + k],
                 T = (double)mom[3 * ps + k];
    rho[k] = r;
    rhoux[k] = r * ux;
    rhouy[k] = r * uy;
    rhoE[k] = 0.5 * r * (ux * ux + uy * uy) + r * cv * T;
  }
}

__global__ void export_shifts_kernel(const uint8_t* lat, size_t n, signed char* ux,
                                     signed char* uy) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const int c = lat[k];
    ux[k] = (signed char)lat_ux(c);
    uy[k] = (signed char)lat_uy(c);
  }
}

__global__ void equilibrium_kernel(const double* rho, const double* ubx, const double* uby,
                                   const double* T, int n, double tol, int maxit, int precision,
                                   double* feq, double* lambda, int* iters, int* status) {
  __shared__ double s_tab[32];
  load_exptab(s_tab);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double lam[NM], p[Q];
  const double r = rho[k];
  Params pr{};
  pr.tol = tol;
  pr.maxit = maxit;
  SolveCount cnt;
  int st = NEWTON_UNREALIZABLE;
  if (r > 0.0)
    st = precision == 0
             ? node_equilibrium<double>(pr, ubx[k], uby[k], T[k], s_tab, nullptr, lam, p, &cnt)
             : node_equilibrium<float>(pr, ubx[k], uby[k], T[k], s_tab, nullptr, lam, p, &cnt);
#pragma unroll
  for (int i = 0; i < Q; ++i) feq[(size_t)k * Q + i] = r * p[i];
  if (lambda)
#pragma unroll
    for (int j = 0; j < NM; ++j) lambda[(size_t)k * NM + j] = lam[j];
  if (iters) iters[k] = precision == 0 ? (int)cnt.fp64_iters : (int)cnt.fp64_evals;
  if (status) status[k] = st;
}

__global__ void exp_neg_kernel(const double* s, int n, double* out) {
  __shared__ double s_tab[32];
  load_exptab(s_tab);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = exp_neg(s[k], s_tab);
}

__global__ void select_kernel(const double* rho, const double* rhou, int n, double n0, int umax,
                              signed char* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = (signed char)select_shift(rhou[k] / rho[k], n0, umax);
}

// ----------------------------------------------------------------- launchers

static dim3 grid_of(const Params& p) { return dim3((p.nx + BLOCK - 1) / BLOCK, p.ny); }

cudaError_t launch_init(FlowDev& f, const double* rho, const double* rhoux, const double* rhouy,
                        const double* rhoE, cudaStream_t s) {
  const int out = f.cur;
  if (f.precision == 0) {
    InitArgs<double> a{rho, rhoux, rhouy, rhoE, (double*)f.pop[out], (double*)f.mom[out],
                       f.lat[out], f.nxt[out], nullptr, f.ps, f.prm, f.ctr};
    init_kernel<double><<<grid_of(f.prm), BLOCK, NPLANES * BLOCK * sizeof(double), s>>>(a);
  } else {
    InitArgs<float> a{rho, rhoux, rhouy, rhoE, (float*)f.pop[out], (float*)f.mom[out],
                      f.lat[out], f.nxt[out], f.lam[out], f.ps, f.prm, f.ctr};
    init_kernel<float><<<grid_of(f.prm), BLOCK, NPLANES * BLOCK * sizeof(float), s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(FlowDev& f, cudaStream_t s) {
  const int in = f.cur, out = f.cur ^ 1;
  if (f.precision == 0) {
    StepArgs<double> a{(const double*)f.pop[in], (double*)f.pop[out], (const double*)f.mom[in],
                       (double*)f.mom[out], f.lat[in], f.nxt[in], f.lat[out], f.nxt[out],
                       nullptr, nullptr, f.ps, f.prm, f.ctr};
    step_kernel<double><<<grid_of(f.prm), BLOCK, NPLANES * BLOCK * sizeof(double), s>>>(a);
  } else {
    StepArgs<float> a{(const float*)f.pop[in], (float*)f.pop[out], (const float*)f.mom[in],
                      (float*)f.mom[out], f.lat[in], f.nxt[in], f.lat[out], f.nxt[out],
                      f.lam[in], f.lam[out], f.ps, f.prm, f.ctr};
    step_kernel<float><<<grid_of(f.prm), BLOCK, NPLANES * BLOCK * sizeof(float), s>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) f.cur = out;
  return e;
}

cudaError_t launch_export_moments(const FlowDev& f, double* rho, double* rhoux, double* rhouy,
                                  double* rhoE, cudaStream_t s) {
  const int blocks = (int)((f.n + 255) / 256 < 4096 ? (f.n + 255) / 256 : 4096);
  if (f.precision == 0)
    export_moments_kernel<double><<<blocks, 256, 0, s>>>((const double*)f.mom[f.cur], f.ps, f.n,
                                                         f.prm.cv, rho, rhoux, rhouy, rhoE);
  else
    export_moments_kernel<float><<<blocks, 256, 0, s>>>((const float*)f.mom[f.cur], f.ps, f.n,
                                                        f.prm.cv, rho, rhoux, rhouy, rhoE);
  return cudaGetLastError();
}

cudaError_t launch_export_shifts(const FlowDev& f, signed char* ux, signed char* uy,
                                 cudaStream_t s) {
  const int blocks = (int)((f.n + 255) / 256 < 4096 ? (f.n + 255) / 256 : 4096);
  export_shifts_kernel<<<blocks, 256, 0, s>>>(f.lat[f.cur], f.n, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_equilibrium(const double* rho, const double* ubx, const double* uby,
                               const double* T, int n, double tol, int maxit, int precision,
                               double* feq, double* lambda, int* iters, int* status,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  equilibrium_kernel<<<(n + 127) / 128, 128, 0, s>>>(rho, ubx, uby, T, n, tol, maxit, precision,
                                                     feq, lambda, iters, status);
  return cudaGetLastError();
}

cudaError_t launch_exp_neg(const double* x, int n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  exp_neg_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_select(const double* rho, const double* rhou, int n, double n0, int umax,
                          signed char* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  select_kernel<<<(n + 255) / 256, 256, 0, s>>>(rho, rhou, n, n0, umax, out);
  return cudaGetLastError();
}

}  // namespace alb
