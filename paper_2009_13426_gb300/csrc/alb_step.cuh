// Per-node update of the adaptive D2Q21 LBM step (Sec. IV.A.3), shared by the
// single-flow and the batched kernels.
//
// One thread updates one node. Its pulled populations (42, precision P) and
// the 21 FP64 equilibrium values per unit density of its latest equilibrium
// solve sit in two columns of the block's dynamic shared memory, with the
// block size as stride.
#pragma once

#include <type_traits>

#include "alb_internal.h"
#include "alb_mixed.cuh"

namespace alb {

constexpr int BLOCK = 128;

template <typename P, int B = BLOCK>
constexpr size_t smem_bytes() {
  return (size_t)NPLANES * B * sizeof(P) + (size_t)Q * B * sizeof(double);
}

// Shared columns of this thread: populations (P) and equilibrium (double),
// both with stride B (the block size).
template <typename P, int B>
struct Columns {
  P* pop;
  double* eq;
  __device__ __forceinline__ Columns(unsigned char* smem) {
    pop = reinterpret_cast<P*>(smem) + threadIdx.x;
    eq = reinterpret_cast<double*>(smem + (size_t)NPLANES * B * sizeof(P)) + threadIdx.x;
  }
};

// Equilibrium of one node in the storage precision P: the full FP64 Newton for
// the FP64 plain path, the mixed FP32/FP64 solver for the FP32 form, both
// started from `warm` (multipliers in precision P) when given. The
// equilibrium per unit density lands in eq[i * B], the multipliers (in the
// precision P the warm start keeps them in) in lam.
template <typename P, int B = BLOCK>
__device__ __forceinline__ int node_equilibrium(const Params& pr, double ubx, double uby,
                                                double T, const double* tab, const P* warm,
                                                double* eq, P lam[NM], SolveCount* cnt) {
  if (pr.moments == 4) {
    // reduced model: FP64 4x4 Newton in both precisions
    double w8[NM], l8[NM];
    if (warm)
#pragma unroll
      for (int k = 0; k < NM; ++k) w8[k] = (double)warm[k];
    int it = 0, ev = 0;
    int st = newton4_fp64g(ubx, uby, T, pr.tol, pr.maxit, tab, eq, B, l8, &it, &ev,
                           warm ? w8 : nullptr);
    cnt->fp64_iters += it;
    cnt->fp64_evals += ev;
    if (warm && st != NEWTON_OK && st != NEWTON_UNREALIZABLE) {
      st = newton4_fp64g(ubx, uby, T, pr.tol, pr.maxit, tab, eq, B, l8, &it, &ev, nullptr);
      cnt->fp64_iters += it;
      cnt->fp64_evals += ev;
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) lam[k] = (P)l8[k];
    return st;
  }
  if constexpr (std::is_same<P, float>::value) {
    return equilibrium_mixed(ubx, uby, T, pr.tol, pr.maxit, tab, warm, eq, B, lam, nullptr, cnt);
  } else {
    int it = 0, ev = 0;
    int st = newton_fp64g(ubx, uby, T, pr.tol, pr.maxit, tab, eq, B, lam, &it, &ev, warm);
    cnt->fp64_iters += it;
    cnt->fp64_evals += ev;
    if (warm && st != NEWTON_OK && st != NEWTON_UNREALIZABLE) {
      // the previous multipliers led nowhere: start again from the Maxwellian
      st = newton_fp64g(ubx, uby, T, pr.tol, pr.maxit, tab, eq, B, lam, &it, &ev, nullptr);
      cnt->fp64_iters += it;
      cnt->fp64_evals += ev;
    }
    return st;
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
  __device__ __forceinline__ double val() const { return cvt_f64(s + c); }
  __device__ __forceinline__ float valf() const { return s + c; }
};

// Multipliers stored for node k (8 planes of L), moved into the frame of
// lattice (Ux, Uy) from the lattice code they were computed in.
template <typename L>
__device__ __forceinline__ void load_warm(const L* lam, size_t ps, size_t k, int code_from,
                                          int Ux, int Uy, L w[NM]) {
  L l[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) l[j] = lam[j * ps + k];
  const int dx = lat_ux(code_from) - Ux, dy = lat_uy(code_from) - Uy;
  if (dx == 0 && dy == 0) {
#pragma unroll
    for (int j = 0; j < NM; ++j) w[j] = l[j];
  } else {
    shift_multipliers<L>(l, (L)dx, (L)dy, w);
  }
}

// Grad rebuild of a missing pull (Sec. III.B.2, IV.A.3): the post-collision
// population of velocity i = (cx, cy) in the receiver's lattice (Upx, Upy),
// built from the sender's moments at (sx, sy) (possibly a ghost), their
// central differences and the sender's relaxation time:
// h* = h^eq (1 + (1 - 1/tau) phi_h), plus (1/tau - 1/tau_Pr) h^eq phi_h,q for
// Pr != 1 (the collision of App. E applied to the Grad population). Uses the
// thread's equilibrium column as scratch. Returns 1 if the root finder failed
// and the Maxwellian-guess fallback was used. With eq_led given, the
// equilibrium of this sender in this lattice has been solved already (by
// another pull of the block): its column eq_led and whether that solve
// failed (led_failed) take the place of the solve.
template <typename P, int B>
__device__ __noinline__ int rebuild_pull(const Params pr, const P* __restrict__ mom, size_t ps,
                                         int i, int cx, int cy, int Upx, int Upy, int sx, int sy,
                                         double* fi, double* gi, const double* tab, double* eq,
                                         const P* lam_in, const uint8_t* lat_in,
                                         SolveCount* cnt, const double* eq_led = nullptr,
                                         int led_failed = 0) {
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
  int st;
  if (eq_led) {
    st = led_failed ? NEWTON_MAXIT : NEWTON_OK;
    eq = const_cast<double*>(eq_led);  // read only below
  } else {
    P lam[NM];
    P wbuf[NM];
    const P* warm = nullptr;
    if (pr.warm) {
      load_warm<P>(lam_in, ps, ks, lat_in[ks], Upx, Upy, wbuf);
      warm = wbuf;
    }
    st = (rho > 0.0) ? node_equilibrium<P, B>(pr, ubx, uby, T, tab, warm, eq, lam, cnt)
                     : NEWTON_UNREALIZABLE;
  }
  const double gfac = (2.0 * pr.cv - 2.0) * T;
  if (st != NEWTON_OK) {
    if (T > 0.0) {
      double lam[NM];
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
  const double feq = rho * eq[i * B];
  const double cbx = (double)(cx + Upx) - ux;
  const double cby = (double)(cy + Upy) - uy;
  double phf, phg, phq;
  grad_phi(pr, rho, T, cbx, cby, du, dT, &phf, &phg, &phq);
  if (pr.shakhov) {
    const double w = 1.0 / tau - 1.0 / (0.5 + (pr.nu / pr.prandtl) / T);
    *fi = feq * (1.0 + omega * phf + w * phq);
    *gi = gfac * feq * (1.0 + omega * phg + w * phg);
  } else {
    *fi = feq * (1.0 + omega * phf);
    *gi = gfac * feq * (1.0 + omega * phg);
  }
  return 0;
}

// The equilibrium column (FP64 values per unit density at stride B) in the
// population precision. In the FP32 form every value is rounded to FP32 once,
// in place, into the first word of its slot (the FP64 value is not read
// again), so that the sensor, the BGK update and the App. E term read the
// same float; the rounding runs on the integer pipe (cvt_f32_rn), not the
// FP64 pipe. Element i is then at [i * eq_stride<P, B>()].
template <typename P, int B>
__device__ __forceinline__ const P* eq_in_precision(double* eq) {
  if constexpr (std::is_same<P, float>::value) {
    float* v = reinterpret_cast<float*>(eq);
#pragma unroll
    for (int i = 0; i < Q; ++i) v[2 * i * B] = cvt_f32_rn(eq[i * B]);
    return v;
  } else {
    return eq;
  }
}
template <typename P, int B>
__host__ __device__ constexpr int eq_stride() {
  return std::is_same<P, float>::value ? 2 * B : B;
}

// |f - fe| / fe of the kinetic sensor (Eq. DeltaAvg): a fast division in
// FP32 (its relative error, about 1e-7, is that of the FP32 populations
// themselves, and alpha is continuous in eps), IEEE division in FP64.
__device__ __forceinline__ float rel_dev(float f, float fe) {
  return __fdividef(fabsf(f - fe), fe);
}
__device__ __forceinline__ double rel_dev(double f, double fe) { return fabs(f - fe) / fe; }

// Store of a collided node for Pr != 1: BGK plus the heat-flux term of App. E
// (Eqs. Shakhov, prandtlPoly),
//   f* += (1/tau - 1/tau_Pr) q.cbar / (rho Cp T^2) (|cbar|^2 / (2T) - Cp) f^eq,
//   g* += (1/tau - 1/tau_Pr) 2 q.cbar / (rho Cp) g^eq,
// with q_a = 1/2 sum_i cbar_ia (|cbar_i|^2 f_i + g_i) of the pre-collision
// populations st, cbar_i = xi_i - (u - U) (lattice frame, U of lattice
// `code`), tau_Pr = 1/2 + (nu/Pr)/T, both relaxation times scaled by the
// sensor factor tau / (1/2 + nu/T).
template <typename P, int B>
__device__ __forceinline__ void store_shakhov(const Params& pr, const P* st, const P* eqv,
                                              double rho, double ux, double uy, double T,
                                              int code, P tau, size_t k, size_t ps,
                                              P* __restrict__ pop_out) {
  const P Tp = (P)T, rp = (P)rho;
  const P bx = (P)(ux - (double)lat_ux(code)), by = (P)(uy - (double)lat_uy(code));
  const P cp = (P)pr.cp;
  const P gp = ((P)2 * (P)pr.cv - (P)2) * Tp;
  const P tau_pr = ((P)0.5 + (P)(pr.nu / pr.prandtl) / Tp) * (tau / ((P)0.5 + (P)pr.nu / Tp));
  const P om = (P)1 / tau;
  const P w = om - (P)1 / tau_pr;
  P qx = 0, qy = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const P cx = (P)XI_X(i) - bx, cy = (P)XI_Y(i) - by;
    const P e = (cx * cx + cy * cy) * st[i * B] + st[(Q + i) * B];
    qx += cx * e;
    qy += cy * e;
  }
  qx *= (P)0.5;
  qy *= (P)0.5;
  const P af = w / (rp * cp * Tp * Tp);
  const P ag = w * (P)2 / (rp * cp);
  const P h = (P)0.5 / Tp;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const P fe = eqv[i * eq_stride<P, B>()] * rp;
    const P ge = gp * fe;
    const P f = st[i * B];
    const P g = st[(Q + i) * B];
    const P cx = (P)XI_X(i) - bx, cy = (P)XI_Y(i) - by;
    const P c2 = cx * cx + cy * cy;
    const P qc = qx * cx + qy * cy;
    __stcs(&pop_out[i * ps + k], fma(om, fe - f, f) + af * qc * (c2 * h - cp) * fe);
    __stcs(&pop_out[(Q + i) * ps + k], fma(om, ge - g, g) + ag * qc * ge);
  }
}

// Moments, next shift, equilibrium and BGK of one node whose 42 pre-collision
// populations sit in its shared column, then store.
template <typename P, int B>
__device__ __forceinline__ void collide_store(const Params& pr, const Columns<P, B>& cl, int code,
                                              size_t k, size_t ps, P* __restrict__ pop_out,
                                              P* __restrict__ mom_out, uint8_t* lat_out,
                                              uint8_t* nxt_out, const double* tab,
                                              const P* warm, P* lam_out,
                                              SolveCount* cnt, unsigned* n_fail,
                                              const uint8_t* nb = nullptr) {
  const P* st = cl.pop;
  const int Ux = lat_ux(code), Uy = lat_uy(code);
  Acc<P> ar, ajx, ajy, ae;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const P f = st[i * B];
    const P g = st[(Q + i) * B];
    ar.add(f);
    if (XI_X(i) != 0) ajx.add(XI_X(i) == 1 ? f : XI_X(i) == -1 ? -f : (P)XI_X(i) * f);
    if (XI_Y(i) != 0) ajy.add(XI_Y(i) == 1 ? f : XI_Y(i) == -1 ? -f : (P)XI_Y(i) * f);
    const int c2 = XI_X(i) * XI_X(i) + XI_Y(i) * XI_Y(i);
    if (c2 != 0) ae.add(c2 == 1 ? f : (P)c2 * f);
    ae.add(g);
  }
  // Moments (Eq. polyTemp). The velocity and temperature that define the
  // equilibrium's targets are formed in FP64 from the (FP32 or FP64) sums, so
  // that the collision conserves the sums to their own precision; the next
  // lattice (Eq. criterion) is chosen from u = (rho u) / rho in FP64.
  const double rho = ar.val();
  double ubx, uby, T;
  if constexpr (std::is_same<P, float>::value) {
    // FP32 sums: one FP64 reciprocal serves the three quotients (their last
    // FP64 bit lies far below the sums' own precision); 1/(2 Cv) = (gamma-1)/2
    const double ir = 1.0 / rho;
    ubx = ajx.val() * ir;
    uby = ajy.val() * ir;
    T = (ae.val() - rho * (ubx * ubx + uby * uby)) * ir * pr.half_gm1;
  } else {
    ubx = ajx.val() / rho;
    uby = ajy.val() / rho;
    T = (ae.val() - rho * (ubx * ubx + uby * uby)) / (2.0 * rho * pr.cv);
  }
  const double ux = ubx + cvt_f64(Ux), uy = uby + cvt_f64(Uy);
  // next lattice: Eq. criterion, or overlapping ranges chosen by history or
  // by the neighbours' current lattices nb[0..7]
  const bool by_nb = order_key(pr.overlap) > 0 && pr.rule == 1 && nb;
  const int code2 = by_nb ? lat_code(select_shift_neighbours(ux, 0, nb, pr),
                                     select_shift_neighbours(uy, 1, nb, pr))
                          : lat_code(select_shift_kept(ux, Ux, pr), select_shift_kept(uy, Uy, pr));

  P lam[NM];
  const int ns = (rho > 0.0) ? node_equilibrium<P, B>(pr, ubx, uby, T, tab, warm, cl.eq, lam, cnt)
                             : NEWTON_UNREALIZABLE;
  // multipliers for the next step's warm start (lattice `code`), if stored
  if (lam_out) {
    if (ns == NEWTON_OK) {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = lam[j];
    } else if (warm) {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = warm[j];
    } else {
#pragma unroll
      for (int j = 0; j < NM; ++j) lam_out[j * ps + k] = j == 3 || j == 5 ? (P)0.5 : (P)0;
    }
  }
  if (ns == NEWTON_OK) {
    // f^eq = rho p, g^eq = (2 Cv - D) T f^eq and tau = 1/2 + nu/T in the
    // population precision (in the FP32 form from the FP64 equilibrium)
    const P Tp = to_p<P>(T);
    const P gp = ((P)2 * to_p<P>(pr.cv) - (P)2) * Tp;
    P tau = (P)0.5 + to_p<P>(pr.nu) / Tp;
    const P rp = to_p<P>(rho);
    const P* eqv = eq_in_precision<P, B>(cl.eq);
    constexpr int es = eq_stride<P, B>();
    if (pr.sensor) {
      P eps = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const P fe = eqv[i * es] * rp;
        eps += rel_dev(st[i * B], fe);
      }
      eps /= (P)Q;
      tau *= sensor_alpha<P>(pr, eps);
    }
    if (pr.shakhov) {
      store_shakhov<P, B>(pr, st, eqv, rho, ux, uy, T, code, tau, k, ps, pop_out);
    } else {
      const P om = (P)1 / tau;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const P fe = eqv[i * es] * rp;
        const P ge = gp * fe;
        const P f = st[i * B];
        const P g = st[(Q + i) * B];
        __stcs(&pop_out[i * ps + k], fma(om, fe - f, f));
        __stcs(&pop_out[(Q + i) * ps + k], fma(om, ge - g, g));
      }
    }
  } else {
    *n_fail += 1;
#pragma unroll
    for (int i = 0; i < NPLANES; ++i) pop_out[i * ps + k] = st[i * B];
  }
  mom_out[k] = to_p<P>(rho);
  mom_out[ps + k] = to_p<P>(ux);
  mom_out[2 * ps + k] = to_p<P>(uy);
  mom_out[3 * ps + k] = to_p<P>(T);
  lat_out[k] = (uint8_t)code;
  nxt_out[k] = (uint8_t)code2;
}

// Current lattices of the eight nodes around (x, y) (boundary rule for
// positions outside the grid), in a fixed order.
__device__ __forceinline__ void neighbour_codes(const Params& pr, const uint8_t* cur, int x, int y,
                                                uint8_t nb[8]) {
  int m = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      bool gh = false;
      const int rx = resolve(x + dx, pr.nx, pr.bcx, &gh);
      const int ry = resolve(y + dy, pr.ny, pr.bcy, &gh);
      nb[m++] = cur[(size_t)ry * pr.nx + rx];
    }
}

// Counts of one node update, added to the flow's counters warp by warp.
struct NodeCount {
  SolveCount solve;
  unsigned rec = 0, rec_fail = 0, fail = 0, calls = 0;
};

__device__ __forceinline__ void flush_counts(unsigned long long* ctr, const NodeCount& c) {
  warp_count(ctr + CTR_NEWTON_ITERS, c.solve.fp64_iters);
  warp_count(ctr + CTR_FP64_EVALS, c.solve.fp64_evals);
  warp_count(ctr + CTR_FP32_ITERS, c.solve.fp32_iters);
  warp_count(ctr + CTR_FP64_UPDATES, c.solve.fp64_updates);
  warp_count(ctr + CTR_NEWTON_CALLS, c.calls);
  warp_count(ctr + CTR_NEWTON_FAIL, c.fail);
  warp_count(ctr + CTR_REC, c.rec);
  warp_count(ctr + CTR_REC_FAIL, c.rec_fail);
}

// Shared state of a block's rebuild queue: one entry (owner thread << 5 | i)
// per missing pull of the block's nodes, at most Q per node.
template <int B>
struct RebuildQueue {
  unsigned short entry[Q * B];
  unsigned key[B];             // (receiver lattice, sender position in the tile's frame)
  unsigned char failed[B];     // the entry's own solve fell back
  unsigned short slot[B];      // leader entry solved by thread j
  unsigned short solver[B];    // thread solving a leader entry
  int wsum[B / 32];            // missing pulls per warp
  int count;
};

// One time step of the nodes of a tile (Sec. IV.A.3), one node per thread:
// thread t updates node (x0 + (t & (2^lg - 1)), y0 + (t >> lg)) if it lies in
// the grid. Phase 1 pulls every population whose sender lives in the node's
// new lattice and queues the missing ones; phase 2 rebuilds the queued pulls
// with all threads of the block (each Grad rebuild is a full equilibrium
// solve, so spreading them keeps the warps of interface nodes from waiting on
// a few lanes); phase 3 collides and stores. A rebuilt value depends only on
// its inputs, not on the thread that computes it. All threads of the block
// must call this (it holds barriers).
template <typename P, int B>
__device__ __forceinline__ void tile_step(const StepArgs<P>& a, int x0, int y0, int lg,
                                          const Columns<P, B>& cl, const double* s_tab,
                                          RebuildQueue<B>& rq, NodeCount& nc) {
  const Params& pr = a.prm;
  const size_t ps = a.ps;
  const int t = threadIdx.x;
  const int mask = (1 << lg) - 1;
  const int x = x0 + (t & mask), y = y0 + (t >> lg);
  const bool active = x < pr.nx && y < pr.ny;
  size_t k = 0;
  int code = 0;
  unsigned own = 0;  // bit i: the sender of velocity i lives in lattice `code`
  if (active) {
    k = (size_t)y * pr.nx + x;
    code = a.nxt_in[k];
    const int Upx = lat_ux(code), Upy = lat_uy(code);
    // All loads first, so that they are in flight together (a pull's load
    // written straight to shared memory would wait for the previous
    // velocity's): for every velocity the sender's lattice code and its two
    // populations, whether or not the sender turns out to live in this node's
    // lattice (the index is inside the grid even for a ghost: resolve clamps
    // it). Then the populations of the senders in this lattice go to the
    // shared-memory column; the others are dropped and queued for a rebuild.
    // Populations are read once and written once per step: streaming
    // (evict-first) loads and stores keep L2 for the lattice codes and the
    // threads' stack.
    int sc[Q];
    P v[2 * Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bool gh = false;
      const int rx = resolve(x - XI_X(i) - Upx, pr.nx, pr.bcx, &gh);
      const int ry = resolve(y - XI_Y(i) - Upy, pr.ny, pr.bcy, &gh);
      const size_t ks = (size_t)ry * pr.nx + rx;
      sc[i] = gh ? -1 : (int)a.lat_in[ks];  // a ghost sender is always rebuilt
      v[i] = __ldcs(&a.pop_in[i * ps + ks]);
      v[Q + i] = __ldcs(&a.pop_in[(Q + i) * ps + ks]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) own |= (sc[i] == code ? 1u : 0u) << i;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (own & (1u << i)) {
        cl.pop[i * B] = v[i];
        cl.pop[(Q + i) * B] = v[Q + i];
      }
    }
  }
  // The queue of missing pulls in (thread, velocity) order, placed by a
  // block-wide prefix sum of the threads' counts, so that its order, and with
  // it which pulls share a solve below, does not depend on scheduling. A tile
  // without missing pulls passes one barrier and skips the rest.
  int nq = 0;
  {
    const unsigned miss = active ? (~own & ((1u << Q) - 1u)) : 0u;
    const int nmiss = __popc(miss), lane = t & 31, warp = t >> 5;
    int incl = nmiss;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += u;
    }
    if (lane == 31) rq.wsum[warp] = incl;
    if (__syncthreads_or(nmiss)) {
      int pos = incl - nmiss;
      for (int w = 0; w < warp; ++w) pos += rq.wsum[w];
      for (unsigned m = miss; m; m &= m - 1)
        rq.entry[pos++] = (unsigned short)((t << 5) | (__ffs(m) - 1));
      if (t == B - 1) rq.count = pos;  // the last thread's end: the total
      __syncthreads();
      nq = rq.count;
    }
  }
  P* pop0 = cl.pop - t;  // column 0 of the block
  // Entries in chunks of B. The pulls of one sender in one receiver lattice
  // need the same equilibrium (the sender's state in that lattice, from the
  // same warm start). Within a chunk, the first entry of each such group (its
  // leader) is solved, by threads 0, 1, ... in entry order, so that the solves
  // fill as few warps as possible; every other entry then reads its leader's
  // column after a barrier. A solve's result does not depend on the thread,
  // so sharing it changes no value.
  static_assert(B % 32 == 0 && B <= 1000, "whole warps; tile sides fit the keys' 10-bit fields");
  const int lane = t & 31, warp = t >> 5;
#pragma unroll 1
  for (int base = 0; base < nq; base += B) {
    const int ne = min(nq - base, B);
    if (t < ne) {
      const int owner = rq.entry[base + t] >> 5, i = rq.entry[base + t] & 31;
      const int ox = x0 + (owner & mask), oy = y0 + (owner >> lg);
      const int ocode = a.nxt_in[(size_t)oy * pr.nx + ox];
      // the sender lies within 6 nodes of the tile (|xi| <= 3, |U| <= 3) and
      // the tile's sides are at most B <= 1000: 10 bits per coordinate
      const int sx = ox - XI_X(i) - lat_ux(ocode) - x0 + 8;
      const int sy = oy - XI_Y(i) - lat_uy(ocode) - y0 + 8;
      rq.key[t] = ((unsigned)ocode << 20) | ((unsigned)sy << 10) | (unsigned)sx;
    }
    __syncthreads();
    int lead = -1;
    if (t < ne) {
      const unsigned key = rq.key[t];
      lead = t;
      for (int e = 0; e < t; ++e)
        if (rq.key[e] == key) {
          lead = e;
          break;
        }
    }
    // number the leaders (block-wide prefix sum of the leader flags)
    const int isl = (t < ne && lead == t) ? 1 : 0;
    int incl = isl;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += u;
    }
    if (lane == 31) rq.wsum[warp] = incl;
    __syncthreads();
    int nlead = 0, rank = incl - isl;
    for (int w = 0; w < B / 32; ++w) {
      nlead += rq.wsum[w];
      if (w < warp) rank += rq.wsum[w];
    }
    if (isl) {
      rq.slot[rank] = (unsigned short)t;    // solver thread rank -> leader entry
      rq.solver[t] = (unsigned short)rank;  // leader entry -> its solver thread
    }
    __syncthreads();
    // pass 0: thread j < nlead solves the j-th leader entry; pass 1: every
    // other entry, with its leader's column
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      if (pass) __syncthreads();
      const int e = pass == 0 ? (t < nlead ? (int)rq.slot[t] : -1)
                              : (t < ne && lead != t ? t : -1);
      if (e >= 0) {
        const int owner = rq.entry[base + e] >> 5, i = rq.entry[base + e] & 31;
        const int ox = x0 + (owner & mask), oy = y0 + (owner >> lg);
        const int ocode = a.nxt_in[(size_t)oy * pr.nx + ox];
        const int Upx = lat_ux(ocode), Upy = lat_uy(ocode);
        const int cx = XI_X(i), cy = XI_Y(i);
        const int j = pass ? (int)rq.solver[lead] : t;  // thread whose column holds the solve
        double fd, gd;
        const int failed = rebuild_pull<P, B>(
            pr, a.mom_in, ps, i, cx, cy, Upx, Upy, ox - cx - Upx, oy - cy - Upy, &fd, &gd, s_tab,
            cl.eq, a.lam_in, a.lat_in, &nc.solve, pass ? cl.eq - t + j : nullptr,
            pass ? rq.failed[lead] : 0);
        if (!pass) {
          rq.failed[e] = (unsigned char)failed;
          nc.calls += 1;
        }
        nc.rec += 1;
        nc.rec_fail += failed;
        pop0[i * B + owner] = (P)fd;
        pop0[(Q + i) * B + owner] = (P)gd;
      }
    }
    // the next chunk reuses the columns, keys and slots; the last chunk's
    // rebuilt pulls are in place before the collisions
    __syncthreads();
  }
  if (active) {
    const int Upx = lat_ux(code), Upy = lat_uy(code);
    P wbuf[NM];
    const P* warm = nullptr;
    if (pr.warm) {
      load_warm<P>(a.lam_in, ps, k, a.lat_in[k], Upx, Upy, wbuf);
      warm = wbuf;
    }
    uint8_t nb[8];
    if (order_key(pr.overlap) > 0 && pr.rule == 1) neighbour_codes(pr, a.nxt_in, x, y, nb);
    collide_store<P, B>(pr, cl, code, k, ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out, s_tab,
                        warm, a.lam_out, &nc.solve, &nc.fail, nb);
    nc.calls += 1;
  }
}

}  // namespace alb
