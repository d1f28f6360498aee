// Kernels of the adaptive D2Q21 LBM step (one node per thread).
//
//  step_kernel   pull (Eq. stream) in the receiver's lattice with Grad rebuild
//                of missing pulls (Eqs. GradGeneral*), moments (Eq. polyTemp),
//                shift for the next pull (Eq. criterion), numerical equilibrium
//                (Eq. feqNum_8Mom), g^eq (Eq. gEq), optional sensor
//                (Eq. DeltaAvg), BGK (Eq. coll), store.
//  init_kernel   Grad-regularised initial populations, then the same collision.
//  export / equilibrium / select kernels for the C ABI.
//
// Layout: structure of arrays. Plane p (f_0..f_20, g_0..g_20) of a buffer is
// a contiguous nx*ny array, x fastest; lattice codes and moments likewise.
// Each thread owns two columns of the block's dynamic shared memory: its 42
// pulled populations (stride BLOCK) and the 21 FP64 equilibrium values per
// unit density of its latest equilibrium solve (stride BLOCK).
#include <type_traits>

#include "alb_step.cuh"

namespace alb {

// Launch shape of the step kernel per precision: the FP32 form runs blocks of
// 256 threads, two per SM (measured on the 4096^2 shear layer once developed,
// through the batch kernel's compiled shapes: 620 MLUPS against 591 for
// 128 x 4 and 555 for 128 x 3); FP64 plain runs 128 threads with up to 255
// registers each.
template <typename P>
struct StepShape;
template <>
struct StepShape<float> {
  static constexpr int B = 256, MINB = 2, LOG2B = 8;
};
template <>
struct StepShape<double> {
  static constexpr int B = 128, MINB = 1, LOG2B = 7;
};

// One time step of every node: block (bx, by) updates the tile of 2^lg nodes
// along x by B >> lg rows at (bx << lg, by * (B >> lg)).
template <typename P>
__global__ void __launch_bounds__(StepShape<P>::B, StepShape<P>::MINB)
    step_kernel(StepArgs<P> a, int lg) {
  constexpr int B = StepShape<P>::B;
  static_assert((1 << StepShape<P>::LOG2B) == B, "tiles of B nodes");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_tab[EXPT_N];
  __shared__ RebuildQueue<B> s_rq;
  load_exptab(s_tab);  // includes a barrier
  const Columns<P, B> cl(smem_raw);
  NodeCount nc;
  tile_step<P, B>(a, blockIdx.x << lg, blockIdx.y << (StepShape<P>::LOG2B - lg), lg, cl, s_tab,
                  s_rq, nc);
  flush_counts(a.ctr, nc);
}

template <typename P>
struct InitArgs {
  const double *rho, *rhoux, *rhouy, *rhoE;
  P* pop_out;
  P* mom_out;
  uint8_t* lat_out;
  uint8_t* nxt_out;
  P* lam_out;
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
__global__ void __launch_bounds__(BLOCK, (std::is_same<P, float>::value ? 4 : 1))
    init_kernel(InitArgs<P> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_tab[EXPT_N];
  load_exptab(s_tab);
  const Columns<P, BLOCK> cl(smem_raw);
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
    P lam[NM];
    const bool realizable = (r > 0.0) && (T > 0.0) && isfinite(r) && isfinite(T);
    const int ns = realizable ? node_equilibrium<P>(pr, ux - U0x, uy - U0y, T, s_tab, nullptr,
                                                    cl.eq, lam, &cnt)
                              : NEWTON_UNREALIZABLE;
    if (!realizable) n_bad += 1;
    if (ns != NEWTON_OK && realizable) n_fail += 1;
    const double gfac = (2.0 * pr.cv - 2.0) * T;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double cbx = (double)(XI_X(i) + U0x) - ux;
      const double cby = (double)(XI_Y(i) + U0y) - uy;
      double phf = 0.0, phg = 0.0, phq = 0.0;
      double feq = 0.0;
      if (ns == NEWTON_OK) {
        grad_phi(pr, r, T, cbx, cby, du, dT, &phf, &phg, &phq);
        feq = r * cl.eq[i * BLOCK];
      }
      cl.pop[i * BLOCK] = (P)(feq * (1.0 + phf));
      cl.pop[(Q + i) * BLOCK] = (P)(gfac * feq * (1.0 + phg));
    }
    if (ns == NEWTON_OK) {
      // the first collision starts from the multipliers just found if the
      // flow starts its solves from previous multipliers
      P wbuf[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) wbuf[j] = lam[j];
      // with the neighbourhood rule, the neighbours' initial lattices (Eq.
      // criterion on their initial velocities, boundary rule outside the grid)
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
      collide_store<P, BLOCK>(pr, cl, code, k, a.ps, a.pop_out, a.mom_out, a.lat_out, a.nxt_out,
                              s_tab, pr.warm ? wbuf : nullptr, a.lam_out, &cnt, &n_fail, nb);
    } else {
      for (int i = 0; i < NPLANES; ++i) a.pop_out[i * a.ps + k] = (P)0;
      a.mom_out[k] = (P)r;
      a.mom_out[a.ps + k] = (P)ux;
      a.mom_out[2 * a.ps + k] = (P)uy;
      a.mom_out[3 * a.ps + k] = (P)T;
      a.lat_out[k] = (uint8_t)code;
      a.nxt_out[k] = (uint8_t)code;
      if (a.lam_out)
#pragma unroll
        for (int j = 0; j < NM; ++j) a.lam_out[j * a.ps + k] = j == 3 || j == 5 ? (P)0.5 : (P)0;
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

// Planes [p0, p0 + np) of a buffer (population or moment planes, stride ps)
// as FP64 planes of n values each.
template <typename P>
__global__ void export_planes_kernel(const P* src, size_t ps, size_t n, int np, double* dst) {
  const size_t total = (size_t)np * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t p = t / n, k = t - p * n;
    dst[t] = (double)src[p * ps + k];
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

__global__ void __launch_bounds__(BLOCK)
    equilibrium_kernel(const double* rho, const double* ubx, const double* uby, const double* T,
                       int n, double tol, int maxit, int precision, double* feq, double* lambda,
                       int* iters, int* status) {
  __shared__ double s_tab[EXPT_N];
  __shared__ double s_eq[Q * BLOCK];
  load_exptab(s_tab);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double* eq = s_eq + threadIdx.x;
  double lam[NM];
  const double r = rho[k];
  Params pr{};
  pr.tol = tol;
  pr.maxit = maxit;
  SolveCount cnt;
  int st = NEWTON_UNREALIZABLE;
  if (r > 0.0) {
    if (precision == 0) {
      st = node_equilibrium<double>(pr, ubx[k], uby[k], T[k], s_tab, nullptr, eq, lam, &cnt);
    } else {
      float l32[NM];  // the FP64 multipliers are asked for here
      st = equilibrium_mixed(ubx[k], uby[k], T[k], tol, maxit, s_tab, nullptr, eq, BLOCK, l32,
                             lam, &cnt);
    }
  }
  for (int i = 0; i < Q; ++i) feq[(size_t)k * Q + i] = st == NEWTON_UNREALIZABLE ? 0.0 : r * eq[i * BLOCK];
  if (lambda)
#pragma unroll
    for (int j = 0; j < NM; ++j) lambda[(size_t)k * NM + j] = lam[j];
  if (iters)
    iters[k] = precision == 0 ? (int)cnt.fp64_iters : (int)(cnt.fp64_evals + cnt.fp64_updates);
  if (status) status[k] = st;
}

template <bool REFINE>
__global__ void exp_neg_kernel(const double* s, int n, double* out) {
  __shared__ double s_tab[EXPT_N];
  load_exptab(s_tab);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = REFINE ? exp_neg_refine(s[k], (float)s[k], s_tab) : exp_neg(s[k], s_tab);
}

__global__ void select_kernel(const double* rho, const double* rhou, int n, double n0, int umax,
                              signed char* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = (signed char)select_shift(rhou[k] / rho[k], n0, umax);
}

// ----------------------------------------------------------------- launchers

static dim3 grid_of(const Params& p) { return dim3((p.nx + BLOCK - 1) / BLOCK, p.ny); }

// Tiles of the step kernel: 2^lg nodes along x, the smallest power of two that
// holds a row (at least 8, at most the block), and the block's other threads
// on the following rows, so that narrow grids keep the threads busy.
template <typename P>
static dim3 step_grid(const Params& p, int* lg) {
  int l = 3;
  while (l < StepShape<P>::LOG2B && (1 << l) < p.nx) ++l;
  *lg = l;
  const int rows = (1 << StepShape<P>::LOG2B) >> l;
  return dim3((p.nx + (1 << l) - 1) >> l, (p.ny + rows - 1) / rows);
}

// Dynamic shared memory needs an explicit opt-in once static plus dynamic
// shared memory exceed 48 KB; the dynamic size is always declared.
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_init(FlowDev& f, const double* rho, const double* rhoux, const double* rhouy,
                        const double* rhoE, cudaStream_t s) {
  if (f.q == 49) return launch_init_q49(f, rho, rhoux, rhouy, rhoE, s);
  const int out = f.cur;
  cudaError_t e;
  if (f.precision == 0) {
    InitArgs<double> a{rho, rhoux, rhouy, rhoE, (double*)f.pop[out], (double*)f.mom[out],
                       f.lat[out], f.nxt[out], (double*)f.lam[out], f.ps, f.prm, f.ctr};
    if ((e = allow_smem(init_kernel<double>, smem_bytes<double>())) != cudaSuccess) return e;
    init_kernel<double><<<grid_of(f.prm), BLOCK, smem_bytes<double>(), s>>>(a);
  } else {
    InitArgs<float> a{rho, rhoux, rhouy, rhoE, (float*)f.pop[out], (float*)f.mom[out],
                      f.lat[out], f.nxt[out], (float*)f.lam[out], f.ps, f.prm, f.ctr};
    if ((e = allow_smem(init_kernel<float>, smem_bytes<float>())) != cudaSuccess) return e;
    init_kernel<float><<<grid_of(f.prm), BLOCK, smem_bytes<float>(), s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(FlowDev& f, cudaStream_t s) {
  if (f.q == 49) return launch_step_q49(f, s);
  const int in = f.cur, out = f.cur ^ 1;
  cudaError_t e;
  int lg = 0;
  if (f.precision == 0) {
    constexpr int B = StepShape<double>::B;
    const StepArgs<double> a = step_args<double>(f, in);
    const dim3 g = step_grid<double>(f.prm, &lg);
    if ((e = allow_smem(step_kernel<double>, smem_bytes<double, B>())) != cudaSuccess) return e;
    step_kernel<double><<<g, B, smem_bytes<double, B>(), s>>>(a, lg);
  } else {
    constexpr int B = StepShape<float>::B;
    const StepArgs<float> a = step_args<float>(f, in);
    const dim3 g = step_grid<float>(f.prm, &lg);
    if ((e = allow_smem(step_kernel<float>, smem_bytes<float, B>())) != cudaSuccess) return e;
    step_kernel<float><<<g, B, smem_bytes<float, B>(), s>>>(a, lg);
  }
  e = cudaGetLastError();
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

cudaError_t launch_export_planes(const FlowDev& f, int what, int p0, int np, double* dst,
                                 cudaStream_t s) {
  const int buf = f.cur;
  const void* base = what == 0 ? f.pop[buf] : f.mom[buf];
  const size_t total = (size_t)np * f.n;
  const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  if (total == 0) return cudaSuccess;
  if (f.precision == 0)
    export_planes_kernel<double><<<blocks, 256, 0, s>>>((const double*)base + p0 * f.ps, f.ps,
                                                        f.n, np, dst);
  else
    export_planes_kernel<float><<<blocks, 256, 0, s>>>((const float*)base + p0 * f.ps, f.ps,
                                                       f.n, np, dst);
  return cudaGetLastError();
}

cudaError_t launch_export_shifts(const FlowDev& f, signed char* ux, signed char* uy,
                                 cudaStream_t s, bool next) {
  const int blocks = (int)((f.n + 255) / 256 < 4096 ? (f.n + 255) / 256 : 4096);
  export_shifts_kernel<<<blocks, 256, 0, s>>>(next ? f.nxt[f.cur] : f.lat[f.cur], f.n, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_equilibrium(const double* rho, const double* ubx, const double* uby,
                               const double* T, int n, double tol, int maxit, int precision,
                               double* feq, double* lambda, int* iters, int* status,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  equilibrium_kernel<<<(n + BLOCK - 1) / BLOCK, BLOCK, 0, s>>>(rho, ubx, uby, T, n, tol, maxit,
                                                               precision, feq, lambda, iters,
                                                               status);
  return cudaGetLastError();
}

cudaError_t launch_exp_neg(const double* x, int n, double* out, cudaStream_t s, bool refine) {
  if (n <= 0) return cudaSuccess;
  if (refine)
    exp_neg_kernel<true><<<(n + 255) / 256, 256, 0, s>>>(x, n, out);
  else
    exp_neg_kernel<false><<<(n + 255) / 256, 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_select(const double* rho, const double* rhou, int n, double n0, int umax,
                          signed char* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  select_kernel<<<(n + 255) / 256, 256, 0, s>>>(rho, rhou, n, n0, umax, out);
  return cudaGetLastError();
}

}  // namespace alb
