// Riemannian PCG (Algorithm 1, PCG-ATKM) on the device.
//
// Per iteration n (phi = phi_n, Phi = Phi_n of the accepted previous trial):
//   H phi (3 axis passes, fused energy sums) -> mu, r = H phi - mu phi, ||r||
//   alpha -> P r (5 passes) -> PR+ scalars -> p, <H phi, p>, ||p||^2
//   (Step 4 (i): if <H phi, p> >= 0, p is re-formed as J(-P r))
//   H p, Phi' = U_dip * Re(conj(phi) p) -> curvature of Eq. (Energy_Expend)
//   t (Eq. (opt_step) or 0.3) -> retraction (Eq. (retraction)), renormalise,
//   Phi+ by ATKM, E(phi+) -> accept, or halve t and retry (Step 4 (iii)).
// All scalar decisions run in single-thread control kernels on a device
// control block, and the vector kernels read their coefficients from it, so an
// iteration is a fixed kernel sequence on ping-pong buffers: it is captured
// once as a CUDA graph per (precision, buffer parity) and replayed, with one
// host synchronisation per iteration (plus one per rare halving) to read the
// control block for the stop rule and the log.
//
// The trial energy's quadratic part is formed from <A phi,phi>, <A phi,p>,
// <A p,p> with A = -1/2[[Delta]] + V - Omega[[L_z]] (A is linear, so
// <A phi+, phi+> expands exactly in cos/sin of the retraction); only the
// quartic and dipolar terms need phi+ itself.  Reductions are deterministic
// (fixed grid, fixed-order two-level sums).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <utility>
#include <thread>
#include <vector>

#include "atkm_internal.cuh"

namespace atkm {

namespace {

constexpr int kRedGrid = 1216;  // most reduction CTAs of a vector kernel (partial-sum capacity)
constexpr int kRedThreads = 256;

// ------------------------------------------------------------ control block
struct Ctl {
  // constants of the solve
  double hv, beta, lam, tolE_eps;
  // state carried between iterations
  double E, den_prev;
  int have_E, have_prev, force_sd, pad0;
  // loop top of the current iteration
  double kin, rot, pot, f4, dip, mu, norm2, res, alpha;
  // direction
  double b, den, beta_cg, cp0, cp1, cp2, pn2, d1;
  int use_cg, reset, redo, nan;
  // step
  double Hpp, S1, S2, S3, curv, t0, t, pn, Aphiphi, Aphip, App, tolE;
  double cr, sr, nrm2, inv, En, linf, bestE, best_t;
  int accepted, nh, forced, pad1;
  double inv0;   // normalisation of psi_0
  double noise;  // FP32 noise of the residual at phi_0 (automatic hand-over)
  // device-driven loop (Solver::run_device): the decisions the host takes
  // between iterations in the host-driven path, taken by control kernels
  int n, n_start, max_iter, max_halv;
  int caps, status, done, handover;
  int logc, log_cap, f32, f32_iters;
  int total_h, f32_best_n, q, final_top;
  int step_logged, f32_window;
  double tol_res, tol_linf, switch_tol, f32_best, linf_n, f32_gain;
  unsigned long long deadline, guard, guard_max, launches;
  atkm_iter_log* log;  // device array of log_cap entries
};

// ------------------------------------------------------------ reductions
__global__ void k_finalize(const double* __restrict__ part, int nblocks, double* __restrict__ out,
                           const int* __restrict__ pred) {
  if (pred && !*pred) return;
  __shared__ double sh[kRedThreads];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kRedThreads) acc += part[(size_t)s * nblocks + i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[s] = sh[0];
}

// Grid maximum of the block maxima; out = its square root (the partials hold
// squared distances).
__global__ void k_finalize_max(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kRedThreads) acc = fmax(acc, part[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(sh[0]);
}

// Vector kernels of the driver.  Vectors are FP64 in memory.  T is the type
// of the per-element arithmetic: double in the FP64 phase; float in the FP32
// phase of the precision form, where every operand carries FP32-level
// accuracy only (H, ATKM and P ran in FP32) and FP64 products would only burn
// the slow FP64 pipe.  With T = float, loads convert on the integer pipe,
// sums accumulate per thread in FP32 over chunks of kChunk elements and in
// FP64 beyond (block and grid sums are FP64 in both phases).
constexpr int kChunk = 8;

template <typename T> struct V2 { T x, y; };
template <typename T> __device__ __forceinline__ V2<T> ld2(const double2& a) { return V2<T>{tor<T>(a.x), tor<T>(a.y)}; }
template <typename T> __device__ __forceinline__ T ld1(double a) { return tor<T>(a); }
template <typename T> __device__ __forceinline__ T dotr(V2<T> a, V2<T> b) { return a.x * b.x + a.y * b.y; }

template <typename T, int NS> struct Sums {
  double d[NS];
  T f[NS];
  int n;
  __device__ __forceinline__ Sums() : n(0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) { d[s] = 0.0; f[s] = (T)0; }
  }
  // sum_s += a b.  Binary64: one FMA (every instruction here is an FP64-pipe
  // instruction, and these kernels are bound by that pipe).  FP32: the
  // product, then the add.
  __device__ __forceinline__ void mac(int s, T a, T b) {
    if constexpr (sizeof(T) == 8) d[s] = fma(a, b, d[s]);
    else f[s] += a * b;
  }
  // sum_s += Re(a conj b) = a.x b.x + a.y b.y: two FMAs in binary64
  __device__ __forceinline__ void dot(int s, V2<T> a, V2<T> b) {
    if constexpr (sizeof(T) == 8) {
      d[s] = fma(a.x, b.x, d[s]);
      d[s] = fma(a.y, b.y, d[s]);
    } else {
      f[s] += a.x * b.x + a.y * b.y;
    }
  }
  __device__ __forceinline__ void flush() {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int s = 0; s < NS; ++s) { d[s] += tod<T>(f[s]); f[s] = (T)0; }
    }
    n = 0;
  }
  __device__ __forceinline__ void next() {
    if constexpr (sizeof(T) == 4) {
      if (++n == kChunk) flush();
    }
  }
  // Block sums into part[s * gridDim.x + blockIdx.x].  FP32 kernels hand each
  // thread's total to the FP32 warp stage (no per-thread FP64 shuffles).
  __device__ __forceinline__ void store(double* part) {
    flush();
    if constexpr (sizeof(T) == 4) {
      float v[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) v[s] = tor<float>(d[s]);
      block_reduce_store_f32<NS>(v, part, gridDim.x, blockIdx.x);
    } else {
      block_reduce_store<NS>(d, part, gridDim.x, blockIdx.x);
    }
  }
};

#define ATKM_GRID_LOOP(j, N) \
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < (N); j += (size_t)gridDim.x * blockDim.x)

// sum_j Re(u_j conj(v_j)) (FP64).
__global__ void __launch_bounds__(kRedThreads) k_dot(const double2* __restrict__ u, const double2* __restrict__ v,
                                                     size_t N, double* __restrict__ part) {
  Sums<double, 1> acc;
  ATKM_GRID_LOOP(j, N) {
    const double2 a = u[j], b = v[j];
    acc.mac(0, a.x, b.x);
    acc.mac(0, a.y, b.y);
  }
  acc.store(part);
}

// The seven sums of the direction step from one read of its five vectors:
// <Pr,phi>, <r,Pr>, <r,phi>, <r_prev,Pr>, <r_prev,phi>, <p_prev,phi>, <phi,phi>.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_dir_dots(const double2* __restrict__ Pr, const double2* __restrict__ phi, const double2* __restrict__ r,
           const double2* __restrict__ rp, const double2* __restrict__ pp, size_t N, double* __restrict__ part) {
  Sums<T, 7> acc;
  ATKM_GRID_LOOP(j, N) {
    const V2<T> P = ld2<T>(Pr[j]), f = ld2<T>(phi[j]), a = ld2<T>(r[j]), b = ld2<T>(rp[j]), c = ld2<T>(pp[j]);
    acc.dot(0, P, f);
    acc.dot(1, a, P);
    acc.dot(2, a, f);
    acc.dot(3, b, P);
    acc.dot(4, b, f);
    acc.dot(5, c, f);
    acc.dot(6, f, f);
    acc.next();
  }
  acc.store(part);
}

// A coefficient m * (*p) (p may be null: then m).
struct Coef {
  const double* p;
  double m;
};
__device__ __forceinline__ double cval(const Coef& c) { return c.p ? c.m * *c.p : c.m; }

// out = c0 v0 + c1 v1 + c2 v2 (null vectors skipped); sums |out|^2 and
// Re(w conj(out)) when w is given.  Skipped entirely when *pred == 0.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_lincomb(double2* __restrict__ out, const double2* __restrict__ v0, Coef c0, const double2* __restrict__ v1,
          Coef c1, const double2* __restrict__ v2, Coef c2, const double2* __restrict__ w, size_t N,
          double* __restrict__ part, const int* __restrict__ pred) {
  if (pred && !*pred) return;
  const T a0 = tor<T>(cval(c0)), a1 = tor<T>(cval(c1)), a2 = tor<T>(cval(c2));
  Sums<T, 2> acc;
  ATKM_GRID_LOOP(j, N) {
    V2<T> o{(T)0, (T)0};
    if (v0) { const V2<T> a = ld2<T>(v0[j]); o.x += a0 * a.x; o.y += a0 * a.y; }
    if (v1) { const V2<T> a = ld2<T>(v1[j]); o.x += a1 * a.x; o.y += a1 * a.y; }
    if (v2) { const V2<T> a = ld2<T>(v2[j]); o.x += a2 * a.x; o.y += a2 * a.y; }
    out[j] = make_double2(tod<T>(o.x), tod<T>(o.y));
    acc.dot(0, o, o);
    if (w) acc.dot(1, ld2<T>(w[j]), o);
    acc.next();
  }
  acc.store(part);
}

// phi+ *= *inv (FP64: the renormalisation); block max of |phi+ - phi|^2, the
// difference taken in T (FP32 in the FP32 phase, where it is only logged).
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_scale_linf(double2* __restrict__ phin, const double2* __restrict__ phi, const double* __restrict__ invp, size_t N,
             double* __restrict__ part) {
  __shared__ T sh[kRedThreads];
  const double inv = *invp;
  T m = (T)0;
  ATKM_GRID_LOOP(j, N) {
    double2 a = phin[j];
    a.x *= inv; a.y *= inv;
    phin[j] = a;
    const V2<T> x = ld2<T>(a), y = ld2<T>(phi[j]);
    const T dx = x.x - y.x, dy = x.y - y.y;
    m = fmax(m, dx * dx + dy * dy);
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = tod<T>(sh[0]);
}

// Sums for the curvature of the quadratic model:
//   [0] <Hp, p>
//   [1] sum rho'(beta rho' + lambda Phi'),  rho' = Re(conj(phi) p)
//   [2] sum (beta|phi|^2 + lambda Phi) Re(phi conj(p))
//   [3] sum (beta|phi|^2 + lambda Phi) |p|^2
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_curv_sums(const double2* __restrict__ Hp, const double2* __restrict__ phi, const double2* __restrict__ p,
            const double* __restrict__ Phi, const double* __restrict__ Phi1, double beta, double lambda, size_t N,
            double* __restrict__ part) {
  const T bt = tor<T>(beta), lm = tor<T>(lambda);
  Sums<T, 4> acc;
  ATKM_GRID_LOOP(j, N) {
    const V2<T> a = ld2<T>(phi[j]), b = ld2<T>(p[j]), h = ld2<T>(Hp[j]);
    const T rp = dotr(a, b);
    const T w = bt * dotr(a, a) + lm * ld1<T>(Phi[j]);
    acc.dot(0, h, b);
    acc.mac(1, rp, bt * rp + lm * ld1<T>(Phi1[j]));
    acc.mac(2, w, rp);
    acc.mac(3, w, dotr(b, b));
    acc.next();
  }
  acc.store(part);
}

// [0] sum |phi|^4, [1] sum Phi |phi|^2
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_quartic_sums(const double2* __restrict__ phi, const double* __restrict__ Phi, size_t N, double* __restrict__ part) {
  Sums<T, 2> acc;
  ATKM_GRID_LOOP(j, N) {
    const V2<T> a = ld2<T>(phi[j]);
    const T r = dotr(a, a);
    acc.mac(0, r, r);
    acc.mac(1, ld1<T>(Phi[j]), r);
    acc.next();
  }
  acc.store(part);
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

int red_grid(size_t N) {
  size_t b = (N + kRedThreads * 4 - 1) / (kRedThreads * 4);
  if (b < 1) b = 1;
  if (b > (size_t)kRedGrid) b = kRedGrid;
  return (int)b;
}

// Grid of a grid-stride vector kernel: whole waves (SMs x resident blocks of
// that kernel, from the occupancy calculator, cached per kernel), at most
// red_grid(N) -- a partial last wave would leave SMs idle at the end.
int wave_grid(const void* kernel, size_t N) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> cache;
  const int nsm = device_sm_count();
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& kv : cache)
      if (kv.first == kernel) per_sm = kv.second;
    if (per_sm == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRedThreads, 0) != cudaSuccess ||
          per_sm <= 0) {
        cudaGetLastError();
        per_sm = 4;
      }
      cache.emplace_back(kernel, per_sm);
    }
  }
  const size_t cap = (size_t)red_grid(N);
  if (nsm <= 0) return (int)cap;  // SM count unknown: the size-based grid
  const size_t full = (size_t)nsm * per_sm;
  if (cap < full) return (int)cap;
  return (int)(full > (size_t)kRedGrid ? std::max(kRedGrid / nsm, 1) * nsm : full);
}

// Slots of plan->scal used by the driver.
enum {
  S_H = SC_RED,          // 10 slots of the H phi reductions
  S_R = SC_RED + 10,     // |r|^2 (+ unused)
  S_D = SC_RED + 12,     // 7 dots for the direction
  S_P = SC_RED + 20,     // |p|^2, <H phi, p>
  S_C = SC_RED + 22,     // <Hp,p> and the 3 curvature sums
  S_T = SC_RED + 26,     // |phi+|^2 (+ unused)
  S_Q = SC_RED + 28,     // 2 quartic sums of phi+
  S_L = SC_RED + 30,     // linf
  S_N = SC_RED + 31,     // |psi0|^2
  S_Z = SC_RED + 32      // |H phi_0 in FP32 - H phi_0 in FP64|^2 (+ unused)
};

// ------------------------------------------------------------ control kernels
__device__ __forceinline__ bool fin(double v) { return isfinite(v); }

__global__ void k_c_init(Ctl* c, const double* s) {
  const double n0 = sqrt(c->hv * s[S_N]);
  c->nan = !(n0 > 0.0) || !fin(n0);
  c->inv0 = c->nan ? 0.0 : 1.0 / n0;
}

// the FP32 arithmetic's noise in the residual at phi_0: ||H_32 phi_0 - H_64 phi_0||
// (each with its own Phi), in the residual's norm
__global__ void k_c_noise(Ctl* c, const double* s) { c->noise = sqrt(c->hv * s[S_Z]); }

// loop top: energy terms of phi, mu, alpha (Step 2 and the shift of §2.3)
__global__ void k_c_parts(Ctl* c, const double* s) {
  const double hv = c->hv;
  c->kin = hv * (s[S_H + 0] + s[S_H + 2] + s[S_H + 4]);
  c->rot = hv * (s[S_H + 1] + s[S_H + 3]);
  c->pot = hv * s[S_H + 5];
  c->f4 = hv * s[S_H + 6];
  c->dip = hv * s[S_H + 7];
  c->mu = hv * s[S_H + 8];
  c->norm2 = hv * s[S_H + 9];
  if (!c->have_E) {
    c->E = c->kin + c->rot + c->pot + 0.5 * c->beta * c->f4 + 0.5 * c->lam * c->dip;
    c->have_E = 1;
  }
  c->alpha = c->kin + c->pot + c->beta * c->f4 + fabs(c->lam * c->dip);
}

__global__ void k_c_res(Ctl* c, const double* s) {
  c->res = sqrt(c->hv * s[S_R]);
  c->nan = !fin(c->E) || !fin(c->res) || !fin(c->mu);
}

// Step 3: PR+ coefficients, p = cp0 P r + cp1 p_prev + cp2 phi
__global__ void k_c_dir(Ctl* c, const double* s) {
  const double hv = c->hv;
  const double b = hv * s[S_D + 0], rPr = hv * s[S_D + 1], rphi = hv * s[S_D + 2];
  const double rpPr = hv * s[S_D + 3], a = hv * s[S_D + 4], cc = hv * s[S_D + 5], nphi = hv * s[S_D + 6];
  c->b = b;
  c->den = rPr - b * rphi;  // <r, J(P r)>
  c->use_cg = c->have_prev && !c->force_sd;
  c->reset = 0;
  if (c->use_cg) {
    const double jrj = rpPr - 2.0 * a * b + a * b * nphi;  // <J(r_prev), J(P r)>
    const double bcg = fmax((c->den - jrj) / c->den_prev, 0.0);
    c->beta_cg = bcg;
    c->cp0 = -1.0; c->cp1 = bcg; c->cp2 = b - bcg * cc;
  } else {
    c->beta_cg = 0.0;
    c->cp0 = -1.0; c->cp1 = 0.0; c->cp2 = b;
  }
}

// Step 4 (i): keep p if <H phi, p> < 0, otherwise re-form it as J(-P r)
__global__ void k_c_reset(Ctl* c, const double* s) {
  c->pn2 = c->hv * s[S_P];
  c->d1 = c->hv * s[S_P + 1];
  c->redo = 0;
  if (c->d1 >= 0.0) {
    c->reset = 1;
    c->beta_cg = 0.0;
    if (c->use_cg) {
      c->cp0 = -1.0; c->cp1 = 0.0; c->cp2 = c->b;
      c->redo = 1;
    }
  }
}

__global__ void k_c_reset2(Ctl* c, const double* s) {
  if (!c->redo) return;
  c->pn2 = c->hv * s[S_P];
  c->d1 = c->hv * s[S_P + 1];
}

// Step 4 (ii): quadratic model, initial t, first retraction coefficients
__global__ void k_c_step(Ctl* c, const double* s) {
  const double hv = c->hv;
  c->Hpp = hv * s[S_C]; c->S1 = hv * s[S_C + 1]; c->S2 = hv * s[S_C + 2]; c->S3 = hv * s[S_C + 3];
  c->curv = c->Hpp + 2.0 * c->S1 - c->mu * c->pn2;
  c->t = c->curv > 0.0 ? -c->d1 / c->curv : 0.3;
  c->t0 = c->t;
  c->pn = sqrt(c->pn2);
  c->Aphiphi = c->kin + c->rot + c->pot;
  c->Aphip = c->d1 - c->S2;
  c->App = c->Hpp - c->S3;
  c->tolE = c->tolE_eps * fabs(c->E);
  c->nh = 0;
  c->forced = 0;
  c->bestE = INFINITY;
  c->best_t = c->t;
  c->cr = cos(c->t * c->pn);
  c->sr = sin(c->t * c->pn) / c->pn;
}

__global__ void k_c_norm(Ctl* c, const double* s) {
  c->nrm2 = c->hv * s[S_T];
  c->inv = 1.0 / sqrt(c->nrm2);
}

// Step 4 (iii): trial energy and the acceptance test
__global__ void k_c_accept(Ctl* c, const double* s) {
  const double quad = (c->cr * c->cr * c->Aphiphi + 2.0 * c->cr * c->sr * c->Aphip + c->sr * c->sr * c->App) / c->nrm2;
  c->En = quad + 0.5 * c->beta * c->hv * s[S_Q] + 0.5 * c->lam * c->hv * s[S_Q + 1];
  c->linf = s[S_L];
  c->accepted = fin(c->En) && (c->En <= c->E + c->tolE);
  if (!c->accepted && c->En < c->bestE) {
    c->bestE = c->En;
    c->best_t = c->t;
  }
}

// Next trial: halve t, or (mode 1) take the lowest-energy trial seen.
__device__ __forceinline__ void halve_body(Ctl* c, int mode) {
  if (mode == 0) {
    c->t *= 0.5;
    c->nh += 1;
  } else {
    c->t = c->best_t;
    c->forced = 1;
  }
  c->cr = cos(c->t * c->pn);
  c->sr = sin(c->t * c->pn) / c->pn;
}
__global__ void k_c_halve(Ctl* c, int mode) { halve_body(c, mode); }
// The same with the mode taken on the device: halve while halvings remain.
__global__ void k_c_halve_auto(Ctl* c) { halve_body(c, c->nh < c->max_halv ? 0 : 1); }

// End of an iteration: the trial becomes phi_{n+1}.
__global__ void k_c_end(Ctl* c) {
  c->den_prev = c->den;
  c->have_prev = 1;
  c->E = c->En;
  c->force_sd = c->forced;
}

// Host-driven state changes (precision hand-over, start of a solve).
__global__ void k_c_reset_state(Ctl* c, int have_E, int force_sd, int clear_prev) {
  c->have_E = have_E;
  c->force_sd = force_sd;
  if (clear_prev) c->have_prev = 0;
}

// ---------------------------------------------------- device-driven loop
// The iteration loop as a CUDA graph with conditional nodes: the control
// kernels below take, between iterations, exactly the decisions that
// Solver::process takes on the host (stop rule, precision hand-over,
// halving, stagnation, log), and set the graph's condition handles.  Every
// loop is also bounded by a guard counter derived from max_iter and
// max_halvings, so a graph launch always ends.
// FP32 phase stagnation: no halving of the best FP32 residual for this many
// iterations (opts.f32_window, this when 0) hands over to FP64.  A long window
// wastes FP32 iterations at the FP32 residual floor (400 cost the finest level
// of a 256^3 multigrid solve 350 of them); 50 keeps the long bulk phases of
// fast-rotating states within about 10% of their time.
constexpr int kF32Window = 50;
// Automatic hand-over (switch_tol < 0): the FP32 phase ends once its residual
// is within kNoiseFactor of the FP32 noise measured at phi_0 (or at
// |switch_tol|, whichever is larger), where its progress would stop; the floor
// being detected that way, the stagnation window is only a backstop, long
// enough not to end the slow, non-monotone progress of vortex-lattice states
// (their residual can stay above its best for several hundred iterations).
constexpr double kNoiseFactor = 4.0;
constexpr int kF32WindowAuto = 2000;

struct LoopInit {
  int n, max_iter, max_halv, caps, f32, log_cap, q, f32_window;
  double tol_res, tol_linf, switch_tol, linf, time_limit_s, f32_gain;
  atkm_iter_log* log;
  unsigned long long guard_max;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_d_setup(Ctl* c, LoopInit L) {
  c->n = c->n_start = L.n;
  c->max_iter = L.max_iter;
  c->max_halv = L.max_halv;
  c->caps = L.caps;
  c->status = ATKM_NOT_CONVERGED;
  c->done = c->handover = c->final_top = c->step_logged = 0;
  c->logc = 0;
  c->log_cap = L.log_cap;
  c->log = L.log;
  c->f32 = L.f32;
  c->f32_iters = c->total_h = 0;
  c->f32_best_n = L.n;
  c->f32_best = INFINITY;
  c->q = L.q;
  c->f32_window = L.f32_window;
  c->f32_gain = L.f32_gain;
  c->tol_res = L.tol_res;
  c->tol_linf = L.tol_linf;
  c->switch_tol = L.switch_tol;
  c->linf_n = L.linf;
  c->deadline = L.time_limit_s > 0.0 ? global_ns() + (unsigned long long)(L.time_limit_s * 1e9) : 0ull;
  c->guard = 0;
  c->guard_max = L.guard_max;
  c->launches = 1;
}

// After Step 2 (loop top): log entry, stop rule, hand-over test.
__global__ void k_d_check(Ctl* c, cudaGraphConditionalHandle h_rest, int nodes) {
  c->launches += nodes;
  if (c->final_top) {  // the residual of the final state after a stagnated run
    c->final_top = 0;
    c->done = 1;
    cudaGraphSetConditional(h_rest, 0);
    return;
  }
  c->step_logged = 0;
  if (c->log && c->logc < c->log_cap) {
    atkm_iter_log* L = &c->log[c->logc++];
    *L = atkm_iter_log{};
    L->n = c->n; L->E = c->E; L->mu = c->mu; L->residual = c->res; L->linf_step = c->linf_n; L->f32_phase = c->f32;
    c->step_logged = 1;
  }
  if (c->nan) {
    c->status = ATKM_ERR_NAN;
    c->done = 1;
  } else {
    if (c->f32 && c->res < c->f32_gain * c->f32_best) {
      c->f32_best = c->res;
      c->f32_best_n = c->n;
    }
    if (c->f32 && (c->res <= c->switch_tol || c->caps >= 2 || c->n - c->f32_best_n > c->f32_window)) {
      c->handover = 1;  // ends this phase; the entry is re-made by the FP64 phase
      c->done = 1;
      if (c->step_logged) {
        c->logc -= 1;
        c->step_logged = 0;
      }
    } else if (!c->f32 && (c->res <= c->tol_res || (c->tol_linf > 0.0 && c->linf_n <= c->tol_linf))) {
      c->status = ATKM_OK;
      c->done = 1;
    } else if (c->n - c->n_start >= c->max_iter) {
      c->status = ATKM_NOT_CONVERGED;
      c->done = 1;
    } else if (c->deadline && global_ns() >= c->deadline) {
      c->status = ATKM_ERR_TIMEOUT;
      c->done = 1;
    } else if (c->f32) {
      c->f32_iters += 1;
    }
  }
  cudaGraphSetConditional(h_rest, !c->done);
}

// After each trial of Step 4 (iii): another halving (or the forced trial)?
__global__ void k_d_after_trial(Ctl* c, cudaGraphConditionalHandle h_halve, int nodes) {
  c->launches += nodes;
  int more;
  if (c->forced) {
    more = 0;
  } else if (!fin(c->En)) {
    c->status = ATKM_ERR_NAN;
    c->done = 1;
    more = 0;
  } else {
    more = !c->accepted;
  }
  if (more && ++c->guard > c->guard_max) {
    c->status = ATKM_ERR_TIMEOUT;
    c->done = 1;
    more = 0;
  }
  cudaGraphSetConditional(h_halve, more);
}

// End of an iteration: the trial becomes phi_{n+1} (k_c_end), bookkeeping.
__global__ void k_d_end(Ctl* c, int nodes) {
  c->launches += nodes;
  if (c->done) return;
  const int acc = c->accepted && !c->forced;
  c->total_h += c->nh;
  c->caps = acc ? 0 : c->caps + 1;
  if (c->step_logged) {
    atkm_iter_log* L = &c->log[c->logc - 1];
    L->alpha = c->alpha; L->beta_cg = c->beta_cg; L->reset_to_sd = c->reset; L->d1 = c->d1; L->curvature = c->curv;
    L->t0 = c->t0; L->t = c->t; L->halvings = c->nh; L->accepted = acc;
  }
  c->linf_n = c->linf;
  c->den_prev = c->den;
  c->have_prev = 1;
  c->E = c->En;
  c->force_sd = c->forced;
  c->q ^= 1;
  c->n += 1;
  if (c->caps >= 3 && !c->f32) {
    c->status = ATKM_STAGNATED;
    c->done = 1;
    c->final_top = 1;
  }
}

// Between the two iterations of a loop body: run the second one?
__global__ void k_d_gate(Ctl* c, cudaGraphConditionalHandle h_go1, int nodes) {
  c->launches += nodes;
  cudaGraphSetConditional(h_go1, !c->done || c->final_top);
}

// End of a loop body (two iterations): run again?
__global__ void k_d_loop(Ctl* c, cudaGraphConditionalHandle h_run, cudaGraphConditionalHandle h_go0, int nodes) {
  c->launches += nodes;
  int run = !c->done || c->final_top;
  if (run && ++c->guard > c->guard_max) {
    c->status = ATKM_ERR_TIMEOUT;
    c->done = 1;
    c->final_top = 0;
    run = 0;
  }
  cudaGraphSetConditional(h_run, run);
  cudaGraphSetConditional(h_go0, run);
}

// After the FP32 loop: hand over at the parity where it stopped.
__global__ void k_d_phase(Ctl* c, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1, int nodes) {
  c->launches += nodes;
  const int ho = c->handover;
  cudaGraphSetConditional(h0, ho && c->q == 0);
  cudaGraphSetConditional(h1, ho && c->q == 1);
}

// The hand-over's state change (after the FP64 ATKM of phi): FP64 from here.
__global__ void k_d_handover(Ctl* c, double tolE_eps, int nodes) {
  c->launches += nodes;
  c->f32 = 0;
  c->caps = 0;
  c->handover = 0;
  c->done = 0;
  c->have_E = 0;
  c->force_sd = 1;
  c->tolE_eps = tolE_eps;
}

}  // namespace

cudaError_t launch_finalize(atkm_plan* p, int nslots, int nblocks, int dst_slot, cudaStream_t st) {
  k_finalize<<<nslots, kRedThreads, 0, st>>>(p->partials, nblocks, p->scal + dst_slot, nullptr);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------- PCG state
struct PcgBuffers {
  size_t N = 0;
  double2* phi[2] = {nullptr, nullptr};  // ping-pong: phi_n / trial phi+
  double2* r[2] = {nullptr, nullptr};    // r_n / r_{n-1}
  double2* p[2] = {nullptr, nullptr};    // p_n / p_{n-1}
  double* Phi[2] = {nullptr, nullptr};   // Phi_n / trial Phi+
  double2 *Hphi = nullptr, *Pr = nullptr, *Hp = nullptr;
  double* Phi1 = nullptr;
  Ctl* ctl = nullptr;        // device
  Ctl* ctl_h = nullptr;      // pinned host mirror
  cudaStream_t st = nullptr; // plan-owned stream (capturable)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // graphs: [f32][parity][kind: 0 iteration, 1 halve+trial, 2 best+trial]
  // captured graphs per [form: FP64, FP32, FP64 with FP32 auxiliaries][parity][kind]
  cudaGraphExec_t gx[4][2][3] = {};
  int gnodes[4][2][3] = {};
  bool seen[4][2][3] = {};
  bool gprof[4][2][3] = {};                 // captured with profiling events
  std::vector<ProfRec> grecs[4][2][3];      // those events
  const std::vector<ProfRec>* last = nullptr;  // records of the last replay
  bool graphs_ok = true;
  Phys gphys{};
  bool gphys_set = false;
  // resume state (host side)
  bool valid = false, f32 = false;
  int parity = 0, n = 0, caps = 0;
  double linf = INFINITY, sw_eff = 0.0;
  // device-driven solve graphs per [polish form][starts in FP32][start parity]
  cudaGraph_t dg[4][2][2] = {};
  cudaGraphExec_t dx[4][2][2] = {};
  bool dl_ok = true;             // false once building or launching one failed
  atkm_iter_log* dlog = nullptr; // device log of the device-driven loop
  int dlog_cap = 0;
};

static void drop_graph(PcgBuffers* b, int f, int q, int k) {
  if (b->gx[f][q][k]) { cudaGraphExecDestroy(b->gx[f][q][k]); b->gx[f][q][k] = nullptr; }
  for (auto& r : b->grecs[f][q][k]) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  b->grecs[f][q][k].clear();
  b->seen[f][q][k] = false;
  b->gnodes[f][q][k] = 0;
  b->gprof[f][q][k] = false;
}

static void destroy_graphs(PcgBuffers* b) {
  for (int f = 0; f < 4; ++f)
    for (int q = 0; q < 2; ++q)
      for (int k = 0; k < 3; ++k) drop_graph(b, f, q, k);
  for (int f = 0; f < 4; ++f)
    for (int a = 0; a < 2; ++a)
      for (int q = 0; q < 2; ++q) {
        if (b->dx[f][a][q]) cudaGraphExecDestroy(b->dx[f][a][q]);
        if (b->dg[f][a][q]) cudaGraphDestroy(b->dg[f][a][q]);
        b->dx[f][a][q] = nullptr;
        b->dg[f][a][q] = nullptr;
      }
  b->last = nullptr;
}

void pcg_free(atkm_plan* p) {
  if (!p->pcg) return;
  PcgBuffers* b = p->pcg;
  destroy_graphs(b);
  void* ptrs[] = {b->phi[0], b->phi[1], b->r[0], b->r[1], b->p[0], b->p[1], b->Phi[0], b->Phi[1],
                  b->Hphi, b->Pr, b->Hp, b->Phi1, b->ctl, b->dlog};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->ctl_h) cudaFreeHost(b->ctl_h);
  if (b->st) cudaStreamDestroy(b->st);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  delete b;
  p->pcg = nullptr;
}

static cudaError_t pcg_alloc(atkm_plan* p) {
  if (p->pcg) return cudaSuccess;
  PcgBuffers* b = new PcgBuffers();
  p->pcg = b;
  const size_t N = (size_t)p->g.Nx * p->g.Ny * p->g.Nz;
  b->N = N;
  double2** cv[] = {&b->phi[0], &b->phi[1], &b->r[0], &b->r[1], &b->p[0], &b->p[1], &b->Hphi, &b->Pr, &b->Hp};
  cudaError_t e = cudaSuccess;
  for (double2** q : cv)
    if (e == cudaSuccess) e = dev_alloc(p, (void**)q, N * sizeof(double2));
  double** rv[] = {&b->Phi[0], &b->Phi[1], &b->Phi1};
  for (double** q : rv)
    if (e == cudaSuccess) e = dev_alloc(p, (void**)q, N * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc(p, (void**)&b->ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->ctl_h, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  // previous-iteration vectors are read (and ignored) before the first step
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMemset(b->r[i], 0, N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemset(b->p[i], 0, N * sizeof(double2));
  }
  if (e == cudaSuccess) e = cudaMemset(b->ctl, 0, sizeof(Ctl));
  if (e != cudaSuccess) pcg_free(p);
  return e;
}

// Enqueues the kernels of one PCG phase on the plan stream.
struct Seq {
  atkm_plan* p;
  PcgBuffers& B;
  Phys ph;
  bool f32;
  int q;  // buffer parity: phi = B.phi[q], trial into B.phi[q ^ 1]
  cudaError_t err = cudaSuccess;
  // FP64 phase of the split form: the operators that only shape the search
  // direction and the step-size model (P r, H p, the pair ATKM) run in FP32.
  bool aux32 = false;
  // Double-word form of that phase: H phi and the trial-energy ATKM run in
  // double-FP32 arithmetic instead of binary64.
  bool dw = false;
  Ctl* c() const { return B.ctl; }
  const double* s() const { return p->scal; }
  cudaStream_t st() const { return B.st; }
  void chk(cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; }

  void dot(const double2* u, const double2* v, int dst) {
    prof_begin(p, "vec_dots", 32.0 * B.N, 0.0, st());
    const int g = wave_grid((const void*)k_dot, B.N);
    k_dot<<<g, kRedThreads, 0, st()>>>(u, v, B.N, p->partials);
    prof_end(p, st());
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, 1, g, dst, st()));
  }
  // FP64 arithmetic unless this is the FP32 phase and `phase_type` allows it.
  void lincomb(double2* out, const double2* v0, Coef c0, const double2* v1, Coef c1, const double2* v2, Coef c2,
               const double2* w, int dst, const int* pred = nullptr, bool phase_type = true) {
    const double nv = (v0 ? 1 : 0) + (v1 ? 1 : 0) + (v2 ? 1 : 0) + (w ? 1 : 0) + 1;
    prof_begin(p, "vec_lincomb", 16.0 * nv * B.N, 0.0, st());
    const bool fl = f32 && phase_type;
    const int g = fl ? wave_grid((const void*)k_lincomb<float>, B.N) : wave_grid((const void*)k_lincomb<double>, B.N);
    if (fl)
      k_lincomb<float><<<g, kRedThreads, 0, st()>>>(out, v0, c0, v1, c1, v2, c2, w, B.N, p->partials, pred);
    else
      k_lincomb<double><<<g, kRedThreads, 0, st()>>>(out, v0, c0, v1, c1, v2, c2, w, B.N, p->partials, pred);
    prof_end(p, st());
    k_finalize<<<2, kRedThreads, 0, st()>>>(p->partials, g, p->scal + dst, pred);
    count_launches(2);
    chk(cudaGetLastError());
  }
  void atkm(int mode, const double* a, const double* b, double* o, bool aux = false) {
    const bool use32 = f32 || (aux && aux32);
    chk(use32 ? launch_atkm<float>(p, mode, a, b, o, st())
              : dw ? launch_atkm<df>(p, mode, a, b, o, st()) : launch_atkm<double>(p, mode, a, b, o, st()));
  }
  void hop(const double2* f, double2* o, int red, bool aux = false) {
    const double* fp = reinterpret_cast<const double*>(f);
    const double* pp = reinterpret_cast<const double*>(B.phi[q]);
    double* op = reinterpret_cast<double*>(o);
    const bool use32 = f32 || (aux && aux32);
    chk(use32 ? launch_H<float>(p, ph, fp, pp, B.Phi[q], op, red, st())
              : dw ? launch_H<df>(p, ph, fp, pp, B.Phi[q], op, red, st())
                   : launch_H<double>(p, ph, fp, pp, B.Phi[q], op, red, st()));
  }
  template <typename K, typename... A> void ctl1(K kernel, A... args) {
    kernel<<<1, 1, 0, st()>>>(args...);
    count_launches(1);
    chk(cudaGetLastError());
  }

  // Step 2 only (loop top): H phi, parts, r, ||r||.
  void top() {
    hop(B.phi[q], B.Hphi, S_H);
    ctl1(k_c_parts, c(), s());
    lincomb(B.r[q], B.Hphi, Coef{nullptr, 1.0}, B.phi[q], Coef{&c()->mu, -1.0}, nullptr, Coef{nullptr, 0.0}, nullptr,
            S_R);
    ctl1(k_c_res, c(), s());
  }
  // One trial of Step 4 (iii) with the current retraction coefficients.
  void trial() {
    double2* phin = B.phi[q ^ 1];
    lincomb(phin, B.phi[q], Coef{&c()->cr, 1.0}, B.p[q], Coef{&c()->sr, 1.0}, nullptr, Coef{nullptr, 0.0}, nullptr,
            S_T, nullptr, false);  // the retraction stays FP64
    ctl1(k_c_norm, c(), s());
    prof_begin(p, "vec_scale_linf", 48.0 * B.N, 0.0, st());
    const int gs = f32 ? wave_grid((const void*)k_scale_linf<float>, B.N)
                       : wave_grid((const void*)k_scale_linf<double>, B.N);
    if (f32) k_scale_linf<float><<<gs, kRedThreads, 0, st()>>>(phin, B.phi[q], &c()->inv, B.N, p->partials);
    else k_scale_linf<double><<<gs, kRedThreads, 0, st()>>>(phin, B.phi[q], &c()->inv, B.N, p->partials);
    prof_end(p, st());
    k_finalize_max<<<1, kRedThreads, 0, st()>>>(p->partials, gs, p->scal + S_L);
    count_launches(2);
    chk(cudaGetLastError());
    atkm(SRC_PSI, reinterpret_cast<const double*>(phin), nullptr, B.Phi[q ^ 1]);
    prof_begin(p, "vec_quartic", 24.0 * B.N, 0.0, st());
    const int gq = f32 ? wave_grid((const void*)k_quartic_sums<float>, B.N)
                       : wave_grid((const void*)k_quartic_sums<double>, B.N);
    if (f32) k_quartic_sums<float><<<gq, kRedThreads, 0, st()>>>(phin, B.Phi[q ^ 1], B.N, p->partials);
    else k_quartic_sums<double><<<gq, kRedThreads, 0, st()>>>(phin, B.Phi[q ^ 1], B.N, p->partials);
    prof_end(p, st());
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, 2, gq, S_Q, st()));
    ctl1(k_c_accept, c(), s());
  }
  cudaError_t precond() {
    const double* r = reinterpret_cast<const double*>(B.r[q]);
    const double* phi = reinterpret_cast<const double*>(B.phi[q]);
    double* Pr = reinterpret_cast<double*>(B.Pr);
    return (f32 || aux32) ? launch_precond<float>(p, ph, &c()->alpha, r, phi, B.Phi[q], Pr, st())
                          : launch_precond<double>(p, ph, &c()->alpha, r, phi, B.Phi[q], Pr, st());
  }
  // A whole iteration: Steps 2-4 up to the first trial.
  void iteration() {
    top();
    rest();
  }
  // Steps 3-4 up to the first trial (after top()).
  void rest() {
    chk(precond());
    prof_begin(p, "vec_dir_dots", 80.0 * B.N, 0.0, st());
    const int gd = f32 ? wave_grid((const void*)k_dir_dots<float>, B.N)
                       : wave_grid((const void*)k_dir_dots<double>, B.N);
    if (f32)
      k_dir_dots<float><<<gd, kRedThreads, 0, st()>>>(B.Pr, B.phi[q], B.r[q], B.r[q ^ 1], B.p[q ^ 1], B.N,
                                                      p->partials);
    else
      k_dir_dots<double><<<gd, kRedThreads, 0, st()>>>(B.Pr, B.phi[q], B.r[q], B.r[q ^ 1], B.p[q ^ 1], B.N,
                                                       p->partials);
    prof_end(p, st());
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, 7, gd, S_D, st()));
    ctl1(k_c_dir, c(), s());
    lincomb(B.p[q], B.Pr, Coef{&c()->cp0, 1.0}, B.p[q ^ 1], Coef{&c()->cp1, 1.0}, B.phi[q], Coef{&c()->cp2, 1.0},
            B.Hphi, S_P);
    ctl1(k_c_reset, c(), s());
    lincomb(B.p[q], B.Pr, Coef{nullptr, -1.0}, B.phi[q], Coef{&c()->b, 1.0}, nullptr, Coef{nullptr, 0.0}, B.Hphi, S_P,
            &c()->redo);
    ctl1(k_c_reset2, c(), s());
    hop(B.p[q], B.Hp, -1, true);
    atkm(SRC_PAIR, reinterpret_cast<const double*>(B.phi[q]), reinterpret_cast<const double*>(B.p[q]), B.Phi1, true);
    prof_begin(p, "vec_curv_sums", 64.0 * B.N, 0.0, st());
    const int gc = f32 ? wave_grid((const void*)k_curv_sums<float>, B.N)
                       : wave_grid((const void*)k_curv_sums<double>, B.N);
    if (f32)
      k_curv_sums<float><<<gc, kRedThreads, 0, st()>>>(B.Hp, B.phi[q], B.p[q], B.Phi[q], B.Phi1, ph.beta, ph.lambda,
                                                       B.N, p->partials);
    else
      k_curv_sums<double><<<gc, kRedThreads, 0, st()>>>(B.Hp, B.phi[q], B.p[q], B.Phi[q], B.Phi1, ph.beta,
                                                        ph.lambda, B.N, p->partials);
    prof_end(p, st());
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, 4, gc, S_C, st()));
    ctl1(k_c_step, c(), s());
    trial();
  }
  void run(int kind) {
    if (kind == 0) {
      iteration();
    } else {
      ctl1(k_c_halve, c(), kind == 1 ? 0 : 1);
      trial();
    }
  }
};

// Runs a phase through its CUDA graph (captured on the second use) or eagerly.
// With profiling on, the graph carries event-record nodes around each pass;
// B.last then points at them so the caller can accumulate their times after
// the replay has completed.
static cudaError_t run_phase(Seq& S, int kind, bool use_graphs) {
  PcgBuffers& B = S.B;
  atkm_plan* p = S.p;
  const int fi = S.f32 ? 1 : (S.aux32 ? (S.dw ? 3 : 2) : 0);
  const bool prof = p->prof != nullptr;
  B.last = nullptr;
  if (!use_graphs || !B.graphs_ok) {
    S.run(kind);
    return S.err;
  }
  if (B.gx[fi][S.q][kind] && B.gprof[fi][S.q][kind] != prof) drop_graph(&B, fi, S.q, kind);
  cudaGraphExec_t& gx = B.gx[fi][S.q][kind];
  if (gx) {
    count_launches(B.gnodes[fi][S.q][kind]);
    if (prof) B.last = &B.grecs[fi][S.q][kind];
    return cudaGraphLaunch(gx, B.st);
  }
  if (!B.seen[fi][S.q][kind]) {  // first use: run eagerly (prepares kernel attributes)
    B.seen[fi][S.q][kind] = true;
    S.run(kind);
    return S.err;
  }
  const unsigned long long c0 = atkm_launch_count();
  if (cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    B.graphs_ok = false;
    S.run(kind);
    return S.err;
  }
  if (prof) prof_set_sink(p, &B.grecs[fi][S.q][kind]);
  S.run(kind);
  if (prof) prof_set_sink(p, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(B.st, &g);
  const int nodes = (int)(atkm_launch_count() - c0);
  count_launches(-nodes);  // recorded into the graph, not executed
  if (S.err != cudaSuccess || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    drop_graph(&B, fi, S.q, kind);
    B.graphs_ok = false;
    S.err = cudaSuccess;
    S.run(kind);
    return S.err;
  }
  const cudaError_t e = cudaGraphInstantiate(&gx, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    gx = nullptr;
    cudaGetLastError();
    drop_graph(&B, fi, S.q, kind);
    B.graphs_ok = false;
    S.run(kind);
    return S.err;
  }
  B.gnodes[fi][S.q][kind] = nodes;
  B.gprof[fi][S.q][kind] = prof;
  count_launches(nodes);
  if (prof) B.last = &B.grecs[fi][S.q][kind];
  return cudaGraphLaunch(gx, B.st);
}

// ------------------------------------------------------------- solve graph
// Builds the device-driven solve of one instance into a graph (a chain with
// no incoming dependency, so several instances can share one graph):
//   start in FP32: Loop(F32, q0); k_d_phase; IF(ho0) { hand-over at 0;
//     Loop(polish, 0) }; IF(ho1) { hand-over at 1; Loop(polish, 1) }
//   otherwise:     Loop(polish, q0)
// Loop(q) = WHILE(run) { IF(go0) { Iter(q) }; k_d_gate; IF(go1) { Iter(q ^ 1) }; k_d_loop }
// Iter(q) = top; k_d_check; IF(rest) { rest; k_d_after_trial;
//           WHILE(halve) { k_c_halve_auto; trial; k_d_after_trial }; k_d_end }
// The kernels are those of Seq, captured on the plan stream; the condition
// handles belong to the graph the chain is built into, and each is set only
// by kernels of the graph that holds its node (or, for a WHILE node, of its
// body).
struct GraphBuild {
  PcgBuffers& B;
  cudaGraph_t top;
  cudaError_t err = cudaSuccess;

  void chk(cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  }
  cudaGraphConditionalHandle handle(unsigned def) {
    cudaGraphConditionalHandle h = 0;
    if (err == cudaSuccess) chk(cudaGraphConditionalHandleCreate(&h, top, def, cudaGraphCondAssignDefault));
    return h;
  }
  // A conditional node in g after *dep (none when null); *dep becomes the
  // node; returns its body graph.
  cudaGraph_t cond(cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                   cudaGraphConditionalNodeType type) {
    if (err != cudaSuccess) return nullptr;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    chk(cudaGraphAddNode(&node, g, *dep ? dep : nullptr, nullptr, *dep ? 1 : 0, &np));
    if (err != cudaSuccess) return nullptr;
    *dep = node;
    return np.conditional.phGraph_out[0];
  }
  // Captures fn() on the plan stream into g after *dep; *dep becomes the last
  // captured node.  fn gets the number of kernels it has launched so far.
  template <class F> void capture(cudaGraph_t g, cudaGraphNode_t* dep, F fn) {
    if (err != cudaSuccess) return;
    // relaxed: the launchers may set kernel attributes or query occupancy on
    // first use, which the stricter capture modes refuse
    chk(cudaStreamBeginCaptureToGraph(B.st, g, *dep ? dep : nullptr, nullptr, *dep ? 1 : 0,
                                      cudaStreamCaptureModeRelaxed));
    if (err != cudaSuccess) return;
    const unsigned long long c0 = atkm_launch_count();
    fn([c0]() { return (int)(atkm_launch_count() - c0); });
    const int k = (int)(atkm_launch_count() - c0);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    chk(cudaStreamGetCaptureInfo(B.st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
    const cudaGraphNode_t last = (err == cudaSuccess && nd == 1) ? deps[0] : nullptr;
    cudaGraph_t out = nullptr;
    chk(cudaStreamEndCapture(B.st, &out));
    count_launches(-k);  // recorded into the graph, not executed
    if (!last) chk(cudaErrorInvalidValue);  // a segment ends in exactly one node
    *dep = last;
  }

  void iteration(cudaGraph_t g, Seq& S) {
    cudaGraphConditionalHandle h_rest = handle(0), h_halve = handle(0);
    Ctl* c = B.ctl;
    cudaGraphNode_t d = nullptr;
    capture(g, &d, [&](auto sofar) {
      S.top();
      S.ctl1(k_d_check, c, h_rest, sofar() + 1);
    });
    cudaGraph_t rb = cond(g, &d, h_rest, cudaGraphCondTypeIf);
    if (err != cudaSuccess) return;
    cudaGraphNode_t r = nullptr;
    capture(rb, &r, [&](auto sofar) {
      S.rest();
      S.ctl1(k_d_after_trial, c, h_halve, sofar() + 1);
    });
    cudaGraph_t hb = cond(rb, &r, h_halve, cudaGraphCondTypeWhile);
    if (err != cudaSuccess) return;
    cudaGraphNode_t h = nullptr;
    capture(hb, &h, [&](auto sofar) {
      S.ctl1(k_c_halve_auto, c);
      S.trial();
      S.ctl1(k_d_after_trial, c, h_halve, sofar() + 1);
    });
    capture(rb, &r, [&](auto) { S.ctl1(k_d_end, c, 1); });
  }

  void loop(cudaGraph_t g, cudaGraphNode_t* dep, Seq& S0, Seq& S1) {
    cudaGraphConditionalHandle h_run = handle(1), h_go0 = handle(1), h_go1 = handle(0);
    cudaGraph_t body = cond(g, dep, h_run, cudaGraphCondTypeWhile);
    if (err != cudaSuccess) return;
    cudaGraphNode_t d = nullptr;
    cudaGraph_t b0 = cond(body, &d, h_go0, cudaGraphCondTypeIf);
    if (err == cudaSuccess) iteration(b0, S0);
    capture(body, &d, [&](auto) { S0.ctl1(k_d_gate, B.ctl, h_go1, 1); });
    cudaGraph_t b1 = cond(body, &d, h_go1, cudaGraphCondTypeIf);
    if (err == cudaSuccess) iteration(b1, S1);
    capture(body, &d, [&](auto) { S0.ctl1(k_d_loop, B.ctl, h_run, h_go0, 1); });
  }

  // The whole chain of one instance; f32s[q] / pol[q]: the kernel sequences
  // of the FP32 phase and of the polish at parity q.
  void solve(bool start_f32, int q0, Seq* f32s, Seq* pol, double tolE_eps_polish, const LoopInit* init) {
    cudaGraphNode_t d = nullptr;
    if (init) capture(top, &d, [&](auto) { pol[0].ctl1(k_d_setup, B.ctl, *init); });
    if (!start_f32) {
      loop(top, &d, pol[q0], pol[q0 ^ 1]);
      return;
    }
    loop(top, &d, f32s[q0], f32s[q0 ^ 1]);
    cudaGraphConditionalHandle h_ho[2] = {handle(0), handle(0)};
    capture(top, &d, [&](auto) { pol[0].ctl1(k_d_phase, B.ctl, h_ho[0], h_ho[1], 1); });
    for (int qq = 0; qq < 2 && err == cudaSuccess; ++qq) {
      cudaGraph_t hb = cond(top, &d, h_ho[qq], cudaGraphCondTypeIf);
      if (err != cudaSuccess) return;
      cudaGraphNode_t x = nullptr;
      capture(hb, &x, [&](auto sofar) {
        pol[qq].atkm(SRC_PSI, reinterpret_cast<const double*>(B.phi[qq]), nullptr, B.Phi[qq]);
        pol[qq].ctl1(k_d_handover, B.ctl, tolE_eps_polish, sofar() + 1);
      });
      loop(hb, &x, pol[qq], pol[qq ^ 1]);
    }
  }
};

// One PCG solve as a host-side state machine: launch() enqueues the next
// phase (graph or direct launches) and an asynchronous read of the control
// block on the plan stream; wait() synchronises that stream; process() takes
// the decisions of the stop rule, the halving loop and the log.  Several
// solvers on different plans run concurrently (pcg_ground_state_batched).
// With graphs on and profiling off, run_device() replaces that loop by one
// launch of the device-driven solve graph (same kernels, same decisions).

struct Solver {
  enum State { INIT_CHECK, MAIN, HALVE, FORCED, FINAL, DONE };
  atkm_plan* plan = nullptr;
  const atkm_params* prm = nullptr;
  const atkm_pcg_opts* opts = nullptr;
  double* psi = nullptr;
  atkm_result* out = nullptr;
  atkm_iter_log* logbuf = nullptr;
  PcgBuffers* B = nullptr;
  cudaStream_t caller = nullptr;
  Phys ph{};
  bool mixed = false, split = false, dwm = false, use_graphs = true, f32 = false, began = false;
  int q = 0, n = 0, n_start = 0, caps = 0, status = ATKM_NOT_CONVERGED, total_h = 0, f32_iters = 0, logc = 0;
  int f32_best_n = 0, early_code = ATKM_OK;
  double linf = INFINITY, f32_best = INFINITY;
  State st = DONE;
  atkm_iter_log* L = nullptr;
  cudaError_t err = cudaSuccess;
  const double eps64 = 2.220446049250313e-16, eps32 = 1.1920928955078125e-07;
  const double epsdw = 1.4210854715202004e-14;  // 2^-46: double-word operators
  double eps_polish() const { return dwm ? epsdw : eps64; }
  std::chrono::steady_clock::time_point t_start;
  bool ran_device = false;
  bool sw_auto = false;  // hand-over at the measured FP32 noise (switch_tol < 0)
  double sw_eff = 0.0;   // the residual at which the FP32 phase hands over

  void chk(cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; }
  double elapsed_s() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  bool past_time_limit() const { return opts->time_limit_s > 0.0 && elapsed_s() >= opts->time_limit_s; }

  // ---- device-driven run (graphs on, profiling off)
  int fi_polish() const { return (split || dwm) ? (dwm ? 3 : 2) : 0; }
  int f32_window() const {
    return opts->f32_window > 0 ? opts->f32_window : (sw_auto ? kF32WindowAuto : kF32Window);
  }
  double f32_gain() const { return opts->f32_gain > 0.0 && opts->f32_gain < 1.0 ? opts->f32_gain : 0.5; }
  bool device_loop_ok() const { return use_graphs && B->graphs_ok && B->dl_ok && plan->prof == nullptr; }
  Seq seq_q(bool is32, int qq) {
    Seq S{plan, *B, ph, is32, qq};
    S.aux32 = (split || dwm) && !is32;
    S.dw = dwm && !is32;
    return S;
  }
  int log_room() const { return (logbuf && opts->log_capacity > logc) ? opts->log_capacity - logc : 0; }
  cudaError_t ensure_dlog() {
    const int need = log_room();
    if (need <= B->dlog_cap) return cudaSuccess;
    if (B->dlog) cudaFree(B->dlog);
    B->dlog = nullptr;
    B->dlog_cap = 0;
    cudaError_t e = cudaMalloc((void**)&B->dlog, (size_t)need * sizeof(atkm_iter_log));
    if (e == cudaSuccess) B->dlog_cap = need;
    return e;
  }
  LoopInit loop_init() const {
    LoopInit I{};
    I.n = n;
    I.max_iter = opts->max_iter;
    I.max_halv = opts->max_halvings;
    I.caps = caps;
    I.f32 = f32 ? 1 : 0;
    I.log_cap = log_room();
    I.q = q;
    I.f32_window = f32_window();
    I.f32_gain = f32_gain();
    I.tol_res = opts->tol_residual;
    I.tol_linf = opts->tol_linf;
    I.switch_tol = sw_eff;
    I.linf = linf;
    I.time_limit_s = opts->time_limit_s > 0.0 ? std::max(opts->time_limit_s - elapsed_s(), 1e-9) : 0.0;
    I.log = B->dlog;
    // loop bodies of both phases and halving rounds of every iteration
    const unsigned long long mi = (unsigned long long)opts->max_iter, mh = (unsigned long long)opts->max_halvings;
    I.guard_max = 2ull * (mi / 2ull + 3ull) + (mi + 2ull) * (mh + 2ull) + 64ull;
    return I;
  }
  // Builds this solver's chain into graph g (init: the setup kernel's
  // parameters, captured too; null when the caller launches it).
  cudaError_t build_chain(cudaGraph_t g, const LoopInit* init) {
    GraphBuild GB{*B, g};
    Seq F[2] = {seq_q(true, 0), seq_q(true, 1)};
    Seq P[2] = {seq_q(false, 0), seq_q(false, 1)};
    GB.solve(f32, q, F, P, 32.0 * eps_polish(), init);
    for (auto& x : F) GB.chk(x.err);
    for (auto& x : P) GB.chk(x.err);
    return GB.err;
  }
  // The cached solve graph for this solver's state, built on first use.
  cudaGraphExec_t solve_graph() {
    const int fp = fi_polish(), a = f32 ? 1 : 0;
    cudaGraphExec_t& gx = B->dx[fp][a][q];
    if (gx) return gx;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = build_chain(g, nullptr);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ex) cudaGraphExecDestroy(ex);
      if (g) cudaGraphDestroy(g);
      B->dl_ok = false;  // the host-driven loop takes over
      return nullptr;
    }
    B->dg[fp][a][q] = g;
    gx = ex;
    return gx;
  }
  // Enqueues the rest of this solve as one graph launch (and the read of the
  // control block); false when the host-driven loop has to run instead.
  bool start_device() {
    if (st != MAIN || !device_loop_ok()) return false;
    if (ensure_dlog() != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaGraphExec_t gx = solve_graph();
    if (!gx) return false;
    k_d_setup<<<1, 1, 0, B->st>>>(B->ctl, loop_init());
    chk(cudaGetLastError());
    chk(cudaGraphLaunch(gx, B->st));
    fetch_async();
    return true;
  }
  // After the launch has completed: the solve's state and log from the device.
  void absorb_device() {
    if (err != cudaSuccess) return;
    const Ctl& h = H();
    count_launches((int)h.launches);
    if (h.logc > 0 && logbuf)
      chk(cudaMemcpy(logbuf + logc, B->dlog, (size_t)h.logc * sizeof(atkm_iter_log), cudaMemcpyDeviceToHost));
    logc += h.logc;
    n = h.n;
    q = h.q;
    caps = h.caps;
    f32 = h.f32 != 0;
    total_h += h.total_h;
    f32_iters += h.f32_iters;
    linf = h.linf_n;
    status = h.status;
    st = DONE;
    ran_device = true;
  }
  bool done() const { return st == DONE || err != cudaSuccess; }
  Ctl& H() { return *B->ctl_h; }
  Seq seq(bool is32) {
    Seq S{plan, *B, ph, is32, q};
    S.aux32 = (split || dwm) && !is32;
    S.dw = dwm && !is32;
    return S;
  }
  void fetch_async() { chk(cudaMemcpyAsync(B->ctl_h, B->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, B->st)); }
  void set_scalar(double* dst, double v) {
    k_set_scalar<<<1, 1, 0, B->st>>>(dst, v);
    count_launches(1);
    chk(cudaGetLastError());
  }

  int begin(atkm_plan* pl, const atkm_params* pr, const atkm_pcg_opts* op, double* ps, atkm_result* o,
            cudaStream_t cs) {
    plan = pl; prm = pr; opts = op; psi = ps; out = o; caller = cs;
    t_start = std::chrono::steady_clock::now();
    if (!plan || !prm || !opts || !psi || !out) return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: NULL argument");
    if (!(opts->tol_residual >= 0.0) || opts->max_iter < 0 || opts->max_halvings < 0 || !(opts->time_limit_s >= 0.0))
      return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: bad options");
    split = opts->precision_mode == ATKM_PRECISION_F32_SPLIT;
    dwm = opts->precision_mode == ATKM_PRECISION_DF32_SPLIT;
    mixed = opts->precision_mode == ATKM_PRECISION_F32_F64 || split || dwm;
    if (opts->precision_mode != ATKM_PRECISION_F64 && !mixed)
      return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: unknown precision_mode");
    if (mixed && !(plan->flags & ATKM_PLAN_F32))
      return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: mixed precision needs a plan created with ATKM_PLAN_F32");
    if (dwm && !(plan->flags & ATKM_PLAN_DF32))
      return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: the double-word form needs a plan created with ATKM_PLAN_DF32");
    logbuf = out->log;
    memset(out, 0, sizeof(*out));
    out->log = logbuf;
    cudaError_t ae = pcg_alloc(plan);
    if (ae != cudaSuccess) return cuda_fail(plan, ae, "pcg_ground_state: allocation");
    B = plan->pcg;
    ph = make_phys(prm);
    if (B->gphys_set && memcmp(&B->gphys, &ph, sizeof(Phys)) != 0) destroy_graphs(B);
    B->gphys = ph;
    B->gphys_set = true;
    use_graphs = !opts->no_graphs;
    began = true;
    chk(cudaEventRecord(B->ev_in, caller));  // order after the caller's prior work
    chk(cudaStreamWaitEvent(B->st, B->ev_in, 0));
    set_scalar(&B->ctl->hv, plan->hvol);
    set_scalar(&B->ctl->beta, prm->beta);
    set_scalar(&B->ctl->lam, prm->lambda);
    f32 = mixed;
    sw_auto = mixed && opts->switch_tol < 0.0;
    sw_eff = fabs(opts->switch_tol);
    if (opts->resume && B->valid) {
      q = B->parity;
      n = n_start = f32_best_n = B->n;
      caps = B->caps;
      linf = B->linf;
      if (B->f32 && !mixed) {  // continue in FP64 from an FP32-phase state
        Seq S = seq(false);
        S.atkm(SRC_PSI, reinterpret_cast<const double*>(B->phi[q]), nullptr, B->Phi[q]);
        S.ctl1(k_c_reset_state, B->ctl, 0, 1, 0);
        chk(S.err);
        f32 = false;
      } else {
        f32 = B->f32 && mixed;
        if (f32 && sw_auto) sw_eff = std::max(sw_eff, B->sw_eff);
      }
      st = MAIN;
    } else {
      // Normalise psi_0 into phi, Phi_0 by ATKM (Step 1 at n = 0).
      q = 0;
      Seq S = seq(f32);
      const double2* p0 = reinterpret_cast<const double2*>(psi);
      S.dot(p0, p0, S_N);
      S.ctl1(k_c_init, B->ctl, (const double*)plan->scal);
      // the normalisation stays FP64 in every precision form (as the
      // renormalisation after each retraction does)
      S.lincomb(B->phi[0], p0, Coef{&B->ctl->inv0, 1.0}, nullptr, Coef{nullptr, 0.0}, nullptr, Coef{nullptr, 0.0},
                nullptr, S_T, nullptr, false);
      S.atkm(SRC_PSI, reinterpret_cast<const double*>(B->phi[0]), nullptr, B->Phi[0]);
      S.ctl1(k_c_reset_state, B->ctl, 0, 1, 1);
      chk(S.err);
      if (sw_auto) {
        // the residual's FP32 noise at phi_0: H phi_0 with the FP32 operators
        // (and the FP32 Phi_0 just formed) against binary64 throughout
        Seq Z{plan, *B, ph, false, 0};
        const double* p0d = reinterpret_cast<const double*>(B->phi[0]);
        Z.atkm(SRC_PSI, p0d, nullptr, B->Phi1);
        chk(launch_H<double>(plan, ph, p0d, p0d, B->Phi1, reinterpret_cast<double*>(B->Hp), -1, B->st));
        chk(launch_H<float>(plan, ph, p0d, p0d, B->Phi[0], reinterpret_cast<double*>(B->Hphi), -1, B->st));
        Z.lincomb(B->Pr, B->Hp, Coef{nullptr, 1.0}, B->Hphi, Coef{nullptr, -1.0}, nullptr, Coef{nullptr, 0.0},
                  nullptr, S_Z, nullptr, false);
        Z.ctl1(k_c_noise, B->ctl, (const double*)plan->scal);
        chk(Z.err);
      }
      fetch_async();
      st = INIT_CHECK;
    }
    set_scalar(&B->ctl->tolE_eps, 32.0 * (f32 ? eps32 : eps_polish()));
    B->valid = false;  // set again when this solve ends cleanly
    return ATKM_OK;
  }

  void launch() {
    if (st == INIT_CHECK) return;  // its work is already enqueued
    Seq S = seq(f32);
    if (st == MAIN) chk(run_phase(S, 0, use_graphs));
    else if (st == HALVE) chk(run_phase(S, 1, use_graphs));
    else if (st == FORCED) chk(run_phase(S, 2, use_graphs));
    else if (st == FINAL) { S.top(); chk(S.err); }
    fetch_async();
  }

  void wait() {
    chk(cudaStreamSynchronize(B->st));
    if (B->last) {  // graph replay with profiling events: collect its pass times
      prof_accumulate(plan, *B->last);
      B->last = nullptr;
    }
  }

  void finish_iteration(bool accepted) {
    Ctl& h = H();
    total_h += h.nh;
    if (accepted) caps = 0;
    else ++caps;
    if (L) {
      L->alpha = h.alpha; L->beta_cg = h.beta_cg; L->reset_to_sd = h.reset; L->d1 = h.d1; L->curvature = h.curv;
      L->t0 = h.t0; L->t = h.t; L->halvings = h.nh; L->accepted = accepted;
    }
    linf = h.linf;
    Seq S = seq(f32);
    S.ctl1(k_c_end, B->ctl);
    chk(S.err);
    q ^= 1;
    ++n;
    if (caps >= 3 && !f32) {
      status = ATKM_STAGNATED;
      st = FINAL;
    } else {
      st = MAIN;
    }
  }

  void process() {
    if (err != cudaSuccess) return;
    Ctl& h = H();
    switch (st) {
      case INIT_CHECK:
        if (h.nan) {
          status = ATKM_ERR_NAN;
          early_code = ATKM_ERR_NAN;
          st = DONE;
        } else {
          if (sw_auto && isfinite(h.noise) && h.noise > 0.0) sw_eff = std::max(sw_eff, kNoiseFactor * h.noise);
          st = MAIN;
        }
        return;
      case MAIN: {
        L = (logbuf && logc < opts->log_capacity) ? &logbuf[logc] : nullptr;
        if (L) {
          memset(L, 0, sizeof(*L));
          L->n = n; L->E = h.E; L->mu = h.mu; L->residual = h.res; L->linf_step = linf; L->f32_phase = f32;
          ++logc;
        }
        if (h.nan) { status = ATKM_ERR_NAN; st = DONE; return; }
        if (f32 && h.res < f32_gain() * f32_best) { f32_best = h.res; f32_best_n = n; }
        if (f32 && (h.res <= sw_eff || caps >= 2 || n - f32_best_n > f32_window())) {
          // hand over to FP64: recompute Phi in FP64, re-evaluate this phi, restart the direction
          f32 = false;
          caps = 0;
          Seq S = seq(false);
          S.atkm(SRC_PSI, reinterpret_cast<const double*>(B->phi[q]), nullptr, B->Phi[q]);
          S.ctl1(k_c_reset_state, B->ctl, 0, 1, 0);
          chk(S.err);
          set_scalar(&B->ctl->tolE_eps, 32.0 * eps_polish());
          if (L) { --logc; L = nullptr; }
          st = MAIN;
          return;
        }
        if (!f32 && (h.res <= opts->tol_residual || (opts->tol_linf > 0 && linf <= opts->tol_linf))) {
          status = ATKM_OK;
          st = DONE;
          return;
        }
        if (n - n_start >= opts->max_iter) { status = ATKM_NOT_CONVERGED; st = DONE; return; }
        if (past_time_limit()) { status = ATKM_ERR_TIMEOUT; st = DONE; return; }
        if (f32) ++f32_iters;
        decide_trial();
        return;
      }
      case HALVE:
        decide_trial();
        return;
      case FORCED:
        finish_iteration(false);
        return;
      case FINAL:
        st = DONE;
        return;
      default:
        return;
    }
  }

  // Step 4 (iii) after a trial: accept, halve again, or take the best trial.
  void decide_trial() {
    Ctl& h = H();
    if (!isfinite(h.En)) { status = ATKM_ERR_NAN; st = DONE; return; }
    if (h.accepted) { finish_iteration(true); return; }
    st = (h.nh < opts->max_halvings) ? HALVE : FORCED;
  }

  // Called when another instance failed before this one started iterating.
  void abandon() {
    if (began && B) cudaStreamSynchronize(B->st);
  }

  int end() {
    if (!began) return early_code;
    if (err != cudaSuccess) {
      out->status = ATKM_ERR_CUDA;
      cudaStreamSynchronize(B->st);
      return cuda_fail(plan, err, "pcg_ground_state");
    }
    if (early_code == ATKM_ERR_NAN) {
      out->status = ATKM_ERR_NAN;
      B->valid = false;
      chk(cudaEventRecord(B->ev_out, B->st));
      chk(cudaStreamWaitEvent(caller, B->ev_out, 0));
      return fail(plan, ATKM_ERR_NAN, "pcg_ground_state: initial state has zero or non-finite norm");
    }
    Ctl& h = H();
    B->valid = (status == ATKM_OK || status == ATKM_NOT_CONVERGED || status == ATKM_STAGNATED ||
                status == ATKM_ERR_TIMEOUT);
    B->f32 = f32; B->parity = q; B->n = n; B->caps = caps; B->linf = linf; B->sw_eff = sw_eff;
    chk(cudaMemcpyAsync(psi, B->phi[q], B->N * sizeof(double2), cudaMemcpyDeviceToDevice, B->st));
    chk(cudaEventRecord(B->ev_out, B->st));
    chk(cudaStreamWaitEvent(caller, B->ev_out, 0));
    chk(cudaStreamSynchronize(B->st));
    if (err != cudaSuccess) {
      out->status = ATKM_ERR_CUDA;
      return cuda_fail(plan, err, "pcg_ground_state");
    }
    out->E_kin = h.kin;
    out->E_rot = h.rot;
    out->E_pot = h.pot;
    out->E_int = 0.5 * prm->beta * h.f4;
    out->E_dip = 0.5 * prm->lambda * h.dip;
    out->E = out->E_kin + out->E_rot + out->E_pot + out->E_int + out->E_dip;
    out->mu = h.mu;
    out->virial = 2 * out->E_kin - 2 * out->E_pot + 3 * out->E_int + 3 * out->E_dip;
    out->residual = h.res;
    out->linf_step = linf;
    out->iters = n;
    out->halvings = total_h;
    out->f32_iters = f32_iters;
    out->status = status;
    out->log_count = logc;
    out->device_loop = ran_device ? 1 : 0;
    out->switch_residual = mixed ? sw_eff : 0.0;
    if (status != ATKM_OK) {
      const char* why = status == ATKM_NOT_CONVERGED ? "max_iter reached"
                        : status == ATKM_STAGNATED   ? "three consecutive exhausted halving loops"
                        : status == ATKM_ERR_TIMEOUT ? "time limit reached"
                                                     : "non-finite energy or residual";
      fail(plan, status, std::string("pcg_ground_state: ") + why);
    }
    return status;
  }
};

// Every unfinished instance that can run device-driven becomes one chain of
// a single graph (built for this call), launched once on `st` after each
// instance's start-up work; each instance's plan stream is ordered after it.
// Instances are left untouched when the graph cannot be built.
static void batched_single_launch(std::vector<Solver>& S, cudaStream_t st) {
  std::vector<Solver*> run;
  for (auto& s : S)
    if (!s.done() && s.st == Solver::MAIN && s.device_loop_ok()) run.push_back(&s);
  if (run.size() < 2) return;  // one instance: its own cached graph
  for (Solver* s : run)
    if (s->ensure_dlog() != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t gx = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  std::vector<LoopInit> inits;
  inits.reserve(run.size());
  for (Solver* s : run) {
    if (e != cudaSuccess) break;
    inits.push_back(s->loop_init());
    e = s->build_chain(g, &inits.back());
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    return;
  }
  for (Solver* s : run) {  // after each instance's start-up work
    s->chk(cudaEventRecord(s->B->ev_in, s->B->st));
    s->chk(cudaStreamWaitEvent(st, s->B->ev_in, 0));
  }
  e = cudaGraphLaunch(gx, st);
  for (Solver* s : run) {
    s->chk(e);
    s->chk(cudaMemcpyAsync(s->B->ctl_h, s->B->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  }
  const cudaError_t es = cudaStreamSynchronize(st);
  for (Solver* s : run) {
    s->chk(es);
    s->absorb_device();
  }
  cudaGraphExecDestroy(gx);
  cudaGraphDestroy(g);
}

}  // namespace atkm

using namespace atkm;

extern "C" {

int atkm_energy_parts(atkm_plan* plan, const atkm_params* prm, const double* phi, const double* Phi,
                      atkm_energy* out, void* stream) {
  if (!plan || !prm || !phi || !Phi || !out) return fail(plan, ATKM_ERR_ARG, "atkm_energy_parts: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  // W1 holds at least N complex values and is free outside the ATKM passes.
  cudaError_t e = launch_H<double>(plan, make_phys(prm), phi, phi, Phi, reinterpret_cast<double*>(plan->W1), S_H, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->scal_host + S_H, plan->scal + S_H, 10 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(plan, e, "atkm_energy_parts");
  const double hv = plan->hvol;
  const double* h = plan->scal_host;
  out->E_kin = hv * (h[S_H + 0] + h[S_H + 2] + h[S_H + 4]);
  out->E_rot = hv * (h[S_H + 1] + h[S_H + 3]);
  out->E_pot = hv * h[S_H + 5];
  out->E_int = 0.5 * prm->beta * hv * h[S_H + 6];
  out->E_dip = 0.5 * prm->lambda * hv * h[S_H + 7];
  out->E = out->E_kin + out->E_rot + out->E_pot + out->E_int + out->E_dip;
  out->mu = hv * h[S_H + 8];
  out->virial = 2 * out->E_kin - 2 * out->E_pot + 3 * out->E_int + 3 * out->E_dip;
  out->norm2 = hv * h[S_H + 9];
  return ATKM_OK;
}

int apply_preconditioner(atkm_plan* plan, const atkm_params* prm, double alpha, const double* r, const double* phi,
                         const double* Phi, double* Pr, void* stream) {
  if (!plan || !prm || !r || !phi || !Phi || !Pr) return fail(plan, ATKM_ERR_ARG, "apply_preconditioner: NULL argument");
  if (!(alpha > 0.0)) return fail(plan, ATKM_ERR_ARG, "apply_preconditioner: alpha must be > 0");
  if (Pr == r || Pr == phi || Pr == Phi) return fail(plan, ATKM_ERR_ARG, "apply_preconditioner: output aliases an input");
  cudaStream_t st = (cudaStream_t)stream;
  k_set_scalar<<<1, 1, 0, st>>>(plan->scal + SC_ALPHA, alpha);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_precond<double>(plan, make_phys(prm), plan->scal + SC_ALPHA, r, phi, Phi, Pr, st);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "apply_preconditioner");
}

int pcg_ground_state(atkm_plan* plan, const atkm_params* prm, const atkm_pcg_opts* opts, double* psi_inout,
                     atkm_result* out, void* stream) {
  Solver S;
  int code = S.begin(plan, prm, opts, psi_inout, out, (cudaStream_t)stream);
  if (code != ATKM_OK) return code;
  if (S.st == Solver::INIT_CHECK) {  // the start-up work is enqueued: its NaN check
    S.wait();
    S.process();
  }
  if (!S.done() && S.start_device()) {  // the whole loop in one graph launch
    S.wait();
    S.absorb_device();
  }
  while (!S.done()) {  // host-driven loop (profiling on, graphs off, or no device loop)
    S.launch();
    S.wait();
    S.process();
  }
  return S.end();
}

int pcg_ground_state_batched(int count, atkm_plan* const* plans, const atkm_params* prm, const atkm_pcg_opts* opts,
                             double* const* psi, atkm_result* out, void* stream) {
  if (count < 1 || !plans || !prm || !opts || !psi || !out)
    return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_batched: bad count or NULL argument");
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (plans[i] == plans[j])
        return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_batched: each instance needs its own plan");
  std::vector<Solver> S(count);
  int first_err = ATKM_OK;
  for (int i = 0; i < count; ++i) {
    const int code = S[i].begin(plans[i], &prm[i], opts, psi[i], &out[i], (cudaStream_t)stream);
    if (code != ATKM_OK && first_err == ATKM_OK) first_err = code;
  }
  if (first_err != ATKM_OK) {
    for (int i = 0; i < count; ++i) S[i].abandon();
    return first_err;
  }
  for (auto& s : S)
    if (s.st == Solver::INIT_CHECK) {
      s.wait();
      s.process();
    }
  // Device-driven: every instance's whole solve in one graph (one chain per
  // instance, no dependencies between chains), one launch for the sweep.
  batched_single_launch(S, (cudaStream_t)stream);
  // Otherwise each instance's solve graph on its own stream; what still
  // needs the host (profiling, graphs off) runs event-driven: every instance
  // enqueues its next phase as soon as its previous one has been processed,
  // so small grids keep iterating while large ones are still on the GPU.
  std::vector<char> dev(count, 0);
  for (int i = 0; i < count; ++i)
    if (!S[i].done()) dev[i] = S[i].start_device();
  for (int i = 0; i < count; ++i)
    if (dev[i]) {
      S[i].wait();
      S[i].absorb_device();
    }
  for (auto& s : S)
    if (!s.done()) s.launch();
  while (true) {
    bool any = false, progressed = false;
    for (auto& s : S) {
      if (s.done()) continue;
      any = true;
      const cudaError_t q = cudaStreamQuery(s.B->st);
      if (q == cudaErrorNotReady) continue;
      s.wait();  // returns at once (or records the stream's error)
      s.process();
      if (!s.done()) s.launch();
      progressed = true;
    }
    if (!any) break;
    if (!progressed) std::this_thread::yield();
  }
  int worst = ATKM_OK;
  for (auto& s : S) {
    const int code = s.end();
    if (code != ATKM_OK && worst == ATKM_OK) worst = code;
    if (code == ATKM_ERR_CUDA) worst = code;
  }
  return worst;
}

int pcg_ground_state_mg(int levels, atkm_plan* const* plans, const atkm_params* prm, const atkm_pcg_opts* opts,
                        double* const* psi, atkm_result* out, void* stream) {
  if (levels < 1 || !plans || !prm || !opts || !psi || !out)
    return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_mg: bad level count or NULL argument");
  for (int i = 0; i < levels; ++i)
    if (!plans[i] || !psi[i]) return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_mg: NULL plan or buffer");
  for (int i = 0; i + 1 < levels; ++i) {
    const Geo &a = plans[i]->g, &b = plans[i + 1]->g;
    if (plans[i] == plans[i + 1] || psi[i] == psi[i + 1])
      return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_mg: levels need distinct plans and buffers");
    if (b.Nx < a.Nx || b.Ny < a.Ny || b.Nz < a.Nz)
      return fail(nullptr, ATKM_ERR_ARG, "pcg_ground_state_mg: grids must not get coarser");
  }
  atkm_pcg_opts o = *opts;
  o.resume = 0;
  const auto t0 = std::chrono::steady_clock::now();
  int code = ATKM_OK;
  for (int i = 0; i < levels; ++i) {
    if (opts->time_limit_s > 0.0) {  // the limit covers the whole cascade
      const double used = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      o.time_limit_s = std::max(opts->time_limit_s - used, 1e-9);
    }
    o.precision_mode = i < opts->mg_f64_levels ? ATKM_PRECISION_F64 : opts->precision_mode;
    code = pcg_ground_state(plans[i], prm, &o, psi[i], &out[i], stream);
    if (code != ATKM_OK && code != ATKM_NOT_CONVERGED && code != ATKM_STAGNATED) return code;
    if (i + 1 < levels) {
      const int up = atkm_spectral_upsample(plans[i], plans[i + 1], psi[i], psi[i + 1], stream);
      if (up != ATKM_OK) return up;
    }
  }
  return code;
}

}  // extern "C"
