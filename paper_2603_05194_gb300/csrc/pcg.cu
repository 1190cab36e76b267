// Riemannian PCG (Algorithm 1, PCG-ATKM) on the device: deterministic FP64
// reductions (fixed grid, fixed-order two-level sums), fused vector updates,
// and the host-side step control of §2.3 (i)-(iii).
//
// Per iteration n (phi = phi_n, Phi = Phi_n of the accepted previous trial):
//   H phi (3 axis passes, fused energy sums) -> mu, r = H phi - mu phi, ||r||
//   alpha -> P r (5 passes) -> PR+ scalars -> p, <H phi, p>, ||p||^2
//   H p, Phi' = U_dip * Re(conj(phi) p) -> curvature of Eq. (Energy_Expend)
//   t (Eq. (opt_step) or 0.3) -> retraction (Eq. (retraction)), renormalise,
//   Phi+ by ATKM, E(phi+) -> accept or halve.
// The trial energy's quadratic part is formed from <A phi,phi>, <A phi,p>,
// <A p,p> with A = -1/2[[Delta]] + V - Omega[[L_z]] (A is linear, so
// <A phi+, phi+> expands exactly in cos/sin of the retraction); only the
// quartic and dipolar terms need phi+ itself.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "atkm_internal.cuh"

namespace atkm {

namespace {

constexpr int kRedGrid = 1216;  // 8 CTAs per SM on 152 SMs
constexpr int kRedThreads = 256;

// ---------------------------------------------------------- reductions
__global__ void k_finalize(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
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
  if (threadIdx.x == 0) out[0] = sh[0];
}

constexpr int kMaxDots = 8;
struct DotPairs {
  const double2* u[kMaxDots];
  const double2* v[kMaxDots];
  int n;
};

// sum_j Re(u_j conj(v_j)) for up to 8 pairs in one sweep.
__global__ void __launch_bounds__(kRedThreads) k_dots(DotPairs dp, size_t N, double* __restrict__ part) {
  double acc[kMaxDots];
#pragma unroll
  for (int i = 0; i < kMaxDots; ++i) acc[i] = 0.0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < kMaxDots; ++i) {
      if (i < dp.n) {
        const double2 a = dp.u[i][j], b = dp.v[i][j];
        acc[i] += a.x * b.x + a.y * b.y;
      }
    }
  }
  block_reduce_store<kMaxDots>(acc, part, gridDim.x, blockIdx.x);
}

// out = c0 v0 + c1 v1 + c2 v2 (null vectors skipped); sums |out|^2 and
// Re(w conj(out)) when w is given.
__global__ void __launch_bounds__(kRedThreads)
k_lincomb(double2* __restrict__ out, const double2* __restrict__ v0, double c0, const double2* __restrict__ v1,
          double c1, const double2* __restrict__ v2, double c2, const double2* __restrict__ w, size_t N,
          double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
    double2 o = make_double2(0.0, 0.0);
    if (v0) { const double2 a = v0[j]; o.x += c0 * a.x; o.y += c0 * a.y; }
    if (v1) { const double2 a = v1[j]; o.x += c1 * a.x; o.y += c1 * a.y; }
    if (v2) { const double2 a = v2[j]; o.x += c2 * a.x; o.y += c2 * a.y; }
    out[j] = o;
    acc[0] += o.x * o.x + o.y * o.y;
    if (w) { const double2 b = w[j]; acc[1] += b.x * o.x + b.y * o.y; }
  }
  block_reduce_store<2>(acc, part, gridDim.x, blockIdx.x);
}

// phi+ *= inv; block max of |phi+ - phi|.
__global__ void __launch_bounds__(kRedThreads)
k_scale_linf(double2* __restrict__ phin, const double2* __restrict__ phi, double inv, size_t N,
             double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double m = 0.0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
    double2 a = phin[j];
    a.x *= inv; a.y *= inv;
    phin[j] = a;
    const double2 b = phi[j];
    m = fmax(m, hypot(a.x - b.x, a.y - b.y));
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Sums for the curvature and the trial energy:
//   [0] sum rho'(beta rho' + lambda Phi'),  rho' = Re(conj(phi) p)
//   [1] sum (beta|phi|^2 + lambda Phi) Re(phi conj(p))
//   [2] sum (beta|phi|^2 + lambda Phi) |p|^2
__global__ void __launch_bounds__(kRedThreads)
k_curv_sums(const double2* __restrict__ phi, const double2* __restrict__ p, const double* __restrict__ Phi,
            const double* __restrict__ Phi1, double beta, double lambda, size_t N, double* __restrict__ part) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
    const double2 a = phi[j], b = p[j];
    const double rp = a.x * b.x + a.y * b.y;
    const double w = beta * (a.x * a.x + a.y * a.y) + lambda * Phi[j];
    acc[0] += rp * (beta * rp + lambda * Phi1[j]);
    acc[1] += w * rp;
    acc[2] += w * (b.x * b.x + b.y * b.y);
  }
  block_reduce_store<3>(acc, part, gridDim.x, blockIdx.x);
}

// [0] sum |phi|^4, [1] sum Phi |phi|^2
__global__ void __launch_bounds__(kRedThreads)
k_quartic_sums(const double2* __restrict__ phi, const double* __restrict__ Phi, size_t N, double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
    const double2 a = phi[j];
    const double r = a.x * a.x + a.y * a.y;
    acc[0] += r * r;
    acc[1] += Phi[j] * r;
  }
  block_reduce_store<2>(acc, part, gridDim.x, blockIdx.x);
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

int red_grid(size_t N) {
  size_t b = (N + kRedThreads * 4 - 1) / (kRedThreads * 4);
  if (b < 1) b = 1;
  if (b > (size_t)kRedGrid) b = kRedGrid;
  return (int)b;
}

}  // namespace

cudaError_t launch_finalize(atkm_plan* p, int nslots, int nblocks, int dst_slot, cudaStream_t st) {
  k_finalize<<<nslots, kRedThreads, 0, st>>>(p->partials, nblocks, p->scal + dst_slot);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------- PCG state
struct PcgBuffers {
  size_t N = 0;
  double2 *phi = nullptr, *Hphi = nullptr, *r = nullptr, *Pr = nullptr, *p = nullptr, *pprev = nullptr,
          *rprev = nullptr, *Hp = nullptr, *phin = nullptr;
  double *Phi = nullptr, *Phi1 = nullptr, *Phin = nullptr;
  // scalar state carried between calls (resume)
  bool valid = false, f32 = false, have_prev = false, force_sd = true;
  int n = 0, caps = 0;
  double E = 0.0, den_prev = 0.0, linf = INFINITY;
};

void pcg_free(atkm_plan* p) {
  if (!p->pcg) return;
  PcgBuffers* b = p->pcg;
  void* ptrs[] = {b->phi, b->Hphi, b->r, b->Pr, b->p, b->pprev, b->rprev, b->Hp, b->phin, b->Phi, b->Phi1, b->Phin};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete b;
  p->pcg = nullptr;
}

static cudaError_t pcg_alloc(atkm_plan* p) {
  if (p->pcg) return cudaSuccess;
  PcgBuffers* b = new PcgBuffers();
  p->pcg = b;
  const size_t N = (size_t)p->g.Nx * p->g.Ny * p->g.Nz;
  b->N = N;
  double2** cv[] = {&b->phi, &b->Hphi, &b->r, &b->Pr, &b->p, &b->pprev, &b->rprev, &b->Hp, &b->phin};
  for (double2** q : cv) {
    cudaError_t e = dev_alloc(p, (void**)q, N * sizeof(double2));
    if (e != cudaSuccess) { pcg_free(p); return e; }
  }
  double** rv[] = {&b->Phi, &b->Phi1, &b->Phin};
  for (double** q : rv) {
    cudaError_t e = dev_alloc(p, (void**)q, N * sizeof(double));
    if (e != cudaSuccess) { pcg_free(p); return e; }
  }
  // the previous-iteration vectors are read (and ignored) before the first
  // step; give them defined contents
  cudaError_t e = cudaMemset(b->pprev, 0, N * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemset(b->rprev, 0, N * sizeof(double2));
  if (e != cudaSuccess) pcg_free(p);
  return e;
}

// Small helper bundling plan, stream and the scalar read-back.
struct Dev {
  atkm_plan* p;
  cudaStream_t st;
  size_t N;
  cudaError_t err = cudaSuccess;

  void chk(cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; }
  // Launch k_dots for the given pairs into scal[dst..dst+n).
  void dots(std::initializer_list<std::pair<const double2*, const double2*>> pairs, int dst) {
    DotPairs dp;
    memset(&dp, 0, sizeof(dp));
    for (auto& pr : pairs) { dp.u[dp.n] = pr.first; dp.v[dp.n] = pr.second; ++dp.n; }
    const int G = red_grid(N);
    k_dots<<<G, kRedThreads, 0, st>>>(dp, N, p->partials);
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, dp.n, G, dst, st));
  }
  void lincomb(double2* out, const double2* v0, double c0, const double2* v1, double c1, const double2* v2,
               double c2, const double2* w, int dst) {
    const int G = red_grid(N);
    k_lincomb<<<G, kRedThreads, 0, st>>>(out, v0, c0, v1, c1, v2, c2, w, N, p->partials);
    count_launches(1);
    chk(cudaGetLastError());
    chk(launch_finalize(p, 2, G, dst, st));
  }
  // Copies scal[lo..hi) to the pinned mirror and waits.
  void fetch(int lo, int hi) {
    chk(cudaMemcpyAsync(p->scal_host + lo, p->scal + lo, (hi - lo) * sizeof(double), cudaMemcpyDeviceToHost, st));
    chk(cudaStreamSynchronize(st));
  }
  double h(int i) const { return p->scal_host[i]; }
};

// Slots used by the driver.
enum {
  S_H = SC_RED,          // 10 slots of the H phi reductions
  S_R = SC_RED + 10,     // |r|^2 (+ unused)
  S_D = SC_RED + 12,     // 7 dots for the direction
  S_P = SC_RED + 20,     // |p|^2, <H phi, p>
  S_C = SC_RED + 22,     // <Hp,p>  then 3 curvature sums at S_C+1
  S_T = SC_RED + 26,     // |phi+|^2 (+ unused)
  S_Q = SC_RED + 28,     // 2 quartic sums of phi+
  S_L = SC_RED + 30,     // linf
  S_N = SC_RED + 31      // |psi0|^2
};

struct Parts {
  double kin, rot, pot, f4, dip, mu, norm2;
};

static Parts read_parts(const Dev& d, double hvol) {
  Parts q;
  q.kin = hvol * (d.h(S_H + 0) + d.h(S_H + 2) + d.h(S_H + 4));
  q.rot = hvol * (d.h(S_H + 1) + d.h(S_H + 3));
  q.pot = hvol * d.h(S_H + 5);
  q.f4 = hvol * d.h(S_H + 6);
  q.dip = hvol * d.h(S_H + 7);
  q.mu = hvol * d.h(S_H + 8);
  q.norm2 = hvol * d.h(S_H + 9);
  return q;
}

}  // namespace atkm

using namespace atkm;

extern "C" {

int atkm_energy_parts(atkm_plan* plan, const atkm_params* prm, const double* phi, const double* Phi,
                      atkm_energy* out, void* stream) {
  if (!plan || !prm || !phi || !Phi || !out) return fail(plan, ATKM_ERR_ARG, "atkm_energy_parts: NULL argument");
  Dev d{plan, (cudaStream_t)stream, (size_t)plan->g.Nx * plan->g.Ny * plan->g.Nz};
  // W1 holds at least N complex values and is free outside the ATKM passes.
  d.chk(launch_H<double>(plan, make_phys(prm), phi, phi, Phi, reinterpret_cast<double*>(plan->W1), S_H, d.st));
  d.fetch(S_H, S_H + 10);
  if (d.err != cudaSuccess) return cuda_fail(plan, d.err, "atkm_energy_parts");
  const Parts q = read_parts(d, plan->hvol);
  out->E_kin = q.kin;
  out->E_rot = q.rot;
  out->E_pot = q.pot;
  out->E_int = 0.5 * prm->beta * q.f4;
  out->E_dip = 0.5 * prm->lambda * q.dip;
  out->E = out->E_kin + out->E_rot + out->E_pot + out->E_int + out->E_dip;
  out->mu = q.mu;
  out->virial = 2 * out->E_kin - 2 * out->E_pot + 3 * out->E_int + 3 * out->E_dip;
  out->norm2 = q.norm2;
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
  if (!plan || !prm || !opts || !psi_inout || !out) return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: NULL argument");
  if (!(opts->tol_residual >= 0.0) || opts->max_iter < 0 || opts->max_halvings < 0)
    return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: bad options");
  const bool mixed = opts->precision_mode == ATKM_PRECISION_F32_F64;
  if (opts->precision_mode != ATKM_PRECISION_F64 && !mixed)
    return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: unknown precision_mode");
  if (mixed && !(plan->flags & ATKM_PLAN_F32))
    return fail(plan, ATKM_ERR_ARG, "pcg_ground_state: mixed precision needs a plan created with ATKM_PLAN_F32");
  atkm_iter_log* logbuf = out->log;
  memset(out, 0, sizeof(*out));
  out->log = logbuf;
  cudaError_t ae = pcg_alloc(plan);
  if (ae != cudaSuccess) return cuda_fail(plan, ae, "pcg_ground_state: allocation");
  PcgBuffers& B = *plan->pcg;
  Dev d{plan, (cudaStream_t)stream, B.N};
  const double hv = plan->hvol;
  const Phys ph = make_phys(prm);
  const double beta = prm->beta, lam = prm->lambda;
  const double eps64 = 2.220446049250313e-16, eps32 = 1.1920928955078125e-07;

  // Select precision for the spectral operators.
  bool f32 = mixed;
  auto ATKM = [&](int mode, const double* a, const double* b, double* o) {
    d.chk(f32 ? launch_atkm<float>(plan, mode, a, b, o, d.st) : launch_atkm<double>(plan, mode, a, b, o, d.st));
  };
  auto HOP = [&](const double* f, double* o, int red) {
    d.chk(f32 ? launch_H<float>(plan, ph, reinterpret_cast<const double*>(f), reinterpret_cast<const double*>(B.phi),
                                B.Phi, o, red, d.st)
              : launch_H<double>(plan, ph, reinterpret_cast<const double*>(f), reinterpret_cast<const double*>(B.phi),
                                 B.Phi, o, red, d.st));
  };
  auto PREC = [&]() {
    d.chk(f32 ? launch_precond<float>(plan, ph, plan->scal + SC_ALPHA, (double*)B.r, (double*)B.phi, B.Phi,
                                      (double*)B.Pr, d.st)
              : launch_precond<double>(plan, ph, plan->scal + SC_ALPHA, (double*)B.r, (double*)B.phi, B.Phi,
                                       (double*)B.Pr, d.st));
  };
  auto fail_cuda = [&]() {
    out->status = ATKM_ERR_CUDA;
    return cuda_fail(plan, d.err, "pcg_ground_state");
  };

  double E = 0.0, den_prev = 0.0, linf = INFINITY;
  bool have_E = false, force_sd = true, have_prev = false;
  int caps = 0, n = 0, status = ATKM_NOT_CONVERGED, total_h = 0, f32_iters = 0;
  int n_start = 0;
  double f32_best = INFINITY;
  int f32_best_n = 0;
  if (opts->resume && B.valid) {
    // continue the previous solve of this plan
    f32 = B.f32 && mixed;
    if (B.f32 && !mixed) ATKM(SRC_PSI, (const double*)B.phi, nullptr, B.Phi);  // FP64 from here on
    have_E = !(B.f32 && !mixed);
    E = B.E; den_prev = B.den_prev; linf = B.linf; force_sd = B.force_sd || (B.f32 && !mixed);
    have_prev = B.have_prev; caps = B.caps; n = n_start = f32_best_n = B.n;
  } else {
    // Normalise psi0 into phi.
    const double2* psi = reinterpret_cast<const double2*>(psi_inout);
    d.dots({{psi, psi}}, S_N);
    d.fetch(S_N, S_N + 1);
    if (d.err != cudaSuccess) return fail_cuda();
    const double n0 = sqrt(hv * d.h(S_N));
    if (!(n0 > 0.0) || !isfinite(n0)) {
      out->status = ATKM_ERR_NAN;
      B.valid = false;
      return fail(plan, ATKM_ERR_NAN, "pcg_ground_state: initial state has zero or non-finite norm");
    }
    d.lincomb(B.phi, psi, 1.0 / n0, nullptr, 0, nullptr, 0, nullptr, S_T);
    ATKM(SRC_PSI, (const double*)B.phi, nullptr, B.Phi);
  }
  B.valid = false;  // set again when this call ends cleanly
  Parts q{};
  double mu = 0.0, res = 0.0;
  int logc = 0;
  while (true) {
    // ---- Step 2: H phi, mu, r
    HOP((const double*)B.phi, (double*)B.Hphi, S_H);
    d.fetch(S_H, S_H + 10);
    if (d.err != cudaSuccess) return fail_cuda();
    q = read_parts(d, hv);
    mu = q.mu;
    if (!have_E) {
      E = q.kin + q.rot + q.pot + 0.5 * beta * q.f4 + 0.5 * lam * q.dip;
      have_E = true;
    }
    d.lincomb(B.r, B.Hphi, 1.0, B.phi, -mu, nullptr, 0, nullptr, S_R);
    d.fetch(S_R, S_R + 1);
    if (d.err != cudaSuccess) return fail_cuda();
    res = sqrt(hv * d.h(S_R));
    atkm_iter_log* L = (logbuf && logc < opts->log_capacity) ? &logbuf[logc] : nullptr;
    if (L) {
      memset(L, 0, sizeof(*L));
      L->n = n; L->E = E; L->mu = mu; L->residual = res; L->linf_step = linf; L->f32_phase = f32;
      ++logc;
    }
    if (!isfinite(E) || !isfinite(res) || !isfinite(mu)) { status = ATKM_ERR_NAN; break; }
    if (f32) {
      // FP32 stagnation: no halving of the best residual within 100 iterations
      if (res < 0.5 * f32_best) { f32_best = res; f32_best_n = n; }
    }
    if (f32 && (res <= opts->switch_tol || caps >= 2 || n - f32_best_n > 100)) {
      // hand over to FP64: recompute Phi and H phi in FP64, restart the direction
      f32 = false;
      caps = 0;
      force_sd = true;
      have_E = false;
      ATKM(SRC_PSI, (const double*)B.phi, nullptr, B.Phi);
      if (L) --logc;
      continue;
    }
    if (!f32 && (res <= opts->tol_residual || (opts->tol_linf > 0 && linf <= opts->tol_linf))) {
      status = ATKM_OK;
      break;
    }
    if (n - n_start >= opts->max_iter) { status = ATKM_NOT_CONVERGED; break; }
    if (f32) ++f32_iters;
    // ---- Step 3: preconditioned PR+ direction
    const double alpha = q.kin + q.pot + beta * q.f4 + fabs(lam * q.dip);
    k_set_scalar<<<1, 1, 0, d.st>>>(plan->scal + SC_ALPHA, alpha);
  count_launches(1);
    d.chk(cudaGetLastError());
    PREC();
    d.dots({{B.Pr, B.phi}, {B.r, B.Pr}, {B.r, B.phi}, {B.rprev, B.Pr}, {B.rprev, B.phi}, {B.pprev, B.phi},
            {B.phi, B.phi}},
           S_D);
    d.fetch(S_D, S_D + 7);
    if (d.err != cudaSuccess) return fail_cuda();
    const double b_ = hv * d.h(S_D + 0), rPr = hv * d.h(S_D + 1), rphi = hv * d.h(S_D + 2);
    const double rpPr = hv * d.h(S_D + 3), a_ = hv * d.h(S_D + 4), c_ = hv * d.h(S_D + 5), nphi = hv * d.h(S_D + 6);
    const double den = rPr - b_ * rphi;  // <r, J(Pr)>
    double beta_cg = 0.0;
    const bool use_cg = have_prev && !force_sd;
    if (use_cg) {
      const double jrj = rpPr - 2.0 * a_ * b_ + a_ * b_ * nphi;  // <J(r_prev), J(Pr)>
      beta_cg = std::max((den - jrj) / den_prev, 0.0);
      d.lincomb(B.p, B.Pr, -1.0, B.pprev, beta_cg, B.phi, b_ - beta_cg * c_, B.Hphi, S_P);
    } else {
      d.lincomb(B.p, B.Pr, -1.0, B.phi, b_, nullptr, 0, B.Hphi, S_P);
    }
    d.fetch(S_P, S_P + 2);
    if (d.err != cudaSuccess) return fail_cuda();
    double pn2 = hv * d.h(S_P), d1 = hv * d.h(S_P + 1);
    bool reset = false;
    if (d1 >= 0.0) {  // Step 4 (i): PSD fallback
      reset = true;
      beta_cg = 0.0;
      if (use_cg) {
        d.lincomb(B.p, B.Pr, -1.0, B.phi, b_, nullptr, 0, B.Hphi, S_P);
        d.fetch(S_P, S_P + 2);
        if (d.err != cudaSuccess) return fail_cuda();
        pn2 = hv * d.h(S_P);
        d1 = hv * d.h(S_P + 1);
      }
    }
    // ---- Step 4 (ii): quadratic model
    HOP((const double*)B.p, (double*)B.Hp, -1);
    ATKM(SRC_PAIR, (const double*)B.phi, (const double*)B.p, B.Phi1);
    d.dots({{B.Hp, B.p}}, S_C);
    {
      const int G = red_grid(B.N);
      k_curv_sums<<<G, kRedThreads, 0, d.st>>>(B.phi, B.p, B.Phi, B.Phi1, beta, lam, B.N, plan->partials);
      count_launches(1);
      d.chk(cudaGetLastError());
      d.chk(launch_finalize(plan, 3, G, S_C + 1, d.st));
    }
    d.fetch(S_C, S_C + 4);
    if (d.err != cudaSuccess) return fail_cuda();
    const double Hpp = hv * d.h(S_C), S1 = hv * d.h(S_C + 1), S2 = hv * d.h(S_C + 2), S3 = hv * d.h(S_C + 3);
    const double curv = Hpp + 2.0 * S1 - mu * pn2;
    double t = curv > 0.0 ? -d1 / curv : 0.3;
    const double t0 = t;
    const double pn = sqrt(pn2);
    const double Aphiphi = q.kin + q.rot + q.pot;
    const double Aphip = d1 - S2, App = Hpp - S3;
    // ---- Step 4 (iii) + Step 5: retract, renormalise, test the energy
    const double tolE = 32.0 * (f32 ? eps32 : eps64) * fabs(E);
    bool accepted = false;
    int nh = 0;
    double bestE = INFINITY, best_t = t, En = 0.0;
    auto trial = [&](double tt, double& Eout, double& linf_out) {
      const double c = cos(tt * pn), sn = sin(tt * pn) / pn;
      d.lincomb(B.phin, B.phi, c, B.p, sn, nullptr, 0, nullptr, S_T);
      d.fetch(S_T, S_T + 1);
      const double nrm2 = hv * d.h(S_T);
      const int G = red_grid(B.N);
      k_scale_linf<<<G, kRedThreads, 0, d.st>>>(B.phin, B.phi, 1.0 / sqrt(nrm2), B.N, plan->partials);
      count_launches(1);
      d.chk(cudaGetLastError());
      k_finalize_max<<<1, kRedThreads, 0, d.st>>>(plan->partials, G, plan->scal + S_L);
      count_launches(1);
      d.chk(cudaGetLastError());
      ATKM(SRC_PSI, (const double*)B.phin, nullptr, B.Phin);
      k_quartic_sums<<<G, kRedThreads, 0, d.st>>>(B.phin, B.Phin, B.N, plan->partials);
      count_launches(1);
      d.chk(cudaGetLastError());
      d.chk(launch_finalize(plan, 2, G, S_Q, d.st));
      d.fetch(S_Q, S_L + 1);
      const double quad = (c * c * Aphiphi + 2.0 * c * sn * Aphip + sn * sn * App) / nrm2;
      Eout = quad + 0.5 * beta * hv * d.h(S_Q) + 0.5 * lam * hv * d.h(S_Q + 1);
      linf_out = d.h(S_L);
    };
    double linf_new = 0.0;
    while (true) {
      trial(t, En, linf_new);
      if (d.err != cudaSuccess) return fail_cuda();
      if (!isfinite(En)) break;
      if (En <= E + tolE) { accepted = true; break; }
      if (En < bestE) { bestE = En; best_t = t; }
      if (nh >= opts->max_halvings) break;
      t *= 0.5;
      ++nh;
    }
    total_h += nh;
    if (!isfinite(En)) { status = ATKM_ERR_NAN; break; }
    if (accepted) {
      caps = 0;
      force_sd = false;
    } else {
      t = best_t;
      trial(t, En, linf_new);
      if (d.err != cudaSuccess) return fail_cuda();
      ++caps;
      force_sd = true;
    }
    if (L) {
      L->alpha = alpha; L->beta_cg = beta_cg; L->reset_to_sd = reset; L->d1 = d1; L->curvature = curv;
      L->t0 = t0; L->t = t; L->halvings = nh; L->accepted = accepted;
    }
    linf = linf_new;
    std::swap(B.rprev, B.r);
    std::swap(B.pprev, B.p);
    std::swap(B.phi, B.phin);
    std::swap(B.Phi, B.Phin);
    den_prev = den;
    have_prev = true;
    E = En;
    ++n;
    if (caps >= 3 && !f32) {
      status = ATKM_STAGNATED;
      HOP((const double*)B.phi, (double*)B.Hphi, S_H);
      d.fetch(S_H, S_H + 10);
      if (d.err != cudaSuccess) return fail_cuda();
      q = read_parts(d, hv);
      mu = q.mu;
      d.lincomb(B.r, B.Hphi, 1.0, B.phi, -mu, nullptr, 0, nullptr, S_R);
      d.fetch(S_R, S_R + 1);
      res = sqrt(hv * d.h(S_R));
      break;
    }
  }
  // Keep the scalar state for a later resume, copy the state back and report.
  B.valid = (status == ATKM_OK || status == ATKM_NOT_CONVERGED || status == ATKM_STAGNATED);
  B.f32 = f32; B.have_prev = have_prev; B.force_sd = force_sd; B.n = n; B.caps = caps;
  B.E = E; B.den_prev = den_prev; B.linf = linf;
  d.chk(cudaMemcpyAsync(psi_inout, B.phi, B.N * sizeof(double2), cudaMemcpyDeviceToDevice, d.st));
  d.chk(cudaStreamSynchronize(d.st));
  if (d.err != cudaSuccess) return fail_cuda();
  out->E_kin = q.kin;
  out->E_rot = q.rot;
  out->E_pot = q.pot;
  out->E_int = 0.5 * beta * q.f4;
  out->E_dip = 0.5 * lam * q.dip;
  out->E = out->E_kin + out->E_rot + out->E_pot + out->E_int + out->E_dip;
  out->mu = mu;
  out->virial = 2 * out->E_kin - 2 * out->E_pot + 3 * out->E_int + 3 * out->E_dip;
  out->residual = res;
  out->linf_step = linf;
  out->iters = n;
  out->halvings = total_h;
  out->f32_iters = f32_iters;
  out->status = status;
  out->log_count = logc;
  if (status != ATKM_OK) {
    const char* why = status == ATKM_NOT_CONVERGED ? "max_iter reached"
                      : status == ATKM_STAGNATED   ? "three consecutive exhausted halving loops"
                                                   : "non-finite energy or residual";
    fail(plan, status, std::string("pcg_ground_state: ") + why);
  }
  return status;
}

}  // extern "C"
