// Plan creation, the truncated-kernel precompute and the thin C entry points
// of the spectral operators.
//
// Truncated Coulomb coefficients (Eq. (FUk), read with the unshifted basis):
//   U0(nu) = int_{D_2L} e^{-i nu.y} / (4 pi |y|) dy,  D_2L = prod [-a_a, a_a], a_a = 2 L_a,
// at nu_a = pi k_a / a_a, |k_a| = 0..N_a.  With 1/|y| = (2/sqrt(pi)) int_0^inf
// e^{-s^2 |y|^2} ds the box integral separates:
//   U0 = (1 / (2 pi^{3/2})) int_0^inf I_x(s) I_y(s) I_z(s) ds,
//   I_a(s) = int_{-a}^{a} e^{-s^2 y^2} cos(nu y) dy.
// This is the separable Gaussian structure the paper's ATKM reference uses;
// the evaluation below is this library's own:
//   * s in [0, s_lo]: I_a(s) = I_a(0) + O(s^2) (head term s_lo prod I_a(0));
//   * s in [s_lo, s_c], s_c = 7 / min_a a_a: composite 16-point Gauss-Legendre
//     in tau = ln s; I_a by composite Gauss-Legendre in y, written as
//     2 int_0^a expm1(-s^2 y^2) cos(nu y) dy + 2a [k = 0] so the small-s
//     rounding floor scales with s^2, and with the cosine phase reduced
//     exactly (integer part of k u taken mod 2) before cospi;
//     if s a_a >= 7 the box edge is invisible to double precision and
//     I_a = (sqrt(pi)/s) e^{-nu^2/(4 s^2)};
//   * s >= s_c: every factor is Gaussian, the integral is closed form
//     (pi^{3/2} / (2 s_c^2)) (1 - e^{-u}) / u, u = |nu|^2 / (4 s_c^2).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "atkm_internal.cuh"

namespace atkm {

thread_local std::string g_last_error;

static std::atomic<unsigned long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

int fail(atkm_plan* p, int code, const std::string& msg) {
  g_last_error = msg;
  if (p) p->err = msg;
  return code;
}

int cuda_fail(atkm_plan* p, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(p, e == cudaErrorMemoryAllocation ? ATKM_ERR_OOM : ATKM_ERR_CUDA, m);
}

cudaError_t dev_alloc(atkm_plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e == cudaSuccess) p->bytes += bytes;
  else *ptr = nullptr;
  return e;
}

Phys make_phys(const atkm_params* prm) {
  Phys ph;
  ph.gx2 = prm->gamma[0] * prm->gamma[0];
  ph.gy2 = prm->gamma[1] * prm->gamma[1];
  ph.gz2 = prm->gamma[2] * prm->gamma[2];
  ph.beta = prm->beta;
  ph.lambda = prm->lambda;
  ph.Omega = prm->Omega;
  return ph;
}

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kGL = 16;         // Gauss-Legendre points per panel
constexpr double kSlo = 1e-9;   // head cut-off in s
constexpr double kEdge = 7.0;   // s a >= kEdge: box edge below FP64 resolution
constexpr double kTauPanel = 0.75;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n
// (three-term recurrence), the classical Golub-Welsch-free construction.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

struct GLNodes {
  double x[kGL];  // nodes mapped to (0, 1)
  double w[kGL];  // weights for (0, 1)
};

// Twiddles e^{-2 pi i m / L}, and the binary64 ones in multiply-add form
// (lf_cform).
__global__ void k_twiddles(double2* t64, float2* t32, cdf* tdf, double2* lf, int L) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)L, &s, &c);
    t64[m] = make_double2(c, -s);
    t32[m] = make_float2((float)c, (float)-s);
    cdf w;
    w.x = df(c);
    w.y = df(-s);
    tdf[m] = w;
    lf[m] = lf_cform(m, L) ? make_double2(c, -s / c) : make_double2(-s, c / -s);
  }
}

// table[q * (N + 1) + k] = I(s_q; nu_k), nu_k = pi k / a, k = 0..N.
__global__ void k_axis_table(double* __restrict__ table, const double* __restrict__ s_nodes, int Q, int N,
                             double a, GLNodes gl) {
  const int total = Q * (N + 1);
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < total; id += gridDim.x * blockDim.x) {
    const int q = id / (N + 1), k = id - q * (N + 1);
    const double s = s_nodes[q];
    double val;
    if (s * a >= kEdge) {
      const double nu = kPi * k / a;
      val = sqrt(kPi) / s * exp(-nu * nu / (4.0 * s * s));
    } else {
      // 2 a int_0^1 expm1(-(s a u)^2) cospi(k u) du (+ 2a when k = 0),
      // P panels of width 1/P; Neumaier-compensated sum.
      const int P = k / 2 + 2;
      const long twoP = 2L * P;
      double sum = 0.0, comp = 0.0;
      for (int pnl = 0; pnl < P; ++pnl) {
        const double base = (double)(((long)k * pnl) % twoP) / (double)P;  // exact reduction
        for (int i = 0; i < kGL; ++i) {
          const double xi = gl.x[i];
          const double u = (pnl + xi) / P;
          const double su = s * a * u;
          const double th = base + (double)k * xi / (double)P;
          const double term = gl.w[i] * expm1(-su * su) * cospi(th);
          const double tsum = sum + term;
          comp += (fabs(sum) >= fabs(term)) ? (sum - tsum) + term : (term - tsum) + sum;
          sum = tsum;
        }
      }
      val = 2.0 * a * (sum + comp) / P;
      if (k == 0) val += 2.0 * a;
    }
    table[id] = val;
  }
}

// U0 octant from the three tables.
__global__ void k_U0(double* __restrict__ U0, const double* __restrict__ Tx, const double* __restrict__ Ty,
                     const double* __restrict__ Tz, const double* __restrict__ wq, int Q, int Nx, int Ny, int Nz,
                     double ax, double ay, double az, double s_c) {
  const size_t total = (size_t)(Nx + 1) * (Ny + 1) * (Nz + 1);
  for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < total;
       id += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(id % (Nx + 1));
    const int ky = (int)((id / (Nx + 1)) % (Ny + 1));
    const int kz = (int)(id / ((size_t)(Nx + 1) * (Ny + 1)));
    double acc = 0.0, comp = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double term = wq[q] * Tx[(size_t)q * (Nx + 1) + kx] * Ty[(size_t)q * (Ny + 1) + ky] *
                          Tz[(size_t)q * (Nz + 1) + kz];
      const double t = acc + term;
      comp += (fabs(acc) >= fabs(term)) ? (acc - t) + term : (term - t) + acc;
      acc = t;
    }
    acc += comp;
    if (kx == 0 && ky == 0 && kz == 0) acc += kSlo * (2.0 * ax) * (2.0 * ay) * (2.0 * az);
    const double nux = kPi * kx / ax, nuy = kPi * ky / ay, nuz = kPi * kz / az;
    const double u = (nux * nux + nuy * nuy + nuz * nuz) / (4.0 * s_c * s_c);
    const double tailfac = (u == 0.0) ? 1.0 : -expm1(-u) / u;
    acc += kPi * sqrt(kPi) / (2.0 * s_c * s_c) * tailfac;
    U0[id] = acc / (2.0 * kPi * sqrt(kPi));
  }
}

// Full padded multiplier K(k) = -1 + 3 (n.nu)^2 U0 in FFT order.
__global__ void k_multiplier_full(double* __restrict__ K, const double* __restrict__ U0, Geo g, double n0, double n1,
                                  double n2) {
  const size_t total = (size_t)g.Mx * g.My * g.Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.Mx);
    const int y = (int)((i / g.Mx) % g.My);
    const int z = (int)(i / ((size_t)g.Mx * g.My));
    const int kx = x < g.Mx / 2 ? x : x - g.Mx, ky = y < g.My / 2 ? y : y - g.My, kz = z < g.Mz / 2 ? z : z - g.Mz;
    const double nd = n0 * kPi * kx / (2.0 * g.Lx) + n1 * kPi * ky / (2.0 * g.Ly) + n2 * kPi * kz / (2.0 * g.Lz);
    const double u = U0[((size_t)abs(kz) * (g.Ny + 1) + abs(ky)) * (g.Nx + 1) + abs(kx)];
    K[i] = -1.0 + 3.0 * nd * nd * u;
  }
}

// The multiplier of the z pass on the Nx + 1 half-spectrum columns, with the
// inverse transform's 1 / (Mx My Mz) and the factor 1/2 of the x forward
// pass's post-twist (OpAtkmXF) folded in.  A real density's spectrum is
// Hermitian, so the real-data ATKM uses the symmetrised multiplier
// K_sym(k) = (K(k) + K(-k)) / 2 = -1 + 3 U0(nu_k) (A^2 + B^2), where A sums
// n_a nu_a over the axes whose index is not the padded Nyquist index M_a / 2
// and B over those that are: the index of -k has the same Nyquist components
// and the others negated, so the cross term 2AB cancels in the average (the
// Nyquist index M_a / 2 stands for nu = -pi M_a / (4 L_a)).  Layout
// [Mz][My][XS], columns x > Nx zero.
__global__ void k_multiplier_half(double* __restrict__ Kh, const double* __restrict__ U0, Geo g, double n0,
                                  double n1, double n2) {
  const size_t total = (size_t)g.Mz * g.My * g.XS;
  const double px = kPi / (2.0 * g.Lx), py = kPi / (2.0 * g.Ly), pz = kPi / (2.0 * g.Lz);
  const double invM = 0.5 / ((double)g.Mx * g.My * g.Mz);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.XS);
    const int o = (int)((i / g.XS) % g.My);
    const int k = (int)(i / ((size_t)g.XS * g.My));
    if (x > g.Nx) {
      Kh[i] = 0.0;
      continue;
    }
    const int kx = x == g.Nx ? -g.Nx : x;
    const int ky = o < g.My / 2 ? o : o - g.My, kz = k < g.Mz / 2 ? k : k - g.Mz;
    const double tx = n0 * (kx * px), ty = n1 * (ky * py), tz = n2 * (kz * pz);
    double A = 0.0, B = 0.0;
    if (x == g.Nx) B += tx; else A += tx;
    if (o == g.Ny) B += ty; else A += ty;
    if (k == g.Nz) B += tz; else A += tz;
    const double u = U0[((size_t)abs(kz) * (g.Ny + 1) + abs(ky)) * (g.Nx + 1) + x];
    Kh[i] = (3.0 * u * (A * A + B * B) - 1.0) * invM;
  }
}

__global__ void k_to_f32(float* __restrict__ dst, const double* __restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__global__ void k_to_df(df* __restrict__ dst, const double* __restrict__ src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = df(src[i]);
}

// Fine spectrum <- coarse spectrum / Nc: fine frequency k (signed) takes the
// coarse coefficient of the same k when -Nc/2 <= k < Nc/2, zero otherwise.
__global__ void k_embed_spectrum(const double2* __restrict__ coarse, double2* __restrict__ fine, Geo gc, Geo gf,
                                 double scale) {
  const size_t total = (size_t)gf.Nx * gf.Ny * gf.Nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % gf.Nx), y = (int)((i / gf.Nx) % gf.Ny), z = (int)(i / ((size_t)gf.Nx * gf.Ny));
    const int kx = x < gf.Nx / 2 ? x : x - gf.Nx, ky = y < gf.Ny / 2 ? y : y - gf.Ny, kz = z < gf.Nz / 2 ? z : z - gf.Nz;
    double2 v = make_double2(0.0, 0.0);
    if (kx >= -gc.Nx / 2 && kx < gc.Nx / 2 && ky >= -gc.Ny / 2 && ky < gc.Ny / 2 && kz >= -gc.Nz / 2 && kz < gc.Nz / 2) {
      const int cx = (kx + gc.Nx) % gc.Nx, cy = (ky + gc.Ny) % gc.Ny, cz = (kz + gc.Nz) % gc.Nz;
      const double2 c = coarse[((size_t)cz * gc.Ny + cy) * gc.Nx + cx];
      v = make_double2(scale * c.x, scale * c.y);
    }
    fine[i] = v;
  }
}

bool smooth235(int n) {
  if (n <= 0) return false;
  for (int r : {2, 3, 5})
    while (n % r == 0) n /= r;
  return n == 1;
}

bool make_fft_len(int L, FftLen& f) {
  memset(&f, 0, sizeof(f));
  f.L = L;
  int n = L, s = 0;
  const int order[5] = {8, 4, 2, 3, 5};
  for (int r : order) {
    while (n % r == 0) {
      if (s >= kMaxStages) return false;
      f.radix[s++] = r;
      n /= r;
    }
  }
  f.nstages = s;
  return n == 1;
}

void free_plan_memory(atkm_plan* p) {
  void* ptrs[] = {p->tw64, p->tw32, p->twdf, p->lf64, p->axtab, p->Pw, p->U0, p->U0f, p->Kz, p->Kzd, p->W1, p->W2, p->T1, p->W1f, p->W2f, p->T1f,
                  p->partials, p->scal};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->scal_host) cudaFreeHost(p->scal_host);
}

}  // namespace

void pcg_free(atkm_plan* p);  // pcg.cu

// Event-pair record of pass launches (opt-in measurement support).
struct Profiler {
  struct Rec {
    const char* name;
    double bytes, flops;
    cudaEvent_t a, b;
  };
  struct Agg {
    const char* name;
    long launches;
    double ms, bytes, flops;
  };
  std::vector<Rec> recs;                // eager launches since profiling was enabled
  std::vector<Agg> agg;                 // totals accumulated from graph replays
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  bool open = false;
  std::vector<ProfRec>* sink = nullptr;  // graph capture in progress
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  void add(const char* name, double ms, double bytes, double flops) {
    for (auto& a : agg)
      if (strcmp(a.name, name) == 0) {
        a.launches += 1; a.ms += ms; a.bytes += bytes; a.flops += flops;
        return;
      }
    agg.push_back(Agg{name, 1, ms, bytes, flops});
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

void prof_begin(atkm_plan* p, const char* name, double bytes, double flops, cudaStream_t st) {
  Profiler* pr = p->prof;
  if (!pr) return;
  if (pr->sink) {
    ProfRec r{name, bytes, flops, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess) { cudaGetLastError(); return; }
    // external event node: re-recorded on every replay of the captured graph
    if (cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(r.a);
      return;
    }
    pr->sink->push_back(r);
    pr->open = true;
    return;
  }
  Profiler::Rec r{name, bytes, flops, pr->get(), nullptr};
  if (!r.a) return;
  cudaEventRecord(r.a, st);
  pr->recs.push_back(r);
  pr->open = true;
}

void prof_end(atkm_plan* p, cudaStream_t st) {
  Profiler* pr = p->prof;
  if (!pr || !pr->open) return;
  pr->open = false;
  if (pr->sink) {
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess) b = nullptr;
    if (!b || cudaEventRecordWithFlags(b, st, cudaEventRecordExternal) != cudaSuccess) {
      cudaGetLastError();
      if (b) cudaEventDestroy(b);
      pr->sink->back().b = nullptr;  // incomplete record: skipped when accumulating
      return;
    }
    pr->sink->back().b = b;
    return;
  }
  cudaEvent_t b = pr->get();
  if (!b) { pr->recs.pop_back(); return; }
  cudaEventRecord(b, st);
  pr->recs.back().b = b;
}

void prof_set_sink(atkm_plan* p, std::vector<ProfRec>* sink) {
  if (p->prof) p->prof->sink = sink;
}

void prof_accumulate(atkm_plan* p, const std::vector<ProfRec>& recs) {
  Profiler* pr = p->prof;
  if (!pr) return;
  for (const auto& r : recs) {
    if (!r.a || !r.b) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) pr->add(r.name, ms, r.bytes, r.flops);
    else cudaGetLastError();  // do not leave the query's error for the next launch check
  }
}

}  // namespace atkm

using namespace atkm;

extern "C" {

const char* atkm_last_error_string(const atkm_plan* plan) {
  if (plan) return plan->err.c_str();
  return g_last_error.c_str();
}

unsigned long long atkm_plan_device_bytes(const atkm_plan* plan) { return plan ? plan->bytes : 0ull; }

unsigned long long atkm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void atkm_plan_destroy(atkm_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  pcg_free(plan);
  delete plan->prof;
  delete plan->prof_stopped_;
  free_plan_memory(plan);
  delete plan;
}

int atkm_plan_create(atkm_plan** out, const int N[3], const double L[3], const double n[3], unsigned flags,
                     void* stream) {
  if (!out) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_create: out is NULL");
  *out = nullptr;
  if (!N || !L || !n) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_create: NULL argument");
  for (int a = 0; a < 3; ++a) {
    if (!(L[a] > 0.0) || !isfinite(L[a]))
      return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_create: box half-lengths must be positive and finite");
    if (N[a] < 2 || N[a] % 2 != 0 || 2 * N[a] > kMaxLen || !smooth235(N[a]))
      return fail(nullptr, ATKM_ERR_UNSUPPORTED_SIZE,
                  "atkm_plan_create: each N must be even, in [2, 1024] and a product of 2, 3, 5");
  }
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (!isfinite(nn) || fabs(nn - 1.0) > 1e-12)
    return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_create: dipole axis must be a unit vector (| |n|-1 | <= 1e-12)");
  if (flags & ~(unsigned)(ATKM_PLAN_F32 | ATKM_PLAN_DF32 | ATKM_PLAN_GENERIC_FFT | ATKM_PLAN_AUTOTUNE))
    return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_create: unknown flags");

  cudaStream_t st = (cudaStream_t)stream;
  atkm_plan* p = new atkm_plan();
  memset(&p->g, 0, sizeof(p->g));
  p->tw64 = nullptr; p->tw32 = nullptr; p->twdf = nullptr; p->lf64 = nullptr; p->U0 = nullptr;
  p->axtab = nullptr; p->Pw = nullptr;
  p->U0f = nullptr; p->Kz = nullptr; p->Kzd = nullptr;
  p->W1 = p->W2 = p->T1 = nullptr;
  p->W1f = p->W2f = p->T1f = nullptr; p->partials = nullptr; p->scal = nullptr; p->scal_host = nullptr;
  p->pcg = nullptr; p->prof = nullptr; p->prof_stopped_ = nullptr; p->bytes = 0; p->flags = flags;
  p->n_tune = 0;
  Geo& g = p->g;
  g.Nx = N[0]; g.Ny = N[1]; g.Nz = N[2];
  g.Mx = 2 * N[0]; g.My = 2 * N[1]; g.Mz = 2 * N[2];
  g.Xh = N[0] + 1;
  g.XS = (g.Xh + 15) / 16 * 16;
  g.Lx = L[0]; g.Ly = L[1]; g.Lz = L[2];
  g.hx = 2 * L[0] / N[0]; g.hy = 2 * L[1] / N[1]; g.hz = 2 * L[2] / N[2];
  p->hvol = g.hx * g.hy * g.hz;
  for (int a = 0; a < 3; ++a) p->n[a] = n[a];

  auto bail = [&](int code) {
    free_plan_memory(p);
    delete p;
    return code;
  };
  cudaError_t e;
  // ---- FFT descriptors and twiddles
  const int lens[6] = {g.Nx, g.Ny, g.Nz, g.Mx, g.My, g.Mz};
  size_t twtot = 0;
  for (int i = 0; i < 6; ++i) twtot += lens[i];
  if ((e = dev_alloc(p, (void**)&p->tw64, twtot * sizeof(double2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan twiddles"));
  if ((e = dev_alloc(p, (void**)&p->tw32, twtot * sizeof(float2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan twiddles"));
  if ((e = dev_alloc(p, (void**)&p->twdf, twtot * sizeof(cdf))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan twiddles"));
  if ((e = dev_alloc(p, (void**)&p->lf64, twtot * sizeof(double2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan twiddles"));
  size_t off = 0;
  for (int i = 0; i < 6; ++i) {
    FftLen& f = (i < 3) ? p->fN[i] : p->fM[i - 3];
    if (!make_fft_len(lens[i], f)) return bail(fail(nullptr, ATKM_ERR_UNSUPPORTED_SIZE, "plan: FFT factorisation"));
    f.tw64 = p->tw64 + off;
    f.tw32 = p->tw32 + off;
    f.twdf = p->twdf + off;
    f.lf64 = p->lf64 + off;
    k_twiddles<<<(lens[i] + 255) / 256, 256, 0, st>>>(p->tw64 + off, p->tw32 + off, p->twdf + off, p->lf64 + off,
                                                      lens[i]);
    count_launches(1);
    off += lens[i];
  }
  // ---- per-axis tables of the binary64 H and preconditioner passes (AxT):
  // nu_k / N, (nu_k^2 / 2) / N, nu_k^2 / 2 with nu_k = k' pi / L (k' the signed
  // index), and the coordinate x_i = -L + i h with x_i^2 / 2
  {
    const int Ns[3] = {g.Nx, g.Ny, g.Nz};
    const double Ls[3] = {g.Lx, g.Ly, g.Lz}, hs[3] = {g.hx, g.hy, g.hz};
    std::vector<double> tab;
    for (int ax = 0; ax < 3; ++ax) {
      const int n = Ns[ax];
      const double kap = kPi / Ls[ax], invn = 1.0 / (double)n;
      std::vector<double> nuN(n), kinN(n), hnu2(n), xc(n), hxc2(n);
      for (int k = 0; k < n; ++k) {
        const int kk = k < n / 2 ? k : k - n;
        const double nu = (double)kk * kap;
        nuN[k] = nu * invn;
        hnu2[k] = 0.5 * nu * nu;
        kinN[k] = hnu2[k] * invn;
        xc[k] = -Ls[ax] + (double)k * hs[ax];
        hxc2[k] = 0.5 * xc[k] * xc[k];
      }
      for (auto* v : {&nuN, &kinN, &hnu2, &xc, &hxc2}) tab.insert(tab.end(), v->begin(), v->end());
    }
    if ((e = dev_alloc(p, (void**)&p->axtab, tab.size() * sizeof(double))) != cudaSuccess)
      return bail(cuda_fail(nullptr, e, "plan axis tables"));
    if ((e = cudaMemcpyAsync(p->axtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return bail(cuda_fail(nullptr, e, "plan axis tables"));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan axis tables"));
  }
  // ---- U0 octant
  const double a[3] = {2.0 * L[0], 2.0 * L[1], 2.0 * L[2]};
  const double amin = std::min(a[0], std::min(a[1], a[2]));
  const double s_c = kEdge / amin;
  const double tau_lo = log(kSlo), tau_c = log(s_c);
  const int npan = std::max(1, (int)ceil((tau_c - tau_lo) / kTauPanel));
  const int Q = npan * kGL;
  std::vector<double> gx, gw;
  gauss_legendre(kGL, gx, gw);
  GLNodes gl01;
  for (int i = 0; i < kGL; ++i) {
    gl01.x[i] = 0.5 * (gx[i] + 1.0);
    gl01.w[i] = 0.5 * gw[i];
  }
  std::vector<double> s_nodes(Q), w_nodes(Q);
  const double wpan = (tau_c - tau_lo) / npan;
  for (int pnl = 0; pnl < npan; ++pnl)
    for (int i = 0; i < kGL; ++i) {
      const double tau = tau_lo + wpan * (pnl + gl01.x[i]);
      const double s = exp(tau);
      s_nodes[pnl * kGL + i] = s;
      w_nodes[pnl * kGL + i] = wpan * gl01.w[i] * s;  // ds = s dtau
    }
  const size_t n_oct = (size_t)(g.Nx + 1) * (g.Ny + 1) * (g.Nz + 1);
  if ((e = dev_alloc(p, (void**)&p->U0, n_oct * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan U0"));
  double *d_s = nullptr, *d_w = nullptr, *d_T[3] = {nullptr, nullptr, nullptr};
  auto free_tmp = [&]() {
    cudaFree(d_s); cudaFree(d_w);
    for (double* t : d_T) cudaFree(t);
  };
  e = cudaMalloc((void**)&d_s, Q * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_w, Q * sizeof(double));
  for (int ax = 0; ax < 3 && e == cudaSuccess; ++ax) e = cudaMalloc((void**)&d_T[ax], (size_t)Q * (N[ax] + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, s_nodes.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w_nodes.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    for (int ax = 0; ax < 3; ++ax) {
      const int tot = Q * (N[ax] + 1);
      k_axis_table<<<(tot + 127) / 128, 128, 0, st>>>(d_T[ax], d_s, Q, N[ax], a[ax], gl01);
    }
    k_U0<<<(int)std::min<size_t>((n_oct + 255) / 256, 65535), 256, 0, st>>>(p->U0, d_T[0], d_T[1], d_T[2], d_w, Q,
                                                                          g.Nx, g.Ny, g.Nz, a[0], a[1], a[2], s_c);
    count_launches(4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  free_tmp();
  if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan U0 precompute"));
  // ---- z-pass multiplier on the half spectrum (FP64; copies below)
  const size_t n_kz = (size_t)g.Mz * g.My * g.XS;
  if ((e = dev_alloc(p, (void**)&p->Kz, n_kz * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan Kz"));
  k_multiplier_half<<<(int)std::min<size_t>((n_kz + 255) / 256, 4096), 256, 0, st>>>(p->Kz, p->U0, g, p->n[0], p->n[1],
                                                                                     p->n[2]);
  count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan Kz"));
  // ---- workspaces
  const size_t Nt = (size_t)g.Nx * g.Ny * g.Nz;
  const size_t n_w1 = (size_t)g.Nz * g.Ny * g.XS, n_w2 = (size_t)g.Nz * g.My * g.XS;
  if ((e = dev_alloc(p, (void**)&p->W1, n_w1 * sizeof(double2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
  if ((e = dev_alloc(p, (void**)&p->W2, n_w2 * sizeof(double2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
  if ((e = dev_alloc(p, (void**)&p->T1, Nt * sizeof(double2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
  if ((e = dev_alloc(p, (void**)&p->Pw, Nt * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
  if (flags & ATKM_PLAN_F32) {
    if ((e = dev_alloc(p, (void**)&p->W1f, n_w1 * sizeof(float2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
    if ((e = dev_alloc(p, (void**)&p->W2f, n_w2 * sizeof(float2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
    if ((e = dev_alloc(p, (void**)&p->T1f, Nt * sizeof(float2))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan workspace"));
    if ((e = dev_alloc(p, (void**)&p->U0f, n_oct * sizeof(float))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan U0f"));
    k_to_f32<<<(int)std::min<size_t>((n_oct + 255) / 256, 4096), 256, 0, st>>>(p->U0f, p->U0, n_oct);
    count_launches(1);
  }
  if (flags & ATKM_PLAN_DF32) {
    if ((e = dev_alloc(p, (void**)&p->Kzd, n_kz * sizeof(df))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan Kzd"));
    k_to_df<<<(int)std::min<size_t>((n_kz + 255) / 256, 4096), 256, 0, st>>>(p->Kzd, p->Kz, n_kz);
    count_launches(1);
  }
  // reductions: the largest CTA count of a reducing pass, or the vector grid
  long maxb = 1216;
  maxb = std::max<long>(maxb, (long)g.Nz * g.Ny);           // x pass with T = 1
  maxb = std::max<long>(maxb, (long)g.Nz * g.Nx);           // y pass
  maxb = std::max<long>(maxb, (long)g.Ny * g.Nx);           // z pass
  p->partials_cap = (int)(16 * maxb);
  if ((e = dev_alloc(p, (void**)&p->partials, (size_t)p->partials_cap * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan partials"));
  if ((e = dev_alloc(p, (void**)&p->scal, SC_COUNT * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan scalars"));
  if ((e = cudaMallocHost((void**)&p->scal_host, SC_COUNT * sizeof(double))) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan scalars"));
  if ((e = cudaMemsetAsync(p->scal, 0, SC_COUNT * sizeof(double), st)) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan scalars"));
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(nullptr, e, "plan create"));
  if (flags & ATKM_PLAN_AUTOTUNE) {
    const int code = atkm_plan_autotune(p, stream);
    if (code != ATKM_OK) {
      const std::string msg = p->err;
      bail(code);
      return fail(nullptr, code, msg);
    }
  }
  *out = p;
  return ATKM_OK;
}

int atkm_plan_copy_U0(const atkm_plan* plan, double* dst, void* stream) {
  if (!plan || !dst) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_copy_U0: NULL argument");
  const size_t n_oct = (size_t)(plan->g.Nx + 1) * (plan->g.Ny + 1) * (plan->g.Nz + 1);
  cudaError_t e = cudaMemcpyAsync(dst, plan->U0, n_oct * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(nullptr, e, "atkm_plan_copy_U0");
}

int atkm_plan_copy_multiplier(const atkm_plan* plan, double* dst, void* stream) {
  if (!plan || !dst) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_copy_multiplier: NULL argument");
  k_multiplier_full<<<1216, 256, 0, (cudaStream_t)stream>>>(dst, plan->U0, plan->g, plan->n[0], plan->n[1], plan->n[2]);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ATKM_OK : cuda_fail(nullptr, e, "atkm_plan_copy_multiplier");
}

int dipolar_potential(atkm_plan* plan, const double* rho, double* phi, void* stream) {
  if (!plan || !rho || !phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential: NULL argument");
  if (rho == phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential: phi must not alias rho");
  cudaError_t e = launch_atkm<double>(plan, SRC_RHO, rho, nullptr, phi, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "dipolar_potential");
}

int dipolar_potential_from_psi(atkm_plan* plan, const double* psi, double* phi, void* stream) {
  if (!plan || !psi || !phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_psi: NULL argument");
  cudaError_t e = launch_atkm<double>(plan, SRC_PSI, psi, nullptr, phi, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "dipolar_potential_from_psi");
}

int dipolar_potential_from_pair(atkm_plan* plan, const double* a, const double* b, double* phi, void* stream) {
  if (!plan || !a || !b || !phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_pair: NULL argument");
  cudaError_t e = launch_atkm<double>(plan, SRC_PAIR, a, b, phi, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "dipolar_potential_from_pair");
}

int dipolar_potential_from_psi_f32(atkm_plan* plan, const double* psi, double* phi, void* stream) {
  if (!plan || !psi || !phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_psi_f32: NULL argument");
  if (!(plan->flags & ATKM_PLAN_F32)) return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_psi_f32: plan lacks ATKM_PLAN_F32");
  cudaError_t e = launch_atkm<float>(plan, SRC_PSI, psi, nullptr, phi, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "dipolar_potential_from_psi_f32");
}

int dipolar_potential_from_psi_df32(atkm_plan* plan, const double* psi, double* phi, void* stream) {
  if (!plan || !psi || !phi) return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_psi_df32: NULL argument");
  if (!(plan->flags & ATKM_PLAN_DF32))
    return fail(plan, ATKM_ERR_ARG, "dipolar_potential_from_psi_df32: plan lacks ATKM_PLAN_DF32");
  cudaError_t e = launch_atkm<df>(plan, SRC_PSI, psi, nullptr, phi, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "dipolar_potential_from_psi_df32");
}

int apply_H(atkm_plan* plan, const atkm_params* prm, const double* f, const double* phi, const double* Phi,
            double* Hf, void* stream) {
  if (!plan || !prm || !f || !phi || !Phi || !Hf) return fail(plan, ATKM_ERR_ARG, "apply_H: NULL argument");
  if (Hf == f || Hf == phi || Hf == Phi) return fail(plan, ATKM_ERR_ARG, "apply_H: output aliases an input");
  cudaError_t e = launch_H<double>(plan, make_phys(prm), f, phi, Phi, Hf, -1, (cudaStream_t)stream);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(plan, e, "apply_H");
}

int atkm_plan_set_profiling(atkm_plan* plan, int on) {
  if (!plan) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_set_profiling: NULL plan");
  if (on) {
    if (!plan->prof) {
      plan->prof = plan->prof_stopped_ ? plan->prof_stopped_ : new Profiler();
      plan->prof_stopped_ = nullptr;
    }
    cudaDeviceSynchronize();
    plan->prof->recs.clear();
    plan->prof->agg.clear();
    plan->prof->used = 0;
    plan->prof->open = false;
    plan->prof->sink = nullptr;
  } else if (plan->prof) {
    // keep the record for atkm_plan_kernel_stats; stop recording new launches
    delete plan->prof_stopped_;
    plan->prof_stopped_ = plan->prof;
    plan->prof = nullptr;
  }
  return ATKM_OK;
}

int atkm_plan_kernel_stats(atkm_plan* plan, atkm_kernel_stat* out, int capacity, int* count) {
  if (!plan || !count || (capacity > 0 && !out)) return fail(plan, ATKM_ERR_ARG, "atkm_plan_kernel_stats: NULL argument");
  Profiler* pr = plan->prof ? plan->prof : plan->prof_stopped_;
  *count = 0;
  if (!pr) return ATKM_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(plan, e, "atkm_plan_kernel_stats");
  std::vector<atkm_kernel_stat> agg;
  for (const auto& r : pr->recs) {
    if (!r.b) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int k = -1;
    for (size_t i = 0; i < agg.size(); ++i)
      if (strncmp(agg[i].name, r.name, sizeof(agg[i].name)) == 0) k = (int)i;
    if (k < 0) {
      atkm_kernel_stat st;
      memset(&st, 0, sizeof(st));
      strncpy(st.name, r.name, sizeof(st.name) - 1);
      agg.push_back(st);
      k = (int)agg.size() - 1;
    }
    agg[k].launches += 1;
    agg[k].ms_total += ms;
    agg[k].bytes_total += r.bytes;
    agg[k].flops_total += r.flops;
  }
  for (const auto& a : pr->agg) {
    int k = -1;
    for (size_t i = 0; i < agg.size(); ++i)
      if (strncmp(agg[i].name, a.name, sizeof(agg[i].name)) == 0) k = (int)i;
    if (k < 0) {
      atkm_kernel_stat st;
      memset(&st, 0, sizeof(st));
      strncpy(st.name, a.name, sizeof(st.name) - 1);
      agg.push_back(st);
      k = (int)agg.size() - 1;
    }
    agg[k].launches += (int)a.launches;
    agg[k].ms_total += a.ms;
    agg[k].bytes_total += a.bytes;
    agg[k].flops_total += a.flops;
  }
  *count = (int)agg.size();
  for (int i = 0; i < capacity && i < (int)agg.size(); ++i) out[i] = agg[i];
  return ATKM_OK;
}

int atkm_spectral_upsample(atkm_plan* coarse, atkm_plan* fine, const double* psi_c, double* psi_f, void* stream) {
  if (!coarse || !fine || !psi_c || !psi_f) return fail(nullptr, ATKM_ERR_ARG, "atkm_spectral_upsample: NULL argument");
  const Geo &gc = coarse->g, &gf = fine->g;
  const double Lc[3] = {gc.Lx, gc.Ly, gc.Lz}, Lf[3] = {gf.Lx, gf.Ly, gf.Lz};
  const int Nc[3] = {gc.Nx, gc.Ny, gc.Nz}, Nf[3] = {gf.Nx, gf.Ny, gf.Nz};
  for (int a = 0; a < 3; ++a) {
    if (fabs(Lc[a] - Lf[a]) > 1e-12 * Lc[a])
      return fail(fine, ATKM_ERR_ARG, "atkm_spectral_upsample: coarse and fine plans must share the box");
    if (Nf[a] < Nc[a]) return fail(fine, ATKM_ERR_ARG, "atkm_spectral_upsample: fine grid must not be coarser");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nc = (size_t)gc.Nx * gc.Ny * gc.Nz;
  cudaError_t e = cudaMemcpyAsync(coarse->T1, psi_c, nc * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_cfft3<double>(coarse, coarse->T1, -1, st);
  if (e == cudaSuccess) {
    k_embed_spectrum<<<1216, 256, 0, st>>>(coarse->T1, reinterpret_cast<double2*>(psi_f), gc, gf, 1.0 / (double)nc);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_cfft3<double>(fine, reinterpret_cast<double2*>(psi_f), 1, st);
  return e == cudaSuccess ? ATKM_OK : cuda_fail(fine, e, "atkm_spectral_upsample");
}

}  // extern "C"
