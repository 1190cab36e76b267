// FFT-tile autotuner.  Without it, a pass's engine and tile width follow a
// fixed rule (ops.cuh, pass_grid): the power-of-two register engine where the
// line length allows it, else the mixed-radix register engine (3 * 2^a, and
// 5 * 2^a outside binary64), else the generic shared-memory engine at a tile
// width narrowed until the pass has two CTAs per SM.  The tuner replaces the
// rule by measurement for every line length of the plan that is not a power
// of two, per arithmetic the plan carries (binary64, and FP32 / double-word
// with ATKM_PLAN_F32 / ATKM_PLAN_DF32) and per layout (the line-major x pass,
// the strided y and z passes).  Candidates: the mixed-radix register engine
// where run_pass instantiates it (3 * 2^a and 5 * 2^a up to 384 in FP32,
// 3 * 2^a in binary64, none in double-word) and the
// generic engine at its default tile width, half of it and a quarter of it.
// Each candidate is timed on the plan's own operators -- the ATKM of |psi|^2,
// H psi and P r (no preconditioner in double-word) -- with CUDA events, the
// best of three runs after a warm-up, while every other length keeps its
// current choice; lengths are tuned one after another in the order x, then
// the padded and unpadded y and z lengths.  Timing and selection support of
// the library; the paper has no counterpart.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "atkm_internal.cuh"
#include "ops.cuh"

namespace atkm {
namespace {

struct Scratch {
  double* psi = nullptr;
  double* Phi = nullptr;
  double* out = nullptr;
  double* alpha = nullptr;
  ~Scratch() {
    if (psi) cudaFree(psi);
    if (Phi) cudaFree(Phi);
    if (out) cudaFree(out);
    if (alpha) cudaFree(alpha);
  }
};

// The operator set of arithmetic r on the scratch state.
cudaError_t run_ops(atkm_plan* p, int r, const Phys& ph, const Scratch& s, cudaStream_t st) {
  cudaError_t e;
  if (r == 0) {
    e = launch_atkm<double>(p, SRC_PSI, s.psi, nullptr, s.Phi, st);
    if (e == cudaSuccess) e = launch_H<double>(p, ph, s.psi, s.psi, s.Phi, s.out, -1, st);
    if (e == cudaSuccess) e = launch_precond<double>(p, ph, s.alpha, s.psi, s.psi, s.Phi, s.out, st);
  } else if (r == 1) {
    e = launch_atkm<float>(p, SRC_PSI, s.psi, nullptr, s.Phi, st);
    if (e == cudaSuccess) e = launch_H<float>(p, ph, s.psi, s.psi, s.Phi, s.out, -1, st);
    if (e == cudaSuccess) e = launch_precond<float>(p, ph, s.alpha, s.psi, s.psi, s.Phi, s.out, st);
  } else {
    e = launch_atkm<df>(p, SRC_PSI, s.psi, nullptr, s.Phi, st);
    if (e == cudaSuccess) e = launch_H<df>(p, ph, s.psi, s.psi, s.Phi, s.out, -1, st);
  }
  return e;
}

// Best of three timed runs after one warm-up, milliseconds.
cudaError_t time_ops(atkm_plan* p, int r, const Phys& ph, const Scratch& s, cudaStream_t st, cudaEvent_t a,
                     cudaEvent_t b, double* ms_out) {
  double best = 1e300;
  cudaError_t e = run_ops(p, r, ph, s, st);
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = run_ops(p, r, ph, s, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) best = std::min(best, (double)ms);
  }
  *ms_out = best;
  return e;
}

bool default_mix(const atkm_plan* p, int r, int L) {
  return !(p->flags & ATKM_PLAN_GENERIC_FFT) && mix_ok_r(r, L);
}

}  // namespace
}  // namespace atkm

using namespace atkm;

extern "C" {

int atkm_plan_autotune(atkm_plan* plan, void* stream) {
  if (!plan) return fail(nullptr, ATKM_ERR_ARG, "atkm_plan_autotune: plan is NULL");
  if (plan->pcg) return fail(plan, ATKM_ERR_ARG, "atkm_plan_autotune: call it before the plan's first PCG solve");
  cudaStream_t st = (cudaStream_t)stream;
  const Geo& g = plan->g;
  const size_t N = (size_t)g.Nx * g.Ny * g.Nz;
  Scratch s;
  cudaError_t e = cudaMalloc((void**)&s.psi, N * 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s.Phi, N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s.out, N * 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&s.alpha, sizeof(double));
  // every byte 0x3f: each double about 4.8e-4 (normal, positive)
  if (e == cudaSuccess) e = cudaMemsetAsync(s.psi, 0x3f, N * 2 * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.alpha, 0x3f, sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(plan, e, "atkm_plan_autotune: scratch");
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  Phys ph{};
  ph.gx2 = ph.gy2 = 1.0;
  ph.gz2 = 4.0;
  ph.beta = 100.0;
  ph.lambda = 50.0;
  ph.Omega = 0.5;
  // the lengths and layouts of the plan's passes (ATKM x, y, z; H and P x, y, z)
  const int keyL[5] = {g.Nx, g.My, g.Mz, g.Ny, g.Nz};
  const int keyLM[5] = {1, 0, 0, 0, 0};
  plan->n_tune = 0;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    if ((r == 1 && !(plan->flags & ATKM_PLAN_F32)) || (r == 2 && !(plan->flags & ATKM_PLAN_DF32))) continue;
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
      const int L = keyL[k], lm = keyLM[k];
      if (fast_len(L)) continue;
      bool seen = false;
      for (int i = 0; i < plan->n_tune; ++i)
        seen = seen || (plan->tune[i].r == r && plan->tune[i].L == L && plan->tune[i].lm == lm);
      if (seen || plan->n_tune >= kMaxTune) continue;
      std::vector<std::pair<int, int>> cand;
      if (!(plan->flags & ATKM_PLAN_GENERIC_FFT) && mix_ok_r(r, L)) cand.push_back({1, 0});
      for (int sh = 0; sh <= 2; ++sh) cand.push_back({0, sh});
      TuneEntry& te = plan->tune[plan->n_tune++];
      te.r = r;
      te.L = L;
      te.lm = lm;
      const int dmix = default_mix(plan, r, L) ? 1 : 0;
      double best = 1e300, dflt = 0.0;
      int bmix = dmix, bshift = 0;
      for (const auto& c : cand) {
        te.mix = c.first;
        te.shift = c.second;
        double ms = 0.0;
        e = time_ops(plan, r, ph, s, st, a, b, &ms);
        if (e != cudaSuccess) break;
        if (c.first == dmix && c.second == 0) dflt = ms;
        if (ms < best) {
          best = ms;
          bmix = c.first;
          bshift = c.second;
        }
      }
      te.mix = bmix;
      te.shift = bshift;
      te.ms_default = dflt;
      te.ms_best = best;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) {
    plan->n_tune = 0;
    return cuda_fail(plan, e, "atkm_plan_autotune");
  }
  return ATKM_OK;
}

int atkm_plan_tuning(const atkm_plan* plan, atkm_tune_info* out, int cap) {
  if (!plan || (cap > 0 && !out)) return -ATKM_ERR_ARG;
  for (int i = 0; i < plan->n_tune && i < cap; ++i) {
    const TuneEntry& t = plan->tune[i];
    atkm_tune_info& o = out[i];
    memset(&o, 0, sizeof(o));
    o.precision = t.r;
    o.length = t.L;
    o.line_major = t.lm;
    o.engine = t.mix ? 1 : 2;
    o.tile_shift = t.mix ? 0 : t.shift;
    o.ms_default = t.ms_default;
    o.ms_best = t.ms_best;
  }
  return plan->n_tune;
}

}  // extern "C"
