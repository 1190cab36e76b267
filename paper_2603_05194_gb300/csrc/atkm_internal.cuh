// Internal declarations of the GB300 PCG-ATKM library: complex helpers, the
// batched line-FFT engine, the plan structure and the launchers shared by the
// translation units.  Not part of the public interface (see include/atkm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/atkm.h"
#include "df32.cuh"

namespace atkm {

// ---------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<double> { using c = double2; };
template <> struct CT<float> { using c = float2; };
template <> struct CT<df> { using c = cdf; };
template <typename R> using cx = typename CT<R>::c;

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> z; z.x = a; z.y = b; return z;
}
// binary64 <-> binary32 conversions on the integer pipe from the IEEE-754 bit
// layouts (the hardware conversion instructions share the slow FP64 pipe on
// this part; each FP32 pass uses these, the hardware or a mix, whichever was
// measured faster for it: see from64 in ops.cuh).  binary64 -> binary32 rounds the 29
// dropped mantissa bits half-up (a mantissa carry moves into the exponent),
// flushes results below the binary32 normal range to signed zero and
// saturates to infinity (a NaN becomes an infinity); binary32 -> binary64 is
// exact for normal numbers and flushes binary32 subnormals to signed zero.
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned int hi = (unsigned int)__double2hiint(d), lo = (unsigned int)__double2loint(d);
  // the high word with the exponent rebased to binary32: (e32 << 20) | the
  // top 20 mantissa bits; e32 <= 0 flushes, e32 >= 255 saturates (a NaN
  // becomes an infinity)
  int a = (int)(hi & 0x7fffffffu) - 0x38000000;
  const bool tiny = a < 0x00100000;
  a = min(a, 0x0ff00000);
  // (a:lo) + 2^28 rounds the 29 dropped bits half-up; bits 29..60 are the result
  const unsigned int lr = lo + 0x10000000u;
  const unsigned int ar = (unsigned int)a + (lr < lo ? 1u : 0u);
  unsigned int bits = min(__funnelshift_r(lr, ar, 29), 0x7f800000u);
  bits = tiny ? 0u : bits;
  return __uint_as_float(bits | (hi & 0x80000000u));
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sign = u & 0x80000000u;
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned int m = u & 0x7fffffu;
  unsigned int hi, lo;
  if (e == 0u) { hi = sign; lo = 0u; }
  else if (e == 255u) { hi = sign | 0x7ff00000u | (m >> 3); lo = (m & 7u) << 29; }
  else { hi = sign | ((e + 896u) << 20) | (m >> 3); lo = (m & 7u) << 29; }
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
template <typename R> __device__ __forceinline__ R tor(double v);
template <> __device__ __forceinline__ double tor<double>(double v) { return v; }
template <> __device__ __forceinline__ float tor<float>(double v) { return d2f_bits(v); }
template <typename R> __device__ __forceinline__ double tod(R v);
template <> __device__ __forceinline__ double tod<double>(double v) { return v; }
template <> __device__ __forceinline__ double tod<float>(float v) { return f2d_bits(v); }
// binary64 <-> double-word: the leading binary32 part from the bit layout, the
// trailing part from the exact binary64 remainder (one binary64 subtraction).
template <> __device__ __forceinline__ df tor<df>(double v) {
  const float h = d2f_bits(v);
  return df(h, d2f_bits(v - f2d_bits(h)));
}
template <> __device__ __forceinline__ double tod<df>(df v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }

template <typename R> __device__ __forceinline__ cx<R> add(cx<R> a, cx<R> b) {
  if constexpr (std::is_same<R, df>::value) return df_cadd(a, b);
  else return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R> __device__ __forceinline__ cx<R> sub(cx<R> a, cx<R> b) {
  if constexpr (std::is_same<R, df>::value) return df_csub(a, b);
  else return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R> __device__ __forceinline__ cx<R> scl(cx<R> a, R s) {
  if constexpr (std::is_same<R, df>::value) return df_cscl(a, s);
  else return mk<R>(a.x * s, a.y * s);
}
// a * b
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  if constexpr (std::is_same<R, df>::value) return df_cmul(a, b, false);
  else return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  if constexpr (std::is_same<R, df>::value) return df_cmul(a, b, true);
  else return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// s * i * a  (s = +1 or -1)
template <typename R, int S> __device__ __forceinline__ cx<R> mul_si(cx<R> a) {
  return S > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}

// Number of SMs of the current device, queried once per device ordinal and
// cached; 0 when the query fails (callers then size their grids without it).
inline int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 0;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// ------------------------------------------------------------- FFT engine
// A CTA transforms T lines of length L held in shared memory.  Stockham
// auto-sort formulation (Govindaraju et al., "High performance discrete
// Fourier transforms on graphics processors", SC'08): stage s with radix R
// reads element j + r L/R, applies the twiddle w^{(j mod Ns) r} with
// w = e^{sign 2 pi i/(Ns R)}, does an R-point DFT in registers and writes
// element (j - j mod Ns) R + j mod Ns + r Ns.  All butterflies of a stage are
// read into registers before any is written (one shared buffer).
constexpr int kThreads = 256;      // threads per FFT CTA
constexpr int kMaxElems = 4096;    // complex elements per CTA tile (upper bound)
// Tile size per arithmetic type: 8 complex doubles or 16 complex floats per
// thread keep a stage's butterflies in registers without spilling.
template <typename R> struct TileElems;
template <> struct TileElems<double> { static constexpr int value = 2048; };
template <> struct TileElems<float> { static constexpr int value = 4096; };
template <> struct TileElems<df> { static constexpr int value = 2048; };
constexpr int kMaxStages = 12;
constexpr int kMaxLen = 2048;     // longest (padded) line; <= TileElems<double>

struct FftLen {
  int L;
  int nstages;
  int radix[kMaxStages];
  const double2* tw64;  // e^{-2 pi i m / L}, m = 0..L-1
  const float2* tw32;
  const cdf* twdf;      // the binary64 table split into double-word
  const double2* lf64;  // tw64 in multiply-add form (m, t), see lf_cform
};

// Multiply-add form of the twiddle W_j = e^{-2 pi i j / L} = c + i s: with
// |t| <= 1, W_j = m (1 + i t) (m = c, t = s / c) when |c| >= |s| (the
// "c-form"), else W_j = m (t + i) (m = s, t = c / s).  The form follows from j
// alone: |c| >= |s| exactly when q = j mod L/2 lies in [0, L/8] or [3L/8, L/2).
__host__ __device__ __forceinline__ bool lf_cform(int j, int L) {
  const int q = j % (L >> 1);
  return 8 * q <= L || 8 * q >= 3 * L;
}

template <typename R> __host__ __device__ __forceinline__ const cx<R>* tw_table(const FftLen& f);
template <> __host__ __device__ __forceinline__ const double2* tw_table<double>(const FftLen& f) { return f.tw64; }
template <> __host__ __device__ __forceinline__ const float2* tw_table<float>(const FftLen& f) { return f.tw32; }
template <> __host__ __device__ __forceinline__ const cdf* tw_table<df>(const FftLen& f) { return f.twdf; }
template <typename R> inline const cx<R>* tw_table_host(const FftLen& f) { return tw_table<R>(f); }

// Exact trigonometric constants of the small DFTs (closed forms in radicals).
#define ATKM_SQRT1_2 0.70710678118654752440084436210485
#define ATKM_SIN60 0.86602540378443864676372317075294
#define ATKM_C72 0.30901699437494742410229341718282    /* cos(2pi/5) = (sqrt5-1)/4 */
#define ATKM_C144 (-0.80901699437494742410229341718282) /* cos(4pi/5) = -(sqrt5+1)/4 */
#define ATKM_S72 0.95105651629515357211643933337938    /* sin(2pi/5) */
#define ATKM_S144 0.58778525229247312916870595463907   /* sin(4pi/5) */

// In-register R-point DFT, X_q = sum_r v_r e^{S 2 pi i r q / R}.
template <typename R, int RAD, int S> struct Dft;

// run: the full DFT.  run_zu: inputs in the upper half are zero (the zero
// padding of a forward transform) and are not read.  run_lo: only outputs in
// the lower half are formed (the crop after an inverse transform); the others
// are left unspecified.
template <typename R, int S> struct Dft<R, 2, S> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> a = v[0], b = v[1];
    v[0] = add<R>(a, b); v[1] = sub<R>(a, b);
  }
  static __device__ __forceinline__ void run_lo(cx<R>* v) { v[0] = add<R>(v[0], v[1]); }
};
template <typename R, int S> struct Dft<R, 4, S> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> a = add<R>(v[0], v[2]), b = sub<R>(v[0], v[2]);
    cx<R> c = add<R>(v[1], v[3]), d = mul_si<R, S>(sub<R>(v[1], v[3]));
    v[0] = add<R>(a, c); v[2] = sub<R>(a, c);
    v[1] = add<R>(b, d); v[3] = sub<R>(b, d);
  }
  static __device__ __forceinline__ void run_zu(cx<R>* v) {  // v[2] = v[3] = 0
    const cx<R> a = v[0], c = v[1], d = mul_si<R, S>(v[1]);
    v[0] = add<R>(a, c); v[2] = sub<R>(a, c);
    v[1] = add<R>(a, d); v[3] = sub<R>(a, d);
  }
  static __device__ __forceinline__ void run_lo(cx<R>* v) {  // v[0], v[1] only
    cx<R> a = add<R>(v[0], v[2]), b = sub<R>(v[0], v[2]);
    cx<R> c = add<R>(v[1], v[3]), d = mul_si<R, S>(sub<R>(v[1], v[3]));
    v[0] = add<R>(a, c); v[1] = add<R>(b, d);
  }
};
template <typename R, int S> struct Dft<R, 8, S> {
  template <bool ZU, bool LO>
  static __device__ __forceinline__ void go(cx<R>* v) {
    cx<R> e[4] = {v[0], v[2], v[4], v[6]};
    cx<R> o[4] = {v[1], v[3], v[5], v[7]};
    if (ZU) {
      Dft<R, 4, S>::run_zu(e);
      Dft<R, 4, S>::run_zu(o);
    } else {
      Dft<R, 4, S>::run(e);
      Dft<R, 4, S>::run(o);
    }
    const R c = (R)ATKM_SQRT1_2;
    // o_q *= e^{S i pi q / 4}
    cx<R> o1 = mk<R>(c * (o[1].x - S * o[1].y), c * (o[1].y + S * o[1].x));
    cx<R> o2 = mul_si<R, S>(o[2]);
    cx<R> o3 = mk<R>(-c * (o[3].x + S * o[3].y), c * (S * o[3].x - o[3].y));
    v[0] = add<R>(e[0], o[0]);
    v[1] = add<R>(e[1], o1);
    v[2] = add<R>(e[2], o2);
    v[3] = add<R>(e[3], o3);
    if (!LO) {
      v[4] = sub<R>(e[0], o[0]);
      v[5] = sub<R>(e[1], o1);
      v[6] = sub<R>(e[2], o2);
      v[7] = sub<R>(e[3], o3);
    }
  }
  static __device__ __forceinline__ void run(cx<R>* v) { go<false, false>(v); }
  static __device__ __forceinline__ void run_zu(cx<R>* v) { go<true, false>(v); }
  static __device__ __forceinline__ void run_lo(cx<R>* v) { go<false, true>(v); }
};
template <typename R, int S> struct Dft<R, 3, S> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> t1 = add<R>(v[1], v[2]);
    cx<R> t2 = mul_si<R, S>(scl<R>(sub<R>(v[1], v[2]), (R)ATKM_SIN60));
    cx<R> m = sub<R>(v[0], scl<R>(t1, (R)0.5));
    v[0] = add<R>(v[0], t1);
    v[1] = add<R>(m, t2);
    v[2] = sub<R>(m, t2);
  }
};
template <typename R, int S> struct Dft<R, 5, S> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> a1 = add<R>(v[1], v[4]), b1 = sub<R>(v[1], v[4]);
    cx<R> a2 = add<R>(v[2], v[3]), b2 = sub<R>(v[2], v[3]);
    const R c1 = (R)ATKM_C72, c2 = (R)ATKM_C144, s1 = (R)ATKM_S72, s2 = (R)ATKM_S144;
    cx<R> m1 = mk<R>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    cx<R> m2 = mk<R>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    cx<R> n1 = mul_si<R, S>(mk<R>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    cx<R> n2 = mul_si<R, S>(mk<R>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = mk<R>(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
    v[1] = add<R>(m1, n1); v[4] = sub<R>(m1, n1);
    v[2] = add<R>(m2, n2); v[3] = sub<R>(m2, n2);
  }
};

// Element (t, j) of the tile: line-major tiles keep lines contiguous (x
// lines), column tiles keep the T columns of one position contiguous.
template <bool LM> __device__ __forceinline__ int tix(int t, int j, int T, int L) {
  return LM ? t * L + j : j * T + t;
}

template <typename R, int RAD, int S, bool LM>
__device__ __forceinline__ void fft_stage(cx<R>* buf, const cx<R>* tw, int L, int T, int Ns) {
  constexpr int NB = (TileElems<R>::value + RAD * kThreads - 1) / (RAD * kThreads);
  const int nb = L / RAD;
  const int total = nb * T;
  const int tws = L / (Ns * RAD);
  cx<R> v[NB][RAD];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * kThreads;
    if (b < total) {
      int t, j;
      if (LM) { t = b / nb; j = b - t * nb; } else { j = b / T; t = b - j * T; }
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[i][r] = buf[tix<LM>(t, j + r * nb, T, L)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * kThreads;
    if (b < total) {
      int t, j;
      if (LM) { t = b / nb; j = b - t * nb; } else { j = b / T; t = b - j * T; }
      const int k = j % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          cx<R> w = tw[k * r * tws];
          v[i][r] = (S < 0) ? cmul<R>(v[i][r], w) : cmulc<R>(v[i][r], w);
        }
      }
      Dft<R, RAD, S>::run(v[i]);
      const int base = (j - k) * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[tix<LM>(t, base + r * Ns, T, L)] = v[i][r];
    }
  }
  __syncthreads();
}

// Transforms all T lines of the tile (forward S = -1, inverse S = +1,
// unnormalised).  Caller has synchronised after filling the tile; returns
// synchronised.
template <typename R, int S, bool LM>
__device__ __forceinline__ void fft_tile(cx<R>* buf, const cx<R>* tw, const FftLen& f, int T) {
  int Ns = 1;
  for (int s = 0; s < f.nstages; ++s) {
    const int rad = f.radix[s];
    switch (rad) {
      case 8: fft_stage<R, 8, S, LM>(buf, tw, f.L, T, Ns); break;
      case 4: fft_stage<R, 4, S, LM>(buf, tw, f.L, T, Ns); break;
      case 2: fft_stage<R, 2, S, LM>(buf, tw, f.L, T, Ns); break;
      case 3: fft_stage<R, 3, S, LM>(buf, tw, f.L, T, Ns); break;
      default: fft_stage<R, 5, S, LM>(buf, tw, f.L, T, Ns); break;
    }
    Ns *= rad;
  }
}

// Copies the twiddle table of f into shared memory (no sync).
template <typename R> __device__ __forceinline__ void load_tw(cx<R>* dst, const FftLen& f) {
  const cx<R>* src = tw_table<R>(f);
  for (int i = threadIdx.x; i < f.L; i += kThreads) dst[i] = src[i];
}

// Block-wide sum of NS doubles; thread 0 writes part[s * stride + slot].
template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NS], double* part, int stride, int slot) {
  __shared__ double red[NS][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double v = acc[s];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[s][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double v = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) v += red[s][w];
      part[s * stride + slot] = v;
    }
  }
}

// The same for FP32 per-thread partials: the warp stage shuffles and adds in
// FP32 (a 32-term sum, about 5 roundings), each warp's sum is widened once,
// and the block stage adds in FP64 -- so no per-thread FP64 work is done in
// FP32 kernels (the FP64 pipe is slow on this part).
template <int NS>
__device__ __forceinline__ void block_reduce_store_f32(float (&acc)[NS], double* part, int stride, int slot) {
  __shared__ double red[NS][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    float v = acc[s];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[s][warp] = tod<float>(v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double v = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) v += red[s][w];
      part[s * stride + slot] = v;
    }
  }
}

// ---------------------------------------------------------------- plan
struct Geo {
  int Nx, Ny, Nz, Mx, My, Mz;
  int Xh;  // Nx + 1: x-frequencies 0..Nx kept by the real-data ATKM transform
  int XS;  // row stride of the half-spectrum workspaces (Xh rounded up to 16)
  double Lx, Ly, Lz, hx, hy, hz;
};

struct Phys {  // physical parameters passed by value to kernels
  double gx2, gy2, gz2;  // gamma^2
  double beta, lambda, Omega;
};

struct PcgBuffers;  // defined in pcg.cu
struct Profiler;    // defined in plan.cu

// One choice of the FFT-tile autotuner (tune.cu): for the arithmetic r (0
// binary64, 1 FP32, 2 double-word), the line length L and the layout lm (1:
// line-major x pass, 0: strided pass), the engine (mix = 1: the mixed-radix
// register engine, else the generic shared-memory engine with its default
// tile width shifted right by `shift`), with the timed operator set's
// milliseconds under the default rule and under this choice.
struct TuneEntry {
  int r, L, lm, mix, shift;
  double ms_default, ms_best;
};
constexpr int kMaxTune = 48;

}  // namespace atkm

// Scalar slots in plan->scal (device) and their host mirror.
enum {
  SC_ALPHA = 0,
  SC_RED = 8,     // reduction outputs start here
  SC_COUNT = 128
};

struct atkm_plan {
  atkm::Geo g;
  double n[3];
  unsigned flags;
  double hvol;
  atkm::FftLen fN[3];  // unpadded lengths N_x, N_y, N_z
  atkm::FftLen fM[3];  // padded lengths 2N_x, 2N_y, 2N_z
  double2* tw64;       // twiddle pool
  float2* tw32;
  double2* lf64;       // binary64 twiddles in multiply-add form
  double* U0;          // octant (Nz+1)(Ny+1)(Nx+1)
  float* U0f;          // FP32 copy of U0 (FP32 workspaces only)
  double* Kz;          // z-pass multiplier K_sym / (Mx My Mz), [Mz][My][XS] half spectrum
  double* axtab;       // per-axis tables (AxT): for a = x, y, z five arrays of N_a doubles
  double* Pw;          // [Nz][Ny][Nx] preconditioner weights, binary64 passes
  atkm::df* Kzd;       // double-word copy of Kz (ATKM_PLAN_DF32 only)
  atkm::cdf* twdf;     // double-word twiddle pool
  double2* W1;         // [Nz][Ny][XS] half spectrum in x
  double2* W2;         // [Nz][My][XS]
  double2* T1;         // [Nz][Ny][Nx]
  float2* W1f;
  float2* W2f;
  float2* T1f;
  double* partials;    // reduction partials
  int partials_cap;    // doubles
  double* scal;        // device scalars
  double* scal_host;   // pinned mirror
  atkm::PcgBuffers* pcg;
  atkm::TuneEntry tune[atkm::kMaxTune];  // autotuned engine choices (n_tune of them)
  int n_tune;
  atkm::Profiler* prof;  // non-null while profiling is on
  atkm::Profiler* prof_stopped_;  // last record after profiling was switched off
  unsigned long long bytes;
  std::string err;
};

namespace atkm {

extern thread_local std::string g_last_error;

int fail(atkm_plan* p, int code, const std::string& msg);
int cuda_fail(atkm_plan* p, cudaError_t e, const char* where);
cudaError_t dev_alloc(atkm_plan* p, void** ptr, size_t bytes);

// Process-wide count of kernel launches issued by the library.
void count_launches(int n);

// Profiling hooks: no-ops unless profiling is on.  `name` must be a literal.
void prof_begin(atkm_plan* p, const char* name, double bytes, double flops, cudaStream_t st);
void prof_end(atkm_plan* p, cudaStream_t st);

// Event pair of one pass launch recorded into a captured CUDA graph; every
// replay re-records the same events.  The owner destroys the events.
struct ProfRec {
  const char* name;
  double bytes, flops;
  cudaEvent_t a, b;
};
// While a sink is set, prof_begin/prof_end record into it with fresh events
// (for graph capture) instead of the plan's eager record.
void prof_set_sink(atkm_plan* p, std::vector<ProfRec>* sink);
// Adds the elapsed times of a replayed graph's records to the plan's totals
// (call after the replay has completed).
void prof_accumulate(atkm_plan* p, const std::vector<ProfRec>& recs);

// Launchers (passes.cu).  All enqueue on `st`.
enum AtkmSrc { SRC_RHO = 0, SRC_PSI = 1, SRC_PAIR = 2 };
template <typename R>
cudaError_t launch_atkm(atkm_plan* p, int mode, const double* a, const double* b, double* phi,
                        cudaStream_t st);
// H f; if red_slot >= 0 the per-pass energy reductions go to partials and are
// finalised into scal[red_slot .. red_slot + 9].
template <typename R>
cudaError_t launch_H(atkm_plan* p, const Phys& ph, const double* f, const double* phi,
                     const double* Phi, double* Hf, int red_slot, cudaStream_t st);
template <typename R>
cudaError_t launch_precond(atkm_plan* p, const Phys& ph, const double* alpha_dev, const double* r,
                           const double* phi, const double* Phi, double* Pr, cudaStream_t st);

template <typename R> cudaError_t launch_cfft3(atkm_plan* p, cx<R>* buf, int sign, cudaStream_t st);

// Reductions (pcg.cu)
cudaError_t launch_finalize(atkm_plan* p, int nslots, int nblocks, int dst_slot, cudaStream_t st);

Phys make_phys(const atkm_params* prm);

}  // namespace atkm
