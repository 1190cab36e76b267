// Pass layer of the spectral operators: each axis pass of ATKM, H_phi f and
// the preconditioner is an "op" (load / spectral multiply / store, with fused
// reductions) run by one of two line-FFT engines:
//   * FastFft: power-of-two lengths 16..1024 known at compile time; each
//     thread keeps 8 elements of one line in registers, radix-8 Stockham
//     stages (plus one radix-2/4 stage) exchange through padded, double-
//     buffered shared memory with one barrier per stage, and the spectral
//     multiply runs on the registers between forward and inverse transforms;
//   * the generic shared-memory engine of atkm_internal.cuh for the other
//     {2,3,5}-smooth lengths.
// A line is addressed by (o, x): line-major (x-axis) passes use o = line
// index (z N_y + y); strided passes use o = the outer index (blockIdx.y) and
// x = the column, T adjacent columns per CTA so global accesses coalesce.
#pragma once

#include <math.h>

#include <atomic>
#include <type_traits>

#include "atkm_internal.cuh"

namespace atkm {

// ------------------------------------------------------------ constants
template <typename R> struct Cst {
  int Nx, Ny, Nz, Mx, My, Mz;
  R kx, ky, kz;     // pi / L_a: nu of an unpadded frequency index
  R pkx, pky, pkz;  // pi / (2 L_a): nu of a padded frequency index
  R Lx, Ly, Lz, hx, hy, hz;
};

template <typename R> inline Cst<R> make_cst(const Geo& g) {
  const double pi = 3.14159265358979323846264338327950288;
  Cst<R> c;
  c.Nx = g.Nx; c.Ny = g.Ny; c.Nz = g.Nz; c.Mx = g.Mx; c.My = g.My; c.Mz = g.Mz;
  c.kx = (R)(pi / g.Lx); c.ky = (R)(pi / g.Ly); c.kz = (R)(pi / g.Lz);
  c.pkx = (R)(pi / (2.0 * g.Lx)); c.pky = (R)(pi / (2.0 * g.Ly)); c.pkz = (R)(pi / (2.0 * g.Lz));
  c.Lx = (R)g.Lx; c.Ly = (R)g.Ly; c.Lz = (R)g.Lz; c.hx = (R)g.hx; c.hy = (R)g.hy; c.hz = (R)g.hz;
  return c;
}

// Per-axis tables of a plan (binary64, length N_a each), used by the binary64
// H and preconditioner passes instead of forming the same values from integer
// indices at every grid point (each index conversion and product is an
// FP64-pipe instruction there): nu_k / N_a, (nu_k^2 / 2) / N_a, nu_k^2 / 2,
// the coordinate -L_a + i h_a and half its square.
struct AxT {
  const double* nuN;
  const double* kinN;
  const double* hnu2;
  const double* xc;
  const double* hxc2;
};

template <typename R> struct PhysR {
  R gx2, gy2, gz2, beta, lambda, Omega;
};
template <typename R> inline PhysR<R> make_physr(const Phys& p) {
  PhysR<R> q;
  q.gx2 = (R)p.gx2; q.gy2 = (R)p.gy2; q.gz2 = (R)p.gz2;
  q.beta = (R)p.beta; q.lambda = (R)p.lambda; q.Omega = (R)p.Omega;
  return q;
}

__device__ __forceinline__ int kfreq(int m, int M) { return m < (M >> 1) ? m : m - M; }
__device__ __forceinline__ int iabs(int a) { return a < 0 ? -a : a; }

// binary64 <-> binary32 at a pass's FP64 interfaces, three ways: on the
// integer pipe (d2f_bits / f2d_bits), with the hardware conversion (it issues
// on the FP64 pipe), or mixed: the real part in hardware, the imaginary part
// on the integer pipe.  The hardware instruction is the shorter dependency
// chain, the integer routine leaves the FP64 pipe free; which wins depends on
// how many conversions a pass makes per element, and each op below uses the
// way measured fastest for it at 256x256x64 (FP32 H x pass 40.7 -> 30.7 us
// mixed, H y 45.5 -> 38.8 us in hardware, H z 65.1 -> 63.2 us mixed; the
// ATKM x forward pass, four conversions an element, stays on the integer
// pipe).  Both round to nearest for finite values (ties away from zero on the
// integer pipe, to even in hardware).
enum CvtMode { kCvtInt = 0, kCvtMixed = 1, kCvtHw = 2 };
template <typename R, int CV = kCvtInt> __device__ __forceinline__ cx<R> from64(double2 z) {
  if constexpr (std::is_same<R, float>::value && CV == kCvtHw) {
    return mk<R>(__double2float_rn(z.x), __double2float_rn(z.y));
  } else if constexpr (std::is_same<R, float>::value && CV == kCvtMixed) {
    return mk<R>(__double2float_rn(z.x), d2f_bits(z.y));
  } else {
    return mk<R>(tor<R>(z.x), tor<R>(z.y));
  }
}
template <typename R, int CV = kCvtInt> __device__ __forceinline__ double2 to64(R a, R b) {
  if constexpr (std::is_same<R, float>::value && CV == kCvtHw) {
    return make_double2((double)a, (double)b);
  } else if constexpr (std::is_same<R, float>::value && CV == kCvtMixed) {
    return make_double2((double)a, f2d_bits(b));
  } else {
    return make_double2(tod<R>(a), tod<R>(b));
  }
}

// Loads of a pass's read-only inputs through the non-coherent path, so that
// the compiler may issue them ahead of the thread's earlier stores (a pass's
// inputs never alias its outputs): an epilogue then waits for one memory
// round trip, not one per element.
__device__ __forceinline__ double2 ldro(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldro(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double ldro(const double* p) { return __ldg(p); }
__device__ __forceinline__ cdf ldro(const cdf* p) {  // (x.hi, x.lo, y.hi, y.lo), 16-byte aligned
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  cdf r;
  r.x = df(t.x, t.y);
  r.y = df(t.z, t.w);
  return r;
}
template <typename R> __device__ __forceinline__ cx<R> czero() { return mk<R>((R)0, (R)0); }

// Asynchronous global -> shared copies (cp.async): an op that prefetches its
// epilogue inputs issues them before the line transforms, so the loads are in
// flight while the FFT runs; the same thread reads them back after waiting.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename R> __device__ __forceinline__ R rsq(R v);
template <> __device__ __forceinline__ double rsq<double>(double v) { return rsqrt(v); }
template <> __device__ __forceinline__ float rsq<float>(float v) { return rsqrtf(v); }
template <> __device__ __forceinline__ df rsq<df>(df v) { return df_rsqrt(v); }

// ------------------------------------------------------------- FastFft
template <typename R> struct SmemShift;  // one pad element per 128 bytes
template <> struct SmemShift<double> { static constexpr int value = 3; };
template <> struct SmemShift<float> { static constexpr int value = 4; };
template <> struct SmemShift<df> { static constexpr int value = 3; };

constexpr int kFastElems = 2048;  // elements per CTA (256 threads x 8)

template <int L> struct FastCfg {
  static constexpr int TPL = L / 8;             // threads per line
  static constexpr int T = kFastElems / L;      // lines per CTA
  static constexpr int A = (L >= 512) ? 3 : (L >= 64 ? 2 : 1);  // radix-8 stages
  static constexpr int REM = L / (A == 3 ? 512 : (A == 2 ? 64 : 8));  // 1, 2 or 4
};

template <typename R, int L> struct FastSmem {
  static constexpr int buf = kFastElems + (kFastElems >> SmemShift<R>::value) + 1;
  // stage s exchanges through b0 (s even) or b1 (s odd) unless it is the last
  // stage; with one or two radix-8 stages and nothing after them (L <= 64)
  // only b0 is used, so b1 takes no shared memory
  static constexpr bool kTwoBufs = FastCfg<L>::A == 3 || (FastCfg<L>::A == 2 && FastCfg<L>::REM > 1);
  static constexpr size_t bytes = (size_t)(L + (kTwoBufs ? 2 : 1) * buf) * sizeof(cx<R>);
};

template <typename R, int L, bool LM> __device__ __forceinline__ int fsa(int t, int pos) {
  const int lin = LM ? t * L + pos : pos * FastCfg<L>::T + t;
  return lin + (lin >> SmemShift<R>::value);
}

// ---- binary64 twiddled butterflies in multiply-add form (Linzer and Feig's
// modified FFT butterflies).  W = e^{S 2 pi i j / L} is read as (m, t) from
// the multiply-add table of e^{-2 pi i j / L} (conjugated for S > 0), so that
// W x = m y with y one FMA a component, and a +/- W x one FMA more a component:
// 6 FP64 instructions a butterfly instead of 8 (complex product, then add and
// subtract).  The form (lf_cform) is an integer test on j.  Nothing on the
// FP64 pipe depends on it: it swaps operands with selects and flips the sign
// of a scale factor with an integer XOR, and the remaining signs are the same
// for every thread and fold into the FMAs.

// a with its sign flipped when f (an integer operation on the high word).
__device__ __forceinline__ double flip_sign(double a, bool f) {
  return __hiloint2double(__double2hiint(a) ^ (f ? (int)0x80000000 : 0), __double2loint(a));
}

template <int L, int S, bool LO>
__device__ __forceinline__ void lf_bfly(double2& a, double2& x, const double2* lf, int j) {
  const double2 e = lf[j];
  const bool sf = !lf_cform(j, L);
  // W = m_e (1 + i t_e) or m_e (t_e + i): t_e = t and m_e = m for S < 0; for
  // S > 0 (conjugate) t_e = -t, and m_e = -m in the s-form
  const double t = (S > 0) ? -e.y : e.y;
  const double mi = (S > 0) ? flip_sign(e.x, sf) : e.x;
  const double mr = flip_sign(mi, sf);
  // (P, Q) = (x.x, x.y) in the c-form, swapped in the s-form; then
  // W x = (mr u, mi v) with u = P - t_e Q, v = Q + t_e P in both forms
  const double P = sf ? x.y : x.x, Q = sf ? x.x : x.y;
  const double u = fma(-t, Q, P), v = fma(t, P, Q);
  if (!LO) x = make_double2(fma(-mr, u, a.x), fma(-mi, v, a.y));  // a - W x
  a = make_double2(fma(mr, u, a.x), fma(mi, v, a.y));               // a + W x
}

// Twiddled radix-8 step: v[r] <- W^r v[r] (W = W_j), then the DFT of sign S,
// as three layers of four multiply-add butterflies.  With r = 4 b2 + 2 b1 + b0
// the layers apply W^4; W^2 and S i W^2 (= W_{2j + L/4}); and W, theta W,
// theta^2 W, theta^3 W (theta = e^{S i pi / 4}, W_{j + qL/8}), where each odd
// partial sum carries the common factor of its inputs so that one table
// twiddle a butterfly suffices.  LO: only X_0..X_3 are formed.
template <int L, int S, bool LO>
__device__ __forceinline__ void lf_radix8(double2 (&v)[8], const double2* lf, int j) {
  constexpr int L8 = L / 8, L4 = L / 4;
  // v0 +/- W^4 v4, v2 +/- W^4 v6, v1 +/- W^4 v5, v3 +/- W^4 v7
  lf_bfly<L, S, false>(v[0], v[4], lf, 4 * j);
  lf_bfly<L, S, false>(v[2], v[6], lf, 4 * j);
  lf_bfly<L, S, false>(v[1], v[5], lf, 4 * j);
  lf_bfly<L, S, false>(v[3], v[7], lf, 4 * j);
  // evens: E0, E2 in v0, v2; E1, E3 in v4, v6.  Odds / W: in v1, v3 and v5, v7
  lf_bfly<L, S, false>(v[0], v[2], lf, 2 * j);
  lf_bfly<L, S, false>(v[4], v[6], lf, 2 * j + L4);
  lf_bfly<L, S, false>(v[1], v[3], lf, 2 * j);
  lf_bfly<L, S, false>(v[5], v[7], lf, 2 * j + L4);
  // X_q = E_q + theta^q O_q, X_{q+4} = E_q - theta^q O_q
  lf_bfly<L, S, LO>(v[0], v[1], lf, j);           // X0, X4
  lf_bfly<L, S, LO>(v[4], v[5], lf, j + L8);      // X1, X5
  lf_bfly<L, S, LO>(v[2], v[3], lf, j + L4);      // X2, X6
  lf_bfly<L, S, LO>(v[6], v[7], lf, j + 3 * L8);  // X3, X7
  const double2 x1 = v[4], x3 = v[6], x4 = v[1], x6 = v[3];
  v[1] = x1; v[3] = x3; v[4] = x4; v[6] = x6;
}

// Twiddled radix-4 step (W = W_b): v[q] <- W^q v[q], then the DFT of sign S:
// v0 +/- W^2 v2, v1 +/- W^2 v3, then W and S i W (= W_{b + L/4}).  LO: only
// X_0, X_1 are formed.
template <int L, int S, bool LO>
__device__ __forceinline__ void lf_radix4(double2 (&u)[4], const double2* lf, int b) {
  lf_bfly<L, S, false>(u[0], u[2], lf, 2 * b);
  lf_bfly<L, S, false>(u[1], u[3], lf, 2 * b);
  lf_bfly<L, S, LO>(u[0], u[1], lf, b);           // X0, X2
  lf_bfly<L, S, LO>(u[2], u[3], lf, b + L / 4);   // X1, X3
  const double2 x1 = u[2], x2 = u[1];
  u[1] = x1; u[2] = x2;
}

// Transforms the 8 register elements v[r] = line[j + TPL r] of line t in place
// (sign S, unnormalised); on return v[r] holds frequency j + TPL r.  ZU: the
// elements r >= 4 (positions >= L/2) are zero and not read.  LO: only the
// outputs r < 4 (frequencies < L/2) are formed.
template <typename R, int L, int S, bool LM, bool ZU = false, bool LO = false>
__device__ __forceinline__ void fast_fft(cx<R> (&v)[8], cx<R>* b0, cx<R>* b1, const cx<R>* tw, int t, int j) {
  using C = FastCfg<L>;
  static_assert(!(ZU && LO && C::A == 1 && C::REM == 1), "ZU and LO in one radix-8 stage");
  constexpr bool kLF = std::is_same<R, double>::value;  // tw is the multiply-add table
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < C::A; ++s) {
    const int k = j & (Ns - 1);
    const bool last = (s == C::A - 1) && (C::REM == 1);
    if constexpr (kLF) {
      if (s == 0) {
        if (ZU) Dft<R, 8, S>::run_zu(v);
        else Dft<R, 8, S>::run(v);
      } else if (LO && last) {
        lf_radix8<L, S, true>(v, tw, k * (L / (8 * Ns)));
      } else {
        lf_radix8<L, S, false>(v, tw, k * (L / (8 * Ns)));
      }
    } else {
      if (s > 0) {
        const int tws = L / (8 * Ns);
#pragma unroll
        for (int r = 1; r < 8; ++r) {
          const cx<R> w = tw[k * r * tws];
          v[r] = (S < 0) ? cmul<R>(v[r], w) : cmulc<R>(v[r], w);
        }
      }
      if (ZU && s == 0) Dft<R, 8, S>::run_zu(v);
      else if (LO && last) Dft<R, 8, S>::run_lo(v);
      else Dft<R, 8, S>::run(v);
    }
    if (!last) {
      cx<R>* b = (s & 1) ? b1 : b0;
      const int base = (j - k) * 8 + k;
#pragma unroll
      for (int r = 0; r < 8; ++r) b[fsa<R, L, LM>(t, base + r * Ns)] = v[r];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = b[fsa<R, L, LM>(t, j + C::TPL * r)];
    }
    Ns *= 8;
  }
  if constexpr (C::REM > 1) {
    constexpr int Q = C::REM, M = 8 / C::REM;  // M butterflies of radix Q per thread
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int b = j + C::TPL * m;  // butterfly index = its twiddle exponent base (Ns = L/Q)
      cx<R> u[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) u[q] = v[m + M * q];
      if constexpr (kLF && Q == 2) {
        lf_bfly<L, S, LO>(u[0], u[1], tw, b);
      } else if constexpr (kLF && Q == 4) {
        lf_radix4<L, S, LO>(u, tw, b);
      } else {
#pragma unroll
        for (int q = 1; q < Q; ++q) {
          const cx<R> w = tw[b * q];
          u[q] = (S < 0) ? cmul<R>(u[q], w) : cmulc<R>(u[q], w);
        }
        if (LO) Dft<R, Q, S>::run_lo(u);
        else Dft<R, Q, S>::run(u);
      }
#pragma unroll
      for (int q = 0; q < (LO ? Q / 2 : Q); ++q) v[m + M * q] = u[q];
    }
  }
}

// ------------------------------------------------------------ op traits
template <int S1, bool SECOND, int NRED, bool LM> struct OpBase {
  static constexpr int kSign1 = S1;       // sign of the first transform
  static constexpr bool kSecond = SECOND;  // inverse transform after the spectral step
  static constexpr int kRed = NRED;        // fused reduction slots
  static constexpr bool kLM = LM;          // line-major (x) pass
  static constexpr bool kMirror = false;   // post-processing needs the mirror frequency L - k
  static constexpr bool kZeroUpper = false;  // positions >= L/2 of the first transform's input are zero
  static constexpr bool kHalfOut = false;    // only positions < L/2 of the last transform's output are used
  static constexpr bool kNyqTail = false;    // column pass over columns 0..c.Nx (see k_fast)
  static constexpr int kPre = 0;  // bytes per element the op prefetches into shared memory (fast engine)
  // the fast engine keeps the loaded line in registers and hands each element
  // to the epilogue (store_k / store_pre_k), which then need not load it again
  static constexpr bool kKeepIn = false;
  double* part = nullptr;                  // reduction partials [slot][block]
  int pstride = 0;
};

// ------------------------------------------------------------ kernels
template <typename R, int NR>
__device__ __forceinline__ void reduce_out(R (&acc)[NR], double* part, int pstride) {
  if constexpr (sizeof(R) == 4) {
    block_reduce_store_f32<NR>(acc, part, pstride, blockIdx.y * gridDim.x + blockIdx.x);
  } else if constexpr (std::is_same<R, double>::value) {
    block_reduce_store<NR>(acc, part, pstride, blockIdx.y * gridDim.x + blockIdx.x);
  } else {  // double-word partials: widened per thread, FP64 beyond
    double d[NR];
#pragma unroll
    for (int s = 0; s < NR; ++s) d[s] = tod<R>(acc[s]);
    block_reduce_store<NR>(d, part, pstride, blockIdx.y * gridDim.x + blockIdx.x);
  }
}

// CTAs per SM the fast engine is compiled for: 4 in FP32 (64 registers); 3
// (80 registers) with a prefetch buffer of 16 bytes an element, when two
// exchange buffers already limit the shared memory to 3 CTAs, and for
// L < 64, whose instances spill 8-88 bytes at 64 registers (L = 64: 4 bytes);
// 2 otherwise (128 registers).
template <typename R, int L, class Op> constexpr int fast_min_blocks() {
  return sizeof(R) == 4 ? (Op::kPre >= 16 && (FastSmem<R, L>::kTwoBufs || L < 64) ? 3 : 4) : 2;
}

template <typename R, int L, class Op>
__global__ void __launch_bounds__(kThreads, fast_min_blocks<R, L, Op>()) k_fast(Op op, const cx<R>* __restrict__ twg) {
  using C = FastCfg<L>;
  extern __shared__ __align__(16) unsigned char fast_smem[];
  cx<R>* tw = reinterpret_cast<cx<R>*>(fast_smem);
  cx<R>* b0 = tw + L;
  cx<R>* b1 = b0 + FastSmem<R, L>::buf;
  int t, j;
  if (Op::kLM) { t = threadIdx.x / C::TPL; j = threadIdx.x % C::TPL; }
  else { j = threadIdx.x / C::T; t = threadIdx.x % C::T; }
  int o = Op::kLM ? blockIdx.x * C::T + t : blockIdx.y;
  int x = Op::kLM ? 0 : blockIdx.x * C::T + t;
  bool ok;
  static_assert(!Op::kNyqTail || (Op::kRed == 0 && !Op::kLM), "the remapped CTAs that exit write no partial sums");
  if constexpr (Op::kNyqTail) {
    // Half-spectrum column passes (columns 0..Nx): when T divides Nx the last
    // block column would carry column Nx alone; it takes column Nx of T
    // consecutive rows instead, so that no CTA transforms idle columns.
    if (blockIdx.x == gridDim.x - 1 && op.c.Nx % C::T == 0) {
      if (blockIdx.y * C::T >= gridDim.y) return;  // whole CTA: before any barrier
      x = op.c.Nx;
      o = blockIdx.y * C::T + t;
      ok = o < (int)gridDim.y && op.valid(o, x);
    } else {
      ok = op.valid(o, x);
    }
  } else {
    ok = op.valid(o, x);
  }
  // epilogue inputs of this thread's elements, [r][thread] (ops with kPre > 0)
  unsigned char* pre = fast_smem + FastSmem<R, L>::bytes;
  if constexpr (Op::kPre > 0) {
    if (ok) {
#pragma unroll
      for (int r = 0; r < (Op::kHalfOut ? 4 : 8); ++r)
        op.prefetch(o, x, j + C::TPL * r, pre + ((size_t)r * kThreads + threadIdx.x) * Op::kPre);
    }
    cp_async_commit();
  }
  cx<R> v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = (ok && (!Op::kZeroUpper || r < 4)) ? op.load(o, x, j + C::TPL * r) : czero<R>();
  cx<R> vin[Op::kKeepIn ? 8 : 1];
  if constexpr (Op::kKeepIn) {
#pragma unroll
    for (int r = 0; r < 8; ++r) vin[r] = v[r];
  }
  // FP64 twiddles are staged in shared memory; FP32 twiddles are read through
  // L1 from global memory, which avoids the bank conflicts of the strided
  // table accesses (the FP32 passes are issue-bound, the FP64 ones ALU-bound).
  const cx<R>* twsrc = twg;
  if (sizeof(R) == 8) {
    for (int i = threadIdx.x; i < L; i += kThreads) tw[i] = twg[i];
    twsrc = tw;
  }
  __syncthreads();
  constexpr int NR = Op::kRed > 0 ? Op::kRed : 1;
  R acc[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) acc[s] = (R)0;
  constexpr bool kLo1 = Op::kHalfOut && !Op::kSecond && !Op::kMirror;
  fast_fft<R, L, Op::kSign1, Op::kLM, Op::kZeroUpper, kLo1>(v, b0, b1, twsrc, t, j);
  if constexpr (Op::kMirror) {
    // exchange so every thread sees the frequency L - k of each of its k
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) b0[fsa<R, L, Op::kLM>(t, j + C::TPL * r)] = v[r];
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int k = j + C::TPL * r;
        op.post(o, x, k, v[r], b0[fsa<R, L, Op::kLM>(t, (L - k) & (L - 1))], acc);
      }
    }
  } else {
    if (ok) {
#pragma unroll
      for (int r = 0; r < 8; ++r) op.spectral(o, x, j + C::TPL * r, v[r], acc);
    }
    if (Op::kSecond) {
      __syncthreads();
      fast_fft<R, L, -Op::kSign1, Op::kLM, false, Op::kHalfOut>(v, b0, b1, twsrc, t, j);
    }
    if constexpr (Op::kPre > 0) {
      cp_async_wait_all();
      if (ok) {
#pragma unroll
        for (int r = 0; r < (Op::kHalfOut ? 4 : 8); ++r) {
          unsigned char* src = pre + ((size_t)r * kThreads + threadIdx.x) * Op::kPre;
          if constexpr (Op::kKeepIn) op.store_pre_k(o, x, j + C::TPL * r, v[r], acc, src, vin[r]);
          else op.store_pre(o, x, j + C::TPL * r, v[r], acc, src);
        }
      }
    } else if (ok) {
#pragma unroll
      for (int r = 0; r < (Op::kHalfOut ? 4 : 8); ++r) {
        if constexpr (Op::kKeepIn) op.store_k(o, x, j + C::TPL * r, v[r], acc, vin[r]);
        else op.store(o, x, j + C::TPL * r, v[r], acc);
      }
    }
  }
  if (Op::kRed > 0) reduce_out<R, NR>(acc, op.part, op.pstride);
}

template <typename R, class Op>
__global__ void __launch_bounds__(kThreads) k_generic(Op op, FftLen f, int T) {
  extern __shared__ __align__(16) unsigned char gen_smem[];
  cx<R>* tile = reinterpret_cast<cx<R>*>(gen_smem);
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    int t, pos;
    if (Op::kLM) { t = e / L; pos = e - t * L; } else { pos = e / T; t = e - pos * T; }
    const int o = Op::kLM ? blockIdx.x * T + t : blockIdx.y;
    const int x = Op::kLM ? 0 : blockIdx.x * T + t;
    tile[e] = op.valid(o, x) ? op.load(o, x, pos) : czero<R>();
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, Op::kSign1, Op::kLM>(tile, tw, f, T);
  constexpr int NR = Op::kRed > 0 ? Op::kRed : 1;
  R acc[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) acc[s] = (R)0;
  if constexpr (Op::kMirror) {
    for (int e = threadIdx.x; e < T * L; e += kThreads) {
      int t, pos;
      if (Op::kLM) { t = e / L; pos = e - t * L; } else { pos = e / T; t = e - pos * T; }
      const int o = Op::kLM ? blockIdx.x * T + t : blockIdx.y;
      const int x = Op::kLM ? 0 : blockIdx.x * T + t;
      const int pm = pos == 0 ? 0 : L - pos;
      if (op.valid(o, x)) op.post(o, x, pos, tile[e], tile[tix<Op::kLM>(t, pm, T, L)], acc);
    }
    if (Op::kRed > 0) reduce_out<R, NR>(acc, op.part, op.pstride);
    return;
  }
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    int t, pos;
    if (Op::kLM) { t = e / L; pos = e - t * L; } else { pos = e / T; t = e - pos * T; }
    const int o = Op::kLM ? blockIdx.x * T + t : blockIdx.y;
    const int x = Op::kLM ? 0 : blockIdx.x * T + t;
    if (op.valid(o, x)) op.spectral(o, x, pos, tile[e], acc);
  }
  __syncthreads();
  if (Op::kSecond) fft_tile<R, -Op::kSign1, Op::kLM>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    int t, pos;
    if (Op::kLM) { t = e / L; pos = e - t * L; } else { pos = e / T; t = e - pos * T; }
    const int o = Op::kLM ? blockIdx.x * T + t : blockIdx.y;
    const int x = Op::kLM ? 0 : blockIdx.x * T + t;
    if (op.valid(o, x)) op.store(o, x, pos, tile[e], acc);
  }
  if (Op::kRed > 0) reduce_out<R, NR>(acc, op.part, op.pstride);
}

// ------------------------------------------------------------ dispatch
inline bool fast_len(int L) { return L >= 16 && L <= 1024 && (L & (L - 1)) == 0; }

inline int ceil_div_l(long a, long b) { return (int)((a + b - 1) / b); }

// Generic-engine tile sizes (see atkm_internal.cuh).
// Narrower tiles until the pass has at least two CTAs per SM.
template <typename R> inline int gen_lm_tile(int L, long nlines) {
  int T = TileElems<R>::value / L;
  if (T < 1) T = 1;
  const long want = 2L * device_sm_count();
  while (T > 1 && ceil_div_l(nlines, T) < want) T >>= 1;
  return T;
}
template <typename R> inline int gen_col_tile(int L, int X, long outer) {
  int T = TileElems<R>::value / L;
  if (T > X) T = X;
  if (T < 1) T = 1;
  const long want = 2L * device_sm_count();
  while (T > 8 && (long)ceil_div_l(X, T) * outer < want) T >>= 1;
  return T;
}

struct PassGrid {
  dim3 grid;
  int T;
  bool fast;
  bool mix;  // the mixed-radix register engine (mix.cuh)
};

bool mix_len(int L);

// LM passes: `lines` lines; strided passes: `X` columns x `outer` outer indices.
// Engine: the power-of-two register engine, else the mixed-radix register
// engine for 3 * 2^a (FP32 and binary64) and 5 * 2^a (FP32; in binary64 its
// 20 complex doubles a thread make it slower than the generic engine,
// measured), not with ATKM_PLAN_GENERIC_FFT, else the generic shared-memory
// engine.
template <typename R> constexpr int tune_r() {
  return std::is_same<R, double>::value ? 0 : (std::is_same<R, float>::value ? 1 : 2);
}
// An autotuned choice for (R, L, LM) of this plan, or null.
template <typename R> inline const TuneEntry* tuned(const atkm_plan* p, int L, bool LM) {
  for (int i = 0; i < p->n_tune; ++i) {
    const TuneEntry& e = p->tune[i];
    if (e.r == tune_r<R>() && e.L == L && e.lm == (LM ? 1 : 0)) return &e;
  }
  return nullptr;
}

// Lengths the mixed-radix register engine is instantiated for in arithmetic
// R (run_pass's switches): 3 * 2^a and 5 * 2^a in FP32, 3 * 2^a in binary64,
// none in double-word.  Both the fixed rule and the autotuner go through this.
template <typename R> inline bool mix_ok(int L) {
  if (std::is_same<R, df>::value || !mix_len(L)) return false;
  return !(std::is_same<R, double>::value && L % 5 == 0);
}
inline bool mix_ok_r(int r, int L) {
  return r == 0 ? mix_ok<double>(L) : (r == 1 ? mix_ok<float>(L) : mix_ok<df>(L));
}

template <typename R> inline PassGrid pass_grid(const atkm_plan* p, int L, bool LM, long lines, int X, int outer) {
  PassGrid pg;
  pg.fast = fast_len(L);
  pg.mix = !pg.fast && !(p->flags & ATKM_PLAN_GENERIC_FFT) && mix_ok<R>(L);
  const TuneEntry* te = pg.fast ? nullptr : tuned<R>(p, L, LM);
  if (te) pg.mix = te->mix != 0 && mix_ok<R>(L);
  if (pg.fast) pg.T = kFastElems / L;
  else if (pg.mix) pg.T = kThreads / (L / (L % 3 == 0 ? 12 : 20));
  else {
    pg.T = LM ? gen_lm_tile<R>(L, lines) : gen_col_tile<R>(L, X, outer);
    if (te) pg.T = std::max(pg.T >> te->shift, 1);
  }
  if (LM) pg.grid = dim3(ceil_div_l(lines, pg.T), 1, 1);
  else pg.grid = dim3(ceil_div_l(X, pg.T), outer, 1);
  return pg;
}

template <typename K> inline cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Dynamic shared memory above the default must be opted into once per kernel
// and device (the attribute belongs to the device's context); `done` holds
// one bit per device already prepared.
template <typename K>
inline cudaError_t ensure_smem(std::atomic<unsigned long long>& done, K kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set_smem(kernel, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <typename R, int L, class Op>
inline cudaError_t launch_fast_L(const Op& op, const FftLen& f, const PassGrid& pg, cudaStream_t st) {
  static std::atomic<unsigned long long> prepared{0};
  const size_t sm = FastSmem<R, L>::bytes + (size_t)Op::kPre * 8 * kThreads;
  cudaError_t e = ensure_smem(prepared, k_fast<R, L, Op>, sm);
  if (e != cudaSuccess) return e;
  // binary64 passes take the multiply-add form of the twiddles
  const cx<R>* tw = std::is_same<R, double>::value ? reinterpret_cast<const cx<R>*>(f.lf64) : tw_table_host<R>(f);
  k_fast<R, L, Op><<<pg.grid, kThreads, sm, st>>>(op, tw);
  return cudaGetLastError();
}

}  // namespace atkm
#include "mix.cuh"
namespace atkm {

template <typename R, class Op>
inline cudaError_t run_pass(const Op& op, const FftLen& f, const PassGrid& pg, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    if (pg.mix) {
      switch (f.L) {
        case 20: return launch_mix_L<R, 20>(op, f, pg, st);
        case 24: return launch_mix_L<R, 24>(op, f, pg, st);
        case 40: return launch_mix_L<R, 40>(op, f, pg, st);
        case 48: return launch_mix_L<R, 48>(op, f, pg, st);
        case 80: return launch_mix_L<R, 80>(op, f, pg, st);
        case 96: return launch_mix_L<R, 96>(op, f, pg, st);
        case 160: return launch_mix_L<R, 160>(op, f, pg, st);
        case 192: return launch_mix_L<R, 192>(op, f, pg, st);
        case 320: return launch_mix_L<R, 320>(op, f, pg, st);
        case 384: return launch_mix_L<R, 384>(op, f, pg, st);
        default: return cudaErrorInvalidValue;
      }
    }
  } else if constexpr (std::is_same<R, double>::value) {
    if (pg.mix) {
      switch (f.L) {
        case 24: return launch_mix_L<R, 24>(op, f, pg, st);
        case 48: return launch_mix_L<R, 48>(op, f, pg, st);
        case 96: return launch_mix_L<R, 96>(op, f, pg, st);
        case 192: return launch_mix_L<R, 192>(op, f, pg, st);
        case 384: return launch_mix_L<R, 384>(op, f, pg, st);
        default: return cudaErrorInvalidValue;
      }
    }
  }
  if (pg.fast) {
    switch (f.L) {
      case 16: return launch_fast_L<R, 16>(op, f, pg, st);
      case 32: return launch_fast_L<R, 32>(op, f, pg, st);
      case 64: return launch_fast_L<R, 64>(op, f, pg, st);
      case 128: return launch_fast_L<R, 128>(op, f, pg, st);
      case 256: return launch_fast_L<R, 256>(op, f, pg, st);
      case 512: return launch_fast_L<R, 512>(op, f, pg, st);
      case 1024: return launch_fast_L<R, 1024>(op, f, pg, st);
      default: return cudaErrorInvalidValue;
    }
  }
  static std::atomic<unsigned long long> prepared{0};
  cudaError_t e = ensure_smem(prepared, k_generic<R, Op>, (size_t)(TileElems<R>::value + kMaxLen) * sizeof(cx<R>));
  if (e != cudaSuccess) return e;
  const size_t sm = (size_t)(pg.T * f.L + f.L) * sizeof(cx<R>);
  k_generic<R, Op><<<pg.grid, kThreads, sm, st>>>(op, f, pg.T);
  return cudaGetLastError();
}

// ================================================================ ops
// ---- ATKM (twofold-padded grid, real-data form).  The density is real, so
// the x transform of each padded line (length Mx = 2 Nx, upper half zero) is
// taken as a complex FFT of length Nx of z_m = rho_{2m} + i rho_{2m+1} with the
// exact post-twist X_k = (Z_k + conj Z_{Nx-k})/2 - (i/2) e^{-2 pi i k/Mx}
// (Z_k - conj Z_{Nx-k}), k = 0..Nx (Hermitian symmetry gives the rest); the y
// and z passes then run on the Nx + 1 half-spectrum columns only, and the
// inverse x transform rebuilds the real output from that half (C2R).  With a
// real density this equals the real part of the full complex convolution
// once K is symmetrised on the padded Nyquist planes (see OpAtkmZ).  W1 and
// W2 hold 2 X (the post-twist's 1/2 sits in the z pass's multiplier).
// W1: [Nz][Ny][XS], W2: [Nz][My][XS], columns 0..Nx used.
template <typename R, int MODE> struct OpAtkmXF : OpBase<-1, false, 0, true> {
  static constexpr bool kMirror = true;
  static constexpr bool kZeroUpper = true;  // z_m = 0 for m >= Nx/2 = L/2
  const double* a; const double* b; cx<R>* W1; const cx<R>* twM; Cst<R> c; int XS;
  __device__ R dens(size_t idx) const {
    if (MODE == SRC_RHO) return tor<R>(a[idx]);
    if (MODE == SRC_PSI) {
      const cx<R> z = from64<R>(reinterpret_cast<const double2*>(a)[idx]);
      return z.x * z.x + z.y * z.y;
    }
    const cx<R> u = from64<R>(reinterpret_cast<const double2*>(a)[idx]);
    const cx<R> w = from64<R>(reinterpret_cast<const double2*>(b)[idx]);
    return u.x * w.x + u.y * w.y;
  }
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  // z_m = rho_{2m} + i rho_{2m+1}; zero for 2m >= Nx (the padding)
  __device__ cx<R> load(int o, int, int m) const {
    if (2 * m >= c.Nx) return czero<R>();
    const size_t idx = (size_t)o * c.Nx + 2 * m;
    return mk<R>(dens(idx), dens(idx + 1));
  }
  // Stores 2 X_k: the factor 1/2 of E and D is left to the z pass's
  // multiplier, where it costs nothing (a power of two commutes exactly with
  // every later sum and product, so the result is the same to the bit).
  __device__ void post(int o, int, int k, cx<R> Zk, cx<R> Zm, R*) const {
    const cx<R> Zc = mk<R>(Zm.x, -Zm.y);                 // conj Z_{Nx-k}
    const cx<R> E2 = add<R>(Zk, Zc);                      // 2 E
    const cx<R> D2 = sub<R>(Zk, Zc);                      // 2 D
    const cx<R> w = twM[k];                               // e^{-2 pi i k / Mx}
    const cx<R> wD = cmul<R>(w, D2);
    W1[(size_t)o * XS + k] = mk<R>(E2.x + wD.y, E2.y - wD.x);  // 2 (E - i w D)
    if (k == 0) {
      const R xn = Zk.x - Zk.y;
      W1[(size_t)o * XS + c.Nx] = mk<R>(xn + xn, (R)0);
    }
  }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int, int, int, cx<R>, R*) const {}
};

// y forward: o = z, x = kx in [0, Nx]; rows y < Ny of W1, zero beyond.
template <typename R> struct OpAtkmYF : OpBase<-1, false, 0, false> {
  static constexpr bool kZeroUpper = true;  // rows y >= Ny = L/2 are the padding
  static constexpr bool kNyqTail = true;
  const cx<R>* W1; cx<R>* W2; Cst<R> c; int XS;
  __device__ bool valid(int, int x) const { return x <= c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const {
    return pos < c.Ny ? W1[((size_t)o * c.Ny + pos) * XS + x] : czero<R>();
  }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const { W2[((size_t)o * c.My + pos) * XS + x] = v; }
};

// z forward * K_sym / (2 Mx My Mz) * inverse: o = ky, x = kx in [0, Nx]; rows z < Nz
// (the 2 undoes the doubled half spectrum that OpAtkmXF stores).
// K_sym = (K(k) + K(-k))/2 = -1 + 3 U0 (A^2 + B^2), A = sum of n_a nu_a over
// axes whose index is not the padded Nyquist index, B over those that are.
// FP64 and double-word passes are bound by arithmetic: they read K_sym, pre-
// scaled, from the plan's table in the layout of W2 (k_multiplier_half; 8 B a
// point, about 9 FP64 instructions fewer).  FP32 passes are bound by issue and
// bandwidth: they form it from the U0 octant (mostly L2-resident), which
// costs less than the table's extra 4 B a point.
template <typename R> struct OpAtkmZ : OpBase<-1, true, 0, false> {
  static constexpr bool kZeroUpper = true;  // rows z >= Nz = L/2 are the padding
  static constexpr bool kHalfOut = true;    // only rows z < Nz are kept
  static constexpr bool kNyqTail = true;
  static constexpr bool kTable = !std::is_same<R, float>::value;
  cx<R>* W2; const R* K; const R* U0; Cst<R> c; R n0, n1, n2, invM; int XS;
  __device__ bool valid(int, int x) const { return x <= c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const {
    return pos < c.Nz ? W2[((size_t)pos * c.My + o) * XS + x] : czero<R>();
  }
  __device__ void spectral(int o, int x, int k, cx<R>& v, R*) const {
    if constexpr (kTable) {
      v = scl<R>(v, K[((size_t)k * c.My + o) * XS + x]);
    } else {
      const int ky = kfreq(o, c.My), kz = kfreq(k, c.Mz);
      const int kx = x == c.Nx ? -c.Nx : x;  // signed frequency of the half-spectrum column
      const R tx = n0 * ((R)kx * c.pkx), ty = n1 * ((R)ky * c.pky), tz = n2 * ((R)kz * c.pkz);
      R A = (R)0, B = (R)0;
      if (x == c.Nx) B += tx; else A += tx;
      if (o == c.Ny) B += ty; else A += ty;
      if (k == c.Nz) B += tz; else A += tz;
      const R u = U0[((size_t)iabs(kz) * (c.Ny + 1) + iabs(ky)) * (c.Nx + 1) + x];
      v = scl<R>(v, ((R)3 * u * (A * A + B * B) - (R)1) * invM);
    }
  }
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const {
    if (pos < c.Nz) W2[((size_t)pos * c.My + o) * XS + x] = v;
  }
};

// y inverse: o = z, x = kx in [0, Nx]; output rows y < Ny into W1.
template <typename R> struct OpAtkmYI : OpBase<1, false, 0, false> {
  static constexpr bool kHalfOut = true;  // only rows y < Ny = L/2 are kept
  static constexpr bool kNyqTail = true;
  const cx<R>* W2; cx<R>* W1; Cst<R> c; int XS;
  __device__ bool valid(int, int x) const { return x <= c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return W2[((size_t)o * c.My + pos) * XS + x]; }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const {
    if (pos < c.Ny) W1[((size_t)o * c.Ny + pos) * XS + x] = v;
  }
};

// x inverse (C2R): lines o; Z_k = (X_k + conj X_{Nx-k}) + i e^{2 pi i k/Mx}
// (X_k - conj X_{Nx-k}), k < Nx, then an inverse FFT of length Nx gives
// z_m = Phi_{2m} + i Phi_{2m+1}; kept for 2m < Nx (the crop).
template <typename R> struct OpAtkmXI : OpBase<1, false, 0, true> {
  static constexpr bool kHalfOut = true;  // only z_m with 2m < Nx, i.e. m < L/2, are kept
  const cx<R>* W1; double* phi; const cx<R>* twM; Cst<R> c; int XS;
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  __device__ cx<R> load(int o, int, int k) const {
    const cx<R>* row = W1 + (size_t)o * XS;
    const cx<R> X = row[k], Xm = row[c.Nx - k];
    const cx<R> Xc = mk<R>(Xm.x, -Xm.y);
    const cx<R> S = add<R>(X, Xc), D = sub<R>(X, Xc);
    const cx<R> w = twM[k];                               // conj gives e^{+2 pi i k / Mx}
    const cx<R> wD = cmulc<R>(D, w);                      // D e^{+2 pi i k/Mx}
    return mk<R>(S.x - wD.y, S.y + wD.x);                 // S + i wD
  }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int, int m, cx<R> v, R*) const {
    if (2 * m < c.Nx) {
      double2* dst = reinterpret_cast<double2*>(phi + (size_t)o * c.Nx + 2 * m);
      *dst = to64<R, kCvtMixed>(v.x, v.y);
    }
  }
};

// ---- H_phi f (unpadded grid); acc: [Nz][Ny][Nx] kinetic+rotation accumulator.
// x: multiplier nu^2/2 + Omega y nu on lines o = z Ny + y.
template <typename R, bool RED> struct OpHX : OpBase<-1, true, RED ? 2 : 0, true> {
  const double2* f; cx<R>* acc; Cst<R> c; R Omega; AxT ax, ay;
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  __device__ cx<R> load(int o, int, int pos) const { return from64<R, kCvtMixed>(f[(size_t)o * c.Nx + pos]); }
  __device__ void spectral(int o, int, int k, cx<R>& v, R* a) const {
    if constexpr (std::is_same<R, double>::value) {
      const double kin = ax.kinN[k], rot = Omega * ay.xc[o % c.Ny] * ax.nuN[k];
      if (RED) {
        const double a2 = v.x * v.x + v.y * v.y;
        a[0] += kin * a2;
        a[1] += rot * a2;
      }
      v = scl<R>(v, kin + rot);
      return;
    }
    const R invL = (R)1 / (R)c.Nx;
    const R nu = (R)kfreq(k, c.Nx) * c.kx;
    const R y = -c.Ly + (R)(o % c.Ny) * c.hy;
    const R mkin = (R)0.5 * nu * nu, mrot = Omega * y * nu;
    if (RED) {
      const R a2 = (v.x * v.x + v.y * v.y) * invL;
      a[0] += mkin * a2;
      a[1] += mrot * a2;
    }
    v = scl<R>(v, (mkin + mrot) * invL);
  }
  __device__ void store(int o, int, int pos, cx<R> v, R*) const { acc[(size_t)o * c.Nx + pos] = v; }
};

// y: multiplier nu^2/2 - Omega x nu on lines (o = z, x); acc += result.
template <typename R, bool RED> struct OpHY : OpBase<-1, true, RED ? 2 : 0, false> {
  const double2* f; cx<R>* acc; Cst<R> c; R Omega; AxT ax, ay;
  __device__ bool valid(int, int x) const { return x < c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return from64<R, kCvtHw>(f[((size_t)o * c.Ny + pos) * c.Nx + x]); }
  __device__ void spectral(int, int x, int k, cx<R>& v, R* a) const {
    if constexpr (std::is_same<R, double>::value) {
      const double kin = ay.kinN[k], rot = -Omega * ax.xc[x] * ay.nuN[k];
      if (RED) {
        const double a2 = v.x * v.x + v.y * v.y;
        a[0] += kin * a2;
        a[1] += rot * a2;
      }
      v = scl<R>(v, kin + rot);
      return;
    }
    const R invL = (R)1 / (R)c.Ny;
    const R nu = (R)kfreq(k, c.Ny) * c.ky;
    const R xc = -c.Lx + (R)x * c.hx;
    const R mkin = (R)0.5 * nu * nu, mrot = -Omega * xc * nu;
    if (RED) {
      const R a2 = (v.x * v.x + v.y * v.y) * invL;
      a[0] += mkin * a2;
      a[1] += mrot * a2;
    }
    v = scl<R>(v, (mkin + mrot) * invL);
  }
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const {
    const size_t idx = ((size_t)o * c.Ny + pos) * c.Nx + x;
    acc[idx] = add<R>(acc[idx], v);
  }
  // FP32: the accumulator (8 B a point) is prefetched into shared memory
  static constexpr int kPre = std::is_same<R, float>::value ? 8 : 0;
  __device__ void prefetch(int o, int x, int pos, unsigned char* dst) const {
    cp_async8(dst, acc + ((size_t)o * c.Ny + pos) * c.Nx + x);
  }
  __device__ void store_pre(int o, int x, int pos, cx<R> v, R*, const unsigned char* src) const {
    acc[((size_t)o * c.Ny + pos) * c.Nx + x] = add<R>(*reinterpret_cast<const cx<R>*>(src), v);
  }
};

// z: multiplier nu^2/2 on lines (o = y, x), then
// Hf = acc + result + (V + beta |phi|^2 + lambda Phi) f.
// Reductions: kin_z, sum V|f|^2, sum |f|^4, sum Phi |f|^2, sum Re(Hf conj f), sum |f|^2.
template <typename R, bool RED> struct OpHZ : OpBase<-1, true, RED ? 6 : 0, false> {
  const double2* f; const double2* phi; const double* Phi; const cx<R>* acc; double2* Hf; Cst<R> c; PhysR<R> ph;
  AxT ax, ay, az;
  bool same = false;  // f == phi (H phi): phi is not read a second time
  __device__ bool valid(int, int x) const { return x < c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return from64<R, kCvtMixed>(f[((size_t)pos * c.Ny + o) * c.Nx + x]); }
  __device__ void spectral(int, int, int k, cx<R>& v, R* a) const {
    if constexpr (std::is_same<R, double>::value) {
      const double m = az.kinN[k];
      if (RED) a[0] += m * (v.x * v.x + v.y * v.y);
      v = scl<R>(v, m);
      return;
    }
    const R invL = (R)1 / (R)c.Nz;
    const R nu = (R)kfreq(k, c.Nz) * c.kz;
    const R m = (R)0.5 * nu * nu;
    if (RED) a[0] += m * (v.x * v.x + v.y * v.y) * invL;
    v = scl<R>(v, m * invL);
  }
  __device__ void store(int o, int x, int pos, cx<R> v, R* a) const {
    const size_t idx = ((size_t)pos * c.Ny + o) * c.Nx + x;
    finish(o, x, pos, idx, v, a, tor<R>(ldro(Phi + idx)), ldro(acc + idx), from64<R, kCvtMixed>(ldro(f + idx)));
  }
  // FP32 and double-word: f at this point is the element the engine loaded
  // (the same conversion of the same value), kept in registers
  static constexpr bool kKeepIn = !std::is_same<R, double>::value;
  __device__ void store_k(int o, int x, int pos, cx<R> v, R* a, cx<R> fin) const {
    const size_t idx = ((size_t)pos * c.Ny + o) * c.Nx + x;
    finish(o, x, pos, idx, v, a, tor<R>(ldro(Phi + idx)), ldro(acc + idx), fin);
  }
  // FP32: Phi (8 B) and the accumulator (8 B) are prefetched into shared memory
  static constexpr int kPre = std::is_same<R, float>::value ? 16 : 0;
  __device__ void prefetch(int o, int x, int pos, unsigned char* dst) const {
    const size_t idx = ((size_t)pos * c.Ny + o) * c.Nx + x;
    cp_async8(dst, Phi + idx);
    cp_async8(dst + 8, acc + idx);
  }
  __device__ void store_pre(int o, int x, int pos, cx<R> v, R* a, const unsigned char* src) const {
    const size_t idx = ((size_t)pos * c.Ny + o) * c.Nx + x;
    finish(o, x, pos, idx, v, a, tor<R>(*reinterpret_cast<const double*>(src)),
           *reinterpret_cast<const cx<R>*>(src + 8), from64<R, kCvtMixed>(ldro(f + idx)));
  }
  __device__ void store_pre_k(int o, int x, int pos, cx<R> v, R* a, const unsigned char* src, cx<R> fin) const {
    const size_t idx = ((size_t)pos * c.Ny + o) * c.Nx + x;
    finish(o, x, pos, idx, v, a, tor<R>(*reinterpret_cast<const double*>(src)),
           *reinterpret_cast<const cx<R>*>(src + 8), fin);
  }
  __device__ __forceinline__ void finish(int o, int x, int pos, size_t idx, cx<R> v, R* a, R Pd, cx<R> accv,
                                         cx<R> fv) const {
    R V;
    if constexpr (std::is_same<R, double>::value) {
      V = ph.gz2 * az.hxc2[pos] + (ph.gy2 * ay.hxc2[o] + ph.gx2 * ax.hxc2[x]);
    } else {
      const R xc = -c.Lx + (R)x * c.hx, yc = -c.Ly + (R)o * c.hy, zc = -c.Lz + (R)pos * c.hz;
      V = (R)0.5 * (ph.gx2 * xc * xc + ph.gy2 * yc * yc + ph.gz2 * zc * zc);
    }
    const cx<R> pv = same ? fv : from64<R, kCvtMixed>(ldro(phi + idx));
    const R w = V + ph.beta * (pv.x * pv.x + pv.y * pv.y) + ph.lambda * Pd;
    const cx<R> kin = add<R>(accv, v);
    const R ox = kin.x + w * fv.x, oy = kin.y + w * fv.y;
    Hf[idx] = to64<R, kCvtMixed>(ox, oy);
    if (RED) {
      const R f2 = fv.x * fv.x + fv.y * fv.y;
      a[1] += V * f2;
      a[2] += f2 * f2;
      a[3] += Pd * f2;
      a[4] += ox * fv.x + oy * fv.y;
      a[5] += f2;
    }
  }
};

// ---- preconditioner (unpadded grid); Wk: [Nz][Ny][Nx] workspace.
template <typename R>
__device__ __forceinline__ R pv_rsqrt(const Cst<R>& c, const PhysR<R>& ph, R alpha, int x, int y, int z, double2 p64,
                                      double Pd64) {
  const R xc = -c.Lx + (R)x * c.hx, yc = -c.Ly + (R)y * c.hy, zc = -c.Lz + (R)z * c.hz;
  const R V = (R)0.5 * (ph.gx2 * xc * xc + ph.gy2 * yc * yc + ph.gz2 * zc * zc);
  const cx<R> pv = from64<R, kCvtMixed>(p64);
  const R Pd = tor<R>(Pd64);
  const R den = alpha + V + ph.beta * (pv.x * pv.x + pv.y * pv.y) + fabs(ph.lambda) * (Pd > (R)0 ? Pd : (R)0);
  return rsq<R>(den);
}

// Binary64: the weight P_V^{-1/2} of each point is also stored in Pw for the
// x inverse pass, which then reads it instead of forming it again.
template <typename R> struct OpPXF : OpBase<-1, false, 0, true> {
  const double2* r; const double2* phi; const double* Phi; cx<R>* Wk; Cst<R> c; PhysR<R> ph; const double* alpha;
  AxT ax, ay, az; double* Pw;
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  __device__ cx<R> load(int o, int, int pos) const {
    const size_t idx = (size_t)o * c.Nx + pos;
    if constexpr (std::is_same<R, double>::value) {
      const int y = o % c.Ny, z = o / c.Ny;
      const double V = ph.gx2 * ax.hxc2[pos] + (ph.gy2 * ay.hxc2[y] + ph.gz2 * az.hxc2[z]);
      const double2 pv = phi[idx];
      const double Pd = Phi[idx];
      const double den = *alpha + V + ph.beta * (pv.x * pv.x + pv.y * pv.y) + fabs(ph.lambda) * (Pd > 0.0 ? Pd : 0.0);
      const double w = rsqrt(den);
      Pw[idx] = w;
      return scl<R>(r[idx], w);
    }
    const R w = pv_rsqrt<R>(c, ph, tor<R>(*alpha), pos, o % c.Ny, o / c.Ny, phi[idx], Phi[idx]);
    return scl<R>(from64<R, kCvtMixed>(r[idx]), w);
  }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int, int pos, cx<R> v, R*) const { Wk[(size_t)o * c.Nx + pos] = v; }
};

template <typename R, int S> struct OpPY : OpBase<S, false, 0, false> {
  cx<R>* Wk; Cst<R> c;
  __device__ bool valid(int, int x) const { return x < c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return Wk[((size_t)o * c.Ny + pos) * c.Nx + x]; }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const { Wk[((size_t)o * c.Ny + pos) * c.Nx + x] = v; }
};

// z forward * 1/((alpha + |nu|^2/2) N) * inverse on lines (o = y, x).
template <typename R> struct OpPZ : OpBase<-1, true, 0, false> {
  cx<R>* Wk; Cst<R> c; const double* alpha; AxT ax, ay, az;
  __device__ bool valid(int, int x) const { return x < c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return Wk[((size_t)pos * c.Ny + o) * c.Nx + x]; }
  __device__ void spectral(int o, int x, int k, cx<R>& v, R*) const {
    if constexpr (std::is_same<R, double>::value) {
      const double invN = 1.0 / ((double)c.Nx * (double)c.Ny * (double)c.Nz);
      v = scl<R>(v, invN / (*alpha + (ax.hnu2[x] + ay.hnu2[o]) + az.hnu2[k]));
      return;
    }
    const R invN = (R)1 / ((R)c.Nx * (R)c.Ny * (R)c.Nz);
    const R nux = (R)kfreq(x, c.Nx) * c.kx, nuy = (R)kfreq(o, c.Ny) * c.ky, nuz = (R)kfreq(k, c.Nz) * c.kz;
    v = scl<R>(v, invN / (tor<R>(*alpha) + (R)0.5 * (nux * nux + nuy * nuy + nuz * nuz)));
  }
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const { Wk[((size_t)pos * c.Ny + o) * c.Nx + x] = v; }
};

template <typename R> struct OpPXI : OpBase<1, false, 0, true> {
  const cx<R>* Wk; const double2* phi; const double* Phi; double2* Pr; Cst<R> c; PhysR<R> ph; const double* alpha;
  const double* Pw;  // binary64: the weights the x forward pass stored
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  __device__ cx<R> load(int o, int, int pos) const { return Wk[(size_t)o * c.Nx + pos]; }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int, int pos, cx<R> v, R*) const {
    const size_t idx = (size_t)o * c.Nx + pos;
    if constexpr (std::is_same<R, double>::value) {
      const double w = ldro(Pw + idx);
      Pr[idx] = make_double2(w * v.x, w * v.y);
      return;
    }
    const R w = pv_rsqrt<R>(c, ph, tor<R>(*alpha), pos, o % c.Ny, o / c.Ny, ldro(phi + idx), ldro(Phi + idx));
    Pr[idx] = to64<R, kCvtMixed>(w * v.x, w * v.y);
  }
};

// ---- in-place 3D complex FFT on a plan's (unpadded) grid, sign S.
template <typename R, int S> struct OpCX : OpBase<S, false, 0, true> {
  cx<R>* buf; Cst<R> c;
  __device__ bool valid(int o, int) const { return o < c.Nz * c.Ny; }
  __device__ cx<R> load(int o, int, int pos) const { return buf[(size_t)o * c.Nx + pos]; }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int, int pos, cx<R> v, R*) const { buf[(size_t)o * c.Nx + pos] = v; }
};
template <typename R, int S> struct OpCZ : OpBase<S, false, 0, false> {
  cx<R>* buf; Cst<R> c;
  __device__ bool valid(int, int x) const { return x < c.Nx; }
  __device__ cx<R> load(int o, int x, int pos) const { return buf[((size_t)pos * c.Ny + o) * c.Nx + x]; }
  __device__ void spectral(int, int, int, cx<R>&, R*) const {}
  __device__ void store(int o, int x, int pos, cx<R> v, R*) const { buf[((size_t)pos * c.Ny + o) * c.Nx + x] = v; }
};

}  // namespace atkm
