// Mixed-radix register FFT engine for the lengths 3 * 2^a and 5 * 2^a.
//
// The power-of-two engine (k_fast) keeps E = 8 elements of a line per thread;
// a length with a factor 3 or 5 cannot be split that way.  Here a thread keeps
// E = 12 (lengths 3 * 2^a) or E = 20 (lengths 5 * 2^a) elements, so that every
// radix of the length's stages divides E: radix-4 stages, one radix-2 stage
// when the power of two is odd, and the radix-3 or radix-5 stage last.  With
// TPL = L / E threads per line (a power of two, so T = 256 / TPL lines fit a
// CTA exactly), thread j holds the elements j + TPL e, e < E, at the start of
// every stage.  A Stockham stage of radix R with Ns = product of the earlier
// radices is E / R butterflies per thread: butterfly b = j + TPL m takes the
// register elements m + r E / R (positions b + r L / R), applies the twiddles
// w^{k r} (k = b mod Ns, w = e^{S 2 pi i / (Ns R)}), runs the R-point DFT and
// sends output r to position (b - k) R + k + r Ns through shared memory; in
// the last stage (Ns R = L) that position is the thread's own register
// m + r E / R, so the outputs stay in registers: on return element e holds
// frequency j + TPL e, as in k_fast, and the same ops (load, spectral
// multiply, inverse transform, store, mirror post-processing, fused sums,
// prefetched epilogue inputs) run unchanged.  The twofold zero padding and the
// crop are honoured (zero upper inputs are not loaded, only the lower outputs
// are stored) without pruning the arithmetic.
#pragma once

namespace atkm {

constexpr int mix_elems(int L) { return L % 3 == 0 ? 12 : 20; }
constexpr int ilog2c(int v) { return v > 1 ? 1 + ilog2c(v / 2) : 0; }
// The lengths this engine is built for (3 * 2^a and 5 * 2^a up to 384).
inline bool mix_len(int L) {
  switch (L) {
    case 24: case 48: case 96: case 192: case 384: case 20: case 40: case 80: case 160: case 320: return true;
    default: return false;
  }
}

template <int L> struct MixCfg {
  static constexpr int E = mix_elems(L);
  static constexpr int RL = E == 12 ? 3 : 5;  // the last stage's radix
  static constexpr int TPL = L / E;           // threads per line (power of two)
  static constexpr int T = kThreads / TPL;    // lines per CTA
  static constexpr int P2 = L / RL;           // the power-of-two part of L
  static constexpr int N4 = ilog2c(P2) / 2;       // radix-4 stages
  static constexpr bool R2 = (ilog2c(P2) & 1) != 0;  // one radix-2 stage
  static_assert((1 << ilog2c(P2)) == P2 && TPL * E == L && (TPL & (TPL - 1)) == 0, "length not 3 or 5 times 2^a");
  static constexpr int ELEMS = kThreads * E;  // elements per CTA
};

template <typename R, int L> struct MixSmem {
  static constexpr int buf = MixCfg<L>::ELEMS + (MixCfg<L>::ELEMS >> SmemShift<R>::value) + 1;
  static constexpr size_t bytes = (size_t)(L + buf) * sizeof(cx<R>);
};

template <typename R, int L, bool LM> __device__ __forceinline__ int msa(int t, int pos) {
  const int lin = LM ? t * L + pos : pos * MixCfg<L>::T + t;
  return lin + (lin >> SmemShift<R>::value);
}

// One Stockham stage of radix RAD over the E register elements of each
// thread; Ns = product of the earlier radices (a power of two here).  LAST:
// the outputs stay in registers.
template <typename R, int L, int RAD, int S, bool LM, bool LAST>
__device__ __forceinline__ void mix_stage(cx<R> (&v)[MixCfg<L>::E], cx<R>* buf, const cx<R>* tw, int t, int j,
                                          int Ns) {
  using C = MixCfg<L>;
  constexpr int M = C::E / RAD;  // butterflies per thread
  const int tws = L / (Ns * RAD);
  cx<R> out[C::E];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int b = j + C::TPL * m;
    const int k = b & (Ns - 1);
    cx<R> u[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) u[r] = v[m + M * r];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cx<R> w = tw[k * r * tws];
        u[r] = (S < 0) ? cmul<R>(u[r], w) : cmulc<R>(u[r], w);
      }
    }
    Dft<R, RAD, S>::run(u);
    if (LAST) {
#pragma unroll
      for (int r = 0; r < RAD; ++r) out[m + M * r] = u[r];
    } else {
      const int base = (b - k) * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[msa<R, L, LM>(t, base + r * Ns)] = u[r];
    }
  }
  if (LAST) {
#pragma unroll
    for (int e = 0; e < C::E; ++e) v[e] = out[e];
  } else {
    __syncthreads();
#pragma unroll
    for (int e = 0; e < C::E; ++e) v[e] = buf[msa<R, L, LM>(t, j + C::TPL * e)];
    __syncthreads();  // the buffer is written again by the next stage
  }
}

// The whole transform of sign S: radix-4 stages, a radix-2 stage if needed,
// then the radix-3 or radix-5 stage.
template <typename R, int L, int S, bool LM>
__device__ __forceinline__ void mix_fft(cx<R> (&v)[MixCfg<L>::E], cx<R>* buf, const cx<R>* tw, int t, int j) {
  using C = MixCfg<L>;
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < C::N4; ++s) {
    mix_stage<R, L, 4, S, LM, false>(v, buf, tw, t, j, Ns);
    Ns *= 4;
  }
  if constexpr (C::R2) {
    mix_stage<R, L, 2, S, LM, false>(v, buf, tw, t, j, Ns);
    Ns *= 2;
  }
  mix_stage<R, L, C::RL, S, LM, true>(v, buf, tw, t, j, Ns);
}

// Prefetched epilogue inputs only while they take at most 48 KB a CTA (else
// the op's plain epilogue loads).
template <int L, class Op> struct MixUsesPre {
  static constexpr bool value = Op::kPre > 0 && (size_t)Op::kPre * MixCfg<L>::E * kThreads <= 48 * 1024;
};

template <typename R, int L, class Op>
__global__ void __launch_bounds__(kThreads, 2) k_mix(Op op, const cx<R>* __restrict__ twg) {
  using C = MixCfg<L>;
  extern __shared__ __align__(16) unsigned char mix_smem[];
  cx<R>* tw = reinterpret_cast<cx<R>*>(mix_smem);
  cx<R>* buf = tw + L;
  int t, j;
  if (Op::kLM) { t = threadIdx.x / C::TPL; j = threadIdx.x % C::TPL; }
  else { j = threadIdx.x / C::T; t = threadIdx.x % C::T; }
  int o = Op::kLM ? blockIdx.x * C::T + t : blockIdx.y;
  int x = Op::kLM ? 0 : blockIdx.x * C::T + t;
  bool ok;
  static_assert(!Op::kNyqTail || (Op::kRed == 0 && !Op::kLM), "the remapped CTAs that exit write no partial sums");
  if constexpr (Op::kNyqTail) {
    // as in k_fast: the last block column takes column Nx of T rows
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
  unsigned char* pre = mix_smem + MixSmem<R, L>::bytes;
  constexpr int EH = Op::kHalfOut ? C::E / 2 : C::E;  // elements stored (the crop keeps positions < L/2)
  constexpr bool kUsePre = MixUsesPre<L, Op>::value;
  if constexpr (kUsePre) {
    if (ok) {
#pragma unroll
      for (int e = 0; e < EH; ++e)
        op.prefetch(o, x, j + C::TPL * e, pre + ((size_t)e * kThreads + threadIdx.x) * Op::kPre);
    }
    cp_async_commit();
  }
  cx<R> v[C::E];
#pragma unroll
  for (int e = 0; e < C::E; ++e)
    v[e] = (ok && (!Op::kZeroUpper || e < C::E / 2)) ? op.load(o, x, j + C::TPL * e) : czero<R>();
  for (int i = threadIdx.x; i < L; i += kThreads) tw[i] = twg[i];
  __syncthreads();
  constexpr int NR = Op::kRed > 0 ? Op::kRed : 1;
  R acc[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) acc[s] = (R)0;
  mix_fft<R, L, Op::kSign1, Op::kLM>(v, buf, tw, t, j);
  if constexpr (Op::kMirror) {
    // exchange so every thread sees the frequency L - k of each of its k
#pragma unroll
    for (int e = 0; e < C::E; ++e) buf[msa<R, L, Op::kLM>(t, j + C::TPL * e)] = v[e];
    __syncthreads();
    if (ok) {
#pragma unroll
      for (int e = 0; e < C::E; ++e) {
        const int k = j + C::TPL * e;
        op.post(o, x, k, v[e], buf[msa<R, L, Op::kLM>(t, k == 0 ? 0 : L - k)], acc);
      }
    }
  } else {
    if (ok) {
#pragma unroll
      for (int e = 0; e < C::E; ++e) op.spectral(o, x, j + C::TPL * e, v[e], acc);
    }
    if (Op::kSecond) mix_fft<R, L, -Op::kSign1, Op::kLM>(v, buf, tw, t, j);
    if constexpr (kUsePre) {
      cp_async_wait_all();
      if (ok) {
#pragma unroll
        for (int e = 0; e < EH; ++e)
          op.store_pre(o, x, j + C::TPL * e, v[e], acc, pre + ((size_t)e * kThreads + threadIdx.x) * Op::kPre);
      }
    } else if (ok) {
#pragma unroll
      for (int e = 0; e < EH; ++e) op.store(o, x, j + C::TPL * e, v[e], acc);
    }
  }
  if (Op::kRed > 0) reduce_out<R, NR>(acc, op.part, op.pstride);
}

template <typename R, int L, class Op>
inline cudaError_t launch_mix_L(const Op& op, const FftLen& f, const PassGrid& pg, cudaStream_t st) {
  static std::atomic<unsigned long long> prepared{0};
  const size_t sm = MixSmem<R, L>::bytes + (MixUsesPre<L, Op>::value ? (size_t)Op::kPre * MixCfg<L>::E * kThreads : 0);
  cudaError_t e = ensure_smem(prepared, k_mix<R, L, Op>, sm);
  if (e != cudaSuccess) return e;
  k_mix<R, L, Op><<<pg.grid, kThreads, sm, st>>>(op, tw_table_host<R>(f));
  return cudaGetLastError();
}

}  // namespace atkm
