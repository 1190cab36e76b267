// BF16 GEMM on the fifth-generation tensor cores (tcgen05), for the learned-
// guess network's dense contractions.
//
// D[M x N] = A[M x K] B[K x N] with FP32 operands in global memory (any
// strides), rounded to BF16 (round to nearest even) when staged, products
// accumulated in FP32 in tensor memory; D(m, n) is stored to C[m*scm + n*scn]
// (or added atomically when K is split over gridDim.z; the caller zeroes C).
//
// One CTA of 128 threads computes a 128 x BN tile.  Every thread stages a
// 64-wide K slice of A (128 rows) and B (BN rows) into shared memory in the
// canonical K-major layout without swizzle: 8 x 8 "core matrices" of 128
// contiguous bytes (8 rows of 16 bytes), the two core matrices of one 16-wide
// K step next to each other (leading-byte offset 128) and consecutive groups
// of 8 rows 1024 bytes apart (stride-byte offset).  Thread 0 issues the four
// tcgen05.mma (M = 128, N = BN, K = 16 each) of the slice and commits them to
// the stage's mbarrier; the slices alternate between two stages, so the next
// slice is staged while the tensor core works.  The accumulator lives in BN
// tensor-memory columns (lane m = row m of the tile), allocated by warp 0 and
// read back by each warp's quarter of the lanes with tcgen05.ld.
//
// Every mbarrier wait is bounded: a wait that gives up sets *err, the CTA
// stops issuing, waits once more (bounded) for what it already issued, frees
// its tensor memory and leaves.  With wait_test set, each CTA instead waits
// (1000 polls) on an mbarrier that nothing arrives at before issuing any MMA,
// gives up, and takes that path: a check of the error reporting that leaves
// no tensor-core work in flight.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace atkm {
namespace tc {

constexpr int kM = 128;       // tile rows (tensor-memory lanes)
constexpr int kKC = 64;       // K elements staged per slice (4 MMAs of K = 16)
constexpr int kThreads = 128;
constexpr uint32_t kSbo = (kKC / 8) * 128;  // bytes between groups of 8 rows
constexpr uint32_t kLbo = 128;              // bytes between the two core matrices of a K step
constexpr long kWaitPolls = 1L << 22;       // try_wait polls before a wait gives up

template <int BN> struct Cfg {
  static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
  static constexpr uint32_t kABytes = kM * kKC * 2;
  static constexpr uint32_t kBBytes = BN * kKC * 2;
  static constexpr uint32_t kStage = kABytes + kBBytes;
  static constexpr uint32_t kSmem = 2 * kStage + 128;  // + alignment slack
  static constexpr uint32_t kCols = BN;                // tensor-memory columns (power of two >= 32)
  // instruction descriptor of kind::f16: D F32 (bits 4-5 = 1), A and B BF16
  // (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
  // bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t kIdesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading- and stride-byte offsets
// (each >> 4, 14 bits), the descriptor version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(cols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// true once the phase of the given parity has completed; false after `polls` polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long polls = kWaitPolls) {
  for (long i = 0; i < polls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 8 consecutive FP32 columns of this thread's lane (warp w reads lanes 32w ...)
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// byte offset of element (row, k) of a staged slice
__device__ __forceinline__ uint32_t soff(int row, int k) {
  return (uint32_t)(row >> 3) * kSbo + (uint32_t)(k >> 3) * kLbo + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // .x = lo (lower address)
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float ldx(const float* __restrict__ X, long sr, long sk, int r, int k, int rows, int k1) {
  return (r < rows && k < k1) ? __ldg(X + (long)r * sr + (long)k * sk) : 0.f;
}

// rows [r0, r0 + R) x K slice [k0, k1) of X(r, k) = X[r*sr + k*sk] into dst.
// K contiguous (sk = 1): a thread converts 8 consecutive k of one row (two
// float4 loads) into one 16-byte row of a core matrix.  Rows contiguous
// (sr = 1): a thread loads a 4-row x 8-k block (eight float4 along the rows)
// and writes four 16-byte core-matrix rows.  Both need X and the other
// stride 16-byte aligned; ragged edges take scalar loads, anything else the
// scalar path.
template <int R>
__device__ __forceinline__ void stage(unsigned char* dst, const float* __restrict__ X, long sr, long sk, int r0,
                                      int rows, int k0, int k1) {
  const bool a16 = ((uintptr_t)X & 15) == 0;
  if (sk == 1 && a16 && (sr & 3) == 0) {
    for (int e = threadIdx.x; e < R * (kKC / 8); e += kThreads) {
      const int rr = e >> 3, g = e & 7;
      const int r = r0 + rr, k = k0 + 8 * g;
      float v[8];
      if (r < rows && k + 8 <= k1) {
        const float4* src = reinterpret_cast<const float4*>(X + (long)r * sr + k);
        const float4 a = __ldg(src), b = __ldg(src + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = ldx(X, sr, 1, r, k + j, rows, k1);
      }
      *reinterpret_cast<uint4*>(dst + soff(rr, 8 * g)) =
          make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
    }
  } else if (sr == 1 && a16 && (sk & 3) == 0) {
    for (int e = threadIdx.x; e < (R / 4) * (kKC / 8); e += kThreads) {
      const int q = e % (R / 4), g = e / (R / 4);
      const int rr = 4 * q, r = r0 + rr, kb = k0 + 8 * g;
      float v[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = kb + j;
        if (r + 4 <= rows && k < k1) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(X + (long)k * sk + r));
          v[j][0] = a.x; v[j][1] = a.y; v[j][2] = a.z; v[j][3] = a.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) v[j][i] = ldx(X, 1, sk, r + i, k, rows, k1);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<uint4*>(dst + soff(rr + i, 8 * g)) =
            make_uint4(pack2(v[0][i], v[1][i]), pack2(v[2][i], v[3][i]), pack2(v[4][i], v[5][i]),
                       pack2(v[6][i], v[7][i]));
    }
  } else {
    const bool kfast = sk == 1;
    for (int e = threadIdx.x; e < R * kKC; e += kThreads) {
      int rr, kk;
      if (kfast) { rr = e / kKC; kk = e - rr * kKC; }
      else { kk = e / R; rr = e - kk * R; }
      *reinterpret_cast<__nv_bfloat16*>(dst + soff(rr, kk)) =
          __float2bfloat16_rn(ldx(X, sr, sk, r0 + rr, k0 + kk, rows, k1));
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
k_gemm_tc(const float* __restrict__ A, long sam, long sak, const float* __restrict__ Bm, long sbk, long sbn,
          float* __restrict__ C, long scm, long scn, int M, int N, int K, int kchunk, unsigned* err,
          int wait_test) {
  using G = Cfg<BN>;
  extern __shared__ __align__(128) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long bars[3];  // [2]: the wait_test barrier
  __shared__ uint32_t tbase;
  const uint32_t raw = smem_u32(tc_smem);
  unsigned char* base = tc_smem + (((raw + 127u) & ~127u) - raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  if (warp == 0) tmem_alloc(smem_u32(&tbase), G::kCols);
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bars[0]));
    mbar_init(smem_u32(&bars[1]));
    mbar_init(smem_u32(&bars[2]));
    fence_async_smem();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tbase;
  uint32_t phase[2] = {0u, 0u};
  int it = 0;
  bool bad = false;
  if (wait_test) bad = __syncthreads_or(!mbar_wait(smem_u32(&bars[2]), 0u, 1000)) != 0;
  for (int k0 = kb; k0 < ke && !bad; k0 += kKC, ++it) {
    const int s = it & 1;
    unsigned char* sA = base + s * G::kStage;
    unsigned char* sB = sA + G::kABytes;
    if (it >= 2) {  // the MMAs of slice it - 2 read this stage
      const bool ok = mbar_wait(smem_u32(&bars[s]), phase[s]);
      phase[s] ^= 1u;
      if (__syncthreads_or(!ok)) { bad = true; break; }
    }
    stage<kM>(sA, A, sam, sak, m0, M, k0, ke);
    stage<BN>(sB, Bm, sbn, sbk, n0, N, k0, ke);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int q = 0; q < kKC / 16; ++q)
        mma_bf16(tmem, sdesc(a0 + q * 2 * kLbo, kLbo, kSbo), sdesc(b0 + q * 2 * kLbo, kLbo, kSbo), G::kIdesc,
                 (it > 0 || q > 0) ? 1u : 0u);
      commit(smem_u32(&bars[s]));
    }
  }
  // the last commit covers every MMA this CTA issued
  if (it > 0) {
    const int s = (it - 1) & 1;
    const bool ok = mbar_wait(smem_u32(&bars[s]), phase[s]);
    bad = __syncthreads_or(bad || !ok) != 0;
  }
  fence_after();
  if (bad) {
    if (threadIdx.x == 0) atomicOr(err, 1u);
  } else {
    const bool split = gridDim.z > 1;
    const int m = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 8) {
      float v[8];
      if (it > 0) {
        ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
      }
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + c0 + j;
          if (n < N) {
            float* dst = C + (long)m * scm + (long)n * scn;
            if (split) atomicAdd(dst, v[j]);
            else *dst = v[j];
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, G::kCols);
}

}  // namespace tc
}  // namespace atkm
