// Shared device helpers of libhelm: complex arithmetic on interleaved
// (re, im) pairs, cache-hinted loads, deterministic block reductions, the
// TMA bulk-copy / mbarrier primitives used to stage CSR tiles, and the
// handle layout.
//
// FP64 on this GPU: the FP64 pipe retires about two FMA lanes per clock per
// SM (about 1.2 TFLOP/s for the chip), 60x below FP32, and a warp
// instruction costs the same however many lanes are active.  Every complex
// kernel here is therefore written to issue as few warp-level FP64
// instructions as possible: one thread per CSR row (no shuffle trees inside a
// row), partial dot products kept per thread across all tiles a block visits
// and reduced once per launch, and scalar work confined to one thread.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/helm.h"

namespace helm {

// ---------------------------------------------------------------- complex

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a * b   (4 DFMA)
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc - a * b   (4 DFMA)
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b   (4 DFMA)
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc + |a|^2   (2 DFMA)
__device__ __forceinline__ double cabs2_acc(double2 a, double acc) {
  acc = fma(a.x, a.x, acc);
  return fma(a.y, a.y, acc);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm (Smith 1962) for robustness against overflow.
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
// a / b with one real division: a conj(b) / |b|^2 (the scalar recurrences run
// in one thread between kernels, where every dependent division is latency);
// Smith's algorithm when |b|^2 under- or overflows.
__device__ __forceinline__ double2 cdiv_fast(double2 a, double2 b) {
  const double d = fma(b.x, b.x, b.y * b.y);
  if (!(d > 0.0) || !isfinite(d) || d < 1e-290) return cdiv(a, b);
  const double inv = 1.0 / d;
  return make_double2(fma(a.x, b.x, a.y * b.y) * inv, fma(a.y, b.x, -a.x * b.y) * inv);
}
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }
__device__ __forceinline__ bool czero(double2 a) { return a.x == 0.0 && a.y == 0.0; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cfma32(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}

// complex64 counterparts (FP32 pipe)
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) { return cfma32(a, b, acc); }
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float cabs2_acc(float2 a, float acc) {
  acc = fmaf(a.x, a.x, acc);
  return fmaf(a.y, a.y, acc);
}

// ---------------------------------------------------------------- loads

// Matrix entries are read once per SpMV: stream them (evict-first).
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
// Gathered vector entries are reused by neighbouring rows: read-only path.
__device__ __forceinline__ double2 ld_gather(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_gather(const float2* p) { return __ldg(p); }
// Values written by other blocks of the same launch: bypass L1.
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

// ---------------------------------------------------------------- reductions

// Sum K doubles over the block, fixed shuffle pattern then warps in order.
// Result valid in thread 0.  `red` must hold 32*K doubles.  Ends with a
// __syncthreads so `red` can be reused.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = red[k];
      for (int w = 1; w < nwarps; ++w) s += red[w * K + k];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Publish this block's K partial sums, then let the last block to arrive
// (ticket counter) add all partials in block-index order.  Returns true in
// every thread of the last block; `tot` then holds the totals in thread 0.
// The counter is reset by the last block, so a kernel can use it again in its
// next launch.
template <int K>
__device__ __forceinline__ bool grid_sum_last(double (&v)[K], double* partials,
                                              unsigned int* ticket, double* red, double (&tot)[K]) {
  __shared__ bool s_last;
  block_sum<K>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // Thread j sums partials j + T (4 m + q) into accumulator q, then adds the
  // four accumulators in order: a fixed order for every addition (four
  // independent FP64 chains hide the DADD latency); the block tree follows.
  double acc[K], acc4[4][K];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < K; ++k) acc4[q][k] = 0.0;
  const unsigned int T = blockDim.x;
  unsigned int b = threadIdx.x;
  for (; b + 3 * T < gridDim.x; b += 4 * T) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) acc4[q][k] += ld_cg(&partials[(size_t)(b + q * T) * K + k]);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (b + q * T < gridDim.x) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc4[q][k] += ld_cg(&partials[(size_t)(b + q * T) * K + k]);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = (acc4[0][k] + acc4[1][k]) + (acc4[2][k] + acc4[3][k]);
  block_sum<K>(acc, red);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = acc[k];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// ---------------------------------------------------------------- TMA bulk copy

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared, completion counted on `bar` (bytes, 16-byte
// multiple; both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: gives up after `limit_ns` and returns
// false.  No unbounded spin anywhere in the library.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Device error flags (bit set by a kernel that had to give up).
enum : unsigned int { DEVERR_MBAR_TIMEOUT = 1u, DEVERR_BARRIER_TIMEOUT = 2u };

}  // namespace helm
