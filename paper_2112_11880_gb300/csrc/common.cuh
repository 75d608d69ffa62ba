// Shared device helpers of libhelm: complex arithmetic on interleaved
// (re, im) pairs, cache-hinted loads, deterministic block reductions and the
// device clock.
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

// Warp sum of K doubles with a transposed butterfly: at the first exchange
// (and for K > 2 the second) each lane keeps only half of the values it
// carries, so a lane adds K/2 + K/4 + 3 values instead of 5 K -- every FP64
// add is a full warp instruction on GB300 whatever the number of useful
// lanes.  The sum of component k ends in lane lane_of<K>(k).  Fixed pattern:
// bit-for-bit reproducible.
template <int K>
__device__ __forceinline__ int warp_sum_lane(int k) {
  return K == 1 ? 0 : (K == 2 ? (k & 1) * 16 : ((k & 1) * 16 + ((k >> 1) & 1) * 8));
}
template <int K>
__device__ __forceinline__ double warp_sum_t(const double (&v)[K]) {
  const int lane = threadIdx.x & 31;
  if (K == 1) {
    double a = v[0];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    return a;
  } else if (K == 2) {
    const bool up = lane & 16;
    double keep = up ? v[1] : v[0];
    keep += __shfl_xor_sync(0xffffffffu, up ? v[0] : v[1], 16);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, off);
    return keep;  // lane 0: v[0], lane 16: v[1]
  } else {
    // K = 3 or 4 (v[3] = 0 for K = 3): keep components {0,2} / {1,3} across
    // the 16-exchange, then {0}/{2} resp. {1}/{3} across the 8-exchange
    const double w3 = K > 3 ? v[K > 3 ? 3 : 0] : 0.0;
    const bool up16 = lane & 16, up8 = lane & 8;
    double a = up16 ? v[1] : v[0];
    double b = up16 ? w3 : v[2];
    a += __shfl_xor_sync(0xffffffffu, up16 ? v[0] : v[1], 16);
    b += __shfl_xor_sync(0xffffffffu, up16 ? v[2] : w3, 16);
    double keep = up8 ? b : a;
    keep += __shfl_xor_sync(0xffffffffu, up8 ? a : b, 8);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, off);
    return keep;  // lane 0: v[0], 16: v[1], 8: v[2], 24: v[3]
  }
}

// Sum K doubles over the block: warp sums (transposed butterfly), then the
// warp sums of each component added in warp order by one lane per component
// (at most 32 warps).  Result valid in thread 0.  `red` holds 32*K doubles.
// Ends with a __syncthreads so `red` can be reused.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  const double ws = warp_sum_t<K>(v);
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (lane == warp_sum_lane<K>(k)) red[warp * K + k] = ws;
  __syncthreads();
  if (warp == 0) {
    // lane k adds the K-th component over warps in order (one chain each)
    double s = 0.0;
    if (lane < K) {
      for (int w = 0; w < nwarps; ++w) s += red[w * K + lane];
    }
    // gather to thread 0
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double sk = __shfl_sync(0xffffffffu, s, k);
      if (lane == 0) v[k] = sk;
    }
  }
  __syncthreads();
}

// Publish this block's K partial sums, then let the last block to arrive
// (ticket counter) add all partials in block-index order.  Returns true in
// every thread of the last block; `tot` then holds the totals in thread 0.
// The counter is reset by the last block, so a kernel can use it again in its
// next launch.
template <int K, int B = 4>
__device__ __forceinline__ bool grid_sum_last(double (&v)[K], double* partials,
                                              unsigned int* ticket, double* red, double (&tot)[K]) {
  static_assert(B % 4 == 0, "B is a multiple of the four accumulators");
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
  // Thread j sums partials j + T m into accumulator m mod 4, then adds the
  // four accumulators in order: a fixed order for every addition (four
  // independent FP64 chains hide the DADD latency); the block tree follows.
  double acc[K], acc4[4][K];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < K; ++k) acc4[q][k] = 0.0;
  // B partials are loaded before they are added (one L2 round trip per B);
  // partial j + T m goes to accumulator m mod 4 whatever B is.
  const unsigned int T = blockDim.x;
  unsigned int b = threadIdx.x;
  for (; b + (B - 1) * T < gridDim.x; b += B * T) {
    double w[B][K];
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) w[q][k] = ld_cg(&partials[(size_t)(b + q * T) * K + k]);
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) acc4[q & 3][k] += w[q][k];
  }
#pragma unroll
  for (int q = 0; q < B - 1; ++q) {
    if (b + q * T < gridDim.x) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc4[q & 3][k] += ld_cg(&partials[(size_t)(b + q * T) * K + k]);
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

// Two-level form for grids of many small blocks: blocks form groups of
// blockDim.x consecutive blocks; the last block of a group to arrive adds the
// group's partials (one per thread) and stores the group sum after the block
// partials; the last group to finish adds the group sums.  Each level adds in
// a fixed order (thread j takes member j, then the fixed block tree), so the
// result does not depend on arrival order.  gticket holds one counter per
// group (at most 256 groups); partials holds gridDim.x * K + groups * K
// doubles.  The total is valid in thread 0 of the returning block.
template <int K>
__device__ __forceinline__ bool grid_sum_last2(double (&v)[K], double* partials, unsigned int* ticket,
                                               unsigned int* gticket, double* red, double (&tot)[K]) {
  __shared__ bool s_go;
  block_sum<K>(v, red);
  const unsigned int T = blockDim.x;
  const unsigned int g = blockIdx.x / T, ng = (gridDim.x + T - 1) / T;
  const unsigned int g0 = g * T, gn = min(T, gridDim.x - g0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    s_go = atomicAdd(&gticket[g], 1u) == gn - 1;
  }
  __syncthreads();
  if (!s_go) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned int j = threadIdx.x; j < gn; j += T)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += ld_cg(&partials[(size_t)(g0 + j) * K + k]);
  block_sum<K>(acc, red);
  double* gpart = partials + (size_t)gridDim.x * K;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) gpart[(size_t)g * K + k] = acc[k];
    gticket[g] = 0u;
    __threadfence();
    s_go = atomicAdd(ticket, 1u) == ng - 1;
  }
  __syncthreads();
  if (!s_go) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned int j = threadIdx.x; j < ng; j += T)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += ld_cg(&gpart[(size_t)j * K + k]);
  block_sum<K>(acc, red);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = acc[k];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// ---------------------------------------------------------------- timers

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Device error flags (bit set by a kernel that had to give up).
enum : unsigned int { DEVERR_BARRIER_TIMEOUT = 2u };

}  // namespace helm
