// CSR SpMV tile engine (Section 3, Table 8 of the paper: CSR SpMV, 8 flops
// per stored entry in complex arithmetic), for complex128 and complex64.
//
// Layout and schedule, chosen for GB300:
//   * A tile is R = 32 consecutive rows; its stored entries are one
//     contiguous range [s, e) of the values / colind.  One elected thread
//     copies that range into shared memory with two TMA bulk copies
//     (cp.async.bulk, completion on an mbarrier, bounded wait).  HBM sees
//     long, fully coalesced streams; no thread issues per-entry global loads
//     for the matrix.
//   * Complex128 tiles whose entries are all real (Helmholtz FEM rows away
//     from the impedance boundary) are staged from a copy of the real parts
//     and take the real x complex product: 12 instead of 20 bytes per entry
//     and 2 instead of 4 FP64 FMA.  Tiles with a complex entry read the
//     matrix directly from global memory.
//   * Single buffer per block and many small blocks per SM: the copies of
//     some blocks overlap the arithmetic of others.  Each block has R * SPLIT
//     threads; a row's entries are split between SPLIT threads, whose sums
//     meet in shared memory.  No shuffle tree inside a row: the FP64 pipe is
//     what bounds this kernel on GB300.
//   * x is gathered through the read-only path; for FEM orderings the 27
//     neighbours of consecutive rows share cache lines.
//   * Persistent grid (resident blocks x SMs); each block walks tiles
//     blockIdx.x, blockIdx.x + gridDim.x, ...  The epilogue object keeps the
//     block's partial dot products in registers across all its tiles.
//   * A tile with more than CAP entries (very long rows) is multiplied
//     directly from global memory instead; rows of any length are correct.
//   * Bulk copies need 16-byte aligned, 16-byte multiple ranges: each range
//     is widened to the enclosing 16-byte groups, except past the last whole
//     group of the array, where the few trailing entries are read directly.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.hpp"

// Unroll of the staged row loops: how many x gathers a thread has in flight.
#ifndef HELM_SPMV_UNROLL
#define HELM_SPMV_UNROLL 4
#endif

namespace helm {

constexpr int kSpmvUnroll = HELM_SPMV_UNROLL;

// Real type of a complex type.
template <class V> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <class V>
struct CsrDev {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const V* vals;
  // Optional: real_blk[r >> 5] != 0 when every stored
  // entry of rows [32 (r >> 5), 32 (r >> 5) + 32) has a zero imaginary part.
  // Those rows take the real x complex product (2 FMA per entry instead of
  // 4); for finite x the result is bit-identical to the complex product,
  // since the skipped terms are exact zeros.  Helmholtz FEM rows away from
  // the impedance boundary are of this kind (A = K - k^2 M + i k B).
  const uint8_t* real_blk;
  // Optional: the real parts of vals.  Real blocks are staged from it: 8
  // (complex128) or 4 (complex64) bytes per entry in HBM and shared memory
  // instead of 16 or 8.  Without it (or real_blk) no tile is staged.
  const typename RealOf<V>::T* vals_re;
};

// Row sum of a complex128 row whose entries are all real: reads only the
// real parts.
__device__ __forceinline__ double2 mac_real(double a, double2 x, double2 acc) {
  acc.x = fma(a, x.x, acc.x);
  acc.y = fma(a, x.y, acc.y);
  return acc;
}
__device__ __forceinline__ float2 mac_real(float a, float2 x, float2 acc) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  return acc;
}
template <class V>
__device__ __forceinline__ bool row_block_real(const CsrDev<V>& A, int64_t r) {
  return A.real_blk != nullptr && A.vals_re != nullptr && A.real_blk[r >> 5] != 0;
}

__device__ __forceinline__ double2 mac(double2 a, double2 x, double2 acc) { return cfma(a, x, acc); }
__device__ __forceinline__ float2 mac(float2 a, float2 x, float2 acc) { return cfma32(a, x, acc); }
template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }

// Type of a staged value: tiles are staged only when all their entries are
// real, as their real parts.
template <class V> struct StagedVal { using T = typename RealOf<V>::T; };

// Shared-memory footprint of the staged engine: STAGES buffers of CAP
// entries each.
template <class V, int CAP, int STAGES = 2>
struct SpmvStage {
  using T = typename StagedVal<V>::T;
  static_assert(CAP % 4 == 0, "CAP must be a multiple of 4");
  static_assert(STAGES == 1 || STAGES == 2, "one or two buffers");
  static constexpr int kVG = 16 / sizeof(T);  // staged values per 16-byte group
  static constexpr size_t kValsBytes = sizeof(T) * (CAP + 2 * kVG);
  static constexpr size_t kColsBytes = sizeof(int32_t) * (CAP + 8);
  static constexpr size_t kBytes = STAGES * (kValsBytes + kColsBytes) + 2 * sizeof(uint64_t);
  static_assert(kValsBytes % 16 == 0 && kColsBytes % 16 == 0, "16-byte aligned buffers");
};

template <class V> __device__ __forceinline__ V vadd(V a, V b) { return cadd(a, b); }

// multiply-accumulate with a staged (real) value
__device__ __forceinline__ double2 mac_staged(double a, double2 x, double2 acc) { return mac_real(a, x, acc); }
__device__ __forceinline__ float2 mac_staged(float a, float2 x, float2 acc) { return mac_real(a, x, acc); }

// Walk this block's tiles; call epi.row(r, acc) for each row r with
// acc = sum_k vals[k] * x[colind[k]].  epi.prefetch(r) is called by the same
// thread before the row's sum starts (while the tile's copy is in flight), so
// the epilogue can issue its own loads early.  Returns false if a bulk copy
// never completed (error flag set).  Must be called by all threads of the
// block.
//
// Staged tiles: tiles whose entries are all real (copied from vals_re), with
// at most CAP entries.  Other tiles (a complex entry -- for Helmholtz FEM
// only the rows at the impedance boundary -- or very long rows) are
// multiplied with direct loads of vals / colind.
//
// STAGES = 2: the copy of a block's next tile overlaps the current tile.
// STAGES = 1: half the shared memory per block, so more blocks share an SM
// and overlap one another instead.
//
// SPLIT > 1: the block has R * SPLIT threads and thread t takes the entries
// k = k0 + (t / R), k0 + (t / R) + SPLIT, ... of row t % R (more warps per
// staged tile, each with a shorter dependent chain); the SPLIT partial sums
// of a row are added in a fixed order through shared memory, and only the
// threads t < R call epi.row.
// gate(): called by every thread once, after the block's first tile copy is
// issued and before anything else is read (a kernel's wait for its
// predecessor goes there, so the matrix copy overlaps the predecessor's
// tail).  It must return the same value in every thread of the block; on
// false the engine lets the copy land and returns without touching x or
// calling the epilogue.
struct NoGate {
  __device__ __forceinline__ bool operator()() const { return true; }
};

template <class V, int R, int CAP, class Epi, int STAGES = 2, int SPLIT = 1, class Gate = NoGate>
__device__ __forceinline__ bool spmv_tiles(const CsrDev<V>& A, const V* __restrict__ x, Epi& epi,
                                           unsigned char* smem, unsigned int* dev_err, Gate gate = Gate()) {
  using S = SpmvStage<V, CAP, STAGES>;
  using T = typename S::T;
  static_assert(R == 32, "tiles are the 32-row blocks of real_blk");
  __shared__ V s_part[SPLIT > 1 ? (SPLIT - 1) * R : 1];
  const int part = SPLIT > 1 ? static_cast<int>(threadIdx.x) / R : 0;
  const int lrow = SPLIT > 1 ? static_cast<int>(threadIdx.x) % R : static_cast<int>(threadIdx.x);
  constexpr int VG = S::kVG;
  // buffer b: values at smem + b * kValsBytes, columns after the value buffers
  auto sv = [&](int b) { return reinterpret_cast<T*>(smem + b * S::kValsBytes); };
  auto sc = [&](int b) {
    return reinterpret_cast<int32_t*>(smem + STAGES * S::kValsBytes + b * S::kColsBytes);
  };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + STAGES * (S::kValsBytes + S::kColsBytes));
  const T* stage_src = A.vals_re;  // source of the staged values

  const int32_t n = A.n;
  const int32_t ntiles = (n + R - 1) / R;
  const int64_t cend = A.nnz & ~int64_t(3);        // last whole 16-byte group of colind
  const int64_t vend = A.nnz & ~int64_t(VG - 1);   // same for the staged values

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  struct Range {
    int64_t s, e, va0, va1, ca0, ca1;
    bool staged;
  };
  auto range_of = [&](int32_t t) {
    Range g;
    const int32_t r0 = t * R;
    const int32_t r1 = min(r0 + R, n);
    g.s = A.rowptr[r0];
    g.e = A.rowptr[r1];
    g.staged = (g.e - g.s) <= CAP && A.vals_re != nullptr && A.real_blk != nullptr && A.real_blk[t] != 0;
    g.va0 = g.s & ~int64_t(VG - 1);
    g.va1 = min((g.e + VG - 1) & ~int64_t(VG - 1), vend);
    g.ca0 = g.s & ~int64_t(3);
    g.ca1 = min((g.e + 3) & ~int64_t(3), cend);
    return g;
  };
  // Elected thread: stage tile t into buffer b (or only arrive when the tile
  // is not staged, so that every use of a buffer completes one phase).
  auto issue = [&](int32_t t, int b) {
    const Range g = range_of(t);
    uint32_t vbytes = 0, cbytes = 0;
    if (g.staged && g.e > g.s) {
      if (g.va1 > g.va0) vbytes = static_cast<uint32_t>((g.va1 - g.va0) * sizeof(T));
      if (g.ca1 > g.ca0) cbytes = static_cast<uint32_t>((g.ca1 - g.ca0) * sizeof(int32_t));
    }
    mbar_expect_tx(&bar[b], vbytes + cbytes);
    if (vbytes) bulk_g2s(sv(b), stage_src + g.va0, vbytes, &bar[b]);
    if (cbytes) bulk_g2s(sc(b), A.colind + g.ca0, cbytes, &bar[b]);
  };

  bool ok = true;
  int fail_it = 0;
  bool fail_next = false;
  int32_t tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);  // the first copy
  if (!gate()) {
    if (tile < ntiles) (void)mbar_wait_bounded(&bar[0], 0, 100000000ull);
    return true;
  }
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = STAGES == 2 ? (it & 1) : 0;
    const int32_t next = tile + gridDim.x;
    if (threadIdx.x == 0) {
      if (STAGES == 2) {
        if (next < ntiles) {
          fence_proxy_async();  // buffer b^1 was last read through the generic proxy
          issue(next, b ^ 1);
        }
      } else if (it > 0) {
        fence_proxy_async();  // the single buffer was last read through the generic proxy
        issue(tile, 0);
      }
    }
    const Range g = range_of(tile);
    // The row's bounds, its real-block flag and the epilogue's operands are
    // loaded while the tile's copy is in flight.
    const int32_t r = tile * R + lrow;
    const bool row_ok = r < min(tile * R + R, n);
    int64_t k0 = 0, k1 = 0;
    bool rreal = false;
    if (row_ok) {
      k0 = A.rowptr[r] + part;
      k1 = A.rowptr[r + 1];
      rreal = row_block_real(A, r);
      if (part == 0) epi.prefetch(r);
    }
    const uint32_t parity = STAGES == 2 ? ((it >> 1) & 1) : (it & 1);
    // Every thread observes the phase (visibility of the async-proxy
    // writes); the give-up decision is made block-uniform by the vote.
    const bool got = mbar_wait_bounded(&bar[b], parity, 2000000000ull);
    if (!__syncthreads_and(got)) {
      if (threadIdx.x == 0) atomicOr(dev_err, DEVERR_MBAR_TIMEOUT);
      ok = false;
      fail_it = it;
      fail_next = STAGES == 2 && next < ntiles;
      break;
    }
    V acc = vzero<V>();
    if (row_ok) {
      constexpr int KS = SPLIT;
      if (g.staged) {
        const T* v = sv(b) - g.va0;
        const int32_t* c = sc(b) - g.ca0;
        if (g.e <= g.va1 && g.e <= g.ca1) {
#pragma unroll kSpmvUnroll
          for (int64_t k = k0; k < k1; k += KS) acc = mac_staged(v[k], ld_gather(x + c[k]), acc);
        } else {  // entries past the last whole 16-byte group: plain loads
#pragma unroll 2
          for (int64_t k = k0; k < k1; k += KS) {
            const T a = (k < g.va1) ? v[k] : stage_src[k];
            const int32_t col = (k < g.ca1) ? c[k] : ld_stream(A.colind + k);
            acc = mac_staged(a, ld_gather(x + col), acc);
          }
        }
      } else {
        bool done = false;
        if (rreal) {  // real rows of a tile too long to stage
#pragma unroll 4
          for (int64_t k = k0; k < k1; k += KS)
            acc = mac_real(__ldcs(A.vals_re + k), ld_gather(x + ld_stream(A.colind + k)), acc);
          done = true;
        }
        if (!done) {
#pragma unroll 4
          for (int64_t k = k0; k < k1; k += KS)
            acc = mac(ld_stream(A.vals + k), ld_gather(x + ld_stream(A.colind + k)), acc);
        }
      }
    }
    if (SPLIT > 1) {
      if (part > 0) s_part[(part - 1) * R + lrow] = acc;
      __syncthreads();
      if (part == 0 && row_ok) {
#pragma unroll
        for (int q = 1; q < SPLIT; ++q) acc = vadd(acc, s_part[(q - 1) * R + lrow]);
      }
    }
    if (part == 0 && row_ok) epi.row(r, acc);
    __syncthreads();  // buffer b fully consumed before it is refilled
  }
  if (!ok) {
    // Let the copies still in flight land (bounded) before the block's
    // shared memory is released.
    if (STAGES == 2) {
      (void)mbar_wait_bounded(&bar[fail_it & 1], (fail_it >> 1) & 1, 100000000ull);
      if (fail_next)
        (void)mbar_wait_bounded(&bar[(fail_it + 1) & 1], ((fail_it + 1) >> 1) & 1, 100000000ull);
    } else {
      (void)mbar_wait_bounded(&bar[0], fail_it & 1, 100000000ull);
    }
  }
  return ok;
}

// The engine configuration every SpMV-shaped kernel of the library uses.
template <class V> struct Engine;
template <> struct Engine<double2> {
  static constexpr int R = kRows128, CAP = kCap128, SPLIT = kSplit;
  static constexpr int kThreads = R * SPLIT;
  static constexpr size_t kSmem = SpmvStage<double2, CAP, kStages>::kBytes;
};
template <> struct Engine<float2> {
  static constexpr int R = kRows64, CAP = kCap64, SPLIT = kSplit;
  static constexpr int kThreads = R * SPLIT;
  static constexpr size_t kSmem = SpmvStage<float2, CAP, kStages>::kBytes;
};
template <class V, class Epi, class Gate = NoGate>
__device__ __forceinline__ bool spmv_run(const CsrDev<V>& A, const V* __restrict__ x, Epi& epi, unsigned char* smem,
                                         unsigned int* dev_err, Gate gate = Gate()) {
  return spmv_tiles<V, Engine<V>::R, Engine<V>::CAP, Epi, kStages, Engine<V>::SPLIT, Gate>(A, x, epi, smem, dev_err,
                                                                                           gate);
}

}  // namespace helm
