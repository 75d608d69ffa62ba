// CSR SpMV tile engine (Section 3, Table 8 of the paper: CSR SpMV, 8 flops
// per stored entry in complex arithmetic), for complex128 and complex64.
//
// Layout and schedule, chosen for GB300:
//   * A tile is R consecutive rows; its stored entries are one contiguous
//     range [s, e) of vals / colind.  One elected thread copies that range
//     into shared memory with two TMA bulk copies (cp.async.bulk, completion
//     on an mbarrier), double-buffered: while the block multiplies tile i the
//     copy of its next tile is in flight.  HBM sees long, fully coalesced
//     streams; no thread issues per-entry global loads for the matrix.
//   * One thread per row.  The complex multiply-accumulate is 4 FMA per
//     entry and, for complex128, nothing else runs on the FP64 pipe inside a
//     row (no shuffle tree) -- the FP64 pipe is what bounds this kernel on
//     GB300.
//   * x is gathered through the read-only path; for FEM orderings the 27
//     neighbours of consecutive rows share cache lines.
//   * Persistent grid (a multiple of the SM count); each block walks tiles
//     blockIdx.x, blockIdx.x + gridDim.x, ...  The epilogue object keeps the
//     block's partial dot products in registers across all its tiles.
//   * A tile with more than CAP entries (very long rows) is multiplied
//     directly from global memory instead; rows of any length are correct.
//   * Bulk copies need 16-byte aligned, 16-byte multiple ranges: each range
//     is widened to the enclosing 16-byte groups, except past the last whole
//     group of the array, where the few trailing entries are read directly.
#pragma once

#include "common.cuh"

namespace helm {

template <class V>
struct CsrDev {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const V* vals;
};

__device__ __forceinline__ double2 mac(double2 a, double2 x, double2 acc) { return cfma(a, x, acc); }
__device__ __forceinline__ float2 mac(float2 a, float2 x, float2 acc) { return cfma32(a, x, acc); }
template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }

// Shared-memory footprint of the staged engine for CAP entries per tile.
template <class V, int CAP>
struct SpmvStage {
  static_assert(CAP % 4 == 0, "CAP must be a multiple of 4");
  static constexpr int kVG = 16 / sizeof(V);  // values per 16-byte group
  static constexpr size_t kValsBytes = sizeof(V) * (CAP + 2 * kVG);
  static constexpr size_t kColsBytes = sizeof(int32_t) * (CAP + 8);
  static constexpr size_t kBytes = 2 * (kValsBytes + kColsBytes) + 2 * sizeof(uint64_t);
  static_assert(kValsBytes % 16 == 0 && kColsBytes % 16 == 0, "16-byte aligned buffers");
};

// Walk this block's tiles; call epi.row(r, acc) for each row r with
// acc = sum_k vals[k] * x[colind[k]].  Returns false if a bulk copy never
// completed (error flag set).  Must be called by all threads of the block.
template <class V, int R, int CAP, class Epi>
__device__ __forceinline__ bool spmv_tiles(const CsrDev<V>& A, const V* __restrict__ x, Epi& epi,
                                           unsigned char* smem, unsigned int* dev_err) {
  using S = SpmvStage<V, CAP>;
  constexpr int VG = S::kVG;
  // buffer b: values at smem + b * kValsBytes, columns after both value buffers
  auto sv = [&](int b) { return reinterpret_cast<V*>(smem + b * S::kValsBytes); };
  auto sc = [&](int b) { return reinterpret_cast<int32_t*>(smem + 2 * S::kValsBytes + b * S::kColsBytes); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * (S::kValsBytes + S::kColsBytes));

  const int32_t n = A.n;
  const int32_t ntiles = (n + R - 1) / R;
  const int64_t cend = A.nnz & ~int64_t(3);        // last whole 16-byte group of colind
  const int64_t vend = A.nnz & ~int64_t(VG - 1);   // same for vals

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
    g.staged = (g.e - g.s) <= CAP;
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
      if (g.va1 > g.va0) vbytes = static_cast<uint32_t>((g.va1 - g.va0) * sizeof(V));
      if (g.ca1 > g.ca0) cbytes = static_cast<uint32_t>((g.ca1 - g.ca0) * sizeof(int32_t));
    }
    mbar_expect_tx(&bar[b], vbytes + cbytes);
    if (vbytes) bulk_g2s(sv(b), A.vals + g.va0, vbytes, &bar[b]);
    if (cbytes) bulk_g2s(sc(b), A.colind + g.ca0, cbytes, &bar[b]);
  };

  bool ok = true;
  int fail_it = 0;
  bool fail_next = false;
  int32_t tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    const int32_t next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) {
      fence_proxy_async();  // buffer b^1 was last read through the generic proxy
      issue(next, b ^ 1);
    }
    const Range g = range_of(tile);
    // Every thread observes the phase (visibility of the async-proxy
    // writes); the give-up decision is made block-uniform by the vote.
    const bool got = mbar_wait_bounded(&bar[b], (it >> 1) & 1, 2000000000ull);
    if (!__syncthreads_and(got)) {
      if (threadIdx.x == 0) atomicOr(dev_err, DEVERR_MBAR_TIMEOUT);
      ok = false;
      fail_it = it;
      fail_next = next < ntiles;
      break;
    }
    const int32_t r = tile * R + threadIdx.x;
    if (r < min(tile * R + R, n)) {
      const int64_t k0 = A.rowptr[r], k1 = A.rowptr[r + 1];
      V acc = vzero<V>();
      if (g.staged) {
        const V* v = sv(b) - g.va0;
        const int32_t* c = sc(b) - g.ca0;
        if (g.e <= g.va1 && g.e <= g.ca1) {
#pragma unroll 4
          for (int64_t k = k0; k < k1; ++k) acc = mac(v[k], ld_gather(x + c[k]), acc);
        } else {  // entries past the last whole 16-byte group: plain loads
#pragma unroll 2
          for (int64_t k = k0; k < k1; ++k) {
            const V a = (k < g.va1) ? v[k] : ld_stream(A.vals + k);
            const int32_t col = (k < g.ca1) ? c[k] : ld_stream(A.colind + k);
            acc = mac(a, ld_gather(x + col), acc);
          }
        }
      } else {
#pragma unroll 4
        for (int64_t k = k0; k < k1; ++k)
          acc = mac(ld_stream(A.vals + k), ld_gather(x + ld_stream(A.colind + k)), acc);
      }
      epi.row(r, acc);
    }
    __syncthreads();  // buffer b fully consumed before it is refilled
  }
  if (!ok) {
    // Let the copies still in flight land (bounded) before the block's
    // shared memory is released.
    (void)mbar_wait_bounded(&bar[fail_it & 1], (fail_it >> 1) & 1, 100000000ull);
    if (fail_next)
      (void)mbar_wait_bounded(&bar[(fail_it + 1) & 1], ((fail_it + 1) >> 1) & 1, 100000000ull);
  }
  return ok;
}

}  // namespace helm
