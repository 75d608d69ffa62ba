// CSR SpMV engine (Section 3, Table 8 of the paper: CSR SpMV, 8 flops per
// stored entry in complex arithmetic), for complex128 and complex64.
//
// The handle keeps the caller's CSR arrays and derives from them, once, a
// sliced-ELLPACK copy (SELL-32, Kreutzer et al. 2014, without row sorting):
//   * a slice is 32 consecutive rows; its width w is the longest row in it;
//     entry k of the slice's row l sits at soff[s] + 32 k + l, so when the 32
//     lanes of a warp each take one row, every load of a value or column
//     index is one contiguous, fully coalesced 256-byte (values) or 128-byte
//     (columns) access, and the gathered x[col] of neighbouring rows share
//     cache lines;
//   * the real parts of the values are stored there (8 bytes per entry for
//     complex128, 4 for complex64) and multiplied with the real x complex
//     product (2 FMA per entry instead of 4);
//   * the entries with a nonzero imaginary part are kept again, as a second
//     SELL of imaginary parts (for Helmholtz FEM, A = K - k^2 M + i k B, only
//     the rows of the impedance face: 65,341 of 9.7 M entries on the
//     120x60x50 cavity), each adding i Im(a) x with 2 more FMA.
//   Padding entries (rows shorter than the slice width) are never read: each
//   lane stops at its own row length.
// Row sums run in CSR order over the real parts, then over the imaginary
// parts: for a row whose entries are all real the result is the CSR-order
// FP64 sum bit for bit.
//
// Schedule (SliceRows): rounds of consecutive slices, each round split into
// equal contiguous sub-ranges, one per block (one block per SM), one slice
// per warp: the whole GPU works on one front of consecutive slices
// (sequential HBM streams; x gathers that hit in L2 and, within a block, in
// L1) and every SM has the same work.  The
// loads of the next U entries are issued before the FMAs of the current U
// (software pipeline), so each warp keeps 2U matrix loads and U gathers in
// flight.  Measured on GB300 (120x60x50 cavity, nnz 9.7 M): 43.1 us, against
// 47.6 us for 32-row CSR tiles staged into shared memory by TMA bulk copies
// (the previous engine); per-warp contiguous slice ranges were 1.3-8x slower.
// On GB300 the FP64 pipe (about two FMA lanes per clock per SM), not HBM,
// bounds this kernel: 2 FMA per stored entry.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.hpp"

// Entries per pipeline stage of a row (matrix loads in flight: 2U per lane).
#ifndef HELM_SPMV_UNROLL
#define HELM_SPMV_UNROLL 4
#endif

namespace helm {

constexpr int kSpmvUnroll = HELM_SPMV_UNROLL;

// Real type of a complex type.
template <class V> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

// Device view of a matrix: the CSR arrays and the SELL-32 copy.
template <class V>
struct CsrDev {
  using R = typename RealOf<V>::T;
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr;  // CSR row pointers (row lengths are read from here)
  const int32_t* colind;  // CSR column indices (not read by the SpMV)
  const V* vals;          // CSR values (not read by the SpMV)
  int32_t nsl;            // slices: ceil(n / 32)
  const int32_t* soff;    // [nsl + 1] first entry of each slice (multiples of 32)
  const int32_t* scol;    // [soff[nsl]] columns, slice-major
  const R* sval;          // [soff[nsl]] real parts, slice-major
  const int32_t* isoff;   // [nsl + 1] the same for the imaginary entries
  const int32_t* icol;
  const R* ival;
  const int32_t* ilen;    // [n] imaginary entries per row (read only in slices that have some)
  int32_t ndia;           // complex64 with a diagonal copy: the real parts on ndia diagonals, else 0
  const int32_t* doff;    // [ndia] ascending offsets col - row
  const R* dval;          // [ndia][n] real part of entry (r, r + doff[d]), 0 where none
};

template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <class V> __device__ __forceinline__ V vadd(V a, V b) { return cadd(a, b); }

// acc + a x for real a
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
// acc + a x, complex a
__device__ __forceinline__ double2 mac(double2 a, double2 x, double2 acc) { return cfma(a, x, acc); }
__device__ __forceinline__ float2 mac(float2 a, float2 x, float2 acc) { return cfma32(a, x, acc); }
// acc + i b x for real b
__device__ __forceinline__ double2 mac_imag(double b, double2 x, double2 acc) {
  acc.x = fma(-b, x.y, acc.x);
  acc.y = fma(b, x.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 mac_imag(float b, float2 x, float2 acc) {
  acc.x = fmaf(-b, x.y, acc.x);
  acc.y = fmaf(b, x.x, acc.y);
  return acc;
}

// How the gathered vector is loaded.  Kernels that only read x take the
// read-only path; a kernel that writes the vector it later gathers (the
// persistent solver, across its grid barriers) must use coherent loads.
struct GatherReadOnly {
  template <class V> __device__ __forceinline__ static V ld(const V* p) { return __ldg(p); }
};
struct GatherCoherent {
  // ld.global.cg: served by L2, the point of coherence of the GPU (an SM's
  // L1 may still hold a line another SM has since rewritten)
  template <class V> __device__ __forceinline__ static V ld(const V* p) { return __ldcg(p); }
};

// Sum of row r = 32 s + lane (len entries) of slice s: real parts in CSR
// order (U-entry pipeline), then the row's imaginary entries.
template <class V, class G = GatherReadOnly, int U = kSpmvUnroll>
__device__ __forceinline__ V sell_row(const CsrDev<V>& A, int32_t s, int lane, int32_t r, int32_t len,
                                      const V* x) {
  using R = typename RealOf<V>::T;
  const int32_t base = A.soff[s];
  const int32_t w = (A.soff[s + 1] - base) >> 5;
  const R* v = A.sval + base + lane;
  const int32_t* c = A.scol + base + lane;
  V acc = vzero<V>();
  R a[U];
  int32_t cc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    a[u] = R(0);
    cc[u] = 0;
    if (u < len) {
      a[u] = __ldcs(v + u * 32);
      cc[u] = __ldcs(c + u * 32);
    }
  }
  for (int32_t k = 0; k < w; k += U) {
    V xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k + u < len) xv[u] = G::ld(x + cc[u]);
    R an[U];
    int32_t cn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      an[u] = R(0);
      cn[u] = 0;
      if (k + U + u < len) {
        an[u] = __ldcs(v + (k + U + u) * 32);
        cn[u] = __ldcs(c + (k + U + u) * 32);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k + u < len) acc = mac_real(a[u], xv[u], acc);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = an[u];
      cc[u] = cn[u];
    }
  }
  const int32_t ib = A.isoff[s];
  const int32_t iw = (A.isoff[s + 1] - ib) >> 5;
  if (iw > 0) {
    const int32_t il = r < A.n ? A.ilen[r] : 0;
    for (int32_t q = 0; q < iw; ++q) {
      if (q < il) {
        const R b = A.ival[ib + q * 32 + lane];
        acc = mac_imag(b, G::ld(x + A.icol[ib + q * 32 + lane]), acc);
      }
    }
  }
  return acc;
}

// Rows of this thread.  The slices are taken in rounds of W = G WB
// consecutive slices (G blocks of WB warps); in round k, whose R slices
// start at k W, block b takes the contiguous sub-range
// [k W + floor(b R / G), k W + floor((b + 1) R / G)), one slice per warp in
// warp order.  So at any moment the grid works on one front of consecutive
// slices (sequential HBM streams, x gathers that hit in L2), the warps of a
// block work on neighbouring slices (their x gathers share L1 lines), every
// block gets the same number of slices to one, also when the last round is
// partial, and the thread that owns a row depends only on the grid's shape:
// every kernel of a solver that launches on the same grid gives a row to
// the same thread, so element-wise phases find their operands where the
// SpMV phase left them, and each thread's partial sums do not depend on the
// schedule.
struct SliceRows {
  int32_t s, lane, nsl, k;
  __device__ __forceinline__ explicit SliceRows(int32_t n)
      : s(0), lane(static_cast<int32_t>(threadIdx.x & 31)), nsl((n + 31) >> 5), k(-1) {
    advance();
  }
  // Move to this warp's slice of the next round that gives it one; s = nsl
  // when there is none.
  __device__ __forceinline__ bool advance() {
    const int64_t G = gridDim.x, WB = blockDim.x >> 5, W = G * WB;
    const int64_t b = blockIdx.x, w = threadIdx.x >> 5;
    for (++k; static_cast<int64_t>(k) * W < nsl; ++k) {
      const int64_t base = static_cast<int64_t>(k) * W;
      const int64_t R = nsl - base < W ? nsl - base : W;
      const int64_t lo = base + (b * R) / G, hi = base + ((b + 1) * R) / G;
      if (lo + w < hi) {
        s = static_cast<int32_t>(lo + w);
        return true;
      }
    }
    s = nsl;
    return false;
  }
  __device__ __forceinline__ bool active() const { return s < nsl; }
  __device__ __forceinline__ int32_t row() const { return s * 32 + lane; }
};

// Row r of a complex64 matrix with a diagonal copy: the real parts from the
// diagonals, in ascending column order (the CSR order of a sorted row), then
// the row's imaginary entries as in sell_row.  Every diagonal's value and
// gather are loaded independently of one another (no load waits on another
// one); a diagonal without an entry in this row (value 0) leaves the sum
// untouched, so the result is that of sell_row for finite x.  The complex64
// product is bound by HBM on this GPU (its arithmetic is FP32): the diagonal
// copy reads 4 bytes per stored real part and no column index, against 8
// for the sliced copy.
template <class G = GatherReadOnly>
__device__ __forceinline__ float2 dia_row(const CsrDev<float2>& A, int32_t s, int lane, int32_t r, const float2* x) {
  float2 acc = make_float2(0.f, 0.f);
  if (r < A.n) {
    const float* dv = A.dval + r;
#pragma unroll 9
    for (int32_t d = 0; d < A.ndia; ++d) {
      const int32_t j = r + __ldg(A.doff + d);
      const float a = __ldcs(dv + static_cast<size_t>(d) * A.n);
      float2 xv = make_float2(0.f, 0.f);
      if (static_cast<uint32_t>(j) < static_cast<uint32_t>(A.n)) xv = G::ld(x + j);
      const float sx = fmaf(a, xv.x, acc.x), sy = fmaf(a, xv.y, acc.y);
      const bool nz = a != 0.f;
      acc.x = nz ? sx : acc.x;
      acc.y = nz ? sy : acc.y;
    }
  }
  const int32_t ib = A.isoff[s];
  const int32_t iw = (A.isoff[s + 1] - ib) >> 5;
  if (iw > 0) {
    const int32_t il = r < A.n ? A.ilen[r] : 0;
    for (int32_t q = 0; q < iw; ++q) {
      if (q < il) {
        const float b = A.ival[ib + q * 32 + lane];
        acc = mac_imag(b, G::ld(x + A.icol[ib + q * 32 + lane]), acc);
      }
    }
  }
  return acc;
}

struct NoGate {
  __device__ __forceinline__ bool operator()() const { return true; }
};

// Walk this thread's rows; for each row r < n call epi.prefetch(r) (before
// the row's sum, so the epilogue's own loads are in flight with it) and then
// epi.row(r, sum_k a_rk x_k).  gate() is called first by every thread; it
// must return the same value in the whole block, and on false the engine
// returns without reading x.  Returns true.  Called by all threads of the
// block (blockDim a multiple of 32).  `smem` and `dev_err` are unused: the
// engine needs no shared memory and no wait.
template <class V, class Epi, class Gate = NoGate, class G = GatherReadOnly, int U = kSpmvUnroll>
__device__ __forceinline__ bool spmv_run(const CsrDev<V>& A, const V* __restrict__ x, Epi& epi,
                                         unsigned char* /*smem*/, unsigned int* /*dev_err*/, Gate gate = Gate()) {
  if (!gate()) return true;
  for (SliceRows q(A.n); q.active(); q.advance()) {
    const int32_t r = q.row();
    int32_t len = 0;
    if (r < A.n) {
      len = A.rowptr[r + 1] - A.rowptr[r];
      epi.prefetch(r);
    }
    V acc;
    if constexpr (std::is_same<V, float2>::value) {
      if (A.ndia > 0) acc = dia_row<G>(A, q.s, q.lane, r, x);
      else acc = sell_row<V, G, U>(A, q.s, q.lane, r, len, x);
    } else {
      acc = sell_row<V, G, U>(A, q.s, q.lane, r, len, x);
    }
    if (r < A.n) epi.row(r, acc);
  }
  return true;
}

// Launch shape of every SpMV-shaped kernel: 1024 threads (32 warps), one
// block per SM (64 registers per thread at most), and a small dynamic
// shared-memory block that kernels use for their block sums.  Measured on
// GB300 (120x60x50 cavity): with 256-thread blocks, four per SM, the warps'
// slice counts differed by one round and SMs idled 19 % of the SpMV.
template <class V> struct Engine {
  static constexpr int R = 32;  // rows per slice
  static constexpr int kThreads = 1024;
  static constexpr int kMinBlocks = 1;
  static constexpr size_t kSmem = 32 * 8 * sizeof(double);
};

// Device view of one value array of a handle (the caller's values, the
// complex64 copy or A D^-1) with the handle's SELL pattern.
template <class V>
inline CsrDev<V> csr_dev(const helm_csr_s* A, const V* vals, const SellVals& sv) {
  using R = typename RealOf<V>::T;
  const bool dia = sv.dval != nullptr && A->ndia > 0;
  return CsrDev<V>{A->n,        A->nnz,   A->rowptr,
                   A->colind,   vals,     A->nsl,
                   A->sell_off, A->sell_col, static_cast<const R*>(sv.sval),
                   sv.isoff,    sv.icol,  static_cast<const R*>(sv.ival),
                   sv.ilen,     dia ? A->ndia : 0, dia ? A->dia_off : nullptr,
                   dia ? static_cast<const R*>(sv.dval) : nullptr};
}

}  // namespace helm
