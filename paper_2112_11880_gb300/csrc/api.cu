// libhelm C ABI: CSR handle, SpMV, dot product, norm, axpby.
//
// Section 3 of the paper (Tables 2-8) defines the vector kernels and the CSR
// SpMV these calls provide; Section 2 fixes CSR as the storage.  Argument
// checks happen on the host before anything is enqueued; no call aborts.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <climits>
#include <cstdint>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.hpp"
#include "krylov.cuh"
#include "spmv.cuh"

namespace helm {

// ---------------------------------------------------------------- kernels

template <class V>
struct AxpbyEpi {
  V* y;
  V alpha, beta;
  int mode;  // 0: y = acc, 1: y = alpha acc, 2: y = alpha acc + beta y
  V y_old;
  __device__ __forceinline__ void prefetch(int32_t r) {
    if (mode == 2) y_old = y[r];
  }
  __device__ __forceinline__ void row(int32_t r, V acc) {
    if (mode == 0) {
      y[r] = acc;
    } else if (mode == 1) {
      y[r] = cmul(alpha, acc);
    } else {
      y[r] = cadd(cmul(alpha, acc), cmul(beta, y_old));
    }
  }
};

// Stand-alone SpMV: y = alpha A x (+ beta y).  U = entries per pipeline
// stage of the SELL engine; the variant (U and blocks per SM) is chosen per
// matrix at handle creation (autotune_spmv).
template <class V, int U>
__global__ void __launch_bounds__(Engine<V>::kThreads, Engine<V>::kMinBlocks) k_spmv(CsrDev<V> A, const V* __restrict__ x, V* y, V alpha,
                                                              V beta, int mode) {
  AxpbyEpi<V> epi{y, alpha, beta, mode, vzero<V>()};
  (void)spmv_run<V, AxpbyEpi<V>, NoGate, GatherReadOnly, U>(A, x, epi, nullptr, nullptr);
}

// ---------------------------------------------------------------- SELL-32 layout

// Slice widths: w[s] = longest row of rows [32 s, 32 s + 32).
__global__ void k_sell_widths(int32_t n, int32_t nsl, const int32_t* __restrict__ rowptr, int32_t* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nsl; s += (gridDim.x * blockDim.x) >> 5) {
    const int32_t r = s * 32 + lane;
    const int32_t len = r < n ? rowptr[r + 1] - rowptr[r] : 0;
    const int32_t m = __reduce_max_sync(0xffffffffu, len);
    if (lane == 0) w[s] = m;
  }
}

// Imaginary entries per row (ilen) and per-slice maxima (iw).
template <class V>
__global__ void k_sell_imag_counts(int32_t n, int32_t nsl, const int32_t* __restrict__ rowptr,
                                   const V* __restrict__ vals, int32_t* __restrict__ ilen, int32_t* __restrict__ iw) {
  const int lane = threadIdx.x & 31;
  for (int32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nsl; s += (gridDim.x * blockDim.x) >> 5) {
    const int32_t r = s * 32 + lane;
    int32_t c = 0;
    if (r < n) {
      for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) c += vals[k].y != 0 ? 1 : 0;
      ilen[r] = c;
    }
    const int32_t m = __reduce_max_sync(0xffffffffu, c);
    if (lane == 0) iw[s] = m;
  }
}

// Columns in SELL order; padding entries take column 0 (never read).
__global__ void k_sell_fill_cols(int32_t n, int32_t nsl, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind, const int32_t* __restrict__ soff,
                                 int32_t* __restrict__ scol) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < static_cast<int64_t>(nsl) * 32;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t s = static_cast<int32_t>(r >> 5), lane = static_cast<int32_t>(r & 31);
    const int32_t w = (soff[s + 1] - soff[s]) >> 5;
    const int32_t k0 = r < n ? rowptr[r] : 0;
    const int32_t len = r < n ? rowptr[r + 1] - k0 : 0;
    int32_t* out = scol + soff[s] + lane;
    for (int32_t k = 0; k < w; ++k) out[k * 32] = k < len ? colind[k0 + k] : 0;
  }
}

// Real parts in SELL order and the imaginary entries in their own SELL.
template <class V, class R>
__global__ void k_sell_fill_vals(int32_t n, int32_t nsl, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind, const V* __restrict__ vals,
                                 const int32_t* __restrict__ soff, const int32_t* __restrict__ isoff,
                                 R* __restrict__ sval, int32_t* __restrict__ icol, R* __restrict__ ival) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < static_cast<int64_t>(nsl) * 32;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t s = static_cast<int32_t>(r >> 5), lane = static_cast<int32_t>(r & 31);
    const int32_t w = (soff[s + 1] - soff[s]) >> 5;
    const int32_t iw = (isoff[s + 1] - isoff[s]) >> 5;
    const int32_t k0 = r < n ? rowptr[r] : 0;
    const int32_t len = r < n ? rowptr[r + 1] - k0 : 0;
    R* out = sval + soff[s] + lane;
    R* iout = ival + isoff[s] + lane;
    int32_t* ic = icol + isoff[s] + lane;
    int32_t q = 0;
    for (int32_t k = 0; k < w; ++k) {
      R re = R(0);
      if (k < len) {
        const V a = vals[k0 + k];
        re = a.x;
        if (a.y != 0) {
          iout[q * 32] = a.y;
          ic[q * 32] = colind[k0 + k];
          ++q;
        }
      }
      out[k * 32] = re;
    }
    for (; q < iw; ++q) {
      iout[q * 32] = R(0);
      ic[q * 32] = 0;
    }
  }
}

// Right Jacobi: d_i = a_ii (1 when row i stores no nonzero diagonal),
// dinv_i = 1 / d_i.
__global__ void k_jac_diag(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const double2* __restrict__ vals, double2* __restrict__ d, double2* __restrict__ dinv) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 di = make_double2(1.0, 0.0);
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (colind[k] == i) {
        if (!czero(vals[k]) && cfinite(vals[k])) di = vals[k];
        break;
      }
    }
    d[i] = di;
    dinv[i] = cdiv(make_double2(1.0, 0.0), di);
  }
}
// A D^-1: entry k of row i is a_ik dinv_colind[k]
__global__ void k_jac_scale(int64_t nnz, const int32_t* __restrict__ colind, const double2* __restrict__ vals,
                            const double2* __restrict__ dinv, double2* __restrict__ out) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[k] = cmul(vals[k], dinv[colind[k]]);
}
// x_i <- s_i x_i
__global__ void k_jac_apply(int32_t n, const double2* __restrict__ sc, double2* __restrict__ x) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = cmul(sc[i], x[i]);
}

// Per-row statistics and (optionally) validation of the CSR pattern.
__global__ void k_csr_check(int32_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colind, int validate, int* out /* [0]=max row, [1]=bad */) {
  int local_max = 0, bad = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    if (b < a || a < 0 || b > nnz) {
      bad = 1;
      continue;
    }
    const int64_t len = b - a;
    local_max = max(local_max, static_cast<int>(len < 0x7fffffff ? len : 0x7fffffff));
    if (validate) {
      int32_t prev = -1;
      for (int64_t k = a; k < b; ++k) {
        const int32_t c = colind[k];
        if (c < 0 || c >= n || c <= prev) bad = 1;
        prev = c;
      }
    }
  }
  if (local_max) atomicMax(&out[0], local_max);
  if (bad) atomicOr(&out[1], 1);
}

// The BLAS-1 kernels below walk the vectors with a grid-stride loop and take
// four strides per trip: all loads of the trip are issued before the first
// product, so every thread keeps four (axpby: eight) 16-byte loads in flight
// instead of one or two.  A thread still adds its elements i, i+T, i+2T, ...
// (T threads in the grid) in that order, so the sums are the same bits as a
// one-stride loop over the same grid.
constexpr int kVecIlp = 4;

// One block-sized partial of (x, y) per block; complex64 inputs accumulate
// products in FP32 per thread (few terms each) and everything above in FP64.
template <class V, bool CONJ>
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const V* __restrict__ x,
                                                     const V* __restrict__ y, double* partials) {
  __shared__ double red[32 * 2];
  V acc = vzero<V>();
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecIlp - 1) * T < n; i += kVecIlp * T) {
    V a[kVecIlp], b[kVecIlp];
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) a[k] = ld_stream(x + i + k * T);
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) b[k] = ld_stream(y + i + k * T);
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) {
      if (CONJ) a[k].y = -a[k].y;
      acc = mac(a[k], b[k], acc);
    }
  }
  for (; i < n; i += T) {
    V a = ld_stream(x + i);
    if (CONJ) a.y = -a.y;
    acc = mac(a, ld_stream(y + i), acc);
  }
  double v[2] = {static_cast<double>(acc.x), static_cast<double>(acc.y)};
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v[0];
    partials[2 * blockIdx.x + 1] = v[1];
  }
}

template <class V>
__global__ void __launch_bounds__(256) k_nrm2_partial(int64_t n, const V* __restrict__ x, double* partials) {
  __shared__ double red[32];
  using S = decltype(V().x);  // FP64 sums for complex128, FP32 per thread for complex64
  S acc = S(0);
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecIlp - 1) * T < n; i += kVecIlp * T) {
    V a[kVecIlp];
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) a[k] = ld_stream(x + i + k * T);
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) {
      acc = fma(a[k].x, a[k].x, acc);
      acc = fma(a[k].y, a[k].y, acc);
    }
  }
  for (; i < n; i += T) {
    const V a = ld_stream(x + i);
    acc = fma(a.x, a.x, acc);
    acc = fma(a.y, a.y, acc);
  }
  double v[1] = {static_cast<double>(acc)};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// Adds the block partials in block order (one block).
template <int K>
__global__ void __launch_bounds__(256) k_sum_partials(int nparts, const double* __restrict__ partials,
                                                      double* out, int sqrt_result) {
  __shared__ double red[32 * K];
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += partials[(size_t)b * K + k];
  }
  block_sum<K>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = sqrt_result ? sqrt(acc[k]) : acc[k];
  }
}

// y = alpha x + beta y with the kinds of the two scalars fixed at compile
// time (0: zero, 1: one, 2: real, 3: complex), so that a kernel does only the
// products its scalars need: assignment (alpha = 1, beta = 0) is a copy, a real
// scalar costs 2 real products an element, a complex one 4.  On this GPU a
// complex128 axpy with complex alpha is as much FP64-pipe work as memory
// traffic, so the products skipped here are time saved.  The values are those
// of the full complex formula (a zero imaginary part adds exact zeros).
template <class V, int XA, int YB>
__device__ __forceinline__ V axpby_elem(V alpha, V xi, V beta, V yi) {
  V r = vzero<V>();
  if (YB == 1) r = yi;
  if (YB == 2) r = V{beta.x * yi.x, beta.x * yi.y};
  if (YB == 3) r = cmul(beta, yi);
  if (XA == 1) r = YB == 0 ? xi : V{r.x + xi.x, r.y + xi.y};
  if (XA == 2) r = V{fma(alpha.x, xi.x, r.x), fma(alpha.x, xi.y, r.y)};
  if (XA == 3) r = mac(alpha, xi, r);
  return r;
}

template <class V, int XA, int YB>
__global__ void __launch_bounds__(256) k_axpby(int64_t n, V alpha, const V* x, V beta, V* y) {
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i + (kVecIlp - 1) * T < n; i += kVecIlp * T) {
    V xs[kVecIlp], ys[kVecIlp];
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) {
      xs[k] = XA ? ld_stream(x + i + k * T) : vzero<V>();
      ys[k] = YB ? ld_stream(y + i + k * T) : vzero<V>();
    }
#pragma unroll
    for (int k = 0; k < kVecIlp; ++k) __stcs(y + i + k * T, axpby_elem<V, XA, YB>(alpha, xs[k], beta, ys[k]));
  }
  for (; i < n; i += T) {
    const V xi = XA ? ld_stream(x + i) : vzero<V>();
    const V yi = YB ? ld_stream(y + i) : vzero<V>();
    __stcs(y + i, axpby_elem<V, XA, YB>(alpha, xi, beta, yi));
  }
}

template <class V, int XA>
void launch_axpby_yb(int yb, int grid, cudaStream_t s, int64_t n, V alpha, const V* x, V beta, V* y) {
  switch (yb) {
    case 0: k_axpby<V, XA, 0><<<grid, 256, 0, s>>>(n, alpha, x, beta, y); break;
    case 1: k_axpby<V, XA, 1><<<grid, 256, 0, s>>>(n, alpha, x, beta, y); break;
    case 2: k_axpby<V, XA, 2><<<grid, 256, 0, s>>>(n, alpha, x, beta, y); break;
    default: k_axpby<V, XA, 3><<<grid, 256, 0, s>>>(n, alpha, x, beta, y); break;
  }
}

template <class V>
void launch_axpby(int xa, int yb, int grid, cudaStream_t s, int64_t n, V alpha, const V* x, V beta, V* y) {
  switch (xa) {
    case 0: launch_axpby_yb<V, 0>(yb, grid, s, n, alpha, x, beta, y); break;
    case 1: launch_axpby_yb<V, 1>(yb, grid, s, n, alpha, x, beta, y); break;
    case 2: launch_axpby_yb<V, 2>(yb, grid, s, n, alpha, x, beta, y); break;
    default: launch_axpby_yb<V, 3>(yb, grid, s, n, alpha, x, beta, y); break;
  }
}

__global__ void k_c128_to_c64(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = ld_stream(a + i);
    b[i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
}

// ---------------------------------------------------------------- diagonal copy (complex64 products)

// The longest row: key = (length << 32) | row, the largest key wins.
__global__ void k_dia_probe(int32_t n, const int32_t* __restrict__ rowptr, unsigned long long* key) {
  unsigned long long best = 0ull;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long len = static_cast<unsigned long long>(rowptr[i + 1] - rowptr[i]);
    const unsigned long long k = (len << 32) | static_cast<unsigned long long>(static_cast<uint32_t>(i));
    best = k > best ? k : best;
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

struct DiaOffsets {
  int32_t nd;
  int32_t off[32];
};

// Flags an entry whose diagonal col - row is not among D's, and a row whose
// columns are not strictly ascending.
__global__ void k_dia_check(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            DiaOffsets D, int* bad) {
  int local = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int64_t prev = INT64_MIN;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t c = colind[k];
      if (c <= prev) local = 1;
      prev = c;
      const int32_t d = c - i;
      bool found = false;
      for (int q = 0; q < D.nd; ++q) found |= D.off[q] == d;
      if (!found) local = 1;
    }
  }
  if (local) atomicOr(bad, 1);
}

// dval[d][i] = Re a(i, i + off[d]) as float (the array starts zeroed)
template <class V>
__global__ void k_dia_fill(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const V* __restrict__ vals, DiaOffsets D, float* __restrict__ dval) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t d = colind[k] - i;
      int q = 0;
      while (q < D.nd - 1 && D.off[q] != d) ++q;
      dval[static_cast<size_t>(q) * n + i] = static_cast<float>(vals[k].x);
    }
  }
}

// ---------------------------------------------------------------- host helpers

void debug_cuda_error(cudaError_t e, const char* file, int line) {
  static const bool on = std::getenv("HELM_DEBUG") != nullptr;
  if (on) std::fprintf(stderr, "libhelm: %s:%d: %s\n", file, line, cudaGetErrorString(e));
}

std::mutex g_attr_mu;
std::vector<std::pair<const void*, int>> g_attr_done;

// Opt a kernel into more than 48 KB of dynamic shared memory (once per
// kernel and device).
cudaError_t set_smem_attr(const void* fn, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (auto& p : g_attr_done)
    if (p.first == fn && p.second == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) g_attr_done.emplace_back(fn, dev);
  return e;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return std::max(sms, 1);
}

int vec_grid_for(int64_t n) {
  const int64_t want = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
  return static_cast<int>(std::max<int64_t>(1, std::min(want, cap)));
}

namespace {
bool is_zero(const double* z) { return z[0] == 0.0 && z[1] == 0.0; }
bool is_one(const double* z) { return z[0] == 1.0 && z[1] == 0.0; }
}  // namespace

// ---------------------------------------------------------------- stand-alone SpMV

// Variants of the stand-alone SpMV: U (entries per pipeline stage) x block
// size (1024 threads, one block per SM, or 512 threads, two per SM).  Every
// variant computes each row with the same operations in the same order, so
// the choice changes the speed only, never a bit of y.
template <class V>
static void spmv_enqueue(int U, int grid, int threads, const CsrDev<V>& d, const V* x, V* y, V alpha, V beta,
                         int mode, cudaStream_t s) {
  if (U == 2)
    k_spmv<V, 2><<<grid, threads, 0, s>>>(d, x, y, alpha, beta, mode);
  else
    k_spmv<V, 4><<<grid, threads, 0, s>>>(d, x, y, alpha, beta, mode);
}

// Blocks of `threads` that fit on one SM for variant U.
template <class V>
static helm_status spmv_occupancy(int U, int threads, int* per_sm) {
  const void* fn = U == 2 ? reinterpret_cast<const void*>(&k_spmv<V, 2>) : reinterpret_cast<const void*>(&k_spmv<V, 4>);
  HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, 0));
  return HELM_OK;
}

// Autotuning (Section 3: the paper's SpMV is auto-tuned): time the variants
// on the handle's own matrix (3 launches each after one warm-up, CUDA events
// on `s`) and keep the fastest.  Matrices under 2^18 stored entries keep the
// default (U = 4, 1024-thread blocks): their SpMV is launch-bound.
template <class V>
static helm_status autotune_spmv(helm_csr A, const CsrDev<V>& d, cudaStream_t s) {
  struct Cand {
    int U, threads, bps;
    bool full;
  };
  const Cand cand[5] = {{4, 1024, 1, false}, {4, 1024, 1, true}, {2, 1024, 1, false}, {4, 512, 2, false},
                        {2, 512, 2, false}};
  const SliceShape s0 = slice_shape(A->n, A->num_sms, 1024, 1);
  A->spmv_variant = 4;
  A->spmv_grid = s0.grid;
  A->spmv_threads = s0.threads;
  if (A->nnz < (int64_t(1) << 18) || A->n == 0) return HELM_OK;
  V *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  helm_status st = HELM_OK;
  float best = 0.f;
  do {
    if (cudaMalloc(&x, sizeof(V) * static_cast<size_t>(A->n)) != cudaSuccess ||
        cudaMalloc(&y, sizeof(V) * static_cast<size_t>(A->n)) != cudaSuccess) {
      st = HELM_ERR_NOMEM;
      break;
    }
    if (cudaMemsetAsync(x, 0, sizeof(V) * static_cast<size_t>(A->n), s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = HELM_ERR_CUDA;
      break;
    }
    V one, zero;
    one.x = 1;
    one.y = 0;
    zero.x = 0;
    zero.y = 0;
    for (const Cand& c : cand) {
      int fit = 0;
      if (spmv_occupancy<V>(c.U, c.threads, &fit) != HELM_OK || fit < c.bps) continue;
      const SliceShape sh = slice_shape(A->n, A->num_sms, c.threads, c.bps, c.full);
      spmv_enqueue<V>(c.U, sh.grid, sh.threads, d, x, y, one, zero, 0, s);
      cudaEventRecord(e0, s);
      for (int k = 0; k < 3; ++k) spmv_enqueue<V>(c.U, sh.grid, sh.threads, d, x, y, one, zero, 0, s);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = HELM_ERR_CUDA;
        break;
      }
      if (std::getenv("HELM_DEBUG"))
        std::fprintf(stderr, "libhelm: spmv variant U=%d grid=%d threads=%d: %.2f us\n", c.U, sh.grid, sh.threads,
                     ms * 1e3f / 3);
      if (best == 0.f || ms < best) {
        best = ms;
        A->spmv_variant = c.U;
        A->spmv_grid = sh.grid;
        A->spmv_threads = sh.threads;
      }
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  (void)cudaGetLastError();
  return st;
}

template <class V>
static int spmv_mode(V alpha, V beta) {
  const bool a1 = alpha.x == 1 && alpha.y == 0, b0 = beta.x == 0 && beta.y == 0;
  return (a1 && b0) ? 0 : (b0 ? 1 : 2);
}

helm_status launch_spmv128(helm_csr A, const double2* x, double2* y, double2 alpha, double2 beta,
                           cudaStream_t s) {
  if (A->n == 0) return HELM_OK;
  const CsrDev<double2> d = csr_dev<double2>(A, static_cast<const double2*>(A->vals), A->sv);
  spmv_enqueue<double2>(A->spmv_variant, A->spmv_grid, A->spmv_threads, d, x, y, alpha, beta, spmv_mode(alpha, beta), s);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

helm_status launch_spmv64(helm_csr A, const float2* x, float2* y, float2 alpha, float2 beta, cudaStream_t s) {
  if (A->n == 0) return HELM_OK;
  const CsrDev<float2> d = csr_dev<float2>(A, static_cast<const float2*>(A->vals), A->sv);
  spmv_enqueue<float2>(A->spmv_variant, A->spmv_grid, A->spmv_threads, d, x, y, alpha, beta, spmv_mode(alpha, beta), s);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

// ---------------------------------------------------------------- SELL build (host)

// Exclusive prefix sum of 32 * widths into offsets (host); false when the
// total does not fit int32.
static bool widths_to_offsets(const std::vector<int32_t>& w, std::vector<int32_t>* off, int64_t* total) {
  off->assign(w.size() + 1, 0);
  int64_t acc = 0;
  for (size_t s = 0; s < w.size(); ++s) {
    (*off)[s] = static_cast<int32_t>(acc);
    acc += 32 * static_cast<int64_t>(w[s]);
    if (acc >= (int64_t(1) << 31)) return false;
  }
  (*off)[w.size()] = static_cast<int32_t>(acc);
  *total = acc;
  return true;
}

// The pattern: slice widths, offsets and columns.  Synchronises `s`.
static helm_status build_sell_pattern(helm_csr A, cudaStream_t s) {
  const int32_t n = A->n, nsl = (n + 31) / 32;
  A->nsl = nsl;
  std::vector<int32_t> w(nsl), off;
  int32_t* d_w = nullptr;
  if (nsl > 0) {
    HELM_CUDA_TRY(cudaMalloc(&d_w, sizeof(int32_t) * nsl));
    k_sell_widths<<<vec_grid_for(static_cast<int64_t>(nsl) * 32), 256, 0, s>>>(n, nsl, A->rowptr, d_w);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.data(), d_w, sizeof(int32_t) * nsl, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_w);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return HELM_ERR_CUDA;
    }
  }
  int64_t total = 0;
  if (!widths_to_offsets(w, &off, &total)) return HELM_ERR_INVALID;  // padded entries >= 2^31
  A->sell_entries = total;
  HELM_CUDA_TRY(cudaMalloc(&A->sell_off, sizeof(int32_t) * (nsl + 1)));
  HELM_CUDA_TRY(cudaMalloc(&A->sell_col, sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(total, 1))));
  HELM_CUDA_TRY(cudaMemcpyAsync(A->sell_off, off.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice, s));
  if (nsl > 0) {
    k_sell_fill_cols<<<vec_grid_for(static_cast<int64_t>(nsl) * 32), 256, 0, s>>>(n, nsl, A->rowptr, A->colind,
                                                                                   A->sell_off, A->sell_col);
    HELM_CUDA_TRY(cudaGetLastError());
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(s));  // `off` is a host buffer of this frame
  return HELM_OK;
}

// Whether the pattern lies on at most 32 diagonals with little padding: the
// longest row's diagonals are the candidates, one device pass checks every
// entry (and that rows are sorted without duplicates).  Sets A->ndia and
// A->dia_off; leaves ndia = 0 (sliced copy only) otherwise.
constexpr double kDiaMaxFill = 1.5;  // diagonal slots per stored entry at most

static helm_status analyze_diagonals(helm_csr A, cudaStream_t s) {
  A->ndia = 0;
  if (A->n == 0 || A->nnz == 0 || A->max_row > 32) return HELM_OK;
  unsigned long long* d_key = nullptr;
  int* d_bad = nullptr;
  unsigned long long key = 0;
  int bad = 0;
  DiaOffsets D;
  std::memset(&D, 0, sizeof(D));
  helm_status st = HELM_OK;
  do {
    if (cudaMalloc(&d_key, sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) {
      st = HELM_ERR_NOMEM;
      break;
    }
    cudaError_t e = cudaMemsetAsync(d_key, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      k_dia_probe<<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->rowptr, d_key);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&key, d_key, sizeof(key), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = HELM_ERR_CUDA;
      break;
    }
    const int32_t row = static_cast<int32_t>(key & 0xffffffffull), len = static_cast<int32_t>(key >> 32);
    if (len < 1 || len > 32) break;
    if (static_cast<double>(len) * A->n > kDiaMaxFill * static_cast<double>(A->nnz)) break;
    int32_t k0 = 0;
    int32_t cols[32];
    e = cudaMemcpyAsync(&k0, A->rowptr + row, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cols, A->colind + k0, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = HELM_ERR_CUDA;
      break;
    }
    D.nd = len;
    for (int q = 0; q < len; ++q) D.off[q] = cols[q] - row;
    bool ascending = true;
    for (int q = 1; q < len; ++q) ascending &= D.off[q] > D.off[q - 1];
    if (!ascending) break;
    k_dia_check<<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->rowptr, A->colind, D, d_bad);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = HELM_ERR_CUDA;
      break;
    }
    if (bad) break;
    if (cudaMalloc(&A->dia_off, sizeof(int32_t) * len) != cudaSuccess) {
      st = HELM_ERR_NOMEM;
      break;
    }
    if (cudaMemcpyAsync(A->dia_off, D.off, sizeof(int32_t) * len, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = HELM_ERR_CUDA;
      break;
    }
    A->ndia = len;
  } while (false);
  cudaFree(d_key);
  cudaFree(d_bad);
  (void)cudaGetLastError();
  return st;
}

// The diagonal copy of a complex64 value set (when the handle has one).
static helm_status build_dia_vals(helm_csr A, const float2* vals, SellVals* out, cudaStream_t s) {
  if (A->ndia == 0) return HELM_OK;
  DiaOffsets D;
  std::memset(&D, 0, sizeof(D));
  D.nd = A->ndia;
  HELM_CUDA_TRY(cudaMemcpyAsync(D.off, A->dia_off, sizeof(int32_t) * A->ndia, cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  const size_t slots = static_cast<size_t>(A->ndia) * A->n;
  HELM_CUDA_TRY(cudaMalloc(&out->dval, sizeof(float) * slots));
  HELM_CUDA_TRY(cudaMemsetAsync(out->dval, 0, sizeof(float) * slots, s));
  k_dia_fill<float2><<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->rowptr, A->colind, vals, D,
                                                         static_cast<float*>(out->dval));
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

static void free_sell_vals(SellVals* v) {
  cudaFree(v->dval);
  cudaFree(v->sval);
  cudaFree(v->isoff);
  cudaFree(v->icol);
  cudaFree(v->ival);
  cudaFree(v->ilen);
  *v = SellVals();
}

template <class V>
static helm_status build_sell_vals_t(helm_csr A, const V* vals, SellVals* out, cudaStream_t s) {
  using R = typename RealOf<V>::T;
  const int32_t n = A->n, nsl = A->nsl;
  const size_t N = static_cast<size_t>(std::max(n, 1));
  std::vector<int32_t> iw(nsl), ioff;
  HELM_CUDA_TRY(cudaMalloc(&out->ilen, sizeof(int32_t) * N));
  HELM_CUDA_TRY(cudaMalloc(&out->sval, sizeof(R) * static_cast<size_t>(std::max<int64_t>(A->sell_entries, 1))));
  HELM_CUDA_TRY(cudaMalloc(&out->isoff, sizeof(int32_t) * (nsl + 1)));
  if (nsl > 0) {
    int32_t* d_iw = nullptr;
    HELM_CUDA_TRY(cudaMalloc(&d_iw, sizeof(int32_t) * nsl));
    k_sell_imag_counts<V><<<vec_grid_for(static_cast<int64_t>(nsl) * 32), 256, 0, s>>>(n, nsl, A->rowptr, vals,
                                                                                       out->ilen, d_iw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(iw.data(), d_iw, sizeof(int32_t) * nsl, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_iw);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return HELM_ERR_CUDA;
    }
  }
  int64_t itotal = 0;
  if (!widths_to_offsets(iw, &ioff, &itotal)) return HELM_ERR_INVALID;
  HELM_CUDA_TRY(cudaMalloc(&out->icol, sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(itotal, 1))));
  HELM_CUDA_TRY(cudaMalloc(&out->ival, sizeof(R) * static_cast<size_t>(std::max<int64_t>(itotal, 1))));
  HELM_CUDA_TRY(cudaMemcpyAsync(out->isoff, ioff.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice, s));
  if (nsl > 0) {
    k_sell_fill_vals<V, R><<<vec_grid_for(static_cast<int64_t>(nsl) * 32), 256, 0, s>>>(
        n, nsl, A->rowptr, A->colind, vals, A->sell_off, out->isoff, static_cast<R*>(out->sval), out->icol,
        static_cast<R*>(out->ival));
    HELM_CUDA_TRY(cudaGetLastError());
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(s));  // `ioff` is a host buffer of this frame
  return HELM_OK;
}

helm_status build_sell_vals(helm_csr A, const void* vals, helm_dtype dt, SellVals* out, cudaStream_t s) {
  helm_status st = dt == HELM_C128 ? build_sell_vals_t<double2>(A, static_cast<const double2*>(vals), out, s)
                                   : build_sell_vals_t<float2>(A, static_cast<const float2*>(vals), out, s);
  if (st == HELM_OK && dt == HELM_C64) st = build_dia_vals(A, static_cast<const float2*>(vals), out, s);
  if (st != HELM_OK) free_sell_vals(out);
  return st;
}

// Graphs capture buffer addresses: drop them whenever a buffer is replaced.
static void drop_graphs(helm_csr A) {
  for (auto& kv : A->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  A->graphs.clear();
}

helm_status ensure_vectors(helm_csr A, int nvec) {
  if (A->nvec >= nvec) return HELM_OK;
  drop_graphs(A);
  if (A->vec) {
    cudaFree(A->vec);
    A->vec = nullptr;
    A->nvec = 0;
  }
  const size_t bytes = sizeof(double2) * static_cast<size_t>(std::max<int32_t>(A->n, 1)) * nvec;
  HELM_CUDA_TRY(cudaMalloc(&A->vec, bytes));
  A->nvec = nvec;
  return HELM_OK;
}

helm_status ensure_vectors32(helm_csr A, int nvec) {
  if (A->nvec32 >= nvec) return HELM_OK;
  drop_graphs(A);
  if (A->vec32) {
    cudaFree(A->vec32);
    A->vec32 = nullptr;
    A->nvec32 = 0;
  }
  const size_t bytes = sizeof(float2) * static_cast<size_t>(std::max<int32_t>(A->n, 1)) * nvec;
  HELM_CUDA_TRY(cudaMalloc(&A->vec32, bytes));
  A->nvec32 = nvec;
  return HELM_OK;
}

helm_status ensure_vals32(helm_csr A, cudaStream_t s) {
  if (A->vals32) return HELM_OK;
  const size_t NNZ = static_cast<size_t>(std::max<int64_t>(A->nnz, 1));
  HELM_CUDA_TRY(cudaMalloc(&A->vals32, sizeof(float2) * NNZ));
  if (A->nnz) {
    k_c128_to_c64<<<vec_grid_for(A->nnz), 256, 0, s>>>(A->nnz, static_cast<const double2*>(A->vals), A->vals32);
    HELM_CUDA_TRY(cudaGetLastError());
  }
  helm_status st = build_sell_vals(A, A->vals32, HELM_C64, &A->sv32, s);
  if (st != HELM_OK) {
    cudaFree(A->vals32);
    A->vals32 = nullptr;
  }
  return st;
}

}  // namespace helm

using namespace helm;

// ---------------------------------------------------------------- C ABI

namespace helm {
helm_status ensure_jacobi(helm_csr A, cudaStream_t s) {
  if (A->svjac.sval) return HELM_OK;
  const int32_t n = A->n;
  const size_t N = static_cast<size_t>(n > 0 ? n : 1), NNZ = static_cast<size_t>(A->nnz > 0 ? A->nnz : 1);
  if (!A->jac_d) HELM_CUDA_TRY(cudaMalloc(&A->jac_d, N * sizeof(double2)));
  if (!A->jac_dinv) HELM_CUDA_TRY(cudaMalloc(&A->jac_dinv, N * sizeof(double2)));
  if (!A->jac_vals) HELM_CUDA_TRY(cudaMalloc(&A->jac_vals, NNZ * sizeof(double2)));
  const double2* vals = static_cast<const double2*>(A->vals);
  k_jac_diag<<<vec_grid_for(n), 256, 0, s>>>(n, A->rowptr, A->colind, vals, A->jac_d, A->jac_dinv);
  k_jac_scale<<<vec_grid_for(A->nnz), 256, 0, s>>>(A->nnz, A->colind, vals, A->jac_dinv, A->jac_vals);
  HELM_CUDA_TRY(cudaGetLastError());
  return build_sell_vals(A, A->jac_vals, HELM_C128, &A->svjac, s);
}
}  // namespace helm

static helm_status solve_dispatch(helm_csr A, const double2* b, double2* x, const helm_opts& opts, helm_info* info,
                                  cudaStream_t s) {
  if (opts.launch == HELM_LAUNCH_PERSISTENT && (opts.method != HELM_BICGSTAB || opts.precision != HELM_PREC_FP64))
    return HELM_ERR_INVALID;
  if (opts.precision == HELM_PREC_MIXED) {
    if (opts.method != HELM_BICGSTAB) return HELM_ERR_INVALID;
    return solve_mixed(A, b, x, opts, info, s);
  }
  if (opts.precision != HELM_PREC_FP64) return HELM_ERR_INVALID;
  if (opts.method == HELM_TFQMR) return tfqmr_fp64(A, b, x, opts, info, s);
  if (opts.method == HELM_BICGSTABL) return bicgstabl_fp64(A, b, x, opts, info, s);
  if (opts.method != HELM_BICGSTAB) return HELM_ERR_INVALID;
  return bicgstab_fp64(A, b, x, opts, info, s);
}


extern "C" {

const char* helm_status_string(helm_status s) {
  switch (s) {
    case HELM_OK: return "ok";
    case HELM_ERR_INVALID: return "invalid argument or malformed CSR";
    case HELM_ERR_CUDA: return "CUDA runtime error";
    case HELM_ERR_NOMEM: return "device allocation failed";
    case HELM_ERR_NOT_CONVERGED: return "iteration cap reached before the tolerance";
    case HELM_ERR_BREAKDOWN: return "Krylov breakdown (zero denominator)";
    case HELM_ERR_TIMEOUT: return "device deadline expired";
    case HELM_ERR_NONFINITE: return "non-finite value in the recurrence";
  }
  return "unknown status";
}

void helm_opts_default(helm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->maxit = 20000;
  o->use_x0 = 0;
  o->method = HELM_BICGSTAB;
  o->precision = HELM_PREC_FP64;
  o->inner_tol = 1e-3;
  o->deadline_s = 0.0;
  o->ell = 2;
  o->launch = HELM_LAUNCH_AUTO;
  o->precond = HELM_PRECOND_NONE;
}

helm_status helm_csr_create(helm_csr* out, int32_t n, int64_t nnz, const int32_t* d_rowptr,
                            const int32_t* d_colind, const void* d_vals, helm_dtype dt, uint32_t flags,
                            helm_stream_t stream) {
  if (!out) return HELM_ERR_INVALID;
  *out = nullptr;
  if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31)) return HELM_ERR_INVALID;
  if (dt != HELM_C128 && dt != HELM_C64) return HELM_ERR_INVALID;
  if (!d_rowptr || (nnz > 0 && (!d_colind || !d_vals))) return HELM_ERR_INVALID;
  const size_t esz = dt == HELM_C128 ? 16 : 8;
  if (!aligned(d_rowptr, 4) || !aligned(d_colind, 16) || !aligned(d_vals, 16) || esz == 0)
    return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  helm_csr A = new (std::nothrow) helm_csr_s();
  if (!A) return HELM_ERR_NOMEM;
  auto fail = [&](helm_status st) {
    helm_csr_destroy(A);
    return st;
  };
  if (cudaGetDevice(&A->device) != cudaSuccess) return fail(HELM_ERR_CUDA);
  A->num_sms = sm_count();
  A->n = n;
  A->nnz = nnz;
  A->rowptr = d_rowptr;
  A->colind = d_colind;
  A->vals = d_vals;
  A->dt = dt;

  // workspace: partials for the largest grid, tickets, error flags, state
  const size_t nparts = static_cast<size_t>(A->num_sms) * 32 * 8;  // <= 32 blocks/SM x 8 sums
  if (cudaMalloc(&A->partials, nparts * sizeof(double)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMalloc(&A->tickets, (TK_COUNT + 2) * sizeof(unsigned int)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMemsetAsync(A->tickets, 0, (TK_COUNT + 2) * sizeof(unsigned int), s) != cudaSuccess)
    return fail(HELM_ERR_CUDA);
  A->dev_err = A->tickets + TK_COUNT;
  if (cudaMalloc(&A->gtickets, 2 * kGroupTickets * sizeof(unsigned int)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMemsetAsync(A->gtickets, 0, 2 * kGroupTickets * sizeof(unsigned int), s) != cudaSuccess)
    return fail(HELM_ERR_CUDA);
  // two solver states: [0] the Krylov loop, [1] an outer loop (refinement)
  if (cudaMalloc(&A->state, 2 * sizeof(SolverState)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMemsetAsync(A->state, 0, 2 * sizeof(SolverState), s) != cudaSuccess) return fail(HELM_ERR_CUDA);
  if (cudaMallocHost(&A->state_host, 2 * sizeof(SolverState)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  std::memset(A->state_host, 0, 2 * sizeof(SolverState));

  // pattern checks and row statistics: one pass, one synchronisation
  int* d_chk = nullptr;
  int h_chk[2] = {0, 0};
  int32_t h_end[2] = {0, 0};
  if (cudaMalloc(&d_chk, 2 * sizeof(int)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  cudaError_t e = cudaMemsetAsync(d_chk, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess && n > 0) {
    k_csr_check<<<vec_grid_for(n), 256, 0, s>>>(n, nnz, d_rowptr, d_colind, (flags & HELM_CSR_VALIDATE) ? 1 : 0,
                                                d_chk);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_chk, d_chk, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_end[0], d_rowptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_end[1], d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_chk);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(HELM_ERR_CUDA);
  }
  if (h_end[0] != 0 || h_end[1] != nnz || h_chk[1]) return fail(HELM_ERR_INVALID);
  A->max_row = h_chk[0];
  A->vec_grid = vec_grid_for(n);
  // the SELL-32 copy the SpMV engine reads (columns, real parts, imaginary
  // entries), then the stand-alone SpMV variant for this matrix
  helm_status st = build_sell_pattern(A, s);
  // complex64 products read the diagonal copy when the pattern has one
  if (st == HELM_OK && !(flags & HELM_CSR_SLICED_ONLY)) st = analyze_diagonals(A, s);
  if (st == HELM_OK) st = build_sell_vals(A, d_vals, dt, &A->sv, s);
  if (st == HELM_OK)
    st = dt == HELM_C128 ? autotune_spmv<double2>(A, csr_dev<double2>(A, static_cast<const double2*>(d_vals), A->sv), s)
                         : autotune_spmv<float2>(A, csr_dev<float2>(A, static_cast<const float2*>(d_vals), A->sv), s);
  if (st != HELM_OK) return fail(st);
  *out = A;
  return HELM_OK;
}

helm_status helm_csr_destroy(helm_csr A) {
  if (!A) return HELM_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(A->device);
  cudaDeviceSynchronize();
  for (auto& kv : A->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  cudaFree(A->partials);
  cudaFree(A->tickets);
  cudaFree(A->gtickets);
  cudaFree(A->state);
  if (A->state_host) cudaFreeHost(A->state_host);
  cudaFree(A->vec);
  cudaFree(A->vals32);
  cudaFree(A->sell_off);
  cudaFree(A->sell_col);
  cudaFree(A->dia_off);
  free_sell_vals(&A->sv);
  free_sell_vals(&A->sv32);
  free_sell_vals(&A->svjac);
  cudaFree(A->jac_vals);
  cudaFree(A->jac_d);
  cudaFree(A->jac_dinv);
  cudaFree(A->vec32);
  (void)cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
  delete A;
  return HELM_OK;
}

helm_status helm_csr_diagonals(helm_csr A, int32_t* out) {
  if (!A || !out) return HELM_ERR_INVALID;
  *out = A->ndia;
  return HELM_OK;
}

helm_status helm_spmv(helm_csr A, const double* alpha, const void* d_x, const double* beta, void* d_y,
                      helm_stream_t stream) {
  if (!A || !alpha || !beta) return HELM_ERR_INVALID;
  if (A->n > 0 && (!d_x || !d_y)) return HELM_ERR_INVALID;
  const size_t vb = static_cast<size_t>(A->n) * (A->dt == HELM_C128 ? sizeof(double2) : sizeof(float2));
  if (overlaps(d_x, vb, d_y, vb)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (A->dt == HELM_C128) {
    if (!aligned(d_x, 16) || !aligned(d_y, 16)) return HELM_ERR_INVALID;
    return launch_spmv128(A, static_cast<const double2*>(d_x), static_cast<double2*>(d_y),
                          make_double2(alpha[0], alpha[1]), make_double2(beta[0], beta[1]), s);
  }
  if (!aligned(d_x, 8) || !aligned(d_y, 8)) return HELM_ERR_INVALID;
  return launch_spmv64(A, static_cast<const float2*>(d_x),
                       static_cast<float2*>(d_y), make_float2((float)alpha[0], (float)alpha[1]),
                       make_float2((float)beta[0], (float)beta[1]), s);
}

helm_status helm_dot(int64_t n, helm_dtype dt, const void* d_x, const void* d_y, int conj_x, void* d_out,
                     helm_stream_t stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || !d_out || (dt != HELM_C128 && dt != HELM_C64)) return HELM_ERR_INVALID;
  if (n > 0 && (!d_x || !d_y)) return HELM_ERR_INVALID;
  const size_t esz = dt == HELM_C128 ? 16 : 8;
  if (!aligned(d_x, esz) || !aligned(d_y, esz) || !aligned(d_out, 16)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = vec_grid_for(n);
  double* part = nullptr;
  HELM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&part), sizeof(double) * 2 * grid, s));
  if (dt == HELM_C128) {
    if (conj_x)
      k_dot_partial<double2, true><<<grid, 256, 0, s>>>(n, (const double2*)d_x, (const double2*)d_y, part);
    else
      k_dot_partial<double2, false><<<grid, 256, 0, s>>>(n, (const double2*)d_x, (const double2*)d_y, part);
  } else {
    if (conj_x)
      k_dot_partial<float2, true><<<grid, 256, 0, s>>>(n, (const float2*)d_x, (const float2*)d_y, part);
    else
      k_dot_partial<float2, false><<<grid, 256, 0, s>>>(n, (const float2*)d_x, (const float2*)d_y, part);
  }
  k_sum_partials<2><<<1, 256, 0, s>>>(grid, part, static_cast<double*>(d_out), 0);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}

helm_status helm_nrm2(int64_t n, helm_dtype dt, const void* d_x, double* d_out, helm_stream_t stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || !d_out || (dt != HELM_C128 && dt != HELM_C64)) return HELM_ERR_INVALID;
  if (n > 0 && !d_x) return HELM_ERR_INVALID;
  const size_t esz = dt == HELM_C128 ? 16 : 8;
  if (!aligned(d_x, esz) || !aligned(d_out, 8)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = vec_grid_for(n);
  double* part = nullptr;
  HELM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&part), sizeof(double) * grid, s));
  if (dt == HELM_C128)
    k_nrm2_partial<double2><<<grid, 256, 0, s>>>(n, (const double2*)d_x, part);
  else
    k_nrm2_partial<float2><<<grid, 256, 0, s>>>(n, (const float2*)d_x, part);
  k_sum_partials<1><<<1, 256, 0, s>>>(grid, part, d_out, 1);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(part, s);
  if (e != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}

helm_status helm_axpby(int64_t n, helm_dtype dt, const double* alpha, const void* d_x, const double* beta,
                       void* d_y, helm_stream_t stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || !alpha || !beta || (dt != HELM_C128 && dt != HELM_C64))
    return HELM_ERR_INVALID;
  if (n == 0) return HELM_OK;
  if (!d_y || (!is_zero(alpha) && !d_x)) return HELM_ERR_INVALID;
  const size_t esz = dt == HELM_C128 ? 16 : 8;
  if (!aligned(d_x, esz) || !aligned(d_y, esz)) return HELM_ERR_INVALID;
  auto kind = [](const double* z) { return is_zero(z) ? 0 : is_one(z) ? 1 : z[1] == 0.0 ? 2 : 3; };
  const int xa = kind(alpha), yb = kind(beta);
  if (xa == 0 && yb == 1) return HELM_OK;  // y = y
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = vec_grid_for(n);
  if (dt == HELM_C128)
    launch_axpby<double2>(xa, yb, grid, s, n, make_double2(alpha[0], alpha[1]), (const double2*)d_x,
                          make_double2(beta[0], beta[1]), (double2*)d_y);
  else
    launch_axpby<float2>(xa, yb, grid, s, n, make_float2((float)alpha[0], (float)alpha[1]), (const float2*)d_x,
                         make_float2((float)beta[0], (float)beta[1]), (float2*)d_y);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

helm_status helm_bicgstab_solve(helm_csr A, const void* d_b, void* d_x, const helm_opts* o, helm_info* info,
                                helm_stream_t stream) {
  helm_opts opts;
  if (o) opts = *o;
  else helm_opts_default(&opts);
  if (info) std::memset(info, 0, sizeof(*info));
  if (!A || A->dt != HELM_C128) return HELM_ERR_INVALID;
  if (A->n > 0 && (!d_b || !d_x)) return HELM_ERR_INVALID;
  if (!aligned(d_b, 16) || !aligned(d_x, 16)) return HELM_ERR_INVALID;
  if (d_b == d_x || overlaps(d_b, sizeof(double2) * A->n, d_x, sizeof(double2) * A->n)) return HELM_ERR_INVALID;
  if (!(opts.tol >= 0.0) || opts.maxit < 0) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (opts.precond != HELM_PRECOND_NONE && opts.precond != HELM_PRECOND_JACOBI) return HELM_ERR_INVALID;
  if (opts.precond == HELM_PRECOND_JACOBI && opts.precision != HELM_PREC_FP64) return HELM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(A->mu);
  const double2* b = static_cast<const double2*>(d_b);
  double2* x = static_cast<double2*>(d_x);
  if (opts.precond != HELM_PRECOND_JACOBI) return solve_dispatch(A, b, x, opts, info, s);
  // right Jacobi: solve (A D^-1) y = b with y0 = D x0, then x = D^-1 y
  helm_status st = ensure_jacobi(A, s);
  if (st != HELM_OK) return st;
  if (opts.use_x0 && A->n > 0) k_jac_apply<<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->jac_d, x);
  HELM_CUDA_TRY(cudaGetLastError());
  st = solve_dispatch(A, b, x, opts, info, s);
  if (A->n > 0) {
    k_jac_apply<<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->jac_dinv, x);
    if (cudaGetLastError() != cudaSuccess && st == HELM_OK) st = HELM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess && st == HELM_OK) st = HELM_ERR_CUDA;
  }
  return st;
}

}  // extern "C"
