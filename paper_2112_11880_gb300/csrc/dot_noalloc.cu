// helm_dot_noalloc: the dot product of helm_dot for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync) at the point where
// they need a dot product: code running while a CUDA graph is being captured
// with a mode that forbids allocation, real-time loops that must not touch the
// allocator, or hosts embedding this library under a memory manager that owns
// every device allocation.  helm_dot needs a small scratch buffer for its
// per-block partial sums and gets it from the stream-ordered allocator; this
// variant keeps that scratch in a fixed array compiled into the library
// instead, so a call allocates and frees nothing.
//
// The array g_dot_scratch below is a file-scope __device__ variable: every GPU
// that loads libhelm holds one copy of it (64 KiB) until the process exits.
// In host code its name is only a host-side stand-in, not a device address, so
// every call looks up the real device address on the current device with
// cudaGetSymbolAddress and passes it to the kernels.  Nothing is cached: after
// a device reset the library's device code is loaded again (possibly at a new
// address), and the next call sees that address.
#include "common.cuh"
#include "internal.hpp"
#include "spmv.cuh"

namespace helm {

namespace {

// Partial sums: 2 doubles (re, im) per block, at most kNoallocMaxBlocks blocks.
constexpr int kNoallocMaxBlocks = 4096;
constexpr int kNoallocThreads = 256;
static __device__ __align__(256) double g_dot_scratch[2 * kNoallocMaxBlocks];

template <class V, bool CONJ>
__global__ void __launch_bounds__(kNoallocThreads) k_dot_partial_na(int64_t n, const V* __restrict__ x,
                                                                    const V* __restrict__ y, double* partials) {
  __shared__ double red[32 * 2];
  V acc = vzero<V>();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
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

__global__ void __launch_bounds__(kNoallocThreads) k_dot_final_na(int nparts, const double* __restrict__ partials,
                                                                  double* out) {
  __shared__ double red[32 * 2];
  double acc[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    acc[0] += partials[2 * b];
    acc[1] += partials[2 * b + 1];
  }
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

// Device address of g_dot_scratch on the current device.
helm_status scratch_address(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_dot_scratch) != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    return HELM_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return HELM_OK;
}

}  // namespace

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_dot_noalloc(int64_t n, helm_dtype dt, const void* d_x, const void* d_y, int conj_x,
                                        void* d_out, helm_stream_t stream) {
  if (n < 0 || n >= (int64_t(1) << 31)) return HELM_ERR_INVALID;  // beyond the supported maximum
  if (!d_out || (dt != HELM_C128 && dt != HELM_C64)) return HELM_ERR_INVALID;
  if (n > 0 && (!d_x || !d_y)) return HELM_ERR_INVALID;
  const size_t esz = dt == HELM_C128 ? 16 : 8;
  if (!aligned(d_x, esz) || !aligned(d_y, esz) || !aligned(d_out, 16)) return HELM_ERR_INVALID;
  double* scratch = nullptr;
  helm_status st = scratch_address(&scratch);
  if (st != HELM_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The grid never exceeds the scratch capacity; the grid-stride loop covers
  // any n below 2^31 with it.
  int64_t want = (n + kNoallocThreads - 1) / kNoallocThreads;
  int64_t cap = static_cast<int64_t>(sm_count()) * 8;
  if (cap > kNoallocMaxBlocks) cap = kNoallocMaxBlocks;
  const int grid = static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
  if (dt == HELM_C128) {
    if (conj_x)
      k_dot_partial_na<double2, true><<<grid, kNoallocThreads, 0, s>>>(n, (const double2*)d_x, (const double2*)d_y,
                                                                        scratch);
    else
      k_dot_partial_na<double2, false><<<grid, kNoallocThreads, 0, s>>>(n, (const double2*)d_x, (const double2*)d_y,
                                                                         scratch);
  } else {
    if (conj_x)
      k_dot_partial_na<float2, true><<<grid, kNoallocThreads, 0, s>>>(n, (const float2*)d_x, (const float2*)d_y,
                                                                       scratch);
    else
      k_dot_partial_na<float2, false><<<grid, kNoallocThreads, 0, s>>>(n, (const float2*)d_x, (const float2*)d_y,
                                                                        scratch);
  }
  k_dot_final_na<<<1, kNoallocThreads, 0, s>>>(grid, scratch, static_cast<double*>(d_out));
  if (cudaGetLastError() != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}
