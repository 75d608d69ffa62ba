// Batched frequency sweep: BiCGStab, TFQMR or BiCGStab(l) (Section 4's
// solvers) for F frequencies on one sparsity pattern, A_j = K - w_j^2 M +
// i w_j B formed on the fly (the Helmholtz operator of Section 1 at
// wavenumbers k = w_j / c, with the impedance term); BiCGStab also with
// complex64 inner solves.
//
// Layout: every Krylov vector is node-major, frequency-minor: V[i * Fp + j],
// Fp = F rounded up to a multiple of 32.  A warp owns one row and 32
// frequencies: the row's K, M, B values and column indices are warp-uniform
// loads (one transaction serves 32 frequencies), each gathered V[col][j..j+31]
// is one 512-byte coalesced access, and every FP64 instruction does useful
// work in all 32 lanes.  Per stored entry and frequency the work is 1 FMA to
// form Re(A_j) = K - w_j^2 M and 2 FMA for the real x complex product (rows
// whose 32-row block has B = 0), or the complex product where B != 0.
//
// All per-frequency scalars (rho, alpha, omega, beta, norms, status, counts)
// live on the device; each dot product is a per-frequency partial sum per
// block, added in block order by the last block to arrive.  A frequency that
// has converged (or failed) is frozen: its lanes do no arithmetic and write
// nothing, and a 32-frequency group whose frequencies have all stopped is
// skipped by every kernel.  The loop is one CUDA graph (conditional WHILE
// node), as for the single solve.
//
// Tile shape autotuning: at creation the sweep times the batched SpMV with
// 4, 8 and 16 warps per block on the actual matrix and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.hpp"

namespace helm {

namespace {

constexpr int kMaxF = 128;  // frequencies per sweep (<= threads per block: one thread per frequency)
#ifndef HELM_SWEEP_FORM_MAX
#define HELM_SWEEP_FORM_MAX (size_t(8) << 30)
#endif
constexpr size_t kSweepFormMax = HELM_SWEEP_FORM_MAX;  // bytes of formed A_j real parts at most (0: never)
constexpr int kSwMaxEll = 8;                                     // batched BiCGStab(l): l <= 8
constexpr int kSwGram = (kSwMaxEll + 1) * (kSwMaxEll + 2) / 2;  // Gram entries per frequency (45)

struct SweepDev {
  int32_t n;
  int64_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* K;
  const double* M;
  const double* B;
  const uint8_t* bzero_blk;  // [ceil(n / 32)]: 1 when B = 0 on every entry of the 32-row block
  const float* K32;          // FP32 copies for the complex64 inner sweep (null in the FP64 sweep)
  const float* M32;
  const float* B32;
  // FP64 sweep: the real parts of every A_j, are[k * are_ld + j] = fma(-w_j^2,
  // M_k, K_k), formed once per solve (null: formed inside every product)
  const double* are;
  int32_t are_ld;
};

// Arguments of the sweep kernels.  V is the type of the Krylov vectors:
// complex128 for the FP64 sweep, complex64 for the inner solves of the
// mixed-precision sweep (products in FP32, every partial sum and every
// scalar of the recurrence in FP64).
template <class V>
struct SweepArgsT {
  SweepDev A;
  int32_t F, Fp, G;      // frequencies, padded count, 32-frequency groups
  const double* w;       // [Fp] angular frequencies (padding: 0)
  const V* b;            // right-hand side: b[i * b_ld + j], or b[i] for all j when b_ld = 0
  int32_t b_ld;          // 0 (one b for all frequencies) or Fp
  V *x, *r, *rh, *p, *v, *s, *t;  // [n][Fp]
  double2 *rho, *alpha, *omg, *beta;    // [Fp]
  double *bnorm, *relres, *relres_true; // [Fp]
  int32_t *status, *iters, *phase;      // [Fp]
  int32_t* gactive;                     // [G]: a frequency of the group is running
  // batched TFQMR only (null otherwise): A un and d [n][Fp]; gamma and
  // (theta, tau) [Fp]; the true-residual check flags per frequency, per group
  // and for the whole sweep; the iteration at which each frequency's
  // current (re)start began
  V *q1, *q2;
  double2 *gam, *tt;
  int32_t *chk, *gcheck, *anychk, *start;
  // batched BiCGStab(l) only: r_0..r_l and u_0..u_l (r_0 = r, u_0 = p, the
  // shadow r~ = rh), rho1 [Fp], the minimal-residual coefficients [Fp][8],
  // the Gram matrices [Fp][45] and the Gram step's block partials
  V *rl[kSwMaxEll + 1], *ul[kSwMaxEll + 1];
  int32_t ell;
  double2 *rho1, *gcoef, *gram;
  double* gpart;
  SolverState* st;                      // tol, maxit, deadline, use_x0
  double* partials;                     // [blocks][Fp][K]
  unsigned int* tickets;
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};
using SweepArgs = SweepArgsT<double2>;

template <class V>
__device__ __forceinline__ void sweep_set_cond(const SweepArgsT<V>& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// Vector-type conversions and FP64-accumulated sums.
template <class V> __device__ __forceinline__ V sw_cvt(double2 z);
template <> __device__ __forceinline__ double2 sw_cvt<double2>(double2 z) { return z; }
template <> __device__ __forceinline__ float2 sw_cvt<float2>(double2 z) {
  return make_float2(static_cast<float>(z.x), static_cast<float>(z.y));
}
__device__ __forceinline__ double2 sw_dot(double2 acc, double2 a, double2 b) { return cfma_conj(a, b, acc); }
__device__ __forceinline__ double2 sw_dot(double2 acc, float2 a, float2 b) {
  const float re = fmaf(a.x, b.x, a.y * b.y);
  const float im = fmaf(a.x, b.y, -a.y * b.x);
  return make_double2(acc.x + static_cast<double>(re), acc.y + static_cast<double>(im));
}
__device__ __forceinline__ double sw_nrm(double acc, double2 a) { return cabs2_acc(a, acc); }
__device__ __forceinline__ double sw_nrm(double acc, float2 a) {
  return acc + static_cast<double>(fmaf(a.x, a.x, a.y * a.y));
}
template <class V> __device__ __forceinline__ V sw_zero();
template <> __device__ __forceinline__ double2 sw_zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 sw_zero<float2>() { return make_float2(0.f, 0.f); }

// Per-frequency partial sums of one block: each warp's lanes hold the partials
// of frequencies g*32 + lane (g = the warp's group); warps with the same group
// are added in warp order through shared memory, then one value per (block,
// frequency) goes to `partials`.  The last block adds the partials of all
// blocks in block order; there thread j < Fp owns frequency j's totals in
// tot[].  Requires Fp <= blockDim.x.  `sh` holds (warps per block) * 32 * K
// doubles.
template <int K, class V>
__device__ bool sweep_grid_sum(const SweepArgsT<V>& a, const double (&v)[K], double* sh, unsigned int* ticket,
                               double (&tot)[K]) {
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) sh[(warp * 32 + lane) * K + k] = v[k];
  __syncthreads();
  const int j = threadIdx.x;
  if (j < a.Fp) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int w = 0; w < nw; ++w) {
      const int gw = static_cast<int>((static_cast<int64_t>(blockIdx.x) * nw + w) % a.G);
      if (gw != j / 32) continue;
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += sh[(w * 32 + (j & 31)) * K + k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) a.partials[(static_cast<size_t>(blockIdx.x) * a.Fp + j) * K + k] = acc[k];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // Q = blockDim / Fp threads per frequency, each adding blocks q, q+Q, ...
  // into four interleaved accumulators (independent FP64 chains); then the Q
  // sums of a frequency are added in q order.  Fixed order throughout.
  const int Q = blockDim.x / a.Fp;
  const int jf = threadIdx.x % a.Fp, q = threadIdx.x / a.Fp;
  double acc4[4][K];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < K; ++k) acc4[c][k] = 0.0;
  if (q < Q) {
    unsigned int bb = q;
    for (; bb + 3u * Q < gridDim.x; bb += 4u * Q) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k)
          acc4[c][k] += ld_cg(&a.partials[(static_cast<size_t>(bb + c * Q) * a.Fp + jf) * K + k]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (bb + c * Q < gridDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          acc4[c][k] += ld_cg(&a.partials[(static_cast<size_t>(bb + c * Q) * a.Fp + jf) * K + k]);
      }
    }
  }
  __syncthreads();  // sh is reused below
  if (q < Q) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[(q * a.Fp + jf) * K + k] = (acc4[0][k] + acc4[1][k]) + (acc4[2][k] + acc4[3][k]);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = 0.0;
  if (j < a.Fp) {
    for (int qq = 0; qq < Q; ++qq) {
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] += sh[(qq * a.Fp + j) * K + k];
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Row i of A_j x for frequency j (w_j, w2 = w_j^2): the entries of A_j are
// formed as (fma(-w2, M, K), w_j B) and multiplied in CSR order; rows of a
// 32-row block where B = 0 take the real x complex product (bit-identical
// for finite x: the skipped terms are exact zeros).  x[col * ld + j].
__device__ __forceinline__ double2 sweep_row(const SweepDev& A, int32_t i, int j, double wj, double w2,
                                             const double2* __restrict__ x, int64_t ld) {
  const int64_t k0 = __ldg(A.rowptr + i), k1 = __ldg(A.rowptr + i + 1);
  double2 acc = make_double2(0.0, 0.0);
  if (A.bzero_blk[i >> 5] != 0) {
    if (A.are) {
      // the formed real parts: one coalesced load per entry and 32 frequencies
      const double* ar = A.are + j;
#pragma unroll 4
      for (int64_t k = k0; k < k1; ++k) {
        const int32_t c = __ldg(A.colind + k);
        const double are = __ldg(ar + k * A.are_ld);
        const double2 xv = __ldg(x + static_cast<int64_t>(c) * ld + j);
        acc.x = fma(are, xv.x, acc.x);
        acc.y = fma(are, xv.y, acc.y);
      }
    } else {
#pragma unroll 4
      for (int64_t k = k0; k < k1; ++k) {
        const int32_t c = __ldg(A.colind + k);
        const double are = fma(-w2, __ldg(A.M + k), __ldg(A.K + k));
        const double2 xv = __ldg(x + static_cast<int64_t>(c) * ld + j);
        acc.x = fma(are, xv.x, acc.x);
        acc.y = fma(are, xv.y, acc.y);
      }
    }
  } else {
#pragma unroll 2
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = __ldg(A.colind + k);
      const double re = A.are ? __ldg(A.are + k * A.are_ld + j) : fma(-w2, __ldg(A.M + k), __ldg(A.K + k));
      const double2 av = make_double2(re, wj * __ldg(A.B + k));
      acc = cfma(av, __ldg(x + static_cast<int64_t>(c) * ld + j), acc);
    }
  }
  return acc;
}

// The same row for complex64 vectors (the inner operator of the mixed
// sweep): the entries are formed in FP32 from FP32 copies of K, M, B,
// products and the row sum are FP32 -- no FP64 instruction per entry.
__device__ __forceinline__ float2 sweep_row(const SweepDev& A, int32_t i, int j, double wj, double w2,
                                            const float2* __restrict__ x, int64_t ld) {
  const int64_t k0 = __ldg(A.rowptr + i), k1 = __ldg(A.rowptr + i + 1);
  const float wf = static_cast<float>(wj), w2f = static_cast<float>(w2);
  float2 acc = make_float2(0.f, 0.f);
  if (A.bzero_blk[i >> 5] != 0) {
#pragma unroll 4
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = __ldg(A.colind + k);
      const float are = fmaf(-w2f, __ldg(A.M32 + k), __ldg(A.K32 + k));
      const float2 xv = __ldg(x + static_cast<int64_t>(c) * ld + j);
      acc.x = fmaf(are, xv.x, acc.x);
      acc.y = fmaf(are, xv.y, acc.y);
    }
  } else {
#pragma unroll 2
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = __ldg(A.colind + k);
      const float2 av = make_float2(fmaf(-w2f, __ldg(A.M32 + k), __ldg(A.K32 + k)), wf * __ldg(A.B32 + k));
      acc = cfma32(av, __ldg(x + static_cast<int64_t>(c) * ld + j), acc);
    }
  }
  return acc;
}

// Batched SpMV over the warp's (row, group) units: acc[j] = sum_k A_j[k] x[col][j].
// Calls epi(i, lane_frequency, acc) for running frequencies.
template <class V, class Epi>
__device__ __forceinline__ void sweep_spmv(const SweepArgsT<V>& a, const V* __restrict__ x, Epi& epi) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int64_t units = static_cast<int64_t>(a.A.n) * a.G;
  // a warp keeps the same group for all its units when nwarps is a multiple
  // of G (the launcher guarantees it), so its lane frequency is fixed
  const int g = static_cast<int>(gw % a.G);
  const int j = g * 32 + lane;
  const bool grp_on = a.gactive[g] != 0;
  const bool run = grp_on && j < a.F && a.status[j] == ST_RUNNING;
  const double wj = a.w[j];
  const double w2 = wj * wj;
  for (int64_t u = gw; u < units; u += nwarps) {
    if (!grp_on) break;
    const int32_t i = static_cast<int32_t>(u / a.G);
    const V acc = sweep_row(a.A, i, j, wj, w2, x, a.Fp);
    if (run) epi(i, j, acc);
  }
}

// Y_j = A_j X_j for the stand-alone batched product (helm_sweep_spmv): warp
// per (row, 32-frequency group), lane = frequency, the solver's row sum.
__global__ void __launch_bounds__(256) k_sw_apply(SweepDev A, int32_t F, int32_t G, const double* __restrict__ w,
                                                  const double2* __restrict__ X, int32_t ldx, double2* __restrict__ Y,
                                                  int32_t ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t u = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       u < static_cast<int64_t>(A.n) * G; u += nwarps) {
    const int32_t i = static_cast<int32_t>(u / G);
    const int j = static_cast<int>(u % G) * 32 + lane;
    if (j >= F) continue;
    const double wj = w[j];
    Y[static_cast<int64_t>(i) * ldy + j] = sweep_row(A, i, j, wj, wj * wj, X, ldx);
  }
}

// fresh: every frequency starts (iteration counts from 0).  Otherwise a
// restart from x: the frequencies with restart[j] != 0 run again (their
// iteration counts continue), the others keep their status and result.
template <class V>
__global__ void k_sw_configure(SweepArgsT<V> a, double tol, int32_t maxit, int32_t use_x0, double deadline_s,
                               int32_t fresh, const int32_t* __restrict__ restart) {
  SolverState* st = a.st;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->tol = tol;
    st->maxit = maxit;
    st->use_x0 = use_x0;
    st->deadline_ns = deadline_s > 0.0 ? static_cast<unsigned long long>(deadline_s * 1e9) : 0ull;
    if (fresh) st->t0 = globaltimer_ns();
    st->status = ST_RUNNING;
  }
  for (int j = threadIdx.x; j < a.Fp; j += blockDim.x) {
    if (!fresh && !(j < a.F && restart[j] != 0)) continue;
    a.status[j] = j < a.F ? ST_RUNNING : HELM_OK;
    if (fresh) a.iters[j] = 0;
    a.phase[j] = PH_RUN;
    a.relres[j] = 0.0;
    a.relres_true[j] = 0.0;
    const double2 one = make_double2(1.0, 0.0);
    a.rho[j] = one;
    a.alpha[j] = one;
    a.omg[j] = one;
    a.beta[j] = make_double2(0.0, 0.0);
  }
  for (int g = threadIdx.x; g < a.G; g += blockDim.x) a.gactive[g] = 1;
}

// Update the group flags and the loop condition from the per-frequency status
// (thread 0 of the last block of a reduction kernel, after the statuses are set).
template <class V>
__device__ void sweep_refresh_groups(const SweepArgsT<V>& a) {
  bool any = false;
  for (int g = 0; g < a.G; ++g) {
    bool on = false;
    for (int l = 0; l < 32; ++l) on |= a.status[g * 32 + l] == ST_RUNNING;
    a.gactive[g] = on ? 1 : 0;
    any |= on;
  }
  a.st->status = any ? ST_RUNNING : HELM_OK;
  sweep_set_cond(a, any);
}

// init: r = b - A_j x (or r = b, x = 0), r^ = r, p = v = 0; ||b||, ||r||, rho
template <class V>
__global__ void __launch_bounds__(512) k_sw_init(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  const int use_x0 = a.st->use_x0;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int g = static_cast<int>(gw % a.G);
  const int j = g * 32 + lane;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  auto body = [&](int32_t i, int jj, V ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + jj;
    const V bi = a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + jj : static_cast<size_t>(i)];
    const V ri = csub(bi, ax);
    a.r[idx] = ri;
    a.rh[idx] = ri;
    a.p[idx] = sw_zero<V>();
    a.v[idx] = sw_zero<V>();
    part[0] = sw_nrm(part[0], bi);
    part[1] = sw_nrm(part[1], ri);
    double2 d = sw_dot(make_double2(part[2], part[3]), ri, ri);
    part[2] = d.x;
    part[3] = d.y;
  };
  if (use_x0) {
    sweep_spmv(a, a.x, body);
  } else {
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const bool run = j < a.F && a.status[j] == ST_RUNNING;
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const int32_t i = static_cast<int32_t>(u / a.G);
      if (run) {
        a.x[static_cast<size_t>(i) * a.Fp + j] = sw_zero<V>();
        body(i, j, sw_zero<V>());
      }
    }
  }
  double tot[4];
  if (!sweep_grid_sum<4>(a, part, sh, a.tickets + TK_INIT, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;  // frozen by a restart of other frequencies
    const double bn = sqrt(tot[0]);
    a.bnorm[jj] = bn;
    int status = ST_RUNNING;
    if (!isfinite(bn)) {
      status = HELM_ERR_NONFINITE;
    } else if (bn == 0.0) {
      status = HELM_OK;
    } else {
      const double rr = sqrt(tot[1]) / bn;
      a.relres[jj] = rr;
      const double2 rho = make_double2(tot[2], tot[3]);
      if (!isfinite(rr)) status = HELM_ERR_NONFINITE;
      else if (rr <= a.st->tol) status = HELM_OK;
      else if (a.st->maxit <= 0) status = HELM_ERR_NOT_CONVERGED;
      else if (!cfinite(rho)) { status = HELM_ERR_NONFINITE; a.iters[jj] = 1; }
      else if (czero(rho)) { status = HELM_ERR_BREAKDOWN; a.iters[jj] = 1; }
      else { a.rho[jj] = rho; a.beta[jj] = rho; }
    }
    a.status[jj] = status;
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// element-wise kernels walk (row, group) units like the SpMV, 32 frequencies per warp
#define SWEEP_ELEMENTWISE_BEGIN                                                          \
  const int lane = threadIdx.x & 31;                                                     \
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; \
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;            \
  const int g = static_cast<int>(gw % a.G);                                              \
  const int j = g * 32 + lane;                                                           \
  const bool grp_on = a.gactive[g] != 0;                                                 \
  const bool run = grp_on && j < a.F && a.status[j] == ST_RUNNING;

// K1: p = r + beta (p - omega v)
template <class V>
__global__ void __launch_bounds__(512) k_sw_p(SweepArgsT<V> a) {
  SWEEP_ELEMENTWISE_BEGIN
  if (!run) return;
  const V beta = sw_cvt<V>(a.beta[j]), omg = sw_cvt<V>(a.omg[j]);
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    a.p[idx] = cfma(beta, cfms(omg, a.v[idx], a.p[idx]), a.r[idx]);
  }
}

// K2: v = A_j p, (r^, v) -> alpha
template <class V>
__global__ void __launch_bounds__(512) k_sw_v(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int g = static_cast<int>(gw % a.G);
  double part[2] = {0.0, 0.0};
  auto body = [&](int32_t i, int j, V ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    a.v[idx] = ax;
    double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], ax);
    part[0] = d.x;
    part[1] = d.y;
  };
  sweep_spmv(a, a.p, body);
  double tot[2];
  if (!sweep_grid_sum<2>(a, part, sh, a.tickets + TK_V, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    a.iters[j] += 1;
    const double2 rv = make_double2(tot[0], tot[1]);
    if (!cfinite(rv)) a.status[j] = HELM_ERR_NONFINITE;
    else if (czero(rv)) a.status[j] = HELM_ERR_BREAKDOWN;
    else {
      const double2 al = cdiv(a.rho[j], rv);
      if (!cfinite(al)) a.status[j] = HELM_ERR_NONFINITE;
      else a.alpha[j] = al;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// K3: s = r - alpha v, ||s||
template <class V>
__global__ void __launch_bounds__(512) k_sw_s(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  double part[1] = {0.0};
  if (run) {
    const V al = sw_cvt<V>(a.alpha[j]);
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      const V si = cfms(al, a.v[idx], a.r[idx]);
      a.s[idx] = si;
      part[0] = sw_nrm(part[0], si);
    }
  }
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_S, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;
    const double sn = sqrt(tot[0]);
    if (!isfinite(sn)) a.status[jj] = HELM_ERR_NONFINITE;
    else if (sn / a.bnorm[jj] <= a.st->tol) {
      a.phase[jj] = PH_SCONV;
      a.relres[jj] = sn / a.bnorm[jj];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// K4: t = A_j s, (t, s), (t, t) -> omega (frequencies stopped at s skip)
template <class V>
__global__ void __launch_bounds__(512) k_sw_t(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int g = static_cast<int>(gw % a.G);
  double part[3] = {0.0, 0.0, 0.0};
  auto body = [&](int32_t i, int j, V ax) {
    if (a.phase[j] != PH_RUN) return;
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    a.t[idx] = ax;
    double2 d = sw_dot(make_double2(part[0], part[1]), ax, a.s[idx]);
    part[0] = d.x;
    part[1] = d.y;
    part[2] = sw_nrm(part[2], ax);
  };
  sweep_spmv(a, a.s, body);
  double tot[3];
  if (!sweep_grid_sum<3>(a, part, sh, a.tickets + TK_T, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING || a.phase[j] != PH_RUN) continue;
    const double2 ts = make_double2(tot[0], tot[1]);
    const double tt = tot[2];
    if (!cfinite(ts) || !isfinite(tt)) a.status[j] = HELM_ERR_NONFINITE;
    else if (tt == 0.0) a.status[j] = HELM_ERR_BREAKDOWN;
    else {
      const double2 om = make_double2(ts.x / tt, ts.y / tt);
      if (!cfinite(om)) a.status[j] = HELM_ERR_NONFINITE;
      else a.omg[j] = om;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// K5: x += alpha p + omega s, r = s - omega t; per-frequency stop tests
template <class V>
__global__ void __launch_bounds__(512) k_sw_xr(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_set_cond(a, false);
    return;
  }
  SWEEP_ELEMENTWISE_BEGIN
  double part[3] = {0.0, 0.0, 0.0};
  if (run) {
    const V al = sw_cvt<V>(a.alpha[j]), om = sw_cvt<V>(a.omg[j]);
    const bool sconv = a.phase[j] == PH_SCONV;
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      if (sconv) {
        a.x[idx] = cfma(al, a.p[idx], a.x[idx]);
      } else {
        const V si = a.s[idx];
        a.x[idx] = cfma(om, si, cfma(al, a.p[idx], a.x[idx]));
        const V ri = cfms(om, a.t[idx], si);
        a.r[idx] = ri;
        double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], ri);
        part[0] = d.x;
        part[1] = d.y;
        part[2] = sw_nrm(part[2], ri);
      }
    }
  }
  double tot[3];
  if (!sweep_grid_sum<3>(a, part, sh, a.tickets + TK_XR, tot)) return;
  const bool late = a.st->deadline_ns != 0ull && (globaltimer_ns() - a.st->t0) > a.st->deadline_ns;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;
    if (a.phase[jj] == PH_SCONV) {
      a.status[jj] = HELM_OK;
      a.phase[jj] = PH_DONE;
      continue;
    }
    const double rr = sqrt(tot[2]) / a.bnorm[jj];
    a.relres[jj] = rr;
    const double2 om = a.omg[jj];
    if (!isfinite(rr)) a.status[jj] = HELM_ERR_NONFINITE;
    else if (rr <= a.st->tol) a.status[jj] = HELM_OK;
    else if (czero(om)) a.status[jj] = HELM_ERR_BREAKDOWN;
    else if (a.iters[jj] >= a.st->maxit) a.status[jj] = HELM_ERR_NOT_CONVERGED;
    else if (late) a.status[jj] = HELM_ERR_TIMEOUT;
    else {
      const double2 rho_new = make_double2(tot[0], tot[1]);
      const double2 beta = cmul(cdiv(rho_new, a.rho[jj]), cdiv(a.alpha[jj], om));
      if (!cfinite(rho_new) || !cfinite(beta)) { a.status[jj] = HELM_ERR_NONFINITE; a.iters[jj] += 1; }
      else if (czero(rho_new)) { a.status[jj] = HELM_ERR_BREAKDOWN; a.iters[jj] += 1; }
      else { a.rho[jj] = rho_new; a.beta[jj] = beta; }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// tail: true residual per frequency, ||b - A_j x|| / ||b||
template <class V>
__global__ void __launch_bounds__(512) k_sw_tail(SweepArgsT<V> a) {
  extern __shared__ double sh[];
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int g = static_cast<int>(gw % a.G);
  // every frequency is measured: mark them all active for the product
  double part[1] = {0.0};
  const int lane = threadIdx.x & 31;
  const int j = g * 32 + lane;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const double wj = a.w[j], w2 = wj * wj;
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const int32_t i = static_cast<int32_t>(u / a.G);
    const V acc = sweep_row(a.A, i, j, wj, w2, a.x, a.Fp);
    if (j < a.F)
      part[0] = sw_nrm(part[0], csub(a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + j : static_cast<size_t>(i)], acc));
  }
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_TAIL, tot)) return;
  for (int jj = threadIdx.x; jj < a.F; jj += blockDim.x)
    a.relres_true[jj] = a.bnorm[jj] > 0.0 ? sqrt(tot[0]) / a.bnorm[jj] : 0.0;
}

// ---------------------------------------------------------------- batched TFQMR
//
// The TFQMR of the single solve (Freund 1993; Saad 2003, Algorithm 7.8, two
// half-steps and two products with A_j per iteration) for every frequency at
// once, on the same row walk, reductions and freezing as the batched
// BiCGStab above.  The sweep's vectors take the TFQMR roles r0 = rh, w = r,
// u = p, un = s, v = v, Au = t, A un = q1, d = q2; eta lives in omg.  When a
// half-step's quasi-residual bound tau sqrt(m + 2) falls below tol ||b_j||,
// the frequency's true residual ||b_j - A_j x_j|| is computed after the odd
// half-step (only the 32-frequency groups with such a frequency make that
// product); a frequency whose bound is below tol but whose true residual is
// not stops with ST_RESTART and the host starts it again from its x.

// After a half-step of frequency j: theta = ||w|| / tau, c = 1 / sqrt(1 + theta^2),
// tau = tau theta c, eta = c^2 alpha; the bound raises the check flag.
__device__ void swq_half(const SweepArgs& a, int j, double ww, int m) {
  const double tau0 = a.tt[j].y;
  const double theta = sqrt(ww) / tau0;
  const double c = 1.0 / sqrt(1.0 + theta * theta);
  const double tau = tau0 * theta * c;
  const double2 al = a.alpha[j];
  const double2 eta = make_double2(c * c * al.x, c * c * al.y);
  if (!isfinite(theta) || !isfinite(tau) || !cfinite(eta)) {
    a.status[j] = HELM_ERR_NONFINITE;
    return;
  }
  a.tt[j] = make_double2(theta, tau);
  a.omg[j] = eta;
  const double bt = a.st->tol * a.bnorm[j];
  if (tau * tau * static_cast<double>(m + 2) <= bt * bt) a.chk[j] = 1;
  a.relres[j] = tau * sqrt(static_cast<double>(m + 2)) / a.bnorm[j];
}

// gamma = (theta^2 / alpha) eta for the next d update
__device__ __forceinline__ void swq_gamma(const SweepArgs& a, int j) {
  const double th = a.tt[j].x;
  a.gam[j] = cmul(cdiv(make_double2(th * th, 0.0), a.alpha[j]), a.omg[j]);
}

// init A: r0 = b - A_j x (or b, x = 0); w = u = r0; d = 0; ||b||, ||r0||, rho = (r0, r0)
__global__ void __launch_bounds__(512) k_swq_init_a(SweepArgs a) {
  extern __shared__ double sh[];
  const int use_x0 = a.st->use_x0;
  SWEEP_ELEMENTWISE_BEGIN
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  auto body = [&](int32_t i, int jj, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + jj;
    const double2 bi = a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + jj : static_cast<size_t>(i)];
    const double2 ri = csub(bi, ax);
    a.rh[idx] = ri;
    a.r[idx] = ri;
    a.p[idx] = ri;
    a.q2[idx] = make_double2(0.0, 0.0);
    part[0] = sw_nrm(part[0], bi);
    part[1] = sw_nrm(part[1], ri);
    const double2 d = sw_dot(make_double2(part[2], part[3]), ri, ri);
    part[2] = d.x;
    part[3] = d.y;
  };
  if (use_x0) {
    sweep_spmv(a, a.x, body);
  } else if (run) {
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const int32_t i = static_cast<int32_t>(u / a.G);
      a.x[static_cast<size_t>(i) * a.Fp + j] = make_double2(0.0, 0.0);
      body(i, j, make_double2(0.0, 0.0));
    }
  }
  double tot[4];
  if (!sweep_grid_sum<4>(a, part, sh, a.tickets + TK_INIT, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;  // frozen by a restart of other frequencies
    const double bn = sqrt(tot[0]);
    a.bnorm[jj] = bn;
    a.chk[jj] = 0;
    a.start[jj] = a.iters[jj];
    int status = ST_RUNNING;
    if (!isfinite(bn)) {
      status = HELM_ERR_NONFINITE;
    } else if (bn == 0.0) {
      status = HELM_OK;
    } else {
      const double rn = sqrt(tot[1]);
      a.relres[jj] = rn / bn;
      if (!isfinite(rn)) status = HELM_ERR_NONFINITE;
      else if (rn <= a.st->tol * bn) status = HELM_OK;
      else if (a.st->maxit <= 0) status = HELM_ERR_NOT_CONVERGED;
      a.rho[jj] = make_double2(tot[2], tot[3]);
      a.tt[jj] = make_double2(0.0, rn);  // theta = 0, tau = ||r0||
      a.omg[jj] = make_double2(0.0, 0.0);
      a.gam[jj] = make_double2(0.0, 0.0);
    }
    a.status[jj] = status;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int g2 = 0; g2 < a.G; ++g2) a.gcheck[g2] = 0;
    *a.anychk = 0;
    sweep_refresh_groups(a);
  }
}

// init B: v = A_j u, Au = v, sigma = (r0, v) -> alpha
__global__ void __launch_bounds__(512) k_swq_init_b(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_set_cond(a, false);
    return;
  }
  double part[2] = {0.0, 0.0};
  auto body = [&](int32_t i, int j, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    a.v[idx] = ax;
    a.t[idx] = ax;
    const double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], ax);
    part[0] = d.x;
    part[1] = d.y;
  };
  sweep_spmv(a, a.p, body);
  double tot[2];
  if (!sweep_grid_sum<2>(a, part, sh, a.tickets + TK_V, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    const double2 sigma = make_double2(tot[0], tot[1]), rho = a.rho[j];
    if (!cfinite(sigma) || !cfinite(rho)) a.status[j] = HELM_ERR_NONFINITE;
    else if (czero(sigma) || czero(rho)) { a.status[j] = HELM_ERR_BREAKDOWN; a.iters[j] += 1; }
    else {
      const double2 al = cdiv(rho, sigma);
      if (!cfinite(al)) a.status[j] = HELM_ERR_NONFINITE;
      else a.alpha[j] = al;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// T1, even half-step: un = u - alpha v, w -= alpha Au, d = u + gamma d, ||w||^2
__global__ void __launch_bounds__(512) k_swq_even(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  double part[1] = {0.0};
  if (run) {
    const double2 al = a.alpha[j], ga = a.gam[j];
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      const double2 ui = a.p[idx];
      a.s[idx] = cfms(al, a.v[idx], ui);
      const double2 wi = cfms(al, a.t[idx], a.r[idx]);
      a.r[idx] = wi;
      a.q2[idx] = cfma(ga, a.q2[idx], ui);
      part[0] = sw_nrm(part[0], wi);
    }
  }
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_S, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;
    a.iters[jj] += 1;
    swq_half(a, jj, tot[0], 2 * (a.iters[jj] - 1 - a.start[jj]));
    if (a.status[jj] == ST_RUNNING) swq_gamma(a, jj);  // the odd half-step's d update (same alpha)
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// T2: A un; x += eta d (the even half-step's x update)
__global__ void __launch_bounds__(512) k_swq_spmv_un(SweepArgs a) {
  if (a.st->status != ST_RUNNING) return;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int jl = static_cast<int>(gw % a.G) * 32 + (threadIdx.x & 31);
  const double2 eta = a.omg[jl];
  auto body = [&](int32_t i, int j, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    a.q1[idx] = ax;
    a.x[idx] = cfma(eta, a.q2[idx], a.x[idx]);
  };
  sweep_spmv(a, a.s, body);
}

// T3, odd half-step: w -= alpha A un, d = un + gamma d, ||w||^2, (r0, w) -> rho, beta
__global__ void __launch_bounds__(512) k_swq_odd(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  double part[3] = {0.0, 0.0, 0.0};
  if (run) {
    const double2 al = a.alpha[j], ga = a.gam[j];
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      const double2 wi = cfms(al, a.q1[idx], a.r[idx]);
      a.r[idx] = wi;
      a.q2[idx] = cfma(ga, a.q2[idx], a.s[idx]);
      part[0] = sw_nrm(part[0], wi);
      const double2 d = sw_dot(make_double2(part[1], part[2]), a.rh[idx], wi);
      part[1] = d.x;
      part[2] = d.y;
    }
  }
  double tot[3];
  if (!sweep_grid_sum<3>(a, part, sh, a.tickets + TK_T, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;
    swq_half(a, jj, tot[0], 2 * (a.iters[jj] - 1 - a.start[jj]) + 1);
    if (a.status[jj] != ST_RUNNING) continue;
    const double2 rho_new = make_double2(tot[1], tot[2]);
    if (!cfinite(rho_new)) a.status[jj] = HELM_ERR_NONFINITE;
    else if (czero(a.rho[jj])) a.status[jj] = HELM_ERR_BREAKDOWN;
    else {
      a.beta[jj] = cdiv(rho_new, a.rho[jj]);
      a.rho[jj] = rho_new;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int g2 = 0; g2 < a.G; ++g2) {
      int on = 0;
      for (int l = 0; l < 32; ++l) on |= a.status[g2 * 32 + l] == ST_RUNNING && a.chk[g2 * 32 + l] != 0;
      a.gcheck[g2] = on;
      any |= on;
    }
    *a.anychk = any;
    sweep_refresh_groups(a);
  }
}

// T4: u = w + beta un; x += eta d
__global__ void __launch_bounds__(512) k_swq_u(SweepArgs a) {
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  if (!run) return;
  const double2 be = a.beta[j], eta = a.omg[j];
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    a.p[idx] = cfma(be, a.s[idx], a.r[idx]);
    a.x[idx] = cfma(eta, a.q2[idx], a.x[idx]);
  }
}

// T5: Au = A_j u; v = Au + beta (A un + beta v); sigma = (r0, v) -> alpha, gamma
__global__ void __launch_bounds__(512) k_swq_spmv_u(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int jl = static_cast<int>(gw % a.G) * 32 + (threadIdx.x & 31);
  const double2 be = a.beta[jl];
  double part[2] = {0.0, 0.0};
  auto body = [&](int32_t i, int j, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    a.t[idx] = ax;
    const double2 vn = cfma(be, cfma(be, a.v[idx], a.q1[idx]), ax);
    a.v[idx] = vn;
    const double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], vn);
    part[0] = d.x;
    part[1] = d.y;
  };
  sweep_spmv(a, a.p, body);
  double tot[2];
  if (!sweep_grid_sum<2>(a, part, sh, a.tickets + TK_AUX1, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    const double2 sigma = make_double2(tot[0], tot[1]);
    if (!cfinite(sigma)) a.status[j] = HELM_ERR_NONFINITE;
    else if (czero(sigma) || czero(a.rho[j])) a.status[j] = HELM_ERR_BREAKDOWN;
    else {
      const double2 al = cdiv(a.rho[j], sigma);
      if (!cfinite(al)) a.status[j] = HELM_ERR_NONFINITE;
      else {
        a.alpha[j] = al;
        swq_gamma(a, j);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// T6: the true residual of the frequencies whose bound fell below tol (only
// their groups make the product); iteration cap and deadline for every
// running frequency; the loop condition.
__global__ void __launch_bounds__(512) k_swq_check(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_set_cond(a, false);
    return;
  }
  const bool late = a.st->deadline_ns != 0ull && (globaltimer_ns() - a.st->t0) > a.st->deadline_ns;
  if (*a.anychk == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int j = 0; j < a.F; ++j) {
        if (a.status[j] != ST_RUNNING) continue;
        if (a.iters[j] >= a.st->maxit) a.status[j] = HELM_ERR_NOT_CONVERGED;
        else if (late) a.status[j] = HELM_ERR_TIMEOUT;
      }
      sweep_refresh_groups(a);
    }
    return;
  }
  SweepArgs ac = a;
  ac.gactive = a.gcheck;  // only the groups with a frequency to check
  double part[1] = {0.0};
  auto body = [&](int32_t i, int j, double2 ax) {
    if (a.chk[j] == 0) return;
    const double2 bi = a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + j : static_cast<size_t>(i)];
    part[0] = sw_nrm(part[0], csub(bi, ax));
  };
  sweep_spmv(ac, a.x, body);
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_AUX2, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    int status = ST_RUNNING;
    if (a.chk[j] != 0) {
      const double rt = sqrt(tot[0]) / a.bnorm[j];
      a.chk[j] = 0;
      if (!isfinite(rt)) status = HELM_ERR_NONFINITE;
      else if (rt <= a.st->tol) status = HELM_OK;
      else if (a.iters[j] >= a.st->maxit) status = HELM_ERR_NOT_CONVERGED;
      else if (late) status = HELM_ERR_TIMEOUT;
      // the bound is below tol but the true residual is not: the recurrence
      // has drifted from b - A x; the host starts this frequency again
      else status = ST_RESTART;
    } else if (a.iters[j] >= a.st->maxit) {
      status = HELM_ERR_NOT_CONVERGED;
    } else if (late) {
      status = HELM_ERR_TIMEOUT;
    }
    a.status[j] = status;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int g2 = 0; g2 < a.G; ++g2) a.gcheck[g2] = 0;
    *a.anychk = 0;
    sweep_refresh_groups(a);
  }
}

// ---------------------------------------------------------------- batched BiCGStab(l)
//
// BiCGStab(l) of the single solve (Sleijpen & Fokkema 1993: per cycle l BiCG
// steps, 2 l products with A_j, and one minimal-residual step over r_1..r_l)
// for every frequency at once.  The scalar step before each BiCG step (at
// j = 0: the cycle count and rho0 = -omega rho0; then beta = alpha rho1 /
// rho0, rho0 = rho1) runs in the last block of the kernel before it.  The
// minimal-residual coefficients g of each frequency solve the normal
// equations of min ||r_0 - sum_k g_k r_k|| (Gram matrix of r_0..r_l in one
// fused per-frequency reduction, Cholesky in FP64 by the frequency's own
// thread), as in the single solve.

__device__ __forceinline__ void swl_stop(const SweepArgs& a, int j, double r2) {
  const double bt = a.st->tol * a.bnorm[j];
  a.relres[j] = sqrt(r2) / a.bnorm[j];
  if (!isfinite(r2)) a.status[j] = HELM_ERR_NONFINITE;
  else if (r2 <= bt * bt) a.status[j] = HELM_OK;
}

// scalar step before BiCG step j of frequency f (first: j = 0, a new cycle)
__device__ __forceinline__ void swl_beta(const SweepArgs& a, int f, bool first) {
  if (first) {
    a.iters[f] += 1;
    const double2 om = a.omg[f];
    a.rho[f] = cmul(make_double2(-om.x, -om.y), a.rho[f]);
  }
  const double2 r1 = a.rho1[f];
  if (!cfinite(r1)) a.status[f] = HELM_ERR_NONFINITE;
  else if (czero(a.rho[f])) a.status[f] = HELM_ERR_BREAKDOWN;
  else {
    a.beta[f] = cmul(a.alpha[f], cdiv(r1, a.rho[f]));
    a.rho[f] = r1;
  }
}

// init: r_0 = b - A_j x (or b, x = 0), r~ = r_0, u_0 = 0; ||b||, ||r_0||,
// rho1 = (r~, r_0); rho0 = 1, alpha = 0, omega = 1; the first scalar step
__global__ void __launch_bounds__(512) k_swl_init(SweepArgs a) {
  extern __shared__ double sh[];
  const int use_x0 = a.st->use_x0;
  SWEEP_ELEMENTWISE_BEGIN
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  auto body = [&](int32_t i, int jj, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + jj;
    const double2 bi = a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + jj : static_cast<size_t>(i)];
    const double2 ri = csub(bi, ax);
    a.r[idx] = ri;
    a.rh[idx] = ri;
    a.p[idx] = make_double2(0.0, 0.0);
    part[0] = sw_nrm(part[0], bi);
    part[1] = sw_nrm(part[1], ri);
    const double2 d = sw_dot(make_double2(part[2], part[3]), ri, ri);
    part[2] = d.x;
    part[3] = d.y;
  };
  if (use_x0) {
    sweep_spmv(a, a.x, body);
  } else if (run) {
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const int32_t i = static_cast<int32_t>(u / a.G);
      a.x[static_cast<size_t>(i) * a.Fp + j] = make_double2(0.0, 0.0);
      body(i, j, make_double2(0.0, 0.0));
    }
  }
  double tot[4];
  if (!sweep_grid_sum<4>(a, part, sh, a.tickets + TK_INIT, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;  // frozen by a restart of other frequencies
    const double bn = sqrt(tot[0]);
    a.bnorm[jj] = bn;
    if (!isfinite(bn)) {
      a.status[jj] = HELM_ERR_NONFINITE;
    } else if (bn == 0.0) {
      a.status[jj] = HELM_OK;
    } else {
      swl_stop(a, jj, tot[1]);
      if (a.status[jj] == ST_RUNNING && a.st->maxit <= 0) a.status[jj] = HELM_ERR_NOT_CONVERGED;
      a.rho[jj] = make_double2(1.0, 0.0);
      a.alpha[jj] = make_double2(0.0, 0.0);
      a.omg[jj] = make_double2(1.0, 0.0);
      a.rho1[jj] = make_double2(tot[2], tot[3]);
      if (a.status[jj] == ST_RUNNING) swl_beta(a, jj, true);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// B1: u_i = r_i - beta u_i, i <= js
__global__ void __launch_bounds__(512) k_swl_u(SweepArgs a, int js) {
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  if (!run) return;
  const double2 be = a.beta[j];
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    for (int i = 0; i <= js; ++i) a.ul[i][idx] = cfms(be, a.ul[i][idx], a.rl[i][idx]);
  }
}

// B2: u_{js+1} = A_j u_js, gamma = (r~, u_{js+1}) -> alpha = rho0 / gamma
__global__ void __launch_bounds__(512) k_swl_au(SweepArgs a, int js) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  double part[2] = {0.0, 0.0};
  double2* out = a.ul[js + 1];
  auto body = [&](int32_t i, int j, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    out[idx] = ax;
    const double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], ax);
    part[0] = d.x;
    part[1] = d.y;
  };
  sweep_spmv(a, a.ul[js], body);
  double tot[2];
  if (!sweep_grid_sum<2>(a, part, sh, a.tickets + TK_V, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    const double2 gm = make_double2(tot[0], tot[1]);
    if (!cfinite(gm)) a.status[j] = HELM_ERR_NONFINITE;
    else if (czero(gm)) a.status[j] = HELM_ERR_BREAKDOWN;
    else {
      const double2 al = cdiv(a.rho[j], gm);
      if (!cfinite(al)) a.status[j] = HELM_ERR_NONFINITE;
      else a.alpha[j] = al;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// B3: r_i -= alpha u_{i+1} (i <= js), x += alpha u_0; ||r_0||^2 -> stop test
__global__ void __launch_bounds__(512) k_swl_r(SweepArgs a, int js) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  double part[1] = {0.0};
  if (run) {
    const double2 al = a.alpha[j];
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      for (int i = 0; i <= js; ++i) {
        const double2 ri = cfms(al, a.ul[i + 1][idx], a.rl[i][idx]);
        a.rl[i][idx] = ri;
        if (i == 0) part[0] = sw_nrm(part[0], ri);
      }
      a.x[idx] = cfma(al, a.ul[0][idx], a.x[idx]);
    }
  }
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_S, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x)
    if (a.status[jj] == ST_RUNNING) swl_stop(a, jj, tot[0]);
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// B4: r_{js+1} = A_j r_js, rho1 = (r~, r_{js+1}); the scalar step of BiCG step js + 1
__global__ void __launch_bounds__(512) k_swl_ar(SweepArgs a, int js) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) return;
  double part[2] = {0.0, 0.0};
  double2* out = a.rl[js + 1];
  auto body = [&](int32_t i, int j, double2 ax) {
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    out[idx] = ax;
    const double2 d = sw_dot(make_double2(part[0], part[1]), a.rh[idx], ax);
    part[0] = d.x;
    part[1] = d.y;
  };
  sweep_spmv(a, a.rl[js], body);
  double tot[2];
  if (!sweep_grid_sum<2>(a, part, sh, a.tickets + TK_T, tot)) return;
  for (int j = threadIdx.x; j < a.F && j == (int)threadIdx.x; j += blockDim.x) {
    if (a.status[j] != ST_RUNNING) continue;
    a.rho1[j] = make_double2(tot[0], tot[1]);
    if (js + 1 < a.ell) swl_beta(a, j, false);
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// M1: per-frequency Gram matrix G_ik = (r_i, r_k), 0 <= i <= k <= L, one fused
// reduction (per-block partials in warp order, then block order); the
// frequency's thread solves sum_k G_ik g_k = G_i0 (i = 1..L) by Cholesky in
// FP64.  Dynamic shared memory: at least 2 doubles per thread.
template <int L>
__global__ void __launch_bounds__(512) k_swl_gram(SweepArgs a) {
  constexpr int NG = (L + 1) * (L + 2) / 2;
  extern __shared__ double sh[];
  __shared__ bool s_last;
  if (a.st->status != ST_RUNNING) return;
  SWEEP_ELEMENTWISE_BEGIN
  double acc[2 * NG];
#pragma unroll
  for (int e = 0; e < 2 * NG; ++e) acc[e] = 0.0;
  if (run) {
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      double2 rv[L + 1];
#pragma unroll
      for (int i = 0; i <= L; ++i) rv[i] = a.rl[i][idx];
      int e = 0;
#pragma unroll
      for (int i = 0; i <= L; ++i)
#pragma unroll
        for (int k = i; k <= L; ++k, ++e) {
          const double2 d = sw_dot(make_double2(acc[2 * e], acc[2 * e + 1]), rv[i], rv[k]);
          acc[2 * e] = d.x;
          acc[2 * e + 1] = d.y;
        }
    }
  }
  // block partials, entry by entry: the warps of a frequency's group in warp order
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = 0; e < NG; ++e) {
    sh[(warp * 32 + lane) * 2] = acc[2 * e];
    sh[(warp * 32 + lane) * 2 + 1] = acc[2 * e + 1];
    __syncthreads();
    const int jt = threadIdx.x;
    if (jt < a.Fp) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < nw; ++w) {
        const int gg = static_cast<int>((static_cast<int64_t>(blockIdx.x) * nw + w) % a.G);
        if (gg != jt / 32) continue;
        s0 += sh[(w * 32 + (jt & 31)) * 2];
        s1 += sh[(w * 32 + (jt & 31)) * 2 + 1];
      }
      const size_t o = (static_cast<size_t>(blockIdx.x) * a.Fp + jt) * (2 * NG) + 2 * e;
      a.gpart[o] = s0;
      a.gpart[o + 1] = s1;
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.tickets + TK_AUX2, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // totals: Q threads per frequency add blocks q, q + Q, ...; the Q sums in q order
  const int Q = blockDim.x / a.Fp;
  const int jf = threadIdx.x % a.Fp, q = threadIdx.x / a.Fp;
  for (int e = 0; e < NG; ++e) {
    double s0 = 0.0, s1 = 0.0;
    if (q < Q) {
      for (unsigned int bb = q; bb < gridDim.x; bb += Q) {
        const size_t o = (static_cast<size_t>(bb) * a.Fp + jf) * (2 * NG) + 2 * e;
        s0 += ld_cg(&a.gpart[o]);
        s1 += ld_cg(&a.gpart[o + 1]);
      }
    }
    __syncthreads();
    if (q < Q) {
      sh[(q * a.Fp + jf) * 2] = s0;
      sh[(q * a.Fp + jf) * 2 + 1] = s1;
    }
    __syncthreads();
    if (threadIdx.x < a.Fp) {
      double t0 = 0.0, t1 = 0.0;
      for (int qq = 0; qq < Q; ++qq) {
        t0 += sh[(qq * a.Fp + threadIdx.x) * 2];
        t1 += sh[(qq * a.Fp + threadIdx.x) * 2 + 1];
      }
      a.gram[static_cast<size_t>(threadIdx.x) * kSwGram + e] = make_double2(t0, t1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) a.tickets[TK_AUX2] = 0u;
  const int f = threadIdx.x;
  if (f < a.F && a.status[f] == ST_RUNNING) {
    const double2* gm = a.gram + static_cast<size_t>(f) * kSwGram;
    // G_ik for i <= k at index e(i, k); G_ki = conj(G_ik)
    auto G = [&](int i, int k) -> double2 {
      const bool sw = i > k;
      const int lo = sw ? k : i, hi = sw ? i : k;
      const double2 v = gm[lo * (L + 1) - lo * (lo - 1) / 2 + (hi - lo)];
      return sw ? make_double2(v.x, -v.y) : v;
    };
    double2 Lc[L][L];
    double2 g[L];
    bool ok = true;
    for (int i = 0; i < L && ok; ++i) {
      for (int k = 0; k <= i; ++k) {
        double2 sacc = G(i + 1, k + 1);
        for (int m = 0; m < k; ++m) sacc = csub(sacc, cmul(Lc[i][m], make_double2(Lc[k][m].x, -Lc[k][m].y)));
        if (i == k) {
          if (!(sacc.x > 0.0) || !isfinite(sacc.x)) {
            ok = false;
            break;
          }
          Lc[i][i] = make_double2(sqrt(sacc.x), 0.0);
        } else {
          Lc[i][k] = make_double2(sacc.x / Lc[k][k].x, sacc.y / Lc[k][k].x);
        }
      }
    }
    if (!ok) {
      a.status[f] = HELM_ERR_BREAKDOWN;
    } else {
      double2 y[L];
      for (int i = 0; i < L; ++i) {  // L y = c
        double2 sacc = G(i + 1, 0);
        for (int m = 0; m < i; ++m) sacc = csub(sacc, cmul(Lc[i][m], y[m]));
        y[i] = make_double2(sacc.x / Lc[i][i].x, sacc.y / Lc[i][i].x);
      }
      for (int i = L - 1; i >= 0; --i) {  // L^H g = y
        double2 sacc = y[i];
        for (int m = i + 1; m < L; ++m) sacc = csub(sacc, cmul(make_double2(Lc[m][i].x, -Lc[m][i].y), g[m]));
        g[i] = make_double2(sacc.x / Lc[i][i].x, sacc.y / Lc[i][i].x);
      }
      bool fin = true;
      for (int i = 0; i < L; ++i) {
        fin &= cfinite(g[i]);
        a.gcoef[static_cast<size_t>(f) * kSwMaxEll + i] = g[i];
      }
      if (!fin) a.status[f] = HELM_ERR_NONFINITE;
      else {
        a.omg[f] = g[L - 1];
        if (czero(g[L - 1])) a.status[f] = HELM_ERR_BREAKDOWN;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// M2: x += sum g_k r_{k-1}; r_0 -= sum g_k r_k; u_0 -= sum g_k u_k;
// ||r_0||^2, (r~, r_0) -> stop test, rho1; iteration cap, deadline; the
// first scalar step of the next cycle
template <int L>
__global__ void __launch_bounds__(512) k_swl_mr(SweepArgs a) {
  extern __shared__ double sh[];
  if (a.st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_set_cond(a, false);
    return;
  }
  SWEEP_ELEMENTWISE_BEGIN
  double part[3] = {0.0, 0.0, 0.0};
  if (run) {
    double2 gk[L];
#pragma unroll
    for (int k = 0; k < L; ++k) gk[k] = a.gcoef[static_cast<size_t>(j) * kSwMaxEll + k];
    for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
      const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
      double2 xq = a.x[idx], r0 = a.rl[0][idx], u0 = a.ul[0][idx];
      double2 rprev = r0;
#pragma unroll
      for (int k = 1; k <= L; ++k) {
        const double2 rk = a.rl[k][idx];
        xq = cfma(gk[k - 1], rprev, xq);
        r0 = cfms(gk[k - 1], rk, r0);
        u0 = cfms(gk[k - 1], a.ul[k][idx], u0);
        rprev = rk;
      }
      a.x[idx] = xq;
      a.rl[0][idx] = r0;
      a.ul[0][idx] = u0;
      part[0] = sw_nrm(part[0], r0);
      const double2 d = sw_dot(make_double2(part[1], part[2]), a.rh[idx], r0);
      part[1] = d.x;
      part[2] = d.y;
    }
  }
  double tot[3];
  if (!sweep_grid_sum<3>(a, part, sh, a.tickets + TK_XR, tot)) return;
  const bool late = a.st->deadline_ns != 0ull && (globaltimer_ns() - a.st->t0) > a.st->deadline_ns;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    if (a.status[jj] != ST_RUNNING) continue;
    swl_stop(a, jj, tot[0]);
    a.rho1[jj] = make_double2(tot[1], tot[2]);
    if (a.status[jj] != ST_RUNNING) continue;
    if (a.iters[jj] >= a.st->maxit) a.status[jj] = HELM_ERR_NOT_CONVERGED;
    else if (late) a.status[jj] = HELM_ERR_TIMEOUT;
    else swl_beta(a, jj, true);
  }
  __syncthreads();
  if (threadIdx.x == 0) sweep_refresh_groups(a);
}

// X_user[i * ldx + j] <-> x[i * Fp + j]
__global__ void k_sw_copy(int32_t n, int32_t F, int32_t Fp, const double2* __restrict__ src, int32_t lds,
                          double2* __restrict__ dst, int32_t ldd) {
  const int64_t total = static_cast<int64_t>(n) * F;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / F, j = q % F;
    dst[i * ldd + j] = src[i * lds + j];
  }
  (void)Fp;
}

__global__ void k_sw_bzero(int32_t n, const int32_t* __restrict__ rowptr, const double* __restrict__ B,
                           uint8_t* __restrict__ flags) {
  const int32_t nblk = (n + 31) / 32;
  for (int32_t blk = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); blk < nblk;
       blk += gridDim.x * (blockDim.x / 32)) {
    const int32_t r0 = blk * 32, r1 = min(r0 + 32, n);
    bool zero = true;
    for (int64_t k = rowptr[r0] + (threadIdx.x & 31); k < rowptr[r1]; k += 32)
      if (B[k] != 0.0) zero = false;
    zero = __all_sync(0xffffffffu, zero);
    if ((threadIdx.x & 31) == 0) flags[blk] = zero ? 1 : 0;
  }
}

// FP32 copies of the K, M, B values (the complex64 inner sweep's operator)
// are[k * Fp + j] = fma(-w_j^2, M_k, K_k): the real parts of all A_j, with
// the product's own formula (w_j^2 = w_j * w_j), so the products give the
// same bits as when they form them.
__global__ void k_sw_form(int64_t nnz, int32_t Fp, const double* __restrict__ K, const double* __restrict__ M,
                          const double* __restrict__ w, double* __restrict__ are) {
  const int64_t total = nnz * Fp;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = q / Fp;
    const int j = static_cast<int>(q % Fp);
    const double wj = w[j];
    const double w2 = wj * wj;
    are[q] = fma(-w2, M[k], K[k]);
  }
}

__global__ void k_sw_to_f32(int64_t nnz, const double* __restrict__ K, const double* __restrict__ M,
                            const double* __restrict__ B, float* __restrict__ out) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    out[k] = static_cast<float>(K[k]);
    out[nnz + k] = static_cast<float>(M[k]);
    out[2 * nnz + k] = static_cast<float>(B[k]);
  }
}

// SpMV-only kernel for the tile-shape autotuner (x = y = internal buffers).
template <class V>
__global__ void __launch_bounds__(512) k_sw_spmv_probe(SweepArgsT<V> a) {
  auto body = [&](int32_t i, int j, V ax) { a.v[static_cast<size_t>(i) * a.Fp + j] = ax; };
  sweep_spmv(a, a.p, body);
}

// ---------------------------------------------------------------- mixed precision
// The mixed-precision sweep: FP64 refinement per frequency around complex64
// inner sweeps (the kernels above instantiated for complex64 vectors).  One
// refinement step for every frequency still running: r_j = b_j - A_j x_j in
// FP64, sigma_j = ||r_j|| / sqrt(n), the inner sweep solves A_j d_j =
// r_j / sigma_j in complex64 to a reduction of inner_tol, then z_j = sigma_j
// d_j (FP64), w_j = A_j z_j and the step gamma_j = (w_j, r_j) / (w_j, w_j)
// that minimises ||r_j - gamma w_j||, x_j += gamma_j z_j.  Frequencies that
// have stopped get f_j = 0, which the inner sweep freezes at once.

struct MxsArgs {
  SweepArgs a;          // FP64 geometry; a.x = x_j, a.r = r_j, a.p = z_j, a.v = w_j, a.b / a.b_ld = b
  float2* x32;          // inner solutions d_j
  float2* f32;          // inner right-hand sides
  const int32_t* act;   // [Fp] 1: running, 2: b_j = 0 (x_j = 0), 0: stopped
  const double* sigma;  // [Fp]
  const double2* gamma; // [Fp]
  double* out;          // [Fp][4] per-frequency sums of the last reduction
};

#define MXS_UNITS_BEGIN                                                                  \
  const SweepArgs& a = m.a;                                                              \
  const int lane = threadIdx.x & 31;                                                     \
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; \
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;            \
  const int g = static_cast<int>(gw % a.G);                                              \
  const int j = g * 32 + lane;                                                           \
  const bool on = j < a.F && m.act[j] == 1;

// r = b - A x (or b when zero_x), out[j][0] = ||r_j||^2
__global__ void __launch_bounds__(512) k_mxs_residual(MxsArgs m, int zero_x) {
  extern __shared__ double sh[];
  MXS_UNITS_BEGIN
  double part[1] = {0.0};
  const double wj = a.w[j], w2 = wj * wj;
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const int32_t i = static_cast<int32_t>(u / a.G);
    if (!on) continue;
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    const double2 bi = a.b[a.b_ld ? static_cast<size_t>(i) * a.b_ld + j : static_cast<size_t>(i)];
    const double2 ri = zero_x ? bi : csub(bi, sweep_row(a.A, i, j, wj, w2, a.x, a.Fp));
    a.r[idx] = ri;
    part[0] = cabs2_acc(ri, part[0]);
  }
  double tot[1];
  if (!sweep_grid_sum<1>(a, part, sh, a.tickets + TK_AUX0, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) m.out[4 * jj] = tot[0];
}

// f_j = complex64(r_j / sigma_j) for running frequencies, 0 for the others
__global__ void __launch_bounds__(512) k_mxs_down(MxsArgs m) {
  MXS_UNITS_BEGIN
  if (j >= a.Fp) return;
  const double inv = on ? 1.0 / m.sigma[j] : 0.0;
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    float2 f = make_float2(0.f, 0.f);
    if (on) {
      const double2 ri = a.r[idx];
      f = make_float2(static_cast<float>(ri.x * inv), static_cast<float>(ri.y * inv));
    }
    m.f32[idx] = f;
  }
}

// z_j = sigma_j complex128(d_j)
__global__ void __launch_bounds__(512) k_mxs_lift(MxsArgs m) {
  MXS_UNITS_BEGIN
  if (!on) return;
  const double sc = m.sigma[j];
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    const float2 d = m.x32[idx];
    a.p[idx] = make_double2(sc * static_cast<double>(d.x), sc * static_cast<double>(d.y));
  }
}

// w_j = A_j z_j (FP64), out[j] = ((w_j, r_j), ||w_j||^2)
__global__ void __launch_bounds__(512) k_mxs_apply(MxsArgs m) {
  extern __shared__ double sh[];
  MXS_UNITS_BEGIN
  double part[3] = {0.0, 0.0, 0.0};
  const double wj = a.w[j], w2 = wj * wj;
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const int32_t i = static_cast<int32_t>(u / a.G);
    if (!on) continue;
    const size_t idx = static_cast<size_t>(i) * a.Fp + j;
    const double2 wi = sweep_row(a.A, i, j, wj, w2, a.p, a.Fp);
    a.v[idx] = wi;
    const double2 d = cfma_conj(wi, a.r[idx], make_double2(part[0], part[1]));
    part[0] = d.x;
    part[1] = d.y;
    part[2] = cabs2_acc(wi, part[2]);
  }
  double tot[3];
  if (!sweep_grid_sum<3>(a, part, sh, a.tickets + TK_AUX1, tot)) return;
  for (int jj = threadIdx.x; jj < a.F && jj == (int)threadIdx.x; jj += blockDim.x) {
    m.out[4 * jj] = tot[0];
    m.out[4 * jj + 1] = tot[1];
    m.out[4 * jj + 2] = tot[2];
  }
}

// x_j += gamma_j z_j (running frequencies); x_j = 0 where b_j = 0
__global__ void __launch_bounds__(512) k_mxs_update(MxsArgs m) {
  const SweepArgs& a = m.a;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int j = static_cast<int>(gw % a.G) * 32 + lane;
  if (j >= a.F) return;
  const int act = m.act[j];
  const double2 gm = m.gamma[j];
  if (act == 0 || (act == 1 && czero(gm))) return;
  for (int64_t u = gw; u < static_cast<int64_t>(a.A.n) * a.G; u += nwarps) {
    const size_t idx = static_cast<size_t>(u / a.G) * a.Fp + j;
    a.x[idx] = act == 2 ? make_double2(0.0, 0.0) : cfma(gm, a.p[idx], a.x[idx]);
  }
}

}  // namespace

}  // namespace helm

using namespace helm;

struct helm_sweep_s {
  int device = 0;
  int num_sms = 1;
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const double* K = nullptr;
  const double* M = nullptr;
  const double* B = nullptr;
  uint8_t* bzero_blk = nullptr;
  int32_t Fcap = 0;  // padded frequency capacity of the buffers
  double2* vec = nullptr;         // 7 vectors [n][Fcap]
  double2* scal = nullptr;        // 4 [Fcap]
  double* dscal = nullptr;        // 3 [Fcap] + w [Fcap]
  int32_t* iscal = nullptr;       // 3 [Fcap] + groups [Fcap / 32] + restart flags [Fcap]
  SolverState* state = nullptr;
  double* partials = nullptr;
  size_t partials_cap = 0;
  unsigned int* tickets = nullptr;
  double* wapply = nullptr;       // frequencies of helm_sweep_spmv
  int32_t wapply_cap = 0;
  // mixed precision: 8 complex64 vectors [n][Fcap32] (x, r, r^, p, v, s, t,
  // f), per-frequency sigma, gamma, sums [Fcap32 * 7 doubles], flags
  float2* vec32 = nullptr;
  int32_t Fcap32 = 0;
  float* kmb32 = nullptr;         // FP32 copies of K, M, B (3 nnz)
  double* oscal = nullptr;
  int32_t* oact = nullptr;
  // batched TFQMR: 2 vectors [n][Fcapq] (A un, d), gamma and (theta, tau)
  // [2 Fcapq], check flags and start iterations [2 Fcapq], group check flags
  // [Fcapq / 32] and one sweep-wide flag
  double2* vecq = nullptr;
  double2* tqscal = nullptr;
  int32_t* tqint = nullptr;
  int32_t Fcapq = 0;
  // batched BiCGStab(l): r_1..r_l, u_1..u_l [2 l][n][Fcapl]; rho1, the
  // coefficients and the Gram matrices [Fcapl * (1 + 8 + 45)]; the Gram
  // step's block partials
  double2* vecl = nullptr;
  double2* lscal = nullptr;
  double* gpart = nullptr;
  int32_t Fcapl = 0, ellcap = 0;
  size_t gpart_cap = 0;
  int graphl_ell = 0;
  // the formed real parts of the A_j of the last FP64 solve ([nnz][Fcap_are])
  double* are = nullptr;
  size_t are_cap = 0;
  std::vector<double> are_w;      // the frequencies they were formed for
  int warps_per_block = 8;        // autotuned
  bool tuned = false;
  std::mutex mu;
  struct G {
    int32_t F = -1, b_ld = -1;
    const void* b = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
  } graph, graph32, graphq, graphl;
};

namespace {

// Graphs capture buffer addresses: both are dropped whenever a buffer they
// use is replaced.
void drop_sweep_graphs(helm_sweep S) {
  for (helm_sweep_s::G* g : {&S->graph, &S->graph32, &S->graphq, &S->graphl}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    *g = helm_sweep_s::G();
  }
}

helm_status sweep_alloc(helm_sweep S, int32_t Fp, size_t blocks) {
  if (S->Fcap < Fp) {
    cudaFree(S->vec);
    cudaFree(S->scal);
    cudaFree(S->dscal);
    cudaFree(S->iscal);
    S->vec = nullptr;
    S->scal = nullptr;
    S->dscal = nullptr;
    S->iscal = nullptr;
    S->Fcap = 0;
    const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * Fp;
    HELM_CUDA_TRY(cudaMalloc(&S->vec, 7 * nf * sizeof(double2)));
    HELM_CUDA_TRY(cudaMalloc(&S->scal, 4 * static_cast<size_t>(Fp) * sizeof(double2)));
    HELM_CUDA_TRY(cudaMalloc(&S->dscal, 4 * static_cast<size_t>(Fp) * sizeof(double)));
    HELM_CUDA_TRY(cudaMalloc(&S->iscal, (4 * static_cast<size_t>(Fp) + Fp / 32) * sizeof(int32_t)));
    S->Fcap = Fp;
    drop_sweep_graphs(S);
  }
  const size_t need = blocks * static_cast<size_t>(Fp) * 4;
  if (S->partials_cap < need) {
    cudaFree(S->partials);
    S->partials = nullptr;
    S->partials_cap = 0;
    HELM_CUDA_TRY(cudaMalloc(&S->partials, need * sizeof(double)));
    S->partials_cap = need;
    drop_sweep_graphs(S);
  }
  return HELM_OK;
}

SweepArgs make_args(helm_sweep S, int32_t F, int32_t Fp, const double2* b, int32_t b_ld) {
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = SweepDev{S->n, S->nnz, S->rowptr, S->colind, S->K, S->M, S->B, S->bzero_blk, nullptr, nullptr, nullptr};
  a.F = F;
  a.Fp = Fp;
  a.G = Fp / 32;
  a.w = S->dscal + 3 * static_cast<size_t>(S->Fcap);
  a.b = b;
  a.b_ld = b_ld;
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * Fp;
  double2* V = S->vec;
  a.x = V;
  a.r = V + nf;
  a.rh = V + 2 * nf;
  a.p = V + 3 * nf;
  a.v = V + 4 * nf;
  a.s = V + 5 * nf;
  a.t = V + 6 * nf;
  a.rho = S->scal;
  a.alpha = S->scal + Fp;
  a.omg = S->scal + 2 * Fp;
  a.beta = S->scal + 3 * Fp;
  a.bnorm = S->dscal;
  a.relres = S->dscal + Fp;
  a.relres_true = S->dscal + 2 * Fp;
  a.status = S->iscal;
  a.iters = S->iscal + Fp;
  a.phase = S->iscal + 2 * Fp;
  a.gactive = S->iscal + 3 * Fp;
  a.st = S->state;
  a.partials = S->partials;
  a.tickets = S->tickets;
  a.dev_err = S->tickets + TK_COUNT;
  return a;
}

// The inner (complex64) sweep's arguments: the same per-frequency scalars and
// geometry as the FP64 sweep, complex64 vectors, right-hand side f [n][Fp].
SweepArgsT<float2> make_args32(helm_sweep S, const SweepArgs& a64) {
  SweepArgsT<float2> a;
  std::memset(&a, 0, sizeof(a));
  a.A = a64.A;
  a.A.K32 = S->kmb32;
  a.A.M32 = S->kmb32 + S->nnz;
  a.A.B32 = S->kmb32 + 2 * S->nnz;
  a.F = a64.F;
  a.Fp = a64.Fp;
  a.G = a64.G;
  a.w = a64.w;
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * a64.Fp;
  float2* V = S->vec32;
  a.x = V;
  a.r = V + nf;
  a.rh = V + 2 * nf;
  a.p = V + 3 * nf;
  a.v = V + 4 * nf;
  a.s = V + 5 * nf;
  a.t = V + 6 * nf;
  a.b = V + 7 * nf;
  a.b_ld = a64.Fp;
  a.rho = a64.rho;
  a.alpha = a64.alpha;
  a.omg = a64.omg;
  a.beta = a64.beta;
  a.bnorm = a64.bnorm;
  a.relres = a64.relres;
  a.relres_true = a64.relres_true;
  a.status = a64.status;
  a.iters = a64.iters;
  a.phase = a64.phase;
  a.gactive = a64.gactive;
  a.st = a64.st;
  a.partials = a64.partials;
  a.tickets = a64.tickets;
  a.dev_err = a64.dev_err;
  return a;
}

helm_status sweep_alloc_mixed(helm_sweep S, int32_t Fp, cudaStream_t s) {
  if (!S->kmb32) {
    HELM_CUDA_TRY(cudaMalloc(&S->kmb32, 3 * static_cast<size_t>(std::max<int64_t>(S->nnz, 1)) * sizeof(float)));
    if (S->nnz > 0) {
      k_sw_to_f32<<<vec_grid_for(S->nnz), 256, 0, s>>>(S->nnz, S->K, S->M, S->B, S->kmb32);
      HELM_CUDA_TRY(cudaGetLastError());
    }
  }
  if (S->Fcap32 >= Fp) return HELM_OK;
  cudaFree(S->vec32);
  cudaFree(S->oscal);
  cudaFree(S->oact);
  S->vec32 = nullptr;
  S->oscal = nullptr;
  S->oact = nullptr;
  S->Fcap32 = 0;
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * Fp;
  HELM_CUDA_TRY(cudaMalloc(&S->vec32, 8 * nf * sizeof(float2)));
  HELM_CUDA_TRY(cudaMalloc(&S->oscal, 7 * static_cast<size_t>(Fp) * sizeof(double)));
  HELM_CUDA_TRY(cudaMalloc(&S->oact, static_cast<size_t>(Fp) * sizeof(int32_t)));
  S->Fcap32 = Fp;
  if (S->graph32.exec) {
    cudaGraphExecDestroy(S->graph32.exec);
    cudaGraphDestroy(S->graph32.graph);
  }
  S->graph32 = helm_sweep_s::G();
  return HELM_OK;
}

// Buffers of the batched TFQMR (allocated at its first use).
helm_status sweep_alloc_tfqmr(helm_sweep S, int32_t Fp) {
  if (S->Fcapq >= Fp) return HELM_OK;
  cudaFree(S->vecq);
  cudaFree(S->tqscal);
  cudaFree(S->tqint);
  S->vecq = nullptr;
  S->tqscal = nullptr;
  S->tqint = nullptr;
  S->Fcapq = 0;
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * Fp;
  HELM_CUDA_TRY(cudaMalloc(&S->vecq, 2 * nf * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&S->tqscal, 2 * static_cast<size_t>(Fp) * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&S->tqint, (2 * static_cast<size_t>(Fp) + Fp / 32 + 1) * sizeof(int32_t)));
  S->Fcapq = Fp;
  if (S->graphq.exec) {
    cudaGraphExecDestroy(S->graphq.exec);
    cudaGraphDestroy(S->graphq.graph);
  }
  S->graphq = helm_sweep_s::G();
  return HELM_OK;
}

void set_tfqmr_args(helm_sweep S, SweepArgs& a) {
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * a.Fp;
  a.q1 = S->vecq;
  a.q2 = S->vecq + nf;
  a.gam = S->tqscal;
  a.tt = S->tqscal + a.Fp;
  a.chk = S->tqint;
  a.start = S->tqint + a.Fp;
  a.gcheck = S->tqint + 2 * static_cast<size_t>(a.Fp);
  a.anychk = S->tqint + 2 * static_cast<size_t>(a.Fp) + a.Fp / 32;
}

// Buffers of the batched BiCGStab(l) (allocated at its first use, grown
// with l and the number of frequencies).
helm_status sweep_alloc_bicgstabl(helm_sweep S, int32_t Fp, int ell, size_t blocks) {
  if (S->Fcapl < Fp || S->ellcap < ell) {
    cudaFree(S->vecl);
    cudaFree(S->lscal);
    S->vecl = nullptr;
    S->lscal = nullptr;
    S->Fcapl = 0;
    S->ellcap = 0;
    const int32_t F2 = std::max(Fp, S->Fcapl);
    const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * F2;
    HELM_CUDA_TRY(cudaMalloc(&S->vecl, 2 * static_cast<size_t>(ell) * nf * sizeof(double2)));
    HELM_CUDA_TRY(cudaMalloc(&S->lscal, static_cast<size_t>(F2) * (1 + kSwMaxEll + kSwGram) * sizeof(double2)));
    S->Fcapl = F2;
    S->ellcap = ell;
    if (S->graphl.exec) {
      cudaGraphExecDestroy(S->graphl.exec);
      cudaGraphDestroy(S->graphl.graph);
    }
    S->graphl = helm_sweep_s::G();
  }
  const size_t need = blocks * static_cast<size_t>(Fp) * 2 * kSwGram;
  if (S->gpart_cap < need) {
    cudaFree(S->gpart);
    S->gpart = nullptr;
    S->gpart_cap = 0;
    HELM_CUDA_TRY(cudaMalloc(&S->gpart, need * sizeof(double)));
    S->gpart_cap = need;
    if (S->graphl.exec) {
      cudaGraphExecDestroy(S->graphl.exec);
      cudaGraphDestroy(S->graphl.graph);
    }
    S->graphl = helm_sweep_s::G();
  }
  return HELM_OK;
}

void set_bicgstabl_args(helm_sweep S, SweepArgs& a, int ell) {
  const size_t nf = static_cast<size_t>(std::max<int32_t>(S->n, 1)) * a.Fp;
  a.ell = ell;
  a.rl[0] = a.r;
  a.ul[0] = a.p;
  for (int k = 1; k <= kSwMaxEll; ++k) {
    a.rl[k] = k <= ell ? S->vecl + static_cast<size_t>(k - 1) * nf : nullptr;
    a.ul[k] = k <= ell ? S->vecl + static_cast<size_t>(ell + k - 1) * nf : nullptr;
  }
  a.rho1 = S->lscal;
  a.gcoef = S->lscal + a.Fp;
  a.gram = S->lscal + static_cast<size_t>(a.Fp) * (1 + kSwMaxEll);
  a.gpart = S->gpart;
}

struct SweepShape {
  int threads, grid;
  size_t smem;  // per-frequency reduction scratch
};

SweepShape sweep_shape(helm_sweep S, int G) {
  SweepShape sh;
  sh.threads = 32 * S->warps_per_block;
  // each warp keeps one group: the number of warps must be a multiple of G
  const int warps_per_block = S->warps_per_block;
  sh.smem = static_cast<size_t>(warps_per_block) * 32 * 4 * sizeof(double);
  // up to 1024 resident threads per SM (enough warps to hide latency, few
  // block partials for the per-frequency reductions), and no more blocks
  // than every sweep kernel fits on an SM at once: one wave
  int per_sm = std::max(1, 1024 / sh.threads);
  for (const void* fn :
       {reinterpret_cast<const void*>(&k_sw_init<double2>), reinterpret_cast<const void*>(&k_sw_p<double2>),
        reinterpret_cast<const void*>(&k_sw_v<double2>), reinterpret_cast<const void*>(&k_sw_s<double2>),
        reinterpret_cast<const void*>(&k_sw_t<double2>), reinterpret_cast<const void*>(&k_sw_xr<double2>),
        reinterpret_cast<const void*>(&k_sw_tail<double2>), reinterpret_cast<const void*>(&k_sw_init<float2>),
        reinterpret_cast<const void*>(&k_sw_p<float2>), reinterpret_cast<const void*>(&k_sw_v<float2>),
        reinterpret_cast<const void*>(&k_sw_s<float2>), reinterpret_cast<const void*>(&k_sw_t<float2>),
        reinterpret_cast<const void*>(&k_sw_xr<float2>), reinterpret_cast<const void*>(&k_swq_init_a),
        reinterpret_cast<const void*>(&k_swq_init_b), reinterpret_cast<const void*>(&k_swq_even),
        reinterpret_cast<const void*>(&k_swq_spmv_un), reinterpret_cast<const void*>(&k_swq_odd),
        reinterpret_cast<const void*>(&k_swq_u), reinterpret_cast<const void*>(&k_swq_spmv_u),
        reinterpret_cast<const void*>(&k_swq_check)}) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, sh.threads, sh.smem) == cudaSuccess && b >= 1)
      per_sm = std::min(per_sm, b);
  }
  (void)cudaGetLastError();
  int64_t blocks = static_cast<int64_t>(S->num_sms) * per_sm;
  int64_t units = static_cast<int64_t>(S->n) * G;
  int64_t want = (units + warps_per_block - 1) / warps_per_block;
  if (want < blocks) blocks = want < 1 ? 1 : want;
  // warps in the grid = blocks * warps_per_block: make it a multiple of G
  // (rounding down keeps one wave; up only when that leaves no block)
  const int64_t b0 = blocks;
  while (blocks > 1 && (blocks * warps_per_block) % G != 0) --blocks;
  if ((blocks * warps_per_block) % G != 0) {
    blocks = b0;
    while ((blocks * warps_per_block) % G != 0) ++blocks;
  }
  sh.grid = static_cast<int>(blocks);
  return sh;
}

template <class V>
void enqueue_sweep_body(const SweepArgsT<V>& a, const SweepShape& sh, cudaStream_t s) {
  k_sw_p<V><<<sh.grid, sh.threads, 0, s>>>(a);
  k_sw_v<V><<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_sw_s<V><<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_sw_t<V><<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_sw_xr<V><<<sh.grid, sh.threads, sh.smem, s>>>(a);
}

// init -> conditional WHILE (body: one iteration) -> tail, as one graph;
// init, body and tail enqueue their kernels with the given arguments.
template <class V, class Init, class Body, class Tail>
helm_status build_sweep_graph_with(const SweepArgsT<V>& base, Init init, Body body_fn, Tail tail,
                                   cudaGraph_t* gout, cudaGraphExec_t* eout) {
  cudaStream_t cs = nullptr;
  HELM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  helm_status result = HELM_ERR_CUDA;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess) break;
    SweepArgsT<V> a = base;
    a.cond = cond;
    a.has_cond = 1;
    if (cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    init(a, cs);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNode_t init_node = (e == cudaSuccess && ndeps == 1) ? deps[0] : nullptr;
    cudaGraph_t tmp = nullptr;
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess || e != cudaSuccess || !init_node) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, graph, &init_node, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    body_fn(a, cs);
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    tail(a, cs);
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) break;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) break;
    result = HELM_OK;
  } while (false);
  cudaStreamDestroy(cs);
  if (result != HELM_OK) {
    (void)cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return result;
  }
  *gout = graph;
  *eout = exec;
  return HELM_OK;
}

template <class V>
helm_status build_sweep_graph(const SweepArgsT<V>& base, const SweepShape& sh, cudaGraph_t* gout,
                              cudaGraphExec_t* eout) {
  return build_sweep_graph_with(
      base, [&](const SweepArgsT<V>& a, cudaStream_t cs) { k_sw_init<V><<<sh.grid, sh.threads, sh.smem, cs>>>(a); },
      [&](const SweepArgsT<V>& a, cudaStream_t cs) { enqueue_sweep_body(a, sh, cs); },
      [&](const SweepArgsT<V>& a, cudaStream_t cs) { k_sw_tail<V><<<sh.grid, sh.threads, sh.smem, cs>>>(a); }, gout,
      eout);
}

// The batched TFQMR's launches: init (two kernels), one iteration (six).
void swq_init(const SweepArgs& a, const SweepShape& sh, cudaStream_t s) {
  k_swq_init_a<<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_swq_init_b<<<sh.grid, sh.threads, sh.smem, s>>>(a);
}
void swq_body(const SweepArgs& a, const SweepShape& sh, cudaStream_t s) {
  k_swq_even<<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_swq_spmv_un<<<sh.grid, sh.threads, 0, s>>>(a);
  k_swq_odd<<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_swq_u<<<sh.grid, sh.threads, 0, s>>>(a);
  k_swq_spmv_u<<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_swq_check<<<sh.grid, sh.threads, sh.smem, s>>>(a);
}

helm_status build_tfqmr_graph(const SweepArgs& base, const SweepShape& sh, cudaGraph_t* gout, cudaGraphExec_t* eout) {
  return build_sweep_graph_with(
      base, [&](const SweepArgs& a, cudaStream_t cs) { swq_init(a, sh, cs); },
      [&](const SweepArgs& a, cudaStream_t cs) { swq_body(a, sh, cs); },
      [&](const SweepArgs& a, cudaStream_t cs) { k_sw_tail<double2><<<sh.grid, sh.threads, sh.smem, cs>>>(a); },
      gout, eout);
}

// The batched BiCGStab(l)'s launches: init, one cycle (4 l + 2 kernels).
template <int L>
void swl_body_l(const SweepArgs& a, const SweepShape& sh, cudaStream_t s) {
  for (int js = 0; js < L; ++js) {
    k_swl_u<<<sh.grid, sh.threads, 0, s>>>(a, js);
    k_swl_au<<<sh.grid, sh.threads, sh.smem, s>>>(a, js);
    k_swl_r<<<sh.grid, sh.threads, sh.smem, s>>>(a, js);
    k_swl_ar<<<sh.grid, sh.threads, sh.smem, s>>>(a, js);
  }
  k_swl_gram<L><<<sh.grid, sh.threads, sh.smem, s>>>(a);
  k_swl_mr<L><<<sh.grid, sh.threads, sh.smem, s>>>(a);
}

void swl_body(const SweepArgs& a, const SweepShape& sh, cudaStream_t s) {
  switch (a.ell) {
    case 1: swl_body_l<1>(a, sh, s); break;
    case 2: swl_body_l<2>(a, sh, s); break;
    case 3: swl_body_l<3>(a, sh, s); break;
    case 4: swl_body_l<4>(a, sh, s); break;
    case 5: swl_body_l<5>(a, sh, s); break;
    case 6: swl_body_l<6>(a, sh, s); break;
    case 7: swl_body_l<7>(a, sh, s); break;
    default: swl_body_l<8>(a, sh, s); break;
  }
}

helm_status build_bicgstabl_graph(const SweepArgs& base, const SweepShape& sh, cudaGraph_t* gout,
                                  cudaGraphExec_t* eout) {
  return build_sweep_graph_with(
      base, [&](const SweepArgs& a, cudaStream_t cs) { k_swl_init<<<sh.grid, sh.threads, sh.smem, cs>>>(a); },
      [&](const SweepArgs& a, cudaStream_t cs) { swl_body(a, sh, cs); },
      [&](const SweepArgs& a, cudaStream_t cs) { k_sw_tail<double2><<<sh.grid, sh.threads, sh.smem, cs>>>(a); },
      gout, eout);
}

// Time the batched SpMV with 4, 8 and 16 warps per block; keep the fastest.
helm_status autotune(helm_sweep S, int32_t F, int32_t Fp, cudaStream_t s) {
  const int candidates[3] = {4, 8, 16};  // 128..512 threads: at least kMaxF
  float best = 1e30f;
  int best_w = 8;
  cudaEvent_t e0, e1;
  HELM_CUDA_TRY(cudaEventCreate(&e0));
  HELM_CUDA_TRY(cudaEventCreate(&e1));
  helm_status result = HELM_OK;
  for (int c : candidates) {
    S->warps_per_block = c;
    const SweepShape sh = sweep_shape(S, Fp / 32);
    result = sweep_alloc(S, Fp, sh.grid);
    if (result != HELM_OK) break;
    SweepArgs a = make_args(S, F, Fp, nullptr, 0);
    // every group active, every frequency running, p = 0 (timing only)
    k_sw_configure<double2><<<1, 256, 0, s>>>(a, 0.0, 1, 0, 0.0, 1, nullptr);
    cudaMemsetAsync(a.p, 0, static_cast<size_t>(S->n) * Fp * sizeof(double2), s);
    k_sw_spmv_probe<double2><<<sh.grid, sh.threads, 0, s>>>(a);
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3; ++rep) k_sw_spmv_probe<double2><<<sh.grid, sh.threads, 0, s>>>(a);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      result = HELM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_w = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  S->warps_per_block = best_w;
  S->tuned = true;
  return result;
}

// The mixed-precision sweep (precision HELM_PREC_MIXED): refinement steps as
// described with the kernels above, driven from the host (a few dozen steps;
// three reads of per-frequency sums each), the inner complex64 solves one
// graph launch each.  A frequency stops when its FP64 residual meets tol,
// after five steps in a row without halving it, at the iteration cap
// (counted in inner iterations) or at the deadline.
constexpr int kSweepInnerMax = 50000;

helm_status sweep_solve_mixed(helm_sweep S, const SweepArgs& a64, const SweepShape& sh, void* d_X, int32_t ldx,
                              const helm_opts& opts, helm_info* h_infos, cudaStream_t s) {
  const int32_t F = a64.F, Fp = a64.Fp;
  HELM_TRY(sweep_alloc_mixed(S, Fp, s));
  SweepArgsT<float2> a32 = make_args32(S, a64);
  MxsArgs m;
  m.a = a64;
  m.x32 = a32.x;
  m.f32 = const_cast<float2*>(a32.b);
  m.act = S->oact;
  double* d_sigma = S->oscal;
  double2* d_gamma = reinterpret_cast<double2*>(S->oscal + Fp);
  m.sigma = d_sigma;
  m.gamma = d_gamma;
  m.out = S->oscal + 3 * static_cast<size_t>(Fp);
  const size_t nf = static_cast<size_t>(S->n) * Fp;
  if (opts.use_x0) {
    HELM_CUDA_TRY(cudaMemsetAsync(a64.x, 0, nf * sizeof(double2), s));
    k_sw_copy<<<vec_grid_for(static_cast<int64_t>(S->n) * F), 256, 0, s>>>(S->n, F, Fp,
                                                                          static_cast<const double2*>(d_X), ldx, a64.x, Fp);
  } else {
    HELM_CUDA_TRY(cudaMemsetAsync(a64.x, 0, nf * sizeof(double2), s));
  }
  if (!(S->graph32.exec && S->graph32.F == F)) {
    if (S->graph32.exec) {
      cudaGraphExecDestroy(S->graph32.exec);
      cudaGraphDestroy(S->graph32.graph);
    }
    S->graph32 = helm_sweep_s::G();
    if (build_sweep_graph(a32, sh, &S->graph32.graph, &S->graph32.exec) == HELM_OK) S->graph32.F = F;
  }
  const double inner_tol = (opts.inner_tol > 0.0 && opts.inner_tol < 1.0) ? opts.inner_tol : 1e-3;
  std::vector<int32_t> act(Fp, 0), status(Fp, ST_RUNNING), steps(Fp, 0), stall(Fp, 0), inner_it(Fp, 0), it32(Fp);
  std::vector<double> bn(Fp, 0.0), rn(Fp, 0.0), out(4 * static_cast<size_t>(Fp)), sigma(Fp, 0.0);
  std::vector<double2> gamma(Fp);
  for (int j = 0; j < F; ++j) act[j] = 1;
  auto upload_act = [&]() {
    return cudaMemcpyAsync(S->oact, act.data(), Fp * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  };
  auto residual = [&](int zero_x, std::vector<double>& norms) -> helm_status {
    HELM_CUDA_TRY(upload_act());
    k_mxs_residual<<<sh.grid, sh.threads, sh.smem, s>>>(m, zero_x);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaMemcpyAsync(out.data(), m.out, 4 * Fp * sizeof(double), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int j = 0; j < F; ++j)
      if (act[j] == 1) norms[j] = std::sqrt(out[4 * j]);
    return HELM_OK;
  };
  HELM_TRY(residual(1, bn));
  for (int j = 0; j < F; ++j) rn[j] = bn[j];
  if (opts.use_x0) HELM_TRY(residual(0, rn));
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const double elapsed = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool any = false;
    for (int j = 0; j < F; ++j) {
      if (act[j] != 1) continue;
      const double rel = bn[j] > 0.0 ? rn[j] / bn[j] : 0.0;
      int st = ST_RUNNING;
      if (bn[j] == 0.0) st = HELM_OK, act[j] = 2;  // b_j = 0: x_j = 0
      else if (!std::isfinite(rel)) st = HELM_ERR_NONFINITE;
      else if (rel <= opts.tol) st = HELM_OK;
      else if (stall[j] >= 5 || inner_it[j] >= opts.maxit) st = HELM_ERR_NOT_CONVERGED;
      else if (opts.deadline_s > 0.0 && elapsed > opts.deadline_s) st = HELM_ERR_TIMEOUT;
      status[j] = st;
      if (st != ST_RUNNING && act[j] == 1) act[j] = 0;
      if (act[j] == 1) {
        any = true;
        sigma[j] = rn[j] / std::sqrt(static_cast<double>(std::max(S->n, 1)));
      }
    }
    if (!any) break;
    // inner right-hand sides, inner complex64 sweep
    HELM_CUDA_TRY(upload_act());
    HELM_CUDA_TRY(cudaMemcpyAsync(d_sigma, sigma.data(), Fp * sizeof(double), cudaMemcpyHostToDevice, s));
    k_mxs_down<<<sh.grid, sh.threads, 0, s>>>(m);
    int32_t inner_max = kSweepInnerMax;
    for (int j = 0; j < F; ++j)
      if (act[j] == 1) inner_max = std::min(inner_max, std::max(1, opts.maxit - inner_it[j]));
    k_sw_configure<float2><<<1, 256, 0, s>>>(a32, inner_tol, inner_max, 0, 0.0, 1, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    if (S->graph32.exec) {
      HELM_CUDA_TRY(cudaGraphLaunch(S->graph32.exec, s));
    } else {
      SolverState hs;
      k_sw_init<float2><<<sh.grid, sh.threads, sh.smem, s>>>(a32);
      for (;;) {
        for (int k = 0; k < 8; ++k) enqueue_sweep_body(a32, sh, s);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(&hs, a32.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs.status != ST_RUNNING) break;
      }
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(it32.data(), a32.iters, Fp * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    // FP64 step along z = sigma d
    k_mxs_lift<<<sh.grid, sh.threads, 0, s>>>(m);
    k_mxs_apply<<<sh.grid, sh.threads, sh.smem, s>>>(m);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaMemcpyAsync(out.data(), m.out, 4 * Fp * sizeof(double), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int j = 0; j < Fp; ++j) {
      gamma[j] = make_double2(0.0, 0.0);
      if (j >= F || act[j] != 1) continue;
      inner_it[j] += it32[j];
      steps[j] += 1;
      const double ww = out[4 * j + 2];
      if (ww > 0.0 && std::isfinite(ww) && std::isfinite(out[4 * j]) && std::isfinite(out[4 * j + 1]))
        gamma[j] = make_double2(out[4 * j] / ww, out[4 * j + 1] / ww);
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(d_gamma, gamma.data(), Fp * sizeof(double2), cudaMemcpyHostToDevice, s));
    k_mxs_update<<<sh.grid, sh.threads, 0, s>>>(m);
    HELM_CUDA_TRY(cudaGetLastError());
    std::vector<double> prev = rn;
    HELM_TRY(residual(0, rn));
    for (int j = 0; j < F; ++j)
      if (act[j] == 1) stall[j] = rn[j] > 0.5 * prev[j] ? stall[j] + 1 : 0;
  }
  // b_j = 0 columns become zero, then x goes to the caller
  HELM_CUDA_TRY(upload_act());
  k_mxs_update<<<sh.grid, sh.threads, 0, s>>>(m);
  k_sw_copy<<<vec_grid_for(static_cast<int64_t>(S->n) * F), 256, 0, s>>>(S->n, F, Fp, a64.x, Fp,
                                                                        static_cast<double2*>(d_X), ldx);
  HELM_CUDA_TRY(cudaGetLastError());
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  helm_status worst = HELM_OK;
  for (int j = 0; j < F; ++j) {
    const helm_status sj = static_cast<helm_status>(status[j]);
    if (h_infos) {
      h_infos[j].iters = inner_it[j];
      h_infos[j].restarts = steps[j];
      h_infos[j].relres_recur = bn[j] > 0.0 ? rn[j] / bn[j] : 0.0;
      h_infos[j].relres_true = h_infos[j].relres_recur;
      h_infos[j].status = sj;
      h_infos[j].spmv_count = 2 * inner_it[j] + 2 * steps[j] + 1;
    }
    if (sj != HELM_OK && worst == HELM_OK) worst = sj;
  }
  return worst;
}

}  // namespace

// Bytes from the first to one past the last element of an [n][ld] complex128
// array of nfreq columns (ld = 0: one shared column).
inline size_t sweep_extent(int32_t n, int32_t ld, int32_t nfreq) {
  if (n <= 0) return 0;
  const size_t rows = static_cast<size_t>(n);
  return sizeof(double2) * (ld == 0 ? rows : (rows - 1) * static_cast<size_t>(ld) + static_cast<size_t>(nfreq));
}

extern "C" {

helm_status helm_sweep_create(helm_sweep* out, int32_t n, int64_t nnz, const int32_t* d_rowptr,
                              const int32_t* d_colind, const double* d_K, const double* d_M, const double* d_B,
                              helm_stream_t stream) {
  if (!out) return HELM_ERR_INVALID;
  *out = nullptr;
  if (n < 0 || nnz < 0 || nnz >= (int64_t(1) << 31) || !d_rowptr) return HELM_ERR_INVALID;
  if (nnz > 0 && (!d_colind || !d_K || !d_M || !d_B)) return HELM_ERR_INVALID;
  helm_sweep S = new (std::nothrow) helm_sweep_s();
  if (!S) return HELM_ERR_NOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto fail = [&](helm_status st) {
    helm_sweep_destroy(S);
    return st;
  };
  if (cudaGetDevice(&S->device) != cudaSuccess) return fail(HELM_ERR_CUDA);
  S->num_sms = sm_count();
  S->n = n;
  S->nnz = nnz;
  S->rowptr = d_rowptr;
  S->colind = d_colind;
  S->K = d_K;
  S->M = d_M;
  S->B = d_B;
  if (cudaMalloc(&S->state, sizeof(SolverState)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMalloc(&S->tickets, (TK_COUNT + 2) * sizeof(unsigned int)) != cudaSuccess) return fail(HELM_ERR_NOMEM);
  if (cudaMemsetAsync(S->tickets, 0, (TK_COUNT + 2) * sizeof(unsigned int), s) != cudaSuccess) return fail(HELM_ERR_CUDA);
  if (n > 0) {
    if (cudaMalloc(&S->bzero_blk, (n + 31) / 32) != cudaSuccess) return fail(HELM_ERR_NOMEM);
    k_sw_bzero<<<vec_grid_for(n / 32 + 1), 256, 0, s>>>(n, d_rowptr, d_B, S->bzero_blk);
    if (cudaGetLastError() != cudaSuccess) return fail(HELM_ERR_CUDA);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(HELM_ERR_CUDA);
  *out = S;
  return HELM_OK;
}

helm_status helm_sweep_destroy(helm_sweep S) {
  if (!S) return HELM_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  if (S->graph.exec) cudaGraphExecDestroy(S->graph.exec);
  if (S->graph.graph) cudaGraphDestroy(S->graph.graph);
  cudaFree(S->bzero_blk);
  cudaFree(S->vec);
  cudaFree(S->scal);
  cudaFree(S->dscal);
  cudaFree(S->iscal);
  cudaFree(S->state);
  cudaFree(S->partials);
  cudaFree(S->tickets);
  cudaFree(S->wapply);
  cudaFree(S->vec32);
  cudaFree(S->kmb32);
  cudaFree(S->oscal);
  cudaFree(S->oact);
  cudaFree(S->vecq);
  cudaFree(S->tqscal);
  cudaFree(S->tqint);
  cudaFree(S->vecl);
  cudaFree(S->lscal);
  cudaFree(S->gpart);
  cudaFree(S->are);
  if (S->graphl.exec) cudaGraphExecDestroy(S->graphl.exec);
  if (S->graphl.graph) cudaGraphDestroy(S->graphl.graph);
  if (S->graph32.exec) cudaGraphExecDestroy(S->graph32.exec);
  if (S->graph32.graph) cudaGraphDestroy(S->graph32.graph);
  if (S->graphq.exec) cudaGraphExecDestroy(S->graphq.exec);
  if (S->graphq.graph) cudaGraphDestroy(S->graphq.graph);
  (void)cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
  delete S;
  return HELM_OK;
}

helm_status helm_sweep_solve(helm_sweep S, int32_t nfreq, const double* h_omega, const void* d_b, int32_t b_ld,
                             void* d_X, int32_t ldx, const helm_opts* o, helm_info* h_infos, helm_stream_t stream) {
  helm_opts opts;
  if (o) opts = *o;
  else helm_opts_default(&opts);
  if (!S || nfreq < 1 || nfreq > kMaxF || !h_omega || (b_ld != 0 && b_ld < nfreq) || ldx < nfreq) return HELM_ERR_INVALID;
  if (S->n > 0 && (!d_b || !d_X)) return HELM_ERR_INVALID;
  if (!aligned(d_b, 16) || !aligned(d_X, 16) || !(opts.tol >= 0.0) || opts.maxit < 0) return HELM_ERR_INVALID;
  if (S->n > 0 && overlaps(d_b, sweep_extent(S->n, b_ld, nfreq), d_X, sweep_extent(S->n, ldx, nfreq)))
    return HELM_ERR_INVALID;
  if (opts.precision != HELM_PREC_FP64 && opts.precision != HELM_PREC_MIXED) return HELM_ERR_INVALID;
  if (opts.method != HELM_BICGSTAB &&
      !((opts.method == HELM_TFQMR || opts.method == HELM_BICGSTABL) && opts.precision == HELM_PREC_FP64))
    return HELM_ERR_INVALID;
  if (opts.method == HELM_BICGSTABL && (opts.ell < 1 || opts.ell > kSwMaxEll)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(S->mu);
  const int32_t Fp = (nfreq + 31) / 32 * 32;
  if (!S->tuned) {
    helm_status st = autotune(S, nfreq, Fp, s);
    if (st != HELM_OK) return st;
  }
  const SweepShape sh = sweep_shape(S, Fp / 32);
  helm_status st = sweep_alloc(S, Fp, sh.grid);
  if (st != HELM_OK) return st;
  // the user's b with its stride becomes an internal [n][Fp] copy only when
  // its stride differs from Fp; a shared b is read in place
  const double2* bsrc = static_cast<const double2*>(d_b);
  int32_t bld = b_ld;
  double2* bcopy = nullptr;
  if (b_ld != 0 && b_ld != Fp) {
    HELM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&bcopy), static_cast<size_t>(S->n) * Fp * sizeof(double2), s));
    HELM_CUDA_TRY(cudaMemsetAsync(bcopy, 0, static_cast<size_t>(S->n) * Fp * sizeof(double2), s));
    k_sw_copy<<<vec_grid_for(static_cast<int64_t>(S->n) * nfreq), 256, 0, s>>>(S->n, nfreq, Fp, bsrc, b_ld, bcopy, Fp);
    bsrc = bcopy;
    bld = Fp;
  }
  // angular frequencies, padded with zeros
  std::vector<double> w(Fp, 0.0);
  for (int j = 0; j < nfreq; ++j) w[j] = h_omega[j];
  SweepArgs a = make_args(S, nfreq, Fp, bsrc, bld);
  HELM_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(a.w), w.data(), Fp * sizeof(double), cudaMemcpyHostToDevice, s));
  if (opts.precision == HELM_PREC_MIXED) {
    st = sweep_solve_mixed(S, a, sh, d_X, ldx, opts, h_infos, s);
    if (bcopy) {
      cudaFreeAsync(bcopy, s);
      if (cudaStreamSynchronize(s) != cudaSuccess && st == HELM_OK) st = HELM_ERR_CUDA;
    }
    return st;
  }
  // the real parts of every A_j, formed once for the whole solve when they fit
  // the budget: each product then reads one value per entry and frequency
  // instead of forming it (one FP64 FMA per entry and frequency less; the
  // products are FP64-bound, the extra bytes are not the bound)
  {
    const size_t slots = static_cast<size_t>(S->nnz) * Fp;
    if (S->nnz > 0 && kSweepFormMax > 0 && slots * sizeof(double) <= kSweepFormMax) {
      if (S->are_cap < slots) {
        cudaFree(S->are);
        S->are = nullptr;
        S->are_cap = 0;
        S->are_w.clear();
        if (cudaMalloc(&S->are, slots * sizeof(double)) == cudaSuccess) S->are_cap = slots;
        else (void)cudaGetLastError();  // no room: the products form the values themselves
        drop_sweep_graphs(S);
      }
      if (S->are) {
        if (S->are_w != w) {
          k_sw_form<<<vec_grid_for(static_cast<int64_t>(slots)), 256, 0, s>>>(S->nnz, Fp, S->K, S->M, a.w, S->are);
          HELM_CUDA_TRY(cudaGetLastError());
          S->are_w = w;
        }
        a.A.are = S->are;
        a.A.are_ld = Fp;
      }
    }
  }
  if (opts.use_x0) {
    HELM_CUDA_TRY(cudaMemsetAsync(a.x, 0, static_cast<size_t>(S->n) * Fp * sizeof(double2), s));
    k_sw_copy<<<vec_grid_for(static_cast<int64_t>(S->n) * nfreq), 256, 0, s>>>(
        S->n, nfreq, Fp, static_cast<const double2*>(d_X), ldx, a.x, Fp);
  }
  const bool tq = opts.method == HELM_TFQMR;
  const bool bl = opts.method == HELM_BICGSTABL;
  if (tq) {
    st = sweep_alloc_tfqmr(S, Fp);
    if (st != HELM_OK) return st;
    set_tfqmr_args(S, a);
  }
  if (bl) {
    st = sweep_alloc_bicgstabl(S, Fp, opts.ell, sh.grid);
    if (st != HELM_OK) return st;
    set_bicgstabl_args(S, a, opts.ell);
  }
  // graph for (method, l, F, b, stride)
  helm_sweep_s::G& gr = tq ? S->graphq : bl ? S->graphl : S->graph;
  if (!(gr.exec && gr.F == nfreq && gr.b == bsrc && gr.b_ld == bld && (!bl || S->graphl_ell == opts.ell))) {
    if (gr.exec) {
      cudaGraphExecDestroy(gr.exec);
      cudaGraphDestroy(gr.graph);
    }
    gr = helm_sweep_s::G();
    if (!bcopy) {
      const helm_status gs = tq   ? build_tfqmr_graph(a, sh, &gr.graph, &gr.exec)
                             : bl ? build_bicgstabl_graph(a, sh, &gr.graph, &gr.exec)
                                  : build_sweep_graph(a, sh, &gr.graph, &gr.exec);
      if (gs == HELM_OK) {
        gr.F = nfreq;
        gr.b = bsrc;
        gr.b_ld = bld;
        if (bl) S->graphl_ell = opts.ell;
      }
    }
  }
  // restart flags of the frequencies that run again from their x
  int32_t* d_restart = S->iscal + 3 * static_cast<size_t>(Fp) + Fp / 32;
  std::vector<int32_t> status(Fp), iters(Fp), restart(Fp, 0), restarts(nfreq, 0);
  std::vector<double> relres(Fp), relres_true(Fp);
  for (int32_t fresh = 1, use_x0 = opts.use_x0 ? 1 : 0;; fresh = 0, use_x0 = 1) {
    k_sw_configure<double2><<<1, 256, 0, s>>>(a, opts.tol, opts.maxit, use_x0, opts.deadline_s, fresh, d_restart);
    HELM_CUDA_TRY(cudaGetLastError());
    if (gr.exec && !bcopy) {
      HELM_CUDA_TRY(cudaGraphLaunch(gr.exec, s));
    } else {
      SolverState hs;
      if (tq) swq_init(a, sh, s);
      else if (bl) k_swl_init<<<sh.grid, sh.threads, sh.smem, s>>>(a);
      else k_sw_init<double2><<<sh.grid, sh.threads, sh.smem, s>>>(a);
      for (;;) {
        for (int k = 0; k < 8; ++k) {
          if (tq) swq_body(a, sh, s);
          else if (bl) swl_body(a, sh, s);
          else enqueue_sweep_body(a, sh, s);
        }
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(&hs, a.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs.status != ST_RUNNING) break;
      }
      k_sw_tail<double2><<<sh.grid, sh.threads, sh.smem, s>>>(a);
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(status.data(), a.status, Fp * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(iters.data(), a.iters, Fp * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(relres.data(), a.relres, Fp * sizeof(double), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(
        cudaMemcpyAsync(relres_true.data(), a.relres_true, Fp * sizeof(double), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    // a frequency whose recurrence met tol while its true residual did not
    // restarts from its x (iterations permitting), as the single solve does
    bool any = false;
    for (int j = 0; j < Fp; ++j) {
      // (TFQMR: also a frequency whose bound met tol while its true residual
      // did not, reported as ST_RESTART)
      restart[j] = j < nfreq && ((status[j] == HELM_OK && relres_true[j] > opts.tol && iters[j] < opts.maxit) ||
                                 status[j] == ST_RESTART);
      if (restart[j]) {
        any = true;
        restarts[j] += 1;
      }
    }
    if (!any) break;
    HELM_CUDA_TRY(cudaMemcpyAsync(d_restart, restart.data(), Fp * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  k_sw_copy<<<vec_grid_for(static_cast<int64_t>(S->n) * nfreq), 256, 0, s>>>(S->n, nfreq, Fp, a.x, Fp,
                                                                           static_cast<double2*>(d_X), ldx);
  HELM_CUDA_TRY(cudaGetLastError());
  if (bcopy) cudaFreeAsync(bcopy, s);
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  helm_status worst = HELM_OK;
  for (int j = 0; j < nfreq; ++j) {
    helm_status sj = status[j] < 0 ? HELM_ERR_CUDA : static_cast<helm_status>(status[j]);
    if (sj == HELM_OK && !(relres_true[j] <= opts.tol)) sj = HELM_ERR_NOT_CONVERGED;
    if (h_infos) {
      h_infos[j].iters = iters[j];
      h_infos[j].restarts = restarts[j];
      h_infos[j].relres_recur = relres[j];
      h_infos[j].relres_true = relres_true[j];
      h_infos[j].status = sj;
      h_infos[j].spmv_count = 2 * iters[j] * (bl ? opts.ell : 1);
    }
    if (sj != HELM_OK && worst == HELM_OK) worst = sj;
  }
  return worst;
}

helm_status helm_sweep_spmv(helm_sweep S, int32_t nfreq, const double* h_omega, const void* d_X, int32_t ldx,
                            void* d_Y, int32_t ldy, helm_stream_t stream) {
  if (!S || nfreq < 1 || nfreq > kMaxF || !h_omega || ldx < nfreq || ldy < nfreq) return HELM_ERR_INVALID;
  if (S->n == 0) return HELM_OK;
  if (!d_X || !d_Y || !aligned(d_X, 16) || !aligned(d_Y, 16)) return HELM_ERR_INVALID;
  if (overlaps(d_X, sweep_extent(S->n, ldx, nfreq), d_Y, sweep_extent(S->n, ldy, nfreq))) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(S->mu);
  const int32_t Fp = (nfreq + 31) / 32 * 32;
  if (S->wapply_cap < Fp) {
    cudaFree(S->wapply);
    S->wapply = nullptr;
    S->wapply_cap = 0;
    HELM_CUDA_TRY(cudaMalloc(&S->wapply, Fp * sizeof(double)));
    S->wapply_cap = Fp;
  }
  // the frequencies are copied from a pageable host buffer: the copy is
  // complete when cudaMemcpyAsync returns, so h_omega may be reused at once
  HELM_CUDA_TRY(cudaMemcpyAsync(S->wapply, h_omega, nfreq * sizeof(double), cudaMemcpyHostToDevice, s));
  const SweepDev A{S->n, S->nnz, S->rowptr, S->colind, S->K, S->M, S->B, S->bzero_blk, nullptr, nullptr, nullptr};
  const int G = Fp / 32;
  const int64_t warps = static_cast<int64_t>(S->n) * G;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, static_cast<int64_t>(S->num_sms) * 8)));
  k_sw_apply<<<grid, 256, 0, s>>>(A, nfreq, G, S->wapply, static_cast<const double2*>(d_X), ldx,
                                  static_cast<double2*>(d_Y), ldy);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

}  // extern "C"
