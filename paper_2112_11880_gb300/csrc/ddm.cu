// Schwarz domain decomposition on one GPU with the subdomain solves batched:
// the route the paper's closing remarks (Section 4) give for problems beyond
// one GPU's memory, here with every subdomain on the same GPU.
//
// Subdomains: P contiguous blocks of rows [s_p, e_p) of the matrix's own
// numbering (for a structured box in its natural numbering: slabs of node
// planes), each extended by `overlap` rows on both sides, Omega_p = [a_p, b_p).
// A_p is the principal submatrix of A on Omega_p.  All A_p together form one
// block-diagonal matrix D = diag(A_1, ..., A_P) (its own CSR, built on the
// device, and its own handle), so a single solve of D y = R r is the batch of
// all subdomain solves.
//
// Preconditioner (restricted additive Schwarz, Cai & Sarkis 1999):
//   M r = sum_p Rt_p^T A_p^{-1} R_p r,
// R_p the restriction to Omega_p, Rt_p^T the prolongation that keeps only the
// rows p owns ([s_p, e_p)).  With HELM_DDM_IMPEDANCE every row of Omega_p that
// couples to rows outside it gets i sum_{j outside} |a_ij| added to its
// diagonal: an absorbing (impedance) condition on the artificial boundary, in
// the algebraic form of optimized Schwarz methods (Despres 1991; St-Cyr,
// Gander & Thomas 2007).  With the plain principal submatrices (a Dirichlet
// condition on the artificial boundary) the method stagnates on indefinite
// Helmholtz systems even with exact subdomain solves: measured on the 20^3
// box at 1500 Hz, 4 slabs, GMRES(300) stalls at a residual of 8e-2; with the
// impedance term it reaches 1e-8 in 170-186 steps.
// A_p^{-1} is applied approximately (BiCGStab on D to a relative residual
// inner_tol), so M varies from one application to the next and the outer
// method is flexible: GCR over the last `window` directions (the
// minimal-residual step over them; on these systems a window shorter than the
// steps a solve takes stalls it: the 20^3 box at 1500 Hz, 4 slabs, exact
// subdomain solves, needs 186 steps with every direction kept and 651 with
// the last 64).  The outer loop runs on the host
// (one batched inner solve, one product with A, one projection pass over the
// window and a few dot products per step); convergence is decided on the
// FP64 residual, and HELM_OK needs the recomputed true residual at most tol.
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

constexpr int kDdmMaxWindow = 512;  // GCR directions kept at most
constexpr int kDdmInnerMax = 5000;  // iterations of one batched inner solve at most

// D-row g: global row gmap[g] of subdomain sub[g]; counts of the entries of
// that row whose column lies in the subdomain's extended range.
__global__ void k_ddm_count(int32_t nd, const int32_t* __restrict__ gmap, const int32_t* __restrict__ sub,
                            const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                            const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            int32_t* __restrict__ cnt) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nd; g += gridDim.x * blockDim.x) {
    const int32_t i = gmap[g], p = sub[g];
    const int32_t a = lo[p], b = hi[p];
    int32_t c = 0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t j = colind[k];
      c += (j >= a && j < b) ? 1 : 0;
    }
    cnt[g] = c;
  }
}

// |a| of a complex entry (hypot, no overflow for large parts)
__device__ __forceinline__ double cabs_d(double2 v) { return hypot(v.x, v.y); }

// The block-diagonal CSR: row g keeps the entries of its global row that lie
// in its subdomain, columns shifted to the subdomain's place in D.
// With `impedance`, the diagonal entry gets i sum_{j outside} |a_ij| (the
// coupling the row loses at the artificial boundary, in the CSR order of the
// row); a row without a stored diagonal keeps its entries as they are.
__global__ void k_ddm_fill(int32_t nd, const int32_t* __restrict__ gmap, const int32_t* __restrict__ sub,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const int32_t* __restrict__ doff, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ colind, const double2* __restrict__ vals, int impedance,
                           const int32_t* __restrict__ drow, int32_t* __restrict__ dcol, double2* __restrict__ dval) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nd; g += gridDim.x * blockDim.x) {
    const int32_t i = gmap[g], p = sub[g];
    const int32_t a = lo[p], b = hi[p], shift = doff[p] - a;
    double lost = 0.0;
    if (impedance)
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int32_t j = colind[k];
        if (j < a || j >= b) lost += cabs_d(vals[k]);
      }
    int32_t o = drow[g];
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t j = colind[k];
      if (j >= a && j < b) {
        double2 v = vals[k];
        if (j == i) v.y += lost;
        dcol[o] = j + shift;
        dval[o] = v;
        ++o;
      }
    }
  }
}

// Projections of w on the window: part[blk][j] = block blk's share of
// (C_j, w), j < nwin, C_j = C + j n; two directions per pass over the rows
// (the fixed-order block sum takes four doubles).
__global__ void __launch_bounds__(256) k_ddm_proj(int32_t n, int nwin, int wcap, const double2* __restrict__ C,
                                                  const double2* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[32 * 4];
  for (int j0 = 0; j0 < nwin; j0 += 2) {
    const bool two = j0 + 1 < nwin;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 wi = w[i];
      const double2 d0 = cfma_conj(C[static_cast<size_t>(j0) * n + i], wi, make_double2(acc[0], acc[1]));
      acc[0] = d0.x;
      acc[1] = d0.y;
      if (two) {
        const double2 d1 = cfma_conj(C[static_cast<size_t>(j0 + 1) * n + i], wi, make_double2(acc[2], acc[3]));
        acc[2] = d1.x;
        acc[3] = d1.y;
      }
    }
    block_sum<4>(acc, red);
    if (threadIdx.x == 0) {
      double* o = part + (static_cast<size_t>(blockIdx.x) * wcap + j0) * 2;
      o[0] = acc[0];
      o[1] = acc[1];
      if (two) {
        o[2] = acc[2];
        o[3] = acc[3];
      }
    }
  }
}

// beta[j] = sum of the block partials in block order (thread j)
__global__ void k_ddm_proj_sum(int nblk, int nwin, int wcap, const double* __restrict__ part,
                               double2* __restrict__ beta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nwin) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) {
    acc.x += part[(static_cast<size_t>(b) * wcap + j) * 2];
    acc.y += part[(static_cast<size_t>(b) * wcap + j) * 2 + 1];
  }
  beta[j] = acc;
}

// w -= sum_j beta_j C_j, z -= sum_j beta_j Z_j (classical Gram-Schmidt)
__global__ void __launch_bounds__(256) k_ddm_orth(int32_t n, int nwin, const double2* __restrict__ C,
                                                  const double2* __restrict__ Z, const double2* __restrict__ beta,
                                                  double2* __restrict__ w, double2* __restrict__ z) {
  __shared__ double2 bs[kDdmMaxWindow];
  for (int j = threadIdx.x; j < nwin; j += blockDim.x) bs[j] = beta[j];
  __syncthreads();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 wi = w[i], zi = z[i];
    for (int j = 0; j < nwin; ++j) {
      wi = cfms(bs[j], C[static_cast<size_t>(j) * n + i], wi);
      zi = cfms(bs[j], Z[static_cast<size_t>(j) * n + i], zi);
    }
    w[i] = wi;
    z[i] = zi;
  }
}

// rD[g] = r[gmap[g]]  (R r: every subdomain's extended piece)
__global__ void k_ddm_gather(int32_t nd, const int32_t* __restrict__ gmap, const double2* __restrict__ r,
                             double2* __restrict__ rd) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nd; g += gridDim.x * blockDim.x) rd[g] = r[gmap[g]];
}

// z[gmap[g]] = yD[g] for the rows g owns (each global row is owned once)
__global__ void k_ddm_scatter(int32_t nd, const int32_t* __restrict__ gmap, const uint8_t* __restrict__ owned,
                              const double2* __restrict__ yd, double2* __restrict__ z) {
  for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nd; g += gridDim.x * blockDim.x)
    if (owned[g]) z[gmap[g]] = yd[g];
}

}  // namespace

}  // namespace helm

using namespace helm;

struct helm_ddm_s {
  helm_csr A = nullptr;   // the global matrix (borrowed)
  int32_t n = 0, nsub = 0, overlap = 0, nd = 0;
  int64_t nnzd = 0;
  int32_t* gmap = nullptr;   // [nd] global row of each D-row
  uint8_t* owned = nullptr;  // [nd] 1 where the D-row's subdomain owns that global row
  int32_t* drow = nullptr;   // D's CSR
  int32_t* dcol = nullptr;
  double2* dval = nullptr;
  helm_csr D = nullptr;      // handle of D
  double2* vd = nullptr;     // [2 nd]: R r, y
  int32_t window = 0;        // GCR directions kept
  double2* vn = nullptr;     // [(4 + 2 window) n]: r, z, w, (spare), C_j, Z_j
  double2* dots = nullptr;   // [window + 2] device scalars
  double* part = nullptr;    // [proj_grid][window][2] block partials of the projections
  int proj_grid = 1;
  std::vector<int32_t> lo, hi;  // extended ranges (host)
  std::mutex mu;
};

namespace {

helm_status ddm_fail(helm_ddm S, helm_status st) {
  helm_ddm_destroy(S);
  return st;
}

// z = M r (restricted additive Schwarz with the batched inner solve); returns
// the inner solve's iterations in *iters.
helm_status ddm_apply(helm_ddm S, const double2* r, double2* z, double inner_tol, int32_t* iters,
                      cudaStream_t s) {
  const int grid = vec_grid_for(S->nd);
  double2* rd = S->vd;
  double2* yd = S->vd + S->nd;
  k_ddm_gather<<<grid, 256, 0, s>>>(S->nd, S->gmap, r, rd);
  HELM_CUDA_TRY(cudaGetLastError());
  helm_opts io;
  helm_opts_default(&io);
  io.tol = inner_tol;
  io.maxit = kDdmInnerMax;
  helm_info ii;
  const helm_status st = helm_bicgstab_solve(S->D, rd, yd, &io, &ii, reinterpret_cast<helm_stream_t>(s));
  if (st == HELM_ERR_INVALID || st == HELM_ERR_CUDA || st == HELM_ERR_NOMEM) return st;
  if (iters) *iters = ii.iters;
  // an inner solve that broke down or went non-finite leaves y unusable: the
  // step then falls back to z = r (the outer GCR's step length keeps the
  // residual from growing either way)
  if (ii.status == HELM_ERR_NONFINITE || ii.status == HELM_ERR_BREAKDOWN) {
    HELM_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(double2) * S->n, cudaMemcpyDeviceToDevice, s));
    return HELM_OK;
  }
  k_ddm_scatter<<<grid, 256, 0, s>>>(S->nd, S->gmap, S->owned, yd, z);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

// Host copies of device complex scalars (one synchronisation).
helm_status read_dots(helm_ddm S, int k, double2* out, cudaStream_t s) {
  HELM_CUDA_TRY(cudaMemcpyAsync(out, S->dots, sizeof(double2) * k, cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  return HELM_OK;
}

helm_status norm_of(helm_ddm S, const double2* v, double* out, cudaStream_t s) {
  HELM_TRY(helm_nrm2(S->n, HELM_C128, v, reinterpret_cast<double*>(S->dots), reinterpret_cast<helm_stream_t>(s)));
  double2 d;
  HELM_TRY(read_dots(S, 1, &d, s));
  *out = d.x;
  return HELM_OK;
}

}  // namespace

extern "C" {

helm_status helm_ddm_create(helm_ddm* out, helm_csr A, int32_t nsub, int32_t overlap, int32_t window,
                            uint32_t flags, helm_stream_t stream) {
  if (!out) return HELM_ERR_INVALID;
  *out = nullptr;
  if (!A || A->dt != HELM_C128 || nsub < 1 || overlap < 0 || A->n < 1 || nsub > A->n) return HELM_ERR_INVALID;
  if ((flags & ~HELM_DDM_IMPEDANCE) || window < 1 || window > kDdmMaxWindow) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  helm_ddm S = new (std::nothrow) helm_ddm_s();
  if (!S) return HELM_ERR_NOMEM;
  S->A = A;
  S->n = A->n;
  S->nsub = nsub;
  S->overlap = overlap;
  S->window = window;
  const int32_t n = A->n;
  // owned blocks [s_p, e_p) of near-equal size, extended ranges [a_p, b_p)
  std::vector<int32_t> own_lo(nsub), own_hi(nsub), doff(nsub + 1, 0);
  S->lo.resize(nsub);
  S->hi.resize(nsub);
  for (int p = 0; p < nsub; ++p) {
    own_lo[p] = static_cast<int32_t>(static_cast<int64_t>(p) * n / nsub);
    own_hi[p] = static_cast<int32_t>(static_cast<int64_t>(p + 1) * n / nsub);
    S->lo[p] = std::max<int64_t>(0, static_cast<int64_t>(own_lo[p]) - overlap);
    S->hi[p] = static_cast<int32_t>(std::min<int64_t>(n, static_cast<int64_t>(own_hi[p]) + overlap));
    const int64_t nxt = static_cast<int64_t>(doff[p]) + (S->hi[p] - S->lo[p]);
    if (nxt >= (int64_t(1) << 31)) return ddm_fail(S, HELM_ERR_INVALID);
    doff[p + 1] = static_cast<int32_t>(nxt);
  }
  S->nd = doff[nsub];
  const int32_t nd = S->nd;
  std::vector<int32_t> gmap(nd), sub(nd);
  std::vector<uint8_t> owned(nd);
  for (int p = 0; p < nsub; ++p)
    for (int32_t i = S->lo[p]; i < S->hi[p]; ++i) {
      const int32_t g = doff[p] + (i - S->lo[p]);
      gmap[g] = i;
      sub[g] = p;
      owned[g] = (i >= own_lo[p] && i < own_hi[p]) ? 1 : 0;
    }
  int32_t *d_sub = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_doff = nullptr, *d_cnt = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_sub);
    cudaFree(d_lo);
    cudaFree(d_hi);
    cudaFree(d_doff);
    cudaFree(d_cnt);
  };
  auto fail = [&](helm_status st) {
    cleanup();
    return ddm_fail(S, st);
  };
  if (cudaMalloc(&S->gmap, sizeof(int32_t) * nd) != cudaSuccess || cudaMalloc(&S->owned, nd) != cudaSuccess ||
      cudaMalloc(&d_sub, sizeof(int32_t) * nd) != cudaSuccess || cudaMalloc(&d_lo, sizeof(int32_t) * nsub) != cudaSuccess ||
      cudaMalloc(&d_hi, sizeof(int32_t) * nsub) != cudaSuccess ||
      cudaMalloc(&d_doff, sizeof(int32_t) * nsub) != cudaSuccess || cudaMalloc(&d_cnt, sizeof(int32_t) * nd) != cudaSuccess ||
      cudaMalloc(&S->drow, sizeof(int32_t) * (static_cast<size_t>(nd) + 1)) != cudaSuccess)
    return fail(HELM_ERR_NOMEM);
  cudaError_t e = cudaMemcpyAsync(S->gmap, gmap.data(), sizeof(int32_t) * nd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->owned, owned.data(), nd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_sub, sub.data(), sizeof(int32_t) * nd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_lo, S->lo.data(), sizeof(int32_t) * nsub, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_hi, S->hi.data(), sizeof(int32_t) * nsub, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_doff, doff.data(), sizeof(int32_t) * nsub, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(HELM_ERR_CUDA);
  const int grid = vec_grid_for(nd);
  k_ddm_count<<<grid, 256, 0, s>>>(nd, S->gmap, d_sub, d_lo, d_hi, A->rowptr, A->colind, d_cnt);
  std::vector<int32_t> cnt(nd), drow(static_cast<size_t>(nd) + 1, 0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * nd, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(HELM_ERR_CUDA);
  int64_t acc = 0;
  for (int32_t g = 0; g < nd; ++g) {
    drow[g] = static_cast<int32_t>(acc);
    acc += cnt[g];
    if (acc >= (int64_t(1) << 31)) return fail(HELM_ERR_INVALID);
  }
  drow[nd] = static_cast<int32_t>(acc);
  S->nnzd = acc;
  const size_t NNZ = static_cast<size_t>(std::max<int64_t>(acc, 1));
  if (cudaMalloc(&S->dcol, sizeof(int32_t) * NNZ) != cudaSuccess || cudaMalloc(&S->dval, sizeof(double2) * NNZ) != cudaSuccess)
    return fail(HELM_ERR_NOMEM);
  e = cudaMemcpyAsync(S->drow, drow.data(), sizeof(int32_t) * (static_cast<size_t>(nd) + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_ddm_fill<<<grid, 256, 0, s>>>(nd, S->gmap, d_sub, d_lo, d_hi, d_doff, A->rowptr, A->colind,
                                     static_cast<const double2*>(A->vals), (flags & HELM_DDM_IMPEDANCE) ? 1 : 0,
                                     S->drow, S->dcol, S->dval);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays above are of this frame
  if (e != cudaSuccess) return fail(HELM_ERR_CUDA);
  cleanup();
  d_sub = d_lo = d_hi = d_doff = d_cnt = nullptr;
  helm_status st = helm_csr_create(&S->D, nd, acc, S->drow, S->dcol, S->dval, HELM_C128, 0, stream);
  if (st != HELM_OK) return ddm_fail(S, st);
  if (cudaMalloc(&S->vd, sizeof(double2) * 2 * static_cast<size_t>(nd)) != cudaSuccess ||
      cudaMalloc(&S->vn, sizeof(double2) * (4 + 2 * static_cast<size_t>(window)) * static_cast<size_t>(n)) != cudaSuccess ||
      cudaMalloc(&S->dots, sizeof(double2) * (window + 2)) != cudaSuccess)
    return ddm_fail(S, HELM_ERR_NOMEM);
  S->proj_grid = std::max(1, std::min(vec_grid_for(n), sm_count() * 4));
  if (cudaMalloc(&S->part, sizeof(double) * 2 * window * static_cast<size_t>(S->proj_grid)) != cudaSuccess)
    return ddm_fail(S, HELM_ERR_NOMEM);
  *out = S;
  return HELM_OK;
}

helm_status helm_ddm_destroy(helm_ddm S) {
  if (!S) return HELM_OK;
  cudaDeviceSynchronize();
  if (S->D) helm_csr_destroy(S->D);
  cudaFree(S->gmap);
  cudaFree(S->owned);
  cudaFree(S->drow);
  cudaFree(S->dcol);
  cudaFree(S->dval);
  cudaFree(S->vd);
  cudaFree(S->vn);
  cudaFree(S->dots);
  cudaFree(S->part);
  (void)cudaGetLastError();
  delete S;
  return HELM_OK;
}

helm_status helm_ddm_subdomains(helm_ddm S, int32_t* d_rows, int64_t* d_nnz) {
  if (!S) return HELM_ERR_INVALID;
  if (d_rows) *d_rows = S->nd;
  if (d_nnz) *d_nnz = S->nnzd;
  return HELM_OK;
}

helm_status helm_ddm_apply(helm_ddm S, const void* d_r, void* d_z, double inner_tol, helm_stream_t stream) {
  if (!S || !d_r || !d_z || !aligned(d_r, 16) || !aligned(d_z, 16) || !(inner_tol >= 0.0)) return HELM_ERR_INVALID;
  if (overlaps(d_r, sizeof(double2) * S->n, d_z, sizeof(double2) * S->n)) return HELM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t it = 0;
  HELM_TRY(ddm_apply(S, static_cast<const double2*>(d_r), static_cast<double2*>(d_z), inner_tol, &it, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  return HELM_OK;
}

helm_status helm_ddm_solve(helm_ddm S, const void* d_b, void* d_x, const helm_opts* o, helm_info* info,
                           helm_stream_t stream) {
  helm_opts opts;
  if (o) opts = *o;
  else helm_opts_default(&opts);
  if (info) std::memset(info, 0, sizeof(*info));
  if (!S || !d_b || !d_x || !aligned(d_b, 16) || !aligned(d_x, 16)) return HELM_ERR_INVALID;
  if (overlaps(d_b, sizeof(double2) * S->n, d_x, sizeof(double2) * S->n)) return HELM_ERR_INVALID;
  if (!(opts.tol >= 0.0) || opts.maxit < 0) return HELM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  helm_stream_t hs = stream;
  const int32_t n = S->n;
  const size_t N = static_cast<size_t>(n);
  const double2* b = static_cast<const double2*>(d_b);
  double2* x = static_cast<double2*>(d_x);
  double2* r = S->vn;
  double2* z = S->vn + N;
  double2* w = S->vn + 2 * N;
  const int W = S->window;
  double2* Cb = S->vn + 4 * N;                               // C_j = Cb + j n
  double2* Zb = S->vn + (4 + static_cast<size_t>(W)) * N;  // Z_j = Zb + j n
  const double inner_tol = (opts.inner_tol > 0.0 && opts.inner_tol < 1.0) ? opts.inner_tol : 1e-3;
  const double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0}, mone[2] = {-1.0, 0.0};
  const auto t0 = std::chrono::steady_clock::now();
  int32_t steps = 0, inner_total = 0, spmvs = 0, restarts = 0;
  double bn = 0.0, rn = 0.0, rt = 0.0;
  HELM_TRY(norm_of(S, b, &bn, s));
  auto true_residual = [&](double* out) -> helm_status {  // r = b - A x
    HELM_TRY(helm_spmv(S->A, mone, x, zero, r, hs));
    HELM_TRY(helm_axpby(n, HELM_C128, one, b, one, r, hs));
    ++spmvs;
    return norm_of(S, r, out, s);
  };
  helm_status result = HELM_ERR_NOT_CONVERGED;
  if (!std::isfinite(bn)) {
    result = HELM_ERR_NONFINITE;
  } else if (bn == 0.0) {
    HELM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double2) * N, s));
    result = HELM_OK;
  } else {
    if (opts.use_x0) {
      HELM_TRY(true_residual(&rn));
    } else {
      HELM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double2) * N, s));
      HELM_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
      rn = bn;
    }
    int nwin = 0, next = 0;
    for (;;) {
      if (!std::isfinite(rn)) {
        result = HELM_ERR_NONFINITE;
        break;
      }
      if (rn <= opts.tol * bn) {
        // the recurrence residual met tol: decide on the recomputed one
        HELM_TRY(true_residual(&rt));
        rn = rt;
        if (rt <= opts.tol * bn) {
          result = HELM_OK;
          break;
        }
        ++restarts;  // start the window again from the true residual
        nwin = 0;
        next = 0;
        if (steps >= opts.maxit) break;
        continue;
      }
      if (steps >= opts.maxit) break;
      if (opts.deadline_s > 0.0 &&
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > opts.deadline_s) {
        result = HELM_ERR_TIMEOUT;
        break;
      }
      // z = M r, w = A z
      int32_t it = 0;
      HELM_TRY(ddm_apply(S, r, z, inner_tol, &it, s));
      inner_total += it;
      HELM_TRY(helm_spmv(S->A, one, z, zero, w, hs));
      ++spmvs;
      ++steps;
      // classical Gram-Schmidt of w against the window: beta_j = (C_j, w),
      // w -= sum beta_j C_j, z -= sum beta_j Z_j (one pass each, on the device)
      if (nwin > 0) {
        k_ddm_proj<<<S->proj_grid, 256, 0, s>>>(n, nwin, W, Cb, w, S->part);
        k_ddm_proj_sum<<<(nwin + 127) / 128, 128, 0, s>>>(S->proj_grid, nwin, W, S->part, S->dots);
        k_ddm_orth<<<vec_grid_for(n), 256, 0, s>>>(n, nwin, Cb, Zb, S->dots, w, z);
        HELM_CUDA_TRY(cudaGetLastError());
      }
      double cn = 0.0;
      HELM_TRY(norm_of(S, w, &cn, s));
      if (!(cn > 0.0) || !std::isfinite(cn)) {
        result = std::isfinite(cn) ? HELM_ERR_BREAKDOWN : HELM_ERR_NONFINITE;
        break;
      }
      // new direction C = w / ||w||, Z = z / ||w||; step gamma = (C, r)
      const double inv[2] = {1.0 / cn, 0.0};
      double2* Cn = Cb + static_cast<size_t>(next) * N;
      double2* Zn = Zb + static_cast<size_t>(next) * N;
      HELM_TRY(helm_axpby(n, HELM_C128, inv, w, zero, Cn, hs));
      HELM_TRY(helm_axpby(n, HELM_C128, inv, z, zero, Zn, hs));
      HELM_TRY(helm_dot(n, HELM_C128, Cn, r, 1, S->dots, hs));
      double2 gam;
      HELM_TRY(read_dots(S, 1, &gam, s));
      const double g[2] = {gam.x, gam.y}, mg[2] = {-gam.x, -gam.y};
      HELM_TRY(helm_axpby(n, HELM_C128, g, Zn, one, x, hs));
      HELM_TRY(helm_axpby(n, HELM_C128, mg, Cn, one, r, hs));
      HELM_TRY(norm_of(S, r, &rn, s));
      nwin = std::min(nwin + 1, W);
      next = (next + 1) % W;
    }
    if (result != HELM_OK && result != HELM_ERR_NONFINITE) HELM_TRY(true_residual(&rt));
  }
  if (info) {
    info->iters = steps;
    info->restarts = restarts;
    info->relres_recur = bn > 0.0 ? rn / bn : 0.0;
    info->relres_true = bn > 0.0 ? rt / bn : 0.0;
    info->status = result;
    // products with A, and with the block-diagonal D (two per inner iteration)
    info->spmv_count = spmvs + 2 * inner_total;
  }
  if (result == HELM_OK && bn > 0.0 && !(rt <= opts.tol * bn)) result = HELM_ERR_NOT_CONVERGED;
  return result;
}

}  // extern "C"
