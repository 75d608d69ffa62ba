// Mixed-precision solve: complex64 inner BiCGStab inside complex128
// iterative refinement.
//
// The paper's library covers single and double precision (Section 1); here
// single precision is used where it is safe and FP64 where accuracy is
// decided:
//   outer (FP64):  r = b - A x (complex128 SpMV), ||r|| / ||b||  -- the true
//                  residual, the stopping test;
//   scale:         r32 = complex64(r / ||r||)  (unit-norm right-hand side);
//   inner (FP32):  BiCGStab on A32 d = r32 to inner_tol, A32 = complex64 copy
//                  of the values owned by the handle (12 bytes per entry
//                  instead of 20); products and per-thread sums FP32, block
//                  and grid sums and all recurrence scalars FP64;
//   update (FP64): x += ||r|| * complex128(d).
// The outer loop runs on the host with one synchronisation per refinement
// step; each inner solve is one graph launch with a device-driven loop.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

namespace {

constexpr int R128 = Engine<double2>::kThreads;  // threads per SpMV block
constexpr size_t kSmem128 = Engine<double2>::kSmem;

struct IrArgs {
  CsrDev<double2> A;
  const double2* b;
  double2* x;
  double2* r;
  float2* r32;
  float2* d32;
  SolverState* ost;  // outer state: bnorm, relres (true residual), aux[0].x = ||r||
  double* partials;
  unsigned int* tickets;
  unsigned int* dev_err;
};

// r = b - A x (x = 0 and r = b when `zero_x`), ||r||, ||b||.
__global__ void __launch_bounds__(R128) k_ir_residual(IrArgs a, int zero_x) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  double part[2] = {0.0, 0.0};  // |r|^2, |b|^2
  if (zero_x) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const double2 bi = a.b[i];
      a.x[i] = make_double2(0.0, 0.0);
      a.r[i] = bi;
      part[0] = cabs2_acc(bi, part[0]);
    }
    part[1] = part[0];
  } else {
    struct Epi {
      const IrArgs* a;
      double r2, b2;
      double2 bpre;
      __device__ __forceinline__ void prefetch(int32_t i) { bpre = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, double2 ax) {
        const double2 bi = bpre;
        const double2 ri = csub(bi, ax);
        a->r[i] = ri;
        r2 = cabs2_acc(ri, r2);
        b2 = cabs2_acc(bi, b2);
      }
    } epi{&a, 0.0, 0.0, make_double2(0.0, 0.0)};
    spmv_run<double2>(a.A, a.x, epi, smem, a.dev_err);
    part[0] = epi.r2;
    part[1] = epi.b2;
  }
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_AUX0, red, tot)) return;
  if (threadIdx.x != 0) return;
  SolverState* st = a.ost;
  const double rnorm = sqrt(tot[0]), bnorm = sqrt(tot[1]);
  st->bnorm = bnorm;
  st->aux[0].x = rnorm;
  st->relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  if (!zero_x) st->spmv_count += 1;
}

// r32 = complex64(r / ||r||); d32 = 0
__global__ void __launch_bounds__(256) k_ir_scale(IrArgs a) {
  const double rnorm = a.ost->aux[0].x;
  const double inv = rnorm > 0.0 ? 1.0 / rnorm : 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const double2 ri = a.r[i];
    a.r32[i] = make_float2(static_cast<float>(ri.x * inv), static_cast<float>(ri.y * inv));
  }
}

// x += ||r|| * complex128(d32)
__global__ void __launch_bounds__(256) k_ir_update(IrArgs a) {
  const double rnorm = a.ost->aux[0].x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const float2 d = a.d32[i];
    double2 xi = a.x[i];
    xi.x = fma(rnorm, static_cast<double>(d.x), xi.x);
    xi.y = fma(rnorm, static_cast<double>(d.y), xi.y);
    a.x[i] = xi;
  }
}

struct NoTail {
  void operator()(const KArgs<float2>&, cudaStream_t) const {}
};

}  // namespace

helm_status solve_mixed(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                        cudaStream_t s) {
  helm_status st = ensure_vals32(A, s);
  if (st == HELM_OK) st = ensure_vectors(A, kNumVec);
  if (st == HELM_OK) st = ensure_vectors32(A, 8);
  if (st == HELM_OK) st = prepare_krylov_kernels<float2>();
  if (st != HELM_OK) return st;
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_ir_residual), kSmem128));
  KShapes<float2> sh;
  st = krylov_shapes<float2>(A, &sh);
  if (st != HELM_OK) return st;
  int grid128 = 0;
  {
    int per_sm = 0;
    HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ir_residual, R128, kSmem128));
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int ntiles = (A->n + Engine<double2>::R - 1) / Engine<double2>::R;
    grid128 = per_sm * A->num_sms;
    if (ntiles < grid128) grid128 = ntiles < 1 ? 1 : ntiles;
  }
  const int32_t n = A->n;
  const size_t N = static_cast<size_t>(n);
  float2* W = A->vec32;
  SolverState* inner = A->state;
  SolverState* outer = A->state + 1;

  IrArgs ir;
  std::memset(&ir, 0, sizeof(ir));
  ir.A = CsrDev<double2>{n, A->nnz, A->rowptr, A->colind, static_cast<const double2*>(A->vals), A->real_blk};
  ir.b = b;
  ir.x = x;
  ir.r = A->vec;  // FP64 residual
  ir.r32 = W + 6 * N;
  ir.d32 = W + 7 * N;
  ir.ost = outer;
  ir.partials = A->partials;
  ir.tickets = A->tickets;
  ir.dev_err = A->dev_err;

  KArgs<float2> ka;
  std::memset(&ka, 0, sizeof(ka));
  ka.A = CsrDev<float2>{n, A->nnz, A->rowptr, A->colind, A->vals32, nullptr};
  ka.b = ir.r32;
  ka.x = ir.d32;
  ka.r = W;
  ka.rh = W + N;
  ka.p = W + 2 * N;
  ka.v = W + 3 * N;
  ka.s = W + 4 * N;
  ka.t = W + 5 * N;
  ka.st = inner;
  ka.partials = A->partials;
  ka.tickets = A->tickets;
  ka.dev_err = A->dev_err;

  GraphEntry* g = nullptr;
  auto key = std::make_pair(static_cast<const void*>(ir.r32), static_cast<const void*>(ir.d32));
  auto it = A->graphs.find(key);
  if (o.launch == HELM_LAUNCH_HOST) {
  } else if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    GraphEntry e;
    if (build_krylov_graph<float2>(ka, sh, NoTail{}, &e) == HELM_OK) g = &(A->graphs[key] = e);
  }

  SolverState* hs = A->state_host;  // [0] inner, [1] outer
  unsigned int herr = 0;
  k_ir_residual<<<grid128, R128, kSmem128, s>>>(ir, o.use_x0 ? 0 : 1);
  HELM_CUDA_TRY(cudaGetLastError());
  HELM_CUDA_TRY(cudaMemcpyAsync(hs + 1, outer, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  double relres = hs[1].relres;
  const double bnorm = hs[1].bnorm;
  int32_t total_inner = 0, steps = 0, spmv = hs[1].spmv_count, stalls = 0;
  helm_status result = HELM_ERR_NOT_CONVERGED;
  double last_recur = 0.0;
  if (!std::isfinite(bnorm) || !std::isfinite(relres)) {
    result = HELM_ERR_NONFINITE;
  } else if (bnorm == 0.0 || relres <= o.tol) {
    result = HELM_OK;
  } else {
    while (total_inner < o.maxit) {
      k_ir_scale<<<A->vec_grid, 256, 0, s>>>(ir);
      k_configure<<<1, 1, 0, s>>>(inner, o.inner_tol, o.maxit - total_inner, 0, o.deadline_s, 1);
      HELM_CUDA_TRY(cudaGetLastError());
      st = run_krylov<float2>(A, ka, sh, g, NoTail{}, s);
      if (st != HELM_OK) return st;
      k_ir_update<<<A->vec_grid, 256, 0, s>>>(ir);
      k_ir_residual<<<grid128, R128, kSmem128, s>>>(ir, 0);
      HELM_CUDA_TRY(cudaGetLastError());
      HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, 2 * sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaStreamSynchronize(s));
      if (herr) return HELM_ERR_CUDA;
      steps += 1;
      total_inner += hs[0].iter;
      spmv += hs[0].spmv_count + 1;
      last_recur = hs[0].relres;
      const double prev = relres;
      relres = hs[1].relres;
      if (!std::isfinite(relres)) {
        result = HELM_ERR_NONFINITE;
        break;
      }
      if (relres <= o.tol) {
        result = HELM_OK;
        break;
      }
      if (hs[0].status == HELM_ERR_TIMEOUT) {
        result = HELM_ERR_TIMEOUT;
        break;
      }
      // Refinement must contract: give up after three steps without a 2x gain.
      stalls = (relres > 0.5 * prev) ? stalls + 1 : 0;
      if (stalls >= 3 || hs[0].iter == 0) {
        result = hs[0].status == HELM_ERR_BREAKDOWN ? HELM_ERR_BREAKDOWN : HELM_ERR_NOT_CONVERGED;
        break;
      }
    }
  }
  if (info) {
    info->iters = total_inner;
    info->restarts = steps;
    info->relres_recur = last_recur;
    info->relres_true = relres;
    info->status = result;
    info->spmv_count = spmv;
  }
  return result;
}

}  // namespace helm
