// Mixed-precision solve: one complex64 BiCGStab whose residual is replaced by
// the FP64 true residual b - A x at "reliable updates" (Sleijpen & van der
// Vorst 1996; the defect-correction form of iterative refinement that keeps
// the Krylov recurrence running instead of restarting it at every step).
//
// The paper's library covers single and double precision (Section 1); here
// single precision does the bulk of the work and FP64 decides accuracy:
//   inner (FP32):  BiCGStab on A32 (complex64 copy of the values owned by the
//                  handle, 12 bytes per entry instead of 20), vectors
//                  complex64; products and per-thread sums FP32, block and
//                  grid sums and every recurrence scalar FP64.  The inner
//                  vectors carry the residual divided by sigma (unit RMS
//                  entries at the last update); x32 collects the solution
//                  increment since the last update in the same scale.
//   update (FP64): when the recurrence residual has dropped 10x below its
//                  maximum since the last update (or looks converged, or every
//                  2000 iterations):  x += sigma x32, x32 = 0;  r64 = b - A x
//                  in FP64;  stop if ||r64|| / ||b|| <= tol;  new sigma;
//                  r = complex64(r64 / sigma), p and v rescaled, rho and beta
//                  moved to the replaced residual -- or, when the recurrence
//                  had drifted from r64 by more than a tenth of ||r64||, a
//                  fresh process (r^ = r, p = v = 0) as in restarted
//                  iterative refinement.
// The convergence test is always the FP64 true residual.  The whole solve is
// one graph: init (+ first replacement) -> while(5 FP32 kernels + 3 update
// kernels) -> tail; the update kernels return at once when no update is due.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

namespace {

// restart the complex64 Krylov process when ||r64 - sigma r|| > kRelRestart ||r64||
#ifndef HELM_REL_RESTART
#define HELM_REL_RESTART 0.1
#endif
constexpr double kRelRestart = HELM_REL_RESTART;

constexpr int R128 = Engine<double2>::kThreads;  // threads per SpMV block
constexpr size_t kSmem128 = Engine<double2>::kSmem;

struct RuArgs {
  CsrDev<double2> A;  // FP64 matrix
  const double2* b;
  double2* x;         // FP64 solution (the caller's)
  double2* r64;       // FP64 residual
  float2 *x32, *r32, *rh32, *p32, *v32;
  SolverState* st;    // the inner loop's state
  double* partials;
  unsigned int* tickets;
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

__device__ __forceinline__ void ru_cond(const RuArgs& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// One row of the init: r64 and its partial sums ||b||^2, ||r||^2; zero x32,
// p, v (r and r^ are written by the first replacement, once the scale is known).
struct MxRow {
  const RuArgs* a;
  double part[2];
  double2 bi;
  __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
  __device__ __forceinline__ void put(int32_t i, double2 b_i, double2 ri) {
    a->r64[i] = ri;
    const float2 z = make_float2(0.f, 0.f);
    a->x32[i] = z;
    a->p32[i] = z;
    a->v32[i] = z;
    part[0] = cabs2_acc(b_i, part[0]);
    part[1] = cabs2_acc(ri, part[1]);
  }
  __device__ __forceinline__ void row(int32_t i, double2 ax) { put(i, bi, csub(bi, ax)); }
};

// init: r64 = b - A x (or b, x = 0); asks for the first replacement, which
// starts the complex64 recurrence
__global__ void __launch_bounds__(R128) k_mx_init(RuArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  MxRow rows{&a, {0.0, 0.0}, make_double2(0.0, 0.0)};
  if (use_x0) {
    spmv_run<double2>(a.A, a.x, rows, smem, a.dev_err);
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const double2 bi = a.b[i];
      a.x[i] = make_double2(0.0, 0.0);
      rows.put(i, bi, bi);
    }
  }
  double part[2] = {rows.part[0], rows.part[1]};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_INIT, red, tot)) return;
  if (threadIdx.x != 0) return;
  const double bnorm = sqrt(tot[0]);
  st->bnorm = bnorm;
  if (use_x0) st->spmv_count += 1;
  int status = ST_RUNNING;
  const double rn = sqrt(tot[1]);
  st->relres_true = bnorm > 0.0 ? rn / bnorm : 0.0;
  st->relres = st->relres_true;
  if (!isfinite(bnorm)) {
    status = HELM_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    status = HELM_OK;
  } else if (!isfinite(rn)) {
    status = HELM_ERR_NONFINITE;
  } else if (rn <= st->tol * bnorm) {
    status = HELM_OK;
  } else if (st->maxit <= 0) {
    status = HELM_ERR_NOT_CONVERGED;
  }
  st->method = kModeReliable;
  st->aux[0] = make_double2(rn, 0.0);   // ||r64||, iteration of the last update
  st->aux[1] = make_double2(1.0, 0.0);  // replacement due
  st->aux[2] = make_double2(0.0, 0.0);  // no inner scale yet
  st->status = status;
}

// update 1: x += scale * complex128(x32); x32 = 0
__global__ void __launch_bounds__(256) k_mx_fold(RuArgs a, int always) {
  const SolverState* st = a.st;
  if (!always && st->aux[1].x == 0.0) return;
  const double sc = st->aux[2].x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const float2 d = a.x32[i];
    double2 xi = a.x[i];
    xi.x = fma(sc, static_cast<double>(d.x), xi.x);
    xi.y = fma(sc, static_cast<double>(d.y), xi.y);
    a.x[i] = xi;
    a.x32[i] = make_float2(0.f, 0.f);
  }
}

// update 2: r64 = b - A x (FP64), the convergence test, and the gap between
// it and the complex64 recurrence, ||r64 - sigma r||.  A gap above
// kRelRestart ||r64|| means the recurrence no longer tracks the residual (its
// rounding has grown with the iterates): the Krylov process restarts from r64.
__global__ void __launch_bounds__(R128) k_mx_residual(RuArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  if (st->aux[1].x == 0.0) return;
  struct Epi {
    const RuArgs* a;
    double part[2];
    double sigma;
    double2 bi;
    float2 ri32;
    __device__ __forceinline__ void prefetch(int32_t i) {
      bi = a->b[i];
      ri32 = a->r32[i];
    }
    __device__ __forceinline__ void row(int32_t i, double2 ax) {
      const double2 ri = csub(bi, ax);
      a->r64[i] = ri;
      part[0] = cabs2_acc(ri, part[0]);
      const double2 d = make_double2(fma(-sigma, static_cast<double>(ri32.x), ri.x),
                                     fma(-sigma, static_cast<double>(ri32.y), ri.y));
      part[1] = cabs2_acc(d, part[1]);
    }
  } epi{&a, {0.0, 0.0}, st->aux[2].x, make_double2(0.0, 0.0), make_float2(0.f, 0.f)};
  spmv_run<double2>(a.A, a.x, epi, smem, a.dev_err);
  double part[2] = {epi.part[0], epi.part[1]};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_AUX0, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  st->restarts += 1;  // reliable updates performed
  const double rn = sqrt(tot[0]);
  st->relres_true = rn / st->bnorm;
  if (!isfinite(rn)) st->status = HELM_ERR_NONFINITE;
  else if (rn <= st->tol * st->bnorm) {
    st->status = HELM_OK;
    st->relres = st->relres_true;
  }
  st->aux[0] = make_double2(rn, static_cast<double>(st->iter));
  st->aux[1].y = tot[1] > (kRelRestart * kRelRestart) * tot[0] ? 1.0 : 0.0;  // restart
}

// update 3: the recurrence moves to the replaced residual.  The complex64
// vectors are kept at unit RMS entries, sigma = ||r64|| / sqrt(n): with the
// problem's own scale (entries of b ~ h^3) the squared terms of the inner dots
// fall below the smallest normal float long before FP64 convergence.
//   r = complex64(r64 / sigma);  p, v *= sigma_old / sigma  (r^ = r the first
//   time);  rho = (r^, r);  beta moved to the replaced residual.
// Also the deadline and the loop condition of the iteration.
__global__ void __launch_bounds__(256) k_mx_replace(RuArgs a) {
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  const bool due = st->aux[1].x != 0.0;
  if (!due) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (st->status == ST_RUNNING && st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns)
        st->status = HELM_ERR_TIMEOUT;
      ru_cond(a, st->status == ST_RUNNING);
    }
    return;
  }
  const int32_t n = a.A.n;
  const double s_old = st->aux[2].x;
  // a fresh Krylov process at the start and after a restart: r^ = r, p = v = 0
  const bool first = s_old == 0.0 || st->aux[1].y != 0.0;
  const double s_new = st->aux[0].x / sqrt(static_cast<double>(n));
  const double inv = 1.0 / s_new;
  const float c = first ? 0.f : static_cast<float>(s_old * inv);
  double2 rr = make_double2(0.0, 0.0);
  if (st->status == ST_RUNNING) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 ri = a.r64[i];
      const float2 r32 = make_float2(static_cast<float>(ri.x * inv), static_cast<float>(ri.y * inv));
      a.r32[i] = r32;
      float2 h = r32;
      if (first) {
        a.rh32[i] = r32;
        a.p32[i] = make_float2(0.f, 0.f);
        a.v32[i] = make_float2(0.f, 0.f);
      } else {
        h = a.rh32[i];
        const float2 pi = a.p32[i], vi = a.v32[i];
        a.p32[i] = make_float2(c * pi.x, c * pi.y);
        a.v32[i] = make_float2(c * vi.x, c * vi.y);
      }
      rr = cfma_conj(make_double2(h.x, h.y), make_double2(r32.x, r32.y), rr);
    }
  }
  double part[2] = {rr.x, rr.y};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_AUX1, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->aux[1] = make_double2(0.0, 0.0);
  if (st->status == ST_RUNNING) {
    const double2 rho_true = make_double2(tot[0], tot[1]);
    if (!cfinite(rho_true)) {
      st->status = HELM_ERR_NONFINITE;
    } else if (czero(rho_true)) {
      st->status = HELM_ERR_BREAKDOWN;
    } else {
      // a fresh process's first p update gives p = r whatever beta is;
      // otherwise, with every vector scaled by c,
      // beta = beta rho_true / (c rho_recurrence)
      if (!first) {
        const double cd = static_cast<double>(c);
        st->beta = cdiv_fast(cmul(st->beta, rho_true), make_double2(cd * st->rho.x, cd * st->rho.y));
      }
      st->rho = rho_true;
      st->aux[2].x = s_new;
      st->aux[0].x = st->aux[0].x * inv;  // ||r|| in the inner scale
    }
    if (st->status == ST_RUNNING && st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns)
      st->status = HELM_ERR_TIMEOUT;
  }
  ru_cond(a, st->status == ST_RUNNING);
}

// tail: the FP64 true residual for the report (x32 folded just before)
__global__ void __launch_bounds__(R128) k_mx_tail(RuArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  SolverState* st = a.st;
  const double bnorm = st->bnorm;
  double part[1] = {0.0};
  if (bnorm == 0.0) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x)
      a.x[i] = make_double2(0.0, 0.0);
  } else {
    struct Epi {
      const RuArgs* a;
      double part;
      double2 bi;
      __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, double2 ax) { part = cabs2_acc(csub(bi, ax), part); }
    } epi{&a, 0.0, make_double2(0.0, 0.0)};
    spmv_run<double2>(a.A, a.x, epi, smem, a.dev_err);
    part[0] = epi.part;
  }
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_TAIL, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->relres_true = bnorm == 0.0 ? 0.0 : sqrt(tot[0]) / bnorm;
  if (bnorm != 0.0) st->spmv_count += 1;
}

struct MxShapes {
  KShapes<float2> k;
  int grid128;
  int vec_grid;
};

void mx_init(const RuArgs& a, const MxShapes& sh, cudaStream_t s) {
  k_mx_init<<<sh.grid128, R128, kSmem128, s>>>(a);
  k_mx_replace<<<sh.vec_grid, 256, 0, s>>>(a);
}
void mx_body(const RuArgs& a, const KArgs<float2>& k, const MxShapes& sh, cudaStream_t s) {
  enqueue_body(k, sh.k, s);
  k_mx_fold<<<sh.vec_grid, 256, 0, s>>>(a, 0);
  k_mx_residual<<<sh.grid128, R128, kSmem128, s>>>(a);
  k_mx_replace<<<sh.vec_grid, 256, 0, s>>>(a);
}
void mx_tail(const RuArgs& a, const MxShapes& sh, cudaStream_t s) {
  k_mx_fold<<<sh.vec_grid, 256, 0, s>>>(a, 1);
  k_mx_tail<<<sh.grid128, R128, kSmem128, s>>>(a);
}

}  // namespace

helm_status solve_mixed(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                        cudaStream_t s) {
  helm_status st = ensure_vals32(A, s);
  if (st == HELM_OK) st = ensure_vectors(A, kNumVec);
  if (st == HELM_OK) st = ensure_vectors32(A, 8);
  if (st == HELM_OK) st = prepare_krylov_kernels<float2>();
  if (st != HELM_OK) return st;
  for (const void* fn : {reinterpret_cast<const void*>(&k_mx_init), reinterpret_cast<const void*>(&k_mx_residual),
                         reinterpret_cast<const void*>(&k_mx_tail)})
    HELM_CUDA_TRY(set_smem_attr(fn, kSmem128));
  MxShapes sh;
  st = krylov_shapes<float2>(A, &sh.k);
  if (st != HELM_OK) return st;
  {
    int per_sm = 0;
    HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mx_residual, R128, kSmem128));
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int ntiles = (A->n + Engine<double2>::R - 1) / Engine<double2>::R;
    sh.grid128 = per_sm * A->num_sms;
    if (ntiles < sh.grid128) sh.grid128 = ntiles < 1 ? 1 : ntiles;
    sh.vec_grid = A->vec_grid;
  }
  const int32_t n = A->n;
  const size_t N = static_cast<size_t>(n);
  float2* W = A->vec32;

  KArgs<float2> k;
  std::memset(&k, 0, sizeof(k));
  k.A = CsrDev<float2>{n, A->nnz, A->rowptr, A->colind, A->vals32, nullptr, nullptr};
  k.r = W;
  k.rh = W + N;
  k.p = W + 2 * N;
  k.v = W + 3 * N;
  k.s = W + 4 * N;
  k.t = W + 5 * N;
  k.x = W + 6 * N;  // x32: the increment since the last reliable update
  k.b = W + 7 * N;  // not read by the loop body
  k.st = A->state;
  k.partials = A->partials;
  k.tickets = A->tickets;
  k.dev_err = A->dev_err;

  RuArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = CsrDev<double2>{n, A->nnz, A->rowptr, A->colind, static_cast<const double2*>(A->vals), A->real_blk, A->vals_re};
  a.b = b;
  a.x = x;
  a.r64 = A->vec;
  a.x32 = k.x;
  a.r32 = k.r;
  a.rh32 = k.rh;
  a.p32 = k.p;
  a.v32 = k.v;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.dev_err = A->dev_err;

  // graph per (b, x), tagged as mixed in the cache key
  GraphEntry* g = nullptr;
  auto key = std::make_pair(static_cast<const void*>(reinterpret_cast<const char*>(b) + 2),
                            static_cast<const void*>(x));
  auto it = A->graphs.find(key);
  if (o.launch == HELM_LAUNCH_HOST) {
  } else if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    auto wa = [&](cudaGraphConditionalHandle c) {
      RuArgs r = a;
      r.cond = c;
      r.has_cond = 1;
      return r;
    };
    auto wk = [&](cudaGraphConditionalHandle c) {
      KArgs<float2> kk = k;
      kk.cond = c;
      kk.has_cond = 1;
      return kk;
    };
    GraphEntry e;
    if (build_while_graph([&](cudaGraphConditionalHandle c, cudaStream_t cs) { mx_init(wa(c), sh, cs); },
                          [&](cudaGraphConditionalHandle c, cudaStream_t cs) { mx_body(wa(c), wk(c), sh, cs); },
                          [&](cudaGraphConditionalHandle c, cudaStream_t cs) { mx_tail(wa(c), sh, cs); },
                          &e) == HELM_OK)
      g = &(A->graphs[key] = e);
  }

  // an explicit graph request does not fall back to the host-driven loop
  if (!g && o.launch == HELM_LAUNCH_GRAPH) return HELM_ERR_CUDA;
  k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, o.use_x0 ? 1 : 0, o.deadline_s, 1);
  HELM_CUDA_TRY(cudaGetLastError());
  SolverState* hs = A->state_host;
  if (g) {
    HELM_CUDA_TRY(cudaGraphLaunch(g->exec, s));
  } else {
    mx_init(a, sh, s);
    for (;;) {
      for (int q = 0; q < 8; ++q) mx_body(a, k, sh, s);
      HELM_CUDA_TRY(cudaGetLastError());
      HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaStreamSynchronize(s));
      if (hs->status != ST_RUNNING) break;
    }
    mx_tail(a, sh, s);
  }
  unsigned int herr = 0;
  HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) return HELM_ERR_CUDA;
  helm_status result = hs->status == ST_RUNNING ? HELM_ERR_CUDA : static_cast<helm_status>(hs->status);
  if (result == HELM_OK && !(hs->relres_true <= o.tol)) result = HELM_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hs->iter;
    info->restarts = hs->restarts;  // reliable updates
    info->relres_recur = hs->relres;
    info->relres_true = hs->relres_true;
    info->status = result;
    info->spmv_count = hs->spmv_count;
  }
  return result;
}

}  // namespace helm
