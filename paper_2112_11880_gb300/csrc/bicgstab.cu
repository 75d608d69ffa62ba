// Complex128 BiCGStab solver (Section 4 of the paper: P-BiCGSTAB, residual
// tolerance, zero initial guess, iteration cap; identity preconditioner).
// The kernels are the precision-generic ones of krylov.cuh instantiated for
// complex128; this file adds the true-residual tail, the graph cache and the
// restart rule: if the true residual ||b - A x|| / ||b|| exceeds 1.5 tol while
// iterations remain, the solve restarts from the current x.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

__global__ void k_configure(SolverState* st, double tol, int32_t maxit, int32_t use_x0, double deadline_s,
                            int32_t fresh) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (fresh) {
    st->iter = 0;
    st->spmv_count = 0;
    st->restarts = 0;
    st->t0 = globaltimer_ns();
  } else {
    st->restarts += 1;
  }
  st->tol = tol;
  st->maxit = maxit;
  st->use_x0 = use_x0;
  st->method = kModePlain;
  st->deadline_ns = deadline_s > 0.0 ? static_cast<unsigned long long>(deadline_s * 1e9) : 0ull;
  st->status = ST_RUNNING;
  st->phase = PH_RUN;
  st->relres = 0.0;
  st->relres_true = 0.0;
  const double2 one = make_double2(1.0, 0.0);
  st->rho = one;
  st->alpha = one;
  st->omega = one;
  st->beta = make_double2(0.0, 0.0);
}

namespace {

using V = double2;
constexpr int R = Engine<V>::kThreads;  // threads per SpMV block
constexpr size_t kSmem = Engine<V>::kSmem;

// Tail: ||b - A x|| / ||b|| (x = 0 when b = 0).
__global__ void __launch_bounds__(R) k_tail(KArgs<V> a) {
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
      const KArgs<V>* a;
      double part;
      double2 bi;
      __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, double2 acc) { part = cabs2_acc(csub(bi, acc), part); }
    } epi{&a, 0.0, make_double2(0.0, 0.0)};
    spmv_run<V>(a.A, a.x, epi, smem, a.dev_err);
    part[0] = epi.part;
  }
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_TAIL, red, tot)) return;
  if (threadIdx.x != 0) return;
  if (bnorm == 0.0) {
    st->relres_true = 0.0;
  } else {
    st->relres_true = sqrt(tot[0]) / bnorm;
    st->spmv_count += 1;
  }
}

struct TailFp64 {
  int grid;
  void operator()(const KArgs<V>& a, cudaStream_t s) const { k_tail<<<grid, R, kSmem, s>>>(a); }
};

}  // namespace

helm_status bicgstab_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                          cudaStream_t s) {
  helm_status st = ensure_vectors(A, kNumVec);
  if (st != HELM_OK) return st;
  st = prepare_krylov_kernels<V>();
  if (st != HELM_OK) return st;
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_tail), kSmem));
  KShapes<V> sh;
  st = krylov_shapes<V>(A, &sh);
  if (st != HELM_OK) return st;
  const int32_t n = A->n;
  double2* W = A->vec;
  KArgs<V> a;
  std::memset(&a, 0, sizeof(a));
  a.A = csr_for(A, o);
  a.b = b;
  a.x = x;
  a.r = W;
  a.rh = W + (size_t)n;
  a.p = W + 2 * (size_t)n;
  a.v = W + 3 * (size_t)n;
  a.s = W + 4 * (size_t)n;
  a.t = W + 5 * (size_t)n;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.gtickets = A->gtickets;
  a.dev_err = A->dev_err;
  TailFp64 tail{0};
  HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_tail)}, R, kSmem, A->num_sms,
                           (static_cast<int64_t>(n) + Engine<V>::R - 1) / Engine<V>::R, &tail.grid));

  // Graph for this (b, x), built once and reused.
  GraphEntry* g = nullptr;
  const bool use_graph = o.launch != HELM_LAUNCH_HOST;
  auto key = graph_key(b, x, 0, o);
  auto it = A->graphs.find(key);
  if (!use_graph) {
  } else if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    GraphEntry e;
    if (build_krylov_graph<V>(a, sh, tail, &e) == HELM_OK) {
      if (A->graphs.size() >= 16) {  // bound the cache
        for (auto& kv : A->graphs) {
          cudaGraphExecDestroy(kv.second.exec);
          cudaGraphDestroy(kv.second.graph);
        }
        A->graphs.clear();
      }
      g = &(A->graphs[key] = e);
    }
  }
  // an explicit graph request does not fall back to the host-driven loop
  if (!g && o.launch == HELM_LAUNCH_GRAPH) return HELM_ERR_CUDA;

  int32_t use_x0 = o.use_x0 ? 1 : 0;
  int32_t fresh = 1;
  SolverState* hs = A->state_host;
  unsigned int herr = 0;
  for (;;) {
    k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0, o.deadline_s, fresh);
    HELM_CUDA_TRY(cudaGetLastError());
    st = run_krylov<V>(A, a, sh, g, tail, s);
    if (st != HELM_OK) return st;
    HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) return HELM_ERR_CUDA;
    if (hs->status == HELM_OK && hs->relres_true > 1.5 * o.tol && hs->iter < o.maxit) {
      use_x0 = 1;
      fresh = 0;
      continue;
    }
    break;
  }
  helm_status result = hs->status == ST_RUNNING ? HELM_ERR_CUDA : static_cast<helm_status>(hs->status);
  if (result == HELM_OK && !(hs->relres_true <= 1.5 * o.tol)) result = HELM_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hs->iter;
    info->restarts = hs->restarts;
    info->relres_recur = hs->relres;
    info->relres_true = hs->relres_true;
    info->status = result;
    info->spmv_count = hs->spmv_count;
  }
  return result;
}

}  // namespace helm
