// Complex128 BiCGStab with device-resident scalars (Section 4 of the paper:
// P-BiCGSTAB with residual tolerance, zero initial guess and an iteration
// cap; identity preconditioner; the recurrence of van der Vorst 1992 /
// Saad 2003 Algorithm 7.7 with conjugated inner products).
//
// One iteration is five kernels; each dot product the recurrence needs is
// fused into the kernel that produces its operands, and the scalar it feeds
// is formed on the device by the last block to finish (ticket counter):
//   K1  p = r + beta (p - omega v)
//   K2  v = A p          + (r^, v)      -> alpha = rho / (r^, v)
//   K3  s = r - alpha v  + ||s||^2      -> stop at s if ||s|| / ||b|| <= tol
//   K4  t = A s          + (t, s), ||t||^2 -> omega = (t, s) / (t, t)
//   K5  x += alpha p + omega s, r = s - omega t + (r^, r), ||r||^2
//                                       -> stop test, rho, beta
// The loop runs inside one CUDA graph: an init kernel, a conditional WHILE
// node whose body is K1..K5 (K5's last block sets the condition), and a tail
// kernel that recomputes the true residual b - A x.  The host launches the
// graph and reads the final state once.  If the true residual is above
// 1.5 tol while iterations remain, the solve restarts from the current x.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.hpp"
#include "spmv.cuh"

namespace helm {

namespace {

constexpr int R = kRows128;
constexpr int CAP = kCap128;
using Stage = SpmvStage<double2, CAP>;

struct BicgArgs {
  CsrDev<double2> A;
  const double2* b;
  double2* x;
  double2 *r, *rh, *p, *v, *s, *t;
  SolverState* st;
  double* partials;
  unsigned int* tickets;
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

__device__ __forceinline__ void set_cond(const BicgArgs& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

__device__ __forceinline__ bool deadline_passed(const SolverState* st) {
  return st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns;
}

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

// r = b - A x (or r = b, x = 0), r^ = r, p = v = 0; ||b||, ||r||, rho.
__global__ void __launch_bounds__(R) k_init(BicgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  double part[4] = {0.0, 0.0, 0.0, 0.0};  // |b|^2, |r|^2, (r, r)
  const double2 zero = make_double2(0.0, 0.0);
  if (use_x0) {
    struct Epi {
      const BicgArgs* a;
      double part[4];
      __device__ __forceinline__ void row(int32_t i, double2 acc) {
        const double2 bi = a->b[i];
        const double2 ri = csub(bi, acc);
        a->r[i] = ri;
        a->rh[i] = ri;
        a->p[i] = make_double2(0.0, 0.0);
        a->v[i] = make_double2(0.0, 0.0);
        part[0] = cabs2_acc(bi, part[0]);
        part[1] = cabs2_acc(ri, part[1]);
        double2 d = cfma_conj(ri, ri, make_double2(part[2], part[3]));
        part[2] = d.x;
        part[3] = d.y;
      }
    } epi{&a, {0.0, 0.0, 0.0, 0.0}};
    spmv_tiles<double2, R, CAP>(a.A, a.x, epi, smem, a.dev_err);
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k] = epi.part[k];
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const double2 bi = a.b[i];
      a.x[i] = zero;
      a.r[i] = bi;
      a.rh[i] = bi;
      a.p[i] = zero;
      a.v[i] = zero;
      part[0] = cabs2_acc(bi, part[0]);
      double2 d = cfma_conj(bi, bi, make_double2(part[2], part[3]));
      part[2] = d.x;
      part[3] = d.y;
    }
    part[1] = part[0];
  }
  double tot[4];
  if (!grid_sum_last<4>(part, a.partials, a.tickets + TK_INIT, red, tot)) return;
  if (threadIdx.x != 0) return;
  const double bnorm = sqrt(tot[0]);
  st->bnorm = bnorm;
  if (use_x0) st->spmv_count += 1;
  int status = ST_RUNNING;
  if (!isfinite(bnorm)) {
    status = HELM_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    status = HELM_OK;  // b = 0: x = 0 (the tail kernel writes it)
    st->relres = 0.0;
  } else {
    const double relres = sqrt(tot[1]) / bnorm;
    st->relres = relres;
    const double2 rho = make_double2(tot[2], tot[3]);
    if (!isfinite(relres)) {
      status = HELM_ERR_NONFINITE;
    } else if (relres <= st->tol) {
      status = HELM_OK;
    } else if (st->iter >= st->maxit) {
      status = HELM_ERR_NOT_CONVERGED;
    } else if (!cfinite(rho)) {
      status = HELM_ERR_NONFINITE;
      st->iter += 1;
    } else if (czero(rho)) {
      status = HELM_ERR_BREAKDOWN;
      st->iter += 1;
    } else {
      // beta = (rho / 1) (1 / 1): the first p update gives p = r
      st->rho = rho;
      st->beta = rho;
    }
  }
  st->status = status;
  set_cond(a, status == ST_RUNNING);
}

// K1: p = r + beta (p - omega v)
__global__ void __launch_bounds__(256) k_p(BicgArgs a) {
  const SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const double2 beta = st->beta, omega = st->omega;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    a.p[i] = cfma(beta, cfms(omega, a.v[i], a.p[i]), a.r[i]);
  }
}

// K2: v = A p, (r^, v) -> alpha
__global__ void __launch_bounds__(R) k_v(BicgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  struct Epi {
    const BicgArgs* a;
    double part[2];
    __device__ __forceinline__ void row(int32_t i, double2 acc) {
      a->v[i] = acc;
      double2 d = cfma_conj(a->rh[i], acc, make_double2(part[0], part[1]));
      part[0] = d.x;
      part[1] = d.y;
    }
  } epi{&a, {0.0, 0.0}};
  spmv_tiles<double2, R, CAP>(a.A, a.p, epi, smem, a.dev_err);
  double part[2] = {epi.part[0], epi.part[1]};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_V, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->iter += 1;
  st->spmv_count += 1;
  const double2 rv = make_double2(tot[0], tot[1]);
  if (!cfinite(rv)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (czero(rv)) {
    st->status = HELM_ERR_BREAKDOWN;
  } else {
    const double2 alpha = cdiv(st->rho, rv);
    if (!cfinite(alpha)) st->status = HELM_ERR_NONFINITE;
    else st->alpha = alpha;
  }
}

// K3: s = r - alpha v, ||s||
__global__ void __launch_bounds__(256) k_s(BicgArgs a) {
  __shared__ double red[32];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const double2 alpha = st->alpha;
  double part[1] = {0.0};
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const double2 si = cfms(alpha, a.v[i], a.r[i]);
    a.s[i] = si;
    part[0] = cabs2_acc(si, part[0]);
  }
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_S, red, tot)) return;
  if (threadIdx.x != 0) return;
  const double snorm = sqrt(tot[0]);
  if (!isfinite(snorm)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (snorm / st->bnorm <= st->tol) {
    st->phase = PH_SCONV;
    st->relres = snorm / st->bnorm;
  }
}

// K4: t = A s, (t, s), (t, t) -> omega
__global__ void __launch_bounds__(R) k_t(BicgArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING || st->phase != PH_RUN) return;
  struct Epi {
    const BicgArgs* a;
    double part[3];
    __device__ __forceinline__ void row(int32_t i, double2 acc) {
      a->t[i] = acc;
      double2 d = cfma_conj(acc, a->s[i], make_double2(part[0], part[1]));
      part[0] = d.x;
      part[1] = d.y;
      part[2] = cabs2_acc(acc, part[2]);
    }
  } epi{&a, {0.0, 0.0, 0.0}};
  spmv_tiles<double2, R, CAP>(a.A, a.s, epi, smem, a.dev_err);
  double part[3] = {epi.part[0], epi.part[1], epi.part[2]};
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_T, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double2 ts = make_double2(tot[0], tot[1]);
  const double tt = tot[2];
  if (!cfinite(ts) || !isfinite(tt)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (tt == 0.0) {
    st->status = HELM_ERR_BREAKDOWN;
  } else {
    const double2 omega = make_double2(ts.x / tt, ts.y / tt);
    if (!cfinite(omega)) st->status = HELM_ERR_NONFINITE;
    else st->omega = omega;
  }
}

// K5: x += alpha p + omega s, r = s - omega t; stop test; rho, beta
__global__ void __launch_bounds__(256) k_xr(BicgArgs a) {
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  const int status0 = st->status;
  if (status0 != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, false);
    return;
  }
  const double2 alpha = st->alpha, omega = st->omega;
  const int phase = st->phase;
  double part[3] = {0.0, 0.0, 0.0};
  if (phase == PH_SCONV) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x)
      a.x[i] = cfma(alpha, a.p[i], a.x[i]);
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const double2 si = a.s[i];
      a.x[i] = cfma(omega, si, cfma(alpha, a.p[i], a.x[i]));
      const double2 ri = cfms(omega, a.t[i], si);
      a.r[i] = ri;
      double2 d = cfma_conj(a.rh[i], ri, make_double2(part[0], part[1]));
      part[0] = d.x;
      part[1] = d.y;
      part[2] = cabs2_acc(ri, part[2]);
    }
  }
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_XR, red, tot)) return;
  if (threadIdx.x != 0) return;
  int status = ST_RUNNING;
  if (phase == PH_SCONV) {
    status = HELM_OK;
    st->phase = PH_DONE;
  } else {
    const double relres = sqrt(tot[2]) / st->bnorm;
    st->relres = relres;
    if (!isfinite(relres)) {
      status = HELM_ERR_NONFINITE;
    } else if (relres <= st->tol) {
      status = HELM_OK;
    } else if (czero(omega)) {
      status = HELM_ERR_BREAKDOWN;
    } else if (st->iter >= st->maxit) {
      status = HELM_ERR_NOT_CONVERGED;
    } else if (deadline_passed(st)) {
      status = HELM_ERR_TIMEOUT;
    } else {
      const double2 rho_new = make_double2(tot[0], tot[1]);
      const double2 beta = cmul(cdiv(rho_new, st->rho), cdiv(alpha, omega));
      if (!cfinite(rho_new) || !cfinite(beta)) {
        status = HELM_ERR_NONFINITE;
        st->iter += 1;
      } else if (czero(rho_new)) {
        status = HELM_ERR_BREAKDOWN;
        st->iter += 1;
      } else {
        st->rho = rho_new;
        st->beta = beta;
      }
    }
  }
  st->status = status;
  set_cond(a, status == ST_RUNNING);
}

// Tail: ||b - A x|| / ||b|| (x = 0 when b = 0).
__global__ void __launch_bounds__(R) k_tail(BicgArgs a) {
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
      const BicgArgs* a;
      double part[1];
      __device__ __forceinline__ void row(int32_t i, double2 acc) {
        part[0] = cabs2_acc(csub(a->b[i], acc), part[0]);
      }
    } epi{&a, {0.0}};
    spmv_tiles<double2, R, CAP>(a.A, a.x, epi, smem, a.dev_err);
    part[0] = epi.part[0];
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

struct Shapes {
  int spmv_grid, vec_grid;
};

void enqueue_init(const BicgArgs& a, const Shapes& sh, cudaStream_t s) {
  k_init<<<sh.spmv_grid, R, Stage::kBytes, s>>>(a);
}
void enqueue_body(const BicgArgs& a, const Shapes& sh, cudaStream_t s) {
  k_p<<<sh.vec_grid, 256, 0, s>>>(a);
  k_v<<<sh.spmv_grid, R, Stage::kBytes, s>>>(a);
  k_s<<<sh.vec_grid, 256, 0, s>>>(a);
  k_t<<<sh.spmv_grid, R, Stage::kBytes, s>>>(a);
  k_xr<<<sh.vec_grid, 256, 0, s>>>(a);
}
void enqueue_tail(const BicgArgs& a, const Shapes& sh, cudaStream_t s) {
  k_tail<<<sh.spmv_grid, R, Stage::kBytes, s>>>(a);
}

helm_status prepare_kernels() {
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_init), Stage::kBytes));
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_v), Stage::kBytes));
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_t), Stage::kBytes));
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_tail), Stage::kBytes));
  return HELM_OK;
}

// Build the graph init -> while(body) -> tail for fixed (b, x).
helm_status build_graph(const BicgArgs& base, const Shapes& sh, GraphEntry* out) {
  cudaStream_t cs = nullptr;
  HELM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  helm_status result = HELM_ERR_CUDA;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess) break;
    BicgArgs a = base;
    a.cond = cond;
    a.has_cond = 1;
    // init
    if (cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    enqueue_init(a, sh, cs);
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
    cudaGraphNode_t init_node = (e == cudaSuccess && ndeps == 1) ? deps[0] : nullptr;
    cudaGraph_t tmp = nullptr;
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess || e != cudaSuccess || !init_node) break;
    // while node
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, graph, &init_node, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    enqueue_body(a, sh, cs);
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) break;
    // tail
    if (cudaStreamBeginCaptureToGraph(cs, graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    enqueue_tail(a, sh, cs);
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
  out->exec = exec;
  out->graph = graph;
  return HELM_OK;
}

}  // namespace

helm_status bicgstab_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                          cudaStream_t s) {
  helm_status st = ensure_vectors(A, 6);
  if (st != HELM_OK) return st;
  st = prepare_kernels();
  if (st != HELM_OK) return st;
  const int32_t n = A->n;
  double2* V = A->vec;
  BicgArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = CsrDev<double2>{n, A->nnz, A->rowptr, A->colind, static_cast<const double2*>(A->vals)};
  a.b = b;
  a.x = x;
  a.r = V;
  a.rh = V + (size_t)n;
  a.p = V + 2 * (size_t)n;
  a.v = V + 3 * (size_t)n;
  a.s = V + 4 * (size_t)n;
  a.t = V + 5 * (size_t)n;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.dev_err = A->dev_err;
  Shapes sh{A->spmv_grid, A->vec_grid};

  // Graph for this (b, x), built once and reused.
  GraphEntry* g = nullptr;
  auto key = std::make_pair(static_cast<const void*>(b), static_cast<const void*>(x));
  auto it = A->graphs.find(key);
  if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    GraphEntry e;
    if (build_graph(a, sh, &e) == HELM_OK) {
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

  int32_t use_x0 = o.use_x0 ? 1 : 0;
  int32_t fresh = 1;
  SolverState* hs = A->state_host;
  unsigned int herr = 0;
  for (;;) {
    k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0, o.deadline_s, fresh);
    HELM_CUDA_TRY(cudaGetLastError());
    if (g) {
      HELM_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    } else {
      // Host-driven fallback: enqueue chunks of iterations and poll the state.
      enqueue_init(a, sh, s);
      HELM_CUDA_TRY(cudaGetLastError());
      for (;;) {
        for (int k = 0; k < 16; ++k) enqueue_body(a, sh, s);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs->status != ST_RUNNING) break;
      }
      enqueue_tail(a, sh, s);
    }
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
