// Complex128 BiCGStab solver (Section 4 of the paper: P-BiCGSTAB, residual
// tolerance, zero initial guess, iteration cap; identity preconditioner).
// The kernels are the precision-generic ones of krylov.cuh instantiated for
// complex128; this file adds the true-residual tail, the persistent
// (cooperative) form of the whole solve, the graph cache and the restart
// rule: a solve reports HELM_OK only when the true residual
// ||b - A x|| / ||b|| recomputed in FP64 is at most tol; when the recurrence
// converged but the true residual did not, the solve restarts from the
// current x while iterations remain.
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

// after the tail: tot = ||b - A x||^2
__device__ __forceinline__ void sc_tail(SolverState* st, const double (&tot)[1]) {
  if (st->bnorm == 0.0) {
    st->relres_true = 0.0;
  } else {
    st->relres_true = sqrt(tot[0]) / st->bnorm;
    st->spmv_count += 1;
  }
}

struct TailEpi {
  const double2* b;
  double part;
  double2 bi;
  __device__ __forceinline__ void prefetch(int32_t i) { bi = b[i]; }
  __device__ __forceinline__ void row(int32_t i, double2 acc) { part = cabs2_acc(csub(bi, acc), part); }
};

// x = 0 on this thread's rows (b = 0)
__device__ __forceinline__ void ph_zero_x(const KArgs<V>& a) {
  for (SliceRows q(a.A.n); q.active(); q.advance()) {
    const int32_t i = q.row();
    if (i < a.A.n) a.x[i] = make_double2(0.0, 0.0);
  }
}

// Tail: ||b - A x|| / ||b|| (x = 0 when b = 0).
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_tail(KArgs<V> a) {
  __shared__ double red[32];
  SolverState* st = a.st;
  double part[1] = {0.0};
  if (st->bnorm == 0.0) {
    ph_zero_x(a);
  } else {
    TailEpi epi{a.b, 0.0, make_double2(0.0, 0.0)};
    spmv_run<V>(a.A, a.x, epi, nullptr, a.dev_err);
    part[0] = epi.part;
  }
  double tot[1];
  if (!grid_total_last<1>(part, a.partials, a.tickets + TK_TAIL, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_tail(st, tot);
}

// ---------------------------------------------------------------- persistent solve

// A grid barrier for a cooperative launch (all blocks resident): arrival
// counter + generation word; thread 0 of each block arrives and waits.  The
// wait is bounded: after kBarrierLimitNs, or once another block has given
// up, the block sets the abort word (and DEVERR_BARRIER_TIMEOUT) and every
// later barrier returns false at once, so the kernel always ends.
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier words at tickets[TK_BAR_COUNT], [TK_BAR_ABORT], [TK_BAR_GEN]; the
// generation a block waits to leave is kept in shared memory (nothing of the
// barrier stays in registers across the phases).  Returns the same answer in
// every thread of the block: false once the barrier has been abandoned.
__device__ __forceinline__ bool grid_sync(unsigned int* tickets, unsigned int* dev_err, unsigned int* s_gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* count = tickets + TK_BAR_COUNT;
    unsigned int* abort = tickets + TK_BAR_ABORT;
    unsigned int* gen = tickets + TK_BAR_GEN;
    const unsigned int g = *s_gen;
    int ok = ld_acquire_u32(abort) == 0u;
    if (ok) {
      __threadfence();
      if (atomicAdd(count, 1u) == gridDim.x - 1) {
        atomicExch(count, 0u);
        __threadfence();
        atomicAdd(gen, 1u);
      } else {
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(gen) == g) {
          if (ld_acquire_u32(abort) != 0u) {
            ok = 0;
            break;
          }
          if (globaltimer_ns() - t0 > kBarrierLimitNs) {
            atomicOr(dev_err, DEVERR_BARRIER_TIMEOUT);
            atomicExch(abort, 1u);
            ok = 0;
            break;
          }
        }
      }
      *s_gen = g + 1;
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Publish this block's K sums, wait for every block, add all blocks' sums in
// the fixed order (every block the same), totals valid in thread 0.
template <int K>
__device__ __forceinline__ bool all_total(double (&v)[K], double* partials, unsigned int* tickets,
                                          unsigned int* dev_err, unsigned int* s_gen, double* red, double (&tot)[K]) {
  block_sum<K>(v, red);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) partials[static_cast<size_t>(blockIdx.x) * K + k] = v[k];
  if (!grid_sync(tickets, dev_err, s_gen)) return false;
  sum_block_partials<K>(partials, gridDim.x, red, tot);
  return true;
}

// The whole solve (init, iterations, tail, restarts) as one cooperative
// kernel on the solver grid.  Every phase does exactly what the graph
// kernels do, on the same rows of the same threads; the totals of each
// reduction are formed in every block from the same partials in the same
// order, and every block runs the scalar step on its own copy of the state,
// so all blocks take every decision together (the deadline is decided by
// block 0 and carried in the last reduction of each iteration).  Two
// partials buffers alternate, so a block may publish the next phase's sums
// while a slower block still reads the previous ones.  The gathered vectors
// (p, s, x) are written by other blocks of the same launch: they are read
// with coherent loads.
// Entries per pipeline stage of the persistent kernel's SpMV phases
// (measured on the 120x60x50 cavity: 149.8 us per iteration with 2, 154.3
// with 4 -- the longer pipeline spills in this kernel).  Gathers go through
// L2 (ld.global.cg): L1-cached loads measured the same speed.
#ifndef HELM_PERSIST_UNROLL
#define HELM_PERSIST_UNROLL 2
#endif
using PGather = GatherCoherent;
constexpr int kPU = HELM_PERSIST_UNROLL;

__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_bicgstab_persistent(KArgs<V> a) {
  __shared__ double red[32 * 4];
  __shared__ SolverState sst;
  __shared__ unsigned int s_gen;
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    sst = *a.st;
    s_gen = ld_acquire_u32(a.tickets + TK_BAR_GEN);
  }
  __syncthreads();
  // partials buffer of the next reduction: two alternate, every thread
  // toggles its own copy of the index (the same in all threads)
  int buf = 0;
#define HELM_TOTAL(K, part, tot)                                                   \
  {                                                                                \
    buf ^= 1;                                                                      \
    double* pb_ = a.partials + static_cast<size_t>(buf) * gridDim.x * 4;           \
    if (!all_total<K>(part, pb_, a.tickets, a.dev_err, &s_gen, red, tot)) return;  \
  }
  for (;;) {  // one pass per (re)start
    // init: r = b - A x or b
    {
      double acc2[2] = {0.0, 0.0};
      double2 d = make_double2(0.0, 0.0);
      const int use_x0 = sst.use_x0;
      if (use_x0) {
        InitEpi<V> epi = init_epi<V>(a);
        spmv_run<V, InitEpi<V>, NoGate, PGather, kPU>(a.A, a.x, epi, nullptr, nullptr);
        acc2[0] = epi.part[0];
        acc2[1] = epi.part[1];
        d = epi.d;
      } else {
        ph_init_zero<V>(a, acc2, d);
      }
      double acc4[4] = {acc2[0], acc2[1], d.x, d.y};
      double tot[4];
      HELM_TOTAL(4, acc4, tot);
      if (threadIdx.x == 0) sc_init(&sst, tot, use_x0);
      __syncthreads();
    }
    while (sst.status == ST_RUNNING) {
      // P1
      ph_p<V>(a, sst.beta, sst.omega);
      if (!grid_sync(a.tickets, a.dev_err, &s_gen)) return;
      // P2
      {
        VEpi<V> epi = v_epi<V>(a);
        spmv_run<V, VEpi<V>, NoGate, PGather, kPU>(a.A, a.p, epi, nullptr, nullptr);
        double part[2] = {epi.part.x, epi.part.y}, tot[2];
        HELM_TOTAL(2, part, tot);
        if (threadIdx.x == 0) sc_after_v(&sst, tot);
        __syncthreads();
        if (sst.status != ST_RUNNING) break;
      }
      // P3
      {
        double part[1] = {ph_s<V>(a, sst.alpha)}, tot[1];
        HELM_TOTAL(1, part, tot);
        if (threadIdx.x == 0) sc_after_s(&sst, tot);
        __syncthreads();
        if (sst.status != ST_RUNNING) break;
      }
      // P4 (not when the solve stopped at s)
      if (sst.phase == PH_RUN) {
        TEpi<V> epi = t_epi<V>(a);
        spmv_run<V, TEpi<V>, NoGate, PGather, kPU>(a.A, a.s, epi, nullptr, nullptr);
        double part[3] = {epi.ts.x, epi.ts.y, epi.tt}, tot[3];
        HELM_TOTAL(3, part, tot);
        if (threadIdx.x == 0) sc_after_t(&sst, tot);
        __syncthreads();
        if (sst.status != ST_RUNNING) break;
      }
      // P5 (+ block 0's deadline decision as a fourth sum)
      {
        double2 rr = make_double2(0.0, 0.0);
        double r2 = 0.0;
        ph_xr<V>(a, sst.alpha, sst.omega, sst.phase == PH_SCONV, rr, r2);
        const double late = (blockIdx.x == 0 && threadIdx.x == 0 && deadline_passed(&sst)) ? 1.0 : 0.0;
        double part[4] = {rr.x, rr.y, r2, late}, tot[4];
        HELM_TOTAL(4, part, tot);
        if (threadIdx.x == 0) {
          const double t3[3] = {tot[0], tot[1], tot[2]};
          sc_after_xr(&sst, t3, tot[3] > 0.0);
        }
        __syncthreads();
      }
    }
    // tail: x is complete once every block is here
    if (!grid_sync(a.tickets, a.dev_err, &s_gen)) return;
    {
      double part[1] = {0.0}, tot[1];
      if (sst.bnorm == 0.0) {
        ph_zero_x(a);
      } else {
        TailEpi epi{a.b, 0.0, make_double2(0.0, 0.0)};
        spmv_run<V, TailEpi, NoGate, PGather, kPU>(a.A, a.x, epi, nullptr, nullptr);
        part[0] = epi.part;
      }
      HELM_TOTAL(1, part, tot);
      if (threadIdx.x == 0) {
        sc_tail(&sst, tot);
        // restart from x when the recurrence converged but the true residual
        // did not, while iterations remain (as the host does for the graph)
        s_go = sst.status == HELM_OK && sst.relres_true > sst.tol && sst.iter < sst.maxit;
        if (s_go) {
          sst.restarts += 1;
          sst.use_x0 = 1;
          sst.status = ST_RUNNING;
          sst.phase = PH_RUN;
          sst.relres = 0.0;
          sst.relres_true = 0.0;
          const double2 one = make_double2(1.0, 0.0);
          sst.rho = one;
          sst.alpha = one;
          sst.omega = one;
          sst.beta = make_double2(0.0, 0.0);
        }
      }
      __syncthreads();
      if (!s_go) break;
    }
  }
#undef HELM_TOTAL
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.st = sst;
}

}  // namespace

helm_status bicgstab_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                          cudaStream_t s) {
  helm_status st = ensure_vectors(A, kNumVec);
  if (st != HELM_OK) return st;
  KShapes<V> sh;
  st = krylov_shapes<V>(A, &sh, {reinterpret_cast<const void*>(&k_tail),
                                 reinterpret_cast<const void*>(&k_bicgstab_persistent)});
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
  HELM_CUDA_TRY(cudaMemsetAsync(A->dev_err, 0, sizeof(unsigned int), s));
  const int32_t use_x0_first = o.use_x0 ? 1 : 0;
  SolverState* hs = A->state_host;
  unsigned int herr = 0;

  // persistent: the whole solve, restarts included, is one cooperative launch
  // (on request; HELM_LAUNCH_AUTO takes the graph, measured faster)
  bool done = false;
  if (o.launch == HELM_LAUNCH_PERSISTENT) {
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, A->device) == cudaSuccess && coop) {
      k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0_first, o.deadline_s, 1);
      HELM_CUDA_TRY(cudaGetLastError());
      HELM_CUDA_TRY(cudaMemsetAsync(A->tickets + TK_BAR_COUNT, 0, 2 * sizeof(unsigned int), s));  // count, abort
      void* args[] = {&a};
      const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_bicgstab_persistent),
                                                        dim3(sh.grid), dim3(sh.threads), args, 0, s);
      if (e != cudaSuccess) {
        debug_cuda_error(e, __FILE__, __LINE__);
        (void)cudaGetLastError();
        return HELM_ERR_CUDA;
      }
      done = true;
    } else {
      return HELM_ERR_CUDA;
    }
    if (done) {
      HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaStreamSynchronize(s));
      if (herr) return HELM_ERR_CUDA;
    }
  }

  if (!done) {
    struct Tail {
      int grid, threads;
      void operator()(const KArgs<V>& ka, cudaStream_t ss) const { k_tail<<<grid, threads, 0, ss>>>(ka); }
    } tail{sh.grid, sh.threads};
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
    int32_t use_x0 = use_x0_first;
    int32_t fresh = 1;
    for (;;) {
      k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0, o.deadline_s, fresh);
      HELM_CUDA_TRY(cudaGetLastError());
      st = run_krylov<V>(A, a, sh, g, tail, s);
      if (st != HELM_OK) return st;
      HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
      HELM_CUDA_TRY(cudaStreamSynchronize(s));
      if (herr) return HELM_ERR_CUDA;
      if (hs->status == HELM_OK && hs->relres_true > o.tol && hs->iter < o.maxit) {
        use_x0 = 1;
        fresh = 0;
        continue;
      }
      break;
    }
  }
  helm_status result = hs->status == ST_RUNNING ? HELM_ERR_CUDA : static_cast<helm_status>(hs->status);
  if (result == HELM_OK && !(hs->relres_true <= o.tol)) result = HELM_ERR_NOT_CONVERGED;
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
