// Complex128 TFQMR with device-resident scalars: the "P-TFQMR" of Section 4
// (identity preconditioner), following Freund 1993 / Saad 2003 Algorithm 7.8
// with conjugated inner products (r0, y) = sum conj(r0_i) y_i.
//
// One iteration = two half-steps = two products with A, six kernels:
//   T1  un = u - alpha v, w -= alpha Au, d = u + gamma d   + ||w||^2
//         -> theta, c, tau, eta (even half-step), quasi-residual bound
//   T2  Aun = A un;  x += eta d                (the even half-step's x update)
//   T3  w -= alpha Aun, d = un + gamma d       + ||w||^2, (r0, w)
//         -> theta, c, tau, eta (odd half-step), rho, beta
//   T4  u = w + beta un;  x += eta d
//   T5  Au = A u;  v = Au + beta (Aun + beta v) + (r0, v) -> alpha, gamma
//   T6  when a half-step's bound tau sqrt(m + 2) fell below tol ||b||: true
//       residual ||b - A x|| (one SpMV), convergence; iteration cap, deadline;
//       the loop condition.
// The true-residual check runs once per iteration, after the odd half-step,
// so a solve can end one half-step later than a check after every half-step.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

namespace {

using V = double2;
constexpr int RT = Engine<V>::kThreads;  // threads per SpMV block
constexpr size_t kSmem = Engine<V>::kSmem;

struct TqArgs {
  CsrDev<V> A;
  const V* b;
  V* x;
  V *r0, *w, *u, *un, *v, *Au, *Aun, *d;
  SolverState* st;  // rho, alpha, beta; aux[0] = eta, aux[1] = (theta, tau), aux[2] = gamma, aux[3] = (check, start iteration)
  double* partials;
  unsigned int* tickets;
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

__device__ __forceinline__ void tq_cond(const TqArgs& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// After a half-step: theta = ||w|| / tau, c = 1/sqrt(1 + theta^2),
// tau = tau theta c, eta = c^2 alpha; the bound tau sqrt(m + 2) <= tol ||b||
// (m = half-step index) raises the check flag.
__device__ void tq_half_step_scalars(SolverState* st, double ww, int m) {
  const double tau0 = st->aux[1].y;
  const double theta = sqrt(ww) / tau0;
  const double c = 1.0 / sqrt(1.0 + theta * theta);
  const double tau = tau0 * theta * c;
  const double2 alpha = st->alpha;
  const double2 eta = make_double2(c * c * alpha.x, c * c * alpha.y);
  if (!isfinite(theta) || !isfinite(tau) || !cfinite(eta)) {
    st->status = HELM_ERR_NONFINITE;
    return;
  }
  st->aux[1] = make_double2(theta, tau);
  st->aux[0] = eta;
  const double bt = st->tol * st->bnorm;
  if (tau * tau * static_cast<double>(m + 2) <= bt * bt) st->aux[3].x = 1.0;
  st->relres = tau * sqrt(static_cast<double>(m + 2)) / st->bnorm;
}

// gamma = (theta^2 / alpha) eta for the next d update
__device__ __forceinline__ void tq_gamma(SolverState* st) {
  const double th = st->aux[1].x;
  const double2 q = cdiv_fast(make_double2(th * th, 0.0), st->alpha);
  st->aux[2] = cmul(q, st->aux[0]);
}

// init A: r0 = b - A x (or b, x = 0); w = u = r0; d = 0; ||b||, ||r0||, rho = (r0, r0)
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_init_a(TqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  const V zero = make_double2(0.0, 0.0);
  auto put = [&](int32_t i, V bi, V ri) {
    a.r0[i] = ri;
    a.w[i] = ri;
    a.u[i] = ri;
    a.d[i] = zero;
    part[0] = cabs2_acc(bi, part[0]);
    part[1] = cabs2_acc(ri, part[1]);
    const V q = cfma_conj(ri, ri, make_double2(part[2], part[3]));
    part[2] = q.x;
    part[3] = q.y;
  };
  if (use_x0) {
    struct Epi {
      const TqArgs* a;
      double p[4];
      V bi;
      __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, V ax) {
        const V ri = csub(bi, ax);
        a->r0[i] = ri;
        a->w[i] = ri;
        a->u[i] = ri;
        a->d[i] = make_double2(0.0, 0.0);
        p[0] = cabs2_acc(bi, p[0]);
        p[1] = cabs2_acc(ri, p[1]);
        const V q = cfma_conj(ri, ri, make_double2(p[2], p[3]));
        p[2] = q.x;
        p[3] = q.y;
      }
    } epi{&a, {0.0, 0.0, 0.0, 0.0}, zero};
    spmv_run<V>(a.A, a.x, epi, smem, a.dev_err);
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k] = epi.p[k];
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const V bi = a.b[i];
      a.x[i] = zero;
      put(i, bi, bi);
    }
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
    status = HELM_OK;
  } else {
    const double rn = sqrt(tot[1]);
    st->relres = rn / bnorm;
    if (!isfinite(rn)) status = HELM_ERR_NONFINITE;
    else if (rn <= st->tol * bnorm) status = HELM_OK;
    else if (st->maxit <= 0) status = HELM_ERR_NOT_CONVERGED;
    st->rho = make_double2(tot[2], tot[3]);
    st->aux[1] = make_double2(0.0, rn);  // theta = 0, tau = ||r0||
    st->aux[0] = make_double2(0.0, 0.0);  // eta
    st->aux[2] = make_double2(0.0, 0.0);  // gamma
    // check flag; iteration at which this (re)start began (the half-step
    // index m of the bound tau sqrt(m + 2) counts from there)
    st->aux[3] = make_double2(0.0, static_cast<double>(st->iter));
  }
  st->status = status;
}

// init B: v = A u, Au = v, sigma = (r0, v) -> alpha
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_init_b(TqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) tq_cond(a, false);
    return;
  }
  struct Epi {
    const TqArgs* a;
    V sig;
    V r0i;
    __device__ __forceinline__ void prefetch(int32_t i) { r0i = a->r0[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      a->v[i] = ax;
      a->Au[i] = ax;
      sig = cfma_conj(r0i, ax, sig);
    }
  } epi{&a, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.u, epi, smem, a.dev_err);
  double part[2] = {epi.sig.x, epi.sig.y};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_V, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double2 sigma = make_double2(tot[0], tot[1]);
  int status = ST_RUNNING;
  if (!cfinite(sigma) || !cfinite(st->rho)) status = HELM_ERR_NONFINITE;
  else if (czero(sigma) || czero(st->rho)) { status = HELM_ERR_BREAKDOWN; st->iter += 1; }
  else {
    st->alpha = cdiv_fast(st->rho, sigma);
    if (!cfinite(st->alpha)) status = HELM_ERR_NONFINITE;
  }
  st->status = status;
  tq_cond(a, status == ST_RUNNING);
}

// T1: even half-step
__global__ void __launch_bounds__(256) k_tq_even(TqArgs a) {
  __shared__ double red[32];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const V alpha = st->alpha, gamma = st->aux[2];
  double ww = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const V ui = a.u[i];
    a.un[i] = cfms(alpha, a.v[i], ui);
    const V wi = cfms(alpha, a.Au[i], a.w[i]);
    a.w[i] = wi;
    a.d[i] = cfma(gamma, a.d[i], ui);
    ww = cabs2_acc(wi, ww);
  }
  double part[1] = {ww};
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_S, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->iter += 1;
  tq_half_step_scalars(st, tot[0], 2 * (st->iter - 1 - static_cast<int32_t>(st->aux[3].y)));
  if (st->status == ST_RUNNING) tq_gamma(st);  // gamma of the odd half-step's d update (same alpha)
}

// T2: Aun = A un; x += eta d
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_spmv_un(TqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  struct Epi {
    const TqArgs* a;
    V eta;
    V di, xi;
    __device__ __forceinline__ void prefetch(int32_t i) {
      di = a->d[i];
      xi = a->x[i];
    }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      a->Aun[i] = ax;
      a->x[i] = cfma(eta, di, xi);
    }
  } epi{&a, st->aux[0], make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.un, epi, smem, a.dev_err);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->spmv_count += 1;
}

// T3: odd half-step
__global__ void __launch_bounds__(256) k_tq_odd(TqArgs a) {
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const V alpha = st->alpha, gamma = st->aux[2];
  double ww = 0.0;
  V rw = make_double2(0.0, 0.0);
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const V wi = cfms(alpha, a.Aun[i], a.w[i]);
    a.w[i] = wi;
    a.d[i] = cfma(gamma, a.d[i], a.un[i]);
    ww = cabs2_acc(wi, ww);
    rw = cfma_conj(a.r0[i], wi, rw);
  }
  double part[3] = {ww, rw.x, rw.y};
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_T, red, tot)) return;
  if (threadIdx.x != 0) return;
  tq_half_step_scalars(st, tot[0], 2 * (st->iter - 1 - static_cast<int32_t>(st->aux[3].y)) + 1);
  if (st->status != ST_RUNNING) return;
  const double2 rho_new = make_double2(tot[1], tot[2]);
  if (!cfinite(rho_new)) {
    st->status = HELM_ERR_NONFINITE;
    return;
  }
  if (czero(st->rho)) {
    st->status = HELM_ERR_BREAKDOWN;
    return;
  }
  st->beta = cdiv_fast(rho_new, st->rho);
  st->rho = rho_new;
}

// T4: u = w + beta un; x += eta d
__global__ void __launch_bounds__(256) k_tq_u(TqArgs a) {
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const V beta = st->beta, eta = st->aux[0];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    a.u[i] = cfma(beta, a.un[i], a.w[i]);
    a.x[i] = cfma(eta, a.d[i], a.x[i]);
  }
}

// T5: Au = A u; v = Au + beta (Aun + beta v); sigma = (r0, v) -> alpha, gamma
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_spmv_u(TqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  struct Epi {
    const TqArgs* a;
    V beta;
    V sig;
    V auni, vi, r0i;
    __device__ __forceinline__ void prefetch(int32_t i) {
      auni = a->Aun[i];
      vi = a->v[i];
      r0i = a->r0[i];
    }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      a->Au[i] = ax;
      const V vn = cfma(beta, cfma(beta, vi, auni), ax);
      a->v[i] = vn;
      sig = cfma_conj(r0i, vn, sig);
    }
  } epi{&a, st->beta, make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
        make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.u, epi, smem, a.dev_err);
  double part[2] = {epi.sig.x, epi.sig.y};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_AUX1, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double2 sigma = make_double2(tot[0], tot[1]);
  if (!cfinite(sigma)) st->status = HELM_ERR_NONFINITE;
  else if (czero(sigma) || czero(st->rho)) st->status = HELM_ERR_BREAKDOWN;
  else {
    st->alpha = cdiv_fast(st->rho, sigma);
    if (!cfinite(st->alpha)) st->status = HELM_ERR_NONFINITE;
    else tq_gamma(st);
  }
}

// T6: true-residual check when a bound fell below tol; cap, deadline, condition
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_check(TqArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  SolverState* st = a.st;
  const int status0 = st->status;
  const bool check = status0 == ST_RUNNING && st->aux[3].x != 0.0;
  if (!check) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      int status = status0;
      if (status == ST_RUNNING) {
        if (st->iter >= st->maxit) status = HELM_ERR_NOT_CONVERGED;
        else if (st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns) status = HELM_ERR_TIMEOUT;
        st->status = status;
      }
      tq_cond(a, status == ST_RUNNING);
    }
    return;
  }
  struct Epi {
    const TqArgs* a;
    double part;
    V bi;
    __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) { part = cabs2_acc(csub(bi, ax), part); }
  } epi{&a, 0.0, make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.x, epi, smem, a.dev_err);
  double part[1] = {epi.part};
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_AUX2, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double rt = sqrt(tot[0]) / st->bnorm;
  st->aux[3].x = 0.0;
  int status = ST_RUNNING;
  if (!isfinite(rt)) status = HELM_ERR_NONFINITE;
  else if (rt <= st->tol) status = HELM_OK;
  else if (st->iter >= st->maxit) status = HELM_ERR_NOT_CONVERGED;
  else if (st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns) status = HELM_ERR_TIMEOUT;
  // the bound is below tol but the true residual is not: the recurrence has
  // drifted from b - A x, so the host starts again from the current x
  else status = ST_RESTART;
  st->status = status;
  tq_cond(a, status == ST_RUNNING);
}

// tail: ||b - A x|| / ||b|| (x = 0 when b = 0)
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_tq_tail(TqArgs a) {
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
      const TqArgs* a;
      double part;
      V bi;
      __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, V ax) { part = cabs2_acc(csub(bi, ax), part); }
    } epi{&a, 0.0, make_double2(0.0, 0.0)};
    spmv_run<V>(a.A, a.x, epi, smem, a.dev_err);
    part[0] = epi.part;
  }
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_TAIL, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->relres_true = bnorm == 0.0 ? 0.0 : sqrt(tot[0]) / bnorm;
  if (bnorm != 0.0) st->spmv_count += 1;
}

struct TqShapes {
  int spmv_grid, vec_grid;
};

void tq_init(const TqArgs& a, const TqShapes& sh, cudaStream_t s) {
  k_tq_init_a<<<sh.spmv_grid, RT, kSmem, s>>>(a);
  k_tq_init_b<<<sh.spmv_grid, RT, kSmem, s>>>(a);
}
void tq_body(const TqArgs& a, const TqShapes& sh, cudaStream_t s) {
  k_tq_even<<<sh.vec_grid, 256, 0, s>>>(a);
  k_tq_spmv_un<<<sh.spmv_grid, RT, kSmem, s>>>(a);
  k_tq_odd<<<sh.vec_grid, 256, 0, s>>>(a);
  k_tq_u<<<sh.vec_grid, 256, 0, s>>>(a);
  k_tq_spmv_u<<<sh.spmv_grid, RT, kSmem, s>>>(a);
  k_tq_check<<<sh.spmv_grid, RT, kSmem, s>>>(a);
}
void tq_tail(const TqArgs& a, const TqShapes& sh, cudaStream_t s) { k_tq_tail<<<sh.spmv_grid, RT, kSmem, s>>>(a); }

}  // namespace

helm_status tfqmr_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                       cudaStream_t s) {
  helm_status st = ensure_vectors(A, kNumVec);
  if (st != HELM_OK) return st;
  for (const void* fn : {reinterpret_cast<const void*>(&k_tq_init_a), reinterpret_cast<const void*>(&k_tq_init_b),
                         reinterpret_cast<const void*>(&k_tq_spmv_un), reinterpret_cast<const void*>(&k_tq_spmv_u),
                         reinterpret_cast<const void*>(&k_tq_check), reinterpret_cast<const void*>(&k_tq_tail)})
    HELM_CUDA_TRY(set_smem_attr(fn, kSmem));
  TqShapes sh;
  HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_tq_init_a), reinterpret_cast<const void*>(&k_tq_init_b),
                            reinterpret_cast<const void*>(&k_tq_spmv_un), reinterpret_cast<const void*>(&k_tq_spmv_u),
                            reinterpret_cast<const void*>(&k_tq_check), reinterpret_cast<const void*>(&k_tq_tail)},
                           RT, kSmem, A->num_sms, (static_cast<int64_t>(A->n) + Engine<V>::R - 1) / Engine<V>::R,
                           &sh.spmv_grid));
  sh.vec_grid = A->vec_grid;
  const size_t N = static_cast<size_t>(A->n);
  double2* W = A->vec;
  TqArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = csr_for(A, o);
  a.b = b;
  a.x = x;
  a.r0 = W;
  a.w = W + N;
  a.u = W + 2 * N;
  a.un = W + 3 * N;
  a.v = W + 4 * N;
  a.Au = W + 5 * N;
  a.Aun = W + 6 * N;
  a.d = W + 7 * N;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.dev_err = A->dev_err;

  // graph cache: key (b, x, variant), the variant tagged as TFQMR
  GraphEntry* g = nullptr;
  auto key = graph_key(b, x, 1, o);
  auto it = A->graphs.find(key);
  if (o.launch == HELM_LAUNCH_HOST) {
  } else if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    auto with = [&](cudaGraphConditionalHandle c) {
      TqArgs aa = a;
      aa.cond = c;
      aa.has_cond = 1;
      return aa;
    };
    GraphEntry e;
    if (build_while_graph([&](cudaGraphConditionalHandle c, cudaStream_t cs) { tq_init(with(c), sh, cs); },
                          [&](cudaGraphConditionalHandle c, cudaStream_t cs) { tq_body(with(c), sh, cs); },
                          [&](cudaGraphConditionalHandle c, cudaStream_t cs) { tq_tail(with(c), sh, cs); },
                          &e) == HELM_OK)
      g = &(A->graphs[key] = e);
  }

  // an explicit graph request does not fall back to the host-driven loop
  if (!g && o.launch == HELM_LAUNCH_GRAPH) return HELM_ERR_CUDA;
  SolverState* hs = A->state_host;
  unsigned int herr = 0;
  int32_t use_x0 = o.use_x0 ? 1 : 0, fresh = 1;
  HELM_CUDA_TRY(cudaMemsetAsync(A->dev_err, 0, sizeof(unsigned int), s));
  for (;;) {
    k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0, o.deadline_s, fresh);
    HELM_CUDA_TRY(cudaGetLastError());
    if (g) {
      HELM_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    } else {
      tq_init(a, sh, s);
      for (;;) {
        for (int k = 0; k < 8; ++k) tq_body(a, sh, s);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs->status != ST_RUNNING) break;
      }
      tq_tail(a, sh, s);
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) return HELM_ERR_CUDA;
    if (hs->status != ST_RESTART) break;
    use_x0 = 1;  // start again from the current x, iterations counted on
    fresh = 0;
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
