// Mixed-precision solve: FP64 outer GCR (iterative refinement with a window
// of directions) around complex64 BiCGStab inner solves, the whole solve in
// one CUDA graph.
//
// The paper's library covers single and double precision (Section 1); here
// single precision does the bulk of the work and FP64 decides accuracy:
//   inner (FP32):  BiCGStab on A32 (complex64 copy of the values owned by the
//                  handle, 8 bytes per entry for real rows instead of 12), vectors
//                  complex64; products and per-thread sums FP32, block and
//                  grid sums and every recurrence scalar FP64.  The inner
//                  system is A32 d = r / sigma with sigma = ||r|| / sqrt(n)
//                  (unit RMS entries: in the problem's own scale, b ~ h^3,
//                  the squared terms of the inner dots would fall below the
//                  smallest normal float long before FP64 convergence).
//   step (FP64):   when the inner recurrence residual has dropped by
//                  inner_tol since the inner solve began, looks below the
//                  outer tolerance, or after kInnerMax inner iterations, an
//                  outer GCR step on z = sigma d: w = A z; c = w - sum beta_j
//                  C_j and z -= sum beta_j Z_j over a window of the last
//                  kGcr directions (C_j orthonormal, A Z_j = C_j; classical
//                  Gram-Schmidt, beta_j = (C_j, w)); gamma = (c, r) / (c, c)
//                  minimises ||r - gamma c||, so the residual is minimised
//                  over the whole window and a poor inner solve cannot
//                  increase it; x += gamma z; r = b - A x in FP64; stop if
//                  ||r|| / ||b|| <= tol (or, not converged, after five steps
//                  in a row without halving ||r||); else a fresh inner solve
//                  on the new r (r^ = r, p = v = d = 0).
// The inner operator is A rounded to complex64, so plain refinement gains at
// most about kappa eps_float per step; the GCR window lets rough inner
// solves add up instead.  Measured before it: one inner process kept across
// steps with its residual replaced (Sleijpen & van der Vorst 1996) stagnated
// on the strongly indefinite 200x100x80 cavity; plain restarted refinement
// converged slowly and, folded without a step length, diverged whenever an
// inner solve stagnated.  The convergence test is always the FP64 true
// residual.
// Launch structure: init (+ first inner start); then per refinement step one
// launch of the inner graph (a conditional WHILE over the 5 complex64
// kernels, which ends when a step is due or the solve stops) and one of the
// step graph (its 6 kernels), the host reading the state between steps; then
// the tail.  An inner iteration so launches its five kernels and nothing
// else (with the step kernels inside the loop body, returning at once when
// no step is due, an inner iteration cost 84.5 instead of 76.1 us on
// the 120x60x50 cavity).  A conditional IF node around the step kernels
// inside the WHILE body was tried first: adding it fails with
// cudaErrorInvalidValue on this CUDA 13.0 stack (handle on the body or the
// top graph, with or without a default).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

namespace {

// Directions kept by the outer GCR (a window over the refinement steps).
constexpr int kGcr = 8;

constexpr int R128 = Engine<double2>::kThreads;  // threads per SpMV block
constexpr size_t kSmem128 = Engine<double2>::kSmem;

struct RuArgs {
  CsrDev<double2> A;  // FP64 matrix
  const double2* b;
  double2* x;         // FP64 solution (the caller's)
  double2* r64;       // FP64 residual
  double2* d64;       // FP64 copy of the scaled inner solution
  double2* w64;       // A d64
  double2* Cw[kGcr];  // GCR window: orthonormal A z_j
  double2* Zw[kGcr];  //   and the directions z_j
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
// p, v (r and r^ are written by the first inner start, once the scale is known).
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

// init: r64 = b - A x (or b, x = 0); asks for the first inner start, which
// starts the complex64 recurrence
__global__ void __launch_bounds__(R128, kSolverMinBlocks) k_mx_init(RuArgs a) {
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
  st->method = kModeRefine;
  st->aux[0] = make_double2(rn, 0.0);   // ||r64||, iteration of the last step
  st->aux[1] = make_double2(1.0, 0.0);  // inner start due
  st->aux[2] = make_double2(0.0, 0.0);  // no inner scale yet
  st->gcr_n = 0;                         // empty GCR window
  st->gcr_next = 0;
  st->gcr_keep = 0;
  st->status = status;
}

// aux[3].y = the reduction of the inner residual that ends an inner solve
// (opts.inner_tol)
__global__ void k_mx_configure(SolverState* st, double inner_tol) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->aux[3] = make_double2(0.0, inner_tol);
}

// step 1a: d64 = sigma complex128(d); d = 0
__global__ void __launch_bounds__(256) k_mx_lift(RuArgs a, int always) {
  const SolverState* st = a.st;
  if (!always && st->aux[1].x == 0.0) return;
  const double sc = st->aux[2].x;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const float2 d = a.x32[i];
    a.d64[i] = make_double2(sc * static_cast<double>(d.x), sc * static_cast<double>(d.y));
    a.x32[i] = make_float2(0.f, 0.f);
  }
}

// Block and grid sums of K > 4 doubles: slices of four through the fixed-
// order block tree (result in thread 0), then the last block adds the block
// partials in block order.
template <int K>
__device__ __forceinline__ void block_sum_many(double (&v)[K], double* red) {
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 4) {
    double q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = k0 + k < K ? v[k0 + k < K ? k0 + k : 0] : 0.0;
    block_sum<4>(q, red);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k0 + k < K) v[k0 + k < K ? k0 + k : 0] = q[k];
  }
}
template <int K>
__device__ __forceinline__ bool grid_sum_last_many(double (&v)[K], double* partials, unsigned int* ticket,
                                                   double* red, double (&tot)[K]) {
  __shared__ bool s_last;
  block_sum_many<K>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += ld_cg(&partials[(size_t)b * K + k]);
  block_sum_many<K>(acc, red);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = acc[k];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// step 1b: w = A z (FP64, z = d64) and the projections beta_j = (C_j, w) on
// the stored directions (classical Gram-Schmidt against the GCR window).
__global__ void __launch_bounds__(R128, kSolverMinBlocks) k_gcr_project(RuArgs a, int always) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int K = 2 * kGcr;
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  if (!always && st->aux[1].x == 0.0) return;
  const int nw = st->gcr_n;
  struct Epi {
    const RuArgs* a;
    int nw;
    double acc[K];
    __device__ __forceinline__ void prefetch(int32_t) {}
    __device__ __forceinline__ void row(int32_t i, double2 w) {
      a->w64[i] = w;
#pragma unroll
      for (int j = 0; j < kGcr; ++j) {
        if (j < nw) {
          const double2 q = cfma_conj(a->Cw[j][i], w, make_double2(acc[2 * j], acc[2 * j + 1]));
          acc[2 * j] = q.x;
          acc[2 * j + 1] = q.y;
        }
      }
    }
  } epi{&a, nw, {}};
  spmv_run<double2>(a.A, a.d64, epi, smem, a.dev_err);
  double tot[K];
  if (!grid_sum_last_many<K>(epi.acc, a.partials, a.tickets + TK_AUX2, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
#pragma unroll
  for (int j = 0; j < kGcr; ++j) st->gcr_beta[j] = j < nw ? make_double2(tot[2 * j], tot[2 * j + 1]) : make_double2(0.0, 0.0);
}

// step 1c: c = w - sum beta_j C_j, z = d64 - sum beta_j Z_j into the window
// slot; gamma = (c, r64) / (c, c), the step that minimises ||r64 - gamma c||
// over the direction orthogonal to the window (so never an increase of the
// FP64 residual, whatever the inner solve returned).
__global__ void __launch_bounds__(256) k_gcr_orth(RuArgs a, int always) {
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  if (!always && st->aux[1].x == 0.0) return;
  const int nw = st->gcr_n, slot = st->gcr_next;
  double2 beta[kGcr];
#pragma unroll
  for (int j = 0; j < kGcr; ++j) beta[j] = st->gcr_beta[j];
  double2 cr = make_double2(0.0, 0.0);
  double cc = 0.0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    double2 c = a.w64[i], z = a.d64[i];
#pragma unroll
    for (int j = 0; j < kGcr; ++j) {
      if (j < nw) {
        c = cfms(beta[j], a.Cw[j][i], c);
        z = cfms(beta[j], a.Zw[j][i], z);
      }
    }
    a.Cw[slot][i] = c;
    a.Zw[slot][i] = z;
    cr = cfma_conj(c, a.r64[i], cr);
    cc = cabs2_acc(c, cc);
  }
  double part[3] = {cr.x, cr.y, cc};
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_AUX3, red, tot)) return;
  if (threadIdx.x != 0) return;
  double2 gamma = make_double2(0.0, 0.0);
  double nrm = 0.0;
  int keep = 0;
  if (tot[2] > 0.0 && isfinite(tot[2])) {
    const double inv = 1.0 / tot[2];
    gamma = make_double2(tot[0] * inv, tot[1] * inv);
    nrm = sqrt(tot[2]);
    keep = cfinite(gamma) ? 1 : 0;
    if (!keep) gamma = make_double2(0.0, 0.0);
  }
  st->gamma = gamma;
  st->gcr_nrm = nrm;
  st->gcr_keep = keep;
}

// step 1d: x += gamma z, and the window slot normalised (|| C_slot || = 1)
__global__ void __launch_bounds__(256) k_gcr_xupd(RuArgs a, int always) {
  const SolverState* st = a.st;
  if (!always && st->aux[1].x == 0.0) return;
  const double2 gamma = st->gamma;
  const int slot = st->gcr_next, keep = st->gcr_keep;
  const double inv = keep ? 1.0 / st->gcr_nrm : 0.0;
  if (!keep) return;  // rejected direction (zero or non-finite): x stays as it is
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
    const double2 z = a.Zw[slot][i];
    a.x[i] = cfma(gamma, z, a.x[i]);
    const double2 c = a.Cw[slot][i];
    a.Cw[slot][i] = make_double2(c.x * inv, c.y * inv);
    a.Zw[slot][i] = make_double2(z.x * inv, z.y * inv);
  }
}

// step 2: r64 = b - A x (FP64), the convergence test
__global__ void __launch_bounds__(R128, kSolverMinBlocks) k_mx_residual(RuArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  SolverState* st = a.st;
  if (st->aux[1].x == 0.0) return;
  struct Epi {
    const RuArgs* a;
    double part;
    double2 bi;
    __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
    __device__ __forceinline__ void row(int32_t i, double2 ax) {
      const double2 ri = csub(bi, ax);
      a->r64[i] = ri;
      part = cabs2_acc(ri, part);
    }
  } epi{&a, 0.0, make_double2(0.0, 0.0)};
  spmv_run<double2>(a.A, a.x, epi, smem, a.dev_err);
  double part[1] = {epi.part};
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_AUX0, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  st->restarts += 1;  // refinement steps
  const double rn = sqrt(tot[0]);
  st->relres_true = rn / st->bnorm;
  if (!isfinite(rn)) st->status = HELM_ERR_NONFINITE;
  else if (rn <= st->tol * st->bnorm) {
    st->status = HELM_OK;
    st->relres = st->relres_true;
  }
  // refinement must contract: five steps in a row without halving the
  // residual end the solve (the inner operator, A rounded to complex64, is
  // then too far from A for this system)
  const double prev = st->aux[0].x * st->aux[2].x;  // ||r64|| before the step
  st->aux[3].x = rn > 0.5 * prev ? st->aux[3].x + 1.0 : 0.0;
  if (st->status == ST_RUNNING && st->aux[3].x >= 5.0) st->status = HELM_ERR_NOT_CONVERGED;
  st->aux[0] = make_double2(rn, static_cast<double>(st->iter));
  // the step's direction joins the GCR window (the oldest one leaves it)
  if (st->gcr_keep) {
    st->gcr_next = (st->gcr_next + 1) % kGcr;
    if (st->gcr_n < kGcr) st->gcr_n += 1;
    st->gcr_keep = 0;
  }
}

// step 3: a fresh inner solve on r64: sigma = ||r64|| / sqrt(n),
// r = r^ = complex64(r64 / sigma), p = v = 0, rho = (r^, r); the deadline and
// the loop condition of the iteration.
__global__ void __launch_bounds__(256) k_mx_restart(RuArgs a) {
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
  const double s_new = st->aux[0].x / sqrt(static_cast<double>(n));
  const double inv = 1.0 / s_new;
  double2 rr = make_double2(0.0, 0.0);
  if (st->status == ST_RUNNING) {
    const float2 z = make_float2(0.f, 0.f);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 ri = a.r64[i];
      const float2 r32 = make_float2(static_cast<float>(ri.x * inv), static_cast<float>(ri.y * inv));
      a.r32[i] = r32;
      a.rh32[i] = r32;
      a.p32[i] = z;
      a.v32[i] = z;
      rr = cfma_conj(make_double2(r32.x, r32.y), make_double2(r32.x, r32.y), rr);
    }
  }
  double part[2] = {rr.x, rr.y};
  double tot[2];
  if (!grid_sum_last<2>(part, a.partials, a.tickets + TK_AUX1, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->aux[1] = make_double2(0.0, 0.0);
  if (st->status == ST_RUNNING) {
    const double2 rho = make_double2(tot[0], tot[1]);
    if (!cfinite(rho)) {
      st->status = HELM_ERR_NONFINITE;
    } else if (czero(rho)) {
      st->status = HELM_ERR_BREAKDOWN;
    } else {
      st->rho = rho;  // the first p update gives p = r whatever beta is
      st->aux[2].x = s_new;
      st->aux[0].x = st->aux[0].x * inv;  // ||r|| in the inner scale
    }
    if (st->status == ST_RUNNING && st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns)
      st->status = HELM_ERR_TIMEOUT;
  }
  ru_cond(a, st->status == ST_RUNNING);
}

// tail: the FP64 true residual for the report (x32 folded just before)
__global__ void __launch_bounds__(R128, kSolverMinBlocks) k_mx_tail(RuArgs a) {
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
  int grid_proj;  // the projection's 2 kGcr partial sums per block fit the partials buffer
  int vec_grid;
};

void mx_init(const RuArgs& a, const MxShapes& sh, cudaStream_t s) {
  k_mx_init<<<sh.grid128, R128, kSmem128, s>>>(a);
  k_mx_restart<<<sh.vec_grid, 256, 0, s>>>(a);
}
void mx_fold(const RuArgs& a, const MxShapes& sh, int always, cudaStream_t s) {
  k_mx_lift<<<sh.vec_grid, 256, 0, s>>>(a, always);
  k_gcr_project<<<sh.grid_proj, R128, kSmem128, s>>>(a, always);
  k_gcr_orth<<<sh.vec_grid, 256, 0, s>>>(a, always);
  k_gcr_xupd<<<sh.vec_grid, 256, 0, s>>>(a, always);
}
// the refinement step: fold the inner solution into x (GCR), the FP64
// residual and a fresh inner start
void mx_step(const RuArgs& a, const MxShapes& sh, cudaStream_t s) {
  mx_fold(a, sh, 0, s);
  k_mx_residual<<<sh.grid128, R128, kSmem128, s>>>(a);
  k_mx_restart<<<sh.vec_grid, 256, 0, s>>>(a);
}
void mx_body(const RuArgs& a, const KArgs<float2>& k, const MxShapes& sh, cudaStream_t s) {
  enqueue_body(k, sh.k, s);
  mx_step(a, sh, s);
}
// A graph of one conditional WHILE node whose body is body(cond, stream).
template <class Body>
helm_status build_loop_graph(Body body, GraphEntry* out) {
  cudaStream_t cs = nullptr;
  HELM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  helm_status result = HELM_ERR_CUDA;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) break;
    cudaGraph_t tmp = nullptr;
    if (cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    for (int u = 0; u < kBodyUnroll; ++u) body(cond, cs);
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

// A graph of the kernels fn(stream) enqueues (stream capture).
template <class Fn>
helm_status build_plain_graph(Fn fn, GraphEntry* out) {
  cudaStream_t cs = nullptr;
  HELM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  helm_status result = HELM_ERR_CUDA;
  do {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
    fn(cs);
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) break;
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

void mx_tail(const RuArgs& a, const MxShapes& sh, cudaStream_t s) {
  mx_fold(a, sh, 1, s);
  k_mx_tail<<<sh.grid128, R128, kSmem128, s>>>(a);
}

}  // namespace

helm_status solve_mixed(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                        cudaStream_t s) {
  helm_status st = ensure_vals32(A, s);
  if (st == HELM_OK) st = ensure_vectors(A, kNumVec > 3 + 2 * kGcr ? kNumVec : 3 + 2 * kGcr);
  if (st == HELM_OK) st = ensure_vectors32(A, 8);
  if (st == HELM_OK) st = prepare_krylov_kernels<float2>();
  if (st != HELM_OK) return st;
  for (const void* fn : {reinterpret_cast<const void*>(&k_mx_init), reinterpret_cast<const void*>(&k_mx_residual),
                         reinterpret_cast<const void*>(&k_gcr_project), reinterpret_cast<const void*>(&k_mx_tail)})
    HELM_CUDA_TRY(set_smem_attr(fn, kSmem128));
  MxShapes sh;
  st = krylov_shapes<float2>(A, &sh.k);
  if (st != HELM_OK) return st;
  HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_mx_init), reinterpret_cast<const void*>(&k_mx_residual),
                            reinterpret_cast<const void*>(&k_gcr_project), reinterpret_cast<const void*>(&k_mx_tail)},
                           R128, kSmem128, A->num_sms,
                           (static_cast<int64_t>(A->n) + Engine<double2>::R - 1) / Engine<double2>::R, &sh.grid128));
  // partials buffer: num_sms * 32 * 8 doubles (api.cu)
  sh.grid_proj = std::min(sh.grid128, A->num_sms * 32 * 8 / (2 * kGcr));
  sh.vec_grid = A->vec_grid;
  const int32_t n = A->n;
  const size_t N = static_cast<size_t>(n);
  float2* W = A->vec32;

  KArgs<float2> k;
  std::memset(&k, 0, sizeof(k));
  k.A = csr_dev<float2>(A, A->vals32, A->sv32);
  k.r = W;
  k.rh = W + N;
  k.p = W + 2 * N;
  k.v = W + 3 * N;
  k.s = W + 4 * N;
  k.t = W + 5 * N;
  k.x = W + 6 * N;  // d: the inner solution of the current refinement step
  k.b = W + 7 * N;  // not read by the loop body
  k.st = A->state;
  k.partials = A->partials;
  k.tickets = A->tickets;
  k.gtickets = A->gtickets;
  k.dev_err = A->dev_err;

  RuArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = csr_dev<double2>(A, static_cast<const double2*>(A->vals), A->sv);
  a.b = b;
  a.x = x;
  a.r64 = A->vec;
  a.d64 = A->vec + N;
  a.w64 = A->vec + 2 * N;
  for (int j = 0; j < kGcr; ++j) {
    a.Cw[j] = A->vec + (3 + j) * N;
    a.Zw[j] = A->vec + (3 + kGcr + j) * N;
  }
  a.x32 = k.x;
  a.r32 = k.r;
  a.rh32 = k.rh;
  a.p32 = k.p;
  a.v32 = k.v;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.dev_err = A->dev_err;

  // the inner-loop graph and the step graph per (b, x), tagged as mixed in
  // the cache key
  GraphEntry* gi = nullptr;
  GraphEntry* gs = nullptr;
  if (o.launch != HELM_LAUNCH_HOST) {
    auto ki = graph_key(b, x, 2, o), ks = graph_key(b, x, 3, o);
    auto ii = A->graphs.find(ki), is = A->graphs.find(ks);
    if (ii != A->graphs.end() && is != A->graphs.end()) {
      gi = &ii->second;
      gs = &is->second;
    } else {
      GraphEntry ei, es;
      const bool ok_i = build_loop_graph(
                            [&](cudaGraphConditionalHandle c, cudaStream_t cs) {
                              KArgs<float2> kk = k;
                              kk.cond = c;
                              kk.has_cond = 1;
                              enqueue_body(kk, sh.k, cs);
                            },
                            &ei) == HELM_OK;
      const bool ok_s = ok_i && build_plain_graph([&](cudaStream_t cs) { mx_step(a, sh, cs); }, &es) == HELM_OK;
      if (ok_i && ok_s) {
        gi = &(A->graphs[ki] = ei);
        gs = &(A->graphs[ks] = es);
      } else {
        if (ei.exec) cudaGraphExecDestroy(ei.exec);
        if (ei.graph) cudaGraphDestroy(ei.graph);
      }
    }
  }

  // an explicit graph request does not fall back to the host-driven loop
  if (!gi && o.launch == HELM_LAUNCH_GRAPH) return HELM_ERR_CUDA;
  HELM_CUDA_TRY(cudaMemsetAsync(A->dev_err, 0, sizeof(unsigned int), s));
  k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, o.use_x0 ? 1 : 0, o.deadline_s, 1);
  k_mx_configure<<<1, 1, 0, s>>>(A->state, o.inner_tol);
  HELM_CUDA_TRY(cudaGetLastError());
  SolverState* hs = A->state_host;
  mx_init(a, sh, s);
  for (;;) {
    if (gi) {
      HELM_CUDA_TRY(cudaGraphLaunch(gi->exec, s));
      HELM_CUDA_TRY(cudaGraphLaunch(gs->exec, s));
    } else {
      for (int q = 0; q < 8; ++q) mx_body(a, k, sh, s);
      HELM_CUDA_TRY(cudaGetLastError());
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs->status != ST_RUNNING) break;
  }
  mx_tail(a, sh, s);
  HELM_CUDA_TRY(cudaGetLastError());
  unsigned int herr = 0;
  HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) return HELM_ERR_CUDA;
  helm_status result = hs->status == ST_RUNNING ? HELM_ERR_CUDA : static_cast<helm_status>(hs->status);
  if (result == HELM_OK && !(hs->relres_true <= o.tol)) result = HELM_ERR_NOT_CONVERGED;
  if (info) {
    info->iters = hs->iter;
    info->restarts = hs->restarts;  // refinement steps
    info->relres_recur = hs->relres;
    info->relres_true = hs->relres_true;
    info->status = result;
    info->spmv_count = hs->spmv_count;
  }
  return result;
}

}  // namespace helm
