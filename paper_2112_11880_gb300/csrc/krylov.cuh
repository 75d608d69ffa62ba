// BiCGStab kernels with device-resident scalars, generic over the vector
// precision (complex128 for the FP64 solver, complex64 for the inner solve of
// mixed precision).  Section 4 of the paper: P-BiCGSTAB with residual
// tolerance, zero initial guess and an iteration cap; identity preconditioner
// (right Jacobi runs the same kernels on A D^-1); the recurrence of van der
// Vorst 1992 / Saad 2003 Algorithm 7.7 with conjugated inner products.
//
// One iteration is five phases; each dot product the recurrence needs is
// fused into the phase that produces its operands, and the scalar it feeds
// is formed in FP64 on the device:
//   P1  p = r + beta (p - omega v)
//   P2  v = A p          + (r^, v)        -> alpha = rho / (r^, v)
//   P3  s = r - alpha v  + ||s||^2        -> stop at s if ||s|| / ||b|| <= tol
//   P4  t = A s          + (t, s), ||t||^2 -> omega = (t, s) / (t, t)
//   P5  x += alpha p + omega s, r = s - omega t + (r^, r), ||r||^2
//                                         -> stop test, rho, beta
// For complex64 the products and each thread's partial sums are FP32; block
// and grid sums and every scalar of the recurrence are FP64.
//
// Two ways to run the loop, with the same arithmetic bit for bit:
//   * graph: one kernel per phase; the last block to finish a phase (ticket
//     counter) adds the block partials and forms the scalars; the loop is a
//     CUDA graph with a conditional WHILE node (four iterations per pass);
//   * persistent: one cooperative kernel for the whole solve; a grid barrier
//     ends every phase, after which every block adds the block partials
//     itself (same order, so the same scalars in every block) -- no kernel
//     launches, no last-block step.
// Both give each row to the same thread in every phase (SliceRows of the
// SpMV engine) on the same grid, and add the same partials in the same order.
#pragma once

#include <algorithm>
#include <type_traits>
#include <cstring>
#include <initializer_list>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.hpp"
#include "spmv.cuh"

namespace helm {

// The complex128 matrix a solve runs on: A, or A D^-1 under right Jacobi.
inline CsrDev<double2> csr_for(helm_csr A, const helm_opts& o) {
  if (o.precond == HELM_PRECOND_JACOBI) return csr_dev<double2>(A, A->jac_vals, A->svjac);
  return csr_dev<double2>(A, static_cast<const double2*>(A->vals), A->sv);
}

// SolverState::method of the Krylov loop: plain, or the inner loop of the
// mixed-precision solve (aux[0] = (||r|| when the process began, in its
// scale; iteration it began), aux[1].x = refinement step due, aux[2].x =
// scale of the inner residual, aux[3] = (steps in a row without a 2x gain,
// inner_tol)).
constexpr int32_t kModePlain = 0;
constexpr int32_t kModeRefine = 1;
constexpr int kInnerMax = 50000;  // inner iterations per refinement step at most

// Per-thread partial sums of dot products and norms (S real, C complex)
// accumulate in FP64: for complex128 operands the FP64 product (4 or 2 FMA),
// for complex64 operands the product formed in FP32 and added in FP64.
// Measured alternatives for complex64: an uncompensated FP32 running sum
// over the ~10 rows a thread takes on the 200x100x80 cavity slowed the inner
// solves of mixed precision visibly; a compensated (Kahan) FP32 sum made an
// inner iteration 2-6 % faster on the 120x60x50 and 200x100x80 cavities, but
// the 200x100x80 solve to 1e-10 then stalled (289,524 inner iterations, not
// converged, against 188,207 to convergence with FP64 sums).
template <class V> struct Prec;
template <> struct Prec<double2> {
  using S = double;
  using C = double2;
  __device__ static __forceinline__ double2 cvt(double2 z) { return z; }
  __device__ static __forceinline__ S szero() { return 0.0; }
  __device__ static __forceinline__ C czero() { return make_double2(0.0, 0.0); }
};
template <> struct Prec<float2> {
  using S = double;
  using C = double2;
  __device__ static __forceinline__ float2 cvt(double2 z) {
    return make_float2(static_cast<float>(z.x), static_cast<float>(z.y));
  }
  __device__ static __forceinline__ S szero() { return 0.0; }
  __device__ static __forceinline__ C czero() { return make_double2(0.0, 0.0); }
};
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

// acc + conj(a) b and acc + |a|^2 in the precision rules above
__device__ __forceinline__ double2 dot_acc(double2 acc, double2 a, double2 b) { return cfma_conj(a, b, acc); }
__device__ __forceinline__ double2 dot_acc(double2 acc, float2 a, float2 b) {
  const float re = fmaf(a.x, b.x, a.y * b.y);
  const float im = fmaf(a.x, b.y, -a.y * b.x);
  return make_double2(acc.x + static_cast<double>(re), acc.y + static_cast<double>(im));
}
__device__ __forceinline__ double nrm_acc(double acc, double2 a) { return cabs2_acc(a, acc); }
__device__ __forceinline__ double nrm_acc(double acc, float2 a) {
  return acc + static_cast<double>(fmaf(a.x, a.x, a.y * a.y));
}

// Every kernel of the solver: at most 1024 threads, one block per SM.
constexpr int kSolverThreads = Engine<double2>::kThreads;
constexpr int kSolverMinBlocks = Engine<double2>::kMinBlocks;

template <class V>
struct KArgs {
  CsrDev<V> A;
  const V* b;
  V* x;
  V *r, *rh, *p, *v, *s, *t;
  SolverState* st;
  double* partials;
  unsigned int* tickets;
  unsigned int* gtickets;
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

template <class V>
__device__ __forceinline__ void set_cond(const KArgs<V>& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

__device__ __forceinline__ bool deadline_passed(const SolverState* st) {
  return st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns;
}

__global__ void k_configure(SolverState* st, double tol, int32_t maxit, int32_t use_x0, double deadline_s,
                            int32_t fresh);

// Programmatic dependent launch.  The loop's kernels are launched so that a
// kernel's blocks may be scheduled while its predecessor is still running:
// they take the SMs that the predecessor's blocks leave while its last block
// forms the scalars, and wait here until the predecessor grid has completed
// and its writes are visible.  Every kernel of the loop calls this before it
// reads anything, so the order of every operation is that of plain launches
// (with a plain launch the wait returns at once).  Each grid is one wave, so
// the waiting blocks never hold an SM that a block of the predecessor needs.
// Measured on the 120x60x50 cavity (BiCGStab, 19,653 iterations): the
// host-driven loop 148.6 -> 141.4 us per iteration; the graph (the WHILE
// node, or a plain graph of 16 iterations) 138.1 us either way, although its
// body keeps the programmatic edges: a graph launch already hides that gap.
#ifndef HELM_PDL
#define HELM_PDL 1
#endif
__device__ __forceinline__ void pdl_enter() {
#if HELM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// ---------------------------------------------------------------- reductions

// Fixed-order total of the block partials partials[b K + k], b < G: thread j
// adds blocks j, j + T, j + 2T, ... in that order, then the fixed block tree.
// Valid in thread 0.
template <int K>
__device__ __forceinline__ void sum_block_partials(const double* partials, int G, double* red, double (&tot)[K]) {
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < G; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += ld_cg(&partials[static_cast<size_t>(b) * K + k]);
  block_sum<K>(acc, red);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = acc[k];
}

// Graph path: publish this block's K sums; the last block to arrive forms
// the totals (valid in its thread 0) and returns true.
template <int K>
__device__ __forceinline__ bool grid_total_last(double (&v)[K], double* partials, unsigned int* ticket, double* red,
                                                double (&tot)[K]) {
  __shared__ bool s_last;
  block_sum<K>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[static_cast<size_t>(blockIdx.x) * K + k] = v[k];
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  sum_block_partials<K>(partials, gridDim.x, red, tot);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// ---------------------------------------------------------------- scalar steps
// Executed by one thread on the state (in global memory for the graph path,
// in each block's shared memory for the persistent one).

// The inner loop of mixed precision does not end the solve on a breakdown or
// a non-finite scalar of its complex64 recurrence: it asks for a refinement
// step instead (the FP64 step minimises the residual over its window, so a
// poor or non-finite inner iterate is rejected there, and a fresh inner
// process starts from the FP64 residual).  Returns true when the event was
// absorbed that way; the caller then leaves the status running.
__device__ __forceinline__ bool refine_absorb(SolverState* st) {
  if (st->method != kModeRefine) return false;
  st->aux[1].x = 1.0;
  return true;
}
// A refinement step is pending: the rest of the inner iteration is skipped.
__device__ __forceinline__ bool refine_step_pending(const SolverState* st) {
  return st->method == kModeRefine && st->aux[1].x != 0.0;
}

// after the initial residual: tot = (||b||^2, ||r||^2, (r^, r))
__device__ __forceinline__ void sc_init(SolverState* st, const double (&tot)[4], int use_x0) {
  const double bnorm = sqrt(tot[0]);
  st->bnorm = bnorm;
  if (use_x0) st->spmv_count += 1;
  int status = ST_RUNNING;
  if (!isfinite(bnorm)) {
    status = HELM_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    status = HELM_OK;  // b = 0: x = 0 (written by the tail)
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
      st->omega = make_double2(1.0, 0.0);
      st->alpha = make_double2(1.0, 0.0);
    }
  }
  st->phase = PH_RUN;
  st->status = status;
}

// after P2: tot = (r^, v)
__device__ __forceinline__ void sc_after_v(SolverState* st, const double (&tot)[2]) {
  st->iter += 1;
  st->spmv_count += 1;
  const double2 rv = make_double2(tot[0], tot[1]);
  int err = 0;
  if (!cfinite(rv)) {
    err = HELM_ERR_NONFINITE;
  } else if (czero(rv)) {
    err = HELM_ERR_BREAKDOWN;
  } else {
    const double2 alpha = cdiv_fast(st->rho, rv);
    if (!cfinite(alpha)) err = HELM_ERR_NONFINITE;
    else st->alpha = alpha;
  }
  if (err && !refine_absorb(st)) st->status = err;
}

// after P3: tot = ||s||^2; ||s|| / ||b|| <= tol compared squared
__device__ __forceinline__ void sc_after_s(SolverState* st, const double (&tot)[1]) {
  const double s2 = tot[0];
  const double bt = st->bnorm * st->tol;
  if (!isfinite(s2)) {
    if (!refine_absorb(st)) st->status = HELM_ERR_NONFINITE;
  } else if (st->method != kModeRefine && s2 <= bt * bt) {
    st->phase = PH_SCONV;
    st->relres = sqrt(s2) / st->bnorm;
  }
}

// after P4: tot = ((t, s), ||t||^2)
__device__ __forceinline__ void sc_after_t(SolverState* st, const double (&tot)[3]) {
  st->spmv_count += 1;
  const double2 ts = make_double2(tot[0], tot[1]);
  const double tt = tot[2];
  int err = 0;
  if (!cfinite(ts) || !isfinite(tt)) {
    err = HELM_ERR_NONFINITE;
  } else if (tt == 0.0) {
    err = HELM_ERR_BREAKDOWN;
  } else {
    const double inv_tt = 1.0 / tt;
    const double2 omega = make_double2(ts.x * inv_tt, ts.y * inv_tt);
    if (!cfinite(omega)) err = HELM_ERR_NONFINITE;
    else st->omega = omega;
  }
  if (err && !refine_absorb(st)) st->status = err;
}

// after P5: tot = ((r^, r), ||r||^2); `late` = the deadline has passed.
// With phase PH_SCONV (P5 only added alpha p to x) the solve is done.
__device__ __forceinline__ void sc_after_xr(SolverState* st, const double (&tot)[3], bool late) {
  // the inner loop of mixed precision runs on a scaled residual: b - A x ~ aux[2].x * r
  const double sc = st->method == kModeRefine ? st->aux[2].x : 1.0;
  const int phase = st->phase;
  const double2 alpha64 = st->alpha, omega64 = st->omega;
  int status = ST_RUNNING;
  if (phase == PH_SCONV) {
    status = HELM_OK;
    st->phase = PH_DONE;
  } else {
    // ||r|| / ||b|| <= tol compared squared; the square root is taken for the
    // report only when the loop stops
    const double r2 = tot[2];
    const double bt = st->bnorm * st->tol;
    bool stop_ok = r2 * (sc * sc) <= bt * bt;
    if (st->method == kModeRefine && isfinite(r2)) {
      // mixed precision: the recurrence never declares convergence; it asks
      // for a refinement step (FP64 residual, fresh process) when it has
      // dropped by inner_tol since the process began, looks converged, or
      // after kInnerMax iterations (complex64 BiCGStab can stagnate on
      // strongly indefinite systems; the step's minimal-residual length
      // keeps a poor inner iterate from increasing the FP64 residual)
      const double rn = sqrt(r2);
      const double cyc = st->aux[3].y;
      const bool dropped = cyc > 0.0 && cyc < 1.0 && rn <= cyc * st->aux[0].x;
      if (stop_ok || dropped || st->iter - static_cast<int>(st->aux[0].y) >= kInnerMax) st->aux[1].x = 1.0;
      stop_ok = false;
    }
    if (!isfinite(r2)) {
      status = refine_absorb(st) ? ST_RUNNING : HELM_ERR_NONFINITE;
    } else if (stop_ok) {
      status = HELM_OK;
    } else if (czero(omega64)) {
      status = refine_absorb(st) ? ST_RUNNING : HELM_ERR_BREAKDOWN;
    } else if (st->iter >= st->maxit) {
      status = HELM_ERR_NOT_CONVERGED;
    } else if (late) {
      status = HELM_ERR_TIMEOUT;
    } else {
      const double2 rho_new = make_double2(tot[0], tot[1]);
      // beta = (rho_new / rho) (alpha / omega) = (rho_new alpha) / (rho omega)
      const double2 beta = cdiv_fast(cmul(rho_new, alpha64), cmul(st->rho, omega64));
      if (!cfinite(rho_new) || !cfinite(beta)) {
        status = refine_absorb(st) ? ST_RUNNING : HELM_ERR_NONFINITE;
        st->iter += 1;
      } else if (czero(rho_new)) {
        status = refine_absorb(st) ? ST_RUNNING : HELM_ERR_BREAKDOWN;
        st->iter += 1;
      } else {
        st->rho = rho_new;
        st->beta = beta;
      }
    }
    if (status != ST_RUNNING) st->relres = sqrt(tot[2]) * sc / st->bnorm;
  }
  st->status = status;
}

// ---------------------------------------------------------------- phases
// The per-thread work of each phase, shared by the graph kernels and the
// persistent kernel.  Rows are those of SliceRows; each phase returns this
// thread's partial sums.

// init without x0: x = 0, r = r^ = b, p = v = 0; (||b||^2, ||r||^2, (r^, r))
template <class V>
__device__ __forceinline__ void ph_init_zero(const KArgs<V>& a, typename Prec<V>::S (&acc)[2],
                                             typename Prec<V>::C& d) {
  const V z = vzero<V>();
  for (SliceRows q(a.A.n); q.active(); q.advance()) {
    const int32_t i = q.row();
    if (i >= a.A.n) continue;
    const V bi = a.b[i];
    a.x[i] = z;
    a.r[i] = bi;
    a.rh[i] = bi;
    a.p[i] = z;
    a.v[i] = z;
    acc[0] = nrm_acc(acc[0], bi);
    d = dot_acc(d, bi, bi);
  }
  acc[1] = acc[0];
}

// init with x0 (SpMV epilogue): r = r^ = b - A x, p = v = 0
template <class V>
struct InitEpi {
  const V* b;
  V *r, *rh, *p, *v;
  typename Prec<V>::S part[2];
  typename Prec<V>::C d;
  V bpre;
  __device__ __forceinline__ void prefetch(int32_t i) { bpre = b[i]; }
  __device__ __forceinline__ void row(int32_t i, V ax) {
    const V bi = bpre;
    const V ri = csub(bi, ax);
    r[i] = ri;
    rh[i] = ri;
    p[i] = vzero<V>();
    v[i] = vzero<V>();
    part[0] = nrm_acc(part[0], bi);
    part[1] = nrm_acc(part[1], ri);
    d = dot_acc(d, ri, ri);
  }
};
template <class V>
__device__ __forceinline__ InitEpi<V> init_epi(const KArgs<V>& a) {
  return InitEpi<V>{a.b, a.r, a.rh, a.p, a.v, {Prec<V>::szero(), Prec<V>::szero()}, Prec<V>::czero(), vzero<V>()};
}

// P1: p = r + beta (p - omega v); the next row's loads are issued before
// this row is computed
template <class V>
__device__ __forceinline__ void ph_p(const KArgs<V>& a, V beta, V omega) {
  SliceRows q(a.A.n);
  int32_t i = q.row();
  if (!q.active() || i >= a.A.n) return;
  V v0 = a.v[i], p0 = a.p[i], r0 = a.r[i];
  for (;;) {
    SliceRows nq = q;
    const bool more = nq.advance() && nq.row() < a.A.n;
    const int32_t j = nq.row();
    V v1 = v0, p1 = p0, r1 = r0;
    if (more) {
      v1 = a.v[j];
      p1 = a.p[j];
      r1 = a.r[j];
    }
    a.p[i] = cfma(beta, cfms(omega, v0, p0), r0);
    if (!more) break;
    v0 = v1;
    p0 = p1;
    r0 = r1;
    i = j;
    q = nq;
  }
}

// P2 epilogue: v = A p, (r^, v)
template <class V>
struct VEpi {
  V* v;
  const V* rhp;
  typename Prec<V>::C part;
  V rh;
  __device__ __forceinline__ void prefetch(int32_t i) { rh = rhp[i]; }
  __device__ __forceinline__ void row(int32_t i, V ax) {
    v[i] = ax;
    part = dot_acc(part, rh, ax);
  }
};
template <class V>
__device__ __forceinline__ VEpi<V> v_epi(const KArgs<V>& a) {
  return VEpi<V>{a.v, a.rh, Prec<V>::czero(), vzero<V>()};
}

// P3: s = r - alpha v, ||s||^2
template <class V>
__device__ __forceinline__ typename Prec<V>::S ph_s(const KArgs<V>& a, V alpha) {
  using S = typename Prec<V>::S;
  S acc = Prec<V>::szero();
  SliceRows q(a.A.n);
  int32_t i = q.row();
  if (!q.active() || i >= a.A.n) return acc;
  V v0 = a.v[i], r0 = a.r[i];
  for (;;) {
    SliceRows nq = q;
    const bool more = nq.advance() && nq.row() < a.A.n;
    const int32_t j = nq.row();
    V v1 = v0, r1 = r0;
    if (more) {
      v1 = a.v[j];
      r1 = a.r[j];
    }
    const V s0 = cfms(alpha, v0, r0);
    a.s[i] = s0;
    acc = nrm_acc(acc, s0);
    if (!more) break;
    v0 = v1;
    r0 = r1;
    i = j;
    q = nq;
  }
  return acc;
}

// P4 epilogue: t = A s, (t, s), ||t||^2
template <class V>
struct TEpi {
  V* t;
  const V* sp;
  typename Prec<V>::C ts;
  typename Prec<V>::S tt;
  V si;
  __device__ __forceinline__ void prefetch(int32_t i) { si = sp[i]; }
  __device__ __forceinline__ void row(int32_t i, V ax) {
    t[i] = ax;
    ts = dot_acc(ts, ax, si);
    tt = nrm_acc(tt, ax);
  }
};
template <class V>
__device__ __forceinline__ TEpi<V> t_epi(const KArgs<V>& a) {
  return TEpi<V>{a.t, a.s, Prec<V>::czero(), Prec<V>::szero(), vzero<V>()};
}

// P5: x += alpha p + omega s, r = s - omega t; (r^, r), ||r||^2.  With
// sconv (the solve stopped at s) only x += alpha p.
template <class V>
__device__ __forceinline__ void ph_xr(const KArgs<V>& a, V alpha, V omega, bool sconv, typename Prec<V>::C& rr,
                                      typename Prec<V>::S& r2) {
  SliceRows q(a.A.n);
  int32_t i = q.row();
  if (!q.active() || i >= a.A.n) return;
  if (sconv) {
    for (; q.active(); q.advance()) {
      i = q.row();
      if (i < a.A.n) a.x[i] = cfma(alpha, a.p[i], a.x[i]);
    }
    return;
  }
  V s0 = a.s[i], x0 = a.x[i], p0 = a.p[i], t0 = a.t[i], h0 = a.rh[i];
  for (;;) {
    SliceRows nq = q;
    const bool more = nq.advance() && nq.row() < a.A.n;
    const int32_t j = nq.row();
    V sn = s0, xn = x0, pn = p0, tn = t0, hn = h0;
    if (more) {
      sn = a.s[j];
      xn = a.x[j];
      pn = a.p[j];
      tn = a.t[j];
      hn = a.rh[j];
    }
    a.x[i] = cfma(omega, s0, cfma(alpha, p0, x0));
    const V r0 = cfms(omega, t0, s0);
    a.r[i] = r0;
    rr = dot_acc(rr, h0, r0);
    r2 = nrm_acc(r2, r0);
    if (!more) break;
    s0 = sn;
    x0 = xn;
    p0 = pn;
    t0 = tn;
    h0 = hn;
    i = j;
    q = nq;
  }
}

// ---------------------------------------------------------------- graph kernels

template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_init(KArgs<V> a) {
  pdl_enter();
  using S = typename Prec<V>::S;
  using C = typename Prec<V>::C;
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  S acc[2] = {Prec<V>::szero(), Prec<V>::szero()};
  C d = Prec<V>::czero();
  if (use_x0) {
    InitEpi<V> epi = init_epi<V>(a);
    spmv_run<V>(a.A, a.x, epi, nullptr, a.dev_err);
    acc[0] = epi.part[0];
    acc[1] = epi.part[1];
    d = epi.d;
  } else {
    ph_init_zero<V>(a, acc, d);
  }
  const double2 dd = to_d2(d);
  double part[4] = {to_d(acc[0]), to_d(acc[1]), dd.x, dd.y};
  double tot[4];
  if (!grid_total_last<4>(part, a.partials, a.tickets + TK_INIT, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_init(st, tot, use_x0);
  set_cond(a, st->status == ST_RUNNING);
}

// K1: p = r + beta (p - omega v)
template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_p(KArgs<V> a) {
  pdl_enter();
  const SolverState* st = a.st;
  if (st->status != ST_RUNNING || refine_step_pending(st)) return;
  ph_p<V>(a, Prec<V>::cvt(st->beta), Prec<V>::cvt(st->omega));
}

// K2: v = A p, (r^, v) -> alpha
template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_v(KArgs<V> a) {
  pdl_enter();
  __shared__ double red[32 * 2];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING || refine_step_pending(st)) return;
  VEpi<V> epi = v_epi<V>(a);
  spmv_run<V>(a.A, a.p, epi, nullptr, a.dev_err);
  const double2 pd = to_d2(epi.part);
  double part[2] = {pd.x, pd.y};
  double tot[2];
  if (!grid_total_last<2>(part, a.partials, a.tickets + TK_V, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_after_v(st, tot);
}

// K3: s = r - alpha v, ||s||
template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_s(KArgs<V> a) {
  pdl_enter();
  __shared__ double red[32];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING || refine_step_pending(st)) return;
  double part[1] = {to_d(ph_s<V>(a, Prec<V>::cvt(st->alpha)))};
  double tot[1];
  if (!grid_total_last<1>(part, a.partials, a.tickets + TK_S, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_after_s(st, tot);
}

// K4: t = A s, (t, s), (t, t) -> omega
template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_t(KArgs<V> a) {
  pdl_enter();
  using S = typename Prec<V>::S;
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING || st->phase != PH_RUN || refine_step_pending(st)) return;
  TEpi<V> epi = t_epi<V>(a);
  spmv_run<V>(a.A, a.s, epi, nullptr, a.dev_err);
  const double2 tsd = to_d2(epi.ts);
  double part[3] = {tsd.x, tsd.y, to_d(epi.tt)};
  double tot[3];
  if (!grid_total_last<3>(part, a.partials, a.tickets + TK_T, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_after_t(st, tot);
}

// K5: x += alpha p + omega s, r = s - omega t; stop test; rho, beta
template <class V>
__global__ void __launch_bounds__(kSolverThreads, kSolverMinBlocks) k_xr(KArgs<V> a) {
  pdl_enter();
  using S = typename Prec<V>::S;
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, false);
    return;
  }
  if (refine_step_pending(st)) {  // mixed precision: the inner loop ends for the refinement step
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, false);
    return;
  }
  typename Prec<V>::C rr = Prec<V>::czero();
  typename Prec<V>::S r2 = Prec<V>::szero();
  ph_xr<V>(a, Prec<V>::cvt(st->alpha), Prec<V>::cvt(st->omega), st->phase == PH_SCONV, rr, r2);
  const double2 rrd = to_d2(rr);
  double part[3] = {rrd.x, rrd.y, to_d(r2)};
  double tot[3];
  if (!grid_total_last<3>(part, a.partials, a.tickets + TK_XR, red, tot)) return;
  if (threadIdx.x != 0) return;
  sc_after_xr(st, tot, deadline_passed(st));
  set_cond(a, st->status == ST_RUNNING && !refine_step_pending(st));
}

// Solver grid: one wave of the solver kernels -- the blocks that fit on every
// SM at once for each of `fns` (so that none runs a second wave), times the
// SMs, at most enough blocks for one warp per slice.  Every kernel of a solve
// (graph or persistent) runs on this grid: the grid fixes which thread owns
// which row and so the order of every partial sum.
inline helm_status persistent_grid(std::initializer_list<const void*> fns, int threads, size_t smem,
                                   int num_sms, int64_t units, int* grid) {
  int per_sm = 1 << 30;
  for (const void* fn : fns) {
    int b = 0;
    HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem));
    per_sm = b < per_sm ? b : per_sm;
  }
  if (per_sm < 1) per_sm = 1;
  int64_t g = static_cast<int64_t>(per_sm) * num_sms;
  if (units < g) g = units < 1 ? 1 : units;
  *grid = static_cast<int>(g);
  return HELM_OK;
}

template <class V>
struct KShapes {
  int grid;     // every kernel of the loop, init and tail included
  int threads;  // threads per block (a multiple of 32)
};

template <class V>
inline void enqueue_init(const KArgs<V>& a, const KShapes<V>& sh, cudaStream_t s) {
  k_init<V><<<sh.grid, sh.threads, 0, s>>>(a);
}

// A loop kernel launched with programmatic stream serialization (a
// programmatic edge from the kernel before it when captured into a graph);
// see pdl_enter.
template <class V>
inline void launch_loop_kernel(void (*kernel)(KArgs<V>), const KArgs<V>& a, const KShapes<V>& sh, cudaStream_t s) {
#if HELM_PDL
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(sh.grid));
  cfg.blockDim = dim3(static_cast<unsigned>(sh.threads));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, a);  // errors surface at the caller's cudaGetLastError
#else
  kernel<<<sh.grid, sh.threads, 0, s>>>(a);
#endif
}

template <class V>
inline void enqueue_body(const KArgs<V>& a, const KShapes<V>& sh, cudaStream_t s) {
  launch_loop_kernel<V>(k_p<V>, a, sh, s);
  launch_loop_kernel<V>(k_v<V>, a, sh, s);
  launch_loop_kernel<V>(k_s<V>, a, sh, s);
  launch_loop_kernel<V>(k_t<V>, a, sh, s);
  launch_loop_kernel<V>(k_xr<V>, a, sh, s);
}

template <class V>
inline helm_status prepare_krylov_kernels() {
  return HELM_OK;
}

// Shape of a slice-parallel grid: one block per SM (blocks_per_sm with
// smaller blocks), never more blocks than slices, and per block just enough
// warps (at most max_threads / 32) for one slice per warp in each round.
struct SliceShape {
  int grid, threads;
};
inline SliceShape slice_shape(int32_t n, int num_sms, int max_threads, int blocks_per_sm, bool full = false) {
  const int64_t nsl = std::max<int64_t>((static_cast<int64_t>(n) + 31) / 32, 1);
  const int64_t grid = std::min<int64_t>(static_cast<int64_t>(num_sms) * blocks_per_sm, nsl);
  const int64_t wmax = std::max(max_threads / 32, 1);
  // rounds at the widest block, then (unless `full`) the fewest warps that
  // keep that many rounds: every round (the last one too) nearly full
  const int64_t rounds = (nsl + grid * wmax - 1) / (grid * wmax);
  const int64_t warps =
      full ? std::min<int64_t>((nsl + grid - 1) / grid, wmax) : std::min<int64_t>((nsl + grid * rounds - 1) / (grid * rounds), wmax);
  return SliceShape{static_cast<int>(grid), static_cast<int>(32 * std::max<int64_t>(warps, 1))};
}

// Shape of the solver's grid: blocks of at most HELM_SOLVER_THREADS threads,
// HELM_SOLVER_BPS blocks per SM.  A build-time choice, not a run-time one:
// the shape fixes which thread owns which row and so the rounding of every
// reduction, and a solve must give the same bits on every run.
// Measured on the 120x60x50 cavity (graph loop, us per iteration): 1024 x 1
// (832 threads used) 144.6, 512 x 2 138.4, 256 x 4 140.8.
#ifndef HELM_SOLVER_THREADS
#define HELM_SOLVER_THREADS 512
#endif
#ifndef HELM_SOLVER_BPS
#define HELM_SOLVER_BPS 2
#endif
// The complex64 solver (the inner solves of mixed precision, HBM-bound) may
// take another shape.
#ifndef HELM_SOLVER32_THREADS
#define HELM_SOLVER32_THREADS HELM_SOLVER_THREADS
#endif
#ifndef HELM_SOLVER32_BPS
#define HELM_SOLVER32_BPS HELM_SOLVER_BPS
#endif

// Grid of the solver's kernels; the kernels (and `extra` ones: the tail, the
// persistent kernel) must fit HELM_SOLVER_BPS such blocks per SM.
template <class V>
inline helm_status krylov_shapes(helm_csr A, KShapes<V>* sh, std::initializer_list<const void*> extra = {}) {
  std::vector<const void*> fns = {reinterpret_cast<const void*>(&k_init<V>), reinterpret_cast<const void*>(&k_p<V>),
                                  reinterpret_cast<const void*>(&k_v<V>),    reinterpret_cast<const void*>(&k_s<V>),
                                  reinterpret_cast<const void*>(&k_t<V>),    reinterpret_cast<const void*>(&k_xr<V>)};
  for (const void* f : extra) fns.push_back(f);
  const bool c64 = std::is_same<V, float2>::value;
  const int bps = c64 ? HELM_SOLVER32_BPS : HELM_SOLVER_BPS;
  const SliceShape ss = slice_shape(A->n, A->num_sms, c64 ? HELM_SOLVER32_THREADS : HELM_SOLVER_THREADS, bps);
  for (const void* fn : fns) {
    int b = 0;
    HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, ss.threads, 0));
    if (b < bps) return HELM_ERR_CUDA;
  }
  sh->grid = ss.grid;
  sh->threads = ss.threads;
  return HELM_OK;
}

// Iterations (loop bodies) per pass of the while node: each pass re-launches
// the body graph, so several iterations per pass save that cost (measured:
// 164.5 -> 161.3 -> 159.8 us per BiCGStab iteration for 1, 2, 4); once the
// solve has finished, the remaining kernels of a pass return at once.
#ifndef HELM_BODY_UNROLL
#define HELM_BODY_UNROLL 4
#endif
constexpr int kBodyUnroll = HELM_BODY_UNROLL;

// Build a graph  init -> while(body) -> tail.  Each callable enqueues its
// kernels on the capture stream with the loop's conditional handle:
// init(cond, stream), body(cond, stream), tail(cond, stream).
template <class Init, class Body, class Tail>
helm_status build_while_graph(Init init, Body body, Tail tail, GraphEntry* out) {
  cudaStream_t cs = nullptr;
  HELM_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  helm_status result = HELM_ERR_CUDA;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle cond;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    init(cond, cs);
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
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    for (int u = 0; u < kBodyUnroll; ++u) body(cond, cs);
    if (cudaStreamEndCapture(cs, &tmp) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      break;
    tail(cond, cs);
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

// BiCGStab graph  init -> while(K1..K5) -> tail  for fixed vectors.
template <class V, class Tail>
helm_status build_krylov_graph(const KArgs<V>& base, const KShapes<V>& sh, Tail tail, GraphEntry* out) {
  auto with = [&](cudaGraphConditionalHandle cond) {
    KArgs<V> a = base;
    a.cond = cond;
    a.has_cond = 1;
    return a;
  };
  return build_while_graph([&](cudaGraphConditionalHandle c, cudaStream_t s) { enqueue_init(with(c), sh, s); },
                           [&](cudaGraphConditionalHandle c, cudaStream_t s) { enqueue_body(with(c), sh, s); },
                           [&](cudaGraphConditionalHandle c, cudaStream_t s) { tail(with(c), s); }, out);
}

// Run init -> loop -> tail once: through the cached graph when there is one,
// else host-driven (chunks of 16 iterations, state polled between chunks).
template <class V, class Tail>
helm_status run_krylov(helm_csr A, const KArgs<V>& a, const KShapes<V>& sh, GraphEntry* g, Tail tail,
                       cudaStream_t s) {
  if (g && g->exec) {
    HELM_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    return HELM_OK;
  }
  enqueue_init(a, sh, s);
  HELM_CUDA_TRY(cudaGetLastError());
  for (;;) {
    for (int k = 0; k < 16; ++k) enqueue_body(a, sh, s);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaMemcpyAsync(A->state_host, a.st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (A->state_host->status != ST_RUNNING) break;
  }
  tail(a, s);
  HELM_CUDA_TRY(cudaGetLastError());
  return HELM_OK;
}

}  // namespace helm
