// BiCGStab kernels with device-resident scalars, generic over the vector
// precision (complex128 for the FP64 solver, complex64 for the inner solve of
// mixed precision).  Section 4 of the paper: P-BiCGSTAB with residual
// tolerance, zero initial guess and an iteration cap; identity preconditioner
// (right Jacobi runs the same kernels on A D^-1); the recurrence of van der
// Vorst 1992 / Saad 2003 Algorithm 7.7 with conjugated inner products.
//
// One iteration is five kernels; each dot product the recurrence needs is
// fused into the kernel that produces its operands, and the scalar it feeds
// is formed in FP64 on the device by the last block to finish (ticket
// counter):
//   K1  p = r + beta (p - omega v)
//   K2  v = A p          + (r^, v)        -> alpha = rho / (r^, v)
//   K3  s = r - alpha v  + ||s||^2        -> stop at s if ||s|| / ||b|| <= tol
//   K4  t = A s          + (t, s), ||t||^2 -> omega = (t, s) / (t, t)
//   K5  x += alpha p + omega s, r = s - omega t + (r^, r), ||r||^2
//                                         -> stop test, rho, beta
// For complex64 the products and each thread's partial sums are FP32; block
// and grid sums and every scalar of the recurrence are FP64.
//
// The loop runs inside one CUDA graph: an init kernel, a conditional WHILE
// node whose body is four iterations of K1..K5 (K5's last block sets the
// condition) and, for the FP64 solver, a tail kernel that recomputes the true
// residual b - A x.
#pragma once

#include <cstring>
#include <initializer_list>
#include <utility>

#include "common.cuh"
#include "internal.hpp"
#include "spmv.cuh"

namespace helm {

// The complex128 matrix a solve runs on: A, or A D^-1 under right Jacobi.
inline CsrDev<double2> csr_for(helm_csr A, const helm_opts& o) {
  if (o.precond == HELM_PRECOND_JACOBI)
    return CsrDev<double2>{A->n, A->nnz, A->rowptr, A->colind, A->jac_vals, A->jac_real_blk, A->jac_vals_re};
  return CsrDev<double2>{A->n, A->nnz, A->rowptr, A->colind, static_cast<const double2*>(A->vals), A->real_blk,
                         A->vals_re};
}

// SolverState::method of the Krylov loop: plain, or the inner loop of the
// mixed-precision solve (aux[0] = (||r|| when the process began, in its
// scale; iteration it began), aux[1].x = refinement step due, aux[2].x =
// scale of the inner residual, aux[3] = (steps in a row without a 2x gain,
// inner_tol)).
constexpr int32_t kModePlain = 0;
constexpr int32_t kModeRefine = 1;
constexpr int kInnerMax = 50000;  // inner iterations per refinement step at most

template <class V> struct Prec;
template <> struct Prec<double2> {
  using S = double;
  static constexpr int R = Engine<double2>::kThreads;  // threads per SpMV block
  __device__ static __forceinline__ double2 cvt(double2 z) { return z; }
};
template <> struct Prec<float2> {
  using S = float;
  static constexpr int R = Engine<float2>::kThreads;  // threads per SpMV block
  __device__ static __forceinline__ float2 cvt(double2 z) {
    return make_float2(static_cast<float>(z.x), static_cast<float>(z.y));
  }
};

template <class V>
struct KArgs {
  CsrDev<V> A;
  const V* b;
  V* x;
  V *r, *rh, *p, *v, *s, *t;
  SolverState* st;
  double* partials;
  unsigned int* tickets;
  unsigned int* gtickets;  // group counters of the two-level sums of K2 and K4
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

// r = b - A x (or r = b, x = 0), r^ = r, p = v = 0; ||b||, ||r||, rho.
template <class V>
__global__ void __launch_bounds__(Prec<V>::R) k_init(KArgs<V> a) {
  using S = typename Prec<V>::S;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  S acc[4] = {S(0), S(0), S(0), S(0)};  // |b|^2, |r|^2, (r, r)
  if (use_x0) {
    struct Epi {
      const KArgs<V>* a;
      S part[4];
      V bpre;
      __device__ __forceinline__ void prefetch(int32_t i) { bpre = a->b[i]; }
      __device__ __forceinline__ void row(int32_t i, V ax) {
        const V bi = bpre;
        const V ri = csub(bi, ax);
        a->r[i] = ri;
        a->rh[i] = ri;
        a->p[i] = vzero<V>();
        a->v[i] = vzero<V>();
        part[0] = cabs2_acc(bi, part[0]);
        part[1] = cabs2_acc(ri, part[1]);
        V d;
        d.x = part[2];
        d.y = part[3];
        d = cfma_conj(ri, ri, d);
        part[2] = d.x;
        part[3] = d.y;
      }
    } epi{&a, {S(0), S(0), S(0), S(0)}, vzero<V>()};
    spmv_run<V>(a.A, a.x, epi, smem, a.dev_err);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = epi.part[k];
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const V bi = a.b[i];
      a.x[i] = vzero<V>();
      a.r[i] = bi;
      a.rh[i] = bi;
      a.p[i] = vzero<V>();
      a.v[i] = vzero<V>();
      acc[0] = cabs2_acc(bi, acc[0]);
      V d;
      d.x = acc[2];
      d.y = acc[3];
      d = cfma_conj(bi, bi, d);
      acc[2] = d.x;
      acc[3] = d.y;
    }
    acc[1] = acc[0];
  }
  double part[4] = {double(acc[0]), double(acc[1]), double(acc[2]), double(acc[3])};
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
    status = HELM_OK;  // b = 0: x = 0 (written by the tail kernel / caller)
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

// Element-wise kernels: one wave of blocks (grid = resident blocks), each
// thread takes two elements per step with all loads issued before the
// arithmetic, so the 64-clock FP64 latency and the memory latency of one
// element overlap the other's.
constexpr int kVecThreads = 256;
// At most this many element-wise blocks per SM (measured on the 120x60x50
// cavity: 3 -> 161.4, 4 -> 158.2, all that fit (6 for K1, K3) -> 159.1 us per
// iteration).
#ifndef HELM_VEC_MAX_BPS
#define HELM_VEC_MAX_BPS 4
#endif
constexpr int kVecMaxBlocksPerSm = HELM_VEC_MAX_BPS;

// Rows of an element-wise kernel: block b takes the contiguous range
// [b n / G, (b + 1) n / G) (sizes differ by at most one, so every SM of a
// one-wave grid gets the same work), its threads striding by blockDim.
struct RowChunk {
  int32_t begin, end, step;
  __device__ __forceinline__ explicit RowChunk(int32_t n)
      : begin(static_cast<int32_t>(static_cast<int64_t>(blockIdx.x) * n / gridDim.x)),
        end(static_cast<int32_t>((static_cast<int64_t>(blockIdx.x) + 1) * n / gridDim.x)),
        step(static_cast<int32_t>(blockDim.x)) {}
  __device__ __forceinline__ int32_t first() const { return begin + static_cast<int32_t>(threadIdx.x); }
};

// K1: p = r + beta (p - omega v)
template <class V>
__global__ void __launch_bounds__(kVecThreads) k_p(KArgs<V> a) {
  const SolverState* st = a.st;
  // K2 may start staging the matrix at once (it waits for p itself); K1 is
  // launched the ordinary way, after the previous iteration has completed
  pdl_launch_dependents();
  if (st->status != ST_RUNNING) return;
  const V beta = Prec<V>::cvt(st->beta), omega = Prec<V>::cvt(st->omega);
  const RowChunk c(a.A.n);
  int32_t i = c.first();
  if (i >= c.end) return;
  V v0 = a.v[i], p0 = a.p[i], r0 = a.r[i];
  for (;;) {
    // the next row's loads are in flight while this row is computed
    const int32_t j = i + c.step;
    const bool more = j < c.end;
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
  }
}

// K2: v = A p, (r^, v) -> alpha
template <class V>
__global__ void __launch_bounds__(Prec<V>::R) k_v(KArgs<V> a) {
  using S = typename Prec<V>::S;
  extern __shared__ __align__(16) unsigned char smem[];
  // the block sums reuse the staging buffer once the tiles are done (less
  // static shared memory: one more block per SM)
  double* red = reinterpret_cast<double*>(smem);
  SolverState* st = a.st;
  struct Epi {
    const KArgs<V>* a;
    V part;
    V rh;
    __device__ __forceinline__ void prefetch(int32_t i) { rh = a->rh[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      a->v[i] = ax;
      part = cfma_conj(rh, ax, part);
    }
  } epi{&a, vzero<V>(), vzero<V>()};
  // the first tile's copy is in flight while p (the previous kernel's
  // output) is waited for
  bool go = false;
  spmv_run<V>(a.A, a.p, epi, smem, a.dev_err, [&]() {
    pdl_wait();
    pdl_launch_dependents();
    go = st->status == ST_RUNNING;
    return go;
  });
  if (!go) return;
  double part[2] = {double(epi.part.x), double(epi.part.y)};
  double tot[2];
  // many blocks of few threads: the two-level sum keeps the last block short
  if (!grid_sum_last2<2>(part, a.partials, a.tickets + TK_V, a.gtickets, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->iter += 1;
  st->spmv_count += 1;
  const double2 rv = make_double2(tot[0], tot[1]);
  if (!cfinite(rv)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (czero(rv)) {
    st->status = HELM_ERR_BREAKDOWN;
  } else {
    const double2 alpha = cdiv_fast(st->rho, rv);
    if (!cfinite(alpha)) st->status = HELM_ERR_NONFINITE;
    else st->alpha = alpha;
  }
}

// K3: s = r - alpha v, ||s||
template <class V>
__global__ void __launch_bounds__(kVecThreads) k_s(KArgs<V> a) {
  using S = typename Prec<V>::S;
  __shared__ double red[32];
  SolverState* st = a.st;
  const RowChunk c(a.A.n);
  int32_t i = c.first();
  // r was final before the previous kernel started; v and alpha are its output
  V r0 = vzero<V>();
  if (i < c.end) r0 = a.r[i];
  pdl_wait();
  pdl_launch_dependents();
  if (st->status != ST_RUNNING) return;
  const V alpha = Prec<V>::cvt(st->alpha);
  S acc = S(0);
  V v0 = vzero<V>();
  if (i < c.end) v0 = a.v[i];
  while (i < c.end) {
    const int32_t j = i + c.step;
    const bool more = j < c.end;
    V v1 = v0, r1 = r0;
    if (more) {
      v1 = a.v[j];
      r1 = a.r[j];
    }
    const V s0 = cfms(alpha, v0, r0);
    a.s[i] = s0;
    acc = cabs2_acc(s0, acc);
    v0 = v1;
    r0 = r1;
    i = j;
  }
  double part[1] = {double(acc)};
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_S, red, tot)) return;
  if (threadIdx.x != 0) return;
  // ||s|| / ||b|| <= tol compared squared: no square root on the critical path
  const double s2 = tot[0];
  const double bt = st->bnorm * st->tol;
  if (!isfinite(s2)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (st->method != kModeRefine && s2 <= bt * bt) {
    st->phase = PH_SCONV;
    st->relres = sqrt(s2) / st->bnorm;
  }
}

// K4: t = A s, (t, s), (t, t) -> omega
template <class V>
__global__ void __launch_bounds__(Prec<V>::R) k_t(KArgs<V> a) {
  using S = typename Prec<V>::S;
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);  // the staging buffer, once the tiles are done
  SolverState* st = a.st;
  struct Epi {
    const KArgs<V>* a;
    V ts;
    S tt;
    V si;
    __device__ __forceinline__ void prefetch(int32_t i) { si = a->s[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      a->t[i] = ax;
      ts = cfma_conj(ax, si, ts);
      tt = cabs2_acc(ax, tt);
    }
  } epi{&a, vzero<V>(), S(0), vzero<V>()};
  // the first tile's copy is in flight while s and the phase (the previous
  // kernel's output) are waited for
  bool go = false;
  spmv_run<V>(a.A, a.s, epi, smem, a.dev_err, [&]() {
    pdl_wait();
    pdl_launch_dependents();
    go = st->status == ST_RUNNING && st->phase == PH_RUN;
    return go;
  });
  if (!go) return;
  double part[3] = {double(epi.ts.x), double(epi.ts.y), double(epi.tt)};
  double tot[3];
  if (!grid_sum_last2<3>(part, a.partials, a.tickets + TK_T, a.gtickets + kGroupTickets, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double2 ts = make_double2(tot[0], tot[1]);
  const double tt = tot[2];
  if (!cfinite(ts) || !isfinite(tt)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (tt == 0.0) {
    st->status = HELM_ERR_BREAKDOWN;
  } else {
    const double inv_tt = 1.0 / tt;
    const double2 omega = make_double2(ts.x * inv_tt, ts.y * inv_tt);
    if (!cfinite(omega)) st->status = HELM_ERR_NONFINITE;
    else st->omega = omega;
  }
}

// K5: x += alpha p + omega s, r = s - omega t; stop test; rho, beta
template <class V>
__global__ void __launch_bounds__(kVecThreads) k_xr(KArgs<V> a) {
  using S = typename Prec<V>::S;
  __shared__ double red[32 * 3];
  SolverState* st = a.st;
  const RowChunk c(a.A.n);
  int32_t i = c.first();
  // x, p, s and r^ were final before the previous kernel started; t, omega
  // and the status are its output
  V s0 = vzero<V>(), x0 = vzero<V>(), p0 = vzero<V>(), h0 = vzero<V>();
  if (i < c.end) {
    s0 = a.s[i];
    x0 = a.x[i];
    p0 = a.p[i];
    h0 = a.rh[i];
  }
  pdl_wait();
  pdl_launch_dependents();
  const int status0 = st->status;
  if (status0 != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(a, false);
    return;
  }
  const double2 alpha64 = st->alpha, omega64 = st->omega;
  const V alpha = Prec<V>::cvt(alpha64), omega = Prec<V>::cvt(omega64);
  const int phase = st->phase;
  V rr = vzero<V>();
  S r2 = S(0);
  if (phase == PH_SCONV) {
    for (; i < c.end; i += c.step) a.x[i] = cfma(alpha, a.p[i], a.x[i]);
  } else {
    V t0 = vzero<V>();
    if (i < c.end) t0 = a.t[i];
    while (i < c.end) {
      const int32_t j = i + c.step;
      const bool more = j < c.end;
      V s1 = s0, x1 = x0, p1 = p0, t1 = t0, h1 = h0;
      if (more) {
        s1 = a.s[j];
        x1 = a.x[j];
        p1 = a.p[j];
        t1 = a.t[j];
        h1 = a.rh[j];
      }
      a.x[i] = cfma(omega, s0, cfma(alpha, p0, x0));
      const V r0 = cfms(omega, t0, s0);
      a.r[i] = r0;
      rr = cfma_conj(h0, r0, rr);
      r2 = cabs2_acc(r0, r2);
      s0 = s1;
      x0 = x1;
      p0 = p1;
      t0 = t1;
      h0 = h1;
      i = j;
    }
  }
  double part[3] = {double(rr.x), double(rr.y), double(r2)};
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_XR, red, tot)) return;
  if (threadIdx.x != 0) return;
  // the inner loop of mixed precision runs on a scaled residual: b - A x ~ aux[2].x * r
  const double sc = st->method == kModeRefine ? st->aux[2].x : 1.0;
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
      status = HELM_ERR_NONFINITE;
    } else if (stop_ok) {
      status = HELM_OK;
    } else if (czero(omega64)) {
      status = HELM_ERR_BREAKDOWN;
    } else if (st->iter >= st->maxit) {
      status = HELM_ERR_NOT_CONVERGED;
    } else if (deadline_passed(st)) {
      status = HELM_ERR_TIMEOUT;
    } else {
      const double2 rho_new = make_double2(tot[0], tot[1]);
      // beta = (rho_new / rho) (alpha / omega) = (rho_new alpha) / (rho omega)
      const double2 beta = cdiv_fast(cmul(rho_new, alpha64), cmul(st->rho, omega64));
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
  if (phase != PH_SCONV && status != ST_RUNNING) st->relres = sqrt(tot[2]) * sc / st->bnorm;
  st->status = status;
  set_cond(a, status == ST_RUNNING);
}

template <class V>
struct KShapes {
  int spmv_grid;                // K2 and K4
  int init_grid;                // the init kernel
  int vec_grid;
  int grid_p, grid_s, grid_xr;  // one wave of each element-wise kernel
};

// Persistent grid shared by `fns`: the blocks that fit on every SM at once
// for each of them (so that none runs a second wave, which would leave most
// of the GPU idle while it finishes), times the SMs, at most `units`.
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
inline void enqueue_init(const KArgs<V>& a, const KShapes<V>& sh, cudaStream_t s) {
  k_init<V><<<sh.init_grid, Prec<V>::R, Engine<V>::kSmem, s>>>(a);
}
// Launch with programmatic stream serialization: the kernel may start while
// its predecessor finishes (it calls pdl_wait() before it reads that
// kernel's output).  Launch errors surface through cudaGetLastError().
// Measured on GB300 inside the solver graph: 162.5 us per BiCGStab iteration
// without the attribute, 179.1 us with it, so it is off; the kernels' waits
// are no-ops then.
#ifndef HELM_PDL
#define HELM_PDL 0
#endif
template <class... P, class... Args>
inline void launch_dependent(void (*kern)(P...), int grid, int block, size_t smem, cudaStream_t s,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(static_cast<unsigned>(block));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = HELM_PDL ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <class V>
inline void enqueue_body(const KArgs<V>& a, const KShapes<V>& sh, cudaStream_t s) {
  constexpr size_t smem = Engine<V>::kSmem;
  k_p<V><<<sh.grid_p, kVecThreads, 0, s>>>(a);
  launch_dependent(k_v<V>, sh.spmv_grid, Prec<V>::R, smem, s, a);
  launch_dependent(k_s<V>, sh.grid_s, kVecThreads, 0, s, a);
  launch_dependent(k_t<V>, sh.spmv_grid, Prec<V>::R, smem, s, a);
  launch_dependent(k_xr<V>, sh.grid_xr, kVecThreads, 0, s, a);
}

template <class V>
inline helm_status prepare_krylov_kernels() {
  constexpr size_t smem = Engine<V>::kSmem;
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_init<V>), smem));
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_v<V>), smem));
  HELM_CUDA_TRY(set_smem_attr(reinterpret_cast<const void*>(&k_t<V>), smem));
  return HELM_OK;
}

// Grids of the solver's kernels: one wave each.
template <class V>
inline helm_status krylov_shapes(helm_csr A, KShapes<V>* sh) {
  constexpr size_t smem = Engine<V>::kSmem;
  const int64_t ntiles = (static_cast<int64_t>(A->n) + Engine<V>::R - 1) / Engine<V>::R;
  HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_v<V>), reinterpret_cast<const void*>(&k_t<V>)},
                                       Prec<V>::R, smem, A->num_sms, ntiles, &sh->spmv_grid));
  HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_init<V>)}, Prec<V>::R, smem, A->num_sms, ntiles,
                                       &sh->init_grid));
  sh->vec_grid = A->vec_grid;
  // element-wise kernels: the same number of blocks on every SM (one wave,
  // fewer when the rows would not fill them)
  const int64_t per_sm_rows = (static_cast<int64_t>(A->n) + static_cast<int64_t>(A->num_sms) * kVecThreads - 1) /
                              (static_cast<int64_t>(A->num_sms) * kVecThreads);
  auto wave = [&](const void* fn, int* out) -> helm_status {
    int b = 0;
    HELM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kVecThreads, 0));
    if (b > kVecMaxBlocksPerSm) b = kVecMaxBlocksPerSm;
    int64_t per_sm = b < 1 ? 1 : b;
    if (per_sm_rows < per_sm) per_sm = per_sm_rows < 1 ? 1 : per_sm_rows;
    *out = static_cast<int>(per_sm * A->num_sms);
    return HELM_OK;
  };
  helm_status st = wave(reinterpret_cast<const void*>(&k_p<V>), &sh->grid_p);
  if (st == HELM_OK) st = wave(reinterpret_cast<const void*>(&k_s<V>), &sh->grid_s);
  if (st == HELM_OK) st = wave(reinterpret_cast<const void*>(&k_xr<V>), &sh->grid_xr);
  return st;
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
