// Complex128 BiCGStab(l) with device-resident scalars: the "P-BiCGSTAB(l)"
// of Section 4 (identity preconditioner), after Sleijpen & Fokkema 1993.
//
// One iteration = one cycle = l BiCG steps (2 l products with A) and one
// minimal-residual step.  BiCG step j (kernels B1..B4):
//   B1  u_i = r_i - beta u_i, i <= j
//   B2  u_{j+1} = A u_j          + (r~, u_{j+1})       -> alpha = rho0 / gamma
//   B3  r_i -= alpha u_{i+1}, i <= j;  x += alpha u_0  + ||r_0||^2 -> stop test
//   B4  r_{j+1} = A r_j          + (r~, r_{j+1})       -> rho1, beta
// Minimal-residual step (after B4 of j = l-1, r_{i+1} = A r_i and
// u_{i+1} = A u_i hold for i < l):
//   M1  Gram matrix G_ik = (r_i, r_k), 0 <= i <= k <= l, one fused reduction;
//       the last block solves sum_k G_ik g_k = G_i0 (i = 1..l) by Cholesky
//       in FP64: g minimises ||r_0 - sum g_k r_k||, omega = g_l
//   M2  x += sum g_k r_{k-1};  r_0 -= sum g_k r_k;  u_0 -= sum g_k u_k
//       + ||r_0||^2 and (r~, r_0) -> stop test, rho1 and beta of the next cycle
// The minimal-residual coefficients come from the normal equations instead of
// the modified Gram-Schmidt of the original algorithm: the same minimiser in
// exact arithmetic, one reduction pass instead of l(l-1)/2 dependent ones.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace helm {

namespace {

using V = double2;
constexpr int RT = Engine<V>::kThreads;
constexpr size_t kSmem = Engine<V>::kSmem;
constexpr int kMaxEll = 8;
constexpr int kGram = (kMaxEll + 1) * (kMaxEll + 2) / 2;  // 45

struct BlArgs {
  CsrDev<V> A;
  const V* b;
  V* x;
  V* rt;               // shadow r~
  V* r[kMaxEll + 1];
  V* u[kMaxEll + 1];
  int ell;
  SolverState* st;     // rho = rho0, alpha, omega, beta; aux[0] = rho1
  double* partials;
  unsigned int* tickets;
  unsigned int* gtickets;  // group counters of the two-level sums of B2 and B4
  unsigned int* dev_err;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

__device__ __forceinline__ void bl_cond(const BlArgs& a, bool cont) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, cont ? 1u : 0u);
}

// after ||r_0||^2 is known: stop test (status) -- the caller keeps running otherwise
__device__ __forceinline__ void bl_stop_test(SolverState* st, double r2) {
  const double bt = st->tol * st->bnorm;
  st->relres = sqrt(r2) / st->bnorm;
  if (!isfinite(r2)) st->status = HELM_ERR_NONFINITE;
  else if (r2 <= bt * bt) st->status = HELM_OK;
}

// init: r_0 = b - A x (or b, x = 0), r~ = r_0, u_0 = 0; ||b||, ||r_0||;
// rho0 = 1, alpha = 0, omega = 1; rho1 = (r~, r_0) for the first step
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_bl_init(BlArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  SolverState* st = a.st;
  const int use_x0 = st->use_x0;
  struct Row {
    const BlArgs* a;
    double p[4];
    V bi;
    __device__ __forceinline__ void prefetch(int32_t i) { bi = a->b[i]; }
    __device__ __forceinline__ void put(int32_t i, V b_i, V ri) {
      a->r[0][i] = ri;
      a->rt[i] = ri;
      a->u[0][i] = make_double2(0.0, 0.0);
      p[0] = cabs2_acc(b_i, p[0]);
      p[1] = cabs2_acc(ri, p[1]);
      const V q = cfma_conj(ri, ri, make_double2(p[2], p[3]));
      p[2] = q.x;
      p[3] = q.y;
    }
    __device__ __forceinline__ void row(int32_t i, V ax) { put(i, bi, csub(bi, ax)); }
  } rows{&a, {0.0, 0.0, 0.0, 0.0}, make_double2(0.0, 0.0)};
  if (use_x0) {
    spmv_run<V>(a.A, a.x, rows, smem, a.dev_err);
  } else {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.A.n; i += gridDim.x * blockDim.x) {
      const V bi = a.b[i];
      a.x[i] = make_double2(0.0, 0.0);
      rows.put(i, bi, bi);
    }
  }
  double part[4] = {rows.p[0], rows.p[1], rows.p[2], rows.p[3]};
  double tot[4];
  if (!grid_sum_last<4>(part, a.partials, a.tickets + TK_INIT, red, tot)) return;
  if (threadIdx.x != 0) return;
  const double bnorm = sqrt(tot[0]);
  st->bnorm = bnorm;
  if (use_x0) st->spmv_count += 1;
  st->status = ST_RUNNING;
  if (!isfinite(bnorm)) {
    st->status = HELM_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    st->status = HELM_OK;
  } else {
    bl_stop_test(st, tot[1]);
    if (st->status == ST_RUNNING && st->maxit <= 0) st->status = HELM_ERR_NOT_CONVERGED;
    st->rho = make_double2(1.0, 0.0);    // rho0
    st->alpha = make_double2(0.0, 0.0);
    st->omega = make_double2(1.0, 0.0);
    st->aux[0] = make_double2(tot[2], tot[3]);  // rho1 = (r~, r_0)
  }
  bl_cond(a, st->status == ST_RUNNING);
}

// Scalar step before B1 (one thread): at the start of a cycle
// rho0 = -omega rho0; then beta = alpha rho1 / rho0 and rho0 = rho1.
__global__ void k_bl_beta(BlArgs a, int j) {
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  if (j == 0) {
    st->iter += 1;
    st->rho = cmul(make_double2(-st->omega.x, -st->omega.y), st->rho);
  }
  const double2 rho1 = st->aux[0];
  if (!cfinite(rho1)) {
    st->status = HELM_ERR_NONFINITE;
    return;
  }
  if (czero(st->rho)) {
    st->status = HELM_ERR_BREAKDOWN;
    return;
  }
  st->beta = cmul(st->alpha, cdiv_fast(rho1, st->rho));
  st->rho = rho1;
}

__global__ void __launch_bounds__(256) k_bl_u(BlArgs a, int j) {
  const SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const V beta = st->beta;
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.A.n; q += gridDim.x * blockDim.x) {
    for (int i = 0; i <= j; ++i) a.u[i][q] = cfms(beta, a.u[i][q], a.r[i][q]);
  }
}

// B2: u_{j+1} = A u_j, gamma = (r~, u_{j+1}) -> alpha
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_bl_au(BlArgs a, int j) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);  // block-sum scratch (dynamic shared memory)
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  struct Epi {
    V* out;
    const V* rt;
    V acc, rti;
    __device__ __forceinline__ void prefetch(int32_t i) { rti = rt[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      out[i] = ax;
      acc = cfma_conj(rti, ax, acc);
    }
  } epi{a.u[j + 1], a.rt, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.u[j], epi, smem, a.dev_err);
  double part[2] = {epi.acc.x, epi.acc.y};
  double tot[2];
  if (!grid_sum_last2<2>(part, a.partials, a.tickets + TK_V, a.gtickets, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  const double2 gamma = make_double2(tot[0], tot[1]);
  if (!cfinite(gamma)) st->status = HELM_ERR_NONFINITE;
  else if (czero(gamma)) st->status = HELM_ERR_BREAKDOWN;
  else st->alpha = cdiv_fast(st->rho, gamma);
}

// B3: r_i -= alpha u_{i+1} (i <= j), x += alpha u_0; ||r_0||^2 -> stop test
__global__ void __launch_bounds__(256) k_bl_r(BlArgs a, int j) {
  __shared__ double red[32];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  const V alpha = st->alpha;
  double r2 = 0.0;
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.A.n; q += gridDim.x * blockDim.x) {
    for (int i = 0; i <= j; ++i) {
      const V ri = cfms(alpha, a.u[i + 1][q], a.r[i][q]);
      a.r[i][q] = ri;
      if (i == 0) r2 = cabs2_acc(ri, r2);
    }
    a.x[q] = cfma(alpha, a.u[0][q], a.x[q]);
  }
  double part[1] = {r2};
  double tot[1];
  if (!grid_sum_last<1>(part, a.partials, a.tickets + TK_S, red, tot)) return;
  if (threadIdx.x != 0) return;
  bl_stop_test(st, tot[0]);
}

// B4: r_{j+1} = A r_j, rho1 = (r~, r_{j+1})
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_bl_ar(BlArgs a, int j) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* red = reinterpret_cast<double*>(smem);  // block-sum scratch (dynamic shared memory)
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  struct Epi {
    V* out;
    const V* rt;
    V acc, rti;
    __device__ __forceinline__ void prefetch(int32_t i) { rti = rt[i]; }
    __device__ __forceinline__ void row(int32_t i, V ax) {
      out[i] = ax;
      acc = cfma_conj(rti, ax, acc);
    }
  } epi{a.r[j + 1], a.rt, make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  spmv_run<V>(a.A, a.r[j], epi, smem, a.dev_err);
  double part[2] = {epi.acc.x, epi.acc.y};
  double tot[2];
  if (!grid_sum_last2<2>(part, a.partials, a.tickets + TK_T, a.gtickets + kGroupTickets, red, tot)) return;
  if (threadIdx.x != 0) return;
  st->spmv_count += 1;
  st->aux[0] = make_double2(tot[0], tot[1]);  // rho1 of the next BiCG step
}

// M1: Gram matrix of r_0..r_l; the last block solves for g (Cholesky, FP64)
template <int L>
__global__ void __launch_bounds__(256) k_bl_gram(BlArgs a) {
  constexpr int NG = (L + 1) * (L + 2) / 2;
  __shared__ double red[32 * 2];
  __shared__ double gram[2 * NG];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) return;
  double acc[2 * NG];
#pragma unroll
  for (int e = 0; e < 2 * NG; ++e) acc[e] = 0.0;
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.A.n; q += gridDim.x * blockDim.x) {
    V rv[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) rv[i] = a.r[i][q];
    int e = 0;
#pragma unroll
    for (int i = 0; i <= L; ++i)
#pragma unroll
      for (int k = i; k <= L; ++k, ++e) {
        const V g = cfma_conj(rv[i], rv[k], make_double2(acc[2 * e], acc[2 * e + 1]));
        acc[2 * e] = g.x;
        acc[2 * e + 1] = g.y;
      }
  }
  // reduce the NG complex entries two doubles at a time (fixed order)
  __shared__ bool last;
  for (int e = 0; e < NG; ++e) {
    double v2[2] = {acc[2 * e], acc[2 * e + 1]};
    block_sum<2>(v2, red);
    if (threadIdx.x == 0) {
      a.partials[(static_cast<size_t>(blockIdx.x) * NG + e) * 2] = v2[0];
      a.partials[(static_cast<size_t>(blockIdx.x) * NG + e) * 2 + 1] = v2[1];
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.tickets + TK_AUX2, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = 0; e < NG; ++e) {
    double v2[2] = {0.0, 0.0};
    for (unsigned int bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) {
      v2[0] += ld_cg(&a.partials[(static_cast<size_t>(bb) * NG + e) * 2]);
      v2[1] += ld_cg(&a.partials[(static_cast<size_t>(bb) * NG + e) * 2 + 1]);
    }
    block_sum<2>(v2, red);
    if (threadIdx.x == 0) {
      gram[2 * e] = v2[0];
      gram[2 * e + 1] = v2[1];
    }
  }
  if (threadIdx.x != 0) return;
  a.tickets[TK_AUX2] = 0u;
  // G_ik for i <= k at index e(i, k); G_ki = conj(G_ik)
  auto G = [&](int i, int k) -> double2 {
    const bool sw = i > k;
    const int lo = sw ? k : i, hi = sw ? i : k;
    const int e = lo * (L + 1) - lo * (lo - 1) / 2 + (hi - lo);
    const double2 v = make_double2(gram[2 * e], gram[2 * e + 1]);
    return sw ? make_double2(v.x, -v.y) : v;
  };
  // Cholesky of the Hermitian matrix M_ik = G_ik (i, k = 1..L), solve M g = c, c_i = G_i0
  double2 Lc[L][L];
  double2 g[L];
  bool ok = true;
  for (int i = 0; i < L && ok; ++i) {
    for (int k = 0; k <= i; ++k) {
      double2 s = G(i + 1, k + 1);
      for (int m = 0; m < k; ++m) s = csub(s, cmul(Lc[i][m], make_double2(Lc[k][m].x, -Lc[k][m].y)));
      if (i == k) {
        if (!(s.x > 0.0) || !isfinite(s.x)) {
          ok = false;
          break;
        }
        Lc[i][i] = make_double2(sqrt(s.x), 0.0);
      } else {
        Lc[i][k] = make_double2(s.x / Lc[k][k].x, s.y / Lc[k][k].x);
      }
    }
  }
  if (!ok) {
    st->status = HELM_ERR_BREAKDOWN;
    return;
  }
  double2 y[L];
  for (int i = 0; i < L; ++i) {  // L y = c
    double2 s = G(i + 1, 0);
    for (int m = 0; m < i; ++m) s = csub(s, cmul(Lc[i][m], y[m]));
    y[i] = make_double2(s.x / Lc[i][i].x, s.y / Lc[i][i].x);
  }
  for (int i = L - 1; i >= 0; --i) {  // L^H g = y
    double2 s = y[i];
    for (int m = i + 1; m < L; ++m) s = csub(s, cmul(make_double2(Lc[m][i].x, -Lc[m][i].y), g[m]));
    g[i] = make_double2(s.x / Lc[i][i].x, s.y / Lc[i][i].x);
  }
  for (int i = 0; i < L; ++i) {
    if (!cfinite(g[i])) {
      st->status = HELM_ERR_NONFINITE;
      return;
    }
  }
  // coefficients live in the partials tail (read by M2): gcoef[k], k = 1..L
  for (int i = 0; i < L; ++i) {
    a.partials[static_cast<size_t>(gridDim.x) * NG * 2 + 2 * i] = g[i].x;
    a.partials[static_cast<size_t>(gridDim.x) * NG * 2 + 2 * i + 1] = g[i].y;
  }
  st->aux[3].y = static_cast<double>(gridDim.x) * NG * 2;  // where the coefficients start
  st->omega = g[L - 1];
  if (czero(st->omega)) st->status = HELM_ERR_BREAKDOWN;
}

// M2: x += sum g_k r_{k-1}; r_0 -= sum g_k r_k; u_0 -= sum g_k u_k;
// ||r_0||^2, (r~, r_0) -> stop test and rho1 of the next cycle
template <int L>
__global__ void __launch_bounds__(256) k_bl_mr(BlArgs a) {
  __shared__ double red[32 * 3];
  __shared__ double2 gs[L];
  SolverState* st = a.st;
  if (st->status != ST_RUNNING) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bl_cond(a, false);
    return;
  }
  const size_t off = static_cast<size_t>(st->aux[3].y);
  if (threadIdx.x < L)
    gs[threadIdx.x] = make_double2(a.partials[off + 2 * threadIdx.x], a.partials[off + 2 * threadIdx.x + 1]);
  __syncthreads();
  double r2 = 0.0;
  V rr = make_double2(0.0, 0.0);
  for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.A.n; q += gridDim.x * blockDim.x) {
    V xq = a.x[q], r0 = a.r[0][q], u0 = a.u[0][q];
    V rprev = r0;
#pragma unroll
    for (int k = 1; k <= L; ++k) {
      const V rk = a.r[k][q];
      xq = cfma(gs[k - 1], rprev, xq);
      r0 = cfms(gs[k - 1], rk, r0);
      u0 = cfms(gs[k - 1], a.u[k][q], u0);
      rprev = rk;
    }
    a.x[q] = xq;
    a.r[0][q] = r0;
    a.u[0][q] = u0;
    r2 = cabs2_acc(r0, r2);
    rr = cfma_conj(a.rt[q], r0, rr);
  }
  double part[3] = {r2, rr.x, rr.y};
  double tot[3];
  if (!grid_sum_last<3>(part, a.partials, a.tickets + TK_XR, red, tot)) return;
  if (threadIdx.x != 0) return;
  bl_stop_test(st, tot[0]);
  st->aux[0] = make_double2(tot[1], tot[2]);
  if (st->status == ST_RUNNING) {
    if (st->iter >= st->maxit) st->status = HELM_ERR_NOT_CONVERGED;
    else if (st->deadline_ns != 0ull && (globaltimer_ns() - st->t0) > st->deadline_ns) st->status = HELM_ERR_TIMEOUT;
  }
  bl_cond(a, st->status == ST_RUNNING);
}

// tail: true residual (x = 0 when b = 0)
__global__ void __launch_bounds__(RT, kSolverMinBlocks) k_bl_tail(BlArgs a) {
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
      const BlArgs* a;
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

struct BlShapes {
  int spmv_grid;  // B2, B4
  int init_grid;  // init and tail
  int vec_grid, gram_grid;
};

template <int L>
void bl_body_l(const BlArgs& a, const BlShapes& sh, cudaStream_t s) {
  for (int j = 0; j < L; ++j) {
    k_bl_beta<<<1, 1, 0, s>>>(a, j);
    k_bl_u<<<sh.vec_grid, 256, 0, s>>>(a, j);
    k_bl_au<<<sh.spmv_grid, RT, kSmem, s>>>(a, j);
    k_bl_r<<<sh.vec_grid, 256, 0, s>>>(a, j);
    k_bl_ar<<<sh.spmv_grid, RT, kSmem, s>>>(a, j);
  }
  k_bl_gram<L><<<sh.gram_grid, 256, 0, s>>>(a);
  k_bl_mr<L><<<sh.vec_grid, 256, 0, s>>>(a);
}

void bl_body(const BlArgs& a, const BlShapes& sh, cudaStream_t s) {
  switch (a.ell) {
    case 1: bl_body_l<1>(a, sh, s); break;
    case 2: bl_body_l<2>(a, sh, s); break;
    case 3: bl_body_l<3>(a, sh, s); break;
    case 4: bl_body_l<4>(a, sh, s); break;
    case 5: bl_body_l<5>(a, sh, s); break;
    case 6: bl_body_l<6>(a, sh, s); break;
    case 7: bl_body_l<7>(a, sh, s); break;
    default: bl_body_l<8>(a, sh, s); break;
  }
}

}  // namespace

helm_status bicgstabl_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                           cudaStream_t s) {
  const int ell = o.ell;
  if (ell < 1 || ell > kMaxEll) return HELM_ERR_INVALID;
  const int nvec = 2 * (ell + 1) + 1;
  helm_status st = ensure_vectors(A, nvec > kNumVec ? nvec : kNumVec);
  if (st != HELM_OK) return st;
  for (const void* fn : {reinterpret_cast<const void*>(&k_bl_init), reinterpret_cast<const void*>(&k_bl_au),
                         reinterpret_cast<const void*>(&k_bl_ar), reinterpret_cast<const void*>(&k_bl_tail)})
    HELM_CUDA_TRY(set_smem_attr(fn, kSmem));
  BlShapes sh;
  {
    const int64_t ntiles = (static_cast<int64_t>(A->n) + Engine<V>::R - 1) / Engine<V>::R;
    HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_bl_au), reinterpret_cast<const void*>(&k_bl_ar)}, RT,
                             kSmem, A->num_sms, ntiles, &sh.spmv_grid));
    HELM_TRY(persistent_grid({reinterpret_cast<const void*>(&k_bl_init), reinterpret_cast<const void*>(&k_bl_tail)},
                             RT, kSmem, A->num_sms, ntiles, &sh.init_grid));
    sh.vec_grid = A->vec_grid;
    // the Gram kernel keeps 2 (l+1)(l+2)/2 accumulators per thread: few
    // blocks, and its partials (blocks x 45 x 2 doubles + coefficients) must
    // fit the handle's partial-sum buffer
    sh.gram_grid = A->num_sms * 2;
    const size_t cap = static_cast<size_t>(A->num_sms) * 32 * 8;
    while (sh.gram_grid > 1 && static_cast<size_t>(sh.gram_grid) * kGram * 2 + 2 * kMaxEll > cap) sh.gram_grid /= 2;
  }
  const size_t N = static_cast<size_t>(A->n);
  double2* W = A->vec;
  BlArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = csr_for(A, o);
  a.b = b;
  a.x = x;
  a.rt = W;
  for (int i = 0; i <= ell; ++i) {
    a.r[i] = W + (1 + i) * N;
    a.u[i] = W + (2 + ell + i) * N;
  }
  a.ell = ell;
  a.st = A->state;
  a.partials = A->partials;
  a.tickets = A->tickets;
  a.gtickets = A->gtickets;
  a.dev_err = A->dev_err;

  GraphEntry* g = nullptr;
  auto key = graph_key(b, x, 4 + ell, o);
  auto it = A->graphs.find(key);
  if (o.launch == HELM_LAUNCH_HOST) {
  } else if (it != A->graphs.end()) {
    g = &it->second;
  } else {
    auto with = [&](cudaGraphConditionalHandle c) {
      BlArgs aa = a;
      aa.cond = c;
      aa.has_cond = 1;
      return aa;
    };
    GraphEntry e;
    if (build_while_graph(
            [&](cudaGraphConditionalHandle c, cudaStream_t cs) {
              k_bl_init<<<sh.init_grid, RT, kSmem, cs>>>(with(c));
            },
            [&](cudaGraphConditionalHandle c, cudaStream_t cs) { bl_body(with(c), sh, cs); },
            [&](cudaGraphConditionalHandle c, cudaStream_t cs) { k_bl_tail<<<sh.init_grid, RT, kSmem, cs>>>(with(c)); },
            &e) == HELM_OK)
      g = &(A->graphs[key] = e);
  }

  // an explicit graph request does not fall back to the host-driven loop
  if (!g && o.launch == HELM_LAUNCH_GRAPH) return HELM_ERR_CUDA;
  SolverState* hs = A->state_host;
  HELM_CUDA_TRY(cudaMemsetAsync(A->dev_err, 0, sizeof(unsigned int), s));
  // restart from x while the recurrence converged but the true residual did
  // not (and iterations remain), as for BiCGStab
  for (int32_t use_x0 = o.use_x0 ? 1 : 0, fresh = 1;; use_x0 = 1, fresh = 0) {
    k_configure<<<1, 1, 0, s>>>(A->state, o.tol, o.maxit, use_x0, o.deadline_s, fresh);
    HELM_CUDA_TRY(cudaGetLastError());
    if (g) {
      HELM_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    } else {
      k_bl_init<<<sh.init_grid, RT, kSmem, s>>>(a);
      for (;;) {
        for (int q = 0; q < 4; ++q) bl_body(a, sh, s);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs->status != ST_RUNNING) break;
      }
      k_bl_tail<<<sh.init_grid, RT, kSmem, s>>>(a);
    }
    unsigned int herr = 0;
    HELM_CUDA_TRY(cudaMemcpyAsync(hs, A->state, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(&herr, A->dev_err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) return HELM_ERR_CUDA;
    if (!(hs->status == HELM_OK && hs->relres_true > o.tol && hs->iter < o.maxit)) break;
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
