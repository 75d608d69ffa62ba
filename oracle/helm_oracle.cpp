// CPU oracle for the complex Krylov hot path.  TEST INFRASTRUCTURE ONLY:
// nothing in the product library calls, links or includes this file; only the
// test-suite, the smoke check and the benchmark's CPU-baseline leg load it.
//
// Plain, sequential, obviously-correct C++17 on std::complex<double>.  Each
// routine cites the passage of the paper ("Iterative Krylov Methods for
// Acoustic Problems on GPU", arXiv 2112.11880) or the textbook it follows.
// No blocking, fusion or reordering beyond the definitions below.
//
// Pins (what checks this code against something other than itself) live in
// tests/test_oracle_*.py: dense LU on tiny meshes, exact rational dot
// products, a Dirichlet/Robin plane-wave manufactured solution, the 1-D
// closed form of the Q1 discretisation, identity/diagonal special cases and
// central finite differences of the loss.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

// The oracle is sequential.  The benchmark's all-core CPU baseline compiles
// this same file a second time with -fopenmp: then ORACLE_PAR makes the SpMV
// rows and BiCGStab's element-wise loops parallel (each index independent,
// so the results are those of the sequential code), and the two sums below
// take one compensated partial sum per thread over a contiguous chunk, added
// in thread order with compensation.  In the default build ORACLE_PAR is
// empty and nothing of OpenMP is compiled.
#ifdef _OPENMP
#define ORACLE_PAR _Pragma("omp parallel for schedule(static)")
#else
#define ORACLE_PAR
#endif

namespace {

// Status codes, same meaning as the library's (Section 4: tolerance, maximum
// number of iterations; the breakdown rule is this project's reading).
enum {
  ST_OK = 0, ST_INVALID = 1, ST_NOT_CONVERGED = 4, ST_BREAKDOWN = 5, ST_NONFINITE = 7
};

// Neumaier's compensated summation (Neumaier 1974), one accumulator per real
// component.  Used so that the oracle's sums are accurate to about one ulp of
// the sum of magnitudes, independent of n.
struct NeumaierSum {
  double s = 0.0, c = 0.0;
  void add(double v) {
    double t = s + v;
    if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

bool finite(cplx z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

// y = A x for CSR A (Section 2 stores the matrices in CSR; Section 3, SpMV).
// y_i = sum_{k = rowptr[i]}^{rowptr[i+1]-1} vals[k] * x[colind[k]], summed in
// CSR order.
void spmv(int32_t n, const int32_t* rowptr, const int32_t* colind, const cplx* vals,
          const cplx* x, cplx* y) {
  ORACLE_PAR
  for (int32_t i = 0; i < n; ++i) {
    cplx acc(0.0, 0.0);
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += vals[k] * x[colind[k]];
    y[i] = acc;
  }
}

// (x, y) = sum_i conj(x_i) y_i.  Section 3 defines the dot product as an
// element-wise product followed by the sum of all products; the conjugation
// on the first argument is the standard complex inner product (zdotc).
cplx zdotc(int64_t n, const cplx* x, const cplx* y) {
  NeumaierSum re, im;
#ifdef _OPENMP
  const int T = omp_get_max_threads();
  std::vector<NeumaierSum> pre(T), pim(T);
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num();
    for (int64_t i = n * t / T; i < n * (t + 1) / T; ++i) {
      cplx p = std::conj(x[i]) * y[i];
      pre[t].add(p.real());
      pim[t].add(p.imag());
    }
  }
  for (int t = 0; t < T; ++t) {
    re.add(pre[t].s);
    re.add(pre[t].c);
    im.add(pim[t].s);
    im.add(pim[t].c);
  }
#else
  for (int64_t i = 0; i < n; ++i) {
    cplx p = std::conj(x[i]) * y[i];
    re.add(p.real());
    im.add(p.imag());
  }
#endif
  return cplx(re.value(), im.value());
}

// ||x||_2 = sqrt(sum_i |x_i|^2) (Section 3, Table 7 "NormL2").
double dznrm2(int64_t n, const cplx* x) {
  NeumaierSum s;
#ifdef _OPENMP
  const int T = omp_get_max_threads();
  std::vector<NeumaierSum> ps(T);
#pragma omp parallel num_threads(T)
  {
    const int t = omp_get_thread_num();
    for (int64_t i = n * t / T; i < n * (t + 1) / T; ++i)
      ps[t].add(x[i].real() * x[i].real() + x[i].imag() * x[i].imag());
  }
  for (int t = 0; t < T; ++t) {
    s.add(ps[t].s);
    s.add(ps[t].c);
  }
#else
  for (int64_t i = 0; i < n; ++i) s.add(x[i].real() * x[i].real() + x[i].imag() * x[i].imag());
#endif
  return std::sqrt(s.value());
}

struct Csr {
  int32_t n;
  const int32_t* rowptr;
  const int32_t* colind;
  const cplx* vals;
  void apply(const cplx* x, cplx* y) const { spmv(n, rowptr, colind, vals, x, y); }
};

// Unpreconditioned BiCGStab (van der Vorst 1992; Saad 2003, Algorithm 7.7),
// the "P-BiCGSTAB" of Section 4 with the identity as preconditioner.  Complex
// version with conjugated inner products.  Stopping rule (Section 4): the
// recurrence residual ||r|| / ||b|| <= tol, at most maxit iterations.  After
// the loop the true residual b - A x is recomputed; if it exceeds tol while
// iterations remain, the method restarts from the current x, and the solve
// reports ok only with a true residual at most tol.
//
// Breakdown (this project's reading; the paper is silent): rho == 0,
// (r^, v) == 0, (t, t) == 0 or omega == 0 exactly, or any non-finite scalar.
// On breakdown x holds the last iterate.
int bicgstab(const Csr& A, const cplx* b, cplx* x, double tol, int32_t maxit, int use_x0,
             int32_t* iters_out, double* relres_recur_out, double* relres_true_out) {
  const int32_t n = A.n;
  std::vector<cplx> r(n), rhat(n), p(n), v(n), s(n), t(n), tmp(n);
  if (!use_x0) {
    ORACLE_PAR
    for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
  }
  const double bnorm = dznrm2(n, b);
  *iters_out = 0;
  *relres_recur_out = 0.0;
  *relres_true_out = 0.0;
  if (!std::isfinite(bnorm)) return ST_NONFINITE;
  if (bnorm == 0.0) {  // A x = 0 has the solution x = 0
    ORACLE_PAR
    for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
    return ST_OK;
  }
  int32_t it = 0;
  int status = ST_NOT_CONVERGED;
  double relres = 0.0;
  for (;;) {  // one pass per (re)start
    // r = b - A x ; r^ = r ; rho_prev = alpha = omega = 1 ; v = p = 0
    A.apply(x, tmp.data());
    ORACLE_PAR
    for (int32_t i = 0; i < n; ++i) { r[i] = b[i] - tmp[i]; rhat[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
    cplx rho_prev(1.0, 0.0), alpha(1.0, 0.0), omega(1.0, 0.0);
    relres = dznrm2(n, r.data()) / bnorm;
    if (!std::isfinite(relres)) { status = ST_NONFINITE; break; }
    if (relres <= tol) { status = ST_OK; }
    while (status != ST_OK && it < maxit) {
      ++it;
      const cplx rho = zdotc(n, rhat.data(), r.data());
      const cplx beta = (rho / rho_prev) * (alpha / omega);
      if (!finite(rho) || !finite(beta)) { status = ST_NONFINITE; break; }
      if (rho == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      ORACLE_PAR
      for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      A.apply(p.data(), v.data());
      const cplx rv = zdotc(n, rhat.data(), v.data());
      if (!finite(rv)) { status = ST_NONFINITE; break; }
      if (rv == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      alpha = rho / rv;
      if (!finite(alpha)) { status = ST_NONFINITE; break; }
      ORACLE_PAR
      for (int32_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      const double snorm = dznrm2(n, s.data());
      if (!std::isfinite(snorm)) { status = ST_NONFINITE; break; }
      if (snorm / bnorm <= tol) {
        ORACLE_PAR
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
        relres = snorm / bnorm;
        status = ST_OK;
        break;
      }
      A.apply(s.data(), t.data());
      const cplx ts = zdotc(n, t.data(), s.data());
      const cplx tt = zdotc(n, t.data(), t.data());
      if (!finite(ts) || !finite(tt)) { status = ST_NONFINITE; break; }
      if (tt == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      omega = ts / tt;
      if (!finite(omega)) { status = ST_NONFINITE; break; }
      ORACLE_PAR
      for (int32_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i] + omega * s[i];
        r[i] = s[i] - omega * t[i];
      }
      relres = dznrm2(n, r.data()) / bnorm;
      if (!std::isfinite(relres)) { status = ST_NONFINITE; break; }
      if (relres <= tol) { status = ST_OK; break; }
      if (omega == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      rho_prev = rho;
    }
    // true residual
    A.apply(x, tmp.data());
    ORACLE_PAR
    for (int32_t i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
    const double rtrue = dznrm2(n, tmp.data()) / bnorm;
    *relres_true_out = rtrue;
    if (status == ST_OK && rtrue > tol && it < maxit) { status = ST_NOT_CONVERGED; continue; }
    if (status == ST_OK && rtrue > tol) status = ST_NOT_CONVERGED;
    break;
  }
  *iters_out = it;
  *relres_recur_out = relres;
  return status;
}

// Transpose-free QMR (Freund 1993; Saad 2003, Algorithm 7.8), the "P-TFQMR"
// of Section 4 with the identity as preconditioner; complex version, inner
// products (x, y) = sum conj(x_i) y_i with the shadow vector r~ = r0 as first
// argument.  One iteration = two half-steps = two products with A.  The
// quasi-residual bound tau sqrt(m + 1) >= ||r_m|| triggers a true-residual
// check; the solve stops when ||b - A x|| / ||b|| <= tol.  Breakdown:
// (r~, v) == 0 or rho == 0 exactly, or a non-finite scalar.
int tfqmr(const Csr& A, const cplx* b, cplx* x, double tol, int32_t maxit, int use_x0,
          int32_t* iters_out, double* relres_recur_out, double* relres_true_out) {
  const int32_t n = A.n;
  std::vector<cplx> r0(n), w(n), u(n), u_next(n), v(n), Au(n), Au_next(n), d(n), tmp(n);
  if (!use_x0) for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
  const double bnorm = dznrm2(n, b);
  *iters_out = 0;
  *relres_recur_out = 0.0;
  *relres_true_out = 0.0;
  if (!std::isfinite(bnorm)) return ST_NONFINITE;
  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
    return ST_OK;
  }
  auto true_relres = [&]() {
    A.apply(x, tmp.data());
    for (int32_t i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
    return dznrm2(n, tmp.data()) / bnorm;
  };
  // (re)start from the current x: w = u = r0 = b - A x ; v = A u ; d = 0
  double tau = 0.0, theta = 0.0;
  cplx eta(0.0, 0.0), alpha(0.0, 0.0), rho(0.0, 0.0);
  auto start = [&]() {
    A.apply(x, tmp.data());
    for (int32_t i = 0; i < n; ++i) { r0[i] = b[i] - tmp[i]; w[i] = r0[i]; u[i] = r0[i]; d[i] = 0.0; }
    A.apply(u.data(), v.data());
    for (int32_t i = 0; i < n; ++i) Au[i] = v[i];
    tau = dznrm2(n, r0.data());
    theta = 0.0;
    eta = cplx(0.0, 0.0);
    rho = zdotc(n, r0.data(), r0.data());
  };
  start();
  double relres = tau / bnorm;
  *relres_true_out = relres;
  if (!std::isfinite(relres)) return ST_NONFINITE;
  if (relres <= tol) { *relres_recur_out = relres; return ST_OK; }
  int32_t it = 0;
  int status = ST_NOT_CONVERGED;
  for (int64_t m = 0;; ++m) {
    const bool even = (m % 2) == 0;
    if (even) {
      if (it >= maxit) break;
      ++it;
      const cplx sigma = zdotc(n, r0.data(), v.data());
      if (!finite(sigma) || !finite(rho)) { status = ST_NONFINITE; break; }
      if (sigma == cplx(0.0, 0.0) || rho == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      alpha = rho / sigma;
      for (int32_t i = 0; i < n; ++i) u_next[i] = u[i] - alpha * v[i];
    }
    // w = w - alpha A u ; d = u + (theta^2 / alpha) eta d
    const cplx dcoef = (theta * theta / alpha) * eta;
    for (int32_t i = 0; i < n; ++i) {
      w[i] -= alpha * Au[i];
      d[i] = u[i] + dcoef * d[i];
    }
    theta = dznrm2(n, w.data()) / tau;
    const double c = 1.0 / std::sqrt(1.0 + theta * theta);
    tau = tau * theta * c;
    eta = (c * c) * alpha;
    if (!std::isfinite(theta) || !std::isfinite(tau) || !finite(eta)) { status = ST_NONFINITE; break; }
    for (int32_t i = 0; i < n; ++i) x[i] += eta * d[i];
    relres = tau * std::sqrt(static_cast<double>(m + 2)) / bnorm;
    if (relres <= tol) {
      const double rt = true_relres();
      *relres_true_out = rt;
      if (rt <= tol) { status = ST_OK; break; }
      // the bound is below tol but the true residual is not: the recurrence
      // has drifted from b - A x, so start again from the current x
      if (!std::isfinite(rt)) { status = ST_NONFINITE; break; }
      start();
      m = -1;
      continue;
    }
    if (even) {
      for (int32_t i = 0; i < n; ++i) u[i] = u_next[i];
      A.apply(u.data(), Au.data());
    } else {
      const cplx rho_new = zdotc(n, r0.data(), w.data());
      if (!finite(rho_new)) { status = ST_NONFINITE; break; }
      if (rho == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      const cplx beta = rho_new / rho;
      rho = rho_new;
      for (int32_t i = 0; i < n; ++i) u[i] = w[i] + beta * u[i];
      A.apply(u.data(), Au_next.data());
      for (int32_t i = 0; i < n; ++i) {
        v[i] = Au_next[i] + beta * (Au[i] + beta * v[i]);
        Au[i] = Au_next[i];
      }
    }
  }
  *relres_true_out = true_relres();
  *iters_out = it;
  *relres_recur_out = relres;
  return status;
}

// BiCGStab(l) (Sleijpen & Fokkema 1993, Algorithm 3.1), the "P-BiCGSTAB(l)"
// of Section 4 with the identity as preconditioner: l BiCG steps build
// r_0..r_l, u_0..u_l, then a minimal-residual step over r_1..r_l (modified
// Gram-Schmidt) updates x, r_0, u_0.  Complex version: (x, y) = sum conj(x_i)
// y_i, shadow vector r~ = r_0 as first argument of the BiCG inner products;
// the Gram-Schmidt coefficients are the projections <r_i, r_j> / sigma_i.
// One iteration = one outer cycle = 2 l products with A.  Stop when the
// recurrence residual ||r_0|| / ||b|| <= tol, tested after each BiCG step and
// after the minimal-residual step; the true residual is then recomputed and,
// as for BiCGStab, the method restarts from x if it exceeds tol while
// iterations remain, and reports ok only with a true residual at most tol.  Breakdown: rho0, gamma or sigma_j exactly 0, or a
// non-finite scalar.
int bicgstabl(const Csr& A, const cplx* b, cplx* x, int ell, double tol, int32_t maxit, int use_x0,
              int32_t* iters_out, double* relres_recur_out, double* relres_true_out) {
  const int32_t n = A.n;
  if (ell < 1 || ell > 16) return ST_INVALID;
  std::vector<std::vector<cplx>> r(ell + 1, std::vector<cplx>(n)), u(ell + 1, std::vector<cplx>(n));
  std::vector<cplx> rt(n), tmp(n);
  if (!use_x0) for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
  const double bnorm = dznrm2(n, b);
  *iters_out = 0;
  *relres_recur_out = 0.0;
  *relres_true_out = 0.0;
  if (!std::isfinite(bnorm)) return ST_NONFINITE;
  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
    return ST_OK;
  }
  int status = ST_NOT_CONVERGED;
  int32_t it = 0;
  double relres = 0.0;
  std::vector<std::vector<cplx>> tau(ell + 1, std::vector<cplx>(ell + 1));
  std::vector<double> sigma(ell + 1);
  std::vector<cplx> g1(ell + 1), g2(ell + 1), g3(ell + 1);  // gamma', gamma, gamma''
  for (;;) {  // one pass per (re)start
  A.apply(x, tmp.data());
  for (int32_t i = 0; i < n; ++i) { r[0][i] = b[i] - tmp[i]; rt[i] = r[0][i]; u[0][i] = 0.0; }
  cplx rho0(1.0, 0.0), alpha(0.0, 0.0), omega(1.0, 0.0);
  relres = dznrm2(n, r[0].data()) / bnorm;
  if (!std::isfinite(relres)) return ST_NONFINITE;
  if (relres <= tol) status = ST_OK;
  while (status != ST_OK && it < maxit) {
    ++it;
    rho0 = -omega * rho0;
    bool bad = false;
    // BiCG part
    for (int j = 0; j < ell && !bad; ++j) {
      const cplx rho1 = zdotc(n, rt.data(), r[j].data());
      if (!finite(rho1)) { status = ST_NONFINITE; bad = true; break; }
      if (rho0 == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; bad = true; break; }
      const cplx beta = alpha * rho1 / rho0;
      rho0 = rho1;
      for (int i = 0; i <= j; ++i)
        for (int32_t q = 0; q < n; ++q) u[i][q] = r[i][q] - beta * u[i][q];
      A.apply(u[j].data(), u[j + 1].data());
      const cplx gamma = zdotc(n, rt.data(), u[j + 1].data());
      if (!finite(gamma)) { status = ST_NONFINITE; bad = true; break; }
      if (gamma == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; bad = true; break; }
      alpha = rho0 / gamma;
      for (int i = 0; i <= j; ++i)
        for (int32_t q = 0; q < n; ++q) r[i][q] -= alpha * u[i + 1][q];
      A.apply(r[j].data(), r[j + 1].data());
      for (int32_t q = 0; q < n; ++q) x[q] += alpha * u[0][q];
      relres = dznrm2(n, r[0].data()) / bnorm;
      if (!std::isfinite(relres)) { status = ST_NONFINITE; bad = true; break; }
      if (relres <= tol) { status = ST_OK; bad = true; break; }
    }
    if (bad) break;
    // MR part: modified Gram-Schmidt on r_1..r_l
    for (int j = 1; j <= ell && !bad; ++j) {
      for (int i = 1; i < j; ++i) {
        tau[i][j] = zdotc(n, r[i].data(), r[j].data()) / sigma[i];
        for (int32_t q = 0; q < n; ++q) r[j][q] -= tau[i][j] * r[i][q];
      }
      sigma[j] = zdotc(n, r[j].data(), r[j].data()).real();
      if (!std::isfinite(sigma[j])) { status = ST_NONFINITE; bad = true; break; }
      if (sigma[j] == 0.0) { status = ST_BREAKDOWN; bad = true; break; }
      g1[j] = zdotc(n, r[j].data(), r[0].data()) / sigma[j];
    }
    if (bad) break;
    g2[ell] = g1[ell];
    omega = g2[ell];
    for (int j = ell - 1; j >= 1; --j) {
      cplx acc = g1[j];
      for (int i = j + 1; i <= ell; ++i) acc -= tau[j][i] * g2[i];
      g2[j] = acc;
    }
    for (int j = 1; j <= ell - 1; ++j) {
      cplx acc = g2[j + 1];
      for (int i = j + 1; i <= ell - 1; ++i) acc += tau[j][i] * g2[i + 1];
      g3[j] = acc;
    }
    for (int32_t q = 0; q < n; ++q) {
      x[q] += g2[1] * r[0][q];
      r[0][q] -= g1[ell] * r[ell][q];
      u[0][q] -= g2[ell] * u[ell][q];
    }
    for (int j = 1; j <= ell - 1; ++j)
      for (int32_t q = 0; q < n; ++q) {
        u[0][q] -= g2[j] * u[j][q];
        x[q] += g3[j] * r[j][q];
        r[0][q] -= g1[j] * r[j][q];
      }
    if (!finite(omega)) { status = ST_NONFINITE; break; }
    relres = dznrm2(n, r[0].data()) / bnorm;
    if (!std::isfinite(relres)) { status = ST_NONFINITE; break; }
    if (relres <= tol) { status = ST_OK; break; }
    if (omega == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
  }
  A.apply(x, tmp.data());
  for (int32_t i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
  const double rtrue = dznrm2(n, tmp.data()) / bnorm;
  *relres_true_out = rtrue;
  if (status == ST_OK && rtrue > tol && it < maxit) { status = ST_NOT_CONVERGED; continue; }
  if (status == ST_OK && rtrue > tol) status = ST_NOT_CONVERGED;
  break;
  }
  *iters_out = it;
  *relres_recur_out = relres;
  return status;
}

}  // namespace

extern "C" {

void oracle_spmv(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                 const double* x, double* y) {
  spmv(n, rowptr, colind, reinterpret_cast<const cplx*>(vals), reinterpret_cast<const cplx*>(x),
       reinterpret_cast<cplx*>(y));
}

void oracle_zdotc(int64_t n, const double* x, const double* y, double* out) {
  cplx d = zdotc(n, reinterpret_cast<const cplx*>(x), reinterpret_cast<const cplx*>(y));
  out[0] = d.real();
  out[1] = d.imag();
}

double oracle_dznrm2(int64_t n, const double* x) {
  return dznrm2(n, reinterpret_cast<const cplx*>(x));
}

int oracle_bicgstab(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                    const double* b, double* x, double tol, int32_t maxit, int use_x0,
                    int32_t* iters, double* relres_recur, double* relres_true) {
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) return ST_INVALID;
  Csr A{n, rowptr, colind, reinterpret_cast<const cplx*>(vals)};
  return bicgstab(A, reinterpret_cast<const cplx*>(b), reinterpret_cast<cplx*>(x), tol, maxit,
                  use_x0, iters, relres_recur, relres_true);
}

int oracle_tfqmr(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* vals, const double* b,
                 double* x, double tol, int32_t maxit, int use_x0, int32_t* iters, double* relres_recur,
                 double* relres_true) {
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) return ST_INVALID;
  Csr A{n, rowptr, colind, reinterpret_cast<const cplx*>(vals)};
  return tfqmr(A, reinterpret_cast<const cplx*>(b), reinterpret_cast<cplx*>(x), tol, maxit, use_x0, iters,
               relres_recur, relres_true);
}

int oracle_bicgstabl(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* vals,
                     const double* b, double* x, int ell, double tol, int32_t maxit, int use_x0, int32_t* iters,
                     double* relres_recur, double* relres_true) {
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) return ST_INVALID;
  Csr A{n, rowptr, colind, reinterpret_cast<const cplx*>(vals)};
  return bicgstabl(A, reinterpret_cast<const cplx*>(b), reinterpret_cast<cplx*>(x), ell, tol, maxit, use_x0, iters,
                   relres_recur, relres_true);
}

}  // extern "C"
