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

typedef std::complex<double> cplx;

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
  for (int64_t i = 0; i < n; ++i) {
    cplx p = std::conj(x[i]) * y[i];
    re.add(p.real());
    im.add(p.imag());
  }
  return cplx(re.value(), im.value());
}

// ||x||_2 = sqrt(sum_i |x_i|^2) (Section 3, Table 7 "NormL2").
double dznrm2(int64_t n, const cplx* x) {
  NeumaierSum s;
  for (int64_t i = 0; i < n; ++i) s.add(x[i].real() * x[i].real() + x[i].imag() * x[i].imag());
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
// the loop the true residual b - A x is recomputed; if it exceeds 1.5 tol while
// iterations remain, the method restarts from the current x.
//
// Breakdown (this project's reading; the paper is silent): rho == 0,
// (r^, v) == 0, (t, t) == 0 or omega == 0 exactly, or any non-finite scalar.
// On breakdown x holds the last iterate.
int bicgstab(const Csr& A, const cplx* b, cplx* x, double tol, int32_t maxit, int use_x0,
             int32_t* iters_out, double* relres_recur_out, double* relres_true_out) {
  const int32_t n = A.n;
  std::vector<cplx> r(n), rhat(n), p(n), v(n), s(n), t(n), tmp(n);
  if (!use_x0) for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
  const double bnorm = dznrm2(n, b);
  *iters_out = 0;
  *relres_recur_out = 0.0;
  *relres_true_out = 0.0;
  if (!std::isfinite(bnorm)) return ST_NONFINITE;
  if (bnorm == 0.0) {  // A x = 0 has the solution x = 0
    for (int32_t i = 0; i < n; ++i) x[i] = cplx(0.0, 0.0);
    return ST_OK;
  }
  int32_t it = 0;
  int status = ST_NOT_CONVERGED;
  double relres = 0.0;
  for (;;) {  // one pass per (re)start
    // r = b - A x ; r^ = r ; rho_prev = alpha = omega = 1 ; v = p = 0
    A.apply(x, tmp.data());
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
      for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      A.apply(p.data(), v.data());
      const cplx rv = zdotc(n, rhat.data(), v.data());
      if (!finite(rv)) { status = ST_NONFINITE; break; }
      if (rv == cplx(0.0, 0.0)) { status = ST_BREAKDOWN; break; }
      alpha = rho / rv;
      if (!finite(alpha)) { status = ST_NONFINITE; break; }
      for (int32_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      const double snorm = dznrm2(n, s.data());
      if (!std::isfinite(snorm)) { status = ST_NONFINITE; break; }
      if (snorm / bnorm <= tol) {
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
    for (int32_t i = 0; i < n; ++i) tmp[i] = b[i] - tmp[i];
    const double rtrue = dznrm2(n, tmp.data()) / bnorm;
    *relres_true_out = rtrue;
    if (status == ST_OK && rtrue > 1.5 * tol && it < maxit) { status = ST_NOT_CONVERGED; continue; }
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

}  // extern "C"
