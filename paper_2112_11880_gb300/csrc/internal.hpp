// Host-side internals of libhelm shared by the translation units: the CSR
// handle, its workspace, launch shapes, and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "../../include/helm.h"

namespace helm {

// Device-resident state of one Krylov solve (Section 4: the scalars of the
// recurrence never leave the device; the paper's per-dot host copy is gone).
struct SolverState {
  double2 rho, alpha, omega, beta;
  double2 aux[4];          // method-specific scalars
  double2 gamma;           // mixed precision: step length of the last refinement step
  // mixed precision, GCR window over the refinement steps: projections of the
  // new direction on the stored ones, its norm after orthogonalisation,
  // directions stored, next slot, whether this step's direction is kept
  double2 gcr_beta[8];
  double gcr_nrm;
  int32_t gcr_n, gcr_next, gcr_keep;
  double bnorm, tol, relres, relres_true;
  double tau, theta, eta;  // TFQMR
  int32_t iter, maxit, status, phase;
  int32_t use_x0, spmv_count, restarts, method;
  unsigned long long t0, deadline_ns;
};

enum : int32_t { ST_RUNNING = -1, ST_RESTART = -2 };  // ST_RESTART: the host relaunches from the current x
enum : int32_t { PH_RUN = 0, PH_SCONV = 1, PH_DONE = 2 };

// Tickets (arrival counters for last-block reductions), one per kernel kind.
enum : int { TK_INIT = 0, TK_V, TK_S, TK_T, TK_XR, TK_TAIL, TK_AUX0, TK_AUX1, TK_AUX2, TK_AUX3,
             TK_BAR_COUNT, TK_BAR_ABORT, TK_BAR_GEN,  // grid barrier of the persistent solver (count, abort adjacent)
             TK_COUNT };
// Group counters per two-level reduction (groups of blockDim blocks).
constexpr int kGroupTickets = 256;

// Values of a matrix in the SELL-32 layout of the SpMV engine (spmv.cuh);
// the slice offsets and columns are the handle's (shared by every value
// array of one pattern).  Arrays are double for complex128 values, float for
// complex64.
struct SellVals {
  void* sval = nullptr;      // real parts, [sell entries]
  int32_t* isoff = nullptr;  // [nsl + 1] offsets of the imaginary slices
  int32_t* icol = nullptr;   // columns of the imaginary entries
  void* ival = nullptr;      // imaginary parts
  int32_t* ilen = nullptr;   // [n] imaginary entries per row
  void* dval = nullptr;      // complex64 sets of a handle with a diagonal copy: real parts [ndia][n]
};

// complex128 Krylov vectors per handle (BiCGStab uses 6, TFQMR 8)
constexpr int kNumVec = 8;

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

}  // namespace helm

struct helm_csr_s {
  int device = 0;
  int num_sms = 0;
  int32_t n = 0;
  int64_t nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* colind = nullptr;
  const void* vals = nullptr;
  helm_dtype dt = HELM_C128;
  int32_t max_row = 0;

  // launch shapes
  int spmv_grid = 0;   // grid of the stand-alone SpMV (autotuned at creation)
  int spmv_threads = 0;  // its block size
  int spmv_variant = 0;  // its entries per pipeline stage (U), chosen at creation
  int vec_grid = 0;    // grid of element-wise kernels (256 threads)

  // workspace (owned)
  double* partials = nullptr;          // max(grid) * 8 doubles
  unsigned int* tickets = nullptr;     // TK_COUNT counters
  unsigned int* gtickets = nullptr;    // 2 x kGroupTickets group counters (K2, K4)
  unsigned int* dev_err = nullptr;     // device error flags
  helm::SolverState* state = nullptr;  // device
  helm::SolverState* state_host = nullptr;  // pinned host mirror
  double2* vec = nullptr;              // Krylov vectors, nvec * n complex128
  int nvec = 0;
  float2* vals32 = nullptr;            // complex64 copy for mixed precision
  // SELL-32 copy of the pattern (spmv.cuh) and of each value array
  int32_t nsl = 0;                     // slices of 32 rows
  int64_t sell_entries = 0;            // stored entries including padding
  int32_t* sell_off = nullptr;         // [nsl + 1]
  int32_t* sell_col = nullptr;         // [sell_entries]
  // diagonal copy of the pattern (complex64 products): every entry lies on
  // one of ndia <= 32 diagonals col - row = dia_off[d] (ascending)
  int32_t ndia = 0;
  int32_t* dia_off = nullptr;
  helm::SellVals sv;                   // the caller's values (complex128 or complex64)
  helm::SellVals sv32;                 // the complex64 copy (mixed precision, complex128 handles)
  helm::SellVals svjac;                // A D^-1 (right Jacobi)
  // right Jacobi (built at the first preconditioned solve): A D^-1; D and D^-1
  double2* jac_vals = nullptr;
  double2* jac_d = nullptr;
  double2* jac_dinv = nullptr;
  float2* vec32 = nullptr;             // complex64 Krylov vectors
  int nvec32 = 0;

  std::mutex mu;
  std::map<std::tuple<const void*, const void*, int>, helm::GraphEntry> graphs;  // (b, x, variant) -> graph
};

namespace helm {

#define HELM_TRY(expr)                   \
  do {                                   \
    const helm_status _s = (expr);       \
    if (_s != HELM_OK) return _s;        \
  } while (0)

// With the environment variable HELM_DEBUG set, a failing CUDA call is
// reported on stderr (file, line, error string); otherwise nothing prints.
void debug_cuda_error(cudaError_t e, const char* file, int line);

#define HELM_CUDA_TRY(expr)                          \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) {                         \
      helm::debug_cuda_error(_e, __FILE__, __LINE__); \
      (void)cudaGetLastError();                      \
      return _e == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA; \
    }                                                \
  } while (0)

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
// The byte ranges [p, p + pn) and [q, q + qn) share a byte.
inline bool overlaps(const void* p, size_t pn, const void* q, size_t qn) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(q);
  return pn > 0 && qn > 0 && a < b + qn && b < a + pn;
}

// Launch-shape helpers (api.cu).
cudaError_t set_smem_attr(const void* fn, size_t bytes);
int sm_count();
int vec_grid_for(int64_t n);

// Allocate the complex128 Krylov vectors (and FP32 ones) on first use.
helm_status ensure_vectors(helm_csr A, int nvec);
helm_status ensure_vectors32(helm_csr A, int nvec);
helm_status ensure_vals32(helm_csr A, cudaStream_t s);

// SELL-32 values of one value array of the handle (api.cu); `vals` is
// complex128 (dt = HELM_C128) or complex64.
helm_status build_sell_vals(helm_csr A, const void* vals, helm_dtype dt, helm::SellVals* out, cudaStream_t s);

// Launchers implemented in spmv_ops.cu (used by several solvers).
helm_status launch_spmv128(helm_csr A, const double2* x, double2* y, double2 alpha, double2 beta,
                           cudaStream_t s);
helm_status launch_spmv64(helm_csr A, const float2* x, float2* y, float2 alpha, float2 beta, cudaStream_t s);

// Solver entry points implemented in the solver translation units.
// Graph-cache key of a solve: (b, x) and the variant (the method tag and
// the preconditioner), so that each variant keeps its own graph.
inline std::tuple<const void*, const void*, int> graph_key(const void* b, const void* x, int tag, const helm_opts& o) {
  return std::make_tuple(b, x, 2 * tag + (o.precond == HELM_PRECOND_JACOBI ? 1 : 0));
}

helm_status ensure_jacobi(helm_csr A, cudaStream_t s);
helm_status bicgstab_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                          cudaStream_t s);
helm_status tfqmr_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                       cudaStream_t s);
helm_status bicgstabl_fp64(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                           cudaStream_t s);
helm_status solve_mixed(helm_csr A, const double2* b, double2* x, const helm_opts& o, helm_info* info,
                        cudaStream_t s);

}  // namespace helm
