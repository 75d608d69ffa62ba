/*
 * helm.h -- C ABI of libhelm, complex Krylov solvers for Helmholtz
 * finite-element systems on one GB300 GPU (sm_103a).
 *
 * The operations follow "Iterative Krylov Methods for Acoustic Problems on
 * GPU" (Cheik Ahamed & Magoules, arXiv 2112.11880):
 *   - the problem: -lap(u) - k^2 u = g, k = 2 pi F / c, discretised by finite
 *     elements into a sparse complex system A x = b (Section 1);
 *   - matrices in CSR (Section 2);
 *   - complex double-precision vector kernels and CSR SpMV (Section 3,
 *     Tables 2-8);
 *   - preconditioned BiCGStab, BiCGStab(l) and TFQMR with residual
 *     tolerance, zero initial guess and an iteration cap (Section 4).
 *
 * Conventions shared by every call:
 *   - Complex numbers are stored interleaved (re, im): complex128 = two
 *     doubles (16 bytes), complex64 = two floats (8 bytes).  Device arrays
 *     must be aligned to their element size; CSR values and vectors used by
 *     the solvers must be 16-byte aligned (any cudaMalloc'd or PyTorch buffer
 *     is).
 *   - Pointers prefixed d_ are device pointers; all others are host pointers.
 *   - The caller owns every buffer passed in.  A CSR handle borrows rowptr,
 *     colind and values: they must stay allocated and unchanged while the
 *     handle lives.  The handle owns only its own workspace, released by
 *     helm_csr_destroy.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Kernels are
 *     enqueued on it; calls documented as asynchronous return after enqueueing
 *     and report launch errors only.
 *   - Every call returns a helm_status; nothing aborts or traps.  Nothing
 *     prints unless the environment variable HELM_DEBUG is set: then a
 *     failing CUDA call is reported on stderr.  Invalid arguments are
 *     detected on the host before any work is enqueued.
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* helm_stream_t; /* same type as cudaStream_t */

typedef enum {
  HELM_OK = 0,
  HELM_ERR_INVALID = 1,       /* bad argument or malformed CSR */
  HELM_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  HELM_ERR_NOMEM = 3,         /* device allocation failed */
  HELM_ERR_NOT_CONVERGED = 4, /* iteration cap reached before the tolerance */
  HELM_ERR_BREAKDOWN = 5,     /* Krylov breakdown (a zero denominator) */
  HELM_ERR_TIMEOUT = 6,       /* the device-side deadline expired */
  HELM_ERR_NONFINITE = 7      /* NaN or Inf met in a scalar of the recurrence */
} helm_status;

typedef enum { HELM_C128 = 0, HELM_C64 = 1 } helm_dtype;

/* Flags for helm_csr_create. */
#define HELM_CSR_VALIDATE 1u  /* check rowptr monotone, colind in range and
                                 sorted within rows (one device pass + sync) */
#define HELM_CSR_SLICED_ONLY 2u  /* no diagonal copy: complex64 products read
                                    the sliced copy too */

typedef struct helm_csr_s* helm_csr; /* opaque CSR handle */

/*
 * helm_csr_create -- wrap an n x n complex CSR matrix (Section 2: matrices
 * are stored in CSR) and prepare it for SpMV and the solvers.
 *   out      : receives the handle (host).
 *   n        : number of rows = columns, 0 <= n < 2^31.
 *   nnz      : number of stored entries, 0 <= nnz < 2^31, equal to rowptr[n].
 *   d_rowptr : int32[n+1], rowptr[0] = 0, non-decreasing.
 *   d_colind : int32[nnz], column of each entry, 0 <= colind < n.
 *   d_vals   : complex[nnz] of type dt (complex128 or complex64).
 *   flags    : HELM_CSR_VALIDATE, HELM_CSR_SLICED_ONLY (or'ed) or 0.
 * Ownership: the handle keeps the three device pointers (no copy); they must
 * stay valid and unchanged until helm_csr_destroy.  What it derives from them
 * is its own: a sliced-ELLPACK copy of the matrix (slices of 32 rows, entry k
 * of each row at a stride of 32: the columns, the real parts of the values
 * and, separately, the entries with a nonzero imaginary part; about 12 bytes
 * per stored entry for complex128), and the complex64 and right-Jacobi copies
 * (at the first solve that needs them).  When every entry lies on one of at
 * most 32 diagonals col - row = const (the longest row's), rows are sorted
 * without duplicates, and the diagonals hold at most 1.5 slots per stored
 * entry (a structured mesh in its natural numbering), the complex64 value
 * sets also get a diagonal copy of their real parts (float[diagonals][n], no
 * column index; 4 bytes per slot): the complex64 product, bound by HBM on
 * GB300, reads it instead of the sliced copy, with the same result for
 * finite x (the diagonals are summed in column order, empty slots skipped).
 * complex128 products always read the sliced copy (their bound is the FP64
 * pipe, and empty slots would add FP64 work).
 * Work done: row statistics, the sliced copy, workspace allocation, and the
 * choice of SpMV variant: for nnz >= 2^18 the stand-alone SpMV's variants
 * are timed on this matrix and the fastest is kept (every variant gives the
 * same y bit for bit).  Synchronises `stream`.  Returns
 * HELM_ERR_INVALID on bad sizes, a misaligned pointer, (with
 * HELM_CSR_VALIDATE) a malformed pattern, or when the padded sliced copy
 * would hold 2^31 entries or more; HELM_ERR_NOMEM if the workspace cannot be
 * allocated.
 */
helm_status helm_csr_create(helm_csr* out, int32_t n, int64_t nnz, const int32_t* d_rowptr,
                            const int32_t* d_colind, const void* d_vals, helm_dtype dt,
                            uint32_t flags, helm_stream_t stream);

/* helm_csr_destroy -- free the handle's workspace (synchronises the device
 * work of the handle first).  NULL is accepted. */
helm_status helm_csr_destroy(helm_csr A);

/* helm_csr_diagonals -- *out (host) = the number of diagonals of the
 * handle's diagonal copy, 0 when it has none (complex64 products then read
 * the sliced copy).  HELM_ERR_INVALID for a NULL argument. */
helm_status helm_csr_diagonals(helm_csr A, int32_t* out);

/*
 * helm_spmv -- y = alpha * A x + beta * y (Section 3, Table 8: CSR SpMV,
 * complex arithmetic).
 *   alpha, beta : host complex128 scalars (double[2]); for a complex64 handle
 *                 they are rounded to complex64.
 *   d_x         : complex[n] of the handle's type; must not overlap d_y
 *                 (HELM_ERR_INVALID).
 *   d_y         : complex[n]; not read when beta == 0.
 * Asynchronous.
 */
helm_status helm_spmv(helm_csr A, const double* alpha, const void* d_x, const double* beta,
                      void* d_y, helm_stream_t stream);

/*
 * helm_dot -- d_out = (x, y) = sum_i conj(x_i) y_i when conj_x != 0 (zdotc),
 * sum_i x_i y_i when conj_x == 0 (zdotu).  Section 3 computes the dot product
 * as an element-wise product followed by a block-wise sum of the products;
 * here each block sums its share in a fixed order and one block adds the block
 * partials in block order, so the result is bit-for-bit reproducible.
 *   n     : vector length, 0 <= n < 2^31 (n = 0 gives 0).
 *   dt    : element type of x and y; complex64 inputs are accumulated in
 *           double precision.
 *   d_out : device complex128 (double[2]).
 * Asynchronous.  Uses stream-ordered scratch memory (cudaMallocAsync).
 */
helm_status helm_dot(int64_t n, helm_dtype dt, const void* d_x, const void* d_y, int conj_x,
                     void* d_out, helm_stream_t stream);

/*
 * helm_dot_noalloc -- the same result as helm_dot (same arguments, same
 * conventions, same kernels' arithmetic), for callers that cannot allocate
 * device memory when they need a dot product: code that runs while a stream
 * is being captured into a CUDA graph in a mode that forbids allocation,
 * real-time loops that must never enter the allocator, or hosts that embed
 * this library under their own device-memory manager.  The paper has no
 * counterpart; it exists only for those callers.
 *   Scratch: the per-block partial sums live in a fixed 64 KiB array compiled
 *   into the library (a file-scope __device__ array of 2 x 4096 doubles).
 *   Every GPU that loads libhelm holds one copy of it until the process
 *   exits.  No call allocates or frees anything: no cudaMalloc, cudaFree or
 *   stream-ordered allocator.
 *   Maximum size: n < 2^31; larger n returns HELM_ERR_INVALID.  The grid never
 *   exceeds 4096 blocks, so every n below the maximum fits the array.
 *   Address: every call looks up the array's device address on the current
 *   device with cudaGetSymbolAddress (a host-side lookup; the first call on a
 *   device may also load the library's device code).  Nothing is cached, so
 *   a device reset needs nothing special.  A failed lookup returns
 *   HELM_ERR_CUDA.
 *   Sharing: all calls on a device share the one array and it keeps the last
 *   call's contents; nothing in it needs to start at zero (every slot read is
 *   written earlier in the same call).  Calls whose kernels overlap on the
 *   GPU (different streams without ordering) race on the array: order them.
 * Asynchronous.
 */
helm_status helm_dot_noalloc(int64_t n, helm_dtype dt, const void* d_x, const void* d_y, int conj_x,
                             void* d_out, helm_stream_t stream);

/*
 * helm_nrm2 -- d_out = ||x||_2 = sqrt(sum_i |x_i|^2) (Section 3, Table 7).
 *   d_out : device double.
 * Asynchronous, deterministic, stream-ordered scratch as helm_dot.
 */
helm_status helm_nrm2(int64_t n, helm_dtype dt, const void* d_x, double* d_out,
                      helm_stream_t stream);

/*
 * helm_axpby -- y = alpha * x + beta * y (Section 3: ZAXPY, Table 4, is
 * beta = 1; ZSCAL, Table 3, is alpha = 0 with y scaled by beta; ZASSIGN,
 * Table 2, is alpha = 1, beta = 0).
 *   alpha, beta : host complex128 (double[2]).
 *   d_x         : complex[n]; may equal d_y, must not otherwise overlap it.
 *                 Not read when alpha == 0.
 *   d_y         : complex[n]; not read when beta == 0.
 * Asynchronous.
 */
helm_status helm_axpby(int64_t n, helm_dtype dt, const double* alpha, const void* d_x,
                       const double* beta, void* d_y, helm_stream_t stream);

/* Krylov method selector (Section 4). */
typedef enum { HELM_BICGSTAB = 0, HELM_TFQMR = 1, HELM_BICGSTABL = 2 } helm_method;
/* Arithmetic of the solve. */
typedef enum {
  HELM_PREC_FP64 = 0, /* complex128 throughout */
  HELM_PREC_MIXED = 1 /* iterative refinement: complex64 BiCGStab inner
                         solves (values converted once into a handle-owned
                         copy), each ended when its residual has dropped by
                         opts.inner_tol; after each, an FP64 GCR step over a
                         window of the last 8 directions updates the
                         solution, the residual b - A x is recomputed in
                         FP64, and convergence is decided on it */
} helm_precision;
/* How the iteration loop is driven on the device. */
typedef enum {
  HELM_LAUNCH_AUTO = 0,       /* graph; the host-driven loop if the graph
                                 cannot be built */
  HELM_LAUNCH_GRAPH = 1,      /* CUDA graph with a device-driven while node;
                                 HELM_ERR_CUDA if it cannot be built */
  HELM_LAUNCH_PERSISTENT = 2, /* FP64 BiCGStab only (HELM_ERR_INVALID for
                                 the other methods and mixed precision): the
                                 whole solve, restarts included, is one
                                 cooperative kernel whose phases are separated
                                 by grid barriers; the same arithmetic as the
                                 graph, bit for bit.  Every barrier wait gives
                                 up after 2 s: the block sets a device error
                                 flag of the handle, every block leaves the
                                 kernel, and the solve returns HELM_ERR_CUDA.
                                 Every solve clears that flag when it starts,
                                 so a later solve on the handle is unaffected;
                                 helm_spmv has no waits and never sets it.
                                 HELM_ERR_CUDA also if the device cannot
                                 launch the kernel */
  HELM_LAUNCH_HOST = 3        /* host-driven loop of the same kernels, state
                                 polled every 16 iterations (profiling: tools
                                 that cannot see inside conditional graphs) */
} helm_launch;

/* Preconditioner.  Section 4 names its solvers P-BiCGSTAB, P-TFQMR and
 * P-BiCGSTAB(l) without saying which preconditioner they use. */
typedef enum {
  HELM_PRECOND_NONE = 0,
  HELM_PRECOND_JACOBI = 1 /* right Jacobi: the method runs on A D^-1 y = b,
                             D = diag(A) (a row without a stored nonzero
                             diagonal takes 1), and x = D^-1 y at the end.
                             The scaled matrix is a handle-owned copy made at
                             the first such solve (20 bytes per entry).  The
                             residual reported and tested is that of A x = b
                             itself.  FP64 only (HELM_ERR_INVALID with
                             HELM_PREC_MIXED) */
} helm_precond;

typedef struct {
  double tol;          /* target ||b - A x|| / ||b|| (Section 4 uses 1e-9).
                          Every method reports HELM_OK only when this ratio,
                          recomputed in FP64 from x after the loop, is at
                          most tol; when the recurrence met tol but the
                          recomputed residual did not, the solve restarts
                          from the current x while iterations remain
                          (BiCGStab, BiCGStab(l), TFQMR) */
  int32_t maxit;       /* iteration cap (Section 4 uses 1000); each BiCGStab
                          or TFQMR iteration applies A twice */
  int32_t use_x0;      /* 0: start from x = 0 (Section 4); 1: start from d_x */
  int32_t method;      /* helm_method */
  int32_t precision;   /* helm_precision */
  double inner_tol;    /* mixed precision: an inner solve ends when its
                          residual has dropped by this factor (0 or >= 1:
                          only when it looks below tol), or after 50000
                          iterations */
  double deadline_s;   /* device wall-clock limit of one solve; <= 0: none */
  int32_t ell;         /* l of BiCGStab(l), 1..8 */
  int32_t launch;      /* helm_launch */
  int32_t precond;     /* helm_precond */
} helm_opts;

typedef struct {
  int32_t iters;        /* iterations performed (all restarts / refinement
                           steps included; for mixed precision, inner
                           iterations) */
  int32_t restarts;     /* restarts from the current x (BiCGStab, TFQMR; 0 for
                           BiCGStab(l) and the sweep) or FP64 refinement
                           steps (mixed) */
  double relres_recur;  /* last recurrence residual / ||b|| */
  double relres_true;   /* ||b - A x|| / ||b|| recomputed in FP64 at the end */
  helm_status status;
  int32_t spmv_count;   /* applications of A (all precisions) */
} helm_info;

/* Defaults: tol 1e-8, maxit 20000, use_x0 0, BiCGStab, FP64, inner_tol 1e-3,
 * no deadline, ell 2, launch auto, no preconditioner. */
void helm_opts_default(helm_opts* o);

/*
 * helm_bicgstab_solve -- solve A x = b with the Krylov method of o->method
 * (Section 4: P-BiCGSTAB, P-BiCGSTAB(l), P-TFQMR; identity preconditioner).
 *   d_b  : complex128[n] right-hand side.
 *   d_x  : complex128[n] solution, overwritten; read first when o->use_x0.
 *          d_b and d_x must not overlap (HELM_ERR_INVALID).
 *   o    : options (NULL = defaults).
 *   info : host, filled after one synchronisation of `stream` at the end;
 *          may be NULL.
 * Scalars of the recurrence stay on the device: no host round trip per dot
 * product (the paper copies each dot product back; here the whole loop runs
 * on the device and only the final status is read).  The handle must be
 * complex128.  Returns info->status.  d_x always holds the last iterate.
 * Solves on one handle must not overlap (they share the handle's workspace).
 */
helm_status helm_bicgstab_solve(helm_csr A, const void* d_b, void* d_x, const helm_opts* o,
                                helm_info* info, helm_stream_t stream);

/*
 * helm_adjoint -- the backward pass of u = A^{-1} b for a real loss L(u):
 * solves A^T mu = d_dLdu (A^T = A is required: complex symmetric FEM
 * matrices) and, when d_dLdvals != NULL, writes dL/dA_ij = -mu_i u_j on every
 * stored entry (CSR order).  With that, dL/db = conj(mu) * 2 in PyTorch's
 * convention and dL/dtheta = 2 Re sum_ij dL/dA_ij dA_ij/dtheta.
 *   d_u       : complex128[n] forward solution.
 *   d_dLdu    : complex128[n] dL/du in the holomorphic sense
 *               (for L = sum |u_r - d_r|^2: conj(u_r - d_r) on receivers).
 *   d_mu      : complex128[n] output.
 *   d_dLdvals : complex128[nnz] output or NULL.
 * The outputs must not overlap d_u, d_dLdu or each other (HELM_ERR_INVALID).
 * Synchronises once at the end (info as helm_bicgstab_solve).
 */
helm_status helm_adjoint(helm_csr A, const void* d_u, const void* d_dLdu, const helm_opts* o,
                         void* d_mu, void* d_dLdvals, helm_info* info, helm_stream_t stream);

/*
 * helm_grad_sound_speed -- chain dL/dA onto per-element sound speed c (the
 * velocity "different in space" of Section 1): with A = K - w^2 M_c + i w B_c,
 * M_c = sum_e M_e / c_e^2 and B_c = sum_{top e} B_f / c_e,
 *   grad[e] = 2 Re sum_{a,b} dLdvals[map[e][8a+b]] *
 *             ((2 w^2 / c_e^3) Me[8a+b] - i (w / c_e^2) Bf[8a+b] [top[e]]).
 *   d_dLdvals  : complex128[nnz], holomorphic dL/dA (as helm_adjoint writes).
 *   d_elem_map : int32[n_elem][64], CSR slot of local pair (a, b) of each
 *                element, -1 for pairs eliminated by a Dirichlet condition.
 *   h_Me, h_Bf : host double[64], the element mass matrix and the impedance
 *                face matrix (8x8 row-major; Bf zero off the face nodes).
 *   d_top      : uint8[n_elem], 1 for elements carrying the impedance face.
 *   d_c        : double[n_elem]; omega = 2 pi F; d_grad : double[n_elem] out.
 * Asynchronous.
 */
helm_status helm_grad_sound_speed(int32_t n_elem, const void* d_dLdvals, const int32_t* d_elem_map,
                                  const double* h_Me, const double* h_Bf, const uint8_t* d_top,
                                  const double* d_c, double omega, double* d_grad,
                                  helm_stream_t stream);

/*
 * helm_assemble_helmholtz -- the complex values of A(c) = K - w^2 M_c + i w B_c
 * (Section 1: k = w / c with c varying in space) on a fixed CSR pattern, for
 * per-element speeds c, so that c can be a differentiable input.
 *   d_K         : double[nnz], the c-independent stiffness (and identity rows).
 *   d_slot_elem : int32[nnz][8], elements contributing to each slot, in
 *                 increasing element order, padded with -1.
 *   d_slot_pair : uint8[nnz][8], local pair 8a+b of each contribution.
 *   h_Me, h_Bf, d_top, d_c, omega as helm_grad_sound_speed.
 *   d_vals      : complex128[nnz] out.
 * Every sum is taken in element order with round-to-nearest steps and no
 * contraction, so equal inputs give the same values bit for bit (and a
 * symmetric pattern gives A == A^T exactly).  Asynchronous.
 */
helm_status helm_assemble_helmholtz(int64_t nnz, const double* d_K, const int32_t* d_slot_elem,
                                    const uint8_t* d_slot_pair, const double* h_Me, const double* h_Bf,
                                    const uint8_t* d_top, const double* d_c, double omega,
                                    void* d_vals, helm_stream_t stream);

/*
 * helm_conj_scale -- d_y = alpha * conj(d_x) on complex128[n] (d_y may equal
 * d_x).  Converts gradients between the holomorphic convention of
 * helm_adjoint and PyTorch's (grad = 2 conj(dL/dz)).  Asynchronous.
 */
helm_status helm_conj_scale(int64_t n, const double* alpha, const void* d_x, void* d_y,
                            helm_stream_t stream);

/*
 * Frequency sweep (the extension of Section 4's solvers to many wavenumbers
 * k_j = w_j / c on one mesh): BiCGStab, TFQMR or BiCGStab(l) for all
 * frequencies at once on
 *   A_j = K - w_j^2 M + i w_j B,
 * K, M, B real on one CSR pattern (stiffness, mass scaled by 1/c^2, impedance
 * face scaled by 1/c), never assembled as complex matrices: the real parts
 * fma(-w_j^2, M, K) are formed once per solve (or inside every product when
 * they do not fit, the same values) and i w_j B inside the product.  Converged
 * frequencies are frozen; the whole sweep is one graph launch.
 */
typedef struct helm_sweep_s* helm_sweep; /* opaque */

/*
 * helm_sweep_create -- borrow the pattern and the three real value arrays
 * (double[nnz] each, same layout rules as helm_csr_create).  One device pass
 * flags the 32-row blocks where B is zero.  Synchronises `stream`.
 */
helm_status helm_sweep_create(helm_sweep* out, int32_t n, int64_t nnz, const int32_t* d_rowptr,
                              const int32_t* d_colind, const double* d_K, const double* d_M,
                              const double* d_B, helm_stream_t stream);
helm_status helm_sweep_destroy(helm_sweep S);

/*
 * helm_sweep_solve -- solve A_j x_j = b_j for j < nfreq (1 <= nfreq <= 128).
 *   h_omega : host double[nfreq], angular frequencies w_j = 2 pi F_j.
 *   d_b     : complex128 right-hand sides, b_j[i] = d_b[i * b_ld + j] for
 *             b_ld >= nfreq, or b_j[i] = d_b[i] (one b shared by all
 *             frequencies) for b_ld = 0.
 *   d_X     : complex128 solutions, x_j[i] = d_X[i * ldx + j], ldx >= nfreq
 *             (read first when o->use_x0); must not overlap d_b
 *             (HELM_ERR_INVALID).
 *   o       : tol, maxit, use_x0, deadline_s, method, precision, inner_tol
 *             used.  method HELM_BICGSTAB (FP64 or mixed precision),
 *             HELM_TFQMR (FP64 only; the recurrences of helm_bicgstab_solve's
 *             TFQMR per frequency, iterations = two products with A_j; the
 *             quasi-residual bound triggers a true-residual check after each
 *             iteration) or HELM_BICGSTABL (FP64 only, o->ell = 1..8, else
 *             HELM_ERR_INVALID; helm_bicgstab_solve's BiCGStab(l) per
 *             frequency, iterations = cycles of 2 l products with A_j).
 *             precision HELM_PREC_MIXED: FP64 refinement per
 *             frequency around complex64 inner sweeps -- each step forms
 *             r_j = b_j - A_j x_j in FP64, solves A_j d_j = r_j / sigma_j
 *             (sigma_j = ||r_j|| / sqrt(n)) for all running frequencies in
 *             one complex64 sweep to a reduction of inner_tol, and updates
 *             x_j += gamma_j sigma_j d_j with the gamma_j that minimises the
 *             FP64 residual along that direction; a frequency stops when its
 *             FP64 residual meets tol, or not converged after five steps in
 *             a row without halving it; iterations are counted in inner
 *             iterations, restarts in refinement steps.
 *             A frequency reports HELM_OK only when its true residual is at
 *             most tol; one whose recurrence (TFQMR: its bound) met tol while
 *             its true residual did not restarts from its x (the others stay
 *             frozen), its iteration count continuing.
 *   h_infos : host helm_info[nfreq] or NULL; filled after the last pass.
 * The first call on a sweep times three tile shapes of the batched SpMV and
 * keeps the fastest (autotuning).  An FP64 solve forms the real parts of all
 * A_j once (K - w_j^2 M, nnz x F_p doubles held by the sweep, F_p = nfreq
 * rounded up to 32) when they take at most 8 GiB; beyond that, or when the
 * allocation fails, every product forms them (the same values).  Returns
 * HELM_OK when every frequency converged, else the first failing
 * frequency's status.
 */
helm_status helm_sweep_solve(helm_sweep S, int32_t nfreq, const double* h_omega, const void* d_b,
                             int32_t b_ld, void* d_X, int32_t ldx, const helm_opts* o,
                             helm_info* h_infos, helm_stream_t stream);

/*
 * helm_sweep_spmv -- Y_j = A_j X_j for j < nfreq (1 <= nfreq <= 128), with
 * A_j = K - w_j^2 M + i w_j B formed inside the product with the values of
 * helm_sweep_solve (the same row sums: each entry fma(-w_j^2, M, K) +
 * i w_j B, CSR order) -- the frequency sweep's product (Section 3's SpMV at
 * the wavenumbers of Section 1, k_j = w_j / c).
 *   h_omega : host double[nfreq].
 *   d_X     : complex128, x_j[i] = d_X[i * ldx + j], ldx >= nfreq.
 *   d_Y     : complex128 out, y_j[i] = d_Y[i * ldy + j], ldy >= nfreq; must
 *             not overlap d_X (HELM_ERR_INVALID).
 * Asynchronous (h_omega is copied before the call returns).
 */
helm_status helm_sweep_spmv(helm_sweep S, int32_t nfreq, const double* h_omega, const void* d_X, int32_t ldx,
                            void* d_Y, int32_t ldy, helm_stream_t stream);

/* helm_status_string -- static description of a status code. */
/*
 * Schwarz domain decomposition with the subdomain solves batched on one GPU
 * (the route of Section 4's closing remarks for problems beyond one GPU,
 * here with all subdomains on the same device).
 *
 * helm_ddm_create -- split the rows of A (complex128 handle, borrowed: it
 * must outlive the decomposition) into nsub contiguous blocks of near-equal
 * size [s_p, e_p) = [p n / nsub, (p + 1) n / nsub), extend each by `overlap`
 * rows on both sides (clamped to [0, n)), and build on the device the
 * block-diagonal matrix D = diag(A_1, ..., A_nsub) of the subdomain matrices
 * A_p, with its own handle (so one solve of D is the batch of all subdomain
 * solves).  A_p is the principal submatrix of A on the extended block; with
 * flags HELM_DDM_IMPEDANCE every row of it that couples to rows outside the
 * block gets i sum_{j outside} |a_ij| added to its (stored) diagonal, an
 * absorbing condition on the artificial boundary (the algebraic form of
 * optimized Schwarz methods; plain principal submatrices stall on
 * indefinite Helmholtz systems).  For a structured mesh in its natural
 * numbering the blocks are slabs of node planes and an overlap of k planes
 * is k times the plane size.  window: GCR directions helm_ddm_solve keeps
 * (1..512; 2 window + 4 complex128 vectors of length n are allocated).
 * 1 <= nsub <= n, overlap >= 0, flags 0 or HELM_DDM_IMPEDANCE;
 * HELM_ERR_INVALID otherwise or when D would hold 2^31 rows or entries or
 * more.  Synchronises `stream`.
 */
typedef struct helm_ddm_s* helm_ddm; /* opaque */
#define HELM_DDM_IMPEDANCE 1u
helm_status helm_ddm_create(helm_ddm* out, helm_csr A, int32_t nsub, int32_t overlap, int32_t window,
                            uint32_t flags, helm_stream_t stream);
helm_status helm_ddm_destroy(helm_ddm S);

/* helm_ddm_subdomains -- *rows = rows of D (the sum of the extended block
 * sizes), *nnz = its entries; either pointer may be NULL. */
helm_status helm_ddm_subdomains(helm_ddm S, int32_t* rows, int64_t* nnz);

/*
 * helm_ddm_apply -- d_z = M d_r, the restricted additive Schwarz
 * preconditioner (Cai & Sarkis 1999): M r = sum_p Rt_p^T A_p^{-1} R_p r, R_p
 * the restriction to the extended block p, Rt_p^T the prolongation that keeps
 * the rows of the block p owns; the A_p^{-1} together as one BiCGStab solve
 * of D to a relative residual inner_tol (at most 5000 iterations; 0 asks for
 * the tightest it reaches).  d_r, d_z: complex128[n], not overlapping
 * (HELM_ERR_INVALID).  Synchronises
 * `stream`.
 */
helm_status helm_ddm_apply(helm_ddm S, const void* d_r, void* d_z, double inner_tol,
                           helm_stream_t stream);

/*
 * helm_ddm_solve -- A x = b by GCR (the last `window` directions kept, the
 * minimal-residual step over them) preconditioned by helm_ddm_apply:
 * flexible, since each application's inner solve stops at its own
 * tolerance.  o: tol (as for helm_bicgstab_solve: HELM_OK only with the
 * recomputed true residual at most tol; a recurrence that met tol without it
 * starts the window again from the true residual), maxit (outer steps),
 * use_x0, inner_tol (the subdomain solves' relative residual, default 1e-3),
 * deadline_s (host wall clock); the other fields are ignored.  info: iters =
 * outer steps, restarts = window restarts, spmv_count = products with A plus
 * two per inner iteration (products with D).  The outer loop runs on the
 * host; synchronises `stream`.
 */
helm_status helm_ddm_solve(helm_ddm S, const void* d_b, void* d_x, const helm_opts* o,
                           helm_info* info, helm_stream_t stream);

const char* helm_status_string(helm_status s);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */
