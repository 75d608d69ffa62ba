// Adjoint of u = A^{-1} b and the chain onto per-element sound speed.
//
// The paper's problem (Section 1): -lap(u) - k^2 u = g with k = 2 pi F / c and
// c varying in space.  With A(c) = K - w^2 M_c(c) + i w B_c(c) and a real loss
// L(u), the holomorphic derivatives are
//   dL/db    = mu,   A^T mu = dL/du
//   dL/dA_ij = -mu_i u_j
//   dL/dc_e  = 2 Re sum_ij dL/dA_ij dA_ij/dc_e,
//              dA/dc_e = (2 w^2 / c_e^3) M_e - i (w / c_e^2) B_f   (B_f on top elements)
// helm_adjoint does the first two (one BiCGStab solve with the same CSR
// handle, A^T = A for these complex-symmetric FEM matrices, then one pass over
// the stored entries); helm_grad_sound_speed the third; helm_assemble_helmholtz
// forms A(c) itself so that c can be a differentiable input; helm_conj_scale
// converts between the holomorphic convention and PyTorch's (2 conj).
#include <cstring>

#include "common.cuh"
#include "internal.hpp"

namespace helm {

namespace {

struct ElemMats {
  double Me[64];
  double Bf[64];
};

// G_k = -mu_i u_j for every stored entry k = (i, j)
__global__ void __launch_bounds__(256) k_neg_outer(int32_t n, const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ colind, const double2* __restrict__ mu,
                                                   const double2* __restrict__ u, double2* __restrict__ G) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 m = mu[i];
    const double2 nm = make_double2(-m.x, -m.y);
    const int32_t k1 = rowptr[i + 1];
    for (int32_t k = rowptr[i]; k < k1; ++k) G[k] = cmul(nm, __ldg(u + colind[k]));
  }
}

// grad_e = 2 Re sum_ab G[map(e, ab)] ((2 w^2 / c^3) Me_ab - i (w / c^2) Bf_ab [top])
__global__ void __launch_bounds__(256) k_grad_c(int32_t E, const double2* __restrict__ G,
                                                const int32_t* __restrict__ map, ElemMats mats,
                                                const uint8_t* __restrict__ top, const double* __restrict__ c,
                                                double w, double* __restrict__ grad) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int32_t* me = map + static_cast<size_t>(e) * 64;
    double sM = 0.0, sB = 0.0;
    const bool is_top = top[e] != 0;
#pragma unroll 8
    for (int ab = 0; ab < 64; ++ab) {
      const int32_t k = __ldg(me + ab);
      if (k < 0) continue;  // pair eliminated by the Dirichlet condition
      const double2 g = __ldg(G + k);
      sM = fma(g.x, mats.Me[ab], sM);
      if (is_top) sB = fma(g.y, mats.Bf[ab], sB);
    }
    const double ce = c[e];
    const double dM = 2.0 * w * w / (ce * ce * ce);
    const double dB = w / (ce * ce);
    // Re(G (dM Me - i dB Bf)) = Re(G) dM Me + Im(G) dB Bf
    grad[e] = 2.0 * (dM * sM + dB * sB);
  }
}

// vals_k = K_k - w^2 sum Me_ab / c_e^2 + i w sum Bf_ab / c_e over the slot's
// (element, pair) table, in element order; round-to-nearest steps without
// contraction, the same sequence of operations as the input generator.
__global__ void __launch_bounds__(256) k_assemble(int64_t nnz, const double* __restrict__ K,
                                                  const int32_t* __restrict__ slot_elem,
                                                  const uint8_t* __restrict__ slot_pair, ElemMats mats,
                                                  const uint8_t* __restrict__ top, const double* __restrict__ c,
                                                  double w, double2* __restrict__ vals) {
  const double w2 = __dmul_rn(w, w);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    double m = 0.0, bsum = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int32_t e = slot_elem[k * 8 + q];
      if (e < 0) break;
      const int pr = slot_pair[k * 8 + q];
      const double ce = c[e];
      m = __dadd_rn(m, __dmul_rn(mats.Me[pr], __ddiv_rn(1.0, __dmul_rn(ce, ce))));
      if (top[e] && mats.Bf[pr] != 0.0) bsum = __dadd_rn(bsum, __dmul_rn(mats.Bf[pr], __ddiv_rn(1.0, ce)));
    }
    vals[k] = make_double2(__dsub_rn(K[k], __dmul_rn(w2, m)), __dmul_rn(w, bsum));
  }
}

// y = alpha conj(x)
__global__ void __launch_bounds__(256) k_conj_scale(int64_t n, double2 alpha, const double2* __restrict__ x,
                                                    double2* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    y[i] = cmul(alpha, make_double2(v.x, -v.y));
  }
}

bool fill_mats(const double* h_Me, const double* h_Bf, ElemMats* m) {
  if (!h_Me || !h_Bf) return false;
  std::memcpy(m->Me, h_Me, sizeof(m->Me));
  std::memcpy(m->Bf, h_Bf, sizeof(m->Bf));
  return true;
}

}  // namespace

}  // namespace helm

using namespace helm;

extern "C" {

helm_status helm_adjoint(helm_csr A, const void* d_u, const void* d_dLdu, const helm_opts* o, void* d_mu,
                         void* d_dLdvals, helm_info* info, helm_stream_t stream) {
  if (!A || A->dt != HELM_C128) return HELM_ERR_INVALID;
  if (A->n > 0 && (!d_u || !d_dLdu || !d_mu)) return HELM_ERR_INVALID;
  if (!aligned(d_u, 16) || !aligned(d_dLdu, 16) || !aligned(d_mu, 16) || !aligned(d_dLdvals, 16))
    return HELM_ERR_INVALID;
  const size_t vb = sizeof(double2) * static_cast<size_t>(A->n), eb = sizeof(double2) * static_cast<size_t>(A->nnz);
  if (overlaps(d_mu, vb, d_u, vb) || overlaps(d_mu, vb, d_dLdu, vb)) return HELM_ERR_INVALID;
  if (d_dLdvals && (overlaps(d_dLdvals, eb, d_mu, vb) || overlaps(d_dLdvals, eb, d_u, vb))) return HELM_ERR_INVALID;
  // A^T mu = dL/du with A^T = A: the forward solver on the same handle.
  helm_status st = helm_bicgstab_solve(A, d_dLdu, d_mu, o, info, stream);
  if (st != HELM_OK) return st;
  if (d_dLdvals && A->n > 0) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_neg_outer<<<vec_grid_for(A->n), 256, 0, s>>>(A->n, A->rowptr, A->colind, static_cast<const double2*>(d_mu),
                                                   static_cast<const double2*>(d_u), static_cast<double2*>(d_dLdvals));
    if (cudaGetLastError() != cudaSuccess) return HELM_ERR_CUDA;
  }
  return HELM_OK;
}

helm_status helm_grad_sound_speed(int32_t n_elem, const void* d_dLdvals, const int32_t* d_elem_map,
                                  const double* h_Me, const double* h_Bf, const uint8_t* d_top, const double* d_c,
                                  double omega, double* d_grad, helm_stream_t stream) {
  if (n_elem < 0) return HELM_ERR_INVALID;
  if (n_elem == 0) return HELM_OK;
  if (!d_dLdvals || !d_elem_map || !d_top || !d_c || !d_grad || !aligned(d_dLdvals, 16)) return HELM_ERR_INVALID;
  ElemMats m;
  if (!fill_mats(h_Me, h_Bf, &m)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_grad_c<<<vec_grid_for(n_elem), 256, 0, s>>>(n_elem, static_cast<const double2*>(d_dLdvals), d_elem_map, m, d_top,
                                                d_c, omega, d_grad);
  if (cudaGetLastError() != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}

helm_status helm_assemble_helmholtz(int64_t nnz, const double* d_K, const int32_t* d_slot_elem,
                                    const uint8_t* d_slot_pair, const double* h_Me, const double* h_Bf,
                                    const uint8_t* d_top, const double* d_c, double omega, void* d_vals,
                                    helm_stream_t stream) {
  if (nnz < 0) return HELM_ERR_INVALID;
  if (nnz == 0) return HELM_OK;
  if (!d_K || !d_slot_elem || !d_slot_pair || !d_top || !d_c || !d_vals || !aligned(d_vals, 16))
    return HELM_ERR_INVALID;
  ElemMats m;
  if (!fill_mats(h_Me, h_Bf, &m)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_assemble<<<vec_grid_for(nnz), 256, 0, s>>>(nnz, d_K, d_slot_elem, d_slot_pair, m, d_top, d_c, omega,
                                               static_cast<double2*>(d_vals));
  if (cudaGetLastError() != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}

helm_status helm_conj_scale(int64_t n, const double* alpha, const void* d_x, void* d_y, helm_stream_t stream) {
  if (n < 0 || !alpha) return HELM_ERR_INVALID;
  if (n == 0) return HELM_OK;
  if (!d_x || !d_y || !aligned(d_x, 16) || !aligned(d_y, 16)) return HELM_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_conj_scale<<<vec_grid_for(n), 256, 0, s>>>(n, make_double2(alpha[0], alpha[1]), static_cast<const double2*>(d_x),
                                               static_cast<double2*>(d_y));
  if (cudaGetLastError() != cudaSuccess) return HELM_ERR_CUDA;
  return HELM_OK;
}

}  // extern "C"
