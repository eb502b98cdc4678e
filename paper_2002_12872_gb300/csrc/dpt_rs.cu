// Rayleigh-Schroedinger partial sums on the GPU, in FP64: the comparator the paper
// sets DPT against (arXiv:2002.12872, Sec. II.D, Eq. (ARS-alpha); Supplement B).
// Column form, with C^(l) the order-l correction of the eigenvector matrix:
//     C^(0) = I,  eps^(l)_i = (Delta C^(l-1))_ii,
//     C^(l)_ji = ( (Delta C^(l-1))_ji - sum_{s=0}^{l-1} C^(l-1-s)_ji eps^(s+1)_i )
//                / (theta_i - theta_j)            (j != i),   C^(l)_ii = 0,
// and the partial sums A = sum_l lambda^l C^(l), E = theta + sum_l lambda^l eps^(l).
// Each order is one FP64 product Delta C^(l-1) (the GEMM of dpt_full_fp64.cu) and
// one pass over the n^2 entries with the l-term convolution of the earlier orders,
// so k orders cost k products and O(k^2 n^2) element work: the series needs every
// earlier order, where the map needs only its current iterate.
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

// eps^(l) = diag(X), X = Delta C^(l-1); E += lambda^l eps^(l).
__global__ void k_rs_eps(int n, int ld, const double* __restrict__ X, double* __restrict__ eps_l,
                         double lam_l, double* __restrict__ E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double e = X[(int64_t)i * ld + i];
  eps_l[i] = e;
  E[i] = fma(lam_l, e, E[i]);
}

// C^(l) from X = Delta C^(l-1) and the earlier orders C (order s at C + s nn) and
// eps (order s at eps + s n); A += lambda^l C^(l).
__global__ void k_rs_order(int n, int ld, int l, const double* __restrict__ X,
                           double* __restrict__ C, const double* __restrict__ eps,
                           const double* __restrict__ theta, double lam_l,
                           double* __restrict__ A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const int64_t idx = (int64_t)i * ld + j;
  const int64_t nn = (int64_t)ld * n;
  double c = 0.0;
  if (j != i) {
    double acc = X[idx];
    for (int s = 0; s < l; ++s) acc -= C[(int64_t)(l - 1 - s) * nn + idx] * eps[(int64_t)(s + 1) * n + i];
    c = acc / (theta[i] - theta[j]);
  }
  C[(int64_t)l * nn + idx] = c;
  A[idx] = fma(lam_l, c, A[idx]);
}

cudaError_t launch_rs_eps(int n, int ld, const double* X, double* eps_l, double lam_l, double* E,
                          cudaStream_t s) {
  k_rs_eps<<<(n + 255) / 256, 256, 0, s>>>(n, ld, X, eps_l, lam_l, E);
  return cudaGetLastError();
}

cudaError_t launch_rs_order(int n, int ld, int l, const double* X, double* C, const double* eps,
                            const double* theta, double lam_l, double* A, cudaStream_t s) {
  k_rs_order<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, ld, l, X, C, eps, theta, lam_l, A);
  return cudaGetLastError();
}

}  // namespace dpt
