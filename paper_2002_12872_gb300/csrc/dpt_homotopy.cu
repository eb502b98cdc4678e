// Homotopy continuation (arXiv:2002.12872, Discussion): lambda is reached in Q equal
// steps; after each step the problem is re-expressed in the eigenbasis just found,
//     W^T M_{q+1} V = diag(E_q) + (lambda/Q) Delta_q,
// with V the accumulated right and W the left eigenvectors (W^T V = I), and the map
// is iterated again from the identity.  The stage solves are the library's full
// solves; this file holds the FP64 helpers of the basis changes (the products use
// the FP64 GEMM of dpt_full_fp64.cu): M V, the stage perturbation, a tiled
// transpose, the biorthogonal scaling of the left eigenvectors, the Newton-Schulz
// factor and the final chart scaling.
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

// Y = X^T for n x n matrices (both leading dimension ld), 32 x 32 tiles through
// shared memory, block (32, 8).
__global__ void k_h_transpose(int n, int ld, const double* __restrict__ X,
                              double* __restrict__ Y) {
  __shared__ double t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = bx + threadIdx.x, col = by + r;   // X(row, col), rows contiguous
    if (row < n && col < n) t[r][threadIdx.x] = X[(int64_t)col * ld + row];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = by + threadIdx.x, col = bx + r;   // Y(row, col) = X(col, row)
    if (row < n && col < n) Y[(int64_t)col * ld + row] = t[threadIdx.x][r];
  }
}

// Column i of B divided by b_i . a_i (so that B^T A = I for biorthogonal columns).
// One block of 256 per column; a zero or non-finite product marks the input bad.
__global__ void k_h_biorth(int n, int ld, const double* __restrict__ A, double* __restrict__ B,
                           IterState* st) {
  const int i = blockIdx.x;
  const double* a = A + (int64_t)i * ld;
  double* b = B + (int64_t)i * ld;
  double s = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) s = fma(a[j], b[j], s);
  __shared__ double ws[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += ws[q];
  if (tot == 0.0 || !finite_bits(tot)) {
    if (threadIdx.x == 0) atomicExch(&st->bad_input, 1u);
    return;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) b[j] = b[j] / tot;
}

// out column i = V column i / V_ii (the chart of the original problem), leading
// dimension ld_out.
__global__ void k_h_chart(int n, int ld, const double* __restrict__ V, double* __restrict__ out,
                          int64_t ld_out, IterState* st) {
  const int i = blockIdx.x;
  const double* v = V + (int64_t)i * ld;
  const double p = v[i];
  if (p == 0.0 || !finite_bits(p)) {
    if (threadIdx.x == 0) atomicExch(&st->bad_input, 1u);
    return;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    out[(int64_t)i * ld_out + j] = (j == i) ? 1.0 : v[j] / p;
}

// T <- diag(theta) V + c T  (column-major, leading dimension ld): with T = Delta V
// on entry this is M V for M = diag(theta) + c Delta.
__global__ void k_h_mv(int n, int ld, const double* __restrict__ theta,
                       const double* __restrict__ V, double c, double* __restrict__ T) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const int64_t idx = (int64_t)i * ld + j;
  T[idx] = fma(c, T[idx], theta[j] * V[idx]);
}

// S <- (S - diag(e)) / step: the stage perturbation from the transformed matrix.
__global__ void k_h_stage(int n, int ld, const double* __restrict__ e, double step,
                          double* __restrict__ S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const int64_t idx = (int64_t)i * ld + j;
  S[idx] = (j == i ? S[idx] - e[i] : S[idx]) / step;
}

// T <- 2 I - T (the Newton-Schulz factor).
__global__ void k_h_two_minus(int n, int ld, double* __restrict__ T) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const int64_t idx = (int64_t)i * ld + j;
  T[idx] = (j == i ? 2.0 : 0.0) - T[idx];
}

cudaError_t launch_h_mv(int n, int ld, const double* theta, const double* V, double c, double* T,
                        cudaStream_t s) {
  k_h_mv<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, ld, theta, V, c, T);
  return cudaGetLastError();
}

cudaError_t launch_h_stage(int n, int ld, const double* e, double step, double* S,
                           cudaStream_t s) {
  k_h_stage<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, ld, e, step, S);
  return cudaGetLastError();
}

cudaError_t launch_h_two_minus(int n, int ld, double* T, cudaStream_t s) {
  k_h_two_minus<<<dim3((n + 255) / 256, n), 256, 0, s>>>(n, ld, T);
  return cudaGetLastError();
}

cudaError_t launch_h_transpose(int n, int ld, const double* X, double* Y, cudaStream_t s) {
  const dim3 g((n + 31) / 32, (n + 31) / 32), b(32, 8);
  k_h_transpose<<<g, b, 0, s>>>(n, ld, X, Y);
  return cudaGetLastError();
}

cudaError_t launch_h_biorth(int n, int ld, const double* A, double* B, IterState* st,
                            cudaStream_t s) {
  k_h_biorth<<<n, 256, 0, s>>>(n, ld, A, B, st);
  return cudaGetLastError();
}

cudaError_t launch_h_chart(int n, int ld, const double* V, double* out, int64_t ld_out,
                           IterState* st, cudaStream_t s) {
  k_h_chart<<<n, 256, 0, s>>>(n, ld, V, out, ld_out, st);
  return cudaGetLastError();
}

}  // namespace dpt
