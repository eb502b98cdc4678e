// Full-spectrum DPT in plain FP64 on the CUDA cores: the map of Eq. (dyn)
// (arXiv:2002.12872, Sec. II.B) applied literally, column form,
//     P = Delta A_k,   d_i = P_ii,   E_i = theta_i + lambda d_i,
//     A_{k+1,ji} = lambda (P_ji - d_i A_ji) / (theta_i - theta_j),   A_{k+1,ii} = 1,
// with the residual of A_k, R_ji = lambda (P_ji - d_i A_ji) - (theta_i - theta_j) A_ji,
// reduced per column for the convergence test.  Real (double) and complex
// (interleaved double2) variants.  This is the comparator for the mixed path.
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

// ---------------------------------------------------------------------------
// A_0 = I
// ---------------------------------------------------------------------------
__global__ void k_fp64_init(int n, int ld, int cplx, double* A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= ld) return;
  const double v = (i == j) ? 1.0 : 0.0;
  if (cplx) {
    A[2 * ((int64_t)i * ld + j)] = v;
    A[2 * ((int64_t)i * ld + j) + 1] = 0.0;
  } else {
    A[(int64_t)i * ld + j] = v;
  }
}

// A_0 from a caller's start (already copied into A): column i divided by its entry
// i (the chart a_i = 1).  One block per column; a zero or non-finite chart entry or
// any non-finite value marks the input bad.
__global__ void k_fp64_start(int n, int ld, int cplx, double* A, IterState* st) {
  const int i = blockIdx.x;
  bool bad = false;
  if (cplx) {
    double2* col = reinterpret_cast<double2*>(A) + (int64_t)i * ld;
    const double2 p = col[i];
    const double den = p.x * p.x + p.y * p.y;
    if (!(den > 0.0) || !finite_bits(den)) bad = true;
    __syncthreads();   // every thread has read the pivot before it is overwritten
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double2 v = col[j];
      if (!finite_bits(v.x) || !finite_bits(v.y)) bad = true;
      double2 q = make_double2(1.0, 0.0);
      if (j != i) q = bad ? make_double2(0.0, 0.0)
                          : make_double2((v.x * p.x + v.y * p.y) / den,
                                         (v.y * p.x - v.x * p.y) / den);
      col[j] = q;
    }
  } else {
    double* col = A + (int64_t)i * ld;
    const double p = col[i];
    if (p == 0.0 || !finite_bits(p)) bad = true;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = col[j];
      if (!finite_bits(v)) bad = true;
      col[j] = (j == i) ? 1.0 : (bad ? 0.0 : v / p);
    }
  }
  if (bad) atomicExch(&st->bad_input, 1u);
}

// ---------------------------------------------------------------------------
// P = Delta * A, FP64 SIMT GEMM.  64 x 64 tile per block, BK = 16, 256 threads,
// 4 x 4 outputs per thread (rows tm + 16 r, columns tn + 16 c).
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(int n, const double* __restrict__ D,
                                                  int64_t ldd, const double* __restrict__ A,
                                                  int ld, double* __restrict__ P,
                                                  const IterState* st) {
  if (st->status != ST_RUNNING) return;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int t = threadIdx.x;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int tm = t & 15, tn = t >> 4;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += GK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int m = t & 63, k = (t >> 6) + 4 * s;
      As[k][m] = (m0 + m < n && k0 + k < n) ? D[(int64_t)(k0 + k) * ldd + m0 + m] : 0.0;
      const int kb = t & 15, c = (t >> 4) + 16 * s;
      Bs[kb][c] = (k0 + kb < n && n0 + c < n) ? A[(int64_t)(n0 + c) * ld + k0 + kb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][tm + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[k][tn + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int m = m0 + tm + 16 * r, col = n0 + tn + 16 * c;
      if (m < n && col < n) P[(int64_t)col * ld + m] = acc[r][c];
    }
}

// Complex variant: interleaved (re, im); 64 x 32 tile, 4 x 2 outputs per thread.
__global__ void __launch_bounds__(256) k_gemm_c128(int n, const double2* __restrict__ D,
                                                   int64_t ldd, const double2* __restrict__ A,
                                                   int ld, double2* __restrict__ P,
                                                   const IterState* st) {
  if (st->status != ST_RUNNING) return;
  __shared__ double2 As[GK][GT + 1];
  __shared__ double2 Bs[GK][33];
  const int t = threadIdx.x;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * 32;
  const int tm = t & 15, tn = t >> 4;
  double2 acc[4][2] = {};
  for (int k0 = 0; k0 < n; k0 += GK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int m = t & 63, k = (t >> 6) + 4 * s;
      As[k][m] = (m0 + m < n && k0 + k < n) ? D[(int64_t)(k0 + k) * ldd + m0 + m]
                                             : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int kb = t & 15, c = (t >> 4) + 16 * s;
      Bs[kb][c] = (k0 + kb < n && n0 + c < n) ? A[(int64_t)(n0 + c) * ld + k0 + kb]
                                               : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      double2 a[4], b[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][tm + 16 * r];
#pragma unroll
      for (int c = 0; c < 2; ++c) b[c] = Bs[k][tn + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          acc[r][c].x = fma(a[r].x, b[c].x, fma(-a[r].y, b[c].y, acc[r][c].x));
          acc[r][c].y = fma(a[r].x, b[c].y, fma(a[r].y, b[c].x, acc[r][c].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int m = m0 + tm + 16 * r, col = n0 + tn + 16 * c;
      if (m < n && col < n) P[(int64_t)col * ld + m] = acc[r][c];
    }
}

// ---------------------------------------------------------------------------
// Epilogue: one block per column i.  Applies the map to column i, reads out
// E_i of the current iterate and its residual norm; the last block decides.
// In the first iteration it also forms the residual scale s from the row sums
// of |Delta| (one block per row chunk does that before the decision).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool CPLX>
__global__ void __launch_bounds__(256) k_epi_f64(int n, int ld, const double* __restrict__ theta,
                                                 double lam, const double* __restrict__ Pv,
                                                 const double* __restrict__ Acv,
                                                 double* __restrict__ Anv,
                                                 const double* __restrict__ Dl, int64_t ldd,
                                                 double* __restrict__ E, IterState* st,
                                                 int first) {
  if (st->status != ST_RUNNING) return;
  const int i = blockIdx.x;
  const double thi = theta[i];
  // strength of this map application: lambda, or lambda (1 - alpha^k) for the
  // non-autonomous iteration (E and the residual R stay at lambda)
  const double lam_map = st->lam_k;
  double r2 = 0.0, a2 = 0.0, rowabs = 0.0;
  if (CPLX) {
    const double2* P = (const double2*)Pv;
    const double2* Ac = (const double2*)Acv;
    double2* An = (double2*)Anv;
    const double2 d = P[(int64_t)i * ld + i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int64_t idx = (int64_t)i * ld + j;
      const double2 a = Ac[idx];
      a2 += a.x * a.x + a.y * a.y;
      if (j == i) {
        An[idx] = make_double2(1.0, 0.0);
      } else {
        const double gap = thi - theta[j];
        const double2 da = cmul(d, a);
        const double2 tt = make_double2(P[idx].x - da.x, P[idx].y - da.y);
        const double2 R = make_double2(lam * tt.x - gap * a.x, lam * tt.y - gap * a.y);
        r2 += R.x * R.x + R.y * R.y;
        An[idx] = make_double2(lam_map * tt.x / gap, lam_map * tt.y / gap);
      }
      if (first) {   // row sums of |Delta| for the residual scale (row j = i here)
        const double2* D2 = (const double2*)Dl;
        const double2 v = D2[(int64_t)j * ldd + i];
        rowabs += sqrt(v.x * v.x + v.y * v.y);
      }
    }
    if (threadIdx.x == 0) {
      E[2 * i] = thi + lam * d.x;
      E[2 * i + 1] = lam * d.y;
    }
  } else {
    const double d = Pv[(int64_t)i * ld + i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int64_t idx = (int64_t)i * ld + j;
      const double a = Acv[idx];
      a2 += a * a;
      if (j == i) {
        Anv[idx] = 1.0;
      } else {
        const double gap = thi - theta[j];
        const double tt = Pv[idx] - d * a;
        const double R = lam * tt - gap * a;
        r2 += R * R;
        Anv[idx] = lam_map * tt / gap;
      }
      if (first) rowabs += fabs(Dl[(int64_t)j * ldd + i]);
    }
    if (threadIdx.x == 0) E[i] = thi + lam * d;
  }
  // block reductions
  __shared__ double sr[3][8];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    rowabs += __shfl_xor_sync(0xffffffffu, rowabs, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sr[0][w] = r2; sr[1][w] = a2; sr[2][w] = rowabs; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R2 = 0, A2 = 0, RA = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { R2 += sr[0][q]; A2 += sr[1][q]; RA += sr[2][q]; }
    float rr = (float)sqrt(R2 / A2);
    if (!(rr == rr) || isinf(rr)) rr = __int_as_float(0x7f800000);
    atomicMax(&st->rho_bits, __float_as_uint(rr));
    if (first) atomicMax(&st->row_bits, __float_as_uint((float)RA));
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  volatile IterState* vs = st;
  if (first) vs->s = vs->theta_max + fabs(vs->lam) * (double)__uint_as_float(vs->row_bits);
  const double rho = (double)__uint_as_float(vs->rho_bits) / vs->s;
  vs->blocks_done = 0;
  vs->rho_bits = 0;
  decide(vs, rho);
}

__global__ void k_check_finite(int n, const double* __restrict__ D, int64_t ldd, int cplx,
                               IterState* st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= n) return;
  const int64_t idx = (int64_t)i * ldd + j;
  bool ok = cplx ? (isfinite(D[2 * idx]) && isfinite(D[2 * idx + 1])) : isfinite(D[idx]);
  if (!ok) atomicExch(&st->bad_input, 1u);
}

cudaError_t launch_fp64_init(int n, int ld, int cplx, void* A0, cudaStream_t s) {
  dim3 grid((ld + 255) / 256, n);
  k_fp64_init<<<grid, 256, 0, s>>>(n, ld, cplx, (double*)A0);
  return cudaGetLastError();
}

cudaError_t launch_fp64_start(int n, int ld, int cplx, double* A, IterState* st,
                              cudaStream_t s) {
  k_fp64_start<<<n, 256, 0, s>>>(n, ld, cplx, A, st);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(int n, const double* Dl, int64_t ldd, const double* A, int ld,
                            double* P, const IterState* st, cudaStream_t s) {
  dim3 grid((n + GT - 1) / GT, (n + GT - 1) / GT);
  k_gemm_f64<<<grid, 256, 0, s>>>(n, Dl, ldd, A, ld, P, st);
  return cudaGetLastError();
}

cudaError_t launch_gemm_c128(int n, const double* Dl, int64_t ldd, const double* A, int ld,
                             double* P, const IterState* st, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (n + GT - 1) / GT);
  k_gemm_c128<<<grid, 256, 0, s>>>(n, (const double2*)Dl, ldd, (const double2*)A, ld,
                                   (double2*)P, st);
  return cudaGetLastError();
}

cudaError_t launch_epi_f64(int n, int ld, int cplx, const double* theta, double lam,
                           const double* P, const double* Acur, double* Anext,
                           const double* Dl, int64_t ldd, double* E, IterState* st, int first,
                           cudaStream_t s) {
  if (cplx)
    k_epi_f64<true><<<n, 256, 0, s>>>(n, ld, theta, lam, P, Acur, Anext, Dl, ldd, E, st, first);
  else
    k_epi_f64<false><<<n, 256, 0, s>>>(n, ld, theta, lam, P, Acur, Anext, Dl, ldd, E, st, first);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(int n, const double* D, int64_t ldd, int cplx, IterState* st,
                                cudaStream_t s) {
  dim3 grid((n + 255) / 256, n);
  k_check_finite<<<grid, 256, 0, s>>>(n, D, ldd, cplx, st);
  return cudaGetLastError();
}

}  // namespace dpt
