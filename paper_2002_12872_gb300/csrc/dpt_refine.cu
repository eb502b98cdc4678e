// FP64 finish of the columns a mixed solve cannot vouch for.
//
// The mixed full solve carries the map of Eq. (dyn) (Sec. II.B) in increments whose
// products run on the tensor cores with FP32 accumulation.  Each product is rounded
// to about 2^-24 of its largest term, and the recursion never revisits that
// rounding, so the residual it tracks differs from the exact one by about
// 2^-24 |lambda| |Delta| |A_ji - delta_ji| per step; the eigenvector error this leaves
// is that residual error divided by the gap theta_i - theta_j.  The gaps themselves
// are float-float (48 bits of theta), adding 2^-46 max|theta| |A_ji| / |gap|.  For
// weakly coupled columns both are far below 1e-10, but a column with a near-degenerate
// partner j carries a large A_ji over a small gap, and its error grows like
// A_ji^2 (measured: 2e-8 when |theta_i - theta_j| = 5 lambda |Delta_ij|).
//
// Columns are independent maps (Sec. II.B: the maps F_n are only bundled), so such
// columns are finished on their own: the plain FP64 map, with FP64 gaps from the FP64
// theta and FP64 products, started from the mixed result and applied until its step
// falls below the requested accuracy (the fixed point attracting, each step is a
// refinement).  The kernels here are
//   k_risk         per-column bound w_i = max_{j != i} |A_ji| / |theta_i - theta_j| of the
//                  returned iterate, and the list of columns whose bound times the
//                  per-problem factor exceeds the target
//   k_cols_gather / k_cols_scatter   copies of the listed columns
//   k_cols_product P = Delta A_S for the listed columns in FP64, split along K into
//                  partial sums (summed in a fixed order by the epilogue)
//   k_cols_epi     the map on each listed column, its eigenvalue read-out, step and
//                  residual norms, and the maxima over the columns
#include <cuda_runtime.h>

#include "dpt_internal.h"

namespace dpt {

constexpr int RF_ROWS = 256;      // rows per block of the product
constexpr int RF_COLS = 8;        // columns per block of the product
constexpr int RF_KC_MAX = 512;    // largest K chunk per block (shared-memory staging)

// One block per column i of the returned iterate (column-major FP64, leading
// dimension lda).  The gap is formed from the float-float theta: the bound only
// needs a few digits.  Columns with coef * w_i > target are appended to cols (in no
// particular order; the host sorts them).
__global__ void __launch_bounds__(256) k_risk(int n, const double* __restrict__ A, int64_t lda,
                                              const float* __restrict__ thh,
                                              const float* __restrict__ thl, double coef,
                                              double target, int* __restrict__ count,
                                              int* __restrict__ cols) {
  const int i = blockIdx.x;
  const float hi = thh[i], li = thl[i];
  const double* a = A + (int64_t)i * lda;
  float w = 0.f;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (j == i) continue;
    const float g = (hi - thh[j]) + (li - thl[j]);
    // |a| / |g|; a zero float gap (theta_i, theta_j equal to 48 bits) gives +inf
    w = fmaxf(w, fabsf((float)a[j]) / fabsf(g));
  }
  for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
  __shared__ float wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x != 0) return;
  float m = 0.f;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmaxf(m, wm[q]);
  // NaN (never from valid data) also flags the column
  if (!(coef * (double)m <= target)) cols[atomicAdd(count, 1)] = i;
}

// As[c n + j] = A[cols[c] lda + j]
__global__ void k_cols_gather(int n, int nc, const int* __restrict__ cols,
                              const double* __restrict__ A, int64_t lda, double* __restrict__ As) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  if (j >= n || c >= nc) return;
  As[(int64_t)c * n + j] = A[(int64_t)cols[c] * lda + j];
}

// A[cols[c] lda + j] = As[c n + j], E[cols[c]] = Ec[c]
__global__ void k_cols_scatter(int n, int nc, const int* __restrict__ cols,
                               const double* __restrict__ As, const double* __restrict__ Ec,
                               double* __restrict__ A, int64_t lda, double* __restrict__ E) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  if (c >= nc) return;
  if (j < n) A[(int64_t)cols[c] * lda + j] = As[(int64_t)c * n + j];
  if (j == 0) E[cols[c]] = Ec[c];
}

// Partial products over one K chunk: Pp[(ks nc + c) n + j] = sum_{k in chunk ks}
// Delta_jk As[c n + k].  Grid (row blocks, K chunks, column groups of RF_COLS); the
// chunk's rows of As are staged in shared memory and read as broadcasts, Delta is
// read once per column group along its contiguous rows.
__global__ void __launch_bounds__(RF_ROWS) k_cols_product(int n, int nc, const double* __restrict__ D,
                                                          int64_t ldd, const double* __restrict__ As,
                                                          int kc, double* __restrict__ Pp) {
  __shared__ double sa[RF_KC_MAX][RF_COLS];
  const int j = blockIdx.x * RF_ROWS + threadIdx.x;
  const int ks = blockIdx.y, c0 = blockIdx.z * RF_COLS;
  const int k0 = ks * kc, k1 = min(n, k0 + kc);
  const int kn = k1 - k0;
  for (int t = threadIdx.x; t < kn * RF_COLS; t += RF_ROWS) {
    const int kk = t / RF_COLS, cc = t % RF_COLS;
    sa[kk][cc] = (c0 + cc < nc) ? As[(int64_t)(c0 + cc) * n + k0 + kk] : 0.0;
  }
  __syncthreads();
  if (j >= n) return;
  double acc[RF_COLS];
#pragma unroll
  for (int cc = 0; cc < RF_COLS; ++cc) acc[cc] = 0.0;
  const double* Dj = D + j;
#pragma unroll 4
  for (int kk = 0; kk < kn; ++kk) {
    const double d = Dj[(int64_t)(k0 + kk) * ldd];
#pragma unroll
    for (int cc = 0; cc < RF_COLS; ++cc) acc[cc] = fma(d, sa[kk][cc], acc[cc]);
  }
#pragma unroll
  for (int cc = 0; cc < RF_COLS; ++cc)
    if (c0 + cc < nc) Pp[((int64_t)ks * nc + c0 + cc) * n + j] = acc[cc];
}

// One block per listed column c (eigenvector i = cols[c]): P = sum of the K-chunk
// partials in chunk order; with the Epstein-Nesbet partition (theta already shifted
// by lambda diag(Delta)) the diagonal of Delta is taken out of P.  Then, as in the
// plain FP64 map,
//     E_c = theta_i + lambda P_i,   A'_j = lambda (P_j - P_i A_j) / (theta_i - theta_j),
//     R_j = lambda (P_j - P_i A_j) - (theta_i - theta_j) A_j   (= M a - E a, Sec. II.A),
// and the column's relative step |A' - A| / |A| and normalised residual |R| / (s |A|).
// The last block writes the maxima over the columns into ctl.
__global__ void __launch_bounds__(256) k_cols_epi(int n, int nc, int nks, const int* __restrict__ cols,
                                                  const double* __restrict__ theta,
                                                  const double* __restrict__ D, int64_t ldd, int en,
                                                  double lam, double s,
                                                  const double* __restrict__ Pp,
                                                  const double* __restrict__ Ac,
                                                  double* __restrict__ An, double* __restrict__ Ec,
                                                  RefineCtl* ctl) {
  const int c = blockIdx.x;
  const int i = cols[c];
  const double thi = theta[i];
  const double* a = Ac + (int64_t)c * n;
  double* an = An + (int64_t)c * n;
  auto prod = [&](int j) {
    double p = 0.0;
    for (int ks = 0; ks < nks; ++ks) p += Pp[((int64_t)ks * nc + c) * n + j];
    if (en) p -= D[(int64_t)j * ldd + j] * a[j];
    return p;
  };
  __shared__ double dsh;
  if (threadIdx.x == 0) {
    dsh = prod(i);
    Ec[c] = thi + lam * dsh;
  }
  __syncthreads();
  const double d = dsh;
  double st2 = 0.0, a2 = 0.0, r2 = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double aj = a[j];
    a2 += aj * aj;
    if (j == i) {
      an[j] = 1.0;
      st2 += (1.0 - aj) * (1.0 - aj);
      continue;
    }
    const double gap = thi - theta[j];
    const double tt = prod(j) - d * aj;
    const double v = lam * tt / gap;
    const double R = lam * tt - gap * aj;
    an[j] = v;
    st2 += (v - aj) * (v - aj);
    r2 += R * R;
  }
  for (int o = 16; o > 0; o >>= 1) {
    st2 += __shfl_xor_sync(0xffffffffu, st2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  __shared__ double sr[3][8];
  __shared__ bool last;
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sr[0][w] = st2; sr[1][w] = a2; sr[2][w] = r2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S2 = 0.0, A2 = 0.0, R2 = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { S2 += sr[0][q]; A2 += sr[1][q]; R2 += sr[2][q]; }
    double step = sqrt(S2 / A2), rho = sqrt(R2 / A2) / s;
    if (!(step == step)) step = INFINITY;
    if (!(rho == rho)) rho = INFINITY;
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(&ctl->step),
              (unsigned long long)__double_as_longlong(step));
    atomicMax(reinterpret_cast<unsigned long long*>(&ctl->rho),
              (unsigned long long)__double_as_longlong(rho));
    __threadfence();
    last = (atomicAdd(&ctl->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    ctl->blocks_done = 0u;   // ready for the next step (the host reads step and rho)
  }
}

cudaError_t launch_risk(int n, const double* A, int64_t lda, const float* thh, const float* thl,
                        double coef, double target, int* count, int* cols, cudaStream_t s) {
  k_risk<<<n, 256, 0, s>>>(n, A, lda, thh, thl, coef, target, count, cols);
  return cudaGetLastError();
}

cudaError_t launch_cols_gather(int n, int nc, const int* cols, const double* A, int64_t lda,
                               double* As, cudaStream_t s) {
  k_cols_gather<<<dim3((n + 255) / 256, nc), 256, 0, s>>>(n, nc, cols, A, lda, As);
  return cudaGetLastError();
}

cudaError_t launch_cols_scatter(int n, int nc, const int* cols, const double* As, const double* Ec,
                                double* A, int64_t lda, double* E, cudaStream_t s) {
  k_cols_scatter<<<dim3((n + 255) / 256, nc), 256, 0, s>>>(n, nc, cols, As, Ec, A, lda, E);
  return cudaGetLastError();
}

// K chunks of the column product for size n: enough blocks to cover the SMs about
// twice at small column counts, and chunks of at most RF_KC_MAX.
int refine_k_chunks(int n) {
  const int rb = (n + RF_ROWS - 1) / RF_ROWS;
  int ks = (2 * 152 + rb - 1) / rb;
  ks = max(1, min(ks, (n + 63) / 64));
  ks = max(ks, (n + RF_KC_MAX - 1) / RF_KC_MAX);
  return ks;
}

cudaError_t launch_cols_product(int n, int nc, const double* D, int64_t ldd, const double* As,
                                int nks, double* Pp, cudaStream_t s) {
  const int kc = (n + nks - 1) / nks;
  if (kc > RF_KC_MAX || nc < 1) return cudaErrorInvalidValue;
  const dim3 grid((n + RF_ROWS - 1) / RF_ROWS, nks, (nc + RF_COLS - 1) / RF_COLS);
  k_cols_product<<<grid, RF_ROWS, 0, s>>>(n, nc, D, ldd, As, kc, Pp);
  return cudaGetLastError();
}

cudaError_t launch_cols_epi(int n, int nc, int nks, const int* cols, const double* theta,
                            const double* D, int64_t ldd, int en, double lam, double s_scale,
                            const double* Pp, const double* Ac, double* An, double* Ec,
                            RefineCtl* ctl, cudaStream_t s) {
  k_cols_epi<<<nc, 256, 0, s>>>(n, nc, nks, cols, theta, D, ldd, en, lam, s_scale, Pp, Ac, An,
                                Ec, ctl);
  return cudaGetLastError();
}

}  // namespace dpt
