// Dominant eigenvector by the single-vector map of Eq. (single_line_dyn)
// (arXiv:2002.12872, Sec. II.H) with a CSR perturbation:
//     y   = Delta z,     y* = y_{n*},     E = theta_{n*} + lambda y*,
//     R_m = lambda (y_m - y* z_m) - (theta_{n*} - theta_m) z_m      (m != n*)
//     z_m <- z_m + R_m / (theta_{n*} - theta_m)  =  lambda (y_m - y* z_m) / (theta_{n*} - theta_m)
// R is the explicit eigen-residual (M z - E z)_m of the current iterate, so its
// norm is the convergence test.  Two arithmetic variants:
//   FF    z, y, R carried as float-float (about 48 bits) on the FP32 pipes: every
//         nonzero costs a few FP32 operations, no FP64 instruction;
//   FP64  plain double arithmetic (the comparator; FP64-pipe bound on this GPU).
// The matrix stream (FP32 values + int32 column indices) is read once per
// iteration with coalesced loads; z (16 B per row in FF form) is gathered
// through L2.
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

// float-float product of a float and an (h, l) pair, accumulated into (ah, al)
__device__ __forceinline__ void ff_fma_acc(float v, float zh, float zl, float& ah, float& al) {
  float p, pe;
  two_prod(v, zh, p, pe);
  pe = fmaf(v, zl, pe);
  float s, se;
  two_sum(ah, p, s, se);
  se += al + pe;
  fast_two_sum(s, se, ah, al);
}
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  fast_two_sum(s, e, rh, rl);
}
// (ah, al) * (bh, bl)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  float p, pe;
  two_prod(ah, bh, p, pe);
  pe = fmaf(ah, bl, fmaf(al, bh, pe));
  fast_two_sum(p, pe, rh, rl);
}

// ---------------------------------------------------------------------------
// Set-up: theta -> float-float, max |theta| (the residual scale's first term), the
// largest theta (for n*), finiteness.  The CSR indices and values are validated, and
// the row sums of |Delta| formed, by the first pass of the map, which reads them
// anyway (k_dom_iter at k = 0).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dom_setup(int n, const double* __restrict__ theta,
                                                   float* __restrict__ th_hi,
                                                   float* __restrict__ th_lo, DomState* st) {
  float amax = 0.f;
  unsigned long long tmax = 0ull;
  bool bad = false;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const double t = theta[m];
    if (!finite_bits(t)) bad = true;
    float h, l;
    split_double(t, h, l);
    th_hi[m] = h;
    th_lo[m] = l;
    amax = fmaxf(amax, fabsf(h));
    tmax = max(tmax, ordered_bits(t));
  }
  if (bad) atomicExch(&st->bad_input, 1u);
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st->absmax_bits, __float_as_uint(amax));
    atomicMax(&st->theta_bits, tmax);
  }
}

// row_ptr must be monotone from 0 to nnz before any kernel follows it into
// col_idx / vals.  Reads row_ptr only.
__global__ void k_dom_check_rowptr(int n, int64_t nnz, const int32_t* __restrict__ row_ptr,
                                   DomState* st) {
  bool bad = false;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const int a = row_ptr[m], b = row_ptr[m + 1];
    if (a < 0 || b < a || (int64_t)b > nnz) bad = true;
    if (m == 0 && a != 0) bad = true;
    if (m == n - 1 && (int64_t)b != nnz) bad = true;
  }
  if (bad) atomicExch(&st->bad_input, 1u);
}

// n* = first index holding the largest theta.
__global__ void k_dom_argmax(int n, const double* __restrict__ theta, DomState* st) {
  const unsigned long long tmax = st->theta_bits;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
    if (ordered_bits(theta[m]) == tmax) atomicMin(&st->nstar_min, m);
}

__global__ void k_dom_pick(int n, DomState* st) {
  int ns = (st->nstar_req >= 0) ? st->nstar_req : st->nstar_min;
  if (ns < 0 || ns >= n) {   // no index held the largest theta: keep later reads in bounds
    ns = 0;
    st->bad_input = 1u;
  }
  st->nstar = ns;
}

// Number of m with theta_m == theta_{n*} (1 unless the map would divide by zero).
__global__ void k_dom_ties(int n, const double* __restrict__ theta, DomState* st) {
  const double ts = theta[st->nstar];
  unsigned cnt = 0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
    cnt += (theta[m] == ts) ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->ties, cnt);
}

// The checks before the loop, on the device (no host round trip): a malformed row
// pointer or a non-finite theta ends the solve with ST_BADINPUT, a theta equal to
// theta_{n*} elsewhere (the map would divide by zero) with ST_DEGENERATE; every later
// kernel then returns at once, before it follows row_ptr.  One thread, after the
// set-up, selection and tie count.
__global__ void k_dom_gate(DomState* st) {
  if (st->bad_input) st->status = ST_BADINPUT;
  else if (st->ties != 1u) st->status = ST_DEGENERATE;
}

// z_0 = e_{n*}.
__global__ void k_dom_init(int n, float2* __restrict__ z, DomState* st) {
  const int nstar = st->nstar;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x)
    z[m] = make_float2((m == nstar) ? 1.f : 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// Pre-pass: y* = (Delta z)_{n*}, one warp.
// ---------------------------------------------------------------------------
template <bool FF>
__global__ void k_dom_ystar(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                            const float* __restrict__ vals, const float2* __restrict__ z0,
                            const float2* __restrict__ z1, const double* __restrict__ z64_0,
                            const double* __restrict__ z64_1, DomState* st) {
  if (st->status != ST_RUNNING) return;
  const int lane = threadIdx.x;
  const int nstar = st->nstar;
  const int a = row_ptr[nstar], b = row_ptr[nstar + 1];
  // row n*'s indices are checked here: the main pass validates the others before its
  // first gathers (an index out of range is read as column 0 and ends the solve)
  auto col = [&](int q) {
    const int c = col_idx[q];
    if ((unsigned)c >= (unsigned)n) {
      atomicExch(&st->bad_input, 1u);
      return 0;
    }
    return c;
  };
  if (FF) {
    const float2* z = st->cur ? z1 : z0;
    float ah = 0.f, al = 0.f;
    for (int q = a + lane; q < b; q += 32) {
      const float2 zc = z[col(q)];
      ff_fma_acc(vals[q], zc.x, zc.y, ah, al);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, ah, o);
      const float ol = __shfl_xor_sync(0xffffffffu, al, o);
      ff_add(ah, al, oh, ol, ah, al);
    }
    if (lane == 0) { st->ys_hi = ah; st->ys_lo = al; }
  } else {
    const double* z = st->cur ? z64_1 : z64_0;
    double acc = 0.0;
    for (int q = a + lane; q < b; q += 32) acc = fma((double)vals[q], z[col(q)], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) st->ys64 = acc;
  }
}

// ---------------------------------------------------------------------------
// Main pass: one group of V lanes per row (V = 4, 8, 16 or 32 by mean row
// length).  Each group sums its row of Delta z, the group leader applies the
// update and accumulates |R|^2 and |z|^2; per-block partials; the last block
// reduces them and takes the convergence decision.  The first pass (k = 0) also
// validates every index and value before it gathers with it (a bad one is read as
// column 0 with value 0 and ends the solve) and forms the row sums of |Delta| for
// the residual scale s = max|theta| + |lambda| max_m sum_k |Delta_mk|, which its own
// decision needs.
// ---------------------------------------------------------------------------
// The decision after a pass (one thread of the last block): the fields it reads are
// loaded together from L2 (one round trip instead of one per field a branch depends
// on), the eigenvalue and residual of the assessed iterate formed, the residual scale
// on the first pass, then the statuses of the full-spectrum decision, stored back
// field by field.  The grid's other blocks are done with the state by now.
template <bool FF, bool FIRST>
__device__ __forceinline__ void dom_decide(DomState* st, double theta_star, double R2, double Z2) {
  const unsigned bad = __ldcg(&st->bad_input);
  const double lam = __ldcg(&st->lam), tol = __ldcg(&st->tol), best = __ldcg(&st->best);
  const int grown = __ldcg(&st->grown), k = __ldcg(&st->k), max_iter = __ldcg(&st->max_iter);
  const double ys = FF ? (double)__ldcg(&st->ys_hi) + (double)__ldcg(&st->ys_lo)
                       : __ldcg(&st->ys64);
  double s;
  if (FIRST) {
    s = (double)__uint_as_float(__ldcg(&st->absmax_bits)) +
        fabs(lam) * (double)__uint_as_float(__ldcg(&st->row_bits));
    st->s = s;
  } else {
    s = __ldcg(&st->s);
  }
  st->blocks_done = 0;
  st->E = theta_star + lam * ys;   // eigenvalue of the iterate that was just assessed
  const double rho = sqrt(R2) / (s * sqrt(Z2));
  st->rho = rho;
  if (bad) { st->status = ST_BADINPUT; return; }
  if (!(rho == rho) || isinf(rho)) { st->status = ST_DIVERGED; return; }
  if (rho <= tol) { st->status = ST_CONVERGED; return; }
  if (rho < best) {
    st->best = rho;
    st->grown = 0;
  } else if (rho > 10.0 * best) {
    if (grown + 1 >= 20) { st->grown = grown + 1; st->status = ST_DIVERGED; return; }
    st->grown = grown + 1;
  } else {
    st->grown = 0;
  }
  if (k >= max_iter) { st->status = ST_MAXITER; return; }
  st->k = k + 1;
  st->cur = (k + 1) & 1;
  if (__ldcg(&st->ramp_alpha) > 0.0) dom_ramp_advance(st);
}

// the next four entries of a lane in the row: index, value; checked on the first pass
template <bool FIRST>
__device__ __forceinline__ void dom_fetch4(const int32_t* __restrict__ col_idx,
                                           const float* __restrict__ vals, int q, int b, int V,
                                           int n, int (&c)[4], float (&v)[4], bool& bad,
                                           float& rsum) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int qq = q + u * V;
    const bool ok = qq < b;
    c[u] = ok ? col_idx[qq] : 0;
    v[u] = ok ? vals[qq] : 0.f;
  }
  if (FIRST) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if ((unsigned)c[u] >= (unsigned)n || !(fabsf(v[u]) <= 3.4e38f)) {
        bad = true;
        c[u] = 0;
        v[u] = 0.f;
      }
      rsum += fabsf(v[u]);
    }
  }
}
template <bool FF, int V, bool FIRST>
__device__ __forceinline__ void dom_iter_body(int n, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col_idx,
                                                  const float* __restrict__ vals,
                                                  const float* __restrict__ th_hi,
                                                  const float* __restrict__ th_lo,
                                                  const double* __restrict__ theta,
                                                  float2* __restrict__ z0,
                                                  float2* __restrict__ z1,
                                                  double* __restrict__ z64_0,
                                                  double* __restrict__ z64_1,
                                                  double* __restrict__ part, DomState* st) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (V - 1);
  bool bad = false;        // first pass: an index out of range or a non-finite value
  float rmax = 0.f;        // first pass: the largest row sum of |Delta| seen
  const int groups_per_block = blockDim.x / V;
  const int g0 = blockIdx.x * groups_per_block + threadIdx.x / V;
  const int gstride = gridDim.x * groups_per_block;
  const int nstar = st->nstar;
  const bool c1 = st->cur != 0;
  const float lam_h = st->lam_hi, lam_l = st->lam_lo;
  // per-thread norms of the float-float variant in float (FP64 instructions are
  // slow on this GPU even with few active lanes); the block reduction is in double
  float r2f = 0.f, z2f = 0.f;
  double r2 = 0.0, z2 = 0.0;
  if (FF) {
    // z as interleaved (hi, lo): one 8-byte gather per nonzero
    const float2* z = c1 ? z1 : z0;
    float2* nz = c1 ? z0 : z1;
    const float ysh = st->ys_hi, ysl = st->ys_lo;
    const float tsh = th_hi[nstar], tsl = th_lo[nstar];
    const float dlh = st->dlam_hi, dll = st->dlam_lo;   // non-autonomous step (0: off)
    // rows are visited in rounds; every lane runs the same number of rounds
    const int rounds = (n + gstride - 1) / gstride;
    for (int rd = 0; rd < rounds; ++rd) {
      const int m = g0 + rd * gstride;
      float ah = 0.f, al = 0.f, rsum = 0.f;
      if (m < n) {
        const int a = row_ptr[m], b = row_ptr[m + 1];
        // Memory-level parallelism: each pass issues the lane's next four index and
        // value loads, then the four gathers, before any arithmetic.
        int q = a + gl;
        for (;; q += 4 * V) {
          int c[4];
          float v[4];
          float2 zz[4];
          dom_fetch4<FIRST>(col_idx, vals, q, b, V, n, c, v, bad, rsum);
#pragma unroll
          for (int u = 0; u < 4; ++u) zz[u] = z[c[u]];
#pragma unroll
          for (int u = 0; u < 4; ++u) ff_fma_acc(v[u], zz[u].x, zz[u].y, ah, al);
          if (q + 4 * V >= b) break;
        }
      }
#pragma unroll
      for (int o = V / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, ah, o);
        const float ol = __shfl_xor_sync(0xffffffffu, al, o);
        ff_add(ah, al, oh, ol, ah, al);
        if (FIRST) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      }
      if (FIRST && gl == 0 && m < n) rmax = fmaxf(rmax, rsum);
      if (gl == 0 && m < n) {
        const float2 zm2 = z[m];
        const float zmh = zm2.x, zml = zm2.y;
        if (m == nstar) {
          nz[m] = make_float2(1.f, 0.f);
          z2f += 1.f;
        } else {
          // R = lambda (y - y* z) - gap z, all in float-float
          float t1h, t1l, t2h, t2l, gh, gl2, uh, ul, vh, vl, Rh, Rl;
          ff_mul(ysh, ysl, zmh, zml, t1h, t1l);
          ff_add(ah, al, -t1h, -t1l, t2h, t2l);
          ff_mul(lam_h, lam_l, t2h, t2l, uh, ul);
          ff_sub(tsh, tsl, th_hi[m], th_lo[m], gh, gl2);
          ff_mul(gh, gl2, zmh, zml, vh, vl);
          ff_add(uh, ul, -vh, -vl, Rh, Rl);
          // the step applies lambda - dlam: R_step = R - dlam (y - y* z)
          float Sh = Rh;
          if (dlh != 0.f) {
            float wh, wl, sl;
            ff_mul(dlh, dll, t2h, t2l, wh, wl);
            ff_add(Rh, Rl, -wh, -wl, Sh, sl);
          }
          const float dlt = Sh * __frcp_rn(gh);
          float nh, nl;
          ff_add(zmh, zml, dlt, 0.f, nh, nl);
          nz[m] = make_float2(nh, nl);
          r2f = fmaf(Rh, Rh, r2f);
          z2f = fmaf(zmh, zmh, z2f);
        }
      }
    }
  } else {
    const double* z = c1 ? z64_1 : z64_0;
    double* nz = c1 ? z64_0 : z64_1;
    const double ys = st->ys64;
    const double ts = theta[nstar];
    const double lam = st->lam;
    const double dlam = st->dlam;   // non-autonomous step (0: off)
    const int rounds = (n + gstride - 1) / gstride;
    for (int rd = 0; rd < rounds; ++rd) {
      const int m = g0 + rd * gstride;
      double acc = 0.0;
      float rsum = 0.f;
      if (m < n) {
        const int a = row_ptr[m], b = row_ptr[m + 1];
        int q = a + gl;
        for (;; q += 4 * V) {
          int c[4];
          float v[4];
          double zz[4];
          dom_fetch4<FIRST>(col_idx, vals, q, b, V, n, c, v, bad, rsum);
#pragma unroll
          for (int u = 0; u < 4; ++u) zz[u] = z[c[u]];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc = fma((double)v[u], zz[u], acc);
          if (q + 4 * V >= b) break;
        }
      }
#pragma unroll
      for (int o = V / 2; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (FIRST) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
      }
      if (FIRST && gl == 0 && m < n) rmax = fmaxf(rmax, rsum);
      if (gl == 0 && m < n) {
        const double zm = z[m];
        if (m == nstar) {
          nz[m] = 1.0;
          z2 += 1.0;
        } else {
          const double gap = ts - theta[m];
          const double t = acc - ys * zm;
          const double R = lam * t - gap * zm;
          nz[m] = (lam - dlam) * t / gap;
          r2 += R * R;
          z2 += zm * zm;
        }
      }
    }
  }
  if (FF) { r2 = (double)r2f; z2 = (double)z2f; }
  if (FIRST) {
    // row sums and validity of the first pass, visible before this block counts in
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    const bool wbad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      atomicMax(&st->row_bits, __float_as_uint(rmax));
      if (wbad) atomicExch(&st->bad_input, 1u);
      __threadfence();
    }
  }
  // block reduction, then the last block decides
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    z2 += __shfl_xor_sync(0xffffffffu, z2, o);
  }
  __shared__ double sr[2][8];
  __shared__ bool last;
  const int w = threadIdx.x >> 5;
  if (lane == 0) { sr[0][w] = r2; sr[1][w] = z2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R2 = 0.0, Z2 = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { R2 += sr[0][q]; Z2 += sr[1][q]; }
    part[2 * blockIdx.x] = R2;
    part[2 * blockIdx.x + 1] = Z2;
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // deterministic final reduction by the last block
  double R2 = 0.0, Z2 = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
    R2 += ((volatile double*)part)[2 * q];
    Z2 += ((volatile double*)part)[2 * q + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    R2 += __shfl_xor_sync(0xffffffffu, R2, o);
    Z2 += __shfl_xor_sync(0xffffffffu, Z2, o);
  }
  __syncthreads();
  if (lane == 0) { sr[0][w] = R2; sr[1][w] = Z2; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  R2 = 0.0; Z2 = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { R2 += sr[0][q]; Z2 += sr[1][q]; }
  dom_decide<FF, FIRST>(st, theta[nstar], R2, Z2);
}

// The pass as a kernel of its own per variant: the first pass (k = 0; it validates
// the CSR data and forms the row sums) needs more registers than the others, which
// keep the occupancy of the plain pass.
template <bool FF, int V, bool FIRST>
__global__ void __launch_bounds__(256) k_dom_iter(int n, const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col_idx,
                                                  const float* __restrict__ vals,
                                                  const float* __restrict__ th_hi,
                                                  const float* __restrict__ th_lo,
                                                  const double* __restrict__ theta,
                                                  float2* __restrict__ z0,
                                                  float2* __restrict__ z1,
                                                  double* __restrict__ z64_0,
                                                  double* __restrict__ z64_1,
                                                  double* __restrict__ part, DomState* st) {
  if (st->status != ST_RUNNING) return;
  dom_iter_body<FF, V, FIRST>(n, row_ptr, col_idx, vals, th_hi, th_lo, theta, z0, z1, z64_0,
                              z64_1, part, st);
}

// Output: z (float-float or FP64) of the assessed iterate -> FP64.
__global__ void k_dom_out(int n, const float2* __restrict__ z0, const float2* __restrict__ z1,
                          const double* __restrict__ z64_0, const double* __restrict__ z64_1,
                          int ff, double* __restrict__ out, const DomState* st) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const bool c1 = st->cur != 0;
  if (ff) {
    const float2 v = c1 ? z1[m] : z0[m];
    out[m] = f2d_bits(v.x) + f2d_bits(v.y);
  } else {
    out[m] = c1 ? z64_1[m] : z64_0[m];
  }
}

// z_0 from a caller's start vector v: z_m = v_m / v_{n*} (the chart z_{n*} = 1) in
// FP64 and as float pairs, and the residual scale as k_dom_init forms it.  A zero or
// non-finite v_{n*}, or any non-finite v_m, marks the input bad (the first decision
// then ends the solve with DPT_ERR_ARG).
__global__ void k_dom_start(int n, const double* __restrict__ v, float2* __restrict__ z,
                            double* __restrict__ z64, DomState* st) {
  const int nstar = st->nstar;
  const double piv = v[nstar];
  const bool piv_ok = piv != 0.0 && finite_bits(piv);
  bool bad = !piv_ok;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    const double vm = v[m];
    if (!finite_bits(vm)) bad = true;
    const double q = (m == nstar) ? 1.0 : (piv_ok ? vm / piv : 0.0);
    float h, l;
    split_double(q, h, l);
    z[m] = make_float2(h, l);
    if (z64) z64[m] = q;
  }
  if (bad) atomicExch(&st->bad_input, 1u);
}

__global__ void k_dom_init64(int n, double* z, const DomState* st) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) z[m] = (m == st->nstar) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int dom_grid(int n) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 132;
  }
  const int want = (n + 255) / 256;
  return want < 8 * nsm ? (want > 0 ? want : 1) : 8 * nsm;
}

int dom_blocks(int n) { return dom_grid(n); }

cudaError_t launch_dom_check(int n, int64_t nnz, const int32_t* row_ptr, DomState* st,
                             cudaStream_t s) {
  k_dom_check_rowptr<<<dom_grid(n), 256, 0, s>>>(n, nnz, row_ptr, st);
  return cudaGetLastError();
}

// The set-up before the loop: theta split and maxima, n*, the tie count, and the
// device-side gate that ends malformed or degenerate solves before any kernel follows
// row_ptr (the row pointer was checked by launch_dom_check just before).
cudaError_t launch_dom_setup(int n, const double* theta, float* th_hi, float* th_lo, DomState* st,
                             cudaStream_t s) {
  k_dom_setup<<<dom_grid(n), 256, 0, s>>>(n, theta, th_hi, th_lo, st);
  cudaError_t e = launch_dom_select(n, theta, st, s);
  if (e != cudaSuccess) return e;
  k_dom_gate<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_dom_select(int n, const double* theta, DomState* st, cudaStream_t s) {
  const int g = dom_grid(n);
  k_dom_argmax<<<g, 256, 0, s>>>(n, theta, st);
  k_dom_pick<<<1, 1, 0, s>>>(n, st);
  k_dom_ties<<<g, 256, 0, s>>>(n, theta, st);
  return cudaGetLastError();
}

cudaError_t launch_dom_start(int n, const double* v, float2* z, double* z64, DomState* st,
                             cudaStream_t s) {
  k_dom_start<<<dom_grid(n), 256, 0, s>>>(n, v, z, z64, st);
  return cudaGetLastError();
}

cudaError_t launch_dom_init(int n, float2* z, double* z64, int ff, DomState* st,
                            cudaStream_t s) {
  const int g = dom_grid(n);
  k_dom_init<<<g, 256, 0, s>>>(n, z, st);
  if (!ff) k_dom_init64<<<(n + 255) / 256, 256, 0, s>>>(n, z64, st);
  return cudaGetLastError();
}

cudaError_t launch_dom_iter(int n, int vlanes, int ff, const int32_t* row_ptr,
                            const int32_t* col_idx, const float* vals, const float* th_hi,
                            const float* th_lo, const double* theta, float2* z0, float2* z1,
                            double* z64_0, double* z64_1, double* part, DomState* st,
                            cudaStream_t s, bool first) {
  if (ff)
    k_dom_ystar<true><<<1, 32, 0, s>>>(n, row_ptr, col_idx, vals, z0, z1, z64_0, z64_1, st);
  else
    k_dom_ystar<false><<<1, 32, 0, s>>>(n, row_ptr, col_idx, vals, z0, z1, z64_0, z64_1, st);
  const int g = dom_grid(n);
#define DOM_LAUNCH1(FFV, VV, FI)                                                                \
  k_dom_iter<FFV, VV, FI><<<g, 256, 0, s>>>(n, row_ptr, col_idx, vals, th_hi, th_lo, theta, z0, \
                                            z1, z64_0, z64_1, part, st)
#define DOM_LAUNCH(FFV, VV) \
  do { if (first) DOM_LAUNCH1(FFV, VV, true); else DOM_LAUNCH1(FFV, VV, false); } while (0)
  if (ff) {
    switch (vlanes) {
      case 4: DOM_LAUNCH(true, 4); break;
      case 8: DOM_LAUNCH(true, 8); break;
      case 16: DOM_LAUNCH(true, 16); break;
      default: DOM_LAUNCH(true, 32); break;
    }
  } else {
    switch (vlanes) {
      case 4: DOM_LAUNCH(false, 4); break;
      case 8: DOM_LAUNCH(false, 8); break;
      case 16: DOM_LAUNCH(false, 16); break;
      default: DOM_LAUNCH(false, 32); break;
    }
  }
#undef DOM_LAUNCH
#undef DOM_LAUNCH1
  return cudaGetLastError();
}

cudaError_t launch_dom_out(int n, const float2* z0, const float2* z1, const double* z64_0,
                           const double* z64_1, int ff, double* out, const DomState* st,
                           cudaStream_t s) {
  k_dom_out<<<(n + 255) / 256, 256, 0, s>>>(n, z0, z1, z64_0, z64_1, ff, out, st);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Gather probe (a calibration of the roofline, not part of the map): the main pass's
// memory traffic without its arithmetic.  The same grid, the same groups of V lanes
// per row, the same four index loads in flight per lane and the same 8-byte gathers
// of an interleaved float pair per nonzero; each row's sum of the gathered high parts
// is written out so that no load can be dropped.  Reads 4 B of index per nonzero (no
// values) and writes 4 B per row.
// ---------------------------------------------------------------------------
template <int V>
__global__ void __launch_bounds__(256) k_probe_gather(int n, const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col_idx,
                                                      const float2* __restrict__ z,
                                                      float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int gl = lane & (V - 1);
  const int groups_per_block = blockDim.x / V;
  const int g0 = blockIdx.x * groups_per_block + threadIdx.x / V;
  const int gstride = gridDim.x * groups_per_block;
  const int rounds = (n + gstride - 1) / gstride;
  for (int rd = 0; rd < rounds; ++rd) {
    const int m = g0 + rd * gstride;
    float acc = 0.f;
    if (m < n) {
      const int a = row_ptr[m], b = row_ptr[m + 1];
      for (int q = a + gl;; q += 4 * V) {
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int qq = q + u * V;
          // the probe does not validate its input: out-of-range indices are clamped
          c[u] = qq < b ? min(max(col_idx[qq], 0), n - 1) : 0;
        }
        float2 zz[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) zz[u] = z[c[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += zz[u].x;
        if (q + 4 * V >= b) break;
      }
    }
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (gl == 0 && m < n) y[m] = acc;
  }
}

cudaError_t launch_probe_gather(int n, int vlanes, const int32_t* row_ptr, const int32_t* col_idx,
                                const float2* z, float* y, cudaStream_t s) {
  const int g = dom_grid(n);
  switch (vlanes) {
    case 4: k_probe_gather<4><<<g, 256, 0, s>>>(n, row_ptr, col_idx, z, y); break;
    case 8: k_probe_gather<8><<<g, 256, 0, s>>>(n, row_ptr, col_idx, z, y); break;
    case 16: k_probe_gather<16><<<g, 256, 0, s>>>(n, row_ptr, col_idx, z, y); break;
    default: k_probe_gather<32><<<g, 256, 0, s>>>(n, row_ptr, col_idx, z, y); break;
  }
  return cudaGetLastError();
}

}  // namespace dpt
