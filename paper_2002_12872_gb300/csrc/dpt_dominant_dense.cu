// Dominant eigenvector with a dense perturbation: the single-vector map of
// arXiv:2002.12872 (Eq. (single_line_dyn), Sec. II.H) with a GEMV in place of the
// CSR SpMV of dpt_dominant.cu.  For n* (the unperturbed level followed) and the
// iterate z (z_{n*} = 1):
//     y = Delta z,  y* = y_{n*},  E = theta_{n*} + lambda y*,
//     R_m = lambda (y_m - y* z_m) - (theta_{n*} - theta_m) z_m      (m != n*),
//     z'_m = z_m + R_m / (theta_{n*} - theta_m),
// where R is the eigen-residual (M z - E z)_m of the iterate z, so its norm is the
// convergence test.
//
// Each iteration streams Delta (FP64, column-major) from HBM once: the GEMV is
// HBM-bound at 8 bytes and 2 flops per entry.  Its arithmetic avoids the FP64 pipe,
// which on this GPU is slower than HBM even at one operation per entry: each entry
// is split into a float pair with integer operations and multiplied with z held as
// float-float, the row sums kept in float-float (FF = true, DPT_PREC_MIXED).
// FF = false is the literal FP64 arithmetic, the comparator.
//
// Kernels per iteration:
//   k_dd_gemv    grid (row blocks of 256 VEC rows) x (column slices); each thread
//                owns VEC adjacent rows (one 16-byte load per column for VEC = 2)
//                and writes its slice partial of y for them;
//   k_dd_update  one thread per row: sums the partials in slice order (y, and so
//                every result, is deterministic), applies the map, reduces the
//                norms; the last block takes the decision.
// The first pass (on z_0, its own kernel instances) also tests every entry (finite;
// below 2^128 in magnitude for the float-float split, split_double_fast) and sums |Delta| per row for
// the residual scale s = max|theta| + |lambda| max_m sum_k |Delta_mk|.
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

namespace {

constexpr int DD_THREADS = 256;
constexpr int DD_MAX_SLICE = 2048;   // columns of z staged in shared memory per block

// (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void dd_add(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  fast_two_sum(s, e, rh, rl);
}

// (ah, al) += (dh + dl) (zh + zl), the dl zl term dropped (below 2^-48 relative)
__device__ __forceinline__ void dd_fma(float dh, float dl, float zh, float zl, float& ah,
                                       float& al) {
  float p, pe;
  two_prod(dh, zh, p, pe);
  pe = fmaf(dh, zl, fmaf(dl, zh, pe));
  float s, e;
  two_sum(ah, p, s, e);
  e += al + pe;
  fast_two_sum(s, e, ah, al);
}

// (ah, al) (bh, bl)
__device__ __forceinline__ void dd_mul(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  float p, pe;
  two_prod(ah, bh, p, pe);
  pe = fmaf(ah, bl, fmaf(al, bh, pe));
  fast_two_sum(p, pe, rh, rl);
}

template <int VEC> struct DDVec;
template <> struct DDVec<1> {
  using T = double;
  static __device__ __forceinline__ double get(const T& v, int) { return v; }
};
template <> struct DDVec<2> {
  using T = double2;
  static __device__ __forceinline__ double get(const T& v, int i) { return i ? v.y : v.x; }
};

}  // namespace

// theta -> float-float, finiteness, max |theta| and the largest theta.
__global__ void k_dd_setup(int n, const double* __restrict__ theta, float* __restrict__ th_hi,
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

// Slice partials of y = Delta z.  Block (row block, column slice); thread t owns
// rows m = (block row offset + t) VEC .. + VEC - 1 and walks the slice's columns,
// eight 8*VEC-byte loads in flight.  VEC divides n and the leading dimension.
// FIRST (the pass on z_0): also the |Delta| row sums and the entry checks.
template <bool FF, int VEC, bool FIRST>
__global__ void __launch_bounds__(DD_THREADS) k_dd_gemv(DDParams p) {
  const DomState* st = p.st;
  if (st->status != ST_RUNNING) return;
  const bool c1 = st->cur != 0;
  const int n = p.n;
  const int k0 = blockIdx.y * p.slice;
  const int kn = min(n - k0, p.slice);
  __shared__ __align__(16) float2 zs[FF ? DD_MAX_SLICE : 1];
  __shared__ __align__(16) double zs64[FF ? 1 : DD_MAX_SLICE];
  if (FF) {
    const float2* __restrict__ z = c1 ? p.z1 : p.z0;
    for (int q = threadIdx.x; q < kn; q += DD_THREADS) zs[q] = z[k0 + q];
  } else {
    const double* __restrict__ z = c1 ? p.z64_1 : p.z64_0;
    for (int q = threadIdx.x; q < kn; q += DD_THREADS) zs64[q] = z[k0 + q];
  }
  __syncthreads();
  const int m = (blockIdx.x * DD_THREADS + threadIdx.x) * VEC;
  if (m >= n) return;
  using VT = typename DDVec<VEC>::T;
  const int64_t ldv = p.ld / VEC;
  const VT* __restrict__ col = reinterpret_cast<const VT*>(p.delta + (int64_t)k0 * p.ld + m);
  float ah[VEC], al[VEC], ra[VEC];
  double acc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) { ah[v] = 0.f; al[v] = 0.f; ra[v] = 0.f; acc[v] = 0.0; }
  bool bad = false;
  auto step = [&](const VT& dv, int kk) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const double d = DDVec<VEC>::get(dv, v);
      if (FF) {
        float dh, dl;
        split_double_fast(d, dh, dl);
        const float2 zz = zs[kk];
        dd_fma(dh, dl, zz.x, zz.y, ah[v], al[v]);
        if (FIRST) { ra[v] += fabsf(dh); bad |= beyond_float(d); }
      } else {
        acc[v] = fma(d, zs64[kk], acc[v]);
        if (FIRST) { ra[v] += fabsf((float)d); bad |= !finite_bits(d); }
      }
    }
  };
  int k = 0;
  for (; k + 8 <= kn; k += 8) {
    VT d[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) d[u] = col[(int64_t)(k + u) * ldv];
#pragma unroll
    for (int u = 0; u < 8; ++u) step(d[u], k + u);
  }
  for (; k < kn; ++k) step(col[(int64_t)k * ldv], k);
  const int64_t o = (int64_t)blockIdx.y * n + m;
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    if (FF) p.ypart[o + v] = make_float2(ah[v], al[v]);
    else p.ypart64[o + v] = acc[v];
    if (FIRST) p.rowabs[o + v] = ra[v];
  }
  if (FIRST && bad) atomicExch(&p.st->bad_input, 1u);
}

// Map, norms and decision.  One thread per row; every block forms y* from the
// partials of row n* in the same fixed order (one warp, lanes striding over the
// slices, then a fixed shuffle tree), so all blocks use the same y*.
template <bool FF, bool FIRST>
__global__ void __launch_bounds__(DD_THREADS) k_dd_update(DDParams p) {
  DomState* st = p.st;
  if (st->status != ST_RUNNING) return;
  constexpr bool first = FIRST;
  const bool c1 = st->cur != 0;
  const int n = p.n, ns = p.nslices;
  const int nstar = st->nstar;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ float ys_sh[2];
  __shared__ double ys_64;
  if (w == 0) {
    float h = 0.f, l = 0.f;
    double y64 = 0.0;
    for (int q = lane; q < ns; q += 32) {
      if (FF) {
        const float2 v = p.ypart[(int64_t)q * n + nstar];
        dd_add(h, l, v.x, v.y, h, l);
      } else {
        y64 += p.ypart64[(int64_t)q * n + nstar];
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      if (FF) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        dd_add(h, l, oh, ol, h, l);
      } else {
        y64 += __shfl_xor_sync(0xffffffffu, y64, o);
      }
    }
    if (lane == 0) { ys_sh[0] = h; ys_sh[1] = l; ys_64 = y64; }
  }
  __syncthreads();
  float r2f = 0.f, z2f = 0.f, rs = 0.f;
  double r2 = 0.0, z2 = 0.0;
  const int m = blockIdx.x * DD_THREADS + threadIdx.x;
  if (m < n) {
    if (first)
      for (int q = 0; q < ns; ++q) rs += p.rowabs[(int64_t)q * n + m];
    // y_m: partials in slice order, four loads ahead
    float yh = 0.f, yl = 0.f;
    double y64 = 0.0;
    int q = 0;
    for (; q + 4 <= ns; q += 4) {
      if (FF) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = p.ypart[(int64_t)(q + u) * n + m];
#pragma unroll
        for (int u = 0; u < 4; ++u) dd_add(yh, yl, v[u].x, v[u].y, yh, yl);
      } else {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = p.ypart64[(int64_t)(q + u) * n + m];
#pragma unroll
        for (int u = 0; u < 4; ++u) y64 += v[u];
      }
    }
    for (; q < ns; ++q) {
      if (FF) {
        const float2 v = p.ypart[(int64_t)q * n + m];
        dd_add(yh, yl, v.x, v.y, yh, yl);
      } else {
        y64 += p.ypart64[(int64_t)q * n + m];
      }
    }
    if (FF) {
      const float2* z = c1 ? p.z1 : p.z0;
      float2* nz = c1 ? p.z0 : p.z1;
      const float2 zm2 = z[m];
      const float zmh = zm2.x, zml = zm2.y;
      if (m == nstar) {
        nz[m] = make_float2(1.f, 0.f);
        z2f = 1.f;
      } else {
        // R = lambda (y - y* z) - gap z, in float-float
        float t1h, t1l, t2h, t2l, gh, gl, uh, ul, vh, vl, Rh, Rl;
        dd_mul(ys_sh[0], ys_sh[1], zmh, zml, t1h, t1l);
        dd_add(yh, yl, -t1h, -t1l, t2h, t2l);
        dd_mul(st->lam_hi, st->lam_lo, t2h, t2l, uh, ul);
        ff_sub(p.th_hi[nstar], p.th_lo[nstar], p.th_hi[m], p.th_lo[m], gh, gl);
        dd_mul(gh, gl, zmh, zml, vh, vl);
        dd_add(uh, ul, -vh, -vl, Rh, Rl);
        // the step applies lambda - dlam: R_step = R - dlam (y - y* z)
        float Sh = Rh;
        const float dlh = st->dlam_hi;
        if (dlh != 0.f) {
          float wh, wl, sl;
          dd_mul(dlh, st->dlam_lo, t2h, t2l, wh, wl);
          dd_add(Rh, Rl, -wh, -wl, Sh, sl);
        }
        const float dlt = Sh * __frcp_rn(gh);
        float nh, nl;
        dd_add(zmh, zml, dlt, 0.f, nh, nl);
        nz[m] = make_float2(nh, nl);
        r2f = Rh * Rh;
        z2f = zmh * zmh;
      }
    } else {
      const double* z = c1 ? p.z64_1 : p.z64_0;
      double* nz = c1 ? p.z64_0 : p.z64_1;
      const double zm = z[m];
      if (m == nstar) {
        nz[m] = 1.0;
        z2 = 1.0;
      } else {
        const double gap = p.theta[nstar] - p.theta[m];
        const double t = y64 - ys_64 * zm;
        const double R = st->lam * t - gap * zm;
        nz[m] = (st->lam - st->dlam) * t / gap;
        r2 = R * R;
        z2 = zm * zm;
      }
    }
  }
  if (FF) { r2 = (double)r2f; z2 = (double)z2f; }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    z2 += __shfl_xor_sync(0xffffffffu, z2, o);
    rs = fmaxf(rs, __shfl_xor_sync(0xffffffffu, rs, o));
  }
  __shared__ double sr[2][DD_THREADS / 32];
  __shared__ float srs[DD_THREADS / 32];
  __shared__ bool last;
  if (lane == 0) { sr[0][w] = r2; sr[1][w] = z2; srs[w] = rs; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R2 = 0.0, Z2 = 0.0;
    float RS = 0.f;
    for (int q = 0; q < DD_THREADS / 32; ++q) {
      R2 += sr[0][q];
      Z2 += sr[1][q];
      RS = fmaxf(RS, srs[q]);
    }
    p.part[2 * blockIdx.x] = R2;
    p.part[2 * blockIdx.x + 1] = Z2;
    if (first) atomicMax(&st->row_bits, __float_as_uint(RS));
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // deterministic final reduction by the last block
  double R2 = 0.0, Z2 = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += DD_THREADS) {
    R2 += ((volatile double*)p.part)[2 * q];
    Z2 += ((volatile double*)p.part)[2 * q + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    R2 += __shfl_xor_sync(0xffffffffu, R2, o);
    Z2 += __shfl_xor_sync(0xffffffffu, Z2, o);
  }
  __syncthreads();
  if (lane == 0) { sr[0][w] = R2; sr[1][w] = Z2; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  R2 = 0.0;
  Z2 = 0.0;
  for (int q = 0; q < DD_THREADS / 32; ++q) { R2 += sr[0][q]; Z2 += sr[1][q]; }
  volatile DomState* vs = st;
  vs->blocks_done = 0;
  if (first)
    vs->s = (double)__uint_as_float(vs->absmax_bits) +
            fabs(vs->lam) * (double)__uint_as_float(vs->row_bits);
  // eigenvalue of the iterate that was just assessed
  if (FF) {
    vs->ys_hi = ys_sh[0];
    vs->ys_lo = ys_sh[1];
    vs->E = p.theta[nstar] + vs->lam * ((double)ys_sh[0] + (double)ys_sh[1]);
  } else {
    vs->ys64 = ys_64;
    vs->E = p.theta[nstar] + vs->lam * ys_64;
  }
  const double rho = sqrt(R2) / (vs->s * sqrt(Z2));
  vs->rho = rho;
  if (vs->bad_input) { vs->status = ST_BADINPUT; return; }
  if (!(rho == rho) || isinf(rho)) { vs->status = ST_DIVERGED; return; }
  if (rho <= vs->tol) { vs->status = ST_CONVERGED; return; }
  if (rho < vs->best) { vs->best = rho; vs->grown = 0; }
  else if (rho > 10.0 * vs->best) {
    if (++vs->grown >= 20) { vs->status = ST_DIVERGED; return; }
  } else vs->grown = 0;
  if (vs->k >= vs->max_iter) { vs->status = ST_MAXITER; return; }
  vs->k = vs->k + 1;
  vs->cur = vs->k & 1;
  dom_ramp_advance(vs);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int dd_sms() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 132;
  }
  return nsm;
}

// Column slice width: enough blocks for two waves of eight blocks per SM, a
// multiple of 8 columns in [64, DD_MAX_SLICE].
int dd_slice(int n, int vec, int nsm) {
  const int rows = DD_THREADS * vec;
  const int rb = (n + rows - 1) / rows;
  const int target = 16 * nsm;
  const int want = (target + rb - 1) / rb;
  int w = (n + want - 1) / want;
  w = (w + 7) / 8 * 8;
  if (w < 64) w = 64;
  if (w > DD_MAX_SLICE) w = DD_MAX_SLICE;
  return w;
}

void dd_plan(DDParams& p, bool aligned16) {
  p.vec = (aligned16 && p.n % 2 == 0 && p.ld % 2 == 0) ? 2 : 1;
  p.slice = dd_slice(p.n, p.vec, dd_sms());
  p.nslices = (p.n + p.slice - 1) / p.slice;
}

int dd_update_blocks(int n) { return (n + DD_THREADS - 1) / DD_THREADS; }

cudaError_t launch_dd_setup(int n, const double* theta, float* th_hi, float* th_lo, DomState* st,
                            cudaStream_t s) {
  const int want = (n + 255) / 256;
  const int g = want < 8 * dd_sms() ? want : 8 * dd_sms();
  k_dd_setup<<<g, 256, 0, s>>>(n, theta, th_hi, th_lo, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dom_select(n, theta, st, s);
}

cudaError_t launch_dd_gemv(const DDParams& p, int ff, int first, cudaStream_t s) {
  const int rows = DD_THREADS * p.vec;
  const dim3 g((p.n + rows - 1) / rows, p.nslices);
#define DD_GEMV(FFV, VV, FIRSTV) k_dd_gemv<FFV, VV, FIRSTV><<<g, DD_THREADS, 0, s>>>(p)
  if (ff) {
    if (p.vec == 2) { if (first) DD_GEMV(true, 2, true); else DD_GEMV(true, 2, false); }
    else { if (first) DD_GEMV(true, 1, true); else DD_GEMV(true, 1, false); }
  } else {
    if (p.vec == 2) { if (first) DD_GEMV(false, 2, true); else DD_GEMV(false, 2, false); }
    else { if (first) DD_GEMV(false, 1, true); else DD_GEMV(false, 1, false); }
  }
#undef DD_GEMV
  return cudaGetLastError();
}

cudaError_t launch_dd_update(const DDParams& p, int ff, int first, cudaStream_t s) {
  const int g = dd_update_blocks(p.n);
  if (ff) {
    if (first) k_dd_update<true, true><<<g, DD_THREADS, 0, s>>>(p);
    else k_dd_update<true, false><<<g, DD_THREADS, 0, s>>>(p);
  } else {
    if (first) k_dd_update<false, true><<<g, DD_THREADS, 0, s>>>(p);
    else k_dd_update<false, false><<<g, DD_THREADS, 0, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace dpt
