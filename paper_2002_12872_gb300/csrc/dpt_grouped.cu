// Grouped full-spectrum DPT: many independent problems of uneven size advanced
// together, one launch per stage of an iteration for the whole group.
//
// Each problem p has an entry in a device-resident table (GProb): its size, its
// work arrays inside one arena, its own iteration state and its own TMA
// descriptors.  Kernels walk flat work lists of (problem, tile) items built once on
// the host, so one launch covers every problem; items of problems that have
// already converged return at once, so every problem retires at its own
// convergence (arXiv:2002.12872: each problem is its own fixed-point iteration,
// Sec. II.B; the arithmetic per problem is that of the single-problem mixed path,
// see dpt_full_mixed.cu).
//
// Operands: as in the single solve, Delta 2^sig as FP16 slices and each increment as
// FP16 scaled by a power of two chosen from the size of the previous one
// (IterState::sig, sexp[2]); the scales are exact, so every product and partial is
// unscaled by a power of two (see dpt_full_mixed.cu).  Up to three slices (33
// significant bits of Delta): the grouped solves have no FP64 finish of the columns
// two slices leave uncertain (measured: a strongly coupled complex n = 3 problem
// missed the 1e-10 eigenvalue bar with two), and the slice rule drops to two and one
// as the increments shrink by 2^-11 and 2^-22.
//
// Tile shape per problem (chosen on the host from n): M = 128 rows, N = the
// smallest multiple of 32 that covers n in ceil(n / 256) column tiles, so small
// problems do not pay for 256-wide tiles.  The host orders the tile list by cost
// (K extent x width, largest first) so that the round-robin assignment to the
// persistent CTAs stays balanced across problems of very different size.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

constexpr int G_BM = 128;
constexpr int G_BNMAX = 256;
constexpr int G_BK = 64;
constexpr int G_UK = 16;
constexpr int G_STAGES = 4;
constexpr int G_A_TILE = G_BM * G_BK * 2;
constexpr int G_B_TILE = G_BNMAX * G_BK * 2;
constexpr int G_EPI_WARPS = 8;
constexpr int G_NTHREADS = 64 + 32 * G_EPI_WARPS;
constexpr int G_XCH = 32;
constexpr int G_SMEM_TILES = G_STAGES * (G_A_TILE + G_B_TILE);
constexpr int G_SMEM_X = G_BM * G_XCH * 4;

struct __align__(16) GSmem {
  uint64_t full[G_STAGES];
  uint64_t empty[G_STAGES];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint32_t tmem_base;
  float e[2 * G_BNMAX];       // e_i of the tile's columns ((re, im) pairs if complex)
  float dprev[2 * G_BNMAX];   // d_{k-1,i}, likewise
  float thh[G_BNMAX];
  float thl[G_BNMAX];
};
constexpr int G_SMEM_BYTES = G_SMEM_TILES + G_SMEM_X + 1024 + (int)sizeof(GSmem);

__device__ __forceinline__ bool g_running(const GProb* P) {
  return *((volatile const int*)&P->st->status) == ST_RUNNING;
}

// ---------------------------------------------------------------------------
// theta checks: finite and pairwise distinct (one block per problem).
// ---------------------------------------------------------------------------
// A problem found invalid stops here (its status leaves ST_RUNNING exactly once,
// so the group's running count drops exactly once).
__device__ __forceinline__ void g_fail(const GProb* P, int code, int* running) {
  if (atomicCAS(&P->st->status, ST_RUNNING, code) == ST_RUNNING) atomicSub(running, 1);
}

// Grid (problems, chunks of 128 indices i); thread i compares theta_i with every
// theta_j, j > i, chunk by chunk: the block stages each chunk of 128 equality keys of
// theta_j in shared memory, so the comparisons are 64-bit integer compares against
// broadcast reads (the FP64 pipe of GB300 is slow; equal finite doubles have equal
// keys, eq_key).  The chunk's max |theta| goes to the state by atomicMax on the bits of
// a non-negative double (which order like the values).
__global__ void __launch_bounds__(128) k_g_check_theta(const GProb* __restrict__ probs,
                                                       int count, int* running) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const GProb* P = probs + p;
  const int n = P->n;
  const int c0 = blockIdx.y * 128;
  if (c0 >= n) return;
  const int i = c0 + threadIdx.x;
  const double* __restrict__ th = P->theta;
  __shared__ unsigned long long tk[128];
  double amax = 0.0;
  bool fin = false;
  unsigned long long ki = 0ull;
  if (i < n) {
    const double ti = th[i];
    fin = finite_bits(ti);
    if (!fin) g_fail(P, ST_BADINPUT, running);
    else { amax = fabs(ti); ki = eq_key(ti); }
  }
  bool dup = false;
  for (int j0 = c0; j0 < n; j0 += 128) {
    __syncthreads();
    // entries past n hold a pattern no finite value has
    tk[threadIdx.x] = (j0 + (int)threadIdx.x < n) ? eq_key(th[j0 + threadIdx.x]) : ~0ull;
    __syncthreads();
    // the diagonal chunk: only j > i; later chunks: all 128
    const int q0 = (j0 == c0) ? (int)threadIdx.x + 1 : 0;
#pragma unroll 8
    for (int q = 0; q < 128; ++q) dup |= (q >= q0) & (tk[q] == ki);
  }
  if (fin && dup) g_fail(P, ST_DEGENERATE, running);
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0 && amax > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&P->st->theta_max),
              (unsigned long long)__double_as_longlong(amax));
}

// ---------------------------------------------------------------------------
// The FP16 scales of each problem, from its Delta and theta (before the slicing):
// sig places max |Delta| 2^sig in [2^14, 2^15) (entries of the largest slice keep 11
// bits; the second slice takes what the first drops), and the first increment's scale
// sexp[0] places its bound |lambda| max |Delta_ji| / |theta_i - theta_j| at 2^13 (as
// the single solve's k_delta_scales).  Work item: a 128 x 128 tile of iteration 0
// (for a complex problem 128 columns by 64 complex rows); a thread owns a row (a
// complex row: two threads, half of the columns each).  Only integer and float
// operations per entry: magnitudes from the doubles' high words, gaps from theta in
// float-float.  The maxima reach the state by atomicMax on non-negative float /
// double-high-word bits; the problem's last item sets the scales.
// ---------------------------------------------------------------------------
// |v| from the high word of a double (sign cleared): exact to 20 fraction bits as a
// float, 0 below the float range, +inf above it (the slicing rejects those inputs).
// Integer operations only: the FP64 pipe is the GB300's slowest.
__device__ __forceinline__ float abs_hi_float(unsigned hw) {
  const unsigned e = hw >> 20;
  return (e > 896u && e < 1151u) ? __uint_as_float(((e - 896u) << 23) | ((hw & 0xFFFFFu) << 3))
                                 : (e >= 1151u ? __int_as_float(0x7f800000) : 0.f);
}

template <bool CPLX>
__global__ void __launch_bounds__(128) k_g_scales(const GProb* __restrict__ probs,
                                                  const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if ((P->cplx != 0) != CPLX || !g_running(P)) return;
  IterState* st = P->st;
  const int n = P->n;
  const int i0 = it.y * 128, i1 = min(n, i0 + 128);
  // theta of the tile's columns as float-float (the gaps of near-degenerate levels
  // survive in the low part)
  __shared__ float thh[128], thl[128];
  {
    const int i = i0 + (int)threadIdx.x;
    float h = 0.f, l = 0.f;
    if (i < n) split_double(P->theta[i], h, l);
    thh[threadIdx.x] = h;
    thl[threadIdx.x] = l;
  }
  __syncthreads();
  // a real tile's 128 rows: one per thread; a complex tile's 64 complex rows: two
  // threads per row, each taking half of the columns
  const int r = CPLX ? (int)(threadIdx.x & 63) : (int)threadIdx.x;
  const int j = (CPLX ? it.z * 64 : it.z * 128) + r;
  const int ia = CPLX ? i0 + 64 * (int)(threadIdx.x >> 6) : i0;
  const int ib_end = CPLX ? min(i1, ia + 64) : i1;
  unsigned hmax = 0u;
  float gmax = 0.f;
  if (j < n) {
    float tjh, tjl;
    split_double(P->theta[j], tjh, tjl);
    // eight columns' loads in flight per thread (a small problem's pass is one block
    // whose time is its load latencies)
    for (int ib = ia; ib < ib_end; ib += 8) {
      unsigned hw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = ib + u;
        hw[u] = 0u;
        if (i < ib_end) {
          if (CPLX) {
            const double2 v =
                reinterpret_cast<const double2*>(P->delta_in)[(int64_t)i * P->ld_in + j];
            hw[u] = max((unsigned)__double2hiint(v.x) & 0x7FFFFFFFu,
                        (unsigned)__double2hiint(v.y) & 0x7FFFFFFFu);
          } else {
            hw[u] = (unsigned)__double2hiint(P->delta_in[(int64_t)i * P->ld_in + j]) & 0x7FFFFFFFu;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = ib + u;
        hmax = max(hmax, hw[u]);
        if (i < ib_end && i != j) {
          float g = thh[i - i0] - tjh;
          if (g == 0.f) g = thl[i - i0] - tjl;
          // NaN never wins fmaxf
          gmax = fmaxf(gmax, abs_hi_float(hw[u]) * rcp_approx(fabsf(g)));
        }
      }
    }
  }
  hmax = __reduce_max_sync(0xffffffffu, hmax);
  const unsigned gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));
  __shared__ unsigned wh[4], wg[4];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { wh[w] = hmax; wg[w] = gb; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const unsigned a = max(max(wh[0], wh[1]), max(wh[2], wh[3]));
  const unsigned b = max(max(wg[0], wg[1]), max(wg[2], wg[3]));
  atomicMax(&st->amax_bits, a);
  atomicMax(&st->g0max_bits, b);
  __threadfence();
  const unsigned nitems = (unsigned)(P->ntm * ((n + 127) / 128));
  if (atomicAdd(&st->blocks_done, 1u) != nitems - 1u) return;
  __threadfence();
  volatile IterState* vs = st;
  const unsigned hm = vs->amax_bits;
  int sig = 0;
  if (hm != 0u) sig = 14 - ((int)((hm >> 20) & 0x7FFu) - 1023);   // max |Delta| < 2^(e+1)
  sig = max(-120, min(120, sig));
  const double lam = vs->lam;
  const double g0 = (double)__uint_as_float(vs->g0max_bits);
  const int s0 = dt_scale_exp(fabs(lam) * g0, 13, sig, lam);
  vs->sig = sig;
  vs->sexp[0] = s0;
  vs->sexp[1] = s0;
  vs->blocks_done = 0;
}

// ---------------------------------------------------------------------------
// Delta -> three FP16 slices of Delta 2^sig (row-major) and theta -> float-float.
// Work item: (problem, 64-column block, 32-row block); block 32 x 8.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_g_prep(const GProb* __restrict__ probs,
                                                const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (!g_running(P)) return;
  __shared__ double tile[32][65];
  const int n = P->n, ld = P->ld;
  const int by = it.z * 32;
  if (it.y == 0 && threadIdx.y == 0) {   // theta split, rows by..by+31
    const int j = by + threadIdx.x;
    if (j < ld) {
      float h = 0.f, l = 0.f;
      if (j < n) split_double(P->theta[j], h, l);
      P->th_hi[j] = h;
      P->th_lo[j] = l;
    }
  }
  slice16_tile_32x64<3>(P->delta_in, P->ld_in, n, ld, 0, exp2i(P->st->sig), it.y * 64, by,
                        P->Dcat, P->cat_ld, &P->st->bad_input, tile);
}

// ---------------------------------------------------------------------------
// Iteration 0 (A_0 = I) in float-float; work item (problem, 128-col tile, 128-row tile).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_g_iter0(const GProb* __restrict__ probs,
                                                 const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (!g_running(P)) return;
  __shared__ float rows[4][128];
  const int n = P->n, ld = P->ld, ntm = P->ntm;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n0 = it.y * 128, m0 = it.z * 128, tm = it.z;
  const int r0 = 4 * lane, j0 = m0 + r0;
  const int64_t cat_ld = P->cat_ld;
  const float lam_hi = P->lam, lam_lo = P->lam_lo;
  // dt_0 stored as dt_0 2^sexp[0]; the slices hold Delta 2^sig
  const float qs = exp2i(P->st->sexp[0]), iqs = exp2i(-P->st->sexp[0]);
  const float isig = exp2i(-P->st->sig);
  const float4 thj_h = *reinterpret_cast<const float4*>(P->th_hi + j0);
  const float4 thj_l = *reinterpret_cast<const float4*>(P->th_lo + j0);
  const double* delta = P->delta_in;
  const int64_t ld_in = P->ld_in;
  float rowabs[4] = {0.f, 0.f, 0.f, 0.f};
  float mx = 0.f;
  // the warp's columns, each one's loads issued while the one before is computed
  const int cend = min(32, n - (n0 + 32 * w));
  float nth_h = 0.f, nth_l = 0.f;
  uint2 nD[3];
  double nv[4];
  auto fetch = [&](int i) {
    nth_h = P->th_hi[i];
    nth_l = P->th_lo[i];
    const __half* Drow = P->Dcat + (int64_t)i * cat_ld + j0;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) nD[sl] = *reinterpret_cast<const uint2*>(Drow + (int64_t)sl * ld);
#pragma unroll
    for (int e = 0; e < 4; ++e) nv[e] = (j0 + e < n) ? delta[(int64_t)i * ld_in + j0 + e] : 0.0;
  };
  if (cend > 0) fetch(n0 + 32 * w);
  for (int c = 0; c < cend; ++c) {
    const int i = n0 + 32 * w + c;
    const float thi_h = nth_h, thi_l = nth_l;
    uint2 D[3];
    double vv[4];
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) D[sl] = nD[sl];
#pragma unroll
    for (int e = 0; e < 4; ++e) vv[e] = nv[e];
    if (c + 1 < cend) fetch(i + 1);
    float4 oh, oL;
    uint32_t ob[4] = {0u, 0u, 0u, 0u};
    float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      float nh = 0.f, Ln = 0.f, dtn = 0.f;
      if (j < n) {
        const double v = vv[e];
        float vh, vl;
        split_double_fast(v, vh, vl);   // |v| < 2^128: checked by the slicing
        rowabs[e] += fabsf(vh);
        if (j == i) {
          nh = 1.f;
          a2 += 1.f;
          P->d[i] = v;
        } else {
          float pr, pe;
          two_prod(lam_hi, vh, pr, pe);
          pe = fmaf(lam_hi, vl, fmaf(lam_lo, vh, pe));
          float R0h, R0l;
          fast_two_sum(pr, pe, R0h, R0l);
          float gh, gl;
          ff_sub(thi_h, thi_l, f4(thj_h, e), f4(thj_l, e), gh, gl);
          // the remainder below keeps R_0 - Gap dt_0 exactly, so any reciprocal
          // close to 1/gap serves
          dtn = f16_scaled(R0h * rcp_approx(gh), qs, iqs, ob[e]);
          float q, qe;
          two_prod(gh, dtn, q, qe);
          qe = fmaf(gl, dtn, qe);
          Ln = (R0h - q) + (R0l - qe);
          nh = dtn;
          r2 = fmaf(R0h, R0h, r2);
          // e_1 2^sig from the slices (exact products)
          const float p1 = h_at(D[0], e) * dtn;
          const float p23 = fmaf(h_at(D[1], e), dtn, h_at(D[2], e) * dtn);
          float sh, se;
          two_sum(eh, p1, sh, se);
          se += el + p23;
          fast_two_sum(sh, se, eh, el);
          mx = fmaxf(mx, fabsf(dtn));
        }
      }
      f4set(oh, e, nh);
      f4set(oL, e, Ln);
    }
    const int64_t idx = (int64_t)i * ld + j0;
    st4(P->A_hi[1] + idx, oh);
    st4(P->A_lo[1] + idx, make_float4(0.f, 0.f, 0.f, 0.f));
    st4(P->L + idx, oL);
    *reinterpret_cast<uint2*>(P->dt[0] + idx) =
        make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
    warp_sum_ff(r2, a2, eh, el);
    eh *= isig;
    el *= isig;
    if (lane == 0) {
      P->part[((int64_t)0 * ntm + tm) * ld + i] = r2;
      P->part[((int64_t)1 * ntm + tm) * ld + i] = a2;
      P->part[((int64_t)2 * ntm + tm) * ld + i] = eh;
      P->part[((int64_t)3 * ntm + tm) * ld + i] = el;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) rows[w][r0 + e] = rowabs[e];
  __syncthreads();
  const int r = threadIdx.x;
  if (m0 + r < n)
    P->rowpart[(int64_t)it.y * ld + m0 + r] = ((rows[0][r] + rows[1][r]) + rows[2][r]) + rows[3][r];
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.f) atomicMax(&P->st->dmax_bits, __float_as_uint(mx));
}

// ===========================================================================
// Complex problems.  The product is the real GEMM of the interleaved embedding:
// embedded row 2j carries [Re D_jk, -Im D_jk] and row 2j+1 [Im D_jk, Re D_jk] at
// K = (2k, 2k+1), and a complex increment column stored (re, im) interleaved is
// the K-major B operand, so X rows (2j, 2j+1) = (Re, Im) of (Delta dt)_j.  Each
// epilogue lane's four consecutive rows are two complex elements.  theta and
// lambda are real.
// ===========================================================================

// Delta (complex, column-major, interleaved doubles) -> three FP16 slices of the
// embedding of Delta 2^sig; theta -> float-float.  Work item: (problem, 32 complex
// columns, 32 complex rows); block 32 x 8.  Each embedded row pair (2j, 2j+1) gets the
// two FP16 pairs (Re, -Im) and (Im, Re) of element (j, k) at columns (2k, 2k+1), one
// 4-byte store per row and slice, so a warp writes 128 contiguous bytes.
__global__ void __launch_bounds__(256) k_gc_prep(const GProb* __restrict__ probs,
                                                 const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (!g_running(P)) return;
  __shared__ double2 tile[32][33];
  const int n = P->n, ld = P->ld;
  const int bx = it.y * 32, by = it.z * 32;      // complex column k, complex row j
  const double2* __restrict__ delta = reinterpret_cast<const double2*>(P->delta_in);
  const int64_t ld_in = P->ld_in;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = by + threadIdx.x, k = bx + r;
    double2 v = make_double2(0.0, 0.0);
    if (j < n && k < n) {
      v = delta[(int64_t)k * ld_in + j];
      if (!finite_bits(v.x) || !finite_bits(v.y)) atomicExch(&P->st->bad_input, 1u);
    }
    tile[r][threadIdx.x] = v;    // tile[k - bx][j - by]
  }
  if (bx == 0 && threadIdx.y == 0) {
    const int j = by + threadIdx.x;
    if (j < n) {
      float h, l;
      split_double(P->theta[j], h, l);
      P->th_hi[j] = h;
      P->th_lo[j] = l;
    }
  }
  __syncthreads();
  const int64_t cat_ld = P->cat_ld;
  const int k = bx + threadIdx.x;                 // complex column written by this thread
  if (2 * k >= ld) return;
  const double sc = (double)exp2i(P->st->sig);
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = by + r;
    if (j >= n) break;
    const double2 v = (k < n) ? tile[threadIdx.x][r] : make_double2(0.0, 0.0);
    // entries beyond the float range after scaling: rejected (sig keeps the
    // largest below 2^15, so this is a non-finite or overflowing input)
    if (beyond_float(v.x * sc) || beyond_float(v.y * sc)) atomicExch(&P->st->bad_input, 1u);
    float rh, rl, ih, il;
    split_double(v.x * sc, rh, rl);
    split_double(v.y * sc, ih, il);
    __half* row0 = P->Dcat + (int64_t)(2 * j) * cat_ld + 2 * k;
    __half* row1 = row0 + cat_ld;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      // the last slice takes the low parts as well; the remainders are exact in float
      const float tr = sl == 2 ? rh + rl : rh, ti = sl == 2 ? ih + il : ih;
      const __half br = __float2half_rn(tr), bi = __float2half_rn(ti);
      // -Im rounds to -f16(Im): the slices of -Im are the negated slices of Im
      *reinterpret_cast<__half2*>(row0 + (int64_t)sl * ld) = __halves2half2(br, __hneg(bi));
      *reinterpret_cast<__half2*>(row1 + (int64_t)sl * ld) = __halves2half2(bi, br);
      rh = tr - __half2float(br);
      ih = ti - __half2float(bi);
    }
  }
}

// complex product a * b in float
__device__ __forceinline__ void cmulf(float ar, float ai, float br, float bi, float& rr, float& ri) {
  rr = fmaf(ar, br, -ai * bi);
  ri = fmaf(ar, bi, ai * br);
}

// Iteration 0 (A_0 = I) for a complex problem.  Work item (problem, 128-column
// tile, 128-embedded-row tile); lane l owns complex rows jc, jc + 1.
__global__ void __launch_bounds__(128) k_gc_iter0(const GProb* __restrict__ probs,
                                                  const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (!g_running(P)) return;
  __shared__ float rows[4][64];
  const int n = P->n, ld = P->ld, ntm = P->ntm;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n0 = it.y * 128, m0 = it.z * 128, tm = it.z;
  const int r0 = 4 * lane, jc0 = (m0 + r0) / 2;   // embedded rows m0+r0.., complex rows jc0, jc0+1
  const int64_t cat_ld = P->cat_ld;
  const float lam_hi = P->lam, lam_lo = P->lam_lo;
  // dt_0 stored as dt_0 2^sexp[0]; the slices hold Delta 2^sig
  const float qs = exp2i(P->st->sexp[0]), iqs = exp2i(-P->st->sexp[0]);
  const float isig = exp2i(-P->st->sig);
  const double2* delta = reinterpret_cast<const double2*>(P->delta_in);
  const int64_t ld_in = P->ld_in;
  float thj_h[2], thj_l[2];
  for (int e = 0; e < 2; ++e) {
    const int j = jc0 + e;
    thj_h[e] = j < n ? P->th_hi[j] : 0.f;
    thj_l[e] = j < n ? P->th_lo[j] : 0.f;
  }
  float rowabs[2] = {0.f, 0.f};
  float mx = 0.f;
  // the warp's columns, each one's loads issued while the one before is computed
  const int cend = min(32, n - (n0 + 32 * w));
  float nth_h = 0.f, nth_l = 0.f;
  uint2 nD[3];
  double2 nv[2];
  auto fetch = [&](int i) {
    nth_h = P->th_hi[i];
    nth_l = P->th_lo[i];
    // Delta(i, jc0..jc0+1) from embedded row 2i: (Re, -Im) pairs
    const __half* Drow = P->Dcat + (int64_t)(2 * i) * cat_ld + 2 * jc0;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) nD[sl] = *reinterpret_cast<const uint2*>(Drow + (int64_t)sl * ld);
#pragma unroll
    for (int e = 0; e < 2; ++e)
      nv[e] = (jc0 + e < n) ? delta[(int64_t)i * ld_in + jc0 + e] : make_double2(0.0, 0.0);
  };
  if (cend > 0) fetch(n0 + 32 * w);
  for (int c = 0; c < cend; ++c) {
    const int i = n0 + 32 * w + c;
    const float thi_h = nth_h, thi_l = nth_l;
    uint2 D[3];
    double2 vv[2];
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) D[sl] = nD[sl];
#pragma unroll
    for (int e = 0; e < 2; ++e) vv[e] = nv[e];
    if (c + 1 < cend) fetch(i + 1);
    float oh[4], oL[4];
    uint32_t ob[4] = {0u, 0u, 0u, 0u};
    float r2 = 0.f, a2 = 0.f, erh = 0.f, erl = 0.f, eih = 0.f, eil = 0.f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = jc0 + e;
      float dn[2] = {0.f, 0.f}, L2[2] = {0.f, 0.f}, A2[2] = {0.f, 0.f};
      if (j < n) {
        const double2 v = vv[e];
        float vh[2], vl[2];
        split_double_fast(v.x, vh[0], vl[0]);   // |v| < 2^128: checked by the slicing
        split_double_fast(v.y, vh[1], vl[1]);
        rowabs[e] += sqrtf(vh[0] * vh[0] + vh[1] * vh[1]);
        if (j == i) {
          A2[0] = 1.f;
          a2 += 1.f;
          P->d[2 * i] = v.x;
          P->d[2 * i + 1] = v.y;
        } else {
          float gh, gl;
          ff_sub(thi_h, thi_l, thj_h[e], thj_l[e], gh, gl);
          const float g = rcp_approx(gh);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            float pr, pe;
            two_prod(lam_hi, vh[q], pr, pe);
            pe = fmaf(lam_hi, vl[q], fmaf(lam_lo, vh[q], pe));
            float R0h, R0l;
            fast_two_sum(pr, pe, R0h, R0l);
            dn[q] = f16_scaled(R0h * g, qs, iqs, ob[2 * e + q]);
            float qq, qe;
            two_prod(gh, dn[q], qq, qe);
            qe = fmaf(gl, dn[q], qe);
            L2[q] = (R0h - qq) + (R0l - qe);
            A2[q] = dn[q];
            r2 = fmaf(R0h, R0h, r2);
          }
          // e_1 2^sig partial: Delta(i, j) 2^sig dt(j, i), slices exact
          float pr1, pi1, pr2, pi2;
          const float a1 = h_at(D[0], 2 * e), b1 = h_at(D[0], 2 * e + 1);
          pr1 = fmaf(a1, dn[0], b1 * dn[1]);          // a x + b' y   (b' = -Im)
          pi1 = fmaf(a1, dn[1], -b1 * dn[0]);         // a y - b' x
          const float a2s = h_at(D[1], 2 * e) + h_at(D[2], 2 * e);
          const float b2s = h_at(D[1], 2 * e + 1) + h_at(D[2], 2 * e + 1);
          pr2 = fmaf(a2s, dn[0], b2s * dn[1]);
          pi2 = fmaf(a2s, dn[1], -b2s * dn[0]);
          float sh, se;
          two_sum(erh, pr1, sh, se); se += erl + pr2; fast_two_sum(sh, se, erh, erl);
          two_sum(eih, pi1, sh, se); se += eil + pi2; fast_two_sum(sh, se, eih, eil);
          mx = fmaxf(mx, fmaxf(fabsf(dn[0]), fabsf(dn[1])));
        }
      }
      oh[2 * e] = A2[0]; oh[2 * e + 1] = A2[1];
      oL[2 * e] = L2[0]; oL[2 * e + 1] = L2[1];
    }
    const int64_t idx = (int64_t)i * ld + m0 + r0;
    st4(P->A_hi[1] + idx, make_float4(oh[0], oh[1], oh[2], oh[3]));
    st4(P->A_lo[1] + idx, make_float4(0.f, 0.f, 0.f, 0.f));
    st4(P->L + idx, make_float4(oL[0], oL[1], oL[2], oL[3]));
    *reinterpret_cast<uint2*>(P->dt[0] + idx) = make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
    warp_sum_ff(r2, a2, erh, erl);
    float z0 = 0.f, z1 = 0.f;
    warp_sum_ff(z0, z1, eih, eil);
    erh *= isig; erl *= isig; eih *= isig; eil *= isig;
    if (lane == 0) {
      P->part[((int64_t)0 * ntm + tm) * ld + i] = r2;
      P->part[((int64_t)1 * ntm + tm) * ld + i] = a2;
      P->part[((int64_t)2 * ntm + tm) * ld + i] = erh;
      P->part[((int64_t)3 * ntm + tm) * ld + i] = erl;
      P->part[((int64_t)4 * ntm + tm) * ld + i] = eih;
      P->part[((int64_t)5 * ntm + tm) * ld + i] = eil;
    }
  }
  rows[w][2 * lane] = rowabs[0];
  rows[w][2 * lane + 1] = rowabs[1];
  __syncthreads();
  if (threadIdx.x < 64) {
    const int r = threadIdx.x, j = m0 / 2 + r;
    if (j < n)
      P->rowpart[(int64_t)it.y * ld + j] = ((rows[0][r] + rows[1][r]) + rows[2][r]) + rows[3][r];
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.f) atomicMax(&P->st->dmax_bits, __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// Control.  Grid (problems, chunks of 64 columns); 4 threads per column sum every
// 4th tile partial.  Per column: the residual estimate of the assessed iterate,
// its eigenvalue read-out E = theta + lambda d (Sec. II.B), and d advanced by the
// new diagonal increment.  The chunk maxima of the residual (and, at the first
// control, of the row sums of |Delta|) reach the state by atomicMax; the last
// chunk of a problem to finish takes the problem's decision.
// ---------------------------------------------------------------------------
template <bool CPLX>
__global__ void __launch_bounds__(256) k_g_ctrl(const GProb* __restrict__ probs, int count,
                                                int* running) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const GProb* P = probs + p;
  if ((P->cplx != 0) != CPLX) return;
  IterState* st = P->st;
  if (st->status != ST_RUNNING) return;
  const int n = P->n, ld = P->ld, ntm = P->ntm;
  const int nchunk = (n + 63) / 64;
  if ((int)blockIdx.y >= nchunk) return;
  const int ntn128 = (n + 127) / 128;
  const bool first = (st->k == 0);
  __shared__ float sh[3][4][64];
  __shared__ double she[2][4][64];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  const int i = blockIdx.y * 64 + c;
  {
    float r2 = 0.f, a2 = 0.f, rs = 0.f;
    double er = 0.0, ei = 0.0;
    if (i < n) {
      const float* __restrict__ part = P->part;
      for (int t = g; t < ntm; t += 4) {
        r2 += part[((int64_t)0 * ntm + t) * ld + i];
        a2 += part[((int64_t)1 * ntm + t) * ld + i];
        er += (double)part[((int64_t)2 * ntm + t) * ld + i] +
              (double)part[((int64_t)3 * ntm + t) * ld + i];
        if (CPLX)
          ei += (double)part[((int64_t)4 * ntm + t) * ld + i] +
                (double)part[((int64_t)5 * ntm + t) * ld + i];
      }
      if (first)
        for (int t = g; t < ntn128; t += 4) rs += P->rowpart[(int64_t)t * ld + i];
    }
    sh[0][g][c] = r2; sh[1][g][c] = a2; sh[2][g][c] = rs;
    she[0][g][c] = er; she[1][g][c] = ei;
  }
  __syncthreads();
  float rr = 0.f, rsum = 0.f;
  if (g == 0 && i < n) {
    const float r2 = ((sh[0][0][c] + sh[0][1][c]) + sh[0][2][c]) + sh[0][3][c];
    const float a2 = ((sh[1][0][c] + sh[1][1][c]) + sh[1][2][c]) + sh[1][3][c];
    const double er = ((she[0][0][c] + she[0][1][c]) + she[0][2][c]) + she[0][3][c];
    rr = sqrtf(r2 / a2);
    if (!(rr == rr) || isinf(rr)) rr = __int_as_float(0x7f800000);
    if (first) rsum = ((sh[2][0][c] + sh[2][1][c]) + sh[2][2][c]) + sh[2][3][c];
    if (CPLX) {
      const double ei = ((she[1][0][c] + she[1][1][c]) + she[1][2][c]) + she[1][3][c];
      const double dr = P->d[2 * i], di = P->d[2 * i + 1];
      P->E[2 * i] = P->theta[i] + P->lam64 * dr;
      P->E[2 * i + 1] = P->lam64 * di;
      P->dprev_col[2 * i] = (float)dr;
      P->dprev_col[2 * i + 1] = (float)di;
      P->e_col[2 * i] = (float)er;
      P->e_col[2 * i + 1] = (float)ei;
      P->d[2 * i] = dr + er;
      P->d[2 * i + 1] = di + ei;
    } else {
      const double dk = P->d[i];
      P->E[i] = P->theta[i] + P->lam64 * dk;
      P->dprev_col[i] = (float)dk;
      P->e_col[i] = (float)er;
      P->d[i] = dk + er;
    }
  }
  float m = rr, mr = rsum;
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
  }
  __shared__ float wm[2][8];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) { wm[0][threadIdx.x >> 5] = m; wm[1][threadIdx.x >> 5] = mr; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = 0.f, br = 0.f;
    for (int q = 0; q < 8; ++q) { bm = fmaxf(bm, wm[0][q]); br = fmaxf(br, wm[1][q]); }
    atomicMax(&st->rho_bits, __float_as_uint(bm));
    if (first) atomicMax(&st->row_bits, __float_as_uint(br));
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == (unsigned)nchunk - 1u);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  volatile IterState* vs = st;
  if (first) vs->s = vs->theta_max + fabs(vs->lam) * (double)__uint_as_float(vs->row_bits);
  const double rho = (double)__uint_as_float(vs->rho_bits) / vs->s;
  vs->blocks_done = 0;
  vs->rho_bits = 0;
  const float dmax = __uint_as_float(vs->dmax_bits);
  vs->dmax_bits = 0;
  if (!decide(vs, rho)) {
    atomicSub(running, 1);
    return;
  }
  const int S = next_slices_f16(vs, dmax, first, vs->max_slices);
  vs->slices = S;
  vs->slice_gemms = vs->slice_gemms + S;
  // the next product writes dt_k into buffer cur, scaled so that the largest increment
  // of the last step would land at 2^10 (as the single solve's control)
  vs->sexp[vs->cur] = dt_scale_exp((double)dmax, 10, vs->sig, vs->lam);
}

// Output of complex problems (interleaved FP64): thread r owns embedded row r of
// a 128-column tile; the loads of eight columns are issued before their stores.
__global__ void __launch_bounds__(128) k_gc_finalize(const GProb* __restrict__ probs,
                                                     const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (!P->cplx) return;
  const IterState* st = P->st;
  const int n = P->n, ld = P->ld;
  const int k = st->k;
  const bool c1 = st->cur != 0;
  const float* __restrict__ hi = c1 ? P->A_hi[1] : P->A_hi[0];
  const float* __restrict__ lo = c1 ? P->A_lo[1] : P->A_lo[0];
  double* __restrict__ out = P->A_out;
  const int64_t lda2 = 2 * P->ld_a;
  const int r = it.z * 128 + threadIdx.x;       // embedded row
  const int j = r >> 1;
  if (j >= n) return;
  const int i0 = it.y * 128, i1 = min(n, i0 + 128);
  if (k == 0) {
    for (int i = i0; i < i1; ++i) out[(int64_t)i * lda2 + r] = (i == j && (r & 1) == 0) ? 1.0 : 0.0;
  } else {
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
      float h[8], l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = hi[(int64_t)(i + u) * ld + r];
        l[u] = lo[(int64_t)(i + u) * ld + r];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) out[(int64_t)(i + u) * lda2 + r] = f2d_bits(h[u]) + f2d_bits(l[u]);
    }
    for (; i < i1; ++i)
      out[(int64_t)i * lda2 + r] = f2d_bits(hi[(int64_t)i * ld + r]) + f2d_bits(lo[(int64_t)i * ld + r]);
  }
  if (it.y == 0) P->E_out[r] = P->E[r];
}

// ---------------------------------------------------------------------------
// The grouped product kernel (persistent, warp-specialised; one CTA per SM).
// Same structure and arithmetic as k_gemm_epi, with per-tile problem data.
// ---------------------------------------------------------------------------
// Scale factors of a tile's problem for the current product (see dpt_full_mixed.cu's
// EpiConst): the epilogue works on X = (Delta 2^sig)(dt_{k-1} 2^scur) and the stored
// previous increment as they are, with e and d_{k-1} staged as e 2^sig 2^scur and
// d_{k-1} 2^sig and lambda as lambda 2^-sig 2^-scur; the new increment is stored as
// dt_k 2^snew and the diagonal partials (from the slices) are scaled back by 2^-sig.
struct GScale {
  float lams;          // lambda 2^-sig 2^-scur
  float fsig, fcur;    // 2^sig, 2^scur
  float qs, iqs;       // 2^snew, 2^-snew
  float isig;          // 2^-sig
};
__device__ __forceinline__ GScale g_scale(const GProb* P, const IterState* st, int cur) {
  GScale g;
  const int sig = st->sig, scur = st->sexp[cur ^ 1], snew = st->sexp[cur];
  g.lams = (P->lam * exp2i(-sig)) * exp2i(-scur);
  g.fsig = exp2i(sig);
  g.fcur = exp2i(scur);
  g.qs = exp2i(snew);
  g.iqs = exp2i(-snew);
  g.isig = exp2i(-sig);
  return g;
}

struct GTileInfo {
  const GProb* P;
  int tm, tn, m0, n0, bn, S, cur, kbs;
  bool live;
  GScale sc;
};

// with_scale: the epilogue's copy, which needs the problem's scales (the producer and
// the MMA issuer skip their loads)
__device__ __forceinline__ GTileInfo g_tile(const GProb* probs, const int2* tiles, int t,
                                            bool with_scale = false) {
  GTileInfo ti;
  const int2 e = tiles[t];
  ti.P = probs + e.x;
  const IterState* st = ti.P->st;
  ti.live = *((volatile const int*)&st->status) == ST_RUNNING;
  ti.tm = e.y / ti.P->ntn;
  ti.tn = e.y % ti.P->ntn;
  ti.bn = ti.P->bn;
  ti.m0 = ti.tm * G_BM;
  ti.n0 = ti.tn * ti.bn;
  ti.S = st->slices;
  ti.cur = st->cur;
  ti.kbs = ti.P->ld / G_BK;
  if (with_scale) ti.sc = g_scale(ti.P, st, ti.cur);
  return ti;
}

// Column walk of one 32-column chunk (phase 2), warp ew takes 4 columns.
__device__ __forceinline__ void g_epilogue_columns(const GTileInfo& ti, GSmem* ms, const float* Xs,
                                                   int ew, int lane, int c0, float& mx) {
  const GProb* P = ti.P;
  const int n = P->n, ld = P->ld;
  const bool c1 = (ti.cur != 0);
  const float* __restrict__ Ahc = c1 ? P->A_hi[1] : P->A_hi[0];
  const float* __restrict__ Alc = c1 ? P->A_lo[1] : P->A_lo[0];
  float* __restrict__ Ahn = c1 ? P->A_hi[0] : P->A_hi[1];
  float* __restrict__ Aln = c1 ? P->A_lo[0] : P->A_lo[1];
  const __half* __restrict__ dtp = c1 ? P->dt[0] : P->dt[1];
  __half* __restrict__ dtn_out = c1 ? P->dt[1] : P->dt[0];
  float* __restrict__ L = P->L;
  const float lam = ti.sc.lams;     // lambda 2^-sig 2^-scur (see GScale)
  const int r0 = 4 * lane;
  const int j0 = ti.m0 + r0;
  const float4 thj_h = ld4(P->th_hi + j0);
  const float4 thj_l = ld4(P->th_lo + j0);
  const int cb = c0 + 4 * ew;
  if (cb >= ti.bn) return;
  Col4 in[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = ti.n0 + cb + u;
    if (i < n) {
      const int64_t idx = (int64_t)i * ld + j0;
      in[u].ah = ld4(Ahc + idx);
      in[u].al = ld4(Alc + idx);
      in[u].L = ld4(L + idx);
      in[u].dtp = *reinterpret_cast<const uint2*>(dtp + idx);
      // as many slices as this product (the bound of next_slices)
      const __half* Drow = P->Dcat + (int64_t)i * P->cat_ld + j0;
      in[u].D[0] = *reinterpret_cast<const uint2*>(Drow);
      in[u].D[1] = ti.S > 1 ? *reinterpret_cast<const uint2*>(Drow + ld) : make_uint2(0u, 0u);
      in[u].D[2] = ti.S > 2 ? *reinterpret_cast<const uint2*>(Drow + 2 * (int64_t)ld) : make_uint2(0u, 0u);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int cl = cb + u;
    const int i = ti.n0 + cl;
    if (i >= n) continue;
    const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * G_BM + r0);
    const float e_i = ms->e[cl], dp_i = ms->dprev[cl];
    const float thh = ms->thh[cl], thl = ms->thl[cl];
    float4 oh, ol, oL;
    uint32_t ob[4] = {0u, 0u, 0u, 0u};
    float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      const float ah = f4(in[u].ah, e), al = f4(in[u].al, e);
      float nh = 0.f, nl = 0.f, Ln = 0.f, dnew = 0.f;
      if (j == i) {
        nh = 1.f;
        a2 += 1.f;
      } else if (j < n) {
        const float R = f4(in[u].L, e) +
                        lam * (f4(x4, e) - ah * e_i - h_at(in[u].dtp, e) * dp_i);
        float gh, gl;
        ff_sub(thh, thl, f4(thj_h, e), f4(thj_l, e), gh, gl);
        // the remainder keeps R - Gap dt exactly: any reciprocal close to 1/gap serves
        dnew = f16_scaled(R * rcp_approx(gh), ti.sc.qs, ti.sc.iqs, ob[e]);
        Ln = fmaf(-gh, dnew, R) - gl * dnew;
        ff_add_f(ah, al, dnew, nh, nl);
        r2 = fmaf(R, R, r2);
        a2 = fmaf(ah, ah, a2);
        const float p1 = h_at(in[u].D[0], e) * dnew;
        const float p23 = fmaf(h_at(in[u].D[1], e), dnew, h_at(in[u].D[2], e) * dnew);
        float sh, se;
        two_sum(eh, p1, sh, se);
        se += el + p23;
        fast_two_sum(sh, se, eh, el);
        mx = fmaxf(mx, fabsf(dnew));
      }
      f4set(oh, e, nh);
      f4set(ol, e, nl);
      f4set(oL, e, Ln);
    }
    const int64_t idx = (int64_t)i * ld + j0;
    st4(Ahn + idx, oh);
    st4(Aln + idx, ol);
    st4(L + idx, oL);
    *reinterpret_cast<uint2*>(dtn_out + idx) = make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
    warp_sum_ff(r2, a2, eh, el);
    eh *= ti.sc.isig;
    el *= ti.sc.isig;
    if (lane == 0) {
      const int ntm = P->ntm;
      P->part[((int64_t)0 * ntm + ti.tm) * ld + i] = r2;
      P->part[((int64_t)1 * ntm + ti.tm) * ld + i] = a2;
      P->part[((int64_t)2 * ntm + ti.tm) * ld + i] = eh;
      P->part[((int64_t)3 * ntm + ti.tm) * ld + i] = el;
    }
  }
}


// Complex column walk: lane l owns complex rows jc0, jc0+1 (embedded rows r0..r0+3).
__device__ __forceinline__ void gc_epilogue_columns(const GTileInfo& ti, GSmem* ms, const float* Xs,
                                                    int ew, int lane, int c0, float& mx) {
  const GProb* P = ti.P;
  const int n = P->n, ld = P->ld;
  const bool c1 = (ti.cur != 0);
  const float* __restrict__ Ahc = c1 ? P->A_hi[1] : P->A_hi[0];
  const float* __restrict__ Alc = c1 ? P->A_lo[1] : P->A_lo[0];
  float* __restrict__ Ahn = c1 ? P->A_hi[0] : P->A_hi[1];
  float* __restrict__ Aln = c1 ? P->A_lo[0] : P->A_lo[1];
  const __half* __restrict__ dtp = c1 ? P->dt[0] : P->dt[1];
  __half* __restrict__ dtn_out = c1 ? P->dt[1] : P->dt[0];
  float* __restrict__ L = P->L;
  const float lam = ti.sc.lams;     // lambda 2^-sig 2^-scur (see GScale)
  const int r0 = 4 * lane;
  const int jc0 = (ti.m0 + r0) / 2;
  float thj_h[2], thj_l[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = jc0 + e;
    thj_h[e] = j < n ? P->th_hi[j] : 0.f;
    thj_l[e] = j < n ? P->th_lo[j] : 0.f;
  }
  const int cb = c0 + 4 * ew;
  if (cb >= ti.bn) return;
  Col4 in[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = ti.n0 + cb + u;
    if (i < n) {
      const int64_t idx = (int64_t)i * ld + ti.m0 + r0;
      in[u].ah = ld4(Ahc + idx);
      in[u].al = ld4(Alc + idx);
      in[u].L = ld4(L + idx);
      in[u].dtp = *reinterpret_cast<const uint2*>(dtp + idx);
      const __half* Drow = P->Dcat + (int64_t)(2 * i) * P->cat_ld + 2 * jc0;
      in[u].D[0] = *reinterpret_cast<const uint2*>(Drow);
      in[u].D[1] = ti.S > 1 ? *reinterpret_cast<const uint2*>(Drow + ld) : make_uint2(0u, 0u);
      in[u].D[2] = ti.S > 2 ? *reinterpret_cast<const uint2*>(Drow + 2 * (int64_t)ld) : make_uint2(0u, 0u);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int cl = cb + u;
    const int i = ti.n0 + cl;
    if (i >= n) continue;
    const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * G_BM + r0);
    // complex e_i and d_{k-1,i} are stored as (re, im) in the parameter arrays
    const float er = ms->e[2 * cl], ei = ms->e[2 * cl + 1];
    const float dr = ms->dprev[2 * cl], di = ms->dprev[2 * cl + 1];
    const float thh = ms->thh[cl], thl = ms->thl[cl];
    float oh[4], ol[4], oL[4];
    uint32_t ob[4] = {0u, 0u, 0u, 0u};
    float r2 = 0.f, a2 = 0.f, erh = 0.f, erl = 0.f, eih = 0.f, eil = 0.f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = jc0 + e;
      const float ar = f4(in[u].ah, 2 * e), ai = f4(in[u].ah, 2 * e + 1);
      const float alr = f4(in[u].al, 2 * e), ali = f4(in[u].al, 2 * e + 1);
      float nh[2] = {0.f, 0.f}, nl[2] = {0.f, 0.f}, Ln[2] = {0.f, 0.f}, dn[2] = {0.f, 0.f};
      if (j == i) {
        nh[0] = 1.f;
        a2 += 1.f;
      } else if (j < n) {
        float aer, aei, pdr, pdi;
        cmulf(ar, ai, er, ei, aer, aei);
        cmulf(h_at(in[u].dtp, 2 * e), h_at(in[u].dtp, 2 * e + 1), dr, di, pdr, pdi);
        float R[2];
        R[0] = f4(in[u].L, 2 * e) + lam * (f4(x4, 2 * e) - aer - pdr);
        R[1] = f4(in[u].L, 2 * e + 1) + lam * (f4(x4, 2 * e + 1) - aei - pdi);
        float gh, gl;
        ff_sub(thh, thl, thj_h[e], thj_l[e], gh, gl);
        const float g = rcp_approx(gh);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          dn[q] = f16_scaled(R[q] * g, ti.sc.qs, ti.sc.iqs, ob[2 * e + q]);
          Ln[q] = fmaf(-gh, dn[q], R[q]) - gl * dn[q];
          r2 = fmaf(R[q], R[q], r2);
        }
        ff_add_f(ar, alr, dn[0], nh[0], nl[0]);
        ff_add_f(ai, ali, dn[1], nh[1], nl[1]);
        a2 = fmaf(ar, ar, fmaf(ai, ai, a2));
        const float a1 = h_at(in[u].D[0], 2 * e), b1 = h_at(in[u].D[0], 2 * e + 1);
        const float pr1 = fmaf(a1, dn[0], b1 * dn[1]), pi1 = fmaf(a1, dn[1], -b1 * dn[0]);
        const float a2s = h_at(in[u].D[1], 2 * e) + h_at(in[u].D[2], 2 * e);
        const float b2s = h_at(in[u].D[1], 2 * e + 1) + h_at(in[u].D[2], 2 * e + 1);
        const float pr2 = fmaf(a2s, dn[0], b2s * dn[1]), pi2 = fmaf(a2s, dn[1], -b2s * dn[0]);
        float sh, se;
        two_sum(erh, pr1, sh, se); se += erl + pr2; fast_two_sum(sh, se, erh, erl);
        two_sum(eih, pi1, sh, se); se += eil + pi2; fast_two_sum(sh, se, eih, eil);
        mx = fmaxf(mx, fmaxf(fabsf(dn[0]), fabsf(dn[1])));
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        oh[2 * e + q] = nh[q]; ol[2 * e + q] = nl[q]; oL[2 * e + q] = Ln[q];
      }
    }
    const int64_t idx = (int64_t)i * ld + ti.m0 + r0;
    st4(Ahn + idx, make_float4(oh[0], oh[1], oh[2], oh[3]));
    st4(Aln + idx, make_float4(ol[0], ol[1], ol[2], ol[3]));
    st4(L + idx, make_float4(oL[0], oL[1], oL[2], oL[3]));
    *reinterpret_cast<uint2*>(dtn_out + idx) = make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
    warp_sum_ff(r2, a2, erh, erl);
    float z0 = 0.f, z1 = 0.f;
    warp_sum_ff(z0, z1, eih, eil);
    erh *= ti.sc.isig; erl *= ti.sc.isig; eih *= ti.sc.isig; eil *= ti.sc.isig;
    if (lane == 0) {
      const int ntm = P->ntm;
      P->part[((int64_t)0 * ntm + ti.tm) * ld + i] = r2;
      P->part[((int64_t)1 * ntm + ti.tm) * ld + i] = a2;
      P->part[((int64_t)2 * ntm + ti.tm) * ld + i] = erh;
      P->part[((int64_t)3 * ntm + ti.tm) * ld + i] = erl;
      P->part[((int64_t)4 * ntm + ti.tm) * ld + i] = eih;
      P->part[((int64_t)5 * ntm + ti.tm) * ld + i] = eil;
    }
  }
}

__device__ __forceinline__ void g_epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool g_epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 1, 256, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// CPLX: every problem of the launch is complex (the group is of one kind).
template <bool CPLX>
__global__ void __launch_bounds__(G_NTHREADS, 1)
k_g_gemm_epi(const GProb* __restrict__ probs, const int2* __restrict__ tiles, int ntiles,
             unsigned* timeout) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + G_STAGES * G_A_TILE;
  float* Xs = reinterpret_cast<float*>(smem + G_SMEM_TILES);
  GSmem* ms = (GSmem*)(smem + G_SMEM_TILES + G_SMEM_X);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; ++s) { mbar_init(&ms->full[s], 1); mbar_init(&ms->empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&ms->acc_full[b], 1); mbar_init(&ms->acc_empty[b], 1); }
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&ms->tmem_base, 2 * G_BNMAX);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ms->tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    uint32_t it = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
      const GTileInfo ti = g_tile(probs, tiles, t);
      if (!ti.live) continue;
      const CUtensorMap* tA = &ti.P->tmA;
      const CUtensorMap* tB = (ti.cur == 1) ? &ti.P->tmB[0] : &ti.P->tmB[1];
      const uint32_t bytes = G_A_TILE + (uint32_t)ti.bn * G_BK * 2;
      const int nk = ti.S * ti.kbs;
      // a complex problem's column i is dominated by embedded K near 2i
      const int kdiag = CPLX ? 2 * (ti.n0 + ti.bn) - 1 : ti.n0 + ti.bn - 1;
      const int kb_last = min(ti.kbs - 1, kdiag / G_BK);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % G_STAGES;
        const uint32_t ph = (it / G_STAGES) & 1;
        if (!mbar_wait(&ms->empty[s], ph ^ 1, timeout)) { alive = false; break; }
        mbar_arrive_expect_tx(&ms->full[s], bytes);
        // small slices first, the tile's diagonal K-blocks last (see k_gemm_epi)
        const int sl = ti.S - 1 - q / ti.kbs;
        const int kb = (kb_last + 1 + q % ti.kbs) % ti.kbs;
        tma_load_2d(sA + s * G_A_TILE, tA, &ms->full[s], sl * ti.P->ld + kb * G_BK, ti.m0);
        tma_load_2d(sB + s * G_B_TILE, tB, &ms->full[s], kb * G_BK, ti.n0);
      }
    }
    for (uint32_t t = (it > G_STAGES ? it - G_STAGES : 0); t < it; ++t)
      mbar_wait(&ms->full[t % G_STAGES], (t / G_STAGES) & 1, timeout);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    uint32_t it = 0;
    int lt = 0;
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
      const GTileInfo ti = g_tile(probs, tiles, t);
      if (!ti.live) continue;
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      ++lt;
      if (!mbar_wait(&ms->acc_empty[b], (use & 1) ^ 1, timeout)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * G_BNMAX);
      const uint32_t idesc = idesc_f16_f32(G_BM, ti.bn);
      const int nk = ti.S * ti.kbs;
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % G_STAGES;
        const uint32_t ph = (it / G_STAGES) & 1;
        if (!mbar_wait(&ms->full[s], ph, timeout)) { alive = false; break; }
        tc_fence_after();
        const uint64_t da = smem_desc_sw128(sA + s * G_A_TILE);
        const uint64_t db = smem_desc_sw128(sB + s * G_B_TILE);
#pragma unroll
        for (int kk = 0; kk < G_BK / G_UK; ++kk)
          umma_f16(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                    (q > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&ms->empty[s]);
      }
      umma_commit(&ms->acc_full[b]);
    }
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int ew = warp - 2;
    const int qd = warp & 3;
    const int half = ew >> 2;
    const int et = threadIdx.x - 64;
    float mx = 0.f;
    const GProb* mxP = nullptr;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const GTileInfo ti = g_tile(probs, tiles, t, true);
      if (!ti.live) continue;
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      ++lt;
      // the running maximum of |dt| belongs to one problem: flush it on a change
      if (mxP != ti.P) {
        if (mxP) {
          float m = mx;
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0 && m > 0.f) atomicMax(&mxP->st->dmax_bits, __float_as_uint(m));
        }
        mxP = ti.P;
        mx = 0.f;
      }
      g_epi_bar();
      if constexpr (CPLX) {
        // e and d_{k-1} are complex: (re, im) of the tile's columns
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = et + 256 * h;
          const int i = ti.n0 + (q >> 1);
          const bool v = (q < 2 * ti.bn) && (i < ti.P->n);
          ms->e[q] = v ? (ti.P->e_col[2 * ti.n0 + q] * ti.sc.fsig) * ti.sc.fcur : 0.f;
          ms->dprev[q] = v ? ti.P->dprev_col[2 * ti.n0 + q] * ti.sc.fsig : 0.f;
        }
        const int ic = ti.n0 + et;
        const bool vc = (et < ti.bn) && (ic < ti.P->n);
        ms->thh[et] = vc ? ti.P->th_hi[ic] : 0.f;
        ms->thl[et] = vc ? ti.P->th_lo[ic] : 0.f;
      } else {
        const int i = ti.n0 + et;
        const bool v = (et < ti.bn) && (i < ti.P->n);
        ms->e[et] = v ? (ti.P->e_col[i] * ti.sc.fsig) * ti.sc.fcur : 0.f;
        ms->dprev[et] = v ? ti.P->dprev_col[i] * ti.sc.fsig : 0.f;
        ms->thh[et] = v ? ti.P->th_hi[i] : 0.f;
        ms->thl[et] = v ? ti.P->th_lo[i] : 0.f;
      }
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&ms->acc_full[b], use & 1, timeout));
      tc_fence_after();
      const uint32_t src = tmem + (uint32_t)(b * G_BNMAX) + ((uint32_t)(qd * 32) << 16);
      bool all_ok = true;
      for (int c0 = 0; c0 < ti.bn; c0 += G_XCH) {
        if (c0 > 0) g_epi_bar();
        if (ok) {
          float x[16];
          const int cc = half * 16;
          tmem_ld_x16(src + (uint32_t)(c0 + cc), x);
#pragma unroll
          for (int c = 0; c < 16; ++c) Xs[(cc + c) * G_BM + qd * 32 + lane] = x[c];
        }
        if (c0 + G_XCH >= ti.bn) tc_fence_before();
        all_ok = g_epi_bar_and(ok);
        if (c0 + G_XCH >= ti.bn && et == 0) mbar_arrive(&ms->acc_empty[b]);
        if (!all_ok) break;
        if constexpr (CPLX) gc_epilogue_columns(ti, ms, Xs, ew, lane, c0, mx);
        else g_epilogue_columns(ti, ms, Xs, ew, lane, c0, mx);
      }
      if (!all_ok) break;
    }
    if (mxP) {
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(&mxP->st->dmax_bits, __float_as_uint(mx));
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * G_BNMAX);
  }
}

// ===========================================================================
// CTA-pair form of the grouped product (tcgen05 cta_group::2; see k_gemm_epi_pair
// in dpt_full_mixed.cu for the single-problem kernel it follows).  A tile of the
// list is (problem, 256-row x bn pair tile); the two CTAs of a cluster each load
// their 128 rows of the problem's slices and half of its increment columns, the
// leader issues the MMA, and each CTA runs a 16-warp epilogue on its own rows with
// the inputs staged in shared memory by per-lane cp.async one 16-column sub-chunk
// ahead.  The arithmetic per element is that of g_/gc_epilogue_columns, with the
// approximate reciprocal (the increment is rounded to FP16 and the remainder keeps
// R - Gap dt exactly, so any reciprocal close to 1/gap serves).
// ===========================================================================
constexpr int GP_EPI_WARPS = 16;
constexpr int GP_NTHREADS = 64 + 32 * GP_EPI_WARPS;          // 576
constexpr int GP_SLOT = G_A_TILE + 112 * G_BK * 2;           // 30720: A + half of B at bn <= 224
constexpr int GP_STAGES = 4;
constexpr int GP_RING = GP_STAGES * GP_SLOT;                   // 122880 (the planner caps bn at 224)
constexpr int GP_EB_BYTES = GP_EPI_WARPS * 32 * 80;           // 40960: one column per warp
constexpr int GP_SMEM_BYTES = GP_RING + G_SMEM_X + 2 * GP_EB_BYTES + 1024 + (int)sizeof(GSmem);
static_assert(GP_SMEM_BYTES <= 232448, "grouped CTA-pair shared memory over the per-block limit");
static_assert(GP_STAGES <= G_STAGES, "barrier slots");

struct GPairTile {
  const GProb* P;
  int tm2, tn, bn, n0, S, cur, kbs;
  bool live;
  GScale sc;
};

__device__ __forceinline__ GPairTile gp_tile(const GProb* probs, const int2* tiles, int t,
                                             bool with_scale = false) {
  GPairTile ti;
  const int2 e = tiles[t];
  ti.P = probs + e.x;
  const IterState* st = ti.P->st;
  ti.live = *((volatile const int*)&st->status) == ST_RUNNING;
  ti.tm2 = e.y / ti.P->ntn;
  ti.tn = e.y % ti.P->ntn;
  ti.bn = ti.P->bn;
  ti.n0 = ti.tn * ti.bn;
  ti.S = st->slices;
  ti.cur = st->cur;
  ti.kbs = ti.P->ld / G_BK;
  if (with_scale) ti.sc = g_scale(ti.P, st, ti.cur);
  return ti;
}

__device__ __forceinline__ uint8_t* gp_f4(uint8_t* eb, int ew, int f, int lane) {
  return eb + (ew * 3 + f) * 512 + lane * 16;
}
__device__ __forceinline__ uint8_t* gp_u2(uint8_t* eb, int ew, int g, int lane) {
  return eb + GP_EPI_WARPS * 3 * 512 + (ew * 4 + g) * 256 + lane * 8;
}
__device__ __forceinline__ void gp_epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * GP_EPI_WARPS) : "memory");
}
__device__ __forceinline__ bool gp_epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 1, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(32 * GP_EPI_WARPS)
      : "memory");
  return r != 0;
}

// Copies of column n0 + 16 sc + ew (rows m0 + 4 lane .. + 3) of the tile's inputs.
template <bool CPLX>
__device__ __forceinline__ void gp_prefetch(const GPairTile& ti, uint8_t* eb, int ew, int lane,
                                            int m0, int sc) {
  const GProb* P = ti.P;
  const int i = ti.n0 + 16 * sc + ew;
  if (i >= P->n) return;
  const bool c1 = (ti.cur != 0);
  const int64_t idx = (int64_t)i * P->ld + m0 + 4 * lane;
  cp_async16(gp_f4(eb, ew, 0, lane), (c1 ? P->A_hi[1] : P->A_hi[0]) + idx);
  cp_async16(gp_f4(eb, ew, 1, lane), (c1 ? P->A_lo[1] : P->A_lo[0]) + idx);
  cp_async16(gp_f4(eb, ew, 2, lane), P->L + idx);
  cp_async8(gp_u2(eb, ew, 0, lane), (c1 ? P->dt[0] : P->dt[1]) + idx);
  // Delta_ij, j = the lane's rows: row i of the slices (row 2i of the embedding)
  const __half* Drow = P->Dcat + (int64_t)(CPLX ? 2 * i : i) * P->cat_ld + m0 + 4 * lane;
  for (int sl = 0; sl < ti.S; ++sl) cp_async8(gp_u2(eb, ew, 1 + sl, lane), Drow + (int64_t)sl * P->ld);
}

// Real problems: update column n0 + cl (cl = 16 sc + ew) from the staged inputs.
__device__ __forceinline__ void gp_compute_real(const GPairTile& ti, GSmem* ms, const float* Xs,
                                                uint8_t* eb, int ew, int lane, int tm, int m0,
                                                int sc, float& mx) {
  const GProb* P = ti.P;
  const int n = P->n, ld = P->ld;
  const int cl = 16 * sc + ew;
  const int i = ti.n0 + cl;
  if (i >= n) return;
  const bool c1 = (ti.cur != 0);
  float* __restrict__ Ahn = c1 ? P->A_hi[0] : P->A_hi[1];
  float* __restrict__ Aln = c1 ? P->A_lo[0] : P->A_lo[1];
  __half* __restrict__ dtn_out = c1 ? P->dt[1] : P->dt[0];
  const float lam = ti.sc.lams;     // lambda 2^-sig 2^-scur (see GScale)
  const int r0 = 4 * lane, j0 = m0 + r0;
  const float4 thj_h = ld4(P->th_hi + j0);
  const float4 thj_l = ld4(P->th_lo + j0);
  const float4 ah4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 0, lane));
  const float4 al4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 1, lane));
  const float4 L4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 2, lane));
  const uint2 dtp = *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 0, lane));
  uint2 D[3];
  D[0] = *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 1, lane));
  D[1] = ti.S > 1 ? *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 2, lane)) : make_uint2(0u, 0u);
  D[2] = ti.S > 2 ? *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 3, lane)) : make_uint2(0u, 0u);
  const int c0 = 32 * (sc >> 1);
  const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * G_BM + r0);
  const float e_i = ms->e[cl], dp_i = ms->dprev[cl];
  const float thh = ms->thh[cl], thl = ms->thl[cl];
  float4 oh, ol, oL;
  uint32_t ob[4] = {0u, 0u, 0u, 0u};
  float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int j = j0 + e;
    const float ah = f4(ah4, e), al = f4(al4, e);
    float nh = 0.f, nl = 0.f, Ln = 0.f, dnew = 0.f;
    if (j == i) {
      nh = 1.f;
      a2 += 1.f;
    } else if (j < n) {
      const float R = f4(L4, e) + lam * (f4(x4, e) - ah * e_i - h_at(dtp, e) * dp_i);
      float gh, gl;
      ff_sub(thh, thl, f4(thj_h, e), f4(thj_l, e), gh, gl);
      dnew = f16_scaled(R * rcp_approx(gh), ti.sc.qs, ti.sc.iqs, ob[e]);
      Ln = fmaf(-gh, dnew, R) - gl * dnew;
      ff_add_f(ah, al, dnew, nh, nl);
      r2 = fmaf(R, R, r2);
      a2 = fmaf(ah, ah, a2);
      const float p1 = h_at(D[0], e) * dnew;
      const float p23 = fmaf(h_at(D[1], e), dnew, h_at(D[2], e) * dnew);
      float sh, se;
      two_sum(eh, p1, sh, se);
      se += el + p23;
      fast_two_sum(sh, se, eh, el);
      mx = fmaxf(mx, fabsf(dnew));
    }
    f4set(oh, e, nh);
    f4set(ol, e, nl);
    f4set(oL, e, Ln);
  }
  const int64_t idx = (int64_t)i * ld + j0;
  st4(Ahn + idx, oh);
  st4(Aln + idx, ol);
  st4(P->L + idx, oL);
  *reinterpret_cast<uint2*>(dtn_out + idx) = make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
  warp_sum_ff(r2, a2, eh, el);
  eh *= ti.sc.isig;
  el *= ti.sc.isig;
  if (lane == 0) {
    const int ntm = P->ntm;
    P->part[((int64_t)0 * ntm + tm) * ld + i] = r2;
    P->part[((int64_t)1 * ntm + tm) * ld + i] = a2;
    P->part[((int64_t)2 * ntm + tm) * ld + i] = eh;
    P->part[((int64_t)3 * ntm + tm) * ld + i] = el;
  }
}

// Complex problems: lane l owns complex rows jc0, jc0 + 1 (embedded rows r0 .. r0 + 3).
__device__ __forceinline__ void gp_compute_cplx(const GPairTile& ti, GSmem* ms, const float* Xs,
                                                uint8_t* eb, int ew, int lane, int tm, int m0,
                                                int sc, float& mx) {
  const GProb* P = ti.P;
  const int n = P->n, ld = P->ld;
  const int cl = 16 * sc + ew;
  const int i = ti.n0 + cl;
  if (i >= n) return;
  const bool c1 = (ti.cur != 0);
  float* __restrict__ Ahn = c1 ? P->A_hi[0] : P->A_hi[1];
  float* __restrict__ Aln = c1 ? P->A_lo[0] : P->A_lo[1];
  __half* __restrict__ dtn_out = c1 ? P->dt[1] : P->dt[0];
  const float lam = ti.sc.lams;     // lambda 2^-sig 2^-scur (see GScale)
  const int r0 = 4 * lane;
  const int jc0 = (m0 + r0) / 2;
  float thj_h[2], thj_l[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = jc0 + e;
    thj_h[e] = j < n ? P->th_hi[j] : 0.f;
    thj_l[e] = j < n ? P->th_lo[j] : 0.f;
  }
  const float4 ah4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 0, lane));
  const float4 al4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 1, lane));
  const float4 L4 = *reinterpret_cast<const float4*>(gp_f4(eb, ew, 2, lane));
  const uint2 dtp = *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 0, lane));
  uint2 D[3];
  D[0] = *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 1, lane));
  D[1] = ti.S > 1 ? *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 2, lane)) : make_uint2(0u, 0u);
  D[2] = ti.S > 2 ? *reinterpret_cast<const uint2*>(gp_u2(eb, ew, 3, lane)) : make_uint2(0u, 0u);
  const int c0 = 32 * (sc >> 1);
  const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * G_BM + r0);
  const float er = ms->e[2 * cl], ei = ms->e[2 * cl + 1];
  const float dr = ms->dprev[2 * cl], di = ms->dprev[2 * cl + 1];
  const float thh = ms->thh[cl], thl = ms->thl[cl];
  float oh[4], ol[4], oL[4];
  uint32_t ob[4] = {0u, 0u, 0u, 0u};
  float r2 = 0.f, a2 = 0.f, erh = 0.f, erl = 0.f, eih = 0.f, eil = 0.f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int j = jc0 + e;
    const float ar = f4(ah4, 2 * e), ai = f4(ah4, 2 * e + 1);
    const float alr = f4(al4, 2 * e), ali = f4(al4, 2 * e + 1);
    float nh[2] = {0.f, 0.f}, nl[2] = {0.f, 0.f}, Ln[2] = {0.f, 0.f}, dn[2] = {0.f, 0.f};
    if (j == i) {
      nh[0] = 1.f;
      a2 += 1.f;
    } else if (j < n) {
      float aer, aei, pdr, pdi;
      cmulf(ar, ai, er, ei, aer, aei);
      cmulf(h_at(dtp, 2 * e), h_at(dtp, 2 * e + 1), dr, di, pdr, pdi);
      float R[2];
      R[0] = f4(L4, 2 * e) + lam * (f4(x4, 2 * e) - aer - pdr);
      R[1] = f4(L4, 2 * e + 1) + lam * (f4(x4, 2 * e + 1) - aei - pdi);
      float gh, gl;
      ff_sub(thh, thl, thj_h[e], thj_l[e], gh, gl);
      const float g = rcp_approx(gh);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        dn[q] = f16_scaled(R[q] * g, ti.sc.qs, ti.sc.iqs, ob[2 * e + q]);
        Ln[q] = fmaf(-gh, dn[q], R[q]) - gl * dn[q];
        r2 = fmaf(R[q], R[q], r2);
      }
      ff_add_f(ar, alr, dn[0], nh[0], nl[0]);
      ff_add_f(ai, ali, dn[1], nh[1], nl[1]);
      a2 = fmaf(ar, ar, fmaf(ai, ai, a2));
      const float a1 = h_at(D[0], 2 * e), b1 = h_at(D[0], 2 * e + 1);
      const float pr1 = fmaf(a1, dn[0], b1 * dn[1]), pi1 = fmaf(a1, dn[1], -b1 * dn[0]);
      const float a2s = h_at(D[1], 2 * e) + h_at(D[2], 2 * e);
      const float b2s = h_at(D[1], 2 * e + 1) + h_at(D[2], 2 * e + 1);
      const float pr2 = fmaf(a2s, dn[0], b2s * dn[1]), pi2 = fmaf(a2s, dn[1], -b2s * dn[0]);
      float sh, se;
      two_sum(erh, pr1, sh, se); se += erl + pr2; fast_two_sum(sh, se, erh, erl);
      two_sum(eih, pi1, sh, se); se += eil + pi2; fast_two_sum(sh, se, eih, eil);
      mx = fmaxf(mx, fmaxf(fabsf(dn[0]), fabsf(dn[1])));
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      oh[2 * e + q] = nh[q]; ol[2 * e + q] = nl[q]; oL[2 * e + q] = Ln[q];
    }
  }
  const int64_t idx = (int64_t)i * ld + m0 + r0;
  st4(Ahn + idx, make_float4(oh[0], oh[1], oh[2], oh[3]));
  st4(Aln + idx, make_float4(ol[0], ol[1], ol[2], ol[3]));
  st4(P->L + idx, make_float4(oL[0], oL[1], oL[2], oL[3]));
  *reinterpret_cast<uint2*>(dtn_out + idx) = make_uint2(ob[0] | (ob[1] << 16), ob[2] | (ob[3] << 16));
  warp_sum_ff(r2, a2, erh, erl);
  float z0 = 0.f, z1 = 0.f;
  warp_sum_ff(z0, z1, eih, eil);
  erh *= ti.sc.isig; erl *= ti.sc.isig; eih *= ti.sc.isig; eil *= ti.sc.isig;
  if (lane == 0) {
    const int ntm = P->ntm;
    P->part[((int64_t)0 * ntm + tm) * ld + i] = r2;
    P->part[((int64_t)1 * ntm + tm) * ld + i] = a2;
    P->part[((int64_t)2 * ntm + tm) * ld + i] = erh;
    P->part[((int64_t)3 * ntm + tm) * ld + i] = erl;
    P->part[((int64_t)4 * ntm + tm) * ld + i] = eih;
    P->part[((int64_t)5 * ntm + tm) * ld + i] = eil;
  }
}

// PAIR = false: the same kernel without clusters: one CTA per 128-row tile of width
// <= 128, a 3-stage ring of A + B slots, its own MMA (cta_group::1) and the same
// 16-warp staged epilogue; for groups of small problems, whose 128-row tiles would
// leave the second CTA of a pair idle.
template <bool PAIR>
struct GPShape {
  static constexpr int slot = PAIR ? GP_SLOT : G_A_TILE + 128 * G_BK * 2;   // 30720 / 32768
  static constexpr int stages = PAIR ? GP_STAGES : 3;
  static constexpr int rows = PAIR ? 2 * G_BM : G_BM;                         // rows per tile
};
static_assert(GPShape<false>::slot * GPShape<false>::stages <= GP_RING, "single-CTA ring");

template <bool CPLX, bool PAIR>
__global__ void __launch_bounds__(GP_NTHREADS, 1)
k_g_gemm_epi_x(const GProb* __restrict__ probs, const int2* __restrict__ tiles, int ntiles,
               unsigned* timeout) {
  using Sh = GPShape<PAIR>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* Xs = reinterpret_cast<float*>(smem + GP_RING);
  uint8_t* EB = smem + GP_RING + G_SMEM_X;
  GSmem* ms = (GSmem*)(smem + GP_RING + G_SMEM_X + 2 * GP_EB_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const int pair = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int npairs = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Sh::stages; ++s) { mbar_init(&ms->full[s], 1); mbar_init(&ms->empty[s], 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ms->acc_full[b], 1);
      mbar_init(&ms->acc_empty[b], PAIR ? 2 : 1);
    }
    fence_mbar_init();
  }
  if (warp == 0) {
    if constexpr (PAIR) { tmem_alloc_pair(&ms->tmem_base, 2 * G_BNMAX); tmem_relinquish_pair(); }
    else { tmem_alloc(&ms->tmem_base, 2 * G_BNMAX); tmem_relinquish(); }
  }
  tc_fence_before();
  if constexpr (PAIR) cluster_sync();
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ms->tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (both CTAs): completions go to the leader's full[s] ----
    const uint32_t full_leader = PAIR ? mapa_shared(&ms->full[0], 0) : 0u;
    uint32_t it = 0;
    bool alive = true;
    for (int t = pair; t < ntiles && alive; t += npairs) {
      const GPairTile ti = gp_tile(probs, tiles, t);
      if (!ti.live) continue;
      // the slot holds A and this CTA's rows of B: bn/2 <= 112 (pair) or bn <= 128
      const int bh = PAIR ? ti.bn / 2 : ti.bn;
      const uint32_t stage_bytes = (uint32_t)G_A_TILE + (uint32_t)bh * G_BK * 2;
      const CUtensorMap* tA = &ti.P->tmA;
      const CUtensorMap* tB = (ti.cur == 1) ? &ti.P->tmB[0] : &ti.P->tmB[1];
      const int nk = ti.S * ti.kbs;
      const int m0 = ti.tm2 * Sh::rows + (int)rank * G_BM;
      const int kdiag = CPLX ? 2 * (ti.n0 + ti.bn) - 1 : ti.n0 + ti.bn - 1;
      const int kb_last = min(ti.kbs - 1, kdiag / G_BK);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % Sh::stages;
        const uint32_t ph = (it / Sh::stages) & 1;
        if (!mbar_wait(&ms->empty[s], ph ^ 1, timeout)) { alive = false; break; }
        const int sl = ti.S - 1 - q / ti.kbs;
        const int kb = (kb_last + 1 + q % ti.kbs) % ti.kbs;
        uint8_t* slot = smem + (size_t)s * Sh::slot;
        if constexpr (PAIR) {
          if (rank == 0) mbar_arrive_expect_tx(&ms->full[s], 2 * stage_bytes);
          const uint32_t fb = full_leader + (uint32_t)s * 8u;
          tma_load_2d_pair(slot, tA, fb, sl * ti.P->ld + kb * G_BK, m0);
          tma_load_2d_pair(slot + G_A_TILE, tB, fb, kb * G_BK, ti.n0 + (int)rank * bh);
        } else {
          mbar_arrive_expect_tx(&ms->full[s], stage_bytes);
          tma_load_2d(slot, tA, &ms->full[s], sl * ti.P->ld + kb * G_BK, m0);
          tma_load_2d(slot + G_A_TILE, tB, &ms->full[s], kb * G_BK, ti.n0);
        }
      }
    }
    if constexpr (PAIR) {
      for (uint32_t u = (it > (uint32_t)Sh::stages ? it - Sh::stages : 0); u < it; ++u)
        mbar_wait_quiet(&ms->empty[u % Sh::stages], (u / Sh::stages) & 1, kTailWaitNs);
    } else {
      // every issued copy has landed before the CTA can exit
      for (uint32_t u = (it > (uint32_t)Sh::stages ? it - Sh::stages : 0); u < it; ++u)
        mbar_wait_quiet(&ms->full[u % Sh::stages], (u / Sh::stages) & 1, kTailWaitNs);
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---- MMA issuer (the pair's leader, or the CTA itself) ----
    uint32_t it = 0;
    int lt = 0;
    bool alive = true;
    for (int t = pair; t < ntiles && alive; t += npairs) {
      const GPairTile ti = gp_tile(probs, tiles, t);
      if (!ti.live) continue;
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      ++lt;
      if (!mbar_wait(&ms->acc_empty[b], (use & 1) ^ 1, timeout)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * G_BNMAX);
      const uint32_t idesc = idesc_f16_f32(Sh::rows, ti.bn);
      const int nk = ti.S * ti.kbs;
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % Sh::stages;
        const uint32_t ph = (it / Sh::stages) & 1;
        if (!mbar_wait(&ms->full[s], ph, timeout)) { alive = false; break; }
        tc_fence_after();
        uint8_t* slot = smem + (size_t)s * Sh::slot;
        const uint64_t da = smem_desc_sw128(slot);
        const uint64_t db = smem_desc_sw128(slot + G_A_TILE);
#pragma unroll
        for (int kk = 0; kk < G_BK / G_UK; ++kk) {
          if constexpr (PAIR)
            umma_f16_pair(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                           (q > 0 || kk > 0) ? 1u : 0u);
          else
            umma_f16(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                      (q > 0 || kk > 0) ? 1u : 0u);
        }
        if constexpr (PAIR) umma_commit_pair(&ms->empty[s], (uint16_t)3);
        else umma_commit(&ms->empty[s]);
      }
      if constexpr (PAIR) umma_commit_pair(&ms->acc_full[b], (uint16_t)3);
      else umma_commit(&ms->acc_full[b]);
    }
    if constexpr (PAIR)
      for (int u = (lt > 2 ? lt - 2 : 0); u < lt; ++u)
        mbar_wait_quiet(&ms->acc_empty[u & 1], (uint32_t)((u >> 1) & 1), kTailWaitNs);
  } else if (warp >= 2) {
    // ---- epilogue (both CTAs, each on its own 128 rows) ----
    const int ew = warp - 2;
    const int qd = warp & 3;
    const int q4 = ew >> 2;
    const int et = threadIdx.x - 64;
    const uint32_t acc_empty_leader = PAIR ? mapa_shared(&ms->acc_empty[0], 0) : 0u;
    float mx = 0.f;
    const GProb* mxP = nullptr;
    int lt = 0;
    int pref_t = -1;      // tile whose first sub-chunk is in flight
    for (int t = pair; t < ntiles; t += npairs) {
      const GPairTile ti = gp_tile(probs, tiles, t, true);
      if (!ti.live) continue;
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      ++lt;
      // 128-row tile of this CTA: the pair's half, or the tile itself
      const int tm = PAIR ? 2 * ti.tm2 + (int)rank : ti.tm2;
      const int m0 = tm * G_BM;
      const bool work = tm < ti.P->ntm;
      if (mxP != ti.P) {
        if (mxP) {
          float m = mx;
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0 && m > 0.f) atomicMax(&mxP->st->dmax_bits, __float_as_uint(m));
        }
        mxP = ti.P;
        mx = 0.f;
      }
      if (pref_t != t) {
        if (work) gp_prefetch<CPLX>(ti, EB, ew, lane, m0, 0);
        cp_async_commit();
        cp_async_wait<0>();
      }
      gp_epi_bar();
      if constexpr (CPLX) {
        const int i = ti.n0 + (et >> 1);
        const bool v = (et < 2 * ti.bn) && (i < ti.P->n);
        ms->e[et] = v ? (ti.P->e_col[2 * ti.n0 + et] * ti.sc.fsig) * ti.sc.fcur : 0.f;
        ms->dprev[et] = v ? ti.P->dprev_col[2 * ti.n0 + et] * ti.sc.fsig : 0.f;
        if (et < G_BNMAX) {
          const int ic = ti.n0 + et;
          const bool vc = (et < ti.bn) && (ic < ti.P->n);
          ms->thh[et] = vc ? ti.P->th_hi[ic] : 0.f;
          ms->thl[et] = vc ? ti.P->th_lo[ic] : 0.f;
        }
      } else {
        if (et < G_BNMAX) {
          const int i = ti.n0 + et;
          const bool v = (et < ti.bn) && (i < ti.P->n);
          ms->e[et] = v ? (ti.P->e_col[i] * ti.sc.fsig) * ti.sc.fcur : 0.f;
          ms->dprev[et] = v ? ti.P->dprev_col[i] * ti.sc.fsig : 0.f;
          ms->thh[et] = v ? ti.P->th_hi[i] : 0.f;
          ms->thl[et] = v ? ti.P->th_lo[i] : 0.f;
        }
      }
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&ms->acc_full[b], use & 1, timeout));
      tc_fence_after();
      const uint32_t src = tmem + (uint32_t)(b * G_BNMAX) + ((uint32_t)(qd * 32) << 16);
      const int nsub = ti.bn / 16;
      // the next live tile of this pair, for the prefetch at the last sub-chunk
      int tnext = t + npairs;
      bool next_live = false;
      GPairTile nx{};
      if (tnext < ntiles) {
        nx = gp_tile(probs, tiles, tnext);
        next_live = nx.live;
      }
      bool all_ok = true;
#pragma unroll 1
      for (int c0 = 0; c0 < ti.bn; c0 += G_XCH) {
        if (c0 > 0) gp_epi_bar();
        if (ok) {
          float x[8];
          const int cc = q4 * 8;
          tmem_ld_x8(src + (uint32_t)(c0 + cc), x);
#pragma unroll
          for (int c = 0; c < 8; ++c) Xs[(cc + c) * G_BM + qd * 32 + lane] = x[c];
        }
        if (c0 + G_XCH >= ti.bn) tc_fence_before();
        all_ok = gp_epi_bar_and(ok);
        if (c0 + G_XCH >= ti.bn && et == 0) {
          if (rank == 0) mbar_arrive(&ms->acc_empty[b]);
          else if constexpr (PAIR) mbar_arrive_remote(acc_empty_leader + (uint32_t)b * 8u);
        }
        if (!all_ok) break;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int sc = c0 / 16 + h;
          uint8_t* nb = EB + ((sc + 1) & 1) * GP_EB_BYTES;
          pref_t = -1;
          if (sc + 1 < nsub) {
            if (work) gp_prefetch<CPLX>(ti, nb, ew, lane, m0, sc + 1);
          } else if (next_live) {
            const int tmn = PAIR ? 2 * nx.tm2 + (int)rank : nx.tm2;
            if (tmn < nx.P->ntm) gp_prefetch<CPLX>(nx, nb, ew, lane, tmn * G_BM, 0);
            pref_t = tnext;
          }
          cp_async_commit();
          cp_async_wait<1>();
          if (work) {
            uint8_t* cb = EB + (sc & 1) * GP_EB_BYTES;
            if constexpr (CPLX) gp_compute_cplx(ti, ms, Xs, cb, ew, lane, tm, m0, sc, mx);
            else gp_compute_real(ti, ms, Xs, cb, ew, lane, tm, m0, sc, mx);
          }
        }
      }
      if (!all_ok) break;
    }
    cp_async_wait<0>();
    if (mxP) {
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(&mxP->st->dmax_bits, __float_as_uint(mx));
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();
  if (warp == 0) {
    tc_fence_after();
    if constexpr (PAIR) tmem_dealloc_pair(tmem, 2 * G_BNMAX);
    else tmem_dealloc(tmem, 2 * G_BNMAX);
  }
}


// ---------------------------------------------------------------------------
// Output: A (float-float -> FP64) and E; work item (problem, 128-col tile, 128-row
// tile), thread j owns row j; the loads of eight columns are issued before their
// stores.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_g_finalize(const GProb* __restrict__ probs,
                                                    const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const GProb* P = probs + it.x;
  if (P->cplx) return;
  const IterState* st = P->st;
  const int n = P->n, ld = P->ld;
  const int k = st->k;
  const bool c1 = st->cur != 0;
  const float* __restrict__ hi = c1 ? P->A_hi[1] : P->A_hi[0];
  const float* __restrict__ lo = c1 ? P->A_lo[1] : P->A_lo[0];
  double* __restrict__ out = P->A_out;
  const int64_t lda = P->ld_a;
  const int j = it.z * 128 + threadIdx.x;
  if (j >= n) return;
  const int i0 = it.y * 128, i1 = min(n, i0 + 128);
  if (k == 0) {
    for (int i = i0; i < i1; ++i) out[(int64_t)i * lda + j] = (i == j) ? 1.0 : 0.0;
  } else {
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
      float h[8], l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = hi[(int64_t)(i + u) * ld + j];
        l[u] = lo[(int64_t)(i + u) * ld + j];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) out[(int64_t)(i + u) * lda + j] = f2d_bits(h[u]) + f2d_bits(l[u]);
    }
    for (; i < i1; ++i)
      out[(int64_t)i * lda + j] = f2d_bits(hi[(int64_t)i * ld + j]) + f2d_bits(lo[(int64_t)i * ld + j]);
  }
  if (it.y == 0) P->E_out[j] = P->E[j];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t g_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_g_gemm_epi<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_g_gemm_epi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_g_gemm_epi_x<false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_g_gemm_epi_x<true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_g_gemm_epi_x<false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_g_gemm_epi_x<true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, GP_SMEM_BYTES);
  return e;
}

namespace {
// launch configuration of the staged kernel: clusters of two for the pair form
struct StagedLaunch {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  StagedLaunch(int blocks, bool pair, cudaStream_t s) {
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(GP_NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = GP_SMEM_BYTES;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pair ? 2 : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pair ? 1 : 0;
  }
};
}  // namespace

// Clusters of two of the grouped pair kernel that can be resident at once.
int g_pair_clusters() {
  static int cached[64];
  static bool known[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  if (known[dev]) return cached[dev];
  StagedLaunch L(2, true, nullptr);
  int n = 0;
  if (cudaFuncSetAttribute(k_g_gemm_epi_x<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           GP_SMEM_BYTES) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, k_g_gemm_epi_x<false, true>, &L.cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached[dev] = n;
  known[dev] = true;
  return n;
}

cudaError_t launch_g_gemm_epi_pair(const GProb* probs, const int2* tiles, int ntiles,
                                   unsigned* timeout, bool cplx, int npairs, cudaStream_t s) {
  if (npairs < 1) return cudaErrorInvalidValue;
  const int pairs = ntiles < npairs ? ntiles : npairs;
  if (pairs <= 0) return cudaGetLastError();
  StagedLaunch L(2 * pairs, true, s);
  return cplx ? cudaLaunchKernelEx(&L.cfg, k_g_gemm_epi_x<true, true>, probs, tiles, ntiles, timeout)
              : cudaLaunchKernelEx(&L.cfg, k_g_gemm_epi_x<false, true>, probs, tiles, ntiles, timeout);
}

cudaError_t launch_g_gemm_epi_staged(const GProb* probs, const int2* tiles, int ntiles,
                                     unsigned* timeout, bool cplx, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  if (grid <= 0) return cudaGetLastError();
  StagedLaunch L(grid, false, s);
  return cplx ? cudaLaunchKernelEx(&L.cfg, k_g_gemm_epi_x<true, false>, probs, tiles, ntiles, timeout)
              : cudaLaunchKernelEx(&L.cfg, k_g_gemm_epi_x<false, false>, probs, tiles, ntiles, timeout);
}
cudaError_t launch_g_check_theta(const GProb* probs, int count, int max_n, int* running,
                                 cudaStream_t s) {
  if (count > 0 && max_n > 0)
    k_g_check_theta<<<dim3(count, (max_n + 127) / 128), 128, 0, s>>>(probs, count, running);
  return cudaGetLastError();
}
cudaError_t launch_g_scales(const GProb* probs, const int4* items, int nitems, bool cplx,
                            cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (cplx) k_g_scales<true><<<nitems, 128, 0, s>>>(probs, items);
  else k_g_scales<false><<<nitems, 128, 0, s>>>(probs, items);
  return cudaGetLastError();
}

cudaError_t launch_g_prep(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_g_prep<<<nitems, dim3(32, 8), 0, s>>>(probs, items);
  return cudaGetLastError();
}
cudaError_t launch_g_iter0(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_g_iter0<<<nitems, 128, 0, s>>>(probs, items);
  return cudaGetLastError();
}
cudaError_t launch_g_ctrl(const GProb* probs, int count, int max_n, bool cplx, int* running,
                          cudaStream_t s) {
  if (count <= 0 || max_n <= 0) return cudaGetLastError();
  const dim3 grid(count, (max_n + 63) / 64);
  if (cplx) k_g_ctrl<true><<<grid, 256, 0, s>>>(probs, count, running);
  else k_g_ctrl<false><<<grid, 256, 0, s>>>(probs, count, running);
  return cudaGetLastError();
}
cudaError_t launch_g_gemm_epi(const GProb* probs, const int2* tiles, int ntiles, unsigned* timeout,
                              bool cplx, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  if (grid > 0) {
    if (cplx) k_g_gemm_epi<true><<<grid, G_NTHREADS, G_SMEM_BYTES, s>>>(probs, tiles, ntiles, timeout);
    else k_g_gemm_epi<false><<<grid, G_NTHREADS, G_SMEM_BYTES, s>>>(probs, tiles, ntiles, timeout);
  }
  return cudaGetLastError();
}
cudaError_t launch_gc_prep(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_gc_prep<<<nitems, dim3(32, 8), 0, s>>>(probs, items);
  return cudaGetLastError();
}
cudaError_t launch_gc_iter0(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_gc_iter0<<<nitems, 128, 0, s>>>(probs, items);
  return cudaGetLastError();
}
cudaError_t launch_gc_finalize(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_gc_finalize<<<nitems, 128, 0, s>>>(probs, items);
  return cudaGetLastError();
}
cudaError_t launch_g_finalize(const GProb* probs, const int4* items, int nitems, cudaStream_t s) {
  if (nitems) k_g_finalize<<<nitems, 128, 0, s>>>(probs, items);
  return cudaGetLastError();
}

}  // namespace dpt
