// Full-spectrum DPT on the tensor cores (mixed precision), real case.
//
// The map of Eq. (dyn) (arXiv:2002.12872, Sec. II.B), in column form,
//     A_{k+1} = A_k + G o R_k,
//     R_k     = lambda (Delta A_k - A_k diag(d_k)) - Gap o A_k,   d_k = diag(Delta A_k),
// with Gap_ji = theta_i - theta_j and G = 1/Gap off the diagonal, is carried here
// in increment form so that every product acts on a small quantity:
//     X_k   = Delta dt_{k-1}                         (tensor-core GEMM, FP16 in, FP32 acc)
//     e_k   = diag(Delta dt_{k-1}),   d_k = d_{k-1} + e_k
//     R_k   = L_k + lambda (X_k - A_k diag(e_k) - dt_{k-1} diag(d_{k-1}))
//     dt_k  = f16(G o R_k)                           (the increment actually applied)
//     L_{k+1} = R_k - Gap o dt_k                     (carried remainder: exact feedback)
//     A_{k+1} = A_k + dt_k                           (float-float accumulation)
// Substituting A_k = A_{k-1} + dt_{k-1} into R_k shows this is the same recursion
// as the map; the remainder L makes the FP16 rounding of each increment re-enter
// the next step instead of being lost, so the fixed point is the FP64 one: any
// rounding (or clamping) of dt_k is made good by the following steps.
// Delta enters the product as FP16 slices (Delta 2^sig ~ D1 + D2, 11 significant
// bits each; a third on request), concatenated along K, so one GEMM of depth S*n
// gives the sliced product.  The increments dt are FP16 as well, each buffer with
// its own power-of-two scale: FP16 has three more significand bits than BF16 but a
// narrow exponent range, and the scales (exact in both directions) give it the
// range of the data.  Two FP16 slices carry 22 bits where three BF16 slices carried
// 24, so the first products need a third fewer tensor-core passes.
// R_k is, to rounding, the eigen-residual M a_i - E_i a_i of the iterate A_k
// (the residual identity: R = Gap o (F(A) - A)); its column norms give the
// convergence test without a second product.

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <type_traits>

#include "dpt_device.cuh"
#include "dpt_internal.h"

namespace dpt {

constexpr int BM = 128;          // rows j per tile (TMEM lanes)
constexpr int BN = 256;          // widest tile: columns i per tile (TMEM columns per accumulator);
                                 // the launch's width p.bn is a multiple of 32 up to BN
constexpr int BK = 64;           // K per stage: one 128-byte swizzle atom of 16-bit elements
constexpr int UK = 16;           // K per tcgen05.mma (kind::f16)
constexpr int STAGES = 4;        // operand ring depth (bytes in flight cover the L2 latency)
constexpr int MAX_STAGES = 8;    // barrier slots; the CTA-pair kernel fits more, smaller stages
constexpr int NACC = 2;          // TMEM accumulators (double buffer)
constexpr int IT0 = 128;         // rows per block of iteration 0 (its columns: kIter0Cols)
constexpr int NSLICE = 3;        // FP16 slices of Delta the layout holds (the solve writes
                                 // max_slices of them, the product uses the first S)
constexpr int A_TILE = BM * BK * 2;
constexpr int B_TILE = BN * BK * 2;
constexpr int EPI_WARPS = 8;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;   // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int SMEM_TILES = STAGES * (A_TILE + B_TILE);
constexpr int XCH = 32;                         // accumulator columns staged per chunk
constexpr int SMEM_X = BM * XCH * 4;            // accumulator staging (FP32, column-major)

struct __align__(16) GemmSmemMisc {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t acc_full[NACC];
  uint64_t acc_empty[NACC];
  uint32_t tmem_base;
  int k;
  int slices;
  int cur;
  int certify;        // this product only assesses its iterate (IterState::certify)
  int sig;            // the slices hold Delta 2^sig
  int scur;           // dt_{k-1} (the B operand) is stored as dt_{k-1} 2^scur
  int snew;           // dt_k is stored as dt_k 2^snew
  float rpow;         // non-autonomous iteration: this step applies lambda (1 - rpow); 0 off
  float rq, oq;       // the pair kernel's (1 - rpow) 2^snew and rpow 2^snew (see EpiConst)
  float e[BN];        // e_k 2^sig 2^scur for the tile's columns
  float dprev[BN];    // d_{k-1} 2^sig
  float thh[BN];      // theta_i as float-float
  float thl[BN];
};
constexpr int SMEM_BYTES = SMEM_TILES + SMEM_X + 1024 + (int)sizeof(GemmSmemMisc);

// CTA-pair layout: an operand ring, the accumulator staging, and buffers of epilogue
// inputs filled by per-thread asynchronous copies.  The pair kernel's epilogue has 16
// warps (its inputs sit in shared memory, not in registers, so 576 threads fit the
// register file); each warp updates one column of every 16-column sub-chunk.
// With one slice a stage holds A and half of B (30 KB at bn = 224, four stages) and
// the epilogue double-buffers its inputs, copying one sub-chunk ahead: the second
// buffer occupies the end of the ring region.  With two slices (after the first
// product: see k_gemm_epi_pair) a stage holds both slices' A tiles and one B half
// (46 KB at bn = 224, three stages): the increment
// tile is fetched once for both slices, which cuts the operand bytes an SM receives
// per flop by a quarter (the products are bound by that inflow, about 42 B per cycle
// and SM on GB300), and the epilogue, which has time to spare in these launches,
// works from one buffer.
constexpr int P_EPI_WARPS = 16;
constexpr int P_NTHREADS = 64 + 32 * P_EPI_WARPS;       // 576
constexpr int EB_COL = 72;                              // bytes per lane and column
constexpr int EB_BYTES = P_EPI_WARPS * 32 * EB_COL;     // one column per warp: 36864 B
constexpr int P_RREG = 4 * (A_TILE + 112 * BK * 2) + EB_BYTES;   // 159744 B
constexpr int P_SMEM_BYTES = P_RREG + EB_BYTES + SMEM_X + 1024 + (int)sizeof(GemmSmemMisc);
static_assert(P_SMEM_BYTES <= 232448, "CTA-pair shared memory over the per-block limit");

// ---------------------------------------------------------------------------
// Scales of the FP16 operands: the block maxima of the scale pass (256 threads) reach
// the state by integer atomicMax; the grid's last block sets sig (max |Delta| 2^sig in
// [2^14, 2^15)) and the exponent of the first increment (its bound lands at 2^13).
// hmax: high word of max |Delta| (sign cleared); gmax: the first increment's bound
// before the factor |lambda| (with a start: its largest entry); rgmax: max 1 / |gap|.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scales_finish(unsigned hmax, float gmax, float rgmax,
                                              bool start, IterState* st) {
  hmax = __reduce_max_sync(0xffffffffu, hmax);
  unsigned gb = __reduce_max_sync(0xffffffffu, __float_as_uint(gmax));   // gmax >= 0
  unsigned rb = __reduce_max_sync(0xffffffffu, __float_as_uint(rgmax));  // rgmax >= 0
  __shared__ unsigned wh[8], wg[8], wr[8];
  __shared__ bool last;
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { wh[w] = hmax; wg[w] = gb; wr[w] = rb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned a = 0u, b = 0u, r = 0u;
    for (int q = 0; q < 8; ++q) { a = max(a, wh[q]); b = max(b, wg[q]); r = max(r, wr[q]); }
    atomicMax(&st->amax_bits, a);
    atomicMax(&st->g0max_bits, b);
    atomicMax(&st->rgmax_bits, r);
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  volatile IterState* vs = st;
  const unsigned hm = vs->amax_bits;
  int sig = 0;
  if (hm != 0u) sig = 14 - ((int)((hm >> 20) & 0x7FFu) - 1023);   // max |Delta| < 2^(e+1)
  sig = max(-120, min(120, sig));
  const double lam = vs->lam;
  // the bound of the first increment: |lambda| max |Delta_ji / gap|, or with a start
  // the largest entry of its offset from I
  const double g0 = (double)__uint_as_float(vs->g0max_bits);
  const double ref = start ? g0 : fabs(lam) * g0;
  const int s0 = dt_scale_exp(ref, 13, sig, lam);
  vs->sig = sig;
  vs->sexp[0] = s0;
  vs->sexp[1] = s0;
  vs->blocks_done = 0;
}

// |v| to 20 fraction bits as a float from the high word of a double (sign cleared):
// 0 below the float range, +inf beyond it (inputs beyond it are rejected by the
// slicing)
__device__ __forceinline__ float abs_from_hiword(unsigned hw) {
  const unsigned e = hw >> 20;
  return (e > 896u && e < 1151u) ? __uint_as_float(((e - 896u) << 23) | ((hw & 0xFFFFFu) << 3))
                                 : (e >= 1151u ? __int_as_float(0x7f800000) : 0.f);
}
// The same in two integer operations: the high word clamped to [2^-127, 2^128] (the
// clamp drops the fraction at the top, giving +inf) and rebiased from 1023 to 127 in
// the wrapping 32-bit product (896 = 512 + 384; 384 << 23 = 0xC0000000).  It differs
// from abs_from_hiword only in [2^-127, 2^-126), which it keeps as subnormals.
__device__ __forceinline__ float abs_from_hiword_clamped(unsigned hw) {
  const unsigned c = min(max(hw, 896u << 20), 1151u << 20);
  return __uint_as_float(c * 8u + 0x40000000u);
}

// The scale pass without a start.  Thread per row j (theta_j in registers); a work
// item is 256 rows x 8 columns, eight loads in flight per thread (a warp reads 256
// contiguous bytes of each column), and the items are strided over a grid of a few
// blocks per SM, so that the block's reduction (scales_finish) runs once per block.
// Column i's theta is a block-uniform 16-byte load.  The quantities are those of
// k_delta_scales below: the high word of max |Delta_ji| (the diagonal only without
// Epstein-Nesbet), and over j != i the ratio |Delta_ji| / |theta_i - theta_j|
// (|Delta_ji| from its high word, the gap from the float parts of theta, their low
// parts where the high parts coincide) and 1 / |gap|.  (Two rows per thread with
// 16-byte loads measured no faster: about 4.5 TB/s of reads either way.)
constexpr int kScaleCols = 8;   // a multiple of 4 (16-byte theta loads)
__device__ __forceinline__ void scale_entry(unsigned hw, float tih, float til, float tjh,
                                            float tjl, unsigned& hmax, float& gmax,
                                            float& rgmax) {
  hmax = max(hmax, hw);
  float g = tih - tjh;
  if (g == 0.f) g = til - tjl;
  // NaN never wins fmaxf
  const float rg = rcp_approx(fabsf(g));
  gmax = fmaxf(gmax, abs_from_hiword_clamped(hw) * rg);
  rgmax = fmaxf(rgmax, rg);
}
__global__ void __launch_bounds__(256) k_delta_scales_rows(const double* __restrict__ delta,
                                                           int64_t ld_in, int n, int nrb,
                                                           int nitems,
                                                           const float* __restrict__ th_hi,
                                                           const float* __restrict__ th_lo,
                                                           int en, IterState* st) {
  unsigned hmax = 0u;
  float gmax = 0.f, rgmax = 0.f;
  // a full item away from the diagonal takes the fast path; its loads are issued one
  // item ahead, so that they are in flight while the previous item is processed
  auto full_item = [&](int it) {
    const int j = (it % nrb) * 256 + threadIdx.x, i0 = (it / nrb) * kScaleCols;
    return j < n && i0 + kScaleCols <= n && (unsigned)(j - i0) >= (unsigned)kScaleCols;
  };
  double v[kScaleCols];
  auto fetch = [&](int it) {
    if (it < nitems && full_item(it)) {
      const int j = (it % nrb) * 256 + threadIdx.x, i0 = (it / nrb) * kScaleCols;
      const double* p = delta + (int64_t)i0 * ld_in + j;
#pragma unroll
      for (int u = 0; u < kScaleCols; ++u) v[u] = p[(int64_t)u * ld_in];
    }
  };
  fetch(blockIdx.x);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int rb = it % nrb, cb = it / nrb;
    const int j = rb * 256 + threadIdx.x, i0 = cb * kScaleCols;
    if (j >= n) {   // a ragged row block (a later item may hold rows of this thread)
      fetch(it + gridDim.x);
      continue;
    }
    const float tjh = th_hi[j], tjl = th_lo[j];
    if (full_item(it)) {
      unsigned hw[kScaleCols];
#pragma unroll
      for (int u = 0; u < kScaleCols; ++u)
        hw[u] = (unsigned)__double2hiint(v[u]) & 0x7FFFFFFFu;
      fetch(it + gridDim.x);
      float tih[kScaleCols], til[kScaleCols];
#pragma unroll
      for (int u = 0; u < kScaleCols; u += 4) {
        const float4 a = *reinterpret_cast<const float4*>(th_hi + i0 + u);
        const float4 b = *reinterpret_cast<const float4*>(th_lo + i0 + u);
        tih[u] = a.x; tih[u + 1] = a.y; tih[u + 2] = a.z; tih[u + 3] = a.w;
        til[u] = b.x; til[u + 1] = b.y; til[u + 2] = b.z; til[u + 3] = b.w;
      }
#pragma unroll
      for (int u = 0; u < kScaleCols; ++u)
        scale_entry(hw[u], tih[u], til[u], tjh, tjl, hmax, gmax, rgmax);
    } else {
      fetch(it + gridDim.x);
      // the ragged last item, or the one holding the diagonal entry of row j
      const int nc = min(kScaleCols, n - i0);
      for (int u = 0; u < nc; ++u) {
        const int i = i0 + u;
        const unsigned hw = (unsigned)__double2hiint(delta[(int64_t)i * ld_in + j]) & 0x7FFFFFFFu;
        if (i == j) {
          if (!en) hmax = max(hmax, hw);
          continue;
        }
        scale_entry(hw, th_hi[i], th_lo[i], tjh, tjl, hmax, gmax, rgmax);
      }
    }
  }
  scales_finish(hmax, gmax, rgmax, false, st);
}

// ---------------------------------------------------------------------------
// The scale pass from a start.  One block per column i of Delta (rows j contiguous):
// the high word of max |Delta_ji| (the FP64 bits without the sign; with its low word
// filled with ones it bounds max |Delta|) and max_{j != i} |Delta_ji| /
// |theta_i - theta_j|, both by integer atomicMax.  The ratio only places the first
// increment's scale, so it is formed cheaply: |Delta_ji| from its high word (20
// fraction bits) and the gap from the float parts of theta (their low parts where
// the high parts coincide).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_delta_scales(const double* __restrict__ delta,
                                                      int64_t ld_in, int n,
                                                      const float* __restrict__ th_hi,
                                                      const float* __restrict__ th_lo, int en,
                                                      const double* __restrict__ start,
                                                      int64_t ld_s, double* __restrict__ sinv,
                                                      IterState* st) {
  const int i = blockIdx.x;
  const float thh = th_hi[i], thl = th_lo[i];
  const double* col = delta + (int64_t)i * ld_in;
  unsigned hmax = 0u;
  float gmax = 0.f, rgmax = 0.f;   // rgmax: max 1 / |gap| (input of the error bound)
  // With a start (the polisher), the first increment is the start's offset from I:
  // X_0 = v / v_ii off the diagonal (the chart a_i = 1).  Its largest entry places the
  // first increment's scale instead of the bound |lambda| max |Delta_ji / gap|; a zero
  // or non-finite chart entry, or a non-finite entry, marks the input bad.
  float smax = 0.f;
  bool sbad = false;
  double inv = 0.0;
  const double* scol = start ? start + (int64_t)i * ld_s : nullptr;
  if (start) {
    const double piv = scol[i];
    sbad = !(piv != 0.0 && finite_bits(piv));
    inv = sbad ? 0.0 : 1.0 / piv;
    if (threadIdx.x == 0) sinv[i] = inv;
    for (int j = threadIdx.x; j < n; j += 256) {
      const double x = scol[j];
      if (!finite_bits(x)) sbad = true;
      else if (j != i) smax = fmaxf(smax, fabsf((float)(x * inv)));
    }
    if (sbad) atomicExch(&st->bad_input, 1u);
  }
  // four independent loads in flight per thread (the column streams from HBM)
  for (int jb = threadIdx.x; jb < n; jb += 1024) {
    double v[4];
    float tjh[4], tjl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jb + 256 * u;
      v[u] = j < n ? col[j] : 0.0;
      tjh[u] = j < n ? th_hi[j] : 0.f;
      tjl[u] = j < n ? th_lo[j] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jb + 256 * u;
      if (j >= n) break;
      const unsigned hw = (unsigned)__double2hiint(v[u]) & 0x7FFFFFFFu;
      if (j == i) {
        if (!en) hmax = max(hmax, hw);
        continue;
      }
      hmax = max(hmax, hw);
      const float va = abs_from_hiword(hw);
      float g = thh - tjh[u];
      if (g == 0.f) g = thl - tjl[u];
      // NaN never wins fmaxf
      const float rg = rcp_approx(fabsf(g));
      gmax = fmaxf(gmax, va * rg);
      rgmax = fmaxf(rgmax, rg);
    }
  }
  if (start) gmax = smax;   // with a start: the first increment's largest entry
  scales_finish(hmax, gmax, rgmax, start != nullptr, st);
}

// ---------------------------------------------------------------------------
// Preparation: transpose Delta (column-major FP64) into the row-major FP16 slices
// of Delta 2^sig (concatenated along K), zeroing the diagonal when the
// Epstein-Nesbet partition is used.
// ---------------------------------------------------------------------------
template <int NSL>
__global__ void __launch_bounds__(256) k_prep_delta(const double* __restrict__ delta,
                                                    int64_t ld_in, int n, int ld, int en,
                                                    __half* __restrict__ Dcat, IterState* st) {
  __shared__ double tile[32][65];
  const float sc = exp2i(st->sig);
  slice16_tile_32x64<NSL>(delta, ld_in, n, ld, en, sc, blockIdx.x * 64, blockIdx.y * 32, Dcat,
                          (int64_t)NSLICE * ld, &st->bad_input, tile);
}

// ---------------------------------------------------------------------------
// Iteration 0 (A_0 = I), computed from the FP64 input in float-float:
//   R_0 = lambda Delta (off the diagonal), d_0 = diag(Delta),
//   dt_0 = f16(G o R_0) (stored scaled by 2^sexp[0]), L_1 = R_0 - Gap o dt_0,
// plus the column partials of |R_0|^2, |a|^2 = 1, e_1 2^sig = diag(Delta 2^sig dt_0)
// from the FP16 slices (float-float) and the row partials of sum_k |Delta_jk| for the
// residual scale.  A_1 = I + dt_0 is not written: the first product and the output
// kernel form it from dt_0.  One block per 128 x 128 tile, 8 warps; each warp walks
// 16 columns with the next column's loads in flight, lane l owning rows 4l..4l+3
// (vector loads along the contiguous row index).
// ---------------------------------------------------------------------------
// START: the first increment is the start's offset X_0 = v / v_ii from I (the
// polisher), read from the caller's start matrix with the per-column 1 / v_ii of the
// scale pass; otherwise dt_0 = f16(r_0 G o R_0) with r_0 = 1 - alpha for the
// non-autonomous iteration (its first step, the identity, is not run) and 1 without.
template <int NSL, bool START>
__global__ void __launch_bounds__(256) k_iter0(const double* __restrict__ delta, int64_t ld_in,
                                               const float* __restrict__ th_hi,
                                               const float* __restrict__ th_lo, float lam_hi,
                                               float lam_lo, int n, int ld, int ntm, int en,
                                               const __half* __restrict__ Dcat,
                                               __half* __restrict__ dt0,
                                               float* __restrict__ L, double* __restrict__ d,
                                               float* __restrict__ part,
                                               float* __restrict__ rowpart,
                                               const double* __restrict__ start, int64_t ld_s,
                                               const double* __restrict__ sinv, IterState* st) {
  // 128 x 64 tiles: 2048 blocks at n = 4096, 4.5 waves of three resident blocks per SM
  // (128 x 128 tiles left a last wave a quarter full)
  constexpr int W = 8, CPW = kIter0Cols / W;   // warps, columns per warp
  __shared__ float rows[W][IT0];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n0 = blockIdx.x * kIter0Cols, m0 = blockIdx.y * IT0, tm = blockIdx.y;
  const int r0 = 4 * lane, j0 = m0 + r0;
  const int64_t cat_ld = (int64_t)NSLICE * ld;
  const float qs = exp2i(st->sexp[0]), iqs = exp2i(-st->sexp[0]);
  // strength factor of this first step (the ramp's 1 - alpha, else 1), folded into the
  // quotient's scale
  const float qr = START ? qs : qs * (float)(1.0 - st->ramp_pow);
  const float4 thj_h = *reinterpret_cast<const float4*>(th_hi + j0);
  const float4 thj_l = *reinterpret_cast<const float4*>(th_lo + j0);
  // 16-byte loads of the four rows where the column start allows them
  const bool vec = (j0 + 3 < n) && ((((uintptr_t)delta) | ((uintptr_t)ld_in * 8u)) & 15u) == 0;
  float rowabs[4] = {0.f, 0.f, 0.f, 0.f};
  float mx = 0.f;
  const int cb = n0 + CPW * w, ce = min(n, cb + CPW);
  double vn[4] = {0.0, 0.0, 0.0, 0.0};
  double sn[4] = {0.0, 0.0, 0.0, 0.0};   // the start's column (START)
  uint2 Dn[3] = {make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u)};
  auto fetch = [&](int i) {
    if (START) {
      const double* sc = start + (int64_t)i * ld_s + j0;
#pragma unroll
      for (int e = 0; e < 4; ++e) sn[e] = (j0 + e < n) ? sc[e] : 0.0;
    }
    const double* col = delta + (int64_t)i * ld_in + j0;
    if (vec) {
      const double2 x = *reinterpret_cast<const double2*>(col);
      const double2 y = *reinterpret_cast<const double2*>(col + 2);
      vn[0] = x.x; vn[1] = x.y; vn[2] = y.x; vn[3] = y.y;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) vn[e] = (j0 + e < n) ? col[e] : 0.0;
    }
    // Delta_ij (row i of the slices; columns j < ld are all written)
    const __half* Drow = Dcat + (int64_t)i * cat_ld + j0;
#pragma unroll
    for (int sl = 0; sl < NSL; ++sl) Dn[sl] = *reinterpret_cast<const uint2*>(Drow + (int64_t)sl * ld);
  };
  if (cb < ce) fetch(cb);
  for (int i = cb; i < ce; ++i) {   // uniform across the warp
    double v[4], sv[4];
    uint2 D[3];
#pragma unroll
    for (int e = 0; e < 4; ++e) { v[e] = vn[e]; sv[e] = sn[e]; }
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) D[sl] = Dn[sl];
    if (i + 1 < ce) fetch(i + 1);
    const float thi_h = th_hi[i], thi_l = th_lo[i];
    const double inv_i = START ? sinv[i] : 0.0;
    // first pass: R_0 and the scaled quotient of the four rows
    float R0h[4], R0l[4], gh[4], gl[4], q[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      R0h[e] = R0l[e] = gh[e] = gl[e] = q[e] = 0.f;
      if (j < n) {
        float vh, vl;
        split_double_fast(v[e], vh, vl);   // |v| < 2^128: checked by the slicing
        rowabs[e] += fabsf(vh);
        if (j == i) {
          d[i] = en ? 0.0 : v[e];
        } else {
          // R_0 = lambda * Delta_ji as float-float
          float pr, pe;
          two_prod(lam_hi, vh, pr, pe);
          pe = fmaf(lam_hi, vl, fmaf(lam_lo, vh, pe));
          fast_two_sum(pr, pe, R0h[e], R0l[e]);
          ff_sub(thi_h, thi_l, f4(thj_h, e), f4(thj_l, e), gh[e], gl[e]);
          // the remainder below keeps R_0 - Gap dt_0 exactly, so any reciprocal
          // close to 1/gap serves (and any increment at all: with a start it is the
          // start's offset, rounded to FP16 like every increment)
          if (START) {
            float xh, xl;
            split_double_fast(sv[e] * inv_i, xh, xl);
            q[e] = xh * qs;
          } else {
            q[e] = R0h[e] * rcp_approx(gh[e]) * qr;
          }
        }
      }
    }
    const uint2 ob = make_uint2(f16x2_sat(q[0], q[1]), f16x2_sat(q[2], q[3]));
    float4 oL;
    float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = j0 + e;
      float Ln = 0.f;
      if (j == i) {
        a2 += 1.f;
      } else if (j < n) {
        const float dtn = h_at(ob, e) * iqs;
        // L_1 = R_0 - Gap * dt_0; R0h - p is exact (p is R0h to FP16 accuracy)
        float pp, pq;
        two_prod(gh[e], dtn, pp, pq);
        pq = fmaf(gl[e], dtn, pq);
        Ln = (R0h[e] - pp) + (R0l[e] - pq);
        r2 = fmaf(R0h[e], R0h[e], r2);
        const float p1 = h_at(D[0], e) * dtn;
        float p23 = 0.f;
        if (NSL > 2) p23 = h_at(D[2], e) * dtn;
        if (NSL > 1) p23 = fmaf(h_at(D[1], e), dtn, p23);
        float sh, se;
        two_sum(eh, p1, sh, se);
        se += el + p23;
        fast_two_sum(sh, se, eh, el);
        mx = fmaxf(mx, fabsf(dtn));
      }
      f4set(oL, e, Ln);
    }
    const int64_t idx = (int64_t)i * ld + j0;
    st4(L + idx, oL);
    // rows beyond n and the diagonal hold zero increments (q = 0 there)
    *reinterpret_cast<uint2*>(dt0 + idx) = ob;
    warp_sum_ff(r2, a2, eh, el);
    if (lane == 0) {
      part[((int64_t)0 * ntm + tm) * ld + i] = r2;
      part[((int64_t)1 * ntm + tm) * ld + i] = a2;
      part[((int64_t)2 * ntm + tm) * ld + i] = eh;
      part[((int64_t)3 * ntm + tm) * ld + i] = el;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) rows[w][r0 + e] = rowabs[e];
  __syncthreads();
  const int r = threadIdx.x;
  if (r < IT0 && m0 + r < n) {
    float t = 0.f;
#pragma unroll
    for (int q2 = 0; q2 < W; ++q2) t += rows[q2][r];
    rowpart[(int64_t)blockIdx.x * ld + m0 + r] = t;
  }
  // the slice count and scale of the first product depend on the size of dt_0
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.f) atomicMax(&st->dmax_bits, __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// Iteration 0 fused with the slicing of Delta, over pairs of mirrored 64 x 64 tiles.
// Iteration 0 needs, for each entry (j, i), both Delta_ji (its increment, remainder
// and |R_0|^2) and the transposed entry Delta_ij (the diagonal term
// e_i 2^sig = sum_j Delta_ij 2^sig dt0_ji, from the FP16 slices), and the slicing
// writes Delta_ij into row i of the row-major slices.  A block that holds tile
// (M, C) and its mirror (C, M) therefore does both kernels' work while reading each
// entry of Delta from HBM once (the separate slicing pass and the transposed re-read
// of the slices are gone).
//
// Roles (128 threads): threads 0-63 own the columns f of tile C (entries (l, f),
// l in M); threads 64-127 own the columns f of tile M (entries (l, f), l in C) in
// 16-column slabs, 16 threads per column, each over 16 of the 64 rows.  A thread
// that owns entry (l, f) also takes the transposed entry (f, l): its slices go to row
// f of Dcat, its magnitude to the row sum of row f, and its product with the
// increment of (l, f) to e_f.  Every column's sums are then thread-local (no warp
// reductions), and every output a thread writes is a run along its own column (dt0,
// L) or row (Dcat): per slab, 32-byte stores (one sector each; 16-byte stores of half
// slabs measured 14 % slower).  The diagonal tiles (M = C) use the first role only.
//
// Data: slabs of 16 rows of M, staged by TMA (FP64, 16 x 16 boxes, 128-byte swizzle,
// zero fill beyond n) in a two-stage ring: the main slab (rows of the slab x the 64
// columns of C) and the mirror slab (the 64 rows of C x the slab's columns).  With the
// swizzle every shared-memory access pattern below is free of bank conflicts.
// Column partials go to 64-row slots (part, nslot = ld / 64 slots per quantity), row
// partials to rowpart (one per 64 columns, as the unfused kernel).
// ---------------------------------------------------------------------------
constexpr int F0T = 64;                        // tile edge
constexpr int F0_BOX = 16 * 128;               // one 16 x 16 FP64 box (16 lines of 128 B)
constexpr int F0_HALF = (F0T / 16) * F0_BOX;   // main or mirror slab: 8 KB
constexpr int F0_STAGE = 2 * F0_HALF;          // 16 KB per ring stage
constexpr int F0_NST = 2;                      // ring stages
constexpr int F0_SMEM = F0_NST * F0_STAGE + 1024;   // the ring + 1024-byte alignment slack

__device__ __forceinline__ void lds_f64x2(const unsigned char* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ double lds_f64(const unsigned char* p) {
  return *reinterpret_cast<const double*>(p);
}
__device__ __forceinline__ void bar_sync_mirror() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

template <int NSL>
__global__ void __launch_bounds__(128) k_iter0_pairs(const __grid_constant__ CUtensorMap tmD,
                                                     const float* __restrict__ th_hi,
                                                     const float* __restrict__ th_lo,
                                                     float lam_hi, float lam_lo, int n, int ld,
                                                     int nt, int en, __half* __restrict__ Dcat,
                                                     __half* __restrict__ dt0,
                                                     float* __restrict__ L, double* __restrict__ d,
                                                     float* __restrict__ part,
                                                     float* __restrict__ rowpart, IterState* st) {
  extern __shared__ unsigned char f0_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)f0_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[F0_NST];
  __shared__ __align__(16) float thA_h[F0T], thA_l[F0T], thB_h[F0T], thB_l[F0T];   // theta of M, C
  __shared__ float red[4][16];   // second mirror warp's column sums, handed to the first

  // unit -> tile pair (tm <= tc): the off-diagonal pairs first, the diagonal tiles last
  const int u = blockIdx.x;
  const int noff = nt * (nt - 1) / 2;
  int tm, tc;
  if (u < noff) {
    int b = (int)((1.f + sqrtf(1.f + 8.f * (float)u)) * 0.5f);
    while (b * (b - 1) / 2 > u) --b;
    while ((b + 1) * b / 2 <= u) ++b;
    tc = b;
    tm = u - b * (b - 1) / 2;
  } else {
    tm = tc = u - noff;
  }
  const int M0 = tm * F0T, C0 = tc * F0T;
  if (M0 >= n) return;   // both tiles beyond n (M0 <= C0): nothing to write
  const bool diag = (tm == tc);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* tflag = &st->timeout;

  if (tid == 0) {
    for (int q = 0; q < F0_NST; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
  }
  if (tid < F0T) {
    const int r = M0 + tid, c = C0 + tid;
    thA_h[tid] = r < n ? th_hi[r] : 0.f;
    thA_l[tid] = r < n ? th_lo[r] : 0.f;
    thB_h[tid] = c < n ? th_hi[c] : 0.f;
    thB_l[tid] = c < n ? th_lo[c] : 0.f;
  }
  __syncthreads();
  // slab s: main = rows [M0 + 16 s, +16) x columns C, mirror = rows C x those columns
  auto issue = [&](int s) {
    uint64_t* bar = &full[s % F0_NST];
    unsigned char* base = sm + (s % F0_NST) * F0_STAGE;
    mbar_arrive_expect_tx(bar, F0_STAGE);
#pragma unroll
    for (int b = 0; b < F0T / 16; ++b) {
      tma_load_2d(base + b * F0_BOX, &tmD, bar, M0 + 16 * s, C0 + 16 * b);
      tma_load_2d(base + F0_HALF + b * F0_BOX, &tmD, bar, C0 + 16 * b, M0 + 16 * s);
    }
  };
  constexpr int NSLAB = F0T / 16;
  if (tid == 0)
    for (int q = 0; q < F0_NST && q < NSLAB; ++q) issue(q);

  const float sc = exp2i(st->sig);
  const int se0 = st->sexp[0];
  const float iqs = exp2i(-se0);
  // strength factor of this first step (the ramp's 1 - alpha, else 1), folded into the
  // quotient's scale
  const float qr = exp2i(se0) * (float)(1.0 - st->ramp_pow);
  const int64_t cat_ld = (int64_t)NSLICE * ld;
  const bool mainr = tid < F0T;
  const int t = mainr ? tid : tid - F0T;
  const int ml = t & 15, g = t >> 4;   // mirror role: column in the slab, group of 16 rows
  float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f, rows = 0.f, mx = 0.f;
  bool badv = false;
  bool ok = true;
  int s = 0;
  for (; s < NSLAB; ++s) {
    const bool got = mbar_wait(&full[s % F0_NST], (s / F0_NST) & 1, tflag);
    if (!__syncthreads_and(got)) {
      ok = false;
      break;
    }
    const unsigned char* mb = sm + (s % F0_NST) * F0_STAGE;   // main slab
    const unsigned char* rb = mb + F0_HALF;              // mirror slab
    if (mainr || !diag) {
      // the fixed index f (owned column, row of the transposed entries) and the
      // first loop index of this slab
      const int f = mainr ? C0 + t : M0 + 16 * s + ml;
      const float tfh = mainr ? thB_h[t] : thA_h[16 * s + ml];
      const float tfl = mainr ? thB_l[t] : thA_l[16 * s + ml];
      if (!mainr) { r2 = 0.f; eh = 0.f; el = 0.f; rows = 0.f; }
      // Eight loop indices l = lb .. lb + 7 of this thread: the owned entries (l, f) and
      // the transposed ones (f, l).  PLAIN: no diagonal entry and every l < n (all
      // but the diagonal tiles and the ragged last tile), so no per-entry tests.
      auto eight = [&](int h, auto plain_tag, uint32_t(&qw)[4], float(&Lo)[8],
                       uint32_t(&Dw)[NSL][4]) {
        constexpr bool PLAIN = decltype(plain_tag)::value;
        const int lb = mainr ? M0 + 16 * s + 8 * h : C0 + 16 * g + 8 * h;
        const int tl0 = mainr ? 16 * s + 8 * h : 16 * g + 8 * h;   // theta of l, in shared
        const float* tlh = mainr ? thA_h + tl0 : thB_h + tl0;
        const float* tll = mainr ? thA_l + tl0 : thB_l + tl0;
        double vo[8], vr[8];   // owned (l, f), transposed (f, l)
        if (mainr) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            lds_f64x2(mb + t * 128 + (((4 * h + kk) ^ (t & 7)) << 4), vo[2 * kk], vo[2 * kk + 1]);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            vr[k] = lds_f64(rb + (t >> 4) * F0_BOX + (8 * h + k) * 128 +
                            ((((t & 15) >> 1) ^ k) << 4) + ((t & 1) << 3));
        } else {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            lds_f64x2(rb + g * F0_BOX + ml * 128 + (((4 * h + kk) ^ (ml & 7)) << 4), vo[2 * kk],
                      vo[2 * kk + 1]);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            vr[k] = lds_f64(mb + (16 * g + 8 * h + k) * 128 + (((ml >> 1) ^ k) << 4) +
                            ((ml & 1) << 3));
        }
        float tlv_h[8], tlv_l[8];
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
          const float4 a = *reinterpret_cast<const float4*>(tlh + k);
          const float4 b = *reinterpret_cast<const float4*>(tll + k);
          tlv_h[k] = a.x; tlv_h[k + 1] = a.y; tlv_h[k + 2] = a.z; tlv_h[k + 3] = a.w;
          tlv_l[k] = b.x; tlv_l[k + 1] = b.y; tlv_l[k + 2] = b.z; tlv_l[k + 3] = b.w;
        }
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          float R0h[2], R0l[2], gh[2], gl[2], q[2], Ds[NSL][2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int l = lb + k + e;
            const bool on = !PLAIN && (l == f);
            // transposed entry (f, l): FP16 slices of Delta_fl 2^sig, as the slicing
            // kernel forms them (hi 2^sig, then the rounding remainders; the last slice
            // takes lo 2^sig as well); zero on the diagonal with Epstein-Nesbet
            float rh, rl;
            split_double_fast(vr[k + e], rh, rl);
            badv |= beyond_float(vr[k + e]);
            rows += fabsf(rh);
            if (!PLAIN && en && on) rh = rl = 0.f;
            float r = rh * sc;
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl) {
              const float tt = (sl == NSL - 1) ? r + rl * sc : r;
              const float qh = __half2float(__float2half_rn(tt));
              r = tt - qh;
              Ds[sl][e] = qh;
            }
            // owned entry (l, f): R_0 = lambda Delta_lf (float-float), the gap
            // theta_f - theta_l, the scaled quotient
            R0h[e] = R0l[e] = gh[e] = gl[e] = q[e] = 0.f;
            if (on) {
              d[f] = en ? 0.0 : vo[k + e];
              a2 += 1.f;
            } else if (PLAIN || l < n) {
              float vh, vl;
              split_double_fast(vo[k + e], vh, vl);
              float pr, pe;
              two_prod(lam_hi, vh, pr, pe);
              pe = fmaf(lam_hi, vl, fmaf(lam_lo, vh, pe));
              fast_two_sum(pr, pe, R0h[e], R0l[e]);
              ff_sub(tfh, tfl, tlv_h[k + e], tlv_l[k + e], gh[e], gl[e]);
              q[e] = R0h[e] * rcp_approx(gh[e]) * qr;
            }
          }
          const uint32_t w = f16x2_sat(q[0], q[1]);
          qw[k >> 1] = w;
          const float2 dq = __half22float2(*reinterpret_cast<const __half2*>(&w));
          const float dtn[2] = {dq.x * iqs, dq.y * iqs};
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl) {
            const __half2 hp = __floats2half2_rn(Ds[sl][0], Ds[sl][1]);   // exact
            Dw[sl][k >> 1] = *reinterpret_cast<const uint32_t*>(&hp);
          }
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            // L_1 = R_0 - Gap dt_0 (R0h - p exact: p is R0h to FP16 accuracy)
            float pp, pq;
            two_prod(gh[e], dtn[e], pp, pq);
            pq = fmaf(gl[e], dtn[e], pq);
            Lo[k + e] = (R0h[e] - pp) + (R0l[e] - pq);
            r2 = fmaf(R0h[e], R0h[e], r2);
            const float p1 = Ds[0][e] * dtn[e];
            float p23 = 0.f;
            if (NSL > 2) p23 = Ds[2][e] * dtn[e];
            if (NSL > 1) p23 = fmaf(Ds[1][e], dtn[e], p23);
            float sh, se;
            two_sum(eh, p1, sh, se);
            se += el + p23;
            fast_two_sum(sh, se, eh, el);
            mx = fmaxf(mx, fabsf(dtn[e]));
          }
        }
      };
      if (f < n) {
        // the sixteen loop indices of the slab, then 32-byte stores (one FP16 sector of
        // dt_0 and of each slice, two of L_1) along column f and row f
        uint32_t qw[2][4], Dw[2][NSL][4];
        float Lo[2][8];
        const int lend = mainr ? M0 + 16 * s + 16 : C0 + 16 * g + 16;
        if (!diag && lend <= n) {
          eight(0, std::true_type{}, qw[0], Lo[0], Dw[0]);
          eight(1, std::true_type{}, qw[1], Lo[1], Dw[1]);
        } else {
          eight(0, std::false_type{}, qw[0], Lo[0], Dw[0]);
          eight(1, std::false_type{}, qw[1], Lo[1], Dw[1]);
        }
        const int lb = mainr ? M0 + 16 * s : C0 + 16 * g;
        const int64_t oc = (int64_t)f * ld + lb;   // column f, rows lb.. (dt0, L)
        st_global_v8(dt0 + oc, qw[0][0], qw[0][1], qw[0][2], qw[0][3], qw[1][0], qw[1][1],
                     qw[1][2], qw[1][3]);
#pragma unroll
        for (int h = 0; h < 2; ++h)
          st_global_v8(L + oc + 8 * h, __float_as_uint(Lo[h][0]), __float_as_uint(Lo[h][1]),
                       __float_as_uint(Lo[h][2]), __float_as_uint(Lo[h][3]),
                       __float_as_uint(Lo[h][4]), __float_as_uint(Lo[h][5]),
                       __float_as_uint(Lo[h][6]), __float_as_uint(Lo[h][7]));
        const int64_t orow = (int64_t)f * cat_ld + lb;   // row f of the slices
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl)
          st_global_v8(Dcat + orow + (int64_t)sl * ld, Dw[0][sl][0], Dw[0][sl][1], Dw[0][sl][2],
                       Dw[0][sl][3], Dw[1][sl][0], Dw[1][sl][1], Dw[1][sl][2], Dw[1][sl][3]);
      }
      if (!mainr) {
        // column f over the 64 rows of C: the four groups of 16 rows (lanes l and
        // l + 16 of each mirror warp, then the two warps)
        float o2 = __shfl_xor_sync(0xffffffffu, r2, 16);
        float ohh = __shfl_xor_sync(0xffffffffu, eh, 16);
        float oll = __shfl_xor_sync(0xffffffffu, el, 16);
        float orw = __shfl_xor_sync(0xffffffffu, rows, 16);
        {
          float sh, se;
          two_sum(eh, ohh, sh, se);
          se += el + oll;
          fast_two_sum(sh, se, eh, el);
          r2 += o2;
          rows += orw;
        }
        if (warp == 3 && lane < 16) {
          red[0][lane] = r2; red[1][lane] = eh; red[2][lane] = el; red[3][lane] = rows;
        }
        bar_sync_mirror();
        if (warp == 2 && lane < 16 && f < n) {
          float sh, se;
          two_sum(eh, red[1][lane], sh, se);
          se += el + red[2][lane];
          fast_two_sum(sh, se, eh, el);
          r2 += red[0][lane];
          rows += red[3][lane];
          const int nslot = nt;
          part[((int64_t)0 * nslot + tc) * ld + f] = r2;
          part[((int64_t)1 * nslot + tc) * ld + f] = 0.f;
          part[((int64_t)2 * nslot + tc) * ld + f] = eh;
          part[((int64_t)3 * nslot + tc) * ld + f] = el;
          if (C0 < n) rowpart[(int64_t)tc * ld + f] = rows;
        }
      }
    }
    __syncthreads();   // the slab's stage is free again
    if (tid == 0 && s + F0_NST < NSLAB) issue(s + F0_NST);
  }
  if (!ok) {
    // let the copies in flight land before the block exits
    if (tid == 0)
      for (int x = s; x < NSLAB && x < s + F0_NST; ++x)
        mbar_wait_quiet(&full[x % F0_NST], (x / F0_NST) & 1, kTailWaitNs);
    return;
  }
  if (mainr && C0 + t < n) {
    const int f = C0 + t, nslot = nt;
    part[((int64_t)0 * nslot + tm) * ld + f] = r2;
    part[((int64_t)1 * nslot + tm) * ld + f] = a2;
    part[((int64_t)2 * nslot + tm) * ld + f] = eh;
    part[((int64_t)3 * nslot + tm) * ld + f] = el;
    rowpart[(int64_t)tm * ld + f] = rows;
  }
  if (badv) atomicExch(&st->bad_input, 1u);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.f) atomicMax(&st->dmax_bits, __float_as_uint(mx));
}

// ---------------------------------------------------------------------------
// Control: reduce the column partials of the last update, read out the
// eigenvalues of the iterate A_k (E = theta + lambda d_k, Sec. II.B read-out),
// advance d, and decide: converged / diverged / max_iter / continue (and with
// how many Delta slices).  The last block to finish takes the decision.
// ---------------------------------------------------------------------------
// The decision of k_ctrl on the register copy of the state (see state_load).
__device__ __forceinline__ void ctrl_decide(IterState& ls, bool first, bool cert) {
  IterState* vs = &ls;
  if (first) vs->s = vs->theta_max + fabs(vs->lam) * (double)__uint_as_float(vs->row_bits);
  const double rho = (double)__uint_as_float(vs->rho_bits) / vs->s;
  vs->blocks_done = 0;
  vs->rho_bits = 0;
  const float dmax = __uint_as_float(vs->dmax_bits);
  vs->dmax_bits = 0;
  // every increment of the returned iterate is bounded by one of these maxima
  vs->dsum = vs->dsum + (double)dmax;
  // the rounding of the float recursion grows with the residuals it carried
  if (!first) vs->rho_sum = vs->rho_sum + rho;
  if (cert) {
    // the certifying pass assessed A_k: stop if it passed, else run the same
    // iteration again in full (nothing it depends on was touched)
    vs->certify = 0;
    if (decide_final(vs, rho)) vs->slice_gemms = vs->slice_gemms + vs->slices;
    // a pass that certified A_k and wrote it as the FP64 output leaves the output
    // kernel nothing to do
    else if (vs->status == ST_CONVERGED && vs->cert_out) vs->out_done = 1;
    return;
  }
  const double prev = vs->rho_last;
  vs->rho_last = rho;
  if (!decide(vs, rho)) return;
  const int S = next_slices_f16(vs, dmax, first, vs->max_slices);
  vs->slices = S;
  vs->slice_gemms = vs->slice_gemms + S;
  // the next product writes dt_k into buffer cur: scaled so that the largest
  // increment of the last step, dmax, would land at 2^10 (increments shrink as the
  // iteration converges; 32-fold growth still fits, more is clamped and the
  // remainder keeps the rest)
  vs->sexp[vs->cur] = dt_scale_exp((double)dmax, 10, vs->sig, vs->lam);
  // When the residual falls geometrically and the next one is predicted below half
  // the tolerance, the next product only forms the residual of its iterate (no new
  // iterate, increment or remainder is written): the last product of a converging
  // solve then costs little more than its matrix product.
  vs->certify = (vs->certify_on && vs->k >= 3 && prev > 0.0 && rho < prev &&
                 rho * (rho / prev) <= 0.5 * vs->tol) ? 1 : 0;
}

__global__ void __launch_bounds__(256) k_ctrl(int n, int ld, int ntm, int ntn,
                                              const float* __restrict__ part,
                                              const float* __restrict__ rowpart,
                                              const double* __restrict__ theta,
                                              double* __restrict__ d, double* __restrict__ E,
                                              float* __restrict__ e_col,
                                              float* __restrict__ dprev_col, IterState* st,
                                              int hilo, int first_step) {
  // 32 columns per block, 8 threads per column each summing every 8th tile partial
  // (short chains of independent loads: the partials were just written, in L2).  The
  // loads depend on nothing in the state (first_step: this control follows iteration
  // 0), so they are issued before the state is read; the status test follows them.
  __shared__ float sh[3][8][32];
  __shared__ double she[8][32];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + c;
  const bool first = first_step != 0;
  {
    float r2 = 0.f, a2 = 0.f, rs = 0.f;
    double ep = 0.0;
    if (i < n) {
      if (first || hilo) {
#pragma unroll 4
        for (int t = g; t < ntm; t += 8) {
          r2 += part[((int64_t)0 * ntm + t) * ld + i];
          a2 += part[((int64_t)1 * ntm + t) * ld + i];
          ep += (double)part[((int64_t)2 * ntm + t) * ld + i] +
                (double)part[((int64_t)3 * ntm + t) * ld + i];
        }
        if (first)
          for (int t = g; t < ntn; t += 8) rs += rowpart[(int64_t)t * ld + i];
      } else {
        // the pair kernel's diagonal partials are plain floats (their low parts are
        // zero, and x + 0 = x): one conversion and one FP64 add per partial
#pragma unroll 4
        for (int t = g; t < ntm; t += 8) {
          r2 += part[((int64_t)0 * ntm + t) * ld + i];
          a2 += part[((int64_t)1 * ntm + t) * ld + i];
          ep += (double)part[((int64_t)2 * ntm + t) * ld + i];
        }
      }
    }
    sh[0][g][c] = r2; sh[1][g][c] = a2; sh[2][g][c] = rs; she[g][c] = ep;
  }
  if (st->status != ST_RUNNING) return;   // the same for every thread of the launch
  // after a certifying product only its residual norms are valid: the iterate, d and
  // the column parameters of the next product stay as they are
  const bool cert = st->certify != 0;
  // the diagonal partials are of Delta 2^sig dt (FP16 slices): exact rescaling
  const double isg = (double)exp2i(-st->sig);
  __syncthreads();
  float rho_raw = 0.f;
  if (g == 0 && i < n) {
    float r2 = 0.f, a2 = 0.f;
    double ep = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { r2 += sh[0][q][c]; a2 += sh[1][q][c]; ep += she[q][c]; }
    ep *= isg;
    rho_raw = sqrtf(r2 / a2);
    if (!(rho_raw == rho_raw) || isinf(rho_raw)) rho_raw = __int_as_float(0x7f800000);
    const double dk = d[i];
    E[i] = theta[i] + st->lam * dk;
    if (!cert) {
      dprev_col[i] = (float)dk;
      e_col[i] = (float)ep;
      d[i] = dk + ep;
    }
    if (first) {
      float rs = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) rs += sh[2][q][c];
      atomicMax(&st->row_bits, __float_as_uint(rs));
    }
  }
  // block max of rho_raw
  float m = rho_raw;
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wm[32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) bm = fmaxf(bm, wm[q]);
    atomicMax(&st->rho_bits, __float_as_uint(bm));
    __threadfence();
    last = (atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  IterState ls;
  state_load(st, ls);
  ctrl_decide(ls, first, cert);
  state_store(st, ls);
}


// ---------------------------------------------------------------------------
// The tensor-core iteration: X = [D1 D2 D3](:, :S) * dt_{k-1} on tcgen05 with TMA
// loads, fused with the update epilogue.  Persistent and warp-specialised: one
// CTA per SM walks the 128 x 128 output tiles round-robin.
//   warp 0       TMA producer: A (Delta slices) and B (dt) tiles into a STAGES ring
//   warp 1       MMA issuer: one elected thread, accumulators alternate between two
//                TMEM buffers so the next tile's products overlap this tile's epilogue
//   warps 2-9    epilogue, per tile in two phases:
//                (1) TMEM -> shared memory (column-major FP32 tile), then the TMEM
//                    buffer is handed back to the MMA warp;
//                (2) column walk: each warp takes 16 columns, lane l owns rows
//                    4l..4l+3, so every global access is a 16-byte vector along the
//                    contiguous row index and each column's sums are one warp
//                    reduction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// Barrier over the 256 epilogue threads that also returns the AND of `v` over them,
// so every epilogue warp takes the same branch afterwards (and the same number of
// barriers in all).
__device__ __forceinline__ bool epi_bar_and(bool v) {
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

// Phase 2 for one chunk: update the 4 columns [c0 + 4 ew, c0 + 4 ew + 4) of the
// tile; Xs holds the chunk's XCH accumulator columns.
__device__ __forceinline__ void epilogue_columns(const GemmEpiParams& p, GemmSmemMisc* ms,
                                                 const float* Xs, int ew, int lane, int tm,
                                                 int m0, int n0, int c0, float& mx) {
  const int n = p.n, ld = p.ld;
  const int S = ms->slices;
  const bool c1 = (ms->cur != 0);
  // a certifying pass forms only the residual of the current iterate (nothing is
  // written but its norms), see k_ctrl
  const bool cert = ms->certify != 0;
  const bool a1 = ms->k == 1;             // A_1 = I + dt_0, formed from dt_0
  // explicit selects: indexing the parameter arrays with a runtime value would
  // copy the parameter block to local memory
  const float* __restrict__ Ahc = c1 ? p.A_hi[1] : p.A_hi[0];
  const float* __restrict__ Alc = c1 ? p.A_lo[1] : p.A_lo[0];
  float* __restrict__ Ahn = c1 ? p.A_hi[0] : p.A_hi[1];
  float* __restrict__ Aln = c1 ? p.A_lo[0] : p.A_lo[1];
  const __half* __restrict__ dtp = c1 ? p.dt[0] : p.dt[1];   // dt_{k-1} 2^scur
  __half* __restrict__ dtn_out = c1 ? p.dt[1] : p.dt[0];     // dt_k 2^snew
  float* __restrict__ L = p.L;
  // the accumulator holds 2^(sig + scur) Delta dt_{k-1}: lambda carries the inverse
  // scale and the per-column parameters the matching ones (all exact)
  const float lam = (p.lam * exp2i(-ms->sig)) * exp2i(-ms->scur);
  const float qs = exp2i(ms->snew), iqs = exp2i(-ms->snew);
  // non-autonomous step: dt = r G o R - (1 - r)(A - I), r = 1 - rpow (1 without)
  const float rq = (1.f - ms->rpow) * qs, oq = ms->rpow * qs;
  const int r0 = 4 * lane;                // rows r0..r0+3 of the tile
  const int j0 = m0 + r0;
  // rows beyond n lie in the padded part of every work array (ld is a multiple of
  // the tile height): they are read, masked and written back as zeros
  const float4 thj_h = ld4(p.th_hi + j0);
  const float4 thj_l = ld4(p.th_lo + j0);
  constexpr int U = 4;                    // columns in flight per lane
  {
    const int cb = c0 + 4 * ew;           // first tile column of this warp
    Col4 in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = n0 + cb + u;
      if (i < n) {
        const int64_t idx = (int64_t)i * ld + j0;
        in[u].L = ld4(L + idx);
        in[u].dtp = *reinterpret_cast<const uint2*>(dtp + idx);
        if (a1) {   // off the diagonal A_1 = dt_0 (its diagonal entry is never read)
          const float isc = exp2i(-ms->scur);
          in[u].ah = make_float4(h_at(in[u].dtp, 0) * isc, h_at(in[u].dtp, 1) * isc,
                                 h_at(in[u].dtp, 2) * isc, h_at(in[u].dtp, 3) * isc);
        } else {
          in[u].ah = ld4(Ahc + idx);
        }
        in[u].al = (cert || a1) ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(Alc + idx);
        // Delta_ij 2^sig for j = j0..j0+3: row i of the row-major slices.  The
        // diagonal partial uses as many slices as this product: its truncation error
        // then obeys the same bound as the product's (see next_slices_f16)
        const __half* Drow = p.Dcat + (int64_t)i * p.cat_ld + j0;
        const int Se = cert ? 0 : S;
        in[u].D[0] = Se > 0 ? *reinterpret_cast<const uint2*>(Drow) : make_uint2(0u, 0u);
        in[u].D[1] = Se > 1 ? *reinterpret_cast<const uint2*>(Drow + ld) : make_uint2(0u, 0u);
        in[u].D[2] = Se > 2 ? *reinterpret_cast<const uint2*>(Drow + 2 * (int64_t)ld) : make_uint2(0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int cl = cb + u;
      const int i = n0 + cl;
      if (i >= n) continue;   // uniform across the warp
      const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * BM + r0);
      const float e_i = ms->e[cl], dp_i = ms->dprev[cl];
      const float thh = ms->thh[cl], thl = ms->thl[cl];
      float4 oh, ol, oL;
      float r2 = 0.f, a2 = 0.f, eh = 0.f, el = 0.f;
      uint2 ob;
      // two rows at a time: the residual and the scaled quotient R / Gap, one packed
      // FP16 conversion (the increment as applied, so the remainder below keeps
      // R - Gap dt exactly whatever the rounding or clamping did), then the rest
#pragma unroll
      for (int hp = 0; hp < 2; ++hp) {
        float R[2], gh[2], gl[2], q[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int e = 2 * hp + t, j = j0 + e;
          R[t] = gh[t] = gl[t] = q[t] = 0.f;
          if (j != i && j < n) {
            const float ah = f4(in[u].ah, e);
            R[t] = f4(in[u].L, e) + lam * (f4(x4, e) - ah * e_i - h_at(in[u].dtp, e) * dp_i);
            r2 = fmaf(R[t], R[t], r2);
            a2 = fmaf(ah, ah, a2);
            if (!cert) {
              ff_sub(thh, thl, f4(thj_h, e), f4(thj_l, e), gh[t], gl[t]);
              q[t] = fmaf(R[t] * __frcp_rn(gh[t]), rq, -ah * oq);
            }
          }
        }
        const uint32_t w = f16x2_sat(q[0], q[1]);
        if (hp == 0) ob.x = w; else ob.y = w;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int e = 2 * hp + t, j = j0 + e;
          const float ah = f4(in[u].ah, e), al = f4(in[u].al, e);
          float nh = 0.f, nl = 0.f, Ln = 0.f;
          if (j == i) {
            nh = 1.f;
            a2 += 1.f;
          } else if (j < n && !cert) {
            const float dnew = h_at(ob, e) * iqs;
            Ln = fmaf(-gh[t], dnew, R[t]) - gl[t] * dnew;
            ff_add_f(ah, al, dnew, nh, nl);
            // e_{k+1} 2^sig partial Delta_ij 2^sig dt_ji: the slice products are
            // exact (11-bit significands), summed in float-float
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
      }
      const int64_t idx = (int64_t)i * ld + j0;
      if (!cert) {
        st4(Ahn + idx, oh);
        st4(Aln + idx, ol);
        st4(L + idx, oL);
        *reinterpret_cast<uint2*>(dtn_out + idx) = ob;
      }
      warp_sum_ff(r2, a2, eh, el);
      if (lane == 0) {
        p.part[((int64_t)0 * p.ntm + tm) * ld + i] = r2;
        p.part[((int64_t)1 * p.ntm + tm) * ld + i] = a2;
        if (!cert) {
          p.part[((int64_t)2 * p.ntm + tm) * ld + i] = eh;
          p.part[((int64_t)3 * p.ntm + tm) * ld + i] = el;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm_epi(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
           const __grid_constant__ CUtensorMap tmB1, const GemmEpiParams p) {
  extern __shared__ uint8_t smem_raw[];
  IterState* st = p.st;
  if (*((volatile int*)&st->status) != ST_RUNNING) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_TILE;
  float* Xs = reinterpret_cast<float*>(smem + SMEM_TILES);
  GemmSmemMisc* ms = (GemmSmemMisc*)(smem + SMEM_TILES + SMEM_X);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bn = p.bn;
  const int ntn = (p.n + bn - 1) / bn;
  const int ntiles = ntn * p.ntm;

  if (threadIdx.x == 0) {
    ms->k = st->k;
    ms->slices = st->slices;
    ms->certify = st->certify;
    ms->cur = st->cur;
    ms->sig = st->sig;
    ms->scur = st->sexp[st->cur ^ 1];
    ms->snew = st->sexp[st->cur];
    ms->rpow = (float)st->ramp_pow;
    for (int s = 0; s < STAGES; ++s) { mbar_init(&ms->full[s], 1); mbar_init(&ms->empty[s], 1); }
    for (int b = 0; b < NACC; ++b) { mbar_init(&ms->acc_full[b], 1); mbar_init(&ms->acc_empty[b], 1); }
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&ms->tmem_base, NACC * BN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ms->tmem_base;
  const int S = ms->slices;
  const int kb_per_slice = p.ld / BK;
  const int nk = S * kb_per_slice;
  const CUtensorMap* tmB = (ms->cur == 1) ? &tmB0 : &tmB1;   // dt_{k-1} lives in buffer cur^1
  unsigned* tflag = &st->timeout;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    prefetch_tmap(&tmA);
    prefetch_tmap(tmB);
    uint32_t it = 0;   // running stage counter over all tiles
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
      const int tm = t / ntn, tn = t % ntn;
      const int m0 = tm * BM, n0 = tn * bn;
      const int kb_last = min(kb_per_slice - 1, (n0 + bn - 1) / BK);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!mbar_wait(&ms->empty[s], ph ^ 1, tflag)) { alive = false; break; }
        mbar_arrive_expect_tx(&ms->full[s], A_TILE + (uint32_t)bn * BK * 2);
        // Accumulation order.  The tensor core accumulates in FP32 and drops the
        // bits below the running sum at every step, so the error of a chain grows
        // with the size of the partial sums it carries.  Column i of Delta dt is
        // dominated by k near i (G_ki ~ 1/(theta_i - theta_k)), so the small slices
        // go first and each slice's K-blocks are rotated to end on the blocks of
        // this tile's own columns: the large terms enter last, with few steps left.
        const int sl = S - 1 - q / kb_per_slice;
        const int kb = (kb_last + 1 + q % kb_per_slice) % kb_per_slice;
        tma_load_2d(sA + s * A_TILE, &tmA, &ms->full[s], sl * p.ld + kb * BK, m0);
        tma_load_2d(sB + s * B_TILE, tmB, &ms->full[s], kb * BK, n0);
      }
    }
    // drain: every issued copy must have landed before the CTA can exit
    for (uint32_t t = (it > STAGES ? it - STAGES : 0); t < it; ++t)
      mbar_wait(&ms->full[t % STAGES], (t / STAGES) & 1, tflag);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = idesc_f16_f32(BM, bn);
    uint32_t it = 0;
    int lt = 0;   // local tile counter
    bool alive = true;
    for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++lt) {
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      if (!mbar_wait(&ms->acc_empty[b], (use & 1) ^ 1, tflag)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * BN);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!mbar_wait(&ms->full[s], ph, tflag)) { alive = false; break; }
        tc_fence_after();
        const uint64_t da = smem_desc_sw128(sA + s * A_TILE);
        const uint64_t db = smem_desc_sw128(sB + s * B_TILE);
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk) {
          // advance the start address by kk * 32 bytes inside the swizzle atom
          umma_f16(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                    (q > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(&ms->empty[s]);
      }
      umma_commit(&ms->acc_full[b]);
    }
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int ew = warp - 2;        // 0..7
    const int qd = warp & 3;        // TMEM lane quadrant of this warp
    const int half = ew >> 2;       // which 16 of a chunk's 32 columns this warp copies
    const int et = threadIdx.x - 64;
    const float cs = exp2i(ms->scur), cd = exp2i(ms->sig);
    float mx = 0.f;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int tm = t / ntn, tn = t % ntn;
      const int m0 = tm * BM, n0 = tn * bn;
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      epi_bar();   // the previous tile's column walk has finished with Xs and params
      if (et < bn) {
        const int i = n0 + et;
        const bool v = i < p.n;
        ms->e[et] = v ? (p.e_col[i] * cd) * cs : 0.f;   // e_k 2^sig 2^scur
        ms->dprev[et] = v ? p.dprev_col[i] * cd : 0.f;
        ms->thh[et] = v ? p.th_hi[i] : 0.f;
        ms->thl[et] = v ? p.th_lo[i] : 0.f;
      }
      // warp-uniform: the TMEM loads below are .sync.aligned
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&ms->acc_full[b], use & 1, tflag));
      tc_fence_after();
      const uint32_t src = tmem + (uint32_t)(b * BN) + ((uint32_t)(qd * 32) << 16);
      bool all_ok = true;
#pragma unroll 1
      for (int c0 = 0; c0 < bn; c0 += XCH) {
        if (c0 > 0) epi_bar();   // the previous chunk's column walk is done with Xs
        // phase 1: this warp's quadrant, 16 of the chunk's 32 columns
        if (ok) {
          float x[16];
          const int cc = half * 16;
          tmem_ld_x16(src + (uint32_t)(c0 + cc), x);
#pragma unroll
          for (int c = 0; c < 16; ++c) Xs[(cc + c) * BM + qd * 32 + lane] = x[c];
        }
        if (c0 + XCH == bn) tc_fence_before();
        all_ok = epi_bar_and(ok);   // Xs holds the chunk
        // after the last chunk is staged the TMEM buffer can be refilled
        if (c0 + XCH == bn && et == 0) mbar_arrive(&ms->acc_empty[b]);
        if (!all_ok) break;
        epilogue_columns(p, ms, Xs, ew, lane, tm, m0, n0, c0, mx);
      }
      if (!all_ok) break;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.f) atomicMax(&p.st->dmax_bits, __float_as_uint(mx));
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NACC * BN);
  }
}

// ---------------------------------------------------------------------------
// Staged epilogue (CTA-pair kernel).  The column walk of k_gemm_epi, with its
// global inputs brought into shared memory by the lane that will use them, with
// cp.async one sub-chunk ahead, so that their latency overlaps the arithmetic of
// the previous sub-chunk (and, for a tile's first sub-chunk, the wait for its
// accumulator).  A sub-chunk is 16 columns, one per warp.  Each lane keeps its own
// slots (80 B per column: A_hi, A_lo, L as float4, then dt_{k-1} and the Delta
// slices as FP16 quadruples), so no barrier guards them.
// ---------------------------------------------------------------------------
// (the pair kernel's products use at most two slices: the increment and two slices
// fill the three 8-byte slots)
__device__ __forceinline__ uint8_t* eb_f4(uint8_t* eb, int ew, int u, int f, int lane) {
  return eb + ((ew + u) * 3 + f) * 512 + lane * 16;
}
__device__ __forceinline__ uint8_t* eb_u2(uint8_t* eb, int ew, int u, int g, int lane) {
  return eb + P_EPI_WARPS * 3 * 512 + ((ew + u) * 3 + g) * 256 + lane * 8;
}
__device__ __forceinline__ void p_epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * P_EPI_WARPS) : "memory");
}
__device__ __forceinline__ bool p_epi_bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.and.pred po, 1, %2, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(32 * P_EPI_WARPS)
      : "memory");
  return r != 0;
}

// Issue the copies of sub-chunk sc (columns 16 sc .. 16 sc + 15) of tile (m0, n0).
// A certifying pass (cert) needs no slices, and A_lo only to write the FP64 output.
// The first product's iterate A_1 = I + dt_0 is not stored (a1): it is formed from dt_0.
__device__ __forceinline__ void epi_prefetch(const GemmEpiParams& p, bool c1, bool cert, bool a1,
                                             int S, uint8_t* eb, int ew, int lane, int m0, int n0,
                                             int sc) {
  const float* Ahc = c1 ? p.A_hi[1] : p.A_hi[0];
  const float* Alc = c1 ? p.A_lo[1] : p.A_lo[0];
  const __half* dtp = c1 ? p.dt[0] : p.dt[1];
  const int j0 = m0 + 4 * lane;
#pragma unroll
  for (int u = 0; u < 1; ++u) {
    const int i = n0 + 16 * sc + ew + u;
    if (i >= p.n) continue;
    const int64_t idx = (int64_t)i * p.ld + j0;
    if (!a1) cp_async16(eb_f4(eb, ew, u, 0, lane), Ahc + idx);
    if ((!cert || p.Aout) && !a1) cp_async16(eb_f4(eb, ew, u, 1, lane), Alc + idx);
    cp_async16(eb_f4(eb, ew, u, 2, lane), p.L + idx);
    cp_async8(eb_u2(eb, ew, u, 0, lane), dtp + idx);
    if (cert) continue;
    const __half* Drow = p.Dcat + (int64_t)i * p.cat_ld + j0;
    for (int sl = 0; sl < S; ++sl)
      cp_async8(eb_u2(eb, ew, u, 1 + sl, lane), Drow + (int64_t)sl * p.ld);
  }
}

// Tile t of the CTA-pair kernel's order.  The column tiles are p.nw wide ones (p.bn
// columns) and then p.nnar narrow ones (p.bn - 32 columns, from column p.nw p.bn on),
// which together cover n with less padding than one width alone; the order takes
// every row block's wide tiles first, so that the round-robin over the clusters gives
// no cluster more than one wide tile above another and leaves the narrow tiles, with
// their shorter epilogues, for the last round.
struct PairTile {
  int tmc;   // row block (of CR x 128 rows)
  int n0;    // first column
  int w;     // width
};
__device__ __forceinline__ PairTile pair_tile(const GemmEpiParams& p, int t, int ntmc) {
  const int tw = ntmc * p.nw;
  if (t < tw) return {t / p.nw, (t % p.nw) * p.bn, p.bn};
  const int u = t - tw;
  return {u / p.nnar, p.nw * p.bn + (u % p.nnar) * (p.bn - 32), p.bn - 32};
}

// Copies of sub-chunk u of this tile, or, for u >= nsub, of sub-chunk u - nsub of the
// CTA's next tile t_next; then one commit group (empty when there is nothing to copy).
__device__ __forceinline__ void epi_prefetch_at(const GemmEpiParams& p, bool c1, bool cert,
                                                bool a1, int S, uint8_t* eb, int ew, int lane,
                                                bool work, int m0, int n0, int u, int nsub,
                                                int t_next, int ntiles, int ntmc, int crank,
                                                int cr) {
  if (u < nsub) {
    if (work) epi_prefetch(p, c1, cert, a1, S, eb, ew, lane, m0, n0, u);
  } else if (t_next < ntiles) {
    const PairTile nt = pair_tile(p, t_next, ntmc);
    const int tm = cr * nt.tmc + crank;
    if (tm < p.ntm) epi_prefetch(p, c1, cert, a1, S, eb, ew, lane, tm * BM, nt.n0, u - nsub);
  }
  cp_async_commit();
}

// Update this warp's column of sub-chunk sc from the staged inputs in eb and
// the accumulator chunk in Xs (which holds columns c0 .. c0 + 31, c0 = 32 (sc / 2)).
// Launch-constant factors of the staged epilogue (the scales of epilogue_columns),
// formed once per thread, and the tile's row parameters, loaded once per tile.
struct EpiConst {
  float lam;          // lambda 2^-sig 2^-scur
  float qs, iqs;      // 2^snew, 2^-snew
  float isc;          // 2^-scur
};
// The step's increment is dt = r G o R - (1 - r)(A - I) with r = 1 - rpow: the
// non-autonomous map at strength lambda r, from the residual at lambda and the identity
// lambda (P - A diag P) = R + Gap o A; r = 1 without the ramp.  Its scaled factors
// r 2^snew and (1 - r) 2^snew sit in shared memory (GemmSmemMisc::rq, oq).

// One column of a sub-chunk: the update of Eq. (dyn) in increment form for this lane's
// four rows, from the staged inputs in eb and the accumulator chunk in Xs (columns
// c0 .. c0 + 31, c0 = 32 (sc / 2)).  Specialised at compile time on
//   S      the Delta slices this product used (the diagonal partial uses as many),
//   MODE   0: a full step; 1: the first product, whose iterate A_1 = I + dt_0 is
//          formed from the increment (its A_lo is zero); 2: a certifying pass, which
//          forms only the residual norms of its iterate and, given p.Aout, writes the
//          iterate as the FP64 output A_hi + A_lo (used when the pass certifies it),
//   CHECK  the tile holds a diagonal element or rows beyond n (per-element masks).
// Leaves this lane's partial sums (|R|^2, |a|^2, the diagonal increment) in part3.
//
// Arithmetic, per element (j, i), with the scales of EpiConst folded in:
//   R    = L + lambda (X - A e_i - dt_{k-1} d_{k-1,i})        (the residual of A_k)
//   gap  = theta_i - theta_j as gs + gl: gs the float difference of the high parts,
//          gl its exact rounding error plus the difference of the low parts (an
//          unnormalised float-float pair: the quotient only needs gs + gl to float
//          accuracy, the remainder takes both parts)
//   dt_k = f16(R / gap) (packed conversion, scaled), L' = R - gap dt_k (exact feedback)
//   A'   = A + dt_k as the exact sum (two-sum) with the error added to A_lo (the pair
//          stays unnormalised: A_hi alone is read by the recursion, A_hi + A_lo only
//          by the output)
//   e    = sum_j Delta_ij dt_k,ji over this lane's rows in plain float: the slice
//          products are exact (11-bit significands) and these increments follow the
//          first one (summed in float-float by iteration 0), so float sums keep the
//          eigenvalues far inside their tolerance; tiles are summed in FP64 later.
template <int S, int MODE, bool CHECK>
__device__ __forceinline__ void epi_lean(const GemmEpiParams& p, const GemmSmemMisc* ms,
                                         const float* Xs, const uint8_t* eb, int ew, int lane,
                                         int m0, int n0, int sc, float& mx, const EpiConst& kc,
                                         const float4& thj_h, const float4& thj_l,
                                         float (&part3)[3]) {
  constexpr bool CERT = MODE == 2, A1 = MODE == 1;
  const int n = p.n, ld = p.ld;
  const int cl = 16 * sc + ew;
  const int i = n0 + cl;
  part3[0] = part3[1] = part3[2] = 0.f;
  if (i >= n) return;   // uniform across the warp
  const bool c1 = (ms->cur != 0);
  float* __restrict__ Ahn = c1 ? p.A_hi[0] : p.A_hi[1];
  float* __restrict__ Aln = c1 ? p.A_lo[0] : p.A_lo[1];
  __half* __restrict__ dtn_out = c1 ? p.dt[1] : p.dt[0];
  const int r0 = 4 * lane;
  const int j0 = m0 + r0;
  const int c0 = 32 * (sc >> 1);
  uint8_t* e8 = const_cast<uint8_t*>(eb);
  const float4 L4 = *reinterpret_cast<const float4*>(eb_f4(e8, ew, 0, 2, lane));
  const uint2 dtp = *reinterpret_cast<const uint2*>(eb_u2(e8, ew, 0, 0, lane));
  float4 ah4, al4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (A1) {
    ah4 = make_float4(h_at(dtp, 0) * kc.isc, h_at(dtp, 1) * kc.isc, h_at(dtp, 2) * kc.isc,
                      h_at(dtp, 3) * kc.isc);
  } else {
    ah4 = *reinterpret_cast<const float4*>(eb_f4(e8, ew, 0, 0, lane));
    if (!CERT || p.Aout) al4 = *reinterpret_cast<const float4*>(eb_f4(e8, ew, 0, 1, lane));
  }
  uint2 D[3] = {make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u)};
  if (!CERT) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) D[sl] = *reinterpret_cast<const uint2*>(eb_u2(e8, ew, 0, 1 + sl, lane));
  }
  const float4 x4 = *reinterpret_cast<const float4*>(Xs + (cl - c0) * BM + r0);
  const float e_i = ms->e[cl], dp_i = ms->dprev[cl];
  const float thh = ms->thh[cl], thl = ms->thl[cl];
  const float lam = kc.lam, iqs = kc.iqs;
  const float rq = ms->rq, oq = ms->oq;
  float r2 = 0.f, a2 = 0.f, es = 0.f;
  float4 oh, ol, oL;
  uint2 ob;
#pragma unroll
  for (int hp = 0; hp < 2; ++hp) {
    float R[2], gs[2], gl[2], q[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = 2 * hp + t, j = j0 + e;
      R[t] = gs[t] = gl[t] = q[t] = 0.f;
      if (!CHECK || (j != i && j < n)) {
        const float ah = f4(ah4, e);
        R[t] = f4(L4, e) + lam * (f4(x4, e) - ah * e_i - h_at(dtp, e) * dp_i);
        r2 = fmaf(R[t], R[t], r2);
        a2 = fmaf(ah, ah, a2);
        if (!CERT) {
          const float bh = f4(thj_h, e);
          float err;
          two_sum(thh, -bh, gs[t], err);
          gl[t] = err + (thl - f4(thj_l, e));
          // the increment is rounded to FP16 and the remainder keeps R - gap dt exactly,
          // so any reciprocal close to 1/gap serves; with the ramp the increment takes
          // the share r of the quotient and returns (1 - r) of A - I
          q[t] = fmaf(R[t] * rcp_approx(gs[t] + gl[t]), rq, -ah * oq);
        }
      }
    }
    if (!CERT) {
      const uint32_t w = f16x2_sat(q[0], q[1]);
      if (hp == 0) ob.x = w; else ob.y = w;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = 2 * hp + t, j = j0 + e;
      float nh = 0.f, nl = 0.f, Ln = 0.f;
      if (CHECK && j == i) {
        nh = 1.f;
        a2 += 1.f;
      } else if (!CERT && (!CHECK || j < n)) {
        const float dnew = h_at(ob, e) * iqs;
        Ln = fmaf(-gs[t], dnew, R[t]) - gl[t] * dnew;
        float err;
        two_sum(f4(ah4, e), dnew, nh, err);
        nl = f4(al4, e) + err;
        es = fmaf(h_at(D[0], e), dnew, es);
        if (S > 1) es = fmaf(h_at(D[1], e), dnew, es);
        if (S > 2) es = fmaf(h_at(D[2], e), dnew, es);
        mx = fmaxf(mx, fabsf(dnew));
      }
      f4set(oh, e, nh);
      f4set(ol, e, nl);
      f4set(oL, e, Ln);
    }
  }
  if (!CERT) {
    const int64_t idx = (int64_t)i * ld + j0;
    st4(Ahn + idx, oh);
    st4(Aln + idx, ol);
    st4(p.L + idx, oL);
    *reinterpret_cast<uint2*>(dtn_out + idx) = ob;
  } else if (p.Aout) {
    // the iterate as the FP64 output (as the output kernel forms it: hi + lo); rows
    // beyond n are not the caller's
    double v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = f2d_bits(f4(ah4, e)) + f2d_bits(f4(al4, e));
    double* o = p.Aout + (int64_t)i * p.ld_a + j0;
    if (!CHECK && p.aout_v8) {
      st_global_v8(o, __double2loint(v[0]), __double2hiint(v[0]), __double2loint(v[1]),
                   __double2hiint(v[1]), __double2loint(v[2]), __double2hiint(v[2]),
                   __double2loint(v[3]), __double2hiint(v[3]));
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (j0 + e < n) o[e] = v[e];
    }
  }
  part3[0] = r2; part3[1] = a2; part3[2] = es;
}

template <int S, int MODE>
__device__ __forceinline__ void epi_lean_tile(bool check, const GemmEpiParams& p,
                                              const GemmSmemMisc* ms, const float* Xs,
                                              const uint8_t* eb, int ew, int lane, int m0, int n0,
                                              int sc, float& mx, const EpiConst& kc,
                                              const float4& thj_h, const float4& thj_l,
                                              float (&part3)[3]) {
  if (check) epi_lean<S, MODE, true>(p, ms, Xs, eb, ew, lane, m0, n0, sc, mx, kc, thj_h, thj_l, part3);
  else epi_lean<S, MODE, false>(p, ms, Xs, eb, ew, lane, m0, n0, sc, mx, kc, thj_h, thj_l, part3);
}

// Dispatch on the launch's slice count and mode (uniform) and the tile's masks.
__device__ __forceinline__ void epi_lean_any(int S, int mode, bool check, const GemmEpiParams& p,
                                             const GemmSmemMisc* ms, const float* Xs,
                                             const uint8_t* eb, int ew, int lane, int m0, int n0,
                                             int sc, float& mx, const EpiConst& kc,
                                             const float4& thj_h, const float4& thj_l,
                                             float (&part3)[3]) {
#define DPT_EPI_CASE(SS, MM) \
  epi_lean_tile<SS, MM>(check, p, ms, Xs, eb, ew, lane, m0, n0, sc, mx, kc, thj_h, thj_l, part3)
  // the single solve slices Delta into at most two FP16 slices (solve_full_mixed_real)
  if (mode == 2) {          // certifying passes read no slices
    DPT_EPI_CASE(1, 2);
  } else if (mode == 1) {
    if (S == 1) DPT_EPI_CASE(1, 1);
    else DPT_EPI_CASE(2, 1);
  } else {
    if (S == 1) DPT_EPI_CASE(1, 0);
    else DPT_EPI_CASE(2, 0);
  }
#undef DPT_EPI_CASE
}

// Warp sums of two columns' lane partials (|R|^2, |a|^2, the diagonal increment) with
// one transposing exchange: after the first step lanes 0-15 carry column a and lanes
// 16-31 column b, so the remaining four steps serve both.  On return lane 0 holds the
// sums of a, lane 16 those of b.
__device__ __forceinline__ void warp_sum3x2(float (&a)[3], const float (&b)[3], int lane) {
  const bool lo = lane < 16;
  float k[3];
#pragma unroll
  for (int q = 0; q < 3; ++q)
    k[q] = (lo ? a[q] : b[q]) + __shfl_xor_sync(0xffffffffu, lo ? b[q] : a[q], 16);
#pragma unroll
  for (int off = 8; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < 3; ++q) k[q] += __shfl_xor_sync(0xffffffffu, k[q], off);
#pragma unroll
  for (int q = 0; q < 3; ++q) a[q] = k[q];
}

// ---------------------------------------------------------------------------
// CTA-pair form of the product kernel (tcgen05 cta_group::2).  The two CTAs of a
// cluster compute one 256 x bn output tile: each loads its own 128 rows of the A
// operand (Delta slices) and half of the B operand (bn/2 increment columns) into
// its own shared memory; the MMA, issued by the pair's leader (cluster rank 0),
// reads both halves of both operands and leaves each CTA's 128 rows of the
// accumulator in that CTA's tensor memory.  Per SM a K-block stage is then A + B/2
// instead of A + B, so the same shared memory holds six stages instead of four and
// each SM fetches a third fewer operand bytes per flop.  Each CTA runs the fused
// epilogue on its own rows; the arithmetic per element, the slice order and the K
// rotation are those of k_gemm_epi.
// Barriers: the leader's full[s] collects the transaction bytes of both CTAs'
// loads (the leader posts the expectation for both); the MMA commits arrive on
// empty[s] and acc_full[b] of both CTAs (multicast); both epilogues arrive on the
// leader's acc_empty[b] (count 2).  Every thread of both CTAs reaches the final
// cluster barrier, also when a bounded wait has given up.
//
// QUAD: clusters of four CTAs, two pairs stacked along M (a 512 x bn tile), which
// share each B half through TMA multicast: cluster ranks 0 and 1 load B halves 0 and
// 1 into themselves and into ranks 2 and 3, so a stage costs an SM its A tile plus a
// quarter of B in L2 reads instead of a half.  Each destination's copy completes on
// full[s] of its own pair's leader, which therefore expects the same bytes as in a
// lone pair.  Each MMA commit releases the slot in all four CTAs (empty[s] count 2:
// a slot holds data for both pairs' products).
// ---------------------------------------------------------------------------
template <bool QUAD, bool MERGED>
__device__ __forceinline__ void gemm_epi_pair_body(const CUtensorMap& tmA, const CUtensorMap& tmB0,
                                                   const CUtensorMap& tmB1,
                                                   const CUtensorMap& tmB0n,
                                                   const CUtensorMap& tmB1n,
                                                   const GemmEpiParams& p) {
  extern __shared__ uint8_t smem_raw[];
  IterState* st = p.st;
  // read before any cluster barrier; nothing changes it during the launch, so every
  // CTA of a cluster takes the same branch
  if (*((volatile int*)&st->status) != ST_RUNNING) return;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // [operand ring | (second epilogue input buffer) | epilogue input buffer at P_RREG |
  //  accumulator staging | barriers and per-launch constants]
  float* Xs = reinterpret_cast<float*>(smem + P_RREG + EB_BYTES);
  GemmSmemMisc* ms = (GemmSmemMisc*)(smem + P_RREG + EB_BYTES + SMEM_X);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int CR = QUAD ? 4 : 2;       // CTAs per cluster, stacked along M
  const uint32_t crank = cluster_ctarank();
  const uint32_t rank = crank & 1u;      // rank within the pair
  const uint32_t lead = crank & ~1u;     // cluster rank of the pair's leader
  const int bn = p.bn, bh = bn / 2;   // the wide tiles (the ring's stage size)
  const int ntmc = (p.n + CR * BM - 1) / (CR * BM);
  const int ntiles = (p.nw + p.nnar) * ntmc;
  const int pair = blockIdx.x / CR, npairs = gridDim.x / CR;   // clusters

  if (threadIdx.x == 0) {
    ms->k = st->k;
    ms->slices = st->slices;
    ms->certify = st->certify;
    ms->cur = st->cur;
    ms->sig = st->sig;
    ms->scur = st->sexp[st->cur ^ 1];
    ms->snew = st->sexp[st->cur];
    ms->rpow = (float)st->ramp_pow;
    ms->rq = (1.f - ms->rpow) * exp2i(ms->snew);
    ms->oq = ms->rpow * exp2i(ms->snew);
    const uint32_t nempty = QUAD ? 2u : 1u;
    for (int s = 0; s < MAX_STAGES; ++s) { mbar_init(&ms->full[s], 1); mbar_init(&ms->empty[s], nempty); }
    for (int b = 0; b < NACC; ++b) { mbar_init(&ms->acc_full[b], 1); mbar_init(&ms->acc_empty[b], 2); }
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc_pair(&ms->tmem_base, NACC * BN);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync();      // every CTA's barriers initialised and each pair's TMEM allocated
  tc_fence_after();
  const uint32_t tmem = ms->tmem_base;
  const int S = ms->slices;
  // two-slice stages (MERGED: two slices, not the first product): a stage holds both
  // slices' A tiles of one K-block and its B half
  constexpr bool merged = MERGED;
  const int na = merged ? 2 : 1;
  const int kb_per_slice = p.ld / BK;
  const int nk = merged ? kb_per_slice : S * kb_per_slice;
  const uint32_t b_bytes = (uint32_t)bh * BK * 2;
  const uint32_t stage_bytes = (uint32_t)(na * A_TILE) + b_bytes;   // multiple of 1024
  // with one buffer of epilogue inputs the ring takes the whole region
  const uint32_t ring_bytes = (uint32_t)P_RREG - (merged ? 0u : (uint32_t)EB_BYTES);
  const int nst = min(MAX_STAGES, (int)(ring_bytes / stage_bytes));
  // the epilogue input buffers: the second for one slice only; with two slices both
  // names are the one buffer
  uint8_t* EB = smem + P_RREG;
  uint8_t* EB2 = merged ? EB : smem + ring_bytes;
  const CUtensorMap* tmB = (ms->cur == 1) ? &tmB0 : &tmB1;
  const CUtensorMap* tmBn = (ms->cur == 1) ? &tmB0n : &tmB1n;   // boxes of bn/2 - 16 rows
  unsigned* tflag = &st->timeout;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (every CTA): A completes on the leader's full[s] ----
    prefetch_tmap(&tmA);
    prefetch_tmap(tmB);
    if (p.nnar > 0) prefetch_tmap(tmBn);
    const uint32_t full_leader = mapa_shared(&ms->full[0], lead);
    uint32_t it = 0;
    bool alive = true;
    for (int t = pair; t < ntiles && alive; t += npairs) {
      const PairTile pt = pair_tile(p, t, ntmc);
      const int m0 = pt.tmc * CR * BM + (int)crank * BM, n0 = pt.n0;
      // a narrow tile loads B halves of its own width (a smaller stage)
      const bool wide = pt.w == bn;
      const int bh_t = pt.w / 2;
      const CUtensorMap* tb = wide ? tmB : tmBn;
      const uint32_t tx = 2u * ((uint32_t)(na * A_TILE) + (uint32_t)bh_t * BK * 2);
      const int kb_last = min(kb_per_slice - 1, (n0 + pt.w - 1) / BK);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % nst;
        const uint32_t ph = (it / nst) & 1;
        if (!mbar_wait(&ms->empty[s], ph ^ 1, tflag)) { alive = false; break; }
        if (rank == 0) mbar_arrive_expect_tx(&ms->full[s], tx);
        // small slices first, the tile's diagonal K-blocks last (see k_gemm_epi); with
        // both slices in a stage, slice 1 before slice 0 within each K-block
        const int kb = (kb_last + 1 + q % kb_per_slice) % kb_per_slice;
        uint8_t* slot = smem + (size_t)s * stage_bytes;
        const uint32_t fb = full_leader + (uint32_t)s * 8u;
        if (merged) {
          tma_load_2d_pair(slot, &tmA, fb, p.ld + kb * BK, m0);
          tma_load_2d_pair(slot + A_TILE, &tmA, fb, kb * BK, m0);
        } else {
          const int sl = S - 1 - q / kb_per_slice;
          tma_load_2d_pair(slot, &tmA, fb, sl * p.ld + kb * BK, m0);
        }
        uint8_t* bslot = slot + na * A_TILE;
        if (!QUAD)
          tma_load_2d_pair(bslot, tb, fb, kb * BK, n0 + (int)rank * bh_t);
        else if (crank < 2)
          tma_load_2d_pair_multicast(bslot, tb, fb, kb * BK, n0 + (int)rank * bh_t,
                                     (uint16_t)((1u << crank) | (4u << crank)));
      }
    }
    // the MMA's last commits have arrived on this CTA's empty barriers
    for (uint32_t u = (it > (uint32_t)nst ? it - nst : 0); u < it; ++u)
      mbar_wait_quiet(&ms->empty[u % nst], (u / nst) & 1, kTailWaitNs);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---- MMA issuer (pair leaders only) ----
    const uint32_t idesc_w = idesc_f16_f32(2 * BM, bn);
    const uint32_t idesc_n = idesc_f16_f32(2 * BM, bn - 32);
    uint32_t it = 0;
    int lt = 0;
    bool alive = true;
    for (int t = pair; t < ntiles && alive; t += npairs, ++lt) {
      const uint32_t idesc = (t < ntmc * p.nw) ? idesc_w : idesc_n;   // see pair_tile
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      if (!mbar_wait(&ms->acc_empty[b], (use & 1) ^ 1, tflag)) break;
      tc_fence_after();
      const uint32_t dacc = tmem + (uint32_t)(b * BN);
      for (int q = 0; q < nk; ++q, ++it) {
        const int s = it % nst;
        const uint32_t ph = (it / nst) & 1;
        if (!mbar_wait(&ms->full[s], ph, tflag)) { alive = false; break; }
        tc_fence_after();
        uint8_t* slot = smem + (size_t)s * stage_bytes;
        const uint64_t da = smem_desc_sw128(slot);
        const uint64_t db = smem_desc_sw128(slot + na * A_TILE);
#pragma unroll
        for (int kk = 0; kk < BK / UK; ++kk)
          umma_f16_pair(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                         (q > 0 || kk > 0) ? 1u : 0u);
        if (merged) {
          const uint64_t da0 = smem_desc_sw128(slot + A_TILE);
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk)
            umma_f16_pair(dacc, da0 + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, 1u);
        }
        umma_commit_pair(&ms->empty[s], (uint16_t)(QUAD ? 0xF : 0x3));
      }
      umma_commit_pair(&ms->acc_full[b], (uint16_t)(3u << lead));
    }
    // both epilogues have released the last accumulators: their arrivals on this
    // CTA's acc_empty have landed before it can exit
    for (int u = (lt > NACC ? lt - NACC : 0); u < lt; ++u)
      mbar_wait_quiet(&ms->acc_empty[u & 1], (uint32_t)((u >> 1) & 1), kTailWaitNs);
  } else if (warp >= 2) {
    // ---- epilogue (both CTAs, each on its own 128 rows) ----
    const int ew = warp - 2;
    const int qd = warp & 3;
    const int q4 = ew >> 2;                // which 8 of a chunk's 32 columns this warp stages
    const int et = threadIdx.x - 64;
    const uint32_t acc_empty_leader = mapa_shared(&ms->acc_empty[0], lead);
    const bool c1 = (ms->cur != 0);
    const bool cert = ms->certify != 0;
    const bool a1 = ms->k == 1;            // A_1 = I + dt_0 is formed from dt_0
    const int mode = cert ? 2 : (a1 ? 1 : 0);
    const float cs = exp2i(ms->scur), cd = exp2i(ms->sig);
    EpiConst kc;
    kc.lam = (p.lam * exp2i(-ms->sig)) * exp2i(-ms->scur);
    kc.qs = exp2i(ms->snew);
    kc.iqs = exp2i(-ms->snew);
    kc.isc = exp2i(-ms->scur);
    float mx = 0.f;
    int lt = 0;
    // The inputs of sub-chunk sc sit in buffer sc & 1 (one slice) or in the only
    // buffer (two slices), copied two sub-chunks ahead (one slice: into the buffer just
    // updated) or one ahead (two slices: after the update, into the same buffer; each
    // lane copies and reads only its own slots).  The first tile's first sub-chunks,
    // while its products run:
    const int ahead = merged ? 1 : 2;
    for (int u = 0; u < ahead; ++u)   // the first tile's (as the "next" of none)
      epi_prefetch_at(p, c1, cert, a1, S, (u & 1) ? EB2 : EB, ew, lane, false, 0, 0, u, 0,
                      pair, ntiles, ntmc, (int)crank, CR);
    for (int t = pair; t < ntiles; t += npairs, ++lt) {
      const PairTile pt = pair_tile(p, t, ntmc);
      const int tm = CR * pt.tmc + (int)crank;
      const int m0 = tm * BM, n0 = pt.n0;
      const bool work = tm < p.ntm;        // rows of a pair tile beyond the padded matrix
      // the tile's width (see pair_tile), a multiple of 32
      const int w = bn - ((t >= ntmc * p.nw) ? 32 : 0);
      const int nsub = w / 16;             // sub-chunks of the tile
      const int b = lt & 1;
      const uint32_t use = (uint32_t)(lt >> 1);
      // per-element masks only where the tile holds a diagonal element or rows beyond n
      const bool check = (m0 + BM > p.n) || (n0 < m0 + BM && m0 < n0 + w);
      // theta_j of this lane's four rows (padded arrays: rows up to ld exist)
      const float4 thj_h = work ? ld4(p.th_hi + m0 + 4 * lane) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 thj_l = work ? ld4(p.th_lo + m0 + 4 * lane) : make_float4(0.f, 0.f, 0.f, 0.f);
      p_epi_bar();
      if (et < w) {
        const int i = n0 + et;
        const bool v = i < p.n;
        ms->e[et] = v ? (p.e_col[i] * cd) * cs : 0.f;   // e_k 2^sig 2^scur
        ms->dprev[et] = v ? p.dprev_col[i] * cd : 0.f;
        ms->thh[et] = v ? p.th_hi[i] : 0.f;
        ms->thl[et] = v ? p.th_lo[i] : 0.f;
      }
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&ms->acc_full[b], use & 1, tflag));
      tc_fence_after();
      const uint32_t src = tmem + (uint32_t)(b * BN) + ((uint32_t)(qd * 32) << 16);
      bool all_ok = true;
#pragma unroll 1
      for (int c0 = 0; c0 < w; c0 += XCH) {
        if (c0 > 0) p_epi_bar();
        if (ok) {
          float x[8];
          const int cc = q4 * 8;
          tmem_ld_x8(src + (uint32_t)(c0 + cc), x);
#pragma unroll
          for (int c = 0; c < 8; ++c) Xs[(cc + c) * BM + qd * 32 + lane] = x[c];
        }
        if (c0 + XCH == w) tc_fence_before();
        all_ok = p_epi_bar_and(ok);
        if (c0 + XCH == w && et == 0) {
          if (rank == 0) mbar_arrive(&ms->acc_empty[b]);
          else mbar_arrive_remote(acc_empty_leader + (uint32_t)b * 8u);
        }
        if (!all_ok) break;
        float pa[3] = {0.f, 0.f, 0.f}, pb[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int sc = c0 / 16 + h;
          // copies of the next sub-chunk (this tile's, or the next tile's first) into
          // the other buffer before this one is updated, or, with one buffer, into the
          // same buffer after it (each lane copies and reads only its own slots)
          // this lane's copies of sub-chunk sc have landed
          if (merged) cp_async_wait<0>();
          else cp_async_wait<1>();
          uint8_t* eb = (sc & 1) ? EB2 : EB;
          if (work) {
            float cur[3];
            epi_lean_any(S, mode, check, p, ms, Xs, eb, ew, lane, m0, n0, sc, mx, kc, thj_h,
                         thj_l, cur);
#pragma unroll
            for (int q = 0; q < 3; ++q) {   // registers, no indexing by h
              if (h == 0) pa[q] = cur[q];
              else pb[q] = cur[q];
            }
          }
          epi_prefetch_at(p, c1, cert, a1, S, eb, ew, lane, work, m0, n0, sc + ahead, nsub,
                          t + npairs, ntiles, ntmc, (int)crank, CR);
        }
        if (work) {
          // this warp's two columns of the chunk, reduced together
          warp_sum3x2(pa, pb, lane);
          const int i = n0 + c0 + 16 * (lane >> 4) + ew;
          if ((lane & 15) == 0 && i < p.n) {
            const int64_t ld = p.ld;
            p.part[((int64_t)0 * p.ntm + tm) * ld + i] = pa[0];
            p.part[((int64_t)1 * p.ntm + tm) * ld + i] = pa[1];
            if (!cert) {
              // the diagonal increment in plain float: its low part is zero
              p.part[((int64_t)2 * p.ntm + tm) * ld + i] = pa[2];
              p.part[((int64_t)3 * p.ntm + tm) * ld + i] = 0.f;
            }
          }
        }
      }
      if (!all_ok) break;
    }
    cp_async_wait<0>();                    // no copy into shared memory outlives the walk
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.f) atomicMax(&p.st->dmax_bits, __float_as_uint(mx));
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();      // no MMA, load or remote arrival of the cluster is still in flight
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, NACC * BN);
  }
}

// Which body runs: two-slice stages for a two-slice product after the first.  The
// tensor core's FP32 accumulation drops the bits below its running sum at every step,
// so interleaving the small slice with the large one (both slices per K-block) adds
// that loss at the scale of the full partial sums: about twice the accumulator error
// of the per-slice order (measured on the GB300 at n = 256 .. 2048, and in a NumPy model
// of the truncating accumulation).  That error scales with the product's increment,
// and the first one, dt_0, is the largest by the map's contraction, so the first
// product keeps the per-slice order (the increment tile loaded once per slice) and
// the accuracy of the result is that of the per-slice order.  The decision reads
// fields the preceding control kernel set (uniform over the launch).  Each case runs
// a body specialised for it: one body with a runtime flag ran the one-slice products
// 8 % slower.
__device__ __forceinline__ bool two_slice_stages(const IterState* st) {
  return *((const volatile int*)&st->slices) == 2 && *((const volatile int*)&st->k) != 1;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P_NTHREADS, 1)
k_gemm_epi_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
                const __grid_constant__ CUtensorMap tmB1,
                const __grid_constant__ CUtensorMap tmB0n,
                const __grid_constant__ CUtensorMap tmB1n, const GemmEpiParams p) {
  if (two_slice_stages(p.st)) gemm_epi_pair_body<false, true>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
  else gemm_epi_pair_body<false, false>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
}

__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(P_NTHREADS, 1)
k_gemm_epi_quad(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
                const __grid_constant__ CUtensorMap tmB1,
                const __grid_constant__ CUtensorMap tmB0n,
                const __grid_constant__ CUtensorMap tmB1n, const GemmEpiParams p) {
  if (two_slice_stages(p.st)) gemm_epi_pair_body<true, true>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
  else gemm_epi_pair_body<true, false>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
}

// ---------------------------------------------------------------------------
// Output: A (float-float -> FP64) and E of the returned iterate.
// ---------------------------------------------------------------------------
// Output: tiles of 128 rows x 32 columns, strided over a grid of one wave; thread j
// owns row j of the tile and issues the loads of eight columns before their stores.
__global__ void __launch_bounds__(128) k_finalize(int n, int ld, const float* __restrict__ Ahi0,
                                                  const float* __restrict__ Alo0,
                                                  const float* __restrict__ Ahi1,
                                                  const float* __restrict__ Alo1,
                                                  const __half* __restrict__ dt0,
                                                  double* __restrict__ Aout, int64_t ld_a,
                                                  const IterState* st, int only_done) {
  if (only_done && st->status == ST_RUNNING) return;   // not the final iterate yet
  if (only_done && st->out_done) return;   // written by the certifying pass
  const int k = st->k;
  const float isc = exp2i(-st->sexp[0]);
  const float* __restrict__ hi = (st->cur == 0) ? Ahi0 : Ahi1;
  const float* __restrict__ lo = (st->cur == 0) ? Alo0 : Alo1;
  // tiles of 128 rows x 32 columns, strided over one wave of blocks (the launch
  // that finds nothing to do then ends at once)
  const int nrt = (n + 127) / 128, ntiles = nrt * ((n + 31) / 32);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int j = (t % nrt) * 128 + threadIdx.x;
    if (j >= n) continue;
    const int i0 = (t / nrt) * 32, i1 = min(n, i0 + 32);
    if (k == 0) {
      for (int i = i0; i < i1; ++i) Aout[(int64_t)i * ld_a + j] = (i == j) ? 1.0 : 0.0;
      continue;
    }
    if (k == 1) {   // A_1 = I + dt_0 (iteration 0 stores only the increment)
      for (int i = i0; i < i1; ++i)
        Aout[(int64_t)i * ld_a + j] =
            (i == j) ? 1.0 : f2d_bits(__half2float(dt0[(int64_t)i * ld + j]) * isc);
      continue;
    }
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
      float h[8], l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        h[u] = hi[(int64_t)(i + u) * ld + j];
        l[u] = lo[(int64_t)(i + u) * ld + j];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        Aout[(int64_t)(i + u) * ld_a + j] = f2d_bits(h[u]) + f2d_bits(l[u]);
    }
    for (; i < i1; ++i)
      Aout[(int64_t)i * ld_a + j] =
          f2d_bits(hi[(int64_t)i * ld + j]) + f2d_bits(lo[(int64_t)i * ld + j]);
  }
}

// Checks of a device-resident theta: finite, pairwise distinct (Sec. II.B: simple
// unperturbed levels), and max |theta| into the state (the residual scale), by
// atomicMax on the bits of a non-negative double.  Grid (256-blocks of i, 32-chunks of
// j), upper triangle only: each block stages its 32 keys of theta_j in shared memory
// and thread i compares theta_i with those j > i (many short blocks: the comparisons
// spread over every SM).  The block whose chunk starts at the i-block's first index
// also tests theta_i for finiteness, takes max |theta_i| and, when hi is given, splits
// theta into float-float (hi, lo) as k_theta_ff does (one launch less for a device
// theta).
// (eq_key: 64-bit integer equality keys of finite doubles, dpt_device.cuh)
constexpr int kThetaChunk = 32;
__global__ void __launch_bounds__(256) k_check_theta(int n, const double* __restrict__ th,
                                                     IterState* st, float* __restrict__ hi,
                                                     float* __restrict__ lo) {
  const int ib = blockIdx.x * 256, j0 = blockIdx.y * kThetaChunk;
  if (j0 + kThetaChunk <= ib) return;   // every j of the chunk is below every i
  __shared__ unsigned long long tj[kThetaChunk];
  const int i = ib + threadIdx.x;
  // entries past n hold a pattern no finite value has
  if (threadIdx.x < kThetaChunk)
    tj[threadIdx.x] = (j0 + (int)threadIdx.x < n) ? eq_key(th[j0 + threadIdx.x]) : ~0ull;
  __syncthreads();
  const bool lead = (j0 == ib);
  double amax = 0.0;
  if (i < n) {
    const double ti = th[i];
    if (hi && lead) {
      const float h = (float)ti;
      hi[i] = h;
      lo[i] = (float)(ti - (double)h);
    }
    if (!finite_bits(ti)) {
      if (lead) atomicCAS(&st->status, ST_RUNNING, ST_BADINPUT);
    } else {
      if (lead) amax = fabs(ti);
      const unsigned long long ki = eq_key(ti);
      // only the j > i of the chunk
      const int q0 = max(0, i + 1 - j0);
      bool dup = false;
#pragma unroll 8
      for (int q = 0; q < kThetaChunk; ++q) dup |= (q >= q0) & (tj[q] == ki);
      if (dup) atomicCAS(&st->status, ST_RUNNING, ST_DEGENERATE);
    }
  }
  if (!lead) return;
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0 && amax > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&st->theta_max),
              (unsigned long long)__double_as_longlong(amax));
}

__global__ void k_theta_ff(int n, const double* __restrict__ th, float* __restrict__ hi,
                           float* __restrict__ lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = (float)th[i];
  hi[i] = h;
  lo[i] = (float)(th[i] - (double)h);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int mixed_smem_bytes() { return SMEM_BYTES; }
// Tile width for an n x n product on nsm SMs.  Every CTA of the persistent kernel
// takes tiles round-robin, so the launch lasts ceil(tiles / nsm) tile times; a
// tile's time grows with its width plus a width-independent part (the A operand's
// share of the TMA traffic and the epilogue's fixed work, about 64 columns' worth).
// The width (a multiple of 32, at most 256) minimises that estimate, so that the
// last wave is not left mostly idle (n = 4096 on 152 SMs: 224 -> 608 tiles = 4
// full waves, against 512 tiles = 3.4 waves at 256).
int mixed_tile_n(int n, int nsm) {
  const int ntm = (n + BM - 1) / BM;
  int best = BN;
  long long best_cost = -1;
  for (int w = BN; w >= 64; w -= 32) {
    const long long tiles = (long long)ntm * ((n + w - 1) / w);
    const long long waves = (tiles + nsm - 1) / nsm;
    const long long cost = waves * (w + 64);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = w; }
  }
  return best;
}

// SM count of the current device, queried once (a thread-safe static initialisation:
// several host threads launch solves); 0 if the query failed
static int device_sms() {
  static const int v = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    return n;
  }();
  return v;
}

cudaError_t launch_delta_scales(const double* delta, int64_t ld_in, int n, const float* th_hi,
                                const float* th_lo, double lam, int en, const double* start,
                                int64_t ld_s, double* sinv, IterState* st, cudaStream_t s) {
  (void)lam;   // read from the state
  if (!start) {
    // one wave of resident blocks (the items are strided over it)
    static const int per_sm = [] {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_delta_scales_rows, 256, 0) !=
          cudaSuccess)
        occ = 1;
      return std::max(1, std::min(occ, 6));
    }();
    const int nsm = device_sms();
    if (nsm <= 0) return cudaErrorInvalidDevice;
    const int nrb = (n + 255) / 256, ncb = (n + kScaleCols - 1) / kScaleCols;
    const long long items = (long long)nrb * ncb;
    if (items > INT_MAX) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(items, (long long)per_sm * nsm);
    k_delta_scales_rows<<<grid, 256, 0, s>>>(delta, ld_in, n, nrb, (int)items, th_hi, th_lo, en,
                                             st);
    return cudaGetLastError();
  }
  // from a start: one block per column
  k_delta_scales<<<n, 256, 0, s>>>(delta, ld_in, n, th_hi, th_lo, en, start, ld_s, sinv, st);
  return cudaGetLastError();
}

cudaError_t launch_prep_delta(const double* delta, int64_t ld_in, int n, int ld, int en, int nsl,
                              __half* Dcat, IterState* st, cudaStream_t s) {
  dim3 grid(ld / 64, (n + 31) / 32), block(32, 8);     // ld is a multiple of 128
  switch (nsl) {
    case 1: k_prep_delta<1><<<grid, block, 0, s>>>(delta, ld_in, n, ld, en, Dcat, st); break;
    case 2: k_prep_delta<2><<<grid, block, 0, s>>>(delta, ld_in, n, ld, en, Dcat, st); break;
    case 3: k_prep_delta<3><<<grid, block, 0, s>>>(delta, ld_in, n, ld, en, Dcat, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_check_theta(int n, const double* th, IterState* st, cudaStream_t s, float* hi,
                               float* lo) {
  k_check_theta<<<dim3((n + 255) / 256, (n + kThetaChunk - 1) / kThetaChunk), 256, 0, s>>>(
      n, th, st, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_theta_ff(int n, const double* th, float* hi, float* lo, cudaStream_t s) {
  k_theta_ff<<<(n + 255) / 256, 256, 0, s>>>(n, th, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_iter0(const double* delta, int64_t ld_in, const float* th_hi,
                         const float* th_lo, double lam, int n, int ld, int en, int nsl,
                         const __half* Dcat, __half* dt0, float* L, double* d, float* part,
                         float* rowpart, const double* start, int64_t ld_s, const double* sinv,
                         IterState* st, cudaStream_t s) {
  if (nsl < 1 || nsl > NSLICE) return cudaErrorInvalidValue;
  const int ntm = (n + IT0 - 1) / IT0, ntn = (n + kIter0Cols - 1) / kIter0Cols;
  const float lh = (float)lam;
  const float ll = (float)(lam - (double)lh);
  const dim3 grid(ntn, ntm);
#define DPT_IT0(NS, SS)                                                                     \
  k_iter0<NS, SS><<<grid, 256, 0, s>>>(delta, ld_in, th_hi, th_lo, lh, ll, n, ld, ntm, en, \
                                       Dcat, dt0, L, d, part, rowpart, start, ld_s, sinv, st)
  if (start) {
    switch (nsl) {
      case 1: DPT_IT0(1, true); break;
      case 2: DPT_IT0(2, true); break;
      default: DPT_IT0(3, true); break;
    }
  } else {
    switch (nsl) {
      case 1: DPT_IT0(1, false); break;
      case 2: DPT_IT0(2, false); break;
      default: DPT_IT0(3, false); break;
    }
  }
#undef DPT_IT0
  return cudaGetLastError();
}

cudaError_t launch_iter0_pairs(const CUtensorMap& tmD, const float* th_hi, const float* th_lo,
                               double lam, int n, int ld, int en, int nsl, __half* Dcat,
                               __half* dt0, float* L, double* d, float* part, float* rowpart,
                               IterState* st, cudaStream_t s) {
  if (nsl < 1 || nsl > NSLICE || ld % F0T) return cudaErrorInvalidValue;
  const cudaError_t ea = mixed_set_attributes();
  if (ea != cudaSuccess) return ea;
  const int nt = ld / F0T;
  const long long units = (long long)nt * (nt + 1) / 2;
  const float lh = (float)lam;
  const float ll = (float)(lam - (double)lh);
#define DPT_IT0P(NS)                                                                         \
  k_iter0_pairs<NS><<<(unsigned)units, 128, F0_SMEM, s>>>(tmD, th_hi, th_lo, lh, ll, n, ld, nt, \
                                                          en, Dcat, dt0, L, d, part, rowpart, st)
  switch (nsl) {
    case 1: DPT_IT0P(1); break;
    case 2: DPT_IT0P(2); break;
    default: DPT_IT0P(3); break;
  }
#undef DPT_IT0P
  return cudaGetLastError();
}

cudaError_t launch_ctrl(int n, int ld, const float* part, const float* rowpart,
                        const double* theta, double* d, double* E, float* e_col,
                        float* dprev_col, IterState* st, cudaStream_t s, int nslot, int hilo,
                        int first_step) {
  // column partials: one per 128-row tile of the product, or nslot of them (the fused
  // iteration 0's 64-row slots); row partials: one per block of kIter0Cols columns of
  // iteration 0
  const int ntm = nslot > 0 ? nslot : (n + BM - 1) / BM;
  const int ntn = (n + kIter0Cols - 1) / kIter0Cols;
  k_ctrl<<<(n + 31) / 32, 256, 0, s>>>(n, ld, ntm, ntn, part, rowpart, theta, d, E, e_col,
                                       dprev_col, st, hilo, first_step);
  return cudaGetLastError();
}

cudaError_t mixed_set_attributes() {
  // once per device (the attribute stays set for the context)
  static std::atomic<bool> done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load()) return cudaSuccess;
  e = cudaFuncSetAttribute(k_gemm_epi, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_epi_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           P_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_epi_quad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           P_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_iter0_pairs<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, F0_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_iter0_pairs<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, F0_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_iter0_pairs<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, F0_SMEM);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(true);
  return e;
}

// Clusters of `ctas` (2: one CTA pair; 4: two pairs sharing B) that can be resident
// at once (0: that form cannot run; call mixed_set_attributes first).  The kernels
// declare their cluster shape at compile time, so the query passes none.
int mixed_pair_clusters(int ctas) {
  static int cached[64][2];
  static bool known[64][2];
  int dev = 0;
  if ((ctas != 2 && ctas != 4) || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  const int q = ctas == 4;
  if (known[dev][q]) return cached[dev][q];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(P_NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = P_SMEM_BYTES;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  int n = 0;
  const cudaError_t e = q ? cudaOccupancyMaxActiveClusters(&n, k_gemm_epi_quad, &cfg)
                          : cudaOccupancyMaxActiveClusters(&n, k_gemm_epi_pair, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached[dev][q] = n;
  known[dev][q] = true;
  return n;
}

// Tile width for the pair forms: as mixed_tile_n with (ctas x 128)-row tiles over
// `nclusters` clusters; half of the width (a multiple of 16) goes to each CTA of a pair.
int mixed_pair_tile_n(int n, int nclusters, int ctas) {
  const int ntmc = (n + ctas * BM - 1) / (ctas * BM);
  int best = BN;
  long long best_cost = -1;
  for (int w = BN; w >= 64; w -= 32) {
    const long long tiles = (long long)ntmc * ((n + w - 1) / w);
    const long long waves = (tiles + nclusters - 1) / nclusters;
    const long long cost = waves * (w + 64);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = w; }
  }
  return best;
}

// The split of the columns into p.nw tiles of bn and nnar tiles of bn - 32 (see
// pair_tile): as many narrow tiles as the padding of ceil(n / bn) wide ones leaves
// room for, where the round-robin over the clusters then ends sooner (the same cost
// model as mixed_pair_tile_n: a tile costs its width plus 64).
void mixed_pair_split(int n, int bn, int nclusters, int ctas, int* nw, int* nnar) {
  const int ntn = (n + bn - 1) / bn;
  const int ntmc = (n + ctas * BM - 1) / (ctas * BM);
  *nw = ntn;
  *nnar = 0;
  if (bn - 32 < 64 || nclusters < 1) return;
  const int bmax = std::min(ntn - 1, (ntn * bn - n) / 32);
  long long best = -1;
  for (int b = 0; b <= bmax; ++b) {
    const int a = ntn - b;
    const long long wide = (long long)ntmc * a, all = (long long)ntmc * ntn;
    // the busiest cluster: the first (all % nclusters) clusters take one tile more;
    // wide tiles come first in the order
    long long worst = 0;
    for (int c = 0; c < nclusters && c < all; ++c) {
      const long long cnt = (all - c + nclusters - 1) / nclusters;   // tiles c, c + ncl, ..
      const long long nwide = wide > c ? std::min(cnt, (wide - c + nclusters - 1) / nclusters) : 0;
      worst = std::max(worst, nwide * (bn + 64) + (cnt - nwide) * (bn - 32 + 64));
    }
    if (best < 0 || worst < best) { best = worst; *nw = a; *nnar = b; }
  }
}

cudaError_t launch_gemm_epi_pair(const CUtensorMap& tmA, const CUtensorMap& tmB0,
                                 const CUtensorMap& tmB1, const CUtensorMap& tmB0n,
                                 const CUtensorMap& tmB1n, const GemmEpiParams& p, int nclusters,
                                 int ctas, cudaStream_t s) {
  if (p.bn < 64 || p.bn > BN || p.bn % 32 || nclusters < 1 || (ctas != 2 && ctas != 4) ||
      p.nw < 1 || p.nnar < 0 || (p.nnar > 0 && p.bn - 32 < 64) ||
      (long long)p.nw * p.bn + (long long)p.nnar * (p.bn - 32) < p.n)
    return cudaErrorInvalidValue;
  const int ntiles = (p.nw + p.nnar) * ((p.n + ctas * BM - 1) / (ctas * BM));
  const int ncl = ntiles < nclusters ? ntiles : nclusters;
  if (ctas == 4)
    k_gemm_epi_quad<<<4 * ncl, P_NTHREADS, P_SMEM_BYTES, s>>>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
  else
    k_gemm_epi_pair<<<2 * ncl, P_NTHREADS, P_SMEM_BYTES, s>>>(tmA, tmB0, tmB1, tmB0n, tmB1n, p);
  return cudaGetLastError();
}

cudaError_t launch_gemm_epi(const CUtensorMap& tmA, const CUtensorMap& tmB0,
                            const CUtensorMap& tmB1, const GemmEpiParams& p, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  if (p.bn < 32 || p.bn > BN || p.bn % 32) return cudaErrorInvalidValue;
  const int ntiles = ((p.n + p.bn - 1) / p.bn) * p.ntm;
  const int grid = ntiles < nsm ? ntiles : nsm;
  k_gemm_epi<<<grid, NTHREADS, SMEM_BYTES, s>>>(tmA, tmB0, tmB1, p);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int n, int ld, const float* Ahi0, const float* Alo0,
                            const float* Ahi1, const float* Alo1, const __half* dt0, double* Aout,
                            int64_t ld_a, const IterState* st, int only_done, cudaStream_t s) {
  const int nsm = device_sms();
  if (nsm <= 0) return cudaErrorInvalidDevice;
  const long long tiles = (long long)((n + 127) / 128) * ((n + 31) / 32);
  const int grid = (int)std::min<long long>(tiles, 16LL * nsm);   // 16 blocks of 128 per SM
  k_finalize<<<grid, 128, 0, s>>>(n, ld, Ahi0, Alo0, Ahi1, Alo1, dt0, Aout, ld_a, st, only_done);
  return cudaGetLastError();
}

}  // namespace dpt
