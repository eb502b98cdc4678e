// Device helpers shared by the libdpt kernels: float-float arithmetic, scaled FP16
// operands, bounded mbarrier waits, TMA loads and tcgen05 (TMEM / UMMA) wrappers
// written as inline PTX for sm_103a.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dpt_internal.h"

namespace dpt {

// ---------------------------------------------------------------------------
// float-float (unevaluated sum hi + lo of two FP32 numbers)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (ah + al) - (bh + bl), renormalised
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl,
                                       float& rh, float& rl) {
  float s, e;
  two_sum(ah, -bh, s, e);
  e += al - bl;
  fast_two_sum(s, e, rh, rl);
}
// (ah + al) + b, renormalised
__device__ __forceinline__ void ff_add_f(float ah, float al, float b, float& rh,
                                         float& rl) {
  float s, e;
  two_sum(ah, b, s, e);
  e += al;
  fast_two_sum(s, e, rh, rl);
}

// Two-product: a*b = p + e exactly (FMA).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Splits a double into hi + lo floats with integer operations only (on this GPU
// every FP64 operation, conversions included, runs on a pipe about 60x slower
// than FP32).  hi is v truncated to 24 significant bits; lo holds the next bits,
// rounded to 24 by the integer-to-float conversion (48 bits in all).  |v| below
// 2^-126 is flushed to zero, beyond the float range it becomes +-inf, NaN stays
// NaN; lo is dropped for |v| < 2^-74.
__device__ __forceinline__ void split_double(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hb = (unsigned)(b >> 32);
  const unsigned sign = hb & 0x80000000u;
  const int e = (int)((hb >> 20) & 0x7FFu);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  lo = 0.f;
  if (e == 0x7FF) {
    hi = __uint_as_float(sign | 0x7F800000u | (mant ? 0x400000u : 0u));
    return;
  }
  const int fe = e - 1023 + 127;
  if (fe <= 0) { hi = __uint_as_float(sign); return; }
  if (fe >= 255) { hi = __uint_as_float(sign | 0x7F800000u); return; }
  hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29));
  const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
  const int le = e - 1075 + 127;   // biased exponent of 2^(e - 1075)
  if (rem == 0u || le <= 0) return;
  lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(rem) * __uint_as_float((unsigned)le << 23)));
}

// Splits a double v into hi + lo floats with a few branch-free integer operations
// (one per streamed entry: split_double's exponent cases cost several times more).
// hi is v truncated to 24 significant bits, lo the next 23 bits truncated, so
// |v - hi - lo| < 2^-46 |v|.  Valid for 2^-103 <= |v| < 2^128; below that lo is 0
// and below 2^-126 hi is 0 as well (such terms are under 2^-103 of the unit-size
// quantities they meet).  Callers reject |v| >= 2^128 and non-finite v with
// beyond_float().
__device__ __forceinline__ void split_double_fast(double v, float& hi, float& lo) {
  const unsigned hb = (unsigned)__double2hiint(v);
  const unsigned lb = (unsigned)__double2loint(v);
  const unsigned e = (hb >> 20) & 0x7FFu;
  // (hb:lb) << 3 puts the exponent's low 9 bits over the top 23 mantissa bits;
  // subtracting 384 from that 9-bit field maps the FP64 bias onto the FP32 bias
  // (e - 1023 + 127 = e - 896 = (e mod 512) - 384 for 897 <= e <= 1150)
  const unsigned t = __funnelshift_l(lb, hb, 3) - (384u << 23);
  const unsigned hib = (t & 0x7FFFFFFFu) | (hb & 0x80000000u);
  // lo: the next 23 mantissa bits as the fraction of a float whose exponent is
  // 23 below hi's, minus that float's leading one (exact, Sterbenz)
  const unsigned base = (hib & 0xFF800000u) - (23u << 23);
  const unsigned gb = base | ((lb >> 6) & 0x7FFFFFu);
  const float l = __uint_as_float(gb) - __uint_as_float(base);
  hi = (e >= 897u) ? __uint_as_float(hib) : __uint_as_float(hb & 0x80000000u);
  lo = (e >= 920u) ? l : 0.f;
}

// Finite doubles are equal exactly when their bit patterns are, once -0 is read as +0:
// the comparisons run as 64-bit integer compares (the FP64 pipe of GB300 is slow).
__device__ __forceinline__ unsigned long long eq_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return b == 0x8000000000000000ull ? 0ull : b;
}

// True for values split_double_fast cannot represent: |v| >= 2^128, inf and NaN.
__device__ __forceinline__ bool beyond_float(double v) {
  return (((unsigned)__double2hiint(v) >> 20) & 0x7FFu) >= 1151u;
}

// True unless v is +-inf or NaN (integer test).
__device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFu) != 0x7FFu;
}

// Order-preserving integer key of a double (larger key <=> larger value, for
// non-NaN values), so that maxima can be taken with integer atomics.
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Exact float -> double by bit construction (zero and normal floats; subnormal
// floats, which this library never produces, fall back to the conversion).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0u) {
    if ((u & 0x7FFFFFu) == 0u) return __longlong_as_double((long long)sign);
    return (double)f;
  }
  const unsigned long long de = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (de << 52) | m));
}

// ---------------------------------------------------------------------------
// Bounded waits.  A wait that does not complete within kWaitNs sets the solve's
// timeout flag and gives up instead of spinning forever.
// ---------------------------------------------------------------------------
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Returns false (and sets *timeout) when the phase did not complete within
// limit_ns, or when another wait of the launch has already given up.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, unsigned* timeout,
                                             uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*((volatile unsigned*)timeout)) return false;
    if (global_ns() - t0 > limit_ns) {
      atomicExch(timeout, 1u);
      return false;
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* timeout) {
  return mbar_wait_ns(bar, parity, timeout, kWaitNs);
}
// Bounded wait that ignores (and never sets) the launch's timeout flag: used at the
// end of a kernel to let asynchronous arrivals land before the CTA exits, also
// after another wait has given up.
__device__ __forceinline__ bool mbar_wait_quiet(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (global_ns() - t0 <= limit_ns)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
constexpr uint64_t kTailWaitNs = 100000000ull;   // 100 ms

// ---------------------------------------------------------------------------
// TMA: 2-D tiled bulk tensor load into shared memory, completion on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, uint64_t* bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// Ampere-style asynchronous copies global -> shared, per thread, in groups
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05: tensor memory allocation, MMA, commit, loads, fences
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem], kind::f16 (16-bit inputs of the type idesc names,
// FP32 accumulator)
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every previously issued MMA of this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 32 lanes x 32 bits, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  // tie the destination registers to the wait so no use is scheduled before it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// CTA pairs (clusters of two): cluster rank, cluster-wide barrier, peer shared
// addresses, and the cta_group::2 forms of the TMEM, TMA and MMA instructions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of both CTAs
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}
// shared::cluster address of the variable at `p` in the CTA of cluster rank `rank`
__device__ __forceinline__ uint32_t mapa_shared(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}
// one warp of each CTA of the pair, collectively
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// TMA load into this CTA's shared memory, completing on an mbarrier that may live
// in either CTA of the pair (given as a shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const void* tmap, uint32_t bar_cluster,
                                                 int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}
// cta_group::2 form of the multicast load: `bar_cluster` is the leader's barrier of
// the issuing CTA's pair; each destination's copy completes on the barrier at that
// offset in the leader of the destination's own pair
__device__ __forceinline__ void tma_load_2d_pair_multicast(void* dst, const void* tmap,
                                                           uint32_t bar_cluster, int32_t x,
                                                           int32_t y, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".multicast::cluster.cta_group::2 [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(bar_cluster), "r"(x), "r"(y), "h"(mask)
      : "memory");
}

// D[tmem of both CTAs] (+)= A[smem of both CTAs, M halves] * B[smem of both CTAs, N halves]
__device__ __forceinline__ void umma_f16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on `bar` (same offset) in every CTA of `mask` once this thread's MMAs completed
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// 32 lanes x 32 bits, 8 consecutive columns per thread
__device__ __forceinline__ void tmem_ld_x8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// Approximate reciprocal (one hardware instruction, ~1 ulp)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle (rows of 64 16-bit elements = 128 B; 8-row groups 1024 B apart).
//   bits  0-13  start address >> 4
//   bits 16-29  leading-dimension byte offset >> 4 (unused for this layout: 1)
//   bits 32-45  stride-dimension byte offset >> 4 (1024 B between 8-row groups)
//   bits 46-47  descriptor version (1)
//   bits 61-63  layout: 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;
  d |= 1ull << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// Instruction descriptor, kind::f16: FP16 A and B (type fields 0; both operands of one
// MMA have the same type), FP32 D, both K-major.
//   bits 4-5 D format (1 = F32), 7-9 A format, 10-12 B format (0 = F16),
//   15/16 A/B major (0 = K), 17-22 N >> 3, 24-28 M >> 4
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// Warp transpose-reduction: each lane holds v[0..15] (16 columns); afterwards
// lane l holds, in v[0], the sum over all 32 lanes of column (l >> 1) & 15.
// (Pairs of lanes hold the same column.)  15 + 1 shuffles for 16 values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16], int lane) {
  // offset 16: keep 8 columns
  {
    const bool up = lane & 16;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float send = up ? v[c] : v[c + 8];
      float keep = up ? v[c + 8] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float send = up ? v[c] : v[c + 4];
      float keep = up ? v[c + 4] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool up = lane & 4;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float send = up ? v[c] : v[c + 2];
      float keep = up ? v[c + 2] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
  }
  {
    const bool up = lane & 2;
    float send = up ? v[0] : v[1];
    float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}
// Column owned by `lane` after warp_transpose_sum16.
__device__ __forceinline__ int transpose_sum16_col(int lane) {
  return ((lane & 16) ? 8 : 0) + ((lane & 8) ? 4 : 0) + ((lane & 4) ? 2 : 0) +
         ((lane & 2) ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Epilogue helpers: four consecutive rows per lane
// ---------------------------------------------------------------------------
struct Col4 {
  float4 ah, al, L;
  uint2 dtp;      // four FP16 (the stored, scaled previous increment)
  uint2 D[3];     // Delta_ij 2^sig as FP16 slices, four rows each
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
// 32-byte global store (one sector; p 32-byte aligned)
__device__ __forceinline__ void st_global_v8(void* p, uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t a4, uint32_t a5, uint32_t a6,
                                             uint32_t a7) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a0),
               "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7)
               : "memory");
}

__device__ __forceinline__ float f4(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}
// Element e (0..3) of four FP16 values packed in a uint2, as a float (exact).
__device__ __forceinline__ float h_at(uint2 u, int e) {
  const uint32_t w = (e < 2) ? u.x : u.y;
  return __half2float(__ushort_as_half((unsigned short)((e & 1) ? (w >> 16) : (w & 0xFFFFu))));
}
// Two floats rounded to FP16 (nearest even) and packed (a in the low half); values
// beyond the FP16 range become +-65504 instead of infinities.
__device__ __forceinline__ uint32_t f16x2_sat(float a, float b) {
  uint32_t r;
  asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
// 2^e as a float, for -126 <= e <= 127 (exact; bit construction).
__device__ __forceinline__ float exp2i(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }
// floor(log2 |x|) of a nonzero finite double, from its bits (normal range).
__device__ __forceinline__ int ilog2_bits(double x) {
  return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7FFu) - 1023;
}

// x qs rounded to FP16 (nearest even, +-65504 beyond the range): the FP16 bits in
// `bits` and the rounded value times iqs (exact for power-of-two qs, iqs = 1 / qs)
__device__ __forceinline__ float f16_scaled(float x, float qs, float iqs, uint32_t& bits) {
  const uint32_t w = f16x2_sat(x * qs, 0.f);
  bits = w & 0xFFFFu;
  return __half2float(__ushort_as_half((unsigned short)bits)) * iqs;
}

// One 32-row x 64-column tile of the Delta -> FP16-slice conversion, block (32, 8).
// Reads Delta (FP64, column-major, rows j contiguous) at rows [by, by+32) and columns
// [bx, bx+64) into shared memory, then writes row j of NSL slices (row-major, pitch ld
// inside a row of cat_ld elements) as FP16 pairs of Delta 2^sig (sc = 2^sig): with
// v = hi + lo (split_double_fast), D1 = f16(hi sc), each further slice the FP16
// rounding of what is left (the remainders are exact in float), the last one taking
// lo sc as well.  Columns in [n, ld) are written as zeros; en != 0 zeroes the
// diagonal.  A non-finite entry, or one of magnitude 2^128 or more (beyond the float
// range), sets *bad.
template <int NSL>
__device__ __forceinline__ void slice16_tile_32x64(const double* __restrict__ delta, int64_t ld_in,
                                                   int n, int ld, int en, float sc, int bx,
                                                   int by, __half* __restrict__ Dcat, int64_t cat_ld,
                                                   unsigned* bad, double (*tile)[65]) {
  const int x = threadIdx.x, y = threadIdx.y;
  {
    // all eight loads are issued before any check (an atomic between them would
    // keep the next load from starting)
    const int j = by + x;
    double v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = bx + y + 8 * m;
      v[m] = (j < n && k < n) ? delta[(int64_t)k * ld_in + j] : 0.0;
    }
    bool badv = false;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = bx + y + 8 * m;
      badv |= beyond_float(v[m]);   // non-finite, or beyond the float range
      if (en && j == k) v[m] = 0.0;
      tile[x][y + 8 * m] = v[m];    // tile[j - by][k - bx]
    }
    if (badv) atomicExch(bad, 1u);
  }
  __syncthreads();
  const int k0 = bx + 2 * x;
  if (k0 >= ld) return;
#pragma unroll
  for (int r = y; r < 32; r += 8) {
    const int j = by + r;
    if (j >= n) break;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    if (k0 < n) split_double_fast(tile[r][2 * x], h0, l0);
    if (k0 + 1 < n) split_double_fast(tile[r][2 * x + 1], h1, l1);
    __half* row = Dcat + (int64_t)j * cat_ld + k0;
    float r0 = h0 * sc, r1 = h1 * sc;
#pragma unroll
    for (int sl = 0; sl < NSL; ++sl) {
      const bool lastsl = (sl == NSL - 1);
      const float t0 = lastsl ? r0 + l0 * sc : r0;
      const float t1 = lastsl ? r1 + l1 * sc : r1;
      const __half q0 = __float2half_rn(t0), q1 = __float2half_rn(t1);
      r0 = t0 - __half2float(q0);
      r1 = t1 - __half2float(q1);
      *reinterpret_cast<__half2*>(row + (int64_t)sl * ld) = __halves2half2(q0, q1);
    }
  }
}

// Warp reduction of the column sums: |R|^2 and |a|^2 in float, the diagonal
// increment (eh, el) in float-float.
__device__ __forceinline__ void warp_sum_ff(float& r2, float& a2, float& eh, float& el) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    const float oh = __shfl_xor_sync(0xffffffffu, eh, o);
    const float ol = __shfl_xor_sync(0xffffffffu, el, o);
    float sh, se;
    two_sum(eh, oh, sh, se);
    se += el + ol;
    fast_two_sum(sh, se, eh, el);
  }
}

// ---------------------------------------------------------------------------
// The state as one register copy.  A control kernel's last block reads the state
// after every other block's atomics: reading each field through a volatile pointer
// costs a round trip to L2 per field that a branch depends on, so the deciding
// thread loads all of it at once (L2 loads, issued together), decides on the copy
// and writes it back.  No other kernel runs meanwhile, and the grid's other blocks
// have finished with the state when the last one takes over.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void state_load(const T* st, T& ls) {
  static_assert(sizeof(T) % 8 == 0, "the state is copied as 8-byte words");
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(st);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&ls);
#pragma unroll
  for (int w = 0; w < (int)(sizeof(T) / 8); ++w) dst[w] = __ldcg(src + w);
}
template <class T>
__device__ __forceinline__ void state_store(T* st, const T& ls) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&ls);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(st);
#pragma unroll
  for (int w = 0; w < (int)(sizeof(T) / 8); ++w) __stcg(dst + w, src[w]);
}

// ---------------------------------------------------------------------------
// Convergence decision shared by the control kernels (run by one thread of the
// last block), on the state or on a register copy of it.  rho is the normalised
// max residual of the iterate A_k.  Returns true when the iteration continues (k
// and cur advanced).
// ---------------------------------------------------------------------------
template <class SP>
__device__ __forceinline__ bool decide(SP* vs, double rho) {
  vs->rho = rho;
  if (vs->bad_input) { vs->status = ST_BADINPUT; return false; }
  if (vs->timeout) { vs->status = ST_TIMEOUT; return false; }
  if (!(rho == rho) || isinf(rho)) { vs->status = ST_DIVERGED; return false; }
  if (rho <= vs->tol) { vs->status = ST_CONVERGED; return false; }
  if (rho < vs->best) { vs->best = rho; vs->grown = 0; }
  else if (rho > 10.0 * vs->best) {
    if (++vs->grown >= 20) { vs->status = ST_DIVERGED; return false; }
  } else vs->grown = 0;
  if (vs->k >= vs->max_iter) { vs->status = ST_MAXITER; return false; }
  vs->k = vs->k + 1;
  vs->cur = vs->k & 1;
  if (vs->ramp_alpha > 0.0) {   // strength lambda (1 - alpha^k) for the next step
    double pw = vs->ramp_pow * vs->ramp_alpha;
    if (pw < 0x1p-60) pw = 0.0;
    vs->ramp_pow = pw;
    vs->lam_k = vs->lam * (1.0 - pw);
  }
  return true;
}

// Decision after a certifying pass (an assessment of A_k that produced no A_{k+1}):
// the statuses of decide() when the iterate fails or passes; otherwise the state is
// left as it is (k not advanced) so that the same iteration runs again in full.
// Returns true when the iteration continues.
template <class SP>
__device__ __forceinline__ bool decide_final(SP* vs, double rho) {
  vs->rho = rho;
  if (vs->bad_input) { vs->status = ST_BADINPUT; return false; }
  if (vs->timeout) { vs->status = ST_TIMEOUT; return false; }
  if (!(rho == rho) || isinf(rho)) { vs->status = ST_DIVERGED; return false; }
  if (rho <= vs->tol) { vs->status = ST_CONVERGED; return false; }
  return true;
}

// The same for a single-vector solve: the next step applies lambda - dlam with
// dlam = lambda alpha^k (carried in FP64 and as a float pair).
template <class SP>
__device__ __forceinline__ void dom_ramp_advance(SP* vs) {
  if (!(vs->ramp_alpha > 0.0)) return;
  double pw = vs->ramp_pow * vs->ramp_alpha;
  if (pw < 0x1p-60) pw = 0.0;
  vs->ramp_pow = pw;
  const double dl = vs->lam * pw;
  vs->dlam = dl;
  const float h = (float)dl;
  vs->dlam_hi = h;
  vs->dlam_lo = (float)(dl - (double)h);
}

// ---------------------------------------------------------------------------
// Slices of Delta for the next product, from the largest increment dmax it will
// multiply.  With S FP16 slices the truncation of Delta is about 2^(-11 S) relative,
// so a product's truncation error is about 2^(-11 S) |Delta| dmax.  The first product
// (nsl slices on the increment dt_0 of size dmax1) sets the error the solve accepts;
// later products take the fewest slices that stay below it.  The carried remainder
// makes the fixed point that of the full Delta either way.
// ---------------------------------------------------------------------------
// The rule for FP16 slices (11 significant bits each, so about 2^(-11 S) relative) of
// a solve whose first product used nsl of them: the accepted truncation is that of the
// first product, 2^(-11 nsl) dmax1, but no finer than the FP32 accumulation's own
// 2^-24 dmax1 (three slices would otherwise keep 33 bits long after the accumulator
// has stopped resolving them); a later product takes the fewest slices S with
// 2^(-11 S) dmax within it, and one below slice_tol.  With nsl = 2 this drops to one
// slice once dmax <= 2^-11 dmax1; with nsl = 3 to two once dmax <= dmax1 / 4 and to
// one once dmax <= 2^-13 dmax1.
template <class SP>
__device__ __forceinline__ int next_slices_f16(SP* vs, float dmax, bool first, int nsl) {
  if (first) vs->dmax1 = dmax;
  const float d1 = vs->dmax1;
  if ((double)dmax < vs->slice_tol) return 1;
  const int b = min(11 * nsl, 24);
  int S = nsl;
  while (S > 1 && dmax <= d1 * exp2i(11 * (S - 1) - b)) --S;
  return S;
}

// Scale exponent s of an FP16 increment buffer (it holds dt * 2^s): the expected
// largest |dt| `ref` lands in [2^top, 2^(top+1)), so FP16's 2^-14 .. 65504 keeps its
// full 11 bits for entries down to 2^-(14+top) of it (the rest rounds; the carried
// remainder keeps what rounding drops).  s is bounded so that lambda 2^-(sig + s),
// the product's multiplier, stays a normal float.  Scaling (Delta, lambda) to
// (2^p Delta, 2^-p lambda) shifts sig by -p and leaves s unchanged.
__device__ __forceinline__ int dt_scale_exp(double ref, int top, int sig, double lam) {
  int s = (ref > 0.0 && ref < 1e300) ? top - ilog2_bits(ref) : 0;
  if (lam != 0.0 && fabs(lam) < 1e300) {
    const int lg = ilog2_bits(lam);
    s = max(lg - 120 - sig, min(lg + 120 - sig, s));
  }
  return max(-120, min(120, s));
}

}  // namespace dpt
