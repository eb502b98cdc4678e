// Internal declarations shared by the libdpt host runtime and its kernels.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dpt {

// Columns per block of the mixed solve's iteration 0 (k_iter0); its row sums of |Delta|
// are left as one partial per such block of columns (rowpart: (n + 63) / 64 rows of ld).
constexpr int kIter0Cols = 64;

enum : int {
  ST_RUNNING = 0,
  ST_CONVERGED = 1,
  ST_BADINPUT = -1,
  ST_DEGENERATE = -2,
  ST_MAXITER = -3,
  ST_DIVERGED = -4,
  ST_TIMEOUT = -7,
  ST_CANCELLED = -11,   // server request cancelled while on the GPU
  ST_IDLE = 2,          // server slot without a problem
};

// Per-solve iteration state, resident in device memory.  The control kernels
// advance it; every iteration kernel reads `status` first and returns at once
// once the solve has finished, so a captured graph of several iterations can be
// replayed past convergence without changing the result.
struct IterState {
  int k;               // index of the current iterate A_k
  int status;          // ST_*
  int slices;          // FP16 slices of Delta used by the next product
  int cur;             // ping-pong index of the buffers holding A_k
  int grown;           // consecutive iterations with residual > 10 x best
  int max_iter;
  int max_slices;
  int slice_gemms;     // running sum of slices used
  unsigned blocks_done;
  unsigned rho_bits;   // atomicMax scratch: max_i sqrt(|R_i|^2 / |a_i|^2)
  unsigned dmax_bits;  // atomicMax scratch: max |delta A| of the last update
  unsigned row_bits;   // atomicMax scratch: max_j sum_k |Delta_jk|
  unsigned bad_input;  // nonzero when a non-finite input value was seen
  unsigned timeout;    // nonzero when a bounded wait expired
  double s;            // residual scale max|theta| + |lambda| max_j sum_k |Delta_jk|
  double theta_max;    // max_j |theta_j|
  double lam;
  double tol;
  double slice_tol;
  double rho;          // normalised max residual of A_k
  double best;
  double rho_last;     // normalised residual of the previous iterate
  float dmax1;         // max |dt_0|: the increment fed to the first product
  double ramp_alpha;   // non-autonomous iteration (0: off)
  double ramp_pow;     // ramp_alpha^k
  double lam_k;        // strength the next map application uses (FP64 path)
  int certify;         // mixed single solve: the next product only assesses its iterate
  int certify_on;      // whether such passes may be scheduled (dpt_options::certify)
  // mixed single solve: Delta and the increments are FP16 tensor-core operands with
  // power-of-two scales (their range is that of FP16, their scale free)
  unsigned amax_bits;  // atomicMax scratch: high word of max |Delta_jk| (FP64 bits)
  unsigned g0max_bits; // atomicMax scratch: max_{j != i} |Delta_ji| / |theta_i - theta_j|
  int sig;             // the FP16 slices hold Delta * 2^sig
  int sexp[2];         // increment buffer q holds dt * 2^sexp[q] in FP16
  int cert_out;        // mixed single solve: a certifying pass also writes the FP64 output
  int out_done;        // ... and the pass that certified the returned iterate wrote it
  double rho_sum;      // sum of the residuals rho_k, k >= 1, the float recursion carried
  // mixed single solve: inputs of the bound on its arithmetic error (see dpt_refine.cu)
  unsigned rgmax_bits; // atomicMax scratch: max_{j != i} 1 / |theta_i - theta_j| (float bits)
  double dsum;         // sum over the updates of max |dt_k|: a bound of max |A_ji - delta_ji|
};

// Maxima of one FP64 step over the refined columns (dpt_refine.cu).
struct RefineCtl {
  unsigned blocks_done;
  unsigned pad;
  double step;         // max over the columns of |A' - A| / |A|
  double rho;          // max over the columns of |M a - E a| / (s |a|) of the step's input
};
cudaError_t launch_risk(int n, const double* A, int64_t lda, const float* thh, const float* thl,
                        double coef, double target, int* count, int* cols, cudaStream_t s);
cudaError_t launch_cols_gather(int n, int nc, const int* cols, const double* A, int64_t lda,
                               double* As, cudaStream_t s);
cudaError_t launch_cols_scatter(int n, int nc, const int* cols, const double* As, const double* Ec,
                                double* A, int64_t lda, double* E, cudaStream_t s);
int refine_k_chunks(int n);
cudaError_t launch_cols_product(int n, int nc, const double* D, int64_t ldd, const double* As,
                                int nks, double* Pp, cudaStream_t s);
cudaError_t launch_cols_epi(int n, int nc, int nks, const int* cols, const double* theta,
                            const double* D, int64_t ldd, int en, double lam, double s_scale,
                            const double* Pp, const double* Ac, double* An, double* Ec,
                            RefineCtl* ctl, cudaStream_t s);

// State of a dominant-eigenvector solve (single-vector map), device resident.
struct DomState {
  int k;                 // index of the current iterate z_k
  int status;            // ST_*
  int cur;               // ping-pong index of z_k
  int grown;
  int max_iter;
  int nstar;             // eigenvector index in use
  int nstar_req;         // requested index, -1 = argmax theta
  int nstar_min;         // first index of the largest theta (atomicMin scratch)
  unsigned ties;         // number of m with theta_m == theta_{n*}
  unsigned blocks_done;
  unsigned row_bits;     // max_m sum_k |Delta_mk| (float bits)
  unsigned absmax_bits;  // max |theta| (float bits)
  unsigned bad_input;
  unsigned pad;
  unsigned long long theta_bits;   // largest theta, order-preserving bits
  double lam;
  float lam_hi, lam_lo;
  float ys_hi, ys_lo;    // y* = (Delta z)_{n*}, float-float
  double ys64;           // y* in FP64 (FP64 variant)
  double s;              // residual scale
  double tol;
  double rho;
  double best;
  double E;              // eigenvalue of the assessed iterate
  double ramp_alpha;     // non-autonomous iteration (0: off)
  double ramp_pow;       // ramp_alpha^k
  double dlam;           // lambda minus the strength of the next map application
  float dlam_hi, dlam_lo;
};

// One problem of a grouped (batched / served) solve: a device-resident table entry
// with the problem's size, tile shape, work arrays, state and TMA descriptors.
struct alignas(128) GProb {
  CUtensorMap tmA;          // Delta slices (row-major scaled FP16, 3 slice places side by side)
  CUtensorMap tmB[2];       // increment buffers dt[0], dt[1]
  // n: problem size; nr: rows of the real product (n, or 2n for a complex problem,
  // whose rows and K index interleave real and imaginary parts); ld: row pitch of
  // every work column (a multiple of 128, >= nr); ntm: 128-row tiles over nr
  int n, ld, ntm, ntn, bn, cplx, nr, pad0;
  float lam, lam_lo;
  double lam64;
  float* A_hi[2];
  float* A_lo[2];
  __half* dt[2];            // increments, FP16 scaled by 2^sexp[buffer] of the state
  float* L;
  __half* Dcat;             // FP16 slices of Delta 2^sig (the state's sig)
  int64_t cat_ld;
  float* th_hi;
  float* th_lo;
  const double* theta;      // input theta (device)
  double* d;
  double* E;
  float* e_col;
  float* dprev_col;
  float* part;              // column partials [6][ntm][n]: |R|^2, |a|^2, diag (hi, lo) x (re, im)
  float* rowpart;
  IterState* st;
  const double* delta_in;   // input Delta (device, column-major; interleaved if complex)
  int64_t ld_in;
  double* A_out;            // outputs (device)
  int64_t ld_a;
  double* E_out;
};

cudaError_t g_set_attributes();
// max_n: the largest problem size among the first `count` table entries
cudaError_t launch_g_check_theta(const GProb* probs, int count, int max_n, int* running,
                                 cudaStream_t s);
// the FP16 scales of every problem (items: the iteration-0 tiles of one kind)
cudaError_t launch_g_scales(const GProb* probs, const int4* items, int nitems, bool cplx,
                            cudaStream_t s);
cudaError_t launch_g_prep(const GProb* probs, const int4* items, int nitems, cudaStream_t s);
cudaError_t launch_g_iter0(const GProb* probs, const int4* items, int nitems, cudaStream_t s);
cudaError_t launch_g_ctrl(const GProb* probs, int count, int max_n, bool cplx, int* running,
                          cudaStream_t s);
cudaError_t launch_g_gemm_epi(const GProb* probs, const int2* tiles, int ntiles,
                              unsigned* timeout, bool cplx, cudaStream_t s);
cudaError_t launch_g_finalize(const GProb* probs, const int4* items, int nitems, cudaStream_t s);
// CTA-pair form of the grouped product: tiles are (problem, 256-row pair tile); the
// problems' increment descriptors have boxes of bn/2 rows
int g_pair_clusters();
cudaError_t launch_g_gemm_epi_pair(const GProb* probs, const int2* tiles, int ntiles,
                                   unsigned* timeout, bool cplx, int npairs, cudaStream_t s);
// One CTA per 128-row tile with the staged 16-warp epilogue (tile widths <= 128).
cudaError_t launch_g_gemm_epi_staged(const GProb* probs, const int2* tiles, int ntiles,
                                     unsigned* timeout, bool cplx, cudaStream_t s);
cudaError_t launch_gc_prep(const GProb* probs, const int4* items, int nitems, cudaStream_t s);
cudaError_t launch_gc_iter0(const GProb* probs, const int4* items, int nitems, cudaStream_t s);
cudaError_t launch_gc_finalize(const GProb* probs, const int4* items, int nitems, cudaStream_t s);

// Arguments of the tensor-core iteration kernel (mixed path, real).
struct GemmEpiParams {
  int n;               // matrix size
  int ld;              // padded leading dimension of every n x n work array (multiple of 128)
  int ntm;             // number of 128-row tiles
  int bn;              // output tile width (columns), a multiple of 32 up to 256
  float lam;
  float* A_hi[2];      // float-float iterate, column-major, ping-pong by iteration parity
  float* A_lo[2];
  __half* dt[2];       // FP16 increments (scaled by 2^sexp), column-major (GEMM B operand), ping-pong
  float* L;            // carried remainder, column-major
  const __half* Dcat;  // Delta * 2^sig as up to 3 FP16 slices, row-major, slices side by side
  int64_t cat_ld;      // row pitch of Dcat (3 * ld)
  const float* th_hi;  // theta as float-float
  const float* th_lo;
  const float* e_col;      // e_k = diag(Delta dt_{k-1})
  const float* dprev_col;  // d_{k-1}
  float* part;         // column partials [4][ntm][ld]: |R|^2, |a|^2, diag hi, diag lo
  IterState* st;
  double* Aout;        // FP64 output (column-major, ld_a), written by certifying passes
  int64_t ld_a;        // of the pair kernel (IterState::cert_out)
  int aout_v8;         // Aout 32-byte aligned and ld_a a multiple of 4 (32-byte stores)
  int nw;              // pair kernel: column tiles of width bn, then
  int nnar;            //   nnar of width bn - 32 (mixed_pair_split)
};

int mixed_smem_bytes();
int mixed_tile_n(int n, int nsm);   // columns per output tile of the product kernel
// CTA-pair forms: clusters of `ctas` = 2 (one pair) or 4 (two pairs sharing B)
int mixed_pair_clusters(int ctas);  // resident clusters of that shape (after mixed_set_attributes)
int mixed_pair_tile_n(int n, int nclusters, int ctas);
void mixed_pair_split(int n, int bn, int nclusters, int ctas, int* nw, int* nnar);
// tmB0n / tmB1n: the increment maps with boxes of bn / 2 - 16 rows (the narrow tiles)
cudaError_t launch_gemm_epi_pair(const CUtensorMap& tmA, const CUtensorMap& tmB0,
                                 const CUtensorMap& tmB1, const CUtensorMap& tmB0n,
                                 const CUtensorMap& tmB1n, const GemmEpiParams& p, int nclusters,
                                 int ctas, cudaStream_t s);
cudaError_t mixed_set_attributes();   // once per device, before any capture
// max |Delta| and max |Delta_ji / (theta_i - theta_j)| (j != i); sets the scales of
// the FP16 slices and of the first increment (IterState::sig, sexp[0]).  With a start
// (device, leading dimension ld_s) the first increment is its offset from I: its
// largest entry sets sexp[0], sinv[i] = 1 / start[i, i] (ld doubles) is written, and a
// zero or non-finite chart entry or value marks the input bad.
cudaError_t launch_delta_scales(const double* delta, int64_t ld_in, int n, const float* th_hi,
                                const float* th_lo, double lam, int en, const double* start,
                                int64_t ld_s, double* sinv, IterState* st, cudaStream_t s);
// nsl FP16 slices of Delta * 2^sig (needs launch_delta_scales first)
cudaError_t launch_prep_delta(const double* delta, int64_t ld_in, int n, int ld, int en, int nsl,
                              __half* Dcat, IterState* st, cudaStream_t s);
cudaError_t launch_theta_ff(int n, const double* th, float* hi, float* lo, cudaStream_t s);
// finite and pairwise distinct theta (status ST_BADINPUT / ST_DEGENERATE), max |theta|
// (hi, lo given: theta split into float-float as launch_theta_ff does, in the same launch)
cudaError_t launch_check_theta(int n, const double* th, IterState* st, cudaStream_t s,
                               float* hi = nullptr, float* lo = nullptr);
// iteration 0 from A_0 = I: dt_0 = f16(r_0 G o R_0), or with a start its offset from I
cudaError_t launch_iter0(const double* delta, int64_t ld_in, const float* th_hi,
                         const float* th_lo, double lam, int n, int ld, int en, int nsl,
                         const __half* Dcat, __half* dt0, float* L, double* d, float* part,
                         float* rowpart, const double* start, int64_t ld_s, const double* sinv,
                         IterState* st, cudaStream_t s);
// iteration 0 fused with the slicing (no start; Delta as an FP64 tensor map with
// 16 x 16 boxes, make_tmap_f64): writes Dcat, dt0, L, d and the column partials in
// ld / 64 slots of 64 rows (pass that count to the first launch_ctrl)
cudaError_t launch_iter0_pairs(const CUtensorMap& tmD, const float* th_hi, const float* th_lo,
                               double lam, int n, int ld, int en, int nsl, __half* Dcat,
                               __half* dt0, float* L, double* d, float* part, float* rowpart,
                               IterState* st, cudaStream_t s);
// nslot > 0: the column partials are in nslot row slots (else one per 128-row tile);
// hilo = 0: the products' diagonal partials have zero low parts (the pair kernel's);
// first_step: the partials are iteration 0's (else a product's)
cudaError_t launch_ctrl(int n, int ld, const float* part, const float* rowpart,
                        const double* theta, double* d, double* E, float* e_col,
                        float* dprev_col, IterState* st, cudaStream_t s, int nslot, int hilo,
                        int first_step);
cudaError_t launch_gemm_epi(const CUtensorMap& tmA, const CUtensorMap& tmB0,
                            const CUtensorMap& tmB1, const GemmEpiParams& p, cudaStream_t s);
// The returned iterate in FP64 (A_1 = I + dt_0 is formed from the first increment dt0).
cudaError_t launch_finalize(int n, int ld, const float* Ahi0, const float* Alo0,
                            const float* Ahi1, const float* Alo1, const __half* dt0, double* Aout,
                            int64_t ld_a, const IterState* st, int only_done, cudaStream_t s);

// Plain FP64 path (real and complex)
cudaError_t launch_fp64_init(int n, int ld, int cplx, void* A0, cudaStream_t s);
cudaError_t launch_gemm_f64(int n, const double* Dl, int64_t ldd, const double* A, int ld,
                            double* P, const IterState* st, cudaStream_t s);
cudaError_t launch_gemm_c128(int n, const double* Dl, int64_t ldd, const double* A, int ld,
                             double* P, const IterState* st, cudaStream_t s);
cudaError_t launch_epi_f64(int n, int ld, int cplx, const double* theta, double lam,
                           const double* P, const double* Acur, double* Anext,
                           const double* Dl, int64_t ldd, double* E, IterState* st,
                           int first, cudaStream_t s);

// Dominant form (CSR)
int dom_blocks(int n);
cudaError_t launch_dom_check(int n, int64_t nnz, const int32_t* row_ptr, DomState* st,
                             cudaStream_t s);
// theta split and maxima, n*, ties, and the gate (statuses of malformed / degenerate
// input set on the device); the first pass validates col_idx / vals and forms s
cudaError_t launch_dom_setup(int n, const double* theta, float* th_hi, float* th_lo, DomState* st,
                             cudaStream_t s);
cudaError_t launch_probe_gather(int n, int vlanes, const int32_t* row_ptr, const int32_t* col_idx,
                                const float2* z, float* y, cudaStream_t s);
cudaError_t launch_dom_init(int n, float2* z, double* z64, int ff, DomState* st,
                            cudaStream_t s);
cudaError_t launch_dom_iter(int n, int vlanes, int ff, const int32_t* row_ptr,
                            const int32_t* col_idx, const float* vals, const float* th_hi,
                            const float* th_lo, const double* theta, float2* z0, float2* z1,
                            double* z64_0, double* z64_1, double* part, DomState* st,
                            cudaStream_t s, bool first = false);
cudaError_t launch_dom_select(int n, const double* theta, DomState* st, cudaStream_t s);
cudaError_t launch_dom_start(int n, const double* v, float2* z, double* z64, DomState* st,
                             cudaStream_t s);
cudaError_t launch_fp64_start(int n, int ld, int cplx, double* A, IterState* st, cudaStream_t s);
cudaError_t launch_h_transpose(int n, int ld, const double* X, double* Y, cudaStream_t s);
cudaError_t launch_h_mv(int n, int ld, const double* theta, const double* V, double c, double* T,
                        cudaStream_t s);
cudaError_t launch_h_stage(int n, int ld, const double* e, double step, double* S,
                           cudaStream_t s);
cudaError_t launch_h_two_minus(int n, int ld, double* T, cudaStream_t s);
cudaError_t launch_rs_eps(int n, int ld, const double* X, double* eps_l, double lam_l, double* E,
                          cudaStream_t s);
cudaError_t launch_rs_order(int n, int ld, int l, const double* X, double* C, const double* eps,
                            const double* theta, double lam_l, double* A, cudaStream_t s);
cudaError_t launch_h_biorth(int n, int ld, const double* A, double* B, IterState* st,
                            cudaStream_t s);
cudaError_t launch_h_chart(int n, int ld, const double* V, double* out, int64_t ld_out,
                           IterState* st, cudaStream_t s);

// Dense dominant form (GEMV): arguments of one iteration's two kernels.
struct DDParams {
  int n, vec, slice, nslices;      // size, rows per thread, columns per slice, slices
  int64_t ld;                      // leading dimension of Delta (elements)
  const double* delta;             // column-major FP64
  float2* z0;                      // z ping-pong, float-float
  float2* z1;
  double* z64_0;                   // z ping-pong, FP64 (comparator)
  double* z64_1;
  float2* ypart;                   // slice partials of y, [nslices][n]
  double* ypart64;
  float* rowabs;                   // slice partials of sum_k |Delta_mk| (first pass)
  const float* th_hi;
  const float* th_lo;
  const double* theta;
  double* part;                    // per-block norm partials of the update kernel
  DomState* st;
};
int dd_slice(int n, int vec, int nsm);
void dd_plan(DDParams& p, bool aligned16);
int dd_update_blocks(int n);
cudaError_t launch_dd_setup(int n, const double* theta, float* th_hi, float* th_lo, DomState* st,
                            cudaStream_t s);
cudaError_t launch_dd_gemv(const DDParams& p, int ff, int first, cudaStream_t s);
cudaError_t launch_dd_update(const DDParams& p, int ff, int first, cudaStream_t s);
cudaError_t launch_dom_out(int n, const float2* z0, const float2* z1, const double* z64_0,
                           const double* z64_1, int ff, double* out, const DomState* st,
                           cudaStream_t s);

}  // namespace dpt
