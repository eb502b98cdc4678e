/* libdpt: dynamical perturbation theory (DPT) eigensolver for one GB300 GPU.
 *
 * Method: M. Kenmoe, M. Smerlak, A. Zadorin, "Dynamical perturbation theory for
 * eigenvalue problems", arXiv:2002.12872.  For M = D + lambda * Delta with
 * D = diag(theta) and simple unperturbed eigenvalues theta (Sec. II.B), the
 * eigenvectors are the fixed points of the map of Eq. (dyn).  In the column
 * convention used throughout this library (column i of A is eigenvector i; the
 * paper stores it as row i and multiplies by Delta'):
 *
 *     A  <-  I + lambda * G o (Delta A - A diag(Delta A)),
 *     G_ji = 1 / (theta_i - theta_j) for j != i,   G_ii = 0,
 *     E  =  theta + lambda * diag(Delta A)          (read-out of Sec. II.B),
 *
 * iterated from A = I.  Every column keeps A_ii = 1 (the affine chart z^n = 1 of
 * Sec. II.A).  The dominant-eigenvector form iterates one column, n* = argmax
 * theta, with a matrix-vector product in place of the matrix product (the
 * single-vector map of Eq. (single_line_dyn), Sec. II.H).
 *
 * Conventions for every entry point:
 *   - Dense matrices are column-major with a leading dimension ld >= n.
 *   - A pointer argument may point to device memory or to host memory (pinned or
 *     pageable); the library checks each pointer with cudaPointerGetAttributes
 *     and stages host buffers through device memory itself.  Host outputs are
 *     complete when the call returns.
 *   - The caller owns every input and output buffer.  Inputs are never modified.
 *     Scratch memory comes from a per-device pool inside the library that grows
 *     on demand and is kept between calls (dpt_release_workspace frees it).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All device
 *     work is ordered on it; the solve calls block until their results are ready.
 *   - Errors are reported only through the returned dpt_status; nothing aborts
 *     and nothing is thrown across this boundary.  On an error the outputs are
 *     unspecified, except that *info (when non-NULL) is filled.
 *   - Calls on different streams may run concurrently; each call uses its own
 *     scratch block from the pool.  The one exception is
 *     dpt_solve_dominant_noalloc, whose calls share a single fixed block and must
 *     not overlap on the GPU.
 */
#ifndef DPT_H
#define DPT_H

#include <stdint.h>

#if defined(__GNUC__)
#define DPT_API __attribute__((visibility("default")))
#else
#define DPT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DPT_OK = 0,
  DPT_PENDING = 1,            /* server request not finished yet */
  DPT_ERR_ARG = -1,           /* invalid argument or non-finite input */
  DPT_ERR_DEGENERATE = -2,    /* theta_i == theta_j for some i != j (Sec. II.B) */
  DPT_ERR_MAXITER = -3,       /* max_iter reached before the tolerance */
  DPT_ERR_DIVERGED = -4,      /* non-finite iterate, or residual growth: the orbit
                                 cycles or escapes outside the convergence domain
                                 (Sec. II.E) */
  DPT_ERR_NOMEM = -5,         /* device or host allocation failed */
  DPT_ERR_CUDA = -6,          /* a CUDA runtime call failed */
  DPT_ERR_TIMEOUT = -7,       /* a bounded device-side wait expired */
  DPT_ERR_UNSUPPORTED = -8,   /* option combination not implemented */
  DPT_ERR_TOO_LARGE = -9,     /* problem larger than a fixed-size entry point or a
                                 server's memory budget accepts */
  DPT_ERR_BUSY = -10,         /* server queue full: the request was not taken */
  DPT_ERR_CANCELLED = -11     /* server request cancelled before it finished */
} dpt_status;

typedef enum {
  DPT_R64 = 0,    /* real: theta, Delta, A, E are double */
  DPT_C128 = 1    /* complex: Delta, A, E are interleaved complex double (re, im);
                     theta and lambda stay real */
} dpt_dtype;

typedef enum {
  DPT_PREC_FP64 = 0,        /* every product in FP64 on the CUDA cores: the map of
                               Eq. (dyn) applied literally */
  DPT_PREC_MIXED = 1        /* tensor-core products: each iteration multiplies Delta,
                               split into FP16 slices, by the FP16 increment of A,
                               with FP32 accumulation (slices and increments carry
                               power-of-two scales chosen per problem); A, the residual
                               and the eigenvalues are carried in extended
                               precision, so the iteration refines to the FP64
                               fixed point.  There is no TF32 variant: on this GPU
                               the TF32 tensor rate is half the 16-bit rate and a
                               TF32 operand takes twice the bytes, while two scaled
                               FP16 slices already carry 22 significant bits of
                               Delta (a TF32 value carries 11) */
} dpt_prec;

typedef struct {
  double tol;              /* stop when max_i rho_i <= tol, where
                              rho_i = ||M a_i - E_i a_i||_2 / (s ||a_i||_2),
                              s = max|theta| + |lambda| max_j sum_k |Delta_jk|.
                              Default 1e-12. */
  int32_t max_iter;        /* maximum map applications (default 200) */
  int32_t prec;            /* dpt_prec (default DPT_PREC_MIXED) */
  int32_t epstein_nesbet;  /* nonzero: move lambda*diag(Delta) into theta first
                              (the partition of Sec. II.H); same eigenpairs */
  int32_t graph_iters;     /* iterations per captured CUDA graph replay between
                              host convergence checks (default 4; 0 = no graph) */
  int32_t max_slices;      /* slices of Delta in the mixed path, 1..3 (default 3): FP16
                              slices (11 significant bits each); a real single solve
                              uses two for max_slices 2 or 3 (its FP64 finish covers
                              the columns two leave uncertain), grouped, served and
                              complex solves that many.  The first products use all of
                              them, and the slices represent Delta to about 2^-11
                              relative per slice: fewer bound the result's accuracy by
                              that representation (the carried remainder makes up for
                              the rounding of the increments, not for that of Delta) */
  int32_t profile;         /* nonzero: time every product kernel with CUDA events on
                              the stream it runs on (reported in dpt_info) */
  double slice_tol;        /* mixed path: the first product uses all its slices; a
                              later one drops a slice for each factor 2^-11 by which
                              its increment's largest entry is below the first
                              increment's, and uses one below slice_tol (default
                              1e-8) */
  int32_t cta_pair;        /* real mixed full solve: 1 (default) runs the product as
                              CTA pairs (tcgen05 cta_group::2, 256-row tiles split
                              over two SMs, epilogue inputs staged in the shared memory
                              this frees) where clusters of two can be resident; 2 as
                              clusters of four (two pairs on 512-row tiles sharing each
                              increment tile through TMA multicast; pairs where such
                              clusters cannot be resident; at n = 4096 on GB300 slower
                              than 1: 254 against 204 us per product); 0 one CTA per
                              128-row tile */
  int32_t grouped_form;    /* grouped solves, complex single solves and the server:
                              1 (what 0, the default, selects) one CTA per 128-row tile
                              with the epilogue reading global memory; 2 one CTA per
                              tile with the epilogue inputs staged in shared memory
                              (tiles at most 128 wide: faster for groups of small
                              problems); 3 CTA pairs (256-row tiles).  Results of one
                              problem are identical across entry points using the
                              same form. */
  double ramp_alpha;       /* 0 (default): the autonomous map.  In (0, 1): the
                              non-autonomous iteration of the Supplement's explicit
                              3x3 example, step k applying the map at
                              lambda (1 - ramp_alpha^k) (step 0 at strength 0), which
                              can reach fixed points the autonomous iteration from
                              the unperturbed vectors misses near the boundary of its
                              convergence domain; E, the residual and the stopping test
                              always refer to lambda.  Supported by both dominant
                              forms and by the real full solve in both precisions: the
                              mixed one forms each step's increment as
                              r G o R - (1 - r)(A - I), r = 1 - alpha^k, from the
                              residual R at lambda it carries (lambda (P - A diag P) =
                              R + Gap o A), and does not run the ramp's identity step
                              0 (it reports one map application fewer).  Complex mixed,
                              batched and served solves return DPT_ERR_UNSUPPORTED. */
  const double* start;     /* NULL (default): iterate from the unperturbed vectors
                              (A_0 = I, z_0 = e_{n*}).  Otherwise the starting iterate,
                              host or device: for the dominant forms n doubles; for
                              the full solve an n x n column-major matrix (complex
                              interleaved for DPT_C128) with leading dimension
                              ld_start.  Each vector is divided by its chart entry
                              (a_i[i], z[n*]), so any nonzero multiple of an
                              eigenvector estimate will do; a zero or non-finite
                              chart entry or a non-finite value gives DPT_ERR_ARG.
                              This is the polisher use of the closing remark of
                              Sec. II.H: approximate eigenvectors from another
                              method, refined by the map's final convergent steps.
                              Supported by both dominant forms and by the real full
                              solve in both precisions (the mixed one applies the
                              start's offset from I as its first increment, rounded
                              to FP16 like every increment, and counts that as a map
                              application); complex mixed, batched and served solves
                              return DPT_ERR_UNSUPPORTED. */
  int64_t ld_start;        /* leading dimension of a full-solve start (>= n) */
  int32_t certify;         /* mixed real full solve: nonzero (default) lets a product whose
                              iterate is predicted to pass the tolerance (the residual
                              falling geometrically below half of it) form only that
                              residual, writing no next iterate; if the iterate does not
                              pass after all, the same iteration runs again in full.
                              Results and iteration counts are those of 0, which always
                              runs the full map. */
  double refine_tol;       /* mixed real full solve: accuracy the eigenvectors must keep
                              against the mixed arithmetic (default 1e-10; <= 0: off).
                              The tensor-core products round to about 2^-24 of their
                              largest term and the gaps are float-float, so a column i
                              with a near-degenerate partner j (a large A_ji over a small
                              theta_i - theta_j) can land further from the fixed point
                              than the tolerance suggests.  After the mixed iteration the
                              solve estimates each column's error as
                              w_i (2^-22 |lambda| max|Delta| + 2^-46 max|theta|),
                              w_i = max_{j != i} |A_ji| / |theta_i - theta_j| (first from
                              a bound that costs nothing, then per column), and finishes
                              the columns above refine_tol with the plain FP64 map (FP64
                              gaps and products) on those columns only, until its step is
                              below refine_tol / 8 (each column is its own map,
                              Sec. II.B); dpt_info reports them. */
  int32_t pair_clusters;   /* mixed real full solve in the CTA-pair form: 0 (default)
                              runs as many clusters as can be resident; k > 0 at most k
                              (the tile schedule of a large problem on a small one:
                              several tiles per cluster and, where they cut the padding,
                              column tiles of two widths).  Results agree with the
                              default to rounding (the tiles' K orders differ). */
} dpt_options;

typedef struct {
  int32_t iters;           /* map applications before the returned iterate */
  int32_t slice_gemms;     /* mixed path: sum over iterations of the slices used */
  double residual;         /* max_i rho_i of the returned iterate, as tracked by
                              the iteration */
  int32_t status;          /* dpt_status of the solve */
  int32_t nstar;           /* dominant form: the eigenvector index used */
  double seconds;          /* wall time of the call */
  int32_t launches;        /* kernels this call launched (graph nodes included) */
  int32_t product_launches;  /* product kernels that did work (one per iteration) */
  double product_ms;       /* with opt->profile: summed device time of those
                              product kernels, else 0 */
  int32_t cta_pair;        /* mixed path: the product form that ran: 1 CTA pairs, 2
                              clusters of four, 0 one CTA per tile */
  int32_t grouped_form;    /* grouped solves: the product form that ran (see
                              dpt_options.grouped_form), else 0 */
  int32_t fp64_iters;      /* mixed real full solve: plain FP64 map steps (included in
                              iters) that finished a strongly coupled solve, whose
                              float recursion could not vouch for the tolerance
                              (2^-23 times the sum of its residuals above
                              max(tol, 1e-11)); 0 otherwise, and for n > 65535 (the
                              plain FP64 path's limit), where the mixed result is
                              returned as it is.  Also counts the FP64 steps that
                              finished the columns of refined_cols. */
  int32_t refined_cols;    /* mixed real full solve: columns finished with plain FP64 map
                              steps because their estimated error exceeded
                              dpt_options.refine_tol (n when the whole problem was
                              finished in FP64, see fp64_iters) */
} dpt_info;

/* Fill *opt with the defaults listed above. */
DPT_API void dpt_options_default(dpt_options* opt);

/* Human-readable name of a status code (static string). */
DPT_API const char* dpt_status_string(dpt_status s);

/* Full spectrum: all n eigenpairs of M = diag(theta) + lambda * Delta.
 *   n          matrix size, 1 <= n <= 2^20 (the mixed path's workspace, about 30
 *              bytes per element, bounds it in practice; the plain FP64 path returns
 *              DPT_ERR_TOO_LARGE beyond 65535)
 *   dtype      DPT_R64 or DPT_C128 (complex mixed solves run through the grouped path
 *              of dpt_solve_batched with one problem)
 *   theta      n doubles, pairwise distinct and finite
 *   delta      n x n, column-major, leading dimension ld_delta >= n, finite (the
 *              mixed path also rejects entries of magnitude 2^128 or more: its slices
 *              hold float-range values; DPT_ERR_ARG)
 *   lambda     real perturbation strength
 *   opt        options (NULL = defaults)
 *   A_out      n x n output, column-major, ld_a >= n: column i is the eigenvector
 *              continued from e_i, normalised so that A_out[i + i*ld_a] == 1
 *   E_out      n outputs: E_i = theta_i + lambda (Delta a_i)_i
 *   info       optional diagnostics
 * Returns DPT_OK when the tolerance was met.  DPT_ERR_MAXITER / DPT_ERR_DIVERGED
 * still write the last iterate and its eigenvalues.  Blocks until done. */
DPT_API dpt_status dpt_solve_full(int64_t n, dpt_dtype dtype, const double* theta,
                          const void* delta, int64_t ld_delta, double lambda,
                          const dpt_options* opt, void* A_out, int64_t ld_a,
                          void* E_out, dpt_info* info, void* stream);

/* Many independent full-spectrum problems in one grouped solve (mixed path): every
 * stage of an iteration is one launch over all problems' tiles, and each problem
 * stops at its own convergence (Sec. II.B: each problem is its own fixed-point
 * iteration).  Arrays of length count:
 *   dtype        DPT_R64, or DPT_C128 (Delta, A, E interleaved complex; theta, lambda real)
 *   n[p]         size of problem p, 1 <= n[p] <= 65536
 *   theta[p]     device pointer, n[p] distinct finite doubles
 *   delta[p]     device pointer, column-major n[p] x n[p], leading dimension ld_delta[p]
 *   lambda[p]    real perturbation strength
 *   A_out[p], E_out[p]   device outputs as for dpt_solve_full (leading dimension ld_a[p])
 *   infos[p]     optional per-problem diagnostics (status of each problem)
 * All pointers must be device pointers (DPT_ERR_UNSUPPORTED otherwise); only
 * opt->prec == DPT_PREC_MIXED without the Epstein-Nesbet shift is supported.
 * Returns DPT_OK when every problem converged, else the first failing problem's
 * status (infos[p] tells which).  Blocks until done. */
DPT_API dpt_status dpt_solve_batched(int64_t count, dpt_dtype dtype, const int64_t* n,
                                     const double* const* theta, const double* const* delta,
                                     const int64_t* ld_delta, const double* lambda,
                                     const dpt_options* opt, double* const* A_out,
                                     const int64_t* ld_a, double* const* E_out,
                                     dpt_info* infos, void* stream);

/* Tile-shape autotuner for grouped solves.  Runs the group twice with each form of the
 * grouped product (dpt_options.grouped_form 1: 128-row tiles up to 256 columns wide, the
 * epilogue reading its inputs from global memory; 2: 128-row tiles up to 128 wide with
 * the epilogue inputs staged in shared memory; 3: 256-row CTA-pair tiles up to 224 wide),
 * the first run untimed (it absorbs the form's one-time set-up costs), the second with
 * per-launch timing of its product kernels, and returns the form whose product
 * launches took the least device time in total.  Pass it as opt->grouped_form to later
 * dpt_solve_batched calls on groups like this one (a problem's result depends on the
 * form, through the tile boundaries of its accumulation order, within the tolerance).
 * Arguments as for dpt_solve_batched (opt->grouped_form and opt->profile are set here);
 * the outputs hold the converged result of the last form tried.
 *   best_form  out: 1, 2 or 3 (0 when no form converged)
 *   form_ms    optional out, 3 doubles: each form's summed product time in ms, or -1
 *              for a form that did not converge or ran as another form (form 3 runs
 *              as 2 where clusters of two cannot be resident)
 * Returns DPT_OK when some form converged for every problem, else the last form's
 * status (DPT_ERR_ARG / DPT_ERR_UNSUPPORTED at once).  Blocks until done. */
DPT_API dpt_status dpt_tune_batched(int64_t count, dpt_dtype dtype, const int64_t* n,
                                    const double* const* theta, const double* const* delta,
                                    const int64_t* ld_delta, const double* lambda,
                                    const dpt_options* opt, double* const* A_out,
                                    const int64_t* ld_a, double* const* E_out,
                                    int32_t* best_form, double* form_ms, void* stream);

/* Device workspace, in bytes, that one dpt_solve_full call of size n takes from the
 * library's pool with the default options and with theta, Delta, A and E in device
 * memory (host buffers add their staging copies: about 8 n^2 bytes each for Delta
 * and A, twice that for DPT_C128).  The pool keeps its blocks, grown to the largest
 * request so far, until dpt_release_workspace.  Mixed real: about 30 bytes per matrix
 * element (room for three FP16 slices of Delta, float-float A and its ping-pong copy,
 * FP16 increments, the carried remainder); plain FP64: 3 n^2 doubles (A, its ping-pong
 * copy and the product) per real component.  Host-only computation (no CUDA call);
 * -1 for n outside [1, 2^20] or an unknown dtype or prec. */
DPT_API int64_t dpt_workspace_bytes(int64_t n, dpt_dtype dtype, dpt_prec prec);

/* Dominant eigenvector: the eigenpair continued from e_{n*}, by the single-vector
 * map of Eq. (single_line_dyn) (Sec. II.H; for a perturbative matrix this is the
 * eigenvector of the largest eigenvalue when n* = argmax theta).
 *   n          size, 1 <= n < 2^31 - 1
 *   theta      n doubles, finite; theta_m != theta_{n*} for every m != n*
 *   row_ptr    n + 1 int32, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col_idx    nnz int32 in [0, n)          (CSR of Delta, rows m)
 *   vals       nnz float (FP32 values; used exactly, promoted to the working precision)
 *   nstar      eigenvector index, or -1 for the first index of max theta
 *   lambda     real perturbation strength
 *   opt        options (prec: DPT_PREC_MIXED = float-float working precision
 *              on the FP32 pipes, DPT_PREC_FP64 = plain FP64 arithmetic)
 *   z_out      n doubles: the eigenvector with z_out[n*] = 1
 *   E_out      one double: E = theta_{n*} + lambda (Delta z)_{n*}
 * Errors as for dpt_solve_full; a malformed CSR structure gives DPT_ERR_ARG
 * before any kernel follows it.  Blocks until done. */
DPT_API dpt_status dpt_solve_dominant(int64_t n, const double* theta, const int32_t* row_ptr,
                                      const int32_t* col_idx, const float* vals, int64_t nstar,
                                      double lambda, const dpt_options* opt, double* z_out,
                                      double* E_out, dpt_info* info, void* stream);

/* Rayleigh-Schroedinger partial sums, the comparator the paper sets DPT against
 * (Sec. II.D, Eq. (ARS-alpha); the recursion of Supplement B), in plain FP64:
 *     A_out = sum_{l=0}^{order} lambda^l C^(l),   E_out = theta + sum_{l=1}^{order} lambda^l eps^(l),
 *     C^(0) = I,  eps^(l)_i = (Delta C^(l-1))_ii,
 *     C^(l)_ji = ((Delta C^(l-1))_ji - sum_{s<l} C^(l-1-s)_ji eps^(s+1)_i) / (theta_i - theta_j),
 *     C^(l)_ii = 0.
 * One FP64 product per order plus an l-term convolution of the earlier orders, all
 * of which stay in device memory: (order + 3) n^2 doubles of workspace.
 *   theta, delta (column-major, ld_delta), A_out (ld_a), E_out: device pointers
 *   (DPT_ERR_UNSUPPORTED otherwise), real; 1 <= n <= 32768; 0 <= order <= 4096.
 * DPT_ERR_DEGENERATE when two theta coincide.  Blocks until done. */
DPT_API dpt_status dpt_rs_series(int64_t n, const double* theta, const double* delta,
                                 int64_t ld_delta, double lambda, int32_t order, double* A_out,
                                 int64_t ld_a, double* E_out, void* stream);

/* Homotopy continuation (the Discussion's extension of the convergence domain):
 * lambda is reached in `stages` equal steps.  After each step the problem is
 * re-expressed in the eigenbasis just found,
 *     W^T (M_q + (lambda/Q) Delta) V = diag(E_q) + (lambda/Q) W^T Delta V,
 * (V right and W left eigenvectors of M_q = diag(theta) + q (lambda/Q) Delta,
 * W^T V = I), and the map is iterated again from the identity: each stage is a
 * perturbation problem of strength lambda/Q around the previous eigenvalues, so
 * a lambda beyond the direct iteration's domain can be reached.  A stage is one
 * full solve for the right eigenvectors (opt->prec: mixed or plain FP64; a mixed
 * last stage is refined by the plain FP64 map started from its result) and, except
 * in the last stage, one on the transposed problem for the left ones.  The basis
 * changes are FP64 matrix products (six per stage, three in the last): the stage
 * matrix is the exact transform W^T M_{q+1} V, so errors of earlier stages enter
 * the next stage's perturbation instead of being lost, and one Newton-Schulz step
 * W <- W (2I - V^T W) keeps W^T V = I to working precision.
 *   n, theta, delta, ld_delta, lambda, A_out, ld_a, E_out   as for dpt_solve_full,
 *              real (DPT_R64) only, all four arrays device pointers
 *              (DPT_ERR_UNSUPPORTED otherwise), 1 <= n <= 32768
 *   stages     Q, 1..1024 (1 is the direct solve)
 *   opt        tol, max_iter, prec, max_slices, slice_tol, graph_iters apply to every
 *              stage solve; start, ramp_alpha and epstein_nesbet must be unset
 *              (DPT_ERR_UNSUPPORTED)
 * A_out columns are scaled to the chart of the original problem (A_ii = 1).  The
 * status is that of the first failing stage solve (DPT_ERR_DEGENERATE when two
 * eigenvalues of a stage coincide); DPT_ERR_DIVERGED when a basis vector has a
 * zero chart entry.  info->iters sums the iterations of all stage solves and
 * info->residual is the last stage's.  Blocks until done. */
DPT_API dpt_status dpt_solve_homotopy(int64_t n, const double* theta, const double* delta,
                                      int64_t ld_delta, double lambda, int32_t stages,
                                      const dpt_options* opt, double* A_out, int64_t ld_a,
                                      double* E_out, dpt_info* info, void* stream);

/* Dominant eigenvector with a dense perturbation: the map of dpt_solve_dominant
 * (Eq. (single_line_dyn), Sec. II.H) with y = Delta z formed by a GEMV.  Every
 * iteration streams Delta from device memory once (8 bytes per entry), so the
 * solve is bound by memory bandwidth.
 *   n          size, 1 <= n <= 2^20 (Delta must fit in device memory)
 *   theta      n doubles, finite; theta_m != theta_{n*} for every m != n*
 *   delta      column-major n x n FP64 (entry (m, k) at delta[m + k ld_delta]),
 *              host or device; a host matrix is first copied to the device
 *   ld_delta   leading dimension, >= n
 *   nstar, lambda, opt, z_out, E_out, info   as for dpt_solve_dominant
 *              (prec DPT_PREC_MIXED: each FP64 entry is split exactly enough
 *              into two floats and the products summed in float-float on the FP32
 *              pipes; DPT_PREC_FP64: plain FP64 arithmetic)
 * A non-finite entry of Delta gives DPT_ERR_ARG (detected during the first pass,
 * before any result is returned), and so does, in the float-float form only, an
 * entry of magnitude 2^128 or more (beyond the FP32 exponent range).  Blocks until
 * done. */
DPT_API dpt_status dpt_solve_dominant_dense(int64_t n, const double* theta, const double* delta,
                                            int64_t ld_delta, int64_t nstar, double lambda,
                                            const dpt_options* opt, double* z_out,
                                            double* E_out, dpt_info* info, void* stream);

/* dpt_solve_dominant for callers that cannot allocate device memory.  (This entry
 * point has no counterpart in the paper; it is a deployment variant of
 * dpt_solve_dominant.)
 *
 * Some callers may not call cudaMalloc at all: processes whose device memory is
 * entirely owned by a framework's caching allocator, and latency-critical loops
 * that must not take the driver's allocation path (cudaMalloc and cudaFree
 * synchronise the device).  The other entry points take their scratch from a pool
 * that grows with cudaMalloc; this one allocates nothing.  Its scratch is a fixed
 * 6.4 MB block of device memory built into the library, which every GPU that
 * loads the library holds until the process exits.
 *
 *   Limits: n <= 262144 rows (larger problems return DPT_ERR_TOO_LARGE at once);
 *   float-float working precision only (the default of dpt_solve_dominant).
 *   theta, row_ptr, col_idx, vals and z_out must be device pointers (there is no
 *   scratch to stage host buffers through); E_out may be host or device.
 *   Arguments otherwise as for dpt_solve_dominant; tol and max_iter replace the
 *   options struct.
 *   The call makes blocking CUDA runtime calls (copies and synchronisations on
 *   `stream`), so it must not be made from a host callback (cudaLaunchHostFunc).
 *   The first call on each device looks up the block's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture begins.
 *   All calls share the one block, which keeps the previous call's contents (each
 *   call rewrites everything it reads).  Calls whose GPU work overlaps — on
 *   different streams or from different threads — race on the block and give
 *   wrong results: issue them in order, e.g. on one stream.
 *   Work runs on `stream`; the call blocks until its results are ready. */
DPT_API dpt_status dpt_solve_dominant_noalloc(int64_t n, const double* theta,
                                              const int32_t* row_ptr, const int32_t* col_idx,
                                              const float* vals, int64_t nstar, double lambda,
                                              double tol, int32_t max_iter, double* z_out,
                                              double* E_out, dpt_info* info, void* stream);

/* ------------------------------------------------------------------------
 * Solve server: continuous batching of independent full-spectrum problems.
 *
 * A server owns one worker thread, one CUDA stream and a fixed budget of device
 * memory on the device current at dpt_server_create.  Requests (dpt_problem)
 * wait in a FIFO queue and are admitted while a slot is free and the budget holds
 * their working set; the worker then advances every admitted problem by one map
 * application per step (one grouped tcgen05 product launch over all of them, the
 * machinery of dpt_solve_batched), and retires each problem at its own
 * convergence (each problem is its own fixed-point iteration, Sec. II.B), writing
 * its outputs and freeing its memory for the queue.  A problem's arithmetic does
 * not depend on which other problems share its steps: its results are the same
 * alone and in any mix.  Mixed precision (DPT_PREC_MIXED) only.
 * ------------------------------------------------------------------------ */
typedef struct dpt_server dpt_server;
typedef int64_t dpt_req;

typedef struct {
  uint64_t hbm_budget;    /* device bytes for request working sets; 0 = 80% of the
                             free device memory at creation.  Allocated once, at
                             creation; admission never allocates. */
  int32_t max_active;     /* problems on the GPU at once (default 64, at most 4096) */
  int32_t max_queue;      /* queued requests beyond which dpt_submit returns
                             DPT_ERR_BUSY (default 65536) */
  dpt_options opt;        /* tol, max_iter, max_slices, slice_tol for requests that
                             do not set their own; prec must be DPT_PREC_MIXED and
                             ramp_alpha 0 */
} dpt_server_cfg;

typedef struct {
  int64_t n;              /* size, 1 <= n <= 65536 */
  int32_t dtype;          /* dpt_dtype */
  const double* theta;    /* n distinct finite doubles, host or device */
  const void* delta;      /* n x n column-major, leading dimension ld_delta, host or device */
  int64_t ld_delta;
  double lambda;          /* real perturbation strength */
  double tol;             /* <= 0: the server's */
  int32_t max_iter;       /* <= 0: the server's */
  void* A_out;            /* n x n column-major output (ld_a), host or device */
  int64_t ld_a;
  void* E_out;            /* n outputs, host or device */
} dpt_problem;

typedef struct {
  int64_t submitted, completed, failed, cancelled, rejected;
  int32_t queued, active;        /* right now */
  int32_t max_queued;            /* largest queue length seen */
  int64_t steps;                 /* grouped product steps run */
  uint64_t hbm_budget, hbm_in_use, hbm_peak;
  double p50_s, p99_s;           /* submit-to-result latency of completed requests */
} dpt_server_stats;

/* Fill *cfg with the defaults listed above. */
DPT_API void dpt_server_cfg_default(dpt_server_cfg* cfg);

/* Create a server on the current device (cfg NULL = defaults).  DPT_ERR_NOMEM
 * when the budget cannot be allocated; DPT_ERR_ARG for invalid settings. */
DPT_API dpt_status dpt_server_create(const dpt_server_cfg* cfg, dpt_server** out);

/* Queue one problem.  The descriptor is copied; the buffers it points to are not:
 * theta and delta must stay valid and unchanged, and A_out / E_out valid, until
 * dpt_poll or dpt_wait reports a final status.  Checks the arguments it can on the
 * host (DPT_ERR_ARG), rejects a problem whose working set exceeds the whole budget
 * (DPT_ERR_TOO_LARGE) and refuses when the queue is full (DPT_ERR_BUSY); nothing is
 * queued then.  Non-finite Delta entries and equal theta values are found on the
 * GPU and end only that request (DPT_ERR_ARG / DPT_ERR_DEGENERATE).  *id
 * identifies the request.  Thread-safe. */
DPT_API dpt_status dpt_submit(dpt_server* srv, const dpt_problem* prob, dpt_req* id);

/* Non-blocking: DPT_PENDING while the request is queued or running, else its final
 * status, with *info (optional) filled: iters, slice_gemms, residual, status, and
 * seconds = submit-to-result latency.  Once a final status has been returned the
 * request is forgotten and its id becomes invalid (DPT_ERR_ARG).  Thread-safe. */
DPT_API dpt_status dpt_poll(dpt_server* srv, dpt_req id, dpt_info* info);

/* As dpt_poll, but waits up to timeout_s seconds (< 0: no limit) for a final status. */
DPT_API dpt_status dpt_wait(dpt_server* srv, dpt_req id, double timeout_s, dpt_info* info);

/* Cancel a queued or running request: it ends with DPT_ERR_CANCELLED (outputs
 * unspecified) at the worker's next step boundary, unless it finishes first.  DPT_OK when the cancel was
 * recorded, DPT_ERR_ARG for an unknown or already finished id.  Thread-safe. */
DPT_API dpt_status dpt_cancel(dpt_server* srv, dpt_req id);

/* Counters and latency percentiles so far.  Thread-safe. */
DPT_API dpt_status dpt_server_stats_get(dpt_server* srv, dpt_server_stats* stats);

/* Stop the worker, end every unfinished request with DPT_ERR_CANCELLED, free the
 * budget.  Requests not yet polled are forgotten. */
DPT_API dpt_status dpt_server_destroy(dpt_server* srv);

/* Self-test of the bounded device waits (a deployment check; no counterpart in the
 * paper).  Every wait inside the library's kernels gives up after a time limit, sets a
 * flag the host reads and lets the kernel return, so a stalled pipeline ends as
 * DPT_ERR_TIMEOUT with the device still usable.  This call runs one kernel whose wait
 * can never complete (an mbarrier phase nobody arrives at) with a limit of `seconds`
 * (0 < seconds <= 5).  Returns DPT_ERR_TIMEOUT when the wait expired and the kernel
 * returned as designed (the expected result), DPT_ERR_ARG for a bad duration,
 * DPT_ERR_CUDA otherwise.  Blocks until done. */
DPT_API dpt_status dpt_selftest_bounded_wait(double seconds, void* stream);

/* Gather probe: a calibration of the CSR form's roofline (no counterpart in the
 * paper).  Each pass of dpt_solve_dominant streams the matrix and gathers one 8-byte
 * float pair of the iterate per nonzero at a random column; at the problem sizes of
 * interest the iterate lives in L2 and the gathers, not HBM, set the pace.  This call
 * runs a kernel with the pass's grid, row groups, index stream and gathers but none
 * of its arithmetic or value loads, `reps` times after one warm-up run, and returns
 * the mean device time of one pass (CUDA events on `stream`) in *ms_per_pass: the
 * fastest a pass with this access pattern can go on this GPU.
 *   n, row_ptr, col_idx   CSR structure as for dpt_solve_dominant (device pointers;
 *                         indices are clamped, not validated)
 *   z                     n interleaved float pairs (device), the gathered vector
 *   y                     n floats (device), written with the per-row sums
 * DPT_ERR_UNSUPPORTED for host pointers.  Blocks until done. */
DPT_API dpt_status dpt_probe_gather(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                    const void* z, float* y, int32_t reps, double* ms_per_pass,
                                    void* stream);

/* Free the scratch pool of the current device (no solve may be running). */
DPT_API void dpt_release_workspace(void);

#ifdef __cplusplus
}
#endif
#endif
