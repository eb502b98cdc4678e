// dpt_solve_dominant_noalloc: the dominant-eigenvector solve of dpt_solve_dominant
// for callers that cannot allocate device memory.
//
// Who needs it: a process whose device memory is fully reserved by another
// allocator (a framework's caching pool that owns the GPU's free memory), or a
// latency-critical loop that must not take the driver's allocation path (whose
// cudaMalloc / cudaFree calls synchronise the device).  The regular entry points
// draw their scratch from a pool that grows with cudaMalloc; this one uses a fixed
// block of device memory that is part of the library image instead.  It still makes
// ordinary blocking CUDA runtime calls (copies and stream synchronisations on the
// caller's stream), so it must not be called from a host callback
// (cudaLaunchHostFunc), where CUDA forbids runtime calls.
//
// The scratch block is a file-scope __device__ array of kScratchBytes bytes.  It
// is created when the library is loaded onto a device and stays resident on every
// GPU that loads the library until the process exits.  Host code cannot use the
// array's name as a device address (in host code the symbol is only a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress, with that device current, and caches it; make that first
// call before any stream capture begins.
//
// Every call shares the one block: two calls whose work overlaps on the GPU (on
// different streams, or from different threads) race on it and give wrong
// results.  Calls must be ordered, e.g. issued on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/dpt.h"
#include "dpt_internal.h"

namespace dpt {
namespace {

constexpr int64_t kMaxN = 1 << 18;                 // largest problem (rows) accepted
constexpr int64_t kPartBytes = 2 * 4096 * 8;       // block partials (2 doubles per block)
constexpr int64_t kStateBytes = 1024;              // DomState, padded
// theta float-float (2n floats) + z float-float ping-pong (4n floats)
constexpr int64_t kScratchBytes = kStateBytes + kPartBytes + 6 * kMaxN * 4;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static_assert(sizeof(DomState) <= kStateBytes, "state slot too small");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

dpt_status status_of(int s) {
  switch (s) {
    case ST_CONVERGED: return DPT_OK;
    case ST_MAXITER: return DPT_ERR_MAXITER;
    case ST_DIVERGED: return DPT_ERR_DIVERGED;
    case ST_TIMEOUT: return DPT_ERR_TIMEOUT;
    case ST_BADINPUT: return DPT_ERR_ARG;
    default: return DPT_ERR_CUDA;
  }
}

}  // namespace
}  // namespace dpt

using namespace dpt;

extern "C" dpt_status dpt_solve_dominant_noalloc(int64_t n, const double* theta,
                                                  const int32_t* row_ptr,
                                                  const int32_t* col_idx, const float* vals,
                                                  int64_t nstar, double lambda, double tol,
                                                  int32_t max_iter, double* z_out,
                                                  double* E_out, dpt_info* info,
                                                  void* stream) {
  if (info) { std::memset(info, 0, sizeof(*info)); info->status = DPT_ERR_ARG; info->nstar = -1; }
  auto done = [&](dpt_status st) {
    if (info) info->status = st;
    return st;
  };
  if (n < 1 || !theta || !row_ptr || !col_idx || !vals || !z_out || !E_out || nstar >= n ||
      !std::isfinite(lambda) || !(tol > 0) || max_iter < 0)
    return done(DPT_ERR_ARG);
  if (n > kMaxN) return done(DPT_ERR_TOO_LARGE);
  if (!on_device(theta) || !on_device(row_ptr) || !on_device(col_idx) || !on_device(vals) ||
      !on_device(z_out))
    return done(DPT_ERR_ARG);
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return done(DPT_ERR_CUDA);
  const int ni = (int)n;
  const int G = dom_blocks(ni);
  if ((int64_t)2 * G * 8 > kPartBytes) return done(DPT_ERR_TOO_LARGE);
  char* b = static_cast<char*>(base);
  DomState* st = reinterpret_cast<DomState*>(b);
  double* part = reinterpret_cast<double*>(b + kStateBytes);
  float* f = reinterpret_cast<float*>(b + kStateBytes + kPartBytes);
  float* thh = f;
  float* thl = f + n;
  float2* z0 = reinterpret_cast<float2*>(f + 2 * n);   // (hi, lo) pairs
  float2* z1 = reinterpret_cast<float2*>(f + 4 * n);

#define NA_CK(call)                                 \
  do {                                              \
    if ((call) != cudaSuccess) {                    \
      cudaStreamSynchronize(s);                     \
      return done(DPT_ERR_CUDA);                    \
    }                                               \
  } while (0)

  int32_t nnz32 = 0;
  NA_CK(cudaMemcpyAsync(&nnz32, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (nnz32 < 0) return done(DPT_ERR_ARG);

  // The block keeps the previous call's contents: the state (counters, flags,
  // scratch maxima) is rewritten in full here; theta, z and the partials are
  // fully written by the kernels before they are read.
  DomState h{};
  h.status = ST_RUNNING;
  h.max_iter = max_iter;
  h.nstar_req = nstar < 0 ? -1 : (int)nstar;
  h.nstar_min = 0x7fffffff;
  h.lam = lambda;
  h.lam_hi = (float)lambda;
  h.lam_lo = (float)(lambda - (double)h.lam_hi);
  h.tol = tol;
  h.best = INFINITY;
  NA_CK(cudaMemcpyAsync(st, &h, sizeof(DomState), cudaMemcpyHostToDevice, s));
  NA_CK(launch_dom_check(ni, nnz32, row_ptr, st, s));
  NA_CK(cudaMemcpyAsync(&h, st, sizeof(DomState), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (h.bad_input) return done(DPT_ERR_ARG);
  NA_CK(launch_dom_setup(ni, theta, thh, thl, st, s));
  NA_CK(cudaMemcpyAsync(&h, st, sizeof(DomState), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (h.bad_input) return done(DPT_ERR_ARG);
  if (h.ties != 1u) return done(DPT_ERR_DEGENERATE);
  NA_CK(launch_dom_init(ni, z0, nullptr, 1, st, s));
  const double avg = (double)nnz32 / (double)n;
  const int V = avg < 24 ? 4 : (avg < 48 ? 8 : (avg < 96 ? 16 : 32));
  // the first pass (k = 0) validates the CSR data and forms the residual scale
  NA_CK(launch_dom_iter(ni, V, 1, row_ptr, col_idx, vals, thh, thl, theta, z0, z1, nullptr,
                        nullptr, part, st, s, /*first=*/true));
  // plain launches (no graph: instantiating one may allocate), host check every 4
  const int per = 4;
  for (int c = 0; c <= max_iter / per + 1; ++c) {
    for (int q = 0; q < per; ++q)
      NA_CK(launch_dom_iter(ni, V, 1, row_ptr, col_idx, vals, thh, thl, theta, z0, z1, nullptr,
                            nullptr, part, st, s));
    NA_CK(cudaMemcpyAsync(&h, st, sizeof(DomState), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (h.status != ST_RUNNING) break;
  }
  NA_CK(launch_dom_out(ni, z0, z1, nullptr, nullptr, 1, z_out, st, s));
  NA_CK(cudaMemcpyAsync(&h, st, sizeof(DomState), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (on_device(E_out)) {
    // ordered on the caller's stream, like every other copy of this call
    NA_CK(cudaMemcpyAsync(E_out, &h.E, sizeof(double), cudaMemcpyHostToDevice, s));
    NA_CK(cudaStreamSynchronize(s));
  } else {
    *E_out = h.E;
  }
#undef NA_CK
  const dpt_status ret = status_of(h.status);
  if (info) {
    info->iters = h.k;
    info->residual = h.rho;
    info->nstar = h.nstar;
  }
  return done(ret);
}
