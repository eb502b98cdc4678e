// Solve server: continuous batching of independent full-spectrum DPT problems on
// one GPU, driving the grouped mixed path (dpt_grouped.cu) one step at a time.
//
// One worker thread owns a CUDA stream, a device table of max_active problem
// slots and one device allocation of hbm_budget bytes, which a first-fit range
// allocator (dpt_sched.h) divides among the admitted requests.  Each pass of its
// loop:
//   1. cancels: requests cancelled while on the GPU are stopped on the device and
//      their slot and memory are freed;
//   2. admission (FIFO): while the queue head fits -- a free slot and a free range
//      of its working-set size -- lay out its arena, stage host inputs, upload its
//      table entry and state, and run its preparation, iteration 0 and first
//      control on the stream;
//   3. one step: the grouped product over the tiles of every admitted problem
//      (one launch per element kind) and the control kernels, which advance or
//      stop each problem on the device (each problem is its own fixed-point
//      iteration, arXiv:2002.12872 Sec. II.B);
//   4. the slot states come back to the host; every problem that stopped is
//      finalised (outputs written), its range and slot are freed and its waiters
//      woken.
// Nothing in a problem's arithmetic depends on the other problems of its steps
// (tile shapes, partial sums and decisions are per problem), so its results are
// the same alone and in any mix.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dpt.h"
#include "dpt_host.h"
#include "dpt_internal.h"
#include "dpt_sched.h"

namespace dpt {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { RQ_QUEUED, RQ_ACTIVE, RQ_DONE };

struct Request {
  dpt_req id = 0;
  dpt_problem p{};
  int cplx = 0;
  bool th_host = false, d_host = false, a_host = false, e_host = false;
  size_t plan_bytes = 0;
  uint64_t bytes = 0;            // working set: plan + staging + work lists
  ReqState state = RQ_QUEUED;
  bool cancel = false;
  dpt_status status = DPT_PENDING;
  dpt_info info{};
  Clock::time_point t_submit;
  // while on the GPU
  int slot = -1;
  uint64_t off = 0;
  GProb P{};
  IterState st0{};
  int4* blk = nullptr;
  int nblk = 0;
  std::vector<int4> items_h;     // host copy of the work lists until the stream syncs
  double* A_stage = nullptr;
  double* E_stage = nullptr;
  int tiles = 0;                 // product tiles per step
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace dpt

using namespace dpt;

struct dpt_server {
  int dev = 0;
  dpt_server_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<dpt_req, Request*> reqs;
  std::vector<Request*> slots;            // active request per slot (nullptr = free)
  std::thread worker;
  bool stop = false;
  dpt_status fatal = DPT_OK;
  dpt_req next_id = 1;
  // device
  char* arena = nullptr;
  RangeAllocator alloc;
  GProb* probs_dev = nullptr;
  IterState* states_dev = nullptr;
  int* flags_dev = nullptr;               // [0] running count (unused), [1] timeout flag
  int2* tiles_dev[2] = {nullptr, nullptr};
  size_t tiles_cap[2] = {0, 0};
  std::vector<int2> tiles_h[2];
  IterState* states_host = nullptr;       // pinned
  int* flags_host = nullptr;              // pinned
  cudaStream_t s = nullptr;
  bool tiles_dirty = true;
  int ntiles[2] = {0, 0};
  int form = G_PLAIN;                     // product form (GForm)
  int npairs = 0;                         // CTA pairs of the pair form
  // statistics (under mu)
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0, steps = 0;
  int32_t max_queued = 0;
  std::vector<double> lat;
};

namespace {

void set_done(dpt_server* S, Request* r, dpt_status st) {
  // caller holds S->mu
  r->state = RQ_DONE;
  r->status = st;
  r->info.status = st;
  r->info.nstar = -1;
  r->info.seconds = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  if (st == DPT_OK) {
    ++S->completed;
    S->lat.push_back(r->info.seconds);
  } else if (st == DPT_ERR_CANCELLED) {
    ++S->cancelled;
  } else {
    ++S->failed;
  }
}

// Frees the slot and the range of a request that left the GPU (holds S->mu).
void release_slot(dpt_server* S, Request* r) {
  if (r->slot >= 0) {
    S->slots[r->slot] = nullptr;
    S->alloc.free(r->off);
    r->slot = -1;
    S->tiles_dirty = true;
  }
}

// Lays out the request's arena and launches its first stage (S->mu not held; the
// request's slot and range are already reserved).
void admit(dpt_server* S, Request* r) {
  const dpt_options& o = S->cfg.opt;
  const int64_t n = r->p.n;
  const int w = r->cplx ? 2 : 1;
  Carve c{S->arena + r->off};
  char* plan_base = c.take<char>(r->plan_bytes);
  const double* th = r->p.theta;
  const double* dl = static_cast<const double*>(r->p.delta);
  int64_t ldd = r->p.ld_delta;
  double* A = static_cast<double*>(r->p.A_out);
  int64_t lda = r->p.ld_a;
  double* E = static_cast<double*>(r->p.E_out);
  if (r->th_host) {
    double* t = c.take<double>(n);
    CK(cudaMemcpyAsync(t, r->p.theta, sizeof(double) * n, cudaMemcpyHostToDevice, S->s));
    th = t;
  }
  if (r->d_host) {
    double* d = c.take<double>((size_t)w * n * n);
    CK(cudaMemcpy2DAsync(d, sizeof(double) * w * n, r->p.delta, sizeof(double) * w * r->p.ld_delta,
                         sizeof(double) * w * n, n, cudaMemcpyHostToDevice, S->s));
    dl = d;
    ldd = n;
  }
  if (r->a_host) {
    r->A_stage = c.take<double>((size_t)w * n * n);
    A = r->A_stage;
    lda = n;
  }
  if (r->e_host) {
    r->E_stage = c.take<double>((size_t)w * n);
    E = r->E_stage;
  }
  GroupPlan g;
  const double lam = r->p.lambda;
  plan_group(g, 1, r->cplx, &n, &th, &dl, &ldd, &lam, &A, &lda, &E, plan_base,
             S->states_dev + r->slot, S->form);
  GProb& P = g.probs[0];
  P.tmA = make_tmap_f16(P.Dcat, (uint64_t)3 * P.ld, P.nr, (uint64_t)3 * P.ld, 128);
  for (int q = 0; q < 2; ++q)
    P.tmB[q] = make_tmap_f16(P.dt[q], P.nr, P.n, P.ld, gform_box(S->form, P.bn));
  r->P = P;
  r->tiles = (int)g.tiles.size();
  const std::vector<int4>& prep = r->cplx ? g.prep_c : g.prep_r;
  const std::vector<int4>& blk = r->cplx ? g.blk_c : g.blk_r;
  const int nprep = (int)prep.size();
  r->nblk = (int)blk.size();
  // prep items then block items, contiguous on both sides
  r->items_h.assign(prep.begin(), prep.end());
  r->items_h.insert(r->items_h.end(), blk.begin(), blk.end());
  int4* prep_dev = c.take<int4>(nprep);
  r->blk = c.take<int4>(r->nblk);
  IterState& h = r->st0;
  h = IterState{};
  h.status = ST_RUNNING;
  h.max_iter = r->p.max_iter > 0 ? r->p.max_iter : o.max_iter;
  // up to three FP16 slices of Delta 2^sig (see dpt_grouped.cu)
  h.max_slices = o.max_slices;
  h.slices = h.max_slices;
  h.lam = lam;
  h.tol = r->p.tol > 0 ? r->p.tol : o.tol;
  h.slice_tol = o.slice_tol;
  h.best = INFINITY;
  GProb* Pd = S->probs_dev + r->slot;
  // every host source lives in the request until the stream has synchronised
  CK(cudaMemcpyAsync(Pd, &r->P, sizeof(GProb), cudaMemcpyHostToDevice, S->s));
  CK(cudaMemcpyAsync(S->states_dev + r->slot, &r->st0, sizeof(IterState), cudaMemcpyHostToDevice,
                     S->s));
  if (nprep) CK(cudaMemcpyAsync(prep_dev, r->items_h.data(), sizeof(int4) * nprep,
                                cudaMemcpyHostToDevice, S->s));
  if (r->nblk) CK(cudaMemcpyAsync(r->blk, r->items_h.data() + nprep, sizeof(int4) * r->nblk,
                                  cudaMemcpyHostToDevice, S->s));
  CK(launch_g_check_theta(Pd, 1, (int)n, S->flags_dev, S->s));
  CK(launch_g_scales(Pd, r->blk, r->nblk, r->cplx != 0, S->s));
  if (r->cplx) {
    CK(launch_gc_prep(Pd, prep_dev, nprep, S->s));
    CK(launch_gc_iter0(Pd, r->blk, r->nblk, S->s));
    CK(launch_g_ctrl(Pd, 1, (int)n, true, S->flags_dev, S->s));
  } else {
    CK(launch_g_prep(Pd, prep_dev, nprep, S->s));
    CK(launch_g_iter0(Pd, r->blk, r->nblk, S->s));
    CK(launch_g_ctrl(Pd, 1, (int)n, false, S->flags_dev, S->s));
  }
}

void upload_tiles(dpt_server* S) {
  std::vector<int2>* t = S->tiles_h;     // kept until the stream has synchronised
  t[0].clear();
  t[1].clear();
  std::vector<GProb> tab(S->slots.size());
  for (size_t q = 0; q < S->slots.size(); ++q) {
    const Request* r = S->slots[q];
    if (!r) continue;
    tab[q] = r->P;
    for (int i = 0; i < r->tiles; ++i) t[r->cplx].push_back(make_int2((int)q, i));
  }
  sort_tiles(t[0], tab.data());
  sort_tiles(t[1], tab.data());
  for (int k = 0; k < 2; ++k) {
    S->ntiles[k] = (int)t[k].size();
    if (t[k].empty()) continue;
    if (t[k].size() > S->tiles_cap[k]) {
      // growth only: at most a few times over a server's life
      CK(cudaStreamSynchronize(S->s));
      if (S->tiles_dev[k]) CK(cudaFree(S->tiles_dev[k]));
      S->tiles_dev[k] = nullptr;
      const size_t cap = t[k].size() * 2;
      if (cudaMalloc(&S->tiles_dev[k], sizeof(int2) * cap) != cudaSuccess) {
        cudaGetLastError();
        S->tiles_cap[k] = 0;
        throw Fail{DPT_ERR_NOMEM};
      }
      S->tiles_cap[k] = cap;
    }
    CK(cudaMemcpyAsync(S->tiles_dev[k], t[k].data(), sizeof(int2) * t[k].size(),
                       cudaMemcpyHostToDevice, S->s));
  }
  S->tiles_dirty = false;
}

// Ends every unfinished request with `st` (holds S->mu).
void fail_all(dpt_server* S, dpt_status st) {
  for (Request*& r : S->slots)
    if (r) {
      Request* q = r;
      release_slot(S, q);
      set_done(S, q, st);
    }
  while (!S->queue.empty()) {
    set_done(S, S->queue.front(), st);
    S->queue.pop_front();
  }
  S->cv_done.notify_all();
}

void worker_loop(dpt_server* S) {
  cudaSetDevice(S->dev);
  static const int kCancelled = ST_CANCELLED;
  std::vector<Request*> admitted, retired;
  while (true) {
    admitted.clear();
    retired.clear();
    int hi = 0;     // slots [0, hi) hold every active request
    {
      std::unique_lock<std::mutex> lk(S->mu);
      auto idle = [&] {
        for (Request* r : S->slots) if (r) return false;
        return true;
      };
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !idle(); });
      if (S->stop) return;
      // cancels of requests on the GPU
      for (Request* r : S->slots)
        if (r && r->cancel) retired.push_back(r);
      for (Request* r : retired) {
        cudaMemcpyAsync(&S->states_dev[r->slot].status, &kCancelled, sizeof(int),
                        cudaMemcpyHostToDevice, S->s);
        release_slot(S, r);
        set_done(S, r, DPT_ERR_CANCELLED);
      }
      if (!retired.empty()) S->cv_done.notify_all();
      retired.clear();
      // FIFO admission while the head fits
      while (!S->queue.empty()) {
        Request* r = S->queue.front();
        int slot = -1;
        for (size_t q = 0; q < S->slots.size(); ++q)
          if (!S->slots[q]) { slot = (int)q; break; }
        if (slot < 0) break;
        uint64_t off;
        if (!S->alloc.alloc(r->bytes, &off)) break;
        S->queue.pop_front();
        r->slot = slot;
        r->off = off;
        r->state = RQ_ACTIVE;
        S->slots[slot] = r;
        S->tiles_dirty = true;
        admitted.push_back(r);
      }
      for (size_t q = 0; q < S->slots.size(); ++q)
        if (S->slots[q]) hi = (int)q + 1;
    }
    try {
      for (Request* r : admitted) {
        try {
          admit(S, r);
        } catch (Fail f) {
          if (cudaPeekAtLastError() != cudaSuccess) throw;
          std::lock_guard<std::mutex> lk(S->mu);
          release_slot(S, r);
          set_done(S, r, f.st);
          S->cv_done.notify_all();
        }
      }
      if (hi == 0) continue;
      if (S->tiles_dirty) upload_tiles(S);
      bool kind[2] = {false, false};
      int max_n[2] = {0, 0};
      for (int q = 0; q < hi; ++q)
        if (const Request* r = S->slots[q]) {
          kind[r->cplx] = true;
          max_n[r->cplx] = std::max(max_n[r->cplx], (int)r->p.n);
        }
      for (int k = 0; k < 2; ++k)
        if (S->ntiles[k])
          CK(launch_gform(S->form, S->probs_dev, S->tiles_dev[k], S->ntiles[k],
                          (unsigned*)(S->flags_dev + 1), k == 1, S->npairs, S->s));
      if (kind[0]) CK(launch_g_ctrl(S->probs_dev, hi, max_n[0], false, S->flags_dev, S->s));
      if (kind[1]) CK(launch_g_ctrl(S->probs_dev, hi, max_n[1], true, S->flags_dev, S->s));
      CK(cudaMemcpyAsync(S->states_host, S->states_dev, sizeof(IterState) * hi,
                         cudaMemcpyDeviceToHost, S->s));
      CK(cudaMemcpyAsync(S->flags_host, S->flags_dev, sizeof(int) * 2, cudaMemcpyDeviceToHost,
                         S->s));
      CK(cudaStreamSynchronize(S->s));
      if (S->flags_host[1]) throw Fail{DPT_ERR_TIMEOUT};
      {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->steps;
      }
      // retire the problems that stopped
      for (int q = 0; q < hi; ++q) {
        Request* r = S->slots[q];
        if (!r) continue;
        const IterState& h = S->states_host[q];
        if (h.status == ST_RUNNING) continue;
        r->info.iters = h.k;
        r->info.slice_gemms = h.slice_gemms;
        r->info.residual = h.rho;
        r->info.product_launches = h.k;
        r->status = from_state(h.status);
        const bool outputs = h.status == ST_CONVERGED || h.status == ST_MAXITER ||
                             h.status == ST_DIVERGED;
        if (outputs) {
          const int64_t n = r->p.n;
          const int w = r->cplx ? 2 : 1;
          if (r->cplx) CK(launch_gc_finalize(S->probs_dev + q, r->blk, r->nblk, S->s));
          else CK(launch_g_finalize(S->probs_dev + q, r->blk, r->nblk, S->s));
          if (r->a_host)
            CK(cudaMemcpy2DAsync(r->p.A_out, sizeof(double) * w * r->p.ld_a, r->A_stage,
                                 sizeof(double) * w * n, sizeof(double) * w * n, n,
                                 cudaMemcpyDeviceToHost, S->s));
          if (r->e_host)
            CK(cudaMemcpyAsync(r->p.E_out, r->E_stage, sizeof(double) * w * n,
                               cudaMemcpyDeviceToHost, S->s));
        }
        retired.push_back(r);
      }
      if (!retired.empty()) {
        CK(cudaStreamSynchronize(S->s));
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* r : retired) {
          release_slot(S, r);
          set_done(S, r, r->status);
        }
        S->cv_done.notify_all();
      }
    } catch (Fail f) {
      cudaStreamSynchronize(S->s);
      std::lock_guard<std::mutex> lk(S->mu);
      S->fatal = f.st == DPT_OK ? DPT_ERR_CUDA : f.st;
      fail_all(S, S->fatal);
      return;
    }
  }
}

bool is_finite(double x) { return std::isfinite(x); }

}  // namespace

extern "C" {

void dpt_server_cfg_default(dpt_server_cfg* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->hbm_budget = 0;
  cfg->max_active = 64;
  cfg->max_queue = 65536;
  dpt_options_default(&cfg->opt);
}

dpt_status dpt_server_create(const dpt_server_cfg* cfg_in, dpt_server** out) {
  if (!out) return DPT_ERR_ARG;
  *out = nullptr;
  dpt_server_cfg cfg;
  dpt_server_cfg_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_active < 1 || cfg.max_active > 4096 || cfg.max_queue < 0 ||
      cfg.opt.prec != DPT_PREC_MIXED || cfg.opt.epstein_nesbet || !(cfg.opt.tol > 0) ||
      cfg.opt.max_iter < 0 || cfg.opt.max_slices < 1 || cfg.opt.max_slices > 3 ||
      cfg.opt.ramp_alpha != 0.0 || cfg.opt.start)
    return DPT_ERR_ARG;
  dpt_server* S = new (std::nothrow) dpt_server();
  if (!S) return DPT_ERR_NOMEM;
  S->cfg = cfg;
  dpt_status ret = DPT_OK;
  try {
    CK(cudaGetDevice(&S->dev));
    size_t freeb = 0, total = 0;
    CK(cudaMemGetInfo(&freeb, &total));
    uint64_t budget = cfg.hbm_budget ? cfg.hbm_budget : (uint64_t)(0.8 * (double)freeb);
    budget = budget / 256 * 256;
    if (budget == 0) throw Fail{DPT_ERR_ARG};
    if (cudaMalloc(&S->arena, budget) != cudaSuccess) {
      cudaGetLastError();
      S->arena = nullptr;
      throw Fail{DPT_ERR_NOMEM};
    }
    S->cfg.hbm_budget = budget;
    S->alloc.reset(budget);
    const int m = cfg.max_active;
    S->slots.assign(m, nullptr);
    CK(cudaMalloc(&S->probs_dev, sizeof(GProb) * m));
    CK(cudaMalloc(&S->states_dev, sizeof(IterState) * m));
    CK(cudaMalloc(&S->flags_dev, sizeof(int) * 4));
    CK(cudaHostAlloc((void**)&S->states_host, sizeof(IterState) * m, cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&S->flags_host, sizeof(int) * 4, cudaHostAllocDefault));
    CK(cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking));
    CK(g_set_attributes());
    S->form = choose_gform(cfg.opt.grouped_form, 0, nullptr, &S->npairs);
    // idle slots: a valid table entry whose state is not running
    std::vector<GProb> p0(m);
    std::vector<IterState> s0(m);
    for (int q = 0; q < m; ++q) {
      p0[q] = GProb{};
      p0[q].st = S->states_dev + q;
      s0[q] = IterState{};
      s0[q].status = ST_IDLE;
    }
    CK(cudaMemcpy(S->probs_dev, p0.data(), sizeof(GProb) * m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(S->states_dev, s0.data(), sizeof(IterState) * m, cudaMemcpyHostToDevice));
    CK(cudaMemset(S->flags_dev, 0, sizeof(int) * 4));
    S->worker = std::thread(worker_loop, S);
  } catch (Fail f) {
    ret = f.st;
  } catch (...) {
    ret = DPT_ERR_NOMEM;
  }
  if (ret != DPT_OK) {
    if (S->arena) cudaFree(S->arena);
    if (S->probs_dev) cudaFree(S->probs_dev);
    if (S->states_dev) cudaFree(S->states_dev);
    if (S->flags_dev) cudaFree(S->flags_dev);
    if (S->states_host) cudaFreeHost(S->states_host);
    if (S->flags_host) cudaFreeHost(S->flags_host);
    if (S->s) cudaStreamDestroy(S->s);
    delete S;
    return ret;
  }
  *out = S;
  return DPT_OK;
}

dpt_status dpt_submit(dpt_server* S, const dpt_problem* prob, dpt_req* id) {
  if (!S || !prob || !id) return DPT_ERR_ARG;
  const dpt_problem& p = *prob;
  auto reject = [&](dpt_status st) {
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->rejected;
    return st;
  };
  if (p.n < 1 || p.n > 65536 || (p.dtype != DPT_R64 && p.dtype != DPT_C128) || !p.theta ||
      !p.delta || !p.A_out || !p.E_out || p.ld_delta < p.n || p.ld_a < p.n ||
      !is_finite(p.lambda) || !(p.tol <= 0 || is_finite(p.tol)))
    return reject(DPT_ERR_ARG);
  Request* r = new (std::nothrow) Request();
  if (!r) return reject(DPT_ERR_NOMEM);
  r->p = p;
  r->cplx = p.dtype == DPT_C128 ? 1 : 0;
  r->th_host = !is_device_ptr(p.theta);
  r->d_host = !is_device_ptr(p.delta);
  r->a_host = !is_device_ptr(p.A_out);
  r->e_host = !is_device_ptr(p.E_out);
  // working set: the grouped layout of this one problem plus staging and work lists
  GroupPlan g;
  const int64_t n = p.n;
  const double* th = nullptr;
  const double* dl = nullptr;
  double* A = nullptr;
  double* E = nullptr;
  const int64_t ld = n;
  const double lam = p.lambda;
  plan_group(g, 1, r->cplx, &n, &th, &dl, &ld, &lam, &A, &ld, &E, nullptr, nullptr, G_PLAIN);
  const int w = r->cplx ? 2 : 1;
  r->plan_bytes = g.bytes;
  size_t b = al256(g.bytes);
  if (r->th_host) b += al256(sizeof(double) * n);
  if (r->d_host) b += al256(sizeof(double) * w * n * n);
  if (r->a_host) b += al256(sizeof(double) * w * n * n);
  if (r->e_host) b += al256(sizeof(double) * w * n);
  b += al256(sizeof(int4) * (r->cplx ? g.prep_c.size() : g.prep_r.size()));
  b += al256(sizeof(int4) * (r->cplx ? g.blk_c.size() : g.blk_r.size()));
  r->bytes = b + 256;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->fatal != DPT_OK) {
    delete r;
    ++S->rejected;
    return S->fatal;
  }
  if (S->alloc.footprint(r->bytes) > S->alloc.capacity()) {
    delete r;
    ++S->rejected;
    return DPT_ERR_TOO_LARGE;
  }
  if ((int64_t)S->queue.size() >= S->cfg.max_queue) {
    delete r;
    ++S->rejected;
    return DPT_ERR_BUSY;
  }
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  S->reqs[r->id] = r;
  S->queue.push_back(r);
  ++S->submitted;
  S->max_queued = std::max<int32_t>(S->max_queued, (int32_t)S->queue.size());
  *id = r->id;
  S->cv_work.notify_one();
  return DPT_OK;
}

static dpt_status take_result(dpt_server* S, std::unordered_map<dpt_req, Request*>::iterator it,
                              dpt_info* info) {
  // caller holds S->mu; the request is done
  Request* r = it->second;
  const dpt_status st = r->status;
  if (info) *info = r->info;
  S->reqs.erase(it);
  delete r;
  return st;
}

dpt_status dpt_poll(dpt_server* S, dpt_req id, dpt_info* info) {
  if (!S) return DPT_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return DPT_ERR_ARG;
  if (it->second->state != RQ_DONE) return DPT_PENDING;
  return take_result(S, it, info);
}

dpt_status dpt_wait(dpt_server* S, dpt_req id, double timeout_s, dpt_info* info) {
  if (!S) return DPT_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return DPT_ERR_ARG;
  Request* r = it->second;
  auto done = [&] { return r->state == RQ_DONE; };
  if (timeout_s < 0) S->cv_done.wait(lk, done);
  else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done))
    return DPT_PENDING;
  return take_result(S, S->reqs.find(id), info);
}

dpt_status dpt_cancel(dpt_server* S, dpt_req id) {
  if (!S) return DPT_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end() || it->second->state == RQ_DONE) return DPT_ERR_ARG;
  Request* r = it->second;
  if (r->state == RQ_QUEUED) {
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
      if (*q == r) { S->queue.erase(q); break; }
    set_done(S, r, DPT_ERR_CANCELLED);
    S->cv_done.notify_all();
  } else {
    r->cancel = true;
    S->cv_work.notify_one();
  }
  return DPT_OK;
}

dpt_status dpt_server_stats_get(dpt_server* S, dpt_server_stats* st) {
  if (!S || !st) return DPT_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->cancelled = S->cancelled;
  st->rejected = S->rejected;
  st->queued = (int32_t)S->queue.size();
  for (Request* r : S->slots) if (r) ++st->active;
  st->max_queued = S->max_queued;
  st->steps = S->steps;
  st->hbm_budget = S->alloc.capacity();
  st->hbm_in_use = S->alloc.in_use();
  st->hbm_peak = S->alloc.peak();
  st->p50_s = percentile(S->lat, 0.50);
  st->p99_s = percentile(S->lat, 0.99);
  return DPT_OK;
}

dpt_status dpt_server_destroy(dpt_server* S) {
  if (!S) return DPT_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->dev);
  cudaStreamSynchronize(S->s);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    fail_all(S, DPT_ERR_CANCELLED);
    for (auto& kv : S->reqs) delete kv.second;
    S->reqs.clear();
  }
  cudaFree(S->arena);
  cudaFree(S->probs_dev);
  cudaFree(S->states_dev);
  cudaFree(S->flags_dev);
  for (int k = 0; k < 2; ++k) if (S->tiles_dev[k]) cudaFree(S->tiles_dev[k]);
  cudaFreeHost(S->states_host);
  cudaFreeHost(S->flags_host);
  cudaStreamDestroy(S->s);
  cudaSetDevice(prev);
  delete S;
  return DPT_OK;
}

}  // extern "C"
