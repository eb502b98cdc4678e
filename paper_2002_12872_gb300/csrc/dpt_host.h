// Host-side helpers shared by the C-ABI translation units: error propagation,
// pointer classification, workspace carving, TMA descriptor encoding and the
// layout of a grouped (multi-problem) solve.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "../../include/dpt.h"
#include "dpt_internal.h"

namespace dpt {

// Thrown inside the host runtime, caught at the C-ABI boundary.
struct Fail {
  dpt_status st;
};

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) throw ::dpt::Fail{DPT_ERR_CUDA};   \
  } while (0)

inline bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Bump allocator over a scratch block (256-byte alignment); base == nullptr
// only measures.
struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (size_t)round_up((int64_t)off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};
template <class F>
size_t measure(F&& f) {
  Carve c{nullptr};
  f(c);
  return (size_t)round_up((int64_t)c.off, 256) + 256;
}

// 2-D tensor map of FP16 elements: inner extent `inner` (contiguous), outer extent
// `outer`, row pitch `pitch_elems`, box 64 x box_rows, 128-byte swizzle.  Throws Fail.
CUtensorMap make_tmap_f16(const void* base, uint64_t inner, uint64_t outer,
                          uint64_t pitch_elems, uint32_t box_rows);
// 2-D FP64 tensor map (column-major, even pitch), 16 x 16 boxes, 128-byte swizzle.
CUtensorMap make_tmap_f64(const void* base, uint64_t inner, uint64_t outer,
                          uint64_t pitch_elems);

// dpt_status of a device-side ST_* code.
dpt_status from_state(int s);

// Column-tile width of the grouped product for a problem of n columns.
int group_tile_n(int n, int wmax);

// Layout of a grouped solve: per-problem tables and the flat work lists.
struct GroupPlan {
  std::vector<GProb> probs;
  std::vector<int2> tiles;      // product kernel: (problem, tile)
  std::vector<int4> prep_r;     // real: (problem, col block, row block) 64 x 32
  std::vector<int4> prep_c;     // complex: (problem, col block, row block) 32 x 32 complex
  std::vector<int4> blk_r;      // real: (problem, col tile, row tile) 128 x 128
  std::vector<int4> blk_c;      // complex: (problem, col tile, embedded-row tile) 128 x 128
  size_t bytes = 0;
};

// Lays out every problem's work arrays in one arena at `base` (nullptr: size
// only) and fills g.  states_dev + p becomes problem p's IterState.
// Forms of the grouped product kernel: tile rows, largest tile width and the rows
// of the increment descriptor's box.
enum GForm { G_PLAIN = 1, G_STAGED = 2, G_PAIR = 3 };
inline int gform_rows(int f) { return f == G_PAIR ? 256 : 128; }
inline int gform_wmax(int f) { return f == G_PAIR ? 224 : (f == G_STAGED ? 128 : 256); }
inline int gform_box(int f, int bn) { return f == G_PAIR ? bn / 2 : bn; }

void plan_group(GroupPlan& g, int count, int cplx, const int64_t* n, const double* const* theta,
                const double* const* delta, const int64_t* ld_delta, const double* lambda,
                double* const* A_out, const int64_t* ld_a, double* const* E_out, char* base,
                IterState* states_dev, int form);

// The product form for a group (opt_form 0: chosen from the sizes) and, for the pair
// form, the number of CTA pairs; launches one product step of a group.
int choose_gform(int opt_form, int count, const int64_t* n, int* npairs);
cudaError_t launch_gform(int form, const GProb* probs, const int2* tiles, int ntiles,
                         unsigned* timeout, bool cplx, int npairs, cudaStream_t s);

// Re-lays a plan's arrays out at `base` (same order as plan_group), states at
// states_dev + p; the work lists are unchanged.
void place_group(GroupPlan& g, char* base, IterState* states_dev);

// Runs enc(p) for every problem on a few host threads (descriptor encoding).
void encode_group_maps(const GProb* probs, int count, const std::function<void(int)>& enc);

// Orders a product tile list (problem, tile) by decreasing cost.
void sort_tiles(std::vector<int2>& tiles, const GProb* probs);

}  // namespace dpt
