// Launch-shape autotuner: times candidate step kernels, tile rows and
// z-range depths on the grid (or batch) it tunes, each candidate for a few
// steps from the current state, restores the state after every trial, and
// keeps the fastest.  The paired and TMA kernels give bit-identical results,
// and the state is restored, so tuning does not change any result.
//
// Paper: none of this is in the paper (its code ran on CPU clusters); it
// serves the batched stepping of many disorder realizations (Sec. "Wide-band
// excitation and gap filling": averages over realizations).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_batch_internal.h"

namespace fdtd {
namespace {

struct Candidate {
  int kind, bx, by, zdepth, grid_blocks, order = FDTD_ORDER_COSTLIEST;
};

// Device copy of a grid's evolving state (fields, CPML and gain memory,
// recorder rings) and its step counter.
struct Snapshot {
  GridBase* g = nullptr;
  std::vector<std::pair<void*, size_t>> blobs;
  std::vector<void*> saved;
  long long steps = 0, limit = 0;
  int kind = 0, bx = 0, by = 0, zdepth = 0, grid_blocks = 0, order = 0;

  int take(GridBase* grid) {
    g = grid;
    g->state_blobs(blobs);
    steps = g->steps;
    limit = g->step_limit;
    kind = g->kernel_kind;
    bx = g->bx;
    by = g->by;
    zdepth = g->zdepth;
    grid_blocks = g->grid_blocks;
    order = g->item_order;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_error(e, "sync");
    for (auto& b : blobs) {
      void* p = nullptr;
      if ((e = cudaMalloc(&p, b.second)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FDTD_E_NOMEM, "autotune: no room for a copy of the state (%zu bytes)", b.second);
      }
      saved.push_back(p);
      if ((e = cudaMemcpyAsync(p, b.first, b.second, cudaMemcpyDeviceToDevice, g->stream)) != cudaSuccess)
        return cuda_error(e, "autotune: copy state");
    }
    return FDTD_OK;
  }
  int restore() {
    cudaError_t e;
    for (size_t q = 0; q < blobs.size(); ++q)
      if ((e = cudaMemcpyAsync(blobs[q].first, saved[q], blobs[q].second, cudaMemcpyDeviceToDevice, g->stream)) !=
          cudaSuccess)
        return cuda_error(e, "autotune: restore state");
    g->set_steps(steps);
    g->step_limit = limit;
    g->tables_dirty = true;
    return FDTD_OK;
  }
  void settings_back() {
    g->kernel_kind = kind;
    g->bx = bx;
    g->by = by;
    g->zdepth = zdepth;
    g->grid_blocks = grid_blocks;
    g->item_order = order;
  }
  ~Snapshot() {
    if (g) cudaStreamSynchronize(g->stream);
    for (void* p : saved) cudaFree(p);
  }
};

std::vector<Candidate> grid_candidates(const GridBase* g) {
  const fdtd_grid_desc& d = g->desc;
  std::vector<Candidate> c;
  if (g->absorber == FDTD_ABSORBER_UPML) return {{1, 32, 8, 0, 0}};  // one launch shape: the UPML launches
  if (d.periodic[0] || d.periodic[1] || d.periodic[2]) {
    c = {{1, 32, 8, 0, 0}, {1, 32, 4, 0, 0}, {1, 64, 4, 0, 0}, {1, 32, 16, 0, 0}};
  } else if (g->precision() == FDTD_FP32) {
    c = {{3, 32, 16, 0, 0}, {3, 32, 8, 0, 0}, {3, 32, 16, 8, 0}, {3, 32, 8, 8, 0}, {2, 32, 8, 0, 0},
         {2, 32, 4, 0, 0},  {2, 32, 8, 8, 0}, {2, 32, 8, 24, 0}};
  } else {
    c = {{2, 32, 8, 0, 0}, {2, 32, 4, 0, 0}, {2, 32, 8, 8, 0}, {2, 32, 4, 16, 0}, {2, 32, 8, 24, 0}};
  }
  // the single-node kernels' items also in plain z order
  const size_t n0 = c.size();
  for (size_t q = 0; q < n0; ++q)
    if (c[q].kind == 2) {
      Candidate z = c[q];
      z.order = FDTD_ORDER_Z;
      c.push_back(z);
    }
  return c;
}

// Mean time of one step over `trial` steps after two warm-up steps.
int time_steps(cudaStream_t st, long long trial, const std::function<int(long long)>& step, double* ms) {
  int r = step(2);
  if (r != FDTD_OK) return r;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  r = step(trial);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (r != FDTD_OK) return r;
  if (e != cudaSuccess) return cuda_error(e, "autotune: timing");
  *ms = (double)t / (double)trial;
  return FDTD_OK;
}

}  // namespace
}  // namespace fdtd

extern "C" {

int fdtd_autotune(fdtd_grid* g, int32_t trial_steps, fdtd_tune_result* out) {
  using namespace fdtd;
  try {
    if (!g || !g->impl) return set_error(FDTD_E_INVAL, "null grid");
    if (trial_steps < 1) return set_error(FDTD_E_INVAL, "trial_steps must be >= 1");
    GridBase* G = g->impl;
    if (!G->finalized) {
      const int r = G->finalize();
      if (r != FDTD_OK) return r;
      G->finalized = true;
    }
    Snapshot snap;
    int r = snap.take(G);
    if (r != FDTD_OK) return r;
    const bool timing = G->timer.on;
    G->timer.on = false;
    G->step_limit = 0x7fffffffffffffffLL;
    const std::vector<Candidate> cands = grid_candidates(G);
    int best = -1;
    double best_ms = 0.0;
    for (size_t q = 0; q < cands.size(); ++q) {
      const Candidate& c = cands[q];
      G->kernel_kind = c.kind;
      G->bx = c.bx;
      G->by = c.by;
      G->zdepth = c.zdepth;
      G->grid_blocks = c.grid_blocks;
      G->item_order = c.order;
      if ((r = G->replan()) != FDTD_OK) break;
      double ms = 0.0;
      r = time_steps(G->stream, trial_steps, [&](long long n) { return G->step(n); }, &ms);
      if (r != FDTD_OK) break;
      if ((r = snap.restore()) != FDTD_OK) break;
      G->step_limit = 0x7fffffffffffffffLL;
      if (best < 0 || ms < best_ms) {
        best = (int)q;
        best_ms = ms;
      }
    }
    G->timer.on = timing;
    if (r != FDTD_OK || best < 0) {
      snap.restore();
      snap.settings_back();
      G->replan();
      return r != FDTD_OK ? r : set_error(FDTD_E_STATE, "autotune: no candidate ran");
    }
    const Candidate& c = cands[best];
    G->kernel_kind = c.kind;
    G->bx = c.bx;
    G->by = c.by;
    G->zdepth = c.zdepth;
    G->grid_blocks = c.grid_blocks;
    G->item_order = c.order;
    if ((r = snap.restore()) != FDTD_OK) return r;
    if ((r = G->replan()) != FDTD_OK) return r;
    if (out) {
      out->kernel = c.kind;
      out->bx = c.bx;
      out->by = c.by;
      out->zdepth = c.zdepth;
      out->grid_blocks = c.grid_blocks;
      out->ms_per_step = best_ms;
      out->candidates = (int32_t)cands.size();
      out->order = c.order;
    }
    return FDTD_OK;
  } catch (...) {
    return set_error(FDTD_E_NOMEM, "autotune: host allocation failed");
  }
}

int fdtd_batch_autotune(fdtd_batch* b, int32_t trial_steps, fdtd_tune_result* out) {
  using namespace fdtd;
  try {
    if (!b || !b->impl) return set_error(FDTD_E_INVAL, "null batch");
    if (trial_steps < 1) return set_error(FDTD_E_INVAL, "trial_steps must be >= 1");
    BatchBase* B = b->impl;
    std::vector<std::unique_ptr<Snapshot>> snaps;
    int r = FDTD_OK;
    if (B->dirty && (r = B->build()) != FDTD_OK) return r;
    for (GridBase* g : B->grids) {
      snaps.emplace_back(new Snapshot());
      if ((r = snaps.back()->take(g)) != FDTD_OK) return r;
    }
    auto restore_all = [&]() {
      int rr = FDTD_OK;
      for (auto& s : snaps) {
        const int x = s->restore();
        if (rr == FDTD_OK) rr = x;
      }
      cudaError_t e = cudaStreamSynchronize(B->stream);
      if (rr == FDTD_OK && e != cudaSuccess) rr = cuda_error(e, "sync");
      return rr;
    };
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    const bool gain = std::any_of(B->grids.begin(), B->grids.end(), [](GridBase* g) { return g->has_gain() != 0; });
    std::vector<Candidate> cands = {{0, 32, 0, 0, 0}, {0, 32, 0, 24, 0}, {0, 32, 0, 8, 0},      {2, 32, 8, 0, 0},
                                    {2, 32, 4, 0, 0}, {2, 32, 8, 8, 0},  {2, 32, 8, 0, 2 * sms}, {2, 32, 8, 24, 0}};
    if (B->grids.front()->precision() == FDTD_FP32) {
      cands.push_back({3, 32, 16, 0, 0});
      cands.push_back({3, 32, 16, 8, 0});
      cands.push_back({3, 32, 8, 0, 0});
    }
    const int kind0 = B->kernel_kind, by0 = B->by, zd0 = B->zdepth, gb0 = B->grid_blocks, graph0 = B->graph_steps;
    const bool timing = B->timer.on;
    B->timer.on = false;
    B->graph_steps = 0;
    for (GridBase* g : B->grids) g->step_limit = 0x7fffffffffffffffLL;
    int best = -1;
    double best_ms = 0.0;
    for (size_t q = 0; q < cands.size() && r == FDTD_OK; ++q) {
      const Candidate& c = cands[q];
      B->kernel_kind = c.kind;
      B->by = c.by;
      B->zdepth = c.zdepth;
      B->grid_blocks = c.grid_blocks;
      B->dirty = true;
      double ms = 0.0;
      r = time_steps(B->stream, trial_steps, [&](long long n) { return B->step(n); }, &ms);
      const int rr = restore_all();
      if (r == FDTD_OK) r = rr;
      for (GridBase* g : B->grids) g->step_limit = 0x7fffffffffffffffLL;
      if (r == FDTD_OK && (best < 0 || ms < best_ms)) {
        best = (int)q;
        best_ms = ms;
      }
    }
    B->timer.on = timing;
    B->graph_steps = graph0;
    if (r != FDTD_OK || best < 0) {
      restore_all();
      B->kernel_kind = kind0;
      B->by = by0;
      B->zdepth = zd0;
      B->grid_blocks = gb0;
      B->dirty = true;
      return r != FDTD_OK ? r : set_error(FDTD_E_STATE, "autotune: no candidate ran");
    }
    const Candidate& c = cands[best];
    B->kernel_kind = c.kind;
    B->by = c.by;
    B->zdepth = c.zdepth;
    B->grid_blocks = c.grid_blocks;
    B->dirty = true;
    if ((r = restore_all()) != FDTD_OK) return r;
    if (out) {
      out->kernel = c.kind;
      out->bx = 32;
      out->by = c.by;
      out->zdepth = c.zdepth;
      out->grid_blocks = c.grid_blocks;
      out->ms_per_step = best_ms;
      out->candidates = (int32_t)cands.size();
      out->order = FDTD_ORDER_COSTLIEST;
    }
    return FDTD_OK;
  } catch (...) {
    return set_error(FDTD_E_NOMEM, "autotune: host allocation failed");
  }
}

}  // extern "C"
