// Batched stepping of many grids of mixed size: every time step of every
// member is one launch of the step kernel over the concatenated work items
// (optionally persistent: a fixed number of blocks looping over the items),
// followed by one observation launch; k steps can be captured into a CUDA
// graph and replayed.  Members keep their own step counters and limits, so a
// member that reaches its limit stops being updated while the others go on.
//
// Paper: the realizations of the disorder studies (Sec. "Wide-band
// excitation and gap filling": results averaged over 10 realizations per
// disorder strength) are independent runs; here they share the GPU in one
// launch per step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_batch_internal.h"
#include "fdtd_internal.cuh"

namespace fdtd {

template <typename T>
struct BatchImpl final : BatchBase {
  StepGrid<T>* d_sg = nullptr;
  ObsGrid<T>* d_og = nullptr;
  TmaGrid* d_tma = nullptr;
  int4* d_items = nullptr;
  int4* d_oitems = nullptr;
  std::vector<int4> items, oitems;
  bool gain = false;
  bool pair = false;  // every member on the paired binary32 kernel
  int oy = 8;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_built_for = 0;

  ~BatchImpl() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
  }

  // Records of every member in the batch's own tables, items re-indexed.
  int build() override {
    const int ng = (int)grids.size();
    cudaError_t e;
    // order: members' pending work before the batch's
    for (GridBase* g : grids) {
      if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_error(e, "sync member");
    }
    gain = false;
    for (GridBase* g : grids) {
      g->kernel_kind = kernel_kind;
      g->bx = bx;
      g->by = by;
      g->zdepth = zdepth > 0 ? zdepth : 16;  // default: short z-ranges (balance across SMs)
      g->grid_blocks = 0;
      int r = g->finalized ? g->replan() : g->finalize();
      if (r != FDTD_OK) return r;
      g->finalized = true;
      gain = gain || g->has_gain();
    }
    // one launch serves all members: they must agree on the kernel and the
    // tile; members that differ fall back to the most general kernel used
    for (int round = 0; round < 3; ++round) {
      int lo = 3, hi = 1;
      for (GridBase* g : grids) {
        const int v = g->uses_pair() ? 3 : (g->uses_tma() ? 2 : 1);
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      bool rows_agree = true;
      for (GridBase* g : grids) rows_agree = rows_agree && g->tile_rows() == grids[0]->tile_rows();
      if (lo == hi && rows_agree) break;
      const int to = (lo == hi) ? 1 : lo;
      for (GridBase* g : grids) {
        g->kernel_kind = to;
        int r = g->replan();
        if (r != FDTD_OK) return r;
      }
    }
    tma = !grids.empty() && grids[0]->uses_tma();
    pair = !grids.empty() && grids[0]->uses_pair();
    oy = grids.empty() ? 8 : grids[0]->tile_rows();
    std::vector<StepGrid<T>> hsg(ng);
    std::vector<ObsGrid<T>> hog(ng);
    items.clear();
    oitems.clear();
    std::vector<std::pair<double, int4>> ranked;
    for (int q = 0; q < ng; ++q) {
      GridBase* g = grids[q];
      std::memcpy(&hsg[q], g->step_record(), sizeof(StepGrid<T>));
      std::memcpy(&hog[q], g->obs_record(), sizeof(ObsGrid<T>));
      hsg[q].step = hog[q].step = g->steps;
      hsg[q].step_end = hog[q].step_end = g->step_limit;
      std::vector<int4> si, oi;
      g->work_items(si, oi);
      // members' lists are ordered longest first; merge them by position so
      // the batch also issues its slab-heavy items first
      for (size_t r = 0; r < si.size(); ++r) {
        int4 it = si[r];
        it.x = q;
        ranked.push_back({(double)r / (double)si.size(), it});
      }
      for (auto it : oi) {
        it.x = q;
        oitems.push_back(it);
      }
    }
    std::stable_sort(ranked.begin(), ranked.end(),
                     [](const std::pair<double, int4>& a, const std::pair<double, int4>& b) { return a.first < b.first; });
    for (auto& w : ranked) items.push_back(w.second);
    mem.release_all();
    d_sg = (StepGrid<T>*)mem.get(sizeof(StepGrid<T>) * ng);
    d_og = (ObsGrid<T>*)mem.get(sizeof(ObsGrid<T>) * ng);
    d_tma = tma ? (TmaGrid*)mem.get(sizeof(TmaGrid) * ng) : nullptr;
    d_items = (int4*)mem.get(sizeof(int4) * std::max<size_t>(items.size(), 1));
    d_oitems = (int4*)mem.get(sizeof(int4) * std::max<size_t>(oitems.size(), 1));
    if (!d_sg || !d_og || (tma && !d_tma) || !d_items || !d_oitems)
      return set_error(FDTD_E_NOMEM, "device allocation failed (batch tables)");
    if ((e = cudaMemcpyAsync(d_sg, hsg.data(), sizeof(StepGrid<T>) * ng, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_og, hog.data(), sizeof(ObsGrid<T>) * ng, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload batch tables");
    if (tma)
      for (int q = 0; q < ng; ++q)
        if ((e = cudaMemcpyAsync(d_tma + q, grids[q]->tma_device(), sizeof(TmaGrid), cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
          return cuda_error(e, "copy tensor maps");
    if (!items.empty() &&
        (e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload items");
    if (!oitems.empty() &&
        (e = cudaMemcpyAsync(d_oitems, oitems.data(), sizeof(int4) * oitems.size(), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload items");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "build batch");
    if (gexec) {
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
    if (graph) {
      cudaGraphDestroy(graph);
      graph = nullptr;
    }
    graph_built_for = 0;
    dirty = false;
    return FDTD_OK;
  }

  size_t nitems() const override { return items.size(); }

  cudaError_t launch_one(int offset, bool timed) {
    cudaError_t e;
    const auto ev = timed ? timer.next() : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) cudaEventRecord(ev.first, stream);
    if (pair)
      // one block per item unless set: the members' items differ in cost,
      // and the hardware's block dispatch balances them better than a
      // persistent grid's fixed stride (measured)
      e = launch_step_pair(reinterpret_cast<const StepGrid<float>*>(d_sg), d_tma, d_items, (int)items.size(), offset,
                           oy, gain, grid_blocks > 0 ? grid_blocks : (int)items.size(), stream);
    else if (tma)
      e = launch_step_tma<T>(d_sg, d_tma, d_items, (int)items.size(), offset, oy, gain, grid_blocks, stream);
    else
      e = launch_step<T>(d_sg, d_items, (int)items.size(), offset, bx, oy + 1, gain, grid_blocks, stream);
    if (e != cudaSuccess) return e;
    if (ev.second) cudaEventRecord(ev.second, stream);
    if (!oitems.empty()) e = launch_observe<T>(d_og, d_oitems, (int)oitems.size(), offset, stream);
    return e;
  }

  int capture(int k) {
    cudaError_t e;
    if (gexec) {
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }
    if (graph) {
      cudaGraphDestroy(graph);
      graph = nullptr;
    }
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_error(e, "capture stream");
    cudaStream_t saved = stream;
    stream = cs;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int s = 0; s < k && e == cudaSuccess; ++s) e = launch_one(s, false);
      if (e == cudaSuccess) e = launch_advance<T>(d_sg, d_og, (int)grids.size(), k, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      if (e == cudaSuccess) e = e2;
    }
    stream = saved;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_error(e, "graph capture");
    }
    if ((e = cudaGraphInstantiate(&gexec, graph, 0)) != cudaSuccess) return cuda_error(e, "graph instantiate");
    graph_built_for = k;
    return FDTD_OK;
  }

  int step(long long n) override {
    cudaError_t e;
    if (dirty) {
      const int r = build();
      if (r != FDTD_OK) return r;
    }
    long long done = 0;
    if (graph_steps > 0 && !timer.on && n >= graph_steps) {
      if (graph_built_for != graph_steps) {
        const int r = capture(graph_steps);
        if (r != FDTD_OK) return r;
      }
      while (n - done >= graph_steps) {
        if ((e = cudaGraphLaunch(gexec, stream)) != cudaSuccess) return cuda_error(e, "graph launch");
        done += graph_steps;
      }
    }
    while (done < n) {
      const int chunk = (int)std::min<long long>(n - done, 1 << 20);
      for (int s = 0; s < chunk; ++s) {
        if ((e = launch_one(s, timer.on)) != cudaSuccess) return cuda_error(e, "batch step");
        if (timer.used >= 4096) {
          if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
          timer.collect();
        }
      }
      if ((e = launch_advance<T>(d_sg, d_og, (int)grids.size(), chunk, stream)) != cudaSuccess)
        return cuda_error(e, "advance");
      done += chunk;
    }
    // host mirrors of the members' counters; member streams wait for this work
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_error(e, "event");
    cudaEventRecord(ev, stream);
    for (GridBase* g : grids) {
      g->set_steps(std::min(g->step_limit, std::max(g->steps, g->steps + n)));
      g->tables_dirty = true;
      if (g->stream != stream) cudaStreamWaitEvent(g->stream, ev, 0);
    }
    cudaEventDestroy(ev);
    return FDTD_OK;
  }
};

BatchBase* make_batch(int precision) {
  if (precision == FDTD_FP32) return new (std::nothrow) BatchImpl<float>();
  return new (std::nothrow) BatchImpl<double>();
}

}  // namespace fdtd
