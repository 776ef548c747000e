// Batched stepping of many grids of mixed size: every time step of every
// member is one launch of each step kernel in use over the concatenated work
// items of its members (optionally persistent: a fixed number of blocks
// looping over the items), followed by one observation launch; k steps can be captured into a CUDA
// graph and replayed.  Members keep their own step counters and limits, so a
// member that reaches its limit stops being updated while the others go on.
//
// Paper: the realizations of the disorder studies (Sec. "Wide-band
// excitation and gap filling": ten of them are averaged for each disorder
// strength) are independent runs; here they share the GPU in one launch per
// step.
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
  // Members stepped by one kernel: the paired kernel (kind 3), the TMA
  // kernel (2) or the plain-load kernel (1), each with one tile shape.
  struct Group {
    bool gain = false;
    int oy = 8;  // tile rows (TMA kernels) or rows of the plain kernel's tile less its halo row
    std::vector<int4> items;
    int4* d_items = nullptr;
  };
  StepGrid<T>* d_sg = nullptr;
  ObsGrid<T>* d_og = nullptr;
  TmaGrid* d_tma = nullptr;
  int4* d_oitems = nullptr;
  std::vector<int4> oitems;
  Group groups[4];  // by kernel kind (index 0 unused)
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_built_for = 0;
  // second stream for the TMA group when the paired group runs too: the two
  // launches of a step overlap (one kernel's blocks fill the SMs that the
  // other's tail leaves idle)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ObsOverlap obs;  // observation launches beside the next step's launches
  bool beside = false;  // every member on the paired kernel: observation on the side stream

  ~BatchImpl() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }

  static int kind_of(const GridBase* g) { return g->uses_pair() ? 3 : (g->uses_tma() ? 2 : 1); }

  // Records of every member in the batch's own tables, items re-indexed and
  // grouped by the members' kernels (kernel 0: each member's automatic
  // choice, so passive binary32 members take the paired kernel and gain
  // members the TMA kernel, one launch each per time step).
  int build() override {
    const int ng = (int)grids.size();
    cudaError_t e;
    // order: members' pending work before the batch's
    for (GridBase* g : grids) {
      if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) return cuda_error(e, "sync member");
    }
    for (GridBase* g : grids) {
      g->kernel_kind = kernel_kind;
      g->bx = bx;
      g->by = by;
      g->zdepth = zdepth > 0 ? zdepth : 16;  // default: short z-ranges (balance across SMs)
      g->grid_blocks = 0;
      int r = g->finalized ? g->replan() : g->finalize();
      if (r != FDTD_OK) return r;
      g->finalized = true;
    }
    // one launch per kernel serves its members: they must share the tile;
    // a member whose rows differ from the first of its kernel's takes the
    // plain-load kernel (whose tile the batch sets for all its members)
    for (GridBase* g : grids) {
      const int k = kind_of(g);
      if (k == 1) continue;
      const GridBase* first = nullptr;
      for (GridBase* h : grids)
        if (kind_of(h) == k) {
          first = h;
          break;
        }
      if (g->tile_rows() != first->tile_rows()) {
        g->kernel_kind = 1;
        int r = g->replan();
        if (r != FDTD_OK) return r;
      }
    }
    tma = false;
    for (Group& gr : groups) {
      gr.gain = false;
      gr.items.clear();
      gr.d_items = nullptr;
    }
    for (GridBase* g : grids) {
      Group& gr = groups[kind_of(g)];
      gr.gain = gr.gain || g->has_gain();
      gr.oy = g->tile_rows();
      tma = tma || g->uses_tma();
    }
    std::vector<StepGrid<T>> hsg(ng);
    std::vector<ObsGrid<T>> hog(ng);
    oitems.clear();
    std::vector<std::pair<double, int4>> ranked[4];
    for (int q = 0; q < ng; ++q) {
      GridBase* g = grids[q];
      std::memcpy(&hsg[q], g->step_record(), sizeof(StepGrid<T>));
      std::memcpy(&hog[q], g->obs_record(), sizeof(ObsGrid<T>));
      hsg[q].step = hog[q].step = g->steps;
      hsg[q].step_end = hog[q].step_end = g->step_limit;
      hsg[q].wait_ns = g->wait_ns;
      std::vector<int4> si, oi;
      g->work_items(si, oi);
      // members' lists are ordered longest first; merge them by position so
      // the batch also issues its slab-heavy items first
      for (size_t r = 0; r < si.size(); ++r) {
        int4 it = si[r];
        it.x = q;
        ranked[kind_of(g)].push_back({(double)r / (double)si.size(), it});
      }
      for (auto it : oi) {
        it.x = q;
        oitems.push_back(it);
      }
    }
    for (int k = 1; k <= 3; ++k) {
      std::stable_sort(ranked[k].begin(), ranked[k].end(),
                       [](const std::pair<double, int4>& a, const std::pair<double, int4>& b) { return a.first < b.first; });
      for (auto& w : ranked[k]) groups[k].items.push_back(w.second);
    }
    mem.release_all();
    d_sg = (StepGrid<T>*)mem.get(sizeof(StepGrid<T>) * ng);
    d_og = (ObsGrid<T>*)mem.get(sizeof(ObsGrid<T>) * ng);
    d_tma = tma ? (TmaGrid*)mem.get(sizeof(TmaGrid) * ng) : nullptr;
    d_oitems = (int4*)mem.get(sizeof(int4) * std::max<size_t>(oitems.size(), 1));
    bool ok = d_sg && d_og && (!tma || d_tma) && d_oitems;
    for (int k = 1; k <= 3 && ok; ++k)
      if (!groups[k].items.empty()) ok = (groups[k].d_items = (int4*)mem.get(sizeof(int4) * groups[k].items.size())) != nullptr;
    if (!ok) return set_error(FDTD_E_NOMEM, "device allocation failed (batch tables)");
    if ((e = cudaMemcpyAsync(d_sg, hsg.data(), sizeof(StepGrid<T>) * ng, cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_og, hog.data(), sizeof(ObsGrid<T>) * ng, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload batch tables");
    if (tma)
      for (int q = 0; q < ng; ++q)
        if (grids[q]->uses_tma() &&
            (e = cudaMemcpyAsync(d_tma + q, grids[q]->tma_device(), sizeof(TmaGrid), cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
          return cuda_error(e, "copy tensor maps");
    for (int k = 1; k <= 3; ++k)
      if (!groups[k].items.empty() &&
          (e = cudaMemcpyAsync(groups[k].d_items, groups[k].items.data(), sizeof(int4) * groups[k].items.size(),
                               cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_error(e, "upload items");
    if (!oitems.empty() &&
        (e = cudaMemcpyAsync(d_oitems, oitems.data(), sizeof(int4) * oitems.size(), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload items");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "build batch");
    beside = !oitems.empty() && groups[1].items.empty() && groups[2].items.empty();
    for (int q = 0; q < ng; ++q) beside = beside && hsg[q].nsets == 3;  // three field sets in every member
    if (beside && (e = obs.ensure()) != cudaSuccess) return cuda_error(e, "observation stream");
    if (!groups[3].items.empty() && !groups[2].items.empty() && !side) {
      if ((e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_error(e, "batch side stream");
    }
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

  size_t nitems() const override { return groups[1].items.size() + groups[2].items.size() + groups[3].items.size(); }

  // One time step of every member: one launch per kernel group (paired,
  // TMA, plain-load), then the observation launch on its own stream.
  cudaError_t launch_one(int offset, bool timed) {
    cudaError_t e = cudaSuccess;
    if (beside && (e = obs.before_step(stream, offset)) != cudaSuccess) return e;
    const auto ev = timed ? timer.next() : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) cudaEventRecord(ev.first, stream);
    const Group& gp = groups[3];
    const Group& gt = groups[2];
    const bool two = side && !gp.items.empty() && !gt.items.empty();
    if (two) {
      if ((e = cudaEventRecord(fork, stream)) != cudaSuccess || (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess)
        return e;
    }
    if (!gp.items.empty())
      // one block per item unless set: the members' items differ in cost,
      // and the hardware's block dispatch balances them better than a
      // persistent grid's fixed stride (measured)
      e = launch_step_pair(reinterpret_cast<const StepGrid<float>*>(d_sg), d_tma, gp.d_items, (int)gp.items.size(),
                           offset, gp.oy, gp.gain, grid_blocks > 0 ? grid_blocks : (int)gp.items.size(), stream);
    if (e == cudaSuccess && !gt.items.empty())
      e = launch_step_tma<T>(d_sg, d_tma, gt.d_items, (int)gt.items.size(), offset, gt.oy, gt.gain, grid_blocks,
                             two ? side : stream);
    if (two) {
      const cudaError_t e2 = cudaEventRecord(join, side);
      const cudaError_t e3 = cudaStreamWaitEvent(stream, join, 0);
      if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    }
    const Group& gl = groups[1];
    if (e == cudaSuccess && !gl.items.empty())
      e = launch_step<T>(d_sg, gl.d_items, (int)gl.items.size(), offset, bx, gl.oy + 1, gl.gain, grid_blocks, stream);
    if (e != cudaSuccess) return e;
    if (ev.second) cudaEventRecord(ev.second, stream);
    if (beside)
      e = obs.observe(stream, offset, [&](cudaStream_t st) {
        return launch_observe<T>(d_og, d_oitems, (int)oitems.size(), offset, st);
      });
    else if (!oitems.empty())
      e = launch_observe<T>(d_og, d_oitems, (int)oitems.size(), offset, stream);
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
      if (e == cudaSuccess && beside) e = obs.join(cs, k);
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
    if (!stream_capturing(stream)) l2_claim(nullptr);  // no grid's CPML memory keeps L2 while the batch steps
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
      if (beside && (e = obs.join(stream, chunk)) != cudaSuccess) return cuda_error(e, "order");
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
