// Host-side batch object behind the opaque fdtd_batch handle.
#pragma once

#include <vector>

#include "fdtd_api_internal.h"

namespace fdtd {

struct BatchBase {
  std::vector<GridBase*> grids;  // members (not owned)
  cudaStream_t stream = nullptr;
  DeviceMemory mem;
  LaunchTimer timer;
  int kernel_kind = 0, bx = 32, by = 0, zdepth = 0, grid_blocks = 0, graph_steps = 0;
  bool tma = false;
  bool dirty = true;  // tables must be rebuilt before the next step

  virtual ~BatchBase() { mem.release_all(); }
  virtual int build() = 0;
  virtual int step(long long n) = 0;
  virtual size_t nitems() const = 0;
};

BatchBase* make_batch(int precision);

}  // namespace fdtd

struct fdtd_batch {
  fdtd::BatchBase* impl;
};
