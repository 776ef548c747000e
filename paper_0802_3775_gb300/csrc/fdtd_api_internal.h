// Host-side grid object behind the opaque fdtd_grid handle.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fdtd.h"

namespace fdtd {

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* where);
extern thread_local std::string g_last_error;

// Device allocations of one owner, released together.
struct DeviceMemory {
  fdtd_allocator alloc{nullptr, nullptr, nullptr};
  void* stream = nullptr;
  std::vector<std::pair<void*, size_t>> blocks;
  void* get(size_t bytes);
  void release_all();
  size_t total() const;
};

// Event pairs bracketing kernel launches (optional per-launch timing).
struct LaunchTimer {
  bool on = false;
  int stride = 1;       // bracket every stride-th launch
  long long seen = 0;   // launches since timing was switched on
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  size_t used = 0;
  double ms = 0.0;
  long long launches = 0;
  ~LaunchTimer() {
    for (auto& e : pool) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  }
  // events for the next launch (nullptr pair when off)
  std::pair<cudaEvent_t, cudaEvent_t> next() {
    if (!on) return {nullptr, nullptr};
    if ((seen++ % stride) != 0) return {nullptr, nullptr};
    if (used == pool.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return {nullptr, nullptr};
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return {nullptr, nullptr};
      }
      pool.push_back({a, b});
    }
    return pool[used++];
  }
  // fold the recorded pairs into the totals (caller synchronized the stream)
  void collect() {
    for (size_t q = 0; q < used; ++q) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pool[q].first, pool[q].second) == cudaSuccess) {
        ms += t;
        launches++;
      }
    }
    used = 0;
  }
};

// Observation launches on a side stream.  With three field sets the
// observation of step s (sets s%3 and (s+1)%3) runs while step s+1 writes the
// third set; step s+2, which writes set s%3 again, and the step-counter update
// wait for it.  Within a chunk of steps s = 0, 1, ...; join() ends a chunk.
// Used for the paired kernel (persistent: an observation block fits beside
// its two resident blocks per SM); beside the TMA kernel, whose four blocks
// per SM fill the register file, the observation blocks took step blocks'
// places and the step ran slower than with the observation in line (140^3
// gain grid 0.1227 -> 0.1260 ms per step, measured).  There the observation
// stays in line and the next step's blocks start without waiting for it.
struct ObsOverlap {
  cudaStream_t side = nullptr;
  cudaEvent_t stepped = nullptr, done[2] = {nullptr, nullptr};

  cudaError_t ensure() {
    cudaError_t e = cudaSuccess;
    if (!side && (e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!stepped && (e = cudaEventCreateWithFlags(&stepped, cudaEventDisableTiming)) != cudaSuccess) return e;
    for (auto& d : done)
      if (!d && (e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming)) != cudaSuccess) return e;
    return e;
  }
  // before step s of a chunk: the observation of step s-2 has finished
  cudaError_t before_step(cudaStream_t main, int s) const {
    return s >= 2 ? cudaStreamWaitEvent(main, done[s & 1], 0) : cudaSuccess;
  }
  // after step s was enqueued on `main`: enqueue its observation on the side stream
  template <typename Launch>
  cudaError_t observe(cudaStream_t main, int s, Launch launch) {
    cudaError_t e;
    if ((e = cudaEventRecord(stepped, main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side, stepped, 0)) != cudaSuccess) return e;
    if ((e = launch(side)) != cudaSuccess) return e;
    return cudaEventRecord(done[s & 1], side);
  }
  // `main` waits for every observation enqueued so far (the last two of the chunk)
  cudaError_t join(cudaStream_t main, int steps_in_chunk) const {
    cudaError_t e = cudaSuccess;
    for (int s = steps_in_chunk - 2; s < steps_in_chunk && e == cudaSuccess; ++s)
      if (s >= 0) e = cudaStreamWaitEvent(main, done[s & 1], 0);
    return e;
  }
  ~ObsOverlap() {
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    if (stepped) cudaEventDestroy(stepped);
    for (auto& d : done)
      if (d) cudaEventDestroy(d);
  }
};

// Precision-independent interface of a grid; GridImpl<T> implements it.
struct GridBase {
  fdtd_grid_desc desc{};
  cudaStream_t stream = nullptr;
  DeviceMemory mem;
  long long ncell = 0;   // nx * ny * nz
  int px = 0;            // x pitch of the device arrays (nx rounded up to 16)
  long long nstore = 0;  // px * ny * nz
  int kernel_kind = 0;   // 0 auto, 1 plain loads, 2 TMA, 3 paired TMA (binary32)
  long long steps = 0;
  double S = 0, dx = 0, dt = 0;
  bool material_set = false;
  bool finalized = false;
  int bx = 32, by = 0, zdepth = 0, grid_blocks = 0;  // by == 0: the step kernel's default tile rows
  uint8_t* d_mat = nullptr;
  LaunchTimer timer;
  long long step_limit = 0x7fffffffffffffffLL;  // no update n >= step_limit
  long long wait_ns = 2000000000LL;              // limit of the TMA step kernels' bounded waits
  int coupling = 0;                              // FDTD_COUPLING_CELL or FDTD_COUPLING_CENTRED
  int item_order = 0;                            // FDTD_ORDER_COSTLIEST or FDTD_ORDER_Z
  int absorber = 0;                              // FDTD_ABSORBER_CPML or FDTD_ABSORBER_UPML
  int l2_resident = 1;                           // keep the CPML memory in a persisting L2 window
  bool l2_applied = false;                       // the window is set on the grid's stream
  virtual int kernel_in_use_kind() const { return 0; }
  bool tables_dirty = false;                     // device records stale (stepped by a batch)

  // Set (on) or clear (off) the persisting L2 window of the CPML memory on
  // the grid's stream; no-op for a grid without CPML memory.
  virtual int apply_l2_window(bool on) { (void)on; return FDTD_OK; }
  virtual ~GridBase() { mem.release_all(); }
  virtual int precision() const = 0;
  virtual size_t word() const = 0;
  virtual int set_gain(const fdtd_gain_params& p) = 0;
  virtual int add_source(const fdtd_source_desc& s) = 0;
  virtual int add_probe(int i, int j, int k) = 0;
  virtual int add_flux(int axis, int index, double sign, int u0, int u1, int v0, int v1) = 0;
  virtual int finalize() = 0;
  virtual int replan() = 0;
  virtual int step(long long n) = 0;
  virtual int read_field(int comp, double* out) = 0;
  virtual int write_field(int comp, const double* in) = 0;
  virtual int read_gain(int what, double* out) = 0;
  virtual int read_probe(int id, long long t0, long long count, double* out) = 0;
  virtual int read_flux(int id, long long t0, long long count, double* out) = 0;
  virtual int nprobes() const = 0;
  virtual int nfluxes() const = 0;
  virtual long long capacity() const = 0;
  virtual int energy(double* out) = 0;
  virtual int error_flags(int* flags) = 0;
  virtual void state_blobs(std::vector<std::pair<void*, size_t>>& v) = 0;
  virtual void set_steps(long long s) = 0;
  // field sets in the grid's cycle, and taking over a state whose fields
  // cycled through `from` sets (a checkpoint of another kernel's grid)
  virtual int field_sets() const = 0;
  virtual int adopt_field_sets(int from) = 0;
  virtual const void* step_record() const = 0;
  virtual const void* obs_record() const = 0;
  virtual size_t step_record_size() const = 0;
  virtual size_t obs_record_size() const = 0;
  virtual int has_gain() const = 0;
  // batch support: device TMA descriptors, kernel path, work items (grid index 0)
  virtual const void* tma_device() const = 0;
  virtual bool uses_tma() const = 0;
  virtual bool uses_pair() const = 0;
  virtual int tile_rows() const = 0;
  virtual void work_items(std::vector<int4>& step_items, std::vector<int4>& obs_items) const = 0;

  int get_material(uint8_t* out) {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    if ((e = cudaMemcpy2D(out, desc.nx, d_mat, px, desc.nx, (size_t)desc.ny * desc.nz, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "read material");
    return FDTD_OK;
  }
  int set_material(const uint8_t* in) {
    cudaError_t e = cudaMemcpy2DAsync(d_mat, px, in, desc.nx, desc.nx, (size_t)desc.ny * desc.nz,
                                      cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_error(e, "set material");
    return FDTD_OK;
  }
};

// The device's persisting L2 set-aside serves one grid at a time: the grid
// stepping alone most recently on that device, if it keeps its CPML memory in
// L2.  l2_claim(g) hands it to g (clearing the previous holder's window and
// returning its lines to normal); l2_claim(nullptr) releases it (a batch
// steps, or a grid switches the option off); l2_forget(g) before g goes away.
void l2_claim(GridBase* g);
void l2_forget(GridBase* g);
// The stream is capturing a graph (no limit or attribute change may happen then).
bool stream_capturing(cudaStream_t st);

GridBase* make_grid(const fdtd_grid_desc& d);
int init_grid(GridBase* g);

}  // namespace fdtd

struct fdtd_grid {
  fdtd::GridBase* impl;
};
