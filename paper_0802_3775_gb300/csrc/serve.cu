// Request server: continuous batching of FDTD runs on one GPU.
//
// A worker thread owns a CUDA stream and a batch of resident runs.  Requests
// (a grid description, a sphere list, optional gain, sources, probes, flux
// planes and a step count) are copied at submission and queued.  At every
// chunk boundary the worker retires finished runs (results copied to host
// memory, device memory returned to the stream-ordered pool), admits queued
// runs first-in first-out while the HBM budget and the slot count allow,
// rebuilds the batch when its membership changed, and steps every resident
// run by one chunk in one launch per time step.  Each run stops exactly at
// its own step count (per-member limits), so a result does not depend on
// which other runs shared the GPU.
//
// Paper: the disorder studies are sets of independent realizations (Sec.
// "Wide-band excitation and gap filling": 10 realizations per disorder
// strength); the server keeps such runs resident and overlaps them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_batch_internal.h"
#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

void* pool_alloc(size_t bytes, void* stream, void*) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void pool_free(void* p, size_t, void* stream, void*) { cudaFreeAsync(p, (cudaStream_t)stream); }

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// Device bytes a run will hold (fields, material, CPML memory, gain state,
// recorders), computed before it is created.
long long estimate_run_bytes(const fdtd_grid_desc& d, bool gain, int nprobe, int nflux) {
  const long long w = d.precision == FDTD_FP32 ? 4 : 8;
  const long long px = (d.nx + 15) / 16 * 16;
  const long long nstore = px * d.ny * d.nz;
  const long long ncell = (long long)d.nx * d.ny * d.nz;
  long long b = 6 * kFieldSets * w * nstore + nstore;
  const int n3[3] = {d.nx, d.ny, d.nz};
  for (int a = 0; a < 3; ++a) b += 6 * w * (long long)(d.npml[2 * a] + d.npml[2 * a + 1]) * (ncell / n3[a]);
  if (gain) b += (w == 4 ? 12 : 9) * w * ((d.nx + 31) / 32 * 32LL) * d.ny * d.nz;  // 32-node records
  b += (long long)d.record_capacity * (nprobe * 3 * w + nflux * 8);
  b += 6 * (long long)(d.nx + d.ny + d.nz) * w + 64 * 1024;
  return b;
}

struct Run {
  uint64_t ticket = 0;
  fdtd_grid_desc desc{};
  std::vector<double> spheres;
  double box_lo[3], box_hi[3];
  bool has_gain = false;
  fdtd_gain_params gain{};
  std::vector<fdtd_source_desc> sources;
  std::vector<int32_t> probes;
  std::vector<fdtd_flux_desc> fluxes;
  long long steps = 0;
  long long bytes = 0;
  fdtd_grid* grid = nullptr;
  // results
  int status = FDTD_E_BUSY;
  double t_submit = 0, t_admit = 0, t_done = 0;
  double energy = 0;
  std::vector<double> probe_series;  // [steps][nprobe][3]
  std::vector<double> flux_series;   // [nflux][steps]
};

struct Server {
  fdtd_server_desc desc{};
  int device = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<Run>> queue;
  std::vector<std::shared_ptr<Run>> active;
  std::map<uint64_t, std::shared_ptr<Run>> runs;
  long long used_bytes = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  fdtd_batch* batch = nullptr;
  bool membership_changed = false;
  fdtd_server_stats stats{};

  int create_run(Run& r) {
    fdtd_allocator a{pool_alloc, pool_free, nullptr};
    fdtd_grid_desc d = r.desc;
    d.record_capacity = std::max<long long>(r.steps, 1);
    int rc = fdtd_create_grid(&d, &a, stream, &r.grid);
    if (rc != FDTD_OK) return rc;
    rc = fdtd_set_eps_from_spheres(r.grid, r.spheres.data(), (int64_t)r.spheres.size() / 4, r.box_lo, r.box_hi);
    if (rc == FDTD_OK && r.has_gain) rc = fdtd_set_gain(r.grid, &r.gain);
    for (size_t q = 0; rc == FDTD_OK && q < r.sources.size(); ++q) rc = fdtd_add_source(r.grid, &r.sources[q], nullptr);
    for (size_t q = 0; rc == FDTD_OK && q + 2 < r.probes.size(); q += 3)
      rc = fdtd_add_probe(r.grid, r.probes[q], r.probes[q + 1], r.probes[q + 2], nullptr);
    for (size_t q = 0; rc == FDTD_OK && q < r.fluxes.size(); ++q) {
      const fdtd_flux_desc& f = r.fluxes[q];
      rc = fdtd_add_flux_plane(r.grid, f.axis, f.index, f.sign, f.u0, f.u1, f.v0, f.v1, nullptr);
    }
    if (rc == FDTD_OK) rc = fdtd_set_step_limit(r.grid, r.steps);
    if (rc == FDTD_OK) rc = fdtd_step_n(r.grid, 0);  // freeze the set-up
    return rc;
  }

  // Copy a run's results to host memory and release its device memory.
  // Returns the run's final status; the caller publishes it under the lock.
  int collect_run(Run& r, int status) {
    if (status == FDTD_OK && r.grid) {
      const int np = (int)r.probes.size() / 3, nf = (int)r.fluxes.size();
      r.probe_series.assign((size_t)r.steps * np * 3, 0.0);
      r.flux_series.assign((size_t)r.steps * nf, 0.0);
      std::vector<double> tmp((size_t)r.steps * 3);
      for (int p = 0; p < np && status == FDTD_OK; ++p) {
        status = fdtd_read_probes(r.grid, p, 0, r.steps, tmp.data());
        for (long long s = 0; s < r.steps; ++s)
          for (int c = 0; c < 3; ++c) r.probe_series[((size_t)s * np + p) * 3 + c] = tmp[s * 3 + c];
      }
      for (int f = 0; f < nf && status == FDTD_OK; ++f)
        status = fdtd_read_flux(r.grid, f, 0, r.steps, r.flux_series.data() + (size_t)f * r.steps);
      if (status == FDTD_OK) status = fdtd_field_energy(r.grid, &r.energy);
      if (status == FDTD_OK) status = fdtd_sync(r.grid);
    }
    if (r.grid) {
      fdtd_destroy_grid(r.grid);
      r.grid = nullptr;
    }
    r.spheres.clear();
    r.spheres.shrink_to_fit();
    return status;
  }

  void publish(Run& r, int status) {  // caller holds mu
    r.t_done = now_s(t0);
    r.status = status;
    used_bytes -= r.bytes;
    if (status == FDTD_OK) {
      stats.completed++;
      stats.cell_updates += (long long)r.desc.nx * r.desc.ny * r.desc.nz * r.steps;
    } else {
      stats.failed++;
    }
  }

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      std::vector<std::shared_ptr<Run>> admit;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
        if (stop && queue.empty() && active.empty()) break;
        if (stop) {
          // drain: fail queued requests, finish active ones below
          while (!queue.empty()) {
            auto r = queue.front();
            queue.pop_front();
            r->status = FDTD_E_STATE;
            r->t_done = now_s(t0);
          }
          cv_done.notify_all();
        }
        while (!queue.empty() && (int)(active.size() + admit.size()) < desc.max_slots &&
               used_bytes + queue.front()->bytes <= desc.hbm_budget_bytes) {
          auto r = queue.front();
          queue.pop_front();
          used_bytes += r->bytes;
          admit.push_back(r);
        }
      }
      for (auto& r : admit) {
        r->t_admit = now_s(t0);
        int rc = create_run(*r);
        if (rc != FDTD_OK) rc = collect_run(*r, rc);
        std::lock_guard<std::mutex> lk(mu);
        if (rc != FDTD_OK) {
          publish(*r, rc);
          cv_done.notify_all();
        } else {
          active.push_back(r);
          membership_changed = true;
          stats.admitted++;
        }
      }
      if (active.empty()) continue;
      if (membership_changed) {
        if (batch) fdtd_batch_destroy(batch);
        batch = nullptr;
        std::vector<fdtd_grid*> gs;
        for (auto& r : active) gs.push_back(r->grid);
        int rc = fdtd_batch_create(gs.data(), (int32_t)gs.size(), stream, &batch);
        if (rc == FDTD_OK) rc = fdtd_batch_set_graph(batch, desc.graph ? desc.steps_per_chunk : 0);
        if (rc != FDTD_OK) {
          for (auto& r : active) {
            const int st = collect_run(*r, rc);
            std::lock_guard<std::mutex> lk(mu);
            publish(*r, st);
          }
          std::lock_guard<std::mutex> lk(mu);
          active.clear();
          cv_done.notify_all();
          continue;
        }
        membership_changed = false;
      }
      // step one chunk, bounded by the longest remaining run
      long long remaining = 0;
      for (auto& r : active) {
        int64_t done = 0;
        fdtd_steps_done(r->grid, &done);
        remaining = std::max(remaining, r->steps - done);
      }
      const long long chunk = std::min<long long>(desc.steps_per_chunk, std::max(1LL, remaining));
      int rc = fdtd_batch_step_n(batch, chunk);
      if (rc == FDTD_OK) rc = fdtd_batch_sync(batch);
      {
        std::lock_guard<std::mutex> lk(mu);
        stats.chunks++;
      }
      std::vector<std::shared_ptr<Run>> done_runs;
      for (auto& r : active) {
        int64_t done = 0;
        fdtd_steps_done(r->grid, &done);
        if (rc != FDTD_OK || done >= r->steps) done_runs.push_back(r);
      }
      if (!done_runs.empty()) {
        if (batch) {
          fdtd_batch_destroy(batch);
          batch = nullptr;
        }
        for (auto& r : done_runs) {
          const int st = collect_run(*r, rc);
          std::lock_guard<std::mutex> lk(mu);
          publish(*r, st);
          active.erase(std::find(active.begin(), active.end(), r));
        }
        membership_changed = true;
        std::lock_guard<std::mutex> lk(mu);
        cv_done.notify_all();
      }
    }
    if (batch) fdtd_batch_destroy(batch);
    batch = nullptr;
  }
};

}  // namespace fdtd

struct fdtd_server {
  fdtd::Server* impl;
};

using fdtd::set_error;

namespace {

// No C++ exception leaves an entry point: host allocation failures (request
// copies, the worker thread) come back as error codes.
template <typename F>
int guard(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return set_error(FDTD_E_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(FDTD_E_INVAL, "%s", e.what());
  } catch (...) {
    return set_error(FDTD_E_INVAL, "unknown error");
  }
}

int server_create_impl(const fdtd_server_desc* desc, void* stream, fdtd_server** out) {
  (void)stream;
  if (!desc || !out) return set_error(FDTD_E_INVAL, "null argument");
  *out = nullptr;
  if (desc->hbm_budget_bytes <= 0 || desc->max_slots < 1 || desc->steps_per_chunk < 1)
    return set_error(FDTD_E_INVAL, "budget, slots and chunk must be positive");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    cudaGetLastError();
    return set_error(FDTD_E_CUDA, "no CUDA device");
  }
  auto* s = new (std::nothrow) fdtd::Server();
  if (!s) return set_error(FDTD_E_NOMEM, "host allocation failed");
  s->desc = *desc;
  cudaGetDevice(&s->device);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return set_error(FDTD_E_CUDA, "stream creation failed");
  }
  auto* h = new (std::nothrow) fdtd_server{s};
  if (h) {
    try {
      s->worker = std::thread([s] { s->loop(); });
    } catch (const std::system_error&) {
      delete h;
      h = nullptr;
    }
  }
  if (!h) {
    cudaStreamDestroy(s->stream);
    delete s;
    return set_error(FDTD_E_NOMEM, "the server's worker thread could not start");
  }
  *out = h;
  return FDTD_OK;
}

int server_destroy_impl(fdtd_server* srv) {
  if (!srv) return FDTD_OK;
  fdtd::Server* s = srv->impl;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->runs)
    if (kv.second->grid) fdtd_destroy_grid(kv.second->grid);
  cudaStreamSynchronize(s->stream);
  cudaStreamDestroy(s->stream);
  delete s;
  delete srv;
  return FDTD_OK;
}

int submit_impl(fdtd_server* srv, const fdtd_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  if (req->steps < 1) return set_error(FDTD_E_INVAL, "steps must be >= 1");
  if (req->n_spheres < 0 || (req->n_spheres > 0 && !req->spheres)) return set_error(FDTD_E_INVAL, "spheres");
  if (req->n_sources < 0 || (req->n_sources > 0 && !req->sources)) return set_error(FDTD_E_INVAL, "sources");
  if (req->n_probes < 0 || (req->n_probes > 0 && !req->probes)) return set_error(FDTD_E_INVAL, "probes");
  if (req->n_fluxes < 0 || (req->n_fluxes > 0 && !req->fluxes)) return set_error(FDTD_E_INVAL, "fluxes");
  if (req->grid.precision != s->desc.precision) return set_error(FDTD_E_INVAL, "request precision differs from the server's");
  auto r = std::make_shared<fdtd::Run>();
  r->desc = req->grid;
  r->desc.record_capacity = req->steps;
  r->spheres.assign(req->spheres, req->spheres + 4 * req->n_spheres);
  for (int q = 0; q < 3; ++q) {
    r->box_lo[q] = req->box_lo[q];
    r->box_hi[q] = req->box_hi[q];
  }
  r->has_gain = req->gain != nullptr;
  if (req->gain) r->gain = *req->gain;
  r->sources.assign(req->sources, req->sources + req->n_sources);
  r->probes.assign(req->probes, req->probes + 3 * req->n_probes);
  r->fluxes.assign(req->fluxes, req->fluxes + req->n_fluxes);
  r->steps = req->steps;
  r->bytes = fdtd::estimate_run_bytes(r->desc, r->has_gain, req->n_probes, req->n_fluxes);
  if (r->bytes > s->desc.hbm_budget_bytes)
    return set_error(FDTD_E_BUDGET, "request needs %lld bytes, the budget is %lld", r->bytes,
                     (long long)s->desc.hbm_budget_bytes);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(FDTD_E_STATE, "server is shutting down");
    r->ticket = s->next_ticket++;
    r->t_submit = fdtd::now_s(s->t0);
    s->runs[r->ticket] = r;
    s->queue.push_back(r);
    s->stats.submitted++;
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return FDTD_OK;
}

int poll_impl(fdtd_server* srv, uint64_t ticket, fdtd_result* out, int32_t timeout_ms) {
  if (!srv || !out) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->runs.find(ticket);
  if (it == s->runs.end()) return set_error(FDTD_E_INVAL, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  if (r->status == FDTD_E_BUSY && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->status != FDTD_E_BUSY; });
  out->status = r->status;
  out->steps = r->steps;
  out->submit_s = r->t_submit;
  out->admit_s = r->t_admit;
  out->done_s = r->t_done;
  out->field_energy = r->energy;
  out->n_probes = (int32_t)(r->probes.size() / 3);
  out->n_fluxes = (int32_t)r->fluxes.size();
  if (r->status == FDTD_E_BUSY) return timeout_ms > 0 ? set_error(FDTD_E_TIMEOUT, "not finished") : FDTD_E_BUSY;
  return FDTD_OK;
}

int result_probes_impl(fdtd_server* srv, uint64_t ticket, double* out) {
  if (!srv || !out) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->runs.find(ticket);
  if (it == s->runs.end()) return set_error(FDTD_E_INVAL, "unknown ticket");
  if (it->second->status != FDTD_OK) return set_error(FDTD_E_STATE, "run not completed");
  std::memcpy(out, it->second->probe_series.data(), sizeof(double) * it->second->probe_series.size());
  return FDTD_OK;
}

int result_flux_impl(fdtd_server* srv, uint64_t ticket, double* out) {
  if (!srv || !out) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->runs.find(ticket);
  if (it == s->runs.end()) return set_error(FDTD_E_INVAL, "unknown ticket");
  if (it->second->status != FDTD_OK) return set_error(FDTD_E_STATE, "run not completed");
  std::memcpy(out, it->second->flux_series.data(), sizeof(double) * it->second->flux_series.size());
  return FDTD_OK;
}

int result_release_impl(fdtd_server* srv, uint64_t ticket) {
  if (!srv) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->runs.find(ticket);
  if (it == s->runs.end()) return set_error(FDTD_E_INVAL, "unknown ticket");
  if (it->second->status == FDTD_E_BUSY) return set_error(FDTD_E_BUSY, "run still pending");
  s->runs.erase(it);
  return FDTD_OK;
}

int server_get_stats_impl(fdtd_server* srv, fdtd_server_stats* out) {
  if (!srv || !out) return set_error(FDTD_E_INVAL, "null argument");
  fdtd::Server* s = srv->impl;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident = (int32_t)s->active.size();
  out->queued = (int32_t)s->queue.size();
  out->used_bytes = s->used_bytes;
  return FDTD_OK;
}

}  // namespace

extern "C" {

int fdtd_server_create(const fdtd_server_desc* desc, void* stream, fdtd_server** out) {
  return guard([&] { return server_create_impl(desc, stream, out); });
}

int fdtd_server_destroy(fdtd_server* srv) {
  return guard([&] { return server_destroy_impl(srv); });
}

int fdtd_submit(fdtd_server* srv, const fdtd_request* req, uint64_t* ticket) {
  return guard([&] { return submit_impl(srv, req, ticket); });
}

int fdtd_poll(fdtd_server* srv, uint64_t ticket, fdtd_result* out, int32_t timeout_ms) {
  return guard([&] { return poll_impl(srv, ticket, out, timeout_ms); });
}

int fdtd_result_probes(fdtd_server* srv, uint64_t ticket, double* out) {
  return guard([&] { return result_probes_impl(srv, ticket, out); });
}

int fdtd_result_flux(fdtd_server* srv, uint64_t ticket, double* out) {
  return guard([&] { return result_flux_impl(srv, ticket, out); });
}

int fdtd_result_release(fdtd_server* srv, uint64_t ticket) {
  return guard([&] { return result_release_impl(srv, ticket); });
}

int fdtd_server_get_stats(fdtd_server* srv, fdtd_server_stats* out) {
  return guard([&] { return server_get_stats_impl(srv, out); });
}

}  // extern "C"
