// extern "C" entry points of include/fdtd.h: argument validation, object
// state checks and dispatch to the grid implementation.  No C++ exception
// crosses this boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_batch_internal.h"
#include "fdtd_internal.cuh"

using fdtd::GridBase;
using fdtd::set_error;

namespace {

template <typename F>
int guarded(F&& f) {
  try {
    fdtd::g_last_error.clear();
    return f();
  } catch (const std::bad_alloc&) {
    return set_error(FDTD_E_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(FDTD_E_INVAL, "%s", e.what());
  } catch (...) {
    return set_error(FDTD_E_INVAL, "unknown error");
  }
}

int axis_len(const fdtd_grid_desc& d, int a) { return a == 0 ? d.nx : a == 1 ? d.ny : d.nz; }

#define CHECK_GRID(g)                                                  \
  if (!(g) || !(g)->impl) return set_error(FDTD_E_INVAL, "null grid"); \
  GridBase* G = (g)->impl

#define BEFORE_FIRST_STEP(G, what) \
  if ((G)->finalized) return set_error(FDTD_E_STATE, "%s is only allowed before the first step", what)

int ensure_finalized(GridBase* G) {
  if (G->finalized) return FDTD_OK;
  const int r = G->finalize();
  if (r == FDTD_OK) G->finalized = true;
  return r;
}

}  // namespace

extern "C" {

const char* fdtd_last_error(void) { return fdtd::g_last_error.c_str(); }

const char* fdtd_version(void) { return "fdtd-gb300 1.0 (sm_103a; Yee/CPML/four-level Maxwell-Bloch)"; }

int fdtd_create_grid(const fdtd_grid_desc* desc, const fdtd_allocator* alloc, void* stream, fdtd_grid** out) {
  return guarded([&]() -> int {
    if (!desc || !out) return set_error(FDTD_E_INVAL, "null argument");
    *out = nullptr;
    const fdtd_grid_desc& d = *desc;
    const int n3[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
      if (n3[a] < 1 || n3[a] > 32767) return set_error(FDTD_E_INVAL, "axis %d length %d out of [1, 32767]", a, n3[a]);
      if (d.npml[2 * a] < 0 || d.npml[2 * a + 1] < 0) return set_error(FDTD_E_INVAL, "negative npml");
      if (d.periodic[a] && (d.npml[2 * a] || d.npml[2 * a + 1]))
        return set_error(FDTD_E_INVAL, "axis %d is periodic and has an absorbing slab", a);
      if (d.npml[2 * a] + d.npml[2 * a + 1] >= n3[a]) return set_error(FDTD_E_INVAL, "absorbing slabs fill axis %d", a);
    }
    if (d.precision != FDTD_FP32 && d.precision != FDTD_FP64) return set_error(FDTD_E_INVAL, "precision");
    if (!(d.res > 0) || !(d.a > 0) || !(d.courant > 0) || !(d.courant <= 1.0))
      return set_error(FDTD_E_INVAL, "res, a must be > 0 and courant in (0, 1]");
    for (int q = 0; q < 3; ++q)
      if (!(d.eps[q] > 0) || !std::isfinite(d.eps[q])) return set_error(FDTD_E_INVAL, "eps[%d] must be finite and > 0", q);
    if (!(d.cpml_m >= 0) || !(d.cpml_sigma_factor >= 0) || !(d.cpml_kappa_max >= 1) || !(d.cpml_alpha_max >= 0))
      return set_error(FDTD_E_INVAL, "CPML parameters");
    if (d.record_capacity < 1) return set_error(FDTD_E_INVAL, "record_capacity must be >= 1");
    int dev_count = 0;
    cudaError_t e = cudaGetDeviceCount(&dev_count);
    if (e != cudaSuccess || dev_count == 0) {
      cudaGetLastError();
      return set_error(FDTD_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    GridBase* G = fdtd::make_grid(d);
    if (!G) return set_error(FDTD_E_NOMEM, "host allocation failed");
    G->desc = d;
    G->stream = (cudaStream_t)stream;
    if (alloc) G->mem.alloc = *alloc;
    G->mem.stream = stream;
    G->ncell = (long long)d.nx * d.ny * d.nz;
    G->S = d.courant / std::sqrt(3.0);
    G->dx = d.a / d.res;
    G->dt = G->S * G->dx / fdtd::kC0;
    const int r = fdtd::init_grid(G);
    if (r != FDTD_OK) {
      delete G;
      return r;
    }
    fdtd_grid* h = new fdtd_grid{G};
    *out = h;
    return FDTD_OK;
  });
}

int fdtd_destroy_grid(fdtd_grid* g) {
  return guarded([&]() -> int {
    if (!g) return FDTD_OK;
    if (g->impl) {
      cudaStreamSynchronize(g->impl->stream);
      delete g->impl;
    }
    delete g;
    return FDTD_OK;
  });
}

int fdtd_set_eps_from_spheres(fdtd_grid* g, const double* spheres, int64_t n, const double box_lo[3],
                              const double box_hi[3]) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_set_eps_from_spheres");
    if (n < 0 || (n > 0 && !spheres) || !box_lo || !box_hi) return set_error(FDTD_E_INVAL, "bad sphere list or box");
    if (n > (int64_t)1 << 26) return set_error(FDTD_E_INVAL, "too many spheres");
    for (int64_t s = 0; s < n; ++s)
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(spheres[4 * s + q])) return set_error(FDTD_E_INVAL, "non-finite sphere %lld", (long long)s);
    for (int64_t s = 0; s < n; ++s)
      if (spheres[4 * s + 3] < 0) return set_error(FDTD_E_INVAL, "negative radius");
    const fdtd_grid_desc& d = G->desc;
    const int B = 8;
    const int bn[3] = {(d.nx + B - 1) / B, (d.ny + B - 1) / B, (d.nz + B - 1) / B};
    const int nb = bn[0] * bn[1] * bn[2];
    // conservative cull: a sphere is listed in every bin whose cells it may touch
    std::vector<int> lo3((size_t)n * 3), hi3((size_t)n * 3);
    std::vector<int> count((size_t)nb + 1, 0);
    for (int64_t s = 0; s < n; ++s) {
      bool empty = false;
      for (int a = 0; a < 3; ++a) {
        const double c = spheres[4 * s + a], r = spheres[4 * s + 3];
        const double lo = std::floor(c - r - 1.0), hi = std::floor(c + r + 1.0);
        const int L = axis_len(d, a);
        const double clo = std::max(lo, 0.0), chi = std::min(hi, (double)(L - 1));
        if (clo > chi) { empty = true; break; }
        lo3[s * 3 + a] = (int)clo / B;
        hi3[s * 3 + a] = (int)chi / B;
      }
      if (empty) { lo3[s * 3] = 1; hi3[s * 3] = 0; continue; }
      for (int bz = lo3[s * 3 + 2]; bz <= hi3[s * 3 + 2]; ++bz)
        for (int by = lo3[s * 3 + 1]; by <= hi3[s * 3 + 1]; ++by)
          for (int bx = lo3[s * 3]; bx <= hi3[s * 3]; ++bx) count[(bz * bn[1] + by) * bn[0] + bx + 1]++;
    }
    for (int b = 0; b < nb; ++b) count[b + 1] += count[b];
    std::vector<int> list((size_t)count[nb]);
    std::vector<int> fill(count.begin(), count.end() - 1);
    for (int64_t s = 0; s < n; ++s) {
      if (lo3[s * 3] > hi3[s * 3]) continue;
      for (int bz = lo3[s * 3 + 2]; bz <= hi3[s * 3 + 2]; ++bz)
        for (int by = lo3[s * 3 + 1]; by <= hi3[s * 3 + 1]; ++by)
          for (int bx = lo3[s * 3]; bx <= hi3[s * 3]; ++bx) list[fill[(bz * bn[1] + by) * bn[0] + bx]++] = (int)s;
    }
    fdtd::DeviceMemory tmp;
    tmp.stream = G->stream;
    double* dsph = (double*)tmp.get(sizeof(double) * 4 * (size_t)std::max<int64_t>(n, 1));
    float* dfsph = (float*)tmp.get(sizeof(float) * 8 * (size_t)std::max<int64_t>(n, 1));
    // binary32 split of each centre (integer part exact, fraction rounded) and r^2, for the rasterizer's pre-test
    std::vector<float> fsph((size_t)8 * (size_t)n);
    for (int64_t s = 0; s < n; ++s) {
      for (int a = 0; a < 3; ++a) {
        const double c = spheres[4 * s + a], fl = std::floor(c);
        fsph[8 * s + a] = (float)fl;
        fsph[8 * s + 4 + a] = (float)(c - fl);
      }
      fsph[8 * s + 3] = (float)(spheres[4 * s + 3] * spheres[4 * s + 3]);
      fsph[8 * s + 7] = 0.0f;
    }
    int* dstart = (int*)tmp.get(sizeof(int) * count.size());
    int* dlist = (int*)tmp.get(sizeof(int) * std::max<size_t>(list.size(), 1));
    if (!dsph || !dfsph || !dstart || !dlist) {
      tmp.release_all();
      return set_error(FDTD_E_NOMEM, "device allocation failed (sphere bins)");
    }
    cudaError_t e = cudaSuccess;
    if (n) e = cudaMemcpyAsync(dsph, spheres, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, G->stream);
    if (n && e == cudaSuccess)
      e = cudaMemcpyAsync(dfsph, fsph.data(), sizeof(float) * 8 * n, cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dstart, count.data(), sizeof(int) * count.size(), cudaMemcpyHostToDevice, G->stream);
    if (e == cudaSuccess && !list.empty())
      e = cudaMemcpyAsync(dlist, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, G->stream);
    const double box[6] = {box_lo[0], box_lo[1], box_lo[2], box_hi[0], box_hi[1], box_hi[2]};
    if (e == cudaSuccess)
      e = fdtd::launch_rasterize(G->d_mat, d.nx, d.ny, d.nz, G->px, dsph, dfsph, dstart, dlist, B, bn[0], bn[1], bn[2],
                                 box, G->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(G->stream);
    tmp.release_all();
    if (e != cudaSuccess) return fdtd::cuda_error(e, "rasterize");
    G->material_set = true;
    return FDTD_OK;
  });
}

int fdtd_set_material(fdtd_grid* g, const uint8_t* mat) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_set_material");
    if (!mat) return set_error(FDTD_E_INVAL, "null material");
    const long long cells = (long long)G->desc.nx * G->desc.ny * G->desc.nz;
    for (long long q = 0; q < cells; ++q) {
      const unsigned b = mat[q];
      if ((b & 0x80u) || (b & 3u) == 3u || ((b >> 2) & 3u) == 3u || ((b >> 4) & 3u) == 3u)
        return set_error(FDTD_E_INVAL, "material byte %u at cell %lld: class 3 or bit 7 set", b, q);
    }
    const int r = G->set_material(mat);
    if (r != FDTD_OK) return r;
    G->material_set = true;
    return FDTD_OK;
  });
}

int fdtd_get_material(fdtd_grid* g, uint8_t* mat) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!mat) return set_error(FDTD_E_INVAL, "null output");
    return G->get_material(mat);
  });
}

int fdtd_set_gain(fdtd_grid* g, const fdtd_gain_params* p) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (G->absorber == FDTD_ABSORBER_UPML)
      return set_error(FDTD_E_INVAL, "the uniaxial PML runs passive grids (no gain medium)");
    BEFORE_FIRST_STEP(G, "fdtd_set_gain");
    if (!p) return set_error(FDTD_E_INVAL, "null gain parameters");
    if (!G->material_set) return set_error(FDTD_E_STATE, "set the material before the gain medium");
    if (!(p->n_total > 0) || !(p->tau32 > 0) || !(p->tau21 > 0) || !(p->tau10 > 0) || !(p->pump >= 0) ||
        !(p->fa_hat > 0) || !(p->dw_rel >= 0) || !(p->noise_amp >= 0) || !(p->kappa >= 0))
      return set_error(FDTD_E_INVAL, "gain parameters out of range");
    if (p->init != FDTD_INIT_STEADY && p->init != FDTD_INIT_GROUND) return set_error(FDTD_E_INVAL, "init");
    return G->set_gain(*p);
  });
}

int fdtd_add_source(fdtd_grid* g, const fdtd_source_desc* s, int32_t* id) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_add_source");
    if (!s) return set_error(FDTD_E_INVAL, "null source");
    if (s->comp < 0 || s->comp > 2) return set_error(FDTD_E_INVAL, "component");
    if (!(s->f0_hat > 0) || !(s->rel_bw > 0) || !std::isfinite(s->amplitude) || !(s->t0_steps >= 0) || !(s->waist >= 0))
      return set_error(FDTD_E_INVAL, "source waveform parameters");
    const fdtd_grid_desc& d = G->desc;
    if (s->kind == FDTD_SRC_POINT) {
      if (s->i < 0 || s->i >= d.nx || s->j < 0 || s->j >= d.ny || s->k < 0 || s->k >= d.nz)
        return set_error(FDTD_E_INVAL, "point source outside the grid");
    } else if (s->kind == FDTD_SRC_SHEET) {
      if (s->axis < 0 || s->axis > 2 || s->index < 0 || s->index >= axis_len(d, s->axis))
        return set_error(FDTD_E_INVAL, "sheet source plane");
    } else {
      return set_error(FDTD_E_INVAL, "source kind");
    }
    const int r = G->add_source(*s);
    if (r == FDTD_OK && id) *id = 0;
    return r;
  });
}

int fdtd_add_probe(fdtd_grid* g, int32_t i, int32_t j, int32_t k, int32_t* id) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_add_probe");
    const fdtd_grid_desc& d = G->desc;
    if (i < 0 || i >= d.nx || j < 0 || j >= d.ny || k < 0 || k >= d.nz) return set_error(FDTD_E_INVAL, "probe outside the grid");
    const int before = G->nprobes();
    const int r = G->add_probe(i, j, k);
    if (r == FDTD_OK && id) *id = before;
    return r;
  });
}

int fdtd_add_flux_plane(fdtd_grid* g, int32_t axis, int32_t index, double sign, int32_t u0, int32_t u1, int32_t v0,
                        int32_t v1, int32_t* id) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_add_flux_plane");
    const fdtd_grid_desc& d = G->desc;
    if (axis < 0 || axis > 2) return set_error(FDTD_E_INVAL, "axis");
    const int n = axis_len(d, axis), n1 = axis_len(d, (axis + 1) % 3), n2 = axis_len(d, (axis + 2) % 3);
    if (index < 1 || index > n - 1) return set_error(FDTD_E_INVAL, "flux plane index out of [1, n-1]");
    if (!(0 <= u0 && u0 <= u1 && u1 <= n1 - 1 && 0 <= v0 && v0 <= v1 && v1 <= n2 - 1))
      return set_error(FDTD_E_INVAL, "flux face range");
    if (!std::isfinite(sign)) return set_error(FDTD_E_INVAL, "sign");
    const int before = G->nfluxes();
    const int r = G->add_flux(axis, index, sign, u0, u1, v0, v1);
    if (r == FDTD_OK && id) *id = before;
    return r;
  });
}

int fdtd_set_launch(fdtd_grid* g, int32_t bx, int32_t by, int32_t zdepth, int32_t grid_blocks) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (bx < 2 || by < 2 || bx * by > 512 || (bx * by) % 32 != 0 || zdepth < 0 || grid_blocks < 0)
      return set_error(FDTD_E_INVAL, "launch shape: need bx, by >= 2, bx*by a multiple of 32 and <= 512");
    G->bx = bx;
    G->by = by;
    G->zdepth = zdepth;
    G->grid_blocks = grid_blocks;
    if (G->finalized) {
      cudaError_t e = cudaStreamSynchronize(G->stream);
      if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
      return G->replan();
    }
    return FDTD_OK;
  });
}

int fdtd_set_kernel(fdtd_grid* g, int32_t kind) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (kind < 0 || kind > 3)
      return set_error(FDTD_E_INVAL, "kernel kind must be 0 (auto), 1 (plain), 2 (TMA) or 3 (paired TMA)");
    const fdtd_grid_desc& d = G->desc;
    if ((kind == 2 || kind == 3) && (d.periodic[0] || d.periodic[1] || d.periodic[2]))
      return set_error(FDTD_E_INVAL, "the TMA step kernels do not handle periodic axes");
    if (kind == 3 && d.precision != FDTD_FP32) return set_error(FDTD_E_INVAL, "the paired step kernel is binary32 only");
    G->kernel_kind = kind;
    if (G->finalized) {
      cudaError_t e = cudaStreamSynchronize(G->stream);
      if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
      return G->replan();
    }
    return FDTD_OK;
  });
}

int fdtd_set_l2_residency(fdtd_grid* g, int32_t on) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (on != 0 && on != 1) return set_error(FDTD_E_INVAL, "L2 residency must be 0 or 1");
    G->l2_resident = on;
    if (on) return FDTD_OK;  // taken at the grid's next step
    cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    fdtd::l2_forget(G);
    return FDTD_OK;
  });
}

int fdtd_kernel_in_use(fdtd_grid* g, int32_t* kind, int32_t* rows) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!kind || !rows) return set_error(FDTD_E_INVAL, "null output");
    if (!G->finalized) return set_error(FDTD_E_STATE, "the launch plan is made at the first step");
    *kind = G->kernel_in_use_kind();
    *rows = G->tile_rows();
    return FDTD_OK;
  });
}

int fdtd_step_n(fdtd_grid* g, int64_t n) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (n < 0) return set_error(FDTD_E_INVAL, "negative step count");
    if (!G->material_set) return set_error(FDTD_E_STATE, "set the permittivity map before stepping");
    int r = ensure_finalized(G);
    if (r != FDTD_OK) return r;
    if (n == 0) return FDTD_OK;
    return G->step(n);
  });
}

int fdtd_set_timing(fdtd_grid* g, int32_t on) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    if (on < 0) return set_error(FDTD_E_INVAL, "timing: 0 (off) or a launch stride >= 1");
    G->timer.collect();
    G->timer.on = on != 0;
    G->timer.stride = on > 0 ? on : 1;
    G->timer.seen = 0;
    G->timer.ms = 0.0;
    G->timer.launches = 0;
    return FDTD_OK;
  });
}

int fdtd_kernel_time(fdtd_grid* g, double* ms, int64_t* launches) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!ms || !launches) return set_error(FDTD_E_INVAL, "null output");
    cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    G->timer.collect();
    *ms = G->timer.ms;
    *launches = G->timer.launches;
    return FDTD_OK;
  });
}

int fdtd_sync(fdtd_grid* g) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    int flags = 0;
    const int r = G->error_flags(&flags);
    if (r != FDTD_OK) return r;
    if (flags & 1) return set_error(FDTD_E_NONFINITE, "a probe, flux or energy value is not finite");
    if (flags & 2) return set_error(FDTD_E_TIMEOUT, "a bounded wait of the step kernel ran out");
    return FDTD_OK;
  });
}

int fdtd_steps_done(fdtd_grid* g, int64_t* n) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!n) return set_error(FDTD_E_INVAL, "null output");
    *n = G->steps;
    return FDTD_OK;
  });
}

static int check_range(GridBase* G, int64_t t0, int64_t count) {
  if (t0 < 0 || count < 0) return set_error(FDTD_E_INVAL, "negative range");
  if (t0 + count > G->steps) return set_error(FDTD_E_INVAL, "range beyond the steps done");
  if (count > 0 && t0 < G->steps - G->capacity()) return set_error(FDTD_E_INVAL, "range older than the recorder holds");
  return FDTD_OK;
}

int fdtd_read_probes(fdtd_grid* g, int32_t id, int64_t t0, int64_t count, double* out) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (id < 0 || id >= G->nprobes()) return set_error(FDTD_E_INVAL, "probe id");
    int r = check_range(G, t0, count);
    if (r != FDTD_OK) return r;
    if (count == 0) return FDTD_OK;
    if (!out) return set_error(FDTD_E_INVAL, "null output");
    return G->read_probe(id, t0, count, out);
  });
}

int fdtd_read_flux(fdtd_grid* g, int32_t id, int64_t t0, int64_t count, double* out) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (id < 0 || id >= G->nfluxes()) return set_error(FDTD_E_INVAL, "flux plane id");
    int r = check_range(G, t0, count);
    if (r != FDTD_OK) return r;
    if (count == 0) return FDTD_OK;
    if (!out) return set_error(FDTD_E_INVAL, "null output");
    return G->read_flux(id, t0, count, out);
  });
}

int fdtd_read_fields(fdtd_grid* g, int32_t comp, double* out) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (comp < 0 || comp > 5 || !out) return set_error(FDTD_E_INVAL, "component or output");
    return G->read_field(comp, out);
  });
}

int fdtd_write_fields(fdtd_grid* g, int32_t comp, const double* in) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    BEFORE_FIRST_STEP(G, "fdtd_write_fields");
    if (comp < 0 || comp > 5 || !in) return set_error(FDTD_E_INVAL, "component or input");
    return G->write_field(comp, in);
  });
}

int fdtd_read_gain(fdtd_grid* g, int32_t what, double* out) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (what < 0 || what > 3 || !out) return set_error(FDTD_E_INVAL, "what or output");
    return G->read_gain(what, out);
  });
}

int fdtd_field_energy(fdtd_grid* g, double* out) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!out) return set_error(FDTD_E_INVAL, "null output");
    return G->energy(out);
  });
}

int fdtd_set_step_limit(fdtd_grid* g, int64_t limit) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (limit < 0) return set_error(FDTD_E_INVAL, "negative step limit");
    G->step_limit = limit;
    G->tables_dirty = true;
    return FDTD_OK;
  });
}

int fdtd_set_absorber(fdtd_grid* g, int32_t absorber) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (absorber != FDTD_ABSORBER_CPML && absorber != FDTD_ABSORBER_UPML)
      return set_error(FDTD_E_INVAL, "absorber must be FDTD_ABSORBER_CPML or FDTD_ABSORBER_UPML");
    if (G->finalized) return set_error(FDTD_E_STATE, "the absorber is only set before the first step");
    if (absorber == FDTD_ABSORBER_UPML && G->has_gain())
      return set_error(FDTD_E_INVAL, "the uniaxial PML runs passive grids (no gain medium)");
    G->absorber = absorber;
    return FDTD_OK;
  });
}

int fdtd_set_item_order(fdtd_grid* g, int32_t order) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (order != FDTD_ORDER_COSTLIEST && order != FDTD_ORDER_Z)
      return set_error(FDTD_E_INVAL, "order must be FDTD_ORDER_COSTLIEST or FDTD_ORDER_Z");
    G->item_order = order;
    if (G->finalized) {
      cudaError_t e = cudaStreamSynchronize(G->stream);
      if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
      return G->replan();
    }
    return FDTD_OK;
  });
}

int fdtd_set_gain_coupling(fdtd_grid* g, int32_t coupling) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (coupling != FDTD_COUPLING_CELL && coupling != FDTD_COUPLING_CENTRED)
      return set_error(FDTD_E_INVAL, "coupling must be FDTD_COUPLING_CELL or FDTD_COUPLING_CENTRED");
    if (G->finalized) return set_error(FDTD_E_STATE, "the coupling is only set before the first step");
    G->coupling = coupling;
    return FDTD_OK;
  });
}

int fdtd_set_wait_limit(fdtd_grid* g, int64_t ns) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (ns < 0) return set_error(FDTD_E_INVAL, "negative wait limit");
    G->wait_ns = ns;
    G->tables_dirty = true;
    return FDTD_OK;
  });
}

#define CHECK_BATCH(b)                                                  \
  if (!(b) || !(b)->impl) return set_error(FDTD_E_INVAL, "null batch"); \
  fdtd::BatchBase* B = (b)->impl

int fdtd_batch_create(fdtd_grid* const* grids, int32_t n, void* stream, fdtd_batch** out) {
  return guarded([&]() -> int {
    if (!grids || !out || n < 1) return set_error(FDTD_E_INVAL, "need at least one grid and an output");
    *out = nullptr;
    int prec = -1;
    for (int q = 0; q < n; ++q) {
      if (!grids[q] || !grids[q]->impl) return set_error(FDTD_E_INVAL, "null member %d", q);
      if (grids[q]->impl->has_gain() && grids[q]->impl->coupling == FDTD_COUPLING_CENTRED)
        return set_error(FDTD_E_INVAL, "member %d has the centred gain coupling: such grids step alone", q);
      if (grids[q]->impl->absorber == FDTD_ABSORBER_UPML)
        return set_error(FDTD_E_INVAL, "member %d has the uniaxial PML: such grids step alone", q);
      GridBase* G = grids[q]->impl;
      if (!G->material_set) return set_error(FDTD_E_STATE, "member %d has no permittivity map", q);
      if (prec >= 0 && G->precision() != prec) return set_error(FDTD_E_INVAL, "members differ in precision");
      prec = G->precision();
      for (int r = 0; r < q; ++r)
        if (grids[r] == grids[q]) return set_error(FDTD_E_INVAL, "member %d listed twice", q);
    }
    fdtd::BatchBase* B = fdtd::make_batch(prec);
    if (!B) return set_error(FDTD_E_NOMEM, "host allocation failed");
    for (int q = 0; q < n; ++q) B->grids.push_back(grids[q]->impl);
    B->stream = (cudaStream_t)stream;
    B->mem.stream = stream;
    *out = new fdtd_batch{B};
    return FDTD_OK;
  });
}

int fdtd_batch_destroy(fdtd_batch* b) {
  return guarded([&]() -> int {
    if (!b) return FDTD_OK;
    if (b->impl) {
      cudaStreamSynchronize(b->impl->stream);
      delete b->impl;
    }
    delete b;
    return FDTD_OK;
  });
}

int fdtd_batch_set_launch(fdtd_batch* b, int32_t kernel, int32_t by, int32_t zdepth, int32_t grid_blocks) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    if (kernel < 0 || kernel > 3 || by < 0 || by == 1 || by > 16 || zdepth < 0 || grid_blocks < 0)
      return set_error(FDTD_E_INVAL, "batch launch shape");
    B->kernel_kind = kernel;
    B->bx = 32;
    B->by = by;
    B->zdepth = zdepth;
    B->grid_blocks = grid_blocks;
    B->dirty = true;
    return FDTD_OK;
  });
}

int fdtd_batch_set_graph(fdtd_batch* b, int32_t steps_per_graph) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    if (steps_per_graph < 0 || steps_per_graph > 100000) return set_error(FDTD_E_INVAL, "steps per graph");
    B->graph_steps = steps_per_graph;
    return FDTD_OK;
  });
}

int fdtd_batch_step_n(fdtd_batch* b, int64_t n) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    if (n < 0) return set_error(FDTD_E_INVAL, "negative step count");
    if (n == 0) return FDTD_OK;
    return B->step(n);
  });
}

int fdtd_batch_sync(fdtd_batch* b) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    for (GridBase* G : B->grids) {
      int flags = 0;
      const int r = G->error_flags(&flags);
      if (r != FDTD_OK) return r;
      if (flags & 1) return set_error(FDTD_E_NONFINITE, "a member produced a non-finite value");
      if (flags & 2) return set_error(FDTD_E_TIMEOUT, "a bounded wait of the step kernel ran out");
    }
    return FDTD_OK;
  });
}

int fdtd_batch_set_timing(fdtd_batch* b, int32_t on) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    if (on < 0) return set_error(FDTD_E_INVAL, "timing: 0 (off) or a launch stride >= 1");
    B->timer.collect();
    B->timer.on = on != 0;
    B->timer.stride = on > 0 ? on : 1;
    B->timer.seen = 0;
    B->timer.ms = 0.0;
    B->timer.launches = 0;
    return FDTD_OK;
  });
}

int fdtd_batch_kernel_time(fdtd_batch* b, double* ms, int64_t* launches) {
  return guarded([&]() -> int {
    CHECK_BATCH(b);
    if (!ms || !launches) return set_error(FDTD_E_INVAL, "null output");
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    B->timer.collect();
    *ms = B->timer.ms;
    *launches = B->timer.launches;
    return FDTD_OK;
  });
}

static const char kMagic[8] = {'F', 'D', 'T', 'D', 'C', 'K', 'P', '3'};

int fdtd_save_state(fdtd_grid* g, const char* path) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!path) return set_error(FDTD_E_INVAL, "null path");
    int r = ensure_finalized(G);
    if (r != FDTD_OK) return r;
    cudaError_t e = cudaStreamSynchronize(G->stream);
    if (e != cudaSuccess) return fdtd::cuda_error(e, "sync");
    std::vector<std::pair<void*, size_t>> blobs;
    G->state_blobs(blobs);
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(FDTD_E_INVAL, "cannot open %s", path);
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    ok = ok && std::fwrite(&G->desc, sizeof(G->desc), 1, f) == 1;
    const long long st = G->steps;
    const long long nb = (long long)blobs.size();
    const int32_t ns = G->field_sets();
    ok = ok && std::fwrite(&st, sizeof(st), 1, f) == 1 && std::fwrite(&nb, sizeof(nb), 1, f) == 1 &&
         std::fwrite(&ns, sizeof(ns), 1, f) == 1;
    std::vector<unsigned char> buf;
    for (auto& b : blobs) {
      if (!ok) break;
      const long long sz = (long long)b.second;
      buf.resize(b.second);
      e = cudaMemcpy(buf.data(), b.first, b.second, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        std::fclose(f);
        return fdtd::cuda_error(e, "save");
      }
      ok = std::fwrite(&sz, sizeof(sz), 1, f) == 1 && std::fwrite(buf.data(), 1, b.second, f) == b.second;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return set_error(FDTD_E_INVAL, "write to %s failed", path);
    return FDTD_OK;
  });
}

int fdtd_load_state(fdtd_grid* g, const char* path) {
  return guarded([&]() -> int {
    CHECK_GRID(g);
    if (!path) return set_error(FDTD_E_INVAL, "null path");
    int r = ensure_finalized(G);
    if (r != FDTD_OK) return r;
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(FDTD_E_INVAL, "cannot open %s", path);
    char magic[8];
    fdtd_grid_desc d;
    long long st = 0, nb = 0;
    int32_t ns = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0;
    ok = ok && std::fread(&d, sizeof(d), 1, f) == 1 && std::memcmp(&d, &G->desc, sizeof(d)) == 0;
    ok = ok && std::fread(&st, sizeof(st), 1, f) == 1 && std::fread(&nb, sizeof(nb), 1, f) == 1 &&
         std::fread(&ns, sizeof(ns), 1, f) == 1 && ns >= 2 && ns <= fdtd::kFieldSets;
    std::vector<std::pair<void*, size_t>> blobs;
    G->state_blobs(blobs);
    ok = ok && nb == (long long)blobs.size();
    std::vector<unsigned char> buf;
    for (auto& b : blobs) {
      if (!ok) break;
      long long sz = 0;
      ok = std::fread(&sz, sizeof(sz), 1, f) == 1 && sz == (long long)b.second;
      if (!ok) break;
      buf.resize(b.second);
      ok = std::fread(buf.data(), 1, b.second, f) == b.second;
      if (ok && cudaMemcpy(b.first, buf.data(), b.second, cudaMemcpyHostToDevice) != cudaSuccess) {
        std::fclose(f);
        return set_error(FDTD_E_CUDA, "load: copy to device failed");
      }
    }
    std::fclose(f);
    if (!ok) return set_error(FDTD_E_INVAL, "%s is not a checkpoint of an identically described grid", path);
    G->set_steps(st);
    r = G->adopt_field_sets(ns);  // the saving grid may have cycled another number of field sets
    if (r != FDTD_OK) return r;
    return G->replan();
  });
}

}  // extern "C"
