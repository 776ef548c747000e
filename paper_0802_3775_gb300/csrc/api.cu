// Host side of the C ABI (include/fdtd.h): grid lifecycle, coefficient
// set-up, launch planning, stepping and read-backs.
//
// The per-cell and per-step arithmetic runs in the kernels of kernels.cu; the
// host computes the grid's constant tables once (CPML grading profiles,
// material-class coefficients, the 4x4 Crank-Nicolson matrices of the gain
// model) and plans the launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_internal.cuh"

// Faces per block of a flux plane (four per thread).  Measured against one
// face per thread (256): the 140^3 lasing step with six flux planes 0.1250 ->
// 0.1231 ms, the 184^3 passive step 0.1131 -> 0.1127 ms (fewer blocks of the
// observation share the SMs with the next step's blocks).
#ifndef FDTD_FLUX_PART_FACES
#define FDTD_FLUX_PART_FACES 1024
#endif

namespace fdtd {

thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  return set_error(FDTD_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ memory
void* DeviceMemory::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (alloc.alloc) {
    p = alloc.alloc(bytes, stream, alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {
    // the kernels move 8- and 16-byte words and TMA boxes: 256-byte alignment required
    if (alloc.free) alloc.free(p, bytes, stream, alloc.ctx);
    else cudaFree(p);
    return nullptr;
  }
  if (p) blocks.push_back({p, bytes});
  return p;
}

void DeviceMemory::release_all() {
  for (auto& b : blocks) {
    if (alloc.free) alloc.free(b.first, b.second, stream, alloc.ctx);
    else cudaFree(b.first);
  }
  blocks.clear();
}

size_t DeviceMemory::total() const {
  size_t s = 0;
  for (auto& b : blocks) s += b.second;
  return s;
}

// ------------------------------------------------------------------ CPML profile
// (1/kappa, b, c) at the nodes of one axis (integer nodes for E-curl terms,
// half-integer nodes for H-curl terms).  Depth rho = (L0 - x)/L0 below L0 and
// (x - (n - L1))/L1 above n - L1; sigma dt/eps0 = factor (m+1) S rho^m /
// sqrt(eps_edge); kappa = 1 + (kappa_max - 1) rho^m; alpha dt/eps0 =
// alpha_max 2 pi f_ref dt (1 - rho); b = exp(-(sigma/kappa + alpha) dt/eps0),
// c = sigma (b - 1)/(sigma kappa + kappa^2 alpha).
static void cpml_profile(const fdtd_grid_desc& d, int axis, bool half, double S, std::vector<double>& ik,
                         std::vector<double>& b, std::vector<double>& c) {
  const int n = axis == 0 ? d.nx : axis == 1 ? d.ny : d.nz;
  const int L0 = d.npml[2 * axis], L1 = d.npml[2 * axis + 1];
  ik.assign(n, 1.0);
  b.assign(n, 1.0);
  c.assign(n, 0.0);
  const double sig_max = d.cpml_sigma_factor * (d.cpml_m + 1.0) * S / std::sqrt(d.eps[0]);
  const double alpha_max = d.cpml_alpha_max * 2.0 * M_PI * d.cpml_f_hat * S / d.res;
  for (int q = 0; q < n; ++q) {
    const double x = q + (half ? 0.5 : 0.0);
    double rho = 0.0;
    if (L0 > 0 && x < L0) rho = (L0 - x) / L0;
    if (L1 > 0 && x > n - L1) rho = (x - (n - L1)) / L1;
    if (rho <= 0.0) continue;
    const double rm = std::pow(rho, d.cpml_m);
    const double sig = sig_max * rm;
    const double kap = 1.0 + (d.cpml_kappa_max - 1.0) * rm;
    const double alp = alpha_max * (1.0 - rho);
    b[q] = std::exp(-(sig / kap + alp));
    c[q] = sig * (b[q] - 1.0) / (sig * kap + kap * kap * alp);
    ik[q] = 1.0 / kap;
  }
}

// Solve the 4x4 system L X = B (columns of B) by Gaussian elimination with
// partial pivoting, in FP64.
static void solve4(const double Lin[4][4], double B[4][5], int ncol) {
  double L[4][4];
  std::memcpy(L, Lin, sizeof(L));
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(L[r][col]) > std::fabs(L[piv][col])) piv = r;
    if (piv != col) {
      for (int q = 0; q < 4; ++q) std::swap(L[col][q], L[piv][q]);
      for (int q = 0; q < ncol; ++q) std::swap(B[col][q], B[piv][q]);
    }
    for (int r = col + 1; r < 4; ++r) {
      const double f = L[r][col] / L[col][col];
      for (int q = col; q < 4; ++q) L[r][q] -= f * L[col][q];
      for (int q = 0; q < ncol; ++q) B[r][q] -= f * B[col][q];
    }
  }
  for (int col = 3; col >= 0; --col) {
    for (int q = 0; q < ncol; ++q) {
      double s = B[col][q];
      for (int r = col + 1; r < 4; ++r) s -= L[col][r] * B[r][q];
      B[col][q] = s / L[col][col];
    }
  }
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// ------------------------------------------------------------------ grid
template <typename T>
struct GridImpl final : GridBase {
  StepGrid<T> sg{};
  ObsGrid<T> og{};
  StepGrid<T>* d_sg = nullptr;
  ObsGrid<T>* d_og = nullptr;
  int4* d_items = nullptr;
  int4* d_oitems = nullptr;
  std::vector<int4> items, oitems;
  int* d_err = nullptr;
  ObsOverlap obs;  // observation launches beside the step launches
  double* d_energy = nullptr;
  double* d_epart = nullptr;
  unsigned int* d_ecount = nullptr;
  T* d_F = nullptr;
  T* d_gain = nullptr;
  size_t gain_words = 0;
  T* d_psi = nullptr;
  size_t psi_words = 0;
  T* d_prof = nullptr;
  T* d_upml = nullptr;     // uniaxial PML: auxiliary fields (6 arrays) and grading tables
  size_t upml_aux_words = 0;
  UpmlDev<T> upml{};
  TmaGrid* d_tma = nullptr;
  bool use_tma = false;
  bool use_pair = false;  // paired binary32 kernel (TMA staging, tiles of 32 x tile_oy)
  int tile_oy = 8;
  int by_eff = 8;          // tile rows in effect (by, or the kernel's default when by == 0)
  double n_total = 0.0, neq[4] = {0, 0, 0, 0};

  int precision() const override { return sizeof(T) == 4 ? FDTD_FP32 : FDTD_FP64; }
  size_t word() const override { return sizeof(T); }

  int init() {
    const long long nc = ncell;
    px = (desc.nx + 15) / 16 * 16;
    nstore = (long long)px * desc.ny * desc.nz;
    d_F = (T*)mem.get(sizeof(T) * 6 * kFieldSets * (size_t)nstore);
    uint8_t* mat = (uint8_t*)mem.get((size_t)nstore);
    d_tma = (TmaGrid*)mem.get(sizeof(TmaGrid));
    d_err = (int*)mem.get(sizeof(int) * 4);
    d_energy = (double*)mem.get(sizeof(double) * 4);
    d_epart = (double*)mem.get(sizeof(double) * kEnergyBlocks);
    d_ecount = (unsigned int*)mem.get(sizeof(unsigned int) * 4);
    d_sg = (StepGrid<T>*)mem.get(sizeof(StepGrid<T>));
    d_og = (ObsGrid<T>*)mem.get(sizeof(ObsGrid<T>));
    if (!d_F || !mat || !d_tma || !d_err || !d_energy || !d_epart || !d_ecount || !d_sg || !d_og)
      return set_error(FDTD_E_NOMEM, "device allocation failed (%lld cells)", nc);
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_F, 0, sizeof(T) * 6 * kFieldSets * (size_t)nstore, stream)) != cudaSuccess)
      return cuda_error(e, "memset fields");
    // background class in every E node of the grid; the pitch padding stays 0
    if ((e = cudaMemsetAsync(mat, 0, (size_t)nstore, stream)) != cudaSuccess) return cuda_error(e, "memset material");
    if ((e = cudaMemset2DAsync(mat, px, 0x15, desc.nx, (size_t)desc.ny * desc.nz, stream)) != cudaSuccess)
      return cuda_error(e, "memset material");
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int) * 4, stream)) != cudaSuccess) return cuda_error(e, "memset err");
    if ((e = cudaMemsetAsync(d_ecount, 0, sizeof(unsigned) * 4, stream)) != cudaSuccess) return cuda_error(e, "memset");
    d_mat = mat;

    sg.nx = og.nx = desc.nx;
    sg.ny = og.ny = desc.ny;
    sg.nz = og.nz = desc.nz;
    sg.px = og.px = px;
    sg.err = d_err;
    sg.per = (desc.periodic[0] ? 1 : 0) | (desc.periodic[1] ? 2 : 0) | (desc.periodic[2] ? 4 : 0);
    for (int q = 0; q < 6; ++q) sg.L[q] = desc.npml[q];
    for (int s = 0; s < kFieldSets; ++s)
      for (int c = 0; c < 6; ++c) {
        sg.F[s][c] = d_F + (size_t)(s * 6 + c) * nstore;
        og.F[s][c] = sg.F[s][c];
      }
    sg.mat = mat;
    sg.nsets = og.nsets = 2;  // three once the grid is frozen on the paired kernel
    sg.step = 0;
    sg.step_end = (long long)0x7fffffffffffffffLL;
    sg.wait_ns = wait_ns;
    og.step = 0;
    og.step_end = sg.step_end;
    og.err = d_err;
    og.dx2_over_eta0 = dx * dx / eta0();

    // CPML memory: per axis with a slab, 2 E-side arrays and 2x2 H-side arrays,
    // each starting on a 128-byte boundary (node pairs move as 8-byte words)
    const int n3[3] = {desc.nx, desc.ny, desc.nz};
    psi_words = 0;
    size_t slab[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
      sg.Sd[d] = desc.npml[2 * d] + desc.npml[2 * d + 1];
      if (sg.Sd[d]) {
        const size_t words = (size_t)sg.Sd[d] * ((size_t)nc / n3[d]);
        const size_t unit = 128 / sizeof(T);
        slab[d] = (words + unit - 1) / unit * unit;
        psi_words += 6 * slab[d];
      }
    }
    if (psi_words) {
      d_psi = (T*)mem.get(sizeof(T) * psi_words);
      if (!d_psi) return set_error(FDTD_E_NOMEM, "device allocation failed (CPML memory)");
      if ((e = cudaMemsetAsync(d_psi, 0, sizeof(T) * psi_words, stream)) != cudaSuccess) return cuda_error(e, "memset psi");
      T* p = d_psi;
      for (int d = 0; d < 3; ++d) {
        if (!slab[d]) continue;
        sg.psiE[d][0] = p; p += slab[d];
        sg.psiE[d][1] = p; p += slab[d];
        for (int s = 0; s < 2; ++s) {
          sg.psiH[s][d][0] = p; p += slab[d];
          sg.psiH[s][d][1] = p; p += slab[d];
        }
      }
    }
    // grading profiles
    const size_t prof_words = (size_t)6 * (desc.nx + desc.ny + desc.nz);
    d_prof = (T*)mem.get(sizeof(T) * prof_words);
    if (!d_prof) return set_error(FDTD_E_NOMEM, "device allocation failed (profiles)");
    std::vector<T> hprof(prof_words);
    size_t off = 0;
    for (int d = 0; d < 3; ++d)
      for (int h = 0; h < 2; ++h) {
        std::vector<double> ik, b, c;
        cpml_profile(desc, d, h == 1, S, ik, b, c);
        const std::vector<double>* arr[3] = {&ik, &b, &c};
        for (int q = 0; q < 3; ++q) {
          sg.prof[d][h][q] = d_prof + off;
          for (int x = 0; x < n3[d]; ++x) hprof[off + x] = (T)(*arr[q])[x];
          off += n3[d];
        }
      }
    if ((e = cudaMemcpyAsync(d_prof, hprof.data(), sizeof(T) * prof_words, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload profiles");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "init");
    sg.cH = (T)S;
    for (int q = 0; q < 3; ++q) {
      sg.cE[q] = (T)(S / desc.eps[q]);
      sg.cP[q] = (T)(1.0 / desc.eps[q]);
    }
    sg.seed = desc.seed;
    return FDTD_OK;
  }

  int set_gain(const fdtd_gain_params& p) override {
    const double e0 = eps0();
    const double omega_a = 2.0 * M_PI * p.fa_hat * kC0 / desc.a;
    const double dw = p.dw_rel * omega_a;
    const double kappa = p.kappa != 0.0 ? p.kappa : 6.0 * M_PI * e0 * kC0 * kC0 * kC0 / (omega_a * omega_a * p.tau21);
    const double g = 0.5 * dw * dt;
    const double a1 = (2.0 - (omega_a * dt) * (omega_a * dt)) / (1.0 + g);
    const double a2 = (1.0 - g) / (1.0 + g);
    const double a3 = kappa * dt * dt / (e0 * (1.0 + g));
    const double W = p.pump;
    const double A[4][4] = {{-W, 1.0 / p.tau10, 0.0, 0.0},
                            {0.0, -1.0 / p.tau10, 1.0 / p.tau21, 0.0},
                            {0.0, 0.0, -1.0 / p.tau21, 1.0 / p.tau32},
                            {W, 0.0, 0.0, -1.0 / p.tau32}};
    double L[4][4];
    double B[4][5];
    for (int r = 0; r < 4; ++r) {
      for (int c = 0; c < 4; ++c) {
        L[r][c] = (r == c ? 1.0 : 0.0) - 0.5 * dt * A[r][c];
        B[r][c] = A[r][c];
      }
      B[r][4] = r == 1 ? -1.0 : r == 2 ? 1.0 : 0.0;
    }
    solve4(L, B, 5);  // B[:, 0:4] = L^-1 A,  B[:, 4] = L^-1 b
    const double n0 = p.n_total / (1.0 + W * (p.tau32 + p.tau21 + p.tau10));
    neq[0] = n0;
    neq[1] = W * p.tau10 * n0;
    neq[2] = W * p.tau21 * n0;
    neq[3] = W * p.tau32 * n0;
    n_total = p.n_total;
    sg.a1 = (T)a1;
    sg.a2 = (T)a2;
    sg.a3 = (T)(a3 * p.n_total);
    sg.n12eq = (T)((neq[1] - neq[2]) / p.n_total);
    sg.q = (T)(e0 / (kHbar * omega_a * p.n_total));
    sg.noise = (T)p.noise_amp;
    for (int k = 0; k < 3; ++k) {
      for (int j = 0; j < 3; ++j) sg.D[k][j] = (T)(dt * (B[k + 1][j + 1] - B[k + 1][0]));
      sg.w[k] = (T)B[k + 1][4];
    }
    // state: P (2 slots x 3), dN (3), compensation (3, binary32 only), in
    // records of 32 x-adjacent nodes (rows padded to whole records)
    sg.gxb = (desc.nx + 31) / 32;
    const long long nslots = (long long)sg.gxb * 32 * desc.ny * desc.nz;
    if (!d_gain) {
      gain_words = (size_t)GainWords<T>::NW * (size_t)nslots;
      d_gain = (T*)mem.get(sizeof(T) * gain_words);
      if (!d_gain) return set_error(FDTD_E_NOMEM, "device allocation failed (gain state)");
    }
    sg.gst = d_gain;
    sg.gain = 1;
    T d1 = 0, d2 = 0, d3 = 0;
    if (p.init == FDTD_INIT_GROUND) {
      d1 = (T)(-neq[1] / p.n_total);
      d2 = (T)(-neq[2] / p.n_total);
      d3 = (T)(-neq[3] / p.n_total);
    }
    cudaError_t e = launch_gain_init<T>(&sg, nslots, d1, d2, d3, stream);
    if (e != cudaSuccess) return cuda_error(e, "gain init");
    return FDTD_OK;
  }

  int add_source(const fdtd_source_desc& s) override {
    if (sg.nsrc >= kMaxSrc) return set_error(FDTD_E_INVAL, "at most %d sources", kMaxSrc);
    SrcDev d{};
    d.kind = s.kind;
    d.comp = s.comp;
    d.amp = s.amplitude;
    const int n3[3] = {desc.nx, desc.ny, desc.nz};
    if (s.kind == FDTD_SRC_POINT) {
      d.i = s.i; d.j = s.j; d.k = s.k;
      d.axis = 0; d.index = -1;
    } else {
      d.axis = s.axis;
      d.index = s.index;
      const int d1 = (s.axis + 1) % 3, d2 = (s.axis + 2) % 3;
      d.lo1 = desc.npml[2 * d1];
      d.hi1 = n3[d1] - desc.npml[2 * d1 + 1];
      d.lo2 = desc.npml[2 * d2];
      d.hi2 = n3[d2] - desc.npml[2 * d2 + 1];
      d.uc = 0.5 * (d.lo1 + d.hi1 - 1);
      d.vc = 0.5 * (d.lo2 + d.hi2 - 1);
      d.inv_w2 = s.waist > 0 ? 1.0 / (s.waist * s.waist) : 0.0;
      d.i = d.j = d.k = -1;
    }
    d.f0dt = s.f0_hat * S / desc.res;
    d.tau = std::sqrt(std::log(2.0)) / (M_PI * s.rel_bw * d.f0dt);
    d.t0 = s.t0_steps > 0 ? s.t0_steps : 5.0 * d.tau;
    sg.src[sg.nsrc++] = d;
    return FDTD_OK;
  }

  int add_probe(int i, int j, int k) override {
    if (og.nprobe >= kMaxProbes) return set_error(FDTD_E_INVAL, "at most %d probes", kMaxProbes);
    og.probe[og.nprobe][0] = i;
    og.probe[og.nprobe][1] = j;
    og.probe[og.nprobe][2] = k;
    og.nprobe++;
    return FDTD_OK;
  }

  int add_flux(int axis, int index, double sign, int u0, int u1, int v0, int v1) override {
    if (og.nflux >= kMaxFlux) return set_error(FDTD_E_INVAL, "at most %d flux planes", kMaxFlux);
    const int f = og.nflux++;
    og.flux_axis[f] = axis;
    og.flux_index[f] = index;
    og.flux_sign[f] = sign;
    og.flux_u0[f] = u0;
    og.flux_u1[f] = u1;
    og.flux_v0[f] = v0;
    og.flux_v1[f] = v1;
    const long long faces = (long long)(u1 - u0) * (v1 - v0);
    int parts = (int)((faces + FDTD_FLUX_PART_FACES - 1) / FDTD_FLUX_PART_FACES);
    og.flux_parts[f] = std::max(1, std::min(kMaxFluxParts, parts));
    return FDTD_OK;
  }

  // Relative cost of a work item: planes (plus the recomputed plane below)
  // times a factor for each absorbing slab the tile's columns or planes cross.
  // Paired kernel: relative cost per plane of a tile's nodes (measured on the
  // 184^3 grid: tiles crossing an x slab 2.3x, a y slab 1.6x an interior
  // tile; a z-slab plane 2.25x an interior plane).
  double pair_tile_cost(int x0, int y0, int ox, int oy) const {
    auto crosses = [](int a0, int a1, int n, int L0, int L1) { return (L0 > 0 && a0 < L0) || (L1 > 0 && a1 > n - L1); };
    const bool sx = crosses(x0 - 2, x0 + ox, desc.nx, desc.npml[0], desc.npml[1]);
    const bool sy = crosses(y0 - 1, y0 + oy, desc.ny, desc.npml[2], desc.npml[3]);
    return 1.0 + 1.3 * sx + 0.6 * sy;
  }
  double pair_item_cost(const int4& it, int ox, int oy) const {
    const int z0 = it.w & 0xffff, z1 = (it.w >> 16) & 0xffff, kstart = z0 > 0 ? z0 - 1 : z0;
    int slab_planes = 0;
    for (int k = kstart; k < z1; ++k) slab_planes += (k < desc.npml[4] || k >= desc.nz - desc.npml[5]);
    return pair_tile_cost(it.y, it.z, ox, oy) * ((z1 - kstart) + 1.25 * slab_planes);
  }

  double item_cost(const int4& it, int ox, int oy) const {
    const int x0 = it.y, y0 = it.z, z0 = it.w & 0xffff, z1 = (it.w >> 16) & 0xffff;
    auto crosses = [](int a0, int a1, int n, int L0, int L1) { return (L0 > 0 && a0 < L0) || (L1 > 0 && a1 > n - L1); };
    const bool sx = crosses(x0 - 1, x0 + ox, desc.nx, desc.npml[0], desc.npml[1]);
    const bool sy = crosses(y0 - 1, y0 + oy, desc.ny, desc.npml[2], desc.npml[3]);
    const bool sz = crosses(z0 - 1, z1, desc.nz, desc.npml[4], desc.npml[5]);
    return (double)(z1 - z0 + 1) * (1.0 + 0.45 * sx + 0.25 * sy + 0.1 * sz + 0.3 * ((int)sx + sy + sz >= 2));
  }

  // Work items of one time step.  TMA kernel: tiles of 32 x by owned columns;
  // plain kernel: tiles of (bx-1) x (by-1) owned columns.  Each tile marches
  // z-ranges of `zdepth` planes (0: chosen so the items fill whole waves).
  void plan_items() {
    items.clear();
    const bool periodic = desc.periodic[0] || desc.periodic[1] || desc.periodic[2];
    const bool enc = tensor_map_encoder() != nullptr;
    // kind 0 (automatic): the paired kernel for passive binary32 grids, the
    // TMA kernel for gain and binary64 grids (measured faster there), the
    // plain-load kernel when an axis is periodic; by == 0: the chosen
    // kernel's default tile rows (paired 16, others 8)
    int kind = kernel_kind;
    if (kind == 0) kind = (sizeof(T) == 4 && !cell_gain()) ? 3 : 2;
    if (upml_grid()) kind = 1;  // its own H and E launches; nothing staged by TMA
    if (kind == 3 && sizeof(T) != 4) kind = 2;  // paired kernel: binary32 only
    use_pair = kind == 3 && !periodic && enc && (by == 0 || by == 8 || by == 16);
    if (kind == 3 && !use_pair) kind = 2;
    by_eff = by > 0 ? by : (use_pair ? 16 : 8);
    use_tma = use_pair || (kind == 2 && !periodic && (by_eff == 4 || by_eff == 8) && enc);
    tile_oy = by_eff;
    const int ox = use_tma ? kTmaOX : bx - 1;
    const int oy = use_tma ? tile_oy : by_eff - 1;
    const int tnx = (desc.nx + ox - 1) / ox, tny = (desc.ny + oy - 1) / oy;
    const int tiles = tnx * tny;
    int depth = zdepth;
    if (depth <= 0) {
      // short z-ranges (16 planes) with the slab-heavy items issued first
      // balance the load across SMs; small grids go shorter so the items fill
      // two waves
      int dev = 0, sms = 152;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaGetLastError();
      const int wave = sms * (use_pair ? step_pair_blocks_per_sm(cell_gain(), tile_oy)
                                       : step_blocks_per_sm<T>(use_tma, cell_gain(), bx, by_eff));
      // (8 for cell-coupled gain grids on the single-node TMA kernel: the gain
      // work per plane varies from tile to tile, and shorter items balance it;
      // measured on the 140^3 lasing grid 0.1168 ms per step with 8 planes,
      // ~0.119 with the 10 this rule gave from 16, 0.1337 with 16)
      depth = (use_tma && !use_pair && cell_gain()) ? 8 : 16;
      while (depth > 4 && (long long)tiles * ((desc.nz + depth - 1) / depth) < 2LL * wave) depth -= 2;
    }
    depth = std::min(depth, desc.nz);
    if (use_tma) depth = std::min(depth, kTmaZMax - 1);  // the item's planes' coefficients fit in shared memory
    std::vector<std::pair<double, int4>> work;
    if (use_pair && zdepth <= 0) {
      // Paired kernel, automatic depth: every tile cuts z at the slab edges
      // and takes z-ranges whose length falls with the tile's and the
      // segment's cost per plane, so the items run about equally long; the
      // costliest go first, and items of equal cost in z order (neighbouring
      // tiles of one z-range run together: their shared halo rows and
      // columns are read from DRAM once and then hit L2).
      const int cuts[4] = {0, std::min(desc.npml[4], desc.nz), std::max(desc.nz - desc.npml[5], std::min(desc.npml[4], desc.nz)), desc.nz};
      for (int ty = 0; ty < tny; ++ty)
        for (int tx = 0; tx < tnx; ++tx) {
          const double ct = pair_tile_cost(tx * ox, ty * oy, ox, oy);
          for (int seg = 0; seg < 3; ++seg) {
            const double cs = ct * (seg == 1 ? 1.0 : 2.25);
            const int d = std::max(4, std::min(depth, (int)std::lround(depth / cs)));
            for (int z0 = cuts[seg]; z0 < cuts[seg + 1]; z0 += d) {
              const int z1 = std::min(cuts[seg + 1], z0 + d);
              const int4 it = make_int4(0, tx * ox, ty * oy, z0 | (z1 << 16));
              work.push_back({pair_item_cost(it, ox, oy), it});
            }
          }
        }
      auto bucket = [](double c) { return (int)std::floor(std::log(c) / std::log(1.2)); };
      std::stable_sort(work.begin(), work.end(), [&](const std::pair<double, int4>& a, const std::pair<double, int4>& b) {
        const int ba = bucket(a.first), bb = bucket(b.first);
        if (ba != bb) return ba > bb;
        const int za = a.second.w & 0xffff, zb = b.second.w & 0xffff;
        if (za != zb) return za < zb;
        if (a.second.z != b.second.z) return a.second.z < b.second.z;
        return a.second.y < b.second.y;
      });
    } else {
      // Items generated in z order (z-range, row, column); by default the
      // costliest go first over the whole launch (items of equal cost stay in
      // z order), with FDTD_ORDER_Z all stay in z order, so the halo rows and
      // columns neighbouring tiles share are read while they sit in L2.
      for (int z0 = 0; z0 < desc.nz; z0 += depth) {
        const int z1 = std::min(desc.nz, z0 + depth);
        for (int ty = 0; ty < tny; ++ty)
          for (int tx = 0; tx < tnx; ++tx) {
            const int4 it = make_int4(0, tx * ox, ty * oy, z0 | (z1 << 16));
            work.push_back({item_cost(it, ox, oy), it});
          }
      }
      if (item_order != FDTD_ORDER_Z)
        std::stable_sort(work.begin(), work.end(), [](const std::pair<double, int4>& a, const std::pair<double, int4>& b) {
          return a.first > b.first;
        });
    }
    for (auto& w : work) items.push_back(w.second);
    oitems.clear();
    if (og.nprobe) oitems.push_back(make_int4(0, -1, 0, 1));
    for (int f = 0; f < og.nflux; ++f)
      for (int p = 0; p < og.flux_parts[f]; ++p) oitems.push_back(make_int4(0, f, p, og.flux_parts[f]));
  }

  // TMA descriptors of the fields (4D: x, y, z, array) and the material (3D).
  int encode_tma() {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return set_error(FDTD_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    TmaGrid h;
    std::memset(&h, 0, sizeof(h));
    const int AX = 16 / (int)sizeof(T);
    const cuuint64_t fdim[4] = {(cuuint64_t)desc.nx, (cuuint64_t)desc.ny, (cuuint64_t)desc.nz, 6 * kFieldSets};
    const cuuint64_t fstr[3] = {(cuuint64_t)px * sizeof(T), (cuuint64_t)px * desc.ny * sizeof(T),
                                (cuuint64_t)nstore * sizeof(T)};
    const cuuint32_t fbox[4] = {(cuuint32_t)(kTmaOX + 2 * AX), (cuuint32_t)(tile_oy + 2), 1, 6};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    CUresult r = enc(&h.fields, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                     (void*)d_F, fdim, fstr, fbox, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FDTD_E_CUDA, "tensor map (fields) encode failed: %d", (int)r);
    const cuuint64_t mdim[3] = {(cuuint64_t)desc.nx, (cuuint64_t)desc.ny, (cuuint64_t)desc.nz};
    const cuuint64_t mstr[2] = {(cuuint64_t)px, (cuuint64_t)px * desc.ny};
    const cuuint32_t mbox[3] = {(cuuint32_t)kTmaOX, (cuuint32_t)tile_oy, 1};
    r = enc(&h.mat, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void*)d_mat, mdim, mstr, mbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FDTD_E_CUDA, "tensor map (material) encode failed: %d", (int)r);
    cudaError_t e = cudaMemcpyAsync(d_tma, &h, sizeof(h), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_error(e, "upload tensor maps");
    return FDTD_OK;
  }

  bool upml_grid() const { return absorber == FDTD_ABSORBER_UPML; }

  // Uniaxial PML: the grading of every axis at integer and half-integer
  // nodes (the CPML's sigma dt/eps0 and kappa, no alpha) as the four factors
  // the update takes, and the auxiliary D~ and B~ arrays (zero).
  int prepare_upml() {
    if (d_upml) return FDTD_OK;
    const int n3[3] = {desc.nx, desc.ny, desc.nz};
    const size_t tab = (size_t)8 * (desc.nx + desc.ny + desc.nz);
    upml_aux_words = (size_t)6 * (size_t)nstore;
    d_upml = (T*)mem.get(sizeof(T) * (upml_aux_words + tab));
    if (!d_upml) return set_error(FDTD_E_NOMEM, "device allocation failed (UPML auxiliary fields)");
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_upml, 0, sizeof(T) * upml_aux_words, stream)) != cudaSuccess)
      return cuda_error(e, "memset UPML fields");
    for (int c = 0; c < 3; ++c) {
      upml.D[c] = d_upml + (size_t)c * nstore;
      upml.B[c] = d_upml + (size_t)(3 + c) * nstore;
    }
    for (int q = 0; q < 6; ++q) upml.L[q] = desc.npml[q];
    std::vector<T> h(tab);
    T* base = d_upml + upml_aux_words;
    size_t off = 0;
    const double sig_max = desc.cpml_sigma_factor * (desc.cpml_m + 1.0) * S / std::sqrt(desc.eps[0]);
    for (int d = 0; d < 3; ++d) {
      const int n = n3[d], L0 = desc.npml[2 * d], L1 = desc.npml[2 * d + 1];
      for (int hf = 0; hf < 2; ++hf)
        for (int qq = 0; qq < 4; ++qq) {
          upml.q[d][hf][qq] = base + off;
          for (int v = 0; v < n; ++v) {
            const double x = v + (hf ? 0.5 : 0.0);
            double rho = 0.0;
            if (L0 > 0 && x < L0) rho = (L0 - x) / L0;
            if (L1 > 0 && x > n - L1) rho = (x - (n - L1)) / L1;
            const double rm = std::pow(rho, desc.cpml_m);
            const double s = sig_max * rm, k = 1.0 + (desc.cpml_kappa_max - 1.0) * rm;
            const double val = qq == 0 ? (k - 0.5 * s) / (k + 0.5 * s)
                             : qq == 1 ? 1.0 / (k + 0.5 * s)
                             : qq == 2 ? k + 0.5 * s : k - 0.5 * s;
            h[off + v] = (T)val;
          }
          off += n;
        }
    }
    if ((e = cudaMemcpyAsync(base, h.data(), sizeof(T) * off, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload UPML grading");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "UPML set-up");
    return FDTD_OK;
  }

  int kernel_in_use_kind() const override { return upml_grid() ? 4 : (use_pair ? 3 : (use_tma ? 2 : 1)); }

  int finalize() override {
    cudaError_t e;
    if (upml_grid()) {
      if (sg.gain) return set_error(FDTD_E_INVAL, "the uniaxial PML runs passive grids (no gain medium)");
      const int r = prepare_upml();
      if (r != FDTD_OK) return r;
    }
    // recorders
    const long long cap = desc.record_capacity;
    og.cap = cap;
    if (og.nprobe) {
      og.probe_ring = (T*)mem.get(sizeof(T) * (size_t)cap * og.nprobe * 3);
      if (!og.probe_ring) return set_error(FDTD_E_NOMEM, "device allocation failed (probe ring)");
    }
    if (og.nflux) {
      og.flux_ring = (double*)mem.get(sizeof(double) * (size_t)cap * og.nflux);
      og.partials = (double*)mem.get(sizeof(double) * kMaxFlux * kMaxFluxParts);
      og.counters = (unsigned int*)mem.get(sizeof(unsigned int) * kMaxFlux);
      if (!og.flux_ring || !og.partials || !og.counters)
        return set_error(FDTD_E_NOMEM, "device allocation failed (flux recorder)");
      if ((e = cudaMemsetAsync(og.counters, 0, sizeof(unsigned) * kMaxFlux, stream)) != cudaSuccess)
        return cuda_error(e, "memset counters");
    }
    const int r = replan();
    // a grid frozen on a TMA-staged kernel cycles through three field sets,
    // so its observation can overlap the next step (set once, at step 0)
    if (r == FDTD_OK && steps == 0) sg.nsets = og.nsets = use_tma ? 3 : 2;
    return r == FDTD_OK ? upload_tables() : r;
  }

  size_t items_cap = 0, oitems_cap = 0;

  int replan() override {
    cudaError_t e;
    plan_items();
    if (use_tma) {
      const int r = encode_tma();
      if (r != FDTD_OK) return r;
    }
    if (items.size() > items_cap) {
      d_items = (int4*)mem.get(sizeof(int4) * items.size());
      items_cap = items.size();
    }
    if (!d_items) return set_error(FDTD_E_NOMEM, "device allocation failed (items)");
    if ((e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_error(e, "upload items");
    if (!oitems.empty()) {
      if (oitems.size() > oitems_cap) {
        d_oitems = (int4*)mem.get(sizeof(int4) * oitems.size());
        oitems_cap = oitems.size();
      }
      if (!d_oitems) return set_error(FDTD_E_NOMEM, "device allocation failed (items)");
      if ((e = cudaMemcpyAsync(d_oitems, oitems.data(), sizeof(int4) * oitems.size(), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_error(e, "upload items");
    }
    return upload_tables();
  }

  int upload_tables() {
    cudaError_t e;
    sg.step = og.step = steps;
    sg.step_end = og.step_end = step_limit;
    sg.wait_ns = wait_ns;
    tables_dirty = false;
    // a grid with the centred coupling steps its fields with the passive
    // step kernel (its record says: no gain) and runs the centred kernels after it
    rec_up = sg;
    if (!cell_gain()) rec_up.gain = 0;
    if (upml_grid())  // no CPML memory: the UPML launches grade the slabs themselves
      for (int d = 0; d < 3; ++d) {
        rec_up.Sd[d] = 0;
        rec_up.L[2 * d] = rec_up.L[2 * d + 1] = 0;
      }
    if ((e = cudaMemcpyAsync(d_sg, &rec_up, sizeof(sg), cudaMemcpyHostToDevice, stream)) != cudaSuccess) return cuda_error(e, "upload grid");
    if ((e = cudaMemcpyAsync(d_og, &og, sizeof(og), cudaMemcpyHostToDevice, stream)) != cudaSuccess) return cuda_error(e, "upload grid");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "upload grid");
    return FDTD_OK;
  }

  // The CPML memory (a few per cent of the state, but read and written at
  // latency-critical points of the slab planes) in a persisting L2 window on
  // the grid's stream: the device's persisting set-aside is raised to its
  // size (at most the device's maximum) and the window's hit ratio scaled to
  // what fits.  Measured on the 184^3 passive grid 0.1126 -> 0.1098 ms per
  // step, on the 140^3 lasing grid 0.1229 -> 0.1210 ms.
  int apply_l2_window(bool on) override {
    if (!d_psi || on == l2_applied) return FDTD_OK;
    cudaError_t e;
    cudaStreamAttrValue a{};
    if (on) {
      int dev = 0, max_persist = 0, max_window = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev)) != cudaSuccess)
        return cuda_error(e, "L2 attributes");
      if (max_persist <= 0 || max_window <= 0) return FDTD_OK;  // no persisting L2 on this device
      const size_t bytes = std::min(sizeof(T) * psi_words, (size_t)max_window);
      if ((e = cudaDeviceGetLimit(&l2_prior_limit, cudaLimitPersistingL2CacheSize)) != cudaSuccess)
        return cuda_error(e, "L2 persisting limit");
      const size_t want = std::min(bytes, (size_t)max_persist);
      if (l2_prior_limit < want && (e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want)) != cudaSuccess)
        return cuda_error(e, "L2 persisting limit");
      a.accessPolicyWindow.base_ptr = d_psi;
      a.accessPolicyWindow.num_bytes = bytes;
      a.accessPolicyWindow.hitRatio = std::min(1.0f, (float)std::max(l2_prior_limit, want) / (float)bytes);
      a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
      a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    } else {
      a.accessPolicyWindow.num_bytes = 0;  // no window
    }
    if ((e = cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &a)) != cudaSuccess)
      return cuda_error(e, "L2 access policy window");
    if (!on) {
      // its lines back to normal, and the set-aside back to what it was
      // before (a set-aside left in place kept L2 from the work after it:
      // measured 0.119 -> 0.182 ms per step on a lasing grid stepped next)
      cudaCtxResetPersistingL2Cache();
      cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, l2_prior_limit);
      cudaGetLastError();
    }
    l2_applied = on;
    return FDTD_OK;
  }
  size_t l2_prior_limit = 0;  // the persisting set-aside before this grid raised it

  ~GridImpl() override {
    cudaStreamSynchronize(stream);
    l2_forget(this);
    cudaGetLastError();
  }

  int step(long long n) override {
    cudaError_t e;
    if (tables_dirty) {
      const int r = upload_tables();
      if (r != FDTD_OK) return r;
    }
    if (l2_resident && !l2_applied && !stream_capturing(stream)) l2_claim(this);
    n = std::min(n, std::max(0LL, step_limit - steps));
    long long done = 0;
    // observation beside the next step's launch (paired kernel), else in line;
    // in line on three field sets, the TMA kernel's blocks of step s+1 start
    // while the observation of step s still runs (it reads sets s%3 and
    // (s+1)%3, step s+1 writes the third)
    const bool beside = use_pair && sg.nsets == 3 && !oitems.empty();
    const bool overlap = !beside && use_tma && !use_pair && sg.nsets == 3 && !oitems.empty() && !centred_gain();
    if (beside && (e = obs.ensure()) != cudaSuccess) return cuda_error(e, "observation stream");
    while (done < n) {
      const int chunk = (int)std::min<long long>(n - done, 1 << 20);
      for (int s = 0; s < chunk; ++s) {
        if (beside && (e = obs.before_step(stream, s)) != cudaSuccess) return cuda_error(e, "order");
        const auto ev = timer.next();
        if (ev.first) cudaEventRecord(ev.first, stream);
        if (upml_grid())
          e = launch_upml<T>(d_sg, upml, desc.nx, desc.ny, desc.nz, s, stream);
        else if (use_pair)
          e = launch_step_pair(reinterpret_cast<const StepGrid<float>*>(d_sg), d_tma, d_items, (int)items.size(), s,
                               tile_oy, cell_gain(), grid_blocks, stream);
        else if (use_tma)
          e = launch_step_tma<T>(d_sg, d_tma, d_items, (int)items.size(), s, tile_oy, cell_gain(), grid_blocks, stream,
                                 !(overlap && s > 0 && !ev.first));
        else
          e = launch_step<T>(d_sg, d_items, (int)items.size(), s, bx, by_eff, cell_gain(), grid_blocks, stream);
        if (e != cudaSuccess) return cuda_error(e, "step kernel");
        if (centred_gain() && (e = launch_centred<T>(d_sg, desc.nx, desc.ny, desc.nz, s, stream)) != cudaSuccess)
          return cuda_error(e, "centred coupling kernels");
        if (ev.second) cudaEventRecord(ev.second, stream);
        if (timer.used >= 4096) {
          if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
          timer.collect();
        }
        if (beside)
          e = obs.observe(stream, s, [&](cudaStream_t st) {
            return launch_observe<T>(d_og, d_oitems, (int)oitems.size(), s, st);
          });
        else if (!oitems.empty())
          e = launch_observe<T>(d_og, d_oitems, (int)oitems.size(), s, stream);
        if (e != cudaSuccess) return cuda_error(e, "observe kernel");
      }
      if (beside && (e = obs.join(stream, chunk)) != cudaSuccess) return cuda_error(e, "order");
      if ((e = launch_advance<T>(d_sg, d_og, 1, chunk, stream)) != cudaSuccess) return cuda_error(e, "advance");
      done += chunk;
      steps += chunk;
    }
    sg.step = og.step = steps;
    return FDTD_OK;
  }

  int read_field(int comp, double* out) override { return copy_out(sg.F[steps % sg.nsets][comp], out); }

  // word w of every node's gain state -> double[nz][ny][nx] on the host (one
  // strided copy: each 32-node record contributes its run of word w)
  int gain_word_out(int w, double* out) {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    const size_t run = sizeof(T) * 32;
    const size_t nruns = (size_t)sg.gxb * desc.ny * desc.nz;
    std::vector<T> h(nruns * 32);
    if ((e = cudaMemcpy2D(h.data(), run, d_gain + (size_t)32 * w, run * GainWords<T>::NW, run, nruns,
                          cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "read gain state");
    const size_t rowp = (size_t)sg.gxb * 32;
    for (long long k = 0; k < desc.nz; ++k)
      for (long long j = 0; j < desc.ny; ++j)
        for (long long i = 0; i < desc.nx; ++i)
          out[(k * desc.ny + j) * desc.nx + i] = (double)h[(size_t)(k * desc.ny + j) * rowp + (size_t)i];
    return FDTD_OK;
  }

  // device array in the pitched layout -> double[nz][ny][nx] on the host
  int copy_out(const T* src, double* out) {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    std::vector<T> h((size_t)ncell);
    if ((e = cudaMemcpy2D(h.data(), sizeof(T) * desc.nx, src, sizeof(T) * px, sizeof(T) * desc.nx,
                          (size_t)desc.ny * desc.nz, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "read");
    for (long long q = 0; q < ncell; ++q) out[q] = (double)h[q];
    return FDTD_OK;
  }

  int write_field(int comp, const double* in) override {
    std::vector<T> h((size_t)ncell);
    for (long long q = 0; q < ncell; ++q) h[q] = (T)in[q];
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    if ((e = cudaMemcpy2D(sg.F[steps % sg.nsets][comp], sizeof(T) * px, h.data(), sizeof(T) * desc.nx, sizeof(T) * desc.nx,
                          (size_t)desc.ny * desc.nz, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_error(e, "write");
    return FDTD_OK;
  }

  int read_gain(int what, double* out) override {
    if (!sg.gain) return set_error(FDTD_E_STATE, "no gain medium");
    int r;
    if (what == 0 || what == 1) {
      const int slot = (int)((steps + (what == 1 ? 1 : 0)) & 1);
      for (int c = 0; c < 3; ++c)
        if ((r = gain_word_out((slot ? GainWords<T>::P1 : GainWords<T>::P0) + c, out + (size_t)c * ncell)) != FDTD_OK)
          return r;
      return FDTD_OK;
    }
    std::vector<uint8_t> m((size_t)ncell);
    if ((r = get_material(m.data())) != FDTD_OK) return r;
    for (int c = 0; c < 3; ++c) {
      if ((r = gain_word_out(GainWords<T>::DN + c, out + (size_t)c * ncell)) != FDTD_OK) return r;
      for (long long q = 0; q < ncell; ++q) {
        double& v = out[(size_t)c * ncell + q];
        if (!((m[q] >> 6) & 1)) v = 0.0;
        else if (what == 2) v = n_total * (neq[c + 1] / n_total + v);
        else v = n_total * v;
      }
    }
    return FDTD_OK;
  }

  int read_probe(int id, long long t0, long long count, double* out) override {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    std::vector<T> ring((size_t)og.cap * og.nprobe * 3);
    if ((e = cudaMemcpy(ring.data(), og.probe_ring, sizeof(T) * ring.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "read probes");
    for (long long q = 0; q < count; ++q) {
      const size_t base = (size_t)((((t0 + q) % og.cap) * og.nprobe + id) * 3);
      for (int c = 0; c < 3; ++c) out[q * 3 + c] = (double)ring[base + c];
    }
    return FDTD_OK;
  }

  int read_flux(int id, long long t0, long long count, double* out) override {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    std::vector<double> ring((size_t)og.cap * og.nflux);
    if ((e = cudaMemcpy(ring.data(), og.flux_ring, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "read flux");
    for (long long q = 0; q < count; ++q) out[q] = ring[(size_t)(((t0 + q) % og.cap) * og.nflux + id)];
    return FDTD_OK;
  }

  int nprobes() const override { return og.nprobe; }
  int nfluxes() const override { return og.nflux; }
  long long capacity() const override { return og.cap; }

  int energy(double* out) override {
    const T* F6[6];
    for (int c = 0; c < 6; ++c) F6[c] = sg.F[steps % sg.nsets][c];
    cudaError_t e = launch_energy<T>(F6, d_mat, desc.eps[0], desc.eps[1], desc.eps[2], nstore, d_epart, d_ecount,
                                     d_energy, d_err, stream);
    if (e != cudaSuccess) return cuda_error(e, "energy kernel");
    double v = 0;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    if ((e = cudaMemcpy(&v, d_energy, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_error(e, "read energy");
    *out = 0.5 * eps0() * dx * dx * dx * v;
    return FDTD_OK;
  }

  int error_flags(int* flags) override {
    cudaError_t e;
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    if ((e = cudaMemcpy(flags, d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_error(e, "read flags");
    return FDTD_OK;
  }

  // state blobs for checkpointing: (device pointer, bytes)
  void state_blobs(std::vector<std::pair<void*, size_t>>& v) override {
    v.clear();
    v.push_back({d_F, sizeof(T) * 6 * kFieldSets * (size_t)nstore});
    v.push_back({(void*)d_mat, (size_t)nstore});
    if (d_psi) v.push_back({d_psi, sizeof(T) * psi_words});
    if (d_upml) v.push_back({d_upml, sizeof(T) * upml_aux_words});
    if (d_gain) v.push_back({d_gain, sizeof(T) * gain_words});
    if (og.probe_ring) v.push_back({og.probe_ring, sizeof(T) * (size_t)og.cap * og.nprobe * 3});
    if (og.flux_ring) v.push_back({og.flux_ring, sizeof(double) * (size_t)og.cap * og.nflux});
  }

  int field_sets() const override { return sg.nsets; }
  int adopt_field_sets(int from) override {
    if (from < 2 || from > kFieldSets) return set_error(FDTD_E_INVAL, "field sets %d", from);
    const int a = (int)(steps % from), b = (int)(steps % sg.nsets);
    if (a == b) return FDTD_OK;
    cudaError_t e;
    for (int c = 0; c < 6; ++c)
      if ((e = cudaMemcpyAsync(sg.F[b][c], sg.F[a][c], sizeof(T) * (size_t)nstore, cudaMemcpyDeviceToDevice, stream)) !=
          cudaSuccess)
        return cuda_error(e, "move the current field set");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_error(e, "sync");
    return FDTD_OK;
  }

  void set_steps(long long s) override {
    steps = s;
    sg.step = og.step = s;
  }

  // batch access
  const void* step_record() const override { return &sg; }
  const void* obs_record() const override { return &og; }
  size_t step_record_size() const override { return sizeof(sg); }
  size_t obs_record_size() const override { return sizeof(og); }
  int has_gain() const override { return sg.gain; }
  // gain coupled on each cell's own E nodes (inside the step kernels) / at the cell centre
  bool cell_gain() const { return sg.gain != 0 && coupling == FDTD_COUPLING_CELL; }
  bool centred_gain() const { return sg.gain != 0 && coupling == FDTD_COUPLING_CENTRED; }
  StepGrid<T> rec_up{};  // the record as uploaded
  const void* tma_device() const override { return d_tma; }
  bool uses_tma() const override { return use_tma; }
  bool uses_pair() const override { return use_pair; }
  int tile_rows() const override { return use_tma ? tile_oy : by_eff - 1; }
  void work_items(std::vector<int4>& si, std::vector<int4>& oi) const override {
    si = items;
    oi = oitems;
  }
};

namespace {
std::mutex g_l2_mutex;
GridBase* g_l2_owner[64] = {};  // per device ordinal
}  // namespace

void l2_claim(GridBase* g) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lock(g_l2_mutex);
  GridBase*& owner = g_l2_owner[dev];
  if (owner == g) {
    if (g && !g->l2_applied) g->apply_l2_window(true);
    return;
  }
  if (owner) owner->apply_l2_window(false);
  owner = nullptr;
  if (g && g->apply_l2_window(true) == FDTD_OK && g->l2_applied) owner = g;
  cudaGetLastError();  // a cache placement: failures leave the grid without a window
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

void l2_forget(GridBase* g) {
  std::lock_guard<std::mutex> lock(g_l2_mutex);
  for (auto& owner : g_l2_owner)
    if (owner == g) {
      g->apply_l2_window(false);
      owner = nullptr;
    }
  cudaGetLastError();
}

GridBase* make_grid(const fdtd_grid_desc& d) {
  if (d.precision == FDTD_FP32) return new (std::nothrow) GridImpl<float>();
  return new (std::nothrow) GridImpl<double>();
}

int init_grid(GridBase* g) {
  if (g->precision() == FDTD_FP32) return static_cast<GridImpl<float>*>(g)->init();
  return static_cast<GridImpl<double>*>(g)->init();
}

}  // namespace fdtd
