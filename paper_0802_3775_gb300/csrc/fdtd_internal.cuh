// Internal declarations of the GB300 Maxwell-Bloch FDTD library.
//
// Device-side grid records and kernel launchers shared by the library's
// translation units.  Nothing here is part of the C ABI (include/fdtd.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

constexpr int kMaxSrc = 8;
constexpr int kMaxProbes = 64;
constexpr int kMaxFlux = 16;
constexpr int kMaxFluxParts = 1024;  // most blocks of one flux plane
constexpr int kEnergyBlocks = 256;
#ifndef FDTD_TMA_STAGES
#define FDTD_TMA_STAGES 3
#endif
constexpr int kTmaStages = FDTD_TMA_STAGES;  // planes resident or in flight per block (TMA step kernel)
constexpr int kTmaOX = 32;        // owned tile width of the TMA step kernel
constexpr int kTmaZMax = 32;      // planes of one TMA work item, its lower halo plane included
// New field values leave the step kernels with the evict-first store hint
// (1): nothing in the launch reads them, and L2 stays with the halo rows
// that neighbouring tiles read and the CPML memory.  Measured: 184^3
// passive step 0.1101 -> 0.1089 ms, 140^3 lasing 0.1217 -> 0.1197 ms.
#ifndef FDTD_STREAM_STORES
#define FDTD_STREAM_STORES 1
#endif

// Field sets: a grid cycles through `nsets` (2 or 3) of the kFieldSets
// allocated sets; set n % nsets holds E^n and H~^{n-1/2} and step n writes set
// (n+1) % nsets.  With three, the observation of step n (sets n%3 and
// (n+1)%3) can run while step n+1 writes the third set.
constexpr int kFieldSets = 3;

// Physical constants (CODATA; mu0 of the 2019 SI, hbar exact).
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kHbar = 1.054571817e-34;
inline double eps0() { return 1.0 / (kMu0 * kC0 * kC0); }
inline double eta0() { return kMu0 * kC0; }

// One soft current source (Gaussian-modulated sine; see fdtd_add_source).
struct SrcDev {
  int kind;          // 0 point, 1 sheet
  int comp;          // driven E component
  int axis, index;   // sheet plane
  int i, j, k;       // point node
  int lo1, hi1, lo2, hi2;  // sheet transverse node ranges along (axis+1)%3, (axis+2)%3
  double uc, vc;     // profile centre (node index units)
  double inv_w2;     // 1/waist^2 (0: uniform)
  double amp;        // amplitude (V/m per step)
  double f0dt;       // f0 * dt
  double tau;        // envelope width in steps
  double t0;         // envelope centre in steps
};

// Words of a node's gain state: P~ in two time slots (x, y, z each), dN~1..3,
// and in binary32 runs three compensation words of the dN~ sums.
template <typename T>
struct GainWords {
  static constexpr int NW = sizeof(T) == 4 ? 12 : 9;
  static constexpr int P0 = 0, P1 = 3, DN = 6, CMP = 9;  // first word of each group
};

// Per-grid record read by the step kernel.  Lives in device memory (a table
// of them for a batched launch); each block copies its grid's record into
// shared memory.
template <typename T>
struct StepGrid {
  int nx, ny, nz;
  int px;               // x pitch of field, material and gain arrays (elements)
  int per;              // bit d set: axis d periodic
  int L[6];             // slab thickness x-,x+,y-,y+,z-,z+
  int Sd[3];            // slab extent per axis (L[2d] + L[2d+1])
  int gain;             // gain medium present
  int nsrc;
  long long step;       // steps completed before this launch sequence
  long long step_end;   // no update n >= step_end is performed
  long long wait_ns;    // limit of a bounded wait of the TMA step kernels (ns; <= 0: give up at once)
  T* F[kFieldSets][6];  // field sets (set n%nsets: E^n, H~^{n-1/2}): Ex Ey Ez Hx Hy Hz
  int nsets;            // field sets in the cycle (2 or 3)
  const uint8_t* mat;   // material bytes
  T* psiE[3][2];        // E-curl CPML memory per axis, slot 0 -> comp (d+1)%3, 1 -> (d+2)%3
  T* psiH[2][3][2];     // H-curl CPML memory, ping-pong like the fields
  const T* prof[3][2][3];  // [axis][0 E-node (integer), 1 H-node (half-integer)][1/kappa, b, c]
  T cH;                 // S
  T cE[3], cP[3];       // S/eps_r and 1/eps_r per material class
  // gain medium (normalized populations N~ = N / n_total): the state words
  // of each run of 32 x-adjacent nodes of a row lie together (see gain_base)
  T* gst;               // gain state: P~ slot 0 and 1 (slot n&1 holds P^n), dN~1..3, compensation words
  int gxb;              // 32-node blocks per row of the gain state (ceil(nx / 32))
  T a1, a2, a3, n12eq, q, noise;
  T D[3][3], w[3];
  unsigned long long seed;
  int* err;             // bit 1: a bounded wait of the step kernel ran out; bit 2: a drain after it ran out too
  SrcDev src[kMaxSrc];
};

// Per-grid record read by the observation kernel (probes, flux).
template <typename T>
struct ObsGrid {
  int nx, ny, nz;
  int px;               // x pitch
  int nprobe, nflux;
  long long step;       // as StepGrid::step
  long long step_end;
  long long cap;        // recorder ring length (steps)
  double dx2_over_eta0; // dx^2 / eta0
  const T* F[kFieldSets][6];
  int nsets;
  int probe[kMaxProbes][3];
  T* probe_ring;        // [cap][nprobe][3]
  int flux_axis[kMaxFlux], flux_index[kMaxFlux];
  int flux_u0[kMaxFlux], flux_u1[kMaxFlux], flux_v0[kMaxFlux], flux_v1[kMaxFlux];
  int flux_parts[kMaxFlux];
  double flux_sign[kMaxFlux];
  double* flux_ring;    // [cap][nflux]
  double* partials;     // [kMaxFlux][kMaxFluxParts] scratch
  unsigned int* counters;  // [kMaxFlux] scratch, zero between launches
  int* err;             // bit 0: non-finite value seen
};

// TMA descriptors of one grid: all twelve field arrays as one 4D tensor
// (x, y, z, array) read with a box of (32 + 2 pad) x (tile rows + 2) x 1 x 6,
// and the material bytes as a 3D tensor read with a box of 32 x rows x 1.
struct alignas(128) TmaGrid {
  CUtensorMap fields;
  CUtensorMap mat;
};

// Work items of the step kernel: (grid, x0, y0, z0 | z1 << 16).
// Work items of the observation kernel: (grid, what, part, nparts) with
// what = -1 for the probes and f >= 0 for flux plane f.

template <typename T>
cudaError_t launch_step(const StepGrid<T>* grids, const int4* items, int nitems, int offset, int bx, int by,
                        bool gain, int grid_blocks, cudaStream_t st);

// wait_prev false: the launch before it is the observation of the step before
// on a grid of three field sets, and its blocks start without waiting for it.
template <typename T>
cudaError_t launch_step_tma(const StepGrid<T>* grids, const TmaGrid* maps, const int4* items, int nitems, int offset,
                            int oy, bool gain, int grid_blocks, cudaStream_t st, bool wait_prev = true);

template <typename T>
size_t step_tma_smem_bytes(int oy);

// Paired binary32 step kernel (two x-adjacent nodes per thread, f32x2
// arithmetic): tiles of 32 x oy columns (oy 8 or 16), the TMA descriptors of
// the single-node TMA kernel for the same oy.
cudaError_t launch_step_pair(const StepGrid<float>* grids, const TmaGrid* maps, const int4* items, int nitems,
                             int offset, int oy, bool gain, int grid_blocks, cudaStream_t st);
size_t step_pair_smem_bytes(int oy);
int step_pair_blocks_per_sm(bool gain, int oy);

// Resident blocks per SM of the step kernel for a launch shape.
template <typename T>
int step_blocks_per_sm(bool tma, bool gain, int bx, int by);

template <typename T>
cudaError_t launch_observe(const ObsGrid<T>* grids, const int4* items, int nitems, int offset, cudaStream_t st);

// Shared-memory bytes of one step block.
template <typename T>
size_t step_smem_bytes(int bx, int by);

// Advance every grid's step counters after a launch sequence of `count` steps.
template <typename T>
cudaError_t launch_advance(StepGrid<T>* sg, ObsGrid<T>* og, int ngrids, int count, cudaStream_t st);

// Rasterization of binned spheres (see fdtd_set_eps_from_spheres).
// fspheres: 8 floats per sphere, (floor cx, floor cy, floor cz, r^2) and
// (cx, cy, cz) - floor(.), rounded to binary32 (16-byte aligned).
cudaError_t launch_rasterize(uint8_t* mat, int nx, int ny, int nz, int px, const double* spheres,
                             const float* fspheres, const int* bin_start, const int* bin_list, int bin, int bnx, int bny,
                             int bnz, const double* box, cudaStream_t st);

// Uniaxial PML of a passive grid: grading tables and auxiliary fields.
template <typename T>
struct UpmlDev {
  const T* q[3][2][4];  // [axis][0 integer node, 1 half-integer node][(k - s/2)/(k + s/2), 1/(k + s/2), k + s/2, k - s/2]
  T* D[3];              // auxiliary D~ of the E nodes (read and written at graded nodes only)
  T* B[3];              // auxiliary B~ of the H~ nodes
  int L[6];             // slab thickness x-,x+,y-,y+,z-,z+
};

// One time step of a grid with the uniaxial PML: the H~ and E launches.
template <typename T>
cudaError_t launch_upml(const StepGrid<T>* g, const UpmlDev<T>& u, int nx, int ny, int nz, int offset,
                        cudaStream_t st);

// Centred Bloch coupling of a gain grid: the polarization, current and
// population kernels that follow the (passive) step kernel of step offset.
template <typename T>
cudaError_t launch_centred(const StepGrid<T>* g, int nx, int ny, int nz, int offset, cudaStream_t st);

// Gain initialization: P slots zero, dN~ = init - N~eq in gain cells.
template <typename T>
cudaError_t launch_gain_init(const StepGrid<T>* g_host_copy, long long nslots, T d1, T d2, T d3, cudaStream_t st);

// Field energy sum (eps_r E^2 + H~^2) over the cells in FP64; result in out[0].
template <typename T>
cudaError_t launch_energy(const T* const* F6, const uint8_t* mat, double e0, double e1, double e2,
                          long long ncell, double* partials, unsigned int* counter, double* out, int* err,
                          cudaStream_t st);

// Convert between the run precision and double (read / write of state).
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_from_double(const double* src, T* dst, long long n, cudaStream_t st);

}  // namespace fdtd
