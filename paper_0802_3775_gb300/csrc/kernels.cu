// Device kernels of the GB300 Maxwell-Bloch FDTD library (sm_103a).
//
// k_step_tma  one time step n -> n+1 of a list of work items (32-column x
//             OY-row tile x z-range of some grid), non-periodic grids.  The
//             tile marches in z; each plane of all six fields (tile plus a
//             one-node halo, x padded to 16-byte alignment) and the tile's
//             material bytes arrive in shared memory by two TMA bulk-tensor
//             copies into a 3-stage mbarrier pipeline (the current plane, the
//             next one, one in flight).  H on the -x / -y halo is recomputed
//             so no block needs a neighbour's output of the same step; fields
//             cycle through nsets sets (read set n % nsets, write the next),
//             H-side CPML memory is double-buffered (read set n&1, write
//             set (n+1)&1); E-side CPML memory and gain state are updated in
//             place by the owning thread; new values are stored from
//             registers; H of a plane goes to one of two shared buffers, so
//             one block barrier per plane suffices.
// k_step      the same step with plain loads and register prefetch of the
//             next plane; any boundary, including periodic axes.
// k_observe   probes (E^{n+1}) and Poynting flux T^n per plane with a
//             fixed-order FP64 reduction (bitwise reproducible).
// k_energy    field energy in FP64, fixed-order reduction.
// k_rasterize sphere list -> material bytes (FP64, no contraction).
//
// Paper: Yee FDTD (Sec. "Sample and numerical approach"), four-level
// Maxwell-Bloch gain solved at the Yee cell (same section), spontaneous-
// emission noise as a random kick (same section), pulsed sources and flux T(t) (Secs.
// "Wide-band excitation", "Dynamical diffusion").
#include <math.h>

#include "cell.cuh"
#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

// Index along an axis of length n: wrapped when periodic, otherwise flagged
// invalid (v = false, reads as zero) outside [0, n).
__device__ __forceinline__ int wrap_index(int i, int n, bool periodic, bool& v) {
  if (i >= 0 && i < n) {
    v = true;
    return i;
  }
  if (periodic) {
    v = true;
    int r = i % n;
    return r < 0 ? r + n : r;
  }
  v = false;
  return 0;
}

template <typename T>
__device__ __forceinline__ T ldz(const T* __restrict__ a, bool v, long long idx) {
  return v ? __ldg(a + idx) : T(0);
}

// =====================================================================
// Plain-load step kernel (any boundary)
// =====================================================================
template <typename T>
size_t step_smem_bytes(int bx, int by) {
  const size_t gs = align128(sizeof(StepGrid<T>));
  const size_t planes = (size_t)3 * (bx + 1) * (by + 1) + (size_t)3 * bx * by;
  return gs + kMaxSrc * sizeof(double) + planes * sizeof(T);
}

template <typename T, bool GAIN>
__global__ void __launch_bounds__(512) k_step(const StepGrid<T>* __restrict__ grids, const int4* __restrict__ items,
                                              int nitems, int offset) {
  extern __shared__ __align__(128) unsigned char smem[];
  StepGrid<T>& G = *reinterpret_cast<StepGrid<T>*>(smem);
  constexpr size_t GS = align128(sizeof(StepGrid<T>));
  double* sg = reinterpret_cast<double*>(smem + GS);
  T* sbase = reinterpret_cast<T*>(smem + GS + kMaxSrc * sizeof(double));
  const int bx = blockDim.x, by = blockDim.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * bx + tx;
  const int EW = bx + 1;
  const int EP = (bx + 1) * (by + 1);
  const int HP = bx * by;
  T* sEx = sbase;
  T* sEy = sEx + EP;
  T* sEz = sEy + EP;
  T* sHx = sEz + EP;
  T* sHy = sHx + HP;
  T* sHz = sHy + HP;
  const int se = ty * EW + tx;  // this thread's slot in an E plane

  int cur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = items[it];
    __syncthreads();
    if (item.x != cur) {
      load_record(grids + item.x, smem, tid, bx * by);
      cur = item.x;
    }
    __syncthreads();
    const long long n = G.step + offset;
    if (n >= G.step_end) continue;
    source_waveforms(G, n, tid, sg, item.w & 0xffff, (item.w >> 16) & 0xffff);
    __syncthreads();

    const int nx = G.nx, ny = G.ny, nz = G.nz, px = G.px;
    const bool perx = G.per & 1, pery = G.per & 2, perz = G.per & 4;
    const int x0 = item.y, y0 = item.z, z0 = item.w & 0xffff, z1 = (item.w >> 16) & 0xffff;
    const int i = x0 - 1 + tx, j = y0 - 1 + ty;
    bool vx, vy, vxp, vyp;
    const int iw = wrap_index(i, nx, perx, vx);
    const int jw = wrap_index(j, ny, pery, vy);
    const bool valid = vx && vy;
    const bool xcol = (tx == bx - 1), yrow = (ty == by - 1);
    const int ip = wrap_index(i + 1, nx, perx, vxp);
    const int jp = wrap_index(j + 1, ny, pery, vyp);
    const bool vcol = xcol && vxp && vy;  // extra column node (i+1, j) exists
    const bool vrow = yrow && vx && vyp;  // extra row node (i, j+1) exists
    const bool owner = tx > 0 && ty > 0 && i < nx && j < ny;

    const int sel = (int)(n & 1);                   // parity: CPML memory and gain slots
    const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;  // field sets read / written
    const T* __restrict__ Ex = G.F[fs][0];
    const T* __restrict__ Ey = G.F[fs][1];
    const T* __restrict__ Ez = G.F[fs][2];
    const T* __restrict__ Hx = G.F[fs][3];
    const T* __restrict__ Hy = G.F[fs][4];
    const T* __restrict__ Hz = G.F[fs][5];

    auto kwrap = [&](int k, bool& v) { return wrap_index(k, nz, perz, v); };

    const int kstart = (z0 > 0 || perz) ? z0 - 1 : z0;
    bool vk0, vk1;
    const int kw0 = kwrap(kstart, vk0);
    const int kw1 = kwrap(kstart + 1, vk1);
    const long long c0 = pidx3(iw, jw, kw0, px, ny);
    const long long c1 = pidx3(iw, jw, kw1, px, ny);
    T eCx = ldz(Ex, valid && vk0, c0), eCy = ldz(Ey, valid && vk0, c0), eCz = ldz(Ez, valid && vk0, c0);
    T eNx = ldz(Ex, valid && vk1, c1), eNy = ldz(Ey, valid && vk1, c1), eNz = ldz(Ez, valid && vk1, c1);
    T hOx = ldz(Hx, valid && vk0, c0), hOy = ldz(Hy, valid && vk0, c0), hOz = ldz(Hz, valid && vk0, c0);
    T xCy, xCz, yCx, yCz;
    {
      const long long cc = pidx3(ip, jw, kw0, px, ny);
      const long long cr = pidx3(iw, jp, kw0, px, ny);
      xCy = ldz(Ey, vcol && vk0, cc);
      xCz = ldz(Ez, vcol && vk0, cc);
      yCx = ldz(Ex, vrow && vk0, cr);
      yCz = ldz(Ez, vrow && vk0, cr);
    }
    T hPx = T(0), hPy = T(0);
    Column col;
    make_column(G, iw, jw, col, owner);

    for (int k = kstart; k < z1; ++k) {
      bool vk;
      const int kw = kwrap(k, vk);
      const bool active = k >= z0;
      const Plane pl = make_plane(G, kw);
      // prefetch the next plane
      T eNNx = T(0), eNNy = T(0), eNNz = T(0), hONx = T(0), hONy = T(0), hONz = T(0);
      T xNy = T(0), xNz = T(0), yNx = T(0), yNz = T(0);
      if (k + 1 < z1) {
        bool va, vb;
        const int ka = kwrap(k + 1, va);
        const int kb = kwrap(k + 2, vb);
        const long long ca = pidx3(iw, jw, ka, px, ny);
        const long long cb = pidx3(iw, jw, kb, px, ny);
        eNNx = ldz(Ex, valid && vb, cb);
        eNNy = ldz(Ey, valid && vb, cb);
        eNNz = ldz(Ez, valid && vb, cb);
        hONx = ldz(Hx, valid && va, ca);
        hONy = ldz(Hy, valid && va, ca);
        hONz = ldz(Hz, valid && va, ca);
        const long long cc = pidx3(ip, jw, ka, px, ny);
        const long long cr = pidx3(iw, jp, ka, px, ny);
        xNy = ldz(Ey, vcol && va, cc);
        xNz = ldz(Ez, vcol && va, cc);
        yNx = ldz(Ex, vrow && va, cr);
        yNz = ldz(Ez, vrow && va, cr);
      }
      const long long cidx = pidx3(iw, jw, kw, px, ny);
      unsigned m = 0;
      if (owner && active) m = __ldg(G.mat + cidx);

      // stage E^n of plane k
      sEx[se] = eCx;
      sEy[se] = eCy;
      sEz[se] = eCz;
      if (xcol) {
        sEy[se + 1] = xCy;
        sEz[se + 1] = xCz;
      }
      if (yrow) {
        sEx[se + EW] = yCx;
        sEz[se + EW] = yCz;
      }
      __syncthreads();

      T hx = T(0), hy = T(0), hz = T(0);
      if (valid && vk) {
        h_node(G, col, pl, sel, owner && active, CoefGlobal<T>{&G, col.i, col.j, pl.k}, sEz[se + EW] - eCz, eNy - eCy, eNx - eCx, sEz[se + 1] - eCz,
               sEy[se + 1] - eCy, sEx[se + EW] - eCx, hOx, hOy, hOz, hx, hy, hz);
      }
      sHx[tid] = hx;
      sHy[tid] = hy;
      sHz[tid] = hz;
      __syncthreads();

      if (owner && active) {
        const bool gcell = GAIN && G.gain && ((m >> 6) & 1);
        GainState<T> gs{};
        const long long gidx = GAIN ? gain_base(G, iw, jw, kw) : 0;
        if (GAIN && gcell) load_gain(G, sel, gidx, gs);
        T enx, eny, enz;
        e_node<T, GAIN>(G, sg, col, pl, sel, n, gidx, m, gcell, gs, CoefGlobal<T>{&G, col.i, col.j, pl.k}, hz - sHz[tid - bx], hy - hPy, hx - hPx,
                        hz - sHz[tid - 1], hy - sHy[tid - 1], hx - sHx[tid - bx], eCx, eCy, eCz, enx, eny, enz);
        G.F[fo][0][cidx] = enx;
        G.F[fo][1][cidx] = eny;
        G.F[fo][2][cidx] = enz;
        G.F[fo][3][cidx] = hx;
        G.F[fo][4][cidx] = hy;
        G.F[fo][5][cidx] = hz;
      }

      hPx = hx;
      hPy = hy;
      eCx = eNx; eCy = eNy; eCz = eNz;
      eNx = eNNx; eNy = eNNy; eNz = eNNz;
      hOx = hONx; hOy = hONy; hOz = hONz;
      xCy = xNy; xCz = xNz; yCx = yNx; yCz = yNz;
    }
  }
}

template <typename T>
cudaError_t launch_step(const StepGrid<T>* grids, const int4* items, int nitems, int offset, int bx, int by,
                        bool gain, int grid_blocks, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = step_smem_bytes<T>(bx, by);
  const int blocks = (grid_blocks > 0 && grid_blocks < nitems) ? grid_blocks : nitems;
  dim3 blk(bx, by);
  if (gain) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_step<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_step<T, true><<<blocks, blk, smem, st>>>(grids, items, nitems, offset);
  } else {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_step<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_step<T, false><<<blocks, blk, smem, st>>>(grids, items, nitems, offset);
  }
  return cudaGetLastError();
}

// =====================================================================
// TMA-staged step kernel (non-periodic grids)
// =====================================================================

// Byte layout of the TMA kernel's shared memory (host and device agree).
template <typename T, int OY>
struct TmaLayout {
  static constexpr int AX = 16 / (int)sizeof(T);  // x pad: one 16-byte unit each side
  static constexpr int BXT = kTmaOX + 2 * AX;     // staged box width
  static constexpr int BYT = OY + 2;              // staged box height (rows y0-1 .. y0+OY)
  static constexpr int PL = BXT * BYT;            // elements of one component plane in a stage
  static constexpr int HW = kTmaOX + 1;           // row length of the H plane buffer
  static constexpr int HPL = (OY + 1) * HW;
  static constexpr size_t sg_off = align128(sizeof(StepGrid<T>));
  static constexpr size_t bar_off = sg_off + align128(kMaxSrc * sizeof(double));
  static constexpr size_t stage_off = bar_off + 128;
  static constexpr int NT = kTmaOX * OY;          // threads = owned nodes of a tile plane
  static constexpr int NH = kTmaOX + OY;           // halo nodes (-y row, -x column)
  static constexpr size_t field_bytes = align128((size_t)6 * PL * sizeof(T));
  static constexpr size_t mat_bytes = align128((size_t)kTmaOX * OY);
  // CPML memory fetched ahead per thread: 4 slots per owned node, 2 per halo node
  static constexpr size_t psi_bytes = align128((size_t)(4 * NT + 2 * NH) * sizeof(T));
  static constexpr size_t stage_bytes = field_bytes + mat_bytes + psi_bytes;
  // H of the plane, two buffers (plane p uses p & 1)
  static constexpr size_t hbuf_bytes = align128((size_t)3 * HPL * sizeof(T));
  static constexpr size_t h_off = stage_off + (size_t)kTmaStages * stage_bytes;
  // CPML grading coefficients of the item: (OX + 1) columns, (OY + 1) rows
  // (the -x / -y halo first) and up to kTmaZMax planes, 6 values each
  static constexpr int CXN = (kTmaOX + 1) * 6, CYN = (OY + 1) * 6, CZN = kTmaZMax * 6;
  static constexpr size_t coef_off = h_off + 2 * hbuf_bytes;
  static constexpr size_t total = coef_off + (size_t)(CXN + CYN + CZN) * sizeof(T) + 128;  // + base alignment slack
};

template <typename T>
size_t step_tma_smem_bytes(int oy) {
  return oy == 4 ? TmaLayout<T, 4>::total : TmaLayout<T, 8>::total;
}

// Four resident blocks of 256 threads per SM (64 registers a thread): the
// sweep of launch shapes on GB300 favoured occupancy over the extra registers.
#ifndef FDTD_TMA_MIN_BLOCKS
#define FDTD_TMA_MIN_BLOCKS 4
#endif

// Threads of a TMA-kernel block.  Binary32: OY warps, one row of 32 nodes
// each, warps 0 and 1 also recomputing H on the -y halo row and the -x halo
// column; 4 blocks per SM at 64 registers (two extra halo warps measured 5 %
// slower on the 140^3 gain grid: fewer resident warps).  Binary64, whose
// blocks shared memory limits to 2 per SM at 8 rows (3 at 4): two extra
// warps recompute the halo row and column, so every warp carries one H
// update per plane, with registers for 2 (3) blocks (the 184^3 binary64 step
// 0.583 -> 0.531 ms; the register budget alone gave 0.569 ms).
template <typename T, int OY>
struct TmaThreads {
  static constexpr bool HALO_WARPS = sizeof(T) == 8;
  static constexpr int ROWS = OY + (HALO_WARPS ? 2 : 0);  // blockDim.y
  static constexpr int NT = kTmaOX * ROWS;
  static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? FDTD_TMA_MIN_BLOCKS * 8 / OY : (OY == 8 ? 2 : 3);
};

template <typename T, bool GAIN, int OY>
__global__ void __launch_bounds__(TmaThreads<T, OY>::NT, TmaThreads<T, OY>::MIN_BLOCKS)
    k_step_tma(const StepGrid<T>* __restrict__ grids, const TmaGrid* __restrict__ maps,
               const int4* __restrict__ items, int nitems, int offset, int wait_prev) {
  using L = TmaLayout<T, OY>;
  constexpr int OX = kTmaOX;
  constexpr int S = kTmaStages;
  constexpr int AX = L::AX, BXT = L::BXT, PL = L::PL, HW = L::HW, HPL = L::HPL;
  constexpr unsigned TX_BYTES = (unsigned)(6 * PL * sizeof(T) + OX * OY);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA sources and destinations need 128-byte alignment: align the dynamic base explicitly
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  StepGrid<T>& G = *reinterpret_cast<StepGrid<T>*>(smem);
  double* sg = reinterpret_cast<double*>(smem + L::sg_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::bar_off);
  unsigned char* stages = smem + L::stage_off;
  T* cfx = reinterpret_cast<T*>(smem + L::coef_off);
  T* cfy = cfx + L::CXN;
  T* cfz = cfy + L::CYN;
  using TT = TmaThreads<T, OY>;
  constexpr int NTALL = TT::NT;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * OX + tx;
  const bool owner = !TT::HALO_WARPS || ty < OY;            // rows 0..OY-1 of the tile
  const bool hwrow = TT::HALO_WARPS ? ty == OY : ty == 0;    // recomputes the -y halo row
  const bool hwcol = TT::HALO_WARPS ? ty == OY + 1 : ty == 1;  // lanes 0..OY-1: the -x halo column

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  // the launch before this one (observation or step) has finished; after the
  // observation of the step before (wait_prev 0) the block starts at once:
  // that observation began after the step it observes had finished, and on
  // three field sets it reads neither the set this step writes nor anything
  // else this step touches
  if (wait_prev) grid_dependency_wait();
  allow_dependents();
  __syncthreads();

  unsigned ld = 0;  // plane loads issued by this block so far (same value in every thread)
  IssuedLoads loads;  // thread 0: the loads it issued, drained if the block gives up
  int cur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = items[it];
    __syncthreads();
    const bool fresh = item.x != cur;
    if (fresh) {
      load_record(grids + item.x, smem, tid, NTALL);
      cur = item.x;
    }
    __syncthreads();
    const long long n = G.step + offset;
    if (n >= G.step_end) continue;
    source_waveforms(G, n, tid, sg, item.w & 0xffff, (item.w >> 16) & 0xffff);

    const int nx = G.nx, ny = G.ny, px = G.px;
    const int x0 = item.y, y0 = item.z, z0 = item.w & 0xffff, z1 = (item.w >> 16) & 0xffff;
    const int kstart = z0 > 0 ? z0 - 1 : z0;
    const int NP = z1 - kstart + 1;  // planes kstart .. z1 (E of plane z1 feeds H of plane z1-1)
    const int sel = (int)(n & 1);                   // parity: CPML memory and gain slots
    const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;  // field sets read / written
    const CUtensorMap* fmap = &maps[item.x].fields;
    const CUtensorMap* mmap = &maps[item.x].mat;
    const unsigned q0 = ld;

    auto issue = [&](unsigned q, int plane) {
      const int s = (int)(q % S);
      unsigned char* dst = stages + (size_t)s * L::stage_bytes;
      loads.note(s);
      mbar_arrive_expect_tx(&full[s], TX_BYTES);
      tma_load_4d(dst, fmap, x0 - AX, y0 - 1, plane, fs * 6, &full[s]);
      tma_load_3d(dst + L::field_bytes, mmap, x0, y0, plane, &full[s]);
    };
    if (tid == 0) {
      if (fresh) {
        tensormap_acquire(fmap);
        tensormap_acquire(mmap);
      }
      fence_proxy_async_smem();
      for (int p = 0; p < S && p < NP; ++p) issue(q0 + p, kstart + p);
    }
    ld = q0 + (unsigned)(NP < S ? NP : S);
    __syncthreads();

    const int i = x0 + tx, j = y0 + ty;
    const bool own = owner && i < nx && j < ny;
    constexpr int xo = AX;      // own node: staged column tx + AX, row ty + 1
    const int oe = (ty + 1) * BXT + tx + xo;
    const int oh = (ty + 1) * HW + tx + 1;
    Column col;
    make_column(G, own ? i : 0, own ? j : 0, col, true);
    const long long cbase = (long long)j * px + i;
    const long long pstride = (long long)px * ny;
    // gain state of the own node in plane 0 and the stride between planes
    const long long gbase = GAIN ? gain_base(G, own ? i : 0, own ? j : 0, 0) : 0;
    const long long gplane = (long long)ny * G.gxb * (GainWords<T>::NW * 32);
    // halo node of this thread, if any: -y row (x0 + tx, y0 - 1) or -x column (x0 - 1, y0 + tx)
    const bool hrow = hwrow && y0 > 0 && i < nx;
    const bool hcolm = hwcol && tx < OY && x0 > 0 && y0 + tx < ny;
    const int hid = hwrow ? tx : OX + tx;
    const int hi = hrow ? i : x0 - 1, hj = hrow ? y0 - 1 : y0 + tx;

    // slab axis whose CPML memory is fetched ahead for a node: z for the planes
    // of a z slab, else x or y for the columns of an x or y slab
    const int col_axis = col.sx >= 0 ? 0 : (col.sy >= 0 ? 1 : -1);
    const int zs_lo = G.Sd[2] ? G.L[4] : 0, zs_hi = G.Sd[2] ? G.nz - G.L[5] : G.nz;
    auto plane_slab = [&](int plane) { return (plane < zs_lo || plane >= zs_hi) ? slab_index(plane, G.nz, G.L[4], G.L[5]) : -1; };
    auto psi_index = [&](const Column& c, int a, int plane, int sz) {
      if (a == 2) return sz * ny * nx + c.pz0;
      if (a == 0) return plane * ny * G.Sd[0] + c.px0;
      return plane * G.Sd[1] * nx + c.py0;
    };
    // slab axes the item's columns (x0-1 .. x0+31), rows (y0-1 .. y0+OY-1) or
    // planes (kstart .. z1-1) reach; an item that reaches none copies no CPML
    // memory or coefficients at all (no copy groups, so its waits are free)
    const bool tsx = G.Sd[0] && (x0 - 1 < G.L[0] || x0 + OX - 1 >= nx - G.L[1]);
    const bool tsy = G.Sd[1] && (y0 - 1 < G.L[2] || y0 + OY - 1 >= ny - G.L[3]);
    const bool tsz = G.Sd[2] && (kstart < G.L[4] || z1 - 1 >= G.nz - G.L[5]);
    const bool psi_item = tsx || tsy || tsz;
    // fetch this thread's CPML memory of `plane` into the stage slots (one commit group per plane)
    auto issue_psi = [&](int plane, int stage) {
      if (!psi_item) return;
      T* slots = reinterpret_cast<T*>(stages + (size_t)stage * L::stage_bytes + L::field_bytes + L::mat_bytes);
      const int sz = plane_slab(plane);
      if (plane < z1 && (sz >= 0 || col_axis >= 0 || hrow || hcolm)) {
        if (own) {
          const int a = sz >= 0 ? 2 : col_axis;
          if (a >= 0) {
            const int pi = psi_index(col, a, plane, sz);
            cp_async_elem(slots + tid, G.psiH[sel][a][0] + pi);
            cp_async_elem(slots + L::NT + tid, G.psiH[sel][a][1] + pi);
            if (plane >= z0) {  // E-side memory of the planes this tile updates
              cp_async_elem(slots + 2 * L::NT + tid, G.psiE[a][0] + pi);
              cp_async_elem(slots + 3 * L::NT + tid, G.psiE[a][1] + pi);
            }
          }
        }
        if (hrow || hcolm) {
          Column hc;
          make_column(G, hi, hj, hc, false);
          const int a = sz >= 0 ? 2 : (hc.sx >= 0 ? 0 : (hc.sy >= 0 ? 1 : -1));
          if (a >= 0) {
            const int pi = psi_index(hc, a, plane, sz);
            cp_async_elem(slots + 4 * L::NT + hid, G.psiH[sel][a][0] + pi);
            cp_async_elem(slots + 4 * L::NT + L::NH + hid, G.psiH[sel][a][1] + pi);
          }
        }
      }
      cp_async_commit();
    };
    // grading coefficients of the columns, rows and planes this item touches
    // (joined to the first plane's copy group; visible after the barrier below)
    {
      // only the axes whose slabs the item reaches: no other entry is read
      const int e0 = tsx ? 0 : (tsy ? L::CXN : L::CXN + L::CYN);
      const int e1 = tsz ? L::CXN + L::CYN + 6 * (NP - 1) : (tsy ? L::CXN + L::CYN : (tsx ? L::CXN : 0));
      for (int e = e0 + tid; e < e1; e += NTALL) {
        int a, pos;
        T* dst;
        if (e < L::CXN) {
          a = 0; pos = x0 - 1 + e / 6; dst = cfx + e;
        } else if (e < L::CXN + L::CYN) {
          a = 1; pos = y0 - 1 + (e - L::CXN) / 6; dst = cfy + (e - L::CXN);
        } else {
          a = 2; pos = kstart + (e - L::CXN - L::CYN) / 6; dst = cfz + (e - L::CXN - L::CYN);
        }
        const int hq = e % 6;  // CXN and CYN are multiples of 6
        const int lim = a == 0 ? nx : (a == 1 ? ny : G.nz);
        const bool t = a == 0 ? tsx : (a == 1 ? tsy : tsz);
        if (t && pos >= 0 && pos < lim) cp_async_elem(dst, G.prof[a][hq / 3][hq % 3] + pos);
      }
    }
    for (int p = 0; p < S; ++p) issue_psi(kstart + p, (int)((q0 + p) % S));
    cp_async_wait<S - 1>();
    __syncthreads();

    T hPx = T(0), hPy = T(0);
    bool ok = true;

    for (int p = 0; p < NP - 1; ++p) {
      const int k = kstart + p;
      const unsigned q = q0 + p;
      T* sHx = reinterpret_cast<T*>(smem + L::h_off + (p & 1) * L::hbuf_bytes);  // H of this plane
      T* sHy = sHx + HPL;
      T* sHz = sHy + HPL;
      if (p == 0) ok = ok && mbar_wait(&full[q % S], (q / S) & 1, G.wait_ns);
      ok = ok && mbar_wait(&full[(q + 1) % S], ((q + 1) / S) & 1, G.wait_ns);
      cp_async_wait<S - 1>();  // this thread's CPML memory of plane p
      const unsigned char* stg = stages + (size_t)(q % S) * L::stage_bytes;
      const T* Fk = reinterpret_cast<const T*>(stg);
      const T* Fn = reinterpret_cast<const T*>(stages + (size_t)((q + 1) % S) * L::stage_bytes);
      const uint8_t* Mk = stg + L::field_bytes;
      const T* slots = reinterpret_cast<const T*>(stg + L::field_bytes + L::mat_bytes);
      const bool active = k >= z0;
      const Plane pl = make_plane(G, k);
      const long long cidx = cbase + (long long)k * pstride;

      // own node: material, gain state (issued before the H work)
      unsigned m = 0;
      bool gcell = false;
      GainState<T> gs{};
      if (ok && own && active) {
        m = Mk[tid];
        gcell = GAIN && G.gain && ((m >> 6) & 1);
        if (GAIN && gcell) load_gain(G, sel, gbase + (long long)k * gplane, gs);
      }
      PsiPre<T> pre;
      pre.axis = own ? (pl.sz >= 0 ? 2 : col_axis) : -1;
      if (pre.axis >= 0) {
        pre.h0 = slots[tid];
        pre.h1 = slots[L::NT + tid];
        pre.e0 = slots[2 * L::NT + tid];
        pre.e1 = slots[3 * L::NT + tid];
      } else {
        pre.h0 = pre.h1 = pre.e0 = pre.e1 = T(0);
      }

      // H^{n+1/2} of plane k at the staged node with offset o
      const T* cz = cfz + 6 * p;
      auto h_at = [&](const Column& c, const CoefShared<T>& cf, int o, bool wr, T& hx, T& hy, T& hz,
                      const PsiPre<T>* pp) {
        const T ex = Fk[o], ey = Fk[PL + o], ez = Fk[2 * PL + o];
        h_node(G, c, pl, sel, wr, cf, Fk[2 * PL + o + BXT] - ez, Fn[PL + o] - ey, Fn[o] - ex, Fk[2 * PL + o + 1] - ez,
               Fk[PL + o + 1] - ey, Fk[o + BXT] - ex, Fk[3 * PL + o], Fk[4 * PL + o], Fk[5 * PL + o], hx, hy, hz,
               pp);
      };

      T hx = T(0), hy = T(0), hz = T(0);
      const CoefShared<T> ocf{cfx + 6 * (tx + 1), cfy + 6 * (ty + 1), cz};
      // E^n of the own node, for the E update
      const T eox = owner ? Fk[oe] : T(0), eoy = owner ? Fk[PL + oe] : T(0), eoz = owner ? Fk[2 * PL + oe] : T(0);
      if (ok && own) h_at(col, ocf, oe, active, hx, hy, hz, &pre);
      if (owner) {
        sHx[oh] = hx;
        sHy[oh] = hy;
        sHz[oh] = hz;
      }
      if (hwrow || (hwcol && tx < OY)) {
        T a = T(0), b = T(0), c = T(0);
        if (ok && (hrow || hcolm)) {
          Column hc;
          make_column(G, hi, hj, hc, false);
          PsiPre<T> hp;
          hp.axis = pl.sz >= 0 ? 2 : (hc.sx >= 0 ? 0 : (hc.sy >= 0 ? 1 : -1));
          hp.h0 = slots[4 * L::NT + hid];
          hp.h1 = slots[4 * L::NT + L::NH + hid];
          hp.e0 = hp.e1 = T(0);
          const CoefShared<T> hcf{hrow ? cfx + 6 * (tx + 1) : cfx, hrow ? cfy : cfy + 6 * (tx + 1), cz};
          h_at(hc, hcf, hrow ? tx + xo : (tx + 1) * BXT + xo - 1, false, a, b, c, &hp);
        }
        const int slot = hwrow ? tx + 1 : (tx + 1) * HW;
        sHx[slot] = a;
        sHy[slot] = b;
        sHz[slot] = c;
      }
      if (__syncthreads_or(!ok)) {
        // a wait ran out: let this thread's copies and the block's loads in
        // flight land (bounded) before the block leaves, then report
        cp_async_wait<0>();
        if (tid == 0) atomicOr(G.err, loads.drain(full, S) ? 2 : 6);
        return;
      }
      // nothing reads the fields of plane p's stage after this barrier: refill it
      if (tid == 0 && p + S < NP) {
        fence_proxy_async_smem();
        issue(q + S, kstart + p + S);
      }

      if (active && own) {
        T enx, eny, enz;
        e_node<T, GAIN>(G, sg, col, pl, sel, n, gbase + (long long)k * gplane, m, gcell, gs, ocf, hz - sHz[oh - HW],
                        hy - hPy, hx - hPx,
                        hz - sHz[oh - 1], hy - sHy[oh - 1], hx - sHx[oh - HW], eox, eoy, eoz, enx, eny, enz, &pre);
        // E^{n+1} and H~^{n+1/2} straight to set (n+1)%3 (a warp row: one contiguous segment)
        T* const* Fo = G.F[fo];
        if (FDTD_STREAM_STORES) {
          // no reader in this launch: the evict-first hint (see fdtd_internal.cuh)
          __stcs(Fo[0] + cidx, enx);
          __stcs(Fo[1] + cidx, eny);
          __stcs(Fo[2] + cidx, enz);
          __stcs(Fo[3] + cidx, hx);
          __stcs(Fo[4] + cidx, hy);
          __stcs(Fo[5] + cidx, hz);
        } else {
          Fo[0][cidx] = enx;
          Fo[1][cidx] = eny;
          Fo[2][cidx] = enz;
          Fo[3][cidx] = hx;
          Fo[4][cidx] = hy;
          Fo[5][cidx] = hz;
        }
      }
      hPx = hx;
      hPy = hy;
      // no second barrier: the next plane writes the other H buffer, and the
      // barrier after its H update orders this plane's E reads before the
      // buffer is written again
      issue_psi(kstart + p + S, (int)(q % S));
    }
    ld = q0 + (unsigned)NP;
  }
  cp_async_wait<0>();
}

template <typename T>
int step_blocks_per_sm(bool tma, bool gain, int bx, int by) {
  int nb = 0;
  cudaError_t e;
  if (tma) {
    const size_t smem = step_tma_smem_bytes<T>(by);
    const void* f = nullptr;
    if (by == 4) f = gain ? (const void*)k_step_tma<T, true, 4> : (const void*)k_step_tma<T, false, 4>;
    else f = gain ? (const void*)k_step_tma<T, true, 8> : (const void*)k_step_tma<T, false, 8>;
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, by == 4 ? TmaThreads<T, 4>::NT : TmaThreads<T, 8>::NT, smem);
  } else {
    const size_t smem = step_smem_bytes<T>(bx, by);
    if (gain) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_step<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<T, true>, bx * by, smem);
    } else {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_step<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<T, false>, bx * by, smem);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

template <typename T, bool GAIN, int OY>
static cudaError_t launch_tma_variant(const StepGrid<T>* grids, const TmaGrid* maps, const int4* items, int nitems,
                                      int offset, int blocks, bool wait_prev, cudaStream_t st) {
  const size_t smem = TmaLayout<T, OY>::total;
  cudaError_t e = cudaFuncSetAttribute(k_step_tma<T, GAIN, OY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_programmatic(k_step_tma<T, GAIN, OY>, dim3(blocks), dim3(kTmaOX, TmaThreads<T, OY>::ROWS), smem, st,
                             grids, maps, items, nitems, offset, wait_prev ? 1 : 0);
}

template <typename T>
cudaError_t launch_step_tma(const StepGrid<T>* grids, const TmaGrid* maps, const int4* items, int nitems, int offset,
                            int oy, bool gain, int grid_blocks, cudaStream_t st, bool wait_prev) {
  if (nitems <= 0) return cudaSuccess;
  const int blocks = (grid_blocks > 0 && grid_blocks < nitems) ? grid_blocks : nitems;
  if (oy == 4)
    return gain ? launch_tma_variant<T, true, 4>(grids, maps, items, nitems, offset, blocks, wait_prev, st)
                : launch_tma_variant<T, false, 4>(grids, maps, items, nitems, offset, blocks, wait_prev, st);
  if (oy == 8)
    return gain ? launch_tma_variant<T, true, 8>(grids, maps, items, nitems, offset, blocks, wait_prev, st)
                : launch_tma_variant<T, false, 8>(grids, maps, items, nitems, offset, blocks, wait_prev, st);
  return cudaErrorInvalidValue;
}

// =====================================================================
// Observers
// =====================================================================
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += red[w];
  }
  return s;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(256) k_observe(const ObsGrid<T>* __restrict__ grids, const int4* __restrict__ items,
                                                 int nitems, int offset) {
  __shared__ double red[32];
  __shared__ bool last;
  // (no-op for a plain launch) the step kernel before this one has finished;
  // the next step launch may start its blocks, which wait for this grid
  grid_dependency_wait();
  allow_dependents();
  const int4 it = items[blockIdx.x];
  const ObsGrid<T>& G = grids[it.x];
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;  // sets n and n+1
  const int px = G.px, ny = G.ny;
  const long long slot = n % G.cap;
  if (it.y < 0) {
    for (int q = threadIdx.x; q < G.nprobe * 3; q += blockDim.x) {
      const int p = q / 3, c = q % 3;
      const T v = G.F[fo][c][pidx3(G.probe[p][0], G.probe[p][1], G.probe[p][2], px, ny)];
      G.probe_ring[(slot * G.nprobe + p) * 3 + c] = v;
      if (!isfinite((double)v)) atomicOr(G.err, 1);
    }
    return;
  }
  const int f = it.y, part = it.z, nparts = it.w;
  const int d = G.flux_axis[f], d1 = (d + 1) % 3, d2 = (d + 2) % 3;
  const int p = G.flux_index[f];
  const int u0 = G.flux_u0[f], v0 = G.flux_v0[f];
  const int nu = G.flux_u1[f] - u0, nv = G.flux_v1[f] - v0;
  const long long total = (long long)nu * nv;
  const long long beg = total * part / nparts, end = total * (part + 1) / nparts;
  const T* E1 = G.F[fs][d1];
  const T* E2 = G.F[fs][d2];
  const T* H1a = G.F[fs][3 + d1];
  const T* H1b = G.F[fo][3 + d1];
  const T* H2a = G.F[fs][3 + d2];
  const T* H2b = G.F[fo][3 + d2];
  // element strides of the plane normal and the two transverse axes
  auto stride = [&](int ax) -> long long { return ax == 0 ? 1LL : (ax == 1 ? (long long)px : (long long)px * ny); };
  const long long sd = stride(d), s1 = stride(d1), s2 = stride(d2);
  const long long base = (long long)p * sd + (long long)u0 * s1 + (long long)v0 * s2;
  // consecutive threads take consecutive x (the fastest memory axis) when x
  // is transverse, else consecutive y (x-normal planes: rows one pitch apart)
  const bool ufast = (d1 == 0) || (d == 0);
  const bool small = total < 0x7fffffffLL;  // face numbers fit 32 bits (every grid that fits in memory)
  double acc = 0.0;
  for (long long q = beg + threadIdx.x; q < end; q += blockDim.x) {
    int du, dv;
    if (small) {
      const unsigned qq = (unsigned)q;
      du = (int)(ufast ? qq % (unsigned)nu : qq / (unsigned)nv);
      dv = (int)(ufast ? qq / (unsigned)nu : qq % (unsigned)nv);
    } else {
      du = (int)(ufast ? q % nu : q / nv);
      dv = (int)(ufast ? q / nu : q % nv);
    }
    // node (p, u, v) of the plane and its +v, +u and -normal neighbours
    const long long a = base + (long long)du * s1 + (long long)dv * s2, av = a + s2, au = a + s1;
    const long long b = a - sd, bv = b + s2, bu = b + s1;
    const T e1 = T(0.5) * (E1[a] + E1[av]);
    const T e2 = T(0.5) * (E2[a] + E2[au]);
    const T h2 = T(0.25) * (T(0.5) * (H2a[b] + H2b[b]) + T(0.5) * (H2a[a] + H2b[a]) +
                            T(0.5) * (H2a[bv] + H2b[bv]) + T(0.5) * (H2a[av] + H2b[av]));
    const T h1 = T(0.25) * (T(0.5) * (H1a[b] + H1b[b]) + T(0.5) * (H1a[a] + H1b[a]) +
                            T(0.5) * (H1a[bu] + H1b[bu]) + T(0.5) * (H1a[au] + H1b[au]));
    acc += (double)(e1 * h2) - (double)(e2 * h1);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    G.partials[f * kMaxFluxParts + part] = s;
    __threadfence();
    const unsigned prev = atomicAdd(&G.counters[f], 1u);
    last = (prev == (unsigned)(nparts - 1));
  }
  __syncthreads();
  if (last) {
    // the last block folds the parts in a fixed order (thread t: parts t,
    // t + 256, ... in sequence, then the fixed block reduction)
    __threadfence();
    const volatile double* pp = G.partials + f * kMaxFluxParts;
    double acc2 = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc2 += pp[q];
    const double tot = block_sum(acc2, red);
    if (threadIdx.x == 0) {
      const double T_n = G.flux_sign[f] * G.dx2_over_eta0 * tot;
      G.flux_ring[slot * G.nflux + f] = T_n;
      if (!isfinite(T_n)) atomicOr(G.err, 1);
      G.counters[f] = 0u;
    }
  }
}

// A plain launch: with the programmatic attribute the observation's blocks
// took SM slots early and a 140^3 gain grid with six flux planes stepped 13 %
// slower (measured); the step launch after it is programmatic instead.
template <typename T>
cudaError_t launch_observe(const ObsGrid<T>* grids, const int4* items, int nitems, int offset, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_observe<T><<<nitems, 256, 0, st>>>(grids, items, nitems, offset);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_advance(StepGrid<T>* sg, ObsGrid<T>* og, int ngrids, int count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrids) return;
  long long s = sg[g].step + count;
  if (s > sg[g].step_end) s = sg[g].step_end;
  if (s < sg[g].step) s = sg[g].step;
  sg[g].step = s;
  og[g].step = s;
}

template <typename T>
cudaError_t launch_advance(StepGrid<T>* sg, ObsGrid<T>* og, int ngrids, int count, cudaStream_t st) {
  k_advance<T><<<(ngrids + 127) / 128, 128, 0, st>>>(sg, og, ngrids, count);
  return cudaGetLastError();
}

// =====================================================================
// Energy
// =====================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_energy(const T* __restrict__ ex, const T* __restrict__ ey,
                                                const T* __restrict__ ez, const T* __restrict__ hx,
                                                const T* __restrict__ hy, const T* __restrict__ hz,
                                                const uint8_t* __restrict__ mat, double e0, double e1, double e2,
                                                long long ncell, double* partials, unsigned int* counter,
                                                double* out, int* err) {
  __shared__ double red[32];
  __shared__ bool last;
  const double epsv[4] = {e0, e1, e2, 0.0};
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride) {
    const unsigned m = mat[c];
    const double vx = (double)ex[c], vy = (double)ey[c], vz = (double)ez[c];
    const double wx = (double)hx[c], wy = (double)hy[c], wz = (double)hz[c];
    acc += epsv[m & 3] * vx * vx + epsv[(m >> 2) & 3] * vy * vy + epsv[(m >> 4) & 3] * vz * vz;
    acc += wx * wx + wy * wy + wz * wz;
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    const volatile double* pp = partials;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += pp[b];
    out[0] = tot;
    if (!isfinite(tot)) atomicOr(err, 1);
    *counter = 0u;
  }
}

template <typename T>
cudaError_t launch_energy(const T* const* F6, const uint8_t* mat, double e0, double e1, double e2, long long ncell,
                          double* partials, unsigned int* counter, double* out, int* err, cudaStream_t st) {
  k_energy<T><<<kEnergyBlocks, 256, 0, st>>>(F6[0], F6[1], F6[2], F6[3], F6[4], F6[5], mat, e0, e1, e2, ncell,
                                             partials, counter, out, err);
  return cudaGetLastError();
}

// =====================================================================
// Rasterizer
// =====================================================================
// The FP64 test of a point against a sphere, (dx*dx + dy*dy) + dz*dz < r*r
// with each operation rounded, decides the material.  Most points lie far
// from every surface, so a binary32 test decides them first: with the
// sphere centre split into floor(c) (exact in binary32) and c - floor(c)
// (rounded to binary32, error <= 2^-25), the binary32 dx, dy, dz are within
// 2^-25 + 2^-24 |d| of i - c, and d2 within 2^-22 (d2 + r^2 + 1) of the
// exact square distance, r^2 rounded within 2^-24 r^2.  Whenever the binary32
// d2 and r^2 differ by more than M = 2^-19 (d2 + r^2 + 1) (eight times that
// bound) the FP64 test gives the same answer; otherwise the FP64 test runs.
// fsph: per sphere (floor cx, floor cy, floor cz, r^2) and (cx, cy, cz) - floor(.), in binary32.
__global__ void k_rasterize(uint8_t* __restrict__ mat, int nx, int ny, int nz, int px, const double* __restrict__ sph,
                            const float4* __restrict__ fsph, const int* __restrict__ bstart,
                            const int* __restrict__ blist, int bin, int bnx, int bny,
                            double lo0, double lo1, double lo2, double hi0, double hi1, double hi2) {
  const long long ncell = (long long)nx * ny * nz;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int i = (int)(c % nx);
  const int j = (int)((c / nx) % ny);
  const int k = (int)(c / ((long long)nx * ny));
  const int b = ((k / bin) * bny + (j / bin)) * bnx + (i / bin);
  const double pxs[4] = {i + 0.5, (double)i, (double)i, i + 0.5};
  const double pys[4] = {(double)j, j + 0.5, (double)j, j + 0.5};
  const double pzs[4] = {(double)k, (double)k, k + 0.5, k + 0.5};
  bool ins[4] = {false, false, false, false};
  const float fi = (float)i, fj = (float)j, fk = (float)k;
  for (int q = bstart[b]; q < bstart[b + 1] && !(ins[0] && ins[1] && ins[2] && ins[3]); ++q) {
    const int s = blist[q];
    const float4 a = fsph[2 * s], f = fsph[2 * s + 1];
    // offsets of the integer and half-integer nodes from the centre
    const float x0 = __fsub_rn(__fsub_rn(fi, a.x), f.x), x1 = __fsub_rn(__fsub_rn(__fadd_rn(fi, 0.5f), a.x), f.x);
    const float y0 = __fsub_rn(__fsub_rn(fj, a.y), f.y), y1 = __fsub_rn(__fsub_rn(__fadd_rn(fj, 0.5f), a.y), f.y);
    const float z0 = __fsub_rn(__fsub_rn(fk, a.z), f.z), z1 = __fsub_rn(__fsub_rn(__fadd_rn(fk, 0.5f), a.z), f.z);
    const float xs[2] = {__fmul_rn(x0, x0), __fmul_rn(x1, x1)}, ys[2] = {__fmul_rn(y0, y0), __fmul_rn(y1, y1)};
    const float zs[2] = {__fmul_rn(z0, z0), __fmul_rn(z1, z1)};
    const int hx[4] = {1, 0, 0, 1}, hy[4] = {0, 1, 0, 1}, hz[4] = {0, 0, 1, 1};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (ins[t]) continue;
      const float d2 = __fadd_rn(__fadd_rn(xs[hx[t]], ys[hy[t]]), zs[hz[t]]);
      const float m = 0x1p-19f * __fadd_rn(__fadd_rn(d2, a.w), 1.0f);
      if (d2 < a.w - m) {
        ins[t] = true;
      } else if (!(d2 > a.w + m)) {
        const double cx = sph[4 * s], cy = sph[4 * s + 1], cz = sph[4 * s + 2], r = sph[4 * s + 3];
        const double dx = __dsub_rn(pxs[t], cx), dy = __dsub_rn(pys[t], cy), dz = __dsub_rn(pzs[t], cz);
        const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        ins[t] = e2 < __dmul_rn(r, r);
      }
    }
  }
  unsigned byte = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const bool inbox = pxs[t] >= lo0 && pxs[t] < hi0 && pys[t] >= lo1 && pys[t] < hi1 && pzs[t] >= lo2 && pzs[t] < hi2;
    if (t < 3) byte |= (inbox ? (ins[t] ? 2u : 1u) : 0u) << (2 * t);
    else if (inbox && ins[t]) byte |= 64u;
  }
  mat[pidx3(i, j, k, px, ny)] = (uint8_t)byte;
}

cudaError_t launch_rasterize(uint8_t* mat, int nx, int ny, int nz, int px, const double* spheres,
                             const float* fspheres, const int* bin_start, const int* bin_list, int bin, int bnx, int bny,
                             int bnz, const double* box, cudaStream_t st) {
  (void)bnz;
  const long long ncell = (long long)nx * ny * nz;
  const int threads = 256;
  const long long blocks = (ncell + threads - 1) / threads;
  k_rasterize<<<(unsigned)blocks, threads, 0, st>>>(mat, nx, ny, nz, px, spheres,
                                                     reinterpret_cast<const float4*>(fspheres), bin_start, bin_list,
                                                     bin, bnx, bny, box[0], box[1], box[2], box[3], box[4], box[5]);
  return cudaGetLastError();
}

// =====================================================================
// Gain initialization and conversions
// =====================================================================
// One thread per node slot of the gain state (rows padded to 32-node
// blocks): both P~ slots and the compensation words zero, dN~ = (d1, d2, d3)
// in gain cells and 0 elsewhere (padding slots included).
template <typename T>
__global__ void k_gain_init(StepGrid<T> G, long long nslots, T d1, T d2, T d3) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const long long rb = t >> 5;  // 32-node block of a row
  const int lane = (int)(t & 31);
  const int i = (int)(rb % G.gxb) * 32 + lane;
  const long long row = rb / G.gxb;
  const int j = (int)(row % G.ny), k = (int)(row / G.ny);
  const bool g = i < G.nx && ((G.mat[((long long)k * G.ny + j) * G.px + i] >> 6) & 1);
  using W = GainWords<T>;
  T* w = G.gst + rb * (W::NW * 32) + lane;
  for (int q = 0; q < W::NW; ++q) w[32 * q] = T(0);
  if (g) {
    w[32 * W::DN] = d1;
    w[32 * W::DN + 32] = d2;
    w[32 * W::DN + 64] = d3;
  }
}

template <typename T>
cudaError_t launch_gain_init(const StepGrid<T>* g, long long nslots, T d1, T d2, T d3, cudaStream_t st) {
  k_gain_init<T><<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(*g, nslots, d1, d2, d3);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ s, double* __restrict__ d, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) d[c] = (double)s[c];
}
template <typename T>
__global__ void k_from_double(const double* __restrict__ s, T* __restrict__ d, long long n) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) d[c] = (T)s[c];
}
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_to_double<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_from_double(const double* src, T* dst, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_from_double<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// =====================================================================
// Instantiations
// =====================================================================
#define FDTD_INST(T)                                                                                           \
  template size_t step_smem_bytes<T>(int, int);                                                                \
  template size_t step_tma_smem_bytes<T>(int);                                                                 \
  template int step_blocks_per_sm<T>(bool, bool, int, int);                                                    \
  template cudaError_t launch_step<T>(const StepGrid<T>*, const int4*, int, int, int, int, bool, int,         \
                                      cudaStream_t);                                                           \
  template cudaError_t launch_step_tma<T>(const StepGrid<T>*, const TmaGrid*, const int4*, int, int, int, bool, \
                                          int, cudaStream_t, bool);                                            \
  template cudaError_t launch_observe<T>(const ObsGrid<T>*, const int4*, int, int, cudaStream_t);             \
  template cudaError_t launch_advance<T>(StepGrid<T>*, ObsGrid<T>*, int, int, cudaStream_t);                  \
  template cudaError_t launch_gain_init<T>(const StepGrid<T>*, long long, T, T, T, cudaStream_t);             \
  template cudaError_t launch_energy<T>(const T* const*, const uint8_t*, double, double, double, long long,   \
                                        double*, unsigned int*, double*, int*, cudaStream_t);                 \
  template cudaError_t launch_to_double<T>(const T*, double*, long long, cudaStream_t);                       \
  template cudaError_t launch_from_double<T>(const double*, T*, long long, cudaStream_t);

FDTD_INST(float)
FDTD_INST(double)

}  // namespace fdtd
