// Paired binary32 step kernel: one time step n -> n+1 of a list of work items
// (32-column x OY-row tile x z-range of some binary32 grid, no periodic axis),
// each thread updating two x-adjacent nodes with packed f32x2 arithmetic.
//
// Same staging as the single-node TMA kernel: every plane of the six fields
// (tile plus a one-node halo, x padded by one 16-byte unit each side) and the
// tile's material bytes arrive in shared memory by two TMA bulk-tensor copies
// into a 3-stage mbarrier pipeline; CPML memory of the planes ahead is fetched
// per thread with cp.async.  What differs:
//   - 16 x OY owner threads, each owning the node pair (x0 + 2 tx, x0 + 2 tx + 1):
//     the pair's values travel as 64-bit shared-memory words and every
//     difference, curl and update of the interior cell is one f32x2 add, sub,
//     mul or fma (sm_100 family), half the instructions of the scalar form;
//   - a ninth warp recomputes H on the -y halo row (16 pairs) and the -x halo
//     column (OY pairs, the x0-1 node kept) while the owners compute their
//     own H, and issues the TMA copies, so no owner warp carries halo work;
//   - the material classes of both nodes index a 64-entry table of
//     (S/eps_x, S/eps_y, S/eps_z) built once per grid record;
//   - the new E and H of a pair leave by 8-byte stores straight from
//     registers (a half-warp writes one 128-byte row segment), and H of a
//     plane goes to one of two shared buffers, so one block barrier per plane
//     suffices (measured: as fast as a TMA store of an output tile, without
//     its 12 KB of shared memory and its second barrier);
//   - a persistent block (the default for single grids) issues the first two
//     planes of its next item into the stages that its current item's last
//     planes free, so an item starts with its planes already in flight;
//   - on gain grids the polarization and populations of both nodes are
//     updated with f32x2 operations on 8-byte words of the gain state.
// Every operation is the one the scalar kernels perform on that node, in the
// same order and rounding (f32x2 lanes round like the scalar instruction), so
// the results equal theirs bit for bit.
//
// Paper: Yee FDTD (Sec. "Sample and numerical approach"), four-level
// Maxwell-Bloch gain solved at the Yee cell (same section), spontaneous-
// emission noise as a random kick (same section).
#include <math.h>

#include "cell.cuh"
#include "fdtd_internal.cuh"
#include "tma.cuh"

namespace fdtd {

// ---------------------------------------------------------------- f32x2
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
#ifndef FDTD_PAIR_X2_INTRINSICS
#define FDTD_PAIR_X2_INTRINSICS 0
#endif
#if FDTD_PAIR_X2_INTRINSICS
// the toolkit's packed float2 intrinsics (the compiler keeps the pairs in
// register pairs); a - b is a + (-b), exactly, lane by lane
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#else
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(r);
}
#endif
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
// new field values: no reader in this launch (FDTD_STREAM_STORES: the evict-first hint)
__device__ __forceinline__ void st2_out(float* p, float2 v) {
  if (FDTD_STREAM_STORES)
    __stcs(reinterpret_cast<float2*>(p), v);
  else
    st2(p, v);
}
__device__ __forceinline__ void st1_out(float* p, float v) {
  if (FDTD_STREAM_STORES)
    __stcs(p, v);
  else
    *p = v;
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// CPML memory of the planes ahead staged per thread by cp.async (1), or read
// from global memory where the update needs it (0: smaller stages).
#ifndef FDTD_PAIR_PSI_STAGED
#define FDTD_PAIR_PSI_STAGED 1
#endif

// Shared-memory layout of the paired kernel (host and device agree).
template <int OY>
struct PairLayout {
  static constexpr int OX = kTmaOX;             // owned tile width (32)
  static constexpr int PXT = OX / 2;            // pair threads per row
  static constexpr int NTO = PXT * OY;          // owner threads
  static constexpr int NT = NTO + 32;           // + the halo / copy warp
  static constexpr int AX = 4;                  // x pad: one 16-byte unit each side
  static constexpr int BXT = OX + 2 * AX;       // staged box width
  static constexpr int PL = BXT * (OY + 2);     // one component plane of a stage (rows y0-1 .. y0+OY)
  static constexpr int HW = OX + 2;             // H row: column 0 = x0-2, 1 = x0-1, 2 + l = x0 + l
  static constexpr int HPL = (OY + 1) * HW;     // row 0 = y0-1
  static constexpr int OPL = OX * OY;           // one component of the output tile
  static constexpr int NC = OPL;                // owned nodes
  static constexpr int NHC = 64;                // halo nodes (32 lanes x 2)
  static constexpr size_t sg_off = align128(sizeof(StepGrid<float>));
  static constexpr size_t bar_off = sg_off + align128(kMaxSrc * sizeof(double));
  static constexpr size_t ctab_off = bar_off + 128;
  static constexpr size_t stage_off = ctab_off + 64 * sizeof(float4);
  static constexpr size_t field_bytes = align128((size_t)6 * PL * sizeof(float));
  static constexpr size_t mat_bytes = align128((size_t)OPL);
  // CPML memory fetched ahead: 4 slots per owned node, 2 per halo node
  static constexpr size_t psi_bytes = FDTD_PAIR_PSI_STAGED ? align128((size_t)(4 * NC + 2 * NHC) * sizeof(float)) : 0;
  static constexpr size_t stage_bytes = field_bytes + mat_bytes + psi_bytes;
  // H of the plane (row 0 = y0-1, column 1 = x0-1), two buffers: plane p uses p & 1
  static constexpr size_t hbuf_bytes = align128((size_t)3 * HPL * sizeof(float));
  static constexpr size_t h_off = stage_off + (size_t)kTmaStages * stage_bytes;
  // CPML grading coefficients: x as [h*3+q][HW column], y as [row][h*3+q], z as [plane][h*3+q]
  static constexpr int CXN = 6 * HW, CYN = 6 * (OY + 1), CZN = 6 * kTmaZMax;
  static constexpr size_t coef_off = h_off + 2 * hbuf_bytes;
  // the block's first kItemCache work items (a persistent block takes every gridDim-th item)
  static constexpr int kItemCache = 32;
  static constexpr size_t items_off = align128(coef_off + (size_t)(CXN + CYN + CZN) * sizeof(float));
  static constexpr size_t total = items_off + kItemCache * sizeof(int4) + 128;
};

size_t step_pair_smem_bytes(int oy) { return oy == 8 ? PairLayout<8>::total : PairLayout<16>::total; }

// The facts of a node pair (i0, i0 + 1) in row j that stay fixed during a z-march.
struct PairCol {
  int i0, j;
  int sx0, sx1, sy;   // slab coordinates (-1 outside); sx1 = -1 also when node 1 is off the grid
  int px0, px1;       // x-slab psi offsets of the two nodes in plane 0
  int py0, pz0;       // y-slab psi offset in plane 0, z-slab offset within a plane (node 0; node 1 is +1)
  bool own1;          // node 1 is on the grid
};

__device__ __forceinline__ void make_pair_col(const StepGrid<float>& G, int i0, int j, PairCol& c) {
  c.i0 = i0;
  c.j = j;
  c.own1 = i0 + 1 < G.nx;
  c.sx0 = G.Sd[0] ? slab_index(i0, G.nx, G.L[0], G.L[1]) : -1;
  c.sx1 = (G.Sd[0] && c.own1) ? slab_index(i0 + 1, G.nx, G.L[0], G.L[1]) : -1;
  c.sy = G.Sd[1] ? slab_index(j, G.ny, G.L[2], G.L[3]) : -1;
  c.px0 = j * G.Sd[0] + c.sx0;
  c.px1 = j * G.Sd[0] + c.sx1;
  c.py0 = c.sy * G.nx + i0;
  c.pz0 = j * G.nx + i0;
}

// CPML on the pair's differences along x (per node), y and z (both nodes
// share the row and the plane).  h = 1: H-curl node (memory of set `sel`
// read, set sel^1 written when `wr`); h = 0: E-curl node (memory updated in
// place when `wr`).  d[a][s]: the difference that psi slot s of axis a
// modifies.  pa: axis whose old memory is in `pre` (-1: none); pre[s] holds
// slot s of the pair (node 0 in .x, node 1 in .y).
// Old CPML memory of both nodes at psi index pi (node 1 at pi + 1, read only
// when `own1`); one 64-bit load when pi is even (both arrays are 8-byte
// aligned and both nodes present).
__device__ __forceinline__ float2 psi_pair(const float* a, int pi, bool own1) {
  if (own1 && !(pi & 1)) return ld2(a + pi);
  return make_float2(a[pi], own1 ? a[pi + 1] : 0.0f);
}
__device__ __forceinline__ void psi_store(float* a, int pi, bool own1, float2 v) {
  if (own1 && !(pi & 1)) {
    st2(a + pi, v);
  } else {
    a[pi] = v.x;
    if (own1) a[pi + 1] = v.y;
  }
}

template <int H>
__device__ __forceinline__ void pair_cpml(const StepGrid<float>& G, const PairCol& c, const Plane& pl, int sel,
                                          bool wr, const float* cfx, int xcol, const float* cfy, const float* cfz,
                                          int pa, const float2* pre, float2& dxA, float2& dxB, float2& dyA,
                                          float2& dyB, float2& dzA, float2& dzB) {
  // psi arrays: H side reads set sel, writes set sel^1; E side in place
  auto rd = [&](int a, int s) -> const float* { return H ? G.psiH[sel][a][s] : G.psiE[a][s]; };
  auto wt = [&](int a, int s) -> float* { return wr ? (H ? G.psiH[sel ^ 1][a][s] : G.psiE[a][s]) : (float*)nullptr; };
  constexpr int HW = PairLayout<8>::HW;
  if (c.sx0 >= 0 && c.sx1 >= 0) {
    // both nodes in the slab: consecutive memory and coefficient entries
    const int pi = pl.px_plane + c.px0;
    const float2 ik = ld2(cfx + (3 * H + 0) * HW + xcol), b = ld2(cfx + (3 * H + 1) * HW + xcol),
                 cc = ld2(cfx + (3 * H + 2) * HW + xcol);
    const float2 s0 = pa == 0 ? pre[0] : psi_pair(rd(0, 0), pi, true);
    const float2 s1 = pa == 0 ? pre[1] : psi_pair(rd(0, 1), pi, true);
    const float2 p0 = fma2(b, s0, mul2(cc, dxA));
    const float2 p1 = fma2(b, s1, mul2(cc, dxB));
    if (wr) {
      psi_store(wt(0, 0), pi, true, p0);
      psi_store(wt(0, 1), pi, true, p1);
    }
    dxA = fma2(ik, dxA, p0);
    dxB = fma2(ik, dxB, p1);
  } else if (c.sx0 >= 0 || c.sx1 >= 0) {
    // one node in the slab (slab edge at an odd index, or the halo column)
    float* o0 = wt(0, 0);
    float* o1 = wt(0, 1);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int sx = e ? c.sx1 : c.sx0;
      if (sx < 0) continue;
      const int pi = pl.px_plane + (e ? c.px1 : c.px0);
      const float ik = cfx[(3 * H + 0) * HW + xcol + e];
      const float b = cfx[(3 * H + 1) * HW + xcol + e];
      const float cc = cfx[(3 * H + 2) * HW + xcol + e];
      const float s0 = pa == 0 ? (e ? pre[0].y : pre[0].x) : rd(0, 0)[pi];
      const float s1 = pa == 0 ? (e ? pre[1].y : pre[1].x) : rd(0, 1)[pi];
      float& A = e ? dxA.y : dxA.x;
      float& B = e ? dxB.y : dxB.x;
      A = pml_term_c(A, ik, b, cc, s0, o0, pi);
      B = pml_term_c(B, ik, b, cc, s1, o1, pi);
    }
  }
  // y and z: the two nodes share the coefficients
  auto both = [&](int a, int pi, const float* cf, float2& A, float2& B) {
    const float2 ik = bc2(cf[3 * H + 0]), b = bc2(cf[3 * H + 1]), cc = bc2(cf[3 * H + 2]);
    const float2 s0 = pa == a ? pre[0] : psi_pair(rd(a, 0), pi, c.own1);
    const float2 s1 = pa == a ? pre[1] : psi_pair(rd(a, 1), pi, c.own1);
    const float2 p0 = fma2(b, s0, mul2(cc, A));
    const float2 p1 = fma2(b, s1, mul2(cc, B));
    if (wr) {
      psi_store(wt(a, 0), pi, c.own1, p0);
      psi_store(wt(a, 1), pi, c.own1, p1);
    }
    A = fma2(ik, A, p0);
    B = fma2(ik, B, p1);
  };
  if (c.sy >= 0) both(1, pl.py_plane + c.py0, cfy, dyA, dyB);
  if (pl.sz >= 0) both(2, pl.pz_plane + c.pz0, cfz, dzA, dzB);
}

// H~^{n+1/2} of the pair whose node 0 sits at staged offset o (even); CPML:
// the pair's node or plane may lie in an absorbing slab.
template <bool CPML>
__device__ __forceinline__ void pair_h(const StepGrid<float>& G, const PairCol& c, const Plane& pl, int sel, bool wr,
                                       const float* Fk, const float* Fn, int o, int PL, int BXT, const float* cfx,
                                       int xcol, const float* cfy, const float* cfz, int pa, const float2* pre,
                                       float2 ncH, float2& ex, float2& ey, float2& ez, float2& hx, float2& hy,
                                       float2& hz) {
  ex = ld2(Fk + o);
  ey = ld2(Fk + PL + o);
  ez = ld2(Fk + 2 * PL + o);
  float2 dyEz = sub2(ld2(Fk + 2 * PL + o + BXT), ez);
  float2 dzEy = sub2(ld2(Fn + PL + o), ey);
  float2 dzEx = sub2(ld2(Fn + o), ex);
  float2 dxEz = sub2(make_float2(ez.y, Fk[2 * PL + o + 2]), ez);
  float2 dxEy = sub2(make_float2(ey.y, Fk[PL + o + 2]), ey);
  float2 dyEx = sub2(ld2(Fk + o + BXT), ex);
  if (CPML && (c.sx0 >= 0 || c.sx1 >= 0 || c.sy >= 0 || pl.sz >= 0))
    pair_cpml<1>(G, c, pl, sel, wr, cfx, xcol, cfy, cfz, pa, pre, dxEz, dxEy, dyEx, dyEz, dzEy, dzEx);
  hx = fma2(ncH, sub2(dyEz, dzEy), ld2(Fk + 3 * PL + o));
  hy = fma2(ncH, sub2(dzEx, dxEz), ld2(Fk + 4 * PL + o));
  hz = fma2(ncH, sub2(dxEy, dyEx), ld2(Fk + 5 * PL + o));
}

// Gain state of a node pair (node 0 in .x, node 1 in .y), loaded at the
// start of the plane so the loads' latency hides behind the H work.
struct PairGain {
  float2 pnx, pny, pnz, pmx, pmy, pmz, d1, d2, d3, k1, k2, k3;
};

// Load the gain state of the pair whose node 0 sits at gain index g0 (even:
// 8-byte words); slot `sel` holds P~^n.
__device__ __forceinline__ void load_pair_gain(const StepGrid<float>& G, int sel, long long g0, PairGain& s) {
  using W = GainWords<float>;
  const float* gw = G.gst + g0;
  const float* pnw = gw + 32 * (sel ? W::P1 : W::P0);
  const float* pmw = gw + 32 * (sel ? W::P0 : W::P1);
  s.pnx = ld2(pnw);
  s.pny = ld2(pnw + 32);
  s.pnz = ld2(pnw + 64);
  s.pmx = ld2(pmw);
  s.pmy = ld2(pmw + 32);
  s.pmz = ld2(pmw + 64);
  s.d1 = ld2(gw + 32 * W::DN);
  s.d2 = ld2(gw + 32 * W::DN + 32);
  s.d3 = ld2(gw + 32 * W::DN + 64);
  s.k1 = ld2(gw + 32 * W::CMP);
  s.k2 = ld2(gw + 32 * W::CMP + 32);
  s.k3 = ld2(gw + 32 * W::CMP + 64);
}

// Sources, gain and PEC of the node pair (the general part of the E update):
// (enx, eny, enz) hold fmad(cE, curl, E^n) of both nodes on entry.  The gain
// state of both nodes is read and written as 8-byte words (node 0 at gain
// index g0, even; node 1 at g0 + 1 in the same 32-node record), and the
// polarization and population updates of both nodes run as f32x2 operations
// in the scalar kernels' order; a node that is not a gain cell (or is off the
// grid) keeps its state and gets no polarization current.
// PRE: the pair's gain state was loaded ahead into `gs`; otherwise it is
// loaded here, the polarization words first and the population words after
// the field update (fewer registers live at once).
template <bool GAIN, bool PRE>
__device__ __forceinline__ void pair_extras(const StepGrid<float>& G, const double* sg, const PairCol& c,
                                            const Plane& pl, int sel, long long n, long long g0, unsigned m0,
                                            unsigned m1, unsigned s0, unsigned s1, float2 ex, float2 ey, float2 ez,
                                            const PairGain& gs, float2& enx, float2& eny, float2& enz) {
  using W = GainWords<float>;
  const bool ga = GAIN && G.gain && ((m0 >> 6) & 1);
  const bool gb = GAIN && G.gain && c.own1 && ((m1 >> 6) & 1);
  float2 srx = make_float2(0.0f, 0.0f), sry = srx, srz = srx;
  if (s0 | s1) {
    Column col;
    col.j = c.j;
    if (s0) {
      col.i = c.i0;
      col.src = s0;
      source_drive(G, sg, col, pl, srx.x, sry.x, srz.x);
    }
    if (s1) {
      col.i = c.i0 + 1;
      col.src = s1;
      source_drive(G, sg, col, pl, srx.y, sry.y, srz.y);
    }
  }
  float2 dPx = make_float2(0.0f, 0.0f), dPy = dPx, dPz = dPx;
  float2 d1, d2;
  float* gw = G.gst + g0;
  if (GAIN && (ga || gb)) {
    float* pmw = gw + 32 * (sel ? W::P0 : W::P1);  // P~^{n-1}, receives P~^{n+1}
    const float* pnw = gw + 32 * (sel ? W::P1 : W::P0);
    const float2 pnx = PRE ? gs.pnx : ld2(pnw), pny = PRE ? gs.pny : ld2(pnw + 32), pnz = PRE ? gs.pnz : ld2(pnw + 64);
    const float2 pmx = PRE ? gs.pmx : ld2(pmw), pmy = PRE ? gs.pmy : ld2(pmw + 32), pmz = PRE ? gs.pmz : ld2(pmw + 64);
    d1 = PRE ? gs.d1 : ld2(gw + 32 * W::DN);
    d2 = PRE ? gs.d2 : ld2(gw + 32 * W::DN + 32);
    const float2 drive = mul2(bc2(G.a3), add2(bc2(G.n12eq), sub2(d1, d2)));
    const float2 a1 = bc2(G.a1), na2 = bc2(-G.a2);
    float2 Px = fma2(drive, ex, fma2(a1, pnx, mul2(na2, pmx)));
    float2 Py = fma2(drive, ey, fma2(a1, pny, mul2(na2, pmy)));
    float2 Pz = fma2(drive, ez, fma2(a1, pnz, mul2(na2, pmz)));
    if (G.noise != 0.0f) {
      float xa, xb, xc;
      const long long lcell = ((long long)pl.k * G.ny + c.j) * G.nx + c.i0;
      if (ga) {
        gain_normals(G.seed, lcell, n, xa, xb, xc);
        Px.x = fmad(G.noise, xa, Px.x);
        Py.x = fmad(G.noise, xb, Py.x);
        Pz.x = fmad(G.noise, xc, Pz.x);
      }
      if (gb) {
        gain_normals(G.seed, lcell + 1, n, xa, xb, xc);
        Px.y = fmad(G.noise, xa, Px.y);
        Py.y = fmad(G.noise, xb, Py.y);
        Pz.y = fmad(G.noise, xc, Pz.y);
      }
    }
    dPx = sub2(Px, pnx);
    dPy = sub2(Py, pny);
    dPz = sub2(Pz, pnz);
    if (ga && gb) {
      st2(pmw, Px);
      st2(pmw + 32, Py);
      st2(pmw + 64, Pz);
    } else if (ga) {
      pmw[0] = Px.x;
      pmw[32] = Py.x;
      pmw[64] = Pz.x;
      dPx.y = dPy.y = dPz.y = 0.0f;
    } else {
      pmw[1] = Px.y;
      pmw[33] = Py.y;
      pmw[65] = Pz.y;
      dPx.x = dPy.x = dPz.x = 0.0f;
    }
  }
  if (s0 | s1 | ga | gb) {
    // -1/eps of each node's component classes; a lane with neither a source
    // nor gain adds fma(-1/eps, +0, e) = e
    const float2 cx = make_float2(-G.cP[m0 & 3], -G.cP[m1 & 3]);
    const float2 cy = make_float2(-G.cP[(m0 >> 2) & 3], -G.cP[(m1 >> 2) & 3]);
    const float2 cz = make_float2(-G.cP[(m0 >> 4) & 3], -G.cP[(m1 >> 4) & 3]);
    enx = fma2(cx, add2(dPx, srx), enx);
    eny = fma2(cy, add2(dPy, sry), eny);
    enz = fma2(cz, add2(dPz, srz), enz);
  }
  if (c.j == 0 || pl.pecz) enx = make_float2(0.0f, 0.0f);
  if (c.i0 == 0) eny.x = 0.0f;
  if (pl.pecz) eny = make_float2(0.0f, 0.0f);
  if (c.i0 == 0) enz.x = 0.0f;
  if (c.j == 0) enz = make_float2(0.0f, 0.0f);
  if (GAIN && (ga || gb)) {
    const float2 d3 = PRE ? gs.d3 : ld2(gw + 32 * W::DN + 64);
    const float2 k1 = PRE ? gs.k1 : ld2(gw + 32 * W::CMP), k2 = PRE ? gs.k2 : ld2(gw + 32 * W::CMP + 32),
                 k3 = PRE ? gs.k3 : ld2(gw + 32 * W::CMP + 64);
    const float2 half = bc2(0.5f);
    const float2 hx_ = mul2(half, add2(enx, ex)), hy_ = mul2(half, add2(eny, ey)), hz_ = mul2(half, add2(enz, ez));
    const float2 r = mul2(bc2(G.q), fma2(hz_, dPz, fma2(hy_, dPy, mul2(hx_, dPx))));
    const float2 inc1 = fma2(bc2(G.w[0]), r, fma2(bc2(G.D[0][2]), d3, fma2(bc2(G.D[0][1]), d2, mul2(bc2(G.D[0][0]), d1))));
    const float2 inc2 = fma2(bc2(G.w[1]), r, fma2(bc2(G.D[1][2]), d3, fma2(bc2(G.D[1][1]), d2, mul2(bc2(G.D[1][0]), d1))));
    const float2 inc3 = fma2(bc2(G.w[2]), r, fma2(bc2(G.D[2][2]), d3, fma2(bc2(G.D[2][1]), d2, mul2(bc2(G.D[2][0]), d1))));
    // compensated (Kahan) accumulation of the population deviations
    const float2 y1 = sub2(inc1, k1), y2 = sub2(inc2, k2), y3 = sub2(inc3, k3);
    const float2 t1 = add2(d1, y1), t2 = add2(d2, y2), t3 = add2(d3, y3);
    const float2 n1 = sub2(sub2(t1, d1), y1), n2 = sub2(sub2(t2, d2), y2), n3 = sub2(sub2(t3, d3), y3);
    float* dw = gw + 32 * W::DN;
    float* kw = gw + 32 * W::CMP;
    if (ga && gb) {
      st2(kw, n1);
      st2(kw + 32, n2);
      st2(kw + 64, n3);
      st2(dw, t1);
      st2(dw + 32, t2);
      st2(dw + 64, t3);
    } else {
      const int e = ga ? 0 : 1;
      kw[e] = ga ? n1.x : n1.y;
      kw[e + 32] = ga ? n2.x : n2.y;
      kw[e + 64] = ga ? n3.x : n3.y;
      dw[e] = ga ? t1.x : t1.y;
      dw[e + 32] = ga ? t2.x : t2.y;
      dw[e + 64] = ga ? t3.x : t3.y;
    }
  }
}

// Sources of the grid that can touch node (i, j) (bit s: source s).
__device__ __forceinline__ unsigned node_sources(const StepGrid<float>& G, int i, int j) {
  unsigned m = 0;
  for (int s = 0; s < G.nsrc; ++s) {
    const SrcDev& S = G.src[s];
    bool hit;
    if (S.kind == 0) hit = (i == S.i && j == S.j);
    else if (S.axis == 2) hit = (i >= S.lo1 && i < S.hi1 && j >= S.lo2 && j < S.hi2);
    else if (S.axis == 0) hit = (i == S.index && j >= S.lo1 && j < S.hi1);
    else hit = (j == S.index && i >= S.lo2 && i < S.hi2);
    if (hit) m |= 1u << s;
  }
  return m;
}

// The next work item's planes that the producer fetches while the current
// item finishes (kept in shared memory: only the producer reads or writes it).
struct PairNext {
  const CUtensorMap* fmap;
  const CUtensorMap* mmap;
  int x0, y0, kstart, fs;  // fs: field set the next item reads
  int cnt;  // planes of the next item to issue from the current item's last refills (0..S-1)
};

static_assert(sizeof(PairNext) <= 64, "PairNext lives in the 128-byte barrier area after the stage barriers");

#ifndef FDTD_PAIR_MIN_BLOCKS
#define FDTD_PAIR_MIN_BLOCKS 2
#endif
#ifndef FDTD_PAIR_GAIN8_MIN_BLOCKS
#define FDTD_PAIR_GAIN8_MIN_BLOCKS 3
#endif

// Owner threads of a tile of OY rows when each owns RY rows of node pairs.
template <int OY, int RY>
struct PairThreads {
  static constexpr int NTO = 16 * OY / RY;  // owner threads
  static constexpr int NT = NTO + 32;       // + the halo / copy warp
};

#ifndef FDTD_PAIR_RY
#define FDTD_PAIR_RY 1  // rows of node pairs per owner thread in 32 x 16 tiles (2 measured slower: fewer warps)
#endif

// Resident blocks the register budget is sized for: 2 of 288 threads (32 x
// 16 tiles), 4 of 160 (32 x 8); gain grids on 32 x 8 tiles 3, whose gain
// state (12 words a pair) stays in registers from the start of the plane.
template <bool GAIN, int OY>
constexpr int pair_min_blocks() { return (GAIN && OY == 8) ? FDTD_PAIR_GAIN8_MIN_BLOCKS : FDTD_PAIR_MIN_BLOCKS * 16 / OY; }

template <bool GAIN, int OY, int RY>
__global__ void __launch_bounds__(PairThreads<OY, RY>::NT, pair_min_blocks<GAIN, OY>())
    k_step_pair(const StepGrid<float>* __restrict__ grids, const TmaGrid* __restrict__ maps,
                const int4* __restrict__ items, int nitems, int offset) {
  using L = PairLayout<OY>;
  constexpr int S = kTmaStages;
  constexpr int AX = L::AX, BXT = L::BXT, PL = L::PL, HW = L::HW, NC = L::NC;
  constexpr int NTO = PairThreads<OY, RY>::NTO, NT = PairThreads<OY, RY>::NT;
  constexpr unsigned TX_BYTES = (unsigned)(6 * PL * sizeof(float) + L::OX * OY);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  StepGrid<float>& G = *reinterpret_cast<StepGrid<float>*>(smem);
  double* sg = reinterpret_cast<double*>(smem + L::sg_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::bar_off);
  PairNext& nxt = *reinterpret_cast<PairNext*>(smem + L::bar_off + 64);
  float4* ctab = reinterpret_cast<float4*>(smem + L::ctab_off);
  unsigned char* stages = smem + L::stage_off;
  float* cfx = reinterpret_cast<float*>(smem + L::coef_off);
  float* cfy = cfx + L::CXN;
  float* cfz = cfy + L::CYN;
  int4* sitems = reinterpret_cast<int4*>(smem + L::items_off);
  const int tid = threadIdx.x;
  const bool halo = tid >= NTO;       // the last warp
  const int lane = tid & 31;
  const bool producer = tid == NTO;   // issues the TMA copies
  const int tx = halo ? 0 : tid % 16, ty0 = halo ? 0 : (tid / 16) * RY;  // first owned row of the thread
  const int nrows = halo ? 1 : RY;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  // the launch before this one (observation or step) has finished
  grid_dependency_wait();
  allow_dependents();
  if (tid < L::kItemCache && (int)blockIdx.x + tid * (int)gridDim.x < nitems)
    sitems[tid] = items[blockIdx.x + tid * gridDim.x];
  __syncthreads();

  unsigned ld = 0;     // planes of the items before this one (same value in every thread)
  unsigned phase = 0;  // bit s: parity of the next completion of stage s's barrier
  IssuedLoads loads;   // producer: the loads it issued, drained if the block gives up
  int pf = 0;          // producer: planes of this item already issued by the previous item
  int cur = -1;
  for (int it = blockIdx.x, r = 0; it < nitems; it += gridDim.x, ++r) {
    const int4 item = r < L::kItemCache ? sitems[r] : items[it];
    __syncthreads();
    const bool fresh = item.x != cur;
    if (fresh) {
      load_record(grids + item.x, smem, tid, NT);
      cur = item.x;
    }
    __syncthreads();
    if (fresh && tid < 64) {
      // S/eps of the three E components for every material class triple
      const int c0 = tid & 3, c1 = (tid >> 2) & 3, c2 = (tid >> 4) & 3;
      ctab[tid] = make_float4(G.cE[c0 < 3 ? c0 : 2], G.cE[c1 < 3 ? c1 : 2], G.cE[c2 < 3 ? c2 : 2], 0.0f);
    }
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

    auto issue = [&](int s, int plane) {
      unsigned char* dst = stages + (size_t)s * L::stage_bytes;
      loads.note(s);
      mbar_arrive_expect_tx(&full[s], TX_BYTES);
      tma_load_4d(dst, fmap, x0 - AX, y0 - 1, plane, fs * 6, &full[s]);
      tma_load_3d(dst + L::field_bytes, mmap, x0, y0, plane, &full[s]);
    };
    if (producer) {
      if (fresh) {
        tensormap_acquire(fmap);
        tensormap_acquire(mmap);
      }
      fence_proxy_async_smem();
      for (int p = pf; p < S && p < NP; ++p) issue((int)((q0 + p) % S), kstart + p);
      pf = 0;
      // the next item of this block: its first planes are issued into the
      // stages that this item's last planes free (same grid step, so the
      // planes it reads are not written by this launch)
      nxt.cnt = 0;
      const int nit = it + (int)gridDim.x;
      if (nit < nitems && NP >= S) {
        const int4 ni = r + 1 < L::kItemCache ? sitems[r + 1] : items[nit];
        // the same grid's step and limit are in the block's record
        const StepGrid<float>* ng = grids + ni.x;
        const long long nn = ni.x == item.x ? n : ng->step + offset;
        if (nn < (ni.x == item.x ? G.step_end : ng->step_end)) {
          const int nz0 = ni.w & 0xffff, nz1 = (ni.w >> 16) & 0xffff;
          const int nks = nz0 > 0 ? nz0 - 1 : nz0;
          nxt.fmap = &maps[ni.x].fields;
          nxt.mmap = &maps[ni.x].mat;
          if (ni.x != item.x) {
            tensormap_acquire(nxt.fmap);
            tensormap_acquire(nxt.mmap);
          }
          nxt.x0 = ni.y;
          nxt.y0 = ni.z;
          nxt.kstart = nks;
          nxt.fs = (int)(nn % (ni.x == item.x ? G.nsets : ng->nsets));
          nxt.cnt = min(S - 1, nz1 - nks + 1);
        }
      }
    }

    // this thread's node pairs: RY owned rows (i0, j), or one on the halo row / column
    bool valid[RY];   // node 0 of the pair is a grid node whose H this thread provides
    int o[RY];        // staged offset of node 0
    int hcol[RY];     // H buffer offset of node 0
    int yrow[RY];     // row of the y coefficients
    int sbase[RY];    // slot of node 0 in a stage's CPML area
    int cell[RY];     // pair index in the tile (owned rows): slots, material, output
    PairCol pc[RY];
    unsigned src0[RY], src1[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      valid[r] = false;
      src0[r] = src1[r] = 0u;
      if (r >= nrows) {
        make_pair_col(G, 0, 0, pc[r]);
        o[r] = hcol[r] = yrow[r] = sbase[r] = cell[r] = 0;
      } else if (!halo) {
        const int i0 = x0 + 2 * tx, j = y0 + ty0 + r;
        valid[r] = i0 < nx && j < ny;
        make_pair_col(G, valid[r] ? i0 : 0, valid[r] ? j : 0, pc[r]);
        o[r] = (ty0 + r + 1) * BXT + AX + 2 * tx;
        hcol[r] = (ty0 + r + 1) * HW + 2 + 2 * tx;
        yrow[r] = ty0 + r + 1;
        cell[r] = (ty0 + r) * 16 + tx;
        sbase[r] = 2 * cell[r];
        if (valid[r] && G.nsrc) {
          src0[r] = node_sources(G, i0, j);
          src1[r] = pc[r].own1 ? node_sources(G, i0 + 1, j) : 0u;
        }
      } else if (lane < 16) {
        const int i0 = x0 + 2 * lane, j = y0 - 1;
        valid[r] = y0 > 0 && i0 < nx;
        make_pair_col(G, valid[r] ? i0 : 0, valid[r] ? j : 0, pc[r]);
        o[r] = AX + 2 * lane;
        hcol[r] = 2 + 2 * lane;
        yrow[r] = 0;
        cell[r] = 0;
        sbase[r] = 4 * NC + 2 * lane;
      } else {
        const int rr = lane - 16, j = y0 + rr;
        valid[r] = rr < OY && x0 > 0 && j < ny;  // node 1 of the pair (x0-2, x0-1) is the halo node
        make_pair_col(G, valid[r] ? x0 - 2 : 0, valid[r] ? j : 0, pc[r]);
        pc[r].sx0 = -1;  // node x0-2 is recomputed only to keep the pair aligned: no CPML for it
        o[r] = (rr + 1) * BXT + AX - 2;
        hcol[r] = (rr + 1) * HW;
        yrow[r] = rr + 1;
        cell[r] = 0;
        sbase[r] = 4 * NC + 2 * lane;
      }
      if (!valid[r]) pc[r].sx0 = pc[r].sx1 = pc[r].sy = -1;
    }
    const int sstride = halo ? L::NHC : NC;
    const int xcol = hcol[0] - (hcol[0] / HW) * HW;  // column of node 0 in the x coefficient rows
    const long long pstride = (long long)px * ny;
    // gain state of node 0 of each owned pair in plane 0, and the stride between planes
    long long gbase[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) gbase[r] = (GAIN && !halo && valid[r]) ? gain_base(G, pc[r].i0, pc[r].j, 0) : 0;
    const long long gplane = (long long)ny * G.gxb * (GainWords<float>::NW * 32);

    // slab axis whose CPML memory is fetched ahead: z for the planes of a z
    // slab, else x for pairs in an x slab, else y
    int col_axis[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r)
      col_axis[r] = (pc[r].sx0 >= 0 || pc[r].sx1 >= 0) ? 0 : (pc[r].sy >= 0 ? 1 : -1);
    const int zs_lo = G.Sd[2] ? G.L[4] : 0, zs_hi = G.Sd[2] ? G.nz - G.L[5] : G.nz;
    auto issue_psi = [&](int plane, int stage) {
      if (!FDTD_PAIR_PSI_STAGED) {
        cp_async_commit();
        return;
      }
      float* slots = reinterpret_cast<float*>(stages + (size_t)stage * L::stage_bytes + L::field_bytes + L::mat_bytes);
      const bool zs = plane < zs_lo || plane >= zs_hi;
      const int sz = zs ? slab_index(plane, G.nz, G.L[4], G.L[5]) : -1;
      const bool eside = !halo && plane >= z0;  // E-side memory of the planes this tile updates
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!(valid[r] && plane < z1 && (zs || col_axis[r] >= 0))) continue;
        const int a = zs ? 2 : col_axis[r];
        // psi index of node 0; node 1 follows at +1 whenever it is fetched too
        const int pi0 = a == 2 ? sz * ny * nx + pc[r].pz0
                               : (a == 0 ? plane * ny * G.Sd[0] + (pc[r].sx0 >= 0 ? pc[r].px0 : pc[r].px1 - 1)
                                         : plane * G.Sd[1] * nx + pc[r].py0);
        const bool has0 = a != 0 || pc[r].sx0 >= 0;
        const bool has1 = a == 0 ? pc[r].sx1 >= 0 : pc[r].own1;
        if (has0 && has1 && !(pi0 & 1)) {
          // both nodes, 8-byte aligned: one 8-byte copy per array
          cp_async_pair(slots + sbase[r], G.psiH[sel][a][0] + pi0);
          cp_async_pair(slots + sstride + sbase[r], G.psiH[sel][a][1] + pi0);
          if (eside) {
            cp_async_pair(slots + 2 * NC + sbase[r], G.psiE[a][0] + pi0);
            cp_async_pair(slots + 3 * NC + sbase[r], G.psiE[a][1] + pi0);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (!(e ? has1 : has0)) continue;
            const int pi = pi0 + e;
            cp_async_elem(slots + sbase[r] + e, G.psiH[sel][a][0] + pi);
            cp_async_elem(slots + sstride + sbase[r] + e, G.psiH[sel][a][1] + pi);
            if (eside) {
              cp_async_elem(slots + 2 * NC + sbase[r] + e, G.psiE[a][0] + pi);
              cp_async_elem(slots + 3 * NC + sbase[r] + e, G.psiE[a][1] + pi);
            }
          }
        }
      }
      cp_async_commit();
    };

    // grading coefficients of the columns, rows and planes this item touches
    // (joined to the first plane's copy group; visible after the barrier below)
    {
      // only the axes whose slabs the item's columns (x0-2 .. x0+31), rows
      // (y0-1 .. y0+OY-1) or planes (kstart .. z1-1) reach: no other entry is read
      const bool tsx = G.Sd[0] && (x0 - 2 < G.L[0] || x0 + L::OX - 1 >= nx - G.L[1]);
      const bool tsy = G.Sd[1] && (y0 - 1 < G.L[2] || y0 + OY - 1 >= ny - G.L[3]);
      const bool tsz = G.Sd[2] && (kstart < G.L[4] || z1 - 1 >= G.nz - G.L[5]);
      const int e0 = tsx ? 0 : (tsy ? L::CXN : L::CXN + L::CYN);
      const int e1 = tsz ? L::CXN + L::CYN + 6 * (NP - 1) : (tsy ? L::CXN + L::CYN : (tsx ? L::CXN : 0));
      for (int e = e0 + tid; e < e1; e += NT) {
        int a, pos, hq;
        float* dst;
        if (e < L::CXN) {
          hq = e / HW;
          a = 0; pos = x0 - 2 + (e - hq * HW); dst = cfx + e;
        } else if (e < L::CXN + L::CYN) {
          const int rr = e - L::CXN;
          hq = rr % 6;
          a = 1; pos = y0 - 1 + rr / 6; dst = cfy + rr;
        } else {
          const int rr = e - L::CXN - L::CYN;
          hq = rr % 6;
          a = 2; pos = kstart + rr / 6; dst = cfz + rr;
        }
        const int lim = a == 0 ? nx : (a == 1 ? ny : G.nz);
        const bool t = a == 0 ? tsx : (a == 1 ? tsy : tsz);
        if (t && pos >= 0 && pos < lim) cp_async_elem(dst, G.prof[a][hq / 3][hq % 3] + pos);
      }
    }
    for (int p = 0; p < S; ++p) issue_psi(kstart + p, (int)((q0 + p) % S));
    cp_async_wait<S - 1>();
    __syncthreads();

    float2 hPx[RY], hPy[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) hPx[r] = hPy[r] = make_float2(0.0f, 0.0f);
    bool ok = true;
    const float2 ncH = bc2(-G.cH);
    // Per-warp choice of the node code, decided once per item (columns, rows)
    // and per plane (z slabs, sources, PEC planes): a warp none of whose nodes
    // needs CPML, a source, a PEC hold or gain takes the plain Yee update.
    bool t_slab = false, t_pec = false, t_src = false;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      t_slab = t_slab || (valid[r] && (pc[r].sx0 >= 0 || pc[r].sx1 >= 0 || pc[r].sy >= 0));
      t_pec = t_pec || (valid[r] && (pc[r].i0 == 0 || pc[r].j == 0));
      t_src = t_src || ((src0[r] | src1[r]) != 0u);
    }
    const bool w_slab = __any_sync(0xffffffffu, t_slab);
    const bool w_pec = __any_sync(0xffffffffu, t_pec);
    const bool w_src = __any_sync(0xffffffffu, t_src);
    unsigned src_planes = 0;  // bit p: plane kstart + p holds a node that some source drives
    if (w_src)
      for (int s = 0; s < G.nsrc; ++s) {
        int lo, hi;
        source_planes(G.src[s], lo, hi);
        for (int p = 0; p < NP - 1; ++p)
          if (kstart + p >= lo && kstart + p < hi) src_planes |= 1u << p;
      }

    // stages of the current and the next plane, advanced by rotation
    int sk = (int)(q0 % S), sn = sk + 1 == S ? 0 : sk + 1;
    auto wait_stage = [&](int s) {
      ok = ok && mbar_wait(&full[s], (phase >> s) & 1u, G.wait_ns);
      phase ^= 1u << s;
    };
    for (int p = 0; p < NP - 1; ++p) {
      const int k = kstart + p;
      float* sHx = reinterpret_cast<float*>(smem + L::h_off + (p & 1) * L::hbuf_bytes);
      float* sHy = sHx + L::HPL;
      float* sHz = sHy + L::HPL;
      if (p == 0) wait_stage(sk);
      wait_stage(sn);
      cp_async_wait<S - 1>();  // this thread's CPML memory of plane p
      const unsigned char* stg = stages + (size_t)sk * L::stage_bytes;
      const float* Fk = reinterpret_cast<const float*>(stg);
      const float* Fn = reinterpret_cast<const float*>(stages + (size_t)sn * L::stage_bytes);
      const float* slots = reinterpret_cast<const float*>(stg + L::field_bytes + L::mat_bytes);
      const bool active = k >= z0;
      const bool zslab = k < zs_lo || k >= zs_hi;
      const bool gen_h = w_slab || zslab;                  // warp-uniform
      bool gen_e = gen_h || w_pec || k == 0 || (w_src && ((src_planes >> p) & 1u));
      unsigned mm[RY];
      bool t_gain = false;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        mm[r] = (!halo && active) ? *reinterpret_cast<const unsigned short*>(stg + L::field_bytes + 2 * cell[r]) : 0u;
        t_gain = t_gain || ((((mm[r] >> 6) | (mm[r] >> 14)) & 1u) != 0u);
      }
      if (GAIN && G.gain) gen_e = gen_e || __any_sync(0xffffffffu, t_gain);
      // gain state of this plane's gain pairs: on 32 x 8 tiles (registers for
      // 3 blocks per SM) loaded before the H work, so the loads' latency
      // hides behind it; on 32 x 16 tiles (2 blocks of 288 threads, no
      // registers to spare) loaded where the E update needs it
      PairGain gst[RY];
#pragma unroll
      for (int r = 0; r < RY; ++r)
        if (GAIN && OY == 8 && G.gain && ok && valid[r] && ((((mm[r] >> 6) | (mm[r] >> 14)) & 1u) != 0u))
          load_pair_gain(G, sel, gbase[r] + (long long)k * gplane, gst[r]);
      Plane pl;
      if (gen_h || gen_e) pl = make_plane(G, k);
      const float* cz = cfz + 6 * p;

      float2 hx[RY], hy[RY], hz[RY];
      float2 eox[RY], eoy[RY], eoz[RY];  // E^n of the pair, kept for the E update
      float2 preE[RY][2];
      int pa[RY];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        hx[r] = hy[r] = hz[r] = make_float2(0.0f, 0.0f);
        eox[r] = eoy[r] = eoz[r] = make_float2(0.0f, 0.0f);
        preE[r][0] = preE[r][1] = make_float2(0.0f, 0.0f);
        pa[r] = -1;
        if (r >= nrows || !ok || !valid[r]) continue;
        if (gen_h) {
          // CPML memory of this pair fetched ahead
          float2 pre[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
          pa[r] = FDTD_PAIR_PSI_STAGED ? (zslab ? 2 : col_axis[r]) : -1;
          if (pa[r] >= 0) {
            pre[0] = ld2(slots + sbase[r]);
            pre[1] = ld2(slots + sstride + sbase[r]);
            if (!halo) {
              preE[r][0] = ld2(slots + 2 * NC + sbase[r]);
              preE[r][1] = ld2(slots + 3 * NC + sbase[r]);
            }
          }
          pair_h<true>(G, pc[r], pl, sel, !halo && active, Fk, Fn, o[r], PL, BXT, cfx, xcol, cfy + 6 * yrow[r], cz,
                       pa[r], pre, ncH, eox[r], eoy[r], eoz[r], hx[r], hy[r], hz[r]);
        } else {
          pair_h<false>(G, pc[r], pl, sel, false, Fk, Fn, o[r], PL, BXT, cfx, xcol, cfy, cz, -1, nullptr, ncH, eox[r],
                        eoy[r], eoz[r], hx[r], hy[r], hz[r]);
        }
        if (!pc[r].own1) hx[r].y = hy[r].y = hz[r].y = 0.0f;
      }
      if (halo) {
        if (lane < 16) {
          st2(sHx + hcol[0], hx[0]);
          st2(sHy + hcol[0], hy[0]);
          st2(sHz + hcol[0], hz[0]);
        } else if (lane - 16 < OY) {
          sHx[hcol[0] + 1] = hx[0].y;
          sHy[hcol[0] + 1] = hy[0].y;
          sHz[hcol[0] + 1] = hz[0].y;
        }
      } else {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          st2(sHx + hcol[r], hx[r]);
          st2(sHy + hcol[r], hy[r]);
          st2(sHz + hcol[r], hz[r]);
        }
      }
      if (__syncthreads_or(!ok)) {
        // a wait ran out: let this thread's copies and the block's loads in
        // flight land (bounded) before the block leaves, then report
        cp_async_wait<0>();
        if (producer) atomicOr(G.err, loads.drain(full, S) ? 2 : 6);
        return;
      }
      // nothing reads the fields of plane p's stage after this barrier: refill
      // it with plane p + S (or a first plane of the block's next item) while
      // the owners update E
      if (producer) {
        if (p + S < NP) {
          fence_proxy_async_smem();
          issue(sk, kstart + p + S);
        } else if (p + S - NP < nxt.cnt) {
          fence_proxy_async_smem();
          unsigned char* dst = stages + (size_t)sk * L::stage_bytes;
          loads.note(sk);
          mbar_arrive_expect_tx(&full[sk], TX_BYTES);
          tma_load_4d(dst, nxt.fmap, nxt.x0 - AX, nxt.y0 - 1, nxt.kstart + p + S - NP, nxt.fs * 6, &full[sk]);
          tma_load_3d(dst + L::field_bytes, nxt.mmap, nxt.x0, nxt.y0, nxt.kstart + p + S - NP, &full[sk]);
          ++pf;
        }
      }

      if (active && !halo) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          float2 enx = make_float2(0.0f, 0.0f), eny = enx, enz = enx;
          if (valid[r]) {
            const int oh = hcol[r];
            const float2 ex = eox[r], ey = eoy[r], ez = eoz[r];
            // H of the row below: this thread's previous row when it has one
            const float2 hzJ = (r > 0) ? hz[r - 1] : ld2(sHz + oh - HW);
            const float2 hxJ = (r > 0) ? hx[r - 1] : ld2(sHx + oh - HW);
            float2 dyHz = sub2(hz[r], hzJ);
            float2 dzHy = sub2(hy[r], hPy[r]);
            float2 dzHx = sub2(hx[r], hPx[r]);
            float2 dxHz = sub2(hz[r], make_float2(sHz[oh - 1], hz[r].x));
            float2 dxHy = sub2(hy[r], make_float2(sHy[oh - 1], hy[r].x));
            float2 dyHx = sub2(hx[r], hxJ);
            if (gen_h && (pc[r].sx0 >= 0 || pc[r].sx1 >= 0 || pc[r].sy >= 0 || pl.sz >= 0))
              pair_cpml<0>(G, pc[r], pl, sel, true, cfx, xcol, cfy + 6 * yrow[r], cz, pa[r], preE[r], dxHz, dxHy,
                           dyHx, dyHz, dzHy, dzHx);
            const float2 curlx = sub2(dyHz, dzHy);
            const float2 curly = sub2(dzHx, dxHz);
            const float2 curlz = sub2(dxHy, dyHx);
            const unsigned m0 = mm[r] & 0xffu, m1 = mm[r] >> 8;
            const float4 c0 = ctab[m0 & 63u], c1 = ctab[m1 & 63u];
            enx = fma2(make_float2(c0.x, c1.x), curlx, ex);
            eny = fma2(make_float2(c0.y, c1.y), curly, ey);
            enz = fma2(make_float2(c0.z, c1.z), curlz, ez);
            if (gen_e) {
              const bool pec = pc[r].i0 == 0 || pc[r].j == 0 || pl.pecz;
              const bool gainpair = GAIN && G.gain && (((m0 | m1) >> 6) & 1);
              if (src0[r] | src1[r] | pec | gainpair)
                pair_extras<GAIN, OY == 8>(G, sg, pc[r], pl, sel, n, GAIN ? gbase[r] + (long long)k * gplane : 0, m0, m1,
                                  src0[r], src1[r], ex, ey, ez, gst[r], enx, eny, enz);
            }
            // a node past the grid edge is never stored (its lane holds zeros)
            if (!pc[r].own1) enx.y = eny.y = enz.y = 0.0f;
          }
          // E^{n+1} and H~^{n+1/2} of the pair straight to set (n+1)%3: 8-byte
          // stores, a warp's half-row one 128-byte segment (px is even)
          if (valid[r]) {
            const long long cidx = (long long)pc[r].j * px + pc[r].i0 + (long long)k * pstride;
            float* const* Fo = G.F[fo];
            if (pc[r].own1) {
              st2_out(Fo[0] + cidx, enx);
              st2_out(Fo[1] + cidx, eny);
              st2_out(Fo[2] + cidx, enz);
              st2_out(Fo[3] + cidx, hx[r]);
              st2_out(Fo[4] + cidx, hy[r]);
              st2_out(Fo[5] + cidx, hz[r]);
            } else {
              st1_out(Fo[0] + cidx, enx.x);
              st1_out(Fo[1] + cidx, eny.x);
              st1_out(Fo[2] + cidx, enz.x);
              st1_out(Fo[3] + cidx, hx[r].x);
              st1_out(Fo[4] + cidx, hy[r].x);
              st1_out(Fo[5] + cidx, hz[r].x);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        hPx[r] = hx[r];
        hPy[r] = hy[r];
      }
      // no second barrier: the next plane writes the other H buffer, and the
      // barrier after its H update orders this plane's E reads before the
      // buffer is written again
      issue_psi(kstart + p + S, sk);
      sk = sn;
      sn = sn + 1 == S ? 0 : sn + 1;
    }
    ld = q0 + (unsigned)NP;
  }
  cp_async_wait<0>();
}

// Rows of node pairs per owner thread for a tile of oy rows.
constexpr int pair_rows(int oy) { return oy == 16 ? FDTD_PAIR_RY : 1; }

int step_pair_blocks_per_sm(bool gain, int oy) {
  const size_t smem = step_pair_smem_bytes(oy);
  const void* f;
  int threads;
  if (oy == 8) {
    f = gain ? (const void*)k_step_pair<true, 8, pair_rows(8)> : (const void*)k_step_pair<false, 8, pair_rows(8)>;
    threads = PairThreads<8, pair_rows(8)>::NT;
  } else {
    f = gain ? (const void*)k_step_pair<true, 16, pair_rows(16)> : (const void*)k_step_pair<false, 16, pair_rows(16)>;
    threads = PairThreads<16, pair_rows(16)>::NT;
  }
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

// Resident blocks of the paired kernel on the whole GPU (per template; the
// occupancy query runs once).
static int pair_resident_blocks(bool gain, int oy) {
  static int cache[2][2] = {{0, 0}, {0, 0}};
  int& v = cache[gain ? 1 : 0][oy == 8 ? 1 : 0];
  if (v == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0) {
      cudaGetLastError();
      sms = 1;
    }
    v = step_pair_blocks_per_sm(gain, oy) * sms;
  }
  return v;
}

cudaError_t launch_step_pair(const StepGrid<float>* grids, const TmaGrid* maps, const int4* items, int nitems,
                             int offset, int oy, bool gain, int grid_blocks, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  // grid_blocks 0: persistent, one wave of resident blocks, each taking every
  // gridDim-th item and fetching its next item's first planes ahead
  const int want = grid_blocks > 0 ? grid_blocks : pair_resident_blocks(gain, oy);
  const int blocks = want < nitems ? want : nitems;
  const size_t smem = step_pair_smem_bytes(oy);
  if (oy == 8) {
    auto f = gain ? k_step_pair<true, 8, pair_rows(8)> : k_step_pair<false, 8, pair_rows(8)>;
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_programmatic(f, dim3(blocks), dim3(PairThreads<8, pair_rows(8)>::NT), smem, st, grids, maps, items,
                               nitems, offset);
  }
  auto f = gain ? k_step_pair<true, 16, pair_rows(16)> : k_step_pair<false, 16, pair_rows(16)>;
  cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return launch_programmatic(f, dim3(blocks), dim3(PairThreads<16, pair_rows(16)>::NT), smem, st, grids, maps, items,
                             nitems, offset);
}

}  // namespace fdtd
