// Per-node update arithmetic shared by the step kernels (identical results
// whichever kernel stages the data: every multiply-add is written as an
// explicit fma so the compiler cannot contract differently per kernel).
//
// Paper: Yee leapfrog (Sec. "Sample and numerical approach"), absorbing layer
// (same section; CPML reading), four-level gain with the polarization at the
// Yee node and spontaneous-emission noise as a random kick (same section), soft pulsed
// sources (Secs. "Wide-band excitation", "Dynamical diffusion").
#pragma once

#include <math.h>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ long long pidx3(int i, int j, int k, int px, int ny) {
  return ((long long)k * ny + j) * px + i;
}

__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplications with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 noise_bits(unsigned long long seed, long long cell, long long step) {
  return philox4x32_10(make_uint4((unsigned)cell, (unsigned)((unsigned long long)cell >> 32), (unsigned)step,
                                  (unsigned)((unsigned long long)step >> 32)),
                       make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// Three N(0,1) deviates for (seed, cell, step): Box-Muller on the uniforms
// u = ((x >> 9) + 0.5) 2^-23 (exact in binary32).  Binary32 runs take the
// special-function-unit forms of log, sin and cos (__logf, __sincosf,
// __cosf; documented bounds: absolute error 2^-21.41 for log on [0.5, 2] and
// for sin and cos on [-pi, pi], 3 ulp for log elsewhere), with the angle
// 2 pi u moved to [-pi, pi) by the exact shift u - 1/2 (cos and sin change
// sign).  A deviate then differs from the binary64 Box-Muller value of the
// same uniforms by about 1e-6 relative (larger only where rho is tiny).
__device__ __forceinline__ void gain_normals(unsigned long long seed, long long cell, long long step, float& a,
                                             float& b, float& c) {
  const uint4 x = noise_bits(seed, cell, step);
  const float u0 = ((float)(x.x >> 9) + 0.5f) * 0x1p-23f;
  const float u1 = ((float)(x.y >> 9) + 0.5f) * 0x1p-23f;
  const float u2 = ((float)(x.z >> 9) + 0.5f) * 0x1p-23f;
  const float u3 = ((float)(x.w >> 9) + 0.5f) * 0x1p-23f;
  constexpr float kTwoPi = 6.28318530717958648f;
  // log u < 0, but within its error bound the approximation may come out
  // positive for u just below 1: clamp before the square root
  const float rho = sqrtf(fmaxf(-2.0f * __logf(u0), 0.0f));
  float s, co;
  __sincosf(kTwoPi * (u1 - 0.5f), &s, &co);
  a = -(rho * co);
  b = -(rho * s);
  c = -(sqrtf(fmaxf(-2.0f * __logf(u2), 0.0f)) * __cosf(kTwoPi * (u3 - 0.5f)));
}

__device__ __forceinline__ void gain_normals(unsigned long long seed, long long cell, long long step, double& a,
                                             double& b, double& c) {
  const uint4 x = noise_bits(seed, cell, step);
  const double u0 = ((double)(x.x >> 9) + 0.5) * 0x1p-23;
  const double u1 = ((double)(x.y >> 9) + 0.5) * 0x1p-23;
  const double u2 = ((double)(x.z >> 9) + 0.5) * 0x1p-23;
  const double u3 = ((double)(x.w >> 9) + 0.5) * 0x1p-23;
  const double rho = sqrt(-2.0 * log(u0));
  double s, co;
  sincospi(2.0 * u1, &s, &co);
  a = rho * co;
  b = rho * s;
  c = sqrt(-2.0 * log(u2)) * cospi(2.0 * u3);
}

// CPML grading coefficients of a node: c(axis, h, q) with h = 0 for the
// E-curl (integer) node and 1 for the H-curl (half-integer) node, q = 0, 1, 2
// for 1/kappa, b, c.  CoefGlobal reads the grid's profile arrays; the TMA
// kernel stages the tile's coefficients in shared memory (CoefShared).
template <typename T>
struct CoefGlobal {
  const StepGrid<T>* G;
  int i, j, k;
  __device__ __forceinline__ T x(int h, int q) const { return G->prof[0][h][q][i]; }
  __device__ __forceinline__ T y(int h, int q) const { return G->prof[1][h][q][j]; }
  __device__ __forceinline__ T z(int h, int q) const { return G->prof[2][h][q][k]; }
};

template <typename T>
struct CoefShared {
  const T* px;  // 6 values (h, q) of the node's column, row and plane
  const T* py;
  const T* pz;
  __device__ __forceinline__ T x(int h, int q) const { return px[h * 3 + q]; }
  __device__ __forceinline__ T y(int h, int q) const { return py[h * 3 + q]; }
  __device__ __forceinline__ T z(int h, int q) const { return pz[h * 3 + q]; }
};

// CPML-modified difference D / kappa + psi with psi <- b psi + c D.
template <typename T>
__device__ __forceinline__ T pml_term_c(T D, T ik, T b, T c, T psi_old, T* psi_out, int pi) {
  const T p = fmad(b, psi_old, c * D);
  if (psi_out) psi_out[pi] = p;
  return fmad(ik, D, p);
}

// CPML memory of one slab axis of a node, fetched ahead of its update:
// H-side slots 0, 1 (set sel) and E-side slots 0, 1.  axis < 0: nothing fetched.
template <typename T>
struct PsiPre {
  int axis;
  T h0, h1, e0, e1;
};

// Slab coordinate of node index q on an axis of length n with slabs L0, L1 (-1 outside).
__device__ __forceinline__ int slab_index(int q, int n, int L0, int L1) {
  if (q < L0) return q;
  if (q >= n - L1) return L0 + q - (n - L1);
  return -1;
}

// Planes [lo, hi) whose E nodes source S drives.
__device__ __forceinline__ void source_planes(const SrcDev& S, int& lo, int& hi) {
  if (S.kind == 0) {
    lo = S.k;
    hi = S.k + 1;
  } else if (S.axis == 2) {
    lo = S.index;
    hi = S.index + 1;
  } else if (S.axis == 0) {
    lo = S.lo2;
    hi = S.hi2;
  } else {
    lo = S.lo1;
    hi = S.hi1;
  }
}

// Soft-source waveform at update n (FP64) of every source of the grid that
// drives a node of planes [za, zb), into sg[] (the others are never read).
template <typename T>
__device__ __forceinline__ void source_waveforms(const StepGrid<T>& G, long long n, int tid, double* sg,
                                                 int za = 0, int zb = 0x7fffffff) {
  if (tid < G.nsrc) {
    const SrcDev& s = G.src[tid];
    int lo, hi;
    source_planes(s, lo, hi);
    if (lo < zb && hi > za) {
      const double t = (double)n + 0.5 - s.t0;
      sg[tid] = exp(-t * t / (2.0 * s.tau * s.tau)) * sin(2.0 * 3.14159265358979323846 * s.f0dt * t);
    }
  }
}

// Everything about a node column (i, j) that stays fixed while a tile
// marches in z: CPML slab coordinates and memory offsets, the sources that
// can touch the column, the PEC holds of its x and y faces.
struct Column {
  int i, j;
  int sx, sy;         // slab coordinates, -1 outside the x / y slabs
  int px0, py0, pz0;  // psi offsets of plane 0 (x slab, y slab) and the column offset in a z slab
  unsigned src;       // bit s: source s can touch this column
  bool pecx, pecy;    // i == 0 on a non-periodic x axis, j == 0 on a non-periodic y axis
};

template <typename T>
__device__ __forceinline__ void make_column(const StepGrid<T>& G, int i, int j, Column& c, bool with_sources = true) {
  c.i = i;
  c.j = j;
  c.sx = G.Sd[0] ? slab_index(i, G.nx, G.L[0], G.L[1]) : -1;
  c.sy = G.Sd[1] ? slab_index(j, G.ny, G.L[2], G.L[3]) : -1;
  c.px0 = j * G.Sd[0] + c.sx;
  c.py0 = c.sy * G.nx + i;
  c.pz0 = j * G.nx + i;
  c.pecx = (i == 0) && !(G.per & 1);
  c.pecy = (j == 0) && !(G.per & 2);
  unsigned m = 0;
  for (int s = 0; with_sources && s < G.nsrc; ++s) {
    const SrcDev& S = G.src[s];
    bool hit;
    if (S.kind == 0) {
      hit = (i == S.i && j == S.j);
    } else if (S.axis == 2) {
      hit = (i >= S.lo1 && i < S.hi1 && j >= S.lo2 && j < S.hi2);
    } else if (S.axis == 0) {
      hit = (i == S.index && j >= S.lo1 && j < S.hi1);
    } else {
      hit = (j == S.index && i >= S.lo2 && i < S.hi2);
    }
    if (hit) m |= 1u << s;
  }
  c.src = m;
}

// Per-plane facts shared by all nodes of plane k.
struct Plane {
  int k;
  int sz;        // z slab coordinate, -1 outside
  int pz_plane;  // psi offset of the plane in a z slab
  int px_plane;  // k * ny * Sd0
  int py_plane;  // k * Sd1 * nx
  bool pecz;     // k == 0 on a non-periodic z axis
};

template <typename T>
__device__ __forceinline__ Plane make_plane(const StepGrid<T>& G, int k) {
  Plane p;
  p.k = k;
  p.sz = G.Sd[2] ? slab_index(k, G.nz, G.L[4], G.L[5]) : -1;
  p.pz_plane = p.sz * G.ny * G.nx;
  p.px_plane = k * G.ny * G.Sd[0];
  p.py_plane = k * G.Sd[1] * G.nx;
  p.pecz = (k == 0) && !(G.per & 4);
  return p;
}

// H~^{n+1/2} at node (c.i, c.j, p.k) from the six forward differences of E^n.
// Inside a slab the difference becomes D/kappa + psi; psi^{n-1/2} is read from
// set `sel`, psi^{n+1/2} written to set sel^1 when `wr` (owner of the node).
template <typename T, typename CF>
__device__ __forceinline__ void h_node(const StepGrid<T>& G, const Column& c, const Plane& p, int sel, bool wr,
                                       const CF& cf, T dyEz, T dzEy, T dzEx, T dxEz, T dxEy, T dyEx, T hOx, T hOy,
                                       T hOz, T& hx, T& hy, T& hz, const PsiPre<T>* pre = nullptr) {
  const int pa = pre ? pre->axis : -1;
  if (c.sx >= 0) {
    const int pi = p.px_plane + c.px0;
    T* o0 = wr ? G.psiH[sel ^ 1][0][0] : (T*)nullptr;
    T* o1 = wr ? G.psiH[sel ^ 1][0][1] : (T*)nullptr;
    const T ik = cf.x(1, 0), b = cf.x(1, 1), cc = cf.x(1, 2);
    const T s0 = pa == 0 ? pre->h0 : G.psiH[sel][0][0][pi];
    const T s1 = pa == 0 ? pre->h1 : G.psiH[sel][0][1][pi];
    dxEz = pml_term_c(dxEz, ik, b, cc, s0, o0, pi);
    dxEy = pml_term_c(dxEy, ik, b, cc, s1, o1, pi);
  }
  if (c.sy >= 0) {
    const int pi = p.py_plane + c.py0;
    T* o0 = wr ? G.psiH[sel ^ 1][1][0] : (T*)nullptr;
    T* o1 = wr ? G.psiH[sel ^ 1][1][1] : (T*)nullptr;
    const T ik = cf.y(1, 0), b = cf.y(1, 1), cc = cf.y(1, 2);
    const T s0 = pa == 1 ? pre->h0 : G.psiH[sel][1][0][pi];
    const T s1 = pa == 1 ? pre->h1 : G.psiH[sel][1][1][pi];
    dyEx = pml_term_c(dyEx, ik, b, cc, s0, o0, pi);
    dyEz = pml_term_c(dyEz, ik, b, cc, s1, o1, pi);
  }
  if (p.sz >= 0) {
    const int pi = p.pz_plane + c.pz0;
    T* o0 = wr ? G.psiH[sel ^ 1][2][0] : (T*)nullptr;
    T* o1 = wr ? G.psiH[sel ^ 1][2][1] : (T*)nullptr;
    const T ik = cf.z(1, 0), b = cf.z(1, 1), cc = cf.z(1, 2);
    const T s0 = pa == 2 ? pre->h0 : G.psiH[sel][2][0][pi];
    const T s1 = pa == 2 ? pre->h1 : G.psiH[sel][2][1][pi];
    dzEy = pml_term_c(dzEy, ik, b, cc, s0, o0, pi);
    dzEx = pml_term_c(dzEx, ik, b, cc, s1, o1, pi);
  }
  const T cH = G.cH;
  hx = fmad(-cH, dyEz - dzEy, hOx);
  hy = fmad(-cH, dzEx - dxEz, hOy);
  hz = fmad(-cH, dxEy - dyEx, hOz);
}

// Gain state of one node, loaded ahead of its update.
template <typename T>
struct GainState {
  T pnx, pny, pnz, pmx, pmy, pmz, d1, d2, d3, c1, c2, c3;
};

// Index of word 0 of node (i, j, k)'s gain state.  The state of the 32
// nodes i = 32 b .. 32 b + 31 of a row lies in one record of NW runs of 32
// values (word w of node i at +32 w), so a warp reads or writes each word of
// a row segment as one contiguous 128-byte (binary32) line, and the words of
// a node sit at fixed offsets from one address.
template <typename T>
__device__ __forceinline__ long long gain_base(const StepGrid<T>& G, int i, int j, int k) {
  return (((long long)k * G.ny + j) * G.gxb + (i >> 5)) * (GainWords<T>::NW * 32) + (i & 31);
}

template <typename T>
__device__ __forceinline__ void load_gain(const StepGrid<T>& G, int sel, long long gidx, GainState<T>& s) {
  using W = GainWords<T>;
  const T* g = G.gst + gidx;
  const T* pn = g + 32 * (sel ? W::P1 : W::P0);
  const T* pm = g + 32 * (sel ? W::P0 : W::P1);
  s.pnx = pn[0];
  s.pny = pn[32];
  s.pnz = pn[64];
  s.pmx = pm[0];
  s.pmy = pm[32];
  s.pmz = pm[64];
  s.d1 = g[32 * W::DN];
  s.d2 = g[32 * W::DN + 32];
  s.d3 = g[32 * W::DN + 64];
  if (sizeof(T) == 4) {
    s.c1 = g[32 * W::CMP];
    s.c2 = g[32 * W::CMP + 32];
    s.c3 = g[32 * W::CMP + 64];
  } else {
    s.c1 = s.c2 = s.c3 = T(0);
  }
}

// Soft-source drive of the node's three E components at plane p.k.
template <typename T>
__device__ __forceinline__ void source_drive(const StepGrid<T>& G, const double* sg, const Column& c, const Plane& p,
                                             T& sx, T& sy, T& sz) {
  unsigned m = c.src;
  while (m) {
    const int s = __ffs(m) - 1;
    m &= m - 1;
    const SrcDev& S = G.src[s];
    double w = 0.0;
    if (S.kind == 0) {
      if (p.k == S.k) w = S.amp;
    } else {
      int u, v;
      bool on;
      if (S.axis == 2) {
        on = p.k == S.index;
        u = c.i;
        v = c.j;
      } else if (S.axis == 0) {
        on = p.k >= S.lo2 && p.k < S.hi2;
        u = c.j;
        v = p.k;
      } else {
        on = p.k >= S.lo1 && p.k < S.hi1;
        u = p.k;
        v = c.i;
      }
      if (on) {
        if (S.inv_w2 > 0.0) {
          const double du = u - S.uc, dv = v - S.vc;
          w = S.amp * exp(-(du * du + dv * dv) * S.inv_w2);
        } else {
          w = S.amp;
        }
      }
    }
    if (w != 0.0) {
      const T val = (T)(w * sg[s]);
      if (S.comp == 0) sx += val;
      else if (S.comp == 1) sy += val;
      else sz += val;
    }
  }
}

// E^{n+1} at node (c.i, c.j, p.k) from the six backward differences of
// H~^{n+1/2}, with the CPML (E-side memory updated in place), the soft
// sources, the gain polarization current and populations (state `gs` of a
// gain cell, loaded from and stored back to gain_base index `gidx`), and the
// PEC hold of tangential E on index-0 planes.
template <typename T, bool GAIN, typename CF>
__device__ __forceinline__ void e_node(const StepGrid<T>& G, const double* sg, const Column& c, const Plane& p,
                                       int sel, long long n, long long gidx, unsigned m, bool gcell,
                                       const GainState<T>& gs, const CF& cf, T dyHz, T dzHy, T dzHx, T dxHz, T dxHy,
                                       T dyHx, T eCx, T eCy, T eCz, T& enx, T& eny, T& enz,
                                       const PsiPre<T>* pre = nullptr) {
  const int pa = pre ? pre->axis : -1;
  if (c.sx >= 0) {
    const int pi = p.px_plane + c.px0;
    const T ik = cf.x(0, 0), b = cf.x(0, 1), cc = cf.x(0, 2);
    const T s0 = pa == 0 ? pre->e0 : G.psiE[0][0][pi];
    const T s1 = pa == 0 ? pre->e1 : G.psiE[0][1][pi];
    dxHz = pml_term_c(dxHz, ik, b, cc, s0, G.psiE[0][0], pi);
    dxHy = pml_term_c(dxHy, ik, b, cc, s1, G.psiE[0][1], pi);
  }
  if (c.sy >= 0) {
    const int pi = p.py_plane + c.py0;
    const T ik = cf.y(0, 0), b = cf.y(0, 1), cc = cf.y(0, 2);
    const T s0 = pa == 1 ? pre->e0 : G.psiE[1][0][pi];
    const T s1 = pa == 1 ? pre->e1 : G.psiE[1][1][pi];
    dyHx = pml_term_c(dyHx, ik, b, cc, s0, G.psiE[1][0], pi);
    dyHz = pml_term_c(dyHz, ik, b, cc, s1, G.psiE[1][1], pi);
  }
  if (p.sz >= 0) {
    const int pi = p.pz_plane + c.pz0;
    const T ik = cf.z(0, 0), b = cf.z(0, 1), cc = cf.z(0, 2);
    const T s0 = pa == 2 ? pre->e0 : G.psiE[2][0][pi];
    const T s1 = pa == 2 ? pre->e1 : G.psiE[2][1][pi];
    dzHy = pml_term_c(dzHy, ik, b, cc, s0, G.psiE[2][0], pi);
    dzHx = pml_term_c(dzHx, ik, b, cc, s1, G.psiE[2][1], pi);
  }
  const T curlx = dyHz - dzHy;
  const T curly = dzHx - dxHz;
  const T curlz = dxHy - dyHx;
  const int clx = m & 3, cly = (m >> 2) & 3, clz = (m >> 4) & 3;

  T srcx = T(0), srcy = T(0), srcz = T(0);
  if (c.src) source_drive(G, sg, c, p, srcx, srcy, srcz);

  T dPx = T(0), dPy = T(0), dPz = T(0);
  if (GAIN && gcell) {
    const T dn12 = G.n12eq + (gs.d1 - gs.d2);
    const T drive = G.a3 * dn12;
    const T a1 = G.a1, a2 = G.a2;
    T Pnx = fmad(drive, eCx, fmad(a1, gs.pnx, -(a2 * gs.pmx)));
    T Pny = fmad(drive, eCy, fmad(a1, gs.pny, -(a2 * gs.pmy)));
    T Pnz = fmad(drive, eCz, fmad(a1, gs.pnz, -(a2 * gs.pmz)));
    if (G.noise != T(0)) {
      T xa, xb, xc;
      const long long lcell = ((long long)p.k * G.ny + c.j) * G.nx + c.i;
      gain_normals(G.seed, lcell, n, xa, xb, xc);
      Pnx = fmad(G.noise, xa, Pnx);
      Pny = fmad(G.noise, xb, Pny);
      Pnz = fmad(G.noise, xc, Pnz);
    }
    dPx = Pnx - gs.pnx;
    dPy = Pny - gs.pny;
    dPz = Pnz - gs.pnz;
    T* pm = G.gst + gidx + 32 * (sel ? GainWords<T>::P0 : GainWords<T>::P1);  // receives P~^{n+1}
    pm[0] = Pnx;
    pm[32] = Pny;
    pm[64] = Pnz;
  }

  enx = fmad(-G.cP[clx], dPx + srcx, fmad(G.cE[clx], curlx, eCx));
  eny = fmad(-G.cP[cly], dPy + srcy, fmad(G.cE[cly], curly, eCy));
  enz = fmad(-G.cP[clz], dPz + srcz, fmad(G.cE[clz], curlz, eCz));
  if (c.pecy || p.pecz) enx = T(0);
  if (c.pecx || p.pecz) eny = T(0);
  if (c.pecx || c.pecy) enz = T(0);

  if (GAIN && gcell) {
    const T hx_ = T(0.5) * (enx + eCx), hy_ = T(0.5) * (eny + eCy), hz_ = T(0.5) * (enz + eCz);
    const T r = G.q * fmad(hz_, dPz, fmad(hy_, dPy, hx_ * dPx));
    const T inc1 = fmad(G.w[0], r, fmad(G.D[0][2], gs.d3, fmad(G.D[0][1], gs.d2, G.D[0][0] * gs.d1)));
    const T inc2 = fmad(G.w[1], r, fmad(G.D[1][2], gs.d3, fmad(G.D[1][1], gs.d2, G.D[1][0] * gs.d1)));
    const T inc3 = fmad(G.w[2], r, fmad(G.D[2][2], gs.d3, fmad(G.D[2][1], gs.d2, G.D[2][0] * gs.d1)));
    if (sizeof(T) == 4) {
      // compensated (Kahan) accumulation of the population deviations
      const T y1 = inc1 - gs.c1, y2 = inc2 - gs.c2, y3 = inc3 - gs.c3;
      const T t1 = gs.d1 + y1, t2 = gs.d2 + y2, t3 = gs.d3 + y3;
      T* g = G.gst + gidx;
      g[32 * GainWords<T>::CMP] = (t1 - gs.d1) - y1;
      g[32 * GainWords<T>::CMP + 32] = (t2 - gs.d2) - y2;
      g[32 * GainWords<T>::CMP + 64] = (t3 - gs.d3) - y3;
      g[32 * GainWords<T>::DN] = t1;
      g[32 * GainWords<T>::DN + 32] = t2;
      g[32 * GainWords<T>::DN + 64] = t3;
    } else {
      T* g = G.gst + gidx;
      g[32 * GainWords<T>::DN] = gs.d1 + inc1;
      g[32 * GainWords<T>::DN + 32] = gs.d2 + inc2;
      g[32 * GainWords<T>::DN + 64] = gs.d3 + inc3;
    }
  }
}

}  // namespace fdtd
