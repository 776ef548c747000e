// Per-node update arithmetic shared by the step kernels (identical results
// whichever kernel stages the data).
//
// Paper: Yee leapfrog (Sec. "Sample and numerical approach"), absorbing layer
// (same section; CPML reading), four-level gain with the polarization at the
// Yee node and noise as a stochastic source (same section), soft pulsed
// sources (Secs. "Wide-band excitation", "Dynamical diffusion").
#pragma once

#include <math.h>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ long long pidx3(int i, int j, int k, int px, int ny) {
  return ((long long)k * ny + j) * px + i;
}

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
// u = ((x >> 9) + 0.5) 2^-23 (exact in binary32).
__device__ __forceinline__ void gain_normals(unsigned long long seed, long long cell, long long step, float& a,
                                             float& b, float& c) {
  const uint4 x = noise_bits(seed, cell, step);
  const float u0 = ((float)(x.x >> 9) + 0.5f) * 0x1p-23f;
  const float u1 = ((float)(x.y >> 9) + 0.5f) * 0x1p-23f;
  const float u2 = ((float)(x.z >> 9) + 0.5f) * 0x1p-23f;
  const float u3 = ((float)(x.w >> 9) + 0.5f) * 0x1p-23f;
  const float rho = sqrtf(-2.0f * logf(u0));
  float s, co;
  sincospif(2.0f * u1, &s, &co);
  a = rho * co;
  b = rho * s;
  c = sqrtf(-2.0f * logf(u2)) * cospif(2.0f * u3);
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

// CPML-modified difference: D / kappa + psi with psi <- b psi + c D.
template <typename T>
__device__ __forceinline__ T pml_term(T D, const T* const* pr, int pos, const T* psi_in, T* psi_out,
                                      long long pi) {
  const T p = pr[1][pos] * psi_in[pi] + pr[2][pos] * D;
  if (psi_out) psi_out[pi] = p;
  return pr[0][pos] * D + p;
}

// Slab coordinate of node index q on an axis of length n with slabs L0, L1 (-1 outside).
__device__ __forceinline__ int slab_index(int q, int n, int L0, int L1) {
  if (q < L0) return q;
  if (q >= n - L1) return L0 + q - (n - L1);
  return -1;
}

// Soft-source waveform of every source of the grid at update n (FP64), into sg[].
template <typename T>
__device__ __forceinline__ void source_waveforms(const StepGrid<T>& G, long long n, int tid, double* sg) {
  if (tid < G.nsrc) {
    const SrcDev& s = G.src[tid];
    const double t = (double)n + 0.5 - s.t0;
    sg[tid] = exp(-t * t / (2.0 * s.tau * s.tau)) * sin(2.0 * 3.14159265358979323846 * s.f0dt * t);
  }
}

// H~^{n+1/2} at node (iw, jw, kw) from the six forward differences of E^n.
// Inside a slab the difference becomes D/kappa + psi; psi^{n-1/2} is read from
// set `sel`, psi^{n+1/2} written to set sel^1 when `wr` (owner of the node).
template <typename T>
__device__ __forceinline__ void h_node(const StepGrid<T>& G, int sel, bool wr, int iw, int jw, int kw, T dyEz,
                                       T dzEy, T dzEx, T dxEz, T dxEy, T dyEx, T hOx, T hOy, T hOz, T& hx, T& hy,
                                       T& hz) {
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  if (G.Sd[0]) {
    const int s = slab_index(iw, nx, G.L[0], G.L[1]);
    if (s >= 0) {
      const long long pi = ((long long)kw * ny + jw) * G.Sd[0] + s;
      dxEz = pml_term(dxEz, G.prof[0][1], iw, G.psiH[sel][0][0], wr ? G.psiH[sel ^ 1][0][0] : (T*)nullptr, pi);
      dxEy = pml_term(dxEy, G.prof[0][1], iw, G.psiH[sel][0][1], wr ? G.psiH[sel ^ 1][0][1] : (T*)nullptr, pi);
    }
  }
  if (G.Sd[1]) {
    const int s = slab_index(jw, ny, G.L[2], G.L[3]);
    if (s >= 0) {
      const long long pi = ((long long)kw * G.Sd[1] + s) * nx + iw;
      dyEx = pml_term(dyEx, G.prof[1][1], jw, G.psiH[sel][1][0], wr ? G.psiH[sel ^ 1][1][0] : (T*)nullptr, pi);
      dyEz = pml_term(dyEz, G.prof[1][1], jw, G.psiH[sel][1][1], wr ? G.psiH[sel ^ 1][1][1] : (T*)nullptr, pi);
    }
  }
  if (G.Sd[2]) {
    const int s = slab_index(kw, nz, G.L[4], G.L[5]);
    if (s >= 0) {
      const long long pi = ((long long)s * ny + jw) * nx + iw;
      dzEy = pml_term(dzEy, G.prof[2][1], kw, G.psiH[sel][2][0], wr ? G.psiH[sel ^ 1][2][0] : (T*)nullptr, pi);
      dzEx = pml_term(dzEx, G.prof[2][1], kw, G.psiH[sel][2][1], wr ? G.psiH[sel ^ 1][2][1] : (T*)nullptr, pi);
    }
  }
  hx = hOx - G.cH * (dyEz - dzEy);
  hy = hOy - G.cH * (dzEx - dxEz);
  hz = hOz - G.cH * (dxEy - dyEx);
}

// Gain state of one node, loaded ahead of its update.
template <typename T>
struct GainState {
  T pnx, pny, pnz, pmx, pmy, pmz, d1, d2, d3, c1, c2, c3;
};

template <typename T>
__device__ __forceinline__ void load_gain(const StepGrid<T>& G, int sel, long long cidx, GainState<T>& s) {
  s.pnx = G.P[sel][0][cidx];
  s.pny = G.P[sel][1][cidx];
  s.pnz = G.P[sel][2][cidx];
  s.pmx = G.P[sel ^ 1][0][cidx];
  s.pmy = G.P[sel ^ 1][1][cidx];
  s.pmz = G.P[sel ^ 1][2][cidx];
  s.d1 = G.dN[0][cidx];
  s.d2 = G.dN[1][cidx];
  s.d3 = G.dN[2][cidx];
  if (sizeof(T) == 4) {
    s.c1 = G.cmp[0][cidx];
    s.c2 = G.cmp[1][cidx];
    s.c3 = G.cmp[2][cidx];
  } else {
    s.c1 = s.c2 = s.c3 = T(0);
  }
}

// E^{n+1} at node (iw, jw, kw) from the six backward differences of H~^{n+1/2},
// with the CPML (E-side memory updated in place), the soft sources, the gain
// polarization current and populations (state `gs` of a gain cell), and the
// PEC hold of tangential E on the index-0 planes of non-periodic axes.
template <typename T, bool GAIN>
__device__ __forceinline__ void e_node(const StepGrid<T>& G, const double* sg, int sel, long long n, int iw, int jw,
                                       int kw, long long cidx, unsigned m, bool gcell, const GainState<T>& gs,
                                       T dyHz, T dzHy, T dzHx, T dxHz, T dxHy, T dyHx, T eCx, T eCy, T eCz, T& enx,
                                       T& eny, T& enz) {
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  if (G.Sd[0]) {
    const int s = slab_index(iw, nx, G.L[0], G.L[1]);
    if (s >= 0) {
      const long long pi = ((long long)kw * ny + jw) * G.Sd[0] + s;
      dxHz = pml_term(dxHz, G.prof[0][0], iw, G.psiE[0][0], G.psiE[0][0], pi);
      dxHy = pml_term(dxHy, G.prof[0][0], iw, G.psiE[0][1], G.psiE[0][1], pi);
    }
  }
  if (G.Sd[1]) {
    const int s = slab_index(jw, ny, G.L[2], G.L[3]);
    if (s >= 0) {
      const long long pi = ((long long)kw * G.Sd[1] + s) * nx + iw;
      dyHx = pml_term(dyHx, G.prof[1][0], jw, G.psiE[1][0], G.psiE[1][0], pi);
      dyHz = pml_term(dyHz, G.prof[1][0], jw, G.psiE[1][1], G.psiE[1][1], pi);
    }
  }
  if (G.Sd[2]) {
    const int s = slab_index(kw, nz, G.L[4], G.L[5]);
    if (s >= 0) {
      const long long pi = ((long long)s * ny + jw) * nx + iw;
      dzHy = pml_term(dzHy, G.prof[2][0], kw, G.psiE[2][0], G.psiE[2][0], pi);
      dzHx = pml_term(dzHx, G.prof[2][0], kw, G.psiE[2][1], G.psiE[2][1], pi);
    }
  }
  const T curlx = dyHz - dzHy;
  const T curly = dzHx - dxHz;
  const T curlz = dxHy - dyHx;
  const int clx = m & 3, cly = (m >> 2) & 3, clz = (m >> 4) & 3;

  // soft sources
  T srcx = T(0), srcy = T(0), srcz = T(0);
  for (int s = 0; s < G.nsrc; ++s) {
    const SrcDev& S = G.src[s];
    double w = 0.0;
    if (S.kind == 0) {
      if (iw == S.i && jw == S.j && kw == S.k) w = S.amp;
    } else {
      const int a = S.axis;
      const int along = a == 0 ? iw : a == 1 ? jw : kw;
      if (along == S.index) {
        const int u = a == 0 ? jw : a == 1 ? kw : iw;
        const int v = a == 0 ? kw : a == 1 ? iw : jw;
        if (u >= S.lo1 && u < S.hi1 && v >= S.lo2 && v < S.hi2) {
          if (S.inv_w2 > 0.0) {
            const double du = u - S.uc, dv = v - S.vc;
            w = S.amp * exp(-(du * du + dv * dv) * S.inv_w2);
          } else {
            w = S.amp;
          }
        }
      }
    }
    if (w != 0.0) {
      const T val = (T)(w * sg[s]);
      if (S.comp == 0) srcx += val;
      else if (S.comp == 1) srcy += val;
      else srcz += val;
    }
  }

  T dPx = T(0), dPy = T(0), dPz = T(0);
  if (GAIN && gcell) {
    const T dn12 = G.n12eq + (gs.d1 - gs.d2);
    const T drive = G.a3 * dn12;
    T Pnx = G.a1 * gs.pnx - G.a2 * gs.pmx + drive * eCx;
    T Pny = G.a1 * gs.pny - G.a2 * gs.pmy + drive * eCy;
    T Pnz = G.a1 * gs.pnz - G.a2 * gs.pmz + drive * eCz;
    if (G.noise != T(0)) {
      T xa, xb, xc;
      const long long lcell = ((long long)kw * ny + jw) * nx + iw;
      gain_normals(G.seed, lcell, n, xa, xb, xc);
      Pnx += G.noise * xa;
      Pny += G.noise * xb;
      Pnz += G.noise * xc;
    }
    dPx = Pnx - gs.pnx;
    dPy = Pny - gs.pny;
    dPz = Pnz - gs.pnz;
    G.P[sel ^ 1][0][cidx] = Pnx;
    G.P[sel ^ 1][1][cidx] = Pny;
    G.P[sel ^ 1][2][cidx] = Pnz;
  }

  enx = eCx + G.cE[clx] * curlx - G.cP[clx] * (dPx + srcx);
  eny = eCy + G.cE[cly] * curly - G.cP[cly] * (dPy + srcy);
  enz = eCz + G.cE[clz] * curlz - G.cP[clz] * (dPz + srcz);
  const bool px = G.per & 1, py = G.per & 2, pz = G.per & 4;
  if ((jw == 0 && !py) || (kw == 0 && !pz)) enx = T(0);
  if ((iw == 0 && !px) || (kw == 0 && !pz)) eny = T(0);
  if ((iw == 0 && !px) || (jw == 0 && !py)) enz = T(0);

  if (GAIN && gcell) {
    const T r = G.q * (T(0.5) * (enx + eCx) * dPx + T(0.5) * (eny + eCy) * dPy + T(0.5) * (enz + eCz) * dPz);
    const T inc1 = G.D[0][0] * gs.d1 + G.D[0][1] * gs.d2 + G.D[0][2] * gs.d3 + G.w[0] * r;
    const T inc2 = G.D[1][0] * gs.d1 + G.D[1][1] * gs.d2 + G.D[1][2] * gs.d3 + G.w[1] * r;
    const T inc3 = G.D[2][0] * gs.d1 + G.D[2][1] * gs.d2 + G.D[2][2] * gs.d3 + G.w[2] * r;
    if (sizeof(T) == 4) {
      // compensated (Kahan) accumulation of the population deviations
      const T y1 = inc1 - gs.c1, y2 = inc2 - gs.c2, y3 = inc3 - gs.c3;
      const T t1 = gs.d1 + y1, t2 = gs.d2 + y2, t3 = gs.d3 + y3;
      G.cmp[0][cidx] = (t1 - gs.d1) - y1;
      G.cmp[1][cidx] = (t2 - gs.d2) - y2;
      G.cmp[2][cidx] = (t3 - gs.d3) - y3;
      G.dN[0][cidx] = t1;
      G.dN[1][cidx] = t2;
      G.dN[2][cidx] = t3;
    } else {
      G.dN[0][cidx] = gs.d1 + inc1;
      G.dN[1][cidx] = gs.d2 + inc2;
      G.dN[2][cidx] = gs.d3 + inc3;
    }
  }
}

}  // namespace fdtd
