// Device kernels of the GB300 Maxwell-Bloch FDTD library (sm_103a).
//
// k_step      one time step n -> n+1 of a set of work items (x-y tile x
//             z-range of some grid): H half step with CPML, polarization,
//             E step with CPML, source and gain current, populations, noise.
//             The tile marches in z with the E planes of the tile (plus a
//             one-node halo) staged in shared memory; H on the -x / -y halo is
//             recomputed so that no block needs a neighbour's output of the
//             same step.  Fields and H-side CPML memory are double-buffered
//             (read set n&1, write set (n+1)&1); E-side CPML memory and the
//             gain state are updated in place by the owning thread.
// k_observe   probes (E^{n+1}) and Poynting flux T^n per plane with a
//             fixed-order FP64 reduction (bitwise reproducible).
// k_energy    field energy in FP64, fixed-order reduction.
// k_rasterize sphere list -> material bytes (FP64, no contraction).
//
// Paper: Yee FDTD (Sec. "Sample and numerical approach"), four-level
// Maxwell-Bloch gain solved at the Yee cell (same section), noise as a
// stochastic source (same section), pulsed sources and flux T(t) (Secs.
// "Wide-band excitation", "Dynamical diffusion").
#include <math.h>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ long long lidx(int i, int j, int k, int nx, int ny) {
  return ((long long)k * ny + j) * nx + i;
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

// Three N(0,1) deviates for (seed, cell, step): Box-Muller on the uniforms
// u = ((x >> 9) + 0.5) 2^-23 (exact in binary32).
__device__ __forceinline__ void gain_normals(unsigned long long seed, long long cell, long long step, float& a,
                                             float& b, float& c) {
  const uint4 x = philox4x32_10(
      make_uint4((unsigned)cell, (unsigned)((unsigned long long)cell >> 32), (unsigned)step,
                 (unsigned)((unsigned long long)step >> 32)),
      make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
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
  const uint4 x = philox4x32_10(
      make_uint4((unsigned)cell, (unsigned)((unsigned long long)cell >> 32), (unsigned)step,
                 (unsigned)((unsigned long long)step >> 32)),
      make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
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
                                      long long pidx) {
  const T p = pr[1][pos] * psi_in[pidx] + pr[2][pos] * D;
  if (psi_out) psi_out[pidx] = p;
  return pr[0][pos] * D + p;
}

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

template <typename T>
size_t step_smem_bytes(int bx, int by) {
  const size_t gs = (sizeof(StepGrid<T>) + 15) & ~size_t(15);
  const size_t planes = (size_t)3 * (bx + 1) * (by + 1) + (size_t)3 * bx * by;
  return gs + kMaxSrc * sizeof(double) + planes * sizeof(T);
}

template <typename T, bool GAIN>
__global__ void __launch_bounds__(512) k_step(const StepGrid<T>* __restrict__ grids, const int4* __restrict__ items,
                                              int nitems, int offset) {
  extern __shared__ __align__(16) unsigned char smem[];
  StepGrid<T>& G = *reinterpret_cast<StepGrid<T>*>(smem);
  constexpr size_t GS = (sizeof(StepGrid<T>) + 15) & ~size_t(15);
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
      const int* src = reinterpret_cast<const int*>(grids + item.x);
      int* dst = reinterpret_cast<int*>(smem);
      for (int w = tid; w < (int)(sizeof(StepGrid<T>) / 4); w += bx * by) dst[w] = src[w];
      cur = item.x;
    }
    __syncthreads();
    const long long n = G.step + offset;
    if (n >= G.step_end) continue;
    if (tid < G.nsrc) {
      const SrcDev& s = G.src[tid];
      const double t = (double)n + 0.5 - s.t0;
      sg[tid] = exp(-t * t / (2.0 * s.tau * s.tau)) * sin(2.0 * 3.14159265358979323846 * s.f0dt * t);
    }
    __syncthreads();

    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const bool px = G.per & 1, py = G.per & 2, pz = G.per & 4;
    const int x0 = item.y, y0 = item.z, z0 = item.w & 0xffff, z1 = (item.w >> 16) & 0xffff;
    const int i = x0 - 1 + tx, j = y0 - 1 + ty;
    bool vx, vy, vxp, vyp;
    const int iw = wrap_index(i, nx, px, vx);
    const int jw = wrap_index(j, ny, py, vy);
    const bool valid = vx && vy;
    const bool xcol = (tx == bx - 1), yrow = (ty == by - 1);
    const int ip = wrap_index(i + 1, nx, px, vxp);
    const int jp = wrap_index(j + 1, ny, py, vyp);
    const bool vcol = xcol && vxp && vy;   // extra column node (i+1, j) exists
    const bool vrow = yrow && vx && vyp;   // extra row node (i, j+1) exists
    const bool owner = tx > 0 && ty > 0 && i < nx && j < ny;

    const int sel = (int)(n & 1);
    const T* __restrict__ Ex = G.F[sel][0];
    const T* __restrict__ Ey = G.F[sel][1];
    const T* __restrict__ Ez = G.F[sel][2];
    const T* __restrict__ Hx = G.F[sel][3];
    const T* __restrict__ Hy = G.F[sel][4];
    const T* __restrict__ Hz = G.F[sel][5];

    // CPML slab coordinates of this column
    int sx = -1, sy = -1;
    if (valid && G.Sd[0]) {
      if (iw < G.L[0]) sx = iw;
      else if (iw >= nx - G.L[1]) sx = G.L[0] + iw - (nx - G.L[1]);
    }
    if (valid && G.Sd[1]) {
      if (jw < G.L[2]) sy = jw;
      else if (jw >= ny - G.L[3]) sy = G.L[2] + jw - (ny - G.L[3]);
    }

    auto kwrap = [&](int k, bool& v) { return wrap_index(k, nz, pz, v); };

    const int kstart = (z0 > 0 || pz) ? z0 - 1 : z0;
    bool vk0, vk1;
    const int kw0 = kwrap(kstart, vk0);
    const int kw1 = kwrap(kstart + 1, vk1);
    const long long c0 = lidx(iw, jw, kw0, nx, ny);
    const long long c1 = lidx(iw, jw, kw1, nx, ny);
    T eCx = ldz(Ex, valid && vk0, c0), eCy = ldz(Ey, valid && vk0, c0), eCz = ldz(Ez, valid && vk0, c0);
    T eNx = ldz(Ex, valid && vk1, c1), eNy = ldz(Ey, valid && vk1, c1), eNz = ldz(Ez, valid && vk1, c1);
    T hOx = ldz(Hx, valid && vk0, c0), hOy = ldz(Hy, valid && vk0, c0), hOz = ldz(Hz, valid && vk0, c0);
    T xCy = T(0), xCz = T(0), yCx = T(0), yCz = T(0);
    {
      const long long cc = lidx(ip, jw, kw0, nx, ny);
      const long long cr = lidx(iw, jp, kw0, nx, ny);
      xCy = ldz(Ey, vcol && vk0, cc);
      xCz = ldz(Ez, vcol && vk0, cc);
      yCx = ldz(Ex, vrow && vk0, cr);
      yCz = ldz(Ez, vrow && vk0, cr);
    }
    T hPx = T(0), hPy = T(0);

    for (int k = kstart; k < z1; ++k) {
      bool vk;
      const int kw = kwrap(k, vk);
      const bool active = k >= z0;
      // prefetch the next plane
      T eNNx = T(0), eNNy = T(0), eNNz = T(0), hONx = T(0), hONy = T(0), hONz = T(0);
      T xNy = T(0), xNz = T(0), yNx = T(0), yNz = T(0);
      if (k + 1 < z1) {
        bool va, vb;
        const int ka = kwrap(k + 1, va);
        const int kb = kwrap(k + 2, vb);
        const long long ca = lidx(iw, jw, ka, nx, ny);
        const long long cb = lidx(iw, jw, kb, nx, ny);
        eNNx = ldz(Ex, valid && vb, cb);
        eNNy = ldz(Ey, valid && vb, cb);
        eNNz = ldz(Ez, valid && vb, cb);
        hONx = ldz(Hx, valid && va, ca);
        hONy = ldz(Hy, valid && va, ca);
        hONz = ldz(Hz, valid && va, ca);
        const long long cc = lidx(ip, jw, ka, nx, ny);
        const long long cr = lidx(iw, jp, ka, nx, ny);
        xNy = ldz(Ey, vcol && va, cc);
        xNz = ldz(Ez, vcol && va, cc);
        yNx = ldz(Ex, vrow && va, cr);
        yNz = ldz(Ez, vrow && va, cr);
      }
      // owner loads for the E update of this plane
      const long long cidx = lidx(iw, jw, kw, nx, ny);
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

      // H^{n+1/2} at this node
      T hx = T(0), hy = T(0), hz = T(0);
      if (valid && vk) {
        T dyEz = sEz[se + EW] - eCz;
        T dzEy = eNy - eCy;
        T dzEx = eNx - eCx;
        T dxEz = sEz[se + 1] - eCz;
        T dxEy = sEy[se + 1] - eCy;
        T dyEx = sEx[se + EW] - eCx;
        const bool wr = owner && active;
        if (sx >= 0) {
          const long long pi = ((long long)kw * ny + jw) * G.Sd[0] + sx;
          dxEz = pml_term(dxEz, G.prof[0][1], iw, G.psiH[sel][0][0], wr ? G.psiH[sel ^ 1][0][0] : (T*)nullptr, pi);
          dxEy = pml_term(dxEy, G.prof[0][1], iw, G.psiH[sel][0][1], wr ? G.psiH[sel ^ 1][0][1] : (T*)nullptr, pi);
        }
        if (sy >= 0) {
          const long long pi = ((long long)kw * G.Sd[1] + sy) * nx + iw;
          dyEx = pml_term(dyEx, G.prof[1][1], jw, G.psiH[sel][1][0], wr ? G.psiH[sel ^ 1][1][0] : (T*)nullptr, pi);
          dyEz = pml_term(dyEz, G.prof[1][1], jw, G.psiH[sel][1][1], wr ? G.psiH[sel ^ 1][1][1] : (T*)nullptr, pi);
        }
        if (G.Sd[2]) {
          int sz = -1;
          if (kw < G.L[4]) sz = kw;
          else if (kw >= nz - G.L[5]) sz = G.L[4] + kw - (nz - G.L[5]);
          if (sz >= 0) {
            const long long pi = ((long long)sz * ny + jw) * nx + iw;
            dzEy = pml_term(dzEy, G.prof[2][1], kw, G.psiH[sel][2][0], wr ? G.psiH[sel ^ 1][2][0] : (T*)nullptr, pi);
            dzEx = pml_term(dzEx, G.prof[2][1], kw, G.psiH[sel][2][1], wr ? G.psiH[sel ^ 1][2][1] : (T*)nullptr, pi);
          }
        }
        hx = hOx - G.cH * (dyEz - dzEy);
        hy = hOy - G.cH * (dzEx - dxEz);
        hz = hOz - G.cH * (dxEy - dyEx);
      }
      sHx[tid] = hx;
      sHy[tid] = hy;
      sHz[tid] = hz;
      __syncthreads();

      if (owner && active) {
        T dyHz = hz - sHz[tid - bx];
        T dzHy = hy - hPy;
        T dzHx = hx - hPx;
        T dxHz = hz - sHz[tid - 1];
        T dxHy = hy - sHy[tid - 1];
        T dyHx = hx - sHx[tid - bx];
        if (sx >= 0) {
          const long long pi = ((long long)kw * ny + jw) * G.Sd[0] + sx;
          dxHz = pml_term(dxHz, G.prof[0][0], iw, G.psiE[0][0], G.psiE[0][0], pi);
          dxHy = pml_term(dxHy, G.prof[0][0], iw, G.psiE[0][1], G.psiE[0][1], pi);
        }
        if (sy >= 0) {
          const long long pi = ((long long)kw * G.Sd[1] + sy) * nx + iw;
          dyHx = pml_term(dyHx, G.prof[1][0], jw, G.psiE[1][0], G.psiE[1][0], pi);
          dyHz = pml_term(dyHz, G.prof[1][0], jw, G.psiE[1][1], G.psiE[1][1], pi);
        }
        if (G.Sd[2]) {
          int sz = -1;
          if (kw < G.L[4]) sz = kw;
          else if (kw >= nz - G.L[5]) sz = G.L[4] + kw - (nz - G.L[5]);
          if (sz >= 0) {
            const long long pi = ((long long)sz * ny + jw) * nx + iw;
            dzHy = pml_term(dzHy, G.prof[2][0], kw, G.psiE[2][0], G.psiE[2][0], pi);
            dzHx = pml_term(dzHx, G.prof[2][0], kw, G.psiE[2][1], G.psiE[2][1], pi);
          }
        }
        const T curlx = dyHz - dzHy;
        const T curly = dzHx - dxHz;
        const T curlz = dxHy - dyHx;
        const int clx = m & 3, cly = (m >> 2) & 3, clz = (m >> 4) & 3;

        // soft sources
        T sx_ = T(0), sy_ = T(0), sz_ = T(0);
        for (int s = 0; s < G.nsrc; ++s) {
          const SrcDev& S = G.src[s];
          double w = 0.0;
          if (S.kind == 0) {
            if (iw == S.i && jw == S.j && kw == S.k) w = S.amp;
          } else {
            const int crd[3] = {iw, jw, kw};
            if (crd[S.axis] == S.index) {
              const int u = crd[(S.axis + 1) % 3], v = crd[(S.axis + 2) % 3];
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
            if (S.comp == 0) sx_ += val;
            else if (S.comp == 1) sy_ += val;
            else sz_ += val;
          }
        }

        T dPx = T(0), dPy = T(0), dPz = T(0);
        T Pnx = T(0), Pny = T(0), Pnz = T(0);
        bool gcell = false;
        if (GAIN) gcell = G.gain && ((m >> 6) & 1);
        T d1 = T(0), d2 = T(0), d3 = T(0);
        if (GAIN && gcell) {
          const T* __restrict__ P0x = G.P[sel][0];
          const T* __restrict__ P0y = G.P[sel][1];
          const T* __restrict__ P0z = G.P[sel][2];
          T* __restrict__ P1x = G.P[sel ^ 1][0];
          T* __restrict__ P1y = G.P[sel ^ 1][1];
          T* __restrict__ P1z = G.P[sel ^ 1][2];
          const T pnx = P0x[cidx], pny = P0y[cidx], pnz = P0z[cidx];
          const T pmx = P1x[cidx], pmy = P1y[cidx], pmz = P1z[cidx];
          d1 = G.dN[0][cidx];
          d2 = G.dN[1][cidx];
          d3 = G.dN[2][cidx];
          const T dn12 = G.n12eq + (d1 - d2);
          const T drive = G.a3 * dn12;
          Pnx = G.a1 * pnx - G.a2 * pmx + drive * eCx;
          Pny = G.a1 * pny - G.a2 * pmy + drive * eCy;
          Pnz = G.a1 * pnz - G.a2 * pmz + drive * eCz;
          if (G.noise != T(0)) {
            T xa, xb, xc;
            gain_normals(G.seed, cidx, n, xa, xb, xc);
            Pnx += G.noise * xa;
            Pny += G.noise * xb;
            Pnz += G.noise * xc;
          }
          dPx = Pnx - pnx;
          dPy = Pny - pny;
          dPz = Pnz - pnz;
          P1x[cidx] = Pnx;
          P1y[cidx] = Pny;
          P1z[cidx] = Pnz;
        }

        T enx = eCx + G.cE[clx] * curlx - G.cP[clx] * (dPx + sx_);
        T eny = eCy + G.cE[cly] * curly - G.cP[cly] * (dPy + sy_);
        T enz = eCz + G.cE[clz] * curlz - G.cP[clz] * (dPz + sz_);
        // tangential E held at zero on the index-0 plane of non-periodic axes
        if ((jw == 0 && !py) || (kw == 0 && !pz)) enx = T(0);
        if ((iw == 0 && !px) || (kw == 0 && !pz)) eny = T(0);
        if ((iw == 0 && !px) || (jw == 0 && !py)) enz = T(0);

        if (GAIN && gcell) {
          const T r = G.q * (T(0.5) * (enx + eCx) * dPx + T(0.5) * (eny + eCy) * dPy + T(0.5) * (enz + eCz) * dPz);
          const T inc1 = G.D[0][0] * d1 + G.D[0][1] * d2 + G.D[0][2] * d3 + G.w[0] * r;
          const T inc2 = G.D[1][0] * d1 + G.D[1][1] * d2 + G.D[1][2] * d3 + G.w[1] * r;
          const T inc3 = G.D[2][0] * d1 + G.D[2][1] * d2 + G.D[2][2] * d3 + G.w[2] * r;
          if (sizeof(T) == 4) {
            // compensated (Kahan) accumulation of the population deviations
            T c1 = G.cmp[0][cidx], c2 = G.cmp[1][cidx], c3 = G.cmp[2][cidx];
            const T y1 = inc1 - c1, y2 = inc2 - c2, y3 = inc3 - c3;
            const T t1 = d1 + y1, t2 = d2 + y2, t3 = d3 + y3;
            G.cmp[0][cidx] = (t1 - d1) - y1;
            G.cmp[1][cidx] = (t2 - d2) - y2;
            G.cmp[2][cidx] = (t3 - d3) - y3;
            G.dN[0][cidx] = t1;
            G.dN[1][cidx] = t2;
            G.dN[2][cidx] = t3;
          } else {
            G.dN[0][cidx] = d1 + inc1;
            G.dN[1][cidx] = d2 + inc2;
            G.dN[2][cidx] = d3 + inc3;
          }
        }

        G.F[sel ^ 1][0][cidx] = enx;
        G.F[sel ^ 1][1][cidx] = eny;
        G.F[sel ^ 1][2][cidx] = enz;
        G.F[sel ^ 1][3][cidx] = hx;
        G.F[sel ^ 1][4][cidx] = hy;
        G.F[sel ^ 1][5][cidx] = hz;
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

// ---------------------------------------------------------------- observers
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
  const int4 it = items[blockIdx.x];
  const ObsGrid<T>& G = grids[it.x];
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int sel = (int)(n & 1);
  const int nx = G.nx, ny = G.ny;
  const long long slot = n % G.cap;
  if (it.y < 0) {
    for (int q = threadIdx.x; q < G.nprobe * 3; q += blockDim.x) {
      const int p = q / 3, c = q % 3;
      const T v = G.F[sel ^ 1][c][lidx(G.probe[p][0], G.probe[p][1], G.probe[p][2], nx, ny)];
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
  const T* E1 = G.F[sel][d1];
  const T* E2 = G.F[sel][d2];
  const T* H1a = G.F[sel][3 + d1];
  const T* H1b = G.F[sel ^ 1][3 + d1];
  const T* H2a = G.F[sel][3 + d2];
  const T* H2b = G.F[sel ^ 1][3 + d2];
  double acc = 0.0;
  for (long long q = beg + threadIdx.x; q < end; q += blockDim.x) {
    const int u = u0 + (int)(q / nv), v = v0 + (int)(q % nv);
    int c[3];
    auto at = [&](int pp, int uu, int vv) {
      c[d] = pp;
      c[d1] = uu;
      c[d2] = vv;
      return lidx(c[0], c[1], c[2], nx, ny);
    };
    const long long a = at(p, u, v), av = at(p, u, v + 1), au = at(p, u + 1, v);
    const long long b = at(p - 1, u, v), bv = at(p - 1, u, v + 1), bu = at(p - 1, u + 1, v);
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
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    const volatile double* pp = G.partials + f * kMaxFluxParts;
    for (int q = 0; q < nparts; ++q) tot += pp[q];
    const double T_n = G.flux_sign[f] * G.dx2_over_eta0 * tot;
    G.flux_ring[slot * G.nflux + f] = T_n;
    if (!isfinite(T_n)) atomicOr(G.err, 1);
    G.counters[f] = 0u;
  }
}

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

// ---------------------------------------------------------------- energy
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

// ---------------------------------------------------------------- rasterizer
__global__ void k_rasterize(uint8_t* __restrict__ mat, int nx, int ny, int nz, const double* __restrict__ sph,
                            const int* __restrict__ bstart, const int* __restrict__ blist, int bin, int bnx, int bny,
                            int bnz, double lo0, double lo1, double lo2, double hi0, double hi1, double hi2) {
  const long long ncell = (long long)nx * ny * nz;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int i = (int)(c % nx);
  const int j = (int)((c / nx) % ny);
  const int k = (int)(c / ((long long)nx * ny));
  const int b = ((k / bin) * bny + (j / bin)) * bnx + (i / bin);
  const double px[4] = {i + 0.5, (double)i, (double)i, i + 0.5};
  const double py[4] = {(double)j, j + 0.5, (double)j, j + 0.5};
  const double pz[4] = {(double)k, (double)k, k + 0.5, k + 0.5};
  bool ins[4] = {false, false, false, false};
  for (int q = bstart[b]; q < bstart[b + 1]; ++q) {
    const int s = blist[q];
    const double cx = sph[4 * s], cy = sph[4 * s + 1], cz = sph[4 * s + 2], r = sph[4 * s + 3];
    const double rr = __dmul_rn(r, r);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double dx = __dsub_rn(px[t], cx), dy = __dsub_rn(py[t], cy), dz = __dsub_rn(pz[t], cz);
      const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      ins[t] = ins[t] || (d2 < rr);
    }
  }
  unsigned byte = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const bool inbox = px[t] >= lo0 && px[t] < hi0 && py[t] >= lo1 && py[t] < hi1 && pz[t] >= lo2 && pz[t] < hi2;
    if (t < 3) byte |= (inbox ? (ins[t] ? 2u : 1u) : 0u) << (2 * t);
    else if (inbox && ins[t]) byte |= 64u;
  }
  mat[c] = (uint8_t)byte;
  (void)bnz;
}

cudaError_t launch_rasterize(uint8_t* mat, int nx, int ny, int nz, const double* spheres, const int* bin_start,
                             const int* bin_list, int bin, int bnx, int bny, int bnz, const double* box,
                             cudaStream_t st) {
  const long long ncell = (long long)nx * ny * nz;
  const int threads = 256;
  const long long blocks = (ncell + threads - 1) / threads;
  k_rasterize<<<(unsigned)blocks, threads, 0, st>>>(mat, nx, ny, nz, spheres, bin_start, bin_list, bin, bnx, bny,
                                                     bnz, box[0], box[1], box[2], box[3], box[4], box[5]);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gain init
template <typename T>
__global__ void k_gain_init(StepGrid<T> G, long long ncell, T d1, T d2, T d3) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const bool g = (G.mat[c] >> 6) & 1;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 3; ++q) G.P[s][q][c] = T(0);
  G.dN[0][c] = g ? d1 : T(0);
  G.dN[1][c] = g ? d2 : T(0);
  G.dN[2][c] = g ? d3 : T(0);
  if (G.cmp[0]) {
    G.cmp[0][c] = T(0);
    G.cmp[1][c] = T(0);
    G.cmp[2][c] = T(0);
  }
}

template <typename T>
cudaError_t launch_gain_init(const StepGrid<T>* g, long long ncell, T d1, T d2, T d3, cudaStream_t st) {
  k_gain_init<T><<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(*g, ncell, d1, d2, d3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- conversions
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

// ---------------------------------------------------------------- instantiations
#define FDTD_INST(T)                                                                                          \
  template size_t step_smem_bytes<T>(int, int);                                                               \
  template cudaError_t launch_step<T>(const StepGrid<T>*, const int4*, int, int, int, int, bool, int,        \
                                      cudaStream_t);                                                          \
  template cudaError_t launch_observe<T>(const ObsGrid<T>*, const int4*, int, int, cudaStream_t);            \
  template cudaError_t launch_advance<T>(StepGrid<T>*, ObsGrid<T>*, int, int, cudaStream_t);                 \
  template cudaError_t launch_gain_init<T>(const StepGrid<T>*, long long, T, T, T, cudaStream_t);            \
  template cudaError_t launch_energy<T>(const T* const*, const uint8_t*, double, double, double, long long,  \
                                        double*, unsigned int*, double*, int*, cudaStream_t);                \
  template cudaError_t launch_to_double<T>(const T*, double*, long long, cudaStream_t);                      \
  template cudaError_t launch_from_double<T>(const double*, T*, long long, cudaStream_t);

FDTD_INST(float)
FDTD_INST(double)

}  // namespace fdtd
