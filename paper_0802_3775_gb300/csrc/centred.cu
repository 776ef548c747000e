// Centred Bloch coupling: the polarization and the populations of a gain cell
// sit at the cell centre (the paper solves the Bloch variables in the middle
// of the Yee cell, Sec. "Sample and numerical approach").
//
// A grid with this coupling steps its fields with a passive step kernel
// (CPML, sources, PEC holds; no polarization current), then per time step n:
//   1. k_centred_polarize: every gain cell drives its oscillator with the
//      centre average E_bar^n = A E^n of the four edges of each E component
//      (for E_c with (d1, d2) the other axes in cyclic order,
//      1/4 ((E + E[+d1]) + (E[+d2] + E[+d1+d2])), beyond the grid 0 or the
//      periodic wrap) and writes P~^{n+1} into the slot of P~^{n-1};
//   2. k_centred_current: every E node not held by a PEC wall receives the
//      polarization current of the four cells sharing it,
//      E^{n+1} -= (1/eps_r) A^T dP~ with A^T dP~ = 1/4 ((dP + dP[-d1]) +
//      (dP[-d2] + dP[-d1-d2])) and dP~ = P~^{n+1} - P~^n in gain cells;
//   3. k_centred_populations: every gain cell updates its population
//      deviations with r = q sum_c A((E^{n+1} + E^n)/2)_c dP~_c (the adjoint of
//      step 2's interpolation, so the field-medium exchange balances), Kahan
//      compensated in binary32 like the cell coupling.
// The oscillator, noise, rate-matrix and compensation arithmetic is that of
// the cell coupling (cell.cuh), in the same operation order.
#include "cell.cuh"
#include "fdtd_internal.cuh"

namespace fdtd {
namespace {

template <typename T>
struct CentredCtx {
  const StepGrid<T>& G;
  long long n;
  int fs, fo;  // field sets holding E^n and receiving E^{n+1}
};

// Neighbour index along axis d (offset s = +1 / -1) of (i, j, k), or -1
// outside the grid of a non-periodic axis.
template <typename T>
__device__ __forceinline__ int nb(const StepGrid<T>& G, int d, int v, int s) {
  const int n = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
  int w = v + s;
  if (w < 0 || w >= n) {
    if (!((G.per >> d) & 1)) return -1;
    w = (w + n) % n;
  }
  return w;
}

template <typename T>
__device__ __forceinline__ T at(const T* F, const StepGrid<T>& G, int i, int j, int k) {
  return (i < 0 || j < 0 || k < 0) ? T(0) : F[pidx3(i, j, k, G.px, G.ny)];
}

// Centre average of component c of field array F at cell (i, j, k).
template <typename T>
__device__ __forceinline__ T centre_avg(const StepGrid<T>& G, const T* F, int c, int i, int j, int k) {
  const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
  int p[3] = {i, j, k};
  int q1[3] = {i, j, k}, q2[3] = {i, j, k}, q12[3] = {i, j, k};
  q1[d1] = nb(G, d1, p[d1], +1);
  q2[d2] = nb(G, d2, p[d2], +1);
  q12[d1] = q1[d1];
  q12[d2] = q2[d2];
  const T a = at(F, G, p[0], p[1], p[2]), b = at(F, G, q1[0], q1[1], q1[2]);
  const T c2 = at(F, G, q2[0], q2[1], q2[2]), d = at(F, G, q12[0], q12[1], q12[2]);
  return T(0.25) * ((a + b) + (c2 + d));
}

// Centre average of (E^{n+1} + E^n)/2, each edge averaged in time first.
template <typename T>
__device__ __forceinline__ T centre_avg_half(const StepGrid<T>& G, const T* Fo, const T* Fn, int c, int i, int j,
                                             int k) {
  const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
  int q[4][3] = {{i, j, k}, {i, j, k}, {i, j, k}, {i, j, k}};
  const int u = nb(G, d1, q[0][d1], +1), v = nb(G, d2, q[0][d2], +1);
  q[1][d1] = u;
  q[2][d2] = v;
  q[3][d1] = u;
  q[3][d2] = v;
  T h[4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
    h[e] = T(0.5) * (at(Fo, G, q[e][0], q[e][1], q[e][2]) + at(Fn, G, q[e][0], q[e][1], q[e][2]));
  return T(0.25) * ((h[0] + h[1]) + (h[2] + h[3]));
}

template <typename T>
__device__ __forceinline__ bool gain_cell(const StepGrid<T>& G, int i, int j, int k) {
  return (G.mat[pidx3(i, j, k, G.px, G.ny)] >> 6) & 1;
}

template <typename T>
__global__ void __launch_bounds__(256) k_centred_polarize(const StepGrid<T>* __restrict__ gp, int offset) {
  const StepGrid<T>& G = *gp;
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int fs = (int)(n % G.nsets);
  const int sel = (int)(n & 1);
  using W = GainWords<T>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i < G.nx && j < G.ny) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    if (!gain_cell(G, i, j, k)) return;
    T* g = G.gst + gain_base(G, i, j, k);
    const T* pn = g + 32 * (sel ? W::P1 : W::P0);
    T* pm = g + 32 * (sel ? W::P0 : W::P1);  // P~^{n-1}, receives P~^{n+1}
    const T ex = centre_avg(G, G.F[fs][0], 0, i, j, k);
    const T ey = centre_avg(G, G.F[fs][1], 1, i, j, k);
    const T ez = centre_avg(G, G.F[fs][2], 2, i, j, k);
    const T dn12 = G.n12eq + (g[32 * W::DN] - g[32 * W::DN + 32]);
    const T drive = G.a3 * dn12;
    T Px = fmad(drive, ex, fmad(G.a1, pn[0], -(G.a2 * pm[0])));
    T Py = fmad(drive, ey, fmad(G.a1, pn[32], -(G.a2 * pm[32])));
    T Pz = fmad(drive, ez, fmad(G.a1, pn[64], -(G.a2 * pm[64])));
    if (G.noise != T(0)) {
      T xa, xb, xc;
      gain_normals(G.seed, c, n, xa, xb, xc);
      Px = fmad(G.noise, xa, Px);
      Py = fmad(G.noise, xb, Py);
      Pz = fmad(G.noise, xc, Pz);
    }
    pm[0] = Px;
    pm[32] = Py;
    pm[64] = Pz;
  }
}

// dP~_c = P~^{n+1} - P~^n of cell (i, j, k) (0 outside the grid and in cells without gain).
template <typename T>
__device__ __forceinline__ T cell_dP(const StepGrid<T>& G, int sel, int c, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || !gain_cell(G, i, j, k)) return T(0);
  using W = GainWords<T>;
  const T* g = G.gst + gain_base(G, i, j, k);
  return g[32 * ((sel ? W::P0 : W::P1) + c)] - g[32 * ((sel ? W::P1 : W::P0) + c)];
}

template <typename T>
__global__ void __launch_bounds__(256) k_centred_current(const StepGrid<T>* __restrict__ gp, int offset) {
  const StepGrid<T>& G = *gp;
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;
  const int sel = (int)(n & 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i < G.nx && j < G.ny) {
    const long long o = pidx3(i, j, k, G.px, G.ny);
    const unsigned m = G.mat[o];
    const int p[3] = {i, j, k};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
      // tangential E held at zero on the index-0 planes of non-periodic axes
      if ((p[d1] == 0 && !((G.per >> d1) & 1)) || (p[d2] == 0 && !((G.per >> d2) & 1))) continue;
      int q1[3] = {i, j, k}, q2[3] = {i, j, k}, q12[3] = {i, j, k};
      q1[d1] = nb(G, d1, p[d1], -1);
      q2[d2] = nb(G, d2, p[d2], -1);
      q12[d1] = q1[d1];
      q12[d2] = q2[d2];
      const T a = cell_dP(G, sel, c, i, j, k), b = cell_dP(G, sel, c, q1[0], q1[1], q1[2]);
      const T c2 = cell_dP(G, sel, c, q2[0], q2[1], q2[2]), d = cell_dP(G, sel, c, q12[0], q12[1], q12[2]);
      if (a == T(0) && b == T(0) && c2 == T(0) && d == T(0)) continue;  // next component
      const T dPe = T(0.25) * ((a + b) + (c2 + d));
      T* E = G.F[fo][c];
      E[o] = fmad(-G.cP[(m >> (2 * c)) & 3], dPe, E[o]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_centred_populations(const StepGrid<T>* __restrict__ gp, int offset) {
  const StepGrid<T>& G = *gp;
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;
  const int sel = (int)(n & 1);
  using W = GainWords<T>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i < G.nx && j < G.ny) {
    const long long c = ((long long)k * G.ny + j) * G.nx + i;
    if (!gain_cell(G, i, j, k)) return;
    T* g = G.gst + gain_base(G, i, j, k);
    const T* pnew = g + 32 * (sel ? W::P0 : W::P1);
    const T* pold = g + 32 * (sel ? W::P1 : W::P0);
    const T dPx = pnew[0] - pold[0], dPy = pnew[32] - pold[32], dPz = pnew[64] - pold[64];
    const T hx_ = centre_avg_half(G, G.F[fo][0], G.F[fs][0], 0, i, j, k);
    const T hy_ = centre_avg_half(G, G.F[fo][1], G.F[fs][1], 1, i, j, k);
    const T hz_ = centre_avg_half(G, G.F[fo][2], G.F[fs][2], 2, i, j, k);
    const T r = G.q * fmad(hz_, dPz, fmad(hy_, dPy, hx_ * dPx));
    const T d1 = g[32 * W::DN], d2 = g[32 * W::DN + 32], d3 = g[32 * W::DN + 64];
    const T inc1 = fmad(G.w[0], r, fmad(G.D[0][2], d3, fmad(G.D[0][1], d2, G.D[0][0] * d1)));
    const T inc2 = fmad(G.w[1], r, fmad(G.D[1][2], d3, fmad(G.D[1][1], d2, G.D[1][0] * d1)));
    const T inc3 = fmad(G.w[2], r, fmad(G.D[2][2], d3, fmad(G.D[2][1], d2, G.D[2][0] * d1)));
    if (sizeof(T) == 4) {
      // compensated (Kahan) accumulation of the population deviations
      const T y1 = inc1 - g[32 * W::CMP], y2 = inc2 - g[32 * W::CMP + 32], y3 = inc3 - g[32 * W::CMP + 64];
      const T t1 = d1 + y1, t2 = d2 + y2, t3 = d3 + y3;
      g[32 * W::CMP] = (t1 - d1) - y1;
      g[32 * W::CMP + 32] = (t2 - d2) - y2;
      g[32 * W::CMP + 64] = (t3 - d3) - y3;
      g[32 * W::DN] = t1;
      g[32 * W::DN + 32] = t2;
      g[32 * W::DN + 64] = t3;
    } else {
      g[32 * W::DN] = d1 + inc1;
      g[32 * W::DN + 32] = d2 + inc2;
      g[32 * W::DN + 64] = d3 + inc3;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_centred(const StepGrid<T>* g, int nx, int ny, int nz, int offset, cudaStream_t st) {
  // one thread per cell (node): blocks of 32 x 8 of one plane
  const dim3 block(32, 8, 1), grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), (unsigned)nz);
  k_centred_polarize<T><<<grid, block, 0, st>>>(g, offset);
  k_centred_current<T><<<grid, block, 0, st>>>(g, offset);
  k_centred_populations<T><<<grid, block, 0, st>>>(g, offset);
  return cudaGetLastError();
}

template cudaError_t launch_centred<float>(const StepGrid<float>*, int, int, int, int, cudaStream_t);
template cudaError_t launch_centred<double>(const StepGrid<double>*, int, int, int, int, cudaStream_t);

}  // namespace fdtd
