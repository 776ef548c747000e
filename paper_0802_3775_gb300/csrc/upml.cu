// Uniaxial PML (the paper's absorbing layer, Sec. "Sample and numerical
// approach"): an alternative to the CPML for passive grids, with the same
// grading of sigma dt/eps0 and kappa (no alpha), evaluated at each field
// node's own position on every axis.
//
// A grid with this absorber takes two launches per time step, one thread per
// node: k_upml_h updates H~, k_upml_e updates E.  A node outside every slab
// takes the plain Yee update (and, for E, the soft sources and the PEC
// holds), exactly as the fused step kernels do; a node where some axis is
// graded steps through an auxiliary field (B~ for H~_c, D~ for E_c), the
// uniaxial tensor diag(s_y s_z/s_x, s_z s_x/s_y, s_x s_y/s_z) split into two
// first-order updates: with (d1, d2) the axes after c in cyclic order and
// s = sigma dt/eps0,
//   D~^{n+1} = u1 D~^n + u2 S curl H~,       u1 = (k1 - s1/2)/(k1 + s1/2), u2 = 1/(k1 + s1/2),
//   E^{n+1} = v1 E^n + v2 D~^{n+1} - v3 D~^n, v1 = (k2 - s2/2)/(k2 + s2/2),
//             v2 = (kc + sc/2)/(k2 + s2/2)/eps_r, v3 = (kc - sc/2)/(k2 + s2/2)/eps_r,
// and H~ likewise with B~, -S curl E and eps_r = 1.  E_c sits at the
// half-integer node along c and at integer nodes along the other axes; H~_c
// the other way round.
#include "cell.cuh"
#include "fdtd_internal.cuh"

namespace fdtd {
namespace {

// neighbour index along axis d, or -1 beyond the edge of a non-periodic axis
template <typename T>
__device__ __forceinline__ int nbr(const StepGrid<T>& G, int d, int v, int s) {
  const int n = d == 0 ? G.nx : (d == 1 ? G.ny : G.nz);
  int w = v + s;
  if (w < 0 || w >= n) {
    if (!((G.per >> d) & 1)) return -1;
    w = (w + n) % n;
  }
  return w;
}

template <typename T>
__device__ __forceinline__ T fld(const T* F, const StepGrid<T>& G, int i, int j, int k) {
  return (i < 0 || j < 0 || k < 0) ? T(0) : F[pidx3(i, j, k, G.px, G.ny)];
}

// the grading of axis d is non-zero at node v (+1/2 when `half`): depth
// below L0 or above n - L1, in integers (v + 1/2 < L0 iff v < L0;
// v + 1/2 > n - L1 iff v >= n - L1)
template <typename T>
__device__ __forceinline__ bool graded(const UpmlDev<T>& u, int d, int n, int v, bool half) {
  const int L0 = u.L[2 * d], L1 = u.L[2 * d + 1];
  return (L0 > 0 && v < L0) || (L1 > 0 && (half ? v >= n - L1 : v > n - L1));
}

template <typename T>
__global__ void __launch_bounds__(256) k_upml_h(const StepGrid<T>* __restrict__ gp, UpmlDev<T> u, int offset) {
  const StepGrid<T>& G = *gp;
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;
  const T* Ex = G.F[fs][0];
  const T* Ey = G.F[fs][1];
  const T* Ez = G.F[fs][2];
  const int nn[3] = {G.nx, G.ny, G.nz};
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i < G.nx && j < G.ny) {
    const int p[3] = {i, j, k};
    const long long o = pidx3(i, j, k, G.px, G.ny);
    const int ip = nbr(G, 0, i, 1), jp = nbr(G, 1, j, 1), kp = nbr(G, 2, k, 1);
    const T ex = Ex[o], ey = Ey[o], ez = Ez[o];
    const T dyEz = fld(Ez, G, i, jp, k) - ez, dzEy = fld(Ey, G, i, j, kp) - ey;
    const T dzEx = fld(Ex, G, i, j, kp) - ex, dxEz = fld(Ez, G, ip, j, k) - ez;
    const T dxEy = fld(Ey, G, ip, j, k) - ey, dyEx = fld(Ex, G, i, jp, k) - ex;
    const T curl[3] = {dyEz - dzEy, dzEx - dxEz, dxEy - dyEx};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T hold = G.F[fs][3 + c][o];
      const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
      // H~_c: integer node along c, half-integer along d1 and d2
      const bool layer = graded(u, c, nn[c], p[c], false) || graded(u, d1, nn[d1], p[d1], true) ||
                         graded(u, d2, nn[d2], p[d2], true);
      T hn;
      if (!layer) {
        hn = fmad(-G.cH, curl[c], hold);
      } else {
        const T u1 = u.q[d1][1][0][p[d1]], u2 = u.q[d1][1][1][p[d1]];
        const T v1 = u.q[d2][1][0][p[d2]], a2 = u.q[d2][1][1][p[d2]];
        const T v2 = u.q[c][0][2][p[c]] * a2, v3 = u.q[c][0][3][p[c]] * a2;
        const T b = u.B[c][o];
        const T t = G.cH * curl[c];
        const T bn = fmad(u1, b, -(u2 * t));
        hn = fmad(v1, hold, fmad(v2, bn, -(v3 * b)));
        u.B[c][o] = bn;
      }
      G.F[fo][3 + c][o] = hn;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_upml_e(const StepGrid<T>* __restrict__ gp, UpmlDev<T> u, int offset) {
  const StepGrid<T>& G = *gp;
  const long long n = G.step + offset;
  if (n >= G.step_end) return;
  __shared__ double sg[kMaxSrc];
  source_waveforms(G, n, threadIdx.y * blockDim.x + threadIdx.x, sg);
  __syncthreads();
  const int fs = (int)(n % G.nsets), fo = fs + 1 == G.nsets ? 0 : fs + 1;
  const T* Hx = G.F[fo][3];
  const T* Hy = G.F[fo][4];
  const T* Hz = G.F[fo][5];
  const int nn[3] = {G.nx, G.ny, G.nz};
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i < G.nx && j < G.ny) {
    const int p[3] = {i, j, k};
    const long long o = pidx3(i, j, k, G.px, G.ny);
    const int im = nbr(G, 0, i, -1), jm = nbr(G, 1, j, -1), km = nbr(G, 2, k, -1);
    const T hx = Hx[o], hy = Hy[o], hz = Hz[o];
    const T dyHz = hz - fld(Hz, G, i, jm, k), dzHy = hy - fld(Hy, G, i, j, km);
    const T dzHx = hx - fld(Hx, G, i, j, km), dxHz = hz - fld(Hz, G, im, j, k);
    const T dxHy = hy - fld(Hy, G, im, j, k), dyHx = hx - fld(Hx, G, i, jm, k);
    const T curl[3] = {dyHz - dzHy, dzHx - dxHz, dxHy - dyHx};
    Column col;
    make_column(G, i, j, col, true);
    const Plane pl = make_plane(G, k);
    T src[3] = {T(0), T(0), T(0)};
    if (col.src) source_drive(G, sg, col, pl, src[0], src[1], src[2]);
    const unsigned m = G.mat[o];
    const bool pec[3] = {col.pecy || pl.pecz, col.pecx || pl.pecz, col.pecx || col.pecy};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T eold = G.F[fs][c][o];
      const int cl = (m >> (2 * c)) & 3;
      const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
      // E_c: half-integer node along c, integer along d1 and d2
      const bool layer = graded(u, c, nn[c], p[c], true) || graded(u, d1, nn[d1], p[d1], false) ||
                         graded(u, d2, nn[d2], p[d2], false);
      T en;
      if (!layer) {
        en = fmad(-G.cP[cl], src[c], fmad(G.cE[cl], curl[c], eold));
      } else {
        const T u1 = u.q[d1][0][0][p[d1]], u2 = u.q[d1][0][1][p[d1]];
        const T v1 = u.q[d2][0][0][p[d2]], a2 = u.q[d2][0][1][p[d2]];
        const T v2 = u.q[c][1][2][p[c]] * a2 * G.cP[cl], v3 = u.q[c][1][3][p[c]] * a2 * G.cP[cl];
        const T d = u.D[c][o];
        const T t = G.cH * curl[c];
        const T dn = fmad(u1, d, u2 * t);
        en = fmad(v1, eold, fmad(v2, dn, -(v3 * d)));
        u.D[c][o] = dn;
      }
      if (pec[c]) en = T(0);
      G.F[fo][c][o] = en;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_upml(const StepGrid<T>* g, const UpmlDev<T>& u, int nx, int ny, int nz, int offset,
                        cudaStream_t st) {
  // one thread per node: blocks of 32 x 8 nodes of one plane
  const dim3 block(32, 8, 1), grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), (unsigned)nz);
  k_upml_h<T><<<grid, block, 0, st>>>(g, u, offset);
  k_upml_e<T><<<grid, block, 0, st>>>(g, u, offset);
  return cudaGetLastError();
}

template cudaError_t launch_upml<float>(const StepGrid<float>*, const UpmlDev<float>&, int, int, int, int,
                                        cudaStream_t);
template cudaError_t launch_upml<double>(const StepGrid<double>*, const UpmlDev<double>&, int, int, int, int,
                                         cudaStream_t);

}  // namespace fdtd
