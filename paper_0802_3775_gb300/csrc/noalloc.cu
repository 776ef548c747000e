// Field energy of caller-owned device arrays, computed without allocating
// any memory.
//
// Some callers cannot allocate device memory at the point where they need
// this number: code that runs while another framework owns the device
// allocator and has handed out its whole budget, real-time loops that must
// not enter the allocator, or tools that inspect a simulation's fields in
// place.  This entry point takes the six field arrays and the material bytes
// as device pointers and keeps its reduction scratch (per-block partial sums,
// an arrival counter and the result) in one file-scope __device__ array of
// fixed size, so a call performs no cudaMalloc, cudaFree or other allocating
// call.
//
// The array is shared by every call on a device and keeps the contents of the
// last call; the arrival counter is cleared at the start of each call.  Calls
// that overlap on the GPU (two streams, or two host threads) use the same
// scratch and race; serialize them.  The scratch's device address is looked
// up with the device current on every call whose stream is not being
// captured (a device reset reloads the module and may move the array), and
// kept per device for calls made during a capture, so make the first call on
// each device before capturing any stream into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_api_internal.h"
#include "fdtd_internal.cuh"

namespace fdtd {
namespace {

constexpr int kStaticBlocks = 2048;               // partial sums kept at most
constexpr long long kStaticCellsPerBlock = 65536; // cells folded into one partial sum at most
constexpr long long kStaticMaxCells = kStaticBlocks * kStaticCellsPerBlock;  // 134,217,728 cells

struct StaticScratch {
  double partial[kStaticBlocks];
  double result;
  unsigned int counter;
};

static __device__ __align__(256) StaticScratch g_static_scratch;

std::mutex g_scratch_mu;
std::vector<StaticScratch*> g_scratch_addr;  // per device, the address last looked up

// Device address of the scratch on device `dev` (current).  Looked up again
// unless `capturing`: a device reset between calls reloads the module, and
// the array may then sit elsewhere.
int scratch_address(int dev, bool capturing, StaticScratch** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if ((int)g_scratch_addr.size() <= dev) g_scratch_addr.resize(dev + 1, nullptr);
  if (!g_scratch_addr[dev] || !capturing) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the static scratch");
    g_scratch_addr[dev] = static_cast<StaticScratch*>(p);
  }
  *out = g_scratch_addr[dev];
  return FDTD_OK;
}

template <typename T>
__global__ void __launch_bounds__(256) k_energy_static(const T* __restrict__ ex, const T* __restrict__ ey,
                                                       const T* __restrict__ ez, const T* __restrict__ hx,
                                                       const T* __restrict__ hy, const T* __restrict__ hz,
                                                       const uint8_t* __restrict__ mat, int nx, int ny, int pitch,
                                                       long long ncell, double e0, double e1, double e2,
                                                       StaticScratch* s) {
  __shared__ double red[8];
  __shared__ bool last;
  const double epsv[4] = {e0, e1, e2, 0.0};
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride) {
    const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
    const long long q = (k * ny + j) * pitch + i;
    const unsigned m = mat[q];
    const double vx = (double)ex[q], vy = (double)ey[q], vz = (double)ez[q];
    const double wx = (double)hx[q], wy = (double)hy[q], wz = (double)hz[q];
    acc += epsv[m & 3] * vx * vx + epsv[(m >> 2) & 3] * vy * vy + epsv[(m >> 4) & 3] * vz * vz;
    acc += wx * wx + wy * wy + wz * wz;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    s->partial[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&s->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    const volatile double* pp = s->partial;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += pp[b];
    s->result = tot;
    s->counter = 0u;
  }
}

}  // namespace
}  // namespace fdtd

extern "C" int fdtd_field_energy_noalloc(const void* const fields[6], const uint8_t* mat, int32_t nx, int32_t ny,
                                         int32_t nz, int32_t pitch, int32_t precision, const double eps[3],
                                         double dx, void* stream, double* out) {
  using namespace fdtd;
  if (!fields || !mat || !eps || !out) return set_error(FDTD_E_INVAL, "null argument");
  for (int c = 0; c < 6; ++c)
    if (!fields[c]) return set_error(FDTD_E_INVAL, "null field array %d", c);
  if (nx < 1 || ny < 1 || nz < 1 || pitch < nx) return set_error(FDTD_E_INVAL, "sizes: need nx, ny, nz >= 1 and pitch >= nx");
  if (precision != FDTD_FP32 && precision != FDTD_FP64) return set_error(FDTD_E_INVAL, "precision");
  if (!(dx > 0)) return set_error(FDTD_E_INVAL, "dx must be > 0");
  const long long ncell = (long long)nx * ny * nz;
  if (ncell > kStaticMaxCells)
    return set_error(FDTD_E_INVAL,
                     "%lld cells exceed the static scratch of this entry point (at most %lld cells: %d partial sums "
                     "of %lld cells); use fdtd_field_energy on a grid instead",
                     ncell, kStaticMaxCells, kStaticBlocks, kStaticCellsPerBlock);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
  StaticScratch* s = nullptr;
  int r = scratch_address(dev, cap != cudaStreamCaptureStatusNone, &s);
  if (r != FDTD_OK) return r;
  // the arrival counter must start at zero (an interrupted earlier call may have left it set)
  e = cudaMemsetAsync(&s->counter, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return cuda_error(e, "clear the static scratch counter");
  // at least two blocks per SM (the grid-stride loop takes any count up to
  // the kStaticBlocks partial sums), more when a block would fold more than
  // kStaticCellsPerBlock cells
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_error(e, "cudaDeviceGetAttribute");
  const long long need = (ncell + kStaticCellsPerBlock - 1) / kStaticCellsPerBlock;
  const int blocks = (int)std::min<long long>(kStaticBlocks, std::max<long long>(2LL * sms, need));
  if (precision == FDTD_FP32) {
    const float* const* f = reinterpret_cast<const float* const*>(fields);
    k_energy_static<float><<<blocks, 256, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], mat, nx, ny, pitch, ncell,
                                                   eps[0], eps[1], eps[2], s);
  } else {
    const double* const* f = reinterpret_cast<const double* const*>(fields);
    k_energy_static<double><<<blocks, 256, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5], mat, nx, ny, pitch, ncell,
                                                    eps[0], eps[1], eps[2], s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "energy kernel");
  double v = 0.0;
  if ((e = cudaMemcpyAsync(&v, &s->result, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_error(e, "read the result");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "sync");
  *out = 0.5 * eps0() * dx * dx * dx * v;
  return FDTD_OK;
}
