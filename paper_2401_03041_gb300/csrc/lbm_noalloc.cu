// lbm_noalloc.cu - lbm_field_moments: FP64 mass and first moments of a
// caller-owned device field, computed without allocating any memory.
//
// The computation is the diagnostics reduction of the step kernels (sum phi,
// sum phi x, sum phi y, sum phi z in FP64, two levels in a fixed order)
// applied to a field in memory.  Its intermediate partials (one group of four
// per z plane) and its four results live in a fixed array compiled into the
// library, not in a workspace, so the call needs no allocation by the library
// or by the caller.  The device address of that array is looked up with the
// device current, on the first call made on it; a failed lookup is not kept,
// so a later call on that device tries again.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "launchers.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// [plane][4] partials for up to LBM_MOMENTS_MAX_PLANES planes, then the four
// results.  Every call writes each slot it later reads, so the contents never
// need to start at zero.
static __device__ __align__(256) double g_moment_scratch[(LBM_MOMENTS_MAX_PLANES + 1) * 4];

// Per-device address of g_moment_scratch (nullptr until a lookup succeeded).
double* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Device address of the scratch array on device dev (current), looked up
// once; errors are returned, not remembered.
cudaError_t scratch_for(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_moment_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Fixed-order sum of one value over a block: warp shuffles, then the warps'
// totals in warp order.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
  return s;
}

// One block per z plane: partials[4 z + 0..3] = sum psi, sum psi (x + 1/2),
// sum psi (y + 1/2), sum psi (z + 1/2) over the plane.
__global__ void __launch_bounds__(kThreads)
plane_moments_kernel(const void* __restrict__ field, int dtype, int nx, int ny,
                     double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  const int z = blockIdx.x;
  const unsigned plane = (unsigned)nx * (unsigned)ny;
  const size_t base = (size_t)z * plane;
  double s0 = 0.0, sx = 0.0, sy = 0.0;
  for (unsigned k = threadIdx.x; k < plane; k += kThreads) {
    const double v = dtype == 0 ? static_cast<const double*>(field)[base + k]
                                : (double)static_cast<const float*>(field)[base + k];
    const unsigned y = k / (unsigned)nx, x = k - y * (unsigned)nx;
    s0 += v;
    sx += v * (x + 0.5);
    sy += v * (y + 0.5);
  }
  s0 = block_sum(s0, red);
  sx = block_sum(sx, red);
  sy = block_sum(sy, red);
  if (threadIdx.x == 0) {
    partials[4 * z + 0] = s0;
    partials[4 * z + 1] = sx;
    partials[4 * z + 2] = sy;
    partials[4 * z + 3] = s0 * (z + 0.5);
  }
}

// One block: out[c] = sum over planes of partials[4 z + c], in a fixed order.
__global__ void __launch_bounds__(kThreads)
moments_finalize_kernel(const double* __restrict__ partials, int nz, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  for (int c = 0; c < 4; ++c) {
    double v = 0.0;
    for (int z = threadIdx.x; z < nz; z += kThreads) v += partials[4 * z + c];
    v = block_sum(v, red);
    if (threadIdx.x == 0) out[c] = v;
  }
}

}  // namespace

extern "C" lbm_status lbm_field_moments(const void* field, int dtype, int nx, int ny, int nz,
                                        void* stream, double* out_host) {
  if (!field || !out_host) return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: null pointer");
  if (dtype != 0 && dtype != 1) return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: dtype must be 0 or 1");
  if (nx < 1 || ny < 1 || nz < 1) return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: sizes must be >= 1");
  if (nz > LBM_MOMENTS_MAX_PLANES)
    return lbm::set_error(LBM_ERR_ARG,
                          "lbm_field_moments: nz exceeds LBM_MOMENTS_MAX_PLANES (the fixed scratch holds "
                          "one partial group per plane)");
  if ((long long)nx * ny >= (1LL << 31))
    return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: nx * ny must be < 2^31");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: device index too large");
  // the field must be device (or managed) memory of the current device: the
  // kernels run there and read it directly
  cudaPointerAttributes pa{};
  e = cudaPointerGetAttributes(&pa, field);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: field is not a CUDA pointer");
  }
  if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
    return lbm::set_error(LBM_ERR_ARG,
                          "lbm_field_moments: field must be device memory of the current device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (st) {
    int sdev = -1;
    e = cudaStreamGetDevice(st, &sdev);
    if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (sdev != dev) return lbm::set_error(LBM_ERR_ARG, "lbm_field_moments: stream belongs to another device");
  }
  // set-up on the first call on this device, with that device current
  double* scratch = nullptr;
  e = scratch_for(dev, &scratch);
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  double* results = scratch + 4 * LBM_MOMENTS_MAX_PLANES;

  plane_moments_kernel<<<nz, kThreads, 0, st>>>(field, dtype, nx, ny, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  moments_finalize_kernel<<<1, kThreads, 0, st>>>(scratch, nz, results);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  e = cudaMemcpyAsync(out_host, results, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return lbm::set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
