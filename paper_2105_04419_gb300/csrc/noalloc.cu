// vdbedt_edt_dense_noalloc: the exact truncated transform of a small dense grid that allocates
// nothing.
//
// Some callers cannot call cudaMalloc: code running while another part of the application holds a
// stream capture open, real-time control loops that must not enter the allocator, and embedded or
// plugin hosts whose device memory budget is fixed when the library is loaded.  For them this entry
// point computes the same D as a handle (vdbedt_create + vdbedt_set_occupancy_dense +
// vdbedt_global) but keeps its two intermediate fields (the x-line and in-plane squared distances)
// in a file-scope device array of fixed size instead of allocating them.  That array exists on
// every GPU that loads the library, for as long as the process runs.
//
// The array is shared by every call on a device and keeps the last call's contents; each call
// writes every scratch element it later reads, so nothing needs clearing.  Calls whose work
// overlaps on the GPU (on different streams, or from different threads without ordering) race on
// the array.
//
// Host code must not pass the array's name to a kernel (in host code it is a host-side stand-in,
// not a device address): the device address is looked up once per device with
// cudaGetSymbolAddress, on the first call made while that device is current, and cached.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/vdbedt.h"
#include "vdbedt_internal.cuh"

namespace {

constexpr int64_t kMaxVoxels = VDBEDT_NOALLOC_MAX_VOXELS;
constexpr int kMaxDevices = 64;

// g1 (x-line squared distance) at [0, kMaxVoxels), g2 (in-plane) at [kMaxVoxels, 2 kMaxVoxels).
static __device__ __align__(256) uint16_t g_noalloc_scratch[2 * kMaxVoxels];

std::atomic<uint16_t*> g_scratch_ptr[kMaxDevices];

// x: nearest occupied voxel along the x-line within dmax - 1, squared, saturated at dmax^2.
__global__ void k_dense_x(const uint8_t* __restrict__ occ, int nx, int ny, int nz, int dmax, uint16_t* __restrict__ g1) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int cap = dmax * dmax;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const uint8_t* row = occ + (i - x);
    int best = cap;
    for (int d = 0; d < dmax && d * d < best; ++d) {
      if ((x - d >= 0 && row[x - d]) || (x + d < nx && row[x + d])) best = d * d;
    }
    g1[i] = (uint16_t)best;
  }
}

// y (axis 1) or z (axis 2): min over |d| < dmax of d^2 + the previous field at offset d.
__global__ void k_dense_win(const uint16_t* __restrict__ in, int nx, int ny, int nz, int dmax, int axis,
                            uint16_t* __restrict__ out16, int32_t* __restrict__ out32) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int cap = dmax * dmax;
  const int64_t stride = axis == 1 ? (int64_t)nx : (int64_t)nx * ny;
  const int len = axis == 1 ? ny : nz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = axis == 1 ? (int)((i / nx) % ny) : (int)(i / ((int64_t)nx * ny));
    int best = in[i];
    for (int d = 1; d < dmax && d * d < best; ++d) {
      if (c - d >= 0) best = min(best, d * d + (int)in[i - d * stride]);
      if (c + d < len) best = min(best, d * d + (int)in[i + d * stride]);
    }
    best = min(best, cap);
    if (out32)
      out32[i] = best;
    else
      out16[i] = (uint16_t)best;
  }
}

}  // namespace

extern "C" vdbedt_status vdbedt_edt_dense_noalloc(const uint8_t* occ, int32_t nx, int32_t ny, int32_t nz,
                                                  int32_t dmax, int32_t* out, void* stream) {
  if (!occ || !out || nx < 1 || ny < 1 || nz < 1 || dmax < 1 || dmax > VDBEDT_DMAX_LIMIT) return VDBEDT_EINVAL;
  const int64_t n = (int64_t)nx * ny * nz;
  if (n > kMaxVoxels) return VDBEDT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VDBEDT_ECUDA;
  uint16_t* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return VDBEDT_ECUDA;
    scratch = static_cast<uint16_t*>(p);
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);
  }
  cudaStream_t st = (cudaStream_t)stream;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  uint16_t* g1 = scratch;
  uint16_t* g2 = scratch + kMaxVoxels;
  VDB_LAUNCH(k_dense_x, (unsigned)blocks, 256, 0, st, occ, nx, ny, nz, dmax, g1);
  VDB_LAUNCH(k_dense_win, (unsigned)blocks, 256, 0, st, g1, nx, ny, nz, dmax, 1, g2, (int32_t*)nullptr);
  VDB_LAUNCH(k_dense_win, (unsigned)blocks, 256, 0, st, g2, nx, ny, nz, dmax, 2, (uint16_t*)nullptr, out);
  return cudaGetLastError() == cudaSuccess ? VDBEDT_OK : VDBEDT_ECUDA;
}
