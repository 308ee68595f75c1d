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
// not a device address): the device address comes from cudaGetSymbolAddress, called with the
// device current.  Each call made while its stream is not being captured looks the address up
// again and refreshes the per-device cache, so a context torn down and recreated in between (for
// example by cudaDeviceReset) is followed; a call made during a stream capture uses the cached
// address, which is why the first call on a device must come before any capture.
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

namespace {

vdbedt_status noalloc_fail(vdbedt_status s, const char* msg) {
  vdbedt::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" vdbedt_status vdbedt_edt_dense_noalloc(const uint8_t* occ, int32_t nx, int32_t ny, int32_t nz,
                                                  int32_t dmax, int32_t* out, void* stream) {
  if (!occ || !out) return noalloc_fail(VDBEDT_EINVAL, "vdbedt_edt_dense_noalloc: null pointer");
  if (nx < 1 || ny < 1 || nz < 1) return noalloc_fail(VDBEDT_EINVAL, "vdbedt_edt_dense_noalloc: size < 1");
  if (dmax < 1 || dmax > VDBEDT_DMAX_LIMIT)
    return noalloc_fail(VDBEDT_EINVAL, "vdbedt_edt_dense_noalloc: dmax outside [1, VDBEDT_DMAX_LIMIT]");
  const int64_t n = (int64_t)nx * ny * nz;
  if (n > kMaxVoxels)
    return noalloc_fail(VDBEDT_EINVAL, "vdbedt_edt_dense_noalloc: more than VDBEDT_NOALLOC_MAX_VOXELS voxels");
  // an error left pending by earlier work on this thread is not ours to report or to clear
  if (cudaPeekAtLastError() != cudaSuccess)
    return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: a CUDA error from earlier work is pending "
                                      "(read it with cudaGetLastError first)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: no current device");
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: invalid stream");
  }
  uint16_t* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: scratch address lookup failed");
    }
    scratch = static_cast<uint16_t*>(p);
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);
  } else if (!scratch) {
    return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: first call on this device made during a stream "
                                      "capture (call it once before capturing)");
  }
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  uint16_t* g1 = scratch;
  uint16_t* g2 = scratch + kMaxVoxels;
  VDB_LAUNCH(k_dense_x, (unsigned)blocks, 256, 0, st, occ, nx, ny, nz, dmax, g1);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: x launch");
  VDB_LAUNCH(k_dense_win, (unsigned)blocks, 256, 0, st, g1, nx, ny, nz, dmax, 1, g2, (int32_t*)nullptr);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: y launch");
  VDB_LAUNCH(k_dense_win, (unsigned)blocks, 256, 0, st, g2, nx, ny, nz, dmax, 2, (uint16_t*)nullptr, out);
  if (cudaGetLastError() != cudaSuccess) return noalloc_fail(VDBEDT_ECUDA, "vdbedt_edt_dense_noalloc: z launch");
  return VDBEDT_OK;
}
