// Parallel primitives used to build the sparse grid: exclusive scan and stable LSD radix sort.
//
// Radix sort: 8-bit digits, 4096 keys per block.  Per pass: (1) per-block digit histogram,
// (2) exclusive scan of the digit-major histogram table, (3) stable scatter: each warp walks its
// 512-key sub-tile in rounds of 32 and ranks equal digits with __match_any_sync, after a block
// scan of per-warp digit counts fixes each warp's base.  The real element count may live on the
// device (sizes are upper bounds), so no host synchronisation is needed.
#include "vdbedt_internal.cuh"

namespace vdbedt {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;  // 2048

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim.x == kScanThreads); returns the
// exclusive prefix, writes the block total to *total.
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = warp_incl_scan(v);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kScanThreads / 32 ? wsum[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < kScanThreads / 32) wsum[lane] = si - s;
    if (lane == kScanThreads / 32 - 1) *total = si;
  }
  __syncthreads();
  int r = incl - v + wsum[warp];
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ part,
                              const int32_t* gate) {
  if (gate && *gate == 0) return;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j)
    if (base + j < n) s += in[base + j];
  __shared__ int tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int32_t* part, int64_t nb, int32_t* total, const int32_t* gate) {
  if (gate && *gate == 0) return;
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t off = 0; off < nb; off += kScanThreads) {
    int64_t i = off + threadIdx.x;
    int v = i < nb ? part[i] : 0;
    __shared__ int tot;
    int ex = block_excl_scan(v, &tot);
    if (i < nb) part[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_down(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                            const int32_t* __restrict__ part, const int32_t* gate) {
  if (gate && *gate == 0) return;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    s += v[j];
  }
  __shared__ int tot;
  int ex = block_excl_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < n) out[base + j] = ex;
    ex += v[j];
  }
}

// ---- radix sort ----
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = 4096;
constexpr int kSubTile = kSortTile / kSortWarps;  // 512 per warp

__device__ __forceinline__ int64_t actual_count(int64_t n, const int32_t* count_dev) {
  if (!count_dev) return n;
  int64_t c = *count_dev;
  return c < n ? c : n;
}

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, const int32_t* count_dev, int shift,
                             int32_t* __restrict__ hist, int nblocks) {
  const int64_t cnt = actual_count(n, count_dev);
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (cnt == 0) return;  // the whole sort is idle (the scan and scatter check the same count)
  if (base >= cnt) {
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = 0;
    return;
  }
  __shared__ int sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < kSortTile; j += kSortThreads) {
    int64_t i = base + j;
    if (i < cnt) atomicAdd(&sh[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, uint32_t* __restrict__ kout,
                                const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, int64_t n,
                                const int32_t* count_dev, int shift, const int32_t* __restrict__ offs, int nblocks) {
  const int64_t total = actual_count(n, count_dev);
  if ((int64_t)blockIdx.x * kSortTile >= total) return;  // block-uniform
  __shared__ int cnt[kSortWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < kSortWarps * 256; j += kSortThreads) (&cnt[0][0])[j] = 0;
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kSubTile;
  // phase A: per-warp digit counts
  for (int r = 0; r < kSubTile / 32; ++r) {
    int64_t i = wbase + r * 32 + lane;
    int d = i < total ? (int)((kin[i] >> shift) & 255) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < 256 && lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // phase B: per-digit base of each warp
  {
    int d = threadIdx.x;
    int run = offs[(int64_t)d * nblocks + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      int c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  // phase C: stable scatter
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSubTile / 32; ++r) {
    int64_t i = wbase + r * 32 + lane;
    uint32_t k = 0, v = 0;
    int d = 256;
    if (i < total) {
      k = kin[i];
      if (vin) v = vin[i];
      d = (int)((k >> shift) & 255);
    }
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int pos = 0;
    if (d < 256) pos = cnt[warp][d] + __popc(peers & lt);
    __syncwarp();
    if (d < 256) {
      kout[pos] = k;
      if (vout) vout[pos] = v;
      if (lane == __ffs(peers) - 1) cnt[warp][d] += __popc(peers);
    }
    __syncwarp();
  }
}

}  // namespace

size_t scan_temp_bytes(int64_t n) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)(nb + 1) * sizeof(int32_t) + 256;
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev, void* temp,
                               cudaStream_t st, const int32_t* gate) {
  if (n <= 0) {
    if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(int32_t), st);
    return cudaSuccess;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  int32_t* part = (int32_t*)temp;
  VDB_LAUNCH(k_scan_reduce, (unsigned)nb, kScanThreads, 0, st, in, n, part, gate);
  VDB_LAUNCH(k_scan_partials, 1, kScanThreads, 0, st, part, nb, total_dev, gate);
  VDB_LAUNCH(k_scan_down, (unsigned)nb, kScanThreads, 0, st, in, out, n, part, gate);
  return cudaGetLastError();
}

size_t radix_temp_bytes(int64_t n) {
  int64_t nb = (n + kSortTile - 1) / kSortTile;
  if (nb < 1) nb = 1;
  size_t hist = (size_t)256 * nb * sizeof(int32_t);
  return 2 * hist + scan_temp_bytes(256 * nb) + 512;
}

cudaError_t radix_sort_u32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, int64_t n,
                           const int32_t* count_dev, int bits, void* temp, cudaStream_t st, bool* result_in_b) {
  *result_in_b = false;
  if (n <= 0) return cudaSuccess;
  int64_t nb = (n + kSortTile - 1) / kSortTile;
  int32_t* hist = (int32_t*)temp;
  int32_t* offs = hist + 256 * nb;
  void* stemp = (void*)(offs + 256 * nb);
  int passes = (bits + 7) / 8;
  if (passes < 1) passes = 1;
  uint32_t *ka = keys_a, *kb = keys_b, *va = vals_a, *vb = vals_b;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    VDB_LAUNCH(k_radix_hist, (unsigned)nb, kSortThreads, 0, st, ka, n, count_dev, shift, hist, (int)nb);
    cudaError_t e = exclusive_scan_i32(hist, offs, 256 * nb, nullptr, stemp, st, count_dev);
    if (e != cudaSuccess) return e;
    VDB_LAUNCH(k_radix_scatter, (unsigned)nb, kSortThreads, 0, st, ka, kb, va, vb, n, count_dev, shift, offs, (int)nb);
    uint32_t* t = ka;
    ka = kb;
    kb = t;
    t = va;
    va = vb;
    vb = t;
  }
  *result_in_b = (passes & 1) != 0;
  return cudaGetLastError();
}

}  // namespace vdbedt
