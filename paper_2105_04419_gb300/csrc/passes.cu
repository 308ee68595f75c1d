// The separable transform passes over the sparse brick grid.
//
// D(v) = min(dmax^2, min over occupied o of |v - o|^2) (paper Eq. 1 with the truncation of
// Sec. III) factorises along the axes because min distributes over +:
//   g1(x,y,z) = min over occupied (x',y,z) of (x'-x)^2          (x pass; saturated at dmax^2)
//   g2(x,y,z) = min over |d| <= W of d^2 + g1(x,y+d,z)         (y pass)
//   D(x,y,z)  = min over |d| <= W of d^2 + g2(x,y,z+d)         (z pass)
// with any window W >= dmax - 1 (offsets of dmax or more cost at least dmax^2 and can never beat
// the d = 0 term, which is already saturated).  Here W = 8R, R = floor((dmax + 6) / 8): exactly the
// halo of R bricks that each pass stages.
//
// Kernel "xy": one work item = a run of RUN bricks along y at fixed (bx, bz).  It stages the
// occupancy bits of bricks bx-R..bx+R and by-R..by+RUN-1+R (64 B each) in shared memory, expands
// every x-line into g1 with a find-nearest-set-bit per voxel (clz / ffs on a 64-bit window), then
// evaluates the y pass for the run and stores g2 (16 bit) into the run's bricks.
//
// Kernel "z": one work item = a run of RUN bricks along z at fixed (bx, by).  It stages g2 of
// bricks bz-R..bz+RUN-1+R (1 KB each, contiguous, vectorised 16-byte loads; an absent brick reads
// as dmax^2) and evaluates the z pass, writing D (int32) and the brick's finite flag.
//
// Arithmetic of the windowed minimum: packed half2, two voxels per 32-bit lane.  Every operand is
// an integer in [0, 2048] (values are saturated at dmax^2 <= 2025 for dmax <= 45 before they enter
// a window, and d^2 <= (8R)^2 <= 2304 only ever adds to them): fp16 represents each such integer
// exactly, the sum of two is exact whenever it is below 2048 and rounds to a value >= 2048
// otherwise, and min is exact, so every minimum below dmax^2 is computed exactly and every
// candidate at or above it stays at or above it.  Each thread owns 8 consecutive outputs of two
// neighbouring lines and keeps the 8 + 2W inputs in registers (fully unrolled), pairing offsets
// +d and -d: acc = min(acc, min(v[k-d], v[k+d]) + d^2).
//
// Grids larger than dmax 45 (up to 181) take the generic kernels at the end of the file: int32
// arithmetic read from shared memory with a runtime window.
#include <cuda_fp16.h>

#include "vdbedt_internal.cuh"

namespace vdbedt {

namespace {

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }

// fp16 bit pattern of a non-negative integer n (exact for n <= 2048; larger n map to 2048, which
// is above every saturation value the half kernels use, so such offsets stay irrelevant).
__host__ __device__ constexpr uint32_t half_bits(int n) {
  if (n > 2048) n = 2048;
  if (n == 0) return 0u;
  int e = 0;
  while ((1 << (e + 1)) <= n) ++e;
  uint32_t mant = e <= 10 ? ((uint32_t)(n << (10 - e)) & 0x3FFu) : ((uint32_t)(n >> (e - 10)) & 0x3FFu);
  return ((uint32_t)(e + 15) << 10) | mant;
}
__host__ __device__ constexpr uint32_t half2_bits(int n) { return half_bits(n) | (half_bits(n) << 16); }

// One 8-output window minimum on packed half2 registers:
// out[k] = min over |d| <= W of v[k + W + d] + d^2, pairing +d and -d.
template <int W>
__device__ __forceinline__ void window_min8(const uint32_t (&v)[8 + 2 * W], uint32_t (&out)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    __half2 acc = u2h(v[k + W]);
#pragma unroll
    for (int d = 1; d <= W; ++d) {
      __half2 m = __hmin2(u2h(v[k + W - d]), u2h(v[k + W + d]));
      acc = __hmin2(acc, __hadd2(m, u2h(half2_bits(d * d))));
    }
    out[k] = h2u(acc);
  }
}

template <int R, int RUN>
struct XYShape {
  static constexpr int W = 8 * R;
  static constexpr int NBX = 2 * R + 1;                  // bricks across x
  static constexpr int NBY = RUN + 2 * R;                // bricks along y
  static constexpr int NYR = 8 * NBY;                    // rows along y
  static constexpr int BITS_BYTES = 8 * NYR * NBX;       // [z][row][bxi]
  static constexpr int G1_STRIDE_Z = (NYR + 1) * 4;      // words per z plane (padded by one row)
  static constexpr int G1_WORDS = 8 * G1_STRIDE_Z;       // [z][row][xpair]
  static constexpr int THREADS = 32 * RUN;               // warp per brick of the run
  static constexpr int SLOTS = NBX * NBY;
  static constexpr size_t SMEM = (size_t)BITS_BYTES + (size_t)G1_WORDS * 4 + (size_t)SLOTS * 4 + 16;
};

template <int R, int RUN>
__global__ void __launch_bounds__(32 * RUN) k_xy_half(GridView g, const unsigned long long* __restrict__ items,
                                                      int max_items) {
  using S = XYShape<R, RUN>;
  constexpr int W = S::W;
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t* bits = smem;                                          // [z][row][bxi]
  uint32_t* g1 = reinterpret_cast<uint32_t*>(smem + S::BITS_BYTES);  // [z][row(+pad)][xpair]
  int* slots = reinterpret_cast<int*>(smem + S::BITS_BYTES + (size_t)S::G1_WORDS * 4);
  const int nitems = min(g.counters[C_XY_ITEMS], max_items);
  const int tid = threadIdx.x;
  const __half hinf = __int2half_rn(g.INF);

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx, by0, bz;
    unpack_brick(items[it], bx, by0, bz);
    // 1. slots of the staged bricks
    for (int i = tid; i < S::SLOTS; i += S::THREADS) {
      int bxi = i % S::NBX, byi = i / S::NBX;
      slots[i] = find_brick(g, bx - R + bxi, by0 - R + byi, bz);
    }
    __syncthreads();
    // 2. occupancy bytes: row (y, z) of brick (bxi, byi) is byte y + 8 z of its 64-byte mask
    for (int i = tid; i < S::SLOTS * 64; i += S::THREADS) {
      int b = i >> 6, byte = i & 63;
      int s = slots[b];
      uint8_t v = 0;
      if (s >= 0) v = reinterpret_cast<const uint8_t*>(g.occ)[(size_t)s * 64 + byte];
      int bxi = b % S::NBX, byi = b / S::NBX;
      int y = byte & 7, z = byte >> 3;
      bits[(z * S::NYR + byi * 8 + y) * S::NBX + bxi] = v;
    }
    __syncthreads();
    // 3. x pass: g1 for every (z, row), 8 voxels of the centre brick
    for (int i = tid; i < 8 * S::NYR; i += S::THREADS) {
      const uint8_t* line = bits + i * S::NBX;
      unsigned long long lo = 0, hi = 0;
#pragma unroll
      for (int b = 0; b < S::NBX; ++b) {
        unsigned long long byte = line[b];
        if (b < 8)
          lo |= byte << (8 * b);
        else
          hi |= byte << (8 * (b - 8));
      }
      uint32_t w[4];
      if ((lo | hi) == 0ull) {
        uint32_t p = h2u(__halves2half2(hinf, hinf));
        w[0] = w[1] = w[2] = w[3] = p;
      } else {
        __half hv[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int p = 8 * R + x;  // position of voxel x in the line (p < 64 for R <= 6)
          int best = g.INF;
          unsigned long long L = lo & ((2ull << p) - 1ull);
          if (L) {
            int dl = p - (63 - __clzll((long long)L));
            best = min(best, dl * dl);
          }
          unsigned long long Rm = (lo >> p) | (p ? (hi << (64 - p)) : 0ull);
          if (Rm) {
            int dr = __ffsll((long long)Rm) - 1;
            best = min(best, dr * dr);
          }
          hv[x] = __int2half_rn(best);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = h2u(__halves2half2(hv[2 * q], hv[2 * q + 1]));
      }
      int z = i / S::NYR, row = i % S::NYR;
      uint32_t* dst = g1 + z * S::G1_STRIDE_Z + row * 4;
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    // 4. y pass: warp = brick of the run; lane = (xpair, z); 8 outputs along y
    {
      const int warp = tid >> 5, lane = tid & 31;
      const int xp = lane & 3, z = lane >> 2;
      const int s = slots[(warp + R) * S::NBX + R];
      if (s >= 0) {
        uint32_t v[8 + 2 * W];
        const uint32_t* col = g1 + z * S::G1_STRIDE_Z + xp;
        const int r0 = warp * 8;  // row of output y = 0 minus W, i.e. (warp + R) * 8 - W
#pragma unroll
        for (int j = 0; j < 8 + 2 * W; ++j) v[j] = col[(r0 + j) * 4];
        uint32_t out[8];
        window_min8<W>(v, out);
        uint32_t* dst = reinterpret_cast<uint32_t*>(g.g2 + (size_t)s * kBrickVox) + z * 32 + xp;
#pragma unroll
        for (int y = 0; y < 8; ++y) dst[y * 4] = out[y];
      }
    }
    __syncthreads();
  }
}

template <int R, int RUN>
struct ZShape {
  static constexpr int W = 8 * R;
  static constexpr int NB = RUN + 2 * R;
  static constexpr int WORDS = NB * 256;  // 512 half values per brick
  static constexpr int THREADS = 32 * RUN;
  static constexpr size_t SMEM = (size_t)WORDS * 4 + (size_t)NB * 4 + 16;
};

template <int R, int RUN>
__global__ void __launch_bounds__(32 * RUN) k_z_half(GridView g, const unsigned long long* __restrict__ items,
                                                     int max_items) {
  using S = ZShape<R, RUN>;
  constexpr int W = S::W;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* col = reinterpret_cast<uint32_t*>(smem);  // [brick][z][y][xpair]
  int* slots = reinterpret_cast<int*>(smem + (size_t)S::WORDS * 4);
  const int nitems = min(g.counters[C_Z_ITEMS], max_items);
  const int tid = threadIdx.x;
  const __half hinf = __int2half_rn(g.INF);
  const uint32_t inf2 = h2u(__halves2half2(hinf, hinf));

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx, by, bz0;
    unpack_brick(items[it], bx, by, bz0);
    for (int i = tid; i < S::NB; i += S::THREADS) slots[i] = find_brick(g, bx, by, bz0 - R + i);
    __syncthreads();
    // stage g2 of the column, 16 bytes per thread per step
    for (int i = tid; i < S::NB * 64; i += S::THREADS) {
      int b = i >> 6, q = i & 63;
      int s = slots[b];
      uint4 v = make_uint4(inf2, inf2, inf2, inf2);
      if (s >= 0) v = reinterpret_cast<const uint4*>(g.g2 + (size_t)s * kBrickVox)[q];
      reinterpret_cast<uint4*>(col)[i] = v;
    }
    __syncthreads();
    {
      const int warp = tid >> 5, lane = tid & 31;
      const int xp = lane & 3, y = lane >> 2;
      const int s = slots[warp + R];
      if (s >= 0) {
        uint32_t v[8 + 2 * W];
        const uint32_t* c = col + y * 4 + xp;
        const int p0 = warp * 8;  // plane of output z = 0 minus W
#pragma unroll
        for (int j = 0; j < 8 + 2 * W; ++j) v[j] = c[(p0 + j) * 32];
        uint32_t out[8];
        window_min8<W>(v, out);
        int2* dst = reinterpret_cast<int2*>(g.dist + (size_t)s * kBrickVox) + y * 4 + xp;
        bool finite = false;
#pragma unroll
        for (int z = 0; z < 8; ++z) {
          __half2 h = u2h(out[z]);
          int a = __half2int_rn(__low2half(h)), b = __half2int_rn(__high2half(h));
          finite |= (a < g.INF) | (b < g.INF);
          dst[z * 32] = make_int2(a, b);
        }
        unsigned any = __any_sync(0xffffffffu, finite);
        if (lane == 0) {
          uint32_t f = g.bflags[s];
          f = any ? (f | F_FINITE) : (f & ~F_FINITE);
          g.bflags[s] = f;
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Generic kernels (any dmax up to 181): int32 from shared memory, runtime window W = 8R.
// ------------------------------------------------------------------------------------------------
constexpr int kGenRun = 4;
constexpr int kGenThreads = 256;

__global__ void __launch_bounds__(kGenThreads) k_xy_generic(GridView g, const unsigned long long* __restrict__ items,
                                                            int max_items) {
  const int R = g.R, W = 8 * R, NBX = 2 * R + 1, NBY = kGenRun + 2 * R, NYR = 8 * NBY;
  extern __shared__ __align__(16) unsigned char smem[];
  int* slots = reinterpret_cast<int*>(smem);                        // [NBY][NBX]
  int* g1 = slots + NBX * NBY;                                      // [z][row][x]
  const int nitems = min(g.counters[C_XY_ITEMS], max_items);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx, by0, bz;
    unpack_brick(items[it], bx, by0, bz);
    for (int i = threadIdx.x; i < NBX * NBY; i += blockDim.x)
      slots[i] = find_brick(g, bx - R + i % NBX, by0 - R + i / NBX, bz);
    __syncthreads();
    // x pass straight from the bit masks: scan outward along the line
    for (int i = threadIdx.x; i < 8 * NYR * 8; i += blockDim.x) {
      int x = i & 7, row = (i >> 3) % NYR, z = (i >> 3) / NYR;
      int byi = row >> 3, y = row & 7;
      int best = g.INF;
      for (int d = 0; d <= W && d * d < best; ++d) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          if (d == 0 && sgn > 0) continue;
          int xx = 8 * R + x + sgn * d;  // position in the line of 8 * NBX voxels
          if (xx < 0 || xx >= 8 * NBX) continue;
          int s = slots[byi * NBX + (xx >> 3)];
          if (s < 0) continue;
          uint8_t rowbits = reinterpret_cast<const uint8_t*>(g.occ)[(size_t)s * 64 + y + 8 * z];
          if ((rowbits >> (xx & 7)) & 1) best = min(best, d * d);
        }
      }
      g1[(z * NYR + row) * 8 + x] = best;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kGenRun * 512; i += blockDim.x) {
      int b = i >> 9, v = i & 511;
      int x = v & 7, y = (v >> 3) & 7, z = v >> 6;
      int s = slots[(b + R) * NBX + R];
      if (s < 0) continue;
      int row = (b + R) * 8 + y;
      int best = g.INF;
      for (int d = -W; d <= W; ++d) best = min(best, d * d + g1[(z * NYR + row + d) * 8 + x]);
      g.g2[(size_t)s * kBrickVox + v] = (uint16_t)best;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kGenThreads) k_z_generic(GridView g, const unsigned long long* __restrict__ items,
                                                           int max_items) {
  const int R = g.R, W = 8 * R, NB = kGenRun + 2 * R;
  extern __shared__ __align__(16) unsigned char smem[];
  int* slots = reinterpret_cast<int*>(smem);
  uint16_t* col = reinterpret_cast<uint16_t*>(slots + NB + 3);  // [brick][512]
  const int nitems = min(g.counters[C_Z_ITEMS], max_items);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx, by, bz0;
    unpack_brick(items[it], bx, by, bz0);
    for (int i = threadIdx.x; i < NB; i += blockDim.x) slots[i] = find_brick(g, bx, by, bz0 - R + i);
    __syncthreads();
    for (int i = threadIdx.x; i < NB * 512; i += blockDim.x) {
      int s = slots[i >> 9];
      col[i] = s >= 0 ? g.g2[(size_t)s * kBrickVox + (i & 511)] : (uint16_t)g.INF;
    }
    __syncthreads();
    for (int b = 0; b < kGenRun; ++b) {
      int s = slots[b + R];
      if (s < 0) continue;
      bool finite = false;
      for (int v = threadIdx.x; v < 512; v += blockDim.x) {
        int z = v >> 6, xy = v & 63;
        int plane = (b + R) * 8 + z;
        int best = g.INF;
        for (int d = -W; d <= W; ++d) best = min(best, d * d + (int)col[(plane + d) * 64 + xy]);
        g.dist[(size_t)s * kBrickVox + v] = best;
        finite |= best < g.INF;
      }
      int any = __syncthreads_or(finite);
      if (threadIdx.x == 0) g.bflags[s] = any ? (g.bflags[s] | F_FINITE) : (g.bflags[s] & ~F_FINITE);
    }
    __syncthreads();
  }
}

int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <typename K>
cudaError_t launch_persistent(K kernel, int threads, size_t smem, const GridView& g, const unsigned long long* items,
                              int max_items, cudaStream_t st) {
  if (max_items <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms() * per_sm;
  if (grid > max_items) grid = max_items;
  VDB_LAUNCH(kernel, grid, threads, smem, st, g, items, max_items);
  return cudaGetLastError();
}

template <int R, int RUN>
cudaError_t xy_half(const GridView& g, const unsigned long long* items, int max_items, cudaStream_t st) {
  using S = XYShape<R, RUN>;
  return launch_persistent(k_xy_half<R, RUN>, S::THREADS, S::SMEM, g, items, max_items, st);
}
template <int R, int RUN>
cudaError_t z_half(const GridView& g, const unsigned long long* items, int max_items, cudaStream_t st) {
  using S = ZShape<R, RUN>;
  return launch_persistent(k_z_half<R, RUN>, S::THREADS, S::SMEM, g, items, max_items, st);
}

template <int RUN>
cudaError_t xy_half_r(const GridView& g, const unsigned long long* items, int max_items, cudaStream_t st) {
  switch (g.R) {
    case 1: return xy_half<1, RUN>(g, items, max_items, st);
    case 2: return xy_half<2, RUN>(g, items, max_items, st);
    case 3: return xy_half<3, RUN>(g, items, max_items, st);
    case 4: return xy_half<4, RUN>(g, items, max_items, st);
    case 5: return xy_half<5, RUN>(g, items, max_items, st);
    case 6: return xy_half<6, RUN>(g, items, max_items, st);
  }
  return cudaErrorInvalidValue;
}
template <int RUN>
cudaError_t z_half_r(const GridView& g, const unsigned long long* items, int max_items, cudaStream_t st) {
  switch (g.R) {
    case 1: return z_half<1, RUN>(g, items, max_items, st);
    case 2: return z_half<2, RUN>(g, items, max_items, st);
    case 3: return z_half<3, RUN>(g, items, max_items, st);
    case 4: return z_half<4, RUN>(g, items, max_items, st);
    case 5: return z_half<5, RUN>(g, items, max_items, st);
    case 6: return z_half<6, RUN>(g, items, max_items, st);
  }
  return cudaErrorInvalidValue;
}

bool use_half(const GridView& g) { return g.dmax <= 45 && g.R >= 1 && g.R <= 6; }

}  // namespace

int item_run_xy(const GridView& g, const Tuning& t) { return use_half(g) ? t.xy_run : kGenRun; }
int item_run_z(const GridView& g, const Tuning& t) { return use_half(g) ? t.z_run : kGenRun; }

cudaError_t launch_xy_pass(const GridView& g, const Tuning& t, const unsigned long long* items, int max_items,
                           cudaStream_t st) {
  if (use_half(g)) {
    switch (t.xy_run) {
      case 4: return xy_half_r<4>(g, items, max_items, st);
      case 8: return xy_half_r<8>(g, items, max_items, st);
      case 16: return xy_half_r<16>(g, items, max_items, st);
    }
    return cudaErrorInvalidValue;
  }
  const int R = g.R, NBX = 2 * R + 1, NBY = kGenRun + 2 * R;
  size_t smem = (size_t)NBX * NBY * 4 + (size_t)8 * 8 * NBY * 8 * 4 + 64;
  return launch_persistent(k_xy_generic, kGenThreads, smem, g, items, max_items, st);
}

cudaError_t launch_z_pass(const GridView& g, const Tuning& t, const unsigned long long* items, int max_items,
                          cudaStream_t st) {
  if (use_half(g)) {
    switch (t.z_run) {
      case 4: return z_half_r<4>(g, items, max_items, st);
      case 8: return z_half_r<8>(g, items, max_items, st);
      case 16: return z_half_r<16>(g, items, max_items, st);
    }
    return cudaErrorInvalidValue;
  }
  const int NB = kGenRun + 2 * g.R;
  size_t smem = (size_t)(NB + 3) * 4 + (size_t)NB * 512 * 2 + 64;
  return launch_persistent(k_z_generic, kGenThreads, smem, g, items, max_items, st);
}

}  // namespace vdbedt
