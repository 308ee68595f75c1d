// Reading the field: point queries, dense export, and the differentiable clearance cost.
//
// Query: D at voxel coordinates through the two-level interior (hash probe, child table); voxels
// outside the grid or in unstored bricks return the background dmax^2 (the paper's tile value,
// Sec. IV-A).  Nearest-obstacle query: the occupied voxel a cell's distance is measured to (the
// obstacle the paper keeps per cell, Sec. IV-B), found on the lattice sphere of radius^2 D.
//
// Clearance cost (Eq. 2, clearance term, as a squared hinge): per point p (metres),
//   u = p / vs (float32), i0 = floor(u) clamped to [0, n-2], t = u - i0,
//   corner distance d_c = vs * sqrt(D_c), d = trilinear(d_c, t), c = max(0, tau - d)^2,
//   cost[traj] = sum of c over the trajectory's points.
// Backward: dc/dp = -2 max(0, tau - d) (1 / vs) grad_t(trilinear), scaled by the upstream
// gradient of the trajectory's cost.  One warp per trajectory, points strided over the lanes,
// a warp shuffle sum for the forward.
#include "vdbedt_internal.cuh"

namespace vdbedt {

namespace {

__device__ __forceinline__ int sqdist_at(const GridView& g, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)g.nx || (unsigned)y >= (unsigned)g.ny || (unsigned)z >= (unsigned)g.nz) return g.INF;
  int s = find_brick(g, x >> 3, y >> 3, z >> 3);
  if (s < 0) return g.INF;
  return g.dist[(size_t)s * kBrickVox + (x & 7) + 8 * (y & 7) + 64 * (z & 7)];
}

// caller coordinates are stored shifted by g.off (an unbounded grid's signed coordinates)
__global__ void k_query(GridView g, const int32_t* __restrict__ xyz, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sqdist_at(g, xyz[3 * i] + g.off, xyz[3 * i + 1] + g.off, xyz[3 * i + 2] + g.off);
}

// One warp per x-row of a brick-aligned 8-voxel segment: lanes cover 32 consecutive x.
__global__ void k_export_dense(GridView g, int32_t* __restrict__ out) {
  const int64_t total = (int64_t)g.nx * g.ny * g.nz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % g.nx);
    int64_t r = i / g.nx;
    int y = (int)(r % g.ny), z = (int)(r / g.ny);
    out[i] = sqdist_at(g, x, y, z);
  }
}

// Occupancy bit of voxel (x, y, z) (inside the grid), keeping the thread's last node lookup (key,
// node): the candidates of one sphere walk mostly fall in one interior node, so most lookups skip
// the hash table.
__device__ __forceinline__ bool occupied_at_cached(const GridView& g, int x, int y, int z, unsigned long long& key,
                                                   int& node) {
  const unsigned long long k = node_key_of(g, x >> 3, y >> 3, z >> 3);
  if (k != key) {
    key = k;
    node = find_node(g, k);
  }
  if (node < 0) return false;
  const int s = g.child[(size_t)node * kNodeBricks + local_brick(x >> 3, y >> 3, z >> 3)];
  return s >= 0 && ((g.occ[(size_t)s * 8 + (z & 7)] >> ((x & 7) + 8 * (y & 7))) & 1ull) != 0ull;
}

__device__ __forceinline__ int isqrt_floor(int v) {
  int r = (int)sqrtf((float)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// Nearest occupied voxel of a query voxel: D(v) fixes the squared distance, so the obstacle lies
// on the lattice sphere |o - v|^2 = D; its points are visited in increasing (z, y, x) and the
// first occupied one is returned (ties to the smallest (z, y, x)).  (-1, -1, -1) outside the grid
// or when D = dmax^2 (no obstacle closer than dmax).  Integer square roots come from a shared
// table of floor(sqrt(v)) for v = 0 .. dmax^2 (dynamic shared memory, dmax^2 + 1 bytes).
__global__ void k_query_nearest(GridView g, const int32_t* __restrict__ xyz, int64_t n, int32_t* __restrict__ out) {
  extern __shared__ uint8_t isq[];
  for (int v = threadIdx.x; v <= g.INF; v += blockDim.x) isq[v] = (uint8_t)isqrt_floor(v);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = xyz[3 * i] + g.off, y = xyz[3 * i + 1] + g.off, z = xyz[3 * i + 2] + g.off;
    int rx = -1 + g.off, ry = -1 + g.off, rz = -1 + g.off;
    const int D = sqdist_at(g, x, y, z);
    if ((unsigned)x < (unsigned)g.nx && (unsigned)y < (unsigned)g.ny && (unsigned)z < (unsigned)g.nz && D < g.INF) {
      bool found = false;
      unsigned long long ckey = ~0ull;  // no node looked up yet
      int cnode = -1;
      const int r = isq[D];
      for (int dz = -r; dz <= r && !found; ++dz) {
        const int oz = z + dz, rem = D - dz * dz;
        if ((unsigned)oz >= (unsigned)g.nz) continue;
        const int r2 = isq[rem];
        for (int dy = -r2; dy <= r2 && !found; ++dy) {
          const int oy = y + dy, rem2 = rem - dy * dy;
          const int dx = isq[rem2];
          if (dx * dx != rem2 || (unsigned)oy >= (unsigned)g.ny) continue;
          if (x - dx >= 0 && occupied_at_cached(g, x - dx, oy, oz, ckey, cnode)) {
            rx = x - dx, ry = oy, rz = oz, found = true;
          } else if (dx > 0 && x + dx < g.nx && occupied_at_cached(g, x + dx, oy, oz, ckey, cnode)) {
            rx = x + dx, ry = oy, rz = oz, found = true;
          }
        }
      }
      if (!found) set_error(g, kErrInternal);  // a finite D always has an obstacle on its sphere
    }
    out[3 * i] = rx - g.off;  // (-1, -1, -1) when there is none
    out[3 * i + 1] = ry - g.off;
    out[3 * i + 2] = rz - g.off;
  }
}

struct Corner8 {
  float d[8];  // index a + 2b + 4c for corner (i0+a, j0+b, k0+c)
};

// Corner distances (metres) of the cell holding u; returns the in-cell coordinates.
__device__ __forceinline__ void cell_of(const GridView& g, float vs, float px, float py, float pz, int& i0, int& j0,
                                        int& k0, float& tx, float& ty, float& tz) {
  float ux = px / vs, uy = py / vs, uz = pz / vs;
  float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
  // cells in stored coordinates (shifted by g.off); t measured from the cell in caller coordinates
  const float o = (float)g.off;
  i0 = (int)fminf(fmaxf(fx + o, 0.f), (float)(g.nx - 2));
  j0 = (int)fminf(fmaxf(fy + o, 0.f), (float)(g.ny - 2));
  k0 = (int)fminf(fmaxf(fz + o, 0.f), (float)(g.nz - 2));
  tx = ux - (float)(i0 - g.off);
  ty = uy - (float)(j0 - g.off);
  tz = uz - (float)(k0 - g.off);
}

__device__ __forceinline__ void corners(const GridView& g, float vs, int i0, int j0, int k0, Corner8& c) {
  // most cells sit inside one brick: look the brick up once
  const bool one = ((i0 & 7) != 7) && ((j0 & 7) != 7) && ((k0 & 7) != 7);
  if (one) {
    int s = find_brick(g, i0 >> 3, j0 >> 3, k0 >> 3);
    const float inf_m = vs * sqrtf((float)g.INF);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
      if (s < 0) {
        c.d[q] = inf_m;
      } else {
        int D = g.dist[(size_t)s * kBrickVox + ((i0 + a) & 7) + 8 * ((j0 + b) & 7) + 64 * ((k0 + e) & 7)];
        c.d[q] = vs * sqrtf((float)D);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int a = q & 1, b = (q >> 1) & 1, e = q >> 2;
      c.d[q] = vs * sqrtf((float)sqdist_at(g, i0 + a, j0 + b, k0 + e));
    }
  }
}

__device__ __forceinline__ float trilinear(const Corner8& c, float tx, float ty, float tz) {
  float c00 = c.d[0] + tx * (c.d[1] - c.d[0]);
  float c10 = c.d[2] + tx * (c.d[3] - c.d[2]);
  float c01 = c.d[4] + tx * (c.d[5] - c.d[4]);
  float c11 = c.d[6] + tx * (c.d[7] - c.d[6]);
  float c0 = c00 + ty * (c10 - c00);
  float c1 = c01 + ty * (c11 - c01);
  return c0 + tz * (c1 - c0);
}

__global__ void k_clearance_fwd(GridView g, float vs, const float* __restrict__ pts, int64_t T, int64_t P, float tau,
                                float* __restrict__ cost) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < T; t += nw) {
    float acc = 0.f;
    for (int64_t p = lane; p < P; p += 32) {
      const float* q = pts + (t * P + p) * 3;
      int i0, j0, k0;
      float tx, ty, tz;
      cell_of(g, vs, q[0], q[1], q[2], i0, j0, k0, tx, ty, tz);
      Corner8 c;
      corners(g, vs, i0, j0, k0, c);
      float d = trilinear(c, tx, ty, tz);
      float h = fmaxf(0.f, tau - d);
      acc += h * h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) cost[t] = acc;
  }
}

__global__ void k_clearance_bwd(GridView g, float vs, const float* __restrict__ pts, int64_t T, int64_t P, float tau,
                                const float* __restrict__ gcost, float* __restrict__ gpts) {
  const int64_t n = T * P;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float* q = pts + i * 3;
    int i0, j0, k0;
    float tx, ty, tz;
    cell_of(g, vs, q[0], q[1], q[2], i0, j0, k0, tx, ty, tz);
    Corner8 c;
    corners(g, vs, i0, j0, k0, c);
    float d = trilinear(c, tx, ty, tz);
    float h = fmaxf(0.f, tau - d);
    float go = gcost[i / P];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (h > 0.f) {
      float wx[2] = {1.f - tx, tx}, wy[2] = {1.f - ty, ty}, wz[2] = {1.f - tz, tz};
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          gx += (c.d[1 + 2 * b + 4 * e] - c.d[2 * b + 4 * e]) * wy[b] * wz[e];
          gy += (c.d[2 + b + 4 * e] - c.d[b + 4 * e]) * wx[b] * wz[e];
          gz += (c.d[4 + b + 2 * e] - c.d[b + 2 * e]) * wx[b] * wy[e];
        }
      float s = -2.f * h / vs * go;
      gx *= s;
      gy *= s;
      gz *= s;
    }
    gpts[i * 3] = gx;
    gpts[i * 3 + 1] = gy;
    gpts[i * 3 + 2] = gz;
  }
}

// Distance and its gradient at points (planners): d = trilinear(vs sqrt(D)) as in the clearance
// cost, grad = (1 / vs) grad_t(trilinear), a thread per point.
__global__ void k_distance_at(GridView g, float vs, const float* __restrict__ pts, int64_t n, float* __restrict__ dist,
                              float* __restrict__ grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float* q = pts + i * 3;
    int i0, j0, k0;
    float tx, ty, tz;
    cell_of(g, vs, q[0], q[1], q[2], i0, j0, k0, tx, ty, tz);
    Corner8 c;
    corners(g, vs, i0, j0, k0, c);
    dist[i] = trilinear(c, tx, ty, tz);
    if (grad) {
      float gx = 0.f, gy = 0.f, gz = 0.f;
      const float wx[2] = {1.f - tx, tx}, wy[2] = {1.f - ty, ty}, wz[2] = {1.f - tz, tz};
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          gx += (c.d[1 + 2 * b + 4 * e] - c.d[2 * b + 4 * e]) * wy[b] * wz[e];
          gy += (c.d[2 + b + 4 * e] - c.d[b + 4 * e]) * wx[b] * wz[e];
          gz += (c.d[4 + b + 2 * e] - c.d[b + 2 * e]) * wx[b] * wy[e];
        }
      grad[i * 3] = gx / vs;
      grad[i * 3 + 1] = gy / vs;
      grad[i * 3 + 2] = gz / vs;
    }
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_query(const GridView& g, const int32_t* xyz, int64_t n, int32_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  VDB_LAUNCH(k_query, grid_for(n, 256), 256, 0, st, g, xyz, n, out);
  return cudaGetLastError();
}

cudaError_t launch_distance_at(const GridView& g, float vs, const float* pts, int64_t n, float* dist, float* grad,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  VDB_LAUNCH(k_distance_at, grid_for(n, 256), 256, 0, st, g, vs, pts, n, dist, grad);
  return cudaGetLastError();
}

cudaError_t launch_query_nearest(const GridView& g, const int32_t* xyz, int64_t n, int32_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = (size_t)g.INF + 1;  // at most 32,762 bytes (dmax <= 181)
  VDB_LAUNCH(k_query_nearest, grid_for(n, 128), 128, smem, st, g, xyz, n, out);
  return cudaGetLastError();
}

// Bricks holding an obstacle and bricks holding a finite D, counted on the device (counters
// C_OBST and C_FINITE, cleared by the caller): one atomic per warp and flag.
__global__ void k_count_flags(GridView g) {
  // counts kept per warp over the grid-stride loop, then one atomic per block and counter (the
  // two counters would otherwise take an atomic from every warp)
  __shared__ int wobst[32], wfin[32];
  const int nb = min(g.counters[C_NBRICKS], g.cap);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int obst = 0, fin = 0;
  for (int base = blockIdx.x * blockDim.x; base < nb; base += gridDim.x * blockDim.x) {
    const int s = base + threadIdx.x;
    const uint32_t f = s < nb ? g.bflags[s] : 0u;
    obst += __popc(__ballot_sync(0xffffffffu, (f & F_OBST) != 0u));
    fin += __popc(__ballot_sync(0xffffffffu, (f & F_FINITE) != 0u));
  }
  if (lane == 0) {
    wobst[warp] = obst;
    wfin[warp] = fin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int to = 0, tf = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      to += wobst[w];
      tf += wfin[w];
    }
    if (to) atomicAdd(&g.counters[C_OBST], to);
    if (tf) atomicAdd(&g.counters[C_FINITE], tf);
  }
}

cudaError_t launch_count_flags(const GridView& g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g.counters + C_FINITE, 0, 2 * sizeof(int32_t), st);  // C_FINITE, C_OBST
  if (e != cudaSuccess) return e;
  VDB_LAUNCH(k_count_flags, 304, 256, 0, st, g);
  return cudaGetLastError();
}

namespace {
// Occupancy of a z-range as packed records (x | y << 21 | (z + dz) << 42 | occ << 63): a warp per
// brick (stored bricks, or the bricks the last update changed), a lane per two voxel rows of one
// z-plane pair; records are appended with one atomic per warp per plane pair.  mode 0: occupied
// voxels only (occ = 1); mode 1: every voxel of the brick in the range, occupied or not.
__global__ void k_export_occupancy(GridView g, const int32_t* __restrict__ changed, int z_lo, int z_hi, int dz,
                                   int mode, unsigned long long* __restrict__ out, int64_t max_n,
                                   unsigned long long* __restrict__ count) {
  const int nb = mode == 0 ? min(g.counters[C_NBRICKS], g.cap) : min(g.counters[C_CHANGED], g.cap);
  const int lane = threadIdx.x & 31;
  const int nw = (int)gridDim.x * (int)(blockDim.x >> 5);
  for (int i = (int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); i < nb; i += nw) {
    const int slot = mode == 0 ? i : changed[i];
    const int4 c = g.bcoord[slot];
    const int bz0 = 8 * c.z;
    if (bz0 + 8 <= z_lo || bz0 >= z_hi) continue;  // warp-uniform
    for (int zz = 0; zz < 8; ++zz) {
      const int z = bz0 + zz;
      if (z < z_lo || z >= z_hi) continue;  // warp-uniform
      const unsigned long long word = g.occ[(size_t)slot * 8 + zz];  // bit x + 8 y
      // lane: bits 2 lane, 2 lane + 1 of the plane
      const int b0 = 2 * lane;
      const int e0 = (int)((word >> b0) & 1ull), e1 = (int)((word >> (b0 + 1)) & 1ull);
      // voxels of a brick that hangs over the grid's edge are not part of the grid
      const int y = 8 * c.y + (b0 >> 3), x0 = 8 * c.x + (b0 & 7);
      const bool in0 = x0 < g.nx && y < g.ny, in1 = x0 + 1 < g.nx && y < g.ny;
      const int k0 = (mode == 0 ? e0 : 1) & (int)in0, k1 = (mode == 0 ? e1 : 1) & (int)in1;
      const int mine = k0 + k1;
      int incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (total == 0) continue;
      unsigned long long base = 0;
      if (lane == 31) base = atomicAdd(count, (unsigned long long)total);
      base = __shfl_sync(0xffffffffu, base, 31);
      unsigned long long p = base + (unsigned long long)(incl - mine);
      for (int q = 0; q < 2; ++q) {
        if (!(q ? k1 : k0)) continue;
        if ((int64_t)p < max_n)
          out[p] = pack_rec(x0 + q, y, z + dz, q ? e1 : e0);
        ++p;
      }
    }
  }
}
}  // namespace

cudaError_t launch_export_occupancy(const GridView& g, const int32_t* changed, int z_lo, int z_hi, int dz, int mode,
                                    unsigned long long* out, int64_t max_n, unsigned long long* count,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  VDB_LAUNCH(k_export_occupancy, 152 * 8, 256, 0, st, g, changed, z_lo, z_hi, dz, mode, out, max_n, count);
  return cudaGetLastError();
}

cudaError_t launch_export_dense(const GridView& g, int32_t* out, cudaStream_t st) {
  int64_t n = (int64_t)g.nx * g.ny * g.nz;
  VDB_LAUNCH(k_export_dense, grid_for(n, 256), 256, 0, st, g, out);
  return cudaGetLastError();
}

cudaError_t launch_clearance_fwd(const GridView& g, float vs, const float* pts, int64_t T, int64_t P, float tau,
                                 float* cost, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  VDB_LAUNCH(k_clearance_fwd, grid_for(T * 32, 256), 256, 0, st, g, vs, pts, T, P, tau, cost);
  return cudaGetLastError();
}

cudaError_t launch_clearance_bwd(const GridView& g, float vs, const float* pts, int64_t T, int64_t P, float tau,
                                 const float* gcost, float* gpts, cudaStream_t st) {
  if (T <= 0 || P <= 0) return cudaSuccess;
  VDB_LAUNCH(k_clearance_bwd, grid_for(T * P, 256), 256, 0, st, g, vs, pts, T, P, tau, gcost, gpts);
  return cudaGetLastError();
}

}  // namespace vdbedt
