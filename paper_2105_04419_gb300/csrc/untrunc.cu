// Untruncated transform (VDBEDT_FLAG_UNTRUNCATED): Eq. 1 without the truncation, i.e. the exact
// squared distance to the nearest occupied voxel anywhere in a bounded grid (the paper's
// dmax = infinity runs, Table II).  With no truncation every voxel is in reach of every obstacle,
// so every brick is stored, brick (bx, by, bz) at slot bx + BX (by + BY bz), and the transform runs
// over whole lines of the grid, one axis after the other (Eq. 1's minimum taken per axis):
//   x: per row, the distance to the nearest occupied voxel on either side (a forward sweep that
//      keeps one carry per brick, and a backward sweep that writes g1 = dx^2);
//   y, z: per line, the lower envelope of the parabolas f(i) + (t - i)^2 rooted at the line's
//      finite values (g1, then g2): built on a stack in one sweep, read back in a second.  Two
//      parabolas are compared through their intersection with the denominators multiplied out,
//      exactly: the grid's size limit keeps every f(p) + p^2 below 2^31, so the differences are
//      int32 and each product one widening multiply (below 2^48).
// kNone marks a row, plane or grid without an obstacle.  Only voxels inside the grid are read or
// written; g1 and g2 hold int32 here (their arrays are allocated twice as large).
#include <algorithm>

#include "vdbedt_internal.cuh"

namespace vdbedt {
namespace {

constexpr int kUT = 256;

__device__ __forceinline__ int ut_slot(const GridView& g, int bx, int by, int bz) {
  return bx + g.BX * (by + g.BY * bz);
}

__device__ __forceinline__ int ut_vox(int x, int y, int z) { return (x & 7) + 8 * (y & 7) + 64 * (z & 7); }

// A line's stack in the scratch, interleaved with the other 31 lines of its group of 32 (entry m
// of line t at ((t >> 5) n + m) 32 + (t & 31)): lanes of a warp that push or pop at similar depths
// touch the same 32-byte sectors instead of 32 separate regions.
struct LineStack {
  int2* p;
  __device__ __forceinline__ LineStack(int2* stack, int64_t t, int n)
      : p(stack + (size_t)(t >> 5) * 32 * n + (size_t)(t & 31)) {}
  __device__ __forceinline__ int2& operator[](int m) const { return p[(size_t)m * 32]; }
};

unsigned ut_blocks(int64_t threads) {
  const int64_t b = (threads + kUT - 1) / kUT;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

// Interior nodes of every key of the grid (node indices in creation order).
__global__ void k_ut_nodes(GridView g) {
  const int64_t nk = (int64_t)g.NX * g.NY * g.NZ;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += (int64_t)gridDim.x * blockDim.x)
    get_or_create_node(g, (unsigned long long)k);
}

// Every brick of the grid at its fixed slot, with an empty occupancy.
__global__ void k_ut_bricks(GridView g) {
  const int64_t nb = (int64_t)g.BX * g.BY * g.BZ;
  if (blockIdx.x == 0 && threadIdx.x == 0) g.counters[C_NBRICKS] = (int)nb;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int bx = (int)(b % g.BX), r = (int)(b / g.BX), by = r % g.BY, bz = r / g.BY;
    const int node = find_node(g, node_key_of(g, bx, by, bz));
    if (node < 0) {
      set_error(g, kErrInternal);
      continue;
    }
    g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)] = (int)b;
    g.bcoord[b] = make_int4(bx, by, bz, node);
    g.bflags[b] = 0u;
    g.bepoch[b] = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) g.occ[(size_t)b * 8 + q] = 0ull;
  }
}

// Empty occupancy, flags and brick epochs; the counters start over except the stored bricks and
// nodes.
__global__ void k_ut_reset(GridView g) {
  const int64_t nb = (int64_t)g.BX * g.BY * g.BZ;
  if (blockIdx.x == 0 && (int)threadIdx.x < C_NUM && threadIdx.x != C_NBRICKS && threadIdx.x != C_NNODES)
    g.counters[threadIdx.x] = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb * 8; i += (int64_t)gridDim.x * blockDim.x) {
    g.occ[i] = 0ull;
    if ((i & 7) == 0) {
      g.bflags[i >> 3] = 0u;
      g.bepoch[i >> 3] = 0;  // the update epoch starts over with the counters
    }
  }
}

// Occupancy from a dense uint8 grid [nz][ny][nx] (nonzero = occupied): a thread per (brick,
// plane) assembles the plane's 64-bit word (bit x + 8 y) from eight rows of eight bytes.
__global__ void k_ut_dense(GridView g, const uint8_t* __restrict__ grid) {
  const int64_t nw = (int64_t)g.BX * g.BY * g.BZ * 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x) {
    // i = bx + BX (pz + 8 (by + BY bz)): neighbouring threads read neighbouring 8-byte row pieces
    const int bx = (int)(i % g.BX);
    const int64_t r = i / g.BX;
    const int pz = (int)(r & 7);
    const int64_t rb = r >> 3;
    const int by = (int)(rb % g.BY), bz = (int)(rb / g.BY);
    const int z = 8 * bz + pz;
    unsigned long long w = 0ull;
    if (z < g.nz) {
      for (int py = 0; py < 8; ++py) {
        const int y = 8 * by + py;
        if (y >= g.ny) break;
        const uint8_t* row = grid + ((size_t)z * g.ny + y) * g.nx;
        for (int px = 0; px < 8; ++px) {
          const int x = 8 * bx + px;
          if (x < g.nx && row[x]) w |= 1ull << (px + 8 * py);
        }
      }
    }
    g.occ[(size_t)ut_slot(g, bx, by, bz) * 8 + pz] = w;
  }
}

// x pass: a thread per voxel row (the 64 rows of a brick line on consecutive threads).  A forward
// sweep over the row's occupancy bytes stores, per brick, the last occupied voxel before the brick
// (-1: none) in `carry` (entry bx * rows + t, so that a warp's 32 rows share a 128-byte line); the
// backward sweep then knows, inside each brick, the nearest occupied voxel on the left (the
// brick's own bits at or below the voxel, else the carry) and on the right (followed as it goes),
// and writes g1 = d^2 (kNone: empty row) once per voxel.
// INCR (an update): only the rows whose dirty bit is set, each warp taking and clearing its word;
// the backward sweep compares each g1 with the stored one, writes the bricks' row pieces that
// changed and sets the y-line byte (x, z) of every changed voxel with a plain store.
template <bool INCR>
__global__ void k_ut_x(GridView g, int32_t* __restrict__ carry) {
  int32_t* __restrict__ g1 = reinterpret_cast<int32_t*>(g.g1);
  const int64_t nrows = (int64_t)g.BY * g.BZ * 64;  // a multiple of 64: every warp is whole
  const int lane = threadIdx.x & 31;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nrows; t += (int64_t)gridDim.x * blockDim.x) {
    if (INCR) {
      uint32_t w = 0u;
      if (lane == 0) {
        w = g.ut_bits[t >> 5];
        if (w) {
          g.ut_bits[t >> 5] = 0u;
          atomicAdd(&g.items_ctr[0], __popc(w));
        }
      }
      w = __shfl_sync(0xffffffffu, w, 0);
      if (!((w >> lane) & 1u)) continue;
    }
    const int64_t line = t >> 6;
    const int q = (int)(t & 63);
    const int by = (int)(line % g.BY), bz = (int)(line / g.BY);
    const int y = 8 * by + (q & 7), z = 8 * bz + (q >> 3);
    if (y >= g.ny || z >= g.nz) continue;
    const int shift = 8 * (y & 7);
    const size_t row = (size_t)(8 * (y & 7) + 64 * (z & 7));
    int last = -1;
    for (int bx = 0; bx < g.BX; ++bx) {
      carry[(size_t)bx * nrows + t] = last;
      const uint32_t byte = (uint32_t)(g.occ[(size_t)ut_slot(g, bx, by, bz) * 8 + (z & 7)] >> shift) & 0xFFu;
      if (byte) last = 8 * bx + 31 - __clz(byte);
    }
    int next = -1;
    uint8_t* yflag = INCR ? reinterpret_cast<uint8_t*>(g.ut_bits + ut_row_words(g)) + (size_t)ut_nxp(g) * z : nullptr;
    for (int bx = g.BX - 1; bx >= 0; --bx) {
      const int s = ut_slot(g, bx, by, bz);
      const uint32_t byte = (uint32_t)(g.occ[(size_t)s * 8 + (z & 7)] >> shift) & 0xFFu;
      const int left_in = carry[(size_t)bx * nrows + t];
      int4* dst = reinterpret_cast<int4*>(g1 + (size_t)s * kBrickVox + row);
      int v[8];
#pragma unroll
      for (int i = 7; i >= 0; --i) {
        const int x = 8 * bx + i;
        if ((byte >> i) & 1u) next = x;
        const uint32_t below = byte & ((2u << i) - 1u);  // occupied voxels of the brick at or left of x
        const int lpos = below ? 8 * bx + 31 - __clz(below) : left_in;
        int d = lpos >= 0 ? x - lpos : -1;
        if (next >= 0 && (d < 0 || next - x < d)) d = next - x;
        v[i] = (d < 0 || x >= g.nx) ? kNone : d * d;  // the last brick's padding holds kNone
      }
      if (INCR) {
        const int4 oa = dst[0], ob = dst[1];
        const int old[8] = {oa.x, oa.y, oa.z, oa.w, ob.x, ob.y, ob.z, ob.w};
        uint32_t ch = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (8 * bx + i < g.nx && v[i] != old[i]) ch |= 1u << i;
        if (ch) {
          dst[0] = make_int4(v[0], v[1], v[2], v[3]);
          dst[1] = make_int4(v[4], v[5], v[6], v[7]);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if ((ch >> i) & 1u) yflag[8 * bx + i] = 1;  // the rows of every y write the same y lines
        }
      } else {
        dst[0] = make_int4(v[0], v[1], v[2], v[3]);
        dst[1] = make_int4(v[4], v[5], v[6], v[7]);
      }
    }
  }
}

// Voxel i of line (x, c) along AXIS (1: y, c = z; 2: z, c = y) in a pool of bricks at fixed slots:
// base + (i >> 3) * brick stride + (i & 7) * voxel stride.
template <int AXIS>
struct LineAt {
  size_t base, bstride;
  __device__ __forceinline__ LineAt(const GridView& g, int x, int c) {
    base = AXIS == 1 ? (size_t)ut_slot(g, x >> 3, 0, c >> 3) * kBrickVox + ut_vox(x, 0, c)
                     : (size_t)ut_slot(g, x >> 3, c >> 3, 0) * kBrickVox + ut_vox(x, c, 0);
    bstride = (size_t)kBrickVox * (AXIS == 1 ? g.BX : (size_t)g.BX * g.BY);
  }
  __device__ __forceinline__ size_t operator()(int i) const {
    return base + (size_t)(i >> 3) * bstride + (size_t)((i & 7) * (AXIS == 1 ? 8 : 64));
  }
};

// Lower envelope of the parabolas f(i) + (t - i)^2 over the line's finite values, built on the
// line's stack: entries (p, F = f(p) + p^2), the top two also in registers.  The grid's size limit
// keeps every F below 2^31, so differences of F are int32 and each intersection test compares two
// widening 32 x 32 -> 64-bit products exactly.  The inputs are loaded a brick (8 positions) at a
// time, all eight before any is used.  Returns the entry count.
template <int AXIS>
__device__ __forceinline__ int env_build(const LineStack& st, const LineAt<AXIS>& at, const int32_t* __restrict__ in,
                                         int n) {
  int m = 0, p0 = 0, F0 = 0, p1 = 0, F1 = 0;
  for (int i0 = 0; i0 < n; i0 += 8) {
    int fv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) fv[j] = i0 + j < n ? in[at(i0 + j)] : kNone;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j;
      if (fv[j] == kNone) continue;
      const int Fi = fv[j] + i * i;
      while (m >= 2) {
        // drop the top when the new parabola undercuts it no later than the top undercuts the one
        // below: (Fi - F1) / (i - p1) <= (F1 - F0) / (p1 - p0)
        if ((long long)(Fi - F1) * (p1 - p0) > (long long)(F1 - F0) * (i - p1)) break;
        --m;
        p1 = p0;
        F1 = F0;
        if (m >= 2) {
          const int2 e = st[m - 2];
          p0 = e.x;
          F0 = e.y;
        }
      }
      st[m] = make_int2(i, Fi);
      p0 = p1;
      F0 = F1;
      p1 = i;
      F1 = Fi;
      ++m;
    }
  }
  return m;
}

// Reading an envelope back in increasing position: the lowest parabola only moves forward.
// Entries k, k + 1 and (loaded ahead) k + 2 in registers.
struct EnvRead {
  const LineStack& st;
  int m, k;
  int2 cur, nxt, ahead;
  __device__ __forceinline__ EnvRead(const LineStack& s, int count) : st(s), m(count), k(0) {
    cur = nxt = ahead = make_int2(0, 0);
    if (m > 0) {
      cur = st[0];
      nxt = m > 1 ? st[1] : cur;
      ahead = m > 2 ? st[2] : cur;
    }
  }
  // the envelope at i (i non-decreasing between calls); kNone for an empty envelope
  __device__ __forceinline__ int at(int i) {
    if (m == 0) return kNone;
    while (k + 1 < m) {
      // the next parabola is no higher at i: F(nxt) - F(cur) <= 2 i (nxt - cur)
      if ((long long)(nxt.y - cur.y) > (long long)(2 * i) * (nxt.x - cur.x)) break;
      ++k;
      cur = nxt;
      nxt = ahead;
      if (k + 2 < m) ahead = st[k + 2];
    }
    const int d = i - cur.x;
    return (cur.y - cur.x * cur.x) + d * d;  // f(p) + (i - p)^2
  }
};

// y (AXIS 1: g1 -> g2) or z (AXIS 2: g2 -> D) pass: a thread per line, lines (x, z) or (x, y)
// with x fastest, the line's stack in `stack` (LineStack).
template <int AXIS>
__global__ void k_ut_env(GridView g, const int32_t* __restrict__ in, int32_t* __restrict__ out, int2* __restrict__ stack) {
  const int n = AXIS == 1 ? g.ny : g.nz;
  const int64_t nlines = (int64_t)g.nx * (AXIS == 1 ? g.nz : g.ny);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nlines; t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % g.nx), c = (int)(t / g.nx);  // c: z (AXIS 1) or y (AXIS 2)
    const LineAt<AXIS> at(g, x, c);
    const LineStack st(stack, t, n);
    EnvRead env(st, env_build<AXIS>(st, at, in, n));
    for (int i = 0; i < n; ++i) out[at(i)] = env.at(i);
  }
}

// The update's y (AXIS 1) or z (AXIS 2) pass over the dirty lines: lines (x, c) with x padded to
// NXP, so that a warp's 32 lanes are 32 lines along x at one c and read 32 dirty-line bytes,
// cleared once read.  Each dirty lane builds its line's envelope as k_ut_env does and reads it
// back; the y pass writes the g2 values that changed and sets the z-line byte (x, y) of each.
// The z pass writes D on its dirty lines.
template <int AXIS>
__global__ void k_ut_env_upd(GridView g, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                             int2* __restrict__ stack) {
  const int n = AXIS == 1 ? g.ny : g.nz;
  const int nxp = ut_nxp(g);
  const int64_t nlines = (int64_t)nxp * (AXIS == 1 ? g.nz : g.ny);  // a multiple of 32
  uint8_t* yflag = reinterpret_cast<uint8_t*>(g.ut_bits + ut_row_words(g));
  uint8_t* zflag = reinterpret_cast<uint8_t*>(g.ut_bits + ut_row_words(g) + ut_yline_words(g));
  uint8_t* flag = AXIS == 1 ? yflag : zflag;  // this pass's dirty lines
  const int lane = threadIdx.x & 31;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nlines; t += (int64_t)gridDim.x * blockDim.x) {
    const bool f = flag[t] != 0;
    const uint32_t w = __ballot_sync(0xffffffffu, f);
    if (f) flag[t] = 0;
    if (!w) continue;  // warp-uniform
    if (lane == 0) atomicAdd(&g.items_ctr[AXIS], __popc(w));
    const bool dirty = (w >> lane) & 1u;  // set only for x < nx
    if (!dirty) continue;
    const int x = (int)(t % nxp), c = (int)(t / nxp);  // c: z (AXIS 1) or y (AXIS 2)
    const LineAt<AXIS> at(g, x, c);
    const LineStack st(stack, t, n);
    EnvRead env(st, env_build<AXIS>(st, at, in, n));
    for (int i = 0; i < n; ++i) {
      const int val = env.at(i);
      const size_t a = at(i);
      if (AXIS == 1) {
        if (out[a] != val) {
          out[a] = val;
          zflag[(size_t)nxp * i + x] = 1;
        }
      } else {
        out[a] = val;
      }
    }
  }
}

// Brick flags after the transform: obstacle bits, and finite D (voxel (0, 0, 0) of every brick lies
// inside the grid; with an obstacle anywhere every voxel is finite).
__global__ void k_ut_flags(GridView g) {
  const int64_t nb = (int64_t)g.BX * g.BY * g.BZ;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long any = 0ull;
#pragma unroll
    for (int q = 0; q < 8; ++q) any |= g.occ[(size_t)b * 8 + q];
    uint32_t f = any ? F_OBST : 0u;
    if (g.dist[(size_t)b * kBrickVox] != kNone) f |= F_FINITE | F_G2FIN | F_G1FIN;
    g.bflags[b] = f;
  }
}

}  // namespace

cudaError_t launch_ut_init(const GridView& g, cudaStream_t st) {
  VDB_LAUNCH(k_ut_nodes, ut_blocks((int64_t)g.NX * g.NY * g.NZ), kUT, 0, st, g);
  VDB_LAUNCH(k_ut_bricks, ut_blocks((int64_t)g.BX * g.BY * g.BZ), kUT, 0, st, g);
  return cudaGetLastError();
}

cudaError_t launch_ut_reset(const GridView& g, cudaStream_t st) {
  VDB_LAUNCH(k_ut_reset, ut_blocks((int64_t)g.BX * g.BY * g.BZ * 8), kUT, 0, st, g);
  return cudaGetLastError();
}

cudaError_t launch_ut_dense(const GridView& g, const uint8_t* grid, cudaStream_t st) {
  VDB_LAUNCH(k_ut_dense, ut_blocks((int64_t)g.BX * g.BY * g.BZ * 8), kUT, 0, st, g, grid);
  return cudaGetLastError();
}

// The line stacks (8 bytes per voxel of lines padded along x to a multiple of 32), or the x pass's
// carries (4 bytes per row and brick), whichever is larger.
size_t ut_scratch_bytes(const GridView& g) {
  return std::max((size_t)ut_nxp(g) * g.ny * g.nz * sizeof(int2), (size_t)g.BX * g.BY * g.BZ * 64 * sizeof(int32_t));
}

cudaError_t launch_ut_pass(const GridView& g, int axis, void* scratch, cudaStream_t st) {
  int32_t* g1 = reinterpret_cast<int32_t*>(g.g1);
  int32_t* g2 = reinterpret_cast<int32_t*>(g.g2);
  int2* stack = static_cast<int2*>(scratch);
  if (axis == 0) {
    VDB_LAUNCH(k_ut_x<false>, ut_blocks((int64_t)g.BY * g.BZ * 64), kUT, 0, st, g, static_cast<int32_t*>(scratch));
  } else if (axis == 1) {
    VDB_LAUNCH(k_ut_env<1>, ut_blocks((int64_t)g.nx * g.nz), kUT, 0, st, g, g1, g2, stack);
  } else {
    VDB_LAUNCH(k_ut_env<2>, ut_blocks((int64_t)g.nx * g.ny), kUT, 0, st, g, g2, g.dist, stack);
    VDB_LAUNCH(k_ut_flags, ut_blocks((int64_t)g.BX * g.BY * g.BZ), kUT, 0, st, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_ut_update_pass(const GridView& g, int axis, void* scratch, cudaStream_t st) {
  int32_t* g1 = reinterpret_cast<int32_t*>(g.g1);
  int32_t* g2 = reinterpret_cast<int32_t*>(g.g2);
  if (axis == 0) {
    VDB_LAUNCH(k_ut_x<true>, ut_blocks((int64_t)g.BY * g.BZ * 64), kUT, 0, st, g, static_cast<int32_t*>(scratch));
  } else if (axis == 1) {
    VDB_LAUNCH(k_ut_env_upd<1>, ut_blocks((int64_t)ut_nxp(g) * g.nz), kUT, 0, st, g, g1, g2, static_cast<int2*>(scratch));
  } else {
    VDB_LAUNCH(k_ut_env_upd<2>, ut_blocks((int64_t)ut_nxp(g) * g.ny), kUT, 0, st, g, g2, g.dist,
               static_cast<int2*>(scratch));
    VDB_LAUNCH(k_ut_flags, ut_blocks((int64_t)g.BX * g.BY * g.BZ), kUT, 0, st, g);
  }
  return cudaGetLastError();
}

}  // namespace vdbedt
