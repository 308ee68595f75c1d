// Building and maintaining the sparse brick grid on the device.
//
//   ingest (global form)  staged occupancy records -> brick keys of "set" records -> unique list
//            (one flag per brick of the grid, compacted with one atomic per warp, when records are
//            many; an LSD radix sort + unique + compaction when they are few) -> nodes created first
//            (one thread per flagged node key) -> bricks allocated (slots reserved with one
//            atomic per block) -> occupancy bits set (OR-ed into a dense mask during the count, or
//            per record).  Several records for one voxel: the last one wins -- a per-voxel
//            last-record table (atomicMax of the record index) picks it whenever a record clears a
//            voxel.
//   ingest (incremental form)  only the bricks of "set" records that are not stored yet are
//            appended to a list and allocated; every voxel's last record is applied through the
//            last-record table and each flip's brick joins the changed list once.
//   dense ingest  a whole occupancy grid -> per-brick masks in a scratch (sector-complete loads),
//            then nodes, then the occupied bricks.
//   activation  the compute set: every brick within Chebyshev brick radius R of a brick holding
//            an obstacle (the paper grows the tree only where the limited transform reaches,
//            Sec. IV-A): obstacle bits in per-node 4096-bit masks, halo nodes created, each node's
//            dilation computed from its 3 x 3 x 3 node neighbourhood, absent bricks allocated.
//   items    work lists for the passes: runs of bricks along x, y and z with their slot lists.
//   incremental marking  bricks whose occupancy changed -> their dilation (allocated) -> dirty
//            runs: x within R along x, in-plane within R in x and y, z within R in x, y and z.
//   batches  the per-grid kernels take a view source: one grid, or every grid of a batch with
//            block shares of one launch.
#include <cuda_fp16.h>

#include "vdbedt_internal.cuh"

namespace vdbedt {

namespace {

constexpr int kT = 256;

// Grid of a grid-stride kernel over n items: enough blocks to fill the GPU a few times over.
inline unsigned blocks_for(int64_t n, int t = kT) {
  int64_t b = (n + t - 1) / t;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)b;
}

inline int bits_for(uint64_t maxval) {
  int b = 1;
  while (b < 32 && (1ull << b) <= maxval) ++b;
  return b;
}

// View sources of the kernels that run once per grid.  get() returns the grid of the calling block
// and the block's index and count within that grid's share of the launch: a single grid (the view
// is a kernel parameter, the whole launch is its share), or every grid of a batch (views in device
// memory; grid i owns blocks first[i] .. first[i + 1] - 1 of a one-dimensional launch, shares sized
// to each grid's work, found by binary search).
struct OneView {
  GridView g;
  __device__ __forceinline__ GridView get(int& bid, int& nblk, int& grid) const {
    bid = blockIdx.x;
    nblk = gridDim.x;
    grid = 0;
    return g;
  }
  __device__ __forceinline__ bool skip(const GridView&) const { return false; }
};
struct BatchViews {
  const GridView* v;
  const int* first;  // [k + 1], first[k] = blocks of the launch
  int k;
  __device__ __forceinline__ GridView get(int& bid, int& nblk, int& grid) const {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = k;  // first[lo] <= b < first[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (first[mid] <= b) lo = mid; else hi = mid;
    }
    bid = b - first[lo];
    nblk = first[lo + 1] - first[lo];
    grid = lo;
    return v[lo];
  }
  __device__ __forceinline__ bool skip(const GridView&) const { return false; }
};
// The global form's activation and work-list kernels run inside an incremental update only for
// grids whose update switched to the global form (counters[C_BIG] set after the records were
// applied): one grid (the whole launch is its share), or grid blockIdx.y of a batch.
// An update's choice between its incremental and its global form (the marking would cost (2R + 1)^3
// brick visits per changed brick; beyond kBigUpdate visits per stored brick the global form's
// activation and work lists are cheaper -- measured crossover on the tunnel scene).  Taken from the
// changed-brick count, final once the records are applied, and the stored bricks when the update
// began, so that every kernel of the update, on either stream and at any time, decides alike.
__device__ __forceinline__ bool big_update(const GridView& g) {
  const int64_t nc = min(g.counters[C_CHANGED], g.cap), side = 2 * g.R + 1;
  return nc * side * side * side > (int64_t)kBigUpdate * max(g.counters[C_NB_START], 1);
}

struct GatedOne {
  GridView g;
  __device__ __forceinline__ GridView get(int& bid, int& nblk, int& grid) const {
    bid = blockIdx.x;
    nblk = gridDim.x;
    grid = 0;
    return g;
  }
  __device__ __forceinline__ bool skip(const GridView& v) const { return !big_update(v); }
};
struct GatedBatch {
  const UpdArgs* a;
  __device__ __forceinline__ GridView get(int& bid, int& nblk, int& grid) const {
    bid = blockIdx.x;
    nblk = gridDim.x;
    grid = (int)blockIdx.y;
    return a[blockIdx.y].g;
  }
  __device__ __forceinline__ bool skip(const GridView& v) const { return !big_update(v); }
};
struct OneSrc {
  const uint8_t* p;
  __device__ __forceinline__ const uint8_t* get(int) const { return p; }
};
struct BatchSrc {
  const uint8_t* p[kBatchMax];
  __device__ __forceinline__ const uint8_t* get(int grid) const { return p[grid]; }
};
// Argument sources of the incremental update's kernels: one grid, or the grid blockIdx.y of a batch.
struct UpdOne {
  UpdArgs a;
  __device__ __forceinline__ UpdArgs get() const { return a; }
};
struct UpdBatch {
  const UpdArgs* a;
  __device__ __forceinline__ UpdArgs get() const { return a[blockIdx.y]; }
};

// ---- reset ----
template <class VS>
__global__ void k_reset_nodes(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  (void)gi;
  // per used node: 4096 child slots, 3 x 1024 marks, 128 activity words and 384 work words, all
  // whole 16-byte vectors (the per-node arrays start at multiples of their node strides)
  const int64_t nn = min(g.counters[C_NNODES], g.node_cap);
  const int64_t stride = (int64_t)nblk * blockDim.x, t0 = (int64_t)bid * blockDim.x + threadIdx.x;
  const int4 none = make_int4(kNoSlot, kNoSlot, kNoSlot, kNoSlot), zero = make_int4(0, 0, 0, 0);
  for (int64_t i = t0; i < nn * (kNodeBricks / 4); i += stride) reinterpret_cast<int4*>(g.child)[i] = none;
  for (int64_t i = t0; i < nn * (3 * 1024 / 4); i += stride) reinterpret_cast<int4*>(g.mark)[i] = zero;
  for (int64_t i = t0; i < nn * (128 / 4); i += stride) reinterpret_cast<int4*>(g.amask)[i] = zero;
  for (int64_t i = t0; i < nn * (384 / 4); i += stride) reinterpret_cast<int4*>(g.mwork)[i] = zero;
  for (int64_t i = t0; i < nn * (128 / 4); i += stride) reinterpret_cast<int4*>(g.nclaim)[i] = zero;
  for (int64_t i = t0; i <= (int64_t)g.hmask; i += stride) g.hslots[i] = ~0ull;
}

// Start of an incremental update: clear the per-update counters and advance the update epoch
// (kept on the device, so that a captured update replays with a fresh epoch each time).  In a batch
// every grid's block clears the shared run counters (all store 0).
template <class US>
__global__ void k_begin_update(US us) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const GridView g = us.get().g;
    g.items_ctr[0] = 0;
    g.items_ctr[1] = 0;
    g.items_ctr[2] = 0;
    g.counters[C_CHANGED] = 0;
    g.counters[C_FLIPS] = 0;
    g.counters[C_NEW_BRICKS] = 0;
    g.counters[C_UNIQUE] = 0;
    g.counters[C_HAS_ZERO] = 0;
    g.counters[C_XB] = 0;
    g.counters[C_YB] = 0;
    g.counters[C_ZB] = 0;
    g.counters[C_BIG] = 0;
    g.counters[C_NB_START] = g.counters[C_NBRICKS];
    g.counters[C_EPOCH] += 1;
  }
}

// Batched form: the same, plus the record count of grids staged without a device count.
__global__ void k_begin_batch_update(const UpdArgs* __restrict__ args, BatchCounts counts) {
  pdl_enter();
  if (threadIdx.x == 0) {
    const int i = (int)blockIdx.y;
    const UpdArgs a = args[i];
    if (counts.c[i] >= 0) *const_cast<int32_t*>(a.n_dev) = counts.c[i];
    const GridView& g = a.g;
    g.items_ctr[0] = 0;
    g.items_ctr[1] = 0;
    g.items_ctr[2] = 0;
    g.counters[C_CHANGED] = 0;
    g.counters[C_FLIPS] = 0;
    g.counters[C_NEW_BRICKS] = 0;
    g.counters[C_UNIQUE] = 0;
    g.counters[C_HAS_ZERO] = 0;
    g.counters[C_XB] = 0;
    g.counters[C_YB] = 0;
    g.counters[C_ZB] = 0;
    g.counters[C_BIG] = 0;
    g.counters[C_NB_START] = g.counters[C_NBRICKS];
    g.counters[C_EPOCH] += 1;
  }
}

// ---- brick allocation ----
// Fill a freshly allocated brick: empty occupancy, coordinates, flags (no plane holds a value below
// dmax^2); with `init_fields` also g1, g2 and D at dmax^2 (bricks added by an incremental update may
// be read before a pass writes them).
__device__ __forceinline__ void init_brick_meta(const GridView& g, int slot, int node, int bx, int by, int bz) {
  g.bcoord[slot] = make_int4(bx, by, bz, node);
  g.bflags[slot] = 0u;
  g.bepoch[slot] = 0;
}

// dmax^2 twice in the 16-bit encoding of g1 / g2 (fp16 bits in the windowed form, integers else)
__device__ __forceinline__ uint32_t field_inf2(const GridView& g) {
  uint16_t inf;
  if (g.half) {
    __half h = __int2half_rn(g.INF);
    inf = *reinterpret_cast<uint16_t*>(&h);
  } else {
    inf = (uint16_t)g.INF;
  }
  return (uint32_t)inf | ((uint32_t)inf << 16);
}

// g1, g2 and D of `slot` at dmax^2, written by a whole warp (every lane passes the same slot): each
// store instruction covers 512 contiguous bytes.
__device__ __forceinline__ void init_fields_warp(const GridView& g, int slot, int lane) {
  const uint32_t p = field_inf2(g);
  const uint4 v = make_uint4(p, p, p, p);
  uint4* d1 = reinterpret_cast<uint4*>(g.g1 + (size_t)slot * kBrickVox);
  uint4* d2 = reinterpret_cast<uint4*>(g.g2 + (size_t)slot * kBrickVox);
  d1[lane] = v;
  d1[lane + 32] = v;
  d2[lane] = v;
  d2[lane + 32] = v;
  int4* dd = reinterpret_cast<int4*>(g.dist + (size_t)slot * kBrickVox);
  const int4 w = make_int4(g.INF, g.INF, g.INF, g.INF);
#pragma unroll
  for (int q = 0; q < 4; ++q) dd[lane + 32 * q] = w;
}

// The fields of the slots `ok` lanes hold, a brick at a time by the whole warp (warp-uniform call).
__device__ __forceinline__ void init_fields_ballot(const GridView& g, bool ok, int slot) {
  const int lane = threadIdx.x & 31;
  unsigned todo = __ballot_sync(0xffffffffu, ok);
  while (todo) {
    const int b = __ffs(todo) - 1;
    todo &= todo - 1u;
    init_fields_warp(g, __shfl_sync(0xffffffffu, slot, b), lane);
  }
}

__device__ void init_brick(const GridView& g, int slot, int node, int bx, int by, int bz, bool init_fields) {
  ulonglong2* occ = reinterpret_cast<ulonglong2*>(g.occ + (size_t)slot * 8);
#pragma unroll
  for (int q = 0; q < 4; ++q) occ[q] = make_ulonglong2(0ull, 0ull);
  if (init_fields) {
    const uint32_t p = field_inf2(g);
    uint4* dst = reinterpret_cast<uint4*>(g.g2 + (size_t)slot * kBrickVox);
    for (int q = 0; q < 64; ++q) dst[q] = make_uint4(p, p, p, p);
    uint4* d1 = reinterpret_cast<uint4*>(g.g1 + (size_t)slot * kBrickVox);
    for (int q = 0; q < 64; ++q) d1[q] = make_uint4(p, p, p, p);
    int4* dd = reinterpret_cast<int4*>(g.dist + (size_t)slot * kBrickVox);
    for (int q = 0; q < 128; ++q) dd[q] = make_int4(g.INF, g.INF, g.INF, g.INF);
  }
  init_brick_meta(g, slot, node, bx, by, bz);
}

__device__ __forceinline__ bool brick_has_obstacle(const GridView& g, int s) {
  const ulonglong2* w = reinterpret_cast<const ulonglong2*>(g.occ + (size_t)s * 8);
  ulonglong2 a = w[0], b = w[1], c = w[2], d = w[3];
  return (a.x | a.y | b.x | b.y | c.x | c.y | d.x | d.y) != 0ull;
}

// ---- record ingest ----
__device__ __forceinline__ bool rec_valid(const GridView& g, int4 r) {
  return (unsigned)r.x < (unsigned)g.nx && (unsigned)r.y < (unsigned)g.ny && (unsigned)r.z < (unsigned)g.nz &&
         (unsigned)r.w <= 1u;
}

// Block-wide aggregation: every thread of the block calls it; returns base + the thread's rank
// among the threads with `pred` (-1 without), after one atomicAdd of the block's total on ctr.
__device__ int block_agg_add(int* ctr, bool pred, int* block_total) {
  __shared__ int wsum[32];
  __shared__ int base_sh, tot_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = wsum[w];
      wsum[w] = t;
      t += c;
    }
    tot_sh = t;
    base_sh = t ? atomicAdd(ctr, t) : 0;
  }
  __syncthreads();
  const int r = pred ? base_sh + wsum[warp] + __popc(bal & ((1u << lane) - 1u)) : -1;
  if (block_total) *block_total = tot_sh;
  __syncthreads();
  return r;
}

// Number of staged records to apply: n, or the count in device memory (clamped to n) when the
// records were staged with a device-side count.
__device__ __forceinline__ int64_t rec_count(int64_t n, const int32_t* n_dev) {
  if (!n_dev) return n;
  const int64_t c = *n_dev;
  return c < 0 ? 0 : (c < n ? c : n);
}

// Grid-stride loops below keep every warp iterating together (the index base is block-uniform),
// so warp-wide votes and shuffles inside the loop see all 32 lanes.
#define GRID_STRIDE(i, n)                                                                              \
  for (int64_t i##_base = (int64_t)blockIdx.x * blockDim.x, i = i##_base + threadIdx.x; i##_base < (n); \
       i##_base += (int64_t)gridDim.x * blockDim.x, i = i##_base + threadIdx.x)

// Places for the lanes with `want` in a list counted by *ctr: one atomic per warp (warp-uniform
// call); returns the lane's place (meaningful where want).
// Sets a flag word that only ever goes from 0 to 1, reading it first (L2): once one warp has set
// it the others find it set and issue no atomic on the shared word.
__device__ __forceinline__ void set_once(int32_t* flag) {
  if (!__ldcg(flag)) atomicOr(flag, 1);
}

__device__ __forceinline__ int warp_reserve(int32_t* ctr, bool want) {
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (!m) return 0;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(ctr, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  return base + __popc(m & ((1u << lane) - 1u));
}

__global__ void k_rec_brick_keys(GridView g, const rec_t* __restrict__ rec, int64_t n, const int32_t* n_dev,
                                 uint32_t* __restrict__ keys) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t ne = rec_count(n, n_dev);  // keys past the count are the sentinel
  GRID_STRIDE(i, n) {
    uint32_t key = 0xFFFFFFFFu;
    bool zero = false, bad = false;
    if (i < ne) {
      int4 r = unpack_rec(rec[i]);
      if (!rec_valid(g, r)) {
        bad = true;
      } else if (r.w == 1) {
        key = (uint32_t)((r.x >> 3) + g.BX * ((r.y >> 3) + g.BY * (r.z >> 3)));
      } else {
        zero = true;
      }
    }
    // drop a key equal to the previous lane's (records of one brick tend to be adjacent)
    uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    if (lane > 0 && prev == key) key = 0xFFFFFFFFu;
    if (i < n) keys[i] = key;
    if (__any_sync(0xffffffffu, zero) && lane == 0) set_once(&g.counters[C_HAS_ZERO]);
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(g, kErrInvalidRecord);
  }
}

// Many records: bucket the brick keys of "set" records through one flag per brick of the grid; the
// compaction of the flags is the unique key list.
// With `dbits` (global form), the records' bits are also OR-ed into a dense mask of every brick of
// the grid (64 B per brick; lanes of one x-row merged by a segmented OR), so that allocation can copy
// each new brick's mask whole instead of a second pass over the records.
// One record of the counting-path mark (all lanes of the warp call it together).  The brick flag
// is only ever set, by the first lane of each run of records in one brick, without reading it
// first (no dependent load); the node flags follow from the compacted bricks.
__device__ __forceinline__ void mark_record(const GridView& g, bool have, rec_t packed, int lane,
                                            int32_t* __restrict__ flag, unsigned long long* __restrict__ dbits) {
  bool zero = false, bad = false;
  uint32_t widx = 0xFFFFFFFFu;  // mask word index lb * 8 + z, or none
  uint32_t blo = 0u, bhi = 0u;  // bit x + 8 y of that word, as two halves
  long long lb = -1;            // brick of a "set" record
  if (have) {
    int4 r = unpack_rec(packed);
    if (!rec_valid(g, r)) {
      bad = true;
    } else if (r.w == 1) {
      lb = (r.x >> 3) + (int64_t)g.BX * ((r.y >> 3) + (int64_t)g.BY * (r.z >> 3));
      if (dbits) {
        widx = (uint32_t)(lb * 8 + (r.z & 7));
        const int bit = (r.x & 7) + 8 * (r.y & 7);
        if (bit < 32) blo = 1u << bit; else bhi = 1u << (bit - 32);
      }
    } else {
      zero = true;
    }
  }
  const long long lb_prev = __shfl_up_sync(0xffffffffu, lb, 1);
  if (lb >= 0 && (lane == 0 || lb_prev != lb)) flag[lb] = 1;
  if (dbits) {
    // lanes hitting the same word OR their bits over up to 8 lanes back (runs of equal words are
    // short: records of one x-row are adjacent); the last lane of each run, and every 8th lane of
    // a longer run, issues the atomic
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const uint32_t wp = __shfl_up_sync(0xffffffffu, widx, o);
      const uint32_t lp = __shfl_up_sync(0xffffffffu, blo, o);
      const uint32_t hp = __shfl_up_sync(0xffffffffu, bhi, o);
      if (lane >= o && wp == widx) {
        blo |= lp;
        bhi |= hp;
      }
    }
    const uint32_t wprev = __shfl_up_sync(0xffffffffu, widx, 1);
    const uint32_t wnext = __shfl_down_sync(0xffffffffu, widx, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || wprev != widx);
    const unsigned upto = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
    const int start = 31 - __clz(heads & upto);
    const bool run_end = lane == 31 || wnext != widx;
    if (widx != 0xFFFFFFFFu && (run_end || ((lane - start) & 7) == 7))
      atomicOr(dbits + widx, ((unsigned long long)bhi << 32) | blo);
  }
  if (__any_sync(0xffffffffu, zero) && lane == 0) set_once(&g.counters[C_HAS_ZERO]);
  if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(g, kErrInvalidRecord);
}

__global__ void k_mark_record_bricks(GridView g, const rec_t* __restrict__ rec, int64_t n_max, const int32_t* n_dev,
                                     int32_t* __restrict__ flag, unsigned long long* __restrict__ dbits) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t n = rec_count(n_max, n_dev);
  // kMarkRecs records per thread and iteration, all loaded before any is used (the loop bounds are
  // uniform over the grid, so the warp-wide steps see all 32 lanes); 8 measured no faster than 4
  constexpr int kMarkRecs = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += kMarkRecs * stride) {
    rec_t r[kMarkRecs];
#pragma unroll
    for (int k = 0; k < kMarkRecs; ++k) {
      const int64_t i = base + k * stride + threadIdx.x;
      r[k] = i < n ? __ldg(rec + i) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kMarkRecs; ++k)
      if (base + k * stride < n) mark_record(g, base + k * stride + threadIdx.x < n, r[k], lane, flag, dbits);
  }
}

// A node absent from the table and inserted by exactly one thread, at index idx: its key, then a
// hash slot claimed with the final word (read by later kernels: the kernel boundary orders both).
__device__ void insert_new_node(const GridView& g, unsigned long long key, int idx) {
  if (idx >= g.node_cap) {
    set_error(g, kErrNodeOverflow);
    return;
  }
  g.node_key[idx] = (long long)key;
  const unsigned long long word = (key << kIndexBits) | (uint32_t)idx;
  uint32_t h = hash_key(key) & g.hmask;
  bool placed = false;
  for (uint32_t probe = 0; probe <= g.hmask && !placed; ++probe) {
    placed = atomicCAS(&g.hslots[h], kEmptySlot, word) == kEmptySlot;
    h = (h + 1) & g.hmask;
  }
  if (!placed) set_error(g, kErrNodeOverflow);
}

// Nodes of the obstacle bricks, created before the bricks so that no brick allocation waits on a
// node insertion in progress: one thread per flagged node key absent from the table; indices come
// from one atomic per block, and each key (inserted by exactly one thread) claims an empty hash
// slot with its final word.  Later kernels read the nodes (the kernel boundary orders them).
__device__ __forceinline__ void create_flagged_nodes(const GridView& g, int32_t* __restrict__ nflag, int64_t nkeys) {
  GRID_STRIDE(k, nkeys) {
    bool need = false;
    if (k < nkeys && nflag[k]) {
      nflag[k] = 0;
      need = find_node(g, (unsigned long long)k) < 0;
    }
    const int idx = block_agg_add(&g.counters[C_NNODES], need, nullptr);
    if (need) insert_new_node(g, (unsigned long long)k, idx);
  }
}

__global__ void k_create_flagged_nodes(GridView g, int32_t* __restrict__ nflag, int64_t nkeys) {
  pdl_enter();
  create_flagged_nodes(g, nflag, nkeys);
}

// Node flags of the unique brick keys (radix path).
__global__ void k_flag_key_nodes(GridView g, const uint32_t* __restrict__ uniq, int64_t n, int32_t* __restrict__ nflag) {
  pdl_enter();
  const int64_t cnt = min((int64_t)g.counters[C_UNIQUE], n);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t lb = uniq[j];
    const int bx = (int)(lb % (uint32_t)g.BX), rest = (int)(lb / (uint32_t)g.BX);
    nflag[node_key_of(g, bx, rest % g.BY, rest / g.BY)] = 1;
  }
}

// Compaction of the flagged bricks, one atomic per block for the list positions (a block's bricks
// stay in key order, blocks follow in completion order; one counter word takes about a thousand
// atomics instead of one per warp holding a flagged brick), with the flags of their node keys:
// consecutive bricks mostly share a node, so only the first flagged lane of each run of one node
// key in the warp sets it (without reading it first).
__global__ void k_compact_flag_index(GridView g, const int32_t* __restrict__ flag, int64_t n,
                                     uint32_t* __restrict__ out, int32_t* __restrict__ nflag) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  GRID_STRIDE(i, n) {
    int nk = -1;
    if (i < n && flag[i]) {
      const uint32_t lb = (uint32_t)i, rest = lb / (uint32_t)g.BX;
      nk = (int)node_key_of(g, (int)(lb - rest * (uint32_t)g.BX), (int)(rest % (uint32_t)g.BY),
                            (int)(rest / (uint32_t)g.BY));
    }
    const unsigned set = __ballot_sync(0xffffffffu, nk >= 0);
    const int pos = block_agg_add(&g.counters[C_UNIQUE], nk >= 0, nullptr);  // block-uniform call
    const unsigned below = set & ((1u << lane) - 1u);
    if (nk >= 0) out[pos] = (uint32_t)i;
    const int prev_lane = 31 - __clz(below);  // previous flagged lane, or -1
    const int nk_prev = __shfl_sync(0xffffffffu, nk, prev_lane < 0 ? lane : prev_lane);
    if (nk >= 0 && (prev_lane < 0 || nk_prev != nk)) nflag[nk] = 1;
  }
}

__global__ void k_head_flags(const uint32_t* __restrict__ keys, int64_t n, uint32_t limit, int32_t* __restrict__ flag) {
  pdl_enter();
  GRID_STRIDE(i, n) {
    if (i < n) {
      uint32_t k = keys[i];
      flag[i] = (k < limit && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
  }
}

__global__ void k_compact_keys(const uint32_t* __restrict__ keys, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ pos, int64_t n, uint32_t* __restrict__ out) {
  pdl_enter();
  GRID_STRIDE(i, n) {
    if (i < n && flag[i]) out[pos[i]] = keys[i];
  }
}

// Bricks of the unique keys: node found or inserted, slot reserved with one atomic per block.
__global__ void k_alloc_obstacle_bricks(GridView g, const uint32_t* __restrict__ uniq, int64_t n, bool init,
                                        const unsigned long long* __restrict__ dbits) {
  pdl_enter();
  const int64_t cnt = min((int64_t)g.counters[C_UNIQUE], n);
  GRID_STRIDE(j, cnt) {
    int bx = 0, by = 0, bz = 0, node = -1;
    int* e = nullptr;
    bool need = false;
    uint32_t lb = 0;
    if (j < cnt) {
      lb = uniq[j];
      bx = (int)(lb % (uint32_t)g.BX);
      int rest = (int)(lb / (uint32_t)g.BX);
      by = rest % g.BY;
      bz = rest / g.BY;
      node = get_or_create_node(g, node_key_of(g, bx, by, bz));
      if (node >= 0) {
        e = &g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)];
        need = *e == kNoSlot;
      }
    }
    int total = 0;
    const int slot = block_agg_add(&g.counters[C_NBRICKS], need, &total);
    const ulonglong2* src = dbits ? reinterpret_cast<const ulonglong2*>(dbits + (size_t)lb * 8) : nullptr;
    if (need) {
      if (slot >= g.cap) {
        set_error(g, kErrOverflow);
      } else {
        if (dbits) {  // a new brick takes the records' mask as it is (the dense mask path is untracked)
          init_brick_meta(g, slot, node, bx, by, bz);
          ulonglong2* dst = reinterpret_cast<ulonglong2*>(g.occ + (size_t)slot * 8);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = src[q];
        } else {
          init_brick(g, slot, node, bx, by, bz, init);
        }
        *e = slot;
      }
    } else if (dbits && j < cnt && e) {  // a stored brick ORs the records' mask in
      const int sl = *e;
      if (sl >= 0 && sl < g.cap) {
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(g.occ + (size_t)sl * 8);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ulonglong2 a = src[q], b = dst[q];
          dst[q] = make_ulonglong2(a.x | b.x, a.y | b.y);
        }
      }
    }
    if (threadIdx.x == 0 && total) atomicAdd(&g.counters[C_NEW_BRICKS], total);
  }
}

// All records set voxels: OR the bits in.  Adjacent lanes that hit the same 64-bit word (records
// of one x-row usually sit next to each other) are merged by a segmented OR over the warp, and the
// last lane of each segment issues the atomic.
__global__ void k_apply_set_only(GridView g, const rec_t* __restrict__ rec, int64_t n_max, const int32_t* n_dev) {
  pdl_enter();
  if (g.counters[C_HAS_ZERO]) return;
  const int lane = threadIdx.x & 31;
  const int64_t n = rec_count(n_max, n_dev);
  GRID_STRIDE(i, n) {
    unsigned long long word = 0ull;  // address of the target word, 0 for none
    unsigned long long bits = 0ull;
    if (i < n) {
      int4 r = unpack_rec(rec[i]);
      if (rec_valid(g, r) && r.w == 1) {
        int s = find_brick(g, r.x >> 3, r.y >> 3, r.z >> 3);
        if (s >= 0) {
          word = (unsigned long long)(&g.occ[(size_t)s * 8 + (r.z & 7)]);
          bits = 1ull << ((r.x & 7) + 8 * (r.y & 7));
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long wp = __shfl_up_sync(0xffffffffu, word, o);
      const unsigned long long bp = __shfl_up_sync(0xffffffffu, bits, o);
      if (lane >= o && wp == word) bits |= bp;
    }
    const unsigned long long wn = __shfl_down_sync(0xffffffffu, word, 1);
    if (word && (lane == 31 || wn != word)) atomicOr(reinterpret_cast<unsigned long long*>(word), bits);
  }
}

// Tracked ingest (incremental form), first kernel: each record's brick slot for the ordered
// kernels (rslot).  A "set" record whose brick is not stored yet creates the brick's interior node
// when it is missing (inline, as the marking kernel does) and claims the brick with a per-node bit
// (`nclaim`, the amask layout); the claiming thread allocates the brick (slots reserved a warp at a
// time, fields at dmax^2 written by the whole warp) and publishes its slot in the child table.
// Records that lose the claim, or read the child table before the claimer publishes, look the
// brick up again in the next kernel (rslot -2).  The claimer's record keeps -3 - slot, so that the
// next kernel, when no record of this ingest tests the bit any more, clears it: `nclaim` is zero
// between updates.  Records of stored bricks need no brick work at all.
template <class US>
__global__ void k_rec_slots(US us) {
  pdl_enter();
  const UpdArgs A = us.get();
  const GridView& g = A.g;
  const int lane = threadIdx.x & 31;
  const int64_t n = rec_count(A.n, A.n_dev);
  const rec_t* __restrict__ rec = A.rec;
  GRID_STRIDE(i, n) {  // block-uniform rounds: the warp-wide steps below see all 32 lanes
    bool zero = false, bad = false, claim = false;
    int rs = -1;  // the record's brick slot (-2: looked up once allocated)
    int node = -1, bx = 0, by = 0, bz = 0;
    if (i < n) {
      int4 r = unpack_rec(rec[i]);
      if (!rec_valid(g, r)) {
        bad = true;
      } else if (r.w == 1) {
        bx = r.x >> 3;
        by = r.y >> 3;
        bz = r.z >> 3;
        node = get_or_create_node(g, node_key_of(g, bx, by, bz));
        rs = -2;
        if (node >= 0) {
          const int l = local_brick(bx, by, bz);
          const int sl = g.child[(size_t)node * kNodeBricks + l];
          if (sl >= 0) {
            rs = sl;
          } else {
            const uint32_t b = 1u << (l & 31);
            claim = (atomicOr(&g.nclaim[(size_t)node * 128 + (l >> 5)], b) & b) == 0u;
          }
        }
      } else {
        zero = true;
        // a cleared voxel matters only in a stored brick: one stored now, or one a "set" record of
        // the same ingest adds (looked up again once it is published)
        rs = find_brick(g, r.x >> 3, r.y >> 3, r.z >> 3);
        if (rs < 0) rs = -2;
      }
    }
    const int slot = warp_reserve(&g.counters[C_NBRICKS], claim);
    const bool ok = claim && slot < g.cap;
    if (claim && !ok) {
      set_error(g, kErrOverflow);  // more bricks than the capacity holds: give the claim back
      const int l = local_brick(bx, by, bz);
      atomicAnd(&g.nclaim[(size_t)node * 128 + (l >> 5)], ~(1u << (l & 31)));
    }
    if (ok) init_brick(g, slot, node, bx, by, bz, false);
    init_fields_ballot(g, ok, slot);
    if (ok) {
      g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)] = slot;
      rs = -3 - slot;
    }
    const unsigned made = __ballot_sync(0xffffffffu, ok);
    if (lane == 0 && made) atomicAdd(&g.counters[C_NEW_BRICKS], __popc(made));
    if (i < n) A.rslot[i] = rs;
    if (__any_sync(0xffffffffu, zero) && lane == 0) set_once(&g.counters[C_HAS_ZERO]);
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(g, kErrInvalidRecord);
  }
}

// Ordered path: the last record of each voxel decides its bit.  vlast holds, per voxel of the
// pool (slot * 512 + voxel in brick), the highest index of a record for it (-1 when none): the
// first kernel raises it with atomicMax, the second applies each voxel's winning record and puts
// the entry back to -1, so vlast is all -1 between ingests.  Both run only when some record
// clears a voxel, or when flips are tracked.
// voxel index of a record inside its brick
__device__ __forceinline__ int rec_in_brick(rec_t packed) {
  const int4 r = unpack_rec(packed);
  return (r.x & 7) + 8 * (r.y & 7) + 64 * (r.z & 7);
}

__device__ __forceinline__ int64_t rec_voxel(const GridView& g, rec_t packed) {
  const int4 r = unpack_rec(packed);
  if (!rec_valid(g, r)) return -1;
  const int s = find_brick(g, r.x >> 3, r.y >> 3, r.z >> 3);
  if (s < 0) return -1;
  return (int64_t)s * 512 + ((r.x & 7) + 8 * (r.y & 7) + 64 * (r.z & 7));
}

__device__ __forceinline__ void rec_last(const GridView& g, const rec_t* __restrict__ rec, int64_t n_max,
                                         const int32_t* n_dev, bool force, int32_t* __restrict__ vlast) {
  if (!force && !g.counters[C_HAS_ZERO]) return;
  const int64_t n = rec_count(n_max, n_dev);
  GRID_STRIDE(i, n) {
    if (i < n) {
      const int64_t key = rec_voxel(g, rec[i]);
      if (key >= 0) atomicMax(&vlast[key], (int)i);
    }
  }
}

// Flips are counted; with `track` the brick is appended once per epoch to the changed list.
__device__ __forceinline__ void apply_last(const GridView& g, const rec_t* __restrict__ rec, int64_t n_max,
                                           const int32_t* n_dev, bool force, bool track, int32_t* __restrict__ vlast,
                                           int32_t* __restrict__ changed, const int32_t* __restrict__ rslot = nullptr) {
  if (!force && !g.counters[C_HAS_ZERO]) return;
  const int64_t n = rec_count(n_max, n_dev);
  const int epoch = g.counters[C_EPOCH];
  GRID_STRIDE(j, n) {
    bool flip = false, first = false;
    int slot = 0;
    if (j < n) {
      const rec_t packed = rec[j];
      int64_t key;
      if (rslot) {
        const int sl = rslot[j];
        key = sl >= 0 ? (int64_t)sl * 512 + rec_in_brick(packed) : -1;
      } else {
        key = rec_voxel(g, packed);
      }
      if (key >= 0 && vlast[key] == (int)j) {
        vlast[key] = -1;
        const int s = (int)(key >> 9), v = (int)(key & 511);
        const unsigned long long bit = 1ull << (v & 63);
        unsigned long long* word = &g.occ[(size_t)s * 8 + (v >> 6)];
        const bool cur = (*word & bit) != 0ull;
        if (cur != ((packed >> 63) != 0ull)) {
          atomicXor(word, bit);
          flip = true;
          first = track && atomicExch(&g.bepoch[s], epoch) != epoch;
          slot = s;
          if (track && g.ut_bits) {
            // untruncated grid (brick s at bx + BX (by + BY bz)): the voxel's x row is dirty
            const int64_t row = (int64_t)(s / g.BX) * 64 + (v >> 3);
            atomicOr(&g.ut_bits[row >> 5], 1u << (row & 31));
          }
        }
      }
    }
    // the changed list: each brick once per epoch, a block's bricks with one atomic (as the flip
    // count): the counter words see one atomic per block, not one per warp
    const int p = block_agg_add(&g.counters[C_CHANGED], first, nullptr);
    if (first) changed[p] = slot;
    block_agg_add(&g.counters[C_FLIPS], flip, nullptr);
  }
}

__global__ void k_rec_last(GridView g, const rec_t* __restrict__ rec, int64_t n_max, const int32_t* n_dev, bool force,
                           int32_t* __restrict__ vlast) {
  pdl_enter();
  rec_last(g, rec, n_max, n_dev, force, vlast);
}

__global__ void k_apply_last(GridView g, const rec_t* __restrict__ rec, int64_t n_max, const int32_t* n_dev,
                             bool force, bool track, int32_t* __restrict__ vlast, int32_t* __restrict__ changed) {
  pdl_enter();
  apply_last(g, rec, n_max, n_dev, force, track, vlast, changed);
}

// The tracked forms (incremental update): every record, flips tracked, each record's brick slot
// taken from the first ingest kernel (looked up here only for bricks allocated since).
template <class US>
__global__ void k_upd_rec_last(US us) {
  pdl_enter();
  const UpdArgs A = us.get();
  const GridView& g = A.g;
  const int64_t n = rec_count(A.n, A.n_dev);
  GRID_STRIDE(i, n) {
    if (i < n) {
      const rec_t packed = A.rec[i];
      int s = A.rslot[i];
      if (s <= -3) {
        // the record that allocated its brick: the claim bit goes back to zero
        s = -3 - s;
        const int4 c = g.bcoord[s];
        const int l = local_brick(c.x, c.y, c.z);
        atomicAnd(&g.nclaim[(size_t)c.w * 128 + (l >> 5)], ~(1u << (l & 31)));
        A.rslot[i] = s;
      } else if (s == -2) {
        const int4 r = unpack_rec(packed);
        s = find_brick(g, r.x >> 3, r.y >> 3, r.z >> 3);
        A.rslot[i] = s;
      }
      if (s >= 0) atomicMax(&A.vlast[(int64_t)s * 512 + rec_in_brick(packed)], (int)i);
    }
  }
}

template <class US>
__global__ void k_upd_apply_last(US us) {
  pdl_enter();
  const UpdArgs A = us.get();
  apply_last(A.g, A.rec, A.n, A.n_dev, true, true, A.vlast, A.changed, A.rslot);
}

// ---- dense ingest ----
// Two streaming passes.  (1) Masks: one warp per brick row (below) writes each brick's eight mask
// words into a plane-major scratch, with one flag per brick and one per node key.  (2) After the
// flagged nodes are created, one thread per brick of the grid allocates the occupied bricks (slots
// reserved with one atomic per block) and copies their masks in.  The grid was reset just before,
// so every brick is new; brick fields are left for the global transform that always follows a
// dense ingest.

// Bit i set when byte i of w is nonzero: the high bit of (low seven bits + 0x7F) | byte marks a
// nonzero byte, and one multiply gathers the four marks (bits 7, 15, 23, 31 land on 28 .. 31
// without overlapping any other partial product).
__device__ __forceinline__ uint32_t nonzero4(uint32_t w) {
  const uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
  return (t * 0x00204081u) >> 28;
}

// Scratch of the dense ingest: masks (8 words per brick of the grid, plane-major: plane z of brick
// lb at dbits[z * bricks + lb]), brick flags, node-key flags.
// A single grid's pointers are its own; grid i of a batch adds off[3i], off[3i + 1], off[3i + 2].
struct DenseScratch {
  unsigned long long* dbits;
  int32_t* flag;
  int32_t* nflag;
  const int64_t* off;  // nullptr for a single grid
  __device__ __forceinline__ void at(int gi, unsigned long long*& d, int32_t*& f, int32_t*& nf) const {
    d = dbits;
    f = flag;
    nf = nflag;
    if (off) {
      d += off[3 * gi];
      f += off[3 * gi + 1];
      nf += off[3 * gi + 2];
    }
  }
};

// Pass 1: one warp per unit (a brick row: by, bz and up to kDenseX bricks along x).  The unit's
// 64 input rows form eight contiguous stretches (one per plane z); each lane loads 16 bytes (two
// bricks) of each row, a plane's eight loads issued together, and assembles both bricks' mask word
// of that plane in registers -- no shared memory, no block barrier -- and stores it to the
// plane-major scratch (a warp's stores are one contiguous run).  After the eight planes a lane
// writes its two bricks' flags and marks their nodes.
constexpr int kDenseX = 64;

template <class VS, class SRC>
__global__ void __launch_bounds__(256, 4) k_dense_masks(VS vs, SRC src, DenseScratch ds) {
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  const uint8_t* __restrict__ grid = src.get(gi);
  unsigned long long* dbits;
  int32_t* flag;
  int32_t* nflag;
  ds.at(gi, dbits, flag, nflag);
  const int64_t nbr = (int64_t)g.BX * g.BY * g.BZ;
  const uint32_t nch = (uint32_t)(g.BX + kDenseX - 1) / kDenseX;
  const uint32_t nunits = nch * (uint32_t)g.BY * (uint32_t)g.BZ;
  const int lane = threadIdx.x & 31;
  const bool v16 = (g.nx % 16) == 0 && (reinterpret_cast<uintptr_t>(grid) & 15u) == 0;
  const bool v8 = (g.nx % 8) == 0 && (reinterpret_cast<uintptr_t>(grid) & 7u) == 0;
  const uint32_t nw = (uint32_t)nblk * (blockDim.x >> 5);
  for (uint32_t u = (uint32_t)bid * (blockDim.x >> 5) + (threadIdx.x >> 5); u < nunits; u += nw) {
    const int ch = (int)(u % nch);
    const uint32_t rest = u / nch;
    const int by = (int)(rest % (uint32_t)g.BY), bz = (int)(rest / (uint32_t)g.BY);
    const int bx0 = ch * kDenseX, nbx = min(kDenseX, g.BX - bx0);
    const int j = 2 * lane;  // this lane: bricks j and j + 1 of the chunk
    if (j >= nbx) continue;  // lanes past the row's end (the warp has no collective below)
    const bool two = j + 1 < nbx;
    const int x0 = (bx0 + j) * 8;
    const int nrow = min(8, g.ny - by * 8), nplane = min(8, g.nz - bz * 8);
    const uint8_t* base = grid + ((size_t)bz * 8 * g.ny + (size_t)by * 8) * g.nx + x0;
    const size_t zstride = (size_t)g.ny * g.nx;
    const int64_t lb = (bx0 + j) + (int64_t)g.BX * (by + (int64_t)g.BY * bz);
    unsigned long long any0 = 0ull, any1 = 0ull;
#pragma unroll 2
    for (int z = 0; z < 8; ++z) {
      const uint8_t* pl = base + (size_t)z * zstride;
      const int nr = z < nplane ? nrow : 0;
      uint32_t m[8];  // row y: bits 0-7 brick j, bits 8-15 brick j + 1
      if (v16) {  // nx a multiple of 16: bricks come in whole pairs
        uint4 w[8];
#pragma unroll
        for (int y = 0; y < 8; ++y)
          w[y] = y < nr ? __ldg(reinterpret_cast<const uint4*>(pl + (size_t)y * g.nx)) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int y = 0; y < 8; ++y)
          m[y] = nonzero4(w[y].x) | (nonzero4(w[y].y) << 4) | (nonzero4(w[y].z) << 8) | (nonzero4(w[y].w) << 12);
      } else if (v8) {
        uint2 lo[8], hi[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          lo[y] = y < nr ? __ldg(reinterpret_cast<const uint2*>(pl + (size_t)y * g.nx)) : make_uint2(0u, 0u);
          hi[y] = y < nr && two ? __ldg(reinterpret_cast<const uint2*>(pl + (size_t)y * g.nx + 8)) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int y = 0; y < 8; ++y)
          m[y] = nonzero4(lo[y].x) | (nonzero4(lo[y].y) << 4) | (nonzero4(hi[y].x) << 8) | (nonzero4(hi[y].y) << 12);
      } else {  // ragged rows: byte loads
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          uint32_t v = 0u;
          if (y < nr)
            for (int x = 0; x < 16 && x0 + x < g.nx && (x < 8 || two); ++x) v |= (uint32_t)(pl[(size_t)y * g.nx + x] != 0) << x;
          m[y] = v;
        }
      }
      unsigned long long a = 0ull, b = 0ull;
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        a |= (unsigned long long)(m[y] & 0xffu) << (8 * y);
        b |= (unsigned long long)(m[y] >> 8) << (8 * y);
      }
      unsigned long long* plane = dbits + (size_t)z * nbr;
      plane[lb] = a;
      if (two) plane[lb + 1] = b;
      any0 |= a;
      any1 |= b;
    }
    const int bx = bx0 + j;
    flag[lb] = any0 != 0ull;
    if (any0) nflag[node_key_of(g, bx, by, bz)] = 1;
    if (two) {
      flag[lb + 1] = any1 != 0ull;
      if (any1) nflag[node_key_of(g, bx + 1, by, bz)] = 1;
    }
  }
}

// Nodes of flagged keys, one thread per key (each key inserted by exactly one thread; indices come
// from one atomic per block): no insertion ever waits on another.
template <class VS>
__global__ void __launch_bounds__(256) k_dense_nodes(VS vs, DenseScratch ds) {
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  unsigned long long* dbits;
  int32_t* flag;
  int32_t* nflag;
  ds.at(gi, dbits, flag, nflag);
  const int64_t nkeys = (int64_t)g.NX * g.NY * g.NZ;
  for (int64_t base = (int64_t)bid * blockDim.x; base < nkeys; base += (int64_t)nblk * blockDim.x) {
    const int64_t k = base + threadIdx.x;
    bool need = false;
    if (k < nkeys && nflag[k]) {
      nflag[k] = 0;
      need = find_node(g, (unsigned long long)k) < 0;
    }
    const int idx = block_agg_add(&g.counters[C_NNODES], need, nullptr);
    if (need) insert_new_node(g, (unsigned long long)k, idx);
  }
}

template <class VS>
__global__ void __launch_bounds__(256) k_dense_alloc(VS vs, DenseScratch ds) {
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  unsigned long long* dbits;
  int32_t* flag;
  int32_t* nflag;
  ds.at(gi, dbits, flag, nflag);
  const int64_t nbr = (int64_t)g.BX * g.BY * g.BZ;
  for (int64_t base = (int64_t)bid * blockDim.x; base < nbr; base += (int64_t)nblk * blockDim.x) {
    const int64_t lb = base + threadIdx.x;
    int node = -1, bx = 0, by = 0, bz = 0;
    if (lb < nbr && flag[lb]) {
      const uint32_t l = (uint32_t)lb, r = l / (uint32_t)g.BX;  // bricks < 2^32
      bx = (int)(l - r * (uint32_t)g.BX);
      by = (int)(r % (uint32_t)g.BY);
      bz = (int)(r / (uint32_t)g.BY);
      node = find_node(g, node_key_of(g, bx, by, bz));
    }
    int total = 0;
    const int slot = block_agg_add(&g.counters[C_NBRICKS], node >= 0, &total);
    if (node >= 0) {
      if (slot >= g.cap) {
        set_error(g, kErrOverflow);
      } else {
        init_brick_meta(g, slot, node, bx, by, bz);
        ulonglong2* dst = reinterpret_cast<ulonglong2*>(g.occ + (size_t)slot * 8);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_ulonglong2(dbits[(2 * q) * nbr + lb], dbits[(2 * q + 1) * nbr + lb]);
        g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)] = slot;
      }
    }
    if (threadIdx.x == 0 && total) atomicAdd(&g.counters[C_NEW_BRICKS], total);
  }
}

// ---- activation ----
// Compute set = bricks within Chebyshev brick radius R of an obstacle brick.  Global form: per-node
// 4096-bit masks, obstacle bits first, then a separable dilation (x, then y, then z), each stage a
// pure gather over neighbouring nodes' rows (no atomics).  A mask word holds two 16-brick x-rows:
// word (y >> 1) + 8 z, bits 16 (y & 1) + x.

template <class VS>
__global__ void k_clear_masks(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < (int64_t)nn * 128;
       i += (int64_t)nblk * blockDim.x) {
    g.amask[i] = 0u;
    int64_t node = i >> 7, w = i & 127;
    g.mwork[node * 384 + w] = 0u;
    g.mwork[node * 384 + 128 + w] = 0u;
    g.mwork[node * 384 + 256 + w] = 0u;
  }
}

template <class VS>
__global__ void k_obstacle_flags(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  const int nb = min(g.counters[C_NBRICKS], g.cap);
  for (int s = bid * blockDim.x + threadIdx.x; s < nb; s += nblk * blockDim.x) {
    bool obst = brick_has_obstacle(g, s);
    uint32_t f = g.bflags[s];
    g.bflags[s] = obst ? (f | F_OBST) : (f & ~F_OBST);
    if (obst) {
      int4 c = g.bcoord[s];
      int l = local_brick(c.x, c.y, c.z);
      atomicOr(&g.mwork[(size_t)c.w * 384 + (l >> 5)], 1u << (l & 31));
    }
  }
}

__device__ __forceinline__ uint32_t row16(const uint32_t* m, int y, int z) {
  return (m[(y >> 1) + 8 * z] >> (16 * (y & 1))) & 0xFFFFu;
}

// One warp per node holding obstacle bricks: create the neighbouring nodes that hold a brick within
// R bricks (Chebyshev) of one of its obstacle bricks, the only nodes its dilation reaches.  With
// R <= 16 the neighbours are the 26 adjacent nodes: neighbour (dx, dy, dz) is needed when one
// obstacle brick lies within R bricks of the side shared with it along every axis with a nonzero
// offset.  Each lane classifies 8 of the node's 256 brick rows and the warp ORs the 27-bit set of
// directions they reach.  (R > 16: every node within ceil(R / 16) nodes.)
template <class VS>
__global__ void k_node_halo(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  const int lane = threadIdx.x & 31;
  const int NR = (g.R + 15) / 16, side = 2 * NR + 1;
  for (int node = (bid * blockDim.x + threadIdx.x) >> 5; node < nn; node += (nblk * blockDim.x) >> 5) {
    const uint32_t* om = g.mwork + (size_t)node * 384;
    uint32_t any = om[lane] | om[lane + 32] | om[lane + 64] | om[lane + 96];
    if (!__any_sync(0xffffffffu, any != 0u)) continue;
    int nxn, nyn, nzn;
    node_coords(g, (unsigned long long)g.node_key[node], nxn, nyn, nzn);
    uint32_t dirs = 0xFFFFFFFFu;  // directions o = (dx + 1) + 3 (dy + 1) + 9 (dz + 1) to create
    if (NR == 1) {
      const uint32_t lo = g.R >= 16 ? 0xFFFFu : ((1u << g.R) - 1u), hi = (lo << (16 - g.R)) & 0xFFFFu;
      dirs = 0u;
      for (int r = lane; r < 256; r += 32) {
        const int yy = r & 15, zz = r >> 4;
        const uint32_t row = row16(om, yy, zz);
        if (!row) continue;
        // per axis, bit k: offset k - 1 reachable from this row's obstacle bricks
        const uint32_t ax = ((row & lo) ? 1u : 0u) | 2u | ((row & hi) ? 4u : 0u);
        const uint32_t ay = (yy < g.R ? 1u : 0u) | 2u | (yy >= 16 - g.R ? 4u : 0u);
        const uint32_t az = (zz < g.R ? 1u : 0u) | 2u | (zz >= 16 - g.R ? 4u : 0u);
        for (int kz = 0; kz < 3; ++kz)
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx)
              if ((az >> kz) & (ay >> ky) & (ax >> kx) & 1u) dirs |= 1u << (kx + 3 * (ky + 3 * kz));
      }
      dirs = __reduce_or_sync(0xffffffffu, dirs);
    }
    for (int o = lane; o < side * side * side; o += 32) {
      const int dx = o % side - NR, dy = (o / side) % side - NR, dz = o / (side * side) - NR;
      const int x = nxn + dx, y = nyn + dy, z = nzn + dz;
      if (x < 0 || y < 0 || z < 0 || x >= g.NX || y >= g.NY || z >= g.NZ || (dx == 0 && dy == 0 && dz == 0)) continue;
      if (NR > 1 || ((dirs >> o) & 1u)) get_or_create_node(g, node_key_at(g, x, y, z));
    }
  }
}


__device__ __forceinline__ int node_at(const GridView& g, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.NX || y >= g.NY || z >= g.NZ) return -1;
  return find_node(g, node_key_at(g, x, y, z));
}

// Stage 0 -> 1: dilate each x-row by R across the neighbouring nodes along x.
// Stage 1 -> 2: OR of the rows y - R .. y + R; stage 2 -> amask: rows z - R .. z + R, then clipped
// to the grid.  One thread per (node, mask word), i.e. two rows.
template <int AXIS, class VS>
__global__ void k_dilate_stage(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  const int R = g.R;
  const int src_off = AXIS * 128;  // obstacle bits, then stage 1, then stage 2
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < (int64_t)nn * 128;
       i += (int64_t)nblk * blockDim.x) {
    const int node = (int)(i >> 7), w = (int)(i & 127);
    int nxn, nyn, nzn;
    node_coords(g, (unsigned long long)g.node_key[node], nxn, nyn, nzn);
    const int z = w >> 3;
    uint32_t out = 0u;
    for (int half = 0; half < 2; ++half) {
      const int y = 2 * (w & 7) + half;
      uint32_t r = 0u;
      if (AXIS == 0) {
        // absolute brick x of bit j of chunk c: 16 (nxn + c) + j
        const int NR = (R + 15) / 16;
        for (int c = -NR; c <= NR; ++c) {
          int nb = c == 0 ? node : node_at(g, nxn + c, nyn, nzn);
          if (nb < 0) continue;
          uint32_t v = row16(g.mwork + (size_t)nb * 384 + src_off, y, z);
          if (!v) continue;
          for (int x = 0; x < 16; ++x) {
            int lo = x - R - 16 * c, hi = x + R - 16 * c;  // chunk-local bit range
            if (hi < 0 || lo > 15) continue;
            lo = max(lo, 0);
            hi = min(hi, 15);
            uint32_t msk = ((hi - lo == 31) ? 0xFFFFFFFFu : ((1u << (hi - lo + 1)) - 1u)) << lo;
            if (v & msk) r |= 1u << x;
          }
        }
      } else if (AXIS == 1) {
        for (int d = -R; d <= R; ++d) {
          int yy = y + d;
          int q = (yy >= 0) ? (yy >> 4) : -((15 - yy) >> 4);
          int nb = q == 0 ? node : node_at(g, nxn, nyn + q, nzn);
          if (nb < 0) continue;
          r |= row16(g.mwork + (size_t)nb * 384 + src_off, yy - 16 * q, z);
        }
      } else {
        for (int d = -R; d <= R; ++d) {
          int zz = z + d;
          int q = (zz >= 0) ? (zz >> 4) : -((15 - zz) >> 4);
          int nb = q == 0 ? node : node_at(g, nxn, nyn, nzn + q);
          if (nb < 0) continue;
          r |= row16(g.mwork + (size_t)nb * 384 + src_off, y, zz - 16 * q);
        }
        // clip to the grid
        const int gy = nyn * 16 + y, gz = nzn * 16 + z;
        if (gy >= g.BY || gz >= g.BZ) r = 0u;
        const int xs = g.BX - nxn * 16;
        if (xs < 16) r &= (xs <= 0) ? 0u : ((1u << xs) - 1u);
      }
      out |= r << (16 * half);
    }
    if (AXIS < 2)
      g.mwork[(size_t)node * 384 + (AXIS + 1) * 128 + w] = out;
    else
      g.amask[(size_t)node * 128 + w] = out;
  }
}

// The whole dilation of one node in one block (R <= 16, so the neighbourhood is the 3 x 3 x 3 nodes
// around it): the obstacle rows of the 3 x 3 node columns along y and z are dilated along x
// (48-bit rows across the three nodes along x), then along y, then along z, in shared memory, and
// the node's own 16 x 16 rows are clipped to the grid and written.  Replaces the three separable
// stage launches.
template <class VS>
__global__ void __launch_bounds__(256) k_dilate_nodes(VS vs) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  __shared__ int nbr[27];
  __shared__ uint16_t X[48][48];  // [z' + 16][y' + 16]: rows dilated along x
  __shared__ uint16_t Y[48][16];  // [z' + 16][y]: then along y
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  const int R = g.R;
  for (int node = bid; node < nn; node += nblk) {
    int nxn, nyn, nzn;
    node_coords(g, (unsigned long long)g.node_key[node], nxn, nyn, nzn);
    if (threadIdx.x < 27) {
      const int t = threadIdx.x, dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
      nbr[t] = (dx | dy | dz) == 0 ? node : node_at(g, nxn + dx, nyn + dy, nzn + dz);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < 48 * 48; r += blockDim.x) {
      const int zq = r / 48 - 16, yq = r % 48 - 16;
      const int dy = yq < 0 ? -1 : (yq >= 16 ? 1 : 0), dz = zq < 0 ? -1 : (zq >= 16 ? 1 : 0);
      const int y = yq - 16 * dy, z = zq - 16 * dz;
      unsigned long long w = 0ull;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int nb = nbr[(dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1))];
        if (nb >= 0) w |= (unsigned long long)row16(g.mwork + (size_t)nb * 384, y, z) << (16 * (dx + 1));
      }
      unsigned long long d = w;
      for (int sft = 1; sft <= R; ++sft) d |= (w << sft) | (w >> sft);
      X[zq + 16][yq + 16] = (uint16_t)(d >> 16);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < 48 * 16; r += blockDim.x) {
      const int zi = r / 16, y = r % 16;
      uint32_t o = 0u;
      for (int d = -R; d <= R; ++d) o |= X[zi][y + d + 16];
      Y[zi][y] = (uint16_t)o;
    }
    __syncthreads();
    if (threadIdx.x < 128) {
      const int w = threadIdx.x, z = w >> 3;
      uint32_t out = 0u;
      for (int half = 0; half < 2; ++half) {
        const int y = 2 * (w & 7) + half;
        uint32_t r = 0u;
        for (int d = -R; d <= R; ++d) r |= Y[z + d + 16][y];
        const int gy = nyn * 16 + y, gz = nzn * 16 + z;
        if (gy >= g.BY || gz >= g.BZ) r = 0u;
        const int xs = g.BX - nxn * 16;
        if (xs < 16) r &= (xs <= 0) ? 0u : ((1u << xs) - 1u);
        out |= r << (16 * half);
      }
      g.amask[(size_t)node * 128 + w] = out;
    }
    __syncthreads();
  }
}

// Mark bricks within Chebyshev radius R of brick (bx,by,bz) in amask: one (dy, dz) row (used by the
// incremental form, where few bricks change).
// Places for `cnt` items of each lane in a list counted by *ctr: one atomic per warp (warp-uniform
// call); returns the lane's first place.  *total receives the warp's sum.
__device__ __forceinline__ int warp_reserve_count(int32_t* ctr, int cnt, int* total) {
  const int lane = threadIdx.x & 31;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  *total = __shfl_sync(0xffffffffu, incl, 31);
  int base = 0;
  if (lane == 31 && *total) base = atomicAdd(ctr, *total);
  return __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
}

// Storage for the bricks of a row segment whose compute-set bits (`bits` of amask word `word` of
// `node`; bit b is the brick at x = x16 + (b & 15) of row (y, z)) this thread set first, so that
// exactly one thread handles each: the ones without storage get slots (places reserved a warp at
// a time), their metadata from the thread, their fields at dmax^2 from the whole warp
// (warp-uniform call).
__device__ void alloc_new_bits(const GridView& g, int node, int word, uint32_t bits, int x16, int y, int z) {
  uint32_t need = 0u;
  if (node >= 0)
    for (uint32_t b = bits; b; b &= b - 1u) {
      const int bit = __ffs(b) - 1;
      if (g.child[(size_t)node * kNodeBricks + word * 32 + bit] == kNoSlot) need |= 1u << bit;
    }
  const int cnt = __popc(need);
  int total = 0;
  const int base = warp_reserve_count(&g.counters[C_NBRICKS], cnt, &total);
  if ((threadIdx.x & 31) == 31 && total) atomicAdd(&g.counters[C_NEW_BRICKS], total);
  int k = 0;
  for (uint32_t b = need; b; b &= b - 1u, ++k) {
    const int bit = __ffs(b) - 1, slot = base + k;
    if (slot >= g.cap) {
      set_error(g, kErrOverflow);
      continue;
    }
    init_brick(g, slot, node, x16 + (bit & 15), y, z, false);
    g.child[(size_t)node * kNodeBricks + word * 32 + bit] = slot;
  }
  // fields: round r takes each lane's r-th new brick, a brick at a time by the whole warp
  const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
  for (int r = 0; r < rounds; ++r) init_fields_ballot(g, r < cnt && base + r < g.cap, base + r);
}

// Allocate every marked brick without storage: a block per (node, 256-brick chunk), a brick per
// thread, one atomic per block for the slot range (block scan of the flags).
template <class VS>
__global__ void __launch_bounds__(256) k_alloc_marked(VS vs, bool init_fields) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  (void)gi;
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  for (int b = bid; b < nn * 16; b += nblk) {
    const int node = b >> 4, l = (b & 15) * 256 + threadIdx.x;
    const bool need = ((g.amask[(size_t)node * 128 + (l >> 5)] >> (l & 31)) & 1u) &&
                      g.child[(size_t)node * kNodeBricks + l] == kNoSlot;
    int total = 0;
    const int slot = block_agg_add(&g.counters[C_NBRICKS], need, &total);
    if (threadIdx.x == 0 && total) atomicAdd(&g.counters[C_NEW_BRICKS], total);
    if (need) {
      if (slot >= g.cap) {
        set_error(g, kErrOverflow);
      } else {
        int nxn, nyn, nzn;
        node_coords(g, (unsigned long long)g.node_key[node], nxn, nyn, nzn);
        init_brick(g, slot, node, nxn * 16 + (l & 15), nyn * 16 + ((l >> 4) & 15), nzn * 16 + (l >> 8), init_fields);
        g.child[(size_t)node * kNodeBricks + l] = slot;
      }
    }
  }
}

// ---- work items ----
// Claim the run along `axis` that holds brick (bx, by, bz) (runs are aligned to `run` bricks inside
// the node) for this epoch: true for the one caller that queues it, with the run's first brick in
// `packed`.  A plain read first lets runs already claimed in this epoch skip the exchange (a value
// read before another thread's exchange only leads to the exchange).
__device__ __forceinline__ bool claim_run(const GridView& g, int axis, int bx, int by, int bz, int node, int run,
                                          int epoch, unsigned long long& packed) {
  // run is 4, 8 or 16: a shift and a mask instead of a division
  const int la = axis == 0 ? bx & 15 : (axis == 1 ? by & 15 : bz & 15);
  const int l1 = axis == 0 ? by & 15 : bx & 15, l2 = axis == 2 ? by & 15 : bz & 15;
  int* mk = &g.mark[((size_t)node * 3 + axis) * 1024 + l1 + 16 * (l2 + 16 * (la >> (__ffs(run) - 1)))];
  if (__ldcg(mk) == epoch || atomicExch(mk, epoch) == epoch) return false;
  const int back = la & (run - 1);
  packed = pack_brick(bx - (axis == 0 ? back : 0), by - (axis == 1 ? back : 0), bz - (axis == 2 ? back : 0));
  return true;
}

// Append the claimed runs (won[a]: this thread's run along axis a) to the three axes' work lists
// (block-uniform call; in a batch, igrid records each run's grid): the warps' counts are summed in
// shared memory and each list's counter word takes one atomic per block -- one per warp would
// queue thousands of atomics on the same word in a frame's marking.
__device__ __forceinline__ void emit_runs3(const GridView& g, const bool (&won)[3], const unsigned long long (&packed)[3],
                                           const Items& it, int grid) {
  __shared__ int cnt[3], base[3];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  int off[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const unsigned m = __ballot_sync(0xffffffffu, won[a]);
    int wb = 0;
    if (lane == 0 && m) wb = atomicAdd(&cnt[a], __popc(m));
    off[a] = __shfl_sync(0xffffffffu, wb, 0) + __popc(m & ((1u << lane) - 1u));
  }
  __syncthreads();
  if (threadIdx.x < 3) base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(&g.items_ctr[threadIdx.x], cnt[threadIdx.x]) : 0;
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int p = base[a] + off[a];
    if (won[a] && p < g.item_cap) {
      it.run[a][p] = packed[a];
      if (it.igrid[a]) it.igrid[a][p] = grid;
    }
  }
}

// Global form: every run that holds a stored brick, found node by node.  Block = (node, axis, run
// index along the axis); its 256 threads cover the 16 x 16 lines of the node across the axis.  A
// block-wide scan compacts the runs and one atomic reserves their places; the run slot lists are
// then read straight from the child tables of the node and of its neighbour along the axis
// (R <= 6 < 16, so the halo reaches at most one node each way), one slot per thread.
template <class VS>
__global__ void __launch_bounds__(256) k_items_nodes(VS vs, int rx, int ry, int rz, Items it, bool with_slots) {
  pdl_enter();
  int bid, nblk, gi;
  const GridView g = vs.get(bid, nblk, gi);
  if (vs.skip(g)) return;
  __shared__ int wsum[8];
  __shared__ int base_sh, count_sh;
  __shared__ int nbr_sh[2];
  __shared__ unsigned char lines[256];
  const int nn = min(g.counters[C_NNODES], g.node_cap);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int R = g.R;
  for (int b = bid; b < nn * 12; b += nblk) {
    const int node = b / 12, axis = (b % 12) / 4, qrun = b % 4;
    const int run = axis == 0 ? rx : (axis == 1 ? ry : rz);
    if (qrun >= 16 / run) continue;  // block-uniform
    int q[3];
    node_coords(g, (unsigned long long)g.node_key[node], q[0], q[1], q[2]);
    const int32_t* ch = g.child + (size_t)node * kNodeBricks;
    const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    const int r0 = qrun * run, nb = run + 2 * R;
    if (threadIdx.x < 2) {
      int qq[3] = {q[0], q[1], q[2]};
      qq[axis] += threadIdx.x == 0 ? -1 : 1;
      int n2 = -1;
      if (qq[0] >= 0 && qq[1] >= 0 && qq[2] >= 0 && qq[0] < g.NX && qq[1] < g.NY && qq[2] < g.NZ)
        n2 = find_node(g, node_key_at(g, qq[0], qq[1], qq[2]));
      nbr_sh[threadIdx.x] = n2;
    }
    const int o1 = threadIdx.x & 15, o2 = threadIdx.x >> 4;
    bool any = false;
    {
      // the run's child entries along the line, all read before any is tested
      const int across = (o1 << (4 * a1)) | (o2 << (4 * a2));
      int c[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) c[j] = j < run ? ch[across | ((r0 + j) << (4 * axis))] : -1;
#pragma unroll
      for (int j = 0; j < 16; ++j) any |= c[j] >= 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < 8; ++w) {
        const int t = wsum[w];
        wsum[w] = tot;
        tot += t;
      }
      count_sh = tot;
      base_sh = tot ? atomicAdd(&g.items_ctr[axis], tot) : 0;
    }
    __syncthreads();
    const int base = base_sh, cnt = count_sh;
    if (any) {
      const int pos = wsum[warp] + __popc(bal & ((1u << lane) - 1u));
      lines[pos] = (unsigned char)threadIdx.x;
      const int p = base + pos;
      if (p < g.item_cap) {
        int l0[3];
        l0[axis] = r0;
        l0[a1] = o1;
        l0[a2] = o2;
        it.run[axis][p] = pack_brick(q[0] * 16 + l0[0], q[1] * 16 + l0[1], q[2] * 16 + l0[2]);
        if (it.igrid[axis]) it.igrid[axis][p] = gi;
      }
    }
    __syncthreads();
    if (with_slots) {
      // four slots per thread and round, their child reads issued before any is written
      const int total = cnt * nb;
      for (int idx0 = threadIdx.x; idx0 < total; idx0 += 4 * 256) {
        int sv[4];
        int64_t dst[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = idx0 + u * 256;
          sv[u] = -1;
          dst[u] = -1;
          if (idx < total) {
            const int i = idx / nb, j = idx % nb;
            const int p = base + i;
            if (p < g.item_cap) {
              const int line = lines[i];
              int c = r0 + j - R, src = node;
              if (c < 0) {
                c += 16;
                src = nbr_sh[0];
              } else if (c >= 16) {
                c -= 16;
                src = nbr_sh[1];
              }
              dst[u] = (int64_t)p * kItemSlots + j;
              // local brick: c along the axis, the line's two coordinates across it
              const int lb = (c << (4 * axis)) | ((line & 15) << (4 * a1)) | ((line >> 4) << (4 * a2));
              if (src >= 0) sv[u] = g.child[(size_t)src * kNodeBricks + lb];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (dst[u] >= 0) it.slots[axis][dst[u]] = sv[u] >= 0 ? sv[u] + g.slot_base : -1;
      }
    }
    __syncthreads();
  }
}

// Slots of each queued run's bricks with R bricks of halo on both sides along the axis: a warp per
// queued run, a lane per slot.  A run lies inside one node and its halo (R <= 6 < 16 bricks)
// reaches at most the neighbouring node on each side along the axis, so three node lookups (lanes
// 0-2) serve the whole slot list, read from the child tables.
__device__ __forceinline__ void run_slots(const GridView& g, int axis, int run, unsigned long long packed,
                                          int32_t* __restrict__ dst) {
  const int nb = run + 2 * g.R;
  const int lane = threadIdx.x & 31;
  int bx, by, bz;
  unpack_brick(packed, bx, by, bz);
  const int ba = axis == 0 ? bx : (axis == 1 ? by : bz);
  const int Ba = axis == 0 ? g.BX : (axis == 1 ? g.BY : g.BZ);
  const int NQa = axis == 0 ? g.NX : (axis == 1 ? g.NY : g.NZ);
  int nq = -1;
  if (lane < 3) {
    const int qa = (ba >> 4) + lane - 1;
    if (qa >= 0 && qa < NQa) {
      const int qx = axis == 0 ? qa : bx >> 4, qy = axis == 1 ? qa : by >> 4, qz = axis == 2 ? qa : bz >> 4;
      nq = find_node(g, node_key_at(g, qx, qy, qz));
    }
  }
  const int n_lo = __shfl_sync(0xffffffffu, nq, 0), n_mid = __shfl_sync(0xffffffffu, nq, 1),
            n_hi = __shfl_sync(0xffffffffu, nq, 2);
  int s = -1;
  const int ca = ba + lane - g.R;  // this slot's brick coordinate along the axis
  if (lane < nb && ca >= 0 && ca < Ba) {
    const int node = (ca >> 4) < (ba >> 4) ? n_lo : ((ca >> 4) > (ba >> 4) ? n_hi : n_mid);
    if (node >= 0) {
      const int cx = axis == 0 ? ca : bx, cy = axis == 1 ? ca : by, cz = axis == 2 ? ca : bz;
      s = g.child[(size_t)node * kNodeBricks + local_brick(cx, cy, cz)];
      if (s >= 0) s += g.slot_base;
    }
  }
  dst[lane] = s;
}

// blockIdx.y = axis
__global__ void k_item_slots(GridView g, int rx, int ry, int rz, Items it) {
  pdl_enter();
  if (g.counters[C_BIG]) return;  // the global form's work lists came with their slots
  const int axis = (int)blockIdx.y;
  const int run = axis == 0 ? rx : (axis == 1 ? ry : rz);
  const int n = min(g.items_ctr[axis], g.item_cap);
  const int nw = (int)gridDim.x * (int)(blockDim.x >> 5);
  for (int item = (int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); item < n; item += nw)
    run_slots(g, axis, run, it.run[axis][item], it.slots[axis] + (size_t)item * kItemSlots);
}

// The same for a batch's shared queue: each run's grid comes from it.igrid.
__global__ void k_item_slots_batch(const GridView* __restrict__ views, const int32_t* __restrict__ items_ctr,
                                   int item_cap, int rx, int ry, int rz, Items it) {
  pdl_enter();
  const int axis = (int)blockIdx.y;
  const int run = axis == 0 ? rx : (axis == 1 ? ry : rz);
  const int n = min(items_ctr[axis], item_cap);
  const int nw = (int)gridDim.x * (int)(blockDim.x >> 5);
  for (int item = (int)blockIdx.x * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); item < n; item += nw) {
    const GridView g = views[it.igrid[axis][item]];
    if (g.counters[C_BIG]) continue;  // warp-uniform: that grid's runs came with their slots
    run_slots(g, axis, run, it.run[axis][item], it.slots[axis] + (size_t)item * kItemSlots);
  }
}

// Update statistics only (launched when they are asked for): the stored bricks each pass
// recomputes, i.e. the own entries (R .. R + run - 1) of every run's slot list that hold a slot,
// added to the counters of the run's grid (views == nullptr: every run is grid `one`'s).
// blockIdx.y = axis, a thread per run.
__global__ void k_count_run_bricks(const GridView* __restrict__ views, GridView one, const int32_t* __restrict__ items_ctr,
                                   int item_cap, int rx, int ry, int rz, Items it) {
  const int axis = (int)blockIdx.y;
  const int run = axis == 0 ? rx : (axis == 1 ? ry : rz);
  const int n = min(items_ctr[axis], item_cap);
  for (int item = (int)(blockIdx.x * blockDim.x + threadIdx.x); item < n; item += (int)(gridDim.x * blockDim.x)) {
    const int32_t* sl = it.slots[axis] + (size_t)item * kItemSlots + one.R;
    int own = 0;
    for (int j = 0; j < run; ++j) own += sl[j] >= 0;
    int32_t* ctr = views ? views[it.igrid[axis][item]].counters : one.counters;
    if (own) atomicAdd(&ctr[C_XB + axis], own);
  }
}

// ---- incremental ----
// Voxel gap between two bricks d apart along an axis: the nearest voxels of bricks 0 and d are
// 8 |d| - 7 apart (0 for the same brick).
__device__ __forceinline__ int brick_gap(int d) {
  d = abs(d);
  return d == 0 ? 0 : 8 * d - 7;
}

// For every changed brick c: refresh its obstacle flag; if it holds obstacles, mark its dilation
// (the bricks within R that must be stored); and queue its dirty runs.
// Dirty sets: D(v) depends only on obstacles closer than dmax (Eq. 1 with the truncation), so a
// flip in c can change D only in bricks whose nearest voxels lie closer than dmax to c's -- the
// ball of radius dmax around c at brick granularity, about half the cube of R bricks.  Such a brick
// needs its z pass if it is stored or about to be (every brick of the cube of an obstacle-holding
// c is: the dilation just marked it, and the allocation of the marked bricks runs before the
// passes).  The in-plane values g2 change only in c's z layer, within dmax in the plane (a disk):
// those bricks also need the in-plane pass; the x-line values g1 change only in c's x row: those
// bricks also need the x pass.
// With at most two changed bricks per block, a block per changed brick: its first threads find
// (or, for an obstacle-holding c, create) the interior nodes c's cube spans (at most 4 per axis:
// 2R + 1 <= 47 bricks), then a thread per row (y, z) of the cube sets the row's x extent in the
// allocation masks, and a thread per (column, z run) of the cube queues the run once if one of its
// bricks is in the ball (and c's y run and x run in c's layer).  Runs are aligned to their length
// (4, 8 or 16) inside nodes, hence at multiples of it in grid coordinates.  With more changed bricks
// per block (a batch's share of the launch, a large update), a thread per (changed brick, row) and
// then per (changed brick, offset in its cube), each with its own node lookups, keeps every thread
// of the GPU busy instead.
template <class US>
__global__ void __launch_bounds__(256, 6) k_changed_mark(US us, int rx, int ry, int rz, Items it, bool mark) {
  pdl_enter();
  __shared__ int nodes[64];
  __shared__ int obst_sh;
  const UpdArgs A = us.get();
  const GridView& g = A.g;
  const int32_t* __restrict__ changed = A.changed;
  const int grid = (int)blockIdx.y;
  const int nc = min(g.counters[C_CHANGED], g.cap);
  const int R = g.R, side = 2 * R + 1;
  // an update that takes the global form leaves all this to the gated kernels of the side stream
  if (big_update(g)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) g.counters[C_BIG] = 1;
    return;
  }
  const int epoch = g.counters[C_EPOCH];
  if (nc > 2 * (int)gridDim.x) {
    // dilation: a thread per (changed brick, row), the rounds block-uniform
    const int rows = side * side, nseg = (side + 15) / 16 + 1;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < (int64_t)nc * rows;
         base += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = base + threadIdx.x;
      int s = -1, r = 0;
      bool obst = false;
      if (i < (int64_t)nc * rows) {
        s = changed[i / rows];
        r = (int)(i % rows);
        obst = brick_has_obstacle(g, s);
        if (r == 0) {
          const uint32_t f = g.bflags[s];
          g.bflags[s] = obst ? (f | F_OBST) : (f & ~F_OBST);
        }
      }
      int4 c = make_int4(0, 0, 0, 0);
      if (obst) c = g.bcoord[s];
      const int y = c.y + r % side - R, z = c.z + r / side - R;
      const bool live = obst && (unsigned)y < (unsigned)g.BY && (unsigned)z < (unsigned)g.BZ;
      const int x0 = max(c.x - R, 0), x1 = min(c.x + R, g.BX - 1);
      const int ly = y & 15, lz = z & 15, word = (ly >> 1) + 8 * lz;
      int xa = x0;
      for (int k = 0; k < nseg; ++k) {  // the row's segments, one node each (same count on every lane)
        uint32_t added = 0u;
        int node = -1;
        const int x16 = xa & ~15;
        if (live && xa <= x1) {
          const int xe = min(x1, xa | 15);
          node = get_or_create_node(g, node_key_of(g, xa, y, z));
          if (node >= 0) {
            const uint32_t bitsx = ((1u << ((xe & 15) - (xa & 15) + 1)) - 1u) << (xa & 15);
            const uint32_t add = bitsx << (16 * (ly & 1));
            added = add & ~atomicOr(&g.amask[(size_t)node * 128 + word], add);
          }
          xa = xe + 1;
        }
        alloc_new_bits(g, node, word, added, x16, y, z);
      }
    }
    if (!mark) return;
    // dirty runs: a thread per (changed brick, offset in its cube); a warp spans at most two changed
    // bricks (a cube has at least 27 offsets), whose obstacle bits its first and last lanes read
    const int vol = side * side * side;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < (int64_t)nc * vol;
         base += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = base + threadIdx.x;
      const long long bi = i < (int64_t)nc * vol ? (long long)(i / vol) : -1ll;
      const long long b0 = __shfl_sync(0xffffffffu, bi, 0), b31 = __shfl_sync(0xffffffffu, bi, 31);
      bool o = false;
      if (lane == 0 && b0 >= 0) o = brick_has_obstacle(g, changed[b0]);
      if (lane == 31 && b31 >= 0) o = brick_has_obstacle(g, changed[b31]);
      const bool o0 = __shfl_sync(0xffffffffu, o, 0), o31 = __shfl_sync(0xffffffffu, o, 31);
      bool wx = false, wy = false, wz = false;
      unsigned long long px = 0, py = 0, pz = 0;
      if (bi >= 0) {
        const int r = (int)(i % vol);
        const int dx = r % side - R, dy = (r / side) % side - R, dz = r / (side * side) - R;
        const int s = changed[bi];
        const int4 c = g.bcoord[s];
        const int bx = c.x + dx, by = c.y + dy, bz = c.z + dz;
        const int gx = brick_gap(dx), gy = brick_gap(dy), gz = brick_gap(dz);
        if ((unsigned)bx < (unsigned)g.BX && (unsigned)by < (unsigned)g.BY && (unsigned)bz < (unsigned)g.BZ &&
            gx * gx + gy * gy + gz * gz < g.INF) {
          const bool obst = bi == b0 ? o0 : o31;
          const unsigned long long key = node_key_of(g, bx, by, bz);
          const int node = obst ? get_or_create_node(g, key) : find_node(g, key);
          if (node >= 0 && (obst || g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)] >= 0)) {
            if (dy == 0 && dz == 0) wx = claim_run(g, 0, bx, by, bz, node, rx, epoch, px);
            if (dz == 0) wy = claim_run(g, 1, bx, by, bz, node, ry, epoch, py);
            wz = claim_run(g, 2, bx, by, bz, node, rz, epoch, pz);
          }
        }
      }
      emit_runs3(g, {wx, wy, wz}, {px, py, pz}, it, grid);
    }
    return;
  }
  for (int i = (int)blockIdx.x; i < nc; i += (int)gridDim.x) {
    const int s = changed[i];
    __syncthreads();  // the table of the block's previous brick is no longer read
    const int4 c = g.bcoord[s];
    const int x0 = max(c.x - R, 0), x1 = min(c.x + R, g.BX - 1);
    const int y0 = max(c.y - R, 0), y1 = min(c.y + R, g.BY - 1);
    const int z0 = max(c.z - R, 0), z1 = min(c.z + R, g.BZ - 1);
    const int qx0 = x0 >> 4, qy0 = y0 >> 4, qz0 = z0 >> 4;
    const int nqx = (x1 >> 4) - qx0 + 1, nqy = (y1 >> 4) - qy0 + 1, nqz = (z1 >> 4) - qz0 + 1;
    const int nq = nqx * nqy * nqz;  // at most 4^3
    // at once: the brick's obstacle bit (lanes 0-7 of warp 0, a mask word each) and the lookups of
    // the nodes its cube spans (threads 32 .. 32 + nq - 1); nodes an obstacle brick's dilation
    // needs and that do not exist yet are created after the barrier
    if (threadIdx.x < 8) {
      const bool any = __any_sync(0xffu, g.occ[(size_t)s * 8 + threadIdx.x] != 0ull);
      if (threadIdx.x == 0) {
        const uint32_t f = g.bflags[s];
        g.bflags[s] = any ? (f | F_OBST) : (f & ~F_OBST);
        obst_sh = any;
      }
    } else if ((int)threadIdx.x >= 32 && (int)threadIdx.x < 32 + nq) {
      const int q = (int)threadIdx.x - 32;
      nodes[q] = find_node(g, node_key_at(g, qx0 + q % nqx, qy0 + (q / nqx) % nqy, qz0 + q / (nqx * nqy)));
    }
    __syncthreads();
    const bool obst = obst_sh != 0;  // block-uniform
    if (obst) {
      if ((int)threadIdx.x < nq && nodes[threadIdx.x] < 0) {
        const int q = (int)threadIdx.x;
        nodes[q] = get_or_create_node(g, node_key_at(g, qx0 + q % nqx, qy0 + (q / nqx) % nqy, qz0 + q / (nqx * nqy)));
      }
      __syncthreads();
    }
    if (obst) {
      // dilation: a row's x extent is split at node boundaries (the same segments on every lane);
      // the rounds are block-uniform so that new bricks' slots are reserved a warp at a time
      const int nyr = y1 - y0 + 1, rows = nyr * (z1 - z0 + 1);
      for (int rb = 0; rb < rows; rb += (int)blockDim.x) {
        const int r = rb + (int)threadIdx.x;
        const bool live = r < rows;
        const int y = y0 + (live ? r % nyr : 0), z = z0 + (live ? r / nyr : 0);
        const int ly = y & 15, lz = z & 15, word = (ly >> 1) + 8 * lz;
        const int nrow = nqx * (((y >> 4) - qy0) + nqy * ((z >> 4) - qz0));
        for (int xa = x0; xa <= x1;) {
          const int xe = min(x1, xa | 15);
          const int node = live ? nodes[nrow + (xa >> 4) - qx0] : -1;
          uint32_t added = 0u;
          if (node >= 0) {
            const uint32_t bitsx = ((1u << ((xe & 15) - (xa & 15) + 1)) - 1u) << (xa & 15);
            const uint32_t add = bitsx << (16 * (ly & 1));
            added = add & ~atomicOr(&g.amask[(size_t)node * 128 + word], add);
          }
          alloc_new_bits(g, node, word, added, xa & ~15, y, z);
          xa = xe + 1;
        }
      }
    }
    if (!mark) continue;  // block-uniform
    // dirty runs: a thread per (column, z run) of the cube, block-uniform rounds (the lists' places
    // are reserved a warp at a time); runs are 4, 8 or 16 bricks (shifts, not divisions)
    const int r0 = z0 & ~(rz - 1), nruns = ((z1 - r0) >> (__ffs(rz) - 1)) + 1;
    const int ncx = x1 - x0 + 1, ncol = ncx * (y1 - y0 + 1), total = ncol * nruns;
    for (int u0 = 0; u0 < total; u0 += (int)blockDim.x) {
      const int u = u0 + (int)threadIdx.x;
      bool wx = false, wy = false, wz = false;
      unsigned long long px = 0, py = 0, pz = 0;
      if (u < total) {
        const int zr = u / ncol, col = u - zr * ncol;
        const int cy = col / ncx;
        const int bx = x0 + (col - cy * ncx), by = y0 + cy;
        const int zs = max(r0 + zr * rz, z0), ze = min(r0 + zr * rz + rz - 1, z1);
        const int node = nodes[((bx >> 4) - qx0) + nqx * (((by >> 4) - qy0) + nqy * ((zs >> 4) - qz0))];
        const int gx = brick_gap(bx - c.x), gy = brick_gap(by - c.y), in_plane = gx * gx + gy * gy;
        if (node >= 0 && in_plane < g.INF) {
          const int32_t* ch = g.child + (size_t)node * kNodeBricks;
          bool any = false;
          for (int bz = zs; bz <= ze; ++bz) {
            const bool stored = obst || ch[local_brick(bx, by, bz)] >= 0;
            const int gz = brick_gap(bz - c.z);
            any |= stored && in_plane + gz * gz < g.INF;
            if (bz == c.z && stored) {
              if (by == c.y) wx = claim_run(g, 0, bx, by, bz, node, rx, epoch, px);
              wy = claim_run(g, 1, bx, by, bz, node, ry, epoch, py);
            }
          }
          if (any) wz = claim_run(g, 2, bx, by, zs, node, rz, epoch, pz);
        }
      }
      emit_runs3(g, {wx, wy, wz}, {px, py, pz}, it, grid);
    }
  }
}

// Dirty runs of a batch's update, queued after the bricks the dilation added are stored (so that
// the marking overlaps the batch's gated global-form branch instead of preceding it): a thread per
// (changed brick, offset in its cube), the ball and disk rules of k_changed_mark, stored bricks
// read from the child tables.
template <class US>
__global__ void __launch_bounds__(256) k_mark_runs(US us, int rx, int ry, int rz, Items it) {
  pdl_enter();
  const UpdArgs A = us.get();
  const GridView& g = A.g;
  const int32_t* __restrict__ changed = A.changed;
  const int grid = (int)blockIdx.y;
  if (g.counters[C_BIG]) return;
  const int nc = min(g.counters[C_CHANGED], g.cap);
  const int epoch = g.counters[C_EPOCH];
  const int R = g.R, side = 2 * R + 1, vol = side * side * side;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < (int64_t)nc * vol;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool wx = false, wy = false, wz = false;
    unsigned long long px = 0, py = 0, pz = 0;
    if (i < (int64_t)nc * vol) {
      const int r = (int)(i % vol);
      const int dx = r % side - R, dy = (r / side) % side - R, dz = r / (side * side) - R;
      const int4 c = g.bcoord[changed[i / vol]];
      const int bx = c.x + dx, by = c.y + dy, bz = c.z + dz;
      const int gx = brick_gap(dx), gy = brick_gap(dy), gz = brick_gap(dz);
      if ((unsigned)bx < (unsigned)g.BX && (unsigned)by < (unsigned)g.BY && (unsigned)bz < (unsigned)g.BZ &&
          gx * gx + gy * gy + gz * gz < g.INF) {
        const int node = find_node(g, node_key_of(g, bx, by, bz));
        if (node >= 0 && g.child[(size_t)node * kNodeBricks + local_brick(bx, by, bz)] >= 0) {
          if (dy == 0 && dz == 0) wx = claim_run(g, 0, bx, by, bz, node, rx, epoch, px);
          if (dz == 0) wy = claim_run(g, 1, bx, by, bz, node, ry, epoch, py);
          wz = claim_run(g, 2, bx, by, bz, node, rz, epoch, pz);
        }
      }
    }
    emit_runs3(g, {wx, wy, wz}, {px, py, pz}, it, grid);
  }
}

// The incremental update's kernels for one grid or all grids of a batch (k = gridDim.y).
template <class US>
cudaError_t update_ingest_kernels(US us, int k, int64_t n, cudaStream_t st) {
  const int div = k > 1 ? k : 1;
  auto bx = [&](int64_t work, int hi) {
    int64_t b = (work + kT - 1) / kT;
    const int64_t lim = k > 1 ? (hi / div > 16 ? hi / div : 16) : hi;
    return (unsigned)(b < 1 ? 1 : (b > lim ? lim : b));
  };
  const dim3 gr(bx(n, 152 * 16), k);
  VDB_LAUNCH_PDL(k_rec_slots<US>, gr, kT, 0, st, us);
  VDB_LAUNCH_PDL(k_upd_rec_last<US>, gr, kT, 0, st, us);
  VDB_LAUNCH_PDL(k_upd_apply_last<US>, gr, kT, 0, st, us);
  return cudaGetLastError();
}

template <class US, class GV>
cudaError_t update_mark_kernels(US us, GV gv, int k, int node_cap, int R, bool with_slots, const Tuning& t,
                                const Items& it, const Fork& fk, cudaStream_t st) {
  const unsigned div = k > 1 ? (unsigned)k : 1u;
  auto share = [&](unsigned single) { return k > 1 ? (single / div > 16 ? single / div : 16u) : single; };
  const unsigned nc = (unsigned)node_cap;
  cudaError_t e = cudaSuccess;
  cudaStream_t gs = st;
  if (fk.side) {
    e = cudaEventRecord(fk.fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fk.side, fk.fork, 0);
    if (e != cudaSuccess) return e;
    gs = fk.side;
  }
  // global form, for the grids whose update takes it (each kernel decides for itself; the others'
  // blocks return at once, and the kernels stride over their work, so a launch of at most two
  // blocks per SM keeps that cheap), on the side stream from the end of the ingest on, beside the
  // incremental marking
  auto gated = [&](unsigned single) { return share(single < 304u ? single : 304u); };
  VDB_LAUNCH(k_clear_masks<GV>, dim3(gated(256), k), kT, 0, gs, gv);
  VDB_LAUNCH_PDL(k_obstacle_flags<GV>, dim3(gated(1024), k), kT, 0, gs, gv);
  VDB_LAUNCH_PDL(k_node_halo<GV>, dim3(gated(64), k), kT, 0, gs, gv);
  if (R <= 16) {
    VDB_LAUNCH_PDL(k_dilate_nodes<GV>, dim3(gated(nc < 1024 ? nc : 1024u), k), 256, 0, gs, gv);
  } else {
    VDB_LAUNCH_PDL((k_dilate_stage<0, GV>), dim3(gated(256), k), kT, 0, gs, gv);
    VDB_LAUNCH_PDL((k_dilate_stage<1, GV>), dim3(gated(256), k), kT, 0, gs, gv);
    VDB_LAUNCH_PDL((k_dilate_stage<2, GV>), dim3(gated(256), k), kT, 0, gs, gv);
  }
  VDB_LAUNCH_PDL(k_alloc_marked<GV>, dim3(gated(nc * 16 < 8192 ? nc * 16 : 8192u), k), kT, 0, gs, gv, false);
  VDB_LAUNCH_PDL(k_items_nodes<GV>, dim3(gated(nc * 12 < 8192 ? nc * 12 : 8192u), k), kT, 0, gs, gv, t.run[0], t.run[1],
             t.run[2], it, with_slots);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fk.side) {
    e = cudaEventRecord(fk.join, fk.side);
    if (e != cudaSuccess) return e;
  }
  // incremental form, for the others: the changed bricks' flags, their dilation (with storage for
  // the bricks it adds) and, for a single grid, their dirty runs; a batch's dirty runs after that
  VDB_LAUNCH_PDL(k_changed_mark<US>, dim3(share(2432), k), kT, 0, st, us, t.run[0], t.run[1], t.run[2], it, k == 1);
  if (k > 1) VDB_LAUNCH_PDL(k_mark_runs<US>, dim3(share(2432), k), kT, 0, st, us, t.run[0], t.run[1], t.run[2], it);
  return cudaGetLastError();
}

}  // namespace

cudaError_t ensure_scratch(Scratch& s, size_t bytes) {
  if (s.bytes >= bytes) return cudaSuccess;
  if (s.buf) cudaFree(s.buf);
  s.buf = nullptr;
  s.bytes = 0;
  size_t want = bytes + bytes / 4 + 4096;
  cudaError_t e = cudaMalloc(&s.buf, want);
  if (e != cudaSuccess) return e;
  s.bytes = want;
  return cudaSuccess;
}

cudaError_t launch_reset(const GridView& g, cudaStream_t st) {
  VDB_LAUNCH(k_reset_nodes<OneView>, 1024, kT, 0, st, OneView{g});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(g.counters, 0, sizeof(int32_t) * C_NUM, st);
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Apply staged records.  Bricks of "set" records are found or created through a counting sort over
// one flag per brick of the grid (many records), or a stable radix sort of brick keys, a unique pass
// and a compaction (few records).  Bits: in the global form, when every record sets a voxel, the
// records' bits go to the bricks directly (many records: OR-ed into a dense scratch mask during the
// counting pass and copied whole at allocation; few records: OR-ed per record).  Whenever a record
// clears a voxel, or flips are tracked, each voxel's last record decides its bit through the
// per-voxel last-record table (largest record index per voxel, then applied and reset).  With
// tracking, each flipped voxel's brick is appended once to `changed`.
static size_t ingest_scratch_bytes(const GridView& g, int64_t n, bool track) {
  const int64_t nbr_all = (int64_t)g.BX * g.BY * g.BZ;
  const bool counting = n >= nbr_all / 4;
  const bool dense_bits = counting && !track && nbr_all * 8 < (int64_t)0xFFFFFFFFll;
  const int64_t m = counting && nbr_all > n ? nbr_all : n;  // brick flags only on the counting path
  const size_t nb4 = align_up((size_t)m * 4);
  const size_t nkeys_al = ((size_t)g.NX * g.NY * g.NZ + 63) & ~(size_t)63;
  const size_t flags = align_up(((size_t)m + nkeys_al) * 4);  // node flags, then brick flags
  const size_t dbytes = dense_bits ? align_up((size_t)nbr_all * 64) : 0;
  return 3 * nb4 + flags + align_up(radix_temp_bytes(n)) + align_up(scan_temp_bytes(m)) + dbytes;
}

// The per-voxel last-record table of the ordered path: cap * 512 words, all -1 between ingests.
static cudaError_t ensure_vlast(const GridView& g, Scratch& vl, cudaStream_t st) {
  const size_t want = (size_t)g.cap * 512 * sizeof(int32_t);
  if (vl.bytes >= want) return cudaSuccess;
  cudaError_t e = ensure_scratch(vl, want);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(vl.buf, 0xFF, want, st);
}

cudaError_t reserve_ingest(const GridView& g, int64_t n, Scratch& scr, Scratch& vl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = g.unbounded ? cudaSuccess : ensure_scratch(scr, ingest_scratch_bytes(g, n, false));
  if (e != cudaSuccess) return e;
  return ensure_vlast(g, vl, st);
}

cudaError_t launch_begin_update(const GridView& g, cudaStream_t st) {
  UpdArgs a{};
  a.g = g;
  VDB_LAUNCH(k_begin_update<UpdOne>, 1, 32, 0, st, UpdOne{a});
  return cudaGetLastError();
}

cudaError_t prepare_update_args(const GridView& g, Scratch& vl, UpdArgs& a, cudaStream_t st) {
  cudaError_t e = ensure_vlast(g, vl, st);
  if (e != cudaSuccess) return e;
  a.vlast = (int32_t*)vl.buf;
  return cudaSuccess;
}

// The tracked ingest: with `track` (an incremental update) each flipped voxel's brick joins the
// changed list once; unbounded grids take this path for the global form too (no brick-key sort).
static cudaError_t launch_ingest_tracked(const GridView& g, const rec_t* rec, int64_t n, const int32_t* n_dev,
                                         int32_t* changed, int32_t* rslot, Scratch& vl, cudaStream_t st) {
  UpdArgs a{};
  a.g = g;
  a.rec = rec;
  a.n = n;
  a.n_dev = n_dev;
  a.changed = changed;
  a.rslot = rslot;
  cudaError_t e = prepare_update_args(g, vl, a, st);
  if (e != cudaSuccess) return e;
  return update_ingest_kernels(UpdOne{a}, 1, n, st);
}

cudaError_t launch_ingest_records(const GridView& g, const rec_t* rec, int64_t n, const int32_t* n_dev, bool track,
                                  int32_t* changed, int32_t* rslot, Scratch& scr, Scratch& vl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (track || g.unbounded) return launch_ingest_tracked(g, rec, n, n_dev, changed, rslot, vl, st);
  const int64_t nbr_all = (int64_t)g.BX * g.BY * g.BZ;
  const bool counting = n >= nbr_all / 4;
  // the dense mask is indexed by a 32-bit word number (8 words per brick)
  const bool dense_bits = counting && !track && nbr_all * 8 < (int64_t)0xFFFFFFFFll;
  const int64_t m = counting && nbr_all > n ? nbr_all : n;  // brick flags only on the counting path
  const size_t nb4 = align_up((size_t)m * 4);
  cudaError_t e = ensure_scratch(scr, ingest_scratch_bytes(g, n, track));
  if (e != cudaSuccess) return e;
  e = ensure_vlast(g, vl, st);
  if (e != cudaSuccess) return e;
  int32_t* vlast = (int32_t*)vl.buf;
  char* p = (char*)scr.buf;
  uint32_t* ka = (uint32_t*)p;
  p += nb4;
  uint32_t* kb = (uint32_t*)p;
  p += nb4;
  // one flag per node key (nodes are created before their bricks), then one per brick or record
  const int64_t nkeys = (int64_t)g.NX * g.NY * g.NZ;
  const int64_t nkeys_al = (nkeys + 63) & ~(int64_t)63;
  int32_t* nflag = (int32_t*)p;
  int32_t* flag = nflag + nkeys_al;
  p += align_up(((size_t)m + (size_t)nkeys_al) * 4);
  int32_t* pos = (int32_t*)p;
  p += nb4;
  void* rtemp = p;
  p += align_up(radix_temp_bytes(n));
  void* stemp = p;
  p += align_up(scan_temp_bytes(m));
  unsigned long long* dbits = dense_bits ? (unsigned long long*)p : nullptr;

  const unsigned nbk = blocks_for(n);
  const uint64_t nbr = (uint64_t)nbr_all;
  if (counting) {
    // one flag per brick of the grid, then compaction
    e = cudaMemsetAsync(nflag, 0, sizeof(int32_t) * (size_t)(nkeys_al + (int64_t)nbr), st);
    if (e != cudaSuccess) return e;
    if (dbits) {
      e = cudaMemsetAsync(dbits, 0, (size_t)nbr * 64, st);
      if (e != cudaSuccess) return e;
    }
    VDB_LAUNCH(k_mark_record_bricks, nbk, kT, 0, st, g, rec, n, n_dev, flag, dbits);
    e = cudaMemsetAsync(g.counters + C_UNIQUE, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    VDB_LAUNCH(k_compact_flag_index, blocks_for((int64_t)nbr), kT, 0, st, g, flag, (int64_t)nbr, ka, nflag);
    VDB_LAUNCH_PDL(k_create_flagged_nodes, blocks_for(nkeys), kT, 0, st, g, nflag, nkeys);
    VDB_LAUNCH_PDL(k_alloc_obstacle_bricks, blocks_for((int64_t)nbr), kT, 0, st, g, ka, (int64_t)nbr, track, dbits);
    if (!track && !dbits) VDB_LAUNCH_PDL(k_apply_set_only, nbk, kT, 0, st, g, rec, n, n_dev);
  } else {
    // LSD radix sort of the brick keys, unique, compaction
    VDB_LAUNCH(k_rec_brick_keys, nbk, kT, 0, st, g, rec, n, n_dev, ka);
    // the sentinel 0xFFFFFFFF sorts after every key below 2^bits
    bool in_b = false;
    e = radix_sort_u32(ka, kb, nullptr, nullptr, n, nullptr, bits_for(nbr), rtemp, st, &in_b);
    if (e != cudaSuccess) return e;
    uint32_t* sorted = in_b ? kb : ka;
    uint32_t* uniq = in_b ? ka : kb;
    VDB_LAUNCH(k_head_flags, nbk, kT, 0, st, sorted, n, (uint32_t)nbr, flag);
    e = exclusive_scan_i32(flag, pos, n, g.counters + C_UNIQUE, stemp, st);
    if (e != cudaSuccess) return e;
    VDB_LAUNCH(k_compact_keys, nbk, kT, 0, st, sorted, flag, pos, n, uniq);
    e = cudaMemsetAsync(nflag, 0, sizeof(int32_t) * (size_t)nkeys, st);
    if (e != cudaSuccess) return e;
    VDB_LAUNCH(k_flag_key_nodes, blocks_for(n), kT, 0, st, g, uniq, n, nflag);
    VDB_LAUNCH_PDL(k_create_flagged_nodes, blocks_for(nkeys), kT, 0, st, g, nflag, nkeys);
    VDB_LAUNCH_PDL(k_alloc_obstacle_bricks, blocks_for(n), kT, 0, st, g, uniq, n, track, nullptr);
    if (!track) VDB_LAUNCH_PDL(k_apply_set_only, nbk, kT, 0, st, g, rec, n, n_dev);
  }
  // ordered path (its kernels return at once when no record clears a voxel and flips are untracked)
  VDB_LAUNCH_PDL(k_rec_last, nbk, kT, 0, st, g, rec, n, n_dev, track, vlast);
  VDB_LAUNCH_PDL(k_apply_last, nbk, kT, 0, st, g, rec, n, n_dev, track, track, vlast, changed);
  return cudaGetLastError();
}

size_t dense_scratch_bytes(const GridView& g) {
  const size_t nbr = (size_t)g.BX * g.BY * g.BZ, nkeys = (size_t)g.NX * g.NY * g.NZ;
  return align_up(nbr * 64) + align_up(nbr * 4) + align_up(nkeys * 4);
}

cudaError_t launch_ingest_dense(const GridView& g, const uint8_t* grid, Scratch& scr, cudaStream_t st) {
  cudaError_t e = ensure_scratch(scr, dense_scratch_bytes(g));
  if (e != cudaSuccess) return e;
  const size_t nbr = (size_t)g.BX * g.BY * g.BZ, nkeys = (size_t)g.NX * g.NY * g.NZ;
  char* p = (char*)scr.buf;
  DenseScratch ds{(unsigned long long*)p, (int32_t*)(p + align_up(nbr * 64)),
                  (int32_t*)(p + align_up(nbr * 64) + align_up(nbr * 4)), nullptr};
  e = cudaMemsetAsync(ds.nflag, 0, nkeys * 4, st);
  if (e != cudaSuccess) return e;
  const OneView v{g};
  VDB_LAUNCH((k_dense_masks<OneView, OneSrc>), batch_blocks(g, BK_DENSE), kT, 0, st, v, OneSrc{grid}, ds);
  VDB_LAUNCH(k_dense_nodes<OneView>, batch_blocks(g, BK_DNODES), kT, 0, st, v, ds);
  VDB_LAUNCH(k_dense_alloc<OneView>, batch_blocks(g, BK_DALLOC), kT, 0, st, v, ds);
  return cudaGetLastError();
}

cudaError_t launch_activation_full(const GridView& g, cudaStream_t st) {
  const OneView v{g};
  VDB_LAUNCH_PDL(k_clear_masks<OneView>, 256, kT, 0, st, v);
  VDB_LAUNCH_PDL(k_obstacle_flags<OneView>, 1024, kT, 0, st, v);
  VDB_LAUNCH_PDL(k_node_halo<OneView>, 64, kT, 0, st, v);
  if (g.R <= 16) {
    VDB_LAUNCH_PDL(k_dilate_nodes<OneView>, g.node_cap < 1024 ? g.node_cap : 1024, 256, 0, st, v);
  } else {
    VDB_LAUNCH_PDL((k_dilate_stage<0, OneView>), 256, kT, 0, st, v);
    VDB_LAUNCH_PDL((k_dilate_stage<1, OneView>), 256, kT, 0, st, v);
    VDB_LAUNCH_PDL((k_dilate_stage<2, OneView>), 256, kT, 0, st, v);
  }
  VDB_LAUNCH_PDL(k_alloc_marked<OneView>, g.node_cap * 16 < 8192 ? g.node_cap * 16 : 8192, kT, 0, st, v, false);
  return cudaGetLastError();
}

static cudaError_t clear_item_counters(const GridView& g, cudaStream_t st) {
  return cudaMemsetAsync(g.items_ctr, 0, 3 * sizeof(int32_t), st);
}

cudaError_t launch_build_items_full(const GridView& g, const Tuning& t, const Items& it, bool with_slots,
                                    cudaStream_t st) {
  cudaError_t e = clear_item_counters(g, st);
  if (e != cudaSuccess) return e;
  VDB_LAUNCH(k_items_nodes<OneView>, g.node_cap * 12 < 8192 ? g.node_cap * 12 : 8192, kT, 0, st, OneView{g}, t.run[0],
             t.run[1], t.run[2], it, with_slots);
  return cudaGetLastError();
}

cudaError_t launch_item_slots(const GridView& g, const Tuning& t, const Items& it, cudaStream_t st) {
  VDB_LAUNCH(k_item_slots, dim3(405, 3), kT, 0, st, g, t.run[0], t.run[1], t.run[2], it);
  return cudaGetLastError();
}

cudaError_t launch_count_run_bricks(const GridView* views, const GridView& one, const int32_t* items_ctr, int item_cap,
                                   const Tuning& t, const Items& it, cudaStream_t st) {
  VDB_LAUNCH(k_count_run_bricks, dim3(152, 3), kT, 0, st, views, one, items_ctr, item_cap, t.run[0], t.run[1], t.run[2],
             it);
  return cudaGetLastError();
}

cudaError_t launch_item_slots_batch(const GridView* views, const Tuning& t, const Items& it, int32_t* items_ctr,
                                    int item_cap, cudaStream_t st) {
  VDB_LAUNCH(k_item_slots_batch, dim3(1216, 3), kT, 0, st, views, items_ctr, item_cap, t.run[0], t.run[1], t.run[2],
             it);
  return cudaGetLastError();
}

// ---- batches ----
static int clamp_blocks(int64_t n, int hi) { return (int)(n < 1 ? 1 : (n > hi ? hi : n)); }

int batch_blocks(const GridView& g, int kind) {
  const int64_t t = kT;
  switch (kind) {
    case BK_RESET: return clamp_blocks(((int64_t)g.node_cap * (kNodeBricks / 4) + g.hmask + t) / t, 1024);  // int4 stores
    case BK_DENSE: {
      const int64_t units = (int64_t)((g.BX + kDenseX - 1) / kDenseX) * g.BY * g.BZ;  // a warp each
      return clamp_blocks((units * 32 + t - 1) / t, 152 * 16);
    }
    case BK_DNODES: return clamp_blocks(((int64_t)g.NX * g.NY * g.NZ + t - 1) / t, 1024);
    case BK_DALLOC: return clamp_blocks(((int64_t)g.BX * g.BY * g.BZ + t - 1) / t, 152 * 64);
    case BK_CLEAR: return clamp_blocks(((int64_t)g.node_cap * 128 + t - 1) / t, 256);
    case BK_OBST: return clamp_blocks(((int64_t)g.cap + t - 1) / t, 1024);
    case BK_HALO: return clamp_blocks(((int64_t)g.node_cap * 32 + t - 1) / t, 64);
    case BK_DILATE: return clamp_blocks(g.node_cap, 1024);
    case BK_ALLOC: return clamp_blocks((int64_t)g.node_cap * 8, 8192);  // two 256-brick chunks per block
    case BK_ITEMS: return clamp_blocks((int64_t)g.node_cap * 12, 8192);
  }
  return 1;
}

cudaError_t launch_reset_batch(const GridView* views, const BatchShape& b, int32_t* counters_all, size_t n_counters,
                               cudaStream_t st) {
  if (b.k <= 0) return cudaSuccess;
  VDB_LAUNCH(k_reset_nodes<BatchViews>, b.total[BK_RESET], kT, 0, st, BatchViews{views, b.first[BK_RESET], b.k});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(counters_all, 0, sizeof(int32_t) * n_counters, st);
}

cudaError_t launch_ingest_dense_batch(const GridView* views, const BatchShape& b, const uint8_t* const* srcs,
                                      void* scratch, const int64_t* offsets, size_t nflag_words, int32_t* nflag0,
                                      cudaStream_t st) {
  if (b.k <= 0) return cudaSuccess;
  if (b.k > kBatchMax) return cudaErrorInvalidValue;
  BatchSrc src;
  for (int i = 0; i < kBatchMax; ++i) src.p[i] = i < b.k ? srcs[i] : nullptr;
  cudaError_t e = cudaMemsetAsync(nflag0, 0, nflag_words * 4, st);
  if (e != cudaSuccess) return e;
  char* p = (char*)scratch;
  DenseScratch ds{(unsigned long long*)p, (int32_t*)p, (int32_t*)p, offsets};
  VDB_LAUNCH((k_dense_masks<BatchViews, BatchSrc>), b.total[BK_DENSE], kT, 0, st,
             BatchViews{views, b.first[BK_DENSE], b.k}, src, ds);
  VDB_LAUNCH(k_dense_nodes<BatchViews>, b.total[BK_DNODES], kT, 0, st, BatchViews{views, b.first[BK_DNODES], b.k}, ds);
  VDB_LAUNCH(k_dense_alloc<BatchViews>, b.total[BK_DALLOC], kT, 0, st, BatchViews{views, b.first[BK_DALLOC], b.k}, ds);
  return cudaGetLastError();
}

cudaError_t launch_activation_batch(const GridView* views, const BatchShape& b, cudaStream_t st) {
  if (b.k <= 0) return cudaSuccess;
  VDB_LAUNCH(k_clear_masks<BatchViews>, b.total[BK_CLEAR], kT, 0, st, BatchViews{views, b.first[BK_CLEAR], b.k});
  VDB_LAUNCH(k_obstacle_flags<BatchViews>, b.total[BK_OBST], kT, 0, st, BatchViews{views, b.first[BK_OBST], b.k});
  VDB_LAUNCH(k_node_halo<BatchViews>, b.total[BK_HALO], kT, 0, st, BatchViews{views, b.first[BK_HALO], b.k});
  const BatchViews dv{views, b.first[BK_DILATE], b.k};
  if (b.R <= 16) {
    VDB_LAUNCH(k_dilate_nodes<BatchViews>, b.total[BK_DILATE], 256, 0, st, dv);
  } else {
    VDB_LAUNCH((k_dilate_stage<0, BatchViews>), b.total[BK_DILATE], kT, 0, st, dv);
    VDB_LAUNCH((k_dilate_stage<1, BatchViews>), b.total[BK_DILATE], kT, 0, st, dv);
    VDB_LAUNCH((k_dilate_stage<2, BatchViews>), b.total[BK_DILATE], kT, 0, st, dv);
  }
  VDB_LAUNCH(k_alloc_marked<BatchViews>, b.total[BK_ALLOC], kT, 0, st, BatchViews{views, b.first[BK_ALLOC], b.k},
             false);
  return cudaGetLastError();
}

cudaError_t launch_build_items_batch(const GridView* views, const BatchShape& b, const Tuning& t, const Items& it,
                                     int32_t* items_ctr, cudaStream_t st) {
  if (b.k <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(items_ctr, 0, 3 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  VDB_LAUNCH(k_items_nodes<BatchViews>, b.total[BK_ITEMS], kT, 0, st, BatchViews{views, b.first[BK_ITEMS], b.k},
             t.run[0], t.run[1], t.run[2], it, true);
  return cudaGetLastError();
}

// Incremental: records were already applied with flip tracking (changed list filled).
// (the item counters were cleared when the update began)
cudaError_t launch_incremental_mark(const GridView& g, const Tuning& t, const int32_t* changed, const Items& it,
                                    const Fork& fk, cudaStream_t st) {
  UpdArgs a{};
  a.g = g;
  a.changed = const_cast<int32_t*>(changed);
  return update_mark_kernels(UpdOne{a}, GatedOne{g}, 1, g.node_cap, g.R, half_path(g), t, it, fk, st);
}

// Batched update: begin + tracked ingest of every grid, then the marking (one launch per step).
cudaError_t launch_update_batch_ingest(const UpdArgs* d_args, const BatchUpdShape& s, const BatchCounts& counts,
                                       cudaStream_t st) {
  if (s.k <= 0) return cudaSuccess;
  VDB_LAUNCH(k_begin_batch_update, dim3(1, s.k), 32, 0, st, d_args, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return update_ingest_kernels(UpdBatch{d_args}, s.k, s.max_n, st);
}

cudaError_t launch_update_batch_mark(const UpdArgs* d_args, const BatchUpdShape& s, const Tuning& t, const Items& it,
                                     const Fork& fk, cudaStream_t st) {
  if (s.k <= 0) return cudaSuccess;
  return update_mark_kernels(UpdBatch{d_args}, GatedBatch{d_args}, s.k, (int)s.max_node_cap, s.R, s.half, t, it, fk,
                             st);
}

}  // namespace vdbedt
