// Internal definitions shared by the CUDA translation units of libvdbedt.
//
// Sparse grid layout in device memory (paper Sec. IV-A: a shallow, wide tree with a hashed top
// level, directly indexed lower levels and a background tile value):
//   level 1  hash table of interior nodes (open addressing, linear probing); a node covers
//            16^3 bricks = 128^3 voxels; node key = nx + NX (ny + NY nz) of the node's coordinates
//            (below 2^42); slot word = (node key << 22) | node index (all ones: empty)
//   level 2  per node a dense table of 4096 child slots (int32; -1 = background tile dmax^2)
//            plus a 4096-bit mask of bricks in the compute set
//   leaves   8^3-voxel bricks in a pool indexed by slot:
//              occ   8 x uint64   bit (y*8 + x) of word z  (64 B)
//              g1    512 x uint16 x-line squared distance, saturated, y-major  (1 KB)
//              g2    512 x uint16 in-plane (x, y) squared distance, saturated   (1 KB)
//              dist  512 x int32  D, the output                                 (2 KB)
//            voxel index inside a brick: x + 8 y + 64 z (g1: x + 8 z + 64 y).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/vdbedt.h"

namespace vdbedt {

constexpr int kBrick = 8;
constexpr int kBrickVox = 512;
constexpr int kNodeB = 16;  // bricks per node edge
constexpr int kNodeBricks = kNodeB * kNodeB * kNodeB;
constexpr unsigned long long kEmptySlot = ~0ull;
constexpr int kIndexBits = 22;
constexpr uint32_t kPending = (1u << kIndexBits) - 1u;  // index field of a claimed, unpublished slot
constexpr int kMaxNodes = (1 << kIndexBits) - 2;
// Unbounded grids: coordinates in [-kUnboundedOffset, kUnboundedOffset - 128) on every axis, stored
// shifted by kUnboundedOffset (node coordinates 0 .. 16382, keys below 2^42 - 1).
constexpr int kUnboundedOffset = VDBEDT_UNBOUNDED_OFFSET;
constexpr int kUnboundedSize = VDBEDT_UNBOUNDED_MAX + VDBEDT_UNBOUNDED_OFFSET;
constexpr int32_t kNoSlot = -1;
constexpr int32_t kNone = VDBEDT_D_NONE;  // untruncated grids: no obstacle on the line / in the grid

// device error bits
constexpr int kErrOverflow = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrInvalidRecord = 4;
constexpr int kErrInternal = 8;
constexpr int kErrNodeOverflow = 16;

// device counters
enum Counter : int {
  C_NBRICKS = 0,
  C_NNODES = 1,
  C_ERR = 2,
  C_X_ITEMS = 3,  // work items queued per axis (x, y, z: three consecutive words)
  C_Y_ITEMS = 4,
  C_Z_ITEMS = 5,
  C_CHANGED = 6,
  C_FLIPS = 7,
  C_NEW_BRICKS = 8,
  C_UNIQUE = 9,
  C_HAS_ZERO = 10,
  C_FINITE = 11,
  C_OBST = 12,
  C_NB_START = 13,  // stored bricks when the running update began (its global-vs-incremental choice)
  C_EPOCH = 14,  // incremental update epoch (run and brick dedupe marks)
  C_SPARE = 15,  // unused
  C_XB = 16,  // stored bricks in the update's dirty runs per axis (x, y, z: three consecutive words)
  C_YB = 17,
  C_ZB = 18,
  C_BIG = 19,  // this update's edits reach so far that it takes the global form after applying them
  C_NUM = 20
};

// brick flags
constexpr uint32_t F_OBST = 1u;    // holds an occupied voxel
constexpr uint32_t F_FINITE = 2u;  // holds a voxel with D < dmax^2
constexpr uint32_t F_G2FIN = 4u;   // holds a voxel with in-plane value g2 < dmax^2
constexpr uint32_t F_G1FIN = 8u;   // holds a voxel with x-line value g1 < dmax^2

struct GridView {
  int nx, ny, nz;     // voxels
  int BX, BY, BZ;     // bricks per axis
  int NX, NY, NZ;     // nodes per axis
  int dmax, R, INF;   // truncation, brick radius of influence, dmax^2
  int half;           // 1: g1 / g2 hold fp16 bit patterns (windowed kernels, dmax <= 45); 0: 16-bit
                      // integers (lower-envelope kernels)
  int off;            // added to caller coordinates (0; kUnboundedOffset for an unbounded grid)
  int unbounded;      // 1: no per-node-key arrays (nodes are created where records fall)
  int untrunc;        // 1: no truncation; every brick stored at slot bx + BX (by + BY bz), g1 / g2 hold
                      // int32 (their arrays are twice as large), INF = kNone
  uint32_t hmask;     // hash capacity - 1
  int cap;            // brick capacity
  int node_cap;       // node capacity
  unsigned long long* hslots;  // [hmask+1]
  int32_t* child;     // [node_cap * 4096]
  uint32_t* amask;    // [node_cap * 128] compute-set bits: bit l = bx + 16 by + 256 bz (local)
  uint32_t* mwork;    // [node_cap * 384] obstacle bits and two dilation stages, same layout
  uint32_t* nclaim;   // [node_cap * 128] bricks claimed for allocation by the running ingest (amask layout)
  long long* node_key;  // [node_cap]
  int32_t* mark;      // [node_cap * 3 * 1024] epoch of the last time each run along axis a was queued
  unsigned long long* occ;  // [cap * 8]
  uint16_t* g1;       // [cap * 512]
  uint16_t* g2;       // [cap * 512]
  int32_t* dist;      // [cap * 512]
  int4* bcoord;       // [cap]
  uint32_t* bflags;   // [cap]
  int32_t* bepoch;    // [cap] epoch of the last change (incremental)
  int32_t* counters;  // [C_NUM]
  // Work lists.  A grid of a batch keeps its bricks in a pool shared by the batch, at slots
  // slot_base .. slot_base + cap - 1 of the pool; the per-brick pointers above already point at
  // its first slot.  Work-item slot lists hold pool slots (local slot + slot_base), so that one
  // pass launch can serve every grid of the batch.  Single grids: slot_base = 0.
  int slot_base;
  int item_cap;       // capacity of the work lists (items per axis)
  int32_t* items_ctr; // [3] items queued along x, y, z (the grid's counters, or the batch's)
  // Untruncated grids: the dirty lines of an update (null otherwise), three sets back to back,
  // each cleared by the pass that reads it: x rows (bit (by + BY bz) * 64 + (y & 7) + 8 (z & 7), set
  // by the tracked ingest at each flipped voxel), y lines (a byte per line x + NXP z, set where the
  // x pass changed g1) and z lines (a byte per line x + NXP y, set where the y pass changed g2); the
  // bytes are set with plain stores -- the rows of every y (the y lines of every z) write the same
  // lines, and bytes need no atomics; NXP = nx rounded up to 32, so that a warp's 32 lines along x
  // read 32 consecutive bytes.
  uint32_t* ut_bits;
};

__host__ __device__ inline int ut_nxp(const GridView& g) { return (g.nx + 31) & ~31; }
__host__ __device__ inline int64_t ut_row_words(const GridView& g) { return (int64_t)g.BY * g.BZ * 2; }
__host__ __device__ inline int64_t ut_yline_words(const GridView& g) { return (int64_t)(ut_nxp(g) >> 2) * g.nz; }
__host__ __device__ inline int64_t ut_zline_words(const GridView& g) { return (int64_t)(ut_nxp(g) >> 2) * g.ny; }
__host__ __device__ inline int64_t ut_bits_words(const GridView& g) {
  return ut_row_words(g) + ut_yline_words(g) + ut_zline_words(g);
}

__host__ __device__ inline unsigned long long node_key_of(const GridView& g, int bx, int by, int bz) {
  return (unsigned long long)(bx >> 4) +
         (unsigned long long)g.NX * ((unsigned long long)(by >> 4) + (unsigned long long)g.NY * (unsigned long long)(bz >> 4));
}
// node coordinates of a key
__host__ __device__ inline void node_coords(const GridView& g, unsigned long long key, int& x, int& y, int& z) {
  x = (int)(key % (unsigned long long)g.NX);
  const unsigned long long r = key / (unsigned long long)g.NX;
  y = (int)(r % (unsigned long long)g.NY);
  z = (int)(r / (unsigned long long)g.NY);
}
__host__ __device__ inline unsigned long long node_key_at(const GridView& g, int x, int y, int z) {
  return (unsigned long long)x + (unsigned long long)g.NX * ((unsigned long long)y + (unsigned long long)g.NY * (unsigned long long)z);
}

__host__ __device__ constexpr uint32_t hash32(uint32_t k) {
  k ^= k >> 16;
  k *= 0x7feb352du;
  k ^= k >> 15;
  k *= 0x846ca68bu;
  k ^= k >> 16;
  return k;
}
// slot of a 64-bit node key: the high word folded into the low one before the 32-bit mix (a
// bounded grid's keys have a zero high word, whose fold is the constant kHashFold0)
constexpr uint32_t kHashFold0 = hash32(0x9e3779b9u);
__device__ __forceinline__ uint32_t hash_key(unsigned long long k) {
  const uint32_t hi = (uint32_t)(k >> 32);
  return hash32((uint32_t)k ^ (hi == 0u ? kHashFold0 : hash32(hi + 0x9e3779b9u)));
}

__device__ __forceinline__ void set_error(const GridView& g, int bits) { atomicOr(&g.counters[C_ERR], bits); }

// First statement of a kernel that may be launched with VDB_LAUNCH_PDL: wait until the previous
// kernel of the stream has finished and its writes are visible (returns at once for a kernel
// launched without the attribute), then let the next kernel of the stream begin launching.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Device-side waits give up after kWaitLimitNs of global time (or kWaitMaxPolls polls, whichever
// comes first), set the error word and let the kernel return.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // one second
constexpr uint32_t kWaitMaxPolls = 1u << 28;
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Node index for node key, or -1 when the node is absent.  Readers never wait: a node whose
// insertion is still pending is absent for them (inserts happen in kernels that do not read the
// node's bricks).
__device__ __forceinline__ int find_node(const GridView& g, unsigned long long key) {
  uint32_t h = hash_key(key) & g.hmask;
  for (uint32_t probe = 0; probe <= g.hmask; ++probe) {
    const unsigned long long w = g.hslots[h];
    if (w == kEmptySlot) return -1;
    if ((w >> kIndexBits) == key) {
      const uint32_t v = (uint32_t)(w & kPending);
      return v == kPending ? -1 : (int)v;
    }
    h = (h + 1) & g.hmask;
  }
  return -1;
}

// Find or insert the node with this key.  The inserting thread claims the hash slot with a
// pending marker, allocates the node index, then publishes it; other inserters of the same key
// wait for publication with a bounded spin (error bit on give-up).
__device__ inline int get_or_create_node(const GridView& g, unsigned long long key) {
  uint32_t h = hash_key(key) & g.hmask;
  for (uint32_t probe = 0; probe <= g.hmask; ++probe) {
    unsigned long long w = g.hslots[h];
    if (w == kEmptySlot) {
      const unsigned long long want = (key << kIndexBits) | kPending;
      const unsigned long long old = atomicCAS(&g.hslots[h], w, want);
      if (old == w) {
        int idx = atomicAdd(&g.counters[C_NNODES], 1);
        if (idx >= g.node_cap) {
          set_error(g, kErrNodeOverflow);
          return -1;
        }
        g.node_key[idx] = (long long)key;
        __threadfence();
        atomicExch(&g.hslots[h], (key << kIndexBits) | (uint32_t)idx);
        return idx;
      }
      w = old;
    }
    if ((w >> kIndexBits) == key) {
      if ((uint32_t)(w & kPending) != kPending) return (int)(w & kPending);  // published: no atomic needed
      const unsigned long long t0 = global_ns();
      for (uint32_t spin = 0; spin < kWaitMaxPolls; ++spin) {
        // plain (volatile) reads while waiting: they do not queue behind the publishing exchange
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&g.hslots[h]);
        const uint32_t v = (uint32_t)(cur & kPending);
        if (v != kPending) return (int)v;
        if ((spin & 63u) == 63u && global_ns() - t0 > kWaitLimitNs) break;
        __nanosleep(64);
      }
      set_error(g, kErrTimeout);
      return -1;
    }
    h = (h + 1) & g.hmask;
  }
  set_error(g, kErrNodeOverflow);
  return -1;
}

__device__ __forceinline__ int local_brick(int bx, int by, int bz) {
  return (bx & 15) | ((by & 15) << 4) | ((bz & 15) << 8);
}

// Slot of brick (bx, by, bz), or -1 when it is outside the grid or not stored.
__device__ __forceinline__ int find_brick(const GridView& g, int bx, int by, int bz) {
  if ((unsigned)bx >= (unsigned)g.BX || (unsigned)by >= (unsigned)g.BY || (unsigned)bz >= (unsigned)g.BZ) return -1;
  int n = find_node(g, node_key_of(g, bx, by, bz));
  if (n < 0) return -1;
  int s = g.child[(size_t)n * kNodeBricks + local_brick(bx, by, bz)];
  return s >= 0 ? s : -1;
}

__device__ __forceinline__ unsigned long long pack_brick(int bx, int by, int bz) {
  return (unsigned long long)(uint32_t)bx | ((unsigned long long)(uint32_t)by << 21) |
         ((unsigned long long)(uint32_t)bz << 42);
}
__device__ __forceinline__ void unpack_brick(unsigned long long p, int& bx, int& by, int& bz) {
  bx = (int)(p & 0x1FFFFF);
  by = (int)((p >> 21) & 0x1FFFFF);
  bz = (int)((p >> 42) & 0x1FFFFF);
}

}  // namespace vdbedt

// ---------------------------------------------------------------------------------------------
// Host-side internal interface between translation units
// ---------------------------------------------------------------------------------------------
namespace vdbedt {

// Process-wide count of kernel launches made by the library (reported by vdbedt_kernel_launches).
void note_launch();
// Message returned by vdbedt_last_error(NULL) on this thread (calls that have no handle).
void set_last_error(const char* msg);

#define VDB_LAUNCH(kernel, grid, block, smem, stream, ...)         \
  do {                                                             \
    ::vdbedt::note_launch();                                       \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);    \
  } while (0)

// Launch with programmatic stream serialization: the kernel may be scheduled before the previous
// kernel of the stream has finished, so its launch and block scheduling overlap that kernel's
// tail.  Only for kernels that call pdl_enter() before their first memory access.  Errors are
// left for cudaGetLastError like those of VDB_LAUNCH.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define VDB_LAUNCH_PDL(kernel, grid, block, smem, stream, ...)                         \
  do {                                                                                 \
    ::vdbedt::note_launch();                                                           \
    ::vdbedt::launch_pdl(kernel, dim3(grid), dim3(block), (smem), (stream), __VA_ARGS__); \
  } while (0)

constexpr int kItemSlots = 32;  // slot list entries per work item (run + 2R <= 28 on the half path)
constexpr int kBatchMax = 1024;  // grids per batch (the dense-ingest source table is a kernel parameter)

// Tuning.variant: low bits 1 = full windowed minimum, 3 = windowed minimum with early exit and
// skips (y and z passes); + kVariantXDirect = x pass with plain loads instead of the copy ring;
// kVariantEnvelope = the lower-envelope kernels for all three passes (16-bit integer fields).
constexpr int kVariantXDirect = 4;
// An incremental update whose changed bricks times (2R + 1)^3 exceed kBigUpdate times the stored
// bricks takes the global form's activation and work lists after applying its records.
constexpr int kBigUpdate = 24;
constexpr int kVariantEnvelope = 8;
struct Tuning {
  int run[3] = {4, 4, 4};  // bricks per work item along x, y, z
  int variant = 3;
};

// Work lists of the passes: runs of bricks along each axis, and (half path) the slots of each
// run's bricks with their halo of R bricks on both sides.
struct Items {
  unsigned long long* run[3];  // packed brick coordinates of the first brick of each run
  int32_t* slots[3];           // [cap * kItemSlots]
  int32_t* igrid[3];           // batches: the grid of each queued run (null for a single grid)
};

// primitives (prims.cu)
size_t scan_temp_bytes(int64_t n);
// gate (nullable): a device count; when it is 0 the scan does nothing
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev, void* temp,
                               cudaStream_t st, const int32_t* gate = nullptr);
size_t radix_temp_bytes(int64_t n);
// Stable LSD radix sort of u32 keys (with optional u32 values) on the low `bits` bits, ping-ponging
// between the a and b buffers (input in a).  n is an upper bound; count_dev (nullable) holds the
// actual count on the device (0: every kernel of the sort returns at once).  *result_in_b tells
// which buffer holds the sorted data.
cudaError_t radix_sort_u32(uint32_t* keys_a, uint32_t* keys_b, uint32_t* vals_a, uint32_t* vals_b, int64_t n,
                           const int32_t* count_dev, int bits, void* temp, cudaStream_t st, bool* result_in_b);

// grid build (grid.cu)
// A staged occupancy record in 64 bits: x | y << 21 | z << 42 | value << 63.  A record that failed
// validation carries x = kBadCoord (never inside a grid) and is skipped (and reported).
typedef unsigned long long rec_t;
constexpr int kBadCoord = 0x1FFFFF;
__host__ __device__ inline rec_t pack_rec(int x, int y, int z, int v) {
  return (rec_t)(uint32_t)x | ((rec_t)(uint32_t)y << 21) | ((rec_t)(uint32_t)z << 42) | ((rec_t)(v & 1) << 63);
}
__host__ __device__ inline int4 unpack_rec(rec_t r) {
  return make_int4((int)(r & 0x1FFFFF), (int)((r >> 21) & 0x1FFFFF), (int)((r >> 42) & 0x1FFFFF), (int)(r >> 63));
}
struct Scratch {
  void* buf = nullptr;
  size_t bytes = 0;
};

// Per-grid arguments of the incremental update's kernels: the same kernels serve one grid (the
// arguments are a kernel parameter) or every grid of a batch at once (an array in device memory;
// blockIdx.y picks the grid, blockIdx.x strides over that grid's work).
struct UpdArgs {
  GridView g;
  const rec_t* rec;          // staged records
  int64_t n;                 // staged records (upper bound when counted)
  const int32_t* n_dev;      // device-side count (counted staging) or null
  int32_t* changed;          // bricks holding a flipped voxel (cap entries)
  int32_t* vlast;            // per-voxel last-record table (cap * 512 words, all -1 between ingests)
  int32_t* rslot;            // per staged record: its brick's slot (-1: none, -2: looked up once allocated,
                             // -3 - slot: the brick this record allocated)
};
cudaError_t ensure_scratch(Scratch& s, size_t bytes);

cudaError_t launch_reset(const GridView& g, cudaStream_t st);
// n records at rec; with n_dev (nullable) only the first *n_dev of them (clamped to [0, n]).
// scr: sort / scan scratch of the global form; vl: the per-voxel last-record table (allocated and
// set to -1 on first use, cap * 512 words); rslot: one word per record (n entries) for the tracked
// form's brick slots.
cudaError_t launch_ingest_records(const GridView& g, const rec_t* rec, int64_t n, const int32_t* n_dev, bool track,
                                  int32_t* changed, int32_t* rslot, Scratch& scr, Scratch& vl, cudaStream_t st);
// size the ingest scratch and the last-record table for up to n records
cudaError_t reserve_ingest(const GridView& g, int64_t n, Scratch& scr, Scratch& vl, cudaStream_t st);
// clear the per-update counters and advance the device-side update epoch
cudaError_t launch_begin_update(const GridView& g, cudaStream_t st);
// dense grid -> bricks (scratch: dense_scratch_bytes(g))
size_t dense_scratch_bytes(const GridView& g);
cudaError_t launch_ingest_dense(const GridView& g, const uint8_t* grid, Scratch& scr, cudaStream_t st);
cudaError_t launch_activation_full(const GridView& g, cudaStream_t st);
// every run holding a stored brick, with slot lists when with_slots (half path)
cudaError_t launch_build_items_full(const GridView& g, const Tuning& t, const Items& it, bool with_slots,
                                    cudaStream_t st);
// A side stream for the update's two alternative branches: the global form's activation and work
// lists run there (forked after the decision kernel, joined by the caller before the passes), so
// that when the update stays incremental their launches, which exit at once, overlap the marking.
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// Records fork.join on the side stream; the caller waits on it before the passes.
cudaError_t launch_incremental_mark(const GridView& g, const Tuning& t, const int32_t* changed, const Items& it,
                                    const Fork& fk, cudaStream_t st);
// The last-record table of one grid, allocated on first use; fills a's vlast.
cudaError_t prepare_update_args(const GridView& g, Scratch& vl, UpdArgs& a, cudaStream_t st);
// Batched incremental update of k grids (d_args: their arguments in device memory): the same
// kernels as one grid's update, each launched once for all grids.  max_*: the largest staged
// count and node capacity over the grids (launch shapes).
struct BatchUpdShape {
  int k;
  int64_t max_n, max_node_cap;
  int R;      // common to the batch
  bool half;  // the windowed form (work lists carry slot lists)
};
// record counts of the grids staged without a device count (-1: the grid's count word is already
// written), passed by value to the first kernel
struct BatchCounts {
  int32_t c[kBatchMax];
};
cudaError_t launch_update_batch_ingest(const UpdArgs* d_args, const BatchUpdShape& s, const BatchCounts& counts,
                                       cudaStream_t st);
cudaError_t launch_update_batch_mark(const UpdArgs* d_args, const BatchUpdShape& s, const Tuning& t, const Items& it,
                                     const Fork& fk, cudaStream_t st);
// slot lists of every queued run of a batch (each run's grid from it.igrid)
cudaError_t launch_item_slots_batch(const GridView* views, const Tuning& t, const Items& it, int32_t* items_ctr,
                                    int item_cap, cudaStream_t st);
// Update statistics: stored bricks of every run's slot list per axis into each grid's C_XB .. C_ZB
// (views == nullptr: a single grid `one`).
cudaError_t launch_count_run_bricks(const GridView* views, const GridView& one, const int32_t* items_ctr, int item_cap,
                                   const Tuning& t, const Items& it, cudaStream_t st);
// Untruncated grids: store every brick (at creation), clear the occupancy (reset), take a dense
// uint8 grid, and the transform proper (three whole-line passes; `scratch` holds 8 bytes per voxel).
cudaError_t launch_ut_init(const GridView& g, cudaStream_t st);
cudaError_t launch_ut_reset(const GridView& g, cudaStream_t st);
cudaError_t launch_ut_dense(const GridView& g, const uint8_t* grid, cudaStream_t st);
size_t ut_scratch_bytes(const GridView& g);
cudaError_t launch_ut_pass(const GridView& g, int axis, void* scratch, cudaStream_t st);
// The update's pass along `axis` over the lines its dirty bits name (x: rows holding a flipped
// voxel; y, z: lines whose input changed), marking the next axis's lines where its output changed;
// lines recomputed are counted in items_ctr[axis].  The z pass also refreshes the brick flags.
cudaError_t launch_ut_update_pass(const GridView& g, int axis, void* scratch, cudaStream_t st);
// slot lists of every queued run (half path)
cudaError_t launch_item_slots(const GridView& g, const Tuning& t, const Items& it, cudaStream_t st);

// The same steps for every grid of a batch at once: one launch per step (views: device array of
// the k grids' views; each block finds its grid through the shape's block shares).
// Kernels that run once per grid: in a batch each grid gets a share of one launch sized to its
// work (batch_blocks), the shares laid end to end (first[kind][i] = first block of grid i).
enum BatchKind {
  BK_RESET = 0, BK_DENSE, BK_DNODES, BK_DALLOC, BK_CLEAR, BK_OBST, BK_HALO, BK_DILATE, BK_ALLOC, BK_ITEMS, BK_NUM
};
int batch_blocks(const GridView& g, int kind);
struct BatchShape {
  int k;
  int R;  // brick radius (common to the batch)
  const int* first[BK_NUM];  // device arrays of k + 1 block offsets per kind
  int total[BK_NUM];         // blocks of the launch per kind
};
cudaError_t launch_reset_batch(const GridView* views, const BatchShape& b, int32_t* counters_all, size_t n_counters,
                               cudaStream_t st);
// scratch: grid i's masks, brick flags and node flags start offsets[3i], offsets[3i + 1] and
// offsets[3i + 2] elements (u64, int32, int32) from the scratch base; nflag0 .. nflag0 +
// nflag_words covers every grid's node flags
cudaError_t launch_ingest_dense_batch(const GridView* views, const BatchShape& b, const uint8_t* const* srcs,
                                      void* scratch, const int64_t* offsets, size_t nflag_words, int32_t* nflag0,
                                      cudaStream_t st);
cudaError_t launch_activation_batch(const GridView* views, const BatchShape& b, cudaStream_t st);
cudaError_t launch_build_items_batch(const GridView* views, const BatchShape& b, const Tuning& t, const Items& it,
                                     int32_t* items_ctr, cudaStream_t st);

// passes (passes.cu)
bool half_path(const GridView& g);
// pass along `axis` (0 x, 1 y, 2 z) over the queued runs
cudaError_t launch_pass(const GridView& g, const Tuning& t, int axis, const Items& it, cudaStream_t st);
int effective_run(const GridView& g, const Tuning& t, int axis);
// a bounded device wait that runs out (0: mbarrier phase, 1: pending node), for tests
cudaError_t launch_wait_selftest(const GridView& g, int which, cudaStream_t st);

// queries (query.cu)
cudaError_t launch_query(const GridView& g, const int32_t* xyz, int64_t n, int32_t* out, cudaStream_t st);
// out[3k .. 3k + 2]: nearest occupied voxel of query k (ties to the smallest (z, y, x)), or -1s
cudaError_t launch_query_nearest(const GridView& g, const int32_t* xyz, int64_t n, int32_t* out, cudaStream_t st);
cudaError_t launch_export_dense(const GridView& g, int32_t* out, cudaStream_t st);
// occupancy of planes [z_lo, z_hi) as packed records with z shifted by dz (mode 0: occupied voxels
// of every stored brick; mode 1: every voxel of the bricks in `changed`); *count = records found
// (only the first max_n are written)
cudaError_t launch_export_occupancy(const GridView& g, const int32_t* changed, int z_lo, int z_hi, int dz, int mode,
                                    unsigned long long* out, int64_t max_n, unsigned long long* count,
                                    cudaStream_t st);
// obstacle and finite brick counts into counters C_OBST and C_FINITE
cudaError_t launch_count_flags(const GridView& g, cudaStream_t st);
// d (metres) and, when grad is not null, dd/dp at n points (the clearance cost's interpolation)
cudaError_t launch_distance_at(const GridView& g, float vs, const float* pts, int64_t n, float* dist, float* grad,
                               cudaStream_t st);
cudaError_t launch_clearance_fwd(const GridView& g, float vs, const float* pts, int64_t T, int64_t P, float tau,
                                 float* cost, cudaStream_t st);
cudaError_t launch_clearance_bwd(const GridView& g, float vs, const float* pts, int64_t T, int64_t P, float tau,
                                 const float* gcost, float* gpts, cudaStream_t st);

}  // namespace vdbedt
