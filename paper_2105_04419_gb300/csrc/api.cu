// The C ABI of libvdbedt (declared in include/vdbedt.h): handle lifetime, staging of occupancy
// records (host, device, device-counted, dense), the global and incremental transforms, queries,
// the clearance cost, tuning and phase events, batches of grids sharing one brick pool, and the
// self-test of the bounded device waits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/vdbedt.h"
#include "vdbedt_internal.cuh"

using namespace vdbedt;

namespace {
thread_local std::string g_last_error = "";
}

namespace vdbedt {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
cudaError_t launch_pack_records(const int32_t* xyz, const uint8_t* occ, int64_t n, const int32_t* n_dev,
                                int32_t* count_out, int nx, int ny, int nz, int off, rec_t* dst, int32_t* invalid,
                                int32_t* counters, cudaStream_t st);
cudaError_t launch_check_packed(const uint64_t* src, int64_t n, int nx, int ny, int nz, rec_t* dst, int32_t* invalid,
                                int32_t* counters, cudaStream_t st);
cudaError_t launch_check_bricks(const int32_t* bxyz, const uint64_t* masks, int64_t n, const GridView& g,
                                int32_t* invalid, unsigned long long* count, cudaStream_t st);
cudaError_t launch_expand_bricks(const int32_t* bxyz, const uint64_t* masks, int64_t n, const GridView& g, rec_t* dst,
                                 unsigned long long* cursor, cudaStream_t st);
}

struct vdbedt_batch;

struct vdbedt_map {
  GridView g{};
  vdbedt_batch* batch = nullptr;  // owning batch of a batch grid (its bricks live in the batch's pool)
  vdbedt_config cfg{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  // staged records
  rec_t* stage = nullptr;
  int32_t* stage_slot = nullptr;  // one word per staged record (the tracked ingest's brick slots)
  int64_t stage_n = 0, stage_cap = 0;
  bool stage_counted = false;  // the stage holds up to stage_n records, *d_count of them valid
  int32_t* d_count = nullptr;
  bool dense_pending = false;
  bool computed = false;
  int32_t* d_invalid = nullptr;
  int32_t* h_pinned = nullptr;  // pinned host words for small readbacks
  Scratch scr;
  Scratch vlast;  // per-voxel last-record table of the ordered ingest
  Scratch io;  // host-input staging on the device
  Scratch uts;  // line stacks of the untruncated transform
  Items items{};
  int32_t* changed = nullptr;
  Tuning tune;
  int sticky = VDBEDT_OK;
  std::string err;
  // phase timing (CUDA events on the handle's stream)
  bool profiling = false;
  cudaEvent_t ev[7] = {};
  bool ev_recorded = false;
  Fork fork;  // side stream of the update's global-form branch
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

vdbedt_status fail(vdbedt_map* h, vdbedt_status s, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (s == VDBEDT_ECUDA) h->sticky = VDBEDT_ECUDA;
  } else {
    g_last_error = msg;
  }
  return s;
}

vdbedt_status cuda_fail(vdbedt_map* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, VDBEDT_ENOMEM, m);
  }
  return fail(h, VDBEDT_ECUDA, m);
}

#define CK(h, expr, where)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail((h), _e, where); \
  } while (0)

template <typename T>
cudaError_t dalloc(vdbedt_map* h, T** p, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) {
    h->allocs.push_back((void*)*p);
    h->device_bytes += bytes;
  }
  return e;
}

vdbedt_status check_handle(vdbedt_map* h) {
  if (!h) return fail(nullptr, VDBEDT_EINVAL, "null handle");
  if (h->sticky == VDBEDT_ECUDA) return VDBEDT_ECUDA;
  return VDBEDT_OK;
}

int32_t* batch_error_word(const vdbedt_map* h);

vdbedt_status device_errors(vdbedt_map* h) {
  cudaError_t e =
      cudaMemcpyAsync(h->h_pinned + 32, h->g.counters + C_ERR, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  h->h_pinned[33] = 0;
  if (e == cudaSuccess && h->batch)
    e = cudaMemcpyAsync(h->h_pinned + 33, batch_error_word(h), sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
  int bits = h->h_pinned[32] | h->h_pinned[33];
  if (!bits) return VDBEDT_OK;
  if (bits & (kErrOverflow | kErrNodeOverflow))
    return fail(h, VDBEDT_EOVERFLOW, "brick or node capacity exceeded; the field is incomplete until vdbedt_reset");
  if (bits & kErrTimeout) return fail(h, VDBEDT_ETIMEOUT, "a bounded device-side wait gave up");
  if (bits & kErrInvalidRecord) {
    // invalid device records were skipped; report once
    int zero = bits & ~kErrInvalidRecord;
    cudaMemcpyAsync(h->g.counters + C_ERR, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
    cudaStreamSynchronize(h->st);
    return fail(h, VDBEDT_EINVAL, "invalid occupancy records in device memory were skipped");
  }
  return fail(h, VDBEDT_EINTERNAL, "device-side consistency check failed");
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device address of page-locked (pinned or registered) host memory, or nullptr for pageable memory.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

vdbedt_status ensure_stage(vdbedt_map* h, int64_t need) {
  if (need <= h->stage_cap) return VDBEDT_OK;
  // records are indexed by int32 in the ordered ingest
  if (need > (int64_t)INT32_MAX) return fail(h, VDBEDT_EINVAL, "more than 2^31 - 1 records staged");
  int64_t cap = std::max<int64_t>(need + need / 2, 1 << 16);
  rec_t* p = nullptr;
  int32_t* q = nullptr;
  cudaError_t e = cudaMalloc((void**)&p, sizeof(rec_t) * (size_t)cap);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage alloc");
  e = cudaMalloc((void**)&q, sizeof(int32_t) * (size_t)cap);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(h, e, "stage alloc");
  }
  if (h->stage_n > 0) {
    e = cudaMemcpyAsync(p, h->stage, sizeof(rec_t) * (size_t)h->stage_n, cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "stage copy");
  }
  if (h->stage) {
    cudaStreamSynchronize(h->st);
    cudaFree(h->stage);
    cudaFree(h->stage_slot);
  }
  h->stage = p;
  h->stage_slot = q;
  h->stage_cap = cap;
  return VDBEDT_OK;
}

bool capturing(const vdbedt_map* h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(h->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// phase events are not recorded while the stream is being captured into a graph
void mark(vdbedt_map* h, int i) {
  if (h->profiling && !capturing(h)) cudaEventRecord(h->ev[i], h->st);
}

Tuning effective_tuning(const vdbedt_map* h) {
  Tuning t = h->tune;
  for (int a = 0; a < 3; ++a) t.run[a] = effective_run(h->g, h->tune, a);
  return t;
}

vdbedt_status run_passes(vdbedt_map* h, const Tuning& t, bool need_slots) {
  if (need_slots && half_path(h->g)) CK(h, launch_item_slots(h->g, t, h->items, h->st), "item slots");
  mark(h, 3);
  CK(h, launch_pass(h->g, t, 0, h->items, h->st), "x pass");
  mark(h, 4);
  CK(h, launch_pass(h->g, t, 1, h->items, h->st), "y pass");
  mark(h, 5);
  CK(h, launch_pass(h->g, t, 2, h->items, h->st), "z pass");
  mark(h, 6);
  h->ev_recorded = h->profiling && !capturing(h);
  return VDBEDT_OK;
}

const int32_t* stage_count(const vdbedt_map* h) { return h->stage_counted ? h->d_count : nullptr; }

void clear_stage(vdbedt_map* h) {
  h->stage_n = 0;
  h->stage_counted = false;
}

vdbedt_status do_global(vdbedt_map* h) {
  const Tuning t = effective_tuning(h);
  mark(h, 0);
  CK(h, cudaMemsetAsync(h->g.counters + C_HAS_ZERO, 0, sizeof(int32_t), h->st), "memset");
  if (h->stage_n > 0) {
    CK(h,
       launch_ingest_records(h->g, h->stage, h->stage_n, stage_count(h), false, h->changed, h->stage_slot, h->scr,
                             h->vlast, h->st),
       "ingest");
    clear_stage(h);
  }
  h->dense_pending = false;
  if (h->g.untrunc) {
    // every brick is stored: no activation or work lists, three whole-line passes
    CK(h, ensure_scratch(h->uts, ut_scratch_bytes(h->g)), "untruncated scratch");
    mark(h, 1);
    mark(h, 2);
    mark(h, 3);
    CK(h, launch_ut_pass(h->g, 0, h->uts.buf, h->st), "x pass");
    mark(h, 4);
    CK(h, launch_ut_pass(h->g, 1, h->uts.buf, h->st), "y pass");
    mark(h, 5);
    CK(h, launch_ut_pass(h->g, 2, h->uts.buf, h->st), "z pass");
    mark(h, 6);
    h->ev_recorded = h->profiling && !capturing(h);
    h->computed = true;
    return VDBEDT_OK;
  }
  mark(h, 1);
  CK(h, launch_activation_full(h->g, h->st), "activation");
  mark(h, 2);
  CK(h, launch_build_items_full(h->g, t, h->items, half_path(h->g), h->st), "items");
  vdbedt_status s = run_passes(h, t, false);
  if (s) return s;
  h->computed = true;
  return VDBEDT_OK;
}

// Per-brick storage and work lists of a batch grid, carved from the batch's pool.
struct PoolSlice {
  unsigned long long* occ;
  uint16_t* g1;
  uint16_t* g2;
  int32_t* dist;
  int4* bcoord;
  uint32_t* bflags;
  int32_t* bepoch;
  int32_t* counters;
  int32_t* items_ctr;
  Items items;
  int slot_base;
  int item_cap;
};

// Brick capacity of a configuration (after validation).
int64_t config_cap(const vdbedt_config* cfg) {
  const int64_t nbr = ceil_div(cfg->nx, 8) * ceil_div(cfg->ny, 8) * ceil_div(cfg->nz, 8);
  return cfg->max_bricks > 0 ? std::min<int64_t>(cfg->max_bricks, nbr) : nbr;
}

vdbedt_status create_impl(const vdbedt_config* cfg, const PoolSlice* slice, vdbedt_map** out) {
  if (!cfg || !out) return fail(nullptr, VDBEDT_EINVAL, "null argument");
  const bool unbounded = (cfg->flags & VDBEDT_FLAG_UNBOUNDED) != 0;
  const bool untrunc = (cfg->flags & VDBEDT_FLAG_UNTRUNCATED) != 0;
  if (cfg->flags & ~(uint32_t)(VDBEDT_FLAG_UNBOUNDED | VDBEDT_FLAG_UNTRUNCATED))
    return fail(nullptr, VDBEDT_EINVAL, "unknown flags");
  if (unbounded && slice) return fail(nullptr, VDBEDT_EINVAL, "a batch grid cannot be unbounded");
  if (untrunc && (slice || unbounded))
    return fail(nullptr, VDBEDT_EINVAL, "an untruncated grid is bounded and not part of a batch");
  if (unbounded && (cfg->max_bricks <= 0 || cfg->max_nodes <= 0))
    return fail(nullptr, VDBEDT_EINVAL, "an unbounded grid needs max_bricks and max_nodes");
  const int64_t nx = unbounded ? kUnboundedSize : cfg->nx, ny = unbounded ? kUnboundedSize : cfg->ny,
                nz = unbounded ? kUnboundedSize : cfg->nz;
  if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, VDBEDT_EINVAL, "grid size must be >= 1");
  if (untrunc ? cfg->dmax != 0 : (cfg->dmax < 1 || cfg->dmax > VDBEDT_DMAX_LIMIT))
    return fail(nullptr, VDBEDT_EINVAL, untrunc ? "an untruncated grid takes dmax 0" : "dmax out of range");
  // untruncated: every squared distance of the grid below VDBEDT_D_NONE
  if (untrunc && (nx - 1) * (nx - 1) + (ny - 1) * (ny - 1) + (nz - 1) * (nz - 1) >= (int64_t)VDBEDT_D_NONE)
    return fail(nullptr, VDBEDT_EINVAL, "untruncated grid too large for int32 distances");
  if (!(cfg->voxel_size > 0.f)) return fail(nullptr, VDBEDT_EINVAL, "voxel_size must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, VDBEDT_EINVAL, "no such CUDA device");
  }
  const int64_t BX = ceil_div(nx, 8), BY = ceil_div(ny, 8), BZ = ceil_div(nz, 8);
  // node keys stay below 2^42 - 1 (16,383 nodes per axis at most) and brick keys of bounded grids
  // fit 32 bits
  if (nx > kUnboundedSize || ny > kUnboundedSize || nz > kUnboundedSize ||
      (!unbounded && BX * BY * BZ >= (int64_t)0xFFFFFFFFll))
    return fail(nullptr, VDBEDT_EINVAL, "grid too large");
  const int64_t NX = ceil_div(BX, 16), NY = ceil_div(BY, 16), NZ = ceil_div(BZ, 16);
  int64_t cap = cfg->max_bricks > 0 ? std::min<int64_t>(cfg->max_bricks, BX * BY * BZ) : BX * BY * BZ;
  if (cap * 512 >= (int64_t)0xFFFFFFFFll) return fail(nullptr, VDBEDT_EINVAL, "brick capacity too large (max 8M)");
  const int64_t node_cap = cfg->max_nodes > 0 ? std::min<int64_t>(cfg->max_nodes, NX * NY * NZ) : NX * NY * NZ;
  if (untrunc && (cap < BX * BY * BZ || node_cap < NX * NY * NZ))
    return fail(nullptr, VDBEDT_EINVAL, "an untruncated grid stores every brick (max_bricks, max_nodes 0)");
  if (node_cap > kMaxNodes) return fail(nullptr, VDBEDT_EINVAL, "node capacity too large (max 4,194,302)");

  DeviceGuard guard(cfg->device);
  vdbedt_map* h = new vdbedt_map();
  h->cfg = *cfg;
  h->device = cfg->device;
  GridView& g = h->g;
  g.nx = (int)nx;
  g.ny = (int)ny;
  g.nz = (int)nz;
  g.unbounded = unbounded ? 1 : 0;
  g.off = unbounded ? kUnboundedOffset : 0;
  g.BX = (int)BX;
  g.BY = (int)BY;
  g.BZ = (int)BZ;
  g.NX = (int)NX;
  g.NY = (int)NY;
  g.NZ = (int)NZ;
  g.dmax = cfg->dmax;
  g.R = (cfg->dmax + 6) / 8;
  g.INF = untrunc ? kNone : cfg->dmax * cfg->dmax;
  g.half = (!untrunc && cfg->dmax <= 45 && g.R >= 1 && g.R <= 6) ? 1 : 0;  // fp16 fields unless the envelope form is chosen
  g.untrunc = untrunc ? 1 : 0;
  uint32_t hcap = 64;
  while ((int64_t)hcap < 2 * node_cap) hcap <<= 1;
  g.hmask = hcap - 1;
  g.cap = (int)cap;
  g.node_cap = (int)node_cap;

  auto bail = [&](cudaError_t e, const char* where) {
    vdbedt_status s = cuda_fail(nullptr, e, where);
    for (void* p : h->allocs) cudaFree(p);
    if (h->uts.buf) cudaFree(h->uts.buf);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    if (h->fork.side) cudaStreamDestroy(h->fork.side);
    if (h->fork.fork) cudaEventDestroy(h->fork.fork);
    if (h->fork.join) cudaEventDestroy(h->fork.join);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
    return s;
  };
  cudaError_t e = cudaSuccess;
  if (cfg->stream) {
    h->st = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e, "stream");
    h->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&h->fork.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork.join, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "side stream");
#define AL(ptr, count)                                   \
  do {                                                   \
    e = dalloc(h, &(ptr), (size_t)(count));              \
    if (e != cudaSuccess) return bail(e, "device alloc"); \
  } while (0)
  AL(g.hslots, hcap);
  AL(g.child, node_cap * kNodeBricks);
  AL(g.amask, node_cap * 128);
  AL(g.mwork, node_cap * 384);
  AL(g.nclaim, node_cap * 128);
  AL(g.node_key, node_cap);
  AL(g.mark, node_cap * 3 * 1024);
  if (slice) {
    g.occ = slice->occ;
    g.g1 = slice->g1;
    g.g2 = slice->g2;
    g.dist = slice->dist;
    g.bcoord = slice->bcoord;
    g.bflags = slice->bflags;
    g.bepoch = slice->bepoch;
    g.counters = slice->counters;
    g.items_ctr = slice->items_ctr;
    g.slot_base = slice->slot_base;
    g.item_cap = slice->item_cap;
    h->items = slice->items;
  } else {
    AL(g.occ, cap * 8);
    AL(g.g1, cap * kBrickVox * (untrunc ? 2 : 1));  // int32 intermediates when untruncated
    AL(g.g2, cap * kBrickVox * (untrunc ? 2 : 1));
    AL(g.dist, cap * kBrickVox);
    AL(g.bcoord, cap);
    AL(g.bflags, cap);
    AL(g.bepoch, cap);
    AL(g.counters, C_NUM);
    for (int a = 0; a < 3; ++a) {
      AL(h->items.run[a], cap);
      AL(h->items.slots[a], cap * kItemSlots);
    }
    g.items_ctr = g.counters + C_X_ITEMS;
    g.slot_base = 0;
    g.item_cap = (int)cap;
  }
  AL(h->changed, cap);
  AL(h->d_invalid, 4);
  if (untrunc) AL(g.ut_bits, ut_bits_words(g));
  h->d_count = h->d_invalid + 1;
#undef AL
  e = cudaMallocHost((void**)&h->h_pinned, 64 * sizeof(int32_t));
  if (e != cudaSuccess) return bail(e, "pinned alloc");
  cudaMemsetAsync(g.hslots, 0xFF, sizeof(unsigned long long) * hcap, h->st);
  cudaMemsetAsync(g.child, 0xFF, sizeof(int32_t) * (size_t)node_cap * kNodeBricks, h->st);
  cudaMemsetAsync(g.amask, 0, sizeof(uint32_t) * (size_t)node_cap * 128, h->st);
  cudaMemsetAsync(g.mwork, 0, sizeof(uint32_t) * (size_t)node_cap * 384, h->st);
  cudaMemsetAsync(g.nclaim, 0, sizeof(uint32_t) * (size_t)node_cap * 128, h->st);
  cudaMemsetAsync(g.mark, 0, sizeof(int32_t) * (size_t)node_cap * 3 * 1024, h->st);
  if (!slice) cudaMemsetAsync(g.counters, 0, sizeof(int32_t) * C_NUM, h->st);
  if (untrunc) {
    cudaMemsetAsync(g.ut_bits, 0, sizeof(uint32_t) * (size_t)ut_bits_words(g), h->st);
    // the line stacks too, so that a transform allocates nothing (and can be captured)
    e = ensure_scratch(h->uts, ut_scratch_bytes(g));
    if (e != cudaSuccess) return bail(e, "untruncated scratch");
    e = launch_ut_init(g, h->st);
    if (e != cudaSuccess) return bail(e, "untruncated init");
  }
  e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return bail(e, "init");
  *out = h;
  return VDBEDT_OK;
}

}  // namespace

extern "C" {

vdbedt_status vdbedt_create(const vdbedt_config* cfg, vdbedt_handle* out) {
  vdbedt_map* h = nullptr;
  vdbedt_status s = create_impl(cfg, nullptr, &h);
  if (s == VDBEDT_OK) *out = h;
  return s;
}

}  // extern "C"

namespace {
void destroy_impl(vdbedt_map* h) {
  DeviceGuard guard(h->device);
  cudaStreamSynchronize(h->st);
  for (void* p : h->allocs) cudaFree(p);
  if (h->stage) cudaFree(h->stage);
  if (h->stage_slot) cudaFree(h->stage_slot);
  if (h->scr.buf) cudaFree(h->scr.buf);
  if (h->vlast.buf) cudaFree(h->vlast.buf);
  if (h->io.buf) cudaFree(h->io.buf);
  if (h->uts.buf) cudaFree(h->uts.buf);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  for (int i = 0; i < 7; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->fork.side) cudaStreamDestroy(h->fork.side);
  if (h->fork.fork) cudaEventDestroy(h->fork.fork);
  if (h->fork.join) cudaEventDestroy(h->fork.join);
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
}
}  // namespace

extern "C" {

vdbedt_status vdbedt_destroy(vdbedt_handle h) {
  if (!h) return VDBEDT_OK;
  if (h->batch) return fail(h, VDBEDT_EINVAL, "a batch grid is released with its batch");
  destroy_impl(h);
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_occupancy(vdbedt_handle h, const int32_t* xyz, const uint8_t* occ, int64_t n,
                                   int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0) return fail(h, VDBEDT_EINVAL, "negative record count");
  if (n == 0) return VDBEDT_OK;
  if (!xyz || !occ) return fail(h, VDBEDT_EINVAL, "null records");
  if (h->stage_counted) return fail(h, VDBEDT_EINVAL, "records staged with a device count must be applied first");
  DeviceGuard guard(h->device);
  s = ensure_stage(h, h->stage_n + n);
  if (s) return s;
  rec_t* dst = h->stage + h->stage_n;
  if (on_device) {
    CK(h, launch_pack_records(xyz, occ, n, nullptr, nullptr, h->g.nx, h->g.ny, h->g.nz, h->g.off, dst, nullptr, h->g.counters,
                              h->st), "pack");
  } else {
    // pack and validate on the device, then check before accepting.  Page-locked host arrays are
    // read by the pack kernel in place (mapped host memory); other host arrays are copied first.
    const int32_t* dxyz = static_cast<const int32_t*>(mapped_host(xyz));
    const uint8_t* docc = static_cast<const uint8_t*>(mapped_host(occ));
    if (!dxyz || !docc) {
      size_t bxyz = ((size_t)n * 12 + 255) & ~(size_t)255;
      CK(h, ensure_scratch(h->io, bxyz + (size_t)n + 256), "io alloc");
      int32_t* cxyz = (int32_t*)h->io.buf;
      uint8_t* cocc = (uint8_t*)h->io.buf + bxyz;
      CK(h, cudaMemcpyAsync(cxyz, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, h->st), "h2d");
      CK(h, cudaMemcpyAsync(cocc, occ, (size_t)n, cudaMemcpyHostToDevice, h->st), "h2d");
      dxyz = cxyz;
      docc = cocc;
    }
    CK(h, cudaMemsetAsync(h->d_invalid, 0, sizeof(int32_t), h->st), "memset");
    CK(h, launch_pack_records(dxyz, docc, n, nullptr, nullptr, h->g.nx, h->g.ny, h->g.nz, h->g.off, dst, h->d_invalid,
                              h->g.counters, h->st),
       "pack");
    CK(h, cudaMemcpyAsync(h->h_pinned, h->d_invalid, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st), "d2h");
    CK(h, cudaStreamSynchronize(h->st), "sync");
    if (h->h_pinned[0] != 0)
      return fail(h, VDBEDT_EINVAL, "record outside the grid or occupancy value > 1; call rejected");
  }
  h->stage_n += n;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_occupancy_packed(vdbedt_handle h, const uint64_t* rec, int64_t n, int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0) return fail(h, VDBEDT_EINVAL, "negative record count");
  if (n == 0) return VDBEDT_OK;
  if (!rec) return fail(h, VDBEDT_EINVAL, "null records");
  if (h->stage_counted) return fail(h, VDBEDT_EINVAL, "records staged with a device count must be applied first");
  DeviceGuard guard(h->device);
  s = ensure_stage(h, h->stage_n + n);
  if (s) return s;
  rec_t* dst = h->stage + h->stage_n;
  const uint64_t* src = rec;
  if (!on_device) {
    // page-locked host records are read in place (mapped host memory); others are copied first
    src = static_cast<const uint64_t*>(mapped_host(rec));
    if (!src) {
      CK(h, ensure_scratch(h->io, (size_t)n * 8), "io alloc");
      CK(h, cudaMemcpyAsync(h->io.buf, rec, (size_t)n * 8, cudaMemcpyHostToDevice, h->st), "h2d");
      src = (const uint64_t*)h->io.buf;
    }
    CK(h, cudaMemsetAsync(h->d_invalid, 0, sizeof(int32_t), h->st), "memset");
  }
  CK(h, launch_check_packed(src, n, h->g.nx, h->g.ny, h->g.nz, dst, on_device ? nullptr : h->d_invalid,
                            h->g.counters, h->st),
     "check");
  if (!on_device) {
    CK(h, cudaMemcpyAsync(h->h_pinned, h->d_invalid, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st), "d2h");
    CK(h, cudaStreamSynchronize(h->st), "sync");
    if (h->h_pinned[0] != 0) return fail(h, VDBEDT_EINVAL, "packed record outside the grid; call rejected");
  }
  h->stage_n += n;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_occupancy_bricks(vdbedt_handle h, const int32_t* bxyz, const uint64_t* masks, int64_t n,
                                          int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0) return fail(h, VDBEDT_EINVAL, "negative brick count");
  if (n == 0) return VDBEDT_OK;
  if (!bxyz || !masks) return fail(h, VDBEDT_EINVAL, "null bricks");
  if (h->stage_counted) return fail(h, VDBEDT_EINVAL, "records staged with a device count must be applied first");
  DeviceGuard guard(h->device);
  // the bricks on the device (host arrays copied once: both passes read them), two counter words
  // (invalid bricks, then the 64-bit bit count / write cursor) after them
  const size_t bk = ((size_t)n * 12 + 255) & ~(size_t)255, bm = ((size_t)n * 64 + 255) & ~(size_t)255;
  CK(h, ensure_scratch(h->io, (on_device ? 0 : bk + bm) + 256), "io alloc");
  const int32_t* dk = bxyz;
  const uint64_t* dm = masks;
  char* ctr = (char*)h->io.buf + (on_device ? 0 : bk + bm);
  if (!on_device) {
    CK(h, cudaMemcpyAsync(h->io.buf, bxyz, (size_t)n * 12, cudaMemcpyHostToDevice, h->st), "h2d");
    CK(h, cudaMemcpyAsync((char*)h->io.buf + bk, masks, (size_t)n * 64, cudaMemcpyHostToDevice, h->st), "h2d");
    dk = (const int32_t*)h->io.buf;
    dm = (const uint64_t*)((char*)h->io.buf + bk);
  }
  int32_t* invalid = (int32_t*)ctr;
  unsigned long long* count = (unsigned long long*)(ctr + 8);
  CK(h, cudaMemsetAsync(ctr, 0, 16, h->st), "memset");
  CK(h, launch_check_bricks(dk, dm, n, h->g, invalid, count, h->st), "check bricks");
  CK(h, cudaMemcpyAsync(h->h_pinned + 48, ctr, 16, cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  if (h->h_pinned[48] != 0) return fail(h, VDBEDT_EINVAL, "brick outside the grid or bit for a voxel outside it; call rejected");
  unsigned long long bits = 0;
  memcpy(&bits, h->h_pinned + 50, sizeof(bits));
  if (bits == 0) return VDBEDT_OK;
  s = ensure_stage(h, h->stage_n + (int64_t)bits);
  if (s) return s;
  CK(h, cudaMemsetAsync(count, 0, 8, h->st), "memset");
  CK(h, launch_expand_bricks(dk, dm, n, h->g, h->stage + h->stage_n, count, h->st), "expand bricks");
  h->stage_n += (int64_t)bits;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_occupancy_counted(vdbedt_handle h, const int32_t* xyz, const uint8_t* occ,
                                           const int32_t* n_dev, int64_t n_max) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n_max < 1 || n_max > INT32_MAX || !xyz || !occ || !n_dev)
    return fail(h, VDBEDT_EINVAL, "bad counted records (need n_max in [1, 2^31) and device pointers)");
  if (h->stage_n > 0) return fail(h, VDBEDT_EINVAL, "counted records need an empty stage");
  DeviceGuard guard(h->device);
  s = ensure_stage(h, n_max);
  if (s) return s;
  CK(h, reserve_ingest(h->g, n_max, h->scr, h->vlast, h->st), "ingest scratch");
  CK(h, launch_pack_records(xyz, occ, n_max, n_dev, h->d_count, h->g.nx, h->g.ny, h->g.nz, h->g.off, h->stage, nullptr,
                              h->g.counters, h->st),
     "pack");
  h->stage_n = n_max;
  h->stage_counted = true;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_occupancy_dense(vdbedt_handle h, const uint8_t* grid, int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!grid) return fail(h, VDBEDT_EINVAL, "null grid");
  if (h->g.unbounded) return fail(h, VDBEDT_EINVAL, "an unbounded grid has no dense form");
  DeviceGuard guard(h->device);
  s = vdbedt_reset(h);
  if (s) return s;
  const uint8_t* src = grid;
  if (!on_device) {
    size_t bytes = (size_t)h->g.nx * h->g.ny * h->g.nz;
    CK(h, ensure_scratch(h->io, bytes), "io alloc");
    CK(h, cudaMemcpyAsync(h->io.buf, grid, bytes, cudaMemcpyHostToDevice, h->st), "h2d");
    src = (const uint8_t*)h->io.buf;
  }
  CK(h, h->g.untrunc ? launch_ut_dense(h->g, src, h->st) : launch_ingest_dense(h->g, src, h->scr, h->st),
     "dense ingest");
  if (!on_device) CK(h, cudaStreamSynchronize(h->st), "sync");
  h->dense_pending = true;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_reset(vdbedt_handle h) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  DeviceGuard guard(h->device);
  CK(h, h->g.untrunc ? launch_ut_reset(h->g, h->st) : launch_reset(h->g, h->st), "reset");
  if (h->g.untrunc)
    CK(h, cudaMemsetAsync(h->g.ut_bits, 0, sizeof(uint32_t) * (size_t)ut_bits_words(h->g), h->st), "memset");
  clear_stage(h);
  h->computed = false;
  h->dense_pending = false;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_global(vdbedt_handle h) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  DeviceGuard guard(h->device);
  return do_global(h);
}

vdbedt_status vdbedt_update(vdbedt_handle h, vdbedt_update_stats* stats) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  DeviceGuard guard(h->device);
  const int64_t nrec = h->stage_n;
  const bool counted = h->stage_counted;
  const bool whole = !h->computed || h->dense_pending;
  if (whole) {
    s = do_global(h);
    if (s) return s;
  } else if (h->g.untrunc) {
    // untruncated: the tracked ingest marks the rows of the flipped voxels; each pass recomputes
    // the lines whose input changed and marks the next axis's lines where its output changed
    mark(h, 0);
    CK(h, launch_begin_update(h->g, h->st), "begin update");
    if (h->stage_n > 0) {
      CK(h,
         launch_ingest_records(h->g, h->stage, h->stage_n, stage_count(h), true, h->changed, h->stage_slot, h->scr,
                               h->vlast, h->st),
         "ingest");
      clear_stage(h);
    }
    mark(h, 1);
    mark(h, 2);
    mark(h, 3);
    CK(h, launch_ut_update_pass(h->g, 0, h->uts.buf, h->st), "x pass");
    mark(h, 4);
    CK(h, launch_ut_update_pass(h->g, 1, h->uts.buf, h->st), "y pass");
    mark(h, 5);
    CK(h, launch_ut_update_pass(h->g, 2, h->uts.buf, h->st), "z pass");
    mark(h, 6);
    h->ev_recorded = h->profiling && !capturing(h);
  } else {
    const Tuning t = effective_tuning(h);
    mark(h, 0);
    CK(h, launch_begin_update(h->g, h->st), "begin update");
    if (h->stage_n > 0) {
      CK(h,
         launch_ingest_records(h->g, h->stage, h->stage_n, stage_count(h), true, h->changed, h->stage_slot, h->scr,
                               h->vlast, h->st),
         "ingest");
      clear_stage(h);
    }
    mark(h, 1);
    CK(h, launch_incremental_mark(h->g, t, h->changed, h->items, h->fork, h->st), "mark");
    mark(h, 2);
    // slot lists of the dirty runs (an update that switched to the global form got them with its
    // work lists), then the side stream's branch joins before the passes
    if (half_path(h->g)) CK(h, launch_item_slots(h->g, t, h->items, h->st), "item slots");
    CK(h, cudaStreamWaitEvent(h->st, h->fork.join, 0), "join");
    s = run_passes(h, t, false);
    if (s) return s;
    if (stats && half_path(h->g))
      CK(h, launch_count_run_bricks(nullptr, h->g, h->g.items_ctr, h->g.item_cap, t, h->items, h->st), "count");
  }
  if (stats) {
    CK(h, cudaMemcpyAsync(h->h_pinned, h->g.counters, sizeof(int32_t) * C_NUM, cudaMemcpyDeviceToHost, h->st), "d2h");
    CK(h, cudaMemcpyAsync(h->h_pinned + 44, h->g.items_ctr, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, h->st), "d2h");
    if (counted)
      CK(h, cudaMemcpyAsync(h->h_pinned + 40, h->d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st), "d2h");
    s = device_errors(h);  // synchronises
    if (s) return s;
    const int32_t* c = h->h_pinned;
    stats->records = counted ? h->h_pinned[40] : nrec;
    stats->net_flips = c[C_FLIPS];
    stats->changed_bricks = c[C_CHANGED];
    stats->x_items = c[44];
    stats->y_items = c[45];
    stats->z_items = c[46];
    stats->new_bricks = c[C_NEW_BRICKS];
    stats->x_bricks = c[C_XB];
    stats->y_bricks = c[C_YB];
    stats->z_bricks = c[C_ZB];
    stats->global_form = whole ? 1 : c[C_BIG];
  }
  return VDBEDT_OK;
}

vdbedt_status vdbedt_query(vdbedt_handle h, const int32_t* xyz, int64_t n, int32_t* out_sqdist, int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0 || (n > 0 && (!xyz || !out_sqdist))) return fail(h, VDBEDT_EINVAL, "bad query arguments");
  if (n == 0) return VDBEDT_OK;
  DeviceGuard guard(h->device);
  if (on_device) {
    CK(h, launch_query(h->g, xyz, n, out_sqdist, h->st), "query");
    return VDBEDT_OK;
  }
  size_t bx = ((size_t)n * 12 + 255) & ~(size_t)255;
  CK(h, ensure_scratch(h->io, bx + (size_t)n * 4), "io alloc");
  int32_t* dxyz = (int32_t*)h->io.buf;
  int32_t* dout = (int32_t*)((char*)h->io.buf + bx);
  CK(h, cudaMemcpyAsync(dxyz, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, h->st), "h2d");
  CK(h, launch_query(h->g, dxyz, n, dout, h->st), "query");
  s = device_errors(h);
  if (s) return s;
  CK(h, cudaMemcpyAsync(out_sqdist, dout, (size_t)n * 4, cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_query_nearest(vdbedt_handle h, const int32_t* xyz, int64_t n, int32_t* out_xyz, int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0 || (n > 0 && (!xyz || !out_xyz))) return fail(h, VDBEDT_EINVAL, "bad query arguments");
  if (h->g.untrunc) return fail(h, VDBEDT_EINVAL, "no nearest-obstacle query on an untruncated grid");
  if (n == 0) return VDBEDT_OK;
  DeviceGuard guard(h->device);
  if (on_device) {
    CK(h, launch_query_nearest(h->g, xyz, n, out_xyz, h->st), "nearest");
    return VDBEDT_OK;
  }
  size_t bx = ((size_t)n * 12 + 255) & ~(size_t)255;
  CK(h, ensure_scratch(h->io, 2 * bx), "io alloc");
  int32_t* dxyz = (int32_t*)h->io.buf;
  int32_t* dout = (int32_t*)((char*)h->io.buf + bx);
  CK(h, cudaMemcpyAsync(dxyz, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, h->st), "h2d");
  CK(h, launch_query_nearest(h->g, dxyz, n, dout, h->st), "nearest");
  s = device_errors(h);
  if (s) return s;
  CK(h, cudaMemcpyAsync(out_xyz, dout, (size_t)n * 12, cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_export_dense(vdbedt_handle h, int32_t* out, int on_device) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!out) return fail(h, VDBEDT_EINVAL, "null output");
  if (h->g.unbounded) return fail(h, VDBEDT_EINVAL, "an unbounded grid has no dense form");
  DeviceGuard guard(h->device);
  size_t bytes = (size_t)h->g.nx * h->g.ny * h->g.nz * 4;
  if (on_device) {
    CK(h, launch_export_dense(h->g, out, h->st), "export");
    return VDBEDT_OK;
  }
  CK(h, ensure_scratch(h->io, bytes), "io alloc");
  CK(h, launch_export_dense(h->g, (int32_t*)h->io.buf, h->st), "export");
  s = device_errors(h);
  if (s) return s;
  CK(h, cudaMemcpyAsync(out, h->io.buf, bytes, cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_export_occupancy(vdbedt_handle h, int32_t z_lo, int32_t z_hi, int32_t dz, int32_t mode,
                                      uint64_t* out, int64_t max_n, int64_t* n_out) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!n_out || (max_n > 0 && !out) || max_n < 0 || (mode != 0 && mode != 1))
    return fail(h, VDBEDT_EINVAL, "bad export arguments");
  // caller z -> stored z (an unbounded grid's coordinates are stored shifted)
  const int64_t zl = std::max<int64_t>((int64_t)z_lo + h->g.off, 0), zh = std::min<int64_t>((int64_t)z_hi + h->g.off, h->g.nz);
  z_lo = (int32_t)zl;
  z_hi = (int32_t)std::max<int64_t>(zh, zl);
  if (z_hi <= z_lo) {
    *n_out = 0;
    return VDBEDT_OK;
  }
  if ((int64_t)z_lo + dz < 0 || (int64_t)z_hi + dz > (int64_t)kBadCoord)
    return fail(h, VDBEDT_EINVAL, "shifted z outside [0, 2^21 - 1)");
  DeviceGuard guard(h->device);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(h->d_invalid + 2);
  CK(h, launch_export_occupancy(h->g, h->changed, z_lo, z_hi, dz, mode, reinterpret_cast<unsigned long long*>(out),
                                max_n, cnt, h->st),
     "export occupancy");
  s = device_errors(h);
  if (s) return s;
  CK(h, cudaMemcpyAsync(h->h_pinned + 48, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  unsigned long long c = 0;
  memcpy(&c, h->h_pinned + 48, sizeof(c));
  *n_out = (int64_t)c;
  if ((int64_t)c > max_n) return fail(h, VDBEDT_EOVERFLOW, "more records than max_n (the count is in *n_out)");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_distance_at(vdbedt_handle h, const float* pts, int64_t n, float* dist, float* grad) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (n < 0 || (n > 0 && (!pts || !dist))) return fail(h, VDBEDT_EINVAL, "bad distance arguments");
  if (h->g.nx < 2 || h->g.ny < 2 || h->g.nz < 2) return fail(h, VDBEDT_EINVAL, "grid needs >= 2 voxels per axis");
  DeviceGuard guard(h->device);
  CK(h, launch_distance_at(h->g, h->cfg.voxel_size, pts, n, dist, grad, h->st), "distance");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_clearance_forward(vdbedt_handle h, const float* pts, int64_t T, int64_t P, float tau,
                                       float* cost) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (T < 0 || P < 0 || (T > 0 && (!pts || !cost))) return fail(h, VDBEDT_EINVAL, "bad clearance arguments");
  if (h->g.nx < 2 || h->g.ny < 2 || h->g.nz < 2) return fail(h, VDBEDT_EINVAL, "grid needs >= 2 voxels per axis");
  DeviceGuard guard(h->device);
  CK(h, launch_clearance_fwd(h->g, h->cfg.voxel_size, pts, T, P, tau, cost, h->st), "clearance fwd");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_clearance_backward(vdbedt_handle h, const float* pts, int64_t T, int64_t P, float tau,
                                        const float* grad_cost, float* grad_pts) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (T < 0 || P < 0 || (T > 0 && P > 0 && (!pts || !grad_cost || !grad_pts)))
    return fail(h, VDBEDT_EINVAL, "bad clearance arguments");
  if (h->g.nx < 2 || h->g.ny < 2 || h->g.nz < 2) return fail(h, VDBEDT_EINVAL, "grid needs >= 2 voxels per axis");
  DeviceGuard guard(h->device);
  CK(h, launch_clearance_bwd(h->g, h->cfg.voxel_size, pts, T, P, tau, grad_cost, grad_pts, h->st), "clearance bwd");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_set_tuning(vdbedt_handle h, const vdbedt_tuning* t) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!t) return fail(h, VDBEDT_EINVAL, "null tuning");
  if (h->g.untrunc) return fail(h, VDBEDT_EINVAL, "an untruncated grid has no tuning");
  auto ok_run = [](int r) { return r == 0 || r == 4 || r == 8 || r == 16; };
  const int v = t->variant;
  if (!ok_run(t->x_run) || !ok_run(t->y_run) || !ok_run(t->z_run) ||
      !(v == 0 || v == 1 || v == 3 || v == 5 || v == 7 || v == kVariantEnvelope))
    return fail(h, VDBEDT_EINVAL, "bad tuning");
  const Tuning d;
  h->tune.run[0] = t->x_run ? t->x_run : d.run[0];
  h->tune.run[1] = t->y_run ? t->y_run : d.run[1];
  h->tune.run[2] = t->z_run ? t->z_run : d.run[2];
  h->tune.variant = v ? v : d.variant;
  // the windowed kernels keep fp16 fields, the envelope kernels 16-bit integers: a change of form
  // makes the stored intermediates unusable, so the next update recomputes the whole field
  const int half = (h->cfg.dmax <= 45 && h->g.R >= 1 && h->g.R <= 6 && h->tune.variant != kVariantEnvelope) ? 1 : 0;
  if (half != h->g.half) {
    h->g.half = half;
    h->computed = false;
  }
  return VDBEDT_OK;
}

vdbedt_status vdbedt_synchronize(vdbedt_handle h) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  DeviceGuard guard(h->device);
  return device_errors(h);
}

vdbedt_status vdbedt_get_info(vdbedt_handle h, vdbedt_info* info) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!info) return fail(h, VDBEDT_EINVAL, "null info");
  DeviceGuard guard(h->device);
  CK(h, launch_count_flags(h->g, h->st), "count");
  s = device_errors(h);  // synchronises
  if (s) return s;
  CK(h, cudaMemcpyAsync(h->h_pinned, h->g.counters, sizeof(int32_t) * C_NUM, cudaMemcpyDeviceToHost, h->st), "d2h");
  CK(h, cudaStreamSynchronize(h->st), "sync");
  info->allocated_bricks = std::min(h->h_pinned[C_NBRICKS], h->g.cap);
  info->obstacle_bricks = h->h_pinned[C_OBST];
  info->finite_bricks = h->h_pinned[C_FINITE];
  info->capacity_bricks = h->g.cap;
  info->nodes = h->h_pinned[C_NNODES];
  info->device_bytes =
      (int64_t)(h->device_bytes + h->scr.bytes + h->vlast.bytes + h->io.bytes +
                (sizeof(rec_t) + sizeof(int32_t)) * h->stage_cap);
  info->R = h->g.R;
  info->error_bits = h->h_pinned[C_ERR];
  return VDBEDT_OK;
}

void* vdbedt_stream(vdbedt_handle h) { return h ? (void*)h->st : nullptr; }

vdbedt_status vdbedt_set_profiling(vdbedt_handle h, int on) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  DeviceGuard guard(h->device);
  if (on && !h->ev[0])
    for (int i = 0; i < 7; ++i) CK(h, cudaEventCreate(&h->ev[i]), "event");
  h->profiling = on != 0;
  h->ev_recorded = false;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_get_phase_times(vdbedt_handle h, vdbedt_phase_times* out) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (!out) return fail(h, VDBEDT_EINVAL, "null output");
  if (!h->ev_recorded) return fail(h, VDBEDT_EINVAL, "no profiled transform since profiling was enabled");
  DeviceGuard guard(h->device);
  CK(h, cudaEventSynchronize(h->ev[6]), "event sync");
  float ms[6];
  for (int i = 0; i < 6; ++i) CK(h, cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]), "event time");
  out->ingest_ms = ms[0];
  out->activation_ms = ms[1];
  out->items_ms = ms[2];
  out->x_ms = ms[3];
  out->y_ms = ms[4];
  out->z_ms = ms[5];
  return VDBEDT_OK;
}

int64_t vdbedt_kernel_launches(void) { return (int64_t)g_launches.load(); }

vdbedt_status vdbedt_selftest_wait_timeout(vdbedt_handle h, int32_t which) {
  vdbedt_status s = check_handle(h);
  if (s) return s;
  if (which != 0 && which != 1) return fail(h, VDBEDT_EINVAL, "which must be 0 or 1");
  DeviceGuard guard(h->device);
  CK(h, launch_wait_selftest(h->g, which, h->st), "wait self-test");
  return VDBEDT_OK;
}

const char* vdbedt_last_error(vdbedt_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

}  // extern "C"

// ---- batches of grids ----
struct vdbedt_batch {
  int k = 0;
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<vdbedt_map*> maps;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  GridView pool{};               // pass view over the shared pool (the batch's counters and work lists)
  Items items{};                 // work lists of every grid of the batch
  int32_t* counters = nullptr;   // (k + 1) * C_NUM words: grid i at i * C_NUM, the batch at k * C_NUM
  GridView* d_views = nullptr;   // the k grids' views in device memory
  BatchShape shape{};
  Scratch io;
  Scratch scr;                     // dense-ingest scratch (all grids)
  size_t dense_bytes = 0;          // its size
  int64_t* d_dense_off = nullptr;  // per grid: mask, brick-flag, node-flag element offsets
  size_t dense_nflag_byte = 0, dense_nflag_words = 0;
  Tuning tune;
  std::string err;
  bool profiling = false;
  cudaEvent_t ev[6] = {};
  bool ev_recorded = false;
  UpdArgs* d_upd = nullptr;  // the grids' update arguments in device memory
  UpdArgs* h_upd = nullptr;  // and their page-locked host copy
  Fork fork;                 // side stream of the update's global-form branch
};

namespace {

int32_t* batch_error_word(const vdbedt_map* h) { return h->batch->counters + (size_t)h->batch->k * C_NUM + C_ERR; }

vdbedt_status bfail(vdbedt_batch* b, vdbedt_status s, const std::string& msg) {
  if (b) b->err = msg;
  g_last_error = msg;
  return s;
}

void destroy_batch(vdbedt_batch* b) {
  DeviceGuard guard(b->device);
  if (b->st) cudaStreamSynchronize(b->st);
  for (vdbedt_map* m : b->maps) destroy_impl(m);
  for (void* p : b->allocs) cudaFree(p);
  if (b->io.buf) cudaFree(b->io.buf);
  if (b->scr.buf) cudaFree(b->scr.buf);
  for (int i = 0; i < 6; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  if (b->h_upd) cudaFreeHost(b->h_upd);
  if (b->fork.side) cudaStreamDestroy(b->fork.side);
  if (b->fork.fork) cudaEventDestroy(b->fork.fork);
  if (b->fork.join) cudaEventDestroy(b->fork.join);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

void bmark(vdbedt_batch* b, int i) {
  if (b->profiling) cudaEventRecord(b->ev[i], b->st);
}

vdbedt_status batch_members_ok(vdbedt_batch* b) {
  for (vdbedt_map* m : b->maps)
    if (m->sticky == VDBEDT_ECUDA) return bfail(b, VDBEDT_ECUDA, "a grid of the batch hit a CUDA error");
  return VDBEDT_OK;
}

#define BCK(b, expr, where)                                                                          \
  do {                                                                                             \
    cudaError_t _e = (expr);                                                                       \
    if (_e != cudaSuccess) {                                                                       \
      for (vdbedt_map* _m : (b)->maps) _m->sticky = VDBEDT_ECUDA;                                  \
      return bfail((b), _e == cudaErrorMemoryAllocation ? VDBEDT_ENOMEM : VDBEDT_ECUDA,            \
                   std::string(where) + ": " + cudaGetErrorString(_e));                            \
    }                                                                                              \
  } while (0)

vdbedt_status batch_global(vdbedt_batch* b) {
  vdbedt_status s = batch_members_ok(b);
  if (s) return s;
  DeviceGuard guard(b->device);
  const GridView& g0 = b->maps[0]->g;
  if (!half_path(g0)) {
    // the envelope kernels find bricks through each grid's own tables: grid by grid (the phase
    // events then put the whole transform in the last phase)
    for (int i = 0; i < 5; ++i) bmark(b, i);
    for (vdbedt_map* m : b->maps) {
      s = do_global(m);
      if (s) return bfail(b, s, m->err);
    }
    bmark(b, 5);
    b->ev_recorded = b->profiling;
    return VDBEDT_OK;
  }
  Tuning t = b->tune;
  for (int a = 0; a < 3; ++a) t.run[a] = effective_run(g0, b->tune, a);
  bmark(b, 0);
  // staged records: applied grid by grid (the sort-based ingest keeps per-grid scratch)
  for (vdbedt_map* m : b->maps) {
    if (m->stage_n <= 0) continue;
    BCK(b, cudaMemsetAsync(m->g.counters + C_HAS_ZERO, 0, sizeof(int32_t), b->st), "memset");
    BCK(b,
        launch_ingest_records(m->g, m->stage, m->stage_n, stage_count(m), false, nullptr, m->stage_slot, m->scr,
                              m->vlast, b->st),
        "ingest");
    clear_stage(m);
  }
  bmark(b, 1);
  BCK(b, launch_activation_batch(b->d_views, b->shape, b->st), "activation");
  bmark(b, 2);
  BCK(b, launch_build_items_batch(b->d_views, b->shape, t, b->items, b->pool.items_ctr, b->st), "items");
  bmark(b, 3);
  BCK(b, launch_pass(b->pool, t, 0, b->items, b->st), "x pass");
  bmark(b, 4);
  BCK(b, launch_pass(b->pool, t, 1, b->items, b->st), "y pass");
  BCK(b, launch_pass(b->pool, t, 2, b->items, b->st), "z pass");
  bmark(b, 5);
  b->ev_recorded = b->profiling;
  for (vdbedt_map* m : b->maps) {
    m->computed = true;
    m->dense_pending = false;
  }
  return VDBEDT_OK;
}

// Incremental update of every grid of a batch: each step (begin, tracked ingest, marking, slot
// lists, the three passes) is one launch for all grids; the dirty runs of every grid go to the
// batch's shared work queue, tagged with their grid.
vdbedt_status batch_update(vdbedt_batch* b, vdbedt_update_stats* stats) {
  vdbedt_status s = batch_members_ok(b);
  if (s) return s;
  DeviceGuard guard(b->device);
  const GridView& g0 = b->maps[0]->g;
  bool fresh = true;
  for (vdbedt_map* m : b->maps) fresh &= m->computed && !m->dense_pending;
  std::vector<int64_t> nrec((size_t)b->k);
  std::vector<char> counted((size_t)b->k);
  for (int i = 0; i < b->k; ++i) {
    nrec[(size_t)i] = b->maps[(size_t)i]->stage_n;
    counted[(size_t)i] = b->maps[(size_t)i]->stage_counted;
  }
  if (!fresh) {
    // a grid without a field yet: the global transform of the whole batch (applies the records)
    s = batch_global(b);
    if (s) return s;
  } else if (!half_path(g0)) {
    // the envelope form: grid by grid
    for (vdbedt_map* m : b->maps) {
      s = vdbedt_update(m, nullptr);
      if (s) return bfail(b, s, m->err);
    }
  } else {
    Tuning t = b->tune;
    for (int a = 0; a < 3; ++a) t.run[a] = effective_run(g0, b->tune, a);
    // The grids' arguments in device memory stay fixed while staging does not reallocate (every
    // grid reads its record count from its device count word), so a captured update replays with
    // the same arguments; they are uploaded again only when they change, outside a capture.
    BatchUpdShape shape{b->k, 0, 0, g0.R, half_path(g0)};
    BatchCounts counts{};
    std::vector<UpdArgs> args((size_t)b->k);
    for (int i = 0; i < b->k; ++i) {
      vdbedt_map* m = b->maps[(size_t)i];
      UpdArgs& a = args[(size_t)i];
      a.g = m->g;
      a.rec = m->stage;
      a.n = m->stage_cap;
      a.n_dev = m->d_count;
      a.changed = m->changed;
      a.rslot = m->stage_slot;
      BCK(b, prepare_update_args(m->g, m->vlast, a, b->st), "update scratch");
      counts.c[i] = m->stage_counted ? -1 : (int32_t)m->stage_n;  // -1: the counted staging wrote it
      shape.max_n = std::max<int64_t>(shape.max_n, m->stage_cap);
      shape.max_node_cap = std::max<int64_t>(shape.max_node_cap, m->g.node_cap);
    }
    if (memcmp(args.data(), b->h_upd, sizeof(UpdArgs) * (size_t)b->k) != 0) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(b->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return bfail(b, VDBEDT_EINVAL, "batch update captured before an uncaptured call with the same staging");
      BCK(b, cudaStreamSynchronize(b->st), "sync");  // earlier updates may still read the old arguments
      memcpy(b->h_upd, args.data(), sizeof(UpdArgs) * (size_t)b->k);
      BCK(b, cudaMemcpyAsync(b->d_upd, b->h_upd, sizeof(UpdArgs) * (size_t)b->k, cudaMemcpyHostToDevice, b->st),
          "update arguments");
      BCK(b, cudaStreamSynchronize(b->st), "sync");
    }
    bmark(b, 0);
    BCK(b, launch_update_batch_ingest(b->d_upd, shape, counts, b->st), "ingest");
    for (vdbedt_map* m : b->maps) clear_stage(m);
    bmark(b, 1);
    BCK(b, launch_update_batch_mark(b->d_upd, shape, t, b->items, b->fork, b->st), "mark");
    BCK(b, cudaStreamWaitEvent(b->st, b->fork.join, 0), "join");
    bmark(b, 2);
    BCK(b, launch_item_slots_batch(b->d_views, t, b->items, b->pool.items_ctr, b->pool.item_cap, b->st), "item slots");
    bmark(b, 3);
    BCK(b, launch_pass(b->pool, t, 0, b->items, b->st), "x pass");
    bmark(b, 4);
    BCK(b, launch_pass(b->pool, t, 1, b->items, b->st), "y pass");
    BCK(b, launch_pass(b->pool, t, 2, b->items, b->st), "z pass");
    bmark(b, 5);
    b->ev_recorded = b->profiling;
    if (stats)
      BCK(b, launch_count_run_bricks(b->d_views, g0, b->pool.items_ctr, b->pool.item_cap, t, b->items, b->st), "count");
  }
  if (stats) {
    for (int i = 0; i < b->k; ++i) {
      vdbedt_map* m = b->maps[(size_t)i];
      BCK(b, cudaMemcpyAsync(m->h_pinned, m->g.counters, sizeof(int32_t) * C_NUM, cudaMemcpyDeviceToHost, b->st), "d2h");
      if (counted[(size_t)i])
        BCK(b, cudaMemcpyAsync(m->h_pinned + 40, m->d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, b->st), "d2h");
    }
    BCK(b, cudaMemcpyAsync(b->maps[0]->h_pinned + 44, b->pool.items_ctr, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost,
                           b->st), "d2h");
    BCK(b, cudaStreamSynchronize(b->st), "sync");
    for (int i = 0; i < b->k; ++i) {
      vdbedt_map* m = b->maps[(size_t)i];
      s = device_errors(m);
      if (s) return bfail(b, s, m->err);
      const int32_t* c = m->h_pinned;
      vdbedt_update_stats& o = stats[i];
      o.records = counted[(size_t)i] ? c[40] : nrec[(size_t)i];
      o.net_flips = c[C_FLIPS];
      o.changed_bricks = c[C_CHANGED];
      // the work queue is shared: its run counts are the batch's, reported on every grid
      o.x_items = b->maps[0]->h_pinned[44];
      o.y_items = b->maps[0]->h_pinned[45];
      o.z_items = b->maps[0]->h_pinned[46];
      o.new_bricks = c[C_NEW_BRICKS];
      o.x_bricks = c[C_XB];
      o.y_bricks = c[C_YB];
      o.z_bricks = c[C_ZB];
      o.global_form = c[C_BIG];
    }
  }
  return VDBEDT_OK;
}

}  // namespace

extern "C" {

vdbedt_status vdbedt_batch_update(vdbedt_batch_handle b, vdbedt_update_stats* stats) {
  if (!b) return bfail(nullptr, VDBEDT_EINVAL, "null batch");
  return batch_update(b, stats);
}

vdbedt_status vdbedt_batch_create(const vdbedt_config* cfgs, int32_t k, vdbedt_batch_handle* out) {
  if (!cfgs || !out || k < 1 || k > kBatchMax) return bfail(nullptr, VDBEDT_EINVAL, "need 1 <= k <= VDBEDT_BATCH_MAX configs");
  int64_t total = 0;
  for (int i = 0; i < k; ++i) {
    const vdbedt_config& c = cfgs[i];
    if (c.dmax != cfgs[0].dmax || c.device != cfgs[0].device || c.stream != cfgs[0].stream ||
        c.voxel_size != cfgs[0].voxel_size)
      return bfail(nullptr, VDBEDT_EINVAL, "the grids of a batch share dmax, voxel_size, device and stream");
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || c.nx >= kBadCoord || c.ny >= kBadCoord || c.nz >= kBadCoord)
      return bfail(nullptr, VDBEDT_EINVAL, "grid size out of range");
    total += config_cap(&c);
  }
  if (total * kItemSlots >= (int64_t)INT32_MAX) return bfail(nullptr, VDBEDT_EINVAL, "batch too large");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfgs[0].device < 0 || cfgs[0].device >= ndev) {
    cudaGetLastError();
    return bfail(nullptr, VDBEDT_EINVAL, "no such CUDA device");
  }
  DeviceGuard guard(cfgs[0].device);
  vdbedt_batch* b = new vdbedt_batch();
  b->k = k;
  b->device = cfgs[0].device;
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t err, const char* where) {
    vdbedt_status st = err == cudaErrorMemoryAllocation ? VDBEDT_ENOMEM : VDBEDT_ECUDA;
    cudaGetLastError();
    g_last_error = std::string(where) + ": " + cudaGetErrorString(err);
    destroy_batch(b);
    return st;
  };
  if (cfgs[0].stream) {
    b->st = (cudaStream_t)cfgs[0].stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(e, "stream");
    b->own_stream = true;
  }
  GridView& p = b->pool;
#define BAL(ptr, count)                                                        \
  do {                                                                         \
    size_t bytes_ = std::max<size_t>((size_t)(count) * sizeof(*(ptr)), 256);   \
    e = cudaMalloc((void**)&(ptr), bytes_);                                    \
    if (e != cudaSuccess) return bail(e, "device alloc");                      \
    b->allocs.push_back((void*)(ptr));                                         \
    b->device_bytes += bytes_;                                                 \
  } while (0)
  BAL(p.occ, total * 8);
  BAL(p.g1, total * kBrickVox);
  BAL(p.g2, total * kBrickVox);
  BAL(p.dist, total * kBrickVox);
  BAL(p.bcoord, total);
  BAL(p.bflags, total);
  BAL(p.bepoch, total);
  BAL(b->counters, (size_t)(k + 1) * C_NUM);
  for (int a = 0; a < 3; ++a) {
    BAL(b->items.run[a], total);
    BAL(b->items.slots[a], total * kItemSlots);
    BAL(b->items.igrid[a], total);
  }
  BAL(b->d_views, k);
  BAL(b->d_upd, k);
#undef BAL
  e = cudaMallocHost((void**)&b->h_upd, sizeof(UpdArgs) * (size_t)k);
  if (e != cudaSuccess) return bail(e, "pinned alloc");
  e = cudaStreamCreateWithFlags(&b->fork.side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.join, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "side stream");
  memset(b->h_upd, 0, sizeof(UpdArgs) * (size_t)k);
  e = cudaMemsetAsync(b->counters, 0, sizeof(int32_t) * (size_t)(k + 1) * C_NUM, b->st);
  if (e != cudaSuccess) return bail(e, "memset");
  int32_t* bctr = b->counters + (size_t)k * C_NUM;
  int64_t off = 0;
  std::vector<GridView> views((size_t)k);
  for (int i = 0; i < k; ++i) {
    vdbedt_config c = cfgs[i];
    c.stream = (void*)b->st;
    PoolSlice sl;
    sl.occ = p.occ + (size_t)off * 8;
    sl.g1 = p.g1 + (size_t)off * kBrickVox;
    sl.g2 = p.g2 + (size_t)off * kBrickVox;
    sl.dist = p.dist + (size_t)off * kBrickVox;
    sl.bcoord = p.bcoord + off;
    sl.bflags = p.bflags + off;
    sl.bepoch = p.bepoch + off;
    sl.counters = b->counters + (size_t)i * C_NUM;
    sl.items_ctr = bctr + C_X_ITEMS;
    sl.items = b->items;
    sl.slot_base = (int)off;
    sl.item_cap = (int)total;
    vdbedt_map* m = nullptr;
    vdbedt_status st = create_impl(&c, &sl, &m);
    if (st) {
      destroy_batch(b);
      return st;
    }
    m->batch = b;
    b->maps.push_back(m);
    views[(size_t)i] = m->g;
    off += m->g.cap;
  }
  b->shape.k = k;
  b->shape.R = b->maps[0]->g.R;
  {
    // block shares of the per-grid kernels (one launch each, shares end to end)
    std::vector<int> first((size_t)BK_NUM * (k + 1));
    for (int kind = 0; kind < BK_NUM; ++kind) {
      int acc = 0;
      for (int i = 0; i < k; ++i) {
        first[(size_t)kind * (k + 1) + i] = acc;
        acc += batch_blocks(views[(size_t)i], kind);
      }
      first[(size_t)kind * (k + 1) + k] = acc;
      b->shape.total[kind] = acc;
    }
    int* d_first = nullptr;
    e = cudaMalloc((void**)&d_first, sizeof(int) * first.size());
    if (e != cudaSuccess) return bail(e, "device alloc");
    b->allocs.push_back(d_first);
    e = cudaMemcpy(d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e, "block shares");
    for (int kind = 0; kind < BK_NUM; ++kind) b->shape.first[kind] = d_first + (size_t)kind * (k + 1);
    // dense-ingest scratch layout: every grid's masks, then brick flags, then node flags
    size_t nbr_all = 0, nkeys_all = 0;
    for (const GridView& v : views) {
      nbr_all += (size_t)v.BX * v.BY * v.BZ;
      nkeys_all += (size_t)v.NX * v.NY * v.NZ;
    }
    const size_t dbytes = (nbr_all * 64 + 255) & ~(size_t)255, fbytes = (nbr_all * 4 + 255) & ~(size_t)255;
    std::vector<int64_t> off((size_t)3 * k);
    size_t nb = 0, nk = 0;
    for (int i = 0; i < k; ++i) {
      const GridView& v = views[(size_t)i];
      off[(size_t)3 * i] = (int64_t)(nb * 8);                     // u64 elements
      off[(size_t)3 * i + 1] = (int64_t)((dbytes + nb * 4) / 4);  // int32 elements
      off[(size_t)3 * i + 2] = (int64_t)((dbytes + fbytes + nk * 4) / 4);
      nb += (size_t)v.BX * v.BY * v.BZ;
      nk += (size_t)v.NX * v.NY * v.NZ;
    }
    b->dense_nflag_byte = dbytes + fbytes;
    b->dense_nflag_words = nkeys_all;
    b->dense_bytes = dbytes + fbytes + ((nkeys_all * 4 + 255) & ~(size_t)255);
    e = cudaMalloc((void**)&b->d_dense_off, sizeof(int64_t) * off.size());
    if (e != cudaSuccess) return bail(e, "device alloc");
    b->allocs.push_back(b->d_dense_off);
    e = cudaMemcpy(b->d_dense_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e, "dense offsets");
  }
  // the pool view: shape fields of grid 0 (dmax, R, INF are common), the batch's words and lists
  {
    const GridView& g0 = b->maps[0]->g;
    GridView pv = g0;
    pv.occ = p.occ;
    pv.g1 = p.g1;
    pv.g2 = p.g2;
    pv.dist = p.dist;
    pv.bcoord = p.bcoord;
    pv.bflags = p.bflags;
    pv.bepoch = p.bepoch;
    pv.counters = bctr;
    pv.items_ctr = bctr + C_X_ITEMS;
    pv.slot_base = 0;
    pv.cap = (int)total;
    pv.item_cap = (int)total;
    b->pool = pv;
  }
  e = cudaMemcpy(b->d_views, views.data(), sizeof(GridView) * (size_t)k, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(e, "views");
  e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return bail(e, "init");
  *out = b;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_destroy(vdbedt_batch_handle b) {
  if (b) destroy_batch(b);
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_map(vdbedt_batch_handle b, int32_t i, vdbedt_handle* out) {
  if (!b || !out || i < 0 || i >= b->k) return bfail(b, VDBEDT_EINVAL, "bad batch index");
  *out = b->maps[(size_t)i];
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_set_occupancy_dense(vdbedt_batch_handle b, const uint8_t* const* grids, int on_device) {
  if (!b || !grids) return bfail(b, VDBEDT_EINVAL, "null argument");
  for (int i = 0; i < b->k; ++i)
    if (!grids[i]) return bfail(b, VDBEDT_EINVAL, "null grid");
  vdbedt_status s = batch_members_ok(b);
  if (s) return s;
  DeviceGuard guard(b->device);
  for (vdbedt_map* m : b->maps) {
    clear_stage(m);
    m->computed = false;
    m->dense_pending = true;
  }
  BCK(b, launch_reset_batch(b->d_views, b->shape, b->counters, (size_t)(b->k + 1) * C_NUM, b->st), "reset");
  std::vector<const uint8_t*> src((size_t)b->k);
  if (on_device) {
    for (int i = 0; i < b->k; ++i) src[(size_t)i] = grids[i];
  } else {
    size_t total = 0;
    for (vdbedt_map* m : b->maps) total += ((size_t)m->g.nx * m->g.ny * m->g.nz + 255) & ~(size_t)255;
    BCK(b, ensure_scratch(b->io, total), "io alloc");
    size_t off = 0;
    for (int i = 0; i < b->k; ++i) {
      const GridView& g = b->maps[(size_t)i]->g;
      const size_t bytes = (size_t)g.nx * g.ny * g.nz;
      BCK(b, cudaMemcpyAsync((uint8_t*)b->io.buf + off, grids[i], bytes, cudaMemcpyHostToDevice, b->st), "h2d");
      src[(size_t)i] = (const uint8_t*)b->io.buf + off;
      off += (bytes + 255) & ~(size_t)255;
    }
  }
  BCK(b, ensure_scratch(b->scr, b->dense_bytes), "dense scratch");
  BCK(b, launch_ingest_dense_batch(b->d_views, b->shape, src.data(), b->scr.buf, b->d_dense_off, b->dense_nflag_words,
                                   (int32_t*)((char*)b->scr.buf + b->dense_nflag_byte), b->st),
      "dense ingest");
  if (!on_device) BCK(b, cudaStreamSynchronize(b->st), "sync");
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_global(vdbedt_batch_handle b) {
  if (!b) return bfail(nullptr, VDBEDT_EINVAL, "null batch");
  return batch_global(b);
}

vdbedt_status vdbedt_batch_set_tuning(vdbedt_batch_handle b, const vdbedt_tuning* t) {
  if (!b) return bfail(nullptr, VDBEDT_EINVAL, "null batch");
  for (vdbedt_map* m : b->maps) {
    vdbedt_status s = vdbedt_set_tuning(m, t);
    if (s) return bfail(b, s, m->err);
  }
  b->tune = b->maps[0]->tune;
  if (b->pool.half != b->maps[0]->g.half) {
    // the field form changed: the device copy of the grids' views follows
    DeviceGuard guard(b->device);
    std::vector<GridView> views;
    for (vdbedt_map* m : b->maps) views.push_back(m->g);
    BCK(b, cudaMemcpyAsync(b->d_views, views.data(), sizeof(GridView) * views.size(), cudaMemcpyHostToDevice, b->st),
        "views");
    BCK(b, cudaStreamSynchronize(b->st), "views");
    b->pool.half = b->maps[0]->g.half;
  }
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_synchronize(vdbedt_batch_handle b) {
  if (!b) return bfail(nullptr, VDBEDT_EINVAL, "null batch");
  for (vdbedt_map* m : b->maps) {
    vdbedt_status s = vdbedt_synchronize(m);
    if (s) return bfail(b, s, m->err);
  }
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_set_profiling(vdbedt_batch_handle b, int on) {
  if (!b) return bfail(nullptr, VDBEDT_EINVAL, "null batch");
  DeviceGuard guard(b->device);
  if (on && !b->ev[0])
    for (int i = 0; i < 6; ++i) BCK(b, cudaEventCreate(&b->ev[i]), "event");
  b->profiling = on != 0;
  b->ev_recorded = false;
  return VDBEDT_OK;
}

vdbedt_status vdbedt_batch_get_phase_times(vdbedt_batch_handle b, vdbedt_phase_times* out) {
  if (!b || !out) return bfail(b, VDBEDT_EINVAL, "null argument");
  if (!b->ev_recorded) return bfail(b, VDBEDT_EINVAL, "no profiled batch transform since profiling was enabled");
  DeviceGuard guard(b->device);
  BCK(b, cudaEventSynchronize(b->ev[5]), "event sync");
  float ms[5];
  for (int i = 0; i < 5; ++i) BCK(b, cudaEventElapsedTime(&ms[i], b->ev[i], b->ev[i + 1]), "event time");
  out->ingest_ms = ms[0];
  out->activation_ms = ms[1];
  out->items_ms = ms[2];
  out->x_ms = ms[3];
  out->y_ms = 0.f;  // the y and z passes are timed together
  out->z_ms = ms[4];
  return VDBEDT_OK;
}

const char* vdbedt_batch_last_error(vdbedt_batch_handle b) { return b ? b->err.c_str() : g_last_error.c_str(); }

// Several grids in one call.  When the handles are exactly the grids of one batch (any order),
// each step runs once for all of them (vdbedt_batch_global); otherwise grid by grid.
vdbedt_status vdbedt_global_batched(vdbedt_handle* hs, int32_t k) {
  if (k < 0 || (k > 0 && !hs)) return fail(nullptr, VDBEDT_EINVAL, "bad batch");
  if (k == 0) return VDBEDT_OK;
  for (int32_t i = 0; i < k; ++i)
    if (!hs[i]) return fail(nullptr, VDBEDT_EINVAL, "null handle in batch");
  vdbedt_batch* b = hs[0]->batch;
  bool whole = b && b->k == k;
  if (whole) {
    std::vector<char> seen((size_t)k, 0);
    for (int32_t i = 0; i < k && whole; ++i) {
      int idx = -1;
      if (hs[i]->batch == b)
        for (int j = 0; j < k; ++j)
          if (b->maps[(size_t)j] == hs[i]) idx = j;
      if (idx < 0 || seen[(size_t)idx]) whole = false;
      else seen[(size_t)idx] = 1;
    }
  }
  if (whole) {
    vdbedt_status s = batch_global(b);
    if (s) g_last_error = b->err;
    return s;
  }
  for (int32_t i = 0; i < k; ++i) {
    vdbedt_status s = vdbedt_global(hs[i]);
    if (s) return s;
  }
  return VDBEDT_OK;
}

}  // extern "C"

// ---- record packing ----
namespace vdbedt {
namespace {
// Validate and pack records.  With n_dev, only the first *n_dev of the n records are read; the
// count, clamped to [0, n], is copied to count_out for the ingest kernels, and a count outside that
// range sets the invalid-record error bit.
__global__ void k_pack_records(const int32_t* __restrict__ xyz, const uint8_t* __restrict__ occ, int64_t n_max,
                               const int32_t* n_dev, int32_t* count_out, int nx, int ny, int nz, int off,
                               rec_t* __restrict__ dst, int32_t* invalid, int32_t* counters) {
  int64_t n = n_max;
  if (n_dev) {
    const int64_t c = *n_dev;
    n = c < 0 ? 0 : (c < n_max ? c : n_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *count_out = (int32_t)n;
      if (c < 0 || c > n_max) atomicOr(&counters[C_ERR], kErrInvalidRecord);
    }
  }
  auto put = [&](int64_t i, int x, int y, int z, int v) {
    const bool ok = (unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz && v <= 1;
    if (!ok) {
      if (invalid) atomicAdd(invalid, 1);
      dst[i] = pack_rec(kBadCoord, 0, 0, 0);  // skipped (and reported) by the ingest kernels
    } else {
      dst[i] = pack_rec(x, y, z, v);
    }
  };
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    put(i, xyz[3 * i] + off, xyz[3 * i + 1] + off, xyz[3 * i + 2] + off, occ[i]);
}

// Packed records (x | y << 21 | z << 42 | occ << 63, the stage's own format): copied into the stage
// after a range check; a record outside the grid is counted (host input: the call is rejected) or
// flagged in the error word (device input: reported by the next synchronising call), and replaced
// by a skipped record.
__global__ void k_check_packed(const uint64_t* __restrict__ src, int64_t n, int nx, int ny, int nz,
                               rec_t* __restrict__ dst, int32_t* invalid, int32_t* counters) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const rec_t r = src[i];
    const int4 u = unpack_rec(r);
    const bool ok = u.x < nx && u.y < ny && u.z < nz;
    if (!ok) {
      if (invalid)
        atomicAdd(invalid, 1);
      else
        atomicOr(&counters[C_ERR], kErrInvalidRecord);
    }
    dst[i] = ok ? r : pack_rec(kBadCoord, 0, 0, 0);
  }
}
}  // namespace

// Brick masks: a thread per (brick, plane).  The check pass validates the brick and the plane's
// bits against the grid (ragged edges included) and counts the set bits; the expansion pass writes
// one "set" record per bit, places reserved a warp at a time.
__global__ void k_check_bricks(const int32_t* __restrict__ bxyz, const uint64_t* __restrict__ masks, int64_t n,
                               GridView g, int32_t* invalid, unsigned long long* count) {
  const int64_t nw = n * 8;
  __shared__ unsigned long long bsum;  // the block's bit count: one atomic on *count per block
  if (threadIdx.x == 0) bsum = 0ull;
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nw; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int bits = 0;
    if (i < nw) {
      const int64_t k = i >> 3;
      const int pz = (int)(i & 7);
      const unsigned long long m = masks[i];
      const int bx = bxyz[3 * k] + (g.off >> 3), by = bxyz[3 * k + 1] + (g.off >> 3), bz = bxyz[3 * k + 2] + (g.off >> 3);
      bool ok = (unsigned)bx < (unsigned)g.BX && (unsigned)by < (unsigned)g.BY && (unsigned)bz < (unsigned)g.BZ;
      if (ok && m) {
        // bits past the grid's last voxel on each axis (a ragged last brick)
        const int ex = min(8, g.nx - 8 * bx), ey = min(8, g.ny - 8 * by);
        const unsigned long long row = ex >= 8 ? 0xFFull : ((1ull << ex) - 1ull);
        unsigned long long inside = 0ull;
        for (int y = 0; y < ey; ++y) inside |= row << (8 * y);
        ok = 8 * bz + pz < g.nz ? (m & ~inside) == 0ull : false;
      }
      if (!ok) atomicAdd(invalid, 1);
      bits = ok ? __popcll(m) : 0;
    }
    for (int o = 16; o > 0; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
    if ((threadIdx.x & 31) == 0 && bits) atomicAdd(&bsum, (unsigned long long)bits);
  }
  __syncthreads();
  if (threadIdx.x == 0 && bsum) atomicAdd(count, bsum);
}

__global__ void k_expand_bricks(const int32_t* __restrict__ bxyz, const uint64_t* __restrict__ masks, int64_t n,
                                GridView g, rec_t* __restrict__ dst, unsigned long long* cursor) {
  const int64_t nw = n * 8;
  const int lane = threadIdx.x & 31;
  __shared__ int wtot[32];
  __shared__ unsigned long long woff[32], bbase;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nw; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    unsigned long long m = 0ull;
    int bx = 0, by = 0, z = 0;
    if (i < nw) {
      const int64_t k = i >> 3;
      m = masks[i];
      bx = bxyz[3 * k] + (g.off >> 3);
      by = bxyz[3 * k + 1] + (g.off >> 3);
      z = 8 * (bxyz[3 * k + 2] + (g.off >> 3)) + (int)(i & 7);
    }
    const int bits = __popcll(m);
    // the block's places: an inclusive scan of the bit counts in each warp, the warps' totals
    // scanned by thread 0, one atomic on the cursor per block
    int incl = bits;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0ull;
      for (int w = 0; w < nwarps; ++w) {
        const unsigned long long c = (unsigned long long)wtot[w];
        woff[w] = t;
        t += c;
      }
      bbase = t ? atomicAdd(cursor, t) : 0ull;
    }
    __syncthreads();
    unsigned long long p = bbase + woff[warp] + (unsigned long long)(incl - bits);
    __syncthreads();  // the block's next round rewrites wtot / woff / bbase
    while (m) {
      const int b = __ffsll((long long)m) - 1;
      m &= m - 1ull;
      dst[p++] = pack_rec(8 * bx + (b & 7), 8 * by + (b >> 3), z, 1);
    }
  }
}

cudaError_t launch_check_packed(const uint64_t* src, int64_t n, int nx, int ny, int nz, rec_t* dst, int32_t* invalid,
                                int32_t* counters, cudaStream_t st) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  VDB_LAUNCH(k_check_packed, (unsigned)b, 256, 0, st, src, n, nx, ny, nz, dst, invalid, counters);
  return cudaGetLastError();
}

cudaError_t launch_check_bricks(const int32_t* bxyz, const uint64_t* masks, int64_t n, const GridView& g,
                                int32_t* invalid, unsigned long long* count, cudaStream_t st) {
  int64_t b = (n * 8 + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  VDB_LAUNCH(k_check_bricks, (unsigned)b, 256, 0, st, bxyz, masks, n, g, invalid, count);
  return cudaGetLastError();
}

cudaError_t launch_expand_bricks(const int32_t* bxyz, const uint64_t* masks, int64_t n, const GridView& g, rec_t* dst,
                                 unsigned long long* cursor, cudaStream_t st) {
  int64_t b = (n * 8 + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  VDB_LAUNCH(k_expand_bricks, (unsigned)b, 256, 0, st, bxyz, masks, n, g, dst, cursor);
  return cudaGetLastError();
}

cudaError_t launch_pack_records(const int32_t* xyz, const uint8_t* occ, int64_t n, const int32_t* n_dev,
                                int32_t* count_out, int nx, int ny, int nz, int off, rec_t* dst, int32_t* invalid,
                                int32_t* counters, cudaStream_t st) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  VDB_LAUNCH(k_pack_records, (unsigned)b, 256, 0, st, xyz, occ, n, n_dev, count_out, nx, ny, nz, off, dst, invalid,
             counters);
  return cudaGetLastError();
}
}  // namespace vdbedt
