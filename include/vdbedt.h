/*
 * vdbedt -- exact truncated Euclidean distance transform over a sparse grid of 8^3 voxel bricks,
 * for one NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * What is computed (paper: Zhu et al., "VDB-EDT", arXiv 2105.04419):
 *   For an nx x ny x nz occupancy grid and truncation distance dmax (voxels), every voxel v gets
 *       D(v) = min( dmax^2, min_{o occupied} |v - o|^2 )
 *   the squared Euclidean distance in integer voxel units to the nearest occupied voxel (Sec. III,
 *   Eq. 1), saturated at dmax^2 (the limited transform of Sec. III; Sec. IV-B stores dmax for any
 *   distance at or beyond it).  D is 0 on obstacles.  Results are exact (bit-identical to the
 *   definition), int32.
 *   Two forms, as the paper names them (Sec. I): the global transform recomputes the field from
 *   the occupancy; the incremental transform repairs it after occupancy edits (Alg. 1's
 *   SetObstacle / RemoveObstacle followed by DistanceTransform).
 *
 * Storage: the grid keeps only bricks within reach of an obstacle; everything else reads as the
 * background value dmax^2 (the paper's tile value, Sec. IV-A).
 *
 * Conventions for every call:
 *   - Return codes only; no call aborts or exits.  Out-parameters are written only on VDBEDT_OK.
 *   - Work is stream-ordered on the handle's stream.  Host pointers are read (and host outputs
 *     written) before the call returns.  Device pointers must stay valid until the stream reaches
 *     the call.
 *   - A CUDA runtime error makes the handle fail stickily: every later call returns VDBEDT_ECUDA
 *     until vdbedt_destroy.
 *   - Errors detected on the device (capacity exceeded, a bounded wait that timed out, invalid
 *     records passed through device memory) are reported by the next call that synchronises
 *     with the stream: vdbedt_synchronize, vdbedt_get_info, vdbedt_query / vdbedt_export_dense
 *     with host outputs.
 *   - Coordinates are int32 (x, y, z) triples, 0 <= x < nx etc.; dense arrays are C-ordered
 *     [nz][ny][nx].
 *   - A handle is not thread-safe; distinct handles may be used from distinct threads.
 */
#ifndef VDBEDT_H
#define VDBEDT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vdbedt_map* vdbedt_handle;

typedef enum {
  VDBEDT_OK = 0,
  VDBEDT_EINVAL = 1,    /* bad argument or record; the whole call is rejected */
  VDBEDT_ENOMEM = 2,    /* device or host allocation failed */
  VDBEDT_ECUDA = 3,     /* CUDA runtime error (sticky for the handle) */
  VDBEDT_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  VDBEDT_EOVERFLOW = 5, /* more bricks needed than the handle's capacity */
  VDBEDT_EINTERNAL = 6  /* a device-side consistency check failed */
} vdbedt_status;

/* Largest supported truncation: keeps dmax^2 = 32761 < 2^15 so stored intermediates fit 16 bits. */
#define VDBEDT_DMAX_LIMIT 181

/* Flags of vdbedt_config.
 * VDBEDT_FLAG_UNBOUNDED: a grid without a fixed size that grows where records fall (the paper's
 * motivation for a VDB-style tree, Sec. I and Sec. IV-A): nx, ny, nz are ignored; coordinates are
 * signed, VDBEDT_UNBOUNDED_MIN <= x, y, z < VDBEDT_UNBOUNDED_MAX on every axis (about +-10^6
 * voxels, +-105 km at 0.1 m), and interior nodes and bricks are created only where obstacles and
 * their dilation reach, so max_bricks and max_nodes (both required) bound the memory.  Queries
 * anywhere in that range answer dmax^2 where nothing is mapped.  Not available: the dense entry
 * points (vdbedt_set_occupancy_dense, vdbedt_export_dense) and batches.  Packed records
 * (vdbedt_set_occupancy_packed, vdbedt_export_occupancy) hold each coordinate plus
 * VDBEDT_UNBOUNDED_OFFSET (non-negative).  The clearance query takes points in metres as usual
 * (cells are found in float32: far from the origin the in-cell position is coarser). */
#define VDBEDT_FLAG_UNBOUNDED 1u
#define VDBEDT_UNBOUNDED_OFFSET (1 << 20)
#define VDBEDT_UNBOUNDED_MIN (-(1 << 20))
#define VDBEDT_UNBOUNDED_MAX ((1 << 20) - 128)

/* VDBEDT_FLAG_UNTRUNCATED: no truncation (the paper's dmax = infinity runs, Table II): D is Eq. 1's
 * exact squared distance to the nearest occupied voxel anywhere in the grid, and VDBEDT_D_NONE at
 * every voxel while the grid holds no obstacle (and for queries outside the grid).  dmax must be 0.
 * A bounded grid only, with (nx-1)^2 + (ny-1)^2 + (nz-1)^2 < 2^31 - 1 so that every distance fits
 * int32, and every brick stored from creation (max_bricks and max_nodes 0 or at least the grid's):
 * about 6.2 KB per 8^3 brick (32-bit intermediates) plus 8 bytes per voxel of line scratch (nx
 * rounded up to 32) and three sets of dirty lines, all allocated at creation.  The transform
 * runs whole lines of the grid (x: nearest occupied voxel of the row; y, z: lower envelope of the
 * parabolas rooted at the line's values).  vdbedt_update applies the staged records and recomputes
 * only the lines they reach, exactly: the x rows holding a flipped voxel, then the y lines on which
 * g1 changed, then the z lines on which g2 changed (each pass's output on a line depends only on
 * its input along that line).  Not available: batches, vdbedt_set_tuning, vdbedt_query_nearest and
 * the unbounded flag. */
#define VDBEDT_FLAG_UNTRUNCATED 2u
#define VDBEDT_D_NONE 2147483647

typedef struct {
  int32_t nx, ny, nz;  /* grid size in voxels, each >= 1 (at most 2^21 - 128; ignored when unbounded) */
  int32_t dmax;        /* truncation distance in voxels, 1 <= dmax <= VDBEDT_DMAX_LIMIT (0 when untruncated) */
  float voxel_size;    /* metres per voxel (used by the clearance query), > 0 */
  int32_t device;      /* CUDA device ordinal */
  void* stream;        /* cudaStream_t to run on; NULL: the handle creates and owns one */
  uint32_t flags;      /* 0, VDBEDT_FLAG_UNBOUNDED or VDBEDT_FLAG_UNTRUNCATED */
  int64_t max_bricks;  /* brick capacity; 0: every brick of the grid (always enough) */
  int64_t max_nodes;   /* interior-node capacity (a node covers 16^3 bricks); 0: every node of the grid;
                          at most 4,194,302 */
} vdbedt_config;

typedef struct {
  int64_t allocated_bricks; /* bricks holding storage */
  int64_t obstacle_bricks;  /* bricks with at least one occupied voxel */
  int64_t finite_bricks;    /* bricks with at least one voxel below dmax^2 (the active set) */
  int64_t capacity_bricks;
  int64_t nodes;            /* interior nodes (16^3 bricks each) */
  int64_t device_bytes;     /* device memory held by the handle */
  int32_t R;                /* brick radius of influence, floor((dmax + 6) / 8) */
  int32_t error_bits;       /* device-side error word (0 when healthy) */
} vdbedt_info;

typedef struct {
  int64_t records;        /* staged records consumed */
  int64_t net_flips;      /* voxels whose occupancy changed */
  int64_t changed_bricks; /* bricks holding a flipped voxel */
  int64_t x_items;        /* brick runs recomputed by the x pass (untruncated grid: voxel rows) */
  int64_t y_items;        /* brick runs recomputed by the y pass (untruncated grid: y lines) */
  int64_t z_items;        /* brick runs recomputed by the z pass (untruncated grid: z lines) */
  int64_t new_bricks;     /* bricks allocated by this update */
  int64_t x_bricks;       /* stored bricks in those runs, recomputed by the x pass */
  int64_t y_bricks;       /* ... by the y pass */
  int64_t z_bricks;       /* ... by the z pass (global_form 1: every stored brick; the three counts are 0
                             in the envelope form, variant 8 or dmax > 45) */
  int64_t global_form;    /* 1: the edits reached so far that the update switched to the global form after
                             applying them (same field, lower cost; see vdbedt_update), or the grid had no
                             transform yet (or a new dense grid), which the update then computes whole */
} vdbedt_update_stats;

/* Create a handle for an nx x ny x nz grid with no obstacles (every D = dmax^2; VDBEDT_D_NONE when
 * untruncated).
 * Allocates the grid's storage for cfg->max_bricks bricks (about 4.1 KB each) and cfg->max_nodes
 * interior nodes (about 30 KB each) up front; the record stage and the ingest scratch grow on
 * demand (vdbedt_set_occupancy_counted reserves them ahead).  With both capacities set, the memory
 * follows the mapped part of the grid, not its size: a grid may span up to 2^32 bricks (e.g.
 * 16384 x 16384 x 8184 voxels) with obstacles in a small part of it.  Record-driven ingest and
 * updates work at any grid size; the dense entry points and vdbedt_export_dense scale with the grid.
 * The brick capacity is at most 8,388,607 (max_bricks 0 on a larger grid is EINVAL: set it).
 * Exceeding a capacity during a transform is EOVERFLOW.
 * EINVAL: a size < 1, dmax outside [1, VDBEDT_DMAX_LIMIT] (not 0 with VDBEDT_FLAG_UNTRUNCATED, or a
 * grid or capacities outside that flag's limits), voxel_size <= 0, unknown flags, bad device.
 * ENOMEM: device allocation failed. */
vdbedt_status vdbedt_create(const vdbedt_config* cfg, vdbedt_handle* out);

/* Release everything the handle owns (waits for its stream).  NULL is accepted. */
vdbedt_status vdbedt_destroy(vdbedt_handle h);

/* Stage occupancy records: voxel (xyz[3k], xyz[3k+1], xyz[3k+2]) gets occ[k] (0 = free, 1 =
 * obstacle) -- the edits of Alg. 1's SetObstacle / RemoveObstacle.  Nothing changes until the next
 * vdbedt_global or vdbedt_update, which applies all staged records in order: when a voxel appears
 * more than once, its last record wins.  on_device != 0: xyz and occ are device pointers (read on
 * the stream; an invalid record is skipped and reported as EINVAL by the next synchronising call);
 * otherwise host pointers, validated here: any coordinate outside the grid or occ[k] > 1 rejects
 * the whole call with EINVAL.  n == 0 is a no-op; n < 0 is EINVAL; at most 2^31 - 1 records can be
 * staged at a time (more: EINVAL). */
vdbedt_status vdbedt_set_occupancy(vdbedt_handle h, const int32_t* xyz, const uint8_t* occ, int64_t n,
                                   int on_device);

/* The same records packed in 64 bits each, 8 bytes instead of 13 (for host links, where the record
 * stream is the largest transfer): rec[k] = x | y << 21 | z << 42 | occ << 63 (x, y, z below 2^21,
 * occ 0 or 1).  Semantics, validation and errors as vdbedt_set_occupancy (a coordinate outside the
 * grid rejects a host call; from device memory it is skipped and reported by the next
 * synchronising call); page-locked host arrays are read in place. */
vdbedt_status vdbedt_set_occupancy_packed(vdbedt_handle h, const uint64_t* rec, int64_t n, int on_device);

/* Occupied voxels given brick by brick (Sec. IV-A's 8^3 leaves), 76 bytes per brick however many of
 * its voxels are occupied -- a fraction of the record stream over a host link when obstacles fill
 * bricks densely: bxyz[3k .. 3k + 2] is a brick (bx, by, bz) (caller voxel coordinates divided by 8,
 * rounded down: signed on an unbounded grid) and masks[8k + z] its plane z, bit x + 8 y marking
 * voxel (8 bx + x, 8 by + y, 8 bz + z) occupied.  Equivalent to one "set" record (occ 1) per bit,
 * staged after the records already staged; bits at 0 stage nothing.  The records are written into
 * the stage on the device (a bit count sizes it first, so the call waits for the device, also
 * with on_device != 0).  EINVAL (whole call rejected): a brick outside the grid, a bit for a voxel
 * outside the grid, n < 0; records staged with vdbedt_set_occupancy_counted and not yet applied. */
vdbedt_status vdbedt_set_occupancy_bricks(vdbedt_handle h, const int32_t* bxyz, const uint64_t* masks, int64_t n,
                                          int on_device);

/* Stage up to n_max occupancy records in device memory whose actual count is the int32 at n_dev
 * (device memory), read when the stream reaches the call -- the same edits as vdbedt_set_occupancy
 * with on_device = 1, in a form whose launches do not depend on the count, so that a staging call
 * followed by vdbedt_update can be captured once into a CUDA graph and replayed for frames of
 * different sizes (write the frame into xyz / occ and its count into *n_dev before each replay).
 * The stage must be empty (EINVAL otherwise), and no other records may be staged until the next
 * transform applies these.  The call reserves the stage and the ingest scratch for n_max records,
 * so a capture taken after one uncaptured call with the same n_max allocates nothing.  A count
 * below 0 or above n_max is clamped to [0, n_max] and reported as EINVAL by the next synchronising
 * call, as are invalid records (which are skipped).  n_max must lie in [1, 2^31). */
vdbedt_status vdbedt_set_occupancy_counted(vdbedt_handle h, const int32_t* xyz, const uint8_t* occ,
                                           const int32_t* n_dev, int64_t n_max);

/* Stage a whole occupancy grid grid[nz][ny][nx] (nonzero = obstacle), replacing the current one
 * (records staged earlier are discarded).  on_device selects host or device memory. */
vdbedt_status vdbedt_set_occupancy_dense(vdbedt_handle h, const uint8_t* grid, int on_device);

/* Clear the grid to no obstacles and drop all storage (keeps capacity); staged records are dropped. */
vdbedt_status vdbedt_reset(vdbedt_handle h);

/* Global transform: apply staged records, then recompute the whole field from the occupancy. */
vdbedt_status vdbedt_global(vdbedt_handle h);

/* Incremental transform: apply staged records; recompute only the bricks that a flipped voxel can
 * reach (bricks whose nearest voxels lie closer than dmax to a changed brick's).  Equal, bit for
 * bit, to vdbedt_global on the same occupancy.  When the changed bricks times (2R + 1)^3 exceed 24
 * times the bricks stored when the update began (the marking would then cost more than
 * recomputing the map), the update decides on the device, after applying the records, to rebuild
 * the compute set and work lists as vdbedt_global does (the trade-off of the paper's Sec. V-A
 * between global and incremental transforms); the decision needs no host round trip, so a
 * captured update keeps it.  On an untruncated grid the update recomputes the lines the flips reach
 * (VDBEDT_FLAG_UNTRUNCATED), and its stats count lines (x rows, y lines, z lines) in x_items,
 * y_items and z_items.  stats (nullable) is filled after a stream synchronisation. */
vdbedt_status vdbedt_update(vdbedt_handle h, vdbedt_update_stats* stats);

/* D at n voxel coordinates; coordinates outside the grid or in unstored bricks give dmax^2
 * (VDBEDT_D_NONE when untruncated).
 * on_device != 0: xyz and out_sqdist are device pointers; otherwise host pointers (the call waits). */
vdbedt_status vdbedt_query(vdbedt_handle h, const int32_t* xyz, int64_t n, int32_t* out_sqdist, int on_device);

/* Nearest obstacle of n voxels: out_xyz[3k .. 3k + 2] is the occupied voxel o that D(v) measures
 * to -- the obstacle the paper's map keeps beside each cell's distance (Sec. IV-B) -- found among
 * the lattice points with |o - v|^2 = D(v) in increasing (z, y, x) order, so ties go to the
 * smallest (z, y, x).  (-1, -1, -1) for voxels outside the grid or with D = dmax^2 (no obstacle
 * closer than dmax).  Reads the current field (after vdbedt_global / vdbedt_update).  on_device
 * as for vdbedt_query.  EINVAL on an untruncated grid. */
vdbedt_status vdbedt_query_nearest(vdbedt_handle h, const int32_t* xyz, int64_t n, int32_t* out_xyz, int on_device);

/* The whole field as a dense int32 array out[nz][ny][nx] (host or device). */
vdbedt_status vdbedt_export_dense(vdbedt_handle h, int32_t* out, int on_device);

/* The occupancy of planes z_lo <= z < z_hi as packed records (the format of
 * vdbedt_set_occupancy_packed) with z shifted by dz, into out (device, up to max_n records):
 * mode 0: every occupied voxel (occ = 1); mode 1: every voxel, occupied or free, of the bricks that
 * the last vdbedt_update changed (the bricks holding one of its flipped voxels).  Staged on another
 * handle whose grid covers the shifted planes, they reproduce those planes' occupancy (mode 0 on an
 * empty grid; mode 1 replays the update's changes).  This is how one grid split into z-slabs over
 * several GPUs exchanges only the occupied voxels (or the changed bricks) of each slab's halo band.
 * Synchronises; *n_out (host) receives the number of records; more than max_n is EOVERFLOW (the
 * first max_n are written, *n_out holds the full count).  Record order is unspecified. */
vdbedt_status vdbedt_export_occupancy(vdbedt_handle h, int32_t z_lo, int32_t z_hi, int32_t dz, int32_t mode,
                                      uint64_t* out, int64_t max_n, int64_t* n_out);

/* Distance field for planners: at n points pts[n][3] (metres; device pointers), dist[k] = the
 * trilinear distance d of the clearance cost below (same cell choice and corner values) and, when
 * grad is not NULL, grad[k][0..2] = dd/dp = (1 / voxel_size) * d(trilinear)/dt, the gradient of the
 * distance field a planner follows away from obstacles (the paper's trajectory optimisation pushes
 * trajectories along it, Sec. I, Eq. 2).  Grids with a size < 2 along any axis are EINVAL. */
vdbedt_status vdbedt_distance_at(vdbedt_handle h, const float* pts, int64_t n, float* dist, float* grad);

/* Clearance cost of Eq. 2 (second term) as a squared hinge, for T trajectories of P points.
 * pts: device float [T][P][3], metres; voxel centre (i, j, k) sits at (i, j, k) * voxel_size.
 * Per point: u = p / voxel_size (float32), cell i0 = floor(u) clamped to [0, n - 2] per axis,
 * t = u - i0; d = trilinear interpolation of voxel_size * sqrt(D) over the cell's 8 corners;
 * c = max(0, tau - d)^2.  cost[t] = sum of c over the trajectory's points (device float [T]).
 * Grids with a size < 2 along any axis are EINVAL. */
vdbedt_status vdbedt_clearance_forward(vdbedt_handle h, const float* pts, int64_t T, int64_t P, float tau,
                                       float* cost);

/* Gradient of sum_t grad_cost[t] * cost[t] with respect to pts: grad_pts[t][p] =
 * grad_cost[t] * (-2 max(0, tau - d)) * (1 / voxel_size) * d(trilinear)/dt.  Device pointers. */
vdbedt_status vdbedt_clearance_backward(vdbedt_handle h, const float* pts, int64_t T, int64_t P, float tau,
                                        const float* grad_cost, float* grad_pts);


/* Tuning of the transform passes (0 = automatic for any field).
 *   x_run, y_run, z_run: bricks per work item of the pass along that axis (4, 8 or 16);
 *   variant: 0 automatic, 1 full windowed minimum, 3 windowed minimum with early exit and skips
 *            (the default; both exact); adding 4 (5 or 7) runs the x pass with plain loads instead
 *            of the bulk-copy ring; 8 the lower-envelope form of all three passes (exact, O(1)
 *            amortised work per voxel whatever the window, runs of 16 bricks: the separable
 *            transform of Eq. 1 line by line).  Grids with dmax above 45 always take the envelope
 *            form.  Switching between the windowed and envelope forms changes how intermediate
 *            fields are stored, so the next vdbedt_update recomputes the whole field (as
 *            vdbedt_global).  Other values are EINVAL, and so is any call on an untruncated grid. */
typedef struct {
  int32_t x_run, y_run, z_run, variant;
} vdbedt_tuning;
vdbedt_status vdbedt_set_tuning(vdbedt_handle h, const vdbedt_tuning* t);

/* Phase timing (tracing): with profiling on, vdbedt_global and vdbedt_update record CUDA events
 * on the handle's stream around their phases; vdbedt_get_phase_times waits for the last such call
 * and returns the device time of each phase in milliseconds.  The paper reports wall time per
 * frame (Table II); these are the GPU analogue, per phase.  EINVAL before any profiled call. */
typedef struct {
  float ingest_ms;     /* staged records -> bricks and occupancy bits */
  float activation_ms; /* compute set (dilation by R bricks) and brick allocation */
  float items_ms;      /* work lists of the passes (global form only) */
  float x_ms;          /* x pass (nearest obstacle along each x-line) */
  float y_ms;          /* y pass (in-plane squared distance) */
  float z_ms;          /* z pass, clamp, finite flags */
} vdbedt_phase_times;
vdbedt_status vdbedt_set_profiling(vdbedt_handle h, int on);
vdbedt_status vdbedt_get_phase_times(vdbedt_handle h, vdbedt_phase_times* out);

/* ---- Batches: many grids of uneven size transformed together (no paper counterpart: the paper
 * transforms one map at a time; this is the batched form of its global transform, Sec. IV). ----
 *
 * A batch owns k grids created together.  Their bricks live in one pool, so that each step of
 * the global transform is one launch for all k grids: the per-grid steps (reset, dense ingest,
 * activation, work-list build) launch a block row per grid, and the three passes run as one
 * persistent launch each over a single work queue holding every grid's brick runs.  Each grid is
 * also an ordinary handle (vdbedt_batch_map): records, queries, export, incremental updates and
 * single-grid transforms work on it as on any handle; it is released with the batch (vdbedt_destroy
 * of a batch grid is EINVAL).  Operations on the grids of one batch must not overlap (they share
 * the work lists and run on the batch's stream). */
typedef struct vdbedt_batch* vdbedt_batch_handle;
#define VDBEDT_BATCH_MAX 1024

/* Create k grids (cfgs[i], 1 <= k <= VDBEDT_BATCH_MAX) that share dmax, voxel_size, device and
 * stream (NULL: the batch creates and owns one); sizes and max_bricks may differ.  EINVAL on a
 * bad or inconsistent configuration; ENOMEM when the pool does not fit. */
vdbedt_status vdbedt_batch_create(const vdbedt_config* cfgs, int32_t k, vdbedt_batch_handle* out);
/* Release the batch and its grids (waits for its stream).  NULL is accepted. */
vdbedt_status vdbedt_batch_destroy(vdbedt_batch_handle b);
/* Handle of grid i (owned by the batch). */
vdbedt_status vdbedt_batch_map(vdbedt_batch_handle b, int32_t i, vdbedt_handle* out);
/* Replace the occupancy of every grid: grids[i] is grid i's [nz][ny][nx] uint8 array (nonzero =
 * obstacle), device pointers when on_device != 0 (read on the stream), else host pointers (copied
 * before return).  grids itself is a host array of k pointers. */
vdbedt_status vdbedt_batch_set_occupancy_dense(vdbedt_batch_handle b, const uint8_t* const* grids, int on_device);
/* Global transform of every grid of the batch (records staged on a grid are applied first).
 * Bit-identical to vdbedt_global on each grid.  In the lower-envelope form (dmax above 45, or
 * variant 8) the grids are transformed one after the other, and the batch's phase times put the
 * whole transform in z_ms. */
vdbedt_status vdbedt_batch_global(vdbedt_batch_handle b);
/* Incremental transform of every grid of the batch (Alg. 1's edits followed by DistanceTransform,
 * Sec. IV-B, for k maps at once): the records staged on each grid (vdbedt_set_occupancy or
 * vdbedt_set_occupancy_counted on its handle) are applied, the changed bricks of every grid are
 * dilated by R bricks and their dirty runs recomputed, each step launched once for all grids, the
 * runs of every grid in one shared work queue.  Bit-identical to vdbedt_update on each grid.  A grid
 * without a field yet (no transform since its occupancy was set) makes the call a
 * vdbedt_batch_global.  In the lower-envelope form the grids are updated one after the other.
 * Capturable into a CUDA graph after one uncaptured call with the same staging (counted staging on
 * each grid, so that nothing reallocates): the grids' arguments live in device memory and are
 * uploaded only when their staging changes, which is EINVAL during a capture.  stats (nullable): an
 * array of k entries, filled after a stream synchronisation; the run counts (x/y/z_items) are the
 * shared queue's, the same on every entry. */
vdbedt_status vdbedt_batch_update(vdbedt_batch_handle b, vdbedt_update_stats* stats);
/* vdbedt_set_tuning on every grid of the batch. */
vdbedt_status vdbedt_batch_set_tuning(vdbedt_batch_handle b, const vdbedt_tuning* t);
/* Report device-side errors of any grid (vdbedt_synchronize on each). */
vdbedt_status vdbedt_batch_synchronize(vdbedt_batch_handle b);
/* Phase timing of vdbedt_batch_global (CUDA events on the batch's stream); in the result, ingest_ms
 * is the staged-record ingest, z_ms covers the y and z passes together and y_ms is 0. */
vdbedt_status vdbedt_batch_set_profiling(vdbedt_batch_handle b, int on);
vdbedt_status vdbedt_batch_get_phase_times(vdbedt_batch_handle b, vdbedt_phase_times* out);
const char* vdbedt_batch_last_error(vdbedt_batch_handle b);

/* Global transform of k handles in one call.  When they are exactly the grids of one batch (in
 * any order) this is vdbedt_batch_global; otherwise each handle is transformed in turn on its
 * own stream.  Bit-identical to vdbedt_global on each. */
vdbedt_status vdbedt_global_batched(vdbedt_handle* hs, int32_t k);

/* Number of CUDA kernels this library has launched in this process (all handles). */
int64_t vdbedt_kernel_launches(void);

/* Self-test of the device-side bounded waits (no paper counterpart: it lets a test exercise the
 * timeout path without a GPU fault).  which = 0: one thread waits on an mbarrier phase that never
 * completes (the wait of the pass kernels); which = 1: one thread looks up a node whose insertion
 * is left pending (the wait of node creation; the planted claim leaves the grid's node table
 * invalid until vdbedt_reset).  Each wait gives up after one second, sets the handle's error word
 * and returns, so the context stays usable; the next synchronising call reports VDBEDT_ETIMEOUT
 * until vdbedt_reset.  Other values of which are EINVAL. */
vdbedt_status vdbedt_selftest_wait_timeout(vdbedt_handle h, int32_t which);

/* Dense transform without any allocation (no paper counterpart: this is a deployment feature).
 * For callers that cannot call cudaMalloc -- code running while the application holds a stream
 * capture open, real-time loops that must stay out of the allocator, hosts whose device memory
 * budget is fixed at load time.  Computes D (int32, out[nz][ny][nx]) of the dense occupancy
 * occ[nz][ny][nx] (nonzero = obstacle), exactly as a handle's vdbedt_global would, on the current
 * device and `stream` (cudaStream_t, NULL = legacy default stream).  occ and out are device
 * pointers, owned by the caller.
 * Its two intermediate fields live in a fixed device array of the library (2 x 16 bit x
 * VDBEDT_NOALLOC_MAX_VOXELS = 8 MiB) that every GPU loading the library holds until exit.  Host
 * code needs that array's device address, which the library looks up (cudaGetSymbolAddress) with
 * the device current: every call whose stream is not being captured looks it up again and caches
 * it per device, so a context that was torn down and recreated (cudaDeviceReset) is followed by the
 * next such call; a call made during a stream capture uses the cached address, so make the first
 * call on each device before any capture (one made during a capture first is ECUDA).  All calls on
 * a device share the array: calls whose work overlaps on the GPU race.
 * EINVAL: a null pointer, a size < 1, nx * ny * nz > VDBEDT_NOALLOC_MAX_VOXELS, or dmax outside
 * [1, VDBEDT_DMAX_LIMIT].  ECUDA: a CUDA error of earlier work was already pending on this thread
 * (it is left pending, for its owner to read), the address lookup failed, or a launch failed.
 * Messages: vdbedt_last_error(NULL). */
#define VDBEDT_NOALLOC_MAX_VOXELS (1 << 21)
vdbedt_status vdbedt_edt_dense_noalloc(const uint8_t* occ, int32_t nx, int32_t ny, int32_t nz, int32_t dmax,
                                       int32_t* out, void* stream);

/* Wait for the handle's stream; report device-side errors. */
vdbedt_status vdbedt_synchronize(vdbedt_handle h);

/* Counters of the grid (synchronises). */
vdbedt_status vdbedt_get_info(vdbedt_handle h, vdbedt_info* info);

/* The handle's stream (cudaStream_t). */
void* vdbedt_stream(vdbedt_handle h);

/* Last error message for the handle (or for handle-less failures when h is NULL); never NULL. */
const char* vdbedt_last_error(vdbedt_handle h);

#ifdef __cplusplus
}
#endif

#endif /* VDBEDT_H */
