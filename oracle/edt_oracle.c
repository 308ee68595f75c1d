/*
 * CPU oracle for the truncated Euclidean distance transform -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load this code.  It
 * shares nothing with the CUDA library: no headers, no helpers, no tables.
 *
 * What it computes (paper Sec. III, Eq. 1, and the truncation rule that follows Eq. 2):
 *   for every voxel v of an nx x ny x nz grid with occupancy occ,
 *       D(v) = min( dmax^2, min_{o occupied} |v - o|^2 )
 *   in integer voxel coordinates (squared Euclidean distance, the paper's f), with D = 0 on
 *   obstacles.  dmax is the truncation distance in voxels; D saturates at dmax^2.
 *
 * Three exact evaluations of that definition:
 *   oracle_edt_naive       -- the definition written out: loop over every obstacle.
 *   oracle_edt_factorised  -- the same minimum taken one axis at a time:
 *                             min over dz of dz^2 + min over dy of dy^2 + min over dx of dx^2 + [occ],
 *                             each window |d| < dmax (a farther offset contributes >= dmax^2).
 *                             Exact because min distributes over +.  Plain nested loops.
 *   oracle_edt_at          -- spot values at given voxels by scanning every integer offset of
 *                             squared length < dmax^2 in increasing length (first hit wins).
 *
 * And the paper's own method (Alg. 1, Sec. IV-B): a priority-queue raise/lower transform, global
 * (seed every obstacle, Lower only, Sec. V-A "Global Transform v.s. Incremental Transform") and
 * incremental (SetObstacle / RemoveObstacle per net change, then DistanceTransform).  Readings
 * taken where the paper is silent:
 *   - every d_max inside Alg. 1 is the squared truncation dmax^2 (dist, raise and priorities are
 *     squared distances, as sqDist is);
 *   - isObst(c) is the current occupancy bit of cell c, flipped by SetObstacle/RemoveObstacle;
 *     isObst of an empty obst field is false;
 *   - queue ties pop in insertion order (priority, sequence number);
 *   - Adj26 skips cells outside the grid;
 *   - a frame's edits are reduced to net flips (last write wins) and seeded in ascending linear
 *     index order.
 * Alg. 1 is not claimed by the paper to equal Eq. 1 exactly; the tests count its disagreements.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static int nthreads_of(int t) {
#ifdef _OPENMP
  return t > 0 ? t : omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

int oracle_num_threads(int t) { return nthreads_of(t); }

/* ---------------------------------------------------------------------------------------------- */
/* Eq. 1 written out                                                                               */
/* ---------------------------------------------------------------------------------------------- */

int oracle_edt_naive(const uint8_t* occ, int nx, int ny, int nz, int dmax, int32_t* out, int threads) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || dmax < 1) return 1;
  const i64 n = (i64)nx * ny * nz;
  i64 nobs = 0;
  for (i64 i = 0; i < n; ++i) nobs += occ[i] != 0;
  int32_t* obs = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nobs ? nobs : 1));
  i64 k = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        if (occ[((i64)z * ny + y) * nx + x]) {
          obs[3 * k] = x;
          obs[3 * k + 1] = y;
          obs[3 * k + 2] = z;
          ++k;
        }
  const i64 cap = (i64)dmax * dmax;
  int nt = nthreads_of(threads);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (i64 i = 0; i < n; ++i) {
    int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((i64)nx * ny));
    i64 best = cap;
    for (i64 j = 0; j < nobs; ++j) {
      i64 dx = x - obs[3 * j], dy = y - obs[3 * j + 1], dz = z - obs[3 * j + 2];
      i64 d2 = dx * dx + dy * dy + dz * dz;
      if (d2 < best) best = d2;
    }
    out[i] = (int32_t)best;
  }
  free(obs);
  return 0;
}

/* ---------------------------------------------------------------------------------------------- */
/* Eq. 1 one axis at a time                                                                        */
/* ---------------------------------------------------------------------------------------------- */

int oracle_edt_factorised(const uint8_t* occ, int nx, int ny, int nz, int dmax, int32_t* out, int threads) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || dmax < 1) return 1;
  const i64 n = (i64)nx * ny * nz;
  const int32_t cap = dmax * dmax;
  const int w = dmax - 1; /* largest offset that can stay below the cap */
  int32_t* g1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* g2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!g1 || !g2) {
    free(g1);
    free(g2);
    return 2;
  }
  int nt = nthreads_of(threads);
  /* x: g1 = min over occupied x' with |x'-x| <= w of (x'-x)^2, else cap */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (i64 line = 0; line < (i64)ny * nz; ++line) {
    const uint8_t* o = occ + line * nx;
    int32_t* g = g1 + line * nx;
    for (int x = 0; x < nx; ++x) {
      int32_t best = cap;
      for (int d = -w; d <= w; ++d) {
        int xx = x + d;
        if (xx < 0 || xx >= nx || !o[xx]) continue;
        if (d * d < best) best = d * d;
      }
      g[x] = best;
    }
  }
  /* y: g2 = min(cap, min over |dy| <= w of dy^2 + g1(y + dy)) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (i64 zx = 0; zx < (i64)nz * nx; ++zx) {
    int z = (int)(zx / nx), x = (int)(zx % nx);
    for (int y = 0; y < ny; ++y) {
      int32_t best = cap;
      for (int d = -w; d <= w; ++d) {
        int yy = y + d;
        if (yy < 0 || yy >= ny) continue;
        int32_t c = d * d + g1[((i64)z * ny + yy) * nx + x];
        if (c < best) best = c;
      }
      g2[((i64)z * ny + y) * nx + x] = best;
    }
  }
  /* z: D = min(cap, min over |dz| <= w of dz^2 + g2(z + dz)) */
#pragma omp parallel for schedule(static) num_threads(nt)
  for (i64 yx = 0; yx < (i64)ny * nx; ++yx) {
    int y = (int)(yx / nx), x = (int)(yx % nx);
    for (int z = 0; z < nz; ++z) {
      int32_t best = cap;
      for (int d = -w; d <= w; ++d) {
        int zz = z + d;
        if (zz < 0 || zz >= nz) continue;
        int32_t c = d * d + g2[((i64)zz * ny + y) * nx + x];
        if (c < best) best = c;
      }
      out[((i64)z * ny + y) * nx + x] = best;
    }
  }
  free(g1);
  free(g2);
  return 0;
}

/* ---------------------------------------------------------------------------------------------- */
/* Eq. 1 at sampled voxels: offsets in increasing squared length                                   */
/* ---------------------------------------------------------------------------------------------- */

typedef struct {
  int32_t d2;
  int8_t dx, dy, dz;
} offset_t;

static int cmp_off(const void* a, const void* b) {
  const offset_t* p = (const offset_t*)a;
  const offset_t* q = (const offset_t*)b;
  return (p->d2 > q->d2) - (p->d2 < q->d2);
}

int oracle_edt_at(const uint8_t* occ, int nx, int ny, int nz, int dmax, const int32_t* xyz, i64 m, int32_t* out,
                  int threads) {
  if (dmax < 1 || dmax > 127) return 1;
  const int w = dmax - 1;
  const int32_t cap = dmax * dmax;
  i64 no = 0;
  offset_t* offs = (offset_t*)malloc(sizeof(offset_t) * (size_t)(2 * w + 1) * (2 * w + 1) * (2 * w + 1));
  for (int dz = -w; dz <= w; ++dz)
    for (int dy = -w; dy <= w; ++dy)
      for (int dx = -w; dx <= w; ++dx) {
        int32_t d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < cap) {
          offs[no].d2 = d2;
          offs[no].dx = (int8_t)dx;
          offs[no].dy = (int8_t)dy;
          offs[no].dz = (int8_t)dz;
          ++no;
        }
      }
  qsort(offs, (size_t)no, sizeof(offset_t), cmp_off);
  int nt = nthreads_of(threads);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt) reduction(| : bad)
  for (i64 i = 0; i < m; ++i) {
    int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) {
      out[i] = cap;
      bad = 1;
      continue;
    }
    int32_t best = cap;
    for (i64 k = 0; k < no; ++k) {
      int xx = x + offs[k].dx, yy = y + offs[k].dy, zz = z + offs[k].dz;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
      if (occ[((i64)zz * ny + yy) * nx + xx]) {
        best = offs[k].d2;
        break;
      }
    }
    out[i] = best;
  }
  free(offs);
  return bad ? 3 : 0;
}

/* ---------------------------------------------------------------------------------------------- */
/* Alg. 1: priority-queue raise/lower transform                                                    */
/* ---------------------------------------------------------------------------------------------- */

#define NOT_RAISE (-1) /* Alg. 1 SetObstacle: "notRaise", commented as -1 */
#define NO_OBST (-1)   /* the empty obst field */

typedef struct {
  i64 obst;      /* linear index of the indexed obstacle, or NO_OBST */
  int32_t dist;  /* squared distance (transform radius), saturates at dmax^2 */
  int32_t raise; /* NOT_RAISE or the radius of the raising wave through this cell */
  uint8_t queued;
} cell_t;

typedef struct {
  int32_t prio;
  uint64_t seq;
  i64 cell;
} qent_t;

typedef struct {
  int nx, ny, nz;
  int32_t dmax2;
  i64 n;
  cell_t* c;
  uint8_t* occ; /* isObst */
  qent_t* heap;
  i64 hn, hcap;
  uint64_t seq;
  /* counters (Table II style): cells popped by Lower / Raise, queue inserts */
  i64 n_lower, n_raise, n_insert;
} alg1_t;

static int qless(const qent_t* a, const qent_t* b) {
  return a->prio < b->prio || (a->prio == b->prio && a->seq < b->seq);
}

static void q_insert(alg1_t* s, i64 cell, int32_t prio) {
  if (s->hn == s->hcap) {
    s->hcap = s->hcap ? 2 * s->hcap : 1024;
    s->heap = (qent_t*)realloc(s->heap, sizeof(qent_t) * (size_t)s->hcap);
  }
  i64 i = s->hn++;
  qent_t e = {prio, s->seq++, cell};
  while (i > 0) {
    i64 p = (i - 1) / 2;
    if (!qless(&e, &s->heap[p])) break;
    s->heap[i] = s->heap[p];
    i = p;
  }
  s->heap[i] = e;
  s->n_insert++;
}

static i64 q_pop(alg1_t* s) {
  i64 top = s->heap[0].cell;
  qent_t last = s->heap[--s->hn];
  i64 i = 0;
  for (;;) {
    i64 l = 2 * i + 1, r = l + 1, m = i;
    const qent_t* best = &last;
    if (l < s->hn && qless(&s->heap[l], best)) {
      m = l;
      best = &s->heap[l];
    }
    if (r < s->hn && qless(&s->heap[r], best)) m = r;
    if (m == i) break;
    s->heap[i] = s->heap[m];
    i = m;
  }
  if (s->hn > 0) s->heap[i] = last;
  return top;
}

static inline int32_t sq_dist(const alg1_t* s, i64 a, i64 b) {
  i64 ax = a % s->nx, ay = (a / s->nx) % s->ny, az = a / ((i64)s->nx * s->ny);
  i64 bx = b % s->nx, by = (b / s->nx) % s->ny, bz = b / ((i64)s->nx * s->ny);
  i64 d = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
  return d > 0x7fffffff ? 0x7fffffff : (int32_t)d;
}

static inline int is_obst(const alg1_t* s, i64 cell) { return cell != NO_OBST && s->occ[cell]; }

/* Initialize(s) for every cell: obst <- empty, dist <- dmax^2, raise <- notRaise, notQueued. */
void* alg1_create(int nx, int ny, int nz, int dmax) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || dmax < 1) return NULL;
  alg1_t* s = (alg1_t*)calloc(1, sizeof(alg1_t));
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->dmax2 = dmax * dmax;
  s->n = (i64)nx * ny * nz;
  s->c = (cell_t*)malloc(sizeof(cell_t) * (size_t)s->n);
  s->occ = (uint8_t*)calloc((size_t)s->n, 1);
  if (!s->c || !s->occ) {
    free(s->c);
    free(s->occ);
    free(s);
    return NULL;
  }
  for (i64 i = 0; i < s->n; ++i) {
    s->c[i].obst = NO_OBST;
    s->c[i].dist = s->dmax2;
    s->c[i].raise = NOT_RAISE;
    s->c[i].queued = 0;
  }
  return s;
}

void alg1_destroy(void* h) {
  alg1_t* s = (alg1_t*)h;
  if (!s) return;
  free(s->c);
  free(s->occ);
  free(s->heap);
  free(s);
}

/* SetObstacle(s): a free, unqueued cell becomes its own obstacle at distance 0, lowering wave. */
static void set_obstacle(alg1_t* s, i64 i) {
  cell_t* c = &s->c[i];
  if (!s->occ[i] && !c->queued) {
    c->obst = i;
    c->dist = 0;
    c->raise = NOT_RAISE;
    c->queued = 1;
    q_insert(s, i, 0);
    s->occ[i] = 1;
  }
}

/* RemoveObstacle(s): an occupied, unqueued cell is cleared and starts a raising wave (raise = 0). */
static void remove_obstacle(alg1_t* s, i64 i) {
  cell_t* c = &s->c[i];
  if (s->occ[i] && !c->queued) {
    c->obst = NO_OBST;
    c->dist = s->dmax2;
    c->raise = 0;
    c->queued = 1;
    q_insert(s, i, 0);
    s->occ[i] = 0;
  }
}

static void raise_cell(alg1_t* s, i64 si) {
  const int sx = (int)(si % s->nx), sy = (int)((si / s->nx) % s->ny), sz = (int)(si / ((i64)s->nx * s->ny));
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        int x = sx + dx, y = sy + dy, z = sz + dz;
        if (x < 0 || y < 0 || z < 0 || x >= s->nx || y >= s->ny || z >= s->nz) continue;
        i64 ni = ((i64)z * s->ny + y) * s->nx + x;
        cell_t* n = &s->c[ni];
        if (n->obst == NO_OBST) continue;
        if (!is_obst(s, n->obst)) {
          /* the obstacle n indexes is gone: n joins the raising wave at its own radius (key-1) */
          n->raise = n->dist;
          n->queued = 1;
          q_insert(s, ni, n->dist);
          n->obst = NO_OBST;
          n->dist = s->dmax2;
        } else if (!n->queued) {
          /* a wave boundary: n still holds a valid obstacle and will re-lower the cleared cells */
          n->queued = 1;
          q_insert(s, ni, n->dist);
        }
      }
  s->c[si].raise = NOT_RAISE;
  s->c[si].queued = 0;
}

static void lower_cell(alg1_t* s, i64 si) {
  cell_t* sc = &s->c[si];
  const i64 so = sc->obst;
  const int sx = (int)(si % s->nx), sy = (int)((si / s->nx) % s->ny), sz = (int)(si / ((i64)s->nx * s->ny));
  if (so != NO_OBST) {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int x = sx + dx, y = sy + dy, z = sz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= s->nx || y >= s->ny || z >= s->nz) continue;
          i64 ni = ((i64)z * s->ny + y) * s->nx + x;
          cell_t* n = &s->c[ni];
          int32_t dnew = sq_dist(s, so, ni);
          if (dnew > s->dmax2) dnew = s->dmax2;
          if (n->raise >= dnew) {
            /* key-2: a raising front closer to this lowering wave is lowered at once */
            n->obst = so;
            n->dist = dnew;
            n->raise = NOT_RAISE;
            n->queued = 1;
            q_insert(s, ni, dnew);
            continue;
          } else if (n->raise < 0) {
            int occ = is_obst(s, n->obst);
            int equ = dnew == n->dist, less = dnew < n->dist;
            if (less || (equ && !occ)) {
              n->obst = so;
              n->dist = dnew;
              n->raise = NOT_RAISE;
              if (dnew < s->dmax2) {
                n->queued = 1;
                q_insert(s, ni, dnew);
              }
            }
          }
        }
  }
  sc->raise = NOT_RAISE;
  sc->queued = 0;
}

/* DistanceTransform(): pop in priority order; skip stale entries; raise >= 0 -> Raise else Lower. */
static void distance_transform(alg1_t* s) {
  while (s->hn > 0) {
    i64 i = q_pop(s);
    if (!s->c[i].queued) continue;
    if (s->c[i].raise >= 0) {
      s->n_raise++;
      raise_cell(s, i);
    } else {
      s->n_lower++;
      lower_cell(s, i);
    }
  }
}

/* Global transform: all cells initialised, every occupied cell seeded, Lower only. */
int alg1_global(void* h, const uint8_t* occ) {
  alg1_t* s = (alg1_t*)h;
  for (i64 i = 0; i < s->n; ++i) {
    s->c[i].obst = NO_OBST;
    s->c[i].dist = s->dmax2;
    s->c[i].raise = NOT_RAISE;
    s->c[i].queued = 0;
  }
  memset(s->occ, 0, (size_t)s->n);
  s->hn = 0;
  for (i64 i = 0; i < s->n; ++i)
    if (occ[i]) set_obstacle(s, i);
  distance_transform(s);
  return 0;
}

/* Incremental transform for one frame of edit records (x, y, z, value in {0,1}); the last record
 * for a voxel wins, and only net flips against the pre-frame occupancy seed waves. */
int alg1_update(void* h, const int32_t* xyz, const uint8_t* val, i64 m) {
  alg1_t* s = (alg1_t*)h;
  if (m < 0) return 1;
  for (i64 k = 0; k < m; ++k) {
    int x = xyz[3 * k], y = xyz[3 * k + 1], z = xyz[3 * k + 2];
    if (x < 0 || y < 0 || z < 0 || x >= s->nx || y >= s->ny || z >= s->nz || val[k] > 1) return 1;
  }
  /* last write wins: per-voxel final value, gathered through a scratch index */
  i64* idx = (i64*)malloc(sizeof(i64) * (size_t)(m ? m : 1));
  uint8_t* fin = (uint8_t*)malloc((size_t)(m ? m : 1));
  i64 nu = 0;
  /* sort record positions by (cell, record order); the last of each run is the final value */
  i64* key = (i64*)malloc(sizeof(i64) * (size_t)(m ? m : 1));
  i64* ord = (i64*)malloc(sizeof(i64) * (size_t)(m ? m : 1));
  for (i64 k = 0; k < m; ++k) {
    key[k] = ((i64)xyz[3 * k + 2] * s->ny + xyz[3 * k + 1]) * s->nx + xyz[3 * k];
    ord[k] = k;
  }
  /* insertion into a simple merge sort on (key, k) */
  i64* tmp = (i64*)malloc(sizeof(i64) * (size_t)(m ? m : 1));
  for (i64 width = 1; width < m; width *= 2) {
    for (i64 lo = 0; lo < m; lo += 2 * width) {
      i64 mid = lo + width < m ? lo + width : m, hi = lo + 2 * width < m ? lo + 2 * width : m;
      i64 a = lo, b = mid, o = lo;
      while (a < mid && b < hi) tmp[o++] = (key[ord[b]] < key[ord[a]]) ? ord[b++] : ord[a++];
      while (a < mid) tmp[o++] = ord[a++];
      while (b < hi) tmp[o++] = ord[b++];
    }
    memcpy(ord, tmp, sizeof(i64) * (size_t)m);
  }
  for (i64 k = 0; k < m; ++k) {
    if (k + 1 < m && key[ord[k + 1]] == key[ord[k]]) continue;
    idx[nu] = key[ord[k]];
    fin[nu] = val[ord[k]];
    ++nu;
  }
  for (i64 k = 0; k < nu; ++k) {
    i64 i = idx[k];
    if (fin[k] && !s->occ[i])
      set_obstacle(s, i);
    else if (!fin[k] && s->occ[i])
      remove_obstacle(s, i);
  }
  free(idx);
  free(fin);
  free(key);
  free(ord);
  free(tmp);
  distance_transform(s);
  return 0;
}

void alg1_read(void* h, int32_t* dist_out, uint8_t* occ_out) {
  alg1_t* s = (alg1_t*)h;
  for (i64 i = 0; i < s->n; ++i) dist_out[i] = s->c[i].dist;
  if (occ_out) memcpy(occ_out, s->occ, (size_t)s->n);
}

void alg1_counters(void* h, i64* out3) {
  alg1_t* s = (alg1_t*)h;
  out3[0] = s->n_lower;
  out3[1] = s->n_raise;
  out3[2] = s->n_insert;
}

void alg1_reset_counters(void* h) {
  alg1_t* s = (alg1_t*)h;
  s->n_lower = s->n_raise = s->n_insert = 0;
}
