/*
 * Seeded synthetic workload generators (host C, OpenMP).
 *
 * These produce the occupancy grids, edit streams and query points that both
 * the CPU oracle and the CUDA library consume.  They contain none of the
 * distance-transform arithmetic: only random numbers, geometry of the
 * synthetic scenes and a voxel ray walker that stands in for a lidar-based
 * mapping front end.
 *
 * Random numbers: a counter-based SplitMix64 (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).  The value for
 * (seed, stream, index) is the finaliser applied to
 *     base(seed, stream) + (index + 1) * GAMMA,
 * with base(seed, stream) = mix(seed * GAMMA + stream), i.e. the index-th
 * output of a SplitMix64 sequence keyed by (seed, stream).  The Python module
 * beside this file restates the same definition in numpy so that small inputs
 * can be produced without the compiled library.
 *
 * Built with -ffp-contract=off so that x86-64 and aarch64 produce identical
 * floating-point results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t wl_rng(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t base = mix64(seed * GAMMA + stream);
  return mix64(base + (idx + 1) * GAMMA);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Bernoulli threshold: an event with probability p fires iff rng < thr(p). */
static inline uint64_t bern_thr(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return UINT64_MAX;
  return (uint64_t)(p * 18446744073709551616.0);
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
  int t = nthreads > 0 ? nthreads : omp_get_max_threads();
  return t;
#else
  (void)nthreads;
  return 1;
#endif
}

/* out[i] = 1 iff rng(seed, stream, i) < p * 2^64, for i in [0, n). */
void wl_bernoulli(uint64_t seed, uint64_t stream, double p, int64_t n, uint8_t* out, int nthreads) {
  const uint64_t thr = bern_thr(p);
  const uint64_t base = mix64(seed * GAMMA + stream);
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) out[i] = mix64(base + (uint64_t)(i + 1) * GAMMA) < thr ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Tunnel scene                                                              */
/* ------------------------------------------------------------------------ */

#define CR_STEPS 64        /* samples per Catmull-Rom segment */
#define CR_CTRL 5          /* control points per tunnel        */
#define CR_NSAMP ((CR_CTRL - 1) * CR_STEPS + 1)

int wl_tunnel_nsamples(void) { return CR_NSAMP; }

/* Uniform Catmull-Rom point between p1 and p2 at parameter t in [0,1]. */
static void catmull_rom(const double* p0, const double* p1, const double* p2, const double* p3, double t,
                        double* out) {
  double t2 = t * t, t3 = t2 * t;
  for (int a = 0; a < 3; ++a) {
    out[a] = 0.5 * ((2.0 * p1[a]) + (-p0[a] + p2[a]) * t + (2.0 * p0[a] - 5.0 * p1[a] + 4.0 * p2[a] - p3[a]) * t2 +
                    (-p0[a] + 3.0 * p1[a] - 3.0 * p2[a] + p3[a]) * t3);
  }
}

/* Centre lines and radii of the tunnels (no voxelisation).
 *   radii[ntunnels], centre[ntunnels][CR_NSAMP][3] (voxel units, voxel centres at integers).
 * Tunnel t draws from stream 100 + t: index 0 -> radius U[rmin, rmax], indices 1..15 -> five
 * control points, each uniform in the domain shrunk by r + 2 (z in [r+2, nz-3-r]). */
void wl_tunnel_lines(uint64_t seed, int nx, int ny, int nz, int ntunnels, double rmin, double rmax, double* radii,
                     double* centre) {
  for (int t = 0; t < ntunnels; ++t) {
    uint64_t st = 100 + (uint64_t)t;
    double r = rmin + u01(wl_rng(seed, st, 0)) * (rmax - rmin);
    radii[t] = r;
    double ctrl[CR_CTRL + 2][3];
    double lo[3] = {r + 2.0, r + 2.0, r + 2.0};
    double hi[3] = {nx - 1 - (r + 2.0), ny - 1 - (r + 2.0), nz - 3 - r};
    for (int c = 0; c < CR_CTRL; ++c)
      for (int a = 0; a < 3; ++a) {
        double h = hi[a] > lo[a] ? hi[a] : lo[a];
        ctrl[c + 1][a] = lo[a] + u01(wl_rng(seed, st, 1 + (uint64_t)(c * 3 + a))) * (h - lo[a]);
      }
    for (int a = 0; a < 3; ++a) {
      ctrl[0][a] = ctrl[1][a];
      ctrl[CR_CTRL + 1][a] = ctrl[CR_CTRL][a];
    }
    double* out = centre + (size_t)t * CR_NSAMP * 3;
    int k = 0;
    for (int s = 0; s < CR_CTRL - 1; ++s) {
      for (int i = 0; i < CR_STEPS; ++i) catmull_rom(ctrl[s], ctrl[s + 1], ctrl[s + 2], ctrl[s + 3], (double)i / CR_STEPS, out + 3 * (k++));
    }
    catmull_rom(ctrl[CR_CTRL - 2], ctrl[CR_CTRL - 1], ctrl[CR_CTRL], ctrl[CR_CTRL + 1], 1.0, out + 3 * (k++));
  }
}

static inline double seg_dist2(double px, double py, double pz, const double* a, const double* b) {
  double ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
  double wx = px - a[0], wy = py - a[1], wz = pz - a[2];
  double uu = ux * ux + uy * uy + uz * uz;
  double t = uu > 0.0 ? (wx * ux + wy * uy + wz * uz) / uu : 0.0;
  if (t < 0.0) t = 0.0;
  if (t > 1.0) t = 1.0;
  double dx = wx - t * ux, dy = wy - t * uy, dz = wz - t * uz;
  return dx * dx + dy * dy + dz * dz;
}

/* Voxelise the tunnel scene into out[nz][ny][nx] (1 = wall).
 * A voxel is wall iff, for some tunnel, r <= dist(v, centre line) < r + shell, and it lies inside
 * no tunnel's interior (dist < r), so that crossing tunnels open into one another.  The centre
 * line is the polyline through the Catmull-Rom samples. */
void wl_tunnels(uint64_t seed, int nx, int ny, int nz, int ntunnels, double rmin, double rmax, double shell,
                uint8_t* out, int nthreads) {
  double* radii = (double*)malloc(sizeof(double) * ntunnels);
  double* centre = (double*)malloc(sizeof(double) * (size_t)ntunnels * CR_NSAMP * 3);
  wl_tunnel_lines(seed, nx, ny, nz, ntunnels, rmin, rmax, radii, centre);
  int nt = set_threads(nthreads);
#pragma omp parallel num_threads(nt)
  {
    uint8_t* interior = (uint8_t*)malloc((size_t)nx * ny);
    uint8_t* shellm = (uint8_t*)malloc((size_t)nx * ny);
#pragma omp for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z) {
      memset(interior, 0, (size_t)nx * ny);
      memset(shellm, 0, (size_t)nx * ny);
      int any = 0;
      for (int t = 0; t < ntunnels; ++t) {
        const double r = radii[t], ro = r + shell;
        const double r2 = r * r, ro2 = ro * ro;
        const double* c = centre + (size_t)t * CR_NSAMP * 3;
        for (int s = 0; s + 1 < CR_NSAMP; ++s) {
          const double* a = c + 3 * s;
          const double* b = c + 3 * (s + 1);
          double zlo = fmin(a[2], b[2]) - ro, zhi = fmax(a[2], b[2]) + ro;
          if (z < zlo || z > zhi) continue;
          int x0 = (int)ceil(fmin(a[0], b[0]) - ro), x1 = (int)floor(fmax(a[0], b[0]) + ro);
          int y0 = (int)ceil(fmin(a[1], b[1]) - ro), y1 = (int)floor(fmax(a[1], b[1]) + ro);
          if (x0 < 0) x0 = 0;
          if (y0 < 0) y0 = 0;
          if (x1 > nx - 1) x1 = nx - 1;
          if (y1 > ny - 1) y1 = ny - 1;
          any = 1;
          for (int y = y0; y <= y1; ++y) {
            size_t row = (size_t)y * nx;
            for (int x = x0; x <= x1; ++x) {
              double d2 = seg_dist2((double)x, (double)y, (double)z, a, b);
              if (d2 < r2)
                interior[row + x] = 1;
              else if (d2 < ro2)
                shellm[row + x] = 1;
            }
          }
        }
      }
      uint8_t* o = out + (size_t)z * nx * ny;
      if (!any) {
        memset(o, 0, (size_t)nx * ny);
        continue;
      }
      for (size_t i = 0; i < (size_t)nx * ny; ++i) o[i] = (uint8_t)(shellm[i] & (uint8_t)(interior[i] ^ 1));
    }
    free(interior);
    free(shellm);
  }
  free(radii);
  free(centre);
}

/* ------------------------------------------------------------------------ */
/* Lidar ray walker (stands in for the occupancy-mapping front end)         */
/* ------------------------------------------------------------------------ */

/* Pose on a polyline at arc-length fraction frac in [0, 1]: position and yaw of the local tangent. */
void wl_polyline_pose(const double* pts, int n, double frac, double* pos, double* yaw) {
  double total = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    double dx = pts[3 * i + 3] - pts[3 * i], dy = pts[3 * i + 4] - pts[3 * i + 1], dz = pts[3 * i + 5] - pts[3 * i + 2];
    total += sqrt(dx * dx + dy * dy + dz * dz);
  }
  double target = frac * total, acc = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double* a = pts + 3 * i;
    const double* b = pts + 3 * i + 3;
    double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    double len = sqrt(dx * dx + dy * dy + dz * dz);
    if (acc + len >= target || i + 2 == n) {
      double t = len > 0.0 ? (target - acc) / len : 0.0;
      if (t < 0.0) t = 0.0;
      if (t > 1.0) t = 1.0;
      pos[0] = a[0] + t * dx;
      pos[1] = a[1] + t * dy;
      pos[2] = a[2] + t * dz;
      *yaw = atan2(dy, dx);
      return;
    }
    acc += len;
  }
  pos[0] = pts[0];
  pos[1] = pts[1];
  pos[2] = pts[2];
  *yaw = 0.0;
}

typedef struct {
  int32_t* xyz;
  uint8_t* val;
  int64_t n, cap;
} recbuf;

static void rec_push(recbuf* b, int x, int y, int z, uint8_t v) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 4096;
    b->xyz = (int32_t*)realloc(b->xyz, sizeof(int32_t) * 3 * b->cap);
    b->val = (uint8_t*)realloc(b->val, b->cap);
  }
  b->xyz[3 * b->n] = x;
  b->xyz[3 * b->n + 1] = y;
  b->xyz[3 * b->n + 2] = z;
  b->val[b->n] = v;
  b->n++;
}

/* One lidar frame.  Casts nbeams x nazim rays from pos (voxel units; voxel v spans [v-0.5, v+0.5))
 * with elevations evenly spaced over [elev_lo, elev_hi] (radians) and azimuths evenly spaced over
 * a full turn, rotated by yaw about z.  Each ray walks voxels with the Amanatides-Woo stepping rule
 * ("A fast voxel traversal algorithm for ray tracing", Eurographics 1987) until its entry distance
 * exceeds maxrange or it leaves the domain.
 *
 * Records, in ray order and along each ray in walk order:
 *   - a traversed voxel that `map` holds as occupied -> (v, 0)
 *   - the first voxel that `truth` holds as wall     -> (v, 1), or (v, 0) with probability
 *     noise_p (spurious delete; stream 9)
 *   - with probability noise_p (stream 7), a spurious obstacle at a traversed voxel chosen by
 *     stream 8 -> (u, 1)
 * Every ray sees `map` as it was before the frame.  The records are then applied to `map` in
 * order (last write wins).  Returns the record count, or -(count) when cap is too small (nothing
 * is written to out_* or map in that case). */
int64_t wl_lidar_frame(const uint8_t* truth, uint8_t* map, int nx, int ny, int nz, const double* pos, double yaw,
                       int nbeams, int nazim, double elev_lo, double elev_hi, double maxrange, uint64_t seed,
                       int64_t frame, double noise_p, int32_t* out_xyz, uint8_t* out_val, int64_t cap,
                       int nthreads) {
  const int64_t nrays = (int64_t)nbeams * nazim;
  const uint64_t thr = bern_thr(noise_p);
  int nt = set_threads(nthreads);
  recbuf* bufs = (recbuf*)calloc((size_t)nt, sizeof(recbuf));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    recbuf* rb = &bufs[tid];
    int32_t* trav = (int32_t*)malloc(sizeof(int32_t) * 3 * ((size_t)maxrange * 3 + 8));
#pragma omp for schedule(static)
    for (int64_t k = 0; k < nrays; ++k) {
      int b = (int)(k / nazim), a = (int)(k % nazim);
      double el = nbeams > 1 ? elev_lo + (elev_hi - elev_lo) * b / (nbeams - 1) : 0.5 * (elev_lo + elev_hi);
      double az = 2.0 * M_PI * a / nazim + yaw;
      double d[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
      double q[3] = {pos[0] + 0.5, pos[1] + 0.5, pos[2] + 0.5};
      int v[3], step[3];
      double tmax[3], tdel[3];
      int dims[3] = {nx, ny, nz};
      int ok = 1;
      for (int c = 0; c < 3; ++c) {
        v[c] = (int)floor(q[c]);
        if (v[c] < 0 || v[c] >= dims[c]) ok = 0;
        if (d[c] > 0) {
          step[c] = 1;
          tdel[c] = 1.0 / d[c];
          tmax[c] = (v[c] + 1 - q[c]) / d[c];
        } else if (d[c] < 0) {
          step[c] = -1;
          tdel[c] = -1.0 / d[c];
          tmax[c] = (v[c] - q[c]) / d[c];
        } else {
          step[c] = 0;
          tdel[c] = INFINITY;
          tmax[c] = INFINITY;
        }
      }
      if (!ok) continue;
      int ntrav = 0, hit = 0;
      int64_t base = (int64_t)frame * nrays + k;
      double tentry = 0.0;
      while (tentry <= maxrange) {
        size_t li = ((size_t)v[2] * ny + v[1]) * nx + v[0];
        if (truth[li]) {
          hit = 1;
          break;
        }
        trav[3 * ntrav] = v[0];
        trav[3 * ntrav + 1] = v[1];
        trav[3 * ntrav + 2] = v[2];
        ntrav++;
        if (map[li]) rec_push(rb, v[0], v[1], v[2], 0);
        int c = (tmax[0] < tmax[1]) ? (tmax[0] < tmax[2] ? 0 : 2) : (tmax[1] < tmax[2] ? 1 : 2);
        tentry = tmax[c];
        tmax[c] += tdel[c];
        v[c] += step[c];
        if (v[c] < 0 || v[c] >= dims[c]) break;
      }
      if (hit) {
        uint8_t hv = wl_rng(seed, 9, (uint64_t)base) < thr ? 0 : 1;
        rec_push(rb, v[0], v[1], v[2], hv);
        if (ntrav > 0 && wl_rng(seed, 7, (uint64_t)base) < thr) {
          int j = (int)(wl_rng(seed, 8, (uint64_t)base) % (uint64_t)ntrav);
          rec_push(rb, trav[3 * j], trav[3 * j + 1], trav[3 * j + 2], 1);
        }
      }
    }
    free(trav);
  }
  int64_t total = 0;
  for (int t = 0; t < nt; ++t) total += bufs[t].n;
  int64_t ret = total;
  if (total > cap) {
    ret = -total;
  } else {
    int64_t o = 0;
    for (int t = 0; t < nt; ++t) {
      memcpy(out_xyz + 3 * o, bufs[t].xyz, sizeof(int32_t) * 3 * bufs[t].n);
      memcpy(out_val + o, bufs[t].val, bufs[t].n);
      o += bufs[t].n;
    }
    for (int64_t i = 0; i < total; ++i) {
      size_t li = ((size_t)out_xyz[3 * i + 2] * ny + out_xyz[3 * i + 1]) * nx + out_xyz[3 * i];
      map[li] = out_val[i];
    }
  }
  for (int t = 0; t < nt; ++t) {
    free(bufs[t].xyz);
    free(bufs[t].val);
  }
  free(bufs);
  return ret;
}

/* ------------------------------------------------------------------------ */
/* Batched random maps                                                       */
/* ------------------------------------------------------------------------ */

/* Parameters of map m (stream 1000 + m): side = round(exp(U[ln smin, ln smax])) rounded up to a
 * multiple of 8; p ~ U[pmin, pmax]; k ~ U{0..kmax} boxes. */
void wl_batched_params(uint64_t seed, int m, int smin, int smax, double pmin, double pmax, int kmax, int* side,
                       double* p, int* nboxes) {
  uint64_t st = 1000 + (uint64_t)m;
  double ls = log((double)smin) + u01(wl_rng(seed, st, 0)) * (log((double)smax) - log((double)smin));
  int s = (int)floor(exp(ls) + 0.5);
  s = ((s + 7) / 8) * 8;
  if (s < 8) s = 8;
  *side = s;
  *p = pmin + u01(wl_rng(seed, st, 1)) * (pmax - pmin);
  *nboxes = (int)(wl_rng(seed, st, 2) % (uint64_t)(kmax + 1));
}

/* Map m as a dense side^3 grid: Bernoulli(p) voxels (stream 2000000 + m) plus solid boxes with
 * integer sides U{2..side/4} at uniform positions (stream 1000 + m, indices 3..). */
void wl_batched_map(uint64_t seed, int m, int smin, int smax, double pmin, double pmax, int kmax, uint8_t* out,
                    int nthreads) {
  int s, nb;
  double p;
  wl_batched_params(seed, m, smin, smax, pmin, pmax, kmax, &s, &p, &nb);
  wl_bernoulli(seed, 2000000 + (uint64_t)m, p, (int64_t)s * s * s, out, nthreads);
  uint64_t st = 1000 + (uint64_t)m;
  int smax_box = s / 4 < 2 ? 2 : s / 4;
  for (int k = 0; k < nb; ++k) {
    int sz[3], lo[3];
    for (int a = 0; a < 3; ++a) {
      sz[a] = 2 + (int)(wl_rng(seed, st, 3 + (uint64_t)(6 * k + a)) % (uint64_t)(smax_box - 1));
      lo[a] = (int)(wl_rng(seed, st, 3 + (uint64_t)(6 * k + 3 + a)) % (uint64_t)(s - sz[a] + 1));
    }
    for (int z = lo[2]; z < lo[2] + sz[2]; ++z)
      for (int y = lo[1]; y < lo[1] + sz[1]; ++y) memset(out + ((size_t)z * s + y) * s + lo[0], 1, (size_t)sz[0]);
  }
}

/* ------------------------------------------------------------------------ */
/* Query points in free space                                               */
/* ------------------------------------------------------------------------ */

/* n points (float xyz, metres) uniform in [0, (dim-1) * vs] per axis, rejection-sampled so that the
 * nearest voxel centre is free in occ.  Point i, attempt j draws axis a from stream 20 + a at index
 * i * 256 + j; after 256 failed attempts the last draw is kept.  Returns the number of points that
 * needed the fallback. */
int64_t wl_free_points(uint64_t seed, const uint8_t* occ, int nx, int ny, int nz, double vs, int64_t n, float* out,
                       int nthreads) {
  int dims[3] = {nx, ny, nz};
  int64_t fallback = 0;
  int nt = set_threads(nthreads);
#pragma omp parallel for schedule(static) num_threads(nt) reduction(+ : fallback)
  for (int64_t i = 0; i < n; ++i) {
    float p[3];
    int good = 0;
    for (int j = 0; j < 256 && !good; ++j) {
      int v[3];
      for (int a = 0; a < 3; ++a) {
        double u = u01(wl_rng(seed, 20 + (uint64_t)a, (uint64_t)i * 256 + (uint64_t)j)) * (dims[a] - 1);
        p[a] = (float)(u * vs);
        double vv = floor((double)p[a] / vs + 0.5);
        if (vv < 0) vv = 0;
        if (vv > dims[a] - 1) vv = dims[a] - 1;
        v[a] = (int)vv;
      }
      good = occ[((size_t)v[2] * ny + v[1]) * nx + v[0]] == 0;
    }
    if (!good) fallback++;
    out[3 * i] = p[0];
    out[3 * i + 1] = p[1];
    out[3 * i + 2] = p[2];
  }
  return fallback;
}
