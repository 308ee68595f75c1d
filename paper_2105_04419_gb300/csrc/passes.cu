// The separable transform passes over the sparse brick grid.
//
// D(v) = min(dmax^2, min over occupied o of |v - o|^2) (paper Eq. 1 with the truncation of
// Sec. III) factorises along the axes because min distributes over +:
//   g1(x,y,z) = min over occupied (x',y,z) of (x'-x)^2          (x pass; saturated at dmax^2)
//   g2(x,y,z) = min over |d| <= W of d^2 + g1(x,y+d,z)         (y pass)
//   D(x,y,z)  = min over |d| <= W of d^2 + g2(x,y,z+d)         (z pass)
// with any window W >= dmax - 1 (offsets of dmax or more cost at least dmax^2 and can never beat
// the d = 0 term, which is already saturated).  Here W = 8R, R = floor((dmax + 6) / 8): exactly the
// halo of R bricks a pass reads on each side.  A brick that is not stored has no obstacle within
// R bricks, so every intermediate value in it is dmax^2: absent bricks read as dmax^2.
//
// All three passes run in one warp-specialised kernel, k_pass<R, RUN, AXIS>.  A work item is a run
// of RUN bricks along the pass axis; its slot list (the run plus R bricks of halo on each side) is
// prepared when the item is queued.  A producer warp streams each item's brick inputs into a
// three-stage shared-memory ring with bulk asynchronous copies (cp.async.bulk global -> shared,
// completion counted in bytes on a "full" mbarrier per stage) and fills absent bricks itself;
// RUN consumer warps each own one output brick of the item, wait on the stage's full barrier,
// compute, write, and release the stage on its "empty" barrier.  No block-wide barrier sits on
// the main path, so warps whose windows exit early run ahead.
//   x (AXIS 0): inputs are the 64-byte occupancy masks.  Each lane expands two x-lines: the line's
//     occupancy is gathered from the masks of bricks bx-R..bx+R (one byte each) and the nearest
//     set bit on either side of each voxel is found with clz / ffs on a 64-bit window.  g1 is
//     stored y-major so that the y pass reads it as planes.
//   y, z (AXIS 1, 2): inputs are 1 KB bricks of g1 / g2.  In the staged column a plane along the
//     pass axis is 32 words (two voxels per word) and a lane's line is one word per plane, so the
//     32 lanes of a consumer read 32 consecutive words.
//
// Arithmetic of the windowed minimum: packed half2, two voxels per 32-bit lane.  Every operand is
// an integer in [0, 2048] (values are saturated at dmax^2 <= 2025 for dmax <= 45 before they enter
// a window, and offsets whose square exceeds 2048 are represented by 2048): fp16 represents each
// such integer exactly, the sum of two is exact whenever it is below 2048 and rounds to a value
// >= 2048 otherwise, and min is exact, so every minimum below dmax^2 is computed exactly and every
// candidate at or above it stays at or above it.  Each lane owns 8 consecutive outputs of two
// neighbouring lines, pairing offsets +d and -d: acc = min(acc, v[k-d] + d^2, v[k+d] + d^2), two
// fp16 adds and one three-input minimum taken on the bit patterns as unsigned 16-bit integers
// (non-negative fp16 values order like their bit patterns).  The pruned form stops when (d + 1)^2
// reaches every output's current minimum in the warp, and skips windows whose input bricks hold no
// value below dmax^2.
//
// Grids with dmax above 45 (up to 181), and any grid tuned to variant 8, take the lower-envelope
// kernels at the end of the file: O(1) amortised work per voxel, whatever the window.
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

// Sets or clears one bit of a brick's flags with a reduction (no value returned, so the warp does
// not wait for the word's round trip); each pass owns the bit it writes.
__device__ __forceinline__ void set_flag_bit(const GridView& g, int slot, uint32_t bit, bool on) {
  if (on)
    atomicOr(&g.bflags[slot], bit);
  else
    atomicAnd(&g.bflags[slot], ~bit);
}

// ---- asynchronous bulk copies and mbarriers (inline PTX) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Ordering between this thread's earlier generic-proxy accesses to shared memory and async-proxy
// writes issued after it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait for a phase of an mbarrier: gives up after one second of global time (or
// kWaitMaxPolls polls), sets the device error word and reports failure.
__device__ __forceinline__ bool mbar_wait_bounded(const GridView& g, uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0; i < kWaitMaxPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && global_ns() - t0 > kWaitLimitNs) break;
    if (i > 16) __nanosleep(64);
  }
  set_error(g, kErrTimeout);
  return false;
}

// One 8-output window minimum on packed half2 registers:
//   out[k] = min over |d| <= W of v[k + W + d] + d^2, pairing +d and -d,
// where v[j] is plane j of the lane's staged column (c[j * 32]).  Planes are loaded when first
// needed: the 8 centre planes, then at offset d the two planes that enter the window (W - d and
// W + 7 + d), so only about 16 planes are live at a time and the early exit also skips the loads.
// With `prune`, the offsets stop once (d + 1)^2 is at least every output's current minimum in the
// warp (a farther candidate costs at least (d + 1)^2, so none can lower any output); the test runs
// every 4 offsets and is warp-uniform.
template <int W>
__device__ __forceinline__ void window_min8(const uint32_t* __restrict__ c, uint32_t (&out)[8], bool prune) {
  static_assert(W % 4 == 0, "window is a multiple of 4 offsets");
  uint32_t v[8 + 2 * W];
  uint32_t acc[8];  // fp16x2 bits: non-negative halves order as unsigned 16-bit integers
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k + W] = c[(k + W) * 32];
    acc[k] = v[k + W];
  }
  bool live = true;  // warp-uniform
#pragma unroll
  for (int ch = 0; ch < W / 4; ++ch) {
    if (live) {
#pragma unroll
      for (int dd = 1; dd <= 4; ++dd) {
        const int d = 4 * ch + dd;
        v[W - d] = c[(W - d) * 32];
        v[W + 7 + d] = c[(W + 7 + d) * 32];
        const __half2 sq = u2h(half2_bits(d * d));
#pragma unroll
        for (int k = 0; k < 8; ++k) {  // two fp16 adds, one three-way minimum of the bit patterns
          const uint32_t lo = h2u(__hadd2(u2h(v[k + W - d]), sq)), hi = h2u(__hadd2(u2h(v[k + W + d]), sq));
          acc[k] = __vimin3_u16x2(acc[k], lo, hi);
        }
      }
      if (prune && ch + 1 < W / 4) {
        const int d1 = 4 * ch + 5;  // the next offset
        const uint32_t mx = __vimax3_u16x2(__vimax3_u16x2(acc[0], acc[1], acc[2]), __vimax3_u16x2(acc[3], acc[4], acc[5]),
                                           __vmaxu2(acc[6], acc[7]));
        const bool done = __hbge2(u2h(half2_bits(d1 * d1)), u2h(mx));
        live = !__all_sync(0xffffffffu, done);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = acc[k];
}

// ================================================================================================
// The three passes: warp-specialised kernel with a bulk-copy ring
// ================================================================================================
template <int R, int RUN, int AXIS>
struct ColShape {
  static constexpr int NB = RUN + 2 * R;                     // staged bricks per item
  static constexpr int NS = AXIS == 0 ? 8 : 3;               // ring stages (x stages are 64 B per brick)
  static constexpr int UNIT = AXIS == 0 ? 64 : 1024;         // bytes staged per brick
  static constexpr int STAGE_BYTES = NB * UNIT;
  static constexpr int META = 2 * NB;                        // slots, then input flags
  static constexpr int THREADS = 32 * (RUN + 1);
  static constexpr size_t DATA_BYTES = (size_t)NS * STAGE_BYTES;
  static constexpr size_t META_BYTES = (size_t)NS * META * 4;
  static constexpr size_t LUT_BYTES = 80;  // x pass: fp16 bits of min(d^2, dmax^2), d = 0..32
  static constexpr size_t SMEM = DATA_BYTES + ((META_BYTES + 15) & ~(size_t)15) + 2 * NS * 8 + LUT_BYTES + 16;
};

// x pass of one brick from the staged masks of bricks w .. w + 2R (64 B each; byte y + 8 z is the
// x-row (y, z)).  Lane: z = lane & 7, rows y0 = 2 (lane >> 3) and y0 + 1.  g1 is stored y-major.
// For dmax <= 32 (and R <= 4) a distance of 32 or more is already saturated, so each voxel needs
// only the 32 line bits on either side: two funnel shifts of 32-bit words and a count of leading
// zeros (left) and of trailing zeros (right).  Otherwise the 64-bit form covers the whole line.
template <int R>
__device__ __forceinline__ void x_compute_rows(const GridView& g, const uint32_t (&rows2)[2 * R + 1], int slot,
                                               uint32_t inf2, const uint16_t* lut);

template <int R>
__device__ __forceinline__ void x_compute(const GridView& g, const uint8_t* masks, int slot, uint32_t inf2,
                                          const uint16_t* lut) {
  constexpr int NBX = 2 * R + 1;
  const int lane = threadIdx.x & 31;
  const int z = lane & 7, y0 = (lane >> 3) * 2;
  uint32_t rows2[NBX];
#pragma unroll
  for (int b = 0; b < NBX; ++b) rows2[b] = *reinterpret_cast<const uint16_t*>(masks + b * 64 + y0 + 8 * z);
  x_compute_rows<R>(g, rows2, slot, inf2, lut);
}

// The x-line computation of one brick from the lane's two mask bytes of each brick of the window
// (rows2[b]: bits of x-rows y0 (low byte) and y0 + 1 (high byte) at z, brick bx - R + b).
template <int R>
__device__ __forceinline__ void x_compute_rows(const GridView& g, const uint32_t (&rows2)[2 * R + 1], int slot,
                                               uint32_t inf2, const uint16_t* lut) {
  constexpr int NBX = 2 * R + 1;
  const int lane = threadIdx.x & 31;
  const int z = lane & 7, y0 = (lane >> 3) * 2;
  bool fin = false;
  uint32_t w[2][4];
  bool done = false;
  if constexpr (R <= 4) {
    if (g.dmax <= 32) {
      // E[r][1 + k] holds line bits 32k .. 32k + 31; E[r][0] = 0 stands for positions -32 .. -1.
      // Byte b of the line is brick b's row: gathered with byte permutes (rows y0 and y0 + 1 are
      // the low and high bytes of rows2[b]).
      uint32_t E[2][5] = {{0u, 0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u, 0u}};
#pragma unroll
      for (int k = 1; k <= 3; ++k) {
        const int b0 = 4 * (k - 1);
        if (b0 < NBX) {
          const uint32_t a = rows2[b0], b = b0 + 1 < NBX ? rows2[b0 + 1] : 0u;
          const uint32_t c = b0 + 2 < NBX ? rows2[b0 + 2] : 0u, d = b0 + 3 < NBX ? rows2[b0 + 3] : 0u;
          const uint32_t t01 = __byte_perm(a, b, 0x5140), t23 = __byte_perm(c, d, 0x5140);
          E[0][k] = __byte_perm(t01, t23, 0x5410);
          E[1][k] = __byte_perm(t01, t23, 0x7632);
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if ((E[r][1] | E[r][2] | E[r][3]) == 0u) {
          w[r][0] = w[r][1] = w[r][2] = w[r][3] = inf2;
          continue;
        }
        uint32_t hv[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int P = 8 * R + x + 32;  // position in E
          const int s0 = P - 31;
          const uint32_t Lw = __funnelshift_r(E[r][s0 >> 5], E[r][(s0 >> 5) + 1], s0 & 31);  // bit 31 = P
          const uint32_t Rw = __funnelshift_r(E[r][P >> 5], E[r][(P >> 5) + 1], P & 31);      // bit 0 = P
          const int d = min(__clz(Lw), __clz(__brev(Rw)));  // 32 when the side is empty
          fin |= d < g.dmax;                                  // d^2 < dmax^2
          hv[x] = lut[d];                                     // fp16 bits of min(d^2, dmax^2)
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) w[r][q] = hv[2 * q] | (hv[2 * q + 1] << 16);
      }
      done = true;
    }
  }
  if (!done) {
    unsigned long long lo[2] = {0ull, 0ull}, hi[2] = {0ull, 0ull};
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
      const uint32_t two = rows2[b];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const unsigned long long byte = (two >> (8 * r)) & 0xFFu;
        if (b < 8)
          lo[r] |= byte << (8 * b);
        else
          hi[r] |= byte << (8 * (b - 8));
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if ((lo[r] | hi[r]) == 0ull) {
        w[r][0] = w[r][1] = w[r][2] = w[r][3] = inf2;
      } else {
        __half hv[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int p = 8 * R + x;  // position of voxel x in the line (8 <= p < 64 for 1 <= R <= 6)
          int best = g.INF;
          const unsigned long long L = lo[r] & ((2ull << p) - 1ull);
          if (L) {
            const int dl = p - (63 - __clzll((long long)L));
            best = min(best, dl * dl);
          }
          const unsigned long long Rm = (lo[r] >> p) | (hi[r] << (64 - p));
          if (Rm) {
            const int dr = __ffsll((long long)Rm) - 1;
            best = min(best, dr * dr);
          }
          fin |= best < g.INF;
          hv[x] = __int2half_rn(best);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) w[r][q] = h2u(__halves2half2(hv[2 * q], hv[2 * q + 1]));
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
    *reinterpret_cast<uint4*>(g.g1 + (size_t)slot * kBrickVox + (y0 + r) * 64 + z * 8) =
        make_uint4(w[r][0], w[r][1], w[r][2], w[r][3]);
  const unsigned anyfin = __any_sync(0xffffffffu, fin);
  if (lane == 0) set_flag_bit(g, slot, F_G1FIN, anyfin);
}

// y or z pass of one brick: the staged column holds planes along the pass axis, 32 words each
// (two voxels per word); lane (xpair, a) reads one word per plane.
//   AXIS 1: g1 (y-major) -> g2 (z-major) + F_G2FIN;   AXIS 2: g2 -> D + F_FINITE.
template <int R, int AXIS>
__device__ __forceinline__ void window_compute(const GridView& g, const uint32_t* col, const int* fin_flags, int slot,
                                               int w, bool prune, uint32_t inf2) {
  constexpr int W = 8 * R;
  const int lane = threadIdx.x & 31;
  const int xp = lane & 3, a = lane >> 2;
  const __half2 hinf2 = u2h(inf2);
  bool any_fin = !prune;
#pragma unroll
  for (int b = 0; b <= 2 * R; ++b) any_fin |= fin_flags[w + b] != 0;
  uint32_t out[8];
  if (any_fin) {
    // plane w * 8 of the stage is plane 0 of this output brick's window (output 0 minus W)
    window_min8<W>(col + a * 4 + xp + (size_t)w * 8 * 32, out, prune);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = inf2;
  }
  bool fin = false;
  if (AXIS == 1) {
    // g2, z-major: word z * 32 + y * 4 + xpair, here z = a and y = q
    uint32_t* dst = reinterpret_cast<uint32_t*>(g.g2 + (size_t)slot * kBrickVox) + a * 32 + xp;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      dst[q * 4] = out[q];
      fin |= !__hbge2(u2h(out[q]), hinf2);
    }
  } else {
    // D, z-major int32: pair index z * 32 + y * 4 + xpair, here y = a and z = q
    int2* dst = reinterpret_cast<int2*>(g.dist + (size_t)slot * kBrickVox) + a * 4 + xp;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const __half2 h = u2h(out[q]);
      const int lo = __half2int_rn(__low2half(h)), hi = __half2int_rn(__high2half(h));
      fin |= (lo < g.INF) | (hi < g.INF);
      dst[q * 32] = make_int2(lo, hi);
    }
  }
  const unsigned anyfin = __any_sync(0xffffffffu, fin);
  if (lane == 0) {
    const uint32_t bit = AXIS == 1 ? F_G2FIN : F_FINITE;
    set_flag_bit(g, slot, bit, anyfin);
  }
}

// One work item = a run of RUN bricks along AXIS.  Warp 0 produces: it reads the item's slot list
// (prefetched two items ahead, with the input flags one item ahead), fills absent bricks of the
// stage, and starts one bulk copy per present brick (64 B masks for x, 1 KB g1 / g2 for y / z).
// Warps 1..RUN consume: warp w computes output brick w of the item from the stage, then
// releases it.  Every wait is bounded; on a timeout the error word is set and the block drains.
// Resident blocks per SM the window passes ask the register allocator for (at most 80 registers
// for RUN 4, 72 for RUN 8): enough warps to keep the packed-min pipe busy.
__host__ __device__ constexpr int pass_min_blocks(int run, int axis) {
  return axis == 0 ? (run == 4 ? 10 : (run == 8 ? 7 : 3)) : (run == 4 ? 5 : (run == 8 ? 3 : 1));
}

template <int R, int RUN, int AXIS>
__global__ void __launch_bounds__(32 * (RUN + 1), pass_min_blocks(RUN, AXIS))
    k_pass(GridView g, const int32_t* __restrict__ islots, int max_items, bool prune) {
  pdl_enter();
  using S = ColShape<R, RUN, AXIS>;
  constexpr int NB = S::NB, NS = S::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* data = smem;
  int* meta = reinterpret_cast<int*>(smem + S::DATA_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::DATA_BYTES + ((S::META_BYTES + 15) & ~(size_t)15));
  uint64_t* empty = full + NS;
  uint16_t* lut = reinterpret_cast<uint16_t*>(empty + NS);
  const int nitems = min(g.items_ctr[AXIS], max_items);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const __half hinf = __int2half_rn(g.INF);
  const uint32_t inf2 = h2u(__halves2half2(hinf, hinf));
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RUN);
    }
  }
  if (AXIS == 0 && threadIdx.x <= 32) {
    const __half h = __int2half_rn(min((int)(threadIdx.x * threadIdx.x), g.INF));
    lut[threadIdx.x] = *reinterpret_cast<const uint16_t*>(&h);
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------- producer ----------------
    const void* src_base = AXIS == 0 ? (const void*)g.occ : (AXIS == 1 ? (const void*)g.g1 : (const void*)g.g2);
    const uint32_t in_fin = AXIS == 1 ? F_G1FIN : F_G2FIN;
    auto slot_of = [&](int item) -> int {
      return (item < nitems && lane < NB) ? islots[(size_t)item * kItemSlots + lane] : -1;
    };
    auto flag_of = [&](int slot) -> int { return (AXIS == 0 || slot < 0) ? 0 : ((g.bflags[slot] & in_fin) != 0); };
    int it = blockIdx.x;
    int sl_cur = slot_of(it), sl_nxt = slot_of(it + (int)gridDim.x);
    int fl_cur = flag_of(sl_cur);
    int k = 0;
    for (; it < nitems; it += gridDim.x, ++k) {
      const int sl_nn = slot_of(it + 2 * (int)gridDim.x);  // prefetch two items ahead
      const int fl_nxt = flag_of(sl_nxt);                  // and the next item's flags
      const int s = k % NS, u = k / NS;
      if (u > 0 && !mbar_wait_bounded(g, &empty[s], (u - 1) & 1)) break;
      if (lane < NB) {
        meta[s * S::META + lane] = sl_cur;
        meta[s * S::META + NB + lane] = fl_cur;
      }
      const unsigned present = __ballot_sync(0xffffffffu, lane < NB && sl_cur >= 0);
      unsigned absent = __ballot_sync(0xffffffffu, lane < NB && sl_cur < 0);
      uint4* stage = reinterpret_cast<uint4*>(data + (size_t)s * S::STAGE_BYTES);
      constexpr int U16 = S::UNIT / 16;  // 16-byte words per staged brick
      while (absent) {
        const int b = __ffs(absent) - 1;
        absent &= absent - 1;
        const uint32_t fill = AXIS == 0 ? 0u : inf2;
        for (int q = lane; q < U16; q += 32) stage[b * U16 + q] = make_uint4(fill, fill, fill, fill);
      }
      __syncwarp();
      if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[s], (uint32_t)__popc(present) * (uint32_t)S::UNIT);
      }
      __syncwarp();
      if ((present >> lane) & 1u)
        bulk_copy_g2s(data + (size_t)s * S::STAGE_BYTES + lane * S::UNIT,
                      reinterpret_cast<const unsigned char*>(src_base) + (size_t)sl_cur * S::UNIT, (uint32_t)S::UNIT,
                      &full[s]);
      sl_cur = sl_nxt;
      fl_cur = fl_nxt;
      sl_nxt = sl_nn;
    }
    // after a timeout, let copies already issued land before the block can exit
    if (it < nitems)
      for (int j = max(0, k - NS); j < k; ++j) mbar_wait_bounded(g, &full[j % NS], (j / NS) & 1);
    return;
  }

  // ---------------- consumers ----------------
  const int w = warp - 1;  // output brick of the item
  int k = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++k) {
    const int s = k % NS, u = k / NS;
    if (!mbar_wait_bounded(g, &full[s], u & 1)) break;
    const int* m = meta + s * S::META;
    const int slot = m[w + R];
    if (slot >= 0) {
      const unsigned char* stage = data + (size_t)s * S::STAGE_BYTES;
      if (AXIS == 0)
        x_compute<R>(g, stage + w * 64, slot, inf2, lut);
      else
        window_compute<R, AXIS>(g, reinterpret_cast<const uint32_t*>(stage), m + NB, slot, w, prune, inf2);
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
  }
}

// x pass with plain loads: one warp per output brick of the queued runs; each lane reads its two
// mask bytes of the 2R + 1 bricks of the window straight from global memory (the masks of
// neighbouring bricks are shared through L1 / L2) and writes its 32 bytes of g1.
template <int R>
__global__ void __launch_bounds__(256) k_x_direct(GridView g, const int32_t* __restrict__ islots, int max_items,
                                                  int run) {
  pdl_enter();
  constexpr int NBX = 2 * R + 1;
  const int nitems = min(g.items_ctr[0], max_items);
  const int lane = threadIdx.x & 31;
  const int z = lane & 7, y0 = (lane >> 3) * 2;
  const __half hinf = __int2half_rn(g.INF);
  const uint32_t inf2 = h2u(__halves2half2(hinf, hinf));
  const int64_t total = (int64_t)nitems * run;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned char* occ = reinterpret_cast<const unsigned char*>(g.occ);
  __shared__ uint16_t lut[33];
  if (threadIdx.x <= 32) {
    const __half h = __int2half_rn(min((int)(threadIdx.x * threadIdx.x), g.INF));
    lut[threadIdx.x] = *reinterpret_cast<const uint16_t*>(&h);
  }
  __syncthreads();
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    const int item = (int)(w / run), j = (int)(w % run);
    const int32_t* sl = islots + (size_t)item * kItemSlots + j;
    const int s = lane < NBX ? __ldg(sl + lane) : -1;
    const int slot = __shfl_sync(0xffffffffu, s, R);
    if (slot < 0) continue;  // warp-uniform
    uint32_t rows2[NBX];
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
      const int sb = __shfl_sync(0xffffffffu, s, b);
      rows2[b] = sb >= 0 ? (uint32_t)__ldg(reinterpret_cast<const uint16_t*>(occ + (size_t)sb * 64 + y0 + 8 * z)) : 0u;
    }
    x_compute_rows<R>(g, rows2, slot, inf2, lut);
  }
}

// ------------------------------------------------------------------------------------------------
// Lower-envelope kernels (any dmax up to 181; the only form above 45, variant 8 below it).
//
// Fields hold plain 16-bit integers (g1 y-major, g2 z-major, as in the windowed kernels).  A work
// item is a run of kEnvRun bricks along the pass axis (a node's length); each kernel finds the
// run's bricks and their R bricks of halo on each side through the node tables.
//   x: the distance to the nearest occupied voxel of an x-line, from the line's bits: within the
//      output brick's own byte with one count of leading / trailing zeros, beyond it by scanning
//      the neighbouring bricks' bytes outward until one holds a set bit (a warp per output brick,
//      a lane per two x-rows).
//   y, z: for one line f(0 .. n-1) along the axis (the run and its halo, n = 8 (kEnvRun + 2R)),
//      every output x needs min over q of (x - q)^2 + f(q), the lower envelope of the parabolas
//      rooted at (q, f(q)) evaluated at x (the separable exact transform of Felzenszwalb and
//      Huttenlocher, "Distance Transforms of Sampled Functions", 2012, restated here for integers
//      and a streaming deque).  A thread owns a line.  Input q enters as the parabola with
//      h = f(q) + q^2 (inputs at dmax^2 are left out: they cannot bring an output below dmax^2);
//      the back of the deque is dropped while it is nowhere strictly below both its predecessor and
//      the new parabola -- (h_q - h_b)(v_b - v_a) <= (h_b - h_a)(q - v_b), the intersection test
//      with the denominators multiplied out (no division, exact in int32).  Once q = x + W, output x
//      has seen every input within W (any farther one costs at least (W + 1)^2 >= dmax^2):
//      parabolas rooted more than W before x are dropped from the front, the front is dropped while
//      its successor is at least as low at x (h_b - h_a <= 2x (v_b - v_a)), and the front gives
//      min(dmax^2, h - 2xv + x^2).  Queries advance monotonically, so every parabola enters and
//      leaves once: O(1) amortised per voxel, independent of the window.  The deque holds at most
//      2W + 2 entries (a ring in the thread's local memory, one packed word h << 9 | v each).
// ------------------------------------------------------------------------------------------------
constexpr int kEnvRun = 16;
constexpr int kEnvThreads = 64;  // y, z: one line of an item per thread (8 x 8 lines)

__device__ __forceinline__ int occ_byte(const GridView& g, int slot, int row) {
  return slot >= 0 ? (int)reinterpret_cast<const uint8_t*>(g.occ)[(size_t)slot * 64 + row] : 0;
}

// x pass (lower envelope of a binary line = nearest set bit).  Block = 8 warps; per item the
// slots of the run and its halo along x are looked up once.
__global__ void __launch_bounds__(256) k_env_x(GridView g, const unsigned long long* __restrict__ items, int max_items) {
  __shared__ int slots[kEnvRun + 2 * 23];
  const int R = g.R, NB = kEnvRun + 2 * R, INF = g.INF, dmax = g.dmax;
  const int nitems = min(g.items_ctr[0], max_items);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx0, by, bz;
    unpack_brick(items[it], bx0, by, bz);
    __syncthreads();
    for (int i = threadIdx.x; i < NB; i += blockDim.x) slots[i] = find_brick(g, bx0 - R + i, by, bz);
    __syncthreads();
    for (int b = warp; b < kEnvRun; b += 8) {
      const int slot = slots[b + R];
      if (slot < 0) continue;  // warp-uniform
      bool fin = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = lane + 32 * h;  // y + 8 z: byte of the brick masks
        const int y = row & 7, z = row >> 3;
        const int own = occ_byte(g, slots[b + R], row);
        // distance from the brick's first voxel to the nearest set bit before it, and from its last
        // voxel to the nearest one after it (beyond dmax - 1 counts as none)
        int left = 1 << 20, right = 1 << 20;
        for (int j = 1; j <= R && 8 * j - 7 < dmax; ++j) {
          const int m = occ_byte(g, slots[b + R - j], row);
          if (m) {
            left = 8 * j - (31 - __clz(m));
            break;
          }
        }
        for (int j = 1; j <= R && 8 * j - 7 < dmax; ++j) {
          const int m = occ_byte(g, slots[b + R + j], row);
          if (m) {
            right = 8 * j - 7 + (__ffs(m) - 1);
            break;
          }
        }
        uint16_t v[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const int lm = own & ((2 << x) - 1), rm = own >> x;
          const int dl = lm ? x - (31 - __clz(lm)) : x + left;
          const int dr = rm ? __ffs(rm) - 1 : (7 - x) + right;
          const int d = min(dl, dr);
          const int val = d < dmax ? d * d : INF;
          fin |= val < INF;
          v[x] = (uint16_t)val;
        }
        // g1 is y-major: voxel x + 8 z + 64 y
        uint4 pk;
        pk.x = v[0] | ((uint32_t)v[1] << 16);
        pk.y = v[2] | ((uint32_t)v[3] << 16);
        pk.z = v[4] | ((uint32_t)v[5] << 16);
        pk.w = v[6] | ((uint32_t)v[7] << 16);
        *reinterpret_cast<uint4*>(g.g1 + (size_t)slot * kBrickVox + 64 * y + 8 * z) = pk;
      }
      const unsigned anyfin = __any_sync(0xffffffffu, fin);
      if (lane == 0) set_flag_bit(g, slot, F_G1FIN, anyfin);
    }
  }
}

// y (AXIS 1: g1 -> g2) or z (AXIS 2: g2 -> D) pass by the lower envelope.  Block = one item at a
// time, thread t = the line (t & 7, t >> 3) across the axis.  RING >= 2W + 2.
template <int AXIS, int RING>
__global__ void __launch_bounds__(kEnvThreads) k_env_yz(GridView g, const unsigned long long* __restrict__ items,
                                                        int max_items) {
  __shared__ int slots[kEnvRun + 2 * 23];  // stored bricks of the run and its halo (-1: none)
  __shared__ int inslot[kEnvRun + 2 * 23];  // the same, -1 also where the brick's input is all dmax^2
  __shared__ __align__(16) uint16_t tile[kBrickVox];  // y pass: one output brick, transposed to z-major
  const int R = g.R, W = 8 * R, NB = kEnvRun + 2 * R, n = 8 * NB, INF = g.INF;
  const int nitems = min(g.items_ctr[AXIS], max_items);
  const int t = threadIdx.x;
  const int c0 = t & 7, c1 = t >> 3;  // y pass: (x, z); z pass: (x, y)
  const uint16_t* __restrict__ src = AXIS == 1 ? g.g1 : g.g2;
  const uint32_t in_fin = AXIS == 1 ? F_G1FIN : F_G2FIN;
  int ring[RING];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    int bx, by, bz;
    unpack_brick(items[it], bx, by, bz);
    __syncthreads();  // the previous item's slots are no longer read
    for (int i = t; i < NB; i += blockDim.x) {
      const int s = AXIS == 1 ? find_brick(g, bx, by - R + i, bz) : find_brick(g, bx, by, bz - R + i);
      slots[i] = s;
      inslot[i] = (s >= 0 && (g.bflags[s] & in_fin)) ? s : -1;
    }
    __syncthreads();
    int head = 0, tail = 0, cnt = 0;
    bool fin = false;
    for (int q = 0; q < n; ++q) {
      const int sq = inslot[q >> 3];
      // input (c0, c1) at position q & 7 along the axis: g1 y-major x + 8z + 64y, g2 z-major x + 8y + 64z
      const int f = sq >= 0 ? (int)src[(size_t)sq * kBrickVox + 64 * (q & 7) + 8 * c1 + c0] : INF;
      if (f < INF) {
        const int hq = f + q * q;
        while (cnt >= 2) {
          const int ib = tail == 0 ? RING - 1 : tail - 1, ia = ib == 0 ? RING - 1 : ib - 1;
          const int b = ring[ib], a = ring[ia];
          const int vb = b & 511, hb = b >> 9, va = a & 511, ha = a >> 9;
          if ((hq - hb) * (vb - va) > (hb - ha) * (q - vb)) break;
          tail = ib;
          --cnt;
        }
        ring[tail] = (hq << 9) | q;
        tail = tail + 1 == RING ? 0 : tail + 1;
        ++cnt;
      }
      const int x = q - W;  // output position, once every input within W of it is in
      if (x < W) continue;  // block-uniform
      while (cnt > 0 && (ring[head] & 511) < x - W) {
        head = head + 1 == RING ? 0 : head + 1;
        --cnt;
      }
      while (cnt >= 2) {
        const int ib = head + 1 == RING ? 0 : head + 1;
        const int a = ring[head], b = ring[ib];
        if ((b >> 9) - (a >> 9) > 2 * x * ((b & 511) - (a & 511))) break;
        head = ib;
        --cnt;
      }
      int res = INF;
      if (cnt > 0) {
        const int a = ring[head];
        res = min(INF, (a >> 9) - 2 * x * (a & 511) + x * x);
      }
      fin |= res < INF;
      const int oslot = slots[x >> 3];  // block-uniform
      const int k = x & 7;
      if (AXIS == 1)
        tile[c0 + 8 * k + 64 * c1] = (uint16_t)res;  // g2 z-major: x + 8 y + 64 z
      else if (oslot >= 0)
        g.dist[(size_t)oslot * kBrickVox + 64 * k + 8 * c1 + c0] = res;  // D z-major: x + 8 y + 64 z
      if (k == 7) {  // block-uniform: the output brick is complete
        const int any = __syncthreads_or(fin);
        fin = false;
        if (oslot >= 0) {
          if (AXIS == 1)
            for (int i = t; i < kBrickVox / 8; i += blockDim.x)
              reinterpret_cast<uint4*>(g.g2 + (size_t)oslot * kBrickVox)[i] = reinterpret_cast<const uint4*>(tile)[i];
          if (t == 0) set_flag_bit(g, oslot, AXIS == 1 ? F_G2FIN : F_FINITE, any != 0);
        }
        if (AXIS == 1) __syncthreads();  // the tile is read before the next brick overwrites it
      }
    }
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

// Persistent launch of an envelope kernel: as many blocks as fit on the GPU at once (items are
// taken grid-stride; blocks beyond the queued count exit at once).
template <typename K>
cudaError_t launch_env_kernel(K kernel, int threads, const GridView& g, const unsigned long long* items,
                              cudaStream_t st) {
  if (g.item_cap <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = num_sms() * per_sm;
  if (grid > g.item_cap) grid = g.item_cap;
  VDB_LAUNCH(kernel, grid, threads, 0, st, g, items, g.item_cap);
  return cudaGetLastError();
}

// Envelope pass along `axis`; the deque ring is sized for the grid's window (2W + 2 entries).
cudaError_t launch_env(const GridView& g, int axis, const Items& it, cudaStream_t st) {
  if (axis == 0) return launch_env_kernel(k_env_x, 256, g, it.run[0], st);
  const int need = 2 * 8 * g.R + 2;
  if (axis == 1) {
    if (need <= 130) return launch_env_kernel(k_env_yz<1, 130>, kEnvThreads, g, it.run[1], st);
    if (need <= 258) return launch_env_kernel(k_env_yz<1, 258>, kEnvThreads, g, it.run[1], st);
    return launch_env_kernel(k_env_yz<1, 370>, kEnvThreads, g, it.run[1], st);
  }
  if (need <= 130) return launch_env_kernel(k_env_yz<2, 130>, kEnvThreads, g, it.run[2], st);
  if (need <= 258) return launch_env_kernel(k_env_yz<2, 258>, kEnvThreads, g, it.run[2], st);
  return launch_env_kernel(k_env_yz<2, 370>, kEnvThreads, g, it.run[2], st);
}

template <int R, int RUN, int AXIS>
cudaError_t pass_half(const GridView& g, const int32_t* islots, int max_items, cudaStream_t st, bool prune) {
  using S = ColShape<R, RUN, AXIS>;
  auto kernel = k_pass<R, RUN, AXIS>;
  if (max_items <= 0) return cudaSuccess;
  // attributes and resident blocks per SM, set up once per device (0: not yet)
  static int per_sm_dev[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int per_sm = dev >= 0 && dev < 64 ? per_sm_dev[dev] : 0;
  if (per_sm == 0) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, S::THREADS, S::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev >= 0 && dev < 64) per_sm_dev[dev] = per_sm;
  }
  int grid = num_sms() * per_sm;
  if (grid > max_items) grid = max_items;
  // the y and z passes follow the previous pass directly: their launch overlaps its tail
  if (AXIS > 0)
    VDB_LAUNCH_PDL(kernel, grid, S::THREADS, S::SMEM, st, g, islots, max_items, prune);
  else
    VDB_LAUNCH(kernel, grid, S::THREADS, S::SMEM, st, g, islots, max_items, prune);
  return cudaGetLastError();
}

template <int RUN, int AXIS>
cudaError_t pass_half_r(const GridView& g, const int32_t* islots, int max_items, cudaStream_t st, bool prune) {
  switch (g.R) {
    case 1: return pass_half<1, RUN, AXIS>(g, islots, max_items, st, prune);
    case 2: return pass_half<2, RUN, AXIS>(g, islots, max_items, st, prune);
    case 3: return pass_half<3, RUN, AXIS>(g, islots, max_items, st, prune);
    case 4: return pass_half<4, RUN, AXIS>(g, islots, max_items, st, prune);
    case 5: return pass_half<5, RUN, AXIS>(g, islots, max_items, st, prune);
    case 6: return pass_half<6, RUN, AXIS>(g, islots, max_items, st, prune);
  }
  return cudaErrorInvalidValue;
}

template <int AXIS>
cudaError_t pass_half_run(const GridView& g, int run, const int32_t* islots, int max_items, cudaStream_t st,
                          bool prune) {
  switch (run) {
    case 4: return pass_half_r<4, AXIS>(g, islots, max_items, st, prune);
    case 8: return pass_half_r<8, AXIS>(g, islots, max_items, st, prune);
    case 16: return pass_half_r<16, AXIS>(g, islots, max_items, st, prune);
  }
  return cudaErrorInvalidValue;
}

// Self-test of the bounded waits: one thread waits on a phase that never completes (which = 0: an
// mbarrier with no arrivals, the wait of the pass kernels) or looks up a node whose insertion was
// left pending (which = 1: the wait of node creation).  Each gives up after its poll limit, sets
// the error word and returns.
__global__ void k_wait_selftest(GridView g, int which) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  if (which == 0) {
    mbar_init(&bar, 1);
    mbar_wait_bounded(g, &bar, 0);
  } else {
    const unsigned long long key = 0;
    g.hslots[hash_key(key) & g.hmask] = (key << kIndexBits) | kPending;
    get_or_create_node(g, key);
  }
}

template <int R>
cudaError_t x_direct_r(const GridView& g, const int32_t* islots, int max_items, int run, cudaStream_t st) {
  auto kernel = k_x_direct<R>;
  if (max_items <= 0) return cudaSuccess;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  VDB_LAUNCH(kernel, num_sms() * per_sm, 256, 0, st, g, islots, max_items, run);
  return cudaGetLastError();
}

cudaError_t x_direct(const GridView& g, const int32_t* islots, int max_items, int run, cudaStream_t st) {
  switch (g.R) {
    case 1: return x_direct_r<1>(g, islots, max_items, run, st);
    case 2: return x_direct_r<2>(g, islots, max_items, run, st);
    case 3: return x_direct_r<3>(g, islots, max_items, run, st);
    case 4: return x_direct_r<4>(g, islots, max_items, run, st);
    case 5: return x_direct_r<5>(g, islots, max_items, run, st);
    case 6: return x_direct_r<6>(g, islots, max_items, run, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_wait_selftest(const GridView& g, int which, cudaStream_t st) {
  VDB_LAUNCH(k_wait_selftest, 1, 32, 0, st, g, which);
  return cudaGetLastError();
}

bool half_path(const GridView& g) { return g.half != 0; }

int effective_run(const GridView& g, const Tuning& t, int axis) { return half_path(g) ? t.run[axis] : kEnvRun; }

// The half kernels address bricks by pool slot (the slot lists hold local slot + slot_base):
// their view has the per-brick pointers moved back to the first slot of the pool.
GridView pool_view(const GridView& g) {
  GridView p = g;
  const size_t b = (size_t)g.slot_base;
  p.occ = g.occ - b * 8;
  p.g1 = g.g1 - b * kBrickVox;
  p.g2 = g.g2 - b * kBrickVox;
  p.dist = g.dist - b * kBrickVox;
  p.bcoord = g.bcoord - b;
  p.bflags = g.bflags - b;
  p.bepoch = g.bepoch - b;
  p.slot_base = 0;
  return p;
}

cudaError_t launch_pass(const GridView& g, const Tuning& t, int axis, const Items& it, cudaStream_t st) {
  const bool prune = (t.variant & 3) != 1;
  if (half_path(g)) {
    const GridView p = pool_view(g);
    if (axis == 0 && (t.variant & kVariantXDirect)) return x_direct(p, it.slots[0], g.item_cap, t.run[0], st);
    if (axis == 0) return pass_half_run<0>(p, t.run[0], it.slots[0], g.item_cap, st, prune);
    if (axis == 1) return pass_half_run<1>(p, t.run[1], it.slots[1], g.item_cap, st, prune);
    return pass_half_run<2>(p, t.run[2], it.slots[2], g.item_cap, st, prune);
  }
  // the envelope kernels find bricks through the grid's own tables (local slots)
  return launch_env(g, axis, it, st);
}

}  // namespace vdbedt
