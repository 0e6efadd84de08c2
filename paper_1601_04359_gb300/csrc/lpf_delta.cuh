// Device pieces of the swap-delta evaluation shared by lpf_delta_swap and the
// annealer (see lpf_delta.cu for the method).
//
// Extended cell: bytes, H + 2ry rows of W + 2rx pixels (row stride
// delta_row_stride), entry (ey, ex) = pixel ((ey - ry) mod H, (ex - rx) mod
// W), so a walk of any segment through a pixel never wraps.  A block stages
// it in shared memory with one bulk copy.
#pragma once
#include <cstdint>

#include "lpf_device.cuh"

namespace lpf {

constexpr uint8_t kMarkA = 4;  // phase 1 before the exchange, 0 after
constexpr uint8_t kMarkB = 3;  // phase 0 before the exchange, 1 after
constexpr int kDeltaThreads = 512;  // 16 warps: 3 blocks of 64 KB fill 48 of 64 warp slots
constexpr int kDeltaWarps = kDeltaThreads / 32;
constexpr int kWalkUnroll = 4;  // segment pixels loaded per round of a walk

struct DeltaArgs {
  int H, W, rx, ry, We, He;
  uint32_t ext_bytes;           // staged bytes (multiple of 16)
  const int32_t* dptr;          // CSR pointers of the canonical segments
  const int32_t* doff;          // per segment pixel: sy*We + sx
  const int32_t* chunk;         // vector chunk bounds
  int n_chunks;
  int64_t n_canon, n_full, base;
  const float* target;          // [2][n_full] or null
  const int64_t* counts;        // [2][n_full] or null
  int phase_mask;               // phases in the error: bit p = phase p (3 = both)
  int max_chunk_vecs;           // vectors in the largest chunk
  const uint8_t* sel_ext;       // selected start translations, extended layout (null: all)
  float inv_norm;               // descriptor = count * inv_norm (1/(H W), or 1/N selected)
  // Phase-0 counts (see delta_lookup_vectors): z[v][y][x] = number of phase-0
  // pixels of S(v) + (x, y), one byte per canonical vector and translation;
  // null: count changes by walks.  off16: the segments' pixel offsets
  // (sx, sy) as int16 pairs, CSR by dptr.
  uint8_t* z;
  const int16_t* off16;
  const int16_t* vec16;         // canonical vectors (dx, dy) as int16 pairs
};

// Where a walk finds the target and the current count of vector v for the
// error change: entry v - vbase of t[p] and c[p] (phase p).  Either the
// global arrays (vbase 0, pointers offset by the canonical base) or a
// block's copy of its chunk in shared memory (vbase = first vector).
struct DeltaTerms {
  const float* t[2];
  const long long* c[2];
  int vbase;
};

__device__ __forceinline__ DeltaTerms delta_terms_global(const DeltaArgs& g) {
  DeltaTerms d;
  d.t[0] = g.target ? g.target + g.base : nullptr;
  d.t[1] = g.target ? g.target + g.n_full + g.base : nullptr;
  d.c[0] = g.counts ? reinterpret_cast<const long long*>(g.counts) + g.base : nullptr;
  d.c[1] = g.counts ? reinterpret_cast<const long long*>(g.counts) + g.n_full + g.base : nullptr;
  d.vbase = 0;
  return d;
}

// Row stride (bytes) of the extended cell: at least W + 2 rx, and an odd
// number of 4-byte words, so that 32 lanes reading one byte each from 32
// consecutive rows (the walks of a near-vertical segment) hit 32 different
// shared-memory banks.  The padding columns are never read.
__host__ __device__ inline int delta_row_stride(int W, int rx) {
  int we = W + 2 * rx;
  we = (we + 3) & ~3;
  if ((we >> 2) % 2 == 0) we += 4;
  return we;
}

__device__ __forceinline__ int delta_ext_pos(int c, int W, int We, int rx, int ry) {
  const int cy = c / W, cx = c - cy * W;
  return (cy + ry) * We + (cx + rx);
}

// Write `val` at every periodic copy of pixel c inside the extended cell.
__device__ __forceinline__ void delta_mark(uint8_t* e, int c, uint8_t val, const DeltaArgs& g) {
  const int cy = c / g.W, cx = c - cy * g.W;
  for (int ey = (cy + g.ry) % g.H; ey < g.He; ey += g.H)
    for (int ex = (cx + g.rx) % g.W; ex < g.We; ex += g.W) e[ey * g.We + ex] = val;
}

// Stage the extended cell (bulk copy, bounded wait).  False on timeout.
__device__ __forceinline__ bool delta_stage(uint8_t* sm, const uint8_t* ext, uint32_t bytes, uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(sm, ext, bytes, bar);
  }
  __syncthreads();
  return mbar_wait(bar, 0);
}

// Count changes of the canonical vectors v0 <= v < v1 for the exchange of a
// (phase 1) and b (phase 0), both already marked in `sm`; the calling warp
// handles v = v0 + warp, v0 + warp + kDeltaWarps, ...  Lane 0 writes the
// changes (if dcounts) and returns the float32 error change of its vectors
// over the phases in g.phase_mask (if the target is given), accumulated in
// vector order.
__device__ __forceinline__ float delta_walk_vectors(const uint8_t* sm, const DeltaArgs& g, int a, int b, int v0,
                                                    int v1, int warp, int lane, int32_t* dcounts_k,
                                                    const DeltaTerms& dt) {
  float acc = 0.0f;
  const float invN = g.inv_norm;
  const int pa = delta_ext_pos(a, g.W, g.We, g.rx, g.ry);
  const int pb = delta_ext_pos(b, g.W, g.We, g.rx, g.ry);
  for (int v = v0 + warp; v < v1; v += kDeltaWarps) {
    const int o0 = __ldg(g.dptr + v);
    const int L1 = __ldg(g.dptr + v + 1) - o0;  // pixels of the segment
    int d0 = 0, d1 = 0;
    {
      const int tasks = 2 * L1;
      for (int t0 = 0; t0 < tasks; t0 += 32) {
        const int t = t0 + lane;
        const bool is_a = t < L1;
        const int i = is_a ? t : t - L1;
        bool alive = t < tasks;
        const int pos = (is_a ? pa : pb) - (alive ? __ldg(g.doff + o0 + i) : 0);
        if (alive && g.sel_ext && !__ldg(g.sel_ext + pos)) alive = false;  // start not among the sampled
        int q = -1;
        // kWalkUnroll pixels per round: their offsets (the same in every
        // lane) and then their bytes are loaded independently, so a round
        // costs about one load latency instead of one per pixel; pixels are
        // then judged in segment order, exactly as a pixel-by-pixel walk.
        for (int j0 = 0; j0 < L1; j0 += kWalkUnroll) {
          if (!__any_sync(0xffffffffu, alive)) break;
          int oj[kWalkUnroll], val[kWalkUnroll];
#pragma unroll
          for (int u = 0; u < kWalkUnroll; ++u) oj[u] = j0 + u < L1 ? __ldg(g.doff + o0 + j0 + u) : 0;
#pragma unroll
          for (int u = 0; u < kWalkUnroll; ++u) {
            const int j = j0 + u;
            val[u] = (alive && j < L1 && j != i) ? (int)sm[pos + oj[u]] : -1;
          }
#pragma unroll
          for (int u = 0; u < kWalkUnroll; ++u) {
            const int v = val[u];
            if (v < 0 || !alive) continue;  // beyond the segment, the anchor itself, or already ended
            if (q < 0) {
              if (v > 1) alive = false; else q = v;
            } else if (v != q) {
              alive = false;
            }
          }
        }
        if (alive) {
          // q < 0: the segment is the anchor alone (zero vector), uniform in
          // its phase before and in the other one after
          if (is_a) { if (q != 0) d1 -= 1; if (q != 1) d0 += 1; }
          else      { if (q != 0) d1 += 1; if (q != 1) d0 -= 1; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      }
    }
    if (lane == 0) {
      if (dcounts_k) {
        dcounts_k[v] = d0;
        dcounts_k[g.n_canon + v] = d1;
      }
      if (g.target && (d0 | d1)) {
        // (d - D/N)^2 - d^2 = (D/N) * (D/N - 2 d), with d = target - count/N
        const int iv = v - dt.vbase;
        if (d0 && (g.phase_mask & 1)) {
          const float dd = dt.t[0][iv] - (float)dt.c[0][iv] * invN;
          const float x = (float)d0 * invN;
          acc += x * (x - 2.0f * dd);
        }
        if (d1 && (g.phase_mask & 2)) {
          const float dd = dt.t[1][iv] - (float)dt.c[1][iv] * invN;
          const float x = (float)d1 * invN;
          acc += x * (x - 2.0f * dd);
        }
      }
    }
  }
  return acc;
}

// ---- count changes by lookups of per-translation phase-0 counts -----------
//
// With z_v(x) = number of phase-0 pixels of S(v) + x (L1 = |S(v)| pixels), a
// translation x through a (phase 1 before, 0 after) and not through b lies
// in phase 1 before iff z = 0 (lost by phase 1) and in phase 0 after iff
// z = L1 - 1 (gained by phase 0); through b (0 before, 1 after) and not
// through a, it lies in phase 1 after iff z = 1 (gained) and in phase 0
// before iff z = L1 (lost); a translation through both changes neither
// phase.  These are the same count changes as the walks' (the definition of
// Sec. 2.2 restricted to the translations the exchange touches), read from
// one byte per translation instead of walking the segment.

// Index of translation (x, y) in z_v: row-major for x-major vectors,
// column-major for y-major ones (dy > |dx|), so that the translations
// through one pixel along the segment are mostly consecutive bytes.
__device__ __forceinline__ int delta_z_index(const DeltaArgs& g, int dx, int dy, int x, int y) {
  return dy > (dx < 0 ? -dx : dx) ? x * g.H + y : y * g.W + x;
}

// Canonical vector of canonical index v.
__device__ __forceinline__ void delta_vector(const DeltaArgs& g, int v, int& dx, int& dy) {
  const short2 d = __ldg(reinterpret_cast<const short2*>(g.vec16) + v);
  dx = d.x;
  dy = d.y;
}

// True when pixel (qx, qy) lies on S(v) placed at translation (x, y), on the
// torus (the segment spans fewer than W columns and H rows, so at most one
// period of (qx, qy) is in its bounding box).
__device__ __forceinline__ bool delta_on_segment(const DeltaArgs& g, int o0, int dx, int dy, int x, int y, int qx,
                                                 int qy) {
  int uy = qy - y;                          // in (-H, H)
  if (uy < 0) uy += g.H;
  if (uy > dy) return false;                // canonical: 0 <= sy <= dy
  const int xlo = dx < 0 ? dx : 0, xhi = dx < 0 ? 0 : dx;
  int ux = qx - x - xlo;                    // in (-W, W + rx), rx < W
  if (ux < 0) ux += g.W;
  else if (ux >= g.W) ux -= g.W;
  ux += xlo;
  if (ux > xhi) return false;
  const int adx = dx < 0 ? -dx : dx;
  if (adx >= dy) {                          // x-major: pixel k at sx = sign(dx) k
    const int k = dx < 0 ? -ux : ux;
    return g.off16[2 * (o0 + k) + 1] == uy;
  }
  return g.off16[2 * (o0 + uy)] == ux;      // y-major: pixel k at sy = k
}

// Same contract as delta_walk_vectors (a phase 1, b phase 0; the warp's
// vectors v = v0 + warp, v0 + warp + kDeltaWarps, ...; lane 0 writes and
// returns), from the phase-0 counts g.z.
__device__ __forceinline__ float delta_lookup_vectors_strided(const DeltaArgs& g, int a, int b, int v0, int v1,
                                                              int vstep, int lane, int32_t* dcounts_k,
                                                              const DeltaTerms& dt);

__device__ __forceinline__ float delta_lookup_vectors(const DeltaArgs& g, int a, int b, int v0, int v1, int warp,
                                                      int lane, int32_t* dcounts_k, const DeltaTerms& dt) {
  return delta_lookup_vectors_strided(g, a, b, v0 + warp, v1, kDeltaWarps, lane, dcounts_k, dt);
}

// One warp over all vectors v0 <= v < v1 (in order); lane 0 returns.
__device__ __forceinline__ float delta_lookup_vectors_warp(const DeltaArgs& g, int a, int b, int v0, int v1,
                                                           int lane, int32_t* dcounts_k, const DeltaTerms& dt) {
  return delta_lookup_vectors_strided(g, a, b, v0, v1, 1, lane, dcounts_k, dt);
}

// Vectors v = v0, v0 + vstep, ... < v1.
__device__ __forceinline__ float delta_lookup_vectors_strided(const DeltaArgs& g, int a, int b, int v0, int v1,
                                                              int vstep, int lane, int32_t* dcounts_k,
                                                              const DeltaTerms& dt) {
  float acc = 0.0f;
  const float invN = g.inv_norm;
  const int W = g.W, H = g.H;
  const int ay = a / W, ax = a - ay * W, by = b / W, bx = b - by * W;
  const int64_t hw = (int64_t)H * W;
  for (int v = v0; v < v1; v += vstep) {
    const int o0 = __ldg(g.dptr + v);
    const int L1 = __ldg(g.dptr + v + 1) - o0;
    int dx, dy;
    delta_vector(g, v, dx, dy);
    const uint8_t* zv = g.z + (int64_t)v * hw;
    int d0 = 0, d1 = 0;
    // four lookups per lane in flight: offsets, then counts, then the tests
    for (int t0 = 0; t0 < 2 * L1; t0 += 128) {
      int xs[4], ys[4], zs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + 32 * u + lane;
        const int side = t >= L1;
        const int i = t < 2 * L1 ? (side ? t - L1 : t) : 0;
        const short2 s2 = reinterpret_cast<const short2*>(g.off16)[o0 + i];
        int x = (side ? bx : ax) - s2.x, y = (side ? by : ay) - s2.y;
        xs[u] = x < 0 ? x + W : (x >= W ? x - W : x);
        ys[u] = y < 0 ? y + H : (y >= H ? y - H : y);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)  // read at L2 (the annealer updates z with atomics, which bypass L1)
        zs[u] = t0 + 32 * u + lane < 2 * L1 ? __ldcg(zv + delta_z_index(g, dx, dy, xs[u], ys[u])) : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + 32 * u + lane;
        if (t >= 2 * L1) continue;
        const int x = xs[u], y = ys[u], z = zs[u];
        if (g.sel_ext && !g.sel_ext[(y + g.ry) * g.We + (x + g.rx)]) continue;  // start not sampled
        if (t < L1) {
          if (z == 0) d1 -= 1;
          if (z == L1 - 1 && !delta_on_segment(g, o0, dx, dy, x, y, bx, by)) d0 += 1;
        } else {
          if (z == L1) d0 -= 1;
          if (z == 1 && !delta_on_segment(g, o0, dx, dy, x, y, ax, ay)) d1 += 1;
        }
      }
    }
    // one reduction for both phases: |d0|, |d1| <= 2 L1 < 2^15 per vector
    int dp = d0 + d1 * 65536;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dp += __shfl_xor_sync(0xffffffffu, dp, o);
    d0 = (int)(short)(dp & 0xffff);
    d1 = (dp - d0) / 65536;
    if (lane == 0) {
      if (dcounts_k) {
        dcounts_k[v] = d0;
        dcounts_k[g.n_canon + v] = d1;
      }
      if (g.target && (d0 | d1)) {
        const int iv = v - dt.vbase;
        if (d0 && (g.phase_mask & 1)) {
          const float dd = dt.t[0][iv] - (float)dt.c[0][iv] * invN;
          const float x = (float)d0 * invN;
          acc += x * (x - 2.0f * dd);
        }
        if (d1 && (g.phase_mask & 2)) {
          const float dd = dt.t[1][iv] - (float)dt.c[1][iv] * invN;
          const float x = (float)d1 * invN;
          acc += x * (x - 2.0f * dd);
        }
      }
    }
  }
  return acc;
}

// After exchanging a (now phase 0) and b (now phase 1): z_v += 1 on the
// translations through a and -= 1 on those through b, for the warp's
// vectors of [v0, v1).  A translation through both gets both, which nets 0;
// the byte never wraps in between (it counts b, so it is >= 1 before the
// decrement, and < L1 before the increment), so the two updates may land
// in either order: one 32-bit atomic add per byte.
__device__ __forceinline__ void delta_lookup_update(const DeltaArgs& g, int a, int b, int v0, int v1, int warp,
                                                   int lane) {
  const int W = g.W, H = g.H;
  const int ay = a / W, ax = a - ay * W, by = b / W, bx = b - by * W;
  const int64_t hw = (int64_t)H * W;
  for (int v = v0 + warp; v < v1; v += kDeltaWarps) {
    const int o0 = __ldg(g.dptr + v);
    const int L1 = __ldg(g.dptr + v + 1) - o0;
    int dx, dy;
    delta_vector(g, v, dx, dy);
    uint8_t* zv = g.z + (int64_t)v * hw;
    for (int t = lane; t < 2 * L1; t += 32) {
      const int side = t >= L1;
      const int i = side ? t - L1 : t;
      int x = (side ? bx : ax) - g.off16[2 * (o0 + i)], y = (side ? by : ay) - g.off16[2 * (o0 + i) + 1];
      x = x < 0 ? x + W : (x >= W ? x - W : x);
      y = y < 0 ? y + H : (y >= H ? y - H : y);
      uint8_t* byte = zv + delta_z_index(g, dx, dy, x, y);
      unsigned int* word = reinterpret_cast<unsigned int*>(reinterpret_cast<uintptr_t>(byte) & ~uintptr_t(3));
      const unsigned int sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(byte) & 3);
      atomicAdd(word, side ? (0u - (1u << sh)) : (1u << sh));
    }
  }
}

// Write zero changes for vectors v0 <= v < v1 (identity candidates).
__device__ __forceinline__ void delta_zero_vectors(const DeltaArgs& g, int v0, int v1, int32_t* dcounts_k) {
  if (!dcounts_k) return;
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    dcounts_k[v] = 0;
    dcounts_k[g.n_canon + v] = 0;
  }
}

}  // namespace lpf
