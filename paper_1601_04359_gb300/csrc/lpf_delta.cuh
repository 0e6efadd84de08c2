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
  int max_chunk_entries;        // segment pixels of the largest chunk
  const uint8_t* sel_ext;       // selected start translations, extended layout (null: all)
  float inv_norm;               // descriptor = count * inv_norm (1/(H W), or 1/N selected)
  // Phase-0 counts (see delta_lookup_vectors_strided): byte
  // v H W + delta_z_index(v, x, y) of z = number of phase-0 pixels of
  // S(v) + (x, y), one byte per canonical vector and translation; null:
  // count changes by walks.  off16: the segments' pixel offsets
  // (sx, sy) as int16 pairs, CSR by dptr.
  uint8_t* z;
  const int16_t* off16;
  const int16_t* vec16;         // canonical vectors (dx, dy) as int16 pairs
  const int32_t* shear;         // their delta_shear, or null: z unsheared
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

// Layout of z_v.  The translations whose segment contains one pixel q are
// q - S(v), a digital line along v; z_v is stored sheared along v so that
// such a line is a run of consecutive bytes in one or two rows (a few
// 32-byte sectors per warp instead of one per pixel for diagonal vectors).
// x-major v (|dx| >= dy): translation (x, y) is at row y - sh(x) (mod H),
// column x, rows of W bytes; y-major v (dy > |dx|): at column x - sh(y)
// (mod W), row y, columns of H bytes; sh(t) = floor(t m / 2^16) with
// m = delta_shear(dx, dy), about t dy/dx (x-major) or t dx/dy (y-major).
// For a fixed column (row) the shear is a rotation, so every layout is a
// permutation of the translations; any m would be correct, this one makes
// the lines short.  |sh(t)| < the sheared extent's period along t.
constexpr int kZMaxSide = 32767;  // cells wider or higher than this use walks
__host__ __device__ inline int delta_shear(int dx, int dy) {
  const int adx = dx < 0 ? -dx : dx;
  if (dy > adx) return (int)(((long long)dx * 65536) / dy);
  return adx ? (int)(((long long)dy * 65536) / dx) : 0;
}

// floor(t m / 2^16); t < 2^15 and |m| <= 2^16 (cells on the lookup path
// are narrower and lower than 2^15), so the product fits 32 bits.
__device__ __forceinline__ int delta_shift(int t, int m) { return (t * m) >> 16; }

// t reduced into [0, n).  On a square cell |shear| < n, so t lies in
// (-n, 2n) and one wrap does; otherwise a full modulo.
__device__ __forceinline__ int delta_wrap(const DeltaArgs& g, int t, int n) {
  if (g.H == g.W) return t < 0 ? t + n : (t >= n ? t - n : t);
  return ((t % n) + n) % n;
}

// Index of translation (x, y) in z_v (m = delta_shear of v, or 0 for the
// unsheared layout: rows of W bytes for x-major vectors, columns of H bytes
// for y-major ones).
__device__ __forceinline__ int delta_z_index(const DeltaArgs& g, int dx, int dy, int m, int x, int y) {
  const bool ymajor = dy > (dx < 0 ? -dx : dx);
  if (m == 0) return ymajor ? x * g.H + y : y * g.W + x;
  if (ymajor) return delta_wrap(g, x - delta_shift(y, m), g.W) * g.H + y;
  return delta_wrap(g, y - delta_shift(x, m), g.H) * g.W + x;
}

// Translation (x, y) stored at index p of z_v: the inverse of delta_z_index.
__device__ __forceinline__ void delta_z_translation(const DeltaArgs& g, int dx, int dy, int m, int p, int& x,
                                                    int& y) {
  if (dy > (dx < 0 ? -dx : dx)) {
    const int c = p / g.H;
    y = p - c * g.H;
    x = m == 0 ? c : delta_wrap(g, c + delta_shift(y, m), g.W);
  } else {
    const int r = p / g.W;
    x = p - r * g.W;
    y = m == 0 ? r : delta_wrap(g, r + delta_shift(x, m), g.H);
  }
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
// vectors v = v0, v0 + vstep, ...; lane 0 writes and returns), from the
// phase-0 counts g.z in the unsheared layout (g.shear null).
__device__ __forceinline__ float delta_lookup_vectors_strided(const DeltaArgs& g, int a, int b, int v0, int v1,
                                                              int vstep, int lane, int32_t* dcounts_k,
                                                              const DeltaTerms& dt);

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
      for (int u = 0; u < 4; ++u)  // read at L2 (the annealer updates z in place)
        zs[u] = t0 + 32 * u + lane < 2 * L1 ? __ldcg(zv + delta_z_index(g, dx, dy, 0, xs[u], ys[u])) : -1;
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

// A block's vector chunk for the block-wide lookups of the persistent
// annealer.  The segment pixels of the chunk's vectors v0 <= v < v0 + nv are
// the contiguous entries o_base + [0, pre[nv]) of off16, copied to off;
// vector v0 + i owns entries [pre[i], pre[i + 1]).  d ([2][mv]) and term
// ([mv]) are the block's scratch for count changes and error terms.  All
// arrays are in shared memory.
struct ChunkTables {
  const int32_t* pre;   // [nv + 1] entry offsets
  const short2* vec;    // [nv] the chunk's canonical vectors (dx, dy)
  const int32_t* shear; // [nv] their delta_shear
  const short2* off;    // [pre[nv]] the chunk's segment pixels (sx, sy)
  const uint16_t* vid;  // [pre[nv]] the chunk-relative vector of every entry
  int32_t* d;           // [2][mv] count changes (phase 0, phase 1)
  float* term;          // [mv] error terms
  int nv, mv;
};

// Entries each thread takes per round of the block-wide lookups.
constexpr int kChunkUnroll = 4;

// The chunk-relative vector owning entry e: the largest i with pre[i] <= e
// (the tables builder's search; the kernels read ct.vid).
__device__ __forceinline__ int chunk_vector_of(const int32_t* pre, int nv, int e) {
  int lo = 0, hi = nv - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The pixels of an exchange, split into coordinates once.
struct PixelPair {
  int ax, ay, bx, by;
};

// delta_on_segment for chunk vector i, reading its pixels from the chunk's
// copy in shared memory.
__device__ __forceinline__ bool chunk_on_segment(const DeltaArgs& g, const ChunkTables& ct, int i, int dx, int dy,
                                                 int x, int y, int qx, int qy) {
  int uy = qy - y;
  if (uy < 0) uy += g.H;
  if (uy > dy) return false;
  const int xlo = dx < 0 ? dx : 0, xhi = dx < 0 ? 0 : dx;
  int ux = qx - x - xlo;
  if (ux < 0) ux += g.W;
  else if (ux >= g.W) ux -= g.W;
  ux += xlo;
  if (ux > xhi) return false;
  const short2* o = ct.off + ct.pre[i];
  const int adx = dx < 0 ? -dx : dx;
  if (adx >= dy) return o[dx < 0 ? -ux : ux].y == uy;  // x-major: pixel k at sx = sign(dx) k
  return o[uy].x == ux;                                // y-major: pixel k at sy = k
}

// Translation of chunk entry j for the exchange pixel (qx, qy): the start x
// of the segment whose pixel j is q, wrapped onto the torus, and the byte of
// z holding its phase-0 count (z has fewer than 2^31 bytes on the lookup
// path).
__device__ __forceinline__ void chunk_entry(const DeltaArgs& g, const ChunkTables& ct, int v0, int j, int qx, int qy,
                                            int& i, int& x, int& y, uint32_t& zi) {
  i = ct.vid[j];
  const short2 s2 = ct.off[j];
  x = qx - s2.x;
  y = qy - s2.y;
  x = x < 0 ? x + g.W : (x >= g.W ? x - g.W : x);
  y = y < 0 ? y + g.H : (y >= g.H ? y - g.H : y);
  const short2 dv = ct.vec[i];
  zi = (uint32_t)(v0 + i) * (uint32_t)(g.H * g.W) + (uint32_t)delta_z_index(g, dv.x, dv.y, ct.shear[i], x, y);
}

// Count changes and error change of the chunk's vectors for the exchange of
// a (phase 1) and b (phase 0), from the phase-0 counts z, with the chunk's
// 2 (L + 1) lookups per vector spread evenly over all threads of the block:
// entry e < E looks at the translation through a of pixel e, entry E + e at
// the one through b; kChunkUnroll lookups per thread in flight.  The tests
// are those of delta_lookup_vectors_strided.  When the block has at most
// kChunkUnroll entries per thread, *held receives the thread's counts as
// read (one byte each) and held_zi their offsets in z, for
// delta_chunk_apply_held; else *held is 0.  Every thread calls it; thread 0
// returns the chunk's error change, summed over the vectors in a fixed
// order.
__device__ __forceinline__ float delta_chunk_lookup(const DeltaArgs& g, const PixelPair& q, int v0,
                                                    const ChunkTables& ct, int32_t* dcounts_k,
                                                    const DeltaTerms& dt, uint32_t* held,
                                                    uint32_t (&held_zi)[kChunkUnroll]) {
  const int E = ct.pre[ct.nv];
  for (int i = threadIdx.x; i < ct.nv; i += blockDim.x) {
    ct.d[i] = 0;
    ct.d[ct.mv + i] = 0;
  }
  __syncthreads();
  const int ax = q.ax, ay = q.ay, bx = q.bx, by = q.by;
  const int nthr = blockDim.x;
  uint32_t h = 0;
  for (int e0 = 0; e0 < 2 * E; e0 += kChunkUnroll * nthr) {
    int vi[kChunkUnroll], xs[kChunkUnroll], ys[kChunkUnroll], zs[kChunkUnroll];
    uint32_t zi[kChunkUnroll];
#pragma unroll
    for (int u = 0; u < kChunkUnroll; ++u) {
      const int e = e0 + u * nthr + (int)threadIdx.x;
      vi[u] = -1;
      if (e < 2 * E) {
        const bool side = e >= E;
        chunk_entry(g, ct, v0, side ? e - E : e, side ? bx : ax, side ? by : ay, vi[u], xs[u], ys[u], zi[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kChunkUnroll; ++u) {  // read at L2 (other threads of the block update z)
      zs[u] = vi[u] >= 0 ? (int)__ldcg(g.z + zi[u]) : 0;
      held_zi[u] = zi[u];
    }
#pragma unroll
    for (int u = 0; u < kChunkUnroll; ++u) {
      h |= (uint32_t)zs[u] << (8 * u);
      if (vi[u] < 0) continue;
      const int e = e0 + u * nthr + (int)threadIdx.x;
      const int i = vi[u], x = xs[u], y = ys[u], z = zs[u];
      if (g.sel_ext && !g.sel_ext[(y + g.ry) * g.We + (x + g.rx)]) continue;  // start not sampled
      const int L1 = ct.pre[i + 1] - ct.pre[i];
      const short2 dv = ct.vec[i];
      if (e < E) {
        if (z == 0) atomicAdd(ct.d + ct.mv + i, -1);
        if (z == L1 - 1 && !chunk_on_segment(g, ct, i, dv.x, dv.y, x, y, bx, by)) atomicAdd(ct.d + i, 1);
      } else {
        if (z == L1) atomicAdd(ct.d + i, -1);
        if (z == 1 && !chunk_on_segment(g, ct, i, dv.x, dv.y, x, y, ax, ay)) atomicAdd(ct.d + ct.mv + i, 1);
      }
    }
  }
  *held = 2 * E <= kChunkUnroll * nthr ? h : 0u;
  __syncthreads();
  const float invN = g.inv_norm;
  for (int i = threadIdx.x; i < ct.nv; i += blockDim.x) {
    const int d0 = ct.d[i], d1 = ct.d[ct.mv + i];
    const int v = v0 + i;
    if (dcounts_k) {
      dcounts_k[v] = d0;
      dcounts_k[g.n_canon + v] = d1;
    }
    float acc = 0.0f;
    if (g.target && (d0 | d1)) {
      const int iv = v - dt.vbase;
      if (d0 && (g.phase_mask & 1)) {
        const float dd = dt.t[0][iv] - (float)dt.c[0][iv] * invN;
        const float xx = (float)d0 * invN;
        acc += xx * (xx - 2.0f * dd);
      }
      if (d1 && (g.phase_mask & 2)) {
        const float dd = dt.t[1][iv] - (float)dt.c[1][iv] * invN;
        const float xx = (float)d1 * invN;
        acc += xx * (xx - 2.0f * dd);
      }
    }
    ct.term[i] = acc;
  }
  __syncthreads();
  float sum = 0.0f;
  if (threadIdx.x < 32) {  // lane-strided sums in vector order, then a fixed shuffle tree
    for (int i = threadIdx.x; i < ct.nv; i += 32) sum += ct.term[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  return sum;
}

// Whether some translation of chunk vector i has both exchanged pixels on
// its segment, for a torus displacement (ddx, ddy) = b - a taken in
// [-W/2, W/2) x [-H/2, H/2).  Every pixel (sx, sy) of S(v) lies within a/2
// of the line along v (|sy dx - sx dy| <= a/2, a = max(|dx|, dy): the
// rounding of Sec. 2.2's segments), so a difference of two of its pixels
// lies within a of it and inside the segment's box.  When the box is less
// than half the cell on both axes only that representative of the
// displacement can fit, and the test is exact enough to rule pairs out;
// otherwise it answers "maybe".
__device__ __forceinline__ bool chunk_maybe_both(const DeltaArgs& g, int dx, int dy, int ddx, int ddy) {
  const int adx = dx < 0 ? -dx : dx;
  if (2 * adx >= g.W || 2 * dy >= g.H) return true;
  if ((ddx < 0 ? -ddx : ddx) > adx || (ddy < 0 ? -ddy : ddy) > dy) return false;
  const int cross = ddy * dx - ddx * dy;
  return (cross < 0 ? -cross : cross) <= (adx > dy ? adx : dy);
}

// After exchanging a (now phase 0) and b (now phase 1): z_v += 1 on the
// translations through a and -= 1 on those through b, for the chunk's
// vectors, with the counts delta_chunk_lookup read for this same exchange
// and their offsets, held by each thread (the block had at most
// kChunkUnroll entries per thread): plain stores at L2 -- the block owns
// these bytes.  A
// translation through both pixels keeps its count (its two entries are
// one byte, which neither stores); within one side a vector's translations
// are distinct, so no two threads store the same byte.  Every thread calls
// it with the same pixels as that lookup.
__device__ __forceinline__ void delta_chunk_apply_held(const DeltaArgs& g, const PixelPair& q, int v0,
                                                       const ChunkTables& ct, uint32_t held,
                                                       const uint32_t (&held_zi)[kChunkUnroll]) {
  const int E = ct.pre[ct.nv];
  const int nthr = blockDim.x;
  int ddx = q.bx - q.ax, ddy = q.by - q.ay;
  if (2 * ddx >= g.W) ddx -= g.W;
  else if (2 * ddx < -g.W) ddx += g.W;
  if (2 * ddy >= g.H) ddy -= g.H;
  else if (2 * ddy < -g.H) ddy += g.H;
#pragma unroll
  for (int u = 0; u < kChunkUnroll; ++u) {
    const int e = u * nthr + (int)threadIdx.x;
    if (e >= 2 * E) continue;
    const bool side = e >= E;
    const int j = side ? e - E : e;
    const short2 dv = ct.vec[ct.vid[j]];
    if (chunk_maybe_both(g, dv.x, dv.y, ddx, ddy)) {  // rare: check the other pixel on the segment
      int i, x, y;
      uint32_t zi;
      chunk_entry(g, ct, v0, j, side ? q.bx : q.ax, side ? q.by : q.ay, i, x, y, zi);
      if (chunk_on_segment(g, ct, i, dv.x, dv.y, x, y, side ? q.ax : q.bx, side ? q.ay : q.by)) continue;
    }
    const uint32_t z = (held >> (8 * u)) & 0xffu;
    __stcg(g.z + held_zi[u], (uint8_t)(side ? z - 1u : z + 1u));
  }
}

// The same update without held counts: each byte is loaded and stored at
// L2, first every translation through a, then (after a block barrier) every
// one through b, so that a translation through both gets both changes in
// turn.  Every thread calls it.
__device__ __forceinline__ void delta_chunk_update(const DeltaArgs& g, const PixelPair& q, int v0,
                                                   const ChunkTables& ct) {
  const int E = ct.pre[ct.nv];
  const int nthr = blockDim.x;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const int qx = side ? q.bx : q.ax, qy = side ? q.by : q.ay;
    for (int j0 = 0; j0 < E; j0 += kChunkUnroll * nthr) {
      uint32_t zi[kChunkUnroll], zz[kChunkUnroll];
      bool ok[kChunkUnroll];
#pragma unroll
      for (int u = 0; u < kChunkUnroll; ++u) {
        const int j = j0 + u * nthr + (int)threadIdx.x;
        ok[u] = j < E;
        zi[u] = 0;
        if (ok[u]) {
          int i, x, y;
          chunk_entry(g, ct, v0, j, qx, qy, i, x, y, zi[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kChunkUnroll; ++u) zz[u] = ok[u] ? (uint32_t)__ldcg(g.z + zi[u]) : 0u;
#pragma unroll
      for (int u = 0; u < kChunkUnroll; ++u)
        if (ok[u]) __stcg(g.z + zi[u], (uint8_t)(side ? zz[u] - 1u : zz[u] + 1u));
    }
    __syncthreads();
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
