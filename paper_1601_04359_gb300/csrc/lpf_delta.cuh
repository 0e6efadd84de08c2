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

// Write zero changes for vectors v0 <= v < v1 (identity candidates).
__device__ __forceinline__ void delta_zero_vectors(const DeltaArgs& g, int v0, int v1, int32_t* dcounts_k) {
  if (!dcounts_k) return;
  for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    dcounts_k[v] = 0;
    dcounts_k[g.n_canon + v] = 0;
  }
}

}  // namespace lpf
