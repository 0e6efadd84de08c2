// One warp's walk of one program piece over its tile of translations (the
// body shared by the single-image and the batched walk kernels).
//
// The program is a depth-first walk of the prefix tree of the canonical
// segments, baked into 16-byte groups (see lpf_paths.hpp): a record is a
// header group, then groups of four pixels (two pairs of pixels that read the
// same staged word window, or four single pixels), then at most one group
// with two single pixels.  Every pixel ANDs one funnel-shifted image word
// into the phase-1 mask and its complement into the phase-0 mask; emitting
// records count both masks (popc, warp sum, one atomic per phase);
// push/restore records keep branch masks on a small per-thread stack.  After
// every 8 pixels inside a record and at the end of an emitting or branching
// record the warp votes: once no translation of its tile is left in either
// phase, every count of the subtree below is zero there too, and the warp
// jumps to the record's skip target (the zero-count skip of Sec. 3.2,
// applied to whole subtrees).
#pragma once
#include <cstdint>

#include "lpf_device.cuh"
#include "lpf_paths.hpp"

namespace lpf {

constexpr int kWalkStack = 24;

// The T + 1 staged words of a pixel word's window.
template <int T>
__device__ __forceinline__ void load_window(const uint32_t* lane_base, uint32_t pix, uint32_t (&w)[T + 1]) {
  const uint32_t* s = lane_word(lane_base, pix);
#pragma unroll
  for (int t = 0; t <= T; ++t) w[t] = s[t];
}

// Four single pixels (one group).
template <int T>
__device__ __forceinline__ void walk_singles4(const uint32_t* lane_base, uint4 P, uint32_t (&m1)[T],
                                              uint32_t (&m0)[T]) {
  if (T <= 4) {
    uint32_t wa[T + 1], wb[T + 1], wc[T + 1], wd[T + 1];
    load_window<T>(lane_base, P.x, wa);
    load_window<T>(lane_base, P.y, wb);
    load_window<T>(lane_base, P.z, wc);
    load_window<T>(lane_base, P.w, wd);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], P.x);
      const uint32_t b = __funnelshift_r(wb[t], wb[t + 1], P.y);
      const uint32_t c = __funnelshift_r(wc[t], wc[t + 1], P.z);
      const uint32_t d = __funnelshift_r(wd[t], wd[t + 1], P.w);
      m1[t] = (m1[t] & a & b) & c & d;
      m0[t] = (m0[t] & ~a & ~b) & ~c & ~d;
    }
  } else {  // two pixels at a time (registers)
    uint32_t wa[T + 1], wb[T + 1];
    load_window<T>(lane_base, P.x, wa);
    load_window<T>(lane_base, P.y, wb);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], P.x);
      const uint32_t b = __funnelshift_r(wb[t], wb[t + 1], P.y);
      m1[t] = m1[t] & a & b;
      m0[t] = m0[t] & ~a & ~b;
    }
    load_window<T>(lane_base, P.z, wa);
    load_window<T>(lane_base, P.w, wb);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], P.z);
      const uint32_t b = __funnelshift_r(wb[t], wb[t + 1], P.w);
      m1[t] = m1[t] & a & b;
      m0[t] = m0[t] & ~a & ~b;
    }
  }
}

// Two single pixels.
template <int T>
__device__ __forceinline__ void walk_singles2(const uint32_t* lane_base, uint32_t p, uint32_t q, uint32_t (&m1)[T],
                                              uint32_t (&m0)[T]) {
  uint32_t wa[T + 1], wb[T + 1];
  load_window<T>(lane_base, p, wa);
  load_window<T>(lane_base, q, wb);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], p);
    const uint32_t b = __funnelshift_r(wb[t], wb[t + 1], q);
    m1[t] = m1[t] & a & b;
    m0[t] = m0[t] & ~a & ~b;
  }
}

// Two pairs {window|shift1, shift2} (one group): one window per pair.
template <int T>
__device__ __forceinline__ void walk_pairs2(const uint32_t* lane_base, uint4 P, uint32_t (&m1)[T], uint32_t (&m0)[T]) {
  uint32_t wa[T + 1], wb[T + 1];
  load_window<T>(lane_base, P.x, wa);
  load_window<T>(lane_base, P.z, wb);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const uint32_t a1 = __funnelshift_r(wa[t], wa[t + 1], P.x), a2 = __funnelshift_r(wa[t], wa[t + 1], P.y);
    const uint32_t b1 = __funnelshift_r(wb[t], wb[t + 1], P.z), b2 = __funnelshift_r(wb[t], wb[t + 1], P.w);
    m1[t] = (m1[t] & a1 & a2) & b1 & b2;
    m0[t] = (m0[t] & ~a1 & ~a2) & ~b1 & ~b2;
  }
}

// True when no translation of the warp's tile is left in either phase (one vote).
template <int T>
__device__ __forceinline__ bool warp_empty(const uint32_t (&m1)[T], const uint32_t (&m0)[T]) {
  uint32_t any = 0;
#pragma unroll
  for (int t = 0; t < T; ++t) any |= m1[t] | m0[t];
  return !__any_sync(0xffffffffu, any != 0);
}

// Valid translations of a tile: word t of the lane's row holds translations
// x = 32 (j0 + t) + bit; those with x < W in a row y < H exist (and, with a
// selection, only the selected ones).
template <int T>
__device__ __forceinline__ void tile_valid(int y, int H, int W, int nw, int j0, const uint32_t* __restrict__ sel,
                                           uint32_t (&v)[T]) {
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int j = j0 + t;
    uint32_t m = 0;
    if (y < H && j < nw) {
      const int rem = W - 32 * j;
      m = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
      if (sel) m &= sel[(size_t)y * nw + j];
    }
    v[t] = m;
  }
}

// Walk program groups [pc, end) for this warp's tile.  lane_base points at
// the lane's first staged word (row = the lane's translation row).  Counts
// go to counts[base + vec] (phase 0) and counts[n_full + base + vec] (phase
// 1).  Returns the pixels this warp walked (for the work statistics).
// UNROLL4: pair groups four per loop iteration (less loop control, more
// code: the batched kernel, which inlines every T, keeps two).
template <int T, bool UNROLL4 = true>
__device__ __forceinline__ uint32_t walk_unit(const uint4* __restrict__ prog, uint32_t pc, uint32_t end,
                                              const uint32_t* lane_base, int y, int H, int W, int nw, int j0,
                                              const uint32_t* __restrict__ sel, int lane,
                                              unsigned long long* __restrict__ counts, int64_t n_full,
                                              int64_t base) {
  uint32_t m1[T], m0[T];
  uint32_t st1[kWalkStack][T], st0[kWalkStack][T];
  tile_valid<T>(y, H, W, nw, j0, sel, m1);
#pragma unroll
  for (int t = 0; t < T; ++t) m0[t] = m1[t];
  uint32_t walked = 0;
  uint4 hd = pc < end ? __ldg(prog + pc) : make_uint4(0u, 0u, 0u, 0u);
  while (pc < end) {
    const uint32_t rec = pc;
    const uint32_t hdr = hd.x, skip = hd.z, cnt = hd.w;
    const uint32_t n_pg = cnt & kCntMask, n_sg = (cnt >> kCntBits) & kCntMask, half = cnt >> (2 * kCntBits);
    const uint32_t next = rec + 1u + n_pg + n_sg + half;
    const int vec = (int)hd.y;
    hd = next < end ? __ldg(prog + next) : make_uint4(0u, 0u, 0u, 0u);  // fetched while this record runs
    if (hdr & kReset) {
      tile_valid<T>(y, H, W, nw, j0, sel, m1);
#pragma unroll
      for (int t = 0; t < T; ++t) m0[t] = m1[t];
    }
    if (hdr & kRestore) {
      const int l = (hdr >> kRlevelShift) & kLevelMask;
#pragma unroll
      for (int t = 0; t < T; ++t) { m1[t] = st1[l][t]; m0[t] = st0[l][t]; }
    }
    const uint32_t n = hdr & kNpixMask;
    walked += n;
    bool dead = false;
    const uint4* g = prog + rec + 1u;
    // four groups (16 pixels) per iteration, their program loads issued
    // together, a vote after every two (8 pixels); then pairs of groups
    uint32_t q = 0;
    for (; UNROLL4 && q + 4u <= n_pg; q += 4u) {
      const uint4 P0 = __ldg(g + q), P1 = __ldg(g + q + 1u), P2 = __ldg(g + q + 2u), P3 = __ldg(g + q + 3u);
      walk_pairs2<T>(lane_base, P0, m1, m0);
      walk_pairs2<T>(lane_base, P1, m1, m0);
      if (skip != 0u && warp_empty<T>(m1, m0)) {
        dead = true;
        walked -= n - 4u * (q + 2u);  // pixels not walked (pair groups hold four pixels of the record)
        break;
      }
      walk_pairs2<T>(lane_base, P2, m1, m0);
      walk_pairs2<T>(lane_base, P3, m1, m0);
      if (skip != 0u && warp_empty<T>(m1, m0)) {
        dead = true;
        walked -= n - 4u * (q + 4u);
        break;
      }
    }
    for (; !dead && q + 2u <= n_pg; q += 2u) {
      const uint4 P0 = __ldg(g + q), P1 = __ldg(g + q + 1u);
      walk_pairs2<T>(lane_base, P0, m1, m0);
      walk_pairs2<T>(lane_base, P1, m1, m0);
      if (skip != 0u && warp_empty<T>(m1, m0)) {
        dead = true;
        walked -= n - 4u * (q + 2u);
        break;
      }
    }
    if (!dead && q < n_pg) walk_pairs2<T>(lane_base, __ldg(g + q), m1, m0);
    if (!dead) {
      g += n_pg;
      for (q = 0; q + 2u <= n_sg; q += 2u) {
        const uint4 P0 = __ldg(g + q), P1 = __ldg(g + q + 1u);
        walk_singles4<T>(lane_base, P0, m1, m0);
        walk_singles4<T>(lane_base, P1, m1, m0);
        if (skip != 0u && warp_empty<T>(m1, m0)) {
          dead = true;
          const uint32_t done = 4u * (n_pg + q + 2u);
          walked -= n > done ? n - done : 0u;
          break;
        }
      }
      if (!dead) {
        if (q < n_sg) walk_singles4<T>(lane_base, __ldg(g + q), m1, m0);
        if (half) {
          const uint4 P = __ldg(g + n_sg);
          walk_singles2<T>(lane_base, P.x, P.y, m1, m0);
        }
      }
    }
    if (dead) {
      pc = rec + skip;
      hd = pc < end ? __ldg(prog + pc) : make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    if (hdr & (kEmit | kPush)) {
      // Empty for the whole warp (one vote): so is every count below this node.
      if (skip != 0u && warp_empty<T>(m1, m0)) {
        pc = rec + skip;
        hd = pc < end ? __ldg(prog + pc) : make_uint4(0u, 0u, 0u, 0u);
        continue;
      }
      if (hdr & kEmit) {
        uint32_t c = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) c += (uint32_t)__popc(m1[t]) + ((uint32_t)__popc(m0[t]) << 16);
        c = __reduce_add_sync(0xffffffffu, c);  // one warp-reduce instruction
        if (lane == 0) {
          const uint32_t c1 = c & 0xffffu, c0 = c >> 16;
          if (c0) atomicAdd(counts + base + vec, (unsigned long long)c0);
          if (c1) atomicAdd(counts + n_full + base + vec, (unsigned long long)c1);
        }
      }
    }
    if (hdr & kPush) {
      const int l = (hdr >> kPlevelShift) & kLevelMask;
#pragma unroll
      for (int t = 0; t < T; ++t) { st1[l][t] = m1[t]; st0[l][t] = m0[t]; }
    }
    pc = next;
  }
  return walked;
}

}  // namespace lpf
