// One warp's walk of one program piece over its translation words (the body
// shared by the single-image and the batched walk kernels).
//
// The program is a depth-first walk of the prefix tree of the canonical
// segments (see lpf_paths.hpp for the record format): every pixel ANDs one
// funnel-shifted image word into the phase-1 mask and its complement into the
// phase-0 mask (two pixels of a pair word share one staged word window); emit records count both masks (popc, warp sum, one atomic
// per phase); push/restore records keep branch masks on a small stack.
#pragma once
#include <cstdint>

#include "lpf_device.cuh"
#include "lpf_paths.hpp"

namespace lpf {

constexpr int kWalkStack = 24;

template <int T>
__device__ __forceinline__ void walk_and4(const uint32_t* lane_base, uint4 P, uint32_t (&m1)[T], uint32_t (&m0)[T]) {
  const uint32_t* sa = lane_word(lane_base, P.x);
  const uint32_t* sb = lane_word(lane_base, P.y);
  const uint32_t* sc = lane_word(lane_base, P.z);
  const uint32_t* sd = lane_word(lane_base, P.w);
  uint32_t wa[T + 1], wb[T + 1], wc[T + 1], wd[T + 1];
#pragma unroll
  for (int t = 0; t <= T; ++t) { wa[t] = sa[t]; wb[t] = sb[t]; wc[t] = sc[t]; wd[t] = sd[t]; }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], P.x);
    const uint32_t b = __funnelshift_r(wb[t], wb[t + 1], P.y);
    const uint32_t c = __funnelshift_r(wc[t], wc[t + 1], P.z);
    const uint32_t d = __funnelshift_r(wd[t], wd[t + 1], P.w);
    m1[t] = (m1[t] & a & b) & (c & d);
    m0[t] = (m0[t] & ~(a | b)) & ~(c | d);
  }
}

template <int T>
__device__ __forceinline__ void walk_and1(const uint32_t* lane_base, uint32_t p, uint32_t (&m1)[T], uint32_t (&m0)[T]) {
  const uint32_t* sa = lane_word(lane_base, p);
  uint32_t wa[T + 1];
#pragma unroll
  for (int t = 0; t <= T; ++t) wa[t] = sa[t];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const uint32_t a = __funnelshift_r(wa[t], wa[t + 1], p);
    m1[t] &= a;
    m0[t] &= ~a;
  }
}

// AND of the two pixels of each of 4 pair words (one staged word window per
// pair, two funnel shifts) into both phase masks.
template <int T>
__device__ __forceinline__ void walk_pair4(const uint32_t* lane_base, uint4 P, uint32_t (&m1)[T], uint32_t (&m0)[T]) {
  const uint32_t* sa = pair_word(lane_base, P.x);
  const uint32_t* sb = pair_word(lane_base, P.y);
  const uint32_t* sc = pair_word(lane_base, P.z);
  const uint32_t* sd = pair_word(lane_base, P.w);
  uint32_t wa[T + 1], wb[T + 1], wc[T + 1], wd[T + 1];
#pragma unroll
  for (int t = 0; t <= T; ++t) { wa[t] = sa[t]; wb[t] = sb[t]; wc[t] = sc[t]; wd[t] = sd[t]; }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const uint32_t a1 = __funnelshift_r(wa[t], wa[t + 1], P.x >> 5), a2 = __funnelshift_r(wa[t], wa[t + 1], P.x);
    const uint32_t b1 = __funnelshift_r(wb[t], wb[t + 1], P.y >> 5), b2 = __funnelshift_r(wb[t], wb[t + 1], P.y);
    const uint32_t c1 = __funnelshift_r(wc[t], wc[t + 1], P.z >> 5), c2 = __funnelshift_r(wc[t], wc[t + 1], P.z);
    const uint32_t d1 = __funnelshift_r(wd[t], wd[t + 1], P.w >> 5), d2 = __funnelshift_r(wd[t], wd[t + 1], P.w);
    m1[t] = (((m1[t] & a1 & a2) & b1 & b2) & c1 & c2) & d1 & d2;
    m0[t] = (((m0[t] & ~(a1 | a2)) & ~(b1 | b2)) & ~(c1 | c2)) & ~(d1 | d2);
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

// Walk program words [pc, end) for this warp's T words.  lane_base points at
// the lane's first staged word (row = lane's translation row); valid[t] masks
// the translations that exist (x < W, row < H).
template <int T>
__device__ __forceinline__ void walk_piece(const uint32_t* __restrict__ prog, int64_t pc, int64_t end,
                                           const uint32_t* lane_base, const uint32_t (&valid)[T], int lane,
                                           unsigned long long* __restrict__ counts, int64_t n_full,
                                           int64_t base) {
  uint32_t m1[T], m0[T];
  uint32_t st1[kWalkStack][T], st0[kWalkStack][T];
#pragma unroll
  for (int t = 0; t < T; ++t) { m1[t] = valid[t]; m0[t] = valid[t]; }
  while (pc < end) {
    const int64_t rec = pc;
    const uint32_t hdr = __ldg(prog + pc++);
    if (hdr & kReset) {
#pragma unroll
      for (int t = 0; t < T; ++t) { m1[t] = valid[t]; m0[t] = valid[t]; }
    }
    if (hdr & kRestore) {
      const int l = (hdr >> kRlevelShift) & kLevelMask;
#pragma unroll
      for (int t = 0; t < T; ++t) { m1[t] = st1[l][t]; m0[t] = st0[l][t]; }
    }
    int vec = -1;
    uint32_t skip = 0;
    if (hdr & kEmit) vec = (int)__ldg(prog + pc++);
    if (hdr & (kEmit | kPush)) skip = __ldg(prog + pc++);
    const int np = (int)__ldg(prog + pc++);  // pixel pairs sharing a staged word window
    pc = (pc + 3) & ~int64_t(3);
    const int ns = (int)(hdr & kNpixMask) - 2 * np;
    {  // np is a multiple of 4
      const uint4* q4 = reinterpret_cast<const uint4*>(prog + pc);
      for (int q = 0; q < (np >> 2); ++q) walk_pair4<T>(lane_base, __ldg(q4 + q), m1, m0);
      pc += np;
    }
    const uint4* q4 = reinterpret_cast<const uint4*>(prog + pc);
    const int n4 = ns >> 2;
    if (n4 > 0) {
      uint4 nxt = __ldg(q4);
      for (int q = 0; q < n4; ++q) {
        const uint4 cur = nxt;
        if (q + 1 < n4) nxt = __ldg(q4 + q + 1);
        walk_and4<T>(lane_base, cur, m1, m0);
      }
    }
    for (int i = n4 * 4; i < ns; ++i) walk_and1<T>(lane_base, __ldg(prog + pc + i), m1, m0);
    pc += ns;
    if (hdr & (kEmit | kPush)) {
      // Empty for the whole warp (one vote): so is every count below this node.
      uint32_t any = 0;
#pragma unroll
      for (int t = 0; t < T; ++t) any |= m1[t] | m0[t];
      if (!__any_sync(0xffffffffu, any != 0) && skip != 0) {
        pc = rec + skip;
        continue;
      }
      if (vec >= 0) {
        uint32_t c = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) c += (uint32_t)__popc(m1[t]) + ((uint32_t)__popc(m0[t]) << 16);
        c = warp_sum(c);
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
  }
}

}  // namespace lpf
