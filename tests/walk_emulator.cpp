// Test infrastructure: a CPU emulation of the walk kernels' semantics on the
// programs the library builds and bakes (build_paths, bake_words of
// lpf_paths.cpp), so that -m "not gpu" tests can check the host side -- the
// prefix-tree program, its pieces and prologues, the skip words and the baked
// pixel pairs -- against the oracle without a GPU.
//
// A "warp" here is 32 translation rows x T words of 32 translations, as in
// the device kernels: a unit is one program piece on one such tile; masks are
// ANDed pixel by pixel, counts are added at emitting records, and the walk
// jumps to a record's skip target when no translation of the tile is left (at
// the end of an emitting or branching record, or after every 8 pixels inside
// a record).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_1601_04359_gb300/csrc/lpf_paths.hpp"

using namespace lpf;

namespace {

inline uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t s) {
  return (uint32_t)(((((uint64_t)hi) << 32) | lo) >> (s & 31u));
}

}  // namespace

// Walk every unit of `prog` over the packed layout of the kernels, adding to
// counts and stats.  rx: the program's column offsets lie in [-rx, rx]; ry:
// its row offsets in [-up, ry] (images) or [-ry, ry] (volumes).  Images: one
// slice, packed row y = image row (y - up) mod H.  Volumes: slices of
// Hs = 32 nb + 2 ry packed rows (image row (y'' - ry) mod H of slice z' mod D),
// D + rz slices; a translation row of slice z starts at packed row z Hs + y.
static int emulate_side(const Paths& p, const Program& prog, const uint8_t* img, int D, int H, int W, int rx,
                        int ry, int up, int T, bool volume, int64_t* counts, int64_t* stats,
                        const uint8_t* sel = nullptr) {
  const int rz = p.rz;
  const int nw = (W + 31) / 32, G = (nw + T - 1) / T, r32 = ((rx + 31) / 32) * 32;
  int S = G * T + ((r32 + rx) >> 5) + 1;
  if (!(S & 1)) ++S;
  const int nb = (H + 31) / 32;
  const int Hs = volume ? (32 * nb + 2 * ry + 3) & ~3 : 0;  // as the kernels: a multiple of 4 rows
  const int rows = volume ? (D + rz) * Hs : 32 * nb + ry + up;
  // packed rows: bit b of word k = pixel at column (32k + b - r32) mod W
  std::vector<uint32_t> packed((size_t)rows * S + 4, 0);
  for (int r = 0; r < rows; ++r) {
    const int zs = volume ? (r / Hs) % D : 0;
    const int yi = volume ? (((r % Hs) - ry) % H + H) % H : ((r - up) % H + H) % H;
    for (int k = 0; k < S; ++k) {
      uint32_t bits = 0;
      for (int b = 0; b < 32; ++b) {
        const int x = ((32 * k + b - r32) % W + W) % W;
        bits |= (uint32_t)(img[((size_t)zs * H + yi) * W + x] != 0) << b;
      }
      packed[(size_t)r * S + k] = bits;
    }
  }
  std::vector<uint32_t> w;
  std::vector<int64_t> piece;
  bake_words(p, prog, S, r32, w, piece, Hs, volume ? ry : up);
  const int64_t nf = p.n_full, base = p.base;
  int64_t walked = 0, skips = 0, pairs = 0;
  const int L = 32 * T;
  std::vector<uint32_t> valid(L), m1(L), m0(L), st1((kMaxStack + 1) * L), st0((kMaxStack + 1) * L);
  auto empty = [&]() {
    for (int i = 0; i < L; ++i)
      if (m1[i] | m0[i]) return false;
    return true;
  };
  for (int zs = 0; zs < (volume ? D : 1); ++zs)
  for (int band = 0; band < nb; ++band)
    for (size_t pi = 0; pi + 1 < piece.size(); ++pi)
      for (int g = 0; g < G; ++g) {
        for (int lane = 0; lane < 32; ++lane)
          for (int t = 0; t < T; ++t) {
            const int y = band * 32 + lane, j = g * T + t;
            uint32_t v = 0;
            if (y < H && j < nw) {
              const int rem = W - 32 * j;
              v = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
              if (sel)  // selected start translations only (Monte-Carlo variant)
                for (int b = 0; b < 32 && 32 * j + b < W; ++b)
                  if (!sel[(size_t)y * W + 32 * j + b]) v &= ~(1u << b);
            }
            valid[lane * T + t] = m1[lane * T + t] = m0[lane * T + t] = v;
          }
        // AND pixel `word` ((byte offset << 5) | shift) into the masks; a
        // pair reads the window of `word` with a second shift `shift2`.
        auto and_pixel = [&](uint32_t word, uint32_t shift) {
          for (int lane = 0; lane < 32; ++lane) {
            const uint32_t* lb = packed.data() + (size_t)(zs * Hs + band * 32 + lane) * S + g * T;
            const uint32_t* sa = lb + ((word >> 5) >> 2);  // byte offset -> word
            for (int t = 0; t < T; ++t) {
              const uint32_t a = funnel_r(sa[t], sa[t + 1], shift);
              m1[lane * T + t] &= a;
              m0[lane * T + t] &= ~a;
            }
          }
        };
        int64_t pc = piece[pi];  // in 16-byte groups
        const int64_t end = piece[pi + 1];
        while (pc < end) {
          const int64_t rec = pc;
          const uint32_t* hg = &w[4 * (size_t)pc];
          const uint32_t h = hg[0], vecw = hg[1], skip = hg[2], cnt = hg[3];
          const uint32_t n_pg = cnt & kCntMask, n_sg = (cnt >> kCntBits) & kCntMask, half = cnt >> (2 * kCntBits);
          if (h & kReset) { m1 = valid; m0 = valid; }
          if (h & kRestore) {
            const int l = (h >> kRlevelShift) & kLevelMask;
            for (int i = 0; i < L; ++i) { m1[i] = st1[l * L + i]; m0[i] = st0[l * L + i]; }
          }
          const int vec = (h & kEmit) ? (int)vecw : -1;
          const int n = (int)(h & kNpixMask);
          pairs += 2 * n_pg;
          bool dead = false;
          int64_t done = 0;
          const uint32_t* gp = hg + 4;
          for (uint32_t q = 0; q < n_pg && !dead; ++q, gp += 4) {
            and_pixel(gp[0], gp[0]);
            and_pixel(gp[0], gp[1]);
            and_pixel(gp[2], gp[2]);
            and_pixel(gp[2], gp[3]);
            done += 4;
            if ((q & 1) && skip && empty()) dead = true;
          }
          for (uint32_t q = 0; q < n_sg && !dead; ++q, gp += 4) {
            for (int k = 0; k < 4; ++k) and_pixel(gp[k], gp[k]);
            done += 4;
            if ((q & 1) && skip && empty()) dead = true;
          }
          if (!dead && half) {
            and_pixel(gp[0], gp[0]);
            and_pixel(gp[1], gp[1]);
            done += 2;
          }
          walked += std::min<int64_t>(done, n);
          pc = rec + 1 + n_pg + n_sg + half;
          if (dead) { pc = rec + skip; ++skips; continue; }
          if (h & (kEmit | kPush)) {
            if (skip && empty()) { pc = rec + skip; ++skips; continue; }
            if (vec >= 0) {
              int64_t c0 = 0, c1 = 0;
              for (int i = 0; i < L; ++i) { c0 += __builtin_popcount(m0[i]); c1 += __builtin_popcount(m1[i]); }
              counts[base + vec] += c0;
              counts[nf + base + vec] += c1;
            }
          }
          if (h & kPush) {
            const int l = (h >> kPlevelShift) & kLevelMask;
            for (int i = 0; i < L; ++i) { st1[l * L + i] = m1[i]; st0[l * L + i] = m0[i]; }
          }
        }
      }
  stats[0] += walked;
  stats[1] += prog.n_pixel_words * (int64_t)nb * G * (volume ? D : 1);
  stats[2] += skips;
  stats[3] += pairs;
  return 0;
}

static void mirror(const Paths& p, int64_t* counts) {
  const int64_t nf = p.n_full, base = p.base;
  for (int64_t j = base + 1; j < nf; ++j)
    for (int q = 0; q < 2; ++q) counts[q * nf + nf - 1 - j] = counts[q * nf + j];
}

// An image: the image's program on the image (column offsets up to rx, rows
// 0 .. min(rx, ry)) and the transpose's program on the transposed image
// (column offsets up to ry, rows -h .. h with h = min(rx, ry - 1)).
// sel != null: only the selected start translations count (sel[y][x]).
static int emulate_impl(const Paths& p, bool standard, const uint8_t* img, int H, int W, int T, int64_t* counts,
                        int64_t* stats, const uint8_t* sel = nullptr) {
  std::memset(counts, 0, sizeof(int64_t) * 2 * p.n_full);
  for (int k = 0; k < 4; ++k) stats[k] = 0;
  emulate_side(p, standard ? p.plain : p.tree, img, 1, H, W, p.rx, std::min(p.rx, p.ry), 0, T, false, counts,
               stats, sel);
  if (p.root_t >= 0) {
    // the transposed image; its translation (x', y') is the image's (y', x')
    std::vector<uint8_t> imgT((size_t)H * W), selT(sel ? (size_t)H * W : 0);
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        imgT[(size_t)x * H + y] = img[(size_t)y * W + x];
        if (sel) selT[(size_t)x * H + y] = sel[(size_t)y * W + x];
      }
    const int h = std::min(p.rx, p.ry - 1);
    emulate_side(p, standard ? p.plain_t : p.tree_t, imgT.data(), 1, W, H, p.ry, h, h, T, false, counts, stats,
                 sel ? selT.data() : nullptr);
  }
  mirror(p, counts);
  return 0;
}

// counts: int64 [2][n_full] (phase 0 first), stats: int64 [4] = {pixels
// walked, nominal pixels, skips taken, pairs baked}.  Returns 0 or -1.
extern "C" int emulate_walk(const uint8_t* img, int H, int W, int rx, int ry, int standard, int T,
                            int64_t* counts, int64_t* stats) {
  Paths p;
  std::string err;
  if (build_paths(rx, ry, 0, p, err)) return -1;
  return emulate_impl(p, standard != 0, img, H, W, T, counts, stats);
}

// The walk over selected start translations only (sel[y][x] != 0; the
// Monte-Carlo variant), tree program.
extern "C" int emulate_walk_sel(const uint8_t* img, const uint8_t* sel, int H, int W, int rx, int ry, int T,
                                int64_t* counts, int64_t* stats) {
  Paths p;
  std::string err;
  if (build_paths(rx, ry, 0, p, err)) return -1;
  return emulate_impl(p, false, img, H, W, T, counts, stats, sel);
}

// The same for a volume vol[z][y][x] (D x H x W) and window (rx, ry, rz).
extern "C" int emulate_walk3(const uint8_t* vol, int D, int H, int W, int rx, int ry, int rz, int T,
                             int64_t* counts, int64_t* stats) {
  Paths p;
  std::string err;
  if (build_paths_nd(rx, ry, rz, 3, 0, p, err)) return -1;
  std::memset(counts, 0, sizeof(int64_t) * 2 * p.n_full);
  for (int k = 0; k < 4; ++k) stats[k] = 0;
  emulate_side(p, p.tree, vol, D, H, W, rx, ry, 0, T, true, counts, stats);
  mirror(p, counts);
  return 0;
}
