// Full lineal path function of a periodic two-phase image (Sec. 2.2, Alg. 1
// and Alg. 2 of Sec. 3.1, prefix sharing after Sec. 3.2), bit-parallel.
//
// Layout.  Phase-1 pixels are bit-packed along rows (bit = 1 for phase 1),
// each row periodically extended so that any column offset in [-rx, rx] is a
// plain funnel shift of two adjacent words, and the rows periodically
// extended downwards by ry so that canonical row offsets (0 <= sy <= ry) never
// wrap.  A 32-bit word of a mask holds 32 consecutive translations x of one
// row; one funnel-shifted image word serves both phases (the phase-0 mask
// ANDs its complement).
//
// Work split.  A tile is 32 translation rows (lane = row, so the 32 lanes of
// a warp read 32 different rows: an odd row stride in words puts them in 32
// different shared-memory banks) by T words of translations.  A block stages
// the image rows of a band group (BB bands of 32 rows, all words of the row)
// in shared memory with one bulk copy; its warps then take units, one piece
// of the evaluation program on one tile, from the band group's counter.  The
// program is a depth-first walk of a prefix tree of canonical segments: each
// tree node ANDs one shifted image word (two nodes of a pair share the staged
// words), a node that ends a canonical vector is counted (popc + warp sum +
// one atomic per phase), masks of branching nodes are kept on a per-thread
// stack, and a subtree whose count is zero for the whole tile is skipped.
// Images have two sides: the tree of the x-major vectors over the image and
// the tree of the y-major vectors, transposed, over the transposed image.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "lpf_device.cuh"
#include "lpf_state.hpp"
#include "lpf_walk.cuh"

namespace lpf {

constexpr int kDevStack = kWalkStack;  // deepest prefix-tree stack the kernels hold
constexpr int kMaxSmem = 227 * 1024;
// Control words of a walk: [0] status flags, [2..3] pixel words walked
// (uint64), [kCtlUnits + bg] the unit counter of band group bg.
constexpr int kCtlExecuted = 2;
// Bits of the status word ctl[0]: a bounded wait gave up (1), an index out of
// range (2, swap deltas), a pixel other than 0 or 1 in checked mode (8).
constexpr int kStatusTimeout = 1;
constexpr int kStatusPixel = 8;
constexpr int kCtlUnits = 4;
constexpr int kMaxBandGroups = 8192;  // images: ceil(H / 32) <= 256; volumes: D * ceil(H / (32 BB))
constexpr int kCtlWords = kCtlUnits + kMaxBandGroups;

int layout_side(int H, int W, int rx, int ry, int T, int BB, Geometry& g, int up) {
  g.H = H; g.W = W; g.rx = rx; g.ry = ry; g.up = up;
  g.nw = (W + 31) / 32;
  g.T = T;
  g.G = (g.nw + T - 1) / T;
  g.nbands = (H + 31) / 32;
  g.BB = std::max(1, std::min(BB, g.nbands));
  g.nbg = (g.nbands + g.BB - 1) / g.BB;
  g.r32 = ((rx + 31) / 32) * 32;
  const int nwp = g.G * T;
  g.S = nwp + ((g.r32 + rx) >> 5) + 1;
  if ((g.S & 1) == 0) g.S += 1;
  g.rows = 32 * g.BB * g.nbg + ry + up;
  const size_t band = (size_t)(32 * g.BB + ry + up) * g.S * 4;
  g.band_bytes = (uint32_t)((band + 15) & ~size_t(15));
  g.packed_words = (size_t)g.rows * g.S + 4;
  g.D = 1;
  g.rz = 0;
  g.slice_rows = 0;
  g.nbg_s = g.nbg;
  if (band > (size_t)kMaxSmem - 64) return LPF_EUNSUPPORTED;
  return LPF_OK;
}

int make_geometry(int H, int W, int rx, int ry, int T, int BB, Geometry& g) {
  const int nw = (W + 31) / 32;
  if (T <= 0) T = nw >= 6 ? 8 : (nw >= 3 ? 4 : (nw >= 2 ? 2 : 1));
  while ((nw + T - 1) / T > 16 && T < 8) T *= 2;  // at most 16 warps per band
  const int G = (nw + T - 1) / T;
  const int nbands = (H + 31) / 32;
  if (BB <= 0) BB = std::max(1, std::min(4, 8 / G));
  BB = std::max(1, std::min(BB, nbands));
  while (BB > 1 && G * BB > 16) --BB;              // at most 512 threads per block
  return layout_side(H, W, rx, ry, T, BB, g);
}

int make_sides(const Paths& paths, int H, int W, int T, int BB, Sides& s) {
  const int rx = paths.rx, ry = paths.ry;
  int rc = make_geometry(H, W, rx, std::min(rx, ry), T, BB, s.g[0]);
  if (rc) return rc;
  s.n = paths.root_t >= 0 ? 2 : 1;
  s.off1 = (s.g[0].packed_words + 3) & ~size_t(3);
  s.packed_words = s.g[0].packed_words;
  s.band_bytes = s.g[0].band_bytes;
  s.nbg = s.g[0].nbg;
  int tiles = s.g[0].G * s.g[0].BB;
  if (s.n == 2) {
    const int h = std::min(rx, ry - 1);  // transposed segments: row offsets -h .. h
    rc = layout_side(W, H, ry, h, s.g[0].T, s.g[0].BB, s.g[1], h);
    if (rc) return rc;
    s.packed_words = s.off1 + s.g[1].packed_words;
    s.band_bytes = std::max(s.band_bytes, s.g[1].band_bytes);
    s.nbg += s.g[1].nbg;
    tiles = std::max(tiles, s.g[1].G * s.g[1].BB);
  }
  s.threads = 32 * std::min(16, tiles);
  if (s.nbg > kMaxBandGroups) return LPF_EUNSUPPORTED;
  return LPF_OK;
}

// Volume layout: packed row (z' * slice_rows + y'') holds image row
// (y'' - ry) mod H of slice z' mod D, z' < D + rz; a block of band group
// (z, b) stages rows z * slice_rows + 32 BB b onwards: its 32 BB
// translation rows, ry above and below them, and the rz following slices.
int make_geometry3(int D, int H, int W, int rx, int ry, int rz, int T, int BB, Geometry& g) {
  int rc = make_geometry(H, W, rx, ry, T, BB, g);
  if (rc && rc != LPF_EUNSUPPORTED) return rc;
  g.D = D;
  g.rz = rz;
  g.nbg_s = g.nbg;
  // A band group's bulk copy starts at row z * slice_rows + 32 BB b, which
  // must be a 16-byte boundary (cp.async.bulk): S is odd, so slice_rows is a
  // multiple of 4 (the extra rows hold the periodic continuation).
  g.slice_rows = (32 * g.BB * g.nbg_s + 2 * ry + 3) & ~3;
  g.nbg = D * g.nbg_s;
  g.rows = (D + rz) * g.slice_rows;
  const size_t band = (size_t)(rz * g.slice_rows + 32 * g.BB + 2 * ry) * g.S * 4;
  g.band_bytes = (uint32_t)((band + 15) & ~size_t(15));
  g.packed_words = (size_t)g.rows * g.S + 4;
  if (band > (size_t)kMaxSmem - 64 || g.nbg > kMaxBandGroups) return LPF_EUNSUPPORTED;
  if (((size_t)g.slice_rows * g.S) % 4 != 0 || ((size_t)32 * g.BB * g.S) % 4 != 0) return LPF_EUNSUPPORTED;
  return LPF_OK;
}

// ---------------------------------------------------------------------------
// Kernels

// One side's packed rows: packed[y][k] bit b is the pixel at row
// (y - up) mod Ho, column (32k + b - r32) mod Wo of the side's image, whose
// pixel (r, c) is img[r rs + c cs] (side 0: the image, rs = W, cs = 1,
// up = 0; side 1: its transpose, rs = 1, cs = W, up = its halo above).  Any
// nonzero byte is phase 1.
struct PackSide {
  uint32_t* packed;
  int Ho, Wo, r32, S, rows, rs, cs, up;
};

// Packs side blockIdx.y.  Side 1 runs over its words column by column, so
// that the threads of a warp read consecutive bytes of an image row.  Side
// 0's blocks also zero the walk's n_zero64 counts and n_zero32 control words
// (which would otherwise take two more launches).  pix_flag != null (checked
// mode): a byte other than 0 or 1 sets kStatusPixel in *pix_flag.
__global__ void pack_rows_kernel(const uint8_t* __restrict__ img, PackSide s0, PackSide s1,
                                 unsigned long long* __restrict__ zero64, int64_t n_zero64, int* __restrict__ zero32,
                                 int n_zero32, int* __restrict__ pix_flag) {
  const bool side1 = blockIdx.y != 0;
  const PackSide ps = side1 ? s1 : s0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (!side1) {
    for (int64_t i = i0; i < n_zero64; i += stride) zero64[i] = 0ull;
    for (int64_t i = i0; i < n_zero32; i += stride) zero32[i] = 0;
  }
  const int64_t total = (int64_t)ps.rows * ps.S;
  uint32_t high = 0;  // OR of the bytes' bits above bit 0
  for (int64_t i = i0; i < total; i += stride) {
    int y, k;
    if (side1) { k = (int)(i / ps.rows); y = (int)(i % ps.rows); }
    else { y = (int)(i / ps.S); k = (int)(i % ps.S); }
    const uint8_t* row = img + (int64_t)((y + ps.Ho - ps.up % ps.Ho) % ps.Ho) * ps.rs;
    int x = (32 * k - ps.r32) % ps.Wo;
    if (x < 0) x += ps.Wo;
    uint32_t bits = 0;
#pragma unroll 4
    for (int b = 0; b < 32; ++b) {
      const uint32_t v = row[(int64_t)x * ps.cs];
      bits |= (uint32_t)(v != 0) << b;
      high |= v >> 1;
      if (++x == ps.Wo) x = 0;
    }
    ps.packed[(int64_t)y * ps.S + k] = bits;
  }
  if (pix_flag && high) atomicOr(pix_flag, kStatusPixel);
}

// Volume rows: packed[(z' * slice_rows + y'') * S + k] bit b = voxel at
// slice z' mod D, row (y'' - ry) mod H, column (32k + b - r32) mod W; also
// zeroes the counts and control words as pack_rows_kernel does.
__global__ void pack_vol_kernel(const uint8_t* __restrict__ vol, int D, int H, int W, int ry, int r32, int S,
                                int slice_rows, int rows, uint32_t* __restrict__ packed,
                                unsigned long long* __restrict__ zero64, int64_t n_zero64, int* __restrict__ zero32,
                                int n_zero32, int* __restrict__ pix_flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = i0; i < n_zero64; i += stride) zero64[i] = 0ull;
  for (int64_t i = i0; i < n_zero32; i += stride) zero32[i] = 0;
  const int64_t total = (int64_t)rows * S;
  uint32_t high = 0;
  for (int64_t i = i0; i < total; i += stride) {
    const int64_t r = i / S;
    const int k = (int)(i % S);
    const int zp = (int)(r / slice_rows), yp = (int)(r % slice_rows);
    int y = (yp - ry) % H;
    if (y < 0) y += H;
    const uint8_t* row = vol + ((int64_t)(zp % D) * H + y) * W;
    int x = (32 * k - r32) % W;
    if (x < 0) x += W;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
      const uint32_t v = row[x];
      bits |= (uint32_t)(v != 0) << b;
      high |= v >> 1;
      if (++x == W) x = 0;
    }
    packed[i] = bits;
  }
  if (pix_flag && high) atomicOr(pix_flag, kStatusPixel);
}

// counts[p][n_full-1-i] = counts[p][i] for the canonical entries i > base
// (Eq. (symmetry): the segment of -v is the segment of v).
__global__ void mirror_kernel(unsigned long long* __restrict__ counts, int64_t n_full, int64_t base) {
  const int64_t n = n_full - base - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n, j = base + 1 + i % n;
    counts[p * n_full + (n_full - 1 - j)] = counts[p * n_full + j];
  }
}

// sel_bits[y][j]: bit b set when translation (32j + b, y) of a side is
// selected; the side's translation (x, y) is sel[y rs + x cs] (side 0: rs =
// W, cs = 1; side 1, whose translation (x', y') is the image's (y', x'):
// rs = 1, cs = W).
__global__ void pack_sel_kernel(const uint8_t* __restrict__ sel, int Ho, int Wo, int nw, int rs, int cs,
                                uint32_t* __restrict__ bits) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ho * nw; i += gridDim.x * blockDim.x) {
    const int y = i / nw, j = i - y * nw;
    uint32_t v = 0;
    for (int b = 0; b < 32 && 32 * j + b < Wo; ++b)
      v |= (uint32_t)(sel[(size_t)y * rs + (size_t)(32 * j + b) * cs] != 0) << b;
    bits[i] = v;
  }
}

// One side of a walk (the image or its transpose; volumes have one side):
// its packed rows, translation selection, size, layout and its pieces of the
// program.
struct WalkSide {
  const uint32_t* packed;
  const uint32_t* sel;  // packed translation selection, or null
  int H, W, S, nw, G, BB;
  int nbg, nbg_s, slice_rows;
  int piece0, n_pieces;
  uint32_t band_bytes;
};

// The units of band group lbg of side sd, pulled from its counter ctr until
// none is left: unit u is the side's program piece u / n_tiles on tile
// u % n_tiles (tile = one band and one group of T words, i.e. 32 rows x 32T
// translations).  Returns the pixel words this warp ANDed.
template <int T>
__device__ __forceinline__ unsigned long long walk_band(const WalkSide& sd, int lbg, int* ctr, const uint32_t* sm,
                                                        int lane, const uint4* __restrict__ prog,
                                                        const uint32_t* __restrict__ piece,
                                                        unsigned long long* __restrict__ counts, int64_t n_full,
                                                        int64_t base) {
  const int n_tiles = sd.G * sd.BB;
  const int units = n_tiles * sd.n_pieces;
  unsigned long long executed = 0;
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(ctr, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= units) break;
    const int tile = u % n_tiles, pi = sd.piece0 + u / n_tiles;
    const int bl = tile / sd.G, grp = tile - bl * sd.G;
    const uint32_t* lane_base = sm + (bl * 32 + lane) * sd.S + grp * T;
    const int y = ((lbg % sd.nbg_s) * sd.BB + bl) * 32 + lane;  // translation row within the slice
    executed += walk_unit<T>(prog, piece[pi], piece[pi + 1], lane_base, y, sd.H, sd.W, sd.nw, grp * T, sd.sel, lane,
                             counts, n_full, base);
  }
  return executed;
}

// Persistent walk kernel.  A block stages the packed rows of one band group
// (BB bands of 32 translation rows, plus the halo rows) and its warps pull
// work units from that band group's counter in global memory (walk_band).
// Band groups are numbered side 0 first, then side 1.  Warps never wait for
// one another inside a band group, so warps whose tiles skip zero-count
// subtrees (and finish early) simply take more units.  A block starts on
// band group blockIdx.x mod n_bg and, once that counter is exhausted, moves
// on to the next band group that still has units (one bulk copy and one
// block barrier per move).  The launch bounds cap a thread at 64 registers
// (two 512-thread blocks per SM), which keeps 32 warps resident per SM to
// hide the latency of the shared-memory word loads.
template <int T>
__global__ void __launch_bounds__(512, 2) walk_kernel(WalkSide s0, WalkSide s1, const uint4* __restrict__ prog,
                                                  const uint32_t* __restrict__ piece,
                                                  unsigned long long* __restrict__ counts, int64_t n_full,
                                                  int64_t base, int* __restrict__ ctl, uint32_t extra_tx,
                                                  uint32_t wait_rounds) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort, s_done;
  const int lane = threadIdx.x & 31;
  const int n_bg = s0.nbg + s1.nbg;
  int* unit_ctr = ctl + kCtlUnits;
  if (threadIdx.x == 0) { mbar_init(&bar, 1); s_abort = 0; }
  __syncthreads();
  uint32_t parity = 0;
  bool copy_pending = false;
  unsigned long long executed = 0;  // pixel words this warp ANDs

  for (int k = 0; k < n_bg; ++k) {
    const int bg = (int)((blockIdx.x + (unsigned)k) % (unsigned)n_bg);
    const bool side1 = bg >= s0.nbg;
    const int lbg = side1 ? bg - s0.nbg : bg;
    if (threadIdx.x == 0) {
      const int units = side1 ? s1.G * s1.BB * s1.n_pieces : s0.G * s0.BB * s0.n_pieces;
      s_done = *reinterpret_cast<volatile int*>(unit_ctr + bg) >= units;
    }
    __syncthreads();
    if (s_done) {
      __syncthreads();  // s_done is rewritten next round
      continue;
    }
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const uint32_t bytes = side1 ? s1.band_bytes : s0.band_bytes;
      // (extra_tx > 0 only in the failure-detection self-test: bytes no copy delivers)
      mbar_expect_tx(&bar, bytes + extra_tx);
      // band group lbg = slice lbg / nbg_s (volumes; images have one slice), band lbg % nbg_s
      const int nbg_s = side1 ? s1.nbg_s : s0.nbg_s, BB = side1 ? s1.BB : s0.BB;
      const size_t row0 = (size_t)(lbg / nbg_s) * (side1 ? s1.slice_rows : s0.slice_rows) +
                          (size_t)(lbg % nbg_s) * 32 * BB;
      const uint32_t* src = side1 ? s1.packed + row0 * s1.S : s0.packed + row0 * s0.S;
      bulk_g2s(sm, src, bytes, &bar);
    }
    copy_pending = true;
    if (mbar_wait(&bar, parity, wait_rounds)) copy_pending = false;
    else s_abort = 1;
    parity ^= 1u;
    __syncthreads();
    if (s_abort) break;
    if (side1) executed += walk_band<T>(s1, lbg, unit_ctr + bg, sm, lane, prog, piece, counts, n_full, base);
    else executed += walk_band<T>(s0, lbg, unit_ctr + bg, sm, lane, prog, piece, counts, n_full, base);
    __syncthreads();  // every warp is done with the staged band before it may be replaced
  }
  if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(ctl + kCtlExecuted), executed);
  if (s_abort) {
    atomicOr(ctl, kStatusTimeout);
    if (copy_pending) (void)mbar_wait(&bar, parity ^ 1u, wait_rounds);  // let an outstanding copy land
  }
}

// ---------------------------------------------------------------------------
// Host side

thread_local char g_last_error[256] = "";

int set_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return LPF_OK;
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LPF_ENOMEM : LPF_ECUDA;
}

static int cuda_status(cudaError_t e) { return set_cuda_error(e); }

int ensure_device(lpf_paths* p, size_t packed_words) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (p->device < 0) {
    p->device = dev;
  } else if (p->device != dev) {
    return LPF_EINVAL;  // handle is bound to another device
  }
  if (!p->d_status) {
    if ((e = cudaMalloc(&p->d_status, kCtlWords * sizeof(int))) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemset(p->d_status, 0, kCtlWords * sizeof(int))) != cudaSuccess) return set_cuda_error(e);
  }
  if (packed_words > p->packed_cap) {
    if (p->d_packed) {
      cudaDeviceSynchronize();
      cudaFree(p->d_packed);
      p->d_packed = nullptr;
      p->packed_cap = 0;
    }
    if ((e = cudaMalloc(&p->d_packed, packed_words * 4)) != cudaSuccess) return set_cuda_error(e);
    p->packed_cap = packed_words;
  }
  return LPF_OK;
}

int bake(lpf_paths* p, const Program& prog0, const Geometry& g0, const Program* prog1, const Geometry* g1,
         Baked& b) {
  const int S1 = prog1 ? g1->S : -1, r32_1 = prog1 ? g1->r32 : -1;
  if (b.d_words && b.W == g0.W && b.S == g0.S && b.r32 == g0.r32 && b.slice_rows == g0.slice_rows && b.S1 == S1 &&
      b.r32_1 == r32_1) {
    b.T = g0.T;
    b.BB = g0.BB;
    return LPF_OK;
  }
  if (b.d_words) {
    cudaDeviceSynchronize();
    cudaFree(b.d_words);
    cudaFree(b.d_piece);
    b.d_words = nullptr;
    b.d_piece = nullptr;
  }
  std::vector<uint32_t> out, out1;
  std::vector<int64_t> piece, piece1;
  // a pixel (sx, sy) of a translation on staged row `lane` reads row
  // lane + sy + up (sy >= -up); volumes: a voxel (sx, sy, sz) reads row
  // lane + sz * slice_rows + sy + ry (sy may be negative in 3D)
  bake_words(p->host, prog0, g0.S, g0.r32, out, piece, g0.slice_rows, g0.slice_rows ? g0.ry : g0.up);
  const int n0 = (int)piece.size() - 1;
  if (prog1) {
    bake_words(p->host, *prog1, g1->S, g1->r32, out1, piece1, 0, g1->up);
    const int64_t at = (int64_t)(out.size() / 4);  // side 1's groups follow side 0's
    out.insert(out.end(), out1.begin(), out1.end());
    for (size_t q = 1; q < piece1.size(); ++q) piece.push_back(at + piece1[q]);
  }
  if (out.size() / 4 >= (size_t(1) << 32)) return LPF_EUNSUPPORTED;  // group offsets are 32-bit
  if (out.empty()) out.assign(4, 0u);
  std::vector<uint32_t> piece32(piece.begin(), piece.end());
  cudaError_t e;
  if ((e = cudaMalloc(&b.d_words, out.size() * 4)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMalloc(&b.d_piece, piece32.size() * 4)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(b.d_words, out.data(), out.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return set_cuda_error(e);
  if ((e = cudaMemcpy(b.d_piece, piece32.data(), piece32.size() * 4, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return set_cuda_error(e);
  b.W = g0.W;
  b.S = g0.S;
  b.r32 = g0.r32;
  b.S1 = S1;
  b.r32_1 = r32_1;
  b.T = g0.T;
  b.BB = g0.BB;
  b.slice_rows = g0.slice_rows;
  b.n_pieces = (int)piece.size() - 1;
  b.n_pieces0 = n0;
  return LPF_OK;
}

// True when b holds the programs laid out for the sides' row layouts.
static bool baked_for_sides(const Baked& b, const Sides& sd) {
  return b.d_words && b.W == sd.g[0].W && b.S == sd.g[0].S && b.r32 == sd.g[0].r32 &&
         b.S1 == (sd.n == 2 ? sd.g[1].S : -1) && b.r32_1 == (sd.n == 2 ? sd.g[1].r32 : -1);
}

// Bake the image's programs (tree or plain) for the sides.
static int bake_sides(lpf_paths* p, const Sides& sd, bool standard, Baked& b) {
  const Program& prog0 = standard ? p->host.plain : p->host.tree;
  const Program& prog1 = standard ? p->host.plain_t : p->host.tree_t;
  return bake(p, prog0, sd.g[0], sd.n == 2 ? &prog1 : nullptr, sd.n == 2 ? &sd.g[1] : nullptr, b);
}

static std::once_flag g_attr_once;
static int g_attr_status = LPF_OK;
static int g_max_dyn_smem = 0;  // dynamic shared memory a walk block may use

template <typename K>
static int allow_smem(K kernel, int optin, int& max_dyn) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int dyn = optin - (int)fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e != cudaSuccess) return set_cuda_error(e);
  max_dyn = max_dyn == 0 ? dyn : std::min(max_dyn, dyn);
  return LPF_OK;
}

static void set_kernel_attributes() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) { g_attr_status = set_cuda_error(e); return; }
  int rc = allow_smem(walk_kernel<1>, optin, g_max_dyn_smem);
  if (!rc) rc = allow_smem(walk_kernel<2>, optin, g_max_dyn_smem);
  if (!rc) rc = allow_smem(walk_kernel<4>, optin, g_max_dyn_smem);
  if (!rc) rc = allow_smem(walk_kernel<8>, optin, g_max_dyn_smem);
  g_attr_status = rc;
}

static int g_num_sms = 0;

template <int T>
static int walk_blocks(const Sides& sd) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_kernel<T>, sd.threads, sd.band_bytes);
  if (e != cudaSuccess) return -set_cuda_error(e);
  return std::max(1, per_sm) * g_num_sms;
}

static int walk_blocks_for(const Sides& sd) {
  switch (sd.g[0].T) {
    case 1: return walk_blocks<1>(sd);
    case 2: return walk_blocks<2>(sd);
    case 4: return walk_blocks<4>(sd);
    default: return walk_blocks<8>(sd);
  }
}

static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_cuda_error(e);
  }
  return LPF_OK;
}

// Failure-detection self-test (lpf_paths_set_selftest): the staging wait
// expects 16 bytes more than the copy delivers and gives up after 2^16
// try_wait rounds instead of 2^24.
static uint32_t selftest_extra_tx(const lpf_paths* p) { return p->selftest ? 16u : 0u; }
static uint32_t selftest_wait_rounds(const lpf_paths* p) { return p->selftest ? (1u << 16) : kWaitRounds; }

// The walk's view of the sides: packed rows from `packed` (side 1 at
// sd.off1), selections sel0/sel1 (or null), pieces from b.
static void walk_sides(const Sides& sd, const Baked& b, const uint32_t* packed, const uint32_t* sel0,
                       const uint32_t* sel1, WalkSide& w0, WalkSide& w1) {
  const Geometry& g0 = sd.g[0];
  w0 = WalkSide{packed, sel0, g0.H, g0.W, g0.S, g0.nw, g0.G, g0.BB, g0.nbg, g0.nbg_s, g0.slice_rows,
                0, b.n_pieces0, g0.band_bytes};
  w1 = WalkSide{};
  if (sd.n == 2) {
    const Geometry& g1 = sd.g[1];
    w1 = WalkSide{packed + sd.off1, sel1, g1.H, g1.W, g1.S, g1.nw, g1.G, g1.BB, g1.nbg, g1.nbg_s, g1.slice_rows,
                  b.n_pieces0, b.n_pieces - b.n_pieces0, g1.band_bytes};
  }
}

static void launch_walk(const Sides& sd, const Baked& b, const uint32_t* packed, const uint32_t* sel0,
                        const uint32_t* sel1, unsigned long long* c, int64_t n_full, int64_t base, int* ctl,
                        const lpf_paths* p, int blocks, cudaStream_t s) {
  WalkSide w0, w1;
  walk_sides(sd, b, packed, sel0, sel1, w0, w1);
  const uint4* prog = reinterpret_cast<const uint4*>(b.d_words);
  const uint32_t xt = selftest_extra_tx(p), wr = selftest_wait_rounds(p);
  switch (sd.g[0].T) {
    case 1: walk_kernel<1><<<blocks, sd.threads, sd.band_bytes, s>>>(w0, w1, prog, b.d_piece, c, n_full, base, ctl, xt, wr); break;
    case 2: walk_kernel<2><<<blocks, sd.threads, sd.band_bytes, s>>>(w0, w1, prog, b.d_piece, c, n_full, base, ctl, xt, wr); break;
    case 4: walk_kernel<4><<<blocks, sd.threads, sd.band_bytes, s>>>(w0, w1, prog, b.d_piece, c, n_full, base, ctl, xt, wr); break;
    default: walk_kernel<8><<<blocks, sd.threads, sd.band_bytes, s>>>(w0, w1, prog, b.d_piece, c, n_full, base, ctl, xt, wr); break;
  }
}

// Pack both sides of an image (one launch, one grid row per side), zeroing
// n_zero counts and the walk's control words 1.. of the sides' band groups.
static void launch_pack(const uint8_t* img, const Sides& sd, uint32_t* packed, int64_t* counts, int64_t n_zero,
                        int* ctl, const lpf_paths* p, cudaStream_t s) {
  const Geometry& g0 = sd.g[0];
  const Geometry& g1 = sd.n == 2 ? sd.g[1] : sd.g[0];
  const PackSide s0{packed, g0.H, g0.W, g0.r32, g0.S, g0.rows, g0.W, 1, 0};
  const PackSide s1{packed + sd.off1, g1.H, g1.W, g1.r32, g1.S, g1.rows, 1, g0.W, g1.up};
  const int64_t total = std::max<int64_t>({(int64_t)g0.rows * g0.S, sd.n == 2 ? (int64_t)g1.rows * g1.S : 0, n_zero});
  const int pblocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  pack_rows_kernel<<<dim3(pblocks, sd.n), 256, 0, s>>>(img, s0, s1, reinterpret_cast<unsigned long long*>(counts),
                                                       n_zero, ctl + 1, kCtlUnits - 1 + sd.nbg,
                                                       p->checked ? ctl : nullptr);
}

// Enqueue one full evaluation with launch shape (T, BB) (<= 0: tuned or
// default); `accumulate` adds to the counts instead of replacing them.
static int run_full(const uint8_t* img, int H, int W, lpf_paths* p, int64_t* counts, cudaStream_t s,
                    bool standard, int T = 0, int BB = 0, const uint8_t* sel = nullptr, bool accumulate = false) {
  if (!p || !img || !counts) return LPF_EINVAL;
  if (p->host.dims != 2) return LPF_EINVAL;  // a volume's handle: lpf_full_3d
  if (H < 1 || W < 1 || H > 8192 || W > 8192) return LPF_EINVAL;
  if (p->host.rx >= W || p->host.ry >= H) return LPF_EINVAL;
  const Program& prog0 = standard ? p->host.plain : p->host.tree;
  const Program& prog1 = standard ? p->host.plain_t : p->host.tree_t;
  if (std::max(prog0.stack_depth, prog1.stack_depth) > kDevStack) return LPF_EUNSUPPORTED;
  std::call_once(g_attr_once, set_kernel_attributes);
  if (g_attr_status) return g_attr_status;
  if (T <= 0)
    for (const Tuned& t : p->tuned)
      if (t.H == H && t.W == W) { T = t.T; BB = t.BB; }
  Sides sd;
  int rc = make_sides(p->host, H, W, T, BB, sd);
  if (rc) return rc;
  if ((int)sd.band_bytes > g_max_dyn_smem) return LPF_EUNSUPPORTED;
  rc = ensure_device(p, sd.packed_words);
  if (rc) return rc;
  Baked& b = standard ? p->plain : p->tree;
  rc = bake_sides(p, sd, standard, b);
  if (rc) return rc;
  if ((rc = num_sms())) return rc;
  int blocks = walk_blocks_for(sd);
  if (blocks < 0) return -blocks;
  blocks = std::min(blocks, sd.nbg * b.n_pieces);
  (void)cudaGetLastError();  // clear a stale error left by earlier, unrelated calls

  const int64_t n_full = p->host.n_full, base = p->host.base;
  cudaError_t e = cudaSuccess;
  // pack the rows; zero the counts (unless accumulating) and the work
  // counters (not the status flags)
  launch_pack(img, sd, p->d_packed, counts, accumulate ? 0 : 2 * n_full, p->d_status, p, s);
  const uint32_t* sel0 = nullptr;
  const uint32_t* sel1 = nullptr;
  if (sel) {
    const Geometry& g0 = sd.g[0];
    const size_t words0 = (size_t)g0.H * g0.nw, words = words0 + (sd.n == 2 ? (size_t)sd.g[1].H * sd.g[1].nw : 0);
    if (words > p->sel_cap) {
      if (p->d_sel) { cudaDeviceSynchronize(); cudaFree(p->d_sel); p->d_sel = nullptr; p->sel_cap = 0; }
      e = cudaMalloc(&p->d_sel, words * 4);
      if (e != cudaSuccess) return set_cuda_error(e);
      p->sel_cap = words;
    }
    pack_sel_kernel<<<(int)std::min<size_t>((words0 + 255) / 256, 4096), 256, 0, s>>>(sel, g0.H, g0.W, g0.nw, W, 1,
                                                                                      p->d_sel);
    sel0 = p->d_sel;
    if (sd.n == 2) {
      const Geometry& g1 = sd.g[1];
      const size_t words1 = words - words0;
      pack_sel_kernel<<<(int)std::min<size_t>((words1 + 255) / 256, 4096), 256, 0, s>>>(sel, g1.H, g1.W, g1.nw, 1,
                                                                                        W, p->d_sel + words0);
      sel1 = p->d_sel + words0;
    }
  }
  unsigned long long* c = reinterpret_cast<unsigned long long*>(counts);
  // every warp walks every piece of its side
  p->nominal_pixels = prog0.n_pixel_words * sd.g[0].nbg * sd.g[0].G * sd.g[0].BB;
  if (sd.n == 2) p->nominal_pixels += prog1.n_pixel_words * sd.g[1].nbg * sd.g[1].G * sd.g[1].BB;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  launch_walk(sd, b, p->d_packed, sel0, sel1, c, n_full, base, p->d_status, p, blocks, s);
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (n_full > 1) {
    const int64_t n = 2 * (n_full - base - 1);
    const int mblocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mirror_kernel<<<mblocks, 256, 0, s>>>(c, n_full, base);
  }
  return cuda_status(cudaGetLastError());
}

// Time every admissible (T, BB) for this image size and keep the fastest.
static int autotune_full(const uint8_t* img, int H, int W, lpf_paths* p, int64_t* counts, cudaStream_t s,
                         int* bestT, int* bestBB) {
  const int nw = (W + 31) / 32;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LPF_ECUDA;
  float best = 1e30f;
  int bt = 0, bb = 0;
  int rc = LPF_OK;
  for (int T : {1, 2, 4, 8}) {
    if (T > 1 && (T / 2) >= nw) continue;          // more words per thread than a row has
    for (int BB : {1, 2, 4, 8}) {
      Sides sd;
      if (make_sides(p->host, H, W, T, BB, sd) != LPF_OK) continue;
      if (sd.g[0].T != T || sd.g[0].BB != BB) continue;  // shape not admissible as asked
      if ((int)sd.band_bytes > g_max_dyn_smem && g_max_dyn_smem > 0) continue;
      rc = run_full(img, H, W, p, counts, s, false, T, BB);  // warm-up (uploads tables)
      if (rc) break;
      float t_min = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        rc = run_full(img, H, W, p, counts, s, false, T, BB);
        cudaEventRecord(e1, s);
        if (rc) break;
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t_min = std::min(t_min, ms);
      }
      if (rc) break;
      if (t_min < best) { best = t_min; bt = T; bb = BB; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (bt == 0) return LPF_EUNSUPPORTED;
  {
    // leave the program on the device laid out for the winning shape (the
    // trials re-baked it for each shape they ran)
    Sides sd;
    rc = make_sides(p->host, H, W, bt, bb, sd);
    if (!rc) rc = bake_sides(p, sd, false, p->tree);
    if (rc) return rc;
  }
  for (Tuned& t : p->tuned)
    if (t.H == H && t.W == W) { t.T = bt; t.BB = bb; bt = -bt; break; }
  if (bt > 0) p->tuned.push_back({H, W, bt, bb});
  if (bestT) *bestT = std::abs(bt);
  if (bestBB) *bestBB = bb;
  return LPF_OK;
}

// Full evaluation of a volume (3D handle): pack the slices, walk, mirror.
static int run_full3(const uint8_t* vol, int D, int H, int W, lpf_paths* p, int64_t* counts, cudaStream_t s) {
  if (!p || !vol || !counts) return LPF_EINVAL;
  if (p->host.dims != 3) return LPF_EINVAL;  // an image's handle: lpf_full
  if (D < 1 || H < 1 || W < 1 || D > 4096 || H > 4096 || W > 4096) return LPF_EINVAL;
  if (p->host.rx >= W || p->host.ry >= H || p->host.rz >= D) return LPF_EINVAL;
  const Program& prog = p->host.tree;
  if (prog.stack_depth > kDevStack) return LPF_EUNSUPPORTED;
  std::call_once(g_attr_once, set_kernel_attributes);
  if (g_attr_status) return g_attr_status;
  int T = 0, BB = 0;
  for (const Tuned& t : p->tuned)
    if (t.H == H && t.W == W) { T = t.T; BB = t.BB; }
  Sides sd;  // one side
  int rc = make_geometry3(D, H, W, p->host.rx, p->host.ry, p->host.rz, T, BB, sd.g[0]);
  if (rc) return rc;
  const Geometry& g = sd.g[0];
  sd.n = 1;
  sd.packed_words = g.packed_words;
  sd.band_bytes = g.band_bytes;
  sd.nbg = g.nbg;
  // 16 warps per block whatever the band group's tile count: warps pull
  // units of any tile of the staged band group, and a volume's band group
  // (its slices with their rz halo) is large, so few blocks fit on an SM
  sd.threads = 512;
  if ((int)g.band_bytes > g_max_dyn_smem) return LPF_EUNSUPPORTED;
  rc = ensure_device(p, g.packed_words);
  if (rc) return rc;
  rc = bake(p, prog, g, nullptr, nullptr, p->tree);
  if (rc) return rc;
  if ((rc = num_sms())) return rc;
  int blocks = walk_blocks_for(sd);
  if (blocks < 0) return -blocks;
  blocks = std::min(blocks, g.nbg * p->tree.n_pieces);
  (void)cudaGetLastError();
  const int64_t n_full = p->host.n_full, base = p->host.base;
  {
    const int64_t total = std::max<int64_t>((int64_t)g.rows * g.S, 2 * n_full);
    const int pblocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    pack_vol_kernel<<<pblocks, 256, 0, s>>>(vol, D, H, W, g.ry, g.r32, g.S, g.slice_rows, g.rows, p->d_packed,
                                            reinterpret_cast<unsigned long long*>(counts), 2 * n_full,
                                            p->d_status + 1, kCtlUnits - 1 + g.nbg,
                                            p->checked ? p->d_status : nullptr);
  }
  unsigned long long* c = reinterpret_cast<unsigned long long*>(counts);
  p->nominal_pixels = prog.n_pixel_words * g.nbg * g.G * g.BB;
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  launch_walk(sd, p->tree, p->d_packed, nullptr, nullptr, c, n_full, base, p->d_status, p, blocks, s);
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (n_full > 1) {
    const int64_t n = 2 * (n_full - base - 1);
    const int mblocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mirror_kernel<<<mblocks, 256, 0, s>>>(c, n_full, base);
  }
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Full evaluation without allocating.
//
// lpf_full keeps its per-call work area (the packed image rows and the
// walk's control words: status, walked-work and unit counters) in device
// memory that the handle
// allocates on first use.  Some callers cannot let a library allocate at the
// time they evaluate: a host application that owns every device allocation
// and hands out fixed budgets, a real-time loop where cudaMalloc (which can
// synchronise the whole device) is forbidden, or code that records its work
// into a stream while allocation would break that.  For them this variant
// keeps the same work area in a fixed array compiled into the library (every
// GPU that loads the library holds it until the process exits) and calls no
// allocating routine.
constexpr size_t kNoAllocPackedWords = size_t(1) << 18;  // 1 MiB of packed image rows
static __device__ __align__(256) uint32_t g_noalloc_packed[kNoAllocPackedWords];
static __device__ __align__(256) int g_noalloc_ctl[kCtlWords];  // control words of the walk

namespace {
struct NoAllocSlot {
  uint32_t* packed = nullptr;
  int* ctl = nullptr;
  bool ready = false;
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc_slot[64];

// Device addresses of the fixed arrays on the current device, looked up once
// per device (in host code the array names are only stand-ins).
int noalloc_slot(int dev, NoAllocSlot& out) {
  if (dev < 0 || dev >= 64) return LPF_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocSlot& s = g_noalloc_slot[dev];
  if (!s.ready) {
    void* a = nullptr;
    void* b = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_packed);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&b, g_noalloc_ctl);
    if (e != cudaSuccess) return set_cuda_error(e);
    s.packed = static_cast<uint32_t*>(a);
    s.ctl = static_cast<int*>(b);
    s.ready = true;
  }
  out = s;
  return LPF_OK;
}
}  // namespace

// The fixed status word on device dev if an allocation-free call has run there.
int* noalloc_ctl_if_ready(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  return g_noalloc_slot[dev].ready ? g_noalloc_slot[dev].ctl : nullptr;
}

static int run_full_noalloc(const uint8_t* img, int H, int W, lpf_paths* p, int64_t* counts, cudaStream_t s) {
  if (!p || !img || !counts) return LPF_EINVAL;
  if (p->host.dims != 2) return LPF_EINVAL;
  if (H < 1 || W < 1 || H > 8192 || W > 8192) return LPF_EINVAL;
  if (p->host.rx >= W || p->host.ry >= H) return LPF_EINVAL;
  if (std::max(p->host.tree.stack_depth, p->host.tree_t.stack_depth) > kDevStack) return LPF_EUNSUPPORTED;
  std::call_once(g_attr_once, set_kernel_attributes);
  if (g_attr_status) return g_attr_status;
  int T = 0, BB = 0;
  for (const Tuned& t : p->tuned)
    if (t.H == H && t.W == W) { T = t.T; BB = t.BB; }
  Sides sd;
  int rc = make_sides(p->host, H, W, T, BB, sd);
  if (rc) return rc;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  const Baked& b = p->tree;
  // The programs for this size must already be on this device (an earlier
  // lpf_full call put them there).  When the tuned shape needs other row
  // layouts than the ones they were baked for (lpf_set_launch_shape after
  // that call), the walk runs in the shape they were baked for instead.
  if (b.d_words && b.W == W && !baked_for_sides(b, sd) && b.T > 0) {
    rc = make_sides(p->host, H, W, b.T, b.BB, sd);
    if (rc) return rc;
  }
  if ((int)sd.band_bytes > g_max_dyn_smem) return LPF_EUNSUPPORTED;
  if (sd.packed_words > kNoAllocPackedWords) return LPF_EUNSUPPORTED;  // image too large for the fixed area
  if (p->device != dev || !baked_for_sides(b, sd)) return LPF_EINVAL;
  NoAllocSlot slot;
  rc = noalloc_slot(dev, slot);
  if (rc) return rc;
  if ((rc = num_sms())) return rc;
  int blocks = walk_blocks_for(sd);
  if (blocks < 0) return -blocks;
  blocks = std::min(blocks, sd.nbg * b.n_pieces);
  (void)cudaGetLastError();

  const int64_t n_full = p->host.n_full, base = p->host.base;
  // pack the rows; the counts and the work counters start at 0 (the status
  // word keeps its flags until lpf_paths_status reads and clears them)
  launch_pack(img, sd, slot.packed, counts, 2 * n_full, slot.ctl, p, s);
  unsigned long long* c = reinterpret_cast<unsigned long long*>(counts);
  launch_walk(sd, b, slot.packed, nullptr, nullptr, c, n_full, base, slot.ctl, p, blocks, s);
  if (n_full > 1) {
    const int64_t n = 2 * (n_full - base - 1);
    const int mblocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mirror_kernel<<<mblocks, 256, 0, s>>>(c, n_full, base);
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace lpf

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

const char* lpf_last_error_message(void) { return lpf::g_last_error; }

const char* lpf_strerror(int code) {
  switch (code) {
    case LPF_OK: return "ok";
    case LPF_EINVAL: return "invalid argument";
    case LPF_ENOMEM: return "out of memory";
    case LPF_ECUDA: return "CUDA runtime error";
    case LPF_ETIMEOUT: return "device-side wait timed out";
    case LPF_EUNSUPPORTED: return "size not supported";
    case LPF_EPIXEL: return "pixel value other than 0 or 1 (checked mode)";
    default: return "unknown status";
  }
}

int lpf_build_paths(int32_t rx, int32_t ry, lpf_paths** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (rx < 0 || ry < 0 || rx > 4095 || ry > 4095) return LPF_EINVAL;
  lpf_paths* p = new (std::nothrow) lpf_paths();
  if (!p) return LPF_ENOMEM;
  std::string err;
  int rc;
  try {
    rc = lpf::build_paths(rx, ry, 0, p->host, err);  // pieces sized by the tree
  } catch (const std::bad_alloc&) {
    rc = LPF_ENOMEM;
  }
  if (rc != 0) {
    delete p;
    return rc == LPF_ENOMEM ? LPF_ENOMEM : LPF_EUNSUPPORTED;
  }
  *out = p;
  return LPF_OK;
}

int lpf_build_paths_3d(int32_t rx, int32_t ry, int32_t rz, lpf_paths** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (rx < 0 || ry < 0 || rz < 0 || rx > 1023 || ry > 1023 || rz > 1023) return LPF_EINVAL;
  lpf_paths* p = new (std::nothrow) lpf_paths();
  if (!p) return LPF_ENOMEM;
  std::string err;
  int rc;
  try {
    rc = lpf::build_paths_nd(rx, ry, rz, 3, 0, p->host, err);
  } catch (const std::bad_alloc&) {
    rc = LPF_ENOMEM;
  }
  if (rc != 0) {
    delete p;
    return rc == LPF_ENOMEM ? LPF_ENOMEM : LPF_EUNSUPPORTED;
  }
  *out = p;
  return LPF_OK;
}

int lpf_full_3d(const uint8_t* vol_dev, int32_t D, int32_t H, int32_t W, lpf_paths* paths, int64_t* counts_dev,
                lpf_stream_t stream) {
  return lpf::run_full3(vol_dev, D, H, W, paths, counts_dev, (cudaStream_t)stream);
}

int lpf_paths_info(const lpf_paths* p, int64_t* n_full, int64_t* n_canon, int64_t* n_off) {
  if (!p) return LPF_EINVAL;
  if (n_full) *n_full = p->host.n_full;
  if (n_canon) *n_canon = p->host.n_canon;
  if (n_off) *n_off = p->host.ptr.back();
  return LPF_OK;
}

int lpf_paths_export(const lpf_paths* p, int16_t* vec, int64_t* ptr, int16_t* off) {
  if (!p) return LPF_EINVAL;
  if (vec) std::memcpy(vec, p->host.vec.data(), p->host.vec.size() * sizeof(int16_t));
  if (ptr) std::memcpy(ptr, p->host.ptr.data(), p->host.ptr.size() * sizeof(int64_t));
  if (off) std::memcpy(off, p->host.off.data(), p->host.off.size() * sizeof(int16_t));
  return LPF_OK;
}

int lpf_paths_stats(const lpf_paths* p, int64_t* n_tree_nodes, int32_t* stack_depth, int32_t* n_pieces) {
  if (!p) return LPF_EINVAL;
  if (n_tree_nodes) *n_tree_nodes = p->host.n_nodes();
  if (stack_depth) *stack_depth = std::max(p->host.tree.stack_depth, p->host.tree_t.stack_depth);
  if (n_pieces) *n_pieces = (int32_t)(p->host.tree.piece_pixels.size() + p->host.tree_t.piece_pixels.size());
  return LPF_OK;
}

int lpf_paths_work(const lpf_paths* p, int64_t* executed, int64_t* nominal) {
  if (!p || !executed || !nominal) return LPF_EINVAL;
  *executed = 0;
  *nominal = p->nominal_pixels;
  if (!p->d_status) return LPF_OK;
  unsigned long long h = 0;
  if (cudaMemcpy(&h, p->d_status + lpf::kCtlExecuted, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LPF_ECUDA;
  *executed = (int64_t)h;
  return LPF_OK;
}

void lpf_paths_free(lpf_paths* p) {
  if (!p) return;
  if (p->device >= 0) {
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->tree.d_words);
    cudaFree(p->tree.d_piece);
    cudaFree(p->plain.d_words);
    cudaFree(p->plain.d_piece);
    cudaFree(p->d_packed);
    cudaFree(p->d_status);
    cudaFree(p->delta.d_doff);
    cudaFree(p->delta.d_dptr);
    cudaFree(p->delta.d_chunk);
    cudaFree(p->delta.d_off16);
    cudaFree(p->delta.d_vec16);
    cudaFree(p->delta.d_shear);
    cudaFree(p->d_z);
    cudaFree(p->d_partial);
    cudaFree(p->d_ext);
    cudaFree(p->d_sel);
    if (cur >= 0) cudaSetDevice(cur);
  }
  delete p;
}

int lpf_full(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, int64_t* counts_dev,
             lpf_stream_t stream) {
  return lpf::run_full(img_dev, H, W, paths, counts_dev, (cudaStream_t)stream, false);
}

int lpf_full_mc(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, const uint8_t* sel_dev,
                int64_t* counts_dev, lpf_stream_t stream) {
  if (!sel_dev) return LPF_EINVAL;
  return lpf::run_full(img_dev, H, W, paths, counts_dev, (cudaStream_t)stream, false, 0, 0, sel_dev);
}

int lpf_full_ensemble(const uint8_t* imgs_dev, int32_t n_img, int32_t H, int32_t W, lpf_paths* paths,
                      int64_t* counts_dev, lpf_stream_t stream) {
  if (!imgs_dev || n_img < 1) return LPF_EINVAL;
  for (int32_t i = 0; i < n_img; ++i) {
    // the non-canonical half is rewritten from the accumulated canonical
    // half after every image, so the sum stays exact
    const int rc = lpf::run_full(imgs_dev + (size_t)i * H * W, H, W, paths, counts_dev, (cudaStream_t)stream, false,
                                 0, 0, nullptr, i > 0);
    if (rc) return rc;
  }
  return LPF_OK;
}

int lpf_full_standard(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, int64_t* counts_dev,
                      lpf_stream_t stream) {
  return lpf::run_full(img_dev, H, W, paths, counts_dev, (cudaStream_t)stream, true);
}

int lpf_autotune_full(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, int64_t* counts_dev,
                      lpf_stream_t stream, int32_t* best_T, int32_t* best_BB) {
  if (!paths) return LPF_EINVAL;
  cudaEvent_t a = paths->ev_start, b = paths->ev_stop;
  paths->ev_start = paths->ev_stop = nullptr;
  const int rc = lpf::autotune_full(img_dev, H, W, paths, counts_dev, (cudaStream_t)stream, best_T, best_BB);
  paths->ev_start = a;
  paths->ev_stop = b;
  return rc;
}

int lpf_set_launch_shape(lpf_paths* p, int32_t H, int32_t W, int32_t T, int32_t BB) {
  if (!p || H < 1 || W < 1) return LPF_EINVAL;
  if (T != 1 && T != 2 && T != 4 && T != 8) return LPF_EINVAL;
  if (BB < 1 || BB > 16) return LPF_EINVAL;
  lpf::Geometry g;
  const int rc = lpf::make_geometry(H, W, p->host.rx, p->host.ry, T, BB, g);
  if (rc) return rc;
  if (g.T != T || g.BB != std::min<int>(BB, g.nbands)) return LPF_EUNSUPPORTED;
  for (lpf::Tuned& t : p->tuned)
    if (t.H == H && t.W == W) { t.T = T; t.BB = BB; return LPF_OK; }
  p->tuned.push_back({H, W, T, BB});
  return LPF_OK;
}

int lpf_full_noalloc(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, int64_t* counts_dev,
                     lpf_stream_t stream) {
  return lpf::run_full_noalloc(img_dev, H, W, paths, counts_dev, (cudaStream_t)stream);
}

int lpf_paths_set_timer(lpf_paths* p, void* ev_start, void* ev_stop) {
  if (!p) return LPF_EINVAL;
  p->ev_start = (cudaEvent_t)ev_start;
  p->ev_stop = (cudaEvent_t)ev_stop;
  return LPF_OK;
}

int lpf_paths_status(lpf_paths* p, lpf_stream_t stream) {
  if (!p) return LPF_EINVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LPF_ECUDA;
  int h = 0;
  if (p->d_status) {
    if (cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LPF_ECUDA;
    if (h && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return LPF_ECUDA;
  }
  // the status word of lpf_full_noalloc's fixed work area on this device
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LPF_ECUDA;
  int* ctl = lpf::noalloc_ctl_if_ready(dev);
  if (ctl) {
    int n = 0;
    if (cudaMemcpy(&n, ctl, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LPF_ECUDA;
    if (n && cudaMemset(ctl, 0, sizeof(int)) != cudaSuccess) return LPF_ECUDA;
    h |= n;
  }
  if (h & lpf::kStatusTimeout) return LPF_ETIMEOUT;
  if (h & lpf::kStatusPixel) return LPF_EPIXEL;
  return h ? LPF_EINVAL : LPF_OK;
}

int lpf_set_checked(lpf_paths* p, int32_t on) {
  if (!p || (on != 0 && on != 1)) return LPF_EINVAL;
  p->checked = on;
  return LPF_OK;
}

int lpf_paths_set_selftest(lpf_paths* p, int32_t on) {
  if (!p || (on != 0 && on != 1)) return LPF_EINVAL;
  p->selftest = on;
  return LPF_OK;
}

}  // extern "C"
