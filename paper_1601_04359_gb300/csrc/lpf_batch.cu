// Batched full lineal path functions of many independent images of uneven
// sizes in one run of persistent kernels (the batching form of the evaluation; the
// paper evaluates one image at a time, Sec. 3.1).
//
// Every image brings its own window and program (its own paths handle).  A
// batch is prepared once (programs uploaded, work area allocated, a device
// table of per-image descriptors written); a run is then a few launches with
// no host-device copies -- zero the counts, pack every image into bit rows,
// one persistent walk kernel per words-per-thread choice present, fill the
// mirrored halves -- and can be replayed as a CUDA graph.  All blocks have 8
// warps; each image side gets its own words per thread T (chosen by a
// waste/load cost model or by the batch autotuner), so its rows split into G
// word groups of 32T translations, and its own band groups of BB bands of 32
// rows (G x BB tiles, no band past the side's last where avoidable).  Each
// walk kernel visits a host-built list of band-group slots of its images
// (every band group gets slots in proportion to its work, heaviest first,
// then one more each), a block claiming the next slot from a counter
// whenever it is free; the kernels run side by side on forked streams, so
// one's blocks take the SMs another's leave at its end.  For each slot a block
// stages the band group's rows (one bulk copy, skipped if already
// staged) and its warps pull units (tile, program piece) from that band
// group's counter until none are left, so warps whose tiles skip zero-count
// subtrees take more units instead of waiting for the others.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_device.cuh"
#include "lpf_state.hpp"
#include "lpf_walk.cuh"

namespace lpf {

constexpr int kBatchWarps = 8;
// Slots per resident block, in proportion to work: finer slots balance the
// end of a launch better (measured: 3 -> 13.5 ms, 6 -> 13.0 ms, 12 -> 12.75 ms
// for 256 images of 48-256 px) at the cost of more band copies.
constexpr double kSlotsPerBlock = 12.0;
constexpr int kBatchThreads = 32 * kBatchWarps;

// control words: [0] status, [kBatchCtlSlot + k] slot counter of the walk
// kernel for T = 1 << k, [kBatchCtlUnits + g] unit counter of band group g
constexpr int kBatchCtlSlot = 1;
constexpr int kBatchCtlUnits = 8;
constexpr int kBatchTs = 4;  // T = 1, 2, 4, 8

// One side of one image (the image with the x-major vectors' program, or
// its transpose with the y-major vectors' program; both add to the image's
// counts).  H, W are the side's: the transpose's pixel (r, c) is the image's
// (c, r).
struct BatchDesc {
  const uint8_t* img;
  unsigned long long* counts;
  uint32_t* packed;
  const uint4* prog;        // baked program, 16-byte groups
  const uint32_t* piece;    // piece starts in groups
  int64_t n_full, base;
  int H, W, S, nw, G, BB, T, r32, rows, nbg, n_pieces, bg0;
  int rs, cs;               // the side's pixel (r, c) is img[r rs + c cs]
  int up;                   // packed row y holds the side's row (y - up) mod H
  int primary;              // 1: side 0 (zeroes and mirrors the image's counts)
  uint32_t band_bytes;
};

struct BatchSlot {
  int img, bg, g;  // image, its band group, global band-group index (counter)
};

__global__ void batch_zero_kernel(const BatchDesc* __restrict__ d) {
  const BatchDesc& b = d[blockIdx.y];
  if (!b.primary) return;
  const int64_t n = 2 * b.n_full;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b.counts[i] = 0ull;
}

// Packed rows of every side: bit b of word k of row y is the side's pixel at
// row (y - up) mod H, column (32k + b - r32) mod W.  A transposed side runs over its
// words column by column, so that a warp reads consecutive image bytes.
__global__ void batch_pack_kernel(const BatchDesc* __restrict__ d) {
  const BatchDesc& b = d[blockIdx.y];
  const int64_t total = (int64_t)b.rows * b.S;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int y, k;
    if (b.primary) { y = (int)(i / b.S); k = (int)(i % b.S); }
    else { k = (int)(i / b.rows); y = (int)(i % b.rows); }
    const uint8_t* row = b.img + (int64_t)((y + b.H - b.up % b.H) % b.H) * b.rs;
    int x = (32 * k - b.r32) % b.W;
    if (x < 0) x += b.W;
    uint32_t bits = 0;
    for (int bit = 0; bit < 32; ++bit) {
      bits |= (uint32_t)(row[(int64_t)x * b.cs] != 0) << bit;
      if (++x == b.W) x = 0;
    }
    b.packed[(int64_t)y * b.S + k] = bits;
  }
}

__global__ void batch_mirror_kernel(const BatchDesc* __restrict__ d) {
  const BatchDesc& b = d[blockIdx.y];
  if (!b.primary) return;
  const int64_t n = b.n_full - b.base - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n, j = b.base + 1 + i % n;
    b.counts[p * b.n_full + (b.n_full - 1 - j)] = b.counts[p * b.n_full + j];
  }
}

// One unit; returns the pixels the warp walked.
template <int T>
__device__ __forceinline__ uint32_t batch_unit(const BatchDesc& b, int bg, int tile, int pi, const uint32_t* sm,
                                               int lane) {
  const int bl = tile / b.G, grp = tile - (tile / b.G) * b.G;
  const int y = (bg * b.BB + bl) * 32 + lane;
  const uint32_t* lane_base = sm + (bl * 32 + lane) * b.S + grp * T;
  return walk_unit<T, false>(b.prog, b.piece[pi], b.piece[pi + 1], lane_base, y, b.H, b.W, b.nw, grp * T, nullptr,
                             lane, b.counts, b.n_full, b.base);
}

// The walk of the slots whose images take T words per thread (one kernel per
// T: the four walks inlined behind one switch would share one register
// allocation and spill).  slot_ctr is this kernel's slot counter in ctl.
// T >= 4 keeps its masks and the image's fields in up to 80 registers (3
// blocks per SM; with 64 it spills, measured 3 % slower on the 256 images).
template <int T>
__global__ void __launch_bounds__(kBatchThreads, (T >= 4 ? 3 : 4)) batch_walk_kernel(const BatchDesc* __restrict__ d,
                                                                   const BatchSlot* __restrict__ slots,
                                                                   int n_slots, int* __restrict__ ctl,
                                                                   int slot_ctr,
                                                                   unsigned long long* __restrict__ executed) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort, s_done, s_slot;
  __shared__ uint32_t s_walked[kBatchWarps];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) { mbar_init(&bar, 1); s_abort = 0; }
  __syncthreads();
  uint32_t parity = 0;
  int cur_img = -1, cur_bg = -1;
  bool copy_pending = false;
  for (;;) {
    // the next slot, claimed when this block is free (the slot list ends
    // with one more slot per band group, heaviest first, so that blocks
    // left without work help the band groups that still have units)
    if (threadIdx.x == 0) s_slot = atomicAdd(ctl + slot_ctr, 1);
    __syncthreads();
    const int k = s_slot;
    __syncthreads();  // s_slot is rewritten next round
    if (k >= n_slots) break;
    const BatchSlot sl = slots[k];
    const BatchDesc& b = d[sl.img];
    const int n_tiles = b.G * b.BB;
    const int units = n_tiles * b.n_pieces;
    int* ctr = ctl + kBatchCtlUnits + sl.g;
    if (threadIdx.x == 0) s_done = *reinterpret_cast<volatile int*>(ctr) >= units;
    __syncthreads();
    if (s_done) {
      __syncthreads();  // s_done is rewritten next round
      continue;
    }
    if (sl.img != cur_img || sl.bg != cur_bg) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar, b.band_bytes);
        bulk_g2s(sm, b.packed + (size_t)sl.bg * 32 * b.BB * b.S, b.band_bytes, &bar);
      }
      copy_pending = true;
      if (mbar_wait(&bar, parity)) copy_pending = false;
      else s_abort = 1;
      parity ^= 1u;
      cur_img = sl.img;
      cur_bg = sl.bg;
      __syncthreads();
      if (s_abort) break;
    }
    // (pixels walked are tallied in shared memory, one word per warp, to keep
    // registers for the walk)
    if (lane == 0) s_walked[threadIdx.x >> 5] = 0u;
    for (;;) {
      int u = 0;
      if (lane == 0) u = atomicAdd(ctr, 1);
      u = __shfl_sync(0xffffffffu, u, 0);
      if (u >= units) break;
      const int tile = u % n_tiles, pi = u / n_tiles;
      const uint32_t w = batch_unit<T>(b, sl.bg, tile, pi, sm, lane);
      if (lane == 0) s_walked[threadIdx.x >> 5] += w;
    }
    if (lane == 0 && s_walked[threadIdx.x >> 5])
      atomicAdd(executed + sl.img, (unsigned long long)s_walked[threadIdx.x >> 5]);
    __syncthreads();  // every warp is done with the staged band before it may be replaced
  }
  if (s_abort) {
    atomicOr(ctl, 1);
    if (copy_pending) (void)mbar_wait(&bar, parity ^ 1u);
  }
}

// T = 1 << k.
static inline int t_index(int T) { return T == 1 ? 0 : T == 2 ? 1 : T == 4 ? 2 : 3; }

static const void* batch_walk_fn(int k) {
  switch (k) {
    case 0: return (const void*)batch_walk_kernel<1>;
    case 1: return (const void*)batch_walk_kernel<2>;
    case 2: return (const void*)batch_walk_kernel<4>;
    default: return (const void*)batch_walk_kernel<8>;
  }
}

static void batch_walk_launch(int k, int blocks, uint32_t smem, cudaStream_t s, const BatchDesc* d,
                              const BatchSlot* slots, int n_slots, int* ctl, int slot_ctr,
                              unsigned long long* executed) {
  switch (k) {
    case 0: batch_walk_kernel<1><<<blocks, kBatchThreads, smem, s>>>(d, slots, n_slots, ctl, slot_ctr, executed); break;
    case 1: batch_walk_kernel<2><<<blocks, kBatchThreads, smem, s>>>(d, slots, n_slots, ctl, slot_ctr, executed); break;
    case 2: batch_walk_kernel<4><<<blocks, kBatchThreads, smem, s>>>(d, slots, n_slots, ctl, slot_ctr, executed); break;
    default: batch_walk_kernel<8><<<blocks, kBatchThreads, smem, s>>>(d, slots, n_slots, ctl, slot_ctr, executed); break;
  }
}

// Bands per band group for a side of nbands bands split into G word groups:
// at most ceil(8 / G) (a band group holds about one tile per warp), the
// fewest bands covered past the side's last one, then the most bands (fewer
// copies of the halo rows).  The warps pull units, so G x BB need not be 8.
static int band_group_bands(int nbands, int G) {
  const int cap = std::max(1, std::min(nbands, (kBatchWarps + G - 1) / G));
  int best = 1, best_cov = 1 << 30;
  for (int bb = 1; bb <= cap; ++bb) {
    const int cov = bb * ((nbands + bb - 1) / bb);
    if (cov <= best_cov) { best_cov = cov; best = bb; }
  }
  return best;
}

// Cost of a (T) choice for one image: translation words covered per useful
// word, times shared loads per word.
static double shape_cost(int H, int W, int T) {
  const int nw = (W + 31) / 32;
  const int G = (nw + T - 1) / T;
  if (G > kBatchWarps) return 1e30;
  const int nbands = (H + 31) / 32;
  const int BB = band_group_bands(nbands, G);
  const int nbg = (nbands + BB - 1) / BB;
  const double covered = (double)G * T * 32.0 * BB * 32.0 * nbg;
  const double useful = (double)W * H;
  return covered / useful * (double)(T + 1) / T;
}

}  // namespace lpf

struct lpf_batch {
  int n = 0;
  std::vector<lpf_paths*> paths;
  std::vector<lpf::BatchDesc> desc;  // per side of every image
  std::vector<int> img_desc;         // an image's first descriptor (its side 0)
  lpf::BatchDesc* d_desc = nullptr;
  unsigned long long* d_exec = nullptr;  // per descriptor: pixels the warps walked in the last run
  std::vector<int64_t> nominal;          // per descriptor: the same without the zero-count skip
  uint32_t* d_packed = nullptr;
  int* d_ctl = nullptr;          // [0] status, [kBatchCtlUnits + g] unit counter of band group g
  int ctl_words = 0, ctl_cap = 0;
  lpf::BatchSlot* d_slots = nullptr;
  int n_slots = 0;
  // the walk kernel of T = 1 << k visits slots [slot_off[k], slot_off[k + 1])
  // with blocks_T[k] blocks; the kernels after the first run on the batch's
  // own streams, forked from and joined to the caller's
  int slot_off[lpf::kBatchTs + 1] = {0, 0, 0, 0, 0};
  int run_order[lpf::kBatchTs] = {0, 1, 2, 3};  // T indices, most work first
  int blocks_T[lpf::kBatchTs] = {0, 0, 0, 0};
  cudaStream_t aux[lpf::kBatchTs - 1] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[lpf::kBatchTs - 1] = {nullptr, nullptr, nullptr};
  // The batch's own copies of the programs (one per handle and row stride):
  // evaluating a handle on its own afterwards (another launch shape) re-bakes
  // the handle's program and must not move the batch's.
  std::vector<const lpf_paths*> baked_for;
  std::vector<int> baked_side;   // 0: the image's program, 1: the transpose's
  std::vector<lpf::Baked> baked;
  int desc_cap = 0;
  uint32_t max_band = 0;
  int max_pack = 0, max_full = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace lpf {

// The words per thread of a side from the cost model (0: none admissible).
static int best_T(int H, int W) {
  double best = 1e30;
  int T = 0;
  for (int t : {1, 2, 4, 8}) {
    const double c = shape_cost(H, W, t);
    if (c < best) { best = c; T = t; }
  }
  return T;
}

static bool admissible(int W, int T) {
  const int G = ((W + 31) / 32 + T - 1) / T;
  return (T == 1 || T == 2 || T == 4 || T == 8) && G <= kBatchWarps;
}

static int batch_build(lpf_batch* bt, const uint8_t* const* imgs, const int32_t* H, const int32_t* W,
                       int64_t* const* counts, const int32_t* T_choice) {
  // geometry, programs on the device, work-area layout; one descriptor per
  // side of every image
  size_t packed_total = 0;
  std::vector<size_t> offs;
  bt->desc.clear();
  bt->nominal.clear();
  bt->img_desc.assign(bt->n, 0);
  std::vector<char> used(bt->baked.size(), 0);
  int total_bg = 0;
  std::vector<double> bg_work;  // nominal work of one band group of each side
  bt->max_band = 0;
  bt->max_pack = bt->max_full = 0;
  for (int i = 0; i < bt->n; ++i) {
    lpf_paths* p = bt->paths[i];
    if (!p || !imgs[i] || !counts[i]) return LPF_EINVAL;
    if (H[i] < 1 || W[i] < 1 || H[i] > 8192 || W[i] > 8192) return LPF_EINVAL;
    if (p->host.rx >= W[i] || p->host.ry >= H[i]) return LPF_EINVAL;
    if (std::max(p->host.tree.stack_depth, p->host.tree_t.stack_depth) > kWalkStack) return LPF_EUNSUPPORTED;
    int rc = ensure_device(p, 0);
    if (rc) return rc;
    const int n_sides = p->host.root_t >= 0 ? 2 : 1;
    bt->img_desc[i] = (int)bt->desc.size();
    for (int side = 0; side < n_sides; ++side) {
      // side 1: the transposed image with the y-major vectors' program
      const int Hs = side ? W[i] : H[i], Ws = side ? H[i] : W[i];
      const int rxs = side ? p->host.ry : p->host.rx;
      // row offsets: side 0 0 .. min(rx, ry); side 1 -h .. h, h = min(rx, ry - 1)
      const int rys = side ? std::min(p->host.rx, p->host.ry - 1) : std::min(p->host.rx, p->host.ry);
      const int up = side ? rys : 0;
      int T = T_choice ? T_choice[i] : 0;
      if (T <= 0 || (side && !admissible(Ws, T))) T = best_T(Hs, Ws);
      if (T <= 0 || !admissible(Ws, T)) return LPF_EUNSUPPORTED;
      const int G = ((Ws + 31) / 32 + T - 1) / T;
      Geometry g;
      rc = layout_side(Hs, Ws, rxs, rys, T, band_group_bands((Hs + 31) / 32, G), g, up);
      if (rc) return rc;
      size_t k = 0;  // this handle's copy of this side's program for this row stride, else a new slot
      while (k < bt->baked.size() &&
             !(bt->baked_for[k] == p && bt->baked_side[k] == side && bt->baked[k].S == g.S)) ++k;
      if (k == bt->baked.size()) {
        bt->baked_for.push_back(p);
        bt->baked_side.push_back(side);
        bt->baked.emplace_back();
        used.push_back(0);
      }
      used[k] = 1;
      const Program& prog = side ? p->host.tree_t : p->host.tree;
      rc = bake(p, prog, g, nullptr, nullptr, bt->baked[k]);
      if (rc) return rc;
      BatchDesc d{};
      d.img = imgs[i];
      d.counts = reinterpret_cast<unsigned long long*>(counts[i]);
      d.prog = reinterpret_cast<const uint4*>(bt->baked[k].d_words);
      d.piece = bt->baked[k].d_piece;
      d.n_full = p->host.n_full;
      d.base = p->host.base;
      d.bg0 = total_bg;
      d.H = g.H; d.W = g.W; d.S = g.S; d.nw = g.nw; d.G = g.G; d.BB = g.BB; d.T = g.T; d.r32 = g.r32;
      d.rows = g.rows; d.nbg = g.nbg; d.n_pieces = bt->baked[k].n_pieces; d.band_bytes = g.band_bytes;
      d.up = up;
      d.rs = side ? 1 : W[i];
      d.cs = side ? W[i] : 1;
      d.primary = side == 0;
      bt->desc.push_back(d);
      total_bg += g.nbg;
      bg_work.push_back((double)prog.n_pixel_words * g.G * g.BB * (g.T + 1));
      bt->nominal.push_back(prog.n_pixel_words * (int64_t)g.nbg * g.G * g.BB);  // every warp walks every piece
      offs.push_back(packed_total);
      packed_total += (g.packed_words + 3) & ~size_t(3);  // keep every side 16-byte aligned
      bt->max_band = std::max(bt->max_band, g.band_bytes);
      bt->max_pack = std::max<int>(bt->max_pack, (int)std::min<int64_t>(((int64_t)g.rows * g.S + 255) / 256, 64));
      bt->max_full = std::max<int>(bt->max_full, (int)std::min<int64_t>((2 * d.n_full + 255) / 256, 64));
    }
  }
  const int n_desc = (int)bt->desc.size();
  // drop the copies no image of this build uses (earlier launch shapes)
  for (size_t k = bt->baked.size(); k-- > 0;)
    if (!used[k]) {
      cudaDeviceSynchronize();
      cudaFree(bt->baked[k].d_words);
      cudaFree(bt->baked[k].d_piece);
      bt->baked.erase(bt->baked.begin() + (std::ptrdiff_t)k);
      bt->baked_for.erase(bt->baked_for.begin() + (std::ptrdiff_t)k);
      bt->baked_side.erase(bt->baked_side.begin() + (std::ptrdiff_t)k);
    }
  cudaError_t e;
  if (bt->d_packed) { cudaFree(bt->d_packed); bt->d_packed = nullptr; }
  if ((e = cudaMalloc(&bt->d_packed, std::max<size_t>(16, packed_total * 4))) != cudaSuccess) return set_cuda_error(e);
  for (int i = 0; i < n_desc; ++i) bt->desc[i].packed = bt->d_packed + offs[i];
  if (n_desc > bt->desc_cap) {
    if (bt->d_desc) { cudaFree(bt->d_desc); bt->d_desc = nullptr; }
    if (bt->d_exec) { cudaFree(bt->d_exec); bt->d_exec = nullptr; }
    if ((e = cudaMalloc(&bt->d_desc, sizeof(BatchDesc) * n_desc)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMalloc(&bt->d_exec, sizeof(unsigned long long) * n_desc)) != cudaSuccess) return set_cuda_error(e);
    bt->desc_cap = n_desc;
  }
  if ((e = cudaMemset(bt->d_exec, 0, sizeof(unsigned long long) * n_desc)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(bt->d_desc, bt->desc.data(), sizeof(BatchDesc) * n_desc, cudaMemcpyHostToDevice)) != cudaSuccess)
    return set_cuda_error(e);
  bt->ctl_words = kBatchCtlUnits + total_bg;
  if (bt->ctl_words > bt->ctl_cap) {
    if (bt->d_ctl) { cudaFree(bt->d_ctl); bt->d_ctl = nullptr; }
    if ((e = cudaMalloc(&bt->d_ctl, bt->ctl_words * sizeof(int))) != cudaSuccess) return set_cuda_error(e);
    bt->ctl_cap = bt->ctl_words;
  }
  if ((e = cudaMemset(bt->d_ctl, 0, bt->ctl_words * sizeof(int))) != cudaSuccess) return set_cuda_error(e);
  int dev = 0, optin = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // each T's walk kernel: its shared-memory limit and resident blocks
  int resident_T[kBatchTs];
  for (int k = 0; k < kBatchTs; ++k) {
    const void* fn = batch_walk_fn(k);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return set_cuda_error(e);
    const int max_dyn = optin - (int)fa.sharedSizeBytes;
    if ((int)bt->max_band > max_dyn) return LPF_EUNSUPPORTED;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn)) != cudaSuccess)
      return set_cuda_error(e);
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, bt->max_band)) != cudaSuccess)
      return set_cuda_error(e);
    resident_T[k] = std::max(1, per_sm) * sms;
  }
  // Slots, per T: every band group at least one, more in proportion to its
  // work (about kSlotsPerBlock slots per resident block over the whole
  // batch), heaviest band groups first, then the sweep: every band group once
  // more, heaviest first.  The kernels run most work first.
  {
    std::vector<int> order(n_desc);
    for (int i = 0; i < n_desc; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return bg_work[a] > bg_work[b]; });
    double total = 0, work_T[kBatchTs] = {0, 0, 0, 0};
    for (int i = 0; i < n_desc; ++i) {
      total += bg_work[i] * bt->desc[i].nbg;
      work_T[t_index(bt->desc[i].T)] += bg_work[i] * bt->desc[i].nbg;
    }
    const double per_slot = total / (kSlotsPerBlock * resident_T[0]);
    for (int k = 0; k < kBatchTs; ++k) bt->run_order[k] = k;
    std::stable_sort(bt->run_order, bt->run_order + kBatchTs, [&](int a, int b) { return work_T[a] > work_T[b]; });
    std::vector<BatchSlot> slots;
    for (int k = 0; k < kBatchTs; ++k) {
      bt->slot_off[k] = (int)slots.size();
      for (int i : order)
        if (t_index(bt->desc[i].T) == k)
          for (int bg = 0; bg < bt->desc[i].nbg; ++bg) {
            const int n = std::max(1, (int)std::lround(bg_work[i] / per_slot));
            for (int c = 0; c < n; ++c) slots.push_back({i, bg, bt->desc[i].bg0 + bg});
          }
      for (int i : order)
        if (t_index(bt->desc[i].T) == k)
          for (int bg = 0; bg < bt->desc[i].nbg; ++bg) slots.push_back({i, bg, bt->desc[i].bg0 + bg});
      bt->blocks_T[k] = std::min(resident_T[k], (int)slots.size() - bt->slot_off[k]);
    }
    bt->slot_off[kBatchTs] = (int)slots.size();
    bt->n_slots = (int)slots.size();
    if (bt->d_slots) { cudaFree(bt->d_slots); bt->d_slots = nullptr; }
    if ((e = cudaMalloc(&bt->d_slots, sizeof(BatchSlot) * slots.size())) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemcpy(bt->d_slots, slots.data(), sizeof(BatchSlot) * slots.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return set_cuda_error(e);
  }
  // the batch's streams and events for the walks after the first
  for (int k = 0; k < kBatchTs - 1; ++k) {
    if (!bt->aux[k] && (e = cudaStreamCreateWithFlags(&bt->aux[k], cudaStreamNonBlocking)) != cudaSuccess)
      return set_cuda_error(e);
    if (!bt->ev_join[k] && (e = cudaEventCreateWithFlags(&bt->ev_join[k], cudaEventDisableTiming)) != cudaSuccess)
      return set_cuda_error(e);
  }
  if (!bt->ev_fork && (e = cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
    return set_cuda_error(e);
  if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
  if (bt->graph) { cudaGraphDestroy(bt->graph); bt->graph = nullptr; }
  return LPF_OK;
}

static void batch_enqueue(lpf_batch* bt, cudaStream_t s) {
  cudaMemsetAsync(bt->d_ctl, 0, bt->ctl_words * sizeof(int), s);  // status of this run, unit counters
  const int n_desc = (int)bt->desc.size();
  cudaMemsetAsync(bt->d_exec, 0, sizeof(unsigned long long) * n_desc, s);
  batch_zero_kernel<<<dim3(bt->max_full, n_desc), 256, 0, s>>>(bt->d_desc);
  batch_pack_kernel<<<dim3(bt->max_pack, n_desc), 256, 0, s>>>(bt->d_desc);
  // one walk kernel per T present, the one with the most work on the
  // caller's stream, the others on the batch's streams (their blocks take
  // the SMs the first one's blocks leave at its end); joined before the mirror
  int present = 0;
  for (int k = 0; k < kBatchTs; ++k) present += bt->slot_off[k + 1] > bt->slot_off[k];
  if (present > 1) cudaEventRecord(bt->ev_fork, s);
  int n_fork = 0;
  bool first = true;
  for (int r = 0; r < kBatchTs; ++r) {
    const int k = bt->run_order[r];
    const int n = bt->slot_off[k + 1] - bt->slot_off[k];
    if (n == 0) continue;
    cudaStream_t ks = s;
    if (!first) {
      ks = bt->aux[n_fork];
      cudaStreamWaitEvent(ks, bt->ev_fork, 0);
    }
    batch_walk_launch(k, bt->blocks_T[k], bt->max_band, ks, bt->d_desc, bt->d_slots + bt->slot_off[k], n,
                      bt->d_ctl, kBatchCtlSlot + k, bt->d_exec);
    if (!first) cudaEventRecord(bt->ev_join[n_fork++], ks);
    first = false;
  }
  for (int f = 0; f < n_fork; ++f) cudaStreamWaitEvent(s, bt->ev_join[f], 0);
  batch_mirror_kernel<<<dim3(bt->max_full, n_desc), 256, 0, s>>>(bt->d_desc);
}

}  // namespace lpf

extern "C" {

int lpf_batch_create(int32_t n_img, const uint8_t* const* imgs_dev, const int32_t* H, const int32_t* W,
                     lpf_paths* const* paths, int64_t* const* counts_dev, const int32_t* words_per_thread,
                     lpf_batch** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (n_img < 1 || !imgs_dev || !H || !W || !paths || !counts_dev) return LPF_EINVAL;
  for (int i = 0; i < n_img; ++i)
    if (!paths[i] || paths[i]->host.dims != 2) return LPF_EINVAL;  // images only
  for (int i = 0; i < n_img; ++i)
    for (int j = 0; j < i; ++j)
      if (paths[i] == paths[j] && (H[i] != H[j] || W[i] != W[j])) return LPF_EINVAL;  // one program per handle
  lpf_batch* bt = new (std::nothrow) lpf_batch();
  if (!bt) return LPF_ENOMEM;
  bt->n = n_img;
  bt->paths.assign(paths, paths + n_img);
  const int rc = lpf::batch_build(bt, imgs_dev, H, W, counts_dev, words_per_thread);
  if (rc) { lpf_batch_free(bt); return rc; }
  *out = bt;
  return LPF_OK;
}

int lpf_batch_run(lpf_batch* bt, int32_t use_graph, lpf_stream_t stream) {
  if (!bt) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  if (!use_graph) {
    lpf::batch_enqueue(bt, s);
    return lpf::set_cuda_error(cudaGetLastError());
  }
  cudaError_t e = cudaSuccess;
  if (!bt->exec) {
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      lpf::batch_enqueue(bt, cs);
      e = cudaStreamEndCapture(cs, &bt->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { bt->exec = nullptr; return lpf::set_cuda_error(e); }
  }
  e = cudaGraphLaunch(bt->exec, s);
  return lpf::set_cuda_error(e);
}

int lpf_batch_status(lpf_batch* bt, lpf_stream_t stream) {
  if (!bt) return LPF_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  int h = 0;
  e = cudaMemcpy(&h, bt->d_ctl, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  return h ? LPF_ETIMEOUT : LPF_OK;
}

int lpf_batch_work(lpf_batch* bt, int64_t* executed, int64_t* nominal, lpf_stream_t stream) {
  if (!bt || !executed || !nominal) return LPF_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  const int n_desc = (int)bt->desc.size();
  std::vector<unsigned long long> h(n_desc, 0);
  if (n_desc && (e = cudaMemcpy(h.data(), bt->d_exec, sizeof(unsigned long long) * n_desc,
                                cudaMemcpyDeviceToHost)) != cudaSuccess)
    return lpf::set_cuda_error(e);
  for (int i = 0; i < bt->n; ++i) {
    const int d0 = bt->img_desc[i], d1 = i + 1 < bt->n ? bt->img_desc[i + 1] : n_desc;
    executed[i] = nominal[i] = 0;
    for (int d = d0; d < d1; ++d) {
      executed[i] += (int64_t)h[d];
      nominal[i] += bt->nominal[d];
    }
  }
  return LPF_OK;
}

int lpf_batch_autotune(lpf_batch* bt, const uint8_t* const* imgs_dev, const int32_t* H, const int32_t* W,
                       int64_t* const* counts_dev, lpf_stream_t stream, int32_t* chosen_T) {
  // Per image size class (words per row), try every admissible T with the
  // whole batch and keep the fastest; classes are tuned one after another.
  if (!bt || !imgs_dev || !H || !W || !counts_dev) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> T(bt->n);
  for (int i = 0; i < bt->n; ++i) T[i] = bt->desc[bt->img_desc[i]].T;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_it = [&](float& ms_out) -> int {
    int rc = lpf::batch_build(bt, imgs_dev, H, W, counts_dev, T.data());
    if (rc) return rc;
    lpf::batch_enqueue(bt, s);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0, s);
      lpf::batch_enqueue(bt, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    ms_out = best;
    return lpf::set_cuda_error(cudaGetLastError());
  };
  float cur = 0;
  int rc = time_it(cur);
  for (int nw = 1; nw <= 256 && !rc; ++nw) {
    bool present = false;
    for (int i = 0; i < bt->n; ++i) present |= ((W[i] + 31) / 32 == nw);
    if (!present) continue;
    for (int t : {1, 2, 4, 8}) {
      if ((nw + t - 1) / t > lpf::kBatchWarps) continue;
      std::vector<int32_t> keep = T;
      for (int i = 0; i < bt->n; ++i)
        if ((W[i] + 31) / 32 == nw) T[i] = t;
      float ms = 0;
      rc = time_it(ms);
      if (rc) break;
      if (ms < cur) cur = ms;
      else T = keep;
    }
  }
  if (!rc) rc = lpf::batch_build(bt, imgs_dev, H, W, counts_dev, T.data());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc && chosen_T)
    for (int i = 0; i < bt->n; ++i) chosen_T[i] = T[i];
  return rc;
}

void lpf_batch_free(lpf_batch* bt) {
  if (!bt) return;
  cudaDeviceSynchronize();
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  cudaFree(bt->d_desc);
  cudaFree(bt->d_exec);
  cudaFree(bt->d_packed);
  cudaFree(bt->d_ctl);
  cudaFree(bt->d_slots);
  for (lpf::Baked& b : bt->baked) {
    cudaFree(b.d_words);
    cudaFree(b.d_piece);
  }
  for (int k = 0; k < lpf::kBatchTs - 1; ++k) {
    if (bt->aux[k]) cudaStreamDestroy(bt->aux[k]);
    if (bt->ev_join[k]) cudaEventDestroy(bt->ev_join[k]);
  }
  if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
  delete bt;
}

}  // extern "C"
