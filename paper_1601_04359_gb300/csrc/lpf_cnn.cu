// Learned swap proposer: a small convolutional network that scores every
// pixel of the cell as the phase-1 pixel (channel 1) or the phase-0 pixel
// (channel 0) of an exchange; trained on candidates the annealer drew and
// evaluated exactly, and used by the annealer to draw candidates (every
// accept/reject decision still uses the exact count changes).  The paper has
// no learned part: its modification operator (Sec. 4) draws interfacial pixels
// uniformly, which stays the fallback (epsilon share of draws).
//
// Network: five 3x3 convolutions with circular padding (the medium is
// periodic), ReLU between them: 2 -> 32 -> 64 -> 48 -> 32 -> 2 channels,
// 61,234 parameters.  Input channels: cell value, interfacial mask.
// Weights: float32 master copies updated by Adam, bfloat16 copies used by the
// forward and backward passes.  The convolutions (forward, input gradient,
// weight gradient) are implicit GEMMs on the tensor cores (mma.sync,
// bfloat16 operands, float32 accumulation): activations are kept in float32
// and rounded to bfloat16 where they enter a product; gradients enter as two
// bfloat16 terms (high and low part, about 16 significant bits), because
// their sums over pixels cancel and a single rounding loses too much.
//
// Layouts: activations [H][W][C] (channels innermost); weights [9][Cin][Cout]
// with tap = (dy+1)*3 + (dx+1); parameter vector = for each layer W then b.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <random>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_state.hpp"

namespace lpf {

constexpr int kLayers = 5;
constexpr int kCh[kLayers + 1] = {2, 32, 64, 48, 32, 2};

inline int layer_w_size(int l) { return 9 * kCh[l] * kCh[l + 1]; }

// Input features [H][W][2]: cell value and interfacial mask (torus); cell
// blockIdx.y of a batch of cells [B][H][W] into x [B][H][W][2].
__global__ void cnn_features_kernel(const uint8_t* __restrict__ cell, int H, int W, float* __restrict__ x) {
  cell += (int64_t)blockIdx.y * H * W;
  x += (int64_t)blockIdx.y * H * W * 2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < H * W; p += gridDim.x * blockDim.x) {
    const int y = p / W, xx = p - y * W;
    const int v = cell[p] != 0;
    const int l = cell[y * W + (xx == 0 ? W - 1 : xx - 1)] != 0;
    const int r = cell[y * W + (xx == W - 1 ? 0 : xx + 1)] != 0;
    const int t = cell[(y == 0 ? H - 1 : y - 1) * W + xx] != 0;
    const int b = cell[(y == H - 1 ? 0 : y + 1) * W + xx] != 0;
    x[2 * p] = (float)v;
    x[2 * p + 1] = (float)((l != v) | (r != v) | (t != v) | (b != v));
  }
}

// ---- convolutions as implicit GEMMs on the tensor cores ------------------
//
// Operands are bfloat16 (weights as stored; activations and gradients
// rounded to nearest even when staged), products accumulate in float32 with
// mma.sync.m16n8k16.  A block owns a tile of kTH x kTW output pixels; the
// input tile with its one-pixel circular halo is staged in shared memory as
// [pixel][channel] rows (channel counts padded to multiples of 16, rows
// padded by 8 bf16 so that the fragment loads of 8 consecutive pixels hit
// distinct banks).

constexpr int kTH = 8, kTW = 16;                 // output tile: 8 rows of 16 pixels (one M fragment per row)
constexpr int kHalo = (kTH + 2) * (kTW + 2);     // staged input pixels
constexpr int kConvThreads = 32 * kTH;           // a warp per tile row
constexpr int kDwThreads = 32 * 9;               // a warp per tap

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                                  uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Stage the block's input tile with its circular halo: s[(ly*(kTW+2) + lx)][k]
// = bf16(in[(y0+ly-1) % H][(x0+lx-1) % W][k]) for k < C, 0 up to KC.
// With lo != null (split operand) also lo[...] = bf16(v - hi): the value as
// two bfloat16 terms, hi + lo, about 16 significant bits.
template <int KC>
__device__ __forceinline__ void stage_halo(const float* __restrict__ in, int H, int W, int C, int x0, int y0,
                                           __nv_bfloat16* s, __nv_bfloat16* lo = nullptr) {
  constexpr int KS = KC + 8;
  constexpr int KP = KC / 2;  // channel pairs
  for (int i = threadIdx.x; i < kHalo * KP; i += blockDim.x) {
    const int q = i / KP, k = 2 * (i - q * KP);
    const int ly = q / (kTW + 2), lx = q - ly * (kTW + 2);
    int gy = (y0 + ly - 1) % H; if (gy < 0) gy += H;
    int gx = (x0 + lx - 1) % W; if (gx < 0) gx += W;
    const float* src = in + ((int64_t)gy * W + gx) * C;
    const float v0 = k < C ? src[k] : 0.0f, v1 = k + 1 < C ? src[k + 1] : 0.0f;
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    *reinterpret_cast<__nv_bfloat162*>(s + q * KS + k) = h;
    if (lo) {
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(lo + q * KS + k) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    }
  }
}

// out[p][n] = bias[n] + sum_tap sum_k in[p + off(tap)][k] * B[tap][k][n], circular.
// Forward (flip = 0): k = ci, n = co, B[tap][k][n] = w[tap][k][n] (w of shape
// [9][K][N]).  Input gradient (flip = 1, the transposed convolution): k = the
// layer's output channel, n = its input channel, B[tap][k][n] = w[8 - tap][n][k]
// (w of shape [9][N][K]).  Optional ReLU; optional mask: out = 0 where
// mask[p][n] <= 0 (the ReLU derivative of the layer input).  K <= KC, N <= NC.
// A block stages the weights once and then takes output tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ... of n_snap snapshots (tile t is
// tile t mod tiles-per-snapshot of snapshot t / tiles-per-snapshot; in, out
// and mask advance by in_stride, out_stride and out_stride floats per
// snapshot).
template <int KC, int NC, bool SPLIT>
__global__ void __launch_bounds__(kConvThreads) cnn_conv_mma_kernel(const float* __restrict__ in, int H, int W,
                                                                    int K, int N, const __nv_bfloat16* __restrict__ w,
                                                                    int flip, const float* __restrict__ bias,
                                                                    int relu, const float* __restrict__ mask,
                                                                    float* __restrict__ out, int64_t in_stride,
                                                                    int64_t out_stride, int n_snap) {
  constexpr int KS = KC + 8;
  extern __shared__ __align__(16) __nv_bfloat16 csm[];
  __nv_bfloat16* s_in = csm;                 // [kHalo][KS]
  __nv_bfloat16* s_w = csm + kHalo * KS;     // [9][NC][KS]  (n rows, k contiguous)
  __nv_bfloat16* s_lo = s_w + 9 * NC * KS;   // SPLIT: [kHalo][KS], the input's low bfloat16 terms
  for (int i = threadIdx.x; i < 9 * NC * KC; i += blockDim.x) {
    const int k = i % KC, r = i / KC;
    const int n = r % NC, tap = r / NC;
    float v = 0.0f;
    if (k < K && n < N)
      v = flip ? __bfloat162float(w[((int64_t)(8 - tap) * N + n) * K + k])
               : __bfloat162float(w[((int64_t)tap * K + k) * N + n]);
    s_w[r * KS + k] = __float2bfloat16(v);
  }
  const int tiles_x = (W + kTW - 1) / kTW, per_snap = tiles_x * ((H + kTH - 1) / kTH);
  for (int t = blockIdx.x; t < per_snap * n_snap; t += gridDim.x) {
    const int z = t / per_snap, tr = t - z * per_snap;
    const int x0 = (tr % tiles_x) * kTW, y0 = (tr / tiles_x) * kTH;
    __syncthreads();  // the previous tile's reads of s_in are done
    stage_halo<KC>(in + z * in_stride, H, W, K, x0, y0, s_in, SPLIT ? s_lo : nullptr);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[NC / 8][4];
#pragma unroll
    for (int f = 0; f < NC / 8; ++f) {
      const int n = f * 8 + tig * 2;
      const float b0 = (bias && n < N) ? bias[n] : 0.0f, b1 = (bias && n + 1 < N) ? bias[n + 1] : 0.0f;
      acc[f][0] = b0; acc[f][1] = b1; acc[f][2] = b0; acc[f][3] = b1;
    }
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap - dy * 3;
      // A rows: the 16 output pixels of tile row `warp`, shifted by the tap
      const __nv_bfloat16* arow = s_in + ((warp + dy) * (kTW + 2) + dx) * KS;
      const __nv_bfloat16* brow = s_w + tap * NC * KS;
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        const int kc = kk * 16 + tig * 2;
        const uint32_t a0 = *reinterpret_cast<const uint32_t*>(arow + gid * KS + kc);
        const uint32_t a1 = *reinterpret_cast<const uint32_t*>(arow + (gid + 8) * KS + kc);
        const uint32_t a2 = *reinterpret_cast<const uint32_t*>(arow + gid * KS + kc + 8);
        const uint32_t a3 = *reinterpret_cast<const uint32_t*>(arow + (gid + 8) * KS + kc + 8);
        uint32_t l0 = 0, l1 = 0, l2 = 0, l3 = 0;
        if constexpr (SPLIT) {
          const __nv_bfloat16* lrow = arow - s_in + s_lo;
          l0 = *reinterpret_cast<const uint32_t*>(lrow + gid * KS + kc);
          l1 = *reinterpret_cast<const uint32_t*>(lrow + (gid + 8) * KS + kc);
          l2 = *reinterpret_cast<const uint32_t*>(lrow + gid * KS + kc + 8);
          l3 = *reinterpret_cast<const uint32_t*>(lrow + (gid + 8) * KS + kc + 8);
        }
#pragma unroll
        for (int f = 0; f < NC / 8; ++f) {
          const __nv_bfloat16* bn = brow + (f * 8 + gid) * KS + kc;
          const uint32_t b0 = *reinterpret_cast<const uint32_t*>(bn), b1 = *reinterpret_cast<const uint32_t*>(bn + 8);
          mma_bf16(acc[f], a0, a1, a2, a3, b0, b1);
          if constexpr (SPLIT) mma_bf16(acc[f], l0, l1, l2, l3, b0, b1);
        }
      }
    }
    const int py = y0 + warp;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int px = x0 + gid + 8 * h;
      if (py >= H || px >= W) continue;
      const int64_t p = (int64_t)py * W + px;
#pragma unroll
      for (int f = 0; f < NC / 8; ++f)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int n = f * 8 + tig * 2 + e;
          if (n >= N) continue;
          float v = acc[f][2 * h + e];
          if (relu) v = fmaxf(v, 0.0f);
          if (mask && !(mask[z * out_stride + p * N + n] > 0.0f)) v = 0.0f;
          out[z * out_stride + p * N + n] = v;
        }
    }
  }
}

// Weight and bias gradients of one layer, per block (partial sums over the
// block's output tile): part[blk][tap][ci][co] = sum_p in[p + off(tap)][ci] *
// g[p][co] and part_b[blk][co] = sum_p g[p][co].  GEMM per tap with M = ci,
// N = co, K = the tile's pixels; warp t computes tap t.  Pixels outside the
// image contribute nothing (their gradient rows are staged as zeros).
// blockIdx.z selects a snapshot (in and g advance by in_stride, g_stride
// floats); its tiles' partials follow those of the snapshots before it.
template <int KC, int NC>
__global__ void __launch_bounds__(kDwThreads) cnn_dw_mma_kernel(const float* __restrict__ in,
                                                                const float* __restrict__ g, int H, int W, int CIN,
                                                                int COUT, float* __restrict__ part,
                                                                float* __restrict__ part_b, int64_t in_stride,
                                                                int64_t g_stride) {
  in += blockIdx.z * in_stride;
  g += blockIdx.z * g_stride;
  constexpr int KS = KC + 8, NS = NC + 8;
  extern __shared__ __align__(16) __nv_bfloat16 csm[];
  __nv_bfloat16* s_in = csm;                          // [kHalo][KS]
  __nv_bfloat16* s_g = csm + kHalo * KS;              // [kTH * kTW][NS], gradient high terms
  __nv_bfloat16* s_gl = s_g + kTH * kTW * NS;         // and low terms (the gradient as hi + lo)
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
  const int blk = ((int)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  stage_halo<KC>(in, H, W, CIN, x0, y0, s_in);
  for (int i = threadIdx.x; i < kTH * kTW * (NC / 2); i += blockDim.x) {
    const int q = i / (NC / 2), n = 2 * (i - q * (NC / 2));
    const int py = y0 + q / kTW, px = x0 + q % kTW;
    float v0 = 0.0f, v1 = 0.0f;
    if (py < H && px < W) {
      const float* src = g + ((int64_t)py * W + px) * COUT;
      v0 = n < COUT ? src[n] : 0.0f;
      v1 = n + 1 < COUT ? src[n + 1] : 0.0f;
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162*>(s_g + q * NS + n) = h;
    *reinterpret_cast<__nv_bfloat162*>(s_gl + q * NS + n) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
  }
  // bias partial: fixed order over the tile's pixels (float32, no rounding)
  if ((int)threadIdx.x < COUT) {
    float sb = 0.0f;
    for (int q = 0; q < kTH * kTW; ++q) {
      const int py = y0 + q / kTW, px = x0 + q % kTW;
      if (py < H && px < W) sb += g[((int64_t)py * W + px) * COUT + threadIdx.x];
    }
    part_b[(int64_t)blk * COUT + threadIdx.x] = sb;
  }
  __syncthreads();
  const int tap = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dy = tap / 3, dx = tap - dy * 3;
  float acc[KC / 16][NC / 8][4];
#pragma unroll
  for (int m = 0; m < KC / 16; ++m)
#pragma unroll
    for (int f = 0; f < NC / 8; ++f)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[m][f][e] = 0.0f;
  // ldmatrix row addresses: lane L serves matrix L/8, row L%8
  const int mat = lane >> 3, row = lane & 7;
#pragma unroll 1
  for (int r = 0; r < kTH; ++r) {  // K step: the 16 pixels of tile row r
    const __nv_bfloat16* arow = s_in + ((r + dy) * (kTW + 2) + dx) * KS;  // pixel k of the step -> arow + k*KS
    const __nv_bfloat16* grow = s_g + (r * kTW) * NS;
    const __nv_bfloat16* glow = s_gl + (r * kTW) * NS;
    uint32_t b[NC / 8][2], bl[NC / 8][2];
    if constexpr (NC >= 16) {
#pragma unroll
      for (int f = 0; f < NC / 8; f += 2) {
        // matrices: (k 0-7, n f), (k 8-15, n f), (k 0-7, n f+1), (k 8-15, n f+1)
        const int k = row + ((mat & 1) ? 8 : 0), n = (f + (mat >> 1)) * 8;
        ldmatrix_x4_trans(smem_addr(grow + k * NS + n), b[f][0], b[f][1], b[f + 1][0], b[f + 1][1]);
        ldmatrix_x4_trans(smem_addr(glow + k * NS + n), bl[f][0], bl[f][1], bl[f + 1][0], bl[f + 1][1]);
      }
    } else {
      const int k = row + ((mat & 1) ? 8 : 0);
      ldmatrix_x2_trans(smem_addr(grow + k * NS), b[0][0], b[0][1]);
      ldmatrix_x2_trans(smem_addr(glow + k * NS), bl[0][0], bl[0][1]);
    }
#pragma unroll
    for (int m = 0; m < KC / 16; ++m) {
      // A[m = ci][k = pixel] from s_in[pixel][ci]: matrices (ci 0-7, k 0-7),
      // (ci 8-15, k 0-7), (ci 0-7, k 8-15), (ci 8-15, k 8-15)
      const int k = row + ((mat >> 1) ? 8 : 0), c = m * 16 + ((mat & 1) ? 8 : 0);
      uint32_t a0, a1, a2, a3;
      ldmatrix_x4_trans(smem_addr(arow + k * KS + c), a0, a1, a2, a3);
#pragma unroll
      for (int f = 0; f < NC / 8; ++f) {
        mma_bf16(acc[m][f], a0, a1, a2, a3, b[f][0], b[f][1]);
        mma_bf16(acc[m][f], a0, a1, a2, a3, bl[f][0], bl[f][1]);
      }
    }
  }
  const int gid = lane >> 2, tig = lane & 3;
  float* dst = part + ((int64_t)blk * 9 + tap) * CIN * COUT;
#pragma unroll
  for (int m = 0; m < KC / 16; ++m)
#pragma unroll
    for (int f = 0; f < NC / 8; ++f)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int ci = m * 16 + gid + (e >= 2 ? 8 : 0), co = f * 8 + tig * 2 + (e & 1);
        if (ci < CIN && co < COUT) dst[ci * COUT + co] = acc[m][f][e];
      }
}

// Reduction of the per-tile gradient partials, deterministic and with the
// same additions as reducing the snapshots one by one:
// s[z][i] = sum over the tiles b of snapshot z of part[z][b][i], tiles in
// order (snapshot blockIdx.y; sixteen loads in flight, added in order) ...
__global__ void cnn_reduce_tiles_kernel(const float* __restrict__ part, int n_blk, int n, float* __restrict__ s) {
  const int z = blockIdx.y;
  const float* pz = part + (int64_t)z * n_blk * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    int b = 0;
    for (; b + 16 <= n_blk; b += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = pz[(int64_t)(b + u) * n + i];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc += v[u];
    }
    for (; b < n_blk; ++b) acc += pz[(int64_t)b * n + i];
    s[(int64_t)z * n + i] = acc;
  }
}

// ... then dst[i] = s[0][i] (or dst[i] + s[0][i] when accumulating), then
// dst[i] + s[1][i], ... in snapshot order.
__global__ void cnn_reduce_snaps_kernel(const float* __restrict__ s, int n_snap, int n, float* __restrict__ dst,
                                        int accumulate) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float d = accumulate ? dst[i] : 0.0f;
    for (int z = 0; z < n_snap; ++z) d = (z == 0 && !accumulate) ? s[(int64_t)z * n + i] : d + s[(int64_t)z * n + i];
    dst[i] = d;
  }
}

// g[idx] += v for one contribution per lane, deterministically: lanes with the
// same index are combined by their lowest lane, in lane order.
__device__ __forceinline__ void warp_scatter_add(float* __restrict__ g, int idx, float v, bool active) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  const unsigned peers = __match_any_sync(0xffffffffu, active ? idx : -1) & act;
  const int lane = threadIdx.x & 31;
  float sum = 0.0f;
  for (unsigned m = peers; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    sum += __shfl_sync(peers, v, src);
  }
  if (active && lane == __ffs(peers) - 1) g[idx] += sum;
  __syncwarp();
}

// Warp sum in a fixed tree order.
__device__ __forceinline__ float warp_fsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_fmax(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Loss of snapshot blockIdx.x and dL/d out (two pixels per candidate), one
// warp: candidates in chunks of 32 (lane = candidate), chunks in order
// (deterministic).  out and g are [B][npix][2], pairs [B][n][2], y [B][n];
// g must be zeroed beforehand; loss[z] receives the snapshot's loss.
__global__ void cnn_loss_kernel(const float* __restrict__ out, int npix, const int32_t* __restrict__ pairs,
                                const float* __restrict__ y, int n, float* __restrict__ g, float* __restrict__ loss) {
  if (threadIdx.x >= 32) return;
  const int z = blockIdx.x;
  out += (int64_t)z * npix * 2;
  g += (int64_t)z * npix * 2;
  pairs += (int64_t)z * n * 2;
  y += (int64_t)z * n;
  const int lane = threadIdx.x;
  float l = 0.0f;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const bool on = i < n;
    int a = 0, b = 0;
    float r = 0.0f;
    if (on) {
      a = pairs[2 * i];
      b = pairs[2 * i + 1];
      r = out[2 * a + 1] + out[2 * b] - y[i];
    }
    l += warp_fsum(on ? 0.5f * r * r : 0.0f);
    warp_scatter_add(g, 2 * a + 1, r / n, on);
    warp_scatter_add(g, 2 * b, r / n, on);
  }
  if (lane == 0) loss[z] = l / n;
}

// Listwise loss of one snapshot: L = logsumexp(s) - sum_i q_i s_i with
// s_i = s1[a_i] + s0[b_i] and q = softmax(y / beta); dL/ds_i = p_i - q_i on
// both pixels of candidate i.  One warp per snapshot (blockIdx.x; layouts as
// cnn_loss_kernel), fixed reduction order (deterministic).
__global__ void cnn_listwise_kernel(const float* __restrict__ out, int npix, const int32_t* __restrict__ pairs,
                                    const float* __restrict__ y, int n, float beta, float* __restrict__ g,
                                    float* __restrict__ loss) {
  if (threadIdx.x >= 32) return;
  const int z = blockIdx.x;
  out += (int64_t)z * npix * 2;
  g += (int64_t)z * npix * 2;
  pairs += (int64_t)z * n * 2;
  y += (int64_t)z * n;
  const int lane = threadIdx.x;
  float smax = -3.0e38f, ymax = -3.0e38f;
  for (int i = lane; i < n; i += 32) {
    smax = fmaxf(smax, out[2 * pairs[2 * i] + 1] + out[2 * pairs[2 * i + 1]]);
    ymax = fmaxf(ymax, y[i] / beta);
  }
  smax = warp_fmax(smax);
  ymax = warp_fmax(ymax);
  float zs = 0.0f, zq = 0.0f;
  for (int i = lane; i < n; i += 32) {
    zs += expf(out[2 * pairs[2 * i] + 1] + out[2 * pairs[2 * i + 1]] - smax);
    zq += expf(y[i] / beta - ymax);
  }
  zs = warp_fsum(zs);
  zq = warp_fsum(zq);
  float lq = 0.0f;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const bool on = i < n;
    int a = 0, b = 0;
    float d = 0.0f;
    if (on) {
      a = pairs[2 * i];
      b = pairs[2 * i + 1];
      const float si = out[2 * a + 1] + out[2 * b];
      const float pi = expf(si - smax) / zs, qi = expf(y[i] / beta - ymax) / zq;
      lq += qi * si;
      d = pi - qi;
    }
    warp_scatter_add(g, 2 * a + 1, d, on);
    warp_scatter_add(g, 2 * b, d, on);
  }
  lq = warp_fsum(lq);
  if (lane == 0) loss[z] = smax + logf(zs) - lq;
}

// *total += loss[z] * scale for the snapshots in order (one thread).
__global__ void cnn_add_losses_kernel(const float* __restrict__ loss, int n_snap, float scale,
                                      float* __restrict__ total) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int z = 0; z < n_snap; ++z) *total += loss[z] * scale;
}

__global__ void cnn_to_bf16_kernel(const float* __restrict__ m, int n, __nv_bfloat16* __restrict__ w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w[i] = __float2bfloat16(m[i]);
}

// Adam (Kingma & Ba) on the float32 master parameters, then bfloat16 copies.
__global__ void cnn_adam_kernel(float* __restrict__ m, float* __restrict__ v, float* __restrict__ p,
                                const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                                float c2, float gscale, __nv_bfloat16* __restrict__ wbf, const int* __restrict__ is_w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (is_w[i] >= 0) wbf[is_w[i]] = __float2bfloat16(pi);
  }
}

}  // namespace lpf

struct lpf_cnn {
  int H = 0, W = 0;
  int64_t n_params = 0;
  int64_t w_off[lpf::kLayers] = {}, b_off[lpf::kLayers] = {};  // offsets in the parameter vector
  int64_t wb_off[lpf::kLayers] = {};                             // offsets in the bf16 weight array
  float* d_p = nullptr;       // master parameters
  float* d_m = nullptr;       // Adam first moment
  float* d_v = nullptr;       // Adam second moment
  float* d_g = nullptr;       // gradient accumulator
  __nv_bfloat16* d_wbf = nullptr;
  int* d_isw = nullptr;       // parameter index -> bf16 index (or -1 for biases)
  float* d_act[lpf::kLayers + 1] = {};  // activations of the scored cell [H][W][C_l] (fixed at creation)
  // Training: activations, gradients and partials for up to `cap` snapshots
  // at once (allocated by the first training call, grown, never moved
  // under the scoring buffers above, which captured graphs may hold).
  int cap = 0;
  float* d_tact[lpf::kLayers + 1] = {};  // [cap][H][W][C_l]
  float* d_gact = nullptr;    // gradient buffers (two, ping-pong) [cap][H][W][64]
  float* d_gact2 = nullptr;
  float* d_part = nullptr;    // per-block weight-gradient partials [cap][blocks][9 * 64 * 64]
  float* d_part_b = nullptr;  // per-block bias-gradient partials [cap][blocks][64]
  float* d_loss = nullptr;    // per-snapshot losses [cap]
  float* d_snap = nullptr;    // per-snapshot gradient sums [cap][9 * 64 * 64]
  int n_blk = 0;              // output tiles (blocks) of a convolution
  int64_t step = 0;
  int loss_kind = 0;          // 0: squared error, 1: listwise cross-entropy
  float beta = 1.0f;          // listwise target temperature
};

namespace lpf {

// Buffers for nb snapshots at once (grown, never shrunk; synchronises the
// device when it grows).
constexpr int kTrainChunk = 8;  // snapshots per batched forward/backward
static int cnn_reserve(lpf_cnn* c, int nb) {
  if (nb <= c->cap) return LPF_OK;
  cudaDeviceSynchronize();
  for (int l = 0; l <= kLayers; ++l) { cudaFree(c->d_tact[l]); c->d_tact[l] = nullptr; }
  cudaFree(c->d_gact); cudaFree(c->d_gact2); cudaFree(c->d_part); cudaFree(c->d_part_b); cudaFree(c->d_loss);
  cudaFree(c->d_snap);
  c->d_gact = c->d_gact2 = c->d_part = c->d_part_b = c->d_loss = c->d_snap = nullptr;
  c->cap = 0;
  const size_t npix = (size_t)c->H * c->W, b = (size_t)nb;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l <= kLayers && e == cudaSuccess; ++l) e = cudaMalloc(&c->d_tact[l], b * npix * kCh[l] * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gact, b * npix * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gact2, b * npix * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_part, b * c->n_blk * 9 * 64 * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_part_b, b * c->n_blk * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_loss, b * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_snap, b * 9 * 64 * 64 * 4);
  if (e != cudaSuccess) return set_cuda_error(e);
  c->cap = nb;
  return LPF_OK;
}

static int cnn_alloc(lpf_cnn* c) {
  int64_t off = 0, woff = 0;
  for (int l = 0; l < kLayers; ++l) {
    c->w_off[l] = off;
    off += layer_w_size(l);
    c->b_off[l] = off;
    off += kCh[l + 1];
    c->wb_off[l] = woff;
    woff += layer_w_size(l);
  }
  c->n_params = off;
  const size_t np = (size_t)off;
  const size_t npix = (size_t)c->H * c->W;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&c->d_p, np * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_m, np * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_v, np * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_g, np * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_wbf, (size_t)woff * 2);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_isw, np * 4);
  c->n_blk = ((c->W + kTW - 1) / kTW) * ((c->H + kTH - 1) / kTH);
  for (int l = 0; l <= kLayers && e == cudaSuccess; ++l) e = cudaMalloc(&c->d_act[l], npix * kCh[l] * 4);
  if (e == cudaSuccess) e = cudaMemset(c->d_m, 0, np * 4);
  if (e == cudaSuccess) e = cudaMemset(c->d_v, 0, np * 4);
  if (e != cudaSuccess) return set_cuda_error(e);
  std::vector<int> isw(np, -1);
  for (int l = 0; l < kLayers; ++l)
    for (int i = 0; i < layer_w_size(l); ++i) isw[c->w_off[l] + i] = (int)(c->wb_off[l] + i);
  e = cudaMemcpy(c->d_isw, isw.data(), np * 4, cudaMemcpyHostToDevice);
  return set_cuda_error(e);
}

static void cnn_sync_bf16(lpf_cnn* c, cudaStream_t s) {
  for (int l = 0; l < kLayers; ++l)
    cnn_to_bf16_kernel<<<64, 256, 0, s>>>(c->d_p + c->w_off[l], layer_w_size(l), c->d_wbf + c->wb_off[l]);
}

template <int KC, int NC, bool SPLIT>
static size_t conv_smem() { return (size_t)((SPLIT ? 2 : 1) * kHalo * (KC + 8) + 9 * NC * (KC + 8)) * 2; }
template <int KC, int NC>
static size_t dw_smem() { return (size_t)(kHalo * (KC + 8) + 2 * kTH * kTW * (NC + 8)) * 2; }

// Blocks of a convolution launch: every output tile of the nb snapshots, at
// most the blocks that fit on the GPU at once (each then loops over tiles).
template <int KC, int NC, bool SPLIT>
static int conv_blocks(int tiles) {
  static int resident = 0;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cnn_conv_mma_kernel<KC, NC, SPLIT>, kConvThreads,
                                                  conv_smem<KC, NC, SPLIT>());
    resident = std::max(1, per_sm) * std::max(1, sms);
  }
  return std::max(1, std::min(tiles, resident));
}

// flip = 1 (the input gradient) carries the incoming gradient as two bfloat16 terms.
template <int KC, int NC>
static void conv_mma(const float* in, int H, int W, int K, int N, const __nv_bfloat16* w, int flip,
                     const float* bias, int relu, const float* mask, float* out, int nb, cudaStream_t s) {
  const int tiles = ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH) * nb;
  const int64_t in_stride = (int64_t)H * W * K, out_stride = (int64_t)H * W * N;
  static bool attr[2] = {false, false};  // dynamic shared memory above 48 KB must be allowed once per kernel
  if (flip) {
    const size_t smem = conv_smem<KC, NC, true>();
    if (!attr[1]) {
      cudaFuncSetAttribute(cnn_conv_mma_kernel<KC, NC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr[1] = true;
    }
    cnn_conv_mma_kernel<KC, NC, true><<<conv_blocks<KC, NC, true>(tiles), kConvThreads, smem, s>>>(
        in, H, W, K, N, w, flip, bias, relu, mask, out, in_stride, out_stride, nb);
  } else {
    const size_t smem = conv_smem<KC, NC, false>();
    if (!attr[0]) {
      cudaFuncSetAttribute(cnn_conv_mma_kernel<KC, NC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      attr[0] = true;
    }
    cnn_conv_mma_kernel<KC, NC, false><<<conv_blocks<KC, NC, false>(tiles), kConvThreads, smem, s>>>(
        in, H, W, K, N, w, flip, bias, relu, mask, out, in_stride, out_stride, nb);
  }
}

// Convolution with K input and N output channels of the GEMM (see the kernel).
static void conv_any(int K, int N, const float* in, int H, int W, const __nv_bfloat16* w, int flip,
                     const float* bias, int relu, const float* mask, float* out, int nb, cudaStream_t s) {
  const int key = K * 1000 + N;
  switch (key) {
    // forward layers
    case 2 * 1000 + 32: conv_mma<16, 32>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 32 * 1000 + 64: conv_mma<32, 64>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 64 * 1000 + 48: conv_mma<64, 48>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 48 * 1000 + 32: conv_mma<48, 32>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 32 * 1000 + 2: conv_mma<32, 8>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    // transposed (input gradients of layers 1..4)
    case 64 * 1000 + 32: conv_mma<64, 32>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 48 * 1000 + 64: conv_mma<48, 64>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    case 32 * 1000 + 48: conv_mma<32, 48>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;
    default: conv_mma<16, 32>(in, H, W, K, N, w, flip, bias, relu, mask, out, nb, s); break;  // 2 -> 32
  }
}

template <int KC, int NC>
static void dw_mma(const float* in, const float* g, int H, int W, int CIN, int COUT, float* part, float* part_b,
                   int nb, cudaStream_t s) {
  const size_t smem = dw_smem<KC, NC>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(cnn_dw_mma_kernel<KC, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, nb);
  cnn_dw_mma_kernel<KC, NC><<<grid, kDwThreads, smem, s>>>(in, g, H, W, CIN, COUT, part, part_b,
                                                            (int64_t)H * W * CIN, (int64_t)H * W * COUT);
}

static void dw_any(int CIN, int COUT, const float* in, const float* g, int H, int W, float* part, float* part_b,
                   int nb, cudaStream_t s) {
  switch (CIN * 1000 + COUT) {
    case 2 * 1000 + 32: dw_mma<16, 32>(in, g, H, W, CIN, COUT, part, part_b, nb, s); break;
    case 32 * 1000 + 64: dw_mma<32, 64>(in, g, H, W, CIN, COUT, part, part_b, nb, s); break;
    case 64 * 1000 + 48: dw_mma<64, 48>(in, g, H, W, CIN, COUT, part, part_b, nb, s); break;
    case 48 * 1000 + 32: dw_mma<48, 32>(in, g, H, W, CIN, COUT, part, part_b, nb, s); break;
    default: dw_mma<32, 8>(in, g, H, W, CIN, COUT, part, part_b, nb, s); break;  // 32 -> 2
  }
}

// Forward pass of nb cells [nb][H][W] into act (room for nb snapshots).
static void cnn_forward_batch(lpf_cnn* c, const uint8_t* cells, int nb, float* const* act, cudaStream_t s) {
  const int npix = c->H * c->W;
  cnn_features_kernel<<<dim3((npix + 255) / 256, nb), 256, 0, s>>>(cells, c->H, c->W, act[0]);
  for (int l = 0; l < kLayers; ++l)
    conv_any(kCh[l], kCh[l + 1], act[l], c->H, c->W, c->d_wbf + c->wb_off[l], 0, c->d_p + c->b_off[l],
             l < kLayers - 1, nullptr, act[l + 1], nb, s);
}

// Scores of one cell into the scoring buffers.
void cnn_forward(lpf_cnn* c, const uint8_t* cell, cudaStream_t s) { cnn_forward_batch(c, cell, 1, c->d_act, s); }

// Forward, loss and backward of nb snapshots in one set of launches (their
// tiles side by side in each grid); their gradients are added into d_g in
// snapshot order (written first when accumulate == 0) and their losses,
// times loss_scale, into *loss_dev (when not null) in the same order -- the
// same additions as running the snapshots one after another.
static int cnn_fwd_bwd(lpf_cnn* c, const uint8_t* cells, int nb, const int32_t* pairs, const float* y, int n,
                       int accumulate, float* loss_dev, float loss_scale, cudaStream_t s) {
  const int H = c->H, W = c->W, npix = H * W;
  int rc = cnn_reserve(c, nb);
  if (rc) return rc;
  cnn_forward_batch(c, cells, nb, c->d_tact, s);
  float* g = c->d_gact;
  float* g2 = c->d_gact2;
  cudaMemsetAsync(g, 0, (size_t)nb * npix * kCh[kLayers] * 4, s);
  if (c->loss_kind == 1)
    cnn_listwise_kernel<<<nb, 32, 0, s>>>(c->d_tact[kLayers], npix, pairs, y, n, c->beta, g, c->d_loss);
  else
    cnn_loss_kernel<<<nb, 32, 0, s>>>(c->d_tact[kLayers], npix, pairs, y, n, g, c->d_loss);
  if (loss_dev) cnn_add_losses_kernel<<<1, 1, 0, s>>>(c->d_loss, nb, loss_scale, loss_dev);
  for (int l = kLayers - 1; l >= 0; --l) {
    const int cin = kCh[l], cout = kCh[l + 1];
    // g = dL/d(pre-activation output of layer l) here (ReLU mask already applied)
    dw_any(cin, cout, c->d_tact[l], g, H, W, c->d_part, c->d_part_b, nb, s);
    const int nw_l = 9 * cin * cout;
    cnn_reduce_tiles_kernel<<<dim3((nw_l + 255) / 256, nb), 256, 0, s>>>(c->d_part, c->n_blk, nw_l, c->d_snap);
    cnn_reduce_snaps_kernel<<<(nw_l + 255) / 256, 256, 0, s>>>(c->d_snap, nb, nw_l, c->d_g + c->w_off[l], accumulate);
    cnn_reduce_tiles_kernel<<<dim3(1, nb), 64, 0, s>>>(c->d_part_b, c->n_blk, cout, c->d_snap);
    cnn_reduce_snaps_kernel<<<1, 64, 0, s>>>(c->d_snap, nb, cout, c->d_g + c->b_off[l], accumulate);
    if (l > 0) {
      // dL/d act[l] = transposed conv of g, then times the ReLU mask of act[l]
      conv_any(cout, cin, g, H, W, c->d_wbf + c->wb_off[l], 1, nullptr, 0, c->d_tact[l], g2, nb, s);
      std::swap(g, g2);
    }
  }
  return LPF_OK;
}

const float* cnn_scores(const lpf_cnn* c) { return c->d_act[kLayers]; }
bool cnn_matches(const lpf_cnn* c, int H, int W) { return c && c->H == H && c->W == W; }

}  // namespace lpf

extern "C" {

int lpf_cnn_set_loss(lpf_cnn* cnn, int32_t kind, float beta) {
  if (!cnn || (kind != 0 && kind != 1) || !(beta > 0.0f)) return LPF_EINVAL;
  cnn->loss_kind = kind;
  cnn->beta = beta;
  return LPF_OK;
}

int lpf_cnn_create(int32_t H, int32_t W, uint64_t seed, lpf_cnn** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (H < 3 || W < 3 || (int64_t)H * W > (1 << 22)) return LPF_EINVAL;
  lpf_cnn* c = new (std::nothrow) lpf_cnn();
  if (!c) return LPF_ENOMEM;
  c->H = H;
  c->W = W;
  int rc = lpf::cnn_alloc(c);
  if (rc) { lpf_cnn_free(c); return rc; }
  // He-normal weights (std sqrt(2 / (9 Cin))), zero biases
  std::mt19937_64 gen(seed);
  std::vector<float> p((size_t)c->n_params, 0.0f);
  for (int l = 0; l < lpf::kLayers; ++l) {
    std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (9.0f * lpf::kCh[l])));
    for (int i = 0; i < lpf::layer_w_size(l); ++i) p[c->w_off[l] + i] = nd(gen);
  }
  rc = lpf_cnn_set_params(c, p.data(), c->n_params);
  if (rc) { lpf_cnn_free(c); return rc; }
  *out = c;
  return LPF_OK;
}

int64_t lpf_cnn_num_params(const lpf_cnn* c) { return c ? c->n_params : -1; }

int lpf_cnn_set_params(lpf_cnn* c, const float* host, int64_t n) {
  if (!c || !host || n != c->n_params) return LPF_EINVAL;
  cudaError_t e = cudaMemcpy(c->d_p, host, (size_t)n * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  lpf::cnn_sync_bf16(c, 0);
  e = cudaDeviceSynchronize();
  return lpf::set_cuda_error(e == cudaSuccess ? cudaGetLastError() : e);
}

int lpf_cnn_get_params(const lpf_cnn* c, float* host, int64_t n) {
  if (!c || !host || n != c->n_params) return LPF_EINVAL;
  return lpf::set_cuda_error(cudaMemcpy(host, c->d_p, (size_t)n * 4, cudaMemcpyDeviceToHost));
}

int lpf_cnn_forward(lpf_cnn* c, const uint8_t* cell_dev, float* scores_dev, lpf_stream_t stream) {
  if (!c || !cell_dev) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  lpf::cnn_forward(c, cell_dev, s);
  if (scores_dev)
    cudaMemcpyAsync(scores_dev, c->d_act[lpf::kLayers], (size_t)c->H * c->W * 2 * 4, cudaMemcpyDeviceToDevice, s);
  return lpf::set_cuda_error(cudaGetLastError());
}

int lpf_cnn_gradients(lpf_cnn* c, const uint8_t* cell_dev, const int32_t* pairs_dev, const float* y_dev, int32_t n,
                      float* grads_dev, float* loss_dev, lpf_stream_t stream) {
  if (!c || !cell_dev || !pairs_dev || !y_dev || n < 1) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  if (loss_dev) cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
  const int rc = lpf::cnn_fwd_bwd(c, cell_dev, 1, pairs_dev, y_dev, n, 0, loss_dev, 1.0f, s);
  if (rc) return rc;
  if (grads_dev) cudaMemcpyAsync(grads_dev, c->d_g, (size_t)c->n_params * 4, cudaMemcpyDeviceToDevice, s);
  return lpf::set_cuda_error(cudaGetLastError());
}

int lpf_cnn_train_step(lpf_cnn* c, const uint8_t* cells_dev, int32_t B, const int32_t* pairs_dev,
                       const float* y_dev, int32_t n, float lr, float* loss_dev, lpf_stream_t stream) {
  if (!c || !cells_dev || !pairs_dev || !y_dev || B < 1 || n < 1 || !(lr > 0.0f)) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  if (loss_dev) cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
  const size_t npix = (size_t)c->H * c->W;
  for (int b0 = 0; b0 < B; b0 += lpf::kTrainChunk) {
    const int nb = std::min(B - b0, lpf::kTrainChunk);
    const int rc = lpf::cnn_fwd_bwd(c, cells_dev + b0 * npix, nb, pairs_dev + (size_t)b0 * n * 2,
                                    y_dev + (size_t)b0 * n, n, b0 > 0, loss_dev, 1.0f / B, s);
    if (rc) return rc;
  }
  c->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)c->step), c2 = 1.0f - std::pow(b2, (float)c->step);
  const int n_p = (int)c->n_params;
  lpf::cnn_adam_kernel<<<(n_p + 255) / 256, 256, 0, s>>>(c->d_m, c->d_v, c->d_p, c->d_g, n_p, lr, b1, b2, 1e-8f, c1,
                                                          c2, 1.0f / B, c->d_wbf, c->d_isw);
  return lpf::set_cuda_error(cudaGetLastError());
}

void lpf_cnn_free(lpf_cnn* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->d_p);
  cudaFree(c->d_m);
  cudaFree(c->d_v);
  cudaFree(c->d_g);
  cudaFree(c->d_wbf);
  cudaFree(c->d_isw);
  for (int l = 0; l <= lpf::kLayers; ++l) {
    cudaFree(c->d_act[l]);
    cudaFree(c->d_tact[l]);
  }
  cudaFree(c->d_gact);
  cudaFree(c->d_gact2);
  cudaFree(c->d_part);
  cudaFree(c->d_part_b);
  cudaFree(c->d_loss);
  cudaFree(c->d_snap);
  delete c;
}

}  // extern "C"
