// Two-point probability as the annealing objective (Sec. 2.1, Eq. (S2dis);
// Eq. (LSE) on S2, used for the S2-based compressions of Sec. 6).
//
// Counts.  C(d) = sum over x of chi(x) chi(x + d) (periodic), chi the phase-1
// indicator: W*H times S2 of phase 1 at offset d, an exact integer.
// s2_counts evaluates the double sum directly on bit-packed rows (each row
// stored twice in a row so that every column shift is a funnel shift).
//
// Swap change.  Exchanging a (phase 1) with b (phase 0) turns chi into
// chi - [x = a] + [x = b], and expanding the product gives, with chi taken
// before the exchange,
//   dC(d) = chi(b+d) + chi(b-d) - chi(a+d) - chi(a-d) + 2[d = 0]
//           - [d = b - a] - [d = a - b].
// A block keeps the cell in shared memory as bytes, extended periodically by
// ceil(W/2) columns and ceil(H/2) rows on each side; offsets are taken in the
// centred range dy in [-ceil(H/2), floor(H/2)), dx likewise, so a +- d and
// b +- d never leave the array.  The error change is
//   sum over d of x (x - 2 delta),  x = dC(d)/N, delta = t(d) - C(d)/N,
// in float32, summed per (candidate, row chunk) in a fixed order (each
// thread in its offset order, a shuffle tree per warp, warps in order) and
// then over chunks in chunk order: bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <new>

#include "../../include/lpf.h"
#include "lpf_sa.cuh"
#include "lpf_state.hpp"

namespace lpf {

constexpr int kS2Threads = 256;
constexpr int kS2ChunkOffsets = 2048;  // offsets per block and candidate (about)

// ext[ey][ex] = img[(ey - ry) mod H][(ex - rx) mod W]; zero padding to ext_bytes.
static __global__ void s2_build_ext_kernel(const uint8_t* __restrict__ img, DeltaArgs g, uint8_t* __restrict__ ext) {
  const int total = g.We * g.He;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)g.ext_bytes; i += gridDim.x * blockDim.x) {
    uint8_t v = 0;
    if (i < total) {
      const int ey = i / g.We, ex = i - ey * g.We;
      int y = (ey - g.ry) % g.H; if (y < 0) y += g.H;
      int x = (ex - g.rx) % g.W; if (x < 0) x += g.W;
      v = img[y * g.W + x];
    }
    ext[i] = v;
  }
}

// Exchange geometry of one candidate in an extended cell.
struct S2Pair {
  int pa, pb;    // extended-cell positions of a and b
  int ey, ex;    // offset b - a (wrapped into [0,H) x [0,W))
  int fy, fx;    // offset a - b
};

__device__ __forceinline__ S2Pair s2_pair(const DeltaArgs& g, int a, int b) {
  S2Pair q;
  const int ay = a / g.W, ax = a - ay * g.W, by = b / g.W, bx = b - by * g.W;
  q.pa = (ay + g.ry) * g.We + ax + g.rx;
  q.pb = (by + g.ry) * g.We + bx + g.rx;
  q.ey = by - ay; if (q.ey < 0) q.ey += g.H;
  q.ex = bx - ax; if (q.ex < 0) q.ex += g.W;
  q.fy = q.ey ? g.H - q.ey : 0;
  q.fx = q.ex ? g.W - q.ex : 0;
  return q;
}

// dC at offset (y, x) in [0,H) x [0,W), chi read from e (values 0/1).
__device__ __forceinline__ int s2_count_change(const uint8_t* e, const DeltaArgs& g, const S2Pair& q, int y, int x) {
  const int dy = y < g.H - g.ry ? y : y - g.H;
  const int dx = x < g.W - g.rx ? x : x - g.W;
  const int o = dy * g.We + dx;
  int dc = (int)e[q.pb + o] + (int)e[q.pb - o] - (int)e[q.pa + o] - (int)e[q.pa - o];
  if ((y | x) == 0) dc += 2;
  if (y == q.ey && x == q.ex) dc -= 1;
  if (y == q.fy && x == q.fx) dc -= 1;
  return dc;
}

// Rows y0 <= y < y1 of the offsets: warps take rows, lanes columns.  Writes
// the changes (if dck, [H][W]) and returns this thread's float32 error change
// (if g.target), accumulated in its own offset order.
__device__ __forceinline__ float s2_delta_rows(const uint8_t* sm, const DeltaArgs& g, const S2Pair& q, int y0, int y1,
                                               int32_t* dck) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float invN = 1.0f / ((float)g.H * (float)g.W);
  float acc = 0.0f;
  for (int y = y0 + warp; y < y1; y += nw) {
    for (int x = lane; x < g.W; x += 32) {
      const int dc = s2_count_change(sm, g, q, y, x);
      const int i = y * g.W + x;
      if (dck) dck[i] = dc;
      if (g.target && dc) {
        const float dd = __ldg(g.target + i) - (float)__ldg(g.counts + i) * invN;
        const float xx = (float)dc * invN;
        acc += xx * (xx - 2.0f * dd);
      }
    }
  }
  return acc;
}

// Fixed-order block sum: shuffle tree per warp, then thread 0 adds the warps
// in order.  Valid in thread 0; every thread calls it.
__device__ __forceinline__ float s2_block_sum(float v, float* warp_acc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) warp_acc[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_acc[w];
  return s;
}

// Standalone swap delta: blocks = (row chunk) x (candidate stride).  A pair
// with an index out of range, or a block whose staging wait gave up, yields
// NaN partials (so NaN error changes) and no count changes are written for it.
__global__ void __launch_bounds__(kS2Threads) s2_delta_kernel(const uint8_t* __restrict__ img,
                                                               const uint8_t* __restrict__ ext, DeltaArgs g,
                                                               const int32_t* __restrict__ pairs, int K,
                                                               int32_t* __restrict__ dcounts,
                                                               float* __restrict__ partial) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ float warp_acc[32];
  __shared__ int s_a, s_b, s_skip;
  const int ch = blockIdx.x;
  if ((int)blockIdx.y >= K) return;
  const int npix = g.H * g.W;
  const int y0 = (int)((int64_t)ch * g.H / g.n_chunks), y1 = (int)((int64_t)(ch + 1) * g.H / g.n_chunks);
  const bool staged = delta_stage(sm, ext, g.ext_bytes, &bar);
  if (!staged) (void)mbar_wait(&bar, 0);  // let the copy land before the block uses or leaves it
  for (int k = blockIdx.y; k < K; k += gridDim.y) {
    if (threadIdx.x == 0) {
      int a = pairs[2 * k], b = pairs[2 * k + 1];
      int skip = 0;
      if (!staged || a < 0 || b < 0 || a >= npix || b >= npix) skip = 2;  // error
      else if (img[a] == img[b]) skip = 1;                                 // identity
      else if (img[a] == 0) { const int t = a; a = b; b = t; }             // a holds phase 1
      s_a = a; s_b = b; s_skip = skip;
    }
    __syncthreads();
    const int skip = s_skip;
    int32_t* dk = dcounts ? dcounts + (int64_t)k * npix : nullptr;
    float acc = 0.0f;
    if (skip == 0) {
      acc = s2_delta_rows(sm, g, s2_pair(g, s_a, s_b), y0, y1, dk);
    } else if (skip == 1 && dk) {
      for (int i = y0 * g.W + threadIdx.x; i < y1 * g.W; i += blockDim.x) dk[i] = 0;
    }
    const float s = s2_block_sum(acc, warp_acc);
    if (threadIdx.x == 0 && partial) partial[(int64_t)k * g.n_chunks + ch] = skip == 2 ? __int_as_float(0x7fc00000) : s;
    __syncthreads();
  }
}

// de[k] = sum over chunks of partial[k][c], in chunk order.
__global__ void s2_reduce_kernel(const float* __restrict__ partial, int n_chunks, int K, float* __restrict__ de) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < n_chunks; ++c) s += partial[(int64_t)k * n_chunks + c];
    de[k] = s;
  }
}

// One annealing batch on the S2 objective (same sequence as the lineal-path
// batch: draw, evaluate, last block accepts the first passing candidate).
__global__ void __launch_bounds__(kS2Threads) s2_batch_kernel(SaDev* __restrict__ st, uint8_t* __restrict__ cell,
                                                               uint8_t* __restrict__ ext, DeltaArgs g,
                                                               int32_t* __restrict__ pairs, float* __restrict__ u,
                                                               float* __restrict__ partial,
                                                               unsigned long long* __restrict__ counts,
                                                               int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ float warp_acc[32];
  __shared__ int s_a, s_b;
  const int ch = blockIdx.x;
  const int Keff = st->done ? 0 : st->k_eff;
  const unsigned long long n0 = (unsigned long long)st->n_eval;

  if ((int)blockIdx.y < Keff) {
    if (!delta_stage(sm, ext, g.ext_bytes, &bar)) {
      if (threadIdx.x == 0) atomicOr(status, 1);
      (void)mbar_wait(&bar, 0);
    } else {
      const int y0 = (int)((int64_t)ch * g.H / g.n_chunks), y1 = (int)((int64_t)(ch + 1) * g.H / g.n_chunks);
      for (int k = blockIdx.y; k < Keff; k += gridDim.y) {
        if (threadIdx.x < 32) {
          int a, b;
          float uu;
          draw_candidate_warp(sm, g, n0 + (unsigned long long)k, st->key0, st->key1, a, b, uu, st,
                              (int)threadIdx.x);
          if (threadIdx.x == 0) {
            if (ch == 0) { pairs[2 * k] = a; pairs[2 * k + 1] = b; u[k] = uu; }
            s_a = a;
            s_b = b;
          }
        }
        __syncthreads();
        const float acc = s_a != s_b ? s2_delta_rows(sm, g, s2_pair(g, s_a, s_b), y0, y1, nullptr) : 0.0f;
        const float s = s2_block_sum(acc, warp_acc);
        if (threadIdx.x == 0) partial[(int64_t)k * g.n_chunks + ch] = s;
        __syncthreads();
      }
    }
  }

  if (!sa_last_block(st)) return;
  __shared__ SaDev s_state;
  sa_state_load(&s_state, st);
  const long long left = s_state.n_step - s_state.n_eval;
  const int Kv = (int)min((long long)Keff, max(0LL, left));
  float de_star;
  const int kstar = sa_first_accept(&s_state, Kv, partial, g.n_chunks, u, &de_star);
  if (kstar >= 0) {
    const int a = __ldcg(pairs + 2 * kstar), b = __ldcg(pairs + 2 * kstar + 1);
    if (a != b) {
      // count changes from the extended cell before the exchange
      const S2Pair q = s2_pair(g, a, b);
      for (int y = threadIdx.x >> 5; y < g.H; y += blockDim.x >> 5)
        for (int x = threadIdx.x & 31; x < g.W; x += 32) {
          const int dc = s2_count_change(ext, g, q, y, x);
          if (dc) counts[y * g.W + x] += (unsigned long long)(long long)dc;
        }
      __syncthreads();
      if (threadIdx.x == 0) {
        const uint8_t va = cell[a];
        cell[a] = cell[b];
        cell[b] = va;
        delta_mark(ext, a, cell[a], g);
        delta_mark(ext, b, cell[b], g);
      }
    }
  }
  if (threadIdx.x == 0) sa_advance(&s_state, Keff, Kv, kstar, de_star, kstar >= 0 ? __ldcg(pairs + 2 * kstar) : 0,
                                      kstar >= 0 ? __ldcg(pairs + 2 * kstar + 1) : 0);
  sa_state_store(st, &s_state);
}

// ---- direct counts ----------------------------------------------------------

// P[y][w]: bit k of word w = chi(y, (32w + k) mod W) for 32w + k < 2W, else 0.
__global__ void s2_pack_kernel(const uint8_t* __restrict__ img, int H, int W, int Wd, uint32_t* __restrict__ P) {
  const int64_t n = (int64_t)H * Wd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / Wd), w = (int)(i - (int64_t)y * Wd);
    uint32_t word = 0;
    for (int k = 0; k < 32; ++k) {
      const int j = 32 * w + k;
      if (j < 2 * W && img[(int64_t)y * W + (j < W ? j : j - W)] == 1) word |= 1u << k;
    }
    P[i] = word;
  }
}

// C[dy][dx] = sum over y1 of popc(row y1 & (row (y1+dy) mod H shifted by dx)),
// over the W columns.  Block = one dy; threads loop over dx.
__global__ void s2_counts_kernel(const uint32_t* __restrict__ P, int H, int W, int Wd, int64_t* __restrict__ C) {
  const int dy = blockIdx.x;
  const int nw = (W + 31) / 32;
  const uint32_t last = (W & 31) ? ((1u << (W & 31)) - 1u) : 0xffffffffu;
  for (int dx = threadIdx.x; dx < W; dx += blockDim.x) {
    const int q = dx >> 5, sh = dx & 31;
    long long acc = 0;
    for (int y1 = 0; y1 < H; ++y1) {
      int y2 = y1 + dy;
      if (y2 >= H) y2 -= H;
      const uint32_t* r1 = P + (int64_t)y1 * Wd;
      const uint32_t* r2 = P + (int64_t)y2 * Wd + q;
      for (int w = 0; w < nw; ++w) {
        uint32_t m = __ldg(r1 + w);
        if (w == nw - 1) m &= last;
        const uint32_t s = __funnelshift_r(__ldg(r2 + w), __ldg(r2 + w + 1), sh);
        acc += __popc(m & s);
      }
    }
    C[(int64_t)dy * W + dx] = acc;
  }
}

// ---- host side --------------------------------------------------------------

static int g_s2_max_smem = -1;

static int s2_prepare() {
  if (g_s2_max_smem >= 0) return LPF_OK;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa, fb;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, s2_delta_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fb, s2_batch_kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(s2_delta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(s2_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fb.sharedSizeBytes);
  if (e != cudaSuccess) return set_cuda_error(e);
  g_s2_max_smem = optin - (int)std::max(fa.sharedSizeBytes, fb.sharedSizeBytes) - 64;
  return LPF_OK;
}

// Geometry of the S2 evaluation for an H x W cell (row chunks of about
// kS2ChunkOffsets offsets); false if the extended cell does not fit.
static bool s2_geometry(int H, int W, DeltaArgs& g) {
  g = DeltaArgs{};
  g.H = H;
  g.W = W;
  g.rx = (W + 1) / 2;
  g.ry = (H + 1) / 2;
  g.We = W + 2 * g.rx;
  g.He = H + 2 * g.ry;
  g.ext_bytes = (uint32_t)((((size_t)g.We * g.He) + 15) & ~size_t(15));
  const int64_t npix = (int64_t)H * W;
  g.n_chunks = (int)std::max<int64_t>(1, std::min<int64_t>(H, (npix + kS2ChunkOffsets - 1) / kS2ChunkOffsets));
  g.n_canon = npix;
  g.n_full = npix;
  g.base = 0;
  g.phase_mask = 1;
  return (int64_t)g.ext_bytes <= g_s2_max_smem;
}

int s2_delta_run(const uint8_t* img, int H, int W, const uint8_t* ext, const int32_t* pairs, int K, int32_t* dcounts,
                 const float* target, const int64_t* counts, float* de, float* partial, cudaStream_t s) {
  int rc = s2_prepare();
  if (rc) return rc;
  DeltaArgs g;
  if (!s2_geometry(H, W, g)) return LPF_EUNSUPPORTED;
  g.target = de ? target : nullptr;
  g.counts = de ? counts : nullptr;
  (void)cudaGetLastError();
  uint8_t* own_ext = nullptr;
  float* own_partial = nullptr;
  cudaError_t e = cudaSuccess;
  if (!ext) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&own_ext), g.ext_bytes, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    const int blocks = (int)std::min<int64_t>((g.ext_bytes + 255) / 256, 4096);
    s2_build_ext_kernel<<<blocks, 256, 0, s>>>(img, g, own_ext);
    ext = own_ext;
  }
  if (de && !partial) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&own_partial), (size_t)K * g.n_chunks * sizeof(float), s);
    partial = own_partial;
  }
  if (e == cudaSuccess) {
    const dim3 grid(g.n_chunks, delta_stride(g.n_chunks, K));
    s2_delta_kernel<<<grid, kS2Threads, g.ext_bytes, s>>>(img, ext, g, pairs, K, dcounts, de ? partial : nullptr);
    if (de) {
      const int blocks = std::min((K + 255) / 256, 1024);
      s2_reduce_kernel<<<blocks, 256, 0, s>>>(partial, g.n_chunks, K, de);
    }
    e = cudaGetLastError();
  }
  if (own_ext) cudaFreeAsync(own_ext, s);
  if (own_partial) cudaFreeAsync(own_partial, s);
  return set_cuda_error(e);
}

void s2_enqueue_batch(lpf_sa* sa, cudaStream_t s) {
  s2_batch_kernel<<<sa->grid, kS2Threads, sa->g.ext_bytes, s>>>(
      sa->d_st, sa->cell, sa->d_ext, sa->g, sa->d_pairs, sa->d_u, sa->d_partial,
      reinterpret_cast<unsigned long long*>(sa->counts), sa->d_status);
}

}  // namespace lpf

extern "C" {

int s2_counts(const uint8_t* img_dev, int32_t H, int32_t W, int64_t* counts_dev, lpf_stream_t stream) {
  if (!img_dev || !counts_dev || H < 1 || W < 1) return LPF_EINVAL;
  if ((int64_t)H * W > (1 << 20)) return LPF_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  const int Wd = 2 * ((W + 31) / 32) + 1;
  uint32_t* P = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&P), (size_t)H * Wd * sizeof(uint32_t), s);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  const int blocks = (int)std::min<int64_t>(((int64_t)H * Wd + 255) / 256, 4096);
  lpf::s2_pack_kernel<<<blocks, 256, 0, s>>>(img_dev, H, W, Wd, P);
  lpf::s2_counts_kernel<<<H, 256, 0, s>>>(P, H, W, Wd, counts_dev);
  e = cudaGetLastError();
  cudaFreeAsync(P, s);
  return lpf::set_cuda_error(e);
}

int s2_delta_swap(const uint8_t* img_dev, int32_t H, int32_t W, const int32_t* pairs_dev, int32_t K,
                  int32_t* dcounts_dev, const float* target_dev, const int64_t* counts_dev, float* de_dev,
                  lpf_stream_t stream) {
  if (!img_dev || K < 0 || H < 1 || W < 1) return LPF_EINVAL;
  if (K == 0) return LPF_OK;
  if (!pairs_dev || (!dcounts_dev && !de_dev)) return LPF_EINVAL;
  if (de_dev && (!target_dev || !counts_dev)) return LPF_EINVAL;
  if ((int64_t)H * W > (1 << 24)) return LPF_EUNSUPPORTED;
  return lpf::s2_delta_run(img_dev, H, W, nullptr, pairs_dev, K, dcounts_dev, target_dev, counts_dev, de_dev,
                           nullptr, (cudaStream_t)stream);
}

int s2_sa_create(uint8_t* cell_dev, int32_t H, int32_t W, const float* target_dev, int64_t* counts_dev,
                 const lpf_sa_params* prm, lpf_stream_t stream, lpf_sa** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (!cell_dev || !target_dev || !counts_dev || !prm || H < 2 || W < 2) return LPF_EINVAL;
  if (int rc = lpf::sa_check_params(prm)) return rc;
  if ((int64_t)H * W > (1 << 20)) return LPF_EUNSUPPORTED;
  int rc = lpf::s2_prepare();
  if (rc) return rc;
  lpf::DeltaArgs g;
  if (!lpf::s2_geometry(H, W, g)) return LPF_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  rc = s2_counts(cell_dev, H, W, counts_dev, stream);
  if (rc) return rc;
  lpf_sa* sa = new (std::nothrow) lpf_sa();
  if (!sa) return LPF_ENOMEM;
  sa->cell = cell_dev;
  sa->H = H;
  sa->W = W;
  sa->target = target_dev;
  sa->counts = counts_dev;
  sa->prm = *prm;
  sa->objective = kSaObjectiveS2;
  sa->phase_mask = 1;
  sa->err_n_full = (int64_t)H * W;
  sa->err_base = 0;
  sa->threads = lpf::kS2Threads;
  sa->g = g;
  sa->g.target = target_dev;
  sa->g.counts = counts_dev;
  sa->grid = dim3(g.n_chunks, lpf::delta_stride(g.n_chunks, prm->k_max));
  rc = lpf::sa_start(sa, s);
  if (rc) { lpf_sa_free(sa); return rc; }
  *out = sa;
  return LPF_OK;
}

}  // extern "C"
