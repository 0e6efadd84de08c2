// Count changes of the lineal path function for a batch of candidate pixel
// exchanges (the annealer's modification operator, Sec. 4), and the change of
// the least-square error Eq. (LSE) they cause.
//
// Exchanging pixel a (phase 1) with pixel b (phase 0) changes count_p(v) only
// for translations x whose segment x + S(v) contains a or b: for each of the
// L+1 pixels s_i of S(v), x = a - s_i and x = b - s_i.  A block keeps the cell
// in shared memory as bytes, extended periodically by rx columns and ry rows
// on each side so that every such walk stays inside the array without
// wrapping, and writes the exchange into its copy with two marker values
// (kMarkA at a: phase 1 before, 0 after; kMarkB at b: 0 before, 1 after).
// One early-exit walk of the segment then decides both phases: the first
// pixel other than the anchor fixes the phase q the segment must be uniform
// in, and a marker anywhere else ends the walk.  For the anchor a:
//   q = 1 -> the segment was all phase 1 before and is not after: dcount_1 -= 1
//   q = 0 -> the segment is all phase 0 after (and was not before): dcount_0 += 1
// and for the anchor b (walks that also contain a are counted from a):
//   q = 1 -> dcount_1 += 1,  q = 0 -> dcount_0 -= 1.
// Segments containing both a and b change in neither phase and are ended by
// the marker.  The zero vector never changes.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "lpf_device.cuh"
#include "lpf_state.hpp"

namespace lpf {

constexpr uint8_t kMarkA = 4;
constexpr uint8_t kMarkB = 3;
constexpr int kDeltaThreads = 256;
constexpr int kDeltaWarps = kDeltaThreads / 32;

struct DeltaGeom {
  int We = 0, He = 0;   // extended width / height
  uint32_t smem = 0;    // bytes (multiple of 16)
};

static DeltaGeom delta_geom(int H, int W, int rx, int ry) {
  DeltaGeom g;
  g.We = W + 2 * rx;
  g.He = H + 2 * ry;
  g.smem = (uint32_t)((((size_t)g.We * g.He) + 15) & ~size_t(15));
  return g;
}

// Extended-cell position of pixel index c.
__device__ __forceinline__ int ext_pos(int c, int W, int We, int rx, int ry) {
  const int cy = c / W, cx = c - cy * W;
  return (cy + ry) * We + (cx + rx);
}

// Write `val` at every periodic copy of pixel c inside the extended cell.
__device__ void mark_copies(uint8_t* sm, int c, uint8_t val, int H, int W, int We, int He, int rx, int ry) {
  const int cy = c / W, cx = c - cy * W;
  for (int ey = cy + ry - ((cy + ry) / H) * H; ey < He; ey += H)
    for (int ex = cx + rx - ((cx + rx) / W) * W; ex < We; ex += W) sm[ey * We + ex] = val;
}

__global__ void __launch_bounds__(kDeltaThreads) delta_kernel(
    const uint8_t* __restrict__ img, int H, int W, int rx, int ry, int We, int He,
    const int32_t* __restrict__ dptr, const int32_t* __restrict__ doff, const int32_t* __restrict__ chunk,
    int n_chunks, const int32_t* __restrict__ pairs, int K, const int32_t* __restrict__ k_dev,
    int32_t* __restrict__ dcounts, int64_t n_canon, const float* __restrict__ target,
    const int64_t* __restrict__ counts, int64_t n_full, int64_t base, float* __restrict__ partial,
    int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ float warp_acc[kDeltaWarps];
  __shared__ int s_a, s_b, s_skip;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = blockIdx.x;
  const int Keff = k_dev ? min(K, *k_dev) : K;
  if ((int)blockIdx.y >= Keff) return;

  // extended cell: sm[ey*We + ex] = img[(ey - ry) mod H][(ex - rx) mod W]
  const int total = We * He;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int ey = i / We, ex = i - ey * We;
    int y = (ey - ry) % H; if (y < 0) y += H;
    int x = (ex - rx) % W; if (x < 0) x += W;
    sm[i] = img[y * W + x];
  }
  __syncthreads();

  const int v0 = chunk[ch], v1 = chunk[ch + 1];
  const float invN = 1.0f / ((float)H * (float)W);
  const int npix = H * W;

  for (int k = blockIdx.y; k < Keff; k += gridDim.y) {
    if (threadIdx.x == 0) {
      int a = pairs[2 * k], b = pairs[2 * k + 1];
      int skip = 0;
      if (a < 0 || b < 0 || a >= npix || b >= npix) { skip = 1; atomicOr(status, 2); }
      else if (img[a] == img[b]) skip = 1;       // same phase (or a == b): identity
      else if (img[a] == 0) { const int t = a; a = b; b = t; }  // a holds phase 1
      s_a = a; s_b = b; s_skip = skip;
      if (!skip) {
        mark_copies(sm, a, kMarkA, H, W, We, He, rx, ry);
        mark_copies(sm, b, kMarkB, H, W, We, He, rx, ry);
      }
    }
    __syncthreads();
    const int a = s_a, b = s_b, skip = s_skip;
    float acc = 0.0f;
    const int pa = skip ? 0 : ext_pos(a, W, We, rx, ry);
    const int pb = skip ? 0 : ext_pos(b, W, We, rx, ry);
    for (int v = v0 + warp; v < v1; v += kDeltaWarps) {
      const int o0 = dptr[v];
      const int L1 = dptr[v + 1] - o0;  // pixels of the segment
      int d0 = 0, d1 = 0;
      if (!skip && L1 > 1) {
        const int tasks = 2 * L1;
        for (int t0 = 0; t0 < tasks; t0 += 32) {
          const int t = t0 + lane;
          const bool is_a = t < L1;
          const int i = is_a ? t : t - L1;
          bool alive = t < tasks;
          const int pos = (is_a ? pa : pb) - (alive ? __ldg(doff + o0 + i) : 0);
          int q = -1;
          for (int j = 0; j < L1; ++j) {
            if (!__any_sync(0xffffffffu, alive)) break;
            const int oj = __ldg(doff + o0 + j);
            if (alive && j != i) {
              const int val = sm[pos + oj];
              if (q < 0) {
                if (val > 1) alive = false; else q = val;
              } else if (val != q) {
                alive = false;
              }
            }
          }
          if (alive) {
            if (is_a) { if (q == 1) d1 -= 1; else d0 += 1; }
            else      { if (q == 1) d1 += 1; else d0 -= 1; }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          d0 += __shfl_xor_sync(0xffffffffu, d0, o);
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        }
      }
      if (lane == 0) {
        if (dcounts) {
          dcounts[((int64_t)k * 2 + 0) * n_canon + v] = d0;
          dcounts[((int64_t)k * 2 + 1) * n_canon + v] = d1;
        }
        if (partial && (d0 | d1)) {
          // (d - D/N)^2 - d^2 = (D/N) * (D/N - 2 d), d = target - count/N
          if (d0) {
            const float dd = target[base + v] - (float)counts[base + v] * invN;
            const float x = (float)d0 * invN;
            acc += x * (x - 2.0f * dd);
          }
          if (d1) {
            const float dd = target[n_full + base + v] - (float)counts[n_full + base + v] * invN;
            const float x = (float)d1 * invN;
            acc += x * (x - 2.0f * dd);
          }
        }
      }
    }
    if (lane == 0) warp_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (partial) {
        float s = 0.0f;
        for (int w = 0; w < kDeltaWarps; ++w) s += warp_acc[w];
        partial[(int64_t)k * n_chunks + ch] = s;
      }
      if (!skip) {
        mark_copies(sm, a, 1, H, W, We, He, rx, ry);
        mark_copies(sm, b, 0, H, W, We, He, rx, ry);
      }
    }
    __syncthreads();
  }
}

// de[k] = sum over chunks of partial[k][c], in chunk order.
__global__ void delta_reduce_kernel(const float* __restrict__ partial, int n_chunks, int K,
                                    const int32_t* __restrict__ k_dev, float* __restrict__ de) {
  const int Keff = k_dev ? min(K, *k_dev) : K;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    float s = 0.0f;
    if (k < Keff)
      for (int c = 0; c < n_chunks; ++c) s += partial[(int64_t)k * n_chunks + c];
    de[k] = s;
  }
}

// ---------------------------------------------------------------------------
// Host side

// Device tables for one cell width: CSR of the canonical segments with each
// offset converted to an extended-cell displacement sy*We + sx, and vector
// chunks of similar walk work.
static int bake_delta(lpf_paths* p, int H, int W, DeltaTables& t) {
  const int We = W + 2 * p->host.rx;
  if (t.d_doff && t.We == We) return LPF_OK;
  if (t.d_doff) {
    cudaDeviceSynchronize();
    cudaFree(t.d_doff); cudaFree(t.d_dptr); cudaFree(t.d_chunk);
    t.d_doff = t.d_dptr = t.d_chunk = nullptr;
  }
  const Paths& h = p->host;
  std::vector<int32_t> off(h.ptr.back()), ptr(h.n_canon + 1);
  for (int64_t c = 0; c <= h.n_canon; ++c) ptr[c] = (int32_t)h.ptr[c];
  for (int64_t j = 0; j < h.ptr.back(); ++j) off[j] = (int32_t)h.off[2 * j + 1] * We + (int32_t)h.off[2 * j];
  // chunks balanced by sum of (L+1)^2 (walks per vector times their length bound)
  double total = 0;
  for (int64_t c = 0; c < h.n_canon; ++c) { const double l = (double)(ptr[c + 1] - ptr[c]); total += l * l; }
  const int want = (int)std::max<int64_t>(1, std::min<int64_t>(32, h.n_canon / 64));
  std::vector<int32_t> chunk{0};
  double accw = 0;
  for (int64_t c = 0; c < h.n_canon; ++c) {
    const double l = (double)(ptr[c + 1] - ptr[c]);
    accw += l * l;
    if (accw >= total * (double)chunk.size() / want && (int)chunk.size() < want) chunk.push_back((int32_t)c + 1);
  }
  if (chunk.back() != (int32_t)h.n_canon) chunk.push_back((int32_t)h.n_canon);
  cudaError_t e;
  if ((e = cudaMalloc(&t.d_doff, std::max<size_t>(1, off.size()) * 4)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMalloc(&t.d_dptr, ptr.size() * 4)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMalloc(&t.d_chunk, chunk.size() * 4)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(t.d_doff, off.data(), off.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(t.d_dptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(t.d_chunk, chunk.data(), chunk.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return set_cuda_error(e);
  t.We = We;
  t.n_chunks = (int)chunk.size() - 1;
  return LPF_OK;
}

static int g_delta_max_smem = -1;

int delta_prepare(lpf_paths* p, int H, int W, int K) {
  if (g_delta_max_smem < 0) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, delta_kernel);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(delta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    g_delta_max_smem = optin - (int)fa.sharedSizeBytes;
  }
  const DeltaGeom g = delta_geom(H, W, p->host.rx, p->host.ry);
  if ((int)g.smem > g_delta_max_smem) return LPF_EUNSUPPORTED;
  int rc = ensure_device(p, 0);
  if (rc) return rc;
  rc = bake_delta(p, H, W, p->delta);
  if (rc) return rc;
  const size_t need = (size_t)std::max(K, 1) * p->delta.n_chunks;
  if (need > p->partial_cap) {
    if (p->d_partial) { cudaDeviceSynchronize(); cudaFree(p->d_partial); p->d_partial = nullptr; p->partial_cap = 0; }
    cudaError_t e = cudaMalloc(&p->d_partial, need * sizeof(float));
    if (e != cudaSuccess) return set_cuda_error(e);
    p->partial_cap = need;
  }
  return LPF_OK;
}

int delta_launch(const uint8_t* img, int H, int W, lpf_paths* p, const int32_t* pairs, int K,
                 const int32_t* k_dev, int32_t* dcounts, const float* target, const int64_t* counts, float* de,
                 float* partial, cudaStream_t s) {
  const DeltaGeom g = delta_geom(H, W, p->host.rx, p->host.ry);
  const int n_chunks = p->delta.n_chunks;
  // blocks stride over the candidates: enough of them to fill every SM a few
  // times whatever the (possibly device-side) number of candidates
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int per_chunk = std::max(1, (sms * 8 + n_chunks - 1) / n_chunks);
  dim3 grid(n_chunks, std::min(K, per_chunk));
  if (p->ev_start) cudaEventRecord(p->ev_start, s);
  delta_kernel<<<grid, kDeltaThreads, g.smem, s>>>(
      img, H, W, p->host.rx, p->host.ry, g.We, g.He, p->delta.d_dptr, p->delta.d_doff, p->delta.d_chunk, n_chunks,
      pairs, K, k_dev, dcounts, p->host.n_canon, target, counts, p->host.n_full, p->host.base,
      de ? partial : nullptr, p->d_status);
  if (p->ev_stop) cudaEventRecord(p->ev_stop, s);
  if (de) {
    const int blocks = std::min((K + 255) / 256, 1024);
    delta_reduce_kernel<<<blocks, 256, 0, s>>>(partial, n_chunks, K, k_dev, de);
  }
  return set_cuda_error(cudaGetLastError());
}

}  // namespace lpf

extern "C" int lpf_delta_swap(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths,
                              const int32_t* pairs_dev, int32_t K, int32_t* dcounts_dev, const float* target_dev,
                              const int64_t* counts_dev, float* de_dev, lpf_stream_t stream) {
  if (!paths || !img_dev || K < 0) return LPF_EINVAL;
  if (K == 0) return LPF_OK;
  if (!pairs_dev) return LPF_EINVAL;
  if (H < 1 || W < 1 || H > 8192 || W > 8192) return LPF_EINVAL;
  if (paths->host.rx >= W || paths->host.ry >= H) return LPF_EINVAL;
  if (de_dev && (!target_dev || !counts_dev)) return LPF_EINVAL;
  if (!de_dev && !dcounts_dev) return LPF_EINVAL;  // nothing to compute
  int rc = lpf::delta_prepare(paths, H, W, K);
  if (rc) return rc;
  (void)cudaGetLastError();
  return lpf::delta_launch(img_dev, H, W, paths, pairs_dev, K, nullptr, dcounts_dev, target_dev, counts_dev, de_dev,
                           paths->d_partial, (cudaStream_t)stream);
}
