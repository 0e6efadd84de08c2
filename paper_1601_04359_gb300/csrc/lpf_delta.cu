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
// the marker.  The zero vector (the anchor alone) loses the anchor's old
// phase and gains its new one: over all translations the two exchanged
// pixels cancel, over a sample of translations they need not.
//
// Work split: blocks = (vector chunk) x (candidate stride); each block stages
// the extended cell once (one bulk copy of a copy built per call in global
// memory) and loops over its candidates.  Error changes are summed per
// (candidate, chunk) in a fixed order and then over chunks in chunk order, so
// results are bitwise reproducible.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "lpf_delta.cuh"
#include "lpf_state.hpp"

namespace lpf {

// ext[ey][ex] = (img[(ey - ry) mod H][(ex - rx) mod W] != 0); zero padding to
// `bytes`.  pix_flag != null (checked mode): a byte other than 0 or 1 sets
// status bit 8 in *pix_flag.
__global__ void build_ext_kernel(const uint8_t* __restrict__ img, int H, int W, int rx, int ry, int We, int He,
                                 uint32_t bytes, uint8_t* __restrict__ ext, int* __restrict__ pix_flag) {
  const int total = We * He;
  uint32_t high = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)bytes; i += gridDim.x * blockDim.x) {
    uint8_t v = 0;
    if (i < total) {
      const int ey = i / We, ex = i - ey * We;
      int y = (ey - ry) % H; if (y < 0) y += H;
      int x = (ex - rx) % W; if (x < 0) x += W;
      const uint32_t raw = img[y * W + x];
      high |= raw >> 1;
      v = raw != 0;
    }
    ext[i] = v;
  }
  if (pix_flag && high) atomicOr(pix_flag, 8);
}

__global__ void __launch_bounds__(kDeltaThreads, 3) delta_kernel(const uint8_t* __restrict__ img,
                                                               const uint8_t* __restrict__ ext, DeltaArgs g,
                                                               const int32_t* __restrict__ pairs, int K,
                                                               int32_t* __restrict__ dcounts,
                                                               float* __restrict__ partial, int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ float warp_acc[kDeltaWarps];
  __shared__ int s_a, s_b, s_skip;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = blockIdx.x;
  if ((int)blockIdx.y >= K) return;
  if (!delta_stage(sm, ext, g.ext_bytes, &bar)) {
    if (threadIdx.x == 0) atomicOr(status, 1);
    (void)mbar_wait(&bar, 0);  // let the copy land before the block exits
    return;
  }
  const int v0 = g.chunk[ch], v1 = g.chunk[ch + 1];
  const int npix = g.H * g.W;
  for (int k = blockIdx.y; k < K; k += gridDim.y) {
    if (threadIdx.x == 0) {
      int a = pairs[2 * k], b = pairs[2 * k + 1];
      int skip = 0;
      if (a < 0 || b < 0 || a >= npix || b >= npix) { skip = 1; atomicOr(status, 2); }
      else if ((img[a] != 0) == (img[b] != 0)) skip = 1;         // same phase (or a == b): identity
      else if (img[a] == 0) { const int t = a; a = b; b = t; }   // a holds phase 1
      s_a = a; s_b = b; s_skip = skip;
      if (!skip) { delta_mark(sm, a, kMarkA, g); delta_mark(sm, b, kMarkB, g); }
    }
    __syncthreads();
    const int a = s_a, b = s_b, skip = s_skip;
    int32_t* dk = dcounts ? dcounts + (int64_t)k * 2 * g.n_canon : nullptr;
    float acc = 0.0f;
    if (skip) delta_zero_vectors(g, v0, v1, dk);
    else acc = delta_walk_vectors(sm, g, a, b, v0, v1, warp, lane, dk, delta_terms_global(g));
    if (lane == 0) warp_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (partial) {
        float s = 0.0f;
        for (int w = 0; w < kDeltaWarps; ++w) s += warp_acc[w];
        partial[(int64_t)k * g.n_chunks + ch] = s;
      }
      if (!skip) { delta_mark(sm, a, 1, g); delta_mark(sm, b, 0, g); }
    }
    __syncthreads();
  }
}

// Phase-0 count of S(v) + (x, y) for every canonical vector and translation,
// from the extended cell (0/1 bytes), at delta_z_index in the sheared layout
// (SHEARED, g.shear set) or the unsheared one.  Blocks stage the cell once
// and take vectors at the grid stride; threads take translations.
template <bool SHEARED>
__global__ void __launch_bounds__(kDeltaThreads) z_init_kernel(const uint8_t* __restrict__ ext, DeltaArgs g,
                                                               uint8_t* __restrict__ z, int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  if (!delta_stage(sm, ext, g.ext_bytes, &bar)) {
    if (threadIdx.x == 0) atomicOr(status, 1);
    (void)mbar_wait(&bar, 0);
    return;
  }
  const int hw = g.H * g.W;
  for (int v = blockIdx.x; v < (int)g.n_canon; v += gridDim.x) {
    const int o0 = __ldg(g.dptr + v), L1 = __ldg(g.dptr + v + 1) - o0;
    int dx, dy;
    delta_vector(g, v, dx, dy);
    const int m = SHEARED ? __ldg(g.shear + v) : 0;
    uint8_t* zv = z + (int64_t)v * hw;
    for (int p = threadIdx.x; p < hw; p += blockDim.x) {
      // p runs over the vector's layout (delta_z_index)
      int x, y;
      delta_z_translation(g, dx, dy, m, p, x, y);
      const uint8_t* base = sm + (y + g.ry) * g.We + (x + g.rx);
      int c = 0;
      for (int k = 0; k < L1; ++k) c += base[__ldg(g.doff + o0 + k)] == 0;
      zv[p] = (uint8_t)c;
    }
  }
}

// Count changes (and error changes) of K candidates from the phase-0 counts
// g.z: no staged cell, no block barriers -- a warp takes one candidate at a
// time (candidates k = warp index over the grid's y extent, strided) and all
// vectors of its block's chunk, in vector order, and writes that chunk's
// partial error change.
__global__ void __launch_bounds__(kDeltaThreads) delta_lookup_kernel(const uint8_t* __restrict__ img, DeltaArgs g,
                                                                     const int32_t* __restrict__ pairs, int K,
                                                                     int32_t* __restrict__ dcounts,
                                                                     float* __restrict__ partial,
                                                                     int* __restrict__ status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = blockIdx.x;
  const int v0 = g.chunk[ch], v1 = g.chunk[ch + 1];
  const int npix = g.H * g.W;
  const int stride = gridDim.y * kDeltaWarps;
  for (int k = blockIdx.y * kDeltaWarps + warp; k < K; k += stride) {
    int a = pairs[2 * k], b = pairs[2 * k + 1];
    int skip = 0;
    if (a < 0 || b < 0 || a >= npix || b >= npix) {
      skip = 1;
      if (lane == 0) atomicOr(status, 2);
    } else if ((img[a] != 0) == (img[b] != 0)) {
      skip = 1;                                   // same phase (or a == b): identity
    } else if (img[a] == 0) {
      const int t = a; a = b; b = t;              // a holds phase 1
    }
    int32_t* dk = dcounts ? dcounts + (int64_t)k * 2 * g.n_canon : nullptr;
    float acc = 0.0f;
    if (skip) {
      if (dk)
        for (int v = v0 + lane; v < v1; v += 32) { dk[v] = 0; dk[g.n_canon + v] = 0; }
    } else {
      // the warp's own pass over the chunk: v0, v0 + 1, ... (one warp, so
      // "warp 0 of 1" in the helper's striding)
      acc = delta_lookup_vectors_warp(g, a, b, v0, v1, lane, dk, delta_terms_global(g));
    }
    if (lane == 0 && partial) partial[(int64_t)k * g.n_chunks + ch] = acc;
  }
}

// de[k] = sum over chunks of partial[k][c], in chunk order.
__global__ void delta_reduce_kernel(const float* __restrict__ partial, int n_chunks, int K, float* __restrict__ de) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < n_chunks; ++c) s += partial[(int64_t)k * n_chunks + c];
    de[k] = s;
  }
}

// ---------------------------------------------------------------------------
// Host side

// Device tables for one cell width: CSR of the canonical segments with each
// offset converted to an extended-cell displacement sy*We + sx, and vector
// chunks of similar walk work.
static int bake_delta(lpf_paths* p, int W, int want_chunks, DeltaTables& t) {
  const int We = delta_row_stride(W, p->host.rx);
  if (t.d_doff && t.We == We && t.want == want_chunks) return LPF_OK;
  if (t.d_doff) {
    cudaDeviceSynchronize();
    cudaFree(t.d_doff); cudaFree(t.d_dptr); cudaFree(t.d_chunk); cudaFree(t.d_off16); cudaFree(t.d_vec16);
    cudaFree(t.d_shear);
    t.d_shear = nullptr;
    t.d_doff = t.d_dptr = t.d_chunk = nullptr;
    t.d_off16 = t.d_vec16 = nullptr;
  }
  const Paths& h = p->host;
  std::vector<int32_t> off(h.ptr.back()), ptr(h.n_canon + 1);
  for (int64_t c = 0; c <= h.n_canon; ++c) ptr[c] = (int32_t)h.ptr[c];
  for (int64_t j = 0; j < h.ptr.back(); ++j) off[j] = (int32_t)h.off[2 * j + 1] * We + (int32_t)h.off[2 * j];
  // chunks balanced by work: 2 (L+1) lookups per vector where count changes
  // come from the phase-0 counts (segments up to 255 pixels), else 2 (L+1)
  // walks of up to L+1 pixels
  const bool lookups = std::max(h.rx, h.ry) + 1 <= 255;
  auto weight = [&](int64_t c) {
    const double l = (double)(ptr[c + 1] - ptr[c]);
    return lookups ? l : l * l;
  };
  double total = 0;
  for (int64_t c = 0; c < h.n_canon; ++c) total += weight(c);
  // as many chunks as blocks fit on the GPU at once (but at least 16 vectors
  // each): a single candidate then runs in one wave over every SM (the
  // annealer evaluates batches of one or a few candidates while its
  // acceptance rate is high)
  const int want = (int)std::max<int64_t>(1, std::min<int64_t>(want_chunks, h.n_canon / 16));
  std::vector<int32_t> chunk{0};
  double accw = 0;
  for (int64_t c = 0; c < h.n_canon; ++c) {
    accw += weight(c);
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
  if ((e = cudaMalloc(&t.d_off16, std::max<size_t>(1, h.off.size()) * 2)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(t.d_off16, h.off.data(), h.off.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
    return set_cuda_error(e);
  if ((e = cudaMalloc(&t.d_vec16, std::max<size_t>(1, h.vec.size()) * 2)) != cudaSuccess) return set_cuda_error(e);
  if ((e = cudaMemcpy(t.d_vec16, h.vec.data(), h.vec.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
    return set_cuda_error(e);
  {
    std::vector<int32_t> shear(std::max<int64_t>(1, h.n_canon));
    for (int64_t c = 0; c < h.n_canon; ++c) shear[c] = delta_shear(h.vec[2 * c], h.vec[2 * c + 1]);
    if ((e = cudaMalloc(&t.d_shear, shear.size() * 4)) != cudaSuccess) return set_cuda_error(e);
    if ((e = cudaMemcpy(t.d_shear, shear.data(), shear.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return set_cuda_error(e);
  }
  t.We = We;
  t.want = want_chunks;
  t.n_chunks = (int)chunk.size() - 1;
  t.max_chunk_vecs = 0;
  t.max_chunk_entries = 0;
  for (size_t c = 0; c + 1 < chunk.size(); ++c) {
    t.max_chunk_vecs = std::max(t.max_chunk_vecs, chunk[c + 1] - chunk[c]);
    t.max_chunk_entries = std::max(t.max_chunk_entries, ptr[chunk[c + 1]] - ptr[chunk[c]]);
  }
  return LPF_OK;
}

static int g_delta_max_smem = -1;
static int g_sms = 0;

int delta_geometry(const lpf_paths* p, int H, int W, DeltaArgs& g) {
  g.H = H;
  g.W = W;
  g.rx = p->host.rx;
  g.ry = p->host.ry;
  g.We = delta_row_stride(W, g.rx);
  g.He = H + 2 * g.ry;
  g.ext_bytes = (uint32_t)((((size_t)g.We * g.He) + 15) & ~size_t(15));
  g.dptr = p->delta.d_dptr;
  g.doff = p->delta.d_doff;
  g.chunk = p->delta.d_chunk;
  g.n_chunks = p->delta.n_chunks;
  g.n_canon = p->host.n_canon;
  g.n_full = p->host.n_full;
  g.base = p->host.base;
  g.target = nullptr;
  g.counts = nullptr;
  g.phase_mask = 3;
  g.max_chunk_vecs = p->delta.max_chunk_vecs;
  g.max_chunk_entries = p->delta.max_chunk_entries;
  g.sel_ext = nullptr;
  g.z = nullptr;
  g.off16 = p->delta.d_off16;
  g.vec16 = p->delta.d_vec16;
  g.shear = p->delta.d_shear;
  g.inv_norm = 1.0f / ((float)H * (float)W);
  return LPF_OK;
}

int delta_max_smem() { return g_delta_max_smem; }
int delta_num_sms() { return g_sms; }

int delta_prepare(lpf_paths* p, int H, int W, int K) {
  if (p->host.dims != 2) return LPF_EINVAL;  // swap deltas of images only
  if (g_delta_max_smem < 0) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    // the swap-delta kernel and the annealing batch kernel stage the same
    // extended cell: allow both the opt-in maximum, and limit the cell by the
    // larger of their static shared memory
    cudaFuncAttributes fa, fs, fp;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, delta_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fs, sa_batch_kernel_entry());
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fp, sa_persistent_kernel_entry());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(delta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fa.sharedSizeBytes);
    cudaFuncAttributes fz;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fz, z_init_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(z_init_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fz.sharedSizeBytes);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fz, z_init_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(z_init_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fz.sharedSizeBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sa_batch_kernel_entry(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fs.sharedSizeBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sa_persistent_kernel_entry(),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   optin - (int)fp.sharedSizeBytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    g_delta_max_smem = optin - (int)std::max(std::max(fa.sharedSizeBytes, fs.sharedSizeBytes), fp.sharedSizeBytes);
  }
  const size_t ext = (((size_t)delta_row_stride(W, p->host.rx) * (H + 2 * p->host.ry)) + 15) & ~size_t(15);
  if ((int64_t)ext > g_delta_max_smem) return LPF_EUNSUPPORTED;
  int rc = ensure_device(p, 0);
  if (rc) return rc;
  // one wave: SMs x resident blocks of the delta and annealing kernels for
  // this extended cell
  // (the persistent annealer needs every chunk's block resident at once)
  int occ_d = 0, occ_s = 0, occ_p = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, delta_kernel, kDeltaThreads, (size_t)ext);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, sa_batch_kernel_entry(), kDeltaThreads,
                                                                         (size_t)ext);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, sa_persistent_kernel_entry(), kDeltaThreads, (size_t)ext);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int occ = std::max(1, std::min(std::min(occ_d, occ_s), occ_p));
  // The tables stay as they are while the same cell width asks for the same
  // chunking (annealing runs on this handle hold pointers into them): the
  // chunking below is decided once per (width, occupancy) and remembered by
  // its first request, so calling again (with any K) never re-bakes them.
  const int want0 = occ * g_sms;
  if (!(p->delta.d_doff && p->delta.We == delta_row_stride(W, p->host.rx) && p->delta.want_key == want0)) {
    rc = bake_delta(p, W, want0, p->delta);
    if (rc) return rc;
    // the persistent kernel also keeps its chunk's counts, targets and lookup tables: check
    // the chunking once more with the size it produced
    const size_t persist = persistent_smem_bytes(ext, p->delta.max_chunk_vecs, p->delta.max_chunk_entries);
    int occ2 = 0;
    if ((int64_t)persist <= g_delta_max_smem &&
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, sa_persistent_kernel_entry(), kDeltaThreads,
                                                           persist)) != cudaSuccess)
      return set_cuda_error(e);
    if (occ2 > 0 && occ2 < occ) {
      rc = bake_delta(p, W, occ2 * g_sms, p->delta);
      if (rc) return rc;
    }
    p->delta.want_key = want0;
  }
  if (ext > p->ext_cap) {
    if (p->d_ext) { cudaDeviceSynchronize(); cudaFree(p->d_ext); p->d_ext = nullptr; p->ext_cap = 0; }
    if ((e = cudaMalloc(&p->d_ext, ext)) != cudaSuccess) return set_cuda_error(e);
    p->ext_cap = ext;
  }
  const size_t need = (size_t)std::max(K, 1) * p->delta.n_chunks;
  if (need > p->partial_cap) {
    if (p->d_partial) { cudaDeviceSynchronize(); cudaFree(p->d_partial); p->d_partial = nullptr; p->partial_cap = 0; }
    if ((e = cudaMalloc(&p->d_partial, need * sizeof(float))) != cudaSuccess) return set_cuda_error(e);
    p->partial_cap = need;
  }
  return LPF_OK;
}

// Blocks per vector chunk: enough candidate strides to fill every SM a few times.
int delta_stride(int n_chunks, int K) {
  const int sms = g_sms > 0 ? g_sms : 152;
  return std::max(1, std::min(K, (sms * 4 + n_chunks - 1) / n_chunks));
}

// Bytes of the phase-0 counts z for an H x W cell (one byte per canonical
// vector and translation, plus 4 bytes of padding), or 0
// when they do not apply: segments longer than 255 pixels (a byte count),
// cells wider or higher than kZMaxSide, or more than kZBudget bytes.
constexpr size_t kZBudget = size_t(2) << 30;
size_t delta_z_bytes(const lpf_paths* p, int H, int W) {
  if (std::max(p->host.rx, p->host.ry) + 1 > 255) return 0;
  if (H > kZMaxSide || W > kZMaxSide) return 0;
  const size_t b = (size_t)p->host.n_canon * H * W + 4;
  return b <= kZBudget ? b : 0;
}

int delta_z_prepare(lpf_paths* p, int H, int W) {
  const size_t need = delta_z_bytes(p, H, W);
  if (need > p->z_cap) {
    if (p->d_z) { cudaDeviceSynchronize(); cudaFree(p->d_z); p->d_z = nullptr; p->z_cap = 0; }
    cudaError_t e = cudaMalloc(&p->d_z, need);
    if (e != cudaSuccess) return set_cuda_error(e);
    p->z_cap = need;
  }
  return LPF_OK;
}

void z_init_launch(const uint8_t* ext, const DeltaArgs& g, uint8_t* z, int* status, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(g.n_canon, 2 * (int64_t)(g_sms > 0 ? g_sms : 152));
  if (g.shear) z_init_kernel<true><<<blocks, kDeltaThreads, g.ext_bytes, s>>>(ext, g, z, status);
  else z_init_kernel<false><<<blocks, kDeltaThreads, g.ext_bytes, s>>>(ext, g, z, status);
}

int delta_swap_run(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, const int32_t* pairs_dev,
                   int32_t K, int32_t* dcounts_dev, const float* target_dev, const int64_t* counts_dev, float* de_dev,
                   int phase_mask, cudaStream_t s, const uint8_t* sel_ext, float inv_norm) {
  if (!paths || !img_dev || K < 0) return LPF_EINVAL;
  if (K == 0) return LPF_OK;
  if (!pairs_dev) return LPF_EINVAL;
  if (H < 1 || W < 1 || H > 8192 || W > 8192) return LPF_EINVAL;
  if (paths->host.rx >= W || paths->host.ry >= H) return LPF_EINVAL;
  if (de_dev && (!target_dev || !counts_dev)) return LPF_EINVAL;
  if (!de_dev && !dcounts_dev) return LPF_EINVAL;  // nothing to compute
  int rc = delta_prepare(paths, H, W, K);
  if (rc) return rc;
  (void)cudaGetLastError();
  DeltaArgs g;
  delta_geometry(paths, H, W, g);
  g.target = de_dev ? target_dev : nullptr;
  g.counts = de_dev ? counts_dev : nullptr;
  g.phase_mask = phase_mask;
  g.sel_ext = sel_ext;
  if (inv_norm > 0.0f) g.inv_norm = inv_norm;
  {
    const int blocks = (int)std::min<int64_t>((g.ext_bytes + 255) / 256, 4096);
    build_ext_kernel<<<blocks, 256, 0, s>>>(img_dev, H, W, g.rx, g.ry, g.We, g.He, g.ext_bytes, paths->d_ext,
                                            paths->checked ? paths->d_status : nullptr);
  }
  dim3 grid(g.n_chunks, delta_stride(g.n_chunks, K));
  // Phase-0 counts of every (vector, translation) when they fit the budget:
  // count changes by lookups; otherwise by walks.
  if (delta_z_bytes(paths, H, W) > 0) {
    rc = delta_z_prepare(paths, H, W);
    if (rc) return rc;
    g.z = paths->d_z;
    // unsheared counts: this call reads every candidate's lookups from an L2
    // that holds z, and is bound by instruction issue, not by the sectors
    // each warp touches (the annealer's sheared layout costs it 5 more
    // instructions per lookup)
    g.shear = nullptr;
    z_init_launch(paths->d_ext, g, g.z, paths->d_status, s);
    if (paths->ev_start) cudaEventRecord(paths->ev_start, s);
    // a warp per candidate: enough candidate groups of 16 for a few warps per SM slot
    grid.y = (unsigned)std::max(1, std::min((K + kDeltaWarps - 1) / kDeltaWarps,
                                            (8 * (g_sms > 0 ? g_sms : 152) + g.n_chunks - 1) / g.n_chunks));
    delta_lookup_kernel<<<grid, kDeltaThreads, 0, s>>>(img_dev, g, pairs_dev, K, dcounts_dev,
                                                       de_dev ? paths->d_partial : nullptr, paths->d_status);
    if (paths->ev_stop) cudaEventRecord(paths->ev_stop, s);
  } else {
    if (paths->ev_start) cudaEventRecord(paths->ev_start, s);
    delta_kernel<<<grid, kDeltaThreads, g.ext_bytes, s>>>(img_dev, paths->d_ext, g, pairs_dev, K, dcounts_dev,
                                                          de_dev ? paths->d_partial : nullptr, paths->d_status);
    if (paths->ev_stop) cudaEventRecord(paths->ev_stop, s);
  }
  if (de_dev) {
    const int blocks = std::min((K + 255) / 256, 1024);
    delta_reduce_kernel<<<blocks, 256, 0, s>>>(paths->d_partial, g.n_chunks, K, de_dev);
  }
  return set_cuda_error(cudaGetLastError());
}

}  // namespace lpf

extern "C" int lpf_delta_swap(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths,
                              const int32_t* pairs_dev, int32_t K, int32_t* dcounts_dev, const float* target_dev,
                              const int64_t* counts_dev, float* de_dev, lpf_stream_t stream) {
  return lpf::delta_swap_run(img_dev, H, W, paths, pairs_dev, K, dcounts_dev, target_dev, counts_dev, de_dev, 3,
                             (cudaStream_t)stream, nullptr, 0.0f);
}

namespace lpf {

// Number of selected translations (host copy of the mask; synchronises).
int count_selected(const uint8_t* sel_dev, int H, int W, cudaStream_t s, int64_t* n) {
  std::vector<uint8_t> h((size_t)H * W);
  cudaError_t e = cudaMemcpyAsync(h.data(), sel_dev, h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(e);
  int64_t c = 0;
  for (uint8_t v : h) c += v != 0;
  *n = c;
  return LPF_OK;
}

// The selection mask in the extended-cell layout of the delta kernels, in a
// new device buffer (stream-ordered).
int build_sel_ext(const uint8_t* sel_dev, int H, int W, const lpf_paths* paths, cudaStream_t s, uint8_t** out) {
  DeltaArgs g;
  g.H = H;
  g.W = W;
  g.rx = paths->host.rx;
  g.ry = paths->host.ry;
  g.We = delta_row_stride(W, g.rx);
  g.He = H + 2 * g.ry;
  g.ext_bytes = (uint32_t)((((size_t)g.We * g.He) + 15) & ~size_t(15));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(out), g.ext_bytes, s);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int blocks = (int)std::min<int64_t>((g.ext_bytes + 255) / 256, 4096);
  build_ext_kernel<<<blocks, 256, 0, s>>>(sel_dev, H, W, g.rx, g.ry, g.We, g.He, g.ext_bytes, *out, nullptr);
  return set_cuda_error(cudaGetLastError());
}

}  // namespace lpf

extern "C" int lpf_delta_swap_mc(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths,
                                 const uint8_t* sel_dev, const int32_t* pairs_dev, int32_t K, int32_t* dcounts_dev,
                                 const float* target_dev, const int64_t* counts_dev, float* de_dev,
                                 lpf_stream_t stream) {
  if (!paths || !img_dev || !sel_dev || K < 0 || H < 1 || W < 1) return LPF_EINVAL;
  if (K == 0) return LPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n = 0;
  int rc = lpf::count_selected(sel_dev, H, W, s, &n);
  if (rc) return rc;
  if (n == 0) return LPF_EINVAL;
  uint8_t* sel_ext = nullptr;
  rc = lpf::build_sel_ext(sel_dev, H, W, paths, s, &sel_ext);
  if (!rc)
    rc = lpf::delta_swap_run(img_dev, H, W, paths, pairs_dev, K, dcounts_dev, target_dev, counts_dev, de_dev, 3, s,
                             sel_ext, 1.0f / (float)n);
  if (sel_ext) cudaFreeAsync(sel_ext, s);
  return rc;
}
