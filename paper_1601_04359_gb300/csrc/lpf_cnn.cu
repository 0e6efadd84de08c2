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
// forward and backward passes; activations and accumulation in float32.
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
constexpr int kTile = 16;        // output tile 16 x 16 pixels per block
constexpr int kCinChunk = 8;     // input channels staged per step

inline int layer_w_size(int l) { return 9 * kCh[l] * kCh[l + 1]; }

// Input features [H][W][2]: cell value and interfacial mask (torus).
__global__ void cnn_features_kernel(const uint8_t* __restrict__ cell, int H, int W, float* __restrict__ x) {
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

// out[p][co] = bias[co] + sum_tap sum_ci in[p + off(tap)][ci] * w[tap][ci][co],
// circular; optional ReLU; optional mask: out *= (mask[p][co] > 0).
// `flip` reads the weights as w[8 - tap][co][ci] (the transposed convolution
// used for input gradients; then CIN/COUT are the layer's Cout/Cin).
template <int COUT>
__global__ void __launch_bounds__(kTile* kTile) cnn_conv_kernel(const float* __restrict__ in, int H, int W, int CIN,
                                                               const __nv_bfloat16* __restrict__ w, int flip,
                                                               const float* __restrict__ bias, int relu,
                                                               const float* __restrict__ mask,
                                                               float* __restrict__ out) {
  __shared__ float s_in[(kTile + 2) * (kTile + 2) * kCinChunk];
  __shared__ float s_w[9 * kCinChunk * COUT];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  const int px = x0 + tx, py = y0 + ty;
  float acc[COUT];
#pragma unroll
  for (int c = 0; c < COUT; ++c) acc[c] = bias ? bias[c] : 0.0f;
  for (int c0 = 0; c0 < CIN; c0 += kCinChunk) {
    const int cn = min(kCinChunk, CIN - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < (kTile + 2) * (kTile + 2) * kCinChunk; i += blockDim.x) {
      const int ci = i % kCinChunk, q = i / kCinChunk;
      const int ly = q / (kTile + 2), lx = q - ly * (kTile + 2);
      int gy = (y0 + ly - 1) % H; if (gy < 0) gy += H;
      int gx = (x0 + lx - 1) % W; if (gx < 0) gx += W;
      s_in[i] = ci < cn ? in[((int64_t)gy * W + gx) * CIN + c0 + ci] : 0.0f;
    }
    for (int i = threadIdx.x; i < 9 * kCinChunk * COUT; i += blockDim.x) {
      const int co = i % COUT, r = i / COUT;
      const int ci = r % kCinChunk, tap = r / kCinChunk;
      float v = 0.0f;
      if (ci < cn) {
        const int cig = c0 + ci;
        v = flip ? __bfloat162float(w[((int64_t)(8 - tap) * COUT + co) * CIN + cig])
                 : __bfloat162float(w[((int64_t)tap * CIN + cig) * COUT + co]);
      }
      s_w[i] = v;
    }
    __syncthreads();
    if (px < W && py < H) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        const float* xi = s_in + ((ty + dy) * (kTile + 2) + (tx + dx)) * kCinChunk;
        const float* wi = s_w + tap * kCinChunk * COUT;
        for (int ci = 0; ci < cn; ++ci) {
          const float xv = xi[ci];
#pragma unroll
          for (int c = 0; c < COUT; ++c) acc[c] = fmaf(xv, wi[ci * COUT + c], acc[c]);
        }
      }
    }
  }
  if (px < W && py < H) {
    const int64_t p = (int64_t)py * W + px;
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
      float v = acc[c];
      if (relu) v = fmaxf(v, 0.0f);
      if (mask && !(mask[p * COUT + c] > 0.0f)) v = 0.0f;
      out[p * COUT + c] = v;
    }
  }
}

// dw[tap][ci][co] (+)= sum_p in[p + off(tap)][ci] * g[p][co]; one block per
// (tap, ci), threads = co x 4 row quarters, quarters summed in order.
__global__ void cnn_dw_kernel(const float* __restrict__ in, const float* __restrict__ g, int H, int W, int CIN,
                              int COUT, float* __restrict__ dw, int accumulate) {
  extern __shared__ float s_part[];
  const int tap = blockIdx.x / CIN, ci = blockIdx.x - tap * CIN;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int co = threadIdx.x % COUT, quarter = threadIdx.x / COUT;
  const int y0 = quarter * ((H + 3) / 4), y1 = min(H, y0 + (H + 3) / 4);
  float acc = 0.0f;
  for (int y = y0; y < y1; ++y) {
    int sy = y + dy; sy = sy < 0 ? sy + H : (sy >= H ? sy - H : sy);
    const float* irow = in + (int64_t)sy * W * CIN + ci;
    const float* grow = g + (int64_t)y * W * COUT + co;
    for (int x = 0; x < W; ++x) {
      int sx = x + dx; sx = sx < 0 ? sx + W : (sx >= W ? sx - W : sx);
      acc = fmaf(irow[(int64_t)sx * CIN], grow[(int64_t)x * COUT], acc);
    }
  }
  s_part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < COUT) {
    const float s = ((s_part[co] + s_part[COUT + co]) + s_part[2 * COUT + co]) + s_part[3 * COUT + co];
    const int64_t i = ((int64_t)tap * CIN + ci) * COUT + co;
    dw[i] = accumulate ? dw[i] + s : s;
  }
}

// db[co] (+)= sum_p g[p][co], one block of COUT x 8 threads, parts summed in order.
__global__ void cnn_db_kernel(const float* __restrict__ g, int npix, int COUT, float* __restrict__ db, int accumulate) {
  extern __shared__ float s_part[];
  const int co = threadIdx.x % COUT, part = threadIdx.x / COUT;
  float acc = 0.0f;
  if (part < 8)
    for (int p = part; p < npix; p += 8) acc += g[(int64_t)p * COUT + co];
  s_part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < COUT) {
    float s = 0.0f;
    for (int q = 0; q < 8; ++q) s += s_part[q * COUT + co];
    db[co] = accumulate ? db[co] + s : s;
  }
}

// Loss of one snapshot and dL/d out (two pixels per candidate), in candidate
// order by one thread (deterministic).  g must be zeroed beforehand.
__global__ void cnn_loss_kernel(const float* __restrict__ out, int W, const int32_t* __restrict__ pairs,
                                const float* __restrict__ y, int n, float* __restrict__ g, float* __restrict__ loss,
                                float scale) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float l = 0.0f;
  for (int i = 0; i < n; ++i) {
    const int a = pairs[2 * i], b = pairs[2 * i + 1];
    const float r = out[2 * a + 1] + out[2 * b] - y[i];
    l += 0.5f * r * r;
    g[2 * a + 1] += r / n;
    g[2 * b] += r / n;
  }
  if (loss) *loss += l / n * scale;
}

// Listwise loss of one snapshot: L = logsumexp(s) - sum_i q_i s_i with
// s_i = s1[a_i] + s0[b_i] and q = softmax(y / beta); dL/ds_i = p_i - q_i on
// both pixels of candidate i.  One thread, candidate order (deterministic).
__global__ void cnn_listwise_kernel(const float* __restrict__ out, const int32_t* __restrict__ pairs,
                                    const float* __restrict__ y, int n, float beta, float* __restrict__ g,
                                    float* __restrict__ loss, float scale) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float smax = -3.0e38f, ymax = -3.0e38f;
  for (int i = 0; i < n; ++i) {
    smax = fmaxf(smax, out[2 * pairs[2 * i] + 1] + out[2 * pairs[2 * i + 1]]);
    ymax = fmaxf(ymax, y[i] / beta);
  }
  float zs = 0.0f, zq = 0.0f;
  for (int i = 0; i < n; ++i) {
    zs += expf(out[2 * pairs[2 * i] + 1] + out[2 * pairs[2 * i + 1]] - smax);
    zq += expf(y[i] / beta - ymax);
  }
  float l = smax + logf(zs);
  for (int i = 0; i < n; ++i) {
    const int a = pairs[2 * i], b = pairs[2 * i + 1];
    const float si = out[2 * a + 1] + out[2 * b];
    const float pi = expf(si - smax) / zs, qi = expf(y[i] / beta - ymax) / zq;
    l -= qi * si;
    g[2 * a + 1] += pi - qi;
    g[2 * b] += pi - qi;
  }
  if (loss) *loss += l * scale;
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
  float* d_act[lpf::kLayers + 1] = {};
  float* d_gact = nullptr;    // gradient buffers (two, ping-pong)
  float* d_gact2 = nullptr;
  int64_t step = 0;
  int loss_kind = 0;          // 0: squared error, 1: listwise cross-entropy
  float beta = 1.0f;          // listwise target temperature
};

namespace lpf {

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
  for (int l = 0; l <= kLayers && e == cudaSuccess; ++l) e = cudaMalloc(&c->d_act[l], npix * kCh[l] * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gact, npix * 64 * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gact2, npix * 64 * 4);
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

template <int COUT>
static void conv_launch(const float* in, int H, int W, int CIN, const __nv_bfloat16* w, int flip, const float* bias,
                        int relu, const float* mask, float* out, cudaStream_t s) {
  const dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  cnn_conv_kernel<COUT><<<grid, kTile * kTile, 0, s>>>(in, H, W, CIN, w, flip, bias, relu, mask, out);
}

static void conv_any(int COUT, const float* in, int H, int W, int CIN, const __nv_bfloat16* w, int flip,
                     const float* bias, int relu, const float* mask, float* out, cudaStream_t s) {
  switch (COUT) {
    case 2: conv_launch<2>(in, H, W, CIN, w, flip, bias, relu, mask, out, s); break;
    case 32: conv_launch<32>(in, H, W, CIN, w, flip, bias, relu, mask, out, s); break;
    case 48: conv_launch<48>(in, H, W, CIN, w, flip, bias, relu, mask, out, s); break;
    default: conv_launch<64>(in, H, W, CIN, w, flip, bias, relu, mask, out, s); break;
  }
}

void cnn_forward(lpf_cnn* c, const uint8_t* cell, cudaStream_t s) {
  const int npix = c->H * c->W;
  cnn_features_kernel<<<(npix + 255) / 256, 256, 0, s>>>(cell, c->H, c->W, c->d_act[0]);
  for (int l = 0; l < kLayers; ++l)
    conv_any(kCh[l + 1], c->d_act[l], c->H, c->W, kCh[l], c->d_wbf + c->wb_off[l], 0, c->d_p + c->b_off[l],
             l < kLayers - 1, nullptr, c->d_act[l + 1], s);
}

// Forward, loss and backward of one snapshot; gradients added into d_g
// (or written when accumulate == 0); loss added into *loss_dev (scaled).
static void cnn_fwd_bwd(lpf_cnn* c, const uint8_t* cell, const int32_t* pairs, const float* y, int n, int accumulate,
                        float* loss_dev, float loss_scale, cudaStream_t s) {
  const int H = c->H, W = c->W, npix = H * W;
  cnn_forward(c, cell, s);
  float* g = c->d_gact;
  float* g2 = c->d_gact2;
  cudaMemsetAsync(g, 0, (size_t)npix * kCh[kLayers] * 4, s);
  if (c->loss_kind == 1)
    cnn_listwise_kernel<<<1, 32, 0, s>>>(c->d_act[kLayers], pairs, y, n, c->beta, g, loss_dev, loss_scale);
  else
    cnn_loss_kernel<<<1, 32, 0, s>>>(c->d_act[kLayers], W, pairs, y, n, g, loss_dev, loss_scale);
  for (int l = kLayers - 1; l >= 0; --l) {
    const int cin = kCh[l], cout = kCh[l + 1];
    // g = dL/d(pre-activation output of layer l) here (ReLU mask already applied)
    cnn_dw_kernel<<<9 * cin, 4 * cout, 4 * cout * sizeof(float), s>>>(c->d_act[l], g, H, W, cin, cout,
                                                                       c->d_g + c->w_off[l], accumulate);
    cnn_db_kernel<<<1, 8 * cout, 8 * cout * sizeof(float), s>>>(g, npix, cout, c->d_g + c->b_off[l], accumulate);
    if (l > 0) {
      // dL/d act[l] = transposed conv of g, then times the ReLU mask of act[l]
      conv_any(cin, g, H, W, cout, c->d_wbf + c->wb_off[l], 1, nullptr, 0, c->d_act[l], g2, s);
      std::swap(g, g2);
    }
  }
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
  lpf::cnn_fwd_bwd(c, cell_dev, pairs_dev, y_dev, n, 0, loss_dev, 1.0f, s);
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
  for (int b = 0; b < B; ++b)
    lpf::cnn_fwd_bwd(c, cells_dev + b * npix, pairs_dev + (size_t)b * n * 2, y_dev + (size_t)b * n, n, b > 0,
                     loss_dev, 1.0f / B, s);
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
  for (int l = 0; l <= lpf::kLayers; ++l) cudaFree(c->d_act[l]);
  cudaFree(c->d_gact);
  cudaFree(c->d_gact2);
  delete c;
}

}  // extern "C"
