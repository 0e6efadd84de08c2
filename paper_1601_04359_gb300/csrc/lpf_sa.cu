// Simulated annealing on the GPU (Sec. 4, Alg. 3) driven by exact lineal
// path counts, with candidate swaps evaluated in batches.
//
// Sequential equivalence.  Candidate number n of the run (n = 0, 1, ...) is
// drawn from Philox-4x32-10 with counter (n, 0, 0, 0) and the run's key, from
// the current image, and its Metropolis uniform comes from the same draw.  A
// batch evaluates candidates n_eval .. n_eval + K - 1 against the current
// state; the first one accepted is applied and the rest are discarded (they
// were drawn from, and evaluated on, the state a sequential annealer would
// also have had, because every earlier candidate was rejected and rejections
// do not change the state).  The next batch starts at the evaluation after
// the accepted one.  The run is therefore the sequential annealer, step for
// step, whatever the batch size.
//
// Readings of Alg. 3 (whose printed loop is garbled): a global evaluation
// counter runs to N_step; a temperature stage lasts until c_max attempts or
// s_max acceptances, then T <- T * T_mult with
// T_mult = (T_min / T_max)^(s_max / N_step); a move is accepted when
// Delta e <= 0 or U < exp(-Delta e / T) (minimisation).
// Modification operator (Sec. 4): exchange an interfacial phase-1 pixel with
// an interfacial phase-0 pixel (4-neighbourhood on the torus), each drawn
// uniformly from its list.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_device.cuh"
#include "lpf_state.hpp"

namespace lpf {

// ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

struct SaDev {
  double T, T_mult, e;
  long long n_eval, n_accept, n_batches, n_cand, c_stage, s_stage;
  long long n_step, c_max, s_max;
  double p_est;
  int k_eff, k_min, k_max, done;
  int acc_pair[2];
  float acc_de;
  int n1, n0;          // interfacial list sizes of the current batch
  unsigned int key0, key1;
};

constexpr int kProposeThreads = 1024;

// Interfacial lists (raster order) and the batch's candidates and uniforms.
__global__ void __launch_bounds__(kProposeThreads) sa_propose_kernel(const uint8_t* __restrict__ cell, int H, int W,
                                                                    SaDev* st, int32_t* __restrict__ list1,
                                                                    int32_t* __restrict__ list0,
                                                                    int32_t* __restrict__ pairs, float* __restrict__ u) {
  __shared__ int s_c1[kProposeThreads], s_c0[kProposeThreads];
  const int tid = threadIdx.x;
  const int npix = H * W;
  const int per = (npix + kProposeThreads - 1) / kProposeThreads;
  const int p0 = min(npix, tid * per), p1 = min(npix, p0 + per);
  int c1 = 0, c0 = 0;
  for (int p = p0; p < p1; ++p) {
    const int y = p / W, x = p - y * W;
    const int v = cell[p];
    const int l = cell[y * W + (x == 0 ? W - 1 : x - 1)], r = cell[y * W + (x == W - 1 ? 0 : x + 1)];
    const int t = cell[(y == 0 ? H - 1 : y - 1) * W + x], b = cell[(y == H - 1 ? 0 : y + 1) * W + x];
    const bool inter = (l != v) | (r != v) | (t != v) | (b != v);
    if (inter) { if (v) ++c1; else ++c0; }
  }
  s_c1[tid] = c1;
  s_c0[tid] = c0;
  __syncthreads();
  // exclusive scan (Hillis-Steele on both counts)
  for (int o = 1; o < kProposeThreads; o <<= 1) {
    const int a1 = tid >= o ? s_c1[tid - o] : 0, a0 = tid >= o ? s_c0[tid - o] : 0;
    __syncthreads();
    s_c1[tid] += a1;
    s_c0[tid] += a0;
    __syncthreads();
  }
  int o1 = s_c1[tid] - c1, o0 = s_c0[tid] - c0;
  const int n1 = s_c1[kProposeThreads - 1], n0 = s_c0[kProposeThreads - 1];
  for (int p = p0; p < p1; ++p) {
    const int y = p / W, x = p - y * W;
    const int v = cell[p];
    const int l = cell[y * W + (x == 0 ? W - 1 : x - 1)], r = cell[y * W + (x == W - 1 ? 0 : x + 1)];
    const int t = cell[(y == 0 ? H - 1 : y - 1) * W + x], b = cell[(y == H - 1 ? 0 : y + 1) * W + x];
    const bool inter = (l != v) | (r != v) | (t != v) | (b != v);
    if (inter) { if (v) list1[o1++] = p; else list0[o0++] = p; }
  }
  __syncthreads();
  if (tid == 0) {
    st->n1 = n1;
    st->n0 = n0;
    if (st->done || n1 == 0 || n0 == 0 || st->n_eval >= st->n_step) { st->done = 1; st->k_eff = 0; }
  }
  __syncthreads();
  const int K = st->k_eff;
  const unsigned long long base = (unsigned long long)st->n_eval;
  for (int k = tid; k < K; k += kProposeThreads) {
    const unsigned long long n = base + (unsigned long long)k;
    const U4 r = philox4x32_10(U4{(uint32_t)n, (uint32_t)(n >> 32), 0u, 0u}, st->key0, st->key1);
    const int ia = (int)(((unsigned long long)r.x * (unsigned)n1) >> 32);
    const int ib = (int)(((unsigned long long)r.y * (unsigned)n0) >> 32);
    pairs[2 * k] = list1[ia];
    pairs[2 * k + 1] = list0[ib];
    u[k] = ((float)(r.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
  }
}

// First accepted candidate of the batch, temperature schedule, bookkeeping.
__global__ void sa_accept_kernel(SaDev* st, const int32_t* __restrict__ pairs, const float* __restrict__ u,
                                 const float* __restrict__ de, int32_t* __restrict__ log_idx) {
  const int lane = threadIdx.x;
  const int K = st->k_eff;
  const long long c0 = st->c_stage;
  const long long cmax = st->c_max;
  const double T0 = st->T, Tm = st->T_mult;
  const long long left = st->n_step - st->n_eval;
  const int Kv = (int)min((long long)K, max(0LL, left));
  int kstar = -1;
  for (int b = 0; b < Kv && kstar < 0; b += 32) {
    const int k = b + lane;
    bool acc = false;
    if (k < Kv) {
      const double Tk = T0 * pow(Tm, (double)((c0 + k) / cmax));
      const float d = de[k];
      acc = d <= 0.0f || u[k] < expf(-d / (float)Tk);
    }
    const unsigned m = __ballot_sync(0xffffffffu, acc);
    if (m) kstar = b + __ffs(m) - 1;
  }
  if (lane != 0) return;
  long long consumed = kstar >= 0 ? kstar + 1 : Kv;
  // rejected attempts before the accepted one (or all of them)
  long long rej = kstar >= 0 ? kstar : Kv;
  long long c = c0 + rej, s = st->s_stage;
  double T = T0;
  const long long wraps = c / cmax;
  if (wraps > 0) { s = 0; }
  c -= wraps * cmax;
  T *= pow(Tm, (double)wraps);
  if (kstar >= 0) {
    c += 1;
    s += 1;
    if (c >= cmax || s >= st->s_max) { c = 0; s = 0; T *= Tm; }
    st->acc_pair[0] = pairs[2 * kstar];
    st->acc_pair[1] = pairs[2 * kstar + 1];
    st->acc_de = de[kstar];
    st->e += (double)de[kstar];
    st->n_accept += 1;
  } else {
    st->acc_pair[0] = 0;
    st->acc_pair[1] = 0;
    st->acc_de = 0.0f;
  }
  st->c_stage = c;
  st->s_stage = s;
  st->T = T;
  st->n_eval += consumed;
  st->n_cand += K;
  st->n_batches += 1;
  if (log_idx) log_idx[0] = kstar;
  // batch size for the next batch: about 4 expected acceptances' worth
  if (consumed > 0) {
    const double obs = (kstar >= 0 ? 1.0 : 0.0) / (double)consumed;
    st->p_est = 0.8 * st->p_est + 0.2 * obs;
  }
  const double want = 4.0 / fmax(st->p_est, 1e-9);
  st->k_eff = (int)fmin((double)st->k_max, fmax((double)st->k_min, want));
  if (st->n_eval >= st->n_step) st->done = 1;
}

// counts += change of the accepted exchange (canonical entries and their
// mirrors), then exchange the two pixels of the cell.
__global__ void sa_apply_kernel(SaDev* st, uint8_t* __restrict__ cell, const int32_t* __restrict__ dc,
                                int64_t n_canon, int64_t n_full, int64_t base, unsigned long long* __restrict__ counts) {
  const int a = st->acc_pair[0], b = st->acc_pair[1];
  if (a == b) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * n_canon; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / n_canon, v = i - p * n_canon;
    const long long d = dc[i];
    if (d == 0) continue;
    counts[p * n_full + base + v] += (unsigned long long)d;
    if (v > 0) counts[p * n_full + (n_full - 1 - (base + v))] += (unsigned long long)d;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint8_t t = cell[a];
    cell[a] = cell[b];
    cell[b] = t;
  }
}

// e = sum over both phases and the canonical half of (target - counts/N)^2, in double.
__global__ void sa_error_kernel(const float* __restrict__ target, const int64_t* __restrict__ counts, int64_t n_full,
                                int64_t base, double invN, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  const int64_t n = n_full - base;
  for (int64_t i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const int64_t p = i / n, k = base + i - p * n;
    const double d = (double)target[p * n_full + k] - (double)counts[p * n_full + k] * invN;
    acc += d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void sa_set_error_kernel(SaDev* st, const double* e) { st->e = *e; }

}  // namespace lpf

struct lpf_sa {
  lpf_paths* paths = nullptr;
  uint8_t* cell = nullptr;
  int H = 0, W = 0;
  const float* target = nullptr;
  int64_t* counts = nullptr;
  lpf_sa_params prm{};
  lpf::SaDev* d_st = nullptr;
  int32_t* d_list = nullptr;    // [2][H*W]
  int32_t* d_pairs = nullptr;   // [k_max][2]
  float* d_u = nullptr;         // [k_max]
  float* d_de = nullptr;        // [k_max]
  float* d_partial = nullptr;   // [k_max][n_chunks]
  int32_t* d_dc = nullptr;      // [2][n_canon]
  float* d_partial1 = nullptr;  // [n_chunks] (accepted-pair delta)
  double* d_e = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_batches = 0;
};

namespace lpf {

static void enqueue_batch(lpf_sa* sa, cudaStream_t s) {
  const Paths& h = sa->paths->host;
  sa_propose_kernel<<<1, kProposeThreads, 0, s>>>(sa->cell, sa->H, sa->W, sa->d_st, sa->d_list,
                                                    sa->d_list + (size_t)sa->H * sa->W, sa->d_pairs, sa->d_u);
  delta_launch(sa->cell, sa->H, sa->W, sa->paths, sa->d_pairs, sa->prm.k_max, &sa->d_st->k_eff, nullptr,
               sa->target, sa->counts, sa->d_de, sa->d_partial, s);
  sa_accept_kernel<<<1, 32, 0, s>>>(sa->d_st, sa->d_pairs, sa->d_u, sa->d_de, nullptr);
  delta_launch(sa->cell, sa->H, sa->W, sa->paths, sa->d_st->acc_pair, 1, nullptr, sa->d_dc, nullptr, nullptr,
               nullptr, sa->d_partial1, s);
  const int blocks = (int)std::min<int64_t>((2 * h.n_canon + 255) / 256, 1024);
  sa_apply_kernel<<<blocks, 256, 0, s>>>(sa->d_st, sa->cell, sa->d_dc, h.n_canon, h.n_full, h.base,
                                         reinterpret_cast<unsigned long long*>(sa->counts));
}

}  // namespace lpf

extern "C" {

int lpf_sa_create(uint8_t* cell_dev, int32_t H, int32_t W, lpf_paths* paths, const float* target_dev,
                  int64_t* counts_dev, const lpf_sa_params* prm, lpf_stream_t stream, lpf_sa** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (!cell_dev || !paths || !target_dev || !counts_dev || !prm) return LPF_EINVAL;
  if (prm->k_max < 1 || prm->k_max > (1 << 20) || prm->k_min < 1 || prm->k_min > prm->k_max) return LPF_EINVAL;
  if (prm->n_step < 1 || prm->c_max < 1 || prm->s_max < 1 || !(prm->t_min_ratio > 0.0)) return LPF_EINVAL;
  if ((int64_t)H * W > (1 << 24)) return LPF_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = lpf_full(cell_dev, H, W, paths, counts_dev, stream);
  if (rc) return rc;
  rc = lpf::delta_prepare(paths, H, W, prm->k_max);
  if (rc) return rc;
  lpf_sa* sa = new (std::nothrow) lpf_sa();
  if (!sa) return LPF_ENOMEM;
  sa->paths = paths;
  sa->cell = cell_dev;
  sa->H = H;
  sa->W = W;
  sa->target = target_dev;
  sa->counts = counts_dev;
  sa->prm = *prm;
  const int nch = paths->delta.n_chunks;
  const size_t npix = (size_t)H * W;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_st, sizeof(lpf::SaDev));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_list, 2 * npix * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_pairs, 2 * (size_t)prm->k_max * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_u, (size_t)prm->k_max * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_de, (size_t)prm->k_max * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_partial, (size_t)prm->k_max * nch * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_dc, 2 * (size_t)paths->host.n_canon * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_partial1, (size_t)nch * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_e, sizeof(double));
  if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }

  // initial error from the exact counts
  lpf::sa_error_kernel<<<1, 256, 0, s>>>(target_dev, counts_dev, paths->host.n_full, paths->host.base,
                                         1.0 / ((double)H * (double)W), sa->d_e);
  double e0 = 0.0;
  e = cudaMemcpyAsync(&e0, sa->d_e, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }

  lpf::SaDev st{};
  st.T = prm->t_max;
  st.T_mult = std::pow(prm->t_min_ratio, (double)prm->s_max / (double)prm->n_step);
  st.e = e0;
  st.n_step = prm->n_step;
  st.c_max = prm->c_max;
  st.s_max = prm->s_max;
  st.p_est = 0.5;
  st.k_min = prm->k_min;
  st.k_max = prm->k_max;
  st.k_eff = prm->k_min;
  st.key0 = (unsigned)(prm->seed & 0xffffffffu);
  st.key1 = (unsigned)(prm->seed >> 32);
  e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }

  if (!(prm->t_max > 0.0)) {
    // T_max so that an uphill move of average size is accepted with
    // probability 1/2 at the start: sample k_max candidates of the initial
    // state, T_max = -mean(positive Delta e) / ln(0.5).
    int32_t kk = prm->k_max;
    e = cudaMemcpyAsync(&sa->d_st->k_eff, &kk, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }
    lpf::sa_propose_kernel<<<1, lpf::kProposeThreads, 0, s>>>(cell_dev, H, W, sa->d_st, sa->d_list,
                                                              sa->d_list + npix, sa->d_pairs, sa->d_u);
    rc = lpf::delta_launch(cell_dev, H, W, paths, sa->d_pairs, prm->k_max, nullptr, nullptr, target_dev,
                           counts_dev, sa->d_de, sa->d_partial, s);
    std::vector<float> de(prm->k_max);
    if (!rc) {
      e = cudaMemcpyAsync(de.data(), sa->d_de, de.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = lpf::set_cuda_error(e);
    }
    if (rc) { lpf_sa_free(sa); return rc; }
    double sum = 0.0;
    int npos = 0;
    for (float d : de)
      if (d > 0.0f) { sum += d; ++npos; }
    const double tmax = npos ? -(sum / npos) / std::log(0.5) : 1e-12;
    st.T = tmax;
    sa->prm.t_max = tmax;
    st.k_eff = prm->k_min;
    e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }
  }
  *out = sa;
  return LPF_OK;
}

int lpf_sa_run(lpf_sa* sa, int32_t n_batches, lpf_stream_t stream) {
  if (!sa || n_batches < 0) return LPF_EINVAL;
  if (n_batches == 0) return LPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  // One captured graph holds kGraphBatches batches; replay it, then enqueue
  // the remainder directly.
  const int kGraphBatches = 8;
  cudaError_t e = cudaSuccess;
  if (!sa->exec && n_batches >= kGraphBatches) {
    // the handle's optional timer events are not recorded inside the graph
    cudaEvent_t ta = sa->paths->ev_start, tb = sa->paths->ev_stop;
    sa->paths->ev_start = sa->paths->ev_stop = nullptr;
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int i = 0; i < kGraphBatches; ++i) lpf::enqueue_batch(sa, cs);
      e = cudaStreamEndCapture(cs, &sa->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sa->exec, sa->graph, 0);
    cudaStreamDestroy(cs);
    sa->paths->ev_start = ta;
    sa->paths->ev_stop = tb;
    if (e != cudaSuccess) { sa->exec = nullptr; return lpf::set_cuda_error(e); }
    sa->graph_batches = kGraphBatches;
  }
  int left = n_batches;
  while (sa->exec && left >= sa->graph_batches) {
    e = cudaGraphLaunch(sa->exec, s);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
    left -= sa->graph_batches;
  }
  for (; left > 0; --left) lpf::enqueue_batch(sa, s);
  return lpf::set_cuda_error(cudaGetLastError());
}

int lpf_sa_read(lpf_sa* sa, lpf_sa_stats* out, lpf_stream_t stream) {
  if (!sa || !out) return LPF_EINVAL;
  lpf::SaDev st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&st, sa->d_st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  out->n_eval = st.n_eval;
  out->n_accept = st.n_accept;
  out->n_batches = st.n_batches;
  out->n_candidates = st.n_cand;
  out->temperature = st.T;
  out->error = st.e;
  out->t_max = sa->prm.t_max;
  out->next_batch = st.k_eff;
  out->done = st.done;
  return LPF_OK;
}

int lpf_sa_recompute_error(lpf_sa* sa, double* e_out, lpf_stream_t stream) {
  if (!sa) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::sa_error_kernel<<<1, 256, 0, s>>>(sa->target, sa->counts, sa->paths->host.n_full, sa->paths->host.base,
                                         1.0 / ((double)sa->H * (double)sa->W), sa->d_e);
  lpf::sa_set_error_kernel<<<1, 1, 0, s>>>(sa->d_st, sa->d_e);
  double e = 0.0;
  cudaError_t err = cudaMemcpyAsync(&e, sa->d_e, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return lpf::set_cuda_error(err);
  if (e_out) *e_out = e;
  return LPF_OK;
}

int lpf_sa_propose(lpf_sa* sa, int32_t k, int32_t* pairs_dev, float* u_dev, lpf_stream_t stream) {
  if (!sa || k < 1 || k > sa->prm.k_max || !pairs_dev || !u_dev) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::SaDev st;
  cudaError_t e = cudaMemcpyAsync(&st, sa->d_st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  const int keep = st.k_eff;
  const int done = st.done;
  st.k_eff = k;
  e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  lpf::sa_propose_kernel<<<1, lpf::kProposeThreads, 0, s>>>(sa->cell, sa->H, sa->W, sa->d_st, sa->d_list,
                                                            sa->d_list + (size_t)sa->H * sa->W, pairs_dev, u_dev);
  e = cudaMemcpyAsync(&st, sa->d_st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  st.k_eff = keep;
  st.done = done;
  e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return lpf::set_cuda_error(e == cudaSuccess ? cudaGetLastError() : e);
}

void lpf_sa_free(lpf_sa* sa) {
  if (!sa) return;
  cudaDeviceSynchronize();
  if (sa->exec) cudaGraphExecDestroy(sa->exec);
  if (sa->graph) cudaGraphDestroy(sa->graph);
  cudaFree(sa->d_st);
  cudaFree(sa->d_list);
  cudaFree(sa->d_pairs);
  cudaFree(sa->d_u);
  cudaFree(sa->d_de);
  cudaFree(sa->d_partial);
  cudaFree(sa->d_dc);
  cudaFree(sa->d_partial1);
  cudaFree(sa->d_e);
  delete sa;
}

}  // extern "C"
