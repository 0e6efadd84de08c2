// Annealer state and device pieces shared by its objectives (lineal path
// counts in lpf_sa.cu, the two-point probability in lpf_s2sa.cu).
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lpf.h"
#include "lpf_delta.cuh"

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

constexpr int kMaxTries = 1 << 16;  // rejection-sampling attempts before giving up (identity)

struct SaDev {
  double T, T_mult, e;
  long long n_eval, n_accept, n_batches, n_cand, c_stage, s_stage;
  long long n_step, c_max, s_max;
  double p_est;
  int k_eff, k_min, k_max, done;
  int acc_pair[2];
  float acc_de;
  unsigned int key0, key1;
  unsigned int ticket;   // blocks of the current batch that finished
  // learned proposer (see lpf_sa_set_proposer)
  int use_model;
  float eps;
  const float* cdf1;     // inclusive prefix sums of the phase-1 sampling weights [H*W]
  const float* cdf0;
  float tot1, tot0;
};

// Pixel value (0/1) of cell index c from an extended cell.
__device__ __forceinline__ int ext_pixel(const uint8_t* e, int c, const DeltaArgs& g) {
  return e[delta_ext_pos(c, g.W, g.We, g.rx, g.ry)];
}

__device__ __forceinline__ bool interfacial(const uint8_t* e, int c, const DeltaArgs& g) {
  const int y = c / g.W, x = c - y * g.W;
  const int v = e[(y + g.ry) * g.We + x + g.rx];
  const int l = e[(y + g.ry) * g.We + (x == 0 ? g.W - 1 : x - 1) + g.rx];
  const int r = e[(y + g.ry) * g.We + (x == g.W - 1 ? 0 : x + 1) + g.rx];
  const int t = e[((y == 0 ? g.H - 1 : y - 1) + g.ry) * g.We + x + g.rx];
  const int b = e[((y == g.H - 1 ? 0 : y + 1) + g.ry) * g.We + x + g.rx];
  return (l != v) | (r != v) | (t != v) | (b != v);
}

// Smallest pixel index p with cdf[p] > t (t < cdf[npix-1]).
__device__ __forceinline__ int cdf_search(const float* __restrict__ cdf, int npix, float t) {
  int lo = 0, hi = npix - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cdf + mid) > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Candidate n of the run: (a, b, U); a == b == 0 when no pair was found.
// With a model (use_model and the draw's word 3 >= epsilon), each pixel is
// drawn from the model's sampling weights instead of uniformly.
static __device__ void draw_candidate(const uint8_t* e, const DeltaArgs& g, unsigned long long n, uint32_t k0, uint32_t k1,
                               int& a, int& b, float& u, const SaDev* st = nullptr) {
  const unsigned npix = (unsigned)(g.H * g.W);
  a = -1;
  b = -1;
  bool model = false;
  for (uint32_t j = 0; j < (uint32_t)kMaxTries && (a < 0 || b < 0); ++j) {
    const U4 r = philox4x32_10(U4{(uint32_t)n, (uint32_t)(n >> 32), j, 0u}, k0, k1);
    if (j == 0) {
      u = ((float)(r.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
      model = st && st->use_model && st->tot1 > 0.0f && st->tot0 > 0.0f &&
              ((float)(r.w >> 8) + 0.5f) * (1.0f / 16777216.0f) >= st->eps;
    }
    if (a < 0) {
      const int c = model ? cdf_search(st->cdf1, (int)npix, ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f) * st->tot1)
                          : (int)(((unsigned long long)r.x * npix) >> 32);
      if (ext_pixel(e, c, g) == 1 && interfacial(e, c, g)) a = c;
    }
    if (b < 0) {
      const int c = model ? cdf_search(st->cdf0, (int)npix, ((float)(r.y >> 8) + 0.5f) * (1.0f / 16777216.0f) * st->tot0)
                          : (int)(((unsigned long long)r.y * npix) >> 32);
      if (ext_pixel(e, c, g) == 0 && interfacial(e, c, g)) b = c;
    }
  }
  if (a < 0 || b < 0) { a = 0; b = 0; }
}

// draw_candidate evaluated by a whole warp: lane j tries attempt j0 + j of
// the rejection sampling, and a ballot picks the lowest attempt that found a
// valid phase-1 pixel (and, independently, phase-0 pixel) -- the attempts the
// sequential loop would have kept.  Attempt 0 (lane 0 of the first round)
// gives U and the model choice.  Every lane returns the same (a, b, u).
__device__ __forceinline__ void draw_candidate_warp(const uint8_t* e, const DeltaArgs& g, unsigned long long n,
                                                    uint32_t k0, uint32_t k1, int& a, int& b, float& u,
                                                    const SaDev* st, int lane) {
  const unsigned npix = (unsigned)(g.H * g.W);
  a = -1;
  b = -1;
  bool model = false;
  for (uint32_t j0 = 0; j0 < (uint32_t)kMaxTries && (a < 0 || b < 0); j0 += 32) {
    const U4 r = philox4x32_10(U4{(uint32_t)n, (uint32_t)(n >> 32), j0 + (uint32_t)lane, 0u}, k0, k1);
    if (j0 == 0) {
      const float u0 = ((float)(r.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
      const int m0 = st && st->use_model && st->tot1 > 0.0f && st->tot0 > 0.0f &&
                     ((float)(r.w >> 8) + 0.5f) * (1.0f / 16777216.0f) >= st->eps;
      u = __shfl_sync(0xffffffffu, u0, 0);
      model = __shfl_sync(0xffffffffu, m0, 0) != 0;
    }
    int ca = -1, cb = -1;
    if (a < 0) {
      ca = model ? cdf_search(st->cdf1, (int)npix, ((float)(r.x >> 8) + 0.5f) * (1.0f / 16777216.0f) * st->tot1)
                 : (int)(((unsigned long long)r.x * npix) >> 32);
      if (!(ext_pixel(e, ca, g) == 1 && interfacial(e, ca, g))) ca = -1;
    }
    if (b < 0) {
      cb = model ? cdf_search(st->cdf0, (int)npix, ((float)(r.y >> 8) + 0.5f) * (1.0f / 16777216.0f) * st->tot0)
                 : (int)(((unsigned long long)r.y * npix) >> 32);
      if (!(ext_pixel(e, cb, g) == 0 && interfacial(e, cb, g))) cb = -1;
    }
    const unsigned ba = __ballot_sync(0xffffffffu, ca >= 0), bb = __ballot_sync(0xffffffffu, cb >= 0);
    if (a < 0 && ba) a = __shfl_sync(0xffffffffu, ca, __ffs(ba) - 1);
    if (b < 0 && bb) b = __shfl_sync(0xffffffffu, cb, __ffs(bb) - 1);
  }
  if (a < 0 || b < 0) { a = 0; b = 0; }
}

// ---- end of a batch (last block) -----------------------------------------

// The first candidate k < Kv that passes the Metropolis test (Delta e <= 0 or
// U < exp(-Delta e / T_k), T_k the temperature candidate k would see after k
// rejections), -1 if none; *de_star gets its error change.  A candidate's
// change is the sum of its n_chunks partials, added by one warp in a fixed
// order (lane-strided sums, then a fixed shuffle tree).  Every thread of the
// block calls this.
__device__ __forceinline__ int sa_first_accept(const SaDev* st, int Kv, const float* partial, int n_chunks,
                                               const float* u, float* de_star) {
  __shared__ float s_de[32];
  __shared__ int s_kstar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_kstar = INT_MAX;
  __syncthreads();
  const long long c0 = st->c_stage, cmax = st->c_max;
  const double T0 = st->T, Tm = st->T_mult;
  int k0 = 0;
  for (; k0 < Kv; k0 += nw) {
    const int k = k0 + warp;
    if (k < Kv) {
      // lane-strided sum in chunk order; the first 16 rounds are loaded
      // before they are added so that their latencies overlap
      const float* pk = partial + (int64_t)k * n_chunks;
      float v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = lane + 32 * r < n_chunks ? __ldcg(pk + lane + 32 * r) : 0.0f;
      float de = 0.0f;
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (lane + 32 * r < n_chunks) de += v[r];
      for (int c = lane + 32 * 16; c < n_chunks; c += 32) de += __ldcg(pk + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(0xffffffffu, de, o);
      if (lane == 0) {
        const long long wk = c0 + k >= cmax ? (c0 + k) / cmax : 0;  // stage ends before candidate k
        const double Tk = wk ? T0 * pow(Tm, (double)wk) : T0;
        const bool acc = de <= 0.0f || __ldcg(u + k) < expf(-de / (float)Tk);
        if (acc) atomicMin(&s_kstar, k);
        s_de[warp] = de;
      }
    }
    __syncthreads();
    if (s_kstar != INT_MAX) break;  // the first accepted candidate is known
    __syncthreads();
  }
  // (every exit from the loop, and an empty loop, follows a block barrier
  // after the last writes of s_kstar and s_de)
  const int kstar = s_kstar == INT_MAX ? -1 : s_kstar;
  *de_star = kstar >= 0 ? s_de[kstar - k0] : 0.0f;
  return kstar;
}

// Advance the run past a batch of Keff candidates of which Kv count (the
// rest lie beyond n_step) and kstar (or -1) was accepted: stage counters,
// temperature, error, statistics and the next batch size.  Thread 0 only.
__device__ __forceinline__ void sa_advance(SaDev* st, int Keff, int Kv, int kstar, float de_star, int acc_a,
                                           int acc_b) {
  const long long c0 = st->c_stage, cmax = st->c_max;
  const double Tm = st->T_mult;
  const long long consumed = kstar >= 0 ? kstar + 1 : Kv;
  const long long rej = kstar >= 0 ? kstar : Kv;
  long long c = c0 + rej, s = st->s_stage;
  double T = st->T;
  const long long wraps = c >= cmax ? c / cmax : 0;  // (a 64-bit division only when a stage ends)
  if (wraps > 0) {
    s = 0;
    T *= pow(Tm, (double)wraps);
  }
  c -= wraps * cmax;
  if (kstar >= 0) {
    c += 1;
    s += 1;
    if (c >= cmax || s >= st->s_max) { c = 0; s = 0; T *= Tm; }
    st->acc_pair[0] = acc_a;
    st->acc_pair[1] = acc_b;
    st->acc_de = de_star;
    st->e += (double)de_star;
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
  st->n_cand += Keff;
  if (Keff > 0) st->n_batches += 1;
  if (consumed > 0) {
    const double obs = (kstar >= 0 ? 1.0 : 0.0) / (double)consumed;
    st->p_est = 0.8 * st->p_est + 0.2 * obs;
  }
  // next batch size: a batch costs a fixed latency plus a share per
  // candidate and yields (1 - (1-p)^K) / p evaluations; with the measured
  // costs that ratio is best near K = 1/(2p)
  const float want = ceilf(0.5f / fmaxf((float)st->p_est, 1e-9f));
  st->k_eff = (int)fminf((float)st->k_max, fmaxf((float)st->k_min, want));
  if (st->n_eval >= st->n_step) st->done = 1;
  st->ticket = 0u;
}

// The serial end of a batch works on a copy of the run state in shared
// memory: loaded and stored back with one 8-byte word per thread, so that
// its many small reads and updates do not each wait for L2.
static_assert(sizeof(SaDev) % 8 == 0, "run state is copied in 8-byte words");
constexpr int kSaStateWords = (int)(sizeof(SaDev) / 8);

__device__ __forceinline__ void sa_state_load(SaDev* sh, const SaDev* st) {
  if ((int)threadIdx.x < kSaStateWords)
    reinterpret_cast<unsigned long long*>(sh)[threadIdx.x] =
        __ldcg(reinterpret_cast<const unsigned long long*>(st) + threadIdx.x);
  __syncthreads();
}

__device__ __forceinline__ void sa_state_store(SaDev* st, const SaDev* sh) {
  __syncthreads();
  if ((int)threadIdx.x < kSaStateWords)
    reinterpret_cast<unsigned long long*>(st)[threadIdx.x] = reinterpret_cast<const unsigned long long*>(sh)[threadIdx.x];
}

// Atomic ticket: true in the last block of the grid to get here (after a
// fence, so that it sees every other block's writes).  Every thread calls it.
__device__ __forceinline__ bool sa_last_block(SaDev* st) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y;
    s_last = (atomicAdd(&st->ticket, 1u) == total - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

}  // namespace lpf

enum { kSaObjectiveLineal = 0, kSaObjectiveS2 = 1 };

struct lpf_sa {
  lpf_paths* paths = nullptr;
  uint8_t* cell = nullptr;
  int H = 0, W = 0;
  const float* target = nullptr;
  int64_t* counts = nullptr;
  lpf_sa_params prm{};
  lpf::DeltaArgs g{};
  int delta_key = -1;           // the swap-delta tables' key (DeltaTables::want_key) the run was built on
  dim3 grid;
  lpf::SaDev* d_st = nullptr;
  uint8_t* d_ext = nullptr;
  int32_t* d_pairs = nullptr;   // [k_max][2]
  float* d_u = nullptr;         // [k_max]
  float* d_de = nullptr;        // [k_max]
  float* d_partial = nullptr;   // [k_max][n_chunks]
  int32_t* d_dc = nullptr;      // [k_max][2][n_canon]
  double* d_e = nullptr;
  int* d_status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_batches = 0;
  lpf_cnn* cnn = nullptr;       // learned proposer (optional)
  float tau = 1.0f;
  int refresh = 16;
  float* d_cdf = nullptr;       // [2][H*W] sampling tables
  int objective = kSaObjectiveLineal;
  int phase_mask = 3;           // phases in the lineal-path error
  int64_t err_n_full = 0, err_base = 0;  // error layout: [phase][err_n_full], summed from err_base
  int threads = 0;              // batch kernel block size
  int persistent = 0;           // batches run by the cooperative persistent kernel
  unsigned int* d_bar = nullptr;  // its grid-barrier counter
  uint8_t* d_sel_ext = nullptr; // Monte-Carlo runs: sampled translations, extended layout
  uint8_t* d_sel = nullptr;     // Monte-Carlo runs: the run's copy of the selection, H*W
  uint8_t* d_z = nullptr;       // phase-0 counts per (vector, translation), kept current by the run
  double inv_norm = 0.0;        // descriptor = count * inv_norm
};

namespace lpf {
// Enqueue one batch of the two-point-probability objective (lpf_s2sa.cu).
void s2_enqueue_batch(lpf_sa* sa, cudaStream_t s);
// Enqueue the recomputation of the run's error from its exact counts into
// sa->d_e, in double (lpf_sa.cu).
void sa_enqueue_error(lpf_sa* sa, cudaStream_t s);
// LPF_OK if the run parameters are valid (lpf_sa.cu).
int sa_check_params(const lpf_sa_params* prm);
// Recompute counts (from the cell) and error (from the counts) after a
// bounded wait gave up, and clear the run's status word (lpf_sa.cu).
int sa_recover(lpf_sa* sa, cudaStream_t s);
// Second half of both create calls once sa's geometry, objective and error
// layout are set: work buffers, extended cell, initial error and temperature,
// device state (lpf_sa.cu).
int sa_start(lpf_sa* sa, cudaStream_t s);
// S2 error changes (and count changes [K][H*W] if dcounts) of K candidate
// exchanges; ext/partial may be null (then allocated on the stream) (lpf_s2sa.cu).
int s2_delta_run(const uint8_t* img, int H, int W, const uint8_t* ext, const int32_t* pairs, int K, int32_t* dcounts,
                 const float* target, const int64_t* counts, float* de, float* partial, cudaStream_t s);
}  // namespace lpf

