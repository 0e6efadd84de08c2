// Simulated annealing on the GPU (Sec. 4, Alg. 3) driven by exact lineal
// path counts, with candidate swaps evaluated in batches.
//
// Sequential equivalence.  Candidate number n of the run (n = 0, 1, ...) is
// drawn from Philox-4x32-10 keyed by the run's seed, from the then-current
// cell, and carries its own Metropolis uniform.  A batch evaluates candidates
// n_eval .. n_eval + K - 1 against the current state; the first one accepted
// is applied and the rest are discarded: they were drawn from, and evaluated
// on, the state a sequential annealer would also have had, because every
// earlier candidate was rejected and rejections do not change the state.  The
// next batch starts at the evaluation after the accepted one, so the run is
// the sequential annealer step for step whatever the batch size.
//
// Readings of Alg. 3 (whose printed loop is garbled): a global evaluation
// counter runs to N_step; a temperature stage lasts until c_max attempts or
// s_max acceptances, then T <- T * T_mult with
// T_mult = (T_min / T_max)^(s_max / N_step); a move is accepted when
// Delta e <= 0 or U < exp(-Delta e / T) (minimisation).
// Modification operator (Sec. 4): exchange an interfacial phase-1 pixel with
// an interfacial phase-0 pixel (4-neighbourhood on the torus), each uniform
// over its set: attempt j = 0, 1, ... of candidate n draws Philox with counter
// (n_lo, n_hi, j, 0); word 0 and word 1 propose a pixel each by
// floor(r * H*W / 2^32), and the first proposal of the right phase that is
// interfacial is kept (rejection sampling); word 2 of attempt 0 gives
// U = ((r >> 8) + 1/2) / 2^24 in float32.
//
// One batch is one kernel launch: every block stages the extended cell, draws
// its candidates, writes their count changes and error-change partial sums;
// the last block to finish (atomic ticket) sums the partials in a fixed
// order, finds the first accepted candidate, applies it to the cell, the
// extended cell and the counts, and advances the schedule.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_sa.cuh"
#include "lpf_state.hpp"

namespace lpf {

// Sampling tables of the model: w_p = exp((s_p - max s) / tau) over the
// interfacial pixels of each phase (0 elsewhere), inclusive prefix sums in
// pixel order (one block; fixed summation order).
constexpr int kTableThreads = 1024;
__global__ void __launch_bounds__(kTableThreads) sa_tables_kernel(const uint8_t* __restrict__ ext, DeltaArgs g,
                                                                  const float* __restrict__ scores, float tau,
                                                                  float* __restrict__ cdf1, float* __restrict__ cdf0,
                                                                  SaDev* st) {
  __shared__ float s_red[2][kTableThreads];
  const int npix = g.H * g.W;
  const int per = (npix + kTableThreads - 1) / kTableThreads;
  const int p0 = min(npix, (int)threadIdx.x * per), p1 = min(npix, p0 + per);
  float m1 = -3.0e38f, m0 = -3.0e38f;
  for (int p = p0; p < p1; ++p) {
    if (!interfacial(ext, p, g)) continue;
    if (ext_pixel(ext, p, g)) m1 = fmaxf(m1, scores[2 * p + 1]); else m0 = fmaxf(m0, scores[2 * p]);
  }
  s_red[0][threadIdx.x] = m1;
  s_red[1][threadIdx.x] = m0;
  __syncthreads();
  for (int o = kTableThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_red[0][threadIdx.x] = fmaxf(s_red[0][threadIdx.x], s_red[0][threadIdx.x + o]);
      s_red[1][threadIdx.x] = fmaxf(s_red[1][threadIdx.x], s_red[1][threadIdx.x + o]);
    }
    __syncthreads();
  }
  m1 = s_red[0][0];
  m0 = s_red[1][0];
  __syncthreads();
  float a1 = 0.0f, a0 = 0.0f;
  for (int p = p0; p < p1; ++p) {
    const bool in = interfacial(ext, p, g);
    const int v = ext_pixel(ext, p, g);
    a1 += (in && v) ? __expf((scores[2 * p + 1] - m1) / tau) : 0.0f;
    a0 += (in && !v) ? __expf((scores[2 * p] - m0) / tau) : 0.0f;
  }
  s_red[0][threadIdx.x] = a1;
  s_red[1][threadIdx.x] = a0;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive offsets in thread order
    float c1 = 0.0f, c0 = 0.0f;
    for (int t = 0; t < kTableThreads; ++t) {
      const float x1 = s_red[0][t], x0 = s_red[1][t];
      s_red[0][t] = c1;
      s_red[1][t] = c0;
      c1 += x1;
      c0 += x0;
    }
    st->tot1 = c1;
    st->tot0 = c0;
  }
  __syncthreads();
  a1 = s_red[0][threadIdx.x];
  a0 = s_red[1][threadIdx.x];
  for (int p = p0; p < p1; ++p) {
    const bool in = interfacial(ext, p, g);
    const int v = ext_pixel(ext, p, g);
    a1 += (in && v) ? __expf((scores[2 * p + 1] - m1) / tau) : 0.0f;
    a0 += (in && !v) ? __expf((scores[2 * p] - m0) / tau) : 0.0f;
    cdf1[p] = a1;
    cdf0[p] = a0;
  }
}

// Candidates n0 .. n0+K-1 drawn from the extended cell in global memory.
__global__ void sa_draw_kernel(const uint8_t* __restrict__ ext, DeltaArgs g, unsigned long long n0, int K,
                               uint32_t k0, uint32_t k1, int32_t* __restrict__ pairs, float* __restrict__ u,
                               const SaDev* st) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    int a, b;
    float uu;
    draw_candidate(ext, g, n0 + (unsigned long long)k, k0, k1, a, b, uu, st);
    pairs[2 * k] = a;
    pairs[2 * k + 1] = b;
    u[k] = uu;
  }
}

// One annealing batch (see the file comment).
__global__ void __launch_bounds__(kDeltaThreads, 3) sa_batch_kernel(
    SaDev* __restrict__ st, uint8_t* __restrict__ cell, uint8_t* __restrict__ ext, DeltaArgs g,
    int32_t* __restrict__ pairs, float* __restrict__ u, int32_t* __restrict__ dcounts, float* __restrict__ partial,
    unsigned long long* __restrict__ counts, int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ float warp_acc[kDeltaWarps];
  __shared__ int s_a, s_b;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = blockIdx.x;
  const int Keff = st->done ? 0 : st->k_eff;
  const unsigned long long n0 = (unsigned long long)st->n_eval;

  if ((int)blockIdx.y < Keff) {
      if (!delta_stage(sm, ext, g.ext_bytes, &bar)) {
      if (threadIdx.x == 0) atomicOr(status, 1);
      (void)mbar_wait(&bar, 0);
    } else {
      const int v0 = g.chunk[ch], v1 = g.chunk[ch + 1];
      for (int k = blockIdx.y; k < Keff; k += gridDim.y) {
        if (warp == 0) {
          int a, b;
          float uu;
          draw_candidate_warp(sm, g, n0 + (unsigned long long)k, st->key0, st->key1, a, b, uu, st, lane);
          if (lane == 0) {
            if (ch == 0) { pairs[2 * k] = a; pairs[2 * k + 1] = b; u[k] = uu; }
            s_a = a;
            s_b = b;
            if (a != b) { delta_mark(sm, a, kMarkA, g); delta_mark(sm, b, kMarkB, g); }
          }
        }
        __syncthreads();
        const int a = s_a, b = s_b;
        int32_t* dk = dcounts + (int64_t)k * 2 * g.n_canon;
        float acc = 0.0f;
        if (a == b) delta_zero_vectors(g, v0, v1, dk);
        else acc = delta_walk_vectors(sm, g, a, b, v0, v1, warp, lane, dk, delta_terms_global(g));
        if (lane == 0) warp_acc[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
          float s = 0.0f;
          for (int w = 0; w < kDeltaWarps; ++w) s += warp_acc[w];
          partial[(int64_t)k * g.n_chunks + ch] = s;
          if (a != b) { delta_mark(sm, a, 1, g); delta_mark(sm, b, 0, g); }
        }
        __syncthreads();
      }
    }
  }

  // ---- last block: accept the first passing candidate and apply it ----
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
      // count changes of the accepted candidate: 8 independent loads per
      // round, then fire-and-forget atomic adds (this block alone writes the
      // counts now, so the adds only avoid waiting for each read)
      const int32_t* dk = dcounts + (int64_t)kstar * 2 * g.n_canon;
      const int64_t n2 = 2 * g.n_canon;
      for (int64_t i0 = threadIdx.x; i0 < n2; i0 += 8 * (int64_t)blockDim.x) {
        int d[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int64_t i = i0 + r * (int64_t)blockDim.x;
          d[r] = i < n2 ? __ldcg(dk + i) : 0;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (d[r] == 0) continue;
          const int64_t i = i0 + r * (int64_t)blockDim.x;
          const int64_t p = i / g.n_canon, v = i - p * g.n_canon;
          const unsigned long long dd = (unsigned long long)(long long)d[r];
          atomicAdd(counts + p * g.n_full + g.base + v, dd);
          if (v > 0) atomicAdd(counts + p * g.n_full + (g.n_full - 1 - (g.base + v)), dd);
        }
      }
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

// ---- persistent annealer ----------------------------------------------------
//
// The same sequence of batches as sa_batch_kernel, run by one cooperative
// launch whose blocks stay resident for n_batches batches: block c owns
// vector chunk c (the grid is exactly the chunk count, all blocks co-resident)
// and keeps its extended cell and a copy of the run state in shared memory.
// Per batch every block draws the batch's candidates, evaluates its chunk
// for each (with the phase-0 counts: the chunk's lookups spread over all
// threads of the block, so that every block takes about the same time to
// reach the barrier; else walks) and writes its partial error changes; after one grid barrier every
// block sums the partials of each candidate in the same fixed order, so all
// blocks find the same first accepted candidate, apply it to their own cell
// copy and to the counts of their own vectors, and advance their identical
// copies of the run state.  Partials, pairs and uniforms alternate between
// two buffers by batch parity: batch b + 2 may overwrite batch b's only after
// the barrier of batch b + 1, which no block reaches before it has read them.

constexpr uint32_t kBarrierPolls = 1u << 22;  // polls of a grid barrier before giving up (seconds)

// Grid barrier on a counter that only grows: block arrivals up to the end of
// batch b are (b + 1) * gridDim.x.  False (and status bit 4) if the other
// blocks did not arrive within kBarrierPolls polls.
__device__ __forceinline__ bool sa_grid_barrier(unsigned int* count, unsigned int target, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // arrive with release and acquire semantics (this block's partials and,
    // for block 0, the batch's candidates go out; the others' come in): the
    // last block to arrive sees the full count at once, the others poll
    // with acquiring loads
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
    int ok = old + 1u >= target;
    for (uint32_t it = 0; !ok && it < kBarrierPolls; ++it) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) ok = 1;
      else __nanosleep(32);
    }
    if (!ok) atomicOr(status, 4);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kDeltaThreads, 3) sa_persistent_kernel(
    SaDev* __restrict__ st, uint8_t* __restrict__ cell, uint8_t* __restrict__ ext, DeltaArgs g,
    int32_t* __restrict__ pairs2, float* __restrict__ u2, int32_t* __restrict__ dcounts, float* __restrict__ partial2,
    unsigned long long* __restrict__ counts, int* __restrict__ status, unsigned int* __restrict__ bar, int n_batches,
    int k_max, unsigned int bar_extra, int bar_block) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ SaDev s_state;
  __shared__ float warp_acc[kDeltaWarps];
  __shared__ int s_a, s_b, s_na, s_nb;
  __shared__ PixelPair s_q, s_nq;  // the pixels of s_a, s_b and of s_na, s_nb as coordinates
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = blockIdx.x;
  const int v0 = g.chunk[ch], v1 = g.chunk[ch + 1], nv = v1 - v0;
  sa_state_load(&s_state, st);
  if (!delta_stage(sm, ext, g.ext_bytes, &mbar)) {
    if (threadIdx.x == 0) atomicOr(status, 1);
    (void)mbar_wait(&mbar, 0);
  }
  // this chunk's targets and counts stay in shared memory after the cell
  // for the whole launch; the counts are kept exact there and written through
  const int mv = g.max_chunk_vecs;
  long long* s_cnt = reinterpret_cast<long long*>(sm + g.ext_bytes);  // [2][mv]
  float* s_tgt = reinterpret_cast<float*>(s_cnt + 2 * mv);            // [2][mv]
  // the chunk's tables for the block-wide lookups and updates (lookup path)
  ChunkTables ct;
  int32_t* s_pre = reinterpret_cast<int32_t*>(s_tgt + 2 * mv);        // [mv + 1]
  short2* s_vec = reinterpret_cast<short2*>(s_pre + mv + 1);          // [mv]
  ct.pre = s_pre;
  ct.vec = s_vec;
  ct.d = reinterpret_cast<int32_t*>(s_vec + mv);                      // [2][mv]
  ct.term = reinterpret_cast<float*>(ct.d + 2 * mv);                  // [mv]
  int32_t* s_shear = reinterpret_cast<int32_t*>(ct.term + mv);       // [mv]
  short2* s_off = reinterpret_cast<short2*>(s_shear + mv);            // [max_chunk_entries]
  uint16_t* s_vid = reinterpret_cast<uint16_t*>(s_off + g.max_chunk_entries);  // [max_chunk_entries]
  ct.shear = s_shear;
  ct.off = s_off;
  ct.vid = s_vid;
  ct.nv = nv;
  ct.mv = mv;
  const int o_base = g.dptr[v0], n_ent = g.dptr[v1] - o_base;
  for (int i = threadIdx.x; i <= nv; i += blockDim.x) {
    s_pre[i] = g.dptr[v0 + i] - o_base;
    if (i < nv) {
      const short2 dv = reinterpret_cast<const short2*>(g.vec16)[v0 + i];
      s_vec[i] = dv;
      s_shear[i] = g.shear[v0 + i];
    }
  }
  __syncthreads();  // s_pre is complete
  for (int j = threadIdx.x; j < n_ent; j += blockDim.x) {
    s_off[j] = reinterpret_cast<const short2*>(g.off16)[o_base + j];
    s_vid[j] = (uint16_t)chunk_vector_of(s_pre, nv, j);
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      s_tgt[p * mv + i] = g.target[p * g.n_full + g.base + v0 + i];
      s_cnt[p * mv + i] = (long long)counts[p * g.n_full + g.base + v0 + i];
    }
  }
  __syncthreads();
  DeltaTerms dt;
  dt.t[0] = s_tgt;
  dt.t[1] = s_tgt + mv;
  dt.c[0] = s_cnt;
  dt.c[1] = s_cnt + mv;
  dt.vbase = v0;
  uint32_t held = 0;  // the phase-0 counts this thread read for candidate held_k
  uint32_t held_zi[kChunkUnroll] = {0, 0, 0, 0};  // and where they are in z
  int held_k = -1;
  // Candidate k of batch bi (warp 0): drawn from the block's own cell copy,
  // marked there, kept in *sa / *sb; block 0 also records it for the others.
  // (n0: the batch's first evaluation index; the draw reads only the run
  // state's fixed fields, so it may run while warp 0 advances the rest)
  auto draw = [&](int bi, unsigned long long n0, int k, int* sa, int* sb, PixelPair* sq) {
    int a, b;
    float uu;
    draw_candidate_warp(sm, g, n0 + (unsigned long long)k, s_state.key0, s_state.key1, a, b, uu, &s_state, lane);
    if (lane == 0) {
      if (ch == 0) {
        pairs2[(size_t)(bi & 1) * 2 * k_max + 2 * k] = a;
        pairs2[(size_t)(bi & 1) * 2 * k_max + 2 * k + 1] = b;
        u2[(size_t)(bi & 1) * k_max + k] = uu;
        __threadfence();  // written by a thread other than the one that arrives at the grid barrier
      }
      *sa = a;
      *sb = b;
      sq->ay = a / g.W;
      sq->ax = a - sq->ay * g.W;
      sq->by = b / g.W;
      sq->bx = b - sq->by * g.W;
      if (a != b) { delta_mark(sm, a, kMarkA, g); delta_mark(sm, b, kMarkB, g); }
    }
  };
  // The first candidate of every batch is drawn ahead, by warp 1 at the end
  // of the batch before (while warp 0 advances the run state and the other
  // warps apply the exchange), into s_na, s_nb; later candidates of a batch
  // go through s_a, s_b.
  if (warp == 1 && !s_state.done && n_batches > 0) draw(0, (unsigned long long)s_state.n_eval, 0, &s_na, &s_nb, &s_nq);
  __syncthreads();
  for (int bi = 0; bi < n_batches && !s_state.done; ++bi) {
    const int Keff = s_state.k_eff;
    const unsigned long long n0 = (unsigned long long)s_state.n_eval;
    int32_t* pairs = pairs2 + (size_t)(bi & 1) * 2 * k_max;
    float* u = u2 + (size_t)(bi & 1) * k_max;
    float* partial = partial2 + (size_t)(bi & 1) * k_max * g.n_chunks;
    int last_a = 0, last_b = 0;  // the batch's last candidate
    PixelPair last_q = {0, 0, 0, 0};
    for (int k = 0; k < Keff; ++k) {
      if (k > 0 && warp == 0) draw(bi, n0, k, &s_a, &s_b, &s_q);
      __syncthreads();
      const int a = k == 0 ? s_na : s_a, b = k == 0 ? s_nb : s_b;
      const PixelPair q = k == 0 ? s_nq : s_q;
      last_a = a;
      last_b = b;
      last_q = q;
      int32_t* dk = dcounts + (int64_t)k * 2 * g.n_canon;
      float acc = 0.0f;
      const bool block_sum = a != b && g.z;  // block-wide lookups: thread 0 holds the chunk's sum
      held_k = -1;
      if (a == b) delta_zero_vectors(g, v0, v1, dk);
      else if (g.z) {
        acc = delta_chunk_lookup(g, q, v0, ct, dk, dt, &held, held_zi);
        if (2 * n_ent <= kChunkUnroll * (int)blockDim.x) held_k = k;  // this candidate's counts stay in registers
      }
      else acc = delta_walk_vectors(sm, g, a, b, v0, v1, warp, lane, dk, dt);
      if (!block_sum && lane == 0) warp_acc[warp] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        float sum = 0.0f;
        if (block_sum) sum = acc;
        else
          for (int w = 0; w < kDeltaWarps; ++w) sum += warp_acc[w];
        partial[(int64_t)k * g.n_chunks + ch] = sum;
        if (a != b) { delta_mark(sm, a, 1, g); delta_mark(sm, b, 0, g); }
      }
      __syncthreads();
    }
    // (bar_extra > 0 only in lpf_sa_selftest_timeout: a target that block
    // bar_block, or every block if bar_block < 0, never reaches)
    const unsigned int extra = (bar_block < 0 || (int)blockIdx.x == bar_block) ? bar_extra : 0u;
    if (!sa_grid_barrier(bar, (unsigned int)(bi + 1) * gridDim.x + extra, status)) break;

    const long long left = s_state.n_step - s_state.n_eval;
    const int Kv = (int)min((long long)Keff, max(0LL, left));
    float de_star;
    const int kstar = sa_first_accept(&s_state, Kv, partial, g.n_chunks, u, &de_star);
    int acc_a = 0, acc_b = 0;
    if (kstar >= 0) {
      // every block drew the candidates itself and holds the last one
      const int a = kstar == Keff - 1 ? last_a : __ldcg(pairs + 2 * kstar);
      const int b = kstar == Keff - 1 ? last_b : __ldcg(pairs + 2 * kstar + 1);
      acc_a = a;
      acc_b = b;
      if (a != b) {
        // this block's vectors: apply the accepted candidate's changes
        // (the block-wide lookups of the last candidate left its changes in ct.d)
        const bool in_smem = held_k == kstar && held_k >= 0;
        const int32_t* dk = dcounts + (int64_t)kstar * 2 * g.n_canon;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
          const int v = v0 + i;
          const int d0 = in_smem ? ct.d[i] : dk[v], d1 = in_smem ? ct.d[mv + i] : dk[(int64_t)g.n_canon + v];
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const int d = p ? d1 : d0;
            if (d == 0) continue;
            const long long c = s_cnt[p * mv + i] + d;
            s_cnt[p * mv + i] = c;
            counts[p * g.n_full + g.base + v] = (unsigned long long)c;
            if (v > 0) counts[p * g.n_full + (g.n_full - 1 - (g.base + v))] = (unsigned long long)c;
          }
        }
        // this block's vectors: the phase-0 counts follow the exchange
        if (g.z) {
          if (held_k == kstar) {
            delta_chunk_apply_held(g, last_q, v0, ct, held, held_zi);
          } else {
            const PixelPair qk = {a % g.W, a / g.W, b % g.W, b / g.W};
            delta_chunk_update(g, qk, v0, ct);
          }
        }
      }
    }
    // warp 0 advances the run state (and block 0 writes the exchange to the
    // cell); warp 1 makes the exchange on the block's cell copy and draws
    // the next batch's first candidate on it
    if (warp == 0) {
      if (lane == 0) {
        if (ch == 0 && kstar >= 0 && acc_a != acc_b) {
          cell[acc_a] = 0;
          cell[acc_b] = 1;
          delta_mark(ext, acc_a, 0, g);
          delta_mark(ext, acc_b, 1, g);
        }
        sa_advance(&s_state, Keff, Kv, kstar, de_star, acc_a, acc_b);
      }
    } else if (warp == 1) {
      if (lane == 0 && kstar >= 0 && acc_a != acc_b) {
        delta_mark(sm, acc_a, 0, g);
        delta_mark(sm, acc_b, 1, g);
      }
      __syncwarp();
      const unsigned long long n_next = n0 + (unsigned long long)(kstar >= 0 ? kstar + 1 : Kv);
      if ((long long)n_next < s_state.n_step && bi + 1 < n_batches) draw(bi + 1, n_next, 0, &s_na, &s_nb, &s_nq);
    }
    __syncthreads();
  }
  if (ch == 0) sa_state_store(st, &s_state);
}

// e = sum over the phases p in phase_mask and base <= k < n_full of
// (target[p][k] - counts[p][k] / N)^2, in double (one block of 256 threads).
__global__ void sa_error_kernel(const float* __restrict__ target, const int64_t* __restrict__ counts, int64_t n_full,
                                int64_t base, int phase_mask, double invN, double* __restrict__ out) {
  __shared__ double sh[256];
  double acc = 0.0;
  const int64_t n = n_full - base;
  for (int64_t i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    const int64_t p = i / n, k = base + i - p * n;
    if (!(phase_mask & (1 << p))) continue;
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

__global__ void build_ext_sa_kernel(const uint8_t* __restrict__ img, DeltaArgs g, uint8_t* __restrict__ ext) {
  const int total = g.We * g.He;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)g.ext_bytes; i += gridDim.x * blockDim.x) {
    uint8_t v = 0;
    if (i < total) {
      const int ey = i / g.We, ex = i - ey * g.We;
      int y = (ey - g.ry) % g.H; if (y < 0) y += g.H;
      int x = (ex - g.rx) % g.W; if (x < 0) x += g.W;
      v = img[y * g.W + x] != 0;
    }
    ext[i] = v;
  }
}

}  // namespace lpf

namespace lpf {

const void* sa_batch_kernel_entry() { return reinterpret_cast<const void*>(&sa_batch_kernel); }
const void* sa_persistent_kernel_entry() { return reinterpret_cast<const void*>(&sa_persistent_kernel); }

constexpr int kPersistentBatches = 4096;  // batches per persistent launch (bounds one launch's duration)

static size_t persistent_smem(const DeltaArgs& g) {
  return persistent_smem_bytes(g.ext_bytes, g.max_chunk_vecs, g.max_chunk_entries);
}

// Launch the persistent annealer for nb batches (cooperative launch: every
// block is resident, which its grid barrier relies on).
static int launch_persistent(lpf_sa* sa, int nb, cudaStream_t s, unsigned int bar_extra = 0, int bar_block = -1) {
  cudaError_t e = cudaMemsetAsync(sa->d_bar, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return set_cuda_error(e);
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(sa->counts);
  int k_max = sa->prm.k_max;
  void* args[] = {&sa->d_st, &sa->cell, &sa->d_ext, &sa->g, &sa->d_pairs, &sa->d_u, &sa->d_dc, &sa->d_partial,
                  &counts, &sa->d_status, &sa->d_bar, &nb, &k_max, &bar_extra, &bar_block};
  e = cudaLaunchCooperativeKernel(sa_persistent_kernel_entry(), dim3(sa->g.n_chunks), dim3(kDeltaThreads), args,
                                  persistent_smem(sa->g), s);
  return set_cuda_error(e);
}

// Score the current cell with the network and rebuild the sampling tables.
static void enqueue_refresh(lpf_sa* sa, cudaStream_t s) {
  if (!sa->cnn) return;
  cnn_forward(sa->cnn, sa->cell, s);
  const size_t npix = (size_t)sa->H * sa->W;
  sa_tables_kernel<<<1, kTableThreads, 0, s>>>(sa->d_ext, sa->g, cnn_scores(sa->cnn), sa->tau, sa->d_cdf,
                                               sa->d_cdf + npix, sa->d_st);
}

static void enqueue_batch(lpf_sa* sa, cudaStream_t s) {
  if (sa->objective == kSaObjectiveS2) {
    s2_enqueue_batch(sa, s);
    return;
  }
  sa_batch_kernel<<<sa->grid, kDeltaThreads, sa->g.ext_bytes, s>>>(
      sa->d_st, sa->cell, sa->d_ext, sa->g, sa->d_pairs, sa->d_u, sa->d_dc, sa->d_partial,
      reinterpret_cast<unsigned long long*>(sa->counts), sa->d_status);
}

void sa_enqueue_error(lpf_sa* sa, cudaStream_t s) {
  sa_error_kernel<<<1, 256, 0, s>>>(sa->target, sa->counts, sa->err_n_full, sa->err_base, sa->phase_mask,
                                    sa->inv_norm > 0.0 ? sa->inv_norm : 1.0 / ((double)sa->H * (double)sa->W),
                                    sa->d_e);
}

static int sa_device_state(lpf_sa* sa, SaDev& st, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(&st, sa->d_st, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return set_cuda_error(e);
}

// Make the run state consistent again after a bounded wait gave up.  The
// cell, its extended copy in global memory and the run state are written by
// one block only (block 0 of the persistent kernel, the last block of a batch
// kernel), so they always agree; the counts are written per vector chunk by
// every block, and after a grid barrier that timed out in some blocks only,
// some chunks hold the counts after a swap that the cell does not show.  So
// the counts are recomputed from the cell (exact integers) and the error from
// the counts, and the run continues from the cell's state.
// A lineal-path run reads the swap-delta tables of its paths handle (vector
// chunks, segment pixels, shears).  Another call on the handle with another
// cell width re-bakes them, so before every launch the run asks for its own
// width's tables again (a no-op when they are in place) and takes their
// current addresses; the chunking of a width never changes.
static int sa_bind_tables(lpf_sa* sa) {
  if (sa->objective != kSaObjectiveLineal) return LPF_OK;
  const DeltaTables& t = sa->paths->delta;
  if (!(t.d_doff && t.We == sa->g.We && t.want_key == sa->delta_key)) {  // re-baked for another cell
    const int rc = delta_prepare(sa->paths, sa->H, sa->W, 1);
    if (rc) return rc;
    if (t.want_key != sa->delta_key) return LPF_EINVAL;  // (a cell of this width but another height)
  }
  if (t.n_chunks != sa->g.n_chunks || t.max_chunk_vecs != sa->g.max_chunk_vecs ||
      t.max_chunk_entries != sa->g.max_chunk_entries)
    return LPF_EINVAL;
  if (sa->g.chunk != t.d_chunk || sa->g.dptr != t.d_dptr || sa->g.doff != t.d_doff || sa->g.off16 != t.d_off16 ||
      sa->g.vec16 != t.d_vec16 || sa->g.shear != t.d_shear) {
    sa->g.chunk = t.d_chunk;
    sa->g.dptr = t.d_dptr;
    sa->g.doff = t.d_doff;
    sa->g.off16 = t.d_off16;
    sa->g.vec16 = t.d_vec16;
    sa->g.shear = t.d_shear;
    // a captured graph of batches holds the old addresses
    if (sa->exec) { cudaGraphExecDestroy(sa->exec); sa->exec = nullptr; }
    if (sa->graph) { cudaGraphDestroy(sa->graph); sa->graph = nullptr; }
  }
  return LPF_OK;
}

int sa_recover(lpf_sa* sa, cudaStream_t s) {
  int rc = sa_bind_tables(sa);
  if (rc) return rc;
  if (sa->objective == kSaObjectiveS2) rc = s2_counts(sa->cell, sa->H, sa->W, sa->counts, s);
  else if (sa->d_sel) rc = lpf_full_mc(sa->cell, sa->H, sa->W, sa->paths, sa->d_sel, sa->counts, s);
  else rc = lpf_full(sa->cell, sa->H, sa->W, sa->paths, sa->counts, s);
  if (rc) return rc;
  if (sa->d_z) z_init_launch(sa->d_ext, sa->g, sa->d_z, sa->d_status, s);  // the counts per translation too
  sa_enqueue_error(sa, s);
  sa_set_error_kernel<<<1, 1, 0, s>>>(sa->d_st, sa->d_e);
  cudaError_t e = cudaMemsetAsync(sa->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  return set_cuda_error(e);
}

int sa_check_params(const lpf_sa_params* prm) {
  if (prm->k_max < 1 || prm->k_max > (1 << 16) || prm->k_min < 1 || prm->k_min > prm->k_max) return LPF_EINVAL;
  if (prm->n_step < 1 || prm->c_max < 1 || prm->s_max < 1 || !(prm->t_min_ratio > 0.0)) return LPF_EINVAL;
  if (prm->phases < 0 || prm->phases > 3) return LPF_EINVAL;
  return LPF_OK;
}

// Second half of both create calls, once sa's geometry (g, grid, objective,
// error layout) is set: work buffers, the extended cell, the initial error,
// the initial temperature and the device state.
int sa_start(lpf_sa* sa, cudaStream_t s) {
  const lpf_sa_params* prm = &sa->prm;
  const int nch = sa->g.n_chunks;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_st, sizeof(SaDev));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_ext, sa->g.ext_bytes);
  // pairs, uniforms and partials: two buffers each (the persistent kernel
  // alternates between them by batch parity; the batch kernel uses the first)
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_pairs, 2 * 2 * (size_t)prm->k_max * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_u, 2 * (size_t)prm->k_max * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_de, (size_t)prm->k_max * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_partial, 2 * (size_t)prm->k_max * nch * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_bar, sizeof(unsigned int));
  if (e == cudaSuccess && sa->objective == kSaObjectiveLineal)
    e = cudaMalloc(&sa->d_dc, (size_t)prm->k_max * 2 * (size_t)sa->paths->host.n_canon * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_e, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sa->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(sa->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return set_cuda_error(e);
  {
    const int blocks = (int)std::min<int64_t>((sa->g.ext_bytes + 255) / 256, 4096);
    build_ext_sa_kernel<<<blocks, 256, 0, s>>>(sa->cell, sa->g, sa->d_ext);
  }
  if (sa->objective == kSaObjectiveLineal && sa->persistent) {
    // count changes by lookups of the run's own phase-0 counts, kept current
    // by the persistent kernel after every accepted exchange
    const size_t zb = delta_z_bytes(sa->paths, sa->H, sa->W);
    if (zb > 0) {
      e = cudaMalloc(&sa->d_z, zb);
      if (e != cudaSuccess) return set_cuda_error(e);
      sa->g.z = sa->d_z;
      z_init_launch(sa->d_ext, sa->g, sa->d_z, sa->d_status, s);
    }
  }
  sa_enqueue_error(sa, s);  // initial error from the exact counts
  double e0 = 0.0;
  e = cudaMemcpyAsync(&e0, sa->d_e, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_cuda_error(e);

  SaDev st{};
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

  if (!(prm->t_max > 0.0)) {
    // T_max so that an uphill move of average size is accepted with
    // probability 1/2 at the start: k_max candidates of the initial state,
    // T_max = -mean(positive Delta e) / ln(0.5).
    const int K = prm->k_max;
    sa_draw_kernel<<<(K + 127) / 128, 128, 0, s>>>(sa->d_ext, sa->g, 0ull, K, st.key0, st.key1, sa->d_pairs,
                                                   sa->d_u, nullptr);
    int rc;
    if (sa->objective == kSaObjectiveS2) {
      rc = s2_delta_run(sa->cell, sa->H, sa->W, sa->d_ext, sa->d_pairs, K, nullptr, sa->target, sa->counts, sa->d_de,
                        sa->d_partial, s);
    } else {
      rc = delta_prepare(sa->paths, sa->H, sa->W, K);
      if (!rc)
        rc = delta_swap_run(sa->cell, sa->H, sa->W, sa->paths, sa->d_pairs, K, nullptr, sa->target, sa->counts,
                            sa->d_de, sa->phase_mask, s, sa->d_sel_ext, (float)sa->inv_norm);
    }
    std::vector<float> de(K);
    if (!rc) {
      e = cudaMemcpyAsync(de.data(), sa->d_de, de.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) rc = set_cuda_error(e);
    }
    if (rc) return rc;
    double sum = 0.0;
    int npos = 0;
    for (float d : de)
      if (d > 0.0f) { sum += d; ++npos; }
    st.T = npos ? -(sum / npos) / std::log(0.5) : 1e-12;
    sa->prm.t_max = st.T;
  }
  e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return set_cuda_error(e);
}

}  // namespace lpf

extern "C" {

}  // extern "C"

namespace lpf {

// Lineal-path annealer on all translations (sel_dev null) or on the sampled
// ones (Monte-Carlo variant).
static int sa_create_lineal(uint8_t* cell_dev, int32_t H, int32_t W, lpf_paths* paths, const float* target_dev,
                            int64_t* counts_dev, const uint8_t* sel_dev, const lpf_sa_params* prm,
                            lpf_stream_t stream, lpf_sa** out) {
  if (!out) return LPF_EINVAL;
  *out = nullptr;
  if (!cell_dev || !paths || !target_dev || !counts_dev || !prm) return LPF_EINVAL;
  if (int rc = sa_check_params(prm)) return rc;
  if ((int64_t)H * W > (1 << 24)) return LPF_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t n_sel = 0;
  if (sel_dev) {
    int rc = count_selected(sel_dev, H, W, s, &n_sel);
    if (rc) return rc;
    if (n_sel == 0) return LPF_EINVAL;
  }
  int rc = sel_dev ? lpf_full_mc(cell_dev, H, W, paths, sel_dev, counts_dev, stream)
                   : lpf_full(cell_dev, H, W, paths, counts_dev, stream);
  if (rc) return rc;
  rc = delta_prepare(paths, H, W, 1);
  if (rc) return rc;
  lpf_sa* sa = new (std::nothrow) lpf_sa();
  if (!sa) return LPF_ENOMEM;
  if (sel_dev) {
    rc = build_sel_ext(sel_dev, H, W, paths, s, &sa->d_sel_ext);
    if (rc) { lpf_sa_free(sa); return rc; }
    sa->inv_norm = 1.0 / (double)n_sel;
    // the run's own copy of the selection (counts are recomputed from it after a failed wait)
    cudaError_t e = cudaMalloc(&sa->d_sel, (size_t)H * W);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sa->d_sel, sel_dev, (size_t)H * W, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }
  }
  sa->paths = paths;
  sa->cell = cell_dev;
  sa->H = H;
  sa->W = W;
  sa->target = target_dev;
  sa->counts = counts_dev;
  sa->prm = *prm;
  sa->objective = kSaObjectiveLineal;
  sa->phase_mask = prm->phases ? prm->phases : 3;
  sa->err_n_full = paths->host.n_full;
  sa->err_base = paths->host.base;
  sa->threads = lpf::kDeltaThreads;
  lpf::delta_geometry(paths, H, W, sa->g);
  sa->delta_key = paths->delta.want_key;
  sa->g.target = target_dev;
  sa->g.counts = counts_dev;
  sa->g.phase_mask = sa->phase_mask;
  sa->g.sel_ext = sa->d_sel_ext;
  if (sa->inv_norm > 0.0) sa->g.inv_norm = (float)sa->inv_norm;
  sa->grid = dim3(sa->g.n_chunks, lpf::delta_stride(sa->g.n_chunks, prm->k_max));
  {
    // persistent batches when the device launches cooperatively and every
    // chunk's block fits at once (the chunk count is sized for that)
    int dev = 0, coop = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = lpf::persistent_smem(sa->g);
    if (e == cudaSuccess && (int64_t)smem <= lpf::delta_max_smem())
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lpf::sa_persistent_kernel_entry(), lpf::kDeltaThreads,
                                                        smem);
    if (e != cudaSuccess) { lpf_sa_free(sa); return lpf::set_cuda_error(e); }
    // (the block-wide lookups number a chunk's vectors in 16 bits)
    sa->persistent = (coop && occ > 0 && sa->g.n_chunks <= occ * sms && sa->g.max_chunk_vecs <= 65535) ? 1 : 0;
  }
  rc = lpf::sa_start(sa, s);
  if (rc) { lpf_sa_free(sa); return rc; }
  *out = sa;
  return LPF_OK;
}

}  // namespace lpf

extern "C" {

int lpf_sa_create(uint8_t* cell_dev, int32_t H, int32_t W, lpf_paths* paths, const float* target_dev,
                  int64_t* counts_dev, const lpf_sa_params* prm, lpf_stream_t stream, lpf_sa** out) {
  return lpf::sa_create_lineal(cell_dev, H, W, paths, target_dev, counts_dev, nullptr, prm, stream, out);
}

int lpf_sa_create_mc(uint8_t* cell_dev, int32_t H, int32_t W, lpf_paths* paths, const uint8_t* sel_dev,
                     const float* target_dev, int64_t* counts_dev, const lpf_sa_params* prm, lpf_stream_t stream,
                     lpf_sa** out) {
  if (!sel_dev) return LPF_EINVAL;
  return lpf::sa_create_lineal(cell_dev, H, W, paths, target_dev, counts_dev, sel_dev, prm, stream, out);
}

int lpf_sa_run(lpf_sa* sa, int32_t n_batches, lpf_stream_t stream) {
  if (!sa || n_batches < 0) return LPF_EINVAL;
  if (n_batches == 0) return LPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  (void)cudaGetLastError();
  if (int rc = lpf::sa_bind_tables(sa)) return rc;
  if (sa->persistent) {
    // a proposer is re-scored every `refresh` batches, between launches
    for (int left = n_batches; left > 0;) {
      const int nb = std::min(left, sa->cnn ? sa->refresh : lpf::kPersistentBatches);
      lpf::enqueue_refresh(sa, s);
      const int rc = lpf::launch_persistent(sa, nb, s);
      if (rc) return rc;
      left -= nb;
    }
    return lpf::set_cuda_error(cudaGetLastError());
  }
  // One captured graph holds kGraphBatches batches; replay it, then enqueue
  // the remainder directly.
  const int kGraphBatches = sa->cnn ? sa->refresh : 16;
  cudaError_t e = cudaSuccess;
  if (!sa->exec && n_batches >= kGraphBatches) {
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      lpf::enqueue_refresh(sa, cs);
      for (int i = 0; i < kGraphBatches; ++i) lpf::enqueue_batch(sa, cs);
      e = cudaStreamEndCapture(cs, &sa->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sa->exec, sa->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { sa->exec = nullptr; return lpf::set_cuda_error(e); }
    sa->graph_batches = kGraphBatches;
  }
  int left = n_batches;
  while (sa->exec && left >= sa->graph_batches) {
    e = cudaGraphLaunch(sa->exec, s);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
    left -= sa->graph_batches;
  }
  if (left > 0) lpf::enqueue_refresh(sa, s);
  for (; left > 0; --left) lpf::enqueue_batch(sa, s);
  return lpf::set_cuda_error(cudaGetLastError());
}

int lpf_sa_selftest_timeout(lpf_sa* sa, int32_t block, lpf_stream_t stream) {
  if (!sa) return LPF_EINVAL;
  if (!sa->persistent) return LPF_EUNSUPPORTED;
  if (block < -1 || block >= sa->g.n_chunks) return LPF_EINVAL;
  if (int rc = lpf::sa_bind_tables(sa)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::SaDev before, after;
  int rc = lpf::sa_device_state(sa, before, s);
  if (rc) return rc;
  int status = 0;
  cudaError_t e = cudaMemcpy(&status, sa->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  if (status) return LPF_ETIMEOUT;  // an earlier wait already failed
  rc = lpf::launch_persistent(sa, 1, s, 1u, block);  // one arrival short of the chosen targets
  if (rc) return rc;
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&status, sa->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  rc = lpf::sa_device_state(sa, after, s);
  if (rc) return rc;
  // Every block timed out, or block 0 did: block 0 kept the state of before
  // the batch.  Another block timed out: block 0 took the batch's decision.
  const bool unchanged = after.n_eval == before.n_eval && after.n_accept == before.n_accept &&
                         after.n_batches == before.n_batches && after.T == before.T && after.e == before.e;
  const bool advanced = after.n_batches == before.n_batches + 1;
  rc = lpf::sa_recover(sa, s);  // recount from the cell, clear the status
  if (rc) return rc;
  const bool state_ok = (block <= 0) ? unchanged : advanced;
  return ((status & 4) && state_ok) ? LPF_OK : LPF_ECUDA;
}

int lpf_sa_set_proposer(lpf_sa* sa, lpf_cnn* cnn, float epsilon, float tau, int32_t refresh) {
  if (!sa || !(epsilon >= 0.0f && epsilon <= 1.0f) || !(tau > 0.0f) || refresh < 1) return LPF_EINVAL;
  if (cnn && !lpf::cnn_matches(cnn, sa->H, sa->W)) return LPF_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  if (cnn && !sa->d_cdf) {
    e = cudaMalloc(&sa->d_cdf, 2 * sizeof(float) * (size_t)sa->H * sa->W);
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
  }
  lpf::SaDev st;
  int rc = lpf::sa_device_state(sa, st, 0);
  if (rc) return rc;
  st.use_model = cnn ? 1 : 0;
  st.eps = epsilon;
  st.cdf1 = sa->d_cdf;
  st.cdf0 = sa->d_cdf ? sa->d_cdf + (size_t)sa->H * sa->W : nullptr;
  st.tot1 = st.tot0 = 0.0f;
  e = cudaMemcpy(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return lpf::set_cuda_error(e);
  sa->cnn = cnn;
  sa->tau = tau;
  sa->refresh = refresh;
  if (sa->exec) { cudaGraphExecDestroy(sa->exec); sa->exec = nullptr; }
  if (sa->graph) { cudaGraphDestroy(sa->graph); sa->graph = nullptr; }
  if (cnn) {
    lpf::enqueue_refresh(sa, 0);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return lpf::set_cuda_error(e);
  }
  return lpf::set_cuda_error(cudaGetLastError());
}

int lpf_sa_read(lpf_sa* sa, lpf_sa_stats* out, lpf_stream_t stream) {
  if (!sa || !out) return LPF_EINVAL;
  lpf::SaDev st;
  int rc = lpf::sa_device_state(sa, st, (cudaStream_t)stream);
  if (rc) return rc;
  int status = 0;
  if (cudaMemcpy(&status, sa->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LPF_ECUDA;
  out->n_eval = st.n_eval;
  out->n_accept = st.n_accept;
  out->n_batches = st.n_batches;
  out->n_candidates = st.n_cand;
  out->temperature = st.T;
  out->error = st.e;
  out->t_max = sa->prm.t_max;
  out->next_batch = st.k_eff;
  out->done = st.done;
  if (!status) return LPF_OK;
  // a bounded wait gave up: restore consistent counts and error, then report it once
  rc = lpf::sa_recover(sa, (cudaStream_t)stream);
  if (rc) return rc;
  rc = lpf::sa_device_state(sa, st, (cudaStream_t)stream);
  if (rc) return rc;
  out->error = st.e;
  return LPF_ETIMEOUT;
}

int lpf_sa_export_progress(lpf_sa* sa, lpf_sa_progress* out, lpf_stream_t stream) {
  if (!sa || !out) return LPF_EINVAL;
  lpf::SaDev st;
  const int rc = lpf::sa_device_state(sa, st, (cudaStream_t)stream);
  if (rc) return rc;
  out->n_eval = st.n_eval;
  out->n_accept = st.n_accept;
  out->n_batches = st.n_batches;
  out->n_candidates = st.n_cand;
  out->c_stage = st.c_stage;
  out->s_stage = st.s_stage;
  out->temperature = st.T;
  out->error = st.e;
  out->p_est = st.p_est;
  out->t_max = sa->prm.t_max;
  out->next_batch = st.k_eff;
  out->done = st.done;
  out->seed = sa->prm.seed;
  out->n_step = st.n_step;
  out->c_max = st.c_max;
  out->s_max = st.s_max;
  out->t_min_ratio = sa->prm.t_min_ratio;
  return LPF_OK;
}

int lpf_sa_import_progress(lpf_sa* sa, const lpf_sa_progress* in, lpf_stream_t stream) {
  if (!sa || !in) return LPF_EINVAL;
  if (in->seed != sa->prm.seed || in->n_step != sa->prm.n_step || in->c_max != sa->prm.c_max ||
      in->s_max != sa->prm.s_max || in->t_min_ratio != sa->prm.t_min_ratio || in->next_batch < sa->prm.k_min ||
      in->next_batch > sa->prm.k_max)
    return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::SaDev st;
  int rc = lpf::sa_device_state(sa, st, s);
  if (rc) return rc;
  st.n_eval = in->n_eval;
  st.n_accept = in->n_accept;
  st.n_batches = in->n_batches;
  st.n_cand = in->n_candidates;
  st.c_stage = in->c_stage;
  st.s_stage = in->s_stage;
  st.T = in->temperature;
  st.e = in->error;
  st.p_est = in->p_est;
  st.k_eff = in->next_batch;
  st.done = in->done;
  cudaError_t e = cudaMemcpyAsync(sa->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return lpf::set_cuda_error(e);
}

int lpf_sa_recompute_error(lpf_sa* sa, double* e_out, lpf_stream_t stream) {
  if (!sa) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::sa_enqueue_error(sa, s);
  lpf::sa_set_error_kernel<<<1, 1, 0, s>>>(sa->d_st, sa->d_e);
  double e = 0.0;
  cudaError_t err = cudaMemcpyAsync(&e, sa->d_e, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return lpf::set_cuda_error(err);
  if (e_out) *e_out = e;
  return LPF_OK;
}

int lpf_sa_propose(lpf_sa* sa, int32_t k, int32_t* pairs_dev, float* u_dev, lpf_stream_t stream) {
  if (!sa || k < 1 || !pairs_dev || !u_dev) return LPF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  lpf::SaDev st;
  int rc = lpf::sa_device_state(sa, st, s);
  if (rc) return rc;
  lpf::sa_draw_kernel<<<(k + 127) / 128, 128, 0, s>>>(sa->d_ext, sa->g, (unsigned long long)st.n_eval, k, st.key0,
                                                      st.key1, pairs_dev, u_dev, sa->d_st);
  cudaError_t e = cudaStreamSynchronize(s);
  return lpf::set_cuda_error(e == cudaSuccess ? cudaGetLastError() : e);
}

void lpf_sa_free(lpf_sa* sa) {
  if (!sa) return;
  cudaDeviceSynchronize();
  if (sa->exec) cudaGraphExecDestroy(sa->exec);
  if (sa->graph) cudaGraphDestroy(sa->graph);
  cudaFree(sa->d_st);
  cudaFree(sa->d_ext);
  cudaFree(sa->d_pairs);
  cudaFree(sa->d_u);
  cudaFree(sa->d_de);
  cudaFree(sa->d_partial);
  cudaFree(sa->d_dc);
  cudaFree(sa->d_e);
  cudaFree(sa->d_status);
  cudaFree(sa->d_sel);
  cudaFree(sa->d_z);
  cudaFree(sa->d_cdf);
  cudaFree(sa->d_bar);
  cudaFree(sa->d_sel_ext);
  delete sa;
}

}  // extern "C"
