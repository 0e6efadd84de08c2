// The opaque paths handle and the per-image geometry the kernels use.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "../../include/lpf.h"
#include "lpf_paths.hpp"

namespace lpf {

// Geometry of the bit-packed, periodically extended image for one (H, W) and
// one window.  Packed row y (0 <= y < rows) holds pixels of image row y mod H;
// bit e (word e / 32, bit e % 32) of a row is the pixel at column
// (e - r32) mod W, so a translation x plus an offset sx in [-rx, rx] reads bit
// x + sx + r32 >= 0 of the row without wrapping.
struct Geometry {
  int H = 0, W = 0, rx = 0, ry = 0;
  int nw = 0;      // words holding the W translations of a row
  int T = 0;       // words per thread
  int G = 0;       // warps per band (word groups), G*T >= nw
  int BB = 0;      // 32-row bands per block
  int nbg = 0;     // block-band groups = ceil(nbands / BB)
  int r32 = 0;     // rx rounded up to a multiple of 32
  int S = 0;       // words per packed row (odd, so that 32 rows hit 32 banks)
  int nbands = 0;  // 32-row bands of translations
  int rows = 0;    // packed rows = 32*BB*nbg + ry
  uint32_t band_bytes = 0;   // shared memory of one block's rows (multiple of 16)
  size_t packed_words = 0;   // rows*S plus padding for the last band's bulk copy
  // Volumes (3D): D slices, window rz; every slice is slice_rows packed rows
  // (image rows periodically extended by ry above and below), slices
  // periodically extended by rz; nbg_s band groups per slice.  Images: D = 1,
  // slice_rows = 0, nbg_s = nbg.
  int D = 1, rz = 0, slice_rows = 0, nbg_s = 0;
};

// T, BB <= 0 pick defaults.
int make_geometry(int H, int W, int rx, int ry, int T, int BB, Geometry& g);
// The same for a D x H x W volume and window (rx, ry, rz).
int make_geometry3(int D, int H, int W, int rx, int ry, int rz, int T, int BB, Geometry& g);

// Walk-kernel launch shape chosen for one image size (by lpf_autotune_full).
struct Tuned {
  int H = 0, W = 0, T = 0, BB = 0;
};

// A program with its pixel words converted to packed offsets for one width.
struct Baked {
  int W = -1, S = -1, r32 = -1, slice_rows = 0;
  int T = 0, BB = 0;  // a launch shape whose row layout the program was baked for
  uint32_t* d_words = nullptr;   // 16-byte groups (4 words each)
  uint32_t* d_piece = nullptr;   // piece starts, in groups [n_pieces + 1]
  int n_pieces = 0;
};

// Tables of the swap-delta kernel for one extended cell width.
struct DeltaTables {
  int We = -1;
  int want = -1;               // vector chunks asked for (one wave of blocks)
  int max_chunk_vecs = 0;      // vectors in the largest chunk
  int32_t* d_doff = nullptr;   // per segment pixel: sy*We + sx
  int32_t* d_dptr = nullptr;   // CSR pointers [n_canon + 1]
  int32_t* d_chunk = nullptr;  // vector chunk bounds [n_chunks + 1]
  int n_chunks = 0;
  int16_t* d_off16 = nullptr;  // per segment pixel: (sx, sy)
  int16_t* d_vec16 = nullptr;  // per canonical vector: (dx, dy)
};

}  // namespace lpf

struct lpf_paths {
  lpf::Paths host;
  int device = -1;
  lpf::Baked tree, plain;
  uint32_t* d_packed = nullptr;  // work area: packed image (one at a time)
  size_t packed_cap = 0;         // words
  int* d_status = nullptr;       // [0] status flags since the last check, [1] work counter,
                                 // [2..3] pixel words the walk warps ANDed (uint64)
  int64_t nominal_pixels = 0;    // the same without the zero-count skip, for the last walk
  std::vector<lpf::Tuned> tuned; // autotuned walk launch shapes
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;  // optional kernel timer
  lpf::DeltaTables delta;
  float* d_partial = nullptr;    // work area: per (candidate, chunk) error changes
  size_t partial_cap = 0;        // floats
  uint8_t* d_ext = nullptr;      // work area: periodically extended cell (bytes)
  size_t ext_cap = 0;
  uint32_t* d_sel = nullptr;     // work area: packed translation selection (Monte-Carlo variant)
  size_t sel_cap = 0;            // words
  const uint32_t* d_sel_active = nullptr;  // selection of the walk being enqueued (or null)
  uint8_t* d_z = nullptr;        // work area: phase-0 counts per (vector, translation) of swap deltas
  size_t z_cap = 0;              // bytes
  int checked = 0;               // 1: kernels that read the image flag pixels other than 0 or 1
  int selftest = 0;              // 1: walks wait for bytes no copy delivers (failure-detection test)
};

namespace lpf {
// Record a CUDA error for lpf_last_error_message(); returns the status code.
int set_cuda_error(cudaError_t e);
// Upload/convert `prog` for geometry g (no-op if already baked for g.W/S).
int bake(lpf_paths* p, const Program& prog, const Geometry& g, Baked& b);
// Make sure the handle is bound to the current device and has a status word
// and a packed-image area of at least `words`.
int ensure_device(lpf_paths* p, size_t packed_words);
struct DeltaArgs;
// Swap-delta: check sizes, bake tables, size the handle's work areas for K.
int delta_prepare(lpf_paths* p, int H, int W, int K);
// Fill the kernel arguments of the swap-delta kernels for an H x W cell.
int delta_geometry(const lpf_paths* p, int H, int W, DeltaArgs& g);
// Candidate strides per vector chunk for K candidates.
int delta_stride(int n_chunks, int K);
int delta_max_smem();
// Phase-0 counts for swap deltas by lookup: bytes for an H x W cell (0: not
// used -- too long segments or too much memory), allocation in the handle,
// and the kernel that fills them from an extended cell.
size_t delta_z_bytes(const lpf_paths* p, int H, int W);
int delta_z_prepare(lpf_paths* p, int H, int W);
void z_init_launch(const uint8_t* ext, const DeltaArgs& g, uint8_t* z, int* status, cudaStream_t s);
// The annealing batch kernel of the lineal-path objective (lpf_sa.cu), for
// attribute and occupancy queries.
const void* sa_batch_kernel_entry();
const void* sa_persistent_kernel_entry();
// lpf_delta_swap with the error restricted to the phases in phase_mask and,
// optionally, the walks restricted to selected start translations (sel_ext:
// extended layout, from build_sel_ext) with descriptor = count * inv_norm
// (inv_norm <= 0: 1/(H W)).
int delta_swap_run(const uint8_t* img_dev, int32_t H, int32_t W, lpf_paths* paths, const int32_t* pairs_dev,
                   int32_t K, int32_t* dcounts_dev, const float* target_dev, const int64_t* counts_dev, float* de_dev,
                   int phase_mask, cudaStream_t s, const uint8_t* sel_ext, float inv_norm);
int count_selected(const uint8_t* sel_dev, int H, int W, cudaStream_t s, int64_t* n);
int build_sel_ext(const uint8_t* sel_dev, int H, int W, const lpf_paths* paths, cudaStream_t s, uint8_t** out);
// Learned proposer internals used by the annealer.
void cnn_forward(lpf_cnn* c, const uint8_t* cell, cudaStream_t s);
const float* cnn_scores(const lpf_cnn* c);   // [H][W][2] of the last forward
bool cnn_matches(const lpf_cnn* c, int H, int W);
}  // namespace lpf
