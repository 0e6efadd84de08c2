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
  int up = 0;      // halo rows above the translation rows (packed row y = image row y - up)
  int rows = 0;    // packed rows = 32*BB*nbg + ry + up
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
// The layout of one side for a fixed shape (T words per thread, BB bands per
// block, clamped to the bands there are).
int layout_side(int H, int W, int rx, int ry, int T, int BB, Geometry& g, int up = 0);

// The sides of an image evaluation: side 0 walks the image's program (the
// x-major vectors; column offsets up to rx, row offsets 0 .. min(rx, ry)),
// side 1 the transpose's program on the transposed image (the y-major
// vectors; H and W swapped, column offsets up to ry, row offsets -h .. h,
// h = min(rx, ry - 1), so its packed rows have h halo rows above too).  Both use the same words per thread.  Their packed rows
// share one work area, side 1 from word off1 (a 16-byte boundary); their
// band groups are numbered side 0 first.
struct Sides {
  Geometry g[2];
  int n = 1;                 // 1: no y-major vectors (ry = 0) or a volume
  size_t off1 = 0;           // words
  size_t packed_words = 0;   // both sides
  uint32_t band_bytes = 0;   // the larger side's
  int nbg = 0;               // band groups of both sides
  int threads = 0;           // walk block: one warp per tile of the larger side, at most 16
};
int make_sides(const Paths& paths, int H, int W, int T, int BB, Sides& s);
// The same for a D x H x W volume and window (rx, ry, rz).
int make_geometry3(int D, int H, int W, int rx, int ry, int rz, int T, int BB, Geometry& g);

// Walk-kernel launch shape chosen for one image size (by lpf_autotune_full).
struct Tuned {
  int H = 0, W = 0, T = 0, BB = 0;
};

// The programs of an evaluation with their pixel words converted to packed
// offsets for one row layout per side: side 0's groups, then side 1's.
struct Baked {
  int W = -1, S = -1, r32 = -1, slice_rows = 0;
  int H = -1, S1 = -1, r32_1 = -1;  // side 1 (-1: none)
  int T = 0, BB = 0;  // a launch shape whose row layout the program was baked for
  uint32_t* d_words = nullptr;   // 16-byte groups (4 words each)
  uint32_t* d_piece = nullptr;   // piece starts, in groups [n_pieces + 1]
  int n_pieces = 0;              // both sides
  int n_pieces0 = 0;             // side 0's (pieces n_pieces0.. belong to side 1)
};

// Tables of the swap-delta kernel for one extended cell width.
struct DeltaTables {
  int We = -1;
  int want = -1;               // vector chunks asked for (one wave of blocks)
  int want_key = -1;           // the first request of delta_prepare that produced these tables
  int max_chunk_vecs = 0;      // vectors in the largest chunk
  int max_chunk_entries = 0;   // segment pixels of the largest chunk (by pixels)
  int32_t* d_doff = nullptr;   // per segment pixel: sy*We + sx
  int32_t* d_dptr = nullptr;   // CSR pointers [n_canon + 1]
  int32_t* d_chunk = nullptr;  // vector chunk bounds [n_chunks + 1]
  int n_chunks = 0;
  int16_t* d_off16 = nullptr;  // per segment pixel: (sx, sy)
  int16_t* d_vec16 = nullptr;  // per canonical vector: (dx, dy)
  int32_t* d_shear = nullptr;  // per canonical vector: the shear of its phase-0 counts' layout
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
  uint8_t* d_z = nullptr;        // work area: phase-0 counts per (vector, translation) of swap deltas
  size_t z_cap = 0;              // bytes
  int checked = 0;               // 1: kernels that read the image flag pixels other than 0 or 1
  int selftest = 0;              // 1: walks wait for bytes no copy delivers (failure-detection test)
};

namespace lpf {
// Record a CUDA error for lpf_last_error_message(); returns the status code.
int set_cuda_error(cudaError_t e);
// Upload/convert prog0 for side geometry g0 and, when prog1 is not null,
// prog1 for g1 (no-op if already baked for these row layouts).
int bake(lpf_paths* p, const Program& prog0, const Geometry& g0, const Program* prog1, const Geometry* g1,
         Baked& b);
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
// Dynamic shared memory of the persistent annealer for an extended cell of
// ext_bytes and chunks of at most mv vectors and me segment pixels: the
// cell, the chunk's counts (int64) and targets (float) of both phases, then
// its tables for the block-wide lookups (entry offsets, vectors as int16
// pairs, count changes of both phases, error terms, shears, the segment
// pixels as int16 pairs and the vector of every pixel as uint16).
inline size_t persistent_smem_bytes(size_t ext_bytes, int mv, int me) {
  const size_t m = (size_t)mv;
  return ext_bytes + m * 2 * (sizeof(long long) + sizeof(float)) + (m + 1) * 4 + m * (4 + 2 * 4 + 4 + 4) +
         (size_t)me * (4 + 2) + 16;
}
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
