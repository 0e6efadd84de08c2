// Host-side path tables and evaluation programs for the lineal path function.
//
// A "program" is the order in which the kernels visit the discretised
// segments of every canonical vector.  Segments that share their first pixels
// share the work for those pixels (the idea of the "enhanced" evaluation,
// Sec. 3.2, generalised from the longest shorter overlapping segment to every
// common prefix): the segments form a prefix tree whose nodes are pixels; a
// depth-first walk ANDs one shifted image word per node, counts at nodes that
// end a canonical vector, and keeps the masks of branching nodes on a small
// stack.  Children are visited smallest subtree first and the largest last,
// which bounds the stack by log2 of the node count.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace lpf {

// Record header word (int32) of a program, then a vector id (emitting
// records), then a skip word (emitting or pushing records), then a pair
// count, then zero padding up to the next multiple of 4 words, then the pixel
// words.  In a program as built the pair count is 0 and the pixel words are
// prefix-tree node ids.
//
// A program baked for an image layout (bake_words) is a sequence of 16-byte
// groups (uint4); every record is
//   header group   {hdr, vec (emitting records, else 0), skip (in groups,
//                   0: none), cnt = n_pg | n_sg << 13 | half << 26}
//   n_pg pair groups   two pairs {(byte offset << 5) | shift1, shift2} of
//                      pixels that read the same staged word window
//   n_sg single groups four pixels (byte offset << 5) | shift
//   half (0 or 1)      one group holding two single pixels and two zeros
// with hdr as below (n_pix the record's true pixel count).  The ANDs of a
// record commute and are idempotent, so its pixels are sorted by word window
// and an odd single left over is written twice (so that singles come in
// twos and fours).  Piece starts and skip distances count groups.
//   bits  0..13  number of pixel words that follow (n_pix)
//   bit   14     emit: count the mask into vector `vec`
//   bit   15     restore: mask <- stack[rlevel] before the pixels
//   bit   16     push: stack[plevel] <- mask after the pixels (and emit)
// The skip word is the distance in words from the header to the first later
// record of the piece that lies outside the subtree of the record's last node
// (or to the piece end; 0: none).  Masks only shrink down the tree, so when
// the mask is empty for every translation a warp holds, every count in that
// subtree is zero there and the warp may continue at the skip target (the
// zero-count skip of the "enhanced" evaluation, Sec. 3.2, applied to whole
// subtrees).
//   bits 17..23  rlevel
//   bits 24..30  plevel
//   bit   31     reset: mask <- all valid translations before the pixels
constexpr uint32_t kNpixMask = 0x3FFFu;
constexpr uint32_t kEmit = 1u << 14;
constexpr uint32_t kRestore = 1u << 15;
constexpr uint32_t kPush = 1u << 16;
constexpr int kRlevelShift = 17;
constexpr int kPlevelShift = 24;
constexpr uint32_t kLevelMask = 0x7Fu;
constexpr uint32_t kReset = 1u << 31;
constexpr int kMaxStack = 32;

#ifdef __CUDACC__
#define LPF_HOST_DEVICE __host__ __device__
#else
#define LPF_HOST_DEVICE
#endif
// Words between a record's header and its padding (vector id, skip word,
// pair count), and the position of the skip word after the header.
LPF_HOST_DEVICE inline int record_extra_words(uint32_t hdr) {
  return 1 + ((hdr & kEmit) ? 1 : 0) + ((hdr & (kEmit | kPush)) ? 1 : 0);
}
LPF_HOST_DEVICE inline int record_skip_at(uint32_t hdr) { return 1 + ((hdr & kEmit) ? 1 : 0); }
// Pixel words of a baked record with n_pix pixels of which 2 n_pairs are paired.
LPF_HOST_DEVICE inline uint32_t record_pixel_words(uint32_t n_pix, uint32_t n_pairs) {
  return n_pix - n_pairs;
}

struct Program {
  // Words: headers, vec ids and pixel words.  Pixel words hold an index into
  // `pix` (the (sx, sy) offsets) until they are baked for an image width.
  std::vector<uint32_t> words;
  std::vector<int64_t> piece_begin;   // word offsets where pieces start (size n_pieces + 1)
  std::vector<int64_t> piece_pixels;  // pixel words per piece (incl. prologue)
  int stack_depth = 0;                // levels used
  int64_t n_pixel_words = 0;          // total pixel words (work per translation word)
};

struct Paths {
  int32_t rx = 0, ry = 0, rz = 0;
  int dims = 2;                      // 2: images; 3: volumes (vectors (dx, dy, dz))
  int64_t n_full = 0, n_canon = 0, base = 0;
  // Canonical vectors in canonical order (canonical index = full index - base).
  std::vector<int16_t> vec;          // [n_canon][dims] (dx, dy[, dz])
  std::vector<int64_t> ptr;          // [n_canon + 1] CSR into off
  std::vector<int16_t> off;          // [ptr[n_canon]][dims] (sx, sy[, sz]) pixel offsets
  // Prefix trees of the canonical segments.  Images: the x-major vectors
  // (|dx| >= |dy|) form the tree rooted at node 0, in image coordinates; the
  // y-major vectors (|dy| > |dx|) form the tree rooted at node root_t, in the
  // coordinates of the transposed image (x' = y, y' = x, so y' < 0 for
  // dx < 0).  Both trees then hold only segments that step one pixel along x
  // per node, so most nodes share a staged word window with a neighbour in
  // the same row.  Volumes: one tree of all vectors (root_t = -1).
  std::vector<int32_t> node_parent;  // -1 for a root (pixel (0,0))
  std::vector<int16_t> node_pix;     // [n_nodes][2] (x, y) in its tree's coordinates
  std::vector<int16_t> node_pz;      // [n_nodes] z (3D only, else empty)
  std::vector<int32_t> node_vec;     // canonical index ending here, or -1
  int32_t root_t = -1;               // root of the transposed tree, -1 when there is none
  // Programs: tree walk (shared prefixes) and plain (every segment from
  // scratch), for the image (tree, plain) and its transpose (tree_t, plain_t;
  // empty when root_t < 0).
  Program tree, tree_t;
  Program plain, plain_t;
  int64_t n_nodes() const { return (int64_t)node_parent.size(); }
};

// Canonical half: dy > 0, or dy == 0 and dx >= 0.
inline bool is_canonical(int dx, int dy) { return dy > 0 || (dy == 0 && dx >= 0); }

// Pixel offsets of the segment (0,0) -> (dx,dy), for canonical (dx,dy).
void segment_canonical(int dx, int dy, std::vector<int16_t>& out_xy);
// Voxel offsets (x, y, z triples) of the 3D segment (0,0,0) -> (dx,dy,dz),
// for (dx,dy,dz) in the 3D half-domain (dz > 0, or dz = 0 and (dx,dy) in D).
void segment_canonical3(int dx, int dy, int dz, std::vector<int16_t>& out_xyz);

// Build tables and all programs, split into n_pieces pieces in all (shared
// by the image's and the transpose's programs in proportion to their tree
// nodes; n_pieces < 1: one piece per 2 longest-segment lengths of tree
// nodes, at least 64, and at most kMaxPieces pieces per program).  A piece repeats a prologue of at most one
// segment, cut where the tree is shallow (a few % of the work), and more
// pieces let more warps share a small tree, whose walk is latency-bound.
// Returns 0 or a negative status.
constexpr int64_t kMaxPieces = 1024;
int build_paths(int32_t rx, int32_t ry, int n_pieces, Paths& p, std::string& err);
// The same for dims = 2 (rz ignored) or dims = 3 (vectors |dz| <= rz too).
int build_paths_nd(int32_t rx, int32_t ry, int32_t rz, int dims, int n_pieces, Paths& p, std::string& err);

// Split a program into pieces of similar pixel count; fills piece tables.
void split_program(const Paths& p, Program& prog, int n_pieces);
// Pad records so that pixel lists start on 16-byte boundaries.
void align_program(Program& prog);
// Fill the skip words of an aligned, split program.
void resolve_skips(Program& prog);
// Bake a program for staged rows of S words whose bit e is the pixel at
// column e - r32, in the group layout above (pairs formed per record), skip
// distances and piece starts counted in 16-byte groups.  out holds 4 words
// per group.
constexpr uint32_t kCntBits = 13;
constexpr uint32_t kCntMask = (1u << kCntBits) - 1u;
// 3D programs: a voxel at offset (sx, sy, sz) reads staged row
// sz * slice_rows + sy + row_off (slices of slice_rows packed rows).
void bake_words(const Paths& p, const Program& prog, int S, int r32, std::vector<uint32_t>& out,
                std::vector<int64_t>& piece_out, int slice_rows = 0, int row_off = 0);

}  // namespace lpf
