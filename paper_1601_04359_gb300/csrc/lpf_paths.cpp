// Host-side construction of the discretised segments and of the evaluation
// programs (see lpf_paths.hpp).
#include "lpf_paths.hpp"

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace lpf {

// Bresenham segment in integer error-term form (Sec. 2.2).  For v in the
// half-domain D, the major axis advances one pixel per step; the minor axis
// advances when the accumulated error reaches a full pixel.  The error starts
// at half a step so the minor coordinate is the one nearest the ideal line,
// and an exact half-way point advances (ties go away from the start pixel).
void segment_canonical(int dx, int dy, std::vector<int16_t>& out) {
  const int ax = std::abs(dx), ay = std::abs(dy);
  const bool xmajor = ax >= ay;
  const int a = xmajor ? ax : ay;  // steps along the major axis
  const int b = xmajor ? ay : ax;
  const int gx = dx < 0 ? -1 : 1, gy = dy < 0 ? -1 : 1;
  out.clear();
  int minor = 0;
  int err = a;  // scaled by 2a: err / (2a) is the fractional minor position + 1/2
  for (int i = 0; i <= a; ++i) {
    if (i > 0) {
      err += 2 * b;
      if (err >= 2 * a) { err -= 2 * a; ++minor; }
    }
    const int px = xmajor ? gx * i : gx * minor;
    const int py = xmajor ? gy * minor : gy * i;
    out.push_back((int16_t)px);
    out.push_back((int16_t)py);
  }
}

// 3D segment, the same rule on every minor axis (one error term per axis):
// the major axis advances one voxel per step, each other axis advances when
// its error reaches a full voxel, ties going away from the start.
void segment_canonical3(int dx, int dy, int dz, std::vector<int16_t>& out) {
  const int ad[3] = {std::abs(dx), std::abs(dy), std::abs(dz)};
  const int g[3] = {dx < 0 ? -1 : 1, dy < 0 ? -1 : 1, dz < 0 ? -1 : 1};
  const int a = std::max(ad[0], std::max(ad[1], ad[2]));
  out.clear();
  int pos[3] = {0, 0, 0};
  int err[3] = {a, a, a};
  for (int i = 0; i <= a; ++i) {
    if (i > 0)
      for (int j = 0; j < 3; ++j) {
        err[j] += 2 * ad[j];
        if (err[j] >= 2 * a) { err[j] -= 2 * a; ++pos[j]; }
      }
    for (int j = 0; j < 3; ++j) out.push_back((int16_t)(g[j] * pos[j]));
  }
}

namespace {

// Child slot of a one-pixel move inside an oriented segment.  2D: the move
// is (mx, my) with my in {0, 1} and mx in {-1, 0, 1}, never (0, 0), or
// (1, -1) (a transposed segment of a vector with dx < 0) (6 slots).  3D:
// (mx, my, mz) with mz in {0, 1}, mx, my in {-1, 0, 1} (18 slots, one of
// them unused).
inline int move_slot(int mx, int my) { return my < 0 ? 5 : (my == 0 ? (mx < 0 ? 0 : 1) : 2 + (mx + 1)); }
inline int move_slot3(int mx, int my, int mz) { return mz * 9 + (my + 1) * 3 + (mx + 1); }

struct Trie {
  int slots = 5;                  // children per node
  std::vector<int32_t> parent;
  std::vector<int16_t> pix;       // [n][3] (x, y, z)
  std::vector<int32_t> vec;
  std::vector<int32_t> child5;    // [n][slots]
  std::vector<int32_t> depth;

  int32_t add(int32_t par, int16_t x, int16_t y, int16_t z, int32_t d) {
    const int32_t id = (int32_t)parent.size();
    parent.push_back(par);
    pix.push_back(x);
    pix.push_back(y);
    pix.push_back(z);
    vec.push_back(-1);
    depth.push_back(d);
    for (int k = 0; k < slots; ++k) child5.push_back(-1);
    return id;
  }
};

struct Event {            // one step of the depth-first walk
  enum Kind : uint8_t { kRestoreEv, kPixEv, kEmitEv, kPushEv } kind;
  int8_t lv;              // pixel events: stack level of the walk invocation
  int32_t a;              // level, node or vector id
};

struct Walker {
  const Trie& t;
  const std::vector<int64_t>& subtree;   // nodes in subtree (work)
  const std::vector<int32_t>& cstart;    // CSR children, ordered light -> heavy
  const std::vector<int32_t>& clist;
  std::vector<Event> ev;
  int max_level = 0;

  void node(int32_t n, int level) {
    // Mask of n's parent is current; AND n's pixel, count, then branch.
    for (;;) {
      ev.push_back({Event::kPixEv, (int8_t)level, n});
      if (t.vec[n] >= 0) ev.push_back({Event::kEmitEv, 0, t.vec[n]});
      const int32_t c0 = cstart[n], c1 = cstart[n + 1];
      const int nc = c1 - c0;
      if (nc == 0) return;
      if (nc == 1) { n = clist[c0]; continue; }
      ev.push_back({Event::kPushEv, 0, level});
      max_level = std::max(max_level, level + 1);
      for (int i = 0; i < nc; ++i) {
        if (i > 0) ev.push_back({Event::kRestoreEv, 0, level});
        if (i < nc - 1) node(clist[c0 + i], level + 1);
      }
      // last (heaviest) child reuses this level: tail position
      n = clist[c1 - 1];
    }
  }
};

}  // namespace

// Turn the event list into records.  At every record start the current node
// and the live stack entries (levels 0..top-1, all ancestors of the next
// node) are kept so that the list can be cut into independent pieces.
static void emit_records(const std::vector<Event>& ev, Program& prog,
                         std::vector<int64_t>& rec_word, std::vector<int64_t>& rec_pix,
                         std::vector<int32_t>& rec_cur, std::vector<std::vector<int32_t>>& rec_stack,
                         std::vector<uint8_t>& rec_restores) {
  std::vector<uint32_t>& w = prog.words;
  w.clear();
  std::vector<int32_t> stack(kMaxStack, -1);
  int top = 0;
  int32_t cur = -1;
  size_t i = 0;
  int64_t pix_total = 0;
  std::vector<uint32_t> pixels;
  while (i < ev.size()) {
    rec_word.push_back((int64_t)w.size());
    rec_pix.push_back(pix_total);
    uint32_t hdr = 0;
    bool restores = false;
    if (ev[i].kind == Event::kRestoreEv) {
      hdr |= kRestore | ((uint32_t)ev[i].a << kRlevelShift);
      cur = stack[ev[i].a];
      top = ev[i].a + 1;
      restores = true;
      ++i;
    }
    rec_cur.push_back(cur);
    rec_restores.push_back(restores ? 1 : 0);
    rec_stack.emplace_back(stack.begin(), stack.begin() + top);
    const size_t hdr_pos = w.size();
    w.push_back(0);  // header placeholder
    uint32_t npix = 0;
    int level = 0;
    pixels.clear();
    while (i < ev.size() && ev[i].kind == Event::kPixEv) {
      pixels.push_back((uint32_t)ev[i].a);  // trie node id until baked
      cur = ev[i].a;
      level = ev[i].lv;
      ++npix;
      ++i;
    }
    if (i < ev.size() && ev[i].kind == Event::kEmitEv) {
      hdr |= kEmit;
      w.push_back((uint32_t)ev[i].a);
      ++i;
    }
    if (i < ev.size() && ev[i].kind == Event::kPushEv) {
      hdr |= kPush | ((uint32_t)ev[i].a << kPlevelShift);
      stack[ev[i].a] = cur;
      top = ev[i].a + 1;
      ++i;
    }
    if (hdr & (kEmit | kPush)) w.push_back((uint32_t)level);  // skip word: the walk level until resolve_skips
    w.push_back(0u);                                            // pair count (formed when baked)
    hdr |= npix;
    w[hdr_pos] = hdr;
    for (uint32_t q : pixels) w.push_back(q);
    pix_total += npix;
  }
  rec_word.push_back((int64_t)w.size());
  rec_pix.push_back(pix_total);
}

// The tree program of one prefix tree from its depth-first event list: cut
// into n_pieces pieces of similar pixel count, each with a prologue that
// rebuilds its starting state from the tree's root (no emits).
static void make_tree_program(const Trie& t, const std::vector<Event>& ev, int max_level, int n_pieces,
                              Program& tree) {
  std::vector<int64_t> rec_word, rec_pix;
  std::vector<int32_t> rec_cur;
  std::vector<std::vector<int32_t>> rec_stack;
  std::vector<uint8_t> rec_restores;
  Program full;
  emit_records(ev, full, rec_word, rec_pix, rec_cur, rec_stack, rec_restores);
  const int64_t nrec = (int64_t)rec_word.size() - 1;
  const int64_t total = rec_pix.back();
  // Each cut sits near its share of the pixels, at the record (within a
  // quarter piece either way) whose starting node is shallowest: the
  // piece's prologue re-walks that node's segment prefix.
  std::vector<int64_t> cuts{0};
  const int64_t slack = std::min<int64_t>(4096, nrec / (4 * (int64_t)n_pieces));
  for (int q = 1; q < n_pieces; ++q) {
    const int64_t target = total * q / n_pieces;
    const int64_t r0 = std::lower_bound(rec_pix.begin(), rec_pix.end() - 1, target) - rec_pix.begin();
    const int64_t lo = std::max<int64_t>(cuts.back() + 1, r0 - slack);
    const int64_t hi = std::min<int64_t>(nrec - 1, r0 + slack);
    int64_t r = r0;
    if (lo <= hi) {
      r = lo;
      for (int64_t c = lo + 1; c <= hi; ++c) {
        const int32_t dc = t.depth[rec_cur[c]], dr = t.depth[rec_cur[r]];
        if (dc < dr || (dc == dr && std::llabs(c - r0) < std::llabs(r - r0))) r = c;
      }
    }
    if (r <= cuts.back()) continue;
    if (r >= nrec) break;
    cuts.push_back(r);
  }
  cuts.push_back(nrec);
  tree.words.clear();
  tree.piece_begin.clear();
  tree.piece_pixels.clear();
  tree.stack_depth = max_level;
  tree.n_pixel_words = 0;
  for (size_t q = 0; q + 1 < cuts.size(); ++q) {
    const int64_t r0 = cuts[q], r1 = cuts[q + 1];
    tree.piece_begin.push_back((int64_t)tree.words.size());
    int64_t pix = 0;
    // prologue: walk root -> deepest node of the state, pushing stack entries
    {
      const std::vector<int32_t>& live = rec_stack[r0];
      // after a restore the state is the restored entry; otherwise the
      // current node (a descendant of every live entry)
      const int32_t target = rec_cur[r0];
      std::vector<int32_t> chain;
      for (int32_t x = target; x >= 0; x = t.parent[x]) chain.push_back(x);
      std::reverse(chain.begin(), chain.end());
      size_t li = 0;
      std::vector<uint32_t> run;
      bool first = true;
      for (size_t ci = 0; ci < chain.size(); ++ci) {
        run.push_back((uint32_t)chain[ci]);
        const bool is_push = li < live.size() && live[li] == chain[ci];
        if (is_push || ci + 1 == chain.size()) {
          uint32_t hdr = (uint32_t)run.size() | (first ? kReset : 0u);
          tree.words.push_back(hdr);
          if (is_push) {  // the node pushed at level li belongs to a walk invocation of level li
            tree.words.back() |= kPush | ((uint32_t)li << kPlevelShift);
            tree.words.push_back((uint32_t)li);  // skip word
            ++li;
          }
          tree.words.push_back(0u);  // pair count
          for (uint32_t n : run) tree.words.push_back(n);
          pix += (int64_t)run.size();
          run.clear();
          first = false;
        }
      }
    }
    // body: copy records r0..r1-1; the first record of piece 0 needs reset
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t wb = rec_word[r], we = rec_word[r + 1];
      uint32_t hdr = full.words[wb];
      if (r == 0) hdr |= kReset;
      tree.words.push_back(hdr);
      for (int64_t j = wb + 1; j < we; ++j) tree.words.push_back(full.words[j]);
      pix += rec_pix[r + 1] - rec_pix[r];
    }
    tree.piece_pixels.push_back(pix);
    tree.n_pixel_words += pix;
  }
  tree.piece_begin.push_back((int64_t)tree.words.size());
}

// The plain program of one tree: the segment of every vector of orientation
// o from scratch, in canonical order; its pixel words are the tree's nodes
// along the segment (found by walking its oriented pixels down from root).
static void make_plain_program(const Trie& t, const std::vector<int32_t>& cstart, const std::vector<int32_t>& clist,
                               const std::vector<int16_t>& oseq, const std::vector<int64_t>& ptr,
                               const std::vector<uint8_t>& orient, uint8_t o, int32_t root, int dims,
                               Program& plain) {
  plain.words.clear();
  plain.stack_depth = 0;
  plain.n_pixel_words = 0;
  std::vector<int32_t> chain;
  const int64_t n_canon = (int64_t)ptr.size() - 1;
  for (int64_t c = 0; c < n_canon; ++c) {
    if (orient[c] != o) continue;
    chain.clear();
    int32_t n = root;
    chain.push_back(n);
    for (int64_t j = ptr[c] + 1; j < ptr[c + 1]; ++j) {
      const int16_t x = oseq[dims * j], y = oseq[dims * j + 1], z = dims == 3 ? oseq[dims * j + 2] : 0;
      int32_t found = -1;
      for (int32_t k = cstart[n]; k < cstart[n + 1]; ++k) {
        const int32_t ch = clist[k];
        if (t.pix[3 * ch] == x && t.pix[3 * ch + 1] == y && t.pix[3 * ch + 2] == z) { found = ch; break; }
      }
      n = found;
      chain.push_back(n);
    }
    plain.words.push_back(kReset | kEmit | (uint32_t)chain.size());
    plain.words.push_back((uint32_t)c);
    plain.words.push_back(0u);  // skip word (resolved to the next record)
    plain.words.push_back(0u);  // pair count
    for (int32_t x : chain) plain.words.push_back((uint32_t)x);
    plain.n_pixel_words += (int64_t)chain.size();
  }
}

int build_paths(int32_t rx, int32_t ry, int n_pieces, Paths& p, std::string& err) {
  return build_paths_nd(rx, ry, 0, 2, n_pieces, p, err);
}

int build_paths_nd(int32_t rx, int32_t ry, int32_t rz, int dims, int n_pieces, Paths& p, std::string& err) {
  if (rx < 0 || ry < 0 || rz < 0 || rx > 4095 || ry > 4095 || rz > 4095) {
    err = "window radius out of range [0, 4095]";
    return -1;
  }
  if (dims != 2 && dims != 3) { err = "dims must be 2 or 3"; return -1; }
  if (dims == 2) rz = 0;
  p = Paths();
  p.rx = rx;
  p.ry = ry;
  p.rz = rz;
  p.dims = dims;
  const int64_t nxy = (int64_t)(2 * rx + 1) * (2 * ry + 1);
  p.n_full = nxy * (2 * rz + 1);
  p.base = (p.n_full - 1) / 2;
  p.n_canon = p.n_full - p.base;
  p.vec.resize((size_t)dims * p.n_canon);
  p.ptr.assign(p.n_canon + 1, 0);
  std::vector<int16_t> seg;
  for (int64_t c = 0; c < p.n_canon; ++c) {
    const int64_t k = p.base + c;
    const int dz = (int)(k / nxy) - rz;
    const int64_t rem = k % nxy;
    const int dy = (int)(rem / (2 * rx + 1)) - ry, dx = (int)(rem % (2 * rx + 1)) - rx;
    p.vec[(size_t)dims * c] = (int16_t)dx;
    p.vec[(size_t)dims * c + 1] = (int16_t)dy;
    if (dims == 3) {
      p.vec[(size_t)dims * c + 2] = (int16_t)dz;
      segment_canonical3(dx, dy, dz, seg);
    } else {
      segment_canonical(dx, dy, seg);
    }
    p.ptr[c + 1] = p.ptr[c] + (int64_t)seg.size() / dims;
    p.off.insert(p.off.end(), seg.begin(), seg.end());
  }

  // Oriented segments: an image's y-major vectors go to the transposed tree
  // (see Paths) as the sequence (x', y') = (sy, sx) of their pixels, which
  // starts at (0, 0) and steps one pixel along x'.
  std::vector<uint8_t> orient((size_t)p.n_canon, 0);
  std::vector<int16_t> oseq(p.off);
  bool any_t = false;
  if (dims == 2) {
    for (int64_t c = 0; c < p.n_canon; ++c) {
      const int dx = p.vec[2 * c], dy = p.vec[2 * c + 1];
      if (std::abs(dy) <= std::abs(dx)) continue;
      orient[c] = 1;
      any_t = true;
      for (int64_t j = p.ptr[c]; j < p.ptr[c + 1]; ++j) {
        oseq[2 * j] = p.off[2 * j + 1];
        oseq[2 * j + 1] = p.off[2 * j];
      }
    }
  }

  // Prefix trees; node 0 is pixel (0,0[,0]) of the image's tree, node 1 the
  // root of the transposed tree (when there is one).
  Trie t;
  t.slots = dims == 3 ? 18 : 6;
  const int S5 = t.slots;
  t.add(-1, 0, 0, 0, 0);
  const int32_t root_t = any_t ? t.add(-1, 0, 0, 0, 0) : -1;
  for (int64_t c = 0; c < p.n_canon; ++c) {
    int32_t n = orient[c] ? root_t : 0;
    for (int64_t j = p.ptr[c] + 1; j < p.ptr[c + 1]; ++j) {
      const int16_t x = oseq[dims * j], y = oseq[dims * j + 1], z = dims == 3 ? oseq[dims * j + 2] : 0;
      const int mx = x - t.pix[3 * n], my = y - t.pix[3 * n + 1], mz = z - t.pix[3 * n + 2];
      const int slot = dims == 3 ? move_slot3(mx, my, mz) : move_slot(mx, my);
      int32_t ch = t.child5[(int64_t)S5 * n + slot];
      if (ch < 0) {
        ch = t.add(n, x, y, z, t.depth[n] + 1);
        t.child5[(int64_t)S5 * n + slot] = ch;
      }
      n = ch;
    }
    t.vec[n] = (int32_t)c;
  }
  const int64_t nn = (int64_t)t.parent.size();
  // subtree sizes (children have larger ids than parents)
  std::vector<int64_t> sub(nn, 1);
  for (int64_t n = nn - 1; n > 0; --n)
    if (t.parent[n] >= 0) sub[t.parent[n]] += sub[n];
  std::vector<int32_t> cstart(nn + 1, 0), clist;
  clist.reserve(nn);
  for (int64_t n = 0; n < nn; ++n) {
    int32_t cs[18];
    int m = 0;
    for (int k = 0; k < S5; ++k) if (t.child5[S5 * n + k] >= 0) cs[m++] = t.child5[S5 * n + k];
    std::sort(cs, cs + m, [&](int32_t a, int32_t b) { return sub[a] != sub[b] ? sub[a] < sub[b] : a < b; });
    for (int k = 0; k < m; ++k) clist.push_back(cs[k]);
    cstart[n + 1] = (int32_t)clist.size();
  }
  std::vector<int32_t>().swap(t.child5);

  // Pieces per program: automatic (one per 2 segment lengths of tree nodes,
  // at least 64, at most kMaxPieces) or n_pieces shared in proportion to the
  // trees' nodes.
  auto pieces_for = [&](int64_t nodes) -> int {
    if (n_pieces < 1) {
      const int64_t piece_nodes = std::max<int64_t>(64, 2 * ((int64_t)std::max(rx, ry) + 1));
      return (int)std::max<int64_t>(1, std::min<int64_t>(kMaxPieces, nodes / piece_nodes));
    }
    return (int)std::max<int64_t>(1, std::llround((double)n_pieces * (double)nodes / (double)nn));
  };
  const int n_trees = root_t >= 0 ? 2 : 1;
  for (int o = 0; o < n_trees; ++o) {
    const int32_t root = o ? root_t : 0;
    // Depth-first walk -> events -> records -> pieces.
    Walker wk{t, sub, cstart, clist, {}, 0};
    wk.ev.reserve(sub[root] + 3 * p.n_canon / n_trees);
    wk.node(root, 0);
    if (wk.max_level > kMaxStack) { err = "prefix-tree stack deeper than supported"; return -2; }
    make_tree_program(t, wk.ev, wk.max_level, pieces_for(sub[root]), o ? p.tree_t : p.tree);
    // Plain program: every segment of the tree from scratch (Alg. 1 order).
    make_plain_program(t, cstart, clist, oseq, p.ptr, orient, (uint8_t)o, root, dims, o ? p.plain_t : p.plain);
    split_program(p, o ? p.plain_t : p.plain, pieces_for(sub[root]));
  }
  for (Program* prog : {&p.tree, &p.tree_t, &p.plain, &p.plain_t}) {
    if (prog->piece_begin.empty()) prog->piece_begin.push_back(0);  // no tree: no pieces
    align_program(*prog);
    resolve_skips(*prog);
  }
  p.root_t = root_t;

  p.node_parent = std::move(t.parent);
  p.node_pix.resize(2 * (size_t)nn);
  if (dims == 3) p.node_pz.resize((size_t)nn);
  for (int64_t n = 0; n < nn; ++n) {
    p.node_pix[2 * n] = t.pix[3 * n];
    p.node_pix[2 * n + 1] = t.pix[3 * n + 1];
    if (dims == 3) p.node_pz[n] = t.pix[3 * n + 2];
  }
  p.node_vec = std::move(t.vec);
  return 0;
}

// Re-lay a program so that every record's pixel list starts on a 16-byte
// boundary (words after the header/vec id are padded with zeros up to the
// next multiple of 4), which lets the kernels fetch pixel words four at a
// time.  Piece offsets are remapped.
void align_program(Program& prog) {
  std::vector<uint32_t> out;
  out.reserve(prog.words.size() + prog.words.size() / 4);
  std::vector<int64_t> remap_from, remap_to;
  size_t pi = 0;
  std::vector<int64_t> new_begin(prog.piece_begin.size(), 0);
  for (size_t i = 0; i < prog.words.size();) {
    while (pi < prog.piece_begin.size() && prog.piece_begin[pi] == (int64_t)i) new_begin[pi++] = (int64_t)out.size();
    const uint32_t h = prog.words[i++];
    out.push_back(h);
    for (int k = record_extra_words(h); k > 0; --k) out.push_back(prog.words[i++]);
    while (out.size() % 4) out.push_back(0);
    const uint32_t n = h & kNpixMask;
    for (uint32_t k = 0; k < n; ++k) out.push_back(prog.words[i++]);
  }
  while (pi < prog.piece_begin.size()) new_begin[pi++] = (int64_t)out.size();
  prog.words.swap(out);
  prog.piece_begin.swap(new_begin);
}

// Replace the walk level held in each skip word by the distance to its skip
// target.  The records of the subtree below the last node
// of a record are those that follow it up to the first record that restores a
// stack level below the level of the walk invocation holding that node (the
// invocation's own branches restore its level or deeper ones, and once it
// returns its parent restores one level up) or that resets the mask.
void resolve_skips(Program& prog) {
  std::vector<int64_t> starts;
  for (size_t q = 0; q + 1 < prog.piece_begin.size(); ++q) {
    const int64_t b = prog.piece_begin[q], e = prog.piece_begin[q + 1];
    starts.clear();
    for (int64_t w = b; w < e;) {
      starts.push_back(w);
      const uint32_t h = prog.words[w];
      const int64_t k = (w + 1 + record_extra_words(h) + 3) & ~int64_t(3);
      w = k + (h & kNpixMask);
    }
    // nr[L]: start of the nearest later record that resets or restores a level < L
    int64_t nr[kMaxStack + 2];
    for (int64_t& x : nr) x = e;
    for (size_t r = starts.size(); r-- > 0;) {
      const int64_t w = starts[r];
      const uint32_t h = prog.words[w];
      if (h & (kEmit | kPush)) {
        const int64_t at = w + record_skip_at(h);
        const uint32_t lv = std::min<uint32_t>(prog.words[at], kMaxStack + 1);
        const int64_t d = nr[lv] - w;
        prog.words[at] = d < (int64_t(1) << 32) ? (uint32_t)d : 0u;  // 0: never skip
      }
      if (h & kReset) {
        for (int64_t& x : nr) x = w;
      } else if (h & kRestore) {
        const int l = (int)((h >> kRlevelShift) & kLevelMask);
        for (int L = l + 1; L <= kMaxStack + 1; ++L) nr[L] = w;
      }
    }
  }
}

void bake_words(const Paths& p, const Program& prog, int S, int r32, std::vector<uint32_t>& out,
                std::vector<int64_t>& piece_out, int slice_rows, int row_off) {
  const std::vector<uint32_t>& w = prog.words;
  out.clear();
  out.reserve(w.size() + w.size() / 8);
  std::vector<int64_t> old_start, new_start;  // record starts (old: words, new: groups)
  std::vector<std::pair<uint32_t, uint32_t>> pix;  // (byte offset, shift)
  std::vector<uint32_t> singles;
  for (size_t i = 0; i < w.size();) {
    old_start.push_back((int64_t)i);
    new_start.push_back((int64_t)(out.size() / 4));
    const uint32_t h = w[i];
    const int extra = record_extra_words(h);
    const uint32_t vec = (h & kEmit) ? w[i + 1] : 0u;
    const uint32_t skip = (h & (kEmit | kPush)) ? w[i + (size_t)record_skip_at(h)] : 0u;  // resolved below
    i += 1 + extra;
    while (i % 4) ++i;
    const uint32_t n = h & kNpixMask;
    pix.clear();
    for (uint32_t k = 0; k < n; ++k) {
      const int node = (int)w[i + k];
      const int sxp = p.node_pix[2 * node] + r32;  // >= 0
      const int sz = p.node_pz.empty() ? 0 : p.node_pz[node];
      const int row = sz * slice_rows + p.node_pix[2 * node + 1] + row_off;  // >= 0
      pix.push_back({(uint32_t)(row * S + (sxp >> 5)) * 4u, (uint32_t)(sxp & 31)});
    }
    i += n;
    std::stable_sort(pix.begin(), pix.end(),
                     [](const std::pair<uint32_t, uint32_t>& a, const std::pair<uint32_t, uint32_t>& b) {
                       return a.first < b.first;
                     });
    // pairs of pixels in one word window, two pairs per group; a pair left
    // over and the unpaired pixels are singles
    std::vector<uint32_t> pairs;
    singles.clear();
    for (size_t k = 0; k < pix.size();) {
      if (k + 1 < pix.size() && pix[k].first == pix[k + 1].first) {
        pairs.push_back((pix[k].first << 5) | pix[k].second);
        pairs.push_back(pix[k + 1].second);
        k += 2;
      } else {
        singles.push_back((pix[k].first << 5) | pix[k].second);
        k += 1;
      }
    }
    if ((pairs.size() / 2) & 1) {  // odd number of pairs: the last one becomes two singles
      const uint32_t s2 = pairs.back();
      pairs.pop_back();
      const uint32_t s1 = pairs.back();
      pairs.pop_back();
      singles.push_back(s1);
      singles.push_back((s1 & ~31u) | s2);
    }
    if (singles.size() & 1) singles.push_back(singles.back());  // ANDing a pixel twice changes nothing
    const uint32_t n_pg = (uint32_t)(pairs.size() / 4);
    const uint32_t n_sg = (uint32_t)(singles.size() / 4);
    const uint32_t half = (uint32_t)(singles.size() % 4 != 0);
    out.push_back(h);
    out.push_back(vec);
    out.push_back(skip);
    out.push_back(n_pg | (n_sg << kCntBits) | (half << (2 * kCntBits)));
    out.insert(out.end(), pairs.begin(), pairs.end());
    out.insert(out.end(), singles.begin(), singles.end());
    while (out.size() % 4) out.push_back(0u);
  }
  auto relocate = [&](int64_t old_pos) -> int64_t {  // a record start or the program end, in groups
    if (old_pos >= (int64_t)w.size()) return (int64_t)(out.size() / 4);
    const auto it = std::lower_bound(old_start.begin(), old_start.end(), old_pos);
    return new_start[it - old_start.begin()];
  };
  for (size_t r = 0; r < old_start.size(); ++r) {
    const uint32_t h = w[(size_t)old_start[r]];
    uint32_t& sk = out[4 * (size_t)new_start[r] + 2];
    if (!(h & (kEmit | kPush)) || sk == 0) { sk = 0; continue; }
    const int64_t nd = relocate(old_start[r] + sk) - new_start[r];
    sk = nd < (int64_t(1) << 32) ? (uint32_t)nd : 0u;
  }
  piece_out.resize(prog.piece_begin.size());
  for (size_t q = 0; q < prog.piece_begin.size(); ++q) piece_out[q] = relocate(prog.piece_begin[q]);
}

void split_program(const Paths&, Program& prog, int n_pieces) {
  // Plain programs have only independent records (each starts with reset),
  // so cutting at any record boundary needs no prologue.
  std::vector<int64_t> starts, pixc;
  int64_t pix = 0;
  for (int64_t w = 0; w < (int64_t)prog.words.size();) {
    const uint32_t h = prog.words[w];
    starts.push_back(w);
    pixc.push_back(pix);
    const int64_t np = h & kNpixMask;
    pix += np;
    w += 1 + record_extra_words(h) + np;
  }
  starts.push_back((int64_t)prog.words.size());
  pixc.push_back(pix);
  prog.piece_begin.clear();
  prog.piece_pixels.clear();
  if (n_pieces < 1) n_pieces = 1;
  std::vector<int64_t> cut_rec{0};
  const int64_t nrec = (int64_t)starts.size() - 1;
  for (int q = 1; q < n_pieces; ++q) {
    int64_t r = std::lower_bound(pixc.begin(), pixc.end() - 1, pix * q / n_pieces) - pixc.begin();
    if (r <= cut_rec.back() || r >= nrec) continue;
    cut_rec.push_back(r);
  }
  cut_rec.push_back(nrec);
  for (size_t q = 0; q + 1 < cut_rec.size(); ++q) {
    prog.piece_begin.push_back(starts[cut_rec[q]]);
    prog.piece_pixels.push_back(pixc[cut_rec[q + 1]] - pixc[cut_rec[q]]);
  }
  prog.piece_begin.push_back(starts[nrec]);
}

}  // namespace lpf
