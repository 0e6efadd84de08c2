/*
 * liblpf -- exact lineal path function of periodic two-phase 2D images on
 * NVIDIA GB300 (sm_103a), after Havelka, Kucerova & Sykora, "Compression and
 * Reconstruction of Random Microstructures using Accelerated Lineal Path
 * Function" (arXiv:1601.04359).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Image     uint8, H rows x W columns, row-major: pixel (x, y) is img[y*W + x]
 *            (x = column, y = row).  Values are 0 or 1; "phase p" is the
 *            set of pixels with value p.  The medium is periodic: coordinates
 *            wrap modulo W and H (the "%" convention of Eq. (S2dis), Sec. 2.1).
 *            Other byte values: by default (unchecked) every nonzero byte is
 *            read as phase 1; in checked mode (lpf_set_checked) a kernel that
 *            reads the image also raises a status flag that lpf_paths_status
 *            reports as LPF_EPIXEL, and the results of that call are not to
 *            be used.
 *  Vectors   v = (dx, dy), dx a column offset, dy a row offset, in the window
 *            |dx| <= rx, |dy| <= ry with 0 <= rx < W and 0 <= ry < H.  The
 *            paper's full domain is rx = W-1, ry = H-1 (Eq. (segments), Sec. 2.2).
 *  Segment   S(v): the Bresenham pixels from (0,0) to v (Sec. 2.2).  For v in
 *            the half-domain D (dy > 0, or dy == 0 and dx >= 0) step i = 0..a,
 *            a = max(|dx|,|dy|), moves i along the major axis and round(i*b/a)
 *            along the minor one (b = min(|dx|,|dy|)), an exact half rounding
 *            away from the start; outside D, S(v) = v + S(-v) (the same pixels
 *            seen from the other end), so L(v) = L(-v) exactly (Eq. (symmetry)).
 *  Count     count_p(v) = #{x : img[(x + s) mod (W,H)] == p for all s in S(v)};
 *            the lineal path function is L_p(v) = count_p(v) / (W*H)
 *            (Sec. 2.2 definition; Alg. 1 of Sec. 3.1).
 *  Layouts   full:      [2][(2ry+1)(2rx+1)], entry (dy+ry)*(2rx+1) + (dx+rx),
 *                       phase 0 first.
 *            canonical: [n_canon] with n_canon = ry*(2rx+1) + rx + 1; the
 *                       canonical entries are the tail of the full layout that
 *                       starts at v = (0,0): canonical index = full index - base,
 *                       base = (n_full - 1) / 2.
 *  Memory    "_dev" pointers are device memory owned by the caller; "_host"
 *            pointers are host memory owned by the caller.  Device calls are
 *            asynchronous on the given stream (a cudaStream_t; NULL = legacy
 *            default stream) and return once the work is enqueued.
 *  Errors    every int-returning call returns LPF_OK (0) or a negative code;
 *            arguments are validated on the host before anything is enqueued,
 *            and on error nothing is enqueued.  lpf_strerror() names a code.
 *  Threads   a paths handle is not thread-safe: calls that use one handle must
 *            be issued from one host thread and ordered on one stream (the
 *            handle keeps device tables and a work area that calls reuse).
 */
#ifndef LPF_H
#define LPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LPF_OK 0
#define LPF_EINVAL (-1)      /* bad argument: size, window, pointer, count */
#define LPF_ENOMEM (-2)      /* host or device allocation failed */
#define LPF_ECUDA (-3)       /* a CUDA runtime call failed (no device, launch error) */
#define LPF_ETIMEOUT (-4)    /* a device-side bounded wait gave up (see lpf_paths_status) */
#define LPF_EUNSUPPORTED (-5) /* size beyond what the kernels support (shared memory, width) */
#define LPF_EPIXEL (-6)      /* a pixel other than 0 or 1 was read in checked mode (see lpf_set_checked) */

typedef struct CUstream_st *lpf_stream_t; /* same type as cudaStream_t */
typedef struct lpf_paths lpf_paths;        /* opaque, owned by the library */

/* Name of a status code (static string). */
const char *lpf_strerror(int code);

/* Text of the last CUDA runtime error seen by this thread inside the library
 * (empty if none); stays valid until the thread's next library call. */
const char *lpf_last_error_message(void);

/*
 * Build the discretised segments of every vector of the window |dx| <= rx,
 * |dy| <= ry (Sec. 2.2 segments; Sec. 3.1 step 1, done once) and the
 * evaluation program that shares the work of common segment prefixes (the
 * enhanced evaluation of Sec. 3.2, generalised to all shared prefixes).  The
 * program has two prefix trees: the segments of the x-major vectors
 * (|dx| >= |dy|), walked over the image, and those of the y-major vectors,
 * transposed, walked over the transposed image, so that every segment
 * advances one pixel along a packed row per step (the count of a vector is
 * the same over the transposed image for the transposed segment).
 * Host-only; touches no GPU.  rx, ry in [0, 4095].  *out receives a handle
 * to release with lpf_paths_free().  Device tables are uploaded lazily by the
 * first device call that uses the handle (see lpf_full).
 * Errors: LPF_EINVAL (radius out of range, out == NULL), LPF_ENOMEM.
 */
int lpf_build_paths(int32_t rx, int32_t ry, lpf_paths **out);

/*
 * Sizes of a handle's tables: n_vec_full = (2rx+1)(2ry+1), n_vec_canon =
 * canonical vectors, n_offsets = total pixels of the canonical segments.
 * Any output pointer may be NULL.  Errors: LPF_EINVAL (paths == NULL).
 */
int lpf_paths_info(const lpf_paths *paths, int64_t *n_vec_full, int64_t *n_vec_canon,
                   int64_t *n_offsets);

/*
 * Copy the canonical segments into caller-sized host arrays (CSR form):
 * vec_dxdy_host [n_vec_canon][2] (dx, dy) in canonical order,
 * ptr_host [n_vec_canon + 1] (segment c is offsets ptr[c] .. ptr[c+1]-1),
 * off_dxdy_host [n_offsets][2] (sx, sy) pixel offsets from the start pixel,
 * start pixel first.  For a volume's handle (lpf_build_paths_3d) the vector
 * and offset arrays hold triples (dx, dy, dz) and (sx, sy, sz) instead.  Any
 * output pointer may be NULL.  Errors: LPF_EINVAL (paths == NULL).
 */
int lpf_paths_export(const lpf_paths *paths, int16_t *vec_dxdy_host, int64_t *ptr_host,
                     int16_t *off_dxdy_host);

/*
 * Work statistics: n_tree_nodes = pixels the prefix-sharing program visits
 * per translation word at most (subtrees whose count is zero for all
 * translations a warp holds are skipped: lpf_paths_work reports what a call
 * did), stack_depth = masks it keeps at once, n_pieces =
 * independent program pieces the kernels spread over thread blocks.
 * Any output pointer may be NULL.
 */
int lpf_paths_stats(const lpf_paths *paths, int64_t *n_tree_nodes, int32_t *stack_depth,
                    int32_t *n_pieces);

/*
 * Work of the last lpf_full, lpf_full_standard, lpf_full_mc,
 * lpf_full_ensemble or lpf_full_3d evaluation enqueued with this handle (for
 * an ensemble: its last cut; not the allocation-free variant), counted in
 * pixel (voxel) words
 * ANDed by a warp (one word for each of the warp's 32 translation rows x T
 * words), summed over warps:
 *   executed  what the warps did, after skipping the subtrees of the
 *             prefix tree whose count is zero for all the warp's translations
 *             (the zero-count skip of the "enhanced" evaluation, Sec. 3.2);
 *   nominal   what they would do without that skip.
 * Host pointers, both required.  Synchronises with the device (a blocking
 * copy).  Before any evaluation both are 0.  Errors: LPF_EINVAL, LPF_ECUDA.
 */
int lpf_paths_work(const lpf_paths *paths, int64_t *executed, int64_t *nominal);

/* Release a handle and its device memory (NULL is ignored).  Synchronises
 * the device before freeing device tables. */
void lpf_paths_free(lpf_paths *paths);

/*
 * Checked mode of a handle (default off).  on = 1: every later device call
 * with this handle that reads an image (lpf_full, lpf_full_noalloc,
 * lpf_full_mc, lpf_full_standard, lpf_full_ensemble, lpf_delta_swap,
 * lpf_delta_swap_mc, and the count set-up of lpf_sa_create /
 * lpf_sa_create_mc) also checks that every pixel byte is 0 or 1; a byte
 * outside {0, 1} sets a device status flag that the next lpf_paths_status
 * returns as LPF_EPIXEL (the Sec. 2.2 definition covers two-phase images
 * only, so such a call's results are not to be used).  The check costs one
 * compare per staged byte in kernels that read the image anyway.  on = 0:
 * no check; nonzero bytes are phase 1.  Host-only.  Errors: LPF_EINVAL.
 */
int lpf_set_checked(lpf_paths *paths, int32_t on);

/*
 * Full lineal path counts of both phases for every vector of the handle's
 * window (Sec. 2.2; Alg. 1/Alg. 2 of Sec. 3.1 with the prefix sharing of
 * Sec. 3.2).  img_dev: H*W uint8 (0/1), counts_dev: int64 full layout
 * [2][n_vec_full], overwritten.  Vectors outside D are filled by the point
 * symmetry of Eq. (symmetry).  A warp that finds no translation left (at the
 * end of a prefix, or every 8 pixels inside one) skips the rest of that
 * prefix and the segments that extend it (their counts are zero there too),
 * so the time depends on the image.
 * Requires rx < W, ry < H, 1 <= H, W <= 8192.  The first call with a new
 * image width uploads the handle's program for that width and may allocate
 * the handle's device work area (make that first call before any stream
 * capture); later calls with the same or smaller sizes allocate nothing.
 * Size envelope: a thread block stages a band of 32 translation rows plus ry
 * halo rows, each about (W + 2 rx) / 32 + 2 words, in shared memory (at most
 * about 227 KB), and W <= 4096; e.g. the full domain (rx = W-1, ry = H-1) fits
 * up to about 700 x 700, a window of 256 up to W = 4096.  Outside it:
 * LPF_EUNSUPPORTED.  Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_full(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths,
             int64_t *counts_dev, lpf_stream_t stream);

/*
 * lpf_full for callers that must not allocate device memory when they
 * evaluate.  (The paper has no counterpart: this is a deployment variant.)
 * Such callers include host applications that own every device allocation
 * and give libraries fixed budgets, and real-time or pipelined loops where a
 * cudaMalloc -- which can synchronise the whole device -- is not allowed.
 * Same arguments, layout and results as lpf_full; this call performs no
 * cudaMalloc, cudaFree or other allocation.  Its work area (packed image
 * rows and the walk's control words) is a fixed array of 1 MiB (2^18 words
 * of packed rows) compiled into the library, which every GPU that loads the
 * library holds until the process exits.  Checked mode (lpf_set_checked)
 * applies as for lpf_full.
 *   - Size limit: the packed, periodically extended image must fit in 2^18
 *     words; it takes roughly (H + ry) * (W + 2*rx) / 32 words plus a few
 *     rows and columns of padding (512x512 with |v| <= 256: 25,348 words).
 *     Larger images return LPF_EUNSUPPORTED.
 *   - Set-up: the handle's program for this image size must already be on the
 *     current device -- call lpf_full (or lpf_autotune_full) once for this
 *     H, W during set-up; otherwise LPF_EINVAL.  The walk runs in the launch
 *     shape lpf_full would use (tuned or set), or, where that shape needs
 *     another row layout than the program on the device was prepared for
 *     (e.g. lpf_set_launch_shape after the set-up call), in the shape it was
 *     prepared for.  The first call of this
 *     function on a device looks up the device address of the fixed array
 *     (once per device, with that device current); make that first call
 *     before any stream capture.
 *   - Sharing: every call on a device uses the same fixed array and leaves
 *     its contents behind (each call clears the control words it needs).
 *     Calls whose work overlaps on the GPU -- on different streams, or from
 *     different host threads without ordering -- race on that array and give
 *     wrong counts; order them on one stream.
 *   - Status: a bounded wait that gave up, or a pixel outside {0, 1} in
 *     checked mode, sets a flag in the fixed array's status word; the next
 *     lpf_paths_status on this device, with any handle, reports it
 *     (LPF_ETIMEOUT, LPF_EPIXEL) and clears it.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ECUDA.
 */
int lpf_full_noalloc(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths,
                     int64_t *counts_dev, lpf_stream_t stream);

/*
 * Monte-Carlo approximation of Sec. 3 (opening): the segments are compared
 * with the image only at the selected translations -- sel_dev: H*W uint8,
 * nonzero = translation (x, y) selected (e.g. a random N-combination of the
 * W*H positions).  counts_dev receives, for every vector of D (the canonical
 * half), the number of selected translations whose segment lies in each
 * phase, so that L~ = counts / N; as in the paper, which evaluates D only,
 * the other half is filled by point symmetry.  All translations selected
 * gives lpf_full's counts.  Errors as lpf_full.
 */
int lpf_full_mc(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths, const uint8_t *sel_dev,
                int64_t *counts_dev, lpf_stream_t stream);

/*
 * Autotuner for lpf_full: times every admissible launch shape (words per
 * thread T in {1,2,4,8}, 32-row bands per block BB in {1,2,4,8}) of the walk
 * kernel on this image (3 timed runs each, fastest kept) and stores the
 * fastest in the handle for later lpf_full calls with the same H, W.  Runs
 * and synchronises on `stream`; counts_dev receives valid counts.  best_T /
 * best_BB (may be NULL) receive the choice.  Not for use inside stream
 * capture.  Errors as lpf_full.
 */
int lpf_autotune_full(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths,
                      int64_t *counts_dev, lpf_stream_t stream, int32_t *best_T, int32_t *best_BB);

/*
 * Failure-detection self-test of the walk kernel (no counterpart in the
 * paper).  on = 1: later lpf_full / lpf_full_noalloc calls with this handle
 * make each block's wait for its staging copy expect 16 bytes more than the
 * copy delivers and give up after 2^16 try_wait rounds (instead of 2^24), so
 * every wait runs out (milliseconds to seconds); the kernel then records the
 * timeout and returns, the counts are incomplete, and lpf_paths_status
 * reports LPF_ETIMEOUT.  on = 0 restores normal waits.  Faults nothing; for
 * tests only.  Host-only.  Errors: LPF_EINVAL.
 */
int lpf_paths_set_selftest(lpf_paths *paths, int32_t on);

/*
 * Fix the walk-kernel launch shape used by lpf_full for images of size H x W
 * (T words per thread in {1,2,4,8}, BB bands of 32 rows per block, 1..16),
 * overriding defaults or an autotuned choice.  Host-only.  Errors:
 * LPF_EINVAL (bad value), LPF_EUNSUPPORTED (shape not admissible for this
 * size: more than 16 warps per block, or shared memory too small).
 */
int lpf_set_launch_shape(lpf_paths *paths, int32_t H, int32_t W, int32_t T, int32_t BB);

/*
 * Same as lpf_full but evaluates every segment from scratch, one vector after
 * another (the "standard" evaluation of Sec. 3.2, i.e. Alg. 1 order without
 * any shared work; a warp stops a segment once none of its translations is
 * left, Alg. 1's early break).  Same arguments, layout and errors; for
 * comparison runs.
 */
int lpf_full_standard(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths,
                      int64_t *counts_dev, lpf_stream_t stream);

/*
 * Count changes for a batch of candidate pixel exchanges, and the change of
 * the least-square error they cause -- the modification operator and the
 * objective of the annealer (Sec. 4, swap of two pixels of different phases;
 * Eq. (LSE)).  The paper re-evaluates the whole descriptor per candidate; this
 * call evaluates only the translations whose segment contains a swapped pixel.
 *   img_dev      H*W uint8 (0/1): the current cell (not modified).
 *   pairs_dev    int32 [K][2] linear pixel indices (y*W + x) of the two
 *                pixels of each candidate, in either order.  A pair whose
 *                pixels hold the same value (including a == b) is the
 *                identity: all its changes are 0.  An index outside [0, H*W)
 *                is treated as the identity and raises a device status
 *                flag that lpf_paths_status reports as LPF_EINVAL.
 *   dcounts_dev  int32 [K][2][n_vec_canon] or NULL: count after the exchange
 *                minus count before, phase 0 first, canonical order.
 *   target_dev   float [2][n_vec_full] target descriptor (already divided by
 *                its own image area) and counts_dev int64 [2][n_vec_full] the
 *                current cell's counts (from lpf_full): needed when de_dev is
 *                given.
 *   de_dev       float [K] or NULL: e(after) - e(before) with
 *                e = sum over both phases and the canonical half of
 *                (target - counts/(H*W))^2, computed in float32 from the exact
 *                integer changes; summed in a fixed order (bitwise
 *                reproducible).
 * At least one of dcounts_dev, de_dev must be non-NULL.  Cell limits: the
 * periodically extended cell (W+2rx, padded to an odd number of 4-byte
 * words) x (H+2ry) bytes must fit in shared memory
 * (about 227 KB), else LPF_EUNSUPPORTED.  The first call for a cell width, or
 * with a larger K than before, allocates the handle's tables / work area.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_delta_swap(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths,
                   const int32_t *pairs_dev, int32_t K, int32_t *dcounts_dev,
                   const float *target_dev, const int64_t *counts_dev, float *de_dev,
                   lpf_stream_t stream);

/*
 * Sum of the lpf_full counts of n_img images of equal size H x W stored one
 * after another in imgs_dev (uint8 [n_img][H][W]), e.g. the parallel cuts of
 * a volume: the ensemble average over cuts of Sec. 6.3 is counts / (n_img *
 * H * W).  counts_dev: int64 [2][n_vec_full] as in lpf_full.  The images are
 * evaluated one after another on `stream` (each one pack and walk launch).
 * Errors: as lpf_full; n_img < 1 is LPF_EINVAL.
 */
int lpf_full_ensemble(const uint8_t *imgs_dev, int32_t n_img, int32_t H, int32_t W, lpf_paths *paths,
                      int64_t *counts_dev, lpf_stream_t stream);

/*
 * lpf_delta_swap for the Monte-Carlo lineal path function (Sec. 3 opening):
 * only translations x with sel_dev[x] != 0 (H*W uint8, the sampled
 * positions, N = their number) are counted, as in lpf_full_mc, and the
 * descriptor is count / N.  counts_dev are then the cell's lpf_full_mc counts
 * for the same selection; dcounts_dev and de_dev as in lpf_delta_swap.
 * Copies the selection to the host to count it (synchronises); N = 0 is
 * LPF_EINVAL.  Errors: as lpf_delta_swap.
 */
int lpf_delta_swap_mc(const uint8_t *img_dev, int32_t H, int32_t W, lpf_paths *paths, const uint8_t *sel_dev,
                      const int32_t *pairs_dev, int32_t K, int32_t *dcounts_dev, const float *target_dev,
                      const int64_t *counts_dev, float *de_dev, lpf_stream_t stream);

/*
 * Two-point probability function of phase `phase` (Sec. 2.1), the baseline
 * descriptor: s2_dev[y][x] = 1/(W*H) * IDFT(DFT(chi) * conj(DFT(chi)))(x, y),
 * chi the indicator of the phase, which equals the direct periodic sum of
 * Eq. (S2dis) over (x1, y1) of chi(x1,y1) chi((x1+x)%W, (y1+y)%H) / (W*H).
 * img_dev: H*W uint8 (0/1); s2_dev: float [H][W] (row y = row offset,
 * column x = column offset).  Transforms in double precision (cuFFT), result
 * rounded to float32.  The first call for a size creates FFT plans and a
 * work area (cached per device and size; not for use inside stream capture
 * the first time).  H*W <= 2^26.  Errors: LPF_EINVAL, LPF_ECUDA, LPF_ENOMEM.
 */
int s2_fft(const uint8_t *img_dev, int32_t H, int32_t W, int32_t phase, float *s2_dev,
           lpf_stream_t stream);

/* ---- Volumes (3D extension; Sec. 2 remark on 3D media, Sec. 6.3) ---- */

/*
 * Segments of every vector |dx| <= rx, |dy| <= ry, |dz| <= rz of a volume
 * and the prefix-tree program over them.  The paper mentions the 3D
 * extension without defining 3D segments; this library takes the 2D rule
 * on every minor axis: for v = (dx, dy, dz), a = max(|dx|, |dy|, |dz|), step
 * i = 0..a moves round(i |d_j| / a) along every axis j (exact halves away
 * from the start), |S(v)| = a + 1; the half-domain is dz > 0, or dz = 0 and
 * (dx, dy) in the 2D half-domain, and S(v) = v + S(-v) outside it.
 * Host-only.  rx, ry, rz in [0, 1023].  The handle serves lpf_full_3d,
 * lpf_paths_info / _export / _stats / _work / _status, lpf_set_checked and
 * lpf_paths_free; image calls (lpf_full, lpf_delta_swap, batches,
 * annealers) refuse it with LPF_EINVAL.
 * Errors: LPF_EINVAL, LPF_ENOMEM, LPF_EUNSUPPORTED.
 */
int lpf_build_paths_3d(int32_t rx, int32_t ry, int32_t rz, lpf_paths **out);

/*
 * Full lineal path counts of both phases of a periodic volume: vol_dev
 * uint8 [D][H][W] (0/1), voxel (x, y, z) = vol[z][y][x], coordinates
 * wrapping modulo W, H, D; count_p(v) = #{x : vol[(x + s) mod (W,H,D)] == p
 * for all s in S(v)}.  counts_dev int64 [2][(2rz+1)(2ry+1)(2rx+1)], entry
 * ((dz+rz)(2ry+1) + dy+ry)(2rx+1) + dx+rx, phase 0 first; the other half of
 * the window filled by point symmetry.  The same bit-parallel prefix-tree
 * walk as lpf_full: slices packed as bit rows extended periodically by ry
 * rows and, as slices, by rz; a block stages the rows of its 32-row bands
 * plus the halo rows of the next rz slices.  Requires rx < W, ry < H,
 * rz < D, sizes up to 4096, at most 8192 bands of 32 rows over all slices,
 * and (rz (H + 2ry) + 32 + 2ry) rows of about (W + 2rx)/32 + 2 words in
 * shared memory (about 227 KB), else LPF_EUNSUPPORTED.  First call per size allocates as lpf_full does.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_full_3d(const uint8_t *vol_dev, int32_t D, int32_t H, int32_t W, lpf_paths *paths,
                int64_t *counts_dev, lpf_stream_t stream);

/* ---- Many independent images in one run of persistent walk kernels ---- */

typedef struct lpf_batch lpf_batch; /* opaque, owned by the library */

/*
 * Prepare a batch: n_img images of possibly different sizes, each with its
 * own paths handle (its own window), evaluated together as in lpf_full.
 * Host arrays of n_img entries: imgs_dev[i] device pointer to H[i]*W[i]
 * uint8 (0/1), paths[i] handle (a handle may serve several images only if
 * they have the same H and W), counts_dev[i] device pointer to int64
 * [2][n_vec_full of paths[i]].  The pointers are bound to the batch: later
 * runs read the images' current contents and overwrite the counts.
 * words_per_thread: NULL (cost model) or n_img values in {1,2,4,8} (the
 * walk kernel's words per thread for each image; each image's row words
 * must split into at most 8 groups of that many words, else LPF_EUNSUPPORTED).  Uploads the batch's own copy
 * of each handle's program (so later calls with the handles alone, in any
 * launch shape, leave the batch intact; the handles must outlive the batch
 * only for lpf_batch_autotune) and allocates the batch's work area
 * (synchronous).
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_batch_create(int32_t n_img, const uint8_t *const *imgs_dev, const int32_t *H,
                     const int32_t *W, lpf_paths *const *paths, int64_t *const *counts_dev,
                     const int32_t *words_per_thread, lpf_batch **out);

/*
 * Enqueue one evaluation of every image of the batch: zero counts, pack,
 * one persistent walk kernel per words-per-thread choice present (blocks
 * visit band groups of the images, warps pull (tile, program piece) units;
 * the kernels after the first run on the batch's own streams, forked from
 * `stream` and joined back before the next step), mirror; no host-device
 * copies.  use_graph != 0 captures those launches as a CUDA graph on the
 * first call and replays it.  Runs of one batch share its work area, counters
 * and streams: order them (one stream, or events between streams).
 * Errors: LPF_EINVAL, LPF_ECUDA.
 */
int lpf_batch_run(lpf_batch *batch, int32_t use_graph, lpf_stream_t stream);

/*
 * Autotuner for a batch: for each class of images with the same number of
 * 32-pixel words per row, times every admissible words-per-thread choice on
 * the whole batch (3 runs each) and keeps the fastest; chosen_T (NULL or
 * n_img entries) receives the final choice.  The same host arrays as at
 * creation must be passed.  Synchronous; not for use inside stream capture.
 */
int lpf_batch_autotune(lpf_batch *batch, const uint8_t *const *imgs_dev, const int32_t *H,
                       const int32_t *W, int64_t *const *counts_dev, lpf_stream_t stream,
                       int32_t *chosen_T);

/* Synchronise `stream`; LPF_ETIMEOUT if a bounded wait in the batch's walk
 * kernel gave up during a run so far, else LPF_OK. */
int lpf_batch_status(lpf_batch *batch, lpf_stream_t stream);

/*
 * Work of the last lpf_batch_run, per image (both sides of its walk), in the
 * units of lpf_paths_work: executed[i] = pixel words the warps ANDed for
 * image i after the zero-count skip of Sec. 3.2, nominal[i] = the same
 * without it.  Host arrays of n_img entries, both required.  Synchronises
 * `stream`, then copies from the device.  Before any run executed is 0.
 * Errors: LPF_EINVAL, LPF_ECUDA.
 */
int lpf_batch_work(lpf_batch *batch, int64_t *executed, int64_t *nominal, lpf_stream_t stream);

/* Release a batch (NULL is ignored); synchronises the device. */
void lpf_batch_free(lpf_batch *batch);

/* ---- Simulated annealing (Sec. 4, Alg. 3) on exact lineal path counts ---- */

typedef struct lpf_sa lpf_sa; /* opaque annealer state, owned by the library */

typedef struct {
  int64_t n_step;      /* swap evaluations in the whole run (N_step) */
  int64_t c_max;       /* attempts per temperature stage */
  int64_t s_max;       /* acceptances per temperature stage */
  double t_max;        /* initial temperature; <= 0: chosen so that an average
                          uphill move of the initial image is accepted with
                          probability 1/2 (the paper tunes it by hand for s/c ~ 0.5) */
  double t_min_ratio;  /* T_min / T_max (Tab. annealing: 0.01) */
  int32_t k_max;       /* candidates per batch, upper bound (e.g. 4096) */
  int32_t k_min;       /* candidates per batch, lower bound (e.g. 1) */
  uint64_t seed;       /* Philox-4x32-10 key of the run */
  int32_t phases;      /* lineal-path runs: phases in the error, bit p = phase p
                          (0 or 3: both, the L2 compression of Sec. 6; 2: phase 1
                          only, L2^w of Tab. mutual with phase 1 the particles;
                          1: phase 0 only, L2^b).  Ignored by s2_sa_create. */
} lpf_sa_params;

typedef struct {
  int64_t n_eval;        /* swap evaluations consumed (as a sequential annealer counts them) */
  int64_t n_accept;      /* accepted swaps */
  int64_t n_batches;     /* batches run */
  int64_t n_candidates;  /* candidates evaluated on the GPU, including those discarded
                            after an earlier acceptance in the same batch */
  double temperature;    /* current T */
  double error;          /* current Eq. (LSE) error (running sum of accepted changes) */
  double t_max;          /* initial temperature actually used */
  int32_t next_batch;    /* candidates the next batch will evaluate */
  int32_t done;          /* 1 once n_eval reached n_step (or no swap is possible) */
} lpf_sa_stats;

/*
 * Start an annealing run on the cell cell_dev (H*W uint8, 0/1, modified in
 * place by later lpf_sa_run calls; the caller supplies the random initial
 * image with the wanted volume fraction, Alg. 3 create_random_image).
 * target_dev: float [2][n_vec_full] target descriptor (counts of the original
 * divided by its area, e.g. from lpf_full on the original with the same
 * window: the descriptor cut of Sec. 6).  counts_dev: int64 [2][n_vec_full],
 * filled here with the cell's counts and kept current by the run.  The
 * paths window must satisfy the lpf_delta_swap limits.  Candidate n of the
 * run (n = 0, 1, ...) is an interfacial phase-1 / phase-0 pixel pair, each
 * uniform over its set, drawn by rejection sampling with Philox-4x32-10
 * (attempt j uses counter (n_lo, n_hi, j, 0), key = seed; words 0 and 1
 * propose floor(r*H*W/2^32)) from the then-current cell, with Metropolis
 * uniform U = ((r2 >> 8) + 1/2) / 2^24 from attempt 0, so the run equals the
 * sequential annealer step for step whatever the batch sizes.  The run's
 * device buffers include count changes for k_max candidates
 * (k_max * 2 * n_vec_canon int32).
 * Synchronises `stream`; allocates the run's device buffers.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_sa_create(uint8_t *cell_dev, int32_t H, int32_t W, lpf_paths *paths,
                  const float *target_dev, int64_t *counts_dev, const lpf_sa_params *params,
                  lpf_stream_t stream, lpf_sa **out);

/*
 * lpf_sa_create driven by the Monte-Carlo lineal path function (the
 * reconstructions of Fig. ComMicRec): the cell's descriptor counts only the
 * translations sampled in sel_dev (H*W uint8, fixed for the run, N of them)
 * and is count / N; target_dev is the original's (Monte-Carlo) descriptor,
 * counts_dev receives the cell's lpf_full_mc counts and is kept current.
 * Everything else as lpf_sa_create.  Errors: as lpf_sa_create; N = 0 is
 * LPF_EINVAL.
 */
int lpf_sa_create_mc(uint8_t *cell_dev, int32_t H, int32_t W, lpf_paths *paths, const uint8_t *sel_dev,
                     const float *target_dev, int64_t *counts_dev, const lpf_sa_params *params,
                     lpf_stream_t stream, lpf_sa **out);

/*
 * Enqueue n_batches annealing batches on `stream` without synchronising.
 * A batch draws the next k candidates, evaluates all of them as
 * lpf_delta_swap does, accepts the first that passes the Metropolis test
 * (Delta e <= 0 or U < exp(-Delta e / T)), applies it to the cell and the
 * counts and updates the temperature stage; k adapts to the acceptance rate
 * p (running estimate) as ceil(1/(2p)), clamped to [k_min, k_max].  Batches
 * after the run is done do nothing.
 * Lineal-path runs use one cooperative launch of a persistent kernel for up
 * to 4096 batches (or the proposer's refresh interval), whose resident
 * blocks keep the cell on chip and meet at a bounded grid barrier once per
 * batch.  S2 runs (and devices without cooperative launch) use one kernel
 * launch per batch, the first call with n_batches >= 16 (or >= the refresh
 * interval) capturing that many as a CUDA graph that is replayed afterwards.
 * Both give the same run.  Errors: LPF_EINVAL, LPF_ECUDA.
 */
int lpf_sa_run(lpf_sa *sa, int32_t n_batches, lpf_stream_t stream);

/* Synchronise `stream` and copy the run's counters to *out.  LPF_ETIMEOUT if
 * a bounded wait in a batch kernel gave up (staging copy or grid barrier)
 * since the last read: the library has then already made the state
 * consistent again -- counts recomputed from the cell, the error from the
 * counts, the run's counters those of the cell's last applied batch -- so
 * the run can continue; the flag is cleared (reported once). */
int lpf_sa_read(lpf_sa *sa, lpf_sa_stats *out, lpf_stream_t stream);

/*
 * Checkpoint of an annealing run's progress (no counterpart in the paper,
 * whose runs "lasted days" without one): with the cell at that moment, it
 * resumes the run exactly -- create an annealer on the saved cell with the
 * same parameters and t_max = the saved t_max, then lpf_sa_import_progress.
 * Candidate draws depend only on the seed, the evaluation counter and the
 * cell, and counts are exact integers, so the resumed run equals the
 * uninterrupted one step for step.
 */
typedef struct {
  int64_t n_eval, n_accept, n_batches, n_candidates;
  int64_t c_stage, s_stage;  /* attempts and acceptances in the current temperature stage */
  double temperature, error, p_est, t_max;
  int32_t next_batch, done;
  uint64_t seed;             /* checked on import */
  int64_t n_step, c_max, s_max;  /* checked on import */
  double t_min_ratio;        /* checked on import */
} lpf_sa_progress;

/* Copy the run's progress to *out (synchronises `stream`). */
int lpf_sa_export_progress(lpf_sa *sa, lpf_sa_progress *out, lpf_stream_t stream);

/* Set the run's progress from *in (synchronises).  LPF_EINVAL if the run was
 * created with another seed, n_step, c_max, s_max or t_min_ratio.  A learned
 * proposer is not part of the progress: set it again after the import. */
int lpf_sa_import_progress(lpf_sa *sa, const lpf_sa_progress *in, lpf_stream_t stream);

/* Recompute the error from the exact counts in double precision, store it
 * as the run's current error and return it in *e (may be NULL). Synchronises. */
int lpf_sa_recompute_error(lpf_sa *sa, double *e, lpf_stream_t stream);

/* The next k candidates the run would draw from its current state
 * (pairs_dev int32 [k][2]: phase-1 pixel, phase-0 pixel; u_dev float [k]
 * Metropolis uniforms), without advancing the run.  k <= k_max.
 * Synchronises.  For inspection and tests. */
int lpf_sa_propose(lpf_sa *sa, int32_t k, int32_t *pairs_dev, float *u_dev, lpf_stream_t stream);

/*
 * Check of the annealer's failure detection (no counterpart in the paper):
 * runs one batch of the persistent kernel whose grid barrier waits for one
 * block arrival more than the grid makes -- in every block (block = -1) or in
 * block `block` only (0 <= block < the kernel's grid, the others pass and
 * apply the batch's decision to their vector chunks) -- so that those
 * blocks' bounded waits run out (about a second or two).  Then it restores a
 * consistent state as lpf_sa_read does (counts recomputed from the cell) and
 * clears the status.  Returns LPF_OK when the kernel reported the timeout
 * and the run state is that of before the batch (block = -1 or 0: block 0,
 * which keeps the state, gave up) or that after it (another block gave up);
 * the run continues as the sequential annealer would from that cell.
 * Synchronises.  LPF_EUNSUPPORTED when the run does not use the persistent
 * kernel; LPF_EINVAL for a bad block; LPF_ETIMEOUT if an earlier wait had
 * already failed; LPF_ECUDA if the timeout was not reported.
 */
int lpf_sa_selftest_timeout(lpf_sa *sa, int32_t block, lpf_stream_t stream);

/* Release a run (NULL is ignored); synchronises the device. */
void lpf_sa_free(lpf_sa *sa);

/* ---- Two-point probability as the annealing objective (Sec. 2.1, Sec. 6) ---- */

/*
 * Exact autocorrelation counts of phase 1 (Eq. (S2dis) times W*H):
 * counts_dev[y][x] = sum over (x1, y1) of chi(x1, y1) * chi((x1+x)%W, (y1+y)%H),
 * chi the phase-1 indicator of img_dev (H*W uint8, 0/1).  counts_dev: int64
 * [H][W], device memory owned by the caller.  Direct double sum on bit-packed
 * rows (H*W*H*ceil(W/32) word operations), meant for annealing cells; the
 * float descriptor of a large original comes from s2_fft.  Allocates a work
 * area on `stream` (stream-ordered).  H*W <= 2^20, else LPF_EUNSUPPORTED.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ECUDA.
 */
int s2_counts(const uint8_t *img_dev, int32_t H, int32_t W, int64_t *counts_dev, lpf_stream_t stream);

/*
 * Changes of the S2 counts and of the S2 error for K candidate exchanges of
 * the image img_dev (not modified), the S2 analogue of lpf_delta_swap.
 *   pairs_dev    int32 [K][2] pixel indices y*W + x; a pair of equal phases
 *                (or a == b) is the identity (all changes 0).
 *   dcounts_dev  int32 [K][H][W] or NULL: counts after minus before for
 *                every offset, exact; not written for a pair with an index
 *                out of range.
 *   target_dev   float [H][W]: the target S2 of phase 1 at each offset of the
 *                cell (needed with de_dev); counts_dev int64 [H][W]: the
 *                image's current counts (from s2_counts).
 *   de_dev       float [K] or NULL: e(after) - e(before) with e = sum over all
 *                H*W offsets of (target - counts/(H*W))^2 (Eq. (LSE) on S2),
 *                float32, summed in a fixed order (bitwise reproducible);
 *                NaN for a pair with an index out of range or when a bounded
 *                wait for the staging copy gave up.
 * The periodically extended cell (W + 2 ceil(W/2)) x (H + 2 ceil(H/2)) bytes
 * must fit in shared memory (about 227 KB), else LPF_EUNSUPPORTED.  Work
 * areas are allocated on `stream` (stream-ordered).
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ECUDA.
 */
int s2_delta_swap(const uint8_t *img_dev, int32_t H, int32_t W, const int32_t *pairs_dev, int32_t K,
                  int32_t *dcounts_dev, const float *target_dev, const int64_t *counts_dev, float *de_dev,
                  lpf_stream_t stream);

/*
 * Start an annealing run (Alg. 3) whose objective is the S2 error above
 * instead of the lineal path error: the S2-based compression of Sec. 6
 * (Tab. mutual).  target_dev float [H][W]: the target S2 of phase 1 per
 * offset of the cell (e.g. an original's S2 cut to the cell's centred offset
 * window); counts_dev int64 [H][W]: filled with the cell's counts
 * (s2_counts) and kept current.  Everything else -- proposals, Metropolis
 * test, schedule, batches, graphs -- is that of lpf_sa_create, and the
 * handle is driven and released by lpf_sa_run / lpf_sa_read /
 * lpf_sa_recompute_error / lpf_sa_propose / lpf_sa_set_proposer /
 * lpf_sa_free.  Cell limits: H, W >= 2, H*W <= 2^20 and the extended cell of
 * s2_delta_swap in shared memory.
 * Errors: LPF_EINVAL, LPF_EUNSUPPORTED, LPF_ENOMEM, LPF_ECUDA.
 */
int s2_sa_create(uint8_t *cell_dev, int32_t H, int32_t W, const float *target_dev, int64_t *counts_dev,
                 const lpf_sa_params *params, lpf_stream_t stream, lpf_sa **out);

/* ---- Learned swap proposer (no counterpart in the paper) ---- */

typedef struct lpf_cnn lpf_cnn; /* opaque network, owned by the library */

/*
 * A small convolutional network that scores every pixel of an H x W cell as
 * the phase-1 pixel (output channel 1) or the phase-0 pixel (channel 0) of an
 * exchange.  The paper's modification operator (Sec. 4) draws interfacial
 * pixels uniformly; the network only changes which candidates are drawn --
 * every accept/reject decision of the annealer still uses exact counts.
 * Layers: five 3x3 convolutions with circular padding (periodic medium) and
 * ReLU between them, channels 2 -> 32 -> 64 -> 48 -> 32 -> 2 (61,234
 * parameters); input channels: cell value, interfacial mask.  Weights are
 * kept as float32 masters (updated by Adam) and bfloat16 copies (used by the
 * forward and backward kernels); activations and accumulation are float32.
 * Parameter vector layout (lpf_cnn_set_params / get_params): for each layer,
 * W [9][Cin][Cout] (tap = (dy+1)*3 + (dx+1)) then b [Cout].
 * lpf_cnn_create initialises He-normal weights (seeded) and allocates the
 * network's device memory for H x W cells.  Errors: LPF_EINVAL, LPF_ENOMEM.
 */
int lpf_cnn_create(int32_t H, int32_t W, uint64_t seed, lpf_cnn **out);

/*
 * Training loss of lpf_cnn_gradients / lpf_cnn_train_step.  kind 0 (the
 * default): L = 1/(2n) sum_i (s1[a_i] + s0[b_i] - y_i)^2.  kind 1 (listwise):
 * L = -sum_i q_i log p_i with q = softmax(y / beta) and p = softmax(s1[a] +
 * s0[b]) over the snapshot's candidates (the annealer draws pixels with
 * probability proportional to exp(score / tau)).  Errors: LPF_EINVAL.
 */
int lpf_cnn_set_loss(lpf_cnn *cnn, int32_t kind, float beta);
int64_t lpf_cnn_num_params(const lpf_cnn *cnn);
int lpf_cnn_set_params(lpf_cnn *cnn, const float *params_host, int64_t n);      /* synchronous */
int lpf_cnn_get_params(const lpf_cnn *cnn, float *params_host, int64_t n);      /* synchronous */

/* Scores of a cell: scores_dev float [H][W][2] (may be NULL to only refresh
 * the network's internal output buffer). */
int lpf_cnn_forward(lpf_cnn *cnn, const uint8_t *cell_dev, float *scores_dev, lpf_stream_t stream);

/*
 * Gradient of the loss of one snapshot, for checking: with n logged
 * candidates (pairs_dev int32 [n][2] = phase-1 pixel a, phase-0 pixel b;
 * y_dev float [n] targets), L = 1/(2n) sum_i (s1[a_i] + s0[b_i] - y_i)^2;
 * grads_dev float [n_params] (may be NULL), loss_dev float (may be NULL).
 */
int lpf_cnn_gradients(lpf_cnn *cnn, const uint8_t *cell_dev, const int32_t *pairs_dev, const float *y_dev,
                      int32_t n, float *grads_dev, float *loss_dev, lpf_stream_t stream);

/*
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean loss of B
 * snapshots: cells_dev uint8 [B][H][W], pairs_dev int32 [B][n][2], y_dev
 * float [B][n]; loss_dev (may be NULL) receives the mean loss before the step.
 * Up to 8 snapshots go through the network together (one launch per layer
 * and pass); the first call that trains on more snapshots than any before
 * allocates the training buffers and synchronises the device.  The result
 * does not depend on that grouping.
 */
int lpf_cnn_train_step(lpf_cnn *cnn, const uint8_t *cells_dev, int32_t B, const int32_t *pairs_dev,
                       const float *y_dev, int32_t n, float lr, float *loss_dev, lpf_stream_t stream);

void lpf_cnn_free(lpf_cnn *cnn);

/*
 * Let an annealing run draw candidates from the network: before every graph
 * of batches (every `refresh` batches) the network scores the current cell
 * and the run builds, per phase, sampling weights exp((s - max s) / tau) over
 * the interfacial pixels of that phase; each candidate then takes, with
 * probability epsilon, the uniform draw of lpf_sa_create, and otherwise
 * draws each pixel from these weights (a drawn pixel that no longer has the
 * wanted phase or is no longer interfacial is rejected and drawn again).
 * cnn = NULL restores uniform draws.  The network must stay alive while the
 * run uses it.  Errors: LPF_EINVAL, LPF_ENOMEM, LPF_ECUDA.
 */
int lpf_sa_set_proposer(lpf_sa *sa, lpf_cnn *cnn, float epsilon, float tau, int32_t refresh);

/*
 * Measurement hook: when ev_start/ev_stop (cudaEvent_t, created by the
 * caller) are non-NULL, every later device call on this handle records
 * ev_start on its stream right before its dominant kernel and ev_stop right
 * after it, so a caller can time that kernel alone.  NULL, NULL turns it off.
 * The events stay owned by the caller.  Errors: LPF_EINVAL (paths == NULL).
 */
int lpf_paths_set_timer(lpf_paths *paths, void *ev_start, void *ev_stop);

/*
 * Device-side status of the handle's last calls (and of lpf_full_noalloc
 * calls on the current device): synchronises `stream`, returns LPF_ETIMEOUT
 * if a bounded wait inside a kernel gave up, else LPF_EPIXEL if a kernel read
 * a pixel other than 0 or 1 in checked mode, else LPF_EINVAL if a kernel met
 * an out-of-range pixel index, since the last check (and clears the flags),
 * LPF_OK otherwise.  Errors: LPF_EINVAL (paths == NULL), LPF_ECUDA.
 */
int lpf_paths_status(lpf_paths *paths, lpf_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LPF_H */
