/*
 * Reference ("oracle") implementation of the lineal path function and of the
 * quantities built on it, written as plainly as possible from Havelka,
 * Kucerova & Sykora, "Compression and Reconstruction of Random
 * Microstructures using Accelerated Lineal Path Function" (arXiv:1601.04359).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness definition that the
 * CUDA library is compared against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Conventions (readings of the paper, each restated where it is used):
 *   - image: uint8, H rows x W columns, row-major, pixel (x, y) at img[y*W + x],
 *     x = column, y = row, values 0 or 1; "phase p" means pixel value p.
 *   - periodic medium: every coordinate is taken modulo W (x) and H (y),
 *     the "%" convention of Eq. (S2dis), Sec. 2.1.
 *   - vector window |dx| <= rx, |dy| <= ry with rx < W, ry < H; the paper's
 *     full domain is rx = W-1, ry = H-1 (Eq. segments, Sec. 2.2).
 *   - full output layout: counts[p][(dy+ry)*(2rx+1) + (dx+rx)], p in {0,1}.
 *   - canonical half: dy > 0, or dy == 0 and dx >= 0 (the domain D of
 *     Eq. segments); its entries are the tail of the full layout starting
 *     at v = (0,0), so canonical index = full index - (n_full-1)/2.
 *
 * Nothing here is blocked, fused or reordered beyond the paper's loops.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int imod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }
static int iabs(int a) { return a < 0 ? -a : a; }

/* Threads of later OpenMP loops (n >= 1); for timing the oracle on one core. */
void lpfo_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int lpfo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* 1 when v = (dx, dy) lies in the half-domain D of Eq. segments (Sec. 2.2). */
int lpfo_is_canonical(int dx, int dy) { return dy > 0 || (dy == 0 && dx >= 0); }

/*
 * Pixel offsets of the discretised segment from (0,0) to v = (dx, dy)
 * (Sec. 2.2: Bresenham's segment between the two end pixels).
 *
 * For v in D: a = max(|dx|,|dy|) steps along the major axis; step i = 0..a
 * moves i along the major axis and, along the minor axis, to the pixel
 * nearest the ideal line, i.e. round(i*b/a) with b = min(|dx|,|dy|); the
 * paper does not say how a tie (exactly half-way) is broken, and this reading
 * rounds it away from the start pixel: floor((2*i*b + a) / (2*a)).
 * Both end pixels are included, so the segment has a+1 pixels, which is the
 * per-segment term max(i,j) of the storage count M (Sec. 3.1).
 *
 * For v outside D the segment is the same geometric pixel set as the one of
 * -v, started from the other end: S(v) = v + S(-v).  This keeps the point
 * symmetry L(v) = L(-v) of Eq. (symmetry) exact.
 *
 * Returns the number of pixels, writes them to sx[], sy[] (caller-sized,
 * at least max(|dx|,|dy|)+1 entries).
 */
int lpfo_segment(int dx, int dy, int32_t *sx, int32_t *sy) {
    if (!lpfo_is_canonical(dx, dy)) {
        int n = lpfo_segment(-dx, -dy, sx, sy);
        for (int i = 0; i < n; ++i) { sx[i] += dx; sy[i] += dy; }
        return n;
    }
    int ax = iabs(dx), ay = iabs(dy);
    int a = ax > ay ? ax : ay;
    int b = ax > ay ? ay : ax;
    int gx = dx < 0 ? -1 : 1, gy = dy < 0 ? -1 : 1;
    for (int i = 0; i <= a; ++i) {
        int minor = (a == 0) ? 0 : (2 * i * b + a) / (2 * a);
        if (ax >= ay) { sx[i] = gx * i;     sy[i] = gy * minor; }
        else          { sx[i] = gx * minor; sy[i] = gy * i; }
    }
    return a + 1;
}

/*
 * Number of translations x of the segment S(v) whose every pixel is in phase
 * `phase` -- Alg. 1 (Sec. 3.1) for one segment: loop over the W*H
 * translations, walk the segment's pixels, stop at the first pixel that is not
 * in the phase, count the translation when the walk reached the end.  The
 * paper's 2x2 periodic copy of the image is replaced by the equivalent modulo.
 */
int64_t lpfo_count_segment(const uint8_t *img, int H, int W,
                           const int32_t *sx, const int32_t *sy, int n, int phase) {
    int64_t L = 0;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int pix;
            for (pix = 0; pix < n; ++pix) {
                int xx = imod(x + sx[pix], W), yy = imod(y + sy[pix], H);
                if (img[(int64_t)yy * W + xx] != phase) break;
            }
            if (pix == n) L += 1;
        }
    }
    return L;
}

/* count_phase(v) for one vector v = (dx, dy). */
int64_t lpfo_count(const uint8_t *img, int H, int W, int dx, int dy, int phase) {
    int n = (iabs(dx) > iabs(dy) ? iabs(dx) : iabs(dy)) + 1;
    int32_t *sx = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *sy = (int32_t *)malloc(sizeof(int32_t) * n);
    lpfo_segment(dx, dy, sx, sy);
    int64_t c = lpfo_count_segment(img, H, W, sx, sy, n, phase);
    free(sx); free(sy);
    return c;
}

/*
 * Counts of both phases for every vector of the window, in the full layout
 * counts[p][(dy+ry)*(2rx+1) + (dx+rx)].  Every vector is evaluated directly,
 * including the half that Eq. (symmetry) would let one mirror, so the
 * symmetry itself stays a checkable property of the result.
 * Loops over vectors are shared among OpenMP threads; each vector is Alg. 1.
 */
void lpfo_lpf_full(const uint8_t *img, int H, int W, int rx, int ry, int64_t *counts) {
    int nx = 2 * rx + 1, ny = 2 * ry + 1;
    int64_t nfull = (int64_t)nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nfull; ++k) {
        int dy = (int)(k / nx) - ry, dx = (int)(k % nx) - rx;
        for (int p = 0; p < 2; ++p)
            counts[p * nfull + k] = lpfo_count(img, H, W, dx, dy, p);
    }
}

/*
 * Monte-Carlo approximation of Sec. 3 (opening): the segments are compared
 * with the image only at the selected translations x (sel[y*W + x] != 0);
 * counts[p][k] = number of selected translations whose segment lies in phase
 * p, full layout, every vector evaluated directly (Alg. 1 with the
 * translation loop restricted to the selection).  L~ = counts / N, N = number
 * of selected translations.
 */
void lpfo_lpf_full_sel(const uint8_t *img, int H, int W, int rx, int ry, const uint8_t *sel, int64_t *counts) {
    int nx = 2 * rx + 1, ny = 2 * ry + 1;
    int64_t nfull = (int64_t)nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nfull; ++k) {
        int dy = (int)(k / nx) - ry, dx = (int)(k % nx) - rx;
        int n = (iabs(dx) > iabs(dy) ? iabs(dx) : iabs(dy)) + 1;
        int32_t *sx = (int32_t *)malloc(sizeof(int32_t) * n);
        int32_t *sy = (int32_t *)malloc(sizeof(int32_t) * n);
        lpfo_segment(dx, dy, sx, sy);
        for (int p = 0; p < 2; ++p) {
            int64_t L = 0;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    if (!sel[(int64_t)y * W + x]) continue;
                    int pix;
                    for (pix = 0; pix < n; ++pix) {
                        int xx = imod(x + sx[pix], W), yy = imod(y + sy[pix], H);
                        if (img[(int64_t)yy * W + xx] != p) break;
                    }
                    if (pix == n) L += 1;
                }
            counts[p * nfull + k] = L;
        }
        free(sx); free(sy);
    }
}

/* Counts for an explicit list of vectors: out[2*i + p] for vec (dx[i], dy[i]). */
void lpfo_count_list(const uint8_t *img, int H, int W, const int32_t *dx,
                     const int32_t *dy, int n, int64_t *out) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < 2; ++p)
            out[2 * i + p] = lpfo_count(img, H, W, dx[i], dy[i], p);
}

/*
 * Change of the canonical-half counts caused by exchanging the values of
 * pixels a and b (linear indices y*W + x): the annealer's modification
 * operator (Sec. 4, swapping two pixels of different phases).  Computed by
 * definition: count every canonical vector on the image after the exchange
 * and subtract the count on the image before it.  A pair whose pixels hold
 * the same value leaves the image unchanged, so its change is zero.
 * dcounts layout: [K][2][n_canon], n_canon = ry*(2rx+1) + rx + 1, with
 * canonical index = full index - base, base = (n_full - 1) / 2.
 */
void lpfo_delta_swap(const uint8_t *img, int H, int W, int rx, int ry,
                     const int32_t *pairs, int K, int64_t *dcounts) {
    int nx = 2 * rx + 1;
    int64_t nfull = (int64_t)nx * (2 * ry + 1);
    int64_t base = (nfull - 1) / 2;
    int64_t ncanon = nfull - base;
    int64_t npix = (int64_t)H * W;
    int64_t *before = (int64_t *)malloc(sizeof(int64_t) * 2 * ncanon);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncanon; ++c) {
        int64_t k = base + c;
        int dy = (int)(k / nx) - ry, dx = (int)(k % nx) - rx;
        for (int p = 0; p < 2; ++p) before[p * ncanon + c] = lpfo_count(img, H, W, dx, dy, p);
    }
    uint8_t *work = (uint8_t *)malloc((size_t)npix);
    for (int q = 0; q < K; ++q) {
        int a = pairs[2 * q], b = pairs[2 * q + 1];
        int64_t *out = dcounts + (int64_t)q * 2 * ncanon;
        if (img[a] == img[b]) {
            memset(out, 0, sizeof(int64_t) * 2 * ncanon);
            continue;
        }
        memcpy(work, img, (size_t)npix);
        uint8_t t = work[a]; work[a] = work[b]; work[b] = t;
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < ncanon; ++c) {
            int64_t k = base + c;
            int dy = (int)(k / nx) - ry, dx = (int)(k % nx) - rx;
            for (int p = 0; p < 2; ++p)
                out[p * ncanon + c] = lpfo_count(work, H, W, dx, dy, p) - before[p * ncanon + c];
        }
    }
    free(work); free(before);
}

/*
 * Least-square error of Eq. (LSE) (Sec. 4) between a target descriptor and
 * the descriptor of the current image, over the phases set in `phases`
 * (bit 0: phase 0, bit 1: phase 1; 3 = both, the L2 of Sec. 6's Tab. mutual,
 * 1 or 2 = the single-phase L2^b or L2^w compressions) and over the
 * canonical half D of the window, in double precision.
 * target: float32 [2][n_full] (already normalised, e.g. counts / (W0*H0) of
 * the original); counts: int64 [2][n_full]; the image descriptor is
 * counts / (W*H) of the current cell.
 */
double lpfo_objective(const float *target, const int64_t *counts, int rx, int ry, int H, int W, int phases) {
    int64_t nfull = (int64_t)(2 * rx + 1) * (2 * ry + 1);
    int64_t base = (nfull - 1) / 2;
    double n = (double)H * (double)W, e = 0.0;
    for (int p = 0; p < 2; ++p)
        if (phases & (1 << p))
        for (int64_t k = base; k < nfull; ++k) {
            double d = (double)target[p * nfull + k] - (double)counts[p * nfull + k] / n;
            e += d * d;
        }
    return e;
}

/*
 * Change of Eq. (LSE) for every candidate: e(counts + dcounts[k]) - e(counts),
 * over the phases set in `phases` as above, in double precision, each term
 * written out as the definition.
 */
void lpfo_delta_objective(const float *target, const int64_t *counts, const int64_t *dcounts,
                          int K, int rx, int ry, int H, int W, int phases, double *de) {
    int64_t nfull = (int64_t)(2 * rx + 1) * (2 * ry + 1);
    int64_t base = (nfull - 1) / 2;
    int64_t ncanon = nfull - base;
    double n = (double)H * (double)W;
    for (int q = 0; q < K; ++q) {
        const int64_t *dq = dcounts + (int64_t)q * 2 * ncanon;
        double after = 0.0, before = 0.0;
        for (int p = 0; p < 2; ++p) {
            if (!(phases & (1 << p))) continue;
            for (int64_t c = 0; c < ncanon; ++c) {
                double t = (double)target[p * nfull + base + c];
                double c0 = (double)counts[p * nfull + base + c];
                double d0 = t - c0 / n;
                double d1 = t - (c0 + (double)dq[p * ncanon + c]) / n;
                before += d0 * d0;
                after += d1 * d1;
            }
        }
        de[q] = after - before;
    }
}

/*
 * Autocorrelation counts of phase 1, C[y][x] = sum over (x1, y1) of
 * chi(x1,y1) * chi((x1+x)%W, (y1+y)%H): W*H times S2 of Eq. (S2dis), as
 * exact integers (direct double sum).
 */
void lpfo_s2_counts(const uint8_t *img, int H, int W, int64_t *C) {
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t acc = 0;
            for (int y1 = 0; y1 < H; ++y1)
                for (int x1 = 0; x1 < W; ++x1)
                    acc += (img[(int64_t)y1 * W + x1] == 1) &&
                           (img[(int64_t)((y1 + y) % H) * W + (x1 + x) % W] == 1);
            C[(int64_t)y * W + x] = acc;
        }
}

/*
 * Change of the least-square S2 error e = sum over all offsets d of
 * (t[d] - C[d]/(W*H))^2 (Eq. (LSE) with the phase-1 two-point probability)
 * for exchanging the values of pixels a and b, by definition: recompute the
 * counts on the exchanged image.  Double precision.
 */
void lpfo_s2_delta_objective(const uint8_t *img, int H, int W, const float *t, const int32_t *pairs, int K,
                             double *de) {
    int64_t npix = (int64_t)H * W;
    int64_t *C0 = (int64_t *)malloc(sizeof(int64_t) * npix);
    int64_t *C1 = (int64_t *)malloc(sizeof(int64_t) * npix);
    uint8_t *work = (uint8_t *)malloc((size_t)npix);
    lpfo_s2_counts(img, H, W, C0);
    double inv = 1.0 / (double)npix;
    for (int q = 0; q < K; ++q) {
        memcpy(work, img, (size_t)npix);
        uint8_t v = work[pairs[2 * q]];
        work[pairs[2 * q]] = work[pairs[2 * q + 1]];
        work[pairs[2 * q + 1]] = v;
        lpfo_s2_counts(work, H, W, C1);
        double before = 0.0, after = 0.0;
        for (int64_t d = 0; d < npix; ++d) {
            double e0 = (double)t[d] - (double)C0[d] * inv, e1 = (double)t[d] - (double)C1[d] * inv;
            before += e0 * e0;
            after += e1 * e1;
        }
        de[q] = after - before;
    }
    free(C0); free(C1); free(work);
}

/*
 * Two-point probability of Eq. (S2dis) (Sec. 2.1) by its direct double sum:
 * s2[y][x] = 1/(W*H) * sum over (x1, y1) of chi(x1,y1) * chi((x1+x)%W, (y1+y)%H)
 * with chi the indicator of `phase`.  O((W*H)^2); small images only.
 */
void lpfo_s2_direct(const uint8_t *img, int H, int W, int phase, double *s2) {
    double inv = 1.0 / ((double)W * (double)H);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t acc = 0;
            for (int y1 = 0; y1 < H; ++y1)
                for (int x1 = 0; x1 < W; ++x1) {
                    int c1 = img[(int64_t)y1 * W + x1] == phase;
                    int c2 = img[(int64_t)((y1 + y) % H) * W + (x1 + x) % W] == phase;
                    acc += c1 * c2;
                }
            s2[(int64_t)y * W + x] = (double)acc * inv;
        }
}

/* ---- Three-dimensional extension (Sec. 2, remark on 3D media; Sec. 6.3) ----
 *
 * The paper states that the lineal path function extends to 3D media but
 * defines no 3D segment.  Reading: the same Bresenham rule per minor axis.
 * For v = (dx, dy, dz) with a = max(|dx|, |dy|, |dz|), step i = 0..a moves
 * sgn(d_j) * round(i |d_j| / a) along every axis j (the major axis exactly
 * i), an exact half rounding away from the start; |S(v)| = a + 1.  The
 * half-domain D3 is dz > 0, or dz = 0 and (dy, dx) in the 2D half-domain;
 * outside D3, S(v) = v + S(-v) as in 2D.  Volumes are vol[z][y][x], periodic
 * in all three coordinates.
 */
static int lpfo_is_canonical3(int dx, int dy, int dz) {
    return dz > 0 || (dz == 0 && lpfo_is_canonical(dx, dy));
}

int lpfo_segment3(int dx, int dy, int dz, int32_t *sx, int32_t *sy, int32_t *sz) {
    if (!lpfo_is_canonical3(dx, dy, dz)) {
        int n = lpfo_segment3(-dx, -dy, -dz, sx, sy, sz);
        for (int i = 0; i < n; ++i) { sx[i] += dx; sy[i] += dy; sz[i] += dz; }
        return n;
    }
    int ad[3] = {iabs(dx), iabs(dy), iabs(dz)};
    int g[3] = {dx < 0 ? -1 : 1, dy < 0 ? -1 : 1, dz < 0 ? -1 : 1};
    int a = ad[0];
    if (ad[1] > a) a = ad[1];
    if (ad[2] > a) a = ad[2];
    for (int i = 0; i <= a; ++i) {
        int c[3];
        for (int j = 0; j < 3; ++j) c[j] = (a == 0) ? 0 : g[j] * ((2 * i * ad[j] + a) / (2 * a));
        sx[i] = c[0]; sy[i] = c[1]; sz[i] = c[2];
    }
    return a + 1;
}

/* Alg. 1 in 3D for one segment: every translation of the periodic volume,
 * early break at the first voxel outside the phase. */
int64_t lpfo_count3(const uint8_t *vol, int D, int H, int W, int dx, int dy, int dz, int phase) {
    int ax = iabs(dx), ay = iabs(dy), az = iabs(dz);
    int n = (ax > ay ? ax : ay);
    n = (n > az ? n : az) + 1;
    int32_t *sx = (int32_t *)malloc(sizeof(int32_t) * 3 * n);
    int32_t *sy = sx + n, *sz = sx + 2 * n;
    lpfo_segment3(dx, dy, dz, sx, sy, sz);
    int64_t L = 0;
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int k;
                for (k = 0; k < n; ++k) {
                    int vz = ((z + sz[k]) % D + D) % D;
                    int vy = ((y + sy[k]) % H + H) % H;
                    int vx = ((x + sx[k]) % W + W) % W;
                    if (vol[((int64_t)vz * H + vy) * W + vx] != phase) break;
                }
                if (k == n) ++L;
            }
    free(sx);
    return L;
}

/* Counts of both phases for every vector of |dx| <= rx, |dy| <= ry,
 * |dz| <= rz in the full layout counts[p][((dz+rz)(2ry+1) + dy+ry)(2rx+1) + dx+rx];
 * every vector evaluated directly. */
void lpfo_lpf_full3(const uint8_t *vol, int D, int H, int W, int rx, int ry, int rz, int64_t *counts) {
    int nx = 2 * rx + 1, ny = 2 * ry + 1, nz = 2 * rz + 1;
    int64_t nfull = (int64_t)nx * ny * nz;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nfull; ++k) {
        int dz = (int)(k / ((int64_t)nx * ny)) - rz;
        int rem = (int)(k % ((int64_t)nx * ny));
        int dy = rem / nx - ry, dx = rem % nx - rx;
        for (int p = 0; p < 2; ++p) counts[p * nfull + k] = lpfo_count3(vol, D, H, W, dx, dy, dz, p);
    }
}
