/*
 * CPU oracle for semi-global-matching stereo and the U-/V-disparity maps.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this library.  The
 * CUDA library never calls it, and the two share no source, header, table or
 * helper.  The oracle is deliberately plain and slow: one stage after the
 * other, in the order of the paper's pipeline, full intermediate arrays,
 * integer arithmetic throughout, no blocking, fusion or reordering.
 *
 * Paper: Ruf, Monka, Kollmann, Grinberg, "Real-time on-board obstacle
 * avoidance for UAVs based on embedded stereo vision" (ISPRS TC I, 2018).
 *   Sec. 3.1.1 "Image rectification"      -> oracle_rectify
 *   Sec. 3.1.2 "Image matching", Eq. 1     -> oracle_census, oracle_cost_volume,
 *                                             oracle_sad_cost_volume
 *   Sec. 3.1.3 "SGM optimization", Eq. 2   -> oracle_aggregate_path, oracle_sum_paths,
 *                                             oracle_wta_left
 *   Sec. 3.1.4 "Left-Right consistency"    -> oracle_wta_right, oracle_lr_check
 *   Sec. 3.1.5 "Median filter"             -> oracle_median
 *   Sec. 3.2   "Obstacle Avoidance"        -> oracle_uvmap, oracle_uv_post
 *
 * Readings taken where the paper is silent or garbled (each is pinned by a
 * CPU test against brute force, a closed form or an invariant):
 *   R1 census bit k is 1 iff I(q_k) < I(p); q_k walks the cw x ch window in
 *      raster order (top-left first) with the centre skipped; neighbours
 *      outside the image contribute a 0 bit.
 *   R2 Eq. 1 for p_x - d < 0 (right pixel outside the image): cost = nbits.
 *   R3 Eq. 2 is printed without its minimum; the recurrence used is the
 *      one of Hirschmueller (2008), which the paper cites for it:
 *        L(p,d) = C(p,d) + min(L(q,d), L(q,d-1)+P1, L(q,d+1)+P1, m(q)+P2) - m(q)
 *      with q the predecessor of p on the path and m(q) = min_k L(q,k);
 *      neighbours d-1 < 0 or d+1 >= D are left out; at the first pixel of a
 *      path L = C.  The subtraction of m(q) is the normalisation of Sec. 3.1.3.
 *   R4 winner-takes-all ties go to the smallest disparity.
 *   R5 D_right(x) = argmin over d with x+d < W of S(x+d, d).
 *   R6 LR check: a pixel keeps D_left(x) iff x - D_left(x) >= 0 and
 *      |D_left(x) - D_right(x - D_left(x))| <= tol; otherwise it becomes 0xFF.
 *      tol < 0 switches the check off.
 *   R7 median: k x k window with clamped (replicated) borders; 0xFF takes
 *      part and sorts above every valid value; the ((k*k+1)/2)-th smallest
 *      is kept; k <= 1 copies the input.
 *   R8 U-map U[d][x] and V-map V[y][d] count pixels of the final map with
 *      value d < D; 0xFF is not counted.
 *   R11 map post-processing (Sec. 3.2 names the steps, not their parameters):
 *      binary B = (count >= threshold) inside the region of interest
 *      [r0, r1) x [c0, c1) of the map, 0 outside it; dilation of B by a
 *      (2r+1) x (2r+1) square (cells outside the map count as 0); then a
 *      3x3 binomial Gaussian [1 2 1; 2 4 2; 1 2 1] / 16 of 255 * dilated
 *      (cells outside the map count as 0), rounded half up:
 *      out = (sum w * 255 * b + 8) / 16.
 *   R12 rectification maps point into a source image of the same W x H;
 *      a rectified pixel whose map entry falls outside the source is 0.
 *   R13 SAD cost (Sec. 3.1.2 names a pixel-wise SAD, Sec. 4.1 a 5 x 5
 *      support region for it): C(x,y,d) = sum over the ww x wh window of
 *      |I_l(x+u, y+v) - I_r(x-d+u, y+v)|, each image read with clamped
 *      (replicated) coordinates; for x - d < 0 the cost is the maximum
 *      ww * wh * 255 (R2's rule for the census cost).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 3

/* The eight path directions (dx, dy), bit r of a path mask enables entry r:
 * 0 left->right, 1 right->left, 2 top->bottom, 3 bottom->top,
 * 4 top-left->bottom-right, 5 bottom-right->top-left,
 * 6 top-right->bottom-left, 7 bottom-left->top-right.                       */
static const int ORACLE_DIR[8][2] = {
    {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {-1, 1}, {1, -1}};

int oracle_direction(int r, int *dx, int *dy)
{
    if (r < 0 || r > 7) return ORACLE_EINVAL;
    *dx = ORACLE_DIR[r][0];
    *dy = ORACLE_DIR[r][1];
    return ORACLE_OK;
}

/* Number of bits of a cw x ch census code (centre excluded). */
int oracle_census_bits(int cw, int ch) { return cw * ch - 1; }

/* Census transform, Sec. 3.1.2 (Zabih and Woodfill), reading R1. */
int oracle_census(const uint8_t *img, int W, int H, int pitch, int cw, int ch,
                  uint64_t *codes)
{
    if (W < 1 || H < 1 || pitch < W || cw < 1 || ch < 1 || (cw % 2) == 0 ||
        (ch % 2) == 0 || cw * ch - 1 > 64)
        return ORACLE_EINVAL;
    int rx = cw / 2, ry = ch / 2;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint8_t centre = img[(size_t)y * pitch + x];
            uint64_t code = 0;
            int bit = 0;
            for (int wy = -ry; wy <= ry; wy++) {
                for (int wx = -rx; wx <= rx; wx++) {
                    if (wx == 0 && wy == 0) continue;
                    int qx = x + wx, qy = y + wy;
                    if (qx >= 0 && qx < W && qy >= 0 && qy < H &&
                        img[(size_t)qy * pitch + qx] < centre)
                        code |= (uint64_t)1 << bit;
                    bit++;
                }
            }
            codes[(size_t)y * W + x] = code;
        }
    }
    return ORACLE_OK;
}

/* Number of set bits, counted one bit at a time. */
int oracle_hamming(uint64_t a, uint64_t b)
{
    uint64_t v = a ^ b;
    int n = 0;
    for (int i = 0; i < 64; i++) n += (int)((v >> i) & 1u);
    return n;
}

/* Matching cost volume, Eq. 1 with Phi = Hamming distance of census codes,
 * reading R2.  Layout C[(y*W + x)*D + d]. */
int oracle_cost_volume(const uint64_t *cl, const uint64_t *cr, int W, int H,
                       int D, int nbits, uint16_t *C)
{
    if (W < 1 || H < 1 || D < 1 || nbits < 0 || nbits > 255) return ORACLE_EINVAL;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < D; d++) {
                size_t i = ((size_t)y * W + x) * D + d;
                if (x - d >= 0)
                    C[i] = (uint16_t)oracle_hamming(cl[(size_t)y * W + x],
                                                    cr[(size_t)y * W + x - d]);
                else
                    C[i] = (uint16_t)nbits;
            }
    return ORACLE_OK;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Matching cost volume, Eq. 1 with Phi = sum of absolute differences over a
 * ww x wh support window, reading R13.  Layout C[(y*W + x)*D + d]. */
int oracle_sad_cost_volume(const uint8_t *left, const uint8_t *right, int W, int H,
                           int pitch, int D, int ww, int wh, uint16_t *C)
{
    if (W < 1 || H < 1 || D < 1 || pitch < W || ww < 1 || wh < 1 || !(ww & 1) ||
        !(wh & 1) || ww * wh * 255 > 0xFFFF)
        return ORACLE_EINVAL;
    const int rw = ww / 2, rh = wh / 2, cmax = ww * wh * 255;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < D; d++) {
                int sum = 0;
                if (x - d < 0) {
                    sum = cmax;
                } else {
                    for (int v = -rh; v <= rh; v++)
                        for (int u = -rw; u <= rw; u++) {
                            int yy = clampi(y + v, 0, H - 1);
                            int a = left[(size_t)yy * pitch + clampi(x + u, 0, W - 1)];
                            int b = right[(size_t)yy * pitch + clampi(x - d + u, 0, W - 1)];
                            sum += a > b ? a - b : b - a;
                        }
                }
                C[((size_t)y * W + x) * D + d] = (uint16_t)sum;
            }
    return ORACLE_OK;
}

/* Aggregation along one path direction r, Eq. 2 read as R3.
 * The image is walked so that the predecessor q = p - (dx, dy) of every
 * pixel p has been visited before p: rows top-down for dy >= 0 (bottom-up
 * otherwise), columns left-right for dx >= 0 (right-left otherwise).
 * Output layout L[(y*W + x)*D + d]. */
int oracle_aggregate_path(const uint16_t *C, int W, int H, int D, int r, int P1,
                          int P2, uint16_t *L)
{
    int dx, dy;
    if (oracle_direction(r, &dx, &dy) != ORACLE_OK) return ORACLE_EINVAL;
    if (W < 1 || H < 1 || D < 1 || P1 < 0 || P2 < P1) return ORACLE_EINVAL;
    for (int iy = 0; iy < H; iy++) {
        int y = (dy >= 0) ? iy : H - 1 - iy;
        for (int ix = 0; ix < W; ix++) {
            int x = (dx >= 0) ? ix : W - 1 - ix;
            const uint16_t *c = C + ((size_t)y * W + x) * D;
            uint16_t *l = L + ((size_t)y * W + x) * D;
            int qx = x - dx, qy = y - dy;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                /* first pixel of the path */
                for (int d = 0; d < D; d++) l[d] = c[d];
                continue;
            }
            const uint16_t *lq = L + ((size_t)qy * W + qx) * D;
            int m = lq[0];
            for (int k = 1; k < D; k++)
                if (lq[k] < m) m = lq[k];
            for (int d = 0; d < D; d++) {
                int best = lq[d];
                if (d - 1 >= 0 && lq[d - 1] + P1 < best) best = lq[d - 1] + P1;
                if (d + 1 < D && lq[d + 1] + P1 < best) best = lq[d + 1] + P1;
                if (m + P2 < best) best = m + P2;
                l[d] = (uint16_t)(c[d] + best - m);
            }
        }
    }
    return ORACLE_OK;
}

/* S = sum over the paths of the mask, Sec. 3.1.3 (C_aggr). */
int oracle_sum_paths(const uint16_t *C, int W, int H, int D, int path_mask,
                     int P1, int P2, uint16_t *S)
{
    if (W < 1 || H < 1 || D < 1 || (path_mask & 0xFF) == 0 || (path_mask & ~0xFF))
        return ORACLE_EINVAL;
    size_t n = (size_t)W * H * D;
    uint16_t *L = (uint16_t *)malloc(n * sizeof(uint16_t));
    uint32_t *acc = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!L || !acc) {
        free(L);
        free(acc);
        return ORACLE_ENOMEM;
    }
    int rc = ORACLE_OK;
    for (int r = 0; r < 8 && rc == ORACLE_OK; r++) {
        if (!(path_mask & (1 << r))) continue;
        rc = oracle_aggregate_path(C, W, H, D, r, P1, P2, L);
        for (size_t i = 0; i < n && rc == ORACLE_OK; i++) acc[i] += L[i];
    }
    for (size_t i = 0; i < n && rc == ORACLE_OK; i++) {
        if (acc[i] > 0xFFFFu) { rc = ORACLE_EINVAL; break; }
        S[i] = (uint16_t)acc[i];
    }
    free(L);
    free(acc);
    return rc;
}

/* Winner-takes-all on the left image, D(p) = argmin_d S(p, d), reading R4. */
int oracle_wta_left(const uint16_t *S, int W, int H, int D, uint8_t *DL)
{
    if (W < 1 || H < 1 || D < 1 || D > 255) return ORACLE_EINVAL;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const uint16_t *s = S + ((size_t)y * W + x) * D;
            int best = 0;
            for (int d = 1; d < D; d++)
                if (s[d] < s[best]) best = d;
            DL[(size_t)y * W + x] = (uint8_t)best;
        }
    return ORACLE_OK;
}

/* Right disparity from the same aggregated volume, Sec. 3.1.4, reading R5. */
int oracle_wta_right(const uint16_t *S, int W, int H, int D, uint8_t *DR)
{
    if (W < 1 || H < 1 || D < 1 || D > 255) return ORACLE_EINVAL;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int best = -1, best_s = 0;
            for (int d = 0; d < D && x + d < W; d++) {
                int s = S[((size_t)y * W + x + d) * D + d];
                if (best < 0 || s < best_s) {
                    best = d;
                    best_s = s;
                }
            }
            DR[(size_t)y * W + x] = (uint8_t)best;
        }
    return ORACLE_OK;
}

/* Left-right consistency check, Sec. 3.1.4, reading R6. */
int oracle_lr_check(const uint8_t *DL, const uint8_t *DR, int W, int H, int tol,
                    uint8_t *out)
{
    if (W < 1 || H < 1) return ORACLE_EINVAL;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int dl = DL[(size_t)y * W + x];
            uint8_t v = (uint8_t)dl;
            if (tol >= 0) {
                int xr = x - dl;
                if (xr < 0) {
                    v = 0xFF;
                } else {
                    int diff = dl - (int)DR[(size_t)y * W + xr];
                    if (diff < 0) diff = -diff;
                    if (diff > tol) v = 0xFF;
                }
            }
            out[(size_t)y * W + x] = v;
        }
    return ORACLE_OK;
}

/* k x k median filter, Sec. 3.1.5, reading R7.  The window is sorted with a
 * plain insertion sort. */
int oracle_median(const uint8_t *in, int W, int H, int k, uint8_t *out)
{
    if (W < 1 || H < 1 || k < 0 || k > 15 || (k > 1 && (k % 2) == 0))
        return ORACLE_EINVAL;
    if (k <= 1) {
        memcpy(out, in, (size_t)W * H);
        return ORACLE_OK;
    }
    int r = k / 2, n = k * k;
    uint8_t win[225];
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int cnt = 0;
            for (int wy = -r; wy <= r; wy++)
                for (int wx = -r; wx <= r; wx++) {
                    int qy = y + wy, qx = x + wx;
                    if (qy < 0) qy = 0;
                    if (qy > H - 1) qy = H - 1;
                    if (qx < 0) qx = 0;
                    if (qx > W - 1) qx = W - 1;
                    uint8_t v = in[(size_t)qy * W + qx];
                    int j = cnt++;
                    while (j > 0 && win[j - 1] > v) {
                        win[j] = win[j - 1];
                        j--;
                    }
                    win[j] = v;
                }
            out[(size_t)y * W + x] = win[(n + 1) / 2 - 1];
        }
    return ORACLE_OK;
}

/* U-map (per-column histogram, D x W) and V-map (per-row histogram, H x D),
 * Sec. 3.2, reading R8. */
int oracle_uvmap(const uint8_t *disp, int W, int H, int D, uint16_t *U,
                 uint16_t *V)
{
    if (W < 1 || H < 1 || D < 1 || D > 255 || W > 65535 || H > 65535)
        return ORACLE_EINVAL;
    memset(U, 0, (size_t)D * W * sizeof(uint16_t));
    memset(V, 0, (size_t)H * D * sizeof(uint16_t));
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int d = disp[(size_t)y * W + x];
            if (d >= D) continue;
            U[(size_t)d * W + x]++;
            V[(size_t)y * D + d]++;
        }
    return ORACLE_OK;
}

/* The whole path for one stereo pair, stage after stage.  cost_kind selects
 * the matching cost: 0 = census Hamming distance over a cw x ch window,
 * 1 = SAD over a cw x ch window (the codes outputs are then left untouched).
 * Every stage output pointer except disp may be NULL. */
int oracle_sgm(const uint8_t *left, const uint8_t *right, int W, int H,
               int pitch, int D, int cw, int ch, int cost_kind, int path_mask, int P1, int P2,
               int lr_tol, int median_k, uint64_t *codes_l, uint64_t *codes_r,
               uint16_t *S_out, uint8_t *DL_out, uint8_t *DR_out,
               uint8_t *lr_out, uint8_t *disp, uint16_t *U, uint16_t *V)
{
    if (W < 1 || H < 1 || D < 1 || D > 255 || !disp) return ORACLE_EINVAL;
    if (cost_kind != 0 && cost_kind != 1) return ORACLE_EINVAL;
    size_t npx = (size_t)W * H, nde = npx * D;
    int nbits = oracle_census_bits(cw, ch);
    uint64_t *cl = (uint64_t *)malloc(npx * sizeof(uint64_t));
    uint64_t *cr = (uint64_t *)malloc(npx * sizeof(uint64_t));
    uint16_t *C = (uint16_t *)malloc(nde * sizeof(uint16_t));
    uint16_t *S = (uint16_t *)malloc(nde * sizeof(uint16_t));
    uint8_t *DL = (uint8_t *)malloc(npx), *DR = (uint8_t *)malloc(npx);
    uint8_t *lr = (uint8_t *)malloc(npx);
    int rc = ORACLE_ENOMEM;
    if (!cl || !cr || !C || !S || !DL || !DR || !lr) goto done;
    if (cost_kind == 0) {
        rc = oracle_census(left, W, H, pitch, cw, ch, cl);
        if (rc == ORACLE_OK) rc = oracle_census(right, W, H, pitch, cw, ch, cr);
        if (rc == ORACLE_OK) rc = oracle_cost_volume(cl, cr, W, H, D, nbits, C);
    } else {
        rc = oracle_sad_cost_volume(left, right, W, H, pitch, D, cw, ch, C);
    }
    if (rc == ORACLE_OK) rc = oracle_sum_paths(C, W, H, D, path_mask, P1, P2, S);
    if (rc == ORACLE_OK) rc = oracle_wta_left(S, W, H, D, DL);
    if (rc == ORACLE_OK) rc = oracle_wta_right(S, W, H, D, DR);
    if (rc == ORACLE_OK) rc = oracle_lr_check(DL, DR, W, H, lr_tol, lr);
    if (rc == ORACLE_OK) rc = oracle_median(lr, W, H, median_k, disp);
    if (rc == ORACLE_OK && U && V) rc = oracle_uvmap(disp, W, H, D, U, V);
    if (rc == ORACLE_OK) {
        if (codes_l && cost_kind == 0) memcpy(codes_l, cl, npx * sizeof(uint64_t));
        if (codes_r && cost_kind == 0) memcpy(codes_r, cr, npx * sizeof(uint64_t));
        if (S_out) memcpy(S_out, S, nde * sizeof(uint16_t));
        if (DL_out) memcpy(DL_out, DL, npx);
        if (DR_out) memcpy(DR_out, DR, npx);
        if (lr_out) memcpy(lr_out, lr, npx);
    }
done:
    free(cl);
    free(cr);
    free(C);
    free(S);
    free(DL);
    free(DR);
    free(lr);
    return rc;
}

/* U-/V-map post-processing of Sec. 3.2, reading R11.  map is rows x cols
 * uint16 (row-major); out is rows x cols uint8.  Threshold, region of
 * interest, dilation, Gaussian, in that order. */
int oracle_uv_post(const uint16_t *map, int rows, int cols, int threshold, int r0, int r1,
                   int c0, int c1, int dilate_r, uint8_t *out)
{
    if (rows < 1 || cols < 1 || threshold < 0 || dilate_r < 0 || dilate_r > 7) return ORACLE_EINVAL;
    size_t n = (size_t)rows * cols;
    uint8_t *bin = (uint8_t *)malloc(n), *dil = (uint8_t *)malloc(n);
    if (!bin || !dil) {
        free(bin);
        free(dil);
        return ORACLE_ENOMEM;
    }
    for (int i = 0; i < rows; i++)
        for (int j = 0; j < cols; j++) {
            int inside = i >= r0 && i < r1 && j >= c0 && j < c1;
            bin[(size_t)i * cols + j] = (uint8_t)(inside && map[(size_t)i * cols + j] >= threshold);
        }
    for (int i = 0; i < rows; i++)
        for (int j = 0; j < cols; j++) {
            int v = 0;
            for (int u = -dilate_r; u <= dilate_r; u++)
                for (int w = -dilate_r; w <= dilate_r; w++) {
                    int ii = i + u, jj = j + w;
                    if (ii >= 0 && ii < rows && jj >= 0 && jj < cols && bin[(size_t)ii * cols + jj]) v = 1;
                }
            dil[(size_t)i * cols + j] = (uint8_t)v;
        }
    static const int k[3] = {1, 2, 1};
    for (int i = 0; i < rows; i++)
        for (int j = 0; j < cols; j++) {
            int acc = 0;
            for (int u = -1; u <= 1; u++)
                for (int w = -1; w <= 1; w++) {
                    int ii = i + u, jj = j + w;
                    if (ii >= 0 && ii < rows && jj >= 0 && jj < cols)
                        acc += k[u + 1] * k[w + 1] * 255 * dil[(size_t)ii * cols + jj];
                }
            out[(size_t)i * cols + j] = (uint8_t)((acc + 8) / 16);
        }
    free(bin);
    free(dil);
    return ORACLE_OK;
}

/* Rectification, Sec. 3.1.1: I_rect(x, y) = I(M_x(x, y), M_y(x, y)) with
 * integer maps of the rectified image's size (reading R12). */
int oracle_rectify(const uint8_t *img, int W, int H, int pitch, const uint16_t *mx,
                   const uint16_t *my, uint8_t *out)
{
    if (W < 1 || H < 1 || pitch < W) return ORACLE_EINVAL;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int sx = mx[(size_t)y * W + x], sy = my[(size_t)y * W + x];
            out[(size_t)y * W + x] = (sx < W && sy < H) ? img[(size_t)sy * pitch + sx] : 0;
        }
    return ORACLE_OK;
}
