/*
 * Overlapping domain decomposition for the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Section 2.1: each subdomain is made of *complete* scan frames, so the frame
 * stack splits into disjoint groups and every group's windows lie inside its
 * subdomain; the overlap of two adjacent subdomains is then (probe side -
 * step) for a raster scan.  Section 3.1 generalises to D subdomains with the
 * pair set N~ = {(i1, i2): Omega_i1 and Omega_i2 intersect}.
 *
 * The paper does not say how frames are grouped for a 2-D grid of subdomains
 * or how a requested overlap width enters.  Reading used here:
 *   1. the image is cut into sub_rows x sub_cols core tiles with boundaries
 *      floor(k*H/sub_rows) and floor(k*W/sub_cols) (half-open);
 *   2. frame j belongs to the core tile containing its window centre
 *      offs[j] + (m-1)/2 (compared in doubled integer coordinates);
 *   3. Omega_d is the bounding box of its core tile, grown by
 *      ceil(overlap_px/2) on interior sides and clipped to the image, and of
 *      the windows of its frames.  overlap_px is therefore a minimum width.
 * With overlap_px = 0 and a raster scan this reproduces the paper's
 * partitions (e.g. 13x25 / 12x25 frames with a 56-pixel overlap in section 4.1).
 *
 * Periodic variant (section 4 names periodic boundaries as the usual
 * alternative to its vacuum boundary; it does not decompose a periodic image,
 * so this is a reading): the image is a torus, window j covers the pixels
 * ((offs[j] + a) mod H, (offs[j] + b) mod W), 0 <= offs < (H, W).  Rectangles
 * live in extended coordinates, where pixel (R, C) is the image pixel
 * (R mod H, C mod W):
 *   1. the same core tiles, grown by ceil(overlap_px/2) on every side (every
 *      side of a tile has a neighbour on the torus) and not clipped;
 *   2. frame j is placed at the copy of its offset whose doubled centre
 *      2 o + m - 1 lies in [0, 2H) x [0, 2W) (o - H where it would not) and
 *      joins the core tile holding that centre;
 *   3. Omega_d is the bounding box of the grown tile and of its frames'
 *      windows at their placed offsets (roffs).
 * Pairs: every (d, e, s) with s in {-2, ..., 2}^2 such that Omega_d and Omega_e
 * shifted by (s_r H, s_c W) intersect, except d = e with s = 0 -- a subdomain
 * that reaches around the torus meets a copy of itself.  The intersection is
 * kept in d's coordinates; (e, d, -s) is the same region seen from e.
 */
#include "od2p_oracle.h"

#include <stddef.h>

int orc_geometry_ext(int H, int W, int m, int J, const int32_t *offs, int sub_rows, int sub_cols,
                     int overlap_px, int periodic, int32_t *frame_sub, int32_t *rect, int32_t *roffs)
{
    if (H < m || W < m || m < 1 || J < 0 || sub_rows < 1 || sub_cols < 1 || sub_rows > H ||
        sub_cols > W || overlap_px < 0)
        return -1;
    for (int j = 0; j < J; ++j) {
        int r = offs[2 * j], c = offs[2 * j + 1];
        if (periodic ? (r < 0 || c < 0 || r >= H || c >= W) : (r < 0 || c < 0 || r > H - m || c > W - m))
            return -2;
    }
    const int D = sub_rows * sub_cols;
    const int half = (overlap_px + 1) / 2;
    for (int a = 0; a < sub_rows; ++a)
        for (int b = 0; b < sub_cols; ++b) {
            int d = a * sub_cols + b;
            int r0 = (int)(((long)a * H) / sub_rows), r1 = (int)(((long)(a + 1) * H) / sub_rows);
            int c0 = (int)(((long)b * W) / sub_cols), c1 = (int)(((long)(b + 1) * W) / sub_cols);
            if (periodic || a > 0) r0 -= half;
            if (periodic || a < sub_rows - 1) r1 += half;
            if (periodic || b > 0) c0 -= half;
            if (periodic || b < sub_cols - 1) c1 += half;
            if (!periodic) {
                if (r0 < 0) r0 = 0;
                if (c0 < 0) c0 = 0;
                if (r1 > H) r1 = H;
                if (c1 > W) c1 = W;
            }
            rect[4 * d + 0] = r0;
            rect[4 * d + 1] = c0;
            rect[4 * d + 2] = r1;
            rect[4 * d + 3] = c1;
        }
    for (int j = 0; j < J; ++j) {
        int r0 = offs[2 * j], c0 = offs[2 * j + 1];
        if (periodic) { /* the copy of the window whose centre lies on the image */
            if (2L * r0 + m - 1 >= 2L * H) r0 -= H;
            if (2L * c0 + m - 1 >= 2L * W) c0 -= W;
        }
        long cr2 = 2L * r0 + m - 1, cc2 = 2L * c0 + m - 1;
        int a = 0, b = 0;
        while (a + 1 < sub_rows && 2L * (((long)(a + 1) * H) / sub_rows) <= cr2) ++a;
        while (b + 1 < sub_cols && 2L * (((long)(b + 1) * W) / sub_cols) <= cc2) ++b;
        int d = a * sub_cols + b;
        frame_sub[j] = d;
        if (roffs) {
            roffs[2 * j] = r0;
            roffs[2 * j + 1] = c0;
        }
        if (r0 < rect[4 * d + 0]) rect[4 * d + 0] = r0;
        if (c0 < rect[4 * d + 1]) rect[4 * d + 1] = c0;
        if (r0 + m > rect[4 * d + 2]) rect[4 * d + 2] = r0 + m;
        if (c0 + m > rect[4 * d + 3]) rect[4 * d + 3] = c0 + m;
    }
    if (periodic) /* rectangles inside (-H, 2H) x (-W, 2W): shifts of up to two periods reach every copy */
        for (int d = 0; d < D; ++d)
            if (rect[4 * d] <= -H || rect[4 * d + 2] >= 2 * H || rect[4 * d + 1] <= -W || rect[4 * d + 3] >= 2 * W)
                return -3;
    return D;
}

int orc_geometry(int H, int W, int m, int J, const int32_t *offs, int sub_rows,
                 int sub_cols, int overlap_px, int32_t *frame_sub, int32_t *rect)
{
    return orc_geometry_ext(H, W, m, J, offs, sub_rows, sub_cols, overlap_px, 0, frame_sub, rect, NULL);
}

int orc_pairs_ext(int D, const int32_t *rect, int H, int W, int periodic, int max_pairs, int32_t *pair,
                  int32_t *pair_shift, int32_t *pair_rect)
{
    int n = 0;
    const int smax = periodic ? 2 : 0;
    for (int d = 0; d < D; ++d)
        for (int e = 0; e < D; ++e)
            for (int sr = -smax; sr <= smax; ++sr)
                for (int sc = -smax; sc <= smax; ++sc) {
                    if (d == e && sr == 0 && sc == 0) continue;
                    const int32_t *a = rect + 4 * d, *b = rect + 4 * e;
                    /* Omega_e shifted by (sr H, sc W), intersected with Omega_d */
                    int b0 = b[0] + sr * H, b1 = b[1] + sc * W, b2 = b[2] + sr * H, b3 = b[3] + sc * W;
                    int r0 = a[0] > b0 ? a[0] : b0, c0 = a[1] > b1 ? a[1] : b1;
                    int r1 = a[2] < b2 ? a[2] : b2, c1 = a[3] < b3 ? a[3] : b3;
                    if (r0 >= r1 || c0 >= c1) continue;
                    if (n < max_pairs) {
                        pair[2 * n] = d;
                        pair[2 * n + 1] = e;
                        if (pair_shift) {
                            pair_shift[2 * n] = sr;
                            pair_shift[2 * n + 1] = sc;
                        }
                        pair_rect[4 * n + 0] = r0;
                        pair_rect[4 * n + 1] = c0;
                        pair_rect[4 * n + 2] = r1;
                        pair_rect[4 * n + 3] = c1;
                    }
                    ++n;
                }
    return n;
}

int orc_pairs(int D, const int32_t *rect, int max_pairs, int32_t *pair, int32_t *pair_rect)
{
    return orc_pairs_ext(D, rect, 0, 0, 0, max_pairs, pair, NULL, pair_rect);
}
