/*
 * CPU oracle for connected-components labelling (CCL) of a 2-D binary image.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct ground
 * truth that the GPU path is compared against.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, calls or includes anything from here, and nothing here is
 * shared with the GPU path.
 *
 * What it computes (the plain definition the paper's union-find reaches):
 *   The paper gives every connected region of the grid one unique ID (§I), and
 *   its union-find links the larger root under the smaller one with atomicMin
 *   (§II-A-3, "findAndUnion"), with IDs that are global raster indices
 *   x + y*imgWidth (Kernel 1, local-to-global ID conversion; the Link kernel of
 *   §II-C).  So the root of every component is its smallest raster index.
 *   With F = { i : img[i] != 0 } and the 4- or 8-neighbour graph on F,
 *       out[i] = 0                          if img[i] == 0
 *       out[i] = 1 + min{ j in C(i) }       otherwise,
 *   where C(i) is the component of i and i = y*W + x (0-based).  The "+1, 0 for
 *   background" encoding is this library's convention on top of the paper's
 *   raster-index IDs.
 *
 * Algorithm: scan pixels in raster order; the first unlabelled foreground pixel
 * met is the smallest index of its component, so a breadth-first flood fill
 * from it (explicit FIFO queue) assigns 1 + that index to the whole component.
 * No union-find, no tiling, no minimum reduction.
 *
 * 4-connectivity: Manhattan distance 1 (the connectivity Kernel 1 is written
 * for, §II-A).  8-connectivity: Chebyshev distance 1 (the paper does not treat
 * it; this is the standard definition).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 3

/* Label one image.  img: h*w bytes row-major, nonzero = foreground.
 * out: h*w int32 row-major, written completely.  Returns 0 on success. */
int ccl_oracle_bfs(const uint8_t *img, int32_t *out, int64_t h, int64_t w,
                   int conn)
{
    static const int dx4[4] = {1, -1, 0, 0};
    static const int dy4[4] = {0, 0, 1, -1};
    static const int dx8[8] = {1, -1, 0, 0, 1, 1, -1, -1};
    static const int dy8[8] = {0, 0, 1, -1, 1, -1, 1, -1};
    const int *dx, *dy;
    int nn;
    int64_t n, i, head, tail;
    int32_t *queue;

    if (img == NULL || out == NULL || h < 1 || w < 1)
        return ORACLE_EINVAL;
    if (conn != 4 && conn != 8)
        return ORACLE_EINVAL;
    n = h * w;
    if (n > (int64_t)2147483646)
        return ORACLE_EINVAL;
    if (conn == 4) {
        dx = dx4; dy = dy4; nn = 4;
    } else {
        dx = dx8; dy = dy8; nn = 8;
    }

    memset(out, 0, (size_t)n * sizeof(int32_t));
    queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (queue == NULL)
        return ORACLE_ENOMEM;

    for (i = 0; i < n; ++i) {
        int32_t label;
        if (img[i] == 0 || out[i] != 0)
            continue;
        /* i is the first pixel of its component met in raster order, hence
         * the smallest raster index in that component. */
        label = (int32_t)(i + 1);
        out[i] = label;
        head = 0;
        tail = 0;
        queue[tail++] = (int32_t)i;
        while (head < tail) {
            int32_t p = queue[head++];
            int64_t py = p / w, px = p % w;
            int k;
            for (k = 0; k < nn; ++k) {
                int64_t qx = px + dx[k], qy = py + dy[k], q;
                if (qx < 0 || qx >= w || qy < 0 || qy >= h)
                    continue;
                q = qy * w + qx;
                if (img[q] == 0 || out[q] != 0)
                    continue;
                out[q] = label;
                queue[tail++] = (int32_t)q;
            }
        }
    }
    free(queue);
    return ORACLE_OK;
}

/* Label `count` images of identical size h*w stored back to back (used to
 * sweep every tiny image exhaustively without one foreign call per image). */
int ccl_oracle_bfs_many(const uint8_t *imgs, int32_t *outs, int64_t count,
                        int64_t h, int64_t w, int conn)
{
    int64_t k;
    for (k = 0; k < count; ++k) {
        int rc = ccl_oracle_bfs(imgs + k * h * w, outs + k * h * w, h, w, conn);
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}

/*
 * Volumes (the "2D/3D grid" the paper's introduction names, §I): the same
 * definition one dimension up.  vol: d*h*w bytes, index i = (z*h + y)*w + x,
 * nonzero = foreground; out[i] = 0 for background, else 1 + the smallest index
 * of i's component.  Connectivity: 6 (face neighbours, |dx|+|dy|+|dz| = 1),
 * 18 (faces and edges, |dx|+|dy|+|dz| <= 2) or 26 (max(|dx|,|dy|,|dz|) = 1).
 * Same algorithm: raster scan, breadth-first flood fill from the first
 * unlabelled foreground voxel.
 */
int ccl_oracle_bfs3d(const uint8_t *vol, int32_t *out, int64_t d, int64_t h,
                     int64_t w, int conn)
{
    int off[26][3];
    int nn = 0, a, b, c;
    int64_t n, i, head, tail;
    int32_t *queue;

    if (vol == NULL || out == NULL || d < 1 || h < 1 || w < 1)
        return ORACLE_EINVAL;
    if (conn != 6 && conn != 18 && conn != 26)
        return ORACLE_EINVAL;
    if (d > (int64_t)2147483646 / h || d * h > (int64_t)2147483646 / w)
        return ORACLE_EINVAL;
    n = d * h * w;
    for (c = -1; c <= 1; ++c)
        for (b = -1; b <= 1; ++b)
            for (a = -1; a <= 1; ++a) {
                int s = abs(a) + abs(b) + abs(c);
                if (s == 0 || (conn == 6 && s > 1) || (conn == 18 && s > 2))
                    continue;
                off[nn][0] = a;
                off[nn][1] = b;
                off[nn][2] = c;
                ++nn;
            }

    memset(out, 0, (size_t)n * sizeof(int32_t));
    queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (queue == NULL)
        return ORACLE_ENOMEM;

    for (i = 0; i < n; ++i) {
        int32_t label;
        if (vol[i] == 0 || out[i] != 0)
            continue;
        label = (int32_t)(i + 1);
        out[i] = label;
        head = 0;
        tail = 0;
        queue[tail++] = (int32_t)i;
        while (head < tail) {
            int32_t p = queue[head++];
            int64_t px = p % w, py = (p / w) % h, pz = p / (w * h);
            int k;
            for (k = 0; k < nn; ++k) {
                int64_t qx = px + off[k][0], qy = py + off[k][1], qz = pz + off[k][2], q;
                if (qx < 0 || qx >= w || qy < 0 || qy >= h || qz < 0 || qz >= d)
                    continue;
                q = (qz * h + qy) * w + qx;
                if (vol[q] == 0 || out[q] != 0)
                    continue;
                out[q] = label;
                queue[tail++] = (int32_t)q;
            }
        }
    }
    free(queue);
    return ORACLE_OK;
}
