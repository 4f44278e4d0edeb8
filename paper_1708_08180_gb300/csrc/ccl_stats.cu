// ccl_stats.cu -- per-component statistics of a canonical label image
// (pixel count, bounding box, coordinate sums): the size and location of each
// region that the paper's motivating uses need (§I).
//
// A component's root is the one pixel whose label is 1 + its own raster
// index.  The steps:
//   1. count the roots of every row segment (row y, 256-column tile tx);
//   2. exclusive prefix sums of the counts (three small kernels): the rank of
//      the first root of each row segment in raster order, i.e. in label order;
//   3. write every root's raster index at its rank (the sorted root list) and
//      initialise its accumulators (one array per field);
//   4. every 256 x 64 tile sums its pixels per label in a shared-memory hash
//      table (each thread first merges the runs of equal labels down its
//      column), then adds each label's sums into the accumulators of its
//      component, found by a binary search of the root list of the row
//      segment that holds the label's root;
//   5. pack the accumulators into the records.
#include <algorithm>
#include <climits>

#include "ccl_internal.h"

namespace ccl {
namespace {

constexpr int kSTW = 256;           // tile width (one column per thread)
constexpr int kSTH = 64;            // tile height
constexpr int kHash = 1024;         // per-tile hash table entries (power of two)
constexpr int kScanPer = 16;        // prefix sums: counts per thread
constexpr int kScanBlock = kSTW * kScanPer;   // and per block

// per-component accumulators, one array per field (max_comps entries each):
// the updates of a component that spans many tiles then spread over seven
// cache lines instead of queueing on one
struct Acc {
    int *count, *xmin, *ymin, *xmax, *ymax;
    unsigned long long *sx, *sy;
};

struct StatsGeom {
    int H, W, tiles_x, tiles_y;
    long long nseg;   // row segments: H * tiles_x
};

StatsGeom stats_geom(int H, int W) {
    StatsGeom s;
    s.H = H;
    s.W = W;
    s.tiles_x = (W + kSTW - 1) / kSTW;
    s.tiles_y = (H + kSTH - 1) / kSTH;
    s.nseg = (long long)H * s.tiles_x;
    return s;
}

// most components an image can hold: a 4-connected checkerboard's
long long max_roots(int H, int W) { return ((long long)H * W + 1) / 2 + 1; }

size_t align256(size_t v) { return (v + 255u) & ~(size_t)255u; }

size_t counts_bytes(const StatsGeom &s) { return align256((size_t)(s.nseg + 1) * 4u); }

// block sums of the prefix-sum step: one per kScanBlock counts
size_t bsum_bytes(const StatsGeom &s) {
    return align256((size_t)((s.nseg + kScanBlock - 1) / kScanBlock + 1) * 4u);
}

// 1: roots per row segment.  A warp takes one row of the tile at a time, its
// lanes reading 32 consecutive columns per step (8 steps per 256 columns).
__global__ void __launch_bounds__(kSTW) k_st_count(const int32_t *__restrict__ labels,
                                                   StatsGeom s, int *cnt) {
    const int tx = blockIdx.x % s.tiles_x, ty = blockIdx.x / s.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ly = warp; ly < kSTH; ly += kSTW / 32) {
        const int y = ty * kSTH + ly;
        if (y >= s.H) break;   // warp-uniform
        int c = 0;
#pragma unroll
        for (int k = 0; k < kSTW / 32; ++k) {
            const int x = tx * kSTW + 32 * k + lane;
            const long long p = (long long)y * s.W + x;
            const bool root = x < s.W && __ldg(labels + p) == (int32_t)(p + 1);
            c += __popc(__ballot_sync(0xFFFFFFFFu, root));
        }
        if (lane == 0) cnt[(long long)y * s.tiles_x + tx] = c;
    }
}

// 2: exclusive prefix sums over the n counts, in three steps: every block of
// kScanBlock counts is summed (2a), one block scans those sums (2b), and every
// block rescans its counts from its offset (2c).  cnt[n] and *ncomps receive
// the total.

__device__ __forceinline__ int block_scan_excl(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kSTW / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int d = 1; d < kSTW / 32; d <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < kSTW / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    total = warp_sums[kSTW / 32 - 1];
    const int r = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
    __syncthreads();   // warp_sums may be reused right away
    return r;
}

__global__ void __launch_bounds__(kSTW) k_st_scan_sums(const int *cnt, long long n, int *bsum) {
    __shared__ int warp_sums[kSTW / 32];
    const long long b0 = (long long)blockIdx.x * kScanBlock;
    int v = 0;
    for (int k = 0; k < kScanPer; ++k) {   // coalesced: thread t reads b0 + k * kSTW + t
        const long long i = b0 + (long long)k * kSTW + threadIdx.x;
        if (i < n) v += cnt[i];
    }
    int total;
    block_scan_excl(v, warp_sums, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kSTW) k_st_scan_top(int *bsum, int nb, int *cnt, long long n,
                                                      int32_t *ncomps) {
    __shared__ int warp_sums[kSTW / 32];
    int carry = 0;
    for (int c0 = 0; c0 < nb; c0 += kSTW) {   // block-uniform
        const int i = c0 + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int total;
        const int e = block_scan_excl(v, warp_sums, total);
        if (i < nb) bsum[i] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) {
        cnt[n] = carry;
        *ncomps = (int32_t)carry;
    }
}

__global__ void __launch_bounds__(kSTW) k_st_scan_apply(int *cnt, long long n, const int *bsum) {
    __shared__ int warp_sums[kSTW / 32];
    // thread t rescans counts b0 + t * kScanPer ... + kScanPer - 1
    const long long i0 = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanPer;
    int v[kScanPer];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = i0 + k < n ? cnt[i0 + k] : 0;
        sum += v[k];
    }
    int total;
    int run = bsum[blockIdx.x] + block_scan_excl(sum, warp_sums, total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (i0 + k < n) cnt[i0 + k] = run;
        run += v[k];
    }
}

// 3: the sorted root list, and the accumulators of the first max_comps components
// (same walk as step 1; a root's rank is its row segment's offset plus the
// roots before it in the segment)
__global__ void __launch_bounds__(kSTW) k_st_roots(const int32_t *__restrict__ labels,
                                                   StatsGeom s, const int *base, int *roots,
                                                   long long nroots, Acc acc, int max_comps) {
    const int tx = blockIdx.x % s.tiles_x, ty = blockIdx.x / s.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ly = warp; ly < kSTH; ly += kSTW / 32) {
        const int y = ty * kSTH + ly;
        if (y >= s.H) break;   // warp-uniform
        unsigned bm[kSTW / 32];   // roots of each 32-column step, loaded first
#pragma unroll
        for (int k = 0; k < kSTW / 32; ++k) {
            const int x = tx * kSTW + 32 * k + lane;
            const long long p = (long long)y * s.W + x;
            bm[k] = __ballot_sync(0xFFFFFFFFu, x < s.W && __ldg(labels + p) == (int32_t)(p + 1));
        }
        long long off = base[(long long)y * s.tiles_x + tx];
#pragma unroll
        for (int k = 0; k < kSTW / 32; ++k) {
            const int x = tx * kSTW + 32 * k + lane;
            const long long p = (long long)y * s.W + x;
            const unsigned b = bm[k];
            const bool root = (b >> lane) & 1u;
            if (root) {
                const long long slot = off + __popc(b & ((1u << lane) - 1u));
                if (slot < nroots) roots[slot] = (int)p;
                if (slot < max_comps) {
                    acc.count[slot] = 0;
                    acc.xmin[slot] = INT_MAX;
                    acc.ymin[slot] = INT_MAX;
                    acc.xmax[slot] = -1;
                    acc.ymax[slot] = -1;
                    acc.sx[slot] = 0;
                    acc.sy[slot] = 0;
                }
            }
            off += __popc(b);
        }
    }
}

// rank of root p in the sorted root list (-1 if p is not a root)
__device__ __forceinline__ long long root_rank(const StatsGeom &s, const int *base,
                                               const int *roots, long long nroots, long long p) {
    const long long y = p / s.W, tx = (p % s.W) / kSTW;
    long long lo = base[y * s.tiles_x + tx], hi = base[y * s.tiles_x + tx + 1];
    if (hi > nroots) hi = nroots;   // only for an input that is not canonical
    while (lo < hi) {   // at most log2(kSTW) + 1 steps
        const long long mid = (lo + hi) >> 1;
        const int v = roots[mid];
        if (v == p) return mid;
        if (v < p) lo = mid + 1; else hi = mid;
    }
    return -1;
}

struct Partial {
    int label, count, xmin, ymin, xmax, ymax;
    long long sx, sy;
};

__device__ __forceinline__ void add_global(const StatsGeom &s, const int *base, const int *roots,
                                           long long nroots, const Acc &acc, int max_comps,
                                           const Partial &q) {
    if (q.label < 1 || (long long)q.label > (long long)s.H * s.W) return;   // not canonical
    const long long r = root_rank(s, base, roots, nroots, (long long)q.label - 1);
    if (r < 0 || r >= max_comps) return;
    atomicAdd(acc.count + r, q.count);
    atomicMin(acc.xmin + r, q.xmin);
    atomicMin(acc.ymin + r, q.ymin);
    atomicMax(acc.xmax + r, q.xmax);
    atomicMax(acc.ymax + r, q.ymax);
    atomicAdd(acc.sx + r, (unsigned long long)q.sx);
    atomicAdd(acc.sy + r, (unsigned long long)q.sy);
}

struct SmemHash {
    int key[kHash];   // 0 = empty
    int count[kHash], xmin[kHash], ymin[kHash], xmax[kHash], ymax[kHash];
    unsigned long long sx[kHash], sy[kHash];
};

// 4: per-tile sums, then one update per component and tile
__global__ void __launch_bounds__(kSTW) k_st_acc(const int32_t *__restrict__ labels, StatsGeom s,
                                                 const int *base, const int *roots, long long nroots,
                                                 Acc acc, int max_comps) {
    __shared__ SmemHash h;
    for (int i = threadIdx.x; i < kHash; i += kSTW) {
        h.key[i] = 0;
        h.count[i] = 0;
        h.xmin[i] = INT_MAX;
        h.ymin[i] = INT_MAX;
        h.xmax[i] = -1;
        h.ymax[i] = -1;
        h.sx[i] = 0;
        h.sy[i] = 0;
    }
    __syncthreads();
    const int tx = blockIdx.x % s.tiles_x, ty = blockIdx.x / s.tiles_x;
    const int x = tx * kSTW + threadIdx.x;
    auto flush = [&](const Partial &q) {
        unsigned hh = ((unsigned)q.label * 2654435761u) & (kHash - 1);
        for (int probe = 0; probe < kHash; ++probe, hh = (hh + 1) & (kHash - 1)) {
            const int k = atomicCAS(&h.key[hh], 0, q.label);
            if (k == 0 || k == q.label) {
                atomicAdd(&h.count[hh], q.count);
                atomicMin(&h.xmin[hh], q.xmin);
                atomicMin(&h.ymin[hh], q.ymin);
                atomicMax(&h.xmax[hh], q.xmax);
                atomicMax(&h.ymax[hh], q.ymax);
                atomicAdd(&h.sx[hh], (unsigned long long)q.sx);
                atomicAdd(&h.sy[hh], (unsigned long long)q.sy);
                return;
            }
        }
        add_global(s, base, roots, nroots, acc, max_comps, q);   // table full
    };
    Partial run;   // the current run of equal labels down this thread's column
    run.label = 0;
    if (x < s.W) {
        constexpr int kChunk = 16;   // labels loaded ahead, independent of the flushes
        for (int c0 = 0; c0 < kSTH; c0 += kChunk) {
            int Ls[kChunk];
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                const int y = ty * kSTH + c0 + k;
                Ls[k] = y < s.H ? __ldg(labels + (long long)y * s.W + x) : 0;
            }
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                const int L = Ls[k];
                if (L == 0) continue;
                const int y = ty * kSTH + c0 + k;
                if (L != run.label) {
                    if (run.label != 0) flush(run);
                    run.label = L;
                    run.count = 0;
                    run.xmin = run.xmax = x;
                    run.ymin = y;
                    run.sx = 0;
                    run.sy = 0;
                }
                run.count += 1;
                run.ymax = y;
                run.sx += x;
                run.sy += y;
            }
        }
        if (run.label != 0) flush(run);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHash; i += kSTW) {
        if (h.key[i] == 0) continue;
        Partial q;
        q.label = h.key[i];
        q.count = h.count[i];
        q.xmin = h.xmin[i];
        q.ymin = h.ymin[i];
        q.xmax = h.xmax[i];
        q.ymax = h.ymax[i];
        q.sx = (long long)h.sx[i];
        q.sy = (long long)h.sy[i];
        add_global(s, base, roots, nroots, acc, max_comps, q);
    }
}

// 5: the records of the first min(components, max_comps) components
__global__ void __launch_bounds__(kSTW) k_st_pack(const int *roots, long long nroots, Acc acc,
                                                  const int32_t *ncomps, ccl_component *comps,
                                                  int max_comps) {
    const long long n = min(min((long long)*ncomps, (long long)max_comps), nroots);
    for (long long i = (long long)blockIdx.x * kSTW + threadIdx.x; i < n;
         i += (long long)gridDim.x * kSTW) {
        ccl_component c;
        c.label = roots[i] + 1;
        c.count = acc.count[i];
        c.xmin = acc.xmin[i];
        c.ymin = acc.ymin[i];
        c.xmax = acc.xmax[i];
        c.ymax = acc.ymax[i];
        c.sum_x = (int64_t)acc.sx[i];
        c.sum_y = (int64_t)acc.sy[i];
        comps[i] = c;
    }
}

size_t acc_bytes(int max_comps) {
    return 5 * align256((size_t)max_comps * 4u) + 2 * align256((size_t)max_comps * 8u);
}

Acc acc_layout(char *base, int max_comps) {
    Acc a;
    const size_t i4 = align256((size_t)max_comps * 4u), i8 = align256((size_t)max_comps * 8u);
    a.count = reinterpret_cast<int *>(base);
    a.xmin = reinterpret_cast<int *>(base + i4);
    a.ymin = reinterpret_cast<int *>(base + 2 * i4);
    a.xmax = reinterpret_cast<int *>(base + 3 * i4);
    a.ymax = reinterpret_cast<int *>(base + 4 * i4);
    a.sx = reinterpret_cast<unsigned long long *>(base + 5 * i4);
    a.sy = reinterpret_cast<unsigned long long *>(base + 5 * i4 + i8);
    return a;
}

}  // namespace
}  // namespace ccl

extern "C" size_t ccl_stats_workspace_bytes(int height, int width, int max_comps) {
    if (!ccl::valid_image_dims(height, width) || max_comps < 0) return 0;
    const ccl::StatsGeom s = ccl::stats_geom(height, width);
    return ccl::counts_bytes(s) + ccl::bsum_bytes(s) +
           ccl::align256((size_t)ccl::max_roots(height, width) * 4u) + ccl::acc_bytes(max_comps);
}

extern "C" ccl_status ccl_component_stats(const int32_t *d_labels, int height, int width,
                                          ccl_component *d_comps, int max_comps, int32_t *d_ncomps,
                                          void *d_ws, size_t ws_bytes, ccl_stream stream) {
    if (!d_labels || !d_ncomps || !ccl::valid_image_dims(height, width) || max_comps < 0 ||
        (max_comps > 0 && !d_comps))
        return CCL_ERR_INVALID_ARG;
    const size_t need = ccl_stats_workspace_bytes(height, width, max_comps);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ccl_status st = CCL_OK;
    if (!d_ws) {
        d_ws = ccl::library_workspace(s, need, &st);
        if (st != CCL_OK) return st;
    } else if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        return CCL_ERR_INVALID_ARG;
    }
    const ccl::StatsGeom g = ccl::stats_geom(height, width);
    char *w = static_cast<char *>(d_ws);
    int *cnt = reinterpret_cast<int *>(w);
    w += ccl::counts_bytes(g);
    int *bsum = reinterpret_cast<int *>(w);
    w += ccl::bsum_bytes(g);
    int *roots = reinterpret_cast<int *>(w);
    const long long nroots = ccl::max_roots(height, width);
    w += ccl::align256((size_t)nroots * 4u);
    const ccl::Acc acc = ccl::acc_layout(w, max_comps);
    const unsigned tiles = (unsigned)((long long)g.tiles_x * g.tiles_y);
    const long long nb = (g.nseg + ccl::kScanBlock - 1) / ccl::kScanBlock;
    ccl::k_st_count<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt);
    ccl::k_st_scan_sums<<<(unsigned)nb, ccl::kSTW, 0, s>>>(cnt, g.nseg, bsum);
    ccl::k_st_scan_top<<<1, ccl::kSTW, 0, s>>>(bsum, (int)nb, cnt, g.nseg, d_ncomps);
    ccl::k_st_scan_apply<<<(unsigned)nb, ccl::kSTW, 0, s>>>(cnt, g.nseg, bsum);
    ccl::k_st_roots<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt, roots, nroots, acc, max_comps);
    ccl::k_st_acc<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt, roots, nroots, acc, max_comps);
    if (max_comps > 0) {
        const unsigned pb = (unsigned)std::min<long long>(((long long)max_comps + ccl::kSTW - 1) / ccl::kSTW,
                                                          65535);
        ccl::k_st_pack<<<pb, ccl::kSTW, 0, s>>>(roots, nroots, acc, d_ncomps, d_comps, max_comps);
    }
    if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}
