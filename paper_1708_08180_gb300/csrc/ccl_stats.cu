// ccl_stats.cu -- per-component statistics of a canonical label image
// (pixel count, bounding box, coordinate sums): the size and location of each
// region that the paper's motivating uses need (§I).
//
// A component's root is the one pixel whose label is 1 + its own raster
// index.  Four kernels:
//   1. count the roots of every row segment (row y, 256-column tile tx);
//   2. one block turns the counts into exclusive prefix sums: the rank of the
//      first root of each row segment in raster order, i.e. in label order;
//   3. write every root's raster index at its rank (the sorted root list) and
//      initialise its record;
//   4. every 256 x 64 tile sums its pixels per label in a shared-memory hash
//      table (each thread first merges the runs of equal labels down its
//      column), then adds each label's sums into the record of its component,
//      found by a binary search of the root list of the row segment that
//      holds the label's root.
#include <climits>

#include "ccl_internal.h"

namespace ccl {
namespace {

constexpr int kSTW = 256;           // tile width (one column per thread)
constexpr int kSTH = 64;            // tile height
constexpr int kHash = 1024;         // per-tile hash table entries (power of two)
constexpr int kScanThreads = 1024;

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

// 1: roots per row segment
__global__ void __launch_bounds__(kSTW) k_st_count(const int32_t *__restrict__ labels,
                                                   StatsGeom s, int *cnt) {
    __shared__ int warp_cnt[kSTW / 32];
    const int tx = blockIdx.x % s.tiles_x, ty = blockIdx.x / s.tiles_x;
    const int x = tx * kSTW + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ly = 0; ly < kSTH; ++ly) {
        const int y = ty * kSTH + ly;
        if (y >= s.H) break;   // block-uniform
        bool root = false;
        if (x < s.W) {
            const long long p = (long long)y * s.W + x;
            root = __ldg(labels + p) == (int32_t)(p + 1);
        }
        const unsigned b = __ballot_sync(0xFFFFFFFFu, root);
        if (lane == 0) warp_cnt[warp] = __popc(b);
        __syncthreads();
        if (threadIdx.x == 0) {
            int c = 0;
            for (int k = 0; k < kSTW / 32; ++k) c += warp_cnt[k];
            cnt[(long long)y * s.tiles_x + tx] = c;
        }
        __syncthreads();
    }
}

// 2: exclusive prefix sums over the n counts (one block); cnt[n] and *ncomps
// receive the total
__global__ void __launch_bounds__(kScanThreads) k_st_scan(int *cnt, long long n, int32_t *ncomps) {
    __shared__ long long part[kScanThreads];
    const long long per = (n + kScanThreads - 1) / kScanThreads;
    const long long lo = threadIdx.x * per;
    const long long hi = lo + per < n ? lo + per : n;
    long long sum = 0;
    for (long long i = lo; i < hi; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < kScanThreads; d <<= 1) {   // Hillis-Steele inclusive scan
        const long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;   // exclusive prefix of this thread's range
    for (long long i = lo; i < hi; ++i) {
        const int c = cnt[i];
        cnt[i] = (int)run;
        run += c;
    }
    if (threadIdx.x == kScanThreads - 1) {
        cnt[n] = (int)part[kScanThreads - 1];
        *ncomps = (int32_t)part[kScanThreads - 1];
    }
}

// 3: the sorted root list, and the records of the first max_comps components
__global__ void __launch_bounds__(kSTW) k_st_roots(const int32_t *__restrict__ labels,
                                                   StatsGeom s, const int *base, int *roots,
                                                   long long nroots, ccl_component *comps,
                                                   int max_comps) {
    __shared__ int warp_off[kSTW / 32];
    const int tx = blockIdx.x % s.tiles_x, ty = blockIdx.x / s.tiles_x;
    const int x = tx * kSTW + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int ly = 0; ly < kSTH; ++ly) {
        const int y = ty * kSTH + ly;
        if (y >= s.H) break;   // block-uniform
        const long long p = (long long)y * s.W + x;
        const bool root = x < s.W && __ldg(labels + p) == (int32_t)(p + 1);
        const unsigned b = __ballot_sync(0xFFFFFFFFu, root);
        if (lane == 0) warp_off[warp] = __popc(b);
        __syncthreads();
        if (root) {
            int off = 0;
            for (int k = 0; k < warp; ++k) off += warp_off[k];
            const long long slot = (long long)base[(long long)y * s.tiles_x + tx] + off +
                                   __popc(b & ((1u << lane) - 1u));
            if (slot < nroots) roots[slot] = (int)p;
            if (slot < max_comps) {
                ccl_component c;
                c.label = (int32_t)(p + 1);
                c.count = 0;
                c.xmin = INT_MAX;
                c.ymin = INT_MAX;
                c.xmax = -1;
                c.ymax = -1;
                c.sum_x = 0;
                c.sum_y = 0;
                comps[slot] = c;
            }
        }
        __syncthreads();
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
                                           long long nroots, ccl_component *comps, int max_comps,
                                           const Partial &q) {
    if (q.label < 1 || (long long)q.label > (long long)s.H * s.W) return;   // not canonical
    const long long r = root_rank(s, base, roots, nroots, (long long)q.label - 1);
    if (r < 0 || r >= max_comps) return;
    ccl_component *c = comps + r;
    atomicAdd(&c->count, q.count);
    atomicMin(&c->xmin, q.xmin);
    atomicMin(&c->ymin, q.ymin);
    atomicMax(&c->xmax, q.xmax);
    atomicMax(&c->ymax, q.ymax);
    atomicAdd(reinterpret_cast<unsigned long long *>(&c->sum_x), (unsigned long long)q.sx);
    atomicAdd(reinterpret_cast<unsigned long long *>(&c->sum_y), (unsigned long long)q.sy);
}

struct SmemHash {
    int key[kHash];   // 0 = empty
    int count[kHash], xmin[kHash], ymin[kHash], xmax[kHash], ymax[kHash];
    unsigned long long sx[kHash], sy[kHash];
};

// 4: per-tile sums, then one update per component and tile
__global__ void __launch_bounds__(kSTW) k_st_acc(const int32_t *__restrict__ labels, StatsGeom s,
                                                 const int *base, const int *roots, long long nroots,
                                                 ccl_component *comps, int max_comps) {
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
        add_global(s, base, roots, nroots, comps, max_comps, q);   // table full
    };
    Partial run;   // the current run of equal labels down this thread's column
    run.label = 0;
    if (x < s.W) {
        for (int ly = 0; ly < kSTH; ++ly) {
            const int y = ty * kSTH + ly;
            if (y >= s.H) break;
            const int L = __ldg(labels + (long long)y * s.W + x);
            if (L == 0) continue;
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
        add_global(s, base, roots, nroots, comps, max_comps, q);
    }
}

}  // namespace
}  // namespace ccl

extern "C" size_t ccl_stats_workspace_bytes(int height, int width) {
    if (!ccl::valid_image_dims(height, width)) return 0;
    const ccl::StatsGeom s = ccl::stats_geom(height, width);
    return ccl::counts_bytes(s) + ccl::align256((size_t)ccl::max_roots(height, width) * 4u);
}

extern "C" ccl_status ccl_component_stats(const int32_t *d_labels, int height, int width,
                                          ccl_component *d_comps, int max_comps, int32_t *d_ncomps,
                                          void *d_ws, size_t ws_bytes, ccl_stream stream) {
    if (!d_labels || !d_ncomps || !ccl::valid_image_dims(height, width) || max_comps < 0 ||
        (max_comps > 0 && !d_comps))
        return CCL_ERR_INVALID_ARG;
    const size_t need = ccl_stats_workspace_bytes(height, width);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ccl_status st = CCL_OK;
    if (!d_ws) {
        d_ws = ccl::library_workspace(s, need, &st);
        if (st != CCL_OK) return st;
    } else if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        return CCL_ERR_INVALID_ARG;
    }
    const ccl::StatsGeom g = ccl::stats_geom(height, width);
    int *cnt = static_cast<int *>(d_ws);
    int *roots = reinterpret_cast<int *>(static_cast<char *>(d_ws) + ccl::counts_bytes(g));
    const long long nroots = ccl::max_roots(height, width);
    const unsigned tiles = (unsigned)((long long)g.tiles_x * g.tiles_y);
    ccl::k_st_count<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt);
    ccl::k_st_scan<<<1, ccl::kScanThreads, 0, s>>>(cnt, g.nseg, d_ncomps);
    ccl::k_st_roots<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt, roots, nroots, d_comps, max_comps);
    ccl::k_st_acc<<<tiles, ccl::kSTW, 0, s>>>(d_labels, g, cnt, roots, nroots, d_comps, max_comps);
    if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}
