// ccl_plain.cu -- single-image path: the three kernels (local merge, seam
// unions, link) and the ccl_label / ccl_label_tiled entry points.
#include <atomic>
#include <mutex>
#include <utility>

#include "ccl_internal.h"
#include "ccl_tile.cuh"

namespace ccl {

// local-merge blocks resident per SM (32 registers, shared memory: 8 x SmemMerge;
// the statistics variant, with a per-node record buffer, holds 6)
constexpr int kMergeBlocksPerSm = 8;

// SMs of the current device (cached per device)
static int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 0; }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// The link kernel is launched with programmatic stream serialisation: once
// every seam block has started (and passed its own wait), link blocks may
// start and run the part of their prologue that reads only the local-merge
// output, then wait (pdl_wait in link_tile) for the seam unions.  When the
// local merge fits in one wave of blocks the seam kernel is launched the
// same way, so that its launch overlaps the local merge's last blocks; its
// blocks wait for the local merge before reading anything.  When it takes
// several waves the local merge itself is launched that way, so that its
// blocks are resident when the previous grid on the stream ends; they wait
// for that grid (pdl_wait) before reading anything.
template <int NW, int HS, bool STATS>
__global__ void __launch_bounds__(kThreads, STATS ? 6 : 8) k_merge(ImageArgs a, int local_only, int *err) {
    __shared__ SmemMerge sm;
    __shared__ uint16_t lslot[STATS ? kNodeCap : 2];   // statistics: local record per root
    pdl_wait();
    pdl_launch_dependents();
    merge_tile<NW, HS, STATS>(a, blockIdx.x, local_only != 0, sm, err, STATS ? lslot : nullptr);
}

__global__ void __launch_bounds__(256, 5) k_seams(ImageArgs a, long long nitems, int *err) {
    __shared__ SmemSeams sm;
    pdl_wait();
    pdl_launch_dependents();
    seam_block(a, (long long)blockIdx.x * 256, nitems, sm, err);
}


template <int NW, int HS>
__global__ void __launch_bounds__(kThreads, 8) k_link(ImageArgs a, int *err) {
    __shared__ SmemLink sm;
    pdl_launch_dependents();
    link_tile<NW, HS>(a, blockIdx.x, sm.S, sm.c, err);
}

// The link kernel of ccl_label_with_stats: the same blocks that write the
// labels gather every component's statistics (the per-tile statistics
// tables and the link's shared memory, dynamic).  The statistics work
// (shared-memory tables, register aggregation) fills issue slots that the
// label stores, bound by HBM writes, leave free.
constexpr size_t kLinkFusedSmem = ((sizeof(SmemLinkStats) + 15) & ~(size_t)15) + sizeof(SmemLink);

template <int NW, int HS>
__global__ void __launch_bounds__(kThreads, 4) k_link_stats(ImageArgs a, int *err) {
    extern __shared__ __align__(16) unsigned char dsm[];
    SmemLinkStats *sx = reinterpret_cast<SmemLinkStats *>(dsm);
    SmemLink &sm = *reinterpret_cast<SmemLink *>(dsm + ((sizeof(SmemLinkStats) + 15) & ~(size_t)15));
    pdl_launch_dependents();
    link_tile<NW, HS, true>(a, blockIdx.x, sm.S, sm.c, err, sx);
}

// Statistics, last step: every border root that is its component's global
// root emits the component's record from its accumulator (one slot range per
// 256 border roots of a tile, reserved with one atomic).
__global__ void __launch_bounds__(256) k_stats_pack(ImageArgs a, int *err) {
    __shared__ int warp_sums[kThreads / 32];
    __shared__ int s_base;
    const Geom &g = a.g;
    const int tile = blockIdx.x;
    const int *tw_ = a.tws + (size_t)tile * g.tile_ints;
    const int nb = min(__ldcg(tw_), g.border_cap);
    const gnode *par = reinterpret_cast<const gnode *>(tw_ + g.off_par);
    const BorderAcc *acc = static_cast<const BorderAcc *>(a.bacc) + (size_t)tile * g.border_cap;
    CompRec *recs = static_cast<CompRec *>(a.comps);
    for (int j0 = 0; j0 < nb; j0 += kThreads) {   // block-uniform trip count
        const int j = j0 + (int)threadIdx.x;
        int key = 0;
        bool root = false;
        if (j < nb) {
            key = __ldcg(tw_ + g.off_key + j);
            root = __ldcg(par + j) == make_gnode(key, tile, j);
        }
        int tot;
        const int rank = block_excl_scan(root ? 1 : 0, warp_sums, tot);
        if (threadIdx.x == 0) s_base = tot ? atomicAdd(a.ncomps, tot) : 0;
        __syncthreads();
        const long long o = (long long)s_base + rank;
        if (root && o < a.max_comps) {
            const BorderAcc &b = acc[j];
            CompRec c;
            c.label = 1 + key;
            c.count = (int)b.count;
            c.xmin = b.xmin;
            c.ymin = b.ymin;
            c.xmax = b.xmax;
            c.ymax = b.ymax;
            c.sum_x = (long long)b.sum_x;
            c.sum_y = (long long)b.sum_y;
            recs[o] = c;
        }
        __syncthreads();
    }
}

// link_early: the link kernel directly follows the seam kernel and may start
// early; otherwise (no seam kernel ran) it waits for the local merge as usual
template <int NW, int HS>
static void launch_merge_link(const ImageArgs &a, bool local_only, int *err, cudaStream_t s,
                              bool link, bool link_early, bool stats) {
    const int ntiles = a.g.tiles_x * a.g.tiles_y;
    if (!link) {
        void (*km)(ImageArgs, int, int *) = stats ? k_merge<NW, HS, true> : k_merge<NW, HS, false>;
        if (ntiles > kMergeBlocksPerSm * sm_count())
            launch_pdl(km, (unsigned)ntiles, (unsigned)kThreads, s, a, local_only ? 1 : 0, err);
        else
            km<<<ntiles, kThreads, 0, s>>>(a, local_only ? 1 : 0, err);
    } else if (stats) {   // labels and statistics in one grid
        static bool attr_set = false;   // per template instance; idempotent
        if (!attr_set) {
            cudaFuncSetAttribute(k_link_stats<NW, HS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLinkFusedSmem);
            attr_set = true;
        }
        if (link_early)
            launch_pdl_smem(k_link_stats<NW, HS>, (unsigned)ntiles, (unsigned)kThreads, kLinkFusedSmem, s, a, err);
        else
            k_link_stats<NW, HS><<<ntiles, kThreads, kLinkFusedSmem, s>>>(a, err);
    } else if (link_early) {
        launch_pdl(k_link<NW, HS>, (unsigned)ntiles, (unsigned)kThreads, s, a, err);
    } else {
        k_link<NW, HS><<<ntiles, kThreads, 0, s>>>(a, err);
    }
}

static void launch_tile_kernel(const ImageArgs &a, bool local_only, int *err, cudaStream_t s,
                               bool link, bool link_early = false, bool stats = false) {
    const int nw = a.g.nw, hs = a.g.hs;
#define CCL_CASE(NW_, HS_) \
    if (nw == NW_ && hs == HS_) { launch_merge_link<NW_, HS_>(a, local_only, err, s, link, link_early, stats); return; }
    CCL_CASE(1, 1) CCL_CASE(2, 1) CCL_CASE(4, 1) CCL_CASE(8, 1)
    CCL_CASE(1, 2) CCL_CASE(2, 2) CCL_CASE(4, 2) CCL_CASE(8, 2)
#undef CCL_CASE
}

// Size-class table: the tile width for an image, indexed by the classes of
// its width and height (<= 64, 128, 256, 512, 1024, 2048, > 2048).  Tiles
// are 8192 (4-conn) or 16384 (8-conn) pixels whatever their width, so the
// choice trades idle columns and vertical seams (narrow tiles) against idle
// rows and horizontal seams (wide tiles).  Initialised with the smallest
// power of two >= W (at most 256) and re-measured by ccl_autotune().
static std::atomic<int> g_tile_table[2][kTileClasses][kTileClasses];
static std::once_flag g_tile_once;

static int initial_tile_width(int wc) {
    return wc <= 0 ? 64 : wc == 1 ? 128 : 256;
}

static void init_tile_table() {
    std::call_once(g_tile_once, [] {
        for (int c = 0; c < 2; ++c)
            for (int hc = 0; hc < kTileClasses; ++hc)
                for (int wc = 0; wc < kTileClasses; ++wc)
                    g_tile_table[c][hc][wc].store(initial_tile_width(wc));
    });
}

int tile_class(int extent) {
    int c = 0;
    while (c < kTileClasses - 1 && extent > (64 << c)) ++c;
    return c;
}

int default_tile_width(int height, int width, int conn) {
    init_tile_table();
    int tw = g_tile_table[conn == 8 ? 1 : 0][tile_class(height)][tile_class(width)].load();
    // never wider than needed: the smallest power of two >= W (>= 32)
    int cap = 32;
    while (cap < width && cap < 256) cap <<= 1;
    return tw < cap ? tw : cap;
}

void set_tile_table_entry(int conn, int hc, int wc, int tile_w) {
    init_tile_table();
    g_tile_table[conn == 8 ? 1 : 0][hc][wc].store(tile_w);
}

// per host thread: events for the next enqueue_label call (benchmark hook)
static thread_local cudaEvent_t t_phase_events[4];
static thread_local bool t_phase_armed = false;

// workspace of the statistics mode past the labelling workspace: component
// slots per segment, then border-root accumulators
size_t stats_extra_bytes(const Geom &g) {
    const size_t tiles = (size_t)g.tiles_x * (size_t)g.tiles_y;
    const size_t cs = (tiles * (size_t)cslot_stride(g) * 2u + 255u) & ~(size_t)255u;
    const size_t ba = (tiles * (size_t)g.border_cap * sizeof(BorderAcc) + 255u) & ~(size_t)255u;
    return cs + ba;
}

ccl_status enqueue_label(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                         int conn, int tile_w, unsigned flags, void *d_ws, size_t ws_bytes,
                         cudaStream_t stream, int level, bool merge_out, const StatsOut *so) {
    if (!d_img || !d_labels || !valid_image_dims(height, width) || !valid_conn(conn))
        return CCL_ERR_INVALID_ARG;
    const bool default_tile = tile_w == 0;
    if (default_tile) tile_w = default_tile_width(height, width, conn);
    if (!valid_tile_w(tile_w)) return CCL_ERR_INVALID_ARG;
    if (flags & ~(unsigned)CCL_FLAG_LOCAL_ONLY) return CCL_ERR_INVALID_ARG;
    const Geom g = make_geom(height, width, conn, tile_w);
    if (!geom_fits(g)) return CCL_ERR_INVALID_ARG;
    // the documented contract: ccl_workspace_bytes() for the default tile
    // width (it does not depend on the current table), the exact need otherwise
    size_t need = default_tile ? ccl_workspace_bytes(height, width, conn)
                               : bits_bytes(g) + tiles_bytes(g);
    if (so) {
        // the statistics name a global root by (tile, slot) in 32 bits
        if ((long long)g.tiles_x * g.tiles_y >= (1ll << (32 - kSlotBits))) return CCL_ERR_INVALID_ARG;
        if (!so->comps && so->max_comps > 0) return CCL_ERR_INVALID_ARG;
        if (!so->ncomps || so->max_comps < 0 || (flags & CCL_FLAG_LOCAL_ONLY) || level >= 0)
            return CCL_ERR_INVALID_ARG;
        need = ccl_workspace_bytes_with_stats(height, width, conn);
    }
    ccl_status st = CCL_OK;
    if (!d_ws) {
        d_ws = library_workspace(stream, need, &st);
        if (st != CCL_OK) return st;
    } else if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        return CCL_ERR_INVALID_ARG;
    }
    int *err = device_error_word();
    if (!err) return CCL_ERR_CUDA;
    ImageArgs a;
    a.img = d_img;
    a.labels = d_labels;
    a.bits = static_cast<uint32_t *>(d_ws);
    a.tws = reinterpret_cast<int *>(static_cast<char *>(d_ws) + bits_bytes(g));
    a.g = g;
    a.aligned16 = (width % 16 == 0) && (reinterpret_cast<uintptr_t>(d_img) % 16 == 0);
    a.out_aligned16 = (width % 4 == 0) && (reinterpret_cast<uintptr_t>(d_labels) % 16 == 0);
    a.level = level;
    a.merge_out = merge_out ? 1 : 0;
    a.hops_smem = hop_budget_smem();
    a.hops_glob = hop_budget_glob();
    a.comps = nullptr;
    a.ncomps = nullptr;
    a.cslot = nullptr;
    a.bacc = nullptr;
    a.max_comps = 0;
    if (so) {
        char *x = static_cast<char *>(d_ws) + bits_bytes(g) + tiles_bytes(g);
        x = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(x) + 255u) & ~(uintptr_t)255u);
        a.cslot = reinterpret_cast<uint16_t *>(x);
        const size_t tiles = (size_t)g.tiles_x * (size_t)g.tiles_y;
        a.bacc = x + ((tiles * (size_t)cslot_stride(g) * 2u + 255u) & ~(size_t)255u);
        a.comps = so->comps;
        a.ncomps = so->ncomps;
        a.max_comps = so->max_comps;
        if (cudaMemsetAsync(so->ncomps, 0, sizeof(int), stream) != cudaSuccess) return CCL_ERR_CUDA;
    }
    const bool local_only = (flags & CCL_FLAG_LOCAL_ONLY) != 0;

    const bool timed = t_phase_armed;
    t_phase_armed = false;
    if (timed) cudaEventRecord(t_phase_events[0], stream);
    launch_tile_kernel(a, local_only, err, stream, false, false, so != nullptr);
    if (timed) cudaEventRecord(t_phase_events[1], stream);
    const long long items = seam_items(g);
    const bool seams = !local_only && items > 0;
    if (seams) {
        const long long blocks = (items + 255) / 256;
        if ((long long)g.tiles_x * g.tiles_y <= (long long)kMergeBlocksPerSm * sm_count())
            launch_pdl(k_seams, (unsigned)blocks, 256u, stream, a, items, err);
        else
            k_seams<<<(unsigned)blocks, 256, 0, stream>>>(a, items, err);
    }
    if (timed) cudaEventRecord(t_phase_events[2], stream);
    if (so) {
        launch_tile_kernel(a, local_only, err, stream, true, seams, true);
        k_stats_pack<<<(unsigned)(g.tiles_x * g.tiles_y), 256, 0, stream>>>(a, err);
    } else {
        launch_tile_kernel(a, local_only, err, stream, true, seams, false);
    }
    if (timed) cudaEventRecord(t_phase_events[3], stream);
    if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // namespace ccl

extern "C" int ccl_default_tile_width(int height, int width, int connectivity) {
    if (!ccl::valid_image_dims(height, width) || !ccl::valid_conn(connectivity)) return 0;
    return ccl::default_tile_width(height, width, connectivity);
}

extern "C" size_t ccl_workspace_bytes_tiled(int height, int width, int connectivity,
                                            int tile_w) {
    if (!ccl::valid_image_dims(height, width) || !ccl::valid_conn(connectivity)) return 0;
    if (tile_w == 0) return ccl_workspace_bytes(height, width, connectivity);
    if (!ccl::valid_tile_w(tile_w)) return 0;
    const ccl::Geom g = ccl::make_geom(height, width, connectivity, tile_w);
    if (!ccl::geom_fits(g)) return 0;
    return ccl::bits_bytes(g) + ccl::tiles_bytes(g);
}

// The largest need over every tile width, so that a workspace sized once
// stays large enough when the size-class table is re-tuned.
extern "C" size_t ccl_workspace_bytes(int height, int width, int connectivity) {
    size_t m = 0;
    for (int tw = 32; tw <= 256; tw <<= 1) {
        const size_t b = ccl_workspace_bytes_tiled(height, width, connectivity, tw);
        if (b > m) m = b;
    }
    return m;
}

extern "C" ccl_status ccl_label(const uint8_t *d_img, int32_t *d_labels, int height, int width,
                                int connectivity, void *d_ws, size_t ws_bytes,
                                ccl_stream stream) {
    return ccl::enqueue_label(d_img, d_labels, height, width, connectivity, 0, 0u, d_ws,
                              ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

// The need over every tile width, as ccl_workspace_bytes.
extern "C" size_t ccl_workspace_bytes_with_stats(int height, int width, int connectivity) {
    if (!ccl::valid_image_dims(height, width) || !ccl::valid_conn(connectivity)) return 0;
    size_t m = 0;
    for (int tw = 32; tw <= 256; tw <<= 1) {
        const ccl::Geom g = ccl::make_geom(height, width, connectivity, tw);
        if (!ccl::geom_fits(g)) return 0;
        const size_t b = ((ccl::bits_bytes(g) + ccl::tiles_bytes(g) + 255u) & ~(size_t)255u) +
                         ccl::stats_extra_bytes(g);
        if (b > m) m = b;
    }
    return m;
}

extern "C" ccl_status ccl_label_with_stats(const uint8_t *d_img, int32_t *d_labels, int height,
                                           int width, int connectivity, ccl_component *d_comps,
                                           int max_comps, int32_t *d_ncomps, void *d_ws,
                                           size_t ws_bytes, ccl_stream stream) {
    static_assert(sizeof(ccl_component) == sizeof(ccl::CompRec), "record layout");
    const ccl::StatsOut so{d_comps, max_comps, d_ncomps};
    return ccl::enqueue_label(d_img, d_labels, height, width, connectivity, 0, 0u, d_ws, ws_bytes,
                              reinterpret_cast<cudaStream_t>(stream), -1, false, &so);
}

extern "C" ccl_status ccl_label_regions(const uint8_t *d_img, int32_t *d_labels, int height,
                                        int width, int connectivity, const uint8_t *levels,
                                        int nlevels, void *d_ws, size_t ws_bytes,
                                        ccl_stream stream) {
    if (!levels || nlevels < 1 || nlevels > 256) return CCL_ERR_INVALID_ARG;
    bool seen[256] = {};
    for (int k = 0; k < nlevels; ++k) {
        if (seen[levels[k]]) return CCL_ERR_INVALID_ARG;   // levels must be distinct
        seen[levels[k]] = true;
    }
    // one pass per level: the first writes every pixel, the others only theirs
    for (int k = 0; k < nlevels; ++k) {
        const ccl_status st = ccl::enqueue_label(d_img, d_labels, height, width, connectivity, 0,
                                                 0u, d_ws, ws_bytes,
                                                 reinterpret_cast<cudaStream_t>(stream),
                                                 (int)levels[k], k > 0);
        if (st != CCL_OK) return st;
    }
    return CCL_OK;
}

extern "C" ccl_status ccl_label_tiled(const uint8_t *d_img, int32_t *d_labels, int height,
                                      int width, int connectivity, int tile_w, unsigned flags,
                                      void *d_ws, size_t ws_bytes, ccl_stream stream) {
    return ccl::enqueue_label(d_img, d_labels, height, width, connectivity, tile_w, flags, d_ws,
                              ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" void ccl_set_phase_events(void *const *events) {
    if (!events) { ccl::t_phase_armed = false; return; }
    for (int k = 0; k < 4; ++k) ccl::t_phase_events[k] = static_cast<cudaEvent_t>(events[k]);
    ccl::t_phase_armed = true;
}
