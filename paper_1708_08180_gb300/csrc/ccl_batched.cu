// ccl_batched.cu -- many images of different sizes labelled by one pass of
// three persistent kernels (local merge, seam unions, link) that pull work
// from device queues, captured once into a CUDA graph.
//
// One graph serves every batch: its nodes are (1) a host-to-device copy of
// the batch descriptor table from a pinned staging buffer into a descriptor
// buffer the library owns per (device, stream, slot) and (2) the three
// persistent kernels, whose grids are sized to the GPU (SMs x resident blocks)
// and whose work counts and image/scratch pointers are read from the copied
// table.  Each call rewrites the staging buffer and replays the graph, so the
// graph does not depend on the images or on the caller's workspace.  Two slots
// per (device, stream) let the host prepare batch k+1 while batch k runs.
//
// A small first kernel writes, into the caller's workspace, the image of
// every tile and of every seam chunk, so that a block that takes a work item
// from a queue finds its image with one load.  The seam and link kernels are
// launched with programmatic stream serialisation: their blocks become
// resident as the previous kernel's blocks run out of work, and wait
// (griddepcontrol.wait) before reading that kernel's results.
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "ccl_internal.h"
#include "ccl_tile.cuh"

namespace ccl {

struct BatchImage {
    ImageArgs a;
    int tile_off;          // first global tile index of this image
    int pad0;
    long long chunk_off;   // first global seam chunk (256 items) of this image
};

struct BatchHeader {
    int n;                 // images
    int total_tiles;
    long long total_chunks;
    int merge_ctr;         // work-queue heads (zero in the staged copy)
    int seam_ctr;
    int link_ctr;
    int pad0;
    int *tile_img;         // image of every tile (caller workspace, written by kb_maps)
    int *chunk_img;        // image of every seam chunk
    int pad[4];
};
static_assert(sizeof(BatchHeader) == 64, "header size");

constexpr size_t kHdrBytes = 256;

// The image of every tile and seam chunk, one block per image (grid-stride).
__global__ void __launch_bounds__(256) kb_maps(const BatchHeader *hdr, const BatchImage *imgs) {
    const int n = hdr->n;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const Geom &g = imgs[k].a.g;
        const int t0 = imgs[k].tile_off, nt = g.tiles_x * g.tiles_y;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) hdr->tile_img[t0 + i] = k;
        const long long c0 = imgs[k].chunk_off, nc = (seam_items(g) + 255) / 256;
        for (long long i = threadIdx.x; i < nc; i += blockDim.x) hdr->chunk_img[c0 + i] = k;
    }
}

template <int HS>
__global__ void __launch_bounds__(kThreads, 6) kb_merge(BatchHeader *hdr, const BatchImage *imgs,
                                                     int *err) {
    __shared__ SmemMerge sm;
    __shared__ int s_tile, s_img;
    const int total = hdr->total_tiles;
    pdl_launch_dependents();   // the seam kernel may start (it waits before reading)
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&hdr->merge_ctr, 1);
            s_tile = t;
            s_img = t < total ? __ldcg(hdr->tile_img + t) : 0;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= total) break;
        const ImageArgs a = imgs[s_img].a;
        const int tile = t - imgs[s_img].tile_off;
        switch (a.g.nw) {
            case 1: merge_tile<1, HS>(a, tile, false, sm, err); break;
            case 2: merge_tile<2, HS>(a, tile, false, sm, err); break;
            case 4: merge_tile<4, HS>(a, tile, false, sm, err); break;
            default: merge_tile<8, HS>(a, tile, false, sm, err); break;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256, 4) kb_seams(BatchHeader *hdr, const BatchImage *imgs,
                                                int *err) {
    __shared__ SmemSeams sm;
    __shared__ long long s_chunk;
    __shared__ int s_img;
    const long long total = hdr->total_chunks;
    pdl_wait();                // the local merge is complete and visible
    pdl_launch_dependents();   // the link kernel may start (it waits before its walks)
    for (;;) {
        if (threadIdx.x == 0) {
            const long long c = atomicAdd(&hdr->seam_ctr, 1);
            s_chunk = c;
            s_img = c < total ? __ldcg(hdr->chunk_img + c) : 0;
        }
        __syncthreads();
        const long long c = s_chunk;
        if (c >= total) break;
        const ImageArgs a = imgs[s_img].a;
        seam_block(a, (c - imgs[s_img].chunk_off) * 256, seam_items(a.g), sm, err);
        __syncthreads();
    }
}

template <int HS>
__global__ void __launch_bounds__(kThreads, 8) kb_link(BatchHeader *hdr, const BatchImage *imgs,
                                                    int *err) {
    __shared__ SmemLink sm;
    __shared__ int s_tile, s_img;
    const int total = hdr->total_tiles;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&hdr->link_ctr, 1);
            s_tile = t;
            s_img = t < total ? __ldcg(hdr->tile_img + t) : 0;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= total) break;
        const ImageArgs a = imgs[s_img].a;
        const int tile = t - imgs[s_img].tile_off;
        switch (a.g.nw) {
            case 1: link_tile<1, HS>(a, tile, sm.S, sm.c, err); break;
            case 2: link_tile<2, HS>(a, tile, sm.S, sm.c, err); break;
            case 4: link_tile<4, HS>(a, tile, sm.S, sm.c, err); break;
            default: link_tile<8, HS>(a, tile, sm.S, sm.c, err); break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side

namespace {

struct Layout {
    size_t desc_bytes;      // descriptor table capacity (header + entries)
    size_t total_bytes;     // caller workspace: per-image scratch, then the maps
    size_t maps_off;        // tile map (total_tiles ints), then chunk map
    std::vector<size_t> img_off;   // per image workspace offset (bits, then tiles)
    std::vector<Geom> geom;
    int total_tiles;
    long long total_chunks;
};

size_t align256(size_t v) { return (v + 255u) & ~(size_t)255u; }

// Descriptor tables come in power-of-two capacities >= 64 KB; a graph is
// captured per capacity.
size_t desc_capacity(int n) {
    const size_t need = kHdrBytes + sizeof(BatchImage) * (size_t)n;
    size_t cap = 1u << 16;
    while (cap < need) cap <<= 1;
    return cap;
}

bool plan(const ccl_image *imgs, int n, int conn, Layout &L) {
    if (!imgs || n < 1 || !valid_conn(conn)) return false;
    L.desc_bytes = desc_capacity(n);
    size_t off = 0;
    L.img_off.resize(n);
    L.geom.resize(n);
    long long tiles = 0, chunks = 0;
    for (int k = 0; k < n; ++k) {
        const ccl_image &im = imgs[k];
        if (!im.d_img || !im.d_labels || !valid_image_dims(im.height, im.width)) return false;
        const Geom g = make_geom(im.height, im.width, conn,
                                 default_tile_width(im.height, im.width, conn));
        if (!geom_fits(g)) return false;
        L.geom[k] = g;
        L.img_off[k] = off;
        // sized for the widest need over all tile widths: a workspace sized
        // before a re-tune of the size-class table stays valid after it
        off += align256(ccl_workspace_bytes(im.height, im.width, conn));
        tiles += (long long)g.tiles_x * g.tiles_y;
        chunks += (seam_items(g) + 255) / 256;
    }
    if (tiles > 0x7FFFFFFFLL || chunks > 0x7FFFFFFFLL) return false;
    L.total_tiles = (int)tiles;
    L.total_chunks = chunks;
    L.maps_off = off;
    off += align256((size_t)tiles * 4u) + align256((size_t)chunks * 4u);
    L.total_bytes = off;
    return true;
}

struct Persist {
    int merge_blocks = 0, seam_blocks = 0, link_blocks = 0;
};

struct GraphSlot {
    void *staging = nullptr;        // pinned host copy of header + descriptors
    void *d_desc = nullptr;         // device copy read by the kernels
    size_t desc_bytes = 0;
    cudaEvent_t done = nullptr;     // recorded after the slot's last graph launch
    cudaGraphExec_t exec = nullptr;
    int exec_conn = 0;
};

// Per (device, stream): its two slots and capture stream, under its own
// mutex, so that a call waiting for its slot's previous batch does not hold
// up calls on other streams (g_mu only guards the maps).
struct StreamState {
    std::mutex mu;
    GraphSlot slot[2];
    int next = 0;
    cudaStream_t capture = nullptr;
};

std::mutex g_mu;
std::map<int, Persist> g_persist;
std::map<std::pair<int, cudaStream_t>, std::shared_ptr<StreamState>> g_state;

bool persist_dims(int dev, int conn, Persist &p) {
    auto it = g_persist.find(dev * 16 + conn);
    if (it != g_persist.end()) { p = it->second; return true; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    int bm = 0, bs = 0, bl = 0;
    if (conn == 8) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, kb_merge<2>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, kb_link<2>, kThreads, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, kb_merge<1>, kThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, kb_link<1>, kThreads, 0);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, kb_seams, 256, 0);
    if (cudaGetLastError() != cudaSuccess) return false;
    p.merge_blocks = sms * (bm > 0 ? bm : 1);
    p.seam_blocks = sms * (bs > 0 ? bs : 1);
    p.link_blocks = sms * (bl > 0 ? bl : 1);
    g_persist[dev * 16 + conn] = p;
    return true;
}

void launch_kernels(const Persist &p, int conn, BatchHeader *hdr, const BatchImage *imgs,
                    int *err, cudaStream_t s) {
    kb_maps<<<p.link_blocks, 256, 0, s>>>(hdr, imgs);
    if (conn == 8) {
        kb_merge<2><<<p.merge_blocks, kThreads, 0, s>>>(hdr, imgs, err);
        launch_pdl(kb_seams, (unsigned)p.seam_blocks, 256u, s, hdr, imgs, err);
        launch_pdl(kb_link<2>, (unsigned)p.link_blocks, (unsigned)kThreads, s, hdr, imgs, err);
    } else {
        kb_merge<1><<<p.merge_blocks, kThreads, 0, s>>>(hdr, imgs, err);
        launch_pdl(kb_seams, (unsigned)p.seam_blocks, 256u, s, hdr, imgs, err);
        launch_pdl(kb_link<1>, (unsigned)p.link_blocks, (unsigned)kThreads, s, hdr, imgs, err);
    }
}

void release_slot(GraphSlot &sl) {
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.staging) cudaFreeHost(sl.staging);
    if (sl.d_desc) cudaFree(sl.d_desc);
    sl = GraphSlot();
}

}  // namespace

void free_batched_state() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_state) {
        StreamState &ss = *kv.second;
        std::lock_guard<std::mutex> lks(ss.mu);
        for (auto &sl : ss.slot) {
            if (sl.done) cudaEventSynchronize(sl.done);
            release_slot(sl);
        }
        if (ss.capture) cudaStreamDestroy(ss.capture);
        ss.capture = nullptr;
    }
    g_state.clear();
    g_persist.clear();
}

static ccl_status enqueue_batched(const ccl_image *imgs, int n, int conn, void *d_ws,
                                  size_t ws_bytes, cudaStream_t stream) {
    Layout L;
    if (!plan(imgs, n, conn, L)) return CCL_ERR_INVALID_ARG;
    ccl_status st = CCL_OK;
    if (!d_ws) {
        d_ws = library_workspace(stream, L.total_bytes, &st);
        if (st != CCL_OK) return st;
        ws_bytes = L.total_bytes;
    } else if (ws_bytes < L.total_bytes || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        return CCL_ERR_INVALID_ARG;
    }
    int *err = device_error_word();
    if (!err) return CCL_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CCL_ERR_CUDA;

    Persist p;
    std::shared_ptr<StreamState> ssp;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!persist_dims(dev, conn, p)) return CCL_ERR_CUDA;
        auto &slot_ptr = g_state[{dev, stream}];
        if (!slot_ptr) slot_ptr = std::make_shared<StreamState>();
        ssp = slot_ptr;
    }
    StreamState &ss = *ssp;
    std::lock_guard<std::mutex> lk(ss.mu);
    if (!ss.capture &&
        cudaStreamCreateWithFlags(&ss.capture, cudaStreamNonBlocking) != cudaSuccess)
        return CCL_ERR_CUDA;
    GraphSlot &sl = ss.slot[ss.next];
    ss.next ^= 1;

    // the slot's previous batch must be finished with its staging/descriptor buffers
    if (sl.done && cudaEventSynchronize(sl.done) != cudaSuccess) return CCL_ERR_CUDA;
    if (sl.desc_bytes != L.desc_bytes) {
        release_slot(sl);
        if (cudaHostAlloc(&sl.staging, L.desc_bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&sl.d_desc, L.desc_bytes) != cudaSuccess) {
            cudaGetLastError();
            release_slot(sl);
            return CCL_ERR_OOM;
        }
        sl.desc_bytes = L.desc_bytes;
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
            return CCL_ERR_CUDA;
    }

    // fill the staged header + descriptor table
    char *ws = static_cast<char *>(d_ws);
    BatchHeader *d_hdr = static_cast<BatchHeader *>(sl.d_desc);
    BatchImage *d_imgs = reinterpret_cast<BatchImage *>(static_cast<char *>(sl.d_desc) + kHdrBytes);
    std::memset(sl.staging, 0, kHdrBytes + sizeof(BatchImage) * (size_t)n);
    BatchHeader *h = static_cast<BatchHeader *>(sl.staging);
    h->n = n;
    h->total_tiles = L.total_tiles;
    h->total_chunks = L.total_chunks;
    h->tile_img = reinterpret_cast<int *>(ws + L.maps_off);
    h->chunk_img = reinterpret_cast<int *>(ws + L.maps_off + align256((size_t)L.total_tiles * 4u));
    BatchImage *hi = reinterpret_cast<BatchImage *>(static_cast<char *>(sl.staging) + kHdrBytes);
    int tiles = 0;
    long long chunks = 0;
    for (int k = 0; k < n; ++k) {
        const Geom &g = L.geom[k];
        BatchImage &b = hi[k];
        b.a.img = imgs[k].d_img;
        b.a.labels = imgs[k].d_labels;
        b.a.bits = reinterpret_cast<uint32_t *>(ws + L.img_off[k]);
        b.a.tws = reinterpret_cast<int *>(ws + L.img_off[k] + bits_bytes(g));
        b.a.g = g;
        b.a.aligned16 = (g.W % 16 == 0) && (reinterpret_cast<uintptr_t>(imgs[k].d_img) % 16 == 0);
        b.a.out_aligned16 =
            (g.W % 4 == 0) && (reinterpret_cast<uintptr_t>(imgs[k].d_labels) % 16 == 0);
        b.a.level = -1;
        b.a.merge_out = 0;
        b.a.hops_smem = hop_budget_smem();
        b.a.hops_glob = hop_budget_glob();
        b.tile_off = tiles;
        b.chunk_off = chunks;
        tiles += g.tiles_x * g.tiles_y;
        chunks += (seam_items(g) + 255) / 256;
    }

    // capture the slot's graph once per descriptor capacity and connectivity
    if (!sl.exec || sl.exec_conn != conn) {
        if (sl.exec) { cudaGraphExecDestroy(sl.exec); sl.exec = nullptr; }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(ss.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return CCL_ERR_CUDA;
        cudaMemcpyAsync(sl.d_desc, sl.staging, sl.desc_bytes, cudaMemcpyHostToDevice, ss.capture);
        launch_kernels(p, conn, d_hdr, d_imgs, err, ss.capture);
        if (cudaStreamEndCapture(ss.capture, &graph) != cudaSuccess) {
            cudaGetLastError();
            return CCL_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&sl.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) { cudaGetLastError(); sl.exec = nullptr; return CCL_ERR_CUDA; }
        sl.exec_conn = conn;
    }
    if (cudaGraphLaunch(sl.exec, stream) != cudaSuccess) { cudaGetLastError(); return CCL_ERR_CUDA; }
    if (cudaEventRecord(sl.done, stream) != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}

}  // namespace ccl

extern "C" size_t ccl_batched_workspace_bytes(const ccl_image *imgs, int n, int connectivity) {
    ccl::Layout L;
    if (!ccl::plan(imgs, n, connectivity, L)) return 0;
    return L.total_bytes;
}

extern "C" ccl_status ccl_label_batched(const ccl_image *imgs, int n, int connectivity,
                                        void *d_ws, size_t ws_bytes, ccl_stream stream) {
    return ccl::enqueue_batched(imgs, n, connectivity, d_ws, ws_bytes,
                                reinterpret_cast<cudaStream_t>(stream));
}
