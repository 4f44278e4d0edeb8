// ccl_core.cuh -- device building blocks of the three-phase union-find CCL
// for sm_103a: bit-packed rows, segment ("run") nodes, shared-memory and
// global-memory union-find, tile geometry and per-tile workspace layout.
//
// Phases (Chen et al., "An Optimized Union-Find Algorithm for Connected
// Components Labeling Using GPUs"):
//   local merge     Kernel 1, §II-A: each thread block labels one tile in
//                   shared memory, roots converted to global raster indices;
//   boundary        Kernel 2, §II-B, Eq. 1-2: unions only across tile seams;
//   link            §II-C: every pixel gets the root of its component.
//
// GB300 design (what differs from the paper's per-pixel Pascal kernels):
//   * A pixel is one bit.  A thread owns one 32-pixel word of a tile row (two
//     rows for 8-connectivity) and finds run starts with shifts, so the
//     paper's row scan and coarse row-column unification (§II-A-2) become a
//     handful of integer instructions per 32 pixels.
//   * Union-find nodes are *segments*: maximal runs of a row (4-connectivity)
//     or of the OR of a two-row strip (8-connectivity: within two rows, all
//     pixels of consecutive non-empty columns are 8-connected).  Unions are
//     needed only between consecutive strips, one per touching run pair.
//   * Roots stay the smallest raster index, as with the paper's atomicMin
//     linking (§II-A-3), but the link step uses the value returned by the
//     atomic (a compare-and-swap that fails when the root was linked
//     concurrently) so a concurrent link is never lost.
//   * The link phase does not re-run union-find: the local merge stores one
//     label per segment (compact) plus the bit-packed image, and the link
//     kernel re-derives segments from the bits.  HBM traffic is about
//     1 B/px read + 4 B/px written plus ~0.6 B/px of compact scratch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccl {

constexpr int kThreads = 256;             // threads per tile = strips x words
constexpr int kNodeCap = kThreads * 16;   // at most 16 run starts per 32-bit word
constexpr int kBorderCapMax = 576;        // border segments: <= 2*16*NW + 2*NS for every NW
constexpr int kHdrInts = 4;               // [0] = border-root count, [1] = segment count

constexpr int kQueueCap = 2048;           // unions left after the local forest pass
constexpr int kSlotBits = 10;             // border slots per tile < 2^10
constexpr int kTileBits = 23;             // tiles per image < 2^23
constexpr long long kMaxTiles = 1ll << kTileBits;

// device error word bits
constexpr int kErrSmemFind = 1;
constexpr int kErrSmemUnion = 2;
constexpr int kErrGlobFind = 4;
constexpr int kErrGlobUnion = 8;
constexpr int kErrResolve = 16;
constexpr int kErrBorderCap = 32;
constexpr int kErrQueue = 64;

// Every union-find walk draws on a per-thread budget of pointer hops; when it
// runs out the thread records an error and stops, so no input and no defect
// can keep a kernel spinning.  Valid inputs stay far below both budgets
// (chains are shortened by path halving / compression as they are walked).
// The 2-D kernels take their budgets as arguments (these values unless a test
// lowers them with ccl_set_hop_budget to make a walk run out on purpose).
constexpr int kSmemHopBudget = 1 << 20;   // per thread per tile (shared memory)
constexpr int kGlobHopBudget = 1 << 20;   // per thread per work item (global memory)

// Geometry of one image under one tile shape, and the layout of the per-tile
// workspace (all offsets in ints from the tile's base):
//   [0, kHdrInts)               header: [0] = number of border roots, [1] = number
//                               of segment nodes
//   [kHdrInts, off_key)         label of each segment node (node_cap)
//   [off_key, off_par)          smallest raster index of each border root's component
//                               inside the tile (border_cap)
//   [off_par, off_rec)          parent of each border root in the global forest,
//                               64-bit node ids (border_cap x 2 ints, 8-byte aligned)
//   [off_rec, off_rec + rec)    seam records, global node of the position's root
//                               (64-bit; all ones: none): top[tw], bottom[tw],
//                               left[ns], right[ns]
struct Geom {
    int H, W;
    int nw;         // 32-bit words per tile row: 1, 2, 4, 8
    int ns;         // strips per tile = kThreads / nw
    int hs;         // strip height: 1 (4-conn) or 2 (8-conn)
    int tw, th;     // tile width / height in pixels
    int log2tw;
    int tiles_x, tiles_y;
    int nwg;        // words per bit-image row = ceil(W / 32)
    int node_cap;   // most segment nodes a tile of this image can hold
    int border_cap; // most border roots
    int off_key, off_par, off_rec, tile_ints;
};

__host__ __device__ inline Geom make_geom(int H, int W, int conn, int tile_w) {
    Geom g;
    g.H = H;
    g.W = W;
    g.nw = tile_w / 32;
    g.ns = kThreads / g.nw;
    g.hs = conn == 8 ? 2 : 1;
    g.tw = tile_w;
    g.th = g.ns * g.hs;
    g.log2tw = tile_w == 32 ? 5 : tile_w == 64 ? 6 : tile_w == 128 ? 7 : 8;
    g.tiles_x = (int)(((long long)W + g.tw - 1) / g.tw);
    g.tiles_y = (int)(((long long)H + g.th - 1) / g.th);
    g.nwg = (int)(((long long)W + 31) / 32);
    // a strip row of c valid columns holds at most ceil(c / 2) runs
    const int cols = W < g.tw ? W : g.tw;
    const int per_strip = (cols + 1) / 2;
    g.node_cap = g.ns * per_strip;
    g.border_cap = 2 * per_strip + 2 * g.ns;
    g.off_key = kHdrInts + g.node_cap;
    g.off_par = (g.off_key + g.border_cap + 1) & ~1;
    g.off_rec = g.off_par + 2 * g.border_cap;
    g.tile_ints = (g.off_rec + 2 * (2 * g.tw + 2 * g.ns) + 63) & ~63;   // 256-byte multiple
    return g;
}

// the (tile, slot) fields of a global node id hold every tile of the image
__host__ __device__ inline bool geom_fits(const Geom &g) {
    return (long long)g.tiles_x * g.tiles_y <= kMaxTiles;
}

__host__ __device__ inline size_t bits_bytes(const Geom &g) {
    size_t b = (size_t)g.H * (size_t)g.nwg * 4u;
    return (b + 255u) & ~(size_t)255u;
}

__host__ __device__ inline size_t tiles_bytes(const Geom &g) {
    return (size_t)g.tiles_x * (size_t)g.tiles_y * (size_t)g.tile_ints * 4u;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  A grid launched with
// programmatic stream serialisation may start once every block of the grid
// before it on the stream has called pdl_launch_dependents() (or exited);
// pdl_wait() then blocks until that previous grid has completed and its
// memory writes are visible.  For a grid launched without the attribute both
// are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// L2 eviction priorities: what the local merge writes for the seam and link
// kernels (bit image, per-tile records, labels, parents; ~60 MB at 8192^2)
// is stored with evict-last priority, so that it outlives the streamed input
// image and label writes in L2 until those kernels read it.
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_policy(uint32_t *p, uint32_t v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_policy(int *p, int v, unsigned long long pol) {
    st_policy(reinterpret_cast<uint32_t *>(p), (uint32_t)v, pol);
}
__device__ __forceinline__ void st_policy(unsigned long long *p, unsigned long long v,
                                          unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_policy(long long *p, long long v, unsigned long long pol) {
    st_policy(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v, pol);
}

// ---------------------------------------------------------------------------
// bit helpers

// mask of bits 0..x (x in [-1, 31]); x = -1 gives 0
__device__ __forceinline__ uint32_t le_mask(int x) {
    return x < 0 ? 0u : (0xFFFFFFFFu >> (31 - x));
}

// 4-bit mask of the nonzero bytes of v (byte k -> bit k): the high bit of
// ((b & 0x7f) + 0x7f) | b is set iff b != 0; the multiply gathers the four
// high bits (positions 7, 15, 23, 31 after >>7: 0, 8, 16, 24) into bits 28-31
// with no carries between partial products.
__device__ __forceinline__ uint32_t nz4(uint32_t v) {
    uint32_t x = (((v & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | v) & 0x80808080u;
    return ((x >> 7) * 0x10204080u) >> 28;
}

__device__ __forceinline__ uint32_t nz16(uint4 v) {
    return nz4(v.x) | (nz4(v.y) << 4) | (nz4(v.z) << 8) | (nz4(v.w) << 12);
}

// Foreground bits of pixels [gx, gx + n) of row y (n = min(32, W - gx)),
// bit k = pixel gx + k.  level < 0: foreground = nonzero byte; level in
// [0, 255]: foreground = byte equal to level (a byte equals the level iff
// its XOR with the level is zero).  img_end bounds every byte read.
__device__ __forceinline__ uint32_t load_row_bits(const uint8_t *__restrict__ img,
                                                  const uint8_t *img_end, int y, int gx,
                                                  int W, bool aligned16, int level = -1) {
    int n = W - gx;
    if (n > 32) n = 32;
    const uint32_t rep = level < 0 ? 0u : (uint32_t)level * 0x01010101u;
    const uint8_t *p = img + (size_t)y * (size_t)W + (size_t)gx;
    uint32_t bits;
    if (aligned16) {
        // W % 16 == 0 and 16-byte aligned base: n is 16 or 32
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        v.x ^= rep; v.y ^= rep; v.z ^= rep; v.w ^= rep;
        bits = nz16(v);
        if (n > 16) {
            uint4 u = __ldg(reinterpret_cast<const uint4 *>(p + 16));
            u.x ^= rep; u.y ^= rep; u.z ^= rep; u.w ^= rep;
            bits |= nz16(u) << 16;
        }
    } else {
        uintptr_t a = reinterpret_cast<uintptr_t>(p);
        int off = (int)(a & 3u);
        const uint8_t *wb = p - off;
        int nwords = (off + n + 3) >> 2;
        uint64_t acc = 0;
        for (int k = 0; k < nwords; ++k) {
            const uint8_t *q = wb + 4 * k;
            uint32_t m4;
            if (q >= img && q + 4 <= img_end) {
                m4 = nz4(__ldg(reinterpret_cast<const uint32_t *>(q)) ^ rep);
            } else {
                m4 = 0;
                for (int b = 0; b < 4; ++b)
                    if (q + b >= img && q + b < img_end && (q[b] ^ (rep & 0xFFu)) != 0) m4 |= 1u << b;
            }
            acc |= (uint64_t)m4 << (4 * k);
        }
        bits = (uint32_t)(acc >> off);
    }
    if (level >= 0) bits = ~bits;   // nonzero XOR = not equal to the level
    return n == 32 ? bits : (bits & ((1u << n) - 1u));
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan over kThreads threads (tid order)

__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            int y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    total = warp_sums[kThreads / 32 - 1];
    return x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
}

// ---------------------------------------------------------------------------
// union-find in shared memory over segment nodes.  P[n] = parent (P[n] <= n is
// not required: links go from the root with the larger key to the one with
// the smaller key, so every root is the smallest key of its tree).

// Parents are plain 32-bit ints: shared-memory compare-and-swap is native at
// that width.
typedef int pnode;

__device__ __forceinline__ int sfind(volatile pnode *P, int x, int &budget, int *err) {
    for (;;) {
        if (--budget < 0) { atomicOr(err, kErrSmemFind); return x; }
        const int p = P[x];
        if (p == x) return x;
        const int g = P[p];
        if (g == p) return p;
        P[x] = (pnode)g;   // path halving: g is an ancestor of x (a smaller key)
        x = g;
    }
}

__device__ __forceinline__ void sunion(pnode *P, const uint16_t *K, int a, int b, int &budget,
                                       int *err) {
    volatile pnode *vP = P;
    volatile const uint16_t *vK = K;
    for (;;) {
        a = sfind(vP, a, budget, err);
        b = sfind(vP, b, budget, err);
        if (a == b) return;
        if (budget < 0) { atomicOr(err, kErrSmemUnion); return; }
        if (vK[a] > vK[b]) { int t = a; a = b; b = t; }
        // link root b (larger key) under root a; fails if b stopped being a root
        if (atomicCAS(&P[b], (pnode)b, (pnode)a) == (pnode)b) return;
    }
}

// ---------------------------------------------------------------------------
// union-find in global memory over the border roots of all tiles.  A node id
// is 64-bit: key << 33 | tile << 10 | slot, where key is the smallest raster
// index of the root's component inside its tile; its parent lives in the
// owning tile's workspace.  Comparing ids compares keys (keys are distinct),
// so linking the larger id under the smaller keeps every root at its set's
// smallest raster index (as the paper's atomicMin linking does) with no key
// loads; and the root of a component spanning many tiles settles at once on
// the image-wide minimum, so concurrent unions link other roots under it
// instead of contending for it.

typedef unsigned long long gnode;
constexpr gnode kNoNode = ~0ull;

__device__ __forceinline__ gnode make_gnode(int key, long long tile, int slot) {
    return ((gnode)(uint32_t)key << (kTileBits + kSlotBits)) | ((gnode)tile << kSlotBits) |
           (gnode)slot;
}

__device__ __forceinline__ int gnode_key(gnode n) { return (int)(n >> (kTileBits + kSlotBits)); }

struct GlobalForest {
    int *tws;
    int tile_ints, off_par;
    __device__ __forceinline__ gnode *par(gnode n) const {
        const long long tile = (long long)((n >> kSlotBits) & (kMaxTiles - 1));
        return reinterpret_cast<gnode *>(tws + (size_t)tile * tile_ints + off_par) +
               (n & ((1u << kSlotBits) - 1u));
    }
};

// The walks below take any forest type with `gnode *par(gnode)` (the tiles of
// an image here; the bricks of a volume in the 3-D path).
template <class Forest>
__device__ __forceinline__ gnode gfind(const Forest &F, gnode x, int &budget, int *err) {
    // Walk to the root, remembering the first two nodes passed whose parent
    // is not the root, then point those at the root.  Keys strictly decrease
    // along parent links, so a node seen below the root always has a larger
    // key than the root: the new link can never close a cycle, whatever other
    // threads did to the path meanwhile.
    gnode w0 = kNoNode, w1 = kNoNode;
    gnode r = x, prev = kNoNode;
    for (;;) {
        if (--budget < 0) { atomicOr(err, kErrGlobFind); return r; }
        const gnode p = __ldcg(F.par(r));
        if (p == r) break;
        if (prev != kNoNode) {   // prev -> r -> p: prev's parent is not the root
            if (w0 == kNoNode) w0 = prev; else if (w1 == kNoNode) w1 = prev;
        }
        prev = r;
        r = p;
    }
    if (w0 != kNoNode) __stcg(F.par(w0), r);
    if (w1 != kNoNode) __stcg(F.par(w1), r);
    return r;
}

// Both finds of a union, walked in lock step so their loads overlap (the
// latency is the longer walk, not the sum); same compression rule as gfind.
template <class Forest>
__device__ __forceinline__ void gfind2(const Forest &F, gnode &a, gnode &b, int &budget,
                                       int *err) {
    gnode ra = a, rb = b;
    gnode prev_a = kNoNode, prev_b = kNoNode, wa = kNoNode, wb = kNoNode;
    bool da = false, db = false;
    while (!(da && db)) {
        if (--budget < 0) { atomicOr(err, kErrGlobFind); a = ra; b = rb; return; }
        const gnode pa = da ? ra : __ldcg(F.par(ra));
        const gnode pb = db ? rb : __ldcg(F.par(rb));
        if (!da) {
            if (pa == ra) {
                da = true;
            } else {
                if (prev_a != kNoNode && wa == kNoNode) wa = prev_a;
                prev_a = ra;
                ra = pa;
            }
        }
        if (!db) {
            if (pb == rb) {
                db = true;
            } else {
                if (prev_b != kNoNode && wb == kNoNode) wb = prev_b;
                prev_b = rb;
                rb = pb;
            }
        }
    }
    // a node seen below its root has a larger key than that root: the new
    // link cannot close a cycle
    if (wa != kNoNode) __stcg(F.par(wa), ra);
    if (wb != kNoNode) __stcg(F.par(wb), rb);
    a = ra;
    b = rb;
}

template <class Forest>
__device__ __forceinline__ void gunion(const Forest &F, gnode a, gnode b, int &budget,
                                       int *err) {
    if (a == b) return;
    {   // first try, one atomic: hook the larger node under the smaller if it is
        // still a root (the smaller need not be one: links still only go from
        // a larger id to a smaller); most seam pairs join sets for the first time
        const gnode hi = a > b ? a : b, lo = a > b ? b : a;
        const gnode old = atomicCAS(F.par(hi), hi, lo);
        if (old == hi) return;
        a = old;
        b = lo;
    }
    for (;;) {
        gfind2(F, a, b, budget, err);
        if (a == b) return;
        if (budget < 0) { atomicOr(err, kErrGlobUnion); return; }
        if (a > b) { const gnode t = a; a = b; b = t; }
        // link root b (larger key) under root a; fails if b was linked meanwhile
        if (atomicCAS(F.par(b), b, a) == b) return;
    }
}

}  // namespace ccl
