// ccl_tile.cuh -- per-tile device routines shared by the single-image and
// batched kernels: local merge (Kernel 1, §II-A), seam unions (Kernel 2,
// §II-B) and link (§II-C).
#pragma once

#include "ccl_core.cuh"

namespace ccl {

// Statistics (ccl_label_with_stats): components aggregated per tile in shared
// memory; the ones past these tables are added straight into global memory.
constexpr int kStatLocal = 128;    // components inside the tile
constexpr int kStatBorder = 128;   // global roots of the tile's border roots

// One image as the kernels see it.
struct ImageArgs {
    const uint8_t *img;
    int32_t *labels;       // output label image (written by the link phase only)
    uint32_t *bits;        // bit image: H rows x nwg words
    int *tws;              // per-tile workspace, g.tile_ints ints per tile
    Geom g;
    int aligned16;         // image rows start on 16-byte boundaries (W % 16 == 0)
    int out_aligned16;     // label rows start on 16-byte boundaries (W % 4 == 0)
    int level;             // -1: foreground = nonzero byte; else byte == level
    int merge_out;         // link writes only its foreground pixels, keeping the others
    int hops_smem;         // hop budget of each shared-memory walk sequence (per thread, tile)
    int hops_glob;         // hop budget of each global-forest walk sequence (per thread, item)
    // component statistics (the STATS kernels of ccl_label_with_stats only)
    void *comps;           // output records (CompRec), max_comps of them
    int *ncomps;           // component count (zeroed before the local merge)
    uint16_t *cslot;       // per tile, cslot_stride entries: each segment's component slot
    void *bacc;            // per tile, border_cap BorderAcc: border-root accumulators
    int max_comps;
};

// One component's record, laid out as ccl_component of the C ABI.
struct CompRec {
    int32_t label, count, xmin, ymin, xmax, ymax;
    long long sum_x, sum_y;
};

// Statistics gathered for a border root's component across tiles (global
// coordinates): kept by the border root that is the component's global root.
struct BorderAcc {
    unsigned count;
    int xmin, ymin, xmax, ymax, pad;
    unsigned long long sum_x, sum_y;
};

__device__ __forceinline__ void init_border_acc(BorderAcc *b) {
    b->count = 0u;
    b->xmin = 0x7FFFFFFF;
    b->ymin = 0x7FFFFFFF;
    b->xmax = -1;
    b->ymax = -1;
    b->pad = 0;
    b->sum_x = 0ull;
    b->sum_y = 0ull;
}

// Shared memory of the local-merge phase.
struct SmemMerge {
    pnode P[kNodeCap];             // parent of each segment node
    uint16_t K[kNodeCap];          // key (smallest tile-local pixel index); for a
                                   // root reaching a seam, later its border slot
    uint32_t flag[kNodeCap / 32];  // roots whose component reaches a tile seam
    uint32_t top[kThreads];        // first row of the strip, per word
    uint32_t bot[kThreads];        // last row of the strip, per word (a word's segment
                                   // starts follow from these two words and the word's
                                   // left neighbour's)
    uint16_t base[kThreads];       // rank of the first segment starting in the word
    int warp_sums[kThreads / 32];
    int nborder;
    int nq;
    int nlocal;                    // statistics: components inside the tile
    int out_base;                  // statistics: their first output record
};

// Shared memory of the link phase: the label of every segment node (the
// statistics-only grid has none) and the rest.
struct SmemLinkCore {
    int R[kBorderCapMax];         // final label per border root
    uint32_t rows[2 * kThreads];  // bit rows of the tile: [row][word]
    uint32_t st[kThreads];        // segment starts per (strip, word)
    int base[kThreads];           // rank of the word's first segment start
    int warp_sums[kThreads / 32];
};
struct SmemLink {
    __align__(16) int S[kNodeCap];   // label per segment node
    SmemLinkCore c;
};

// Statistics mode of the link phase: per-tile aggregates of the components
// the tile's segments belong to (tile coordinates), flushed once per tile.
constexpr int kStatHash = 1024;    // global roots of a tile's border roots (hash table)
// A global forest node without its key: tile << kSlotBits | slot (tiles of
// at least 8192 pixels: fewer than 2^18 per image, so this fits 32 bits).
__device__ __forceinline__ uint32_t gnode_site(gnode r) {
    return (uint32_t)(r & ((1ull << (kTileBits + kSlotBits)) - 1ull));
}
constexpr uint32_t kNoSite = 0xFFFFFFFFu;

struct SmemLinkStats {
    __align__(16) uint16_t C[kNodeCap];       // component slot per segment node (cslot encoding)
    uint32_t G[kBorderCapMax];                // global root (site) of each border root
    uint32_t HK[kStatHash];                   // hash table: the distinct global roots ...
    uint16_t HV[kStatHash];                   // ... and their aggregate index in the tile
    uint16_t HJ[kBorderCapMax];               // each border root's hash entry
    uint16_t HR[kBorderCapMax];               // each aggregate index's hash entry
    unsigned LA[kStatLocal][7];               // count, xmin, ymin, xmax, ymax, sum x, sum y
    unsigned BA[kStatBorder][7];              // per global root
    int nroots;                               // distinct global roots in the tile
};

// A segment's component slot, 16 bits: a component inside the tile (its
// record index in the tile, < 2^15), or a border root (bit 15 set, border slot
// in the low bits).
constexpr uint16_t kSlotBorder = 0x8000u;

// per-tile stride of the component-slot array, in 16-bit entries (16-byte
// multiple for cp.async)
__host__ __device__ inline int cslot_stride(const Geom &g) { return (g.node_cap + 7) & ~7; }

// sum of the positions of the set bits of v
__device__ __forceinline__ int bit_position_sum(uint32_t v) {
    return __popc(v & 0xAAAAAAAAu) + 2 * __popc(v & 0xCCCCCCCCu) + 4 * __popc(v & 0xF0F0F0F0u) +
           8 * __popc(v & 0xFF00FF00u) + 16 * __popc(v & 0xFFFF0000u);
}

// rank of the segment containing column bit x (x in [-1, 31]) of a word with
// segment starts `st` whose first start has rank `base`
__device__ __forceinline__ int seg_rank(int base, uint32_t st, int x) {
    return base + __popc(st & le_mask(x)) - 1;
}

// ---------------------------------------------------------------------------
// Kernel 1 body: local merge of tile `tile` (§II-A).
//
// Thread (s, w) = (threadIdx.x / NW, threadIdx.x % NW) owns word w of strip s.
// Output in the tile workspace:
//   labels[n]  for every segment node n (rank order): 1 + global root index
//              when the component stays inside the tile, else -(1 + j) with j
//              the slot of its root in the border-root list;
//   border[j]  global raster index of each root whose component reaches a
//              seam with a neighbouring tile (also initialised as a root in the
//              global union-find array G = labels buffer);
//   records    global root index per seam pixel column/strip (-1: empty).
template <int NW, int HS, bool STATS = false>
__device__ __forceinline__ void merge_tile(const ImageArgs &a, int tile, bool local_only,
                                           SmemMerge &sm, int *err, uint16_t *lslot = nullptr) {
    constexpr int NS = kThreads / NW;
    constexpr int TW = 32 * NW;
    constexpr int TH = NS * HS;
    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int s = tid / NW, w = tid % NW;
    const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
    const int x0 = tx * TW, y0 = ty * TH;
    const int gx = x0 + 32 * w;
    const uint8_t *img_end = a.img + (size_t)g.H * (size_t)g.W;

    // ---- a-1: stage the tile's pixels as bits (nonzero byte = foreground) ----
    uint32_t rows[HS];
#pragma unroll
    for (int j = 0; j < HS; ++j) {
        const int y = y0 + s * HS + j;
        rows[j] = (y < g.H && gx < g.W)
                      ? load_row_bits(a.img, img_end, y, gx, g.W, a.aligned16 != 0, a.level)
                      : 0u;
        if (y < g.H && (x0 / 32 + w) < g.nwg)
            st_policy(a.bits + (size_t)y * g.nwg + (x0 / 32 + w), rows[j], l2_evict_last());
    }
    const uint32_t top = rows[0], bot = rows[HS - 1];
    const uint32_t m = top | bot;
    sm.top[tid] = top;
    sm.bot[tid] = bot;
    uint32_t mL = __shfl_up_sync(0xFFFFFFFFu, m, 1);
    mL = (w > 0) ? (mL >> 31) : 0u;
    const uint32_t st = m & ~((m << 1) | mL);
    int total;
    const int base = block_excl_scan(__popc(st), sm.warp_sums, total);   // syncs: top/bot visible
    sm.base[tid] = (uint16_t)base;
    // segment starts of word o (strip o / NW, word o % NW)
    auto st_of = [&](int o) {
        const uint32_t mo = sm.top[o] | sm.bot[o];
        const uint32_t ml = (o % NW) ? ((sm.top[o - 1] | sm.bot[o - 1]) >> 31) : 0u;
        return mo & ~((mo << 1) | ml);
    };
    // The union queue (entries a | b << 16) lives in the unused ends of P and
    // K, past the tile's segments: at most kQueueCap entries.
    uint32_t *const Q1 = reinterpret_cast<uint32_t *>(sm.P + total);
    const int cap1 = kNodeCap - total;
    const int tot2 = (total + 1) & ~1;
    uint32_t *const Q2 = reinterpret_cast<uint32_t *>(sm.K + tot2);
    const int qcap = min(cap1 + (kNodeCap - tot2) / 2, kQueueCap);
    auto qat = [&](int i) -> uint32_t & { return i < cap1 ? Q1[i] : Q2[i - cap1]; };

    // ---- nodes: parent = self, key = smallest tile-local pixel index ----
    {
        uint32_t rem = st;
        int n = base;
        while (rem) {
            const int i = __ffs(rem) - 1;
            rem &= rem - 1;
            int key;
            if (HS == 2) {
                // the run from bit i inside this word (len <= 32 - i bits)
                const int len = __ffsll(~((unsigned long long)m >> i)) - 1;
                const uint32_t part = (uint32_t)(((1ull << len) - 1ull) << i);
                const uint32_t tp = top & part;
                if (tp) {
                    key = (2 * s) * TW + 32 * w + (__ffs(tp) - 1);
                } else {
                    // no top-row pixel here: the start's bottom pixel, unless the
                    // segment continues and meets a top-row pixel in a later word
                    key = (2 * s + 1) * TW + 32 * w + i;
                    if (i + len == 32) {
                        for (int w2 = w + 1; w2 < NW; ++w2) {
                            const uint32_t t2 = sm.top[tid + (w2 - w)];
                            const uint32_t m2 = t2 | sm.bot[tid + (w2 - w)];
                            const int len2 = __ffsll(~(unsigned long long)m2) - 1;
                            const uint32_t tp2 = t2 & (uint32_t)((1ull << len2) - 1ull);
                            if (tp2) { key = (2 * s) * TW + 32 * w2 + (__ffs(tp2) - 1); break; }
                            if (len2 < 32) break;
                        }
                    }
                }
            } else {
                key = s * TW + 32 * w + i;
            }
            sm.P[n] = (pnode)n;
            sm.K[n] = (uint16_t)key;
            ++n;
        }
    }
    for (int i = tid; i < kNodeCap / 32; i += kThreads) sm.flag[i] = 0u;
    if (tid == 0) { sm.nborder = 0; sm.nq = 0; }
    __syncthreads();

    // ---- a-2: union-find over the segments of the tile ----
    // Contacts join strip s-1 and strip s only.  (1) Every segment takes its
    // first contact as parent (a CAS on a segment that is still its own
    // parent): a forest whose edges all point one strip up, so each tree's
    // root is its smallest key.  A contact whose CAS fails is the union of its
    // upper segment with the parent already taken; it is queued.  (2) Pointer
    // jumping, in lock-step rounds, flattens the forest.  (3) The queued
    // unions are shared out evenly over the block: one CAS hook each of the
    // larger-key root under the smaller; (4) the few that lose a race run as
    // lock-free unions with finds.  (5) Pointer jumping points every node
    // straight at its root.
    int budget = a.hops_smem;
    if (s > 0) {
        const int up = tid - NW;
        const uint32_t av = sm.bot[up];
        const uint32_t bv = sm.top[tid];
        if (bv) {
            const uint32_t aL = w > 0 ? (sm.bot[up - 1] >> 31) : 0u;
            const uint32_t bL = w > 0 ? (sm.top[tid - 1] >> 31) : 0u;
            const int baseA = sm.base[up];
            const uint32_t stA = st_of(up);
            int la = -1, lb = -1;
            auto contact = [&](int ra, int rb) {
                if (ra == la && rb == lb) return;
                la = ra;
                lb = rb;
                const int old = atomicCAS(&sm.P[rb], (pnode)rb, (pnode)ra);
                if (old != rb && old != ra) {
                    const int q = atomicAdd(&sm.nq, 1);
                    if (q < qcap) qat(q) = (uint32_t)ra | ((uint32_t)old << 16);
                    else sunion(sm.P, sm.K, ra, old, budget, err);   // queue full: now
                }
            };
            const uint32_t o = av & bv;
            uint32_t os = o & ~((o << 1) | (aL & bL));
            while (os) {
                const int x = __ffs(os) - 1;
                os &= os - 1;
                contact(seg_rank(baseA, stA, x), seg_rank(base, st, x));
            }
            if (HS == 2) {
                const uint32_t aR = w < NW - 1 ? (sm.bot[up + 1] & 1u) : 0u;
                const uint32_t bR = w < NW - 1 ? (sm.top[tid + 1] & 1u) : 0u;
                const uint32_t stA_next0 = w < NW - 1 ? (st_of(up + 1) & 1u) : 0u;
                // b-run starts at x right after an a-run that ends at x-1
                uint32_t dr = bv & ~av & ~((bv << 1) | bL) & ((av << 1) | aL);
                // b-run ends at x right before an a-run that starts at x+1
                uint32_t dl = bv & ~av & ~((bv >> 1) | (bR << 31)) & ((av >> 1) | (aR << 31));
                while (dr) {
                    const int x = __ffs(dr) - 1;
                    dr &= dr - 1;
                    contact(seg_rank(baseA, stA, x - 1), seg_rank(base, st, x));
                }
                while (dl) {
                    const int x = __ffs(dl) - 1;
                    dl &= dl - 1;
                    contact((x == 31) ? (baseA + __popc(stA) + (int)stA_next0 - 1)
                                      : seg_rank(baseA, stA, x + 1),
                            seg_rank(base, st, x));
                }
            }
        }
    }
    __syncthreads();
    // (2) pointer jumping: every node to the root of its first-contact tree
    volatile pnode *vP = sm.P;
    // Plain loads: within a round any mix of old and new parents is valid
    // (all are ancestors), and the barrier between rounds publishes the stores.
    // A first-contact tree is at most NS - 1 links deep (one per strip), so
    // log2(NS) rounds flatten it; no test round is needed here because the
    // hooks below tolerate a parent that is not a root (the CAS fails and
    // the pair is unioned with finds), and the final jumping tests.
    {
        constexpr int kRounds = NS >= 256 ? 8 : NS >= 128 ? 7 : NS >= 64 ? 6 : 5;
#pragma unroll 1
        for (int round = 0; round < kRounds; ++round) {
#pragma unroll 4
            for (int n = tid; n < total; n += kThreads) {
                const int p = sm.P[n];
                const int gp = sm.P[p];
                if (gp != p) sm.P[n] = (pnode)gp;
            }
            __syncthreads();
        }
    }
    // (3) one round of hooks: each queued pair whose roots differ hooks the
    // root with the larger key under the other (one CAS, no find); a hook
    // that loses a race is queued again with the loser's new parent.  (4) The
    // few pairs that lost run as lock-free unions with finds (path halving).
    constexpr int kPer = kQueueCap / kThreads;   // queue entries per thread
    const int nq0 = min(sm.nq, qcap);            // block-uniform: read after a barrier
    if (nq0 > 0) {
        const int kn = (nq0 + kThreads - 1) / kThreads;   // entries per thread (block-uniform)
        uint32_t e[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (k >= kn) break;
            const int i = tid + k * kThreads;
            e[k] = i < nq0 ? qat(i) : 0xFFFFFFFFu;
        }
        __syncthreads();
        if (tid == 0) sm.nq = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (k >= kn) break;
            if (e[k] == 0xFFFFFFFFu) continue;
            int pa = vP[e[k] & 0xFFFFu], pb = vP[e[k] >> 16];
            if (pa == pb) continue;
            if (sm.K[pa] > sm.K[pb]) { const int t = pa; pa = pb; pb = t; }
            const int old = atomicCAS(&sm.P[pb], (pnode)pb, (pnode)pa);   // hook root pb under pa
            if (old != pb && old != pa) {
                const int q = atomicAdd(&sm.nq, 1);
                if (q < qcap) qat(q) = (uint32_t)pa | ((uint32_t)old << 16);
                else sunion(sm.P, sm.K, pa, old, budget, err);   // queue full: now
            }
        }
        __syncthreads();
        const int nq1 = min(sm.nq, qcap);
        for (int i = tid; i < nq1; i += kThreads) {
            const uint32_t q = qat(i);
            sunion(sm.P, sm.K, (int)(q & 0xFFFFu), (int)(q >> 16), budget, err);
        }
        __syncthreads();
    }
    // (5) pointer jumping until every node points at its root
    for (int round = 0; round < 64; ++round) {
        int changed = 0;
#pragma unroll 4
        for (int n = tid; n < total; n += kThreads) {
            const int p = sm.P[n];
            const int gp = sm.P[p];
            if (gp != p) { sm.P[n] = (pnode)gp; changed = 1; }
        }
        if (!__syncthreads_or(changed)) break;
        if (round == 63) atomicOr(err, kErrSmemFind);
    }

    int *tw_ = a.tws + (size_t)tile * g.tile_ints;
    int *rec = tw_ + g.off_rec;
    auto gkey = [&](int k) -> int {
        const int ly = k >> g.log2tw, lx = k & (TW - 1);
        return (y0 + ly) * g.W + x0 + lx;
    };
    const bool has_up = ty > 0, has_down = ty < g.tiles_y - 1;
    const bool has_left = tx > 0, has_right = tx < g.tiles_x - 1;

    // ---- roots that reach a seam with a neighbouring tile ----
    // Each record position (top/bottom row per column, left/right column per
    // strip) remembers its segment's root; roots of positions that can touch
    // a neighbour are flagged and given a border slot.
    // The first thread to flag a root gives it a border slot and makes it a
    // root node of the global forest (K then holds the slot), so no pass over
    // all nodes is needed to find the flagged roots.
    gnode *par = reinterpret_cast<gnode *>(tw_ + g.off_par);
    auto mark = [&](int r) {
        const uint32_t bit = 1u << (r & 31);
        if (atomicOr(&sm.flag[r >> 5], bit) & bit) return;   // flagged already
        const int j = atomicAdd(&sm.nborder, 1);
        if (j < g.border_cap) {
            const int gk = gkey(sm.K[r]);
            st_policy(tw_ + g.off_key + j, gk, l2_evict_last());
            st_policy(par + j, make_gnode(gk, tile, j), l2_evict_last());
            if (STATS)
                init_border_acc(static_cast<BorderAcc *>(a.bacc) + (size_t)tile * g.border_cap + j);
            sm.K[r] = (uint16_t)j;
        } else {
            atomicOr(err, kErrBorderCap);
        }
    };
    int r_top = -1, r_bot = -1, r_left = -1, r_right = -1;
    if (tid < TW) {
        const int wc = tid >> 5, b = tid & 31;
        {   // top: strip 0
            const int o = wc;
            if ((sm.top[o] | sm.bot[o]) >> b & 1u) {
                r_top = sm.P[seg_rank(sm.base[o], st_of(o), b)];
                if (has_up && !local_only && ((sm.top[o] >> b) & 1u)) mark(r_top);
            }
        }
        {   // bottom: strip NS-1
            const int o = (NS - 1) * NW + wc;
            if ((sm.top[o] | sm.bot[o]) >> b & 1u) {
                r_bot = sm.P[seg_rank(sm.base[o], st_of(o), b)];
                if (has_down && !local_only && ((sm.bot[o] >> b) & 1u)) mark(r_bot);
            }
        }
    }
    if (tid < NS) {
        {   // left: column 0 of strip tid (always a segment start when set)
            const int o = tid * NW;
            if ((sm.top[o] | sm.bot[o]) & 1u) {
                r_left = sm.P[sm.base[o]];
                if (has_left && !local_only) mark(r_left);
            }
        }
        {   // right: column TW-1 of strip tid
            const int o = tid * NW + NW - 1;
            if ((sm.top[o] | sm.bot[o]) >> 31) {
                r_right = sm.P[seg_rank(sm.base[o], st_of(o), 31)];
                if (has_right && !local_only) mark(r_right);
            }
        }
    }
    __syncthreads();
    auto flagged = [&](int r) { return (sm.flag[r >> 5] >> (r & 31)) & 1u; };

    // ---- seam records: the global node of each position's root ----
    long long *rec64 = reinterpret_cast<long long *>(rec);
    auto node_of = [&](int r) {
        return (r >= 0 && flagged(r)) ? (long long)make_gnode(tw_[g.off_key + sm.K[r]], tile, sm.K[r])
                                      : (long long)kNoNode;
    };
    if (tid < TW) {
        st_policy(rec64 + tid, node_of(r_top), l2_evict_last());
        st_policy(rec64 + TW + tid, node_of(r_bot), l2_evict_last());
    }
    if (tid < NS) {
        st_policy(rec64 + 2 * TW + tid, node_of(r_left), l2_evict_last());
        st_policy(rec64 + 2 * TW + NS + tid, node_of(r_right), l2_evict_last());
    }

    // ---- per-segment labels ----
    if (!STATS) {
        for (int n = tid; n < total; n += kThreads) {
            const int r = sm.P[n];
            const int k = sm.K[r];
            st_policy(tw_ + kHdrInts + n, flagged(r) ? -(1 + k) : 1 + gkey(k), l2_evict_last());
        }
    } else {
        // Statistics: every component inside the tile gets an output record
        // (a slot in a range reserved with one atomic per tile) holding its
        // label; each segment also stores its component's slot, local (>= 0)
        // or border (-(1 + border slot)), for the link phase.
        if (tid == 0) sm.nlocal = 0;
        __syncthreads();
        for (int n = tid; n < total; n += kThreads)
            if (sm.P[n] == n && !flagged(n)) lslot[n] = (uint16_t)atomicAdd(&sm.nlocal, 1);
        __syncthreads();
        if (tid == 0) sm.out_base = sm.nlocal ? atomicAdd(a.ncomps, sm.nlocal) : 0;
        __syncthreads();
        const int ob = sm.out_base;
        CompRec *recs = static_cast<CompRec *>(a.comps);
        uint16_t *cs = a.cslot + (size_t)tile * cslot_stride(g);
        for (int n = tid; n < total; n += kThreads) {
            const int r = sm.P[n];
            const int k = sm.K[r];
            const bool f = flagged(r) != 0u;
            st_policy(tw_ + kHdrInts + n, f ? -(1 + k) : 1 + gkey(k), l2_evict_last());
            cs[n] = f ? (uint16_t)(kSlotBorder | k) : lslot[r];
            if (r == n && !f) {
                const long long o = (long long)ob + lslot[n];
                if (o < a.max_comps) {
                    if (lslot[n] < kStatLocal) {   // the statistics flush writes the rest
                        recs[o].label = 1 + gkey(k);
                    } else {                       // added into with atomics: initialise
                        CompRec c;
                        c.label = 1 + gkey(k);
                        c.count = 0;
                        c.xmin = c.ymin = 0x7FFFFFFF;
                        c.xmax = c.ymax = -1;
                        c.sum_x = c.sum_y = 0;
                        recs[o] = c;
                    }
                }
            }
        }
        if (tid == 0) {
            tw_[2] = ob;
            tw_[3] = sm.nlocal;
        }
    }
    if (tid == 0) {
        tw_[0] = local_only ? 0 : min(sm.nborder, g.border_cap);
        tw_[1] = total;
    }
}

// ---------------------------------------------------------------------------
// Kernel 2 body: seam unions (§II-B).  Work items: 4-column groups of the
// horizontal seams (rows y-1, y with y = ty*TH), (tiles_y-1)*nwg*8 of them,
// padded to a multiple of 256 so that no warp or 256-item chunk mixes the two
// kinds; then
// one item per strip of each vertical seam, (tiles_x-1)*tiles_y*NS.  Each
// touching pair of runs across a seam yields one union of the two local roots
// (deduplicated per warp, see seam_block).
__device__ __forceinline__ uint32_t bit_at(const uint32_t *bits, int nwg, int y, int x) {
    return (__ldcg(bits + (size_t)y * nwg + (x >> 5)) >> (x & 31)) & 1u;
}

// horizontal seam items cover kGroupCols = 4 columns each (8 per 32-bit
// word): about one contact per thread at p = 0.5, and few enough live
// records (6 above, 4 below) that the kernel holds 4 blocks per SM
constexpr int kSeamGroupsPerWord = 8;
constexpr int kGroupCols = 32 / kSeamGroupsPerWord;

__host__ __device__ inline long long seam_h_real(const Geom &g) {
    return (long long)(g.tiles_y - 1) * g.nwg * kSeamGroupsPerWord;
}

__host__ __device__ inline long long seam_h_items(const Geom &g) {
    return (seam_h_real(g) + 255) / 256 * 256;
}

__host__ __device__ inline long long seam_items(const Geom &g) {
    return seam_h_items(g) + (long long)(g.tiles_x - 1) * g.tiles_y * g.ns;
}

// Seam unions of one block of 256 items, warp by warp.  Each lane lists the
// pairs (local root above/left, local root below/right) of its item's
// contacts, dropping a pair equal to its previous one and a first pair equal
// to the previous lane's last; one warp scan packs all lanes' pairs into the
// warp's list.  The list is then deduplicated 32 entries at a time
// (__match_any_sync; the first of equal pairs is kept, in place), and the
// lanes run the remaining unions in parallel.  One component crossing a seam
// many times yields the same pair over and over, so a warp costs about one
// union's chain of dependent global loads instead of one per contact.
constexpr int kSeamList = 128;   // pairs per warp before falling back to direct unions

struct SmemSeams {
    gnode list[kThreads / 32][kSeamList][2];
};

// Warp-wide exclusive scan of c; `total` gets the warp's sum.
__device__ __forceinline__ int warp_excl_scan(int c, int &total) {
    const int lane = threadIdx.x & 31;
    int x = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    total = __shfl_sync(0xFFFFFFFFu, x, 31);
    return x - c;
}

// Drops the lane's first kept pair (lowest bit of `keep`) when it equals the
// previous lane's last kept pair (la, lb); the previous lane's pair, or one
// equal to it further left, stays listed.
__device__ __forceinline__ uint32_t drop_left_repeat(uint32_t keep, gnode fa, gnode fb, gnode la,
                                                     gnode lb) {
    const gnode pa = __shfl_up_sync(0xFFFFFFFFu, la, 1);
    const gnode pb = __shfl_up_sync(0xFFFFFFFFu, lb, 1);
    if ((threadIdx.x & 31) > 0 && keep && fa == pa && fb == pb) keep &= keep - 1u;
    return keep;
}

// One block of 256 seam items; every lane of every warp must call it.  Items
// of one warp are all horizontal (4-column groups of a seam row pair) or all
// vertical (strips of a column seam).
__device__ __forceinline__ void seam_block(const ImageArgs &a, long long idx0, long long nitems,
                                           SmemSeams &sm, int *err) {
    const Geom &g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GlobalForest F{a.tws, g.tile_ints, g.off_par};
    int budget = a.hops_glob;
    gnode(*list)[2] = sm.list[warp];
    int n = 0;   // warp-uniform list length
    const long long idx = idx0 + threadIdx.x;
    const long long nh_real = seam_h_real(g);
    const long long nh = seam_h_items(g);
    bool bad = false;   // a contact without a record: a border root was dropped
    if (idx0 < nh) {
        // ---- horizontal: columns [c0, c0 + kGroupCols) of rows y-1 (a) and y (b) ----
        constexpr int GC = kGroupCols;
        uint32_t os = 0, dr = 0, dl = 0;
        gnode u[GC + 2], d[GC];   // records of columns c0-1 .. c0+GC above, c0 .. c0+GC-1 below
#pragma unroll
        for (int k = 0; k < GC + 2; ++k) u[k] = kNoNode;
#pragma unroll
        for (int k = 0; k < GC; ++k) d[k] = kNoNode;
        if (idx < nh_real) {
            // item counts stay below 2^32 (H * W <= 2^31 - 2): 32-bit division
            const unsigned per_row = (unsigned)g.nwg * kSeamGroupsPerWord;
            const int ty = (int)((unsigned)idx / per_row) + 1;
            const int grp = (int)((unsigned)idx % per_row);
            const int j = grp / kSeamGroupsPerWord;
            const int sh = GC * (grp % kSeamGroupsPerWord);
            const int c0 = 32 * j + sh;
            const int y = ty * g.th;
            const uint32_t *ra_ = a.bits + (size_t)(y - 1) * g.nwg;
            const uint32_t *rb_ = a.bits + (size_t)y * g.nwg;
            const long long *up = reinterpret_cast<const long long *>(
                                      a.tws + (size_t)(ty - 1) * g.tiles_x * g.tile_ints + g.off_rec) + g.tw;
            const long long *dn = reinterpret_cast<const long long *>(
                                      a.tws + (size_t)ty * g.tiles_x * g.tile_ints + g.off_rec);
            auto rec = [&](const long long *b, int xg) -> gnode {
                return (xg >= 0 && xg < g.W)
                           ? (gnode)__ldcg(b + (size_t)(xg >> g.log2tw) * (g.tile_ints / 2) + (xg & (g.tw - 1)))
                           : kNoNode;
            };
            // one round of independent loads
            const uint32_t av = __ldcg(ra_ + j), bv = __ldcg(rb_ + j);
            const uint32_t aW = j > 0 ? __ldcg(ra_ + j - 1) : 0u, bW = j > 0 ? __ldcg(rb_ + j - 1) : 0u;
            const uint32_t aE = j < g.nwg - 1 ? __ldcg(ra_ + j + 1) : 0u;
            const uint32_t bE = j < g.nwg - 1 ? __ldcg(rb_ + j + 1) : 0u;
#pragma unroll
            for (int k = 0; k < GC + 2; ++k) u[k] = rec(up, c0 - 1 + k);
#pragma unroll
            for (int k = 0; k < GC; ++k) d[k] = rec(dn, c0 + k);
            const uint32_t aL = aW >> 31, bL = bW >> 31, aR = aE & 1u, bR = bE & 1u;
            const uint32_t o = av & bv;
            const uint32_t gm = ((1u << GC) - 1u) << sh;
            os = (o & ~((o << 1) | (aL & bL)) & gm) >> sh;
            if (g.hs == 2) {
                dr = ((bv & ~av & ~((bv << 1) | bL) & ((av << 1) | aL)) & gm) >> sh;
                dl = ((bv & ~av & ~((bv >> 1) | (bR << 31)) & ((av >> 1) | (aR << 31))) & gm) >> sh;
            }
        }
        // two pair slots per column, bit 2c + kind of `keep`: kind 0 is the
        // overlap or down-right contact at column c0 + c, kind 1 the down-left
        auto pair_of = [&](int c, int kind, gnode &ka, gnode &kb) {
            kb = d[c];
            ka = kind == 0 ? (((os >> c) & 1u) ? u[c + 1] : u[c]) : u[c + 2];
        };
        uint32_t keep = 0u;
        gnode fa = kNoNode, fb = kNoNode, la = kNoNode, lb = kNoNode;
#pragma unroll
        for (int c = 0; c < GC; ++c) {
#pragma unroll
            for (int kind = 0; kind < 2; ++kind) {
                bool have = kind == 0 ? (((os | dr) >> c) & 1u) : ((dl >> c) & 1u);
                gnode ka, kb;
                pair_of(c, kind, ka, kb);
                if (have && (ka == kNoNode || kb == kNoNode)) { bad = true; have = false; }
                if (have && ka == la && kb == lb) have = false;
                if (have) {
                    if (keep == 0u) { fa = ka; fb = kb; }
                    la = ka;
                    lb = kb;
                    keep |= 1u << (2 * c + kind);
                }
            }
        }
        keep = drop_left_repeat(keep, fa, fb, la, lb);
        int slot = warp_excl_scan(__popc(keep), n);
#pragma unroll
        for (int c = 0; c < GC; ++c) {
#pragma unroll
            for (int kind = 0; kind < 2; ++kind) {
                if ((keep >> (2 * c + kind)) & 1u) {
                    gnode ka, kb;
                    pair_of(c, kind, ka, kb);
                    if (slot < kSeamList) { list[slot][0] = ka; list[slot][1] = kb; }
                    else gunion(F, ka, kb, budget, err);   // list full: union now
                    ++slot;
                }
            }
        }
    } else {
        // ---- vertical: strip s of the seam between tiles tx-1 and tx ----
        bool h0 = false, h1 = false, h2 = false;
        gnode kL = kNoNode, kR = kNoNode, kLu = kNoNode, kRu = kNoNode;
        if (idx < nitems) {
            const unsigned v = (unsigned)(idx - nh);
            const int s = (int)(v % (unsigned)g.ns);
            const unsigned t = v / (unsigned)g.ns;
            const int ty = (int)(t % (unsigned)g.tiles_y);
            const int tx = (int)(t / (unsigned)g.tiles_y) + 1;
            const int x = tx * g.tw;
            const int r0 = ty * g.th + s * g.hs;
            if (r0 < g.H) {
                const long long tL = (long long)ty * g.tiles_x + (tx - 1), tR = tL + 1;
                const long long *recL = reinterpret_cast<const long long *>(
                                            a.tws + (size_t)tL * g.tile_ints + g.off_rec) + 2 * g.tw + g.ns;
                const long long *recR = reinterpret_cast<const long long *>(
                                            a.tws + (size_t)tR * g.tile_ints + g.off_rec) + 2 * g.tw;
                const int wq = x >> 5;   // x is a multiple of 32: column x-1 is bit 31 of word wq-1
                const uint32_t *row0 = a.bits + (size_t)r0 * g.nwg;
                const uint32_t A0 = __ldcg(row0 + wq - 1), B0 = __ldcg(row0 + wq);
                uint32_t A1 = 0, B1 = 0, Au = 0, Bu = 0;
                if (g.hs == 2 && r0 + 1 < g.H) {
                    A1 = __ldcg(row0 + g.nwg + wq - 1);
                    B1 = __ldcg(row0 + g.nwg + wq);
                }
                const bool diag = g.hs == 2 && s > 0;
                if (diag) {
                    Au = __ldcg(row0 - g.nwg + wq - 1);
                    Bu = __ldcg(row0 - g.nwg + wq);
                    kLu = (gnode)__ldcg(recL + s - 1);
                    kRu = (gnode)__ldcg(recR + s - 1);
                }
                kL = (gnode)__ldcg(recL + s);
                kR = (gnode)__ldcg(recR + s);
                const uint32_t l0 = A0 >> 31, l1 = A1 >> 31, lu = Au >> 31;
                const uint32_t rr0 = B0 & 1u, rr1 = B1 & 1u, ru = Bu & 1u;
                h0 = (l0 | l1) && (rr0 | rr1);
                // diagonals between the last row of strip s-1 and the first of strip s
                h1 = diag && lu && rr0;
                h2 = diag && l0 && ru;
            }
        }
        // pair k: 0 = (kLu, kR), 1 = (kL, kRu), 2 = (kL, kR), in this order
        auto pair_of = [&](int k, gnode &ka, gnode &kb) {
            ka = k == 0 ? kLu : kL;
            kb = k == 1 ? kRu : kR;
        };
        uint32_t keep = 0u;
        gnode fa = kNoNode, fb = kNoNode, la = kNoNode, lb = kNoNode;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            bool have = k == 0 ? h1 : (k == 1 ? h2 : h0);
            gnode ka, kb;
            pair_of(k, ka, kb);
            if (have && (ka == kNoNode || kb == kNoNode)) { bad = true; have = false; }
            if (have && ka == la && kb == lb) have = false;
            if (have) {
                if (keep == 0u) { fa = ka; fb = kb; }
                la = ka;
                lb = kb;
                keep |= 1u << k;
            }
        }
        keep = drop_left_repeat(keep, fa, fb, la, lb);
        int slot = warp_excl_scan(__popc(keep), n);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if ((keep >> k) & 1u) {
                gnode ka, kb;
                pair_of(k, ka, kb);
                if (slot < kSeamList) { list[slot][0] = ka; list[slot][1] = kb; }
                else gunion(F, ka, kb, budget, err);   // list full: union now
                ++slot;
            }
        }
    }
    if (bad) atomicOr(err, kErrBorderCap);
    __syncwarp();
    // deduplicate the list 32 entries at a time, in place: of equal pairs
    // within a chunk the lowest lane's stays.  Pairs are compared folded into
    // 64 bits; a lane whose pair differs from its elected lane's (a
    // collision) stays too.
    const int m = n < kSeamList ? n : kSeamList;
    int nu = 0;   // warp-uniform count of kept pairs
    for (int i0 = 0; i0 < m; i0 += 32) {
        const int i = i0 + lane;
        const bool have = i < m;
        const gnode ka = have ? list[i][0] : kNoNode;
        const gnode kb = have ? list[i][1] : kNoNode;
        const unsigned long long key = have ? (ka * 0x9E3779B97F4A7C15ull) ^ kb : ~0ull;
        const unsigned same = __match_any_sync(0xFFFFFFFFu, key);
        const int first = __ffs(same) - 1;
        const gnode ea = __shfl_sync(0xFFFFFFFFu, ka, first);
        const gnode eb = __shfl_sync(0xFFFFFFFFu, kb, first);
        const bool keepit = have && (first == lane || ea != ka || eb != kb);
        const unsigned km = __ballot_sync(0xFFFFFFFFu, keepit);
        __syncwarp();   // every lane has read its entry before any is overwritten
        if (keepit) {
            const int o = nu + __popc(km & ((1u << lane) - 1u));   // o <= i
            list[o][0] = ka;
            list[o][1] = kb;
        }
        nu += __popc(km);
    }
    __syncwarp();
    for (int i = lane; i < nu; i += 32) gunion(F, list[i][0], list[i][1], budget, err);
}

// ---------------------------------------------------------------------------
// Link body (§II-C): re-derive the segments of the tile from the bit image,
// give every segment its final label (its local root's, or the resolved label
// of its border root), and write one int32 per pixel.  The stores are laid
// out so that 32 lanes write 128 consecutive pixels (512 bytes) of one row.
// STATS: also gather the component statistics of the tile, in the same
// blocks (ccl_label_with_stats).
template <int NW, int HS, bool STATS = false>
__device__ __forceinline__ void link_tile(const ImageArgs &a, int tile, int *S, SmemLinkCore &sm,
                                          int *err, SmemLinkStats *sx = nullptr) {
    constexpr int NS = kThreads / NW;
    constexpr int TW = 32 * NW;
    constexpr int TH = NS * HS;
    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int s = tid / NW, w = tid % NW;
    const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
    const int x0 = tx * TW, y0 = ty * TH;
    const int gwi = x0 / 32 + w;

    const int *tw_ = a.tws + (size_t)tile * g.tile_ints;
    const int nb = min(__ldcg(tw_), g.border_cap);
    const int nseg = min(__ldcg(tw_ + 1), kNodeCap);
    uint32_t rows[HS];
#pragma unroll
    for (int j = 0; j < HS; ++j) {
        const int y = y0 + s * HS + j;
        rows[j] = (y < g.H && gwi < g.nwg) ? __ldcg(a.bits + (size_t)y * g.nwg + gwi) : 0u;
    }
    // the per-segment labels, copied to shared memory asynchronously
    // (16-byte cp.async; the source starts 16 bytes into the 256-byte aligned
    // tile workspace, and rounding the count up stays inside the workspace)
    for (int c = tid; c < (nseg + 3) / 4; c += kThreads) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&S[4 * c]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                     "l"(tw_ + kHdrInts + 4 * c) : "memory");
    }
    if (STATS) {   // the segments' component slots, the same way
        const uint16_t *cs = a.cslot + (size_t)tile * cslot_stride(g);
        for (int c = tid; c < (nseg + 7) / 8; c += kThreads) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&sx->C[8 * c]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(cs + 8 * c)
                         : "memory");
        }
        if (tid == 0) sx->nroots = 0;
        for (int i = tid; i < kStatLocal + kStatBorder; i += kThreads) {
            unsigned *e = i < kStatLocal ? sx->LA[i] : sx->BA[i - kStatLocal];
            e[0] = 0u;
            e[1] = e[2] = 0xFFFFFFFFu;
            e[3] = e[4] = 0u;
            e[5] = e[6] = 0u;
        }
        for (int i = tid; i < kStatHash; i += kThreads) sx->HK[i] = kNoSite;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
#pragma unroll
    for (int j = 0; j < HS; ++j) sm.rows[(s * HS + j) * NW + w] = rows[j];
    const uint32_t m = rows[0] | rows[HS - 1];
    uint32_t mL = __shfl_up_sync(0xFFFFFFFFu, m, 1);
    mL = (w > 0) ? (mL >> 31) : 0u;
    const uint32_t st = m & ~((m << 1) | mL);
    // final label of each border root: 1 + the key of its global root (a
    // read-only walk, usually one or two hops).  Everything above reads only
    // the local-merge output; the walk needs the seam unions complete, so a
    // grid launched early (programmatic dependent launch) waits here.
    pdl_wait();
    {
        const GlobalForest F{a.tws, g.tile_ints, g.off_par};
        const gnode *par = reinterpret_cast<const gnode *>(tw_ + g.off_par);
        int budget = a.hops_glob;
        for (int j = tid; j < nb; j += kThreads) {
            gnode r = __ldcg(par + j);
            for (;;) {
                if (--budget < 0) { atomicOr(err, kErrGlobFind); break; }
                const gnode p = __ldcg(F.par(r));
                if (p == r) break;
                r = p;
            }
            sm.R[j] = 1 + gnode_key(r);
            if (STATS) sx->G[j] = gnode_site(r);
        }
    }
    int total;
    const int base = block_excl_scan(__popc(st), sm.warp_sums, total);   // syncs: R visible
    sm.st[tid] = st;
    sm.base[tid] = base;
    if (STATS) {
        // border roots of this tile with the same global root share one
        // aggregate: a hash table on the global root gives each distinct root
        // an index, taken by the thread that inserts it
        for (int j = tid; j < nb; j += kThreads) {
            const uint32_t r = sx->G[j];
            unsigned h = (r * 0x9E3779B1u) >> 22;   // 10 bits: kStatHash entries
            for (int probe = 0; probe < kStatHash; ++probe, h = (h + 1) & (kStatHash - 1)) {
                const uint32_t old = atomicCAS(&sx->HK[h], kNoSite, r);
                if (old == kNoSite) {
                    const int id = atomicAdd(&sx->nroots, 1);
                    sx->HV[h] = (uint16_t)id;
                    sx->HR[id] = (uint16_t)h;
                    break;
                }
                if (old == r) break;
            }
            sx->HJ[j] = (uint16_t)h;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // every thread's copies of S have landed
    if (total != nseg) { if (tid == 0) atomicOr(err, kErrBorderCap); }
    for (int n = tid; n < total; n += kThreads) {
        const int v = S[n];
        if (v < 0) {
            const int j = -v - 1;
            if (j < nb) {
                S[n] = sm.R[j];
            } else {
                S[n] = 0;
                atomicOr(err, kErrBorderCap);
            }
        }
    }
    // statistics: each border slot's hash entry becomes its aggregate index
    for (int j = tid; STATS && j < nb; j += kThreads) sx->HJ[j] = sx->HV[sx->HJ[j]];
    __syncthreads();

    if (STATS) {
        // Statistics of every piece of a segment inside this thread's word (the
        // segments starting here, and the part of one continuing from the word
        // before), from its pixels' bits: count, bounding box, coordinate sums.
        // Aggregated per component in shared memory (components beyond the
        // shared tables go straight to their global records), then flushed:
        // a component inside the tile writes its record, a border component
        // adds into the accumulator of its global root.
        const int ob = __ldcg(tw_ + 2), nloc = __ldcg(tw_ + 3);
        CompRec *recs = static_cast<CompRec *>(a.comps);
        BorderAcc *bacc = static_cast<BorderAcc *>(a.bacc);
        auto root_acc = [&](uint32_t r) {   // a global root's site
            return bacc + (size_t)(r >> kSlotBits) * g.border_cap + (int)(r & ((1u << kSlotBits) - 1u));
        };
        // A thread adds up its pieces in registers: the first component it
        // meets that crosses the tile border (in a dense image, the large
        // component most pieces belong to) gathers its pieces' pixel masks and
        // takes their statistics once, from the word's rows; one accumulator
        // holds the current run of pieces of any other component, flushed when
        // the component changes.  The crossing one is flushed at the end with
        // warp reductions among the lanes that hold the same component.
        struct Agg {
            int c;   // component: >= 0 inside the tile, < 0: -(1 + aggregate index)
            unsigned cnt, xmn, ymn, xmx, ymx, sx, sy;
        };
        auto add_to = [&](Agg &d, unsigned cnt, unsigned xmn, unsigned ymn, unsigned xmx,
                          unsigned ymx, unsigned sxl, unsigned syl) {
            d.cnt += cnt;
            d.xmn = min(d.xmn, xmn);
            d.ymn = min(d.ymn, ymn);
            d.xmx = max(d.xmx, xmx);
            d.ymx = max(d.ymx, ymx);
            d.sx += sxl;
            d.sy += syl;
        };
        // one aggregate into the shared tables, or its global record when
        // the tables are full
        auto flush = [&](const Agg &d) {
            const int c = d.c;
            unsigned *e = nullptr;
            if (c >= 0 && c < kStatLocal) e = sx->LA[c];
            else if (c < 0 && -c - 1 < kStatBorder) e = sx->BA[-c - 1];
            if (e) {
                atomicAdd(e + 0, d.cnt);
                atomicMin(e + 1, d.xmn);
                atomicMin(e + 2, d.ymn);
                atomicMax(e + 3, d.xmx);
                atomicMax(e + 4, d.ymx);
                atomicAdd(e + 5, d.sx);
                atomicAdd(e + 6, d.sy);
            } else if (c >= 0) {   // a component inside the tile, past the shared table
                if ((long long)ob + c < a.max_comps) {
                    CompRec *rc = recs + ob + c;
                    atomicAdd(&rc->count, (int)d.cnt);
                    atomicMin(&rc->xmin, x0 + (int)d.xmn);
                    atomicMin(&rc->ymin, y0 + (int)d.ymn);
                    atomicMax(&rc->xmax, x0 + (int)d.xmx);
                    atomicMax(&rc->ymax, y0 + (int)d.ymx);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&rc->sum_x),
                              (unsigned long long)d.sx + (unsigned long long)x0 * d.cnt);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&rc->sum_y),
                              (unsigned long long)d.sy + (unsigned long long)y0 * d.cnt);
                }
            } else {               // a global root past the shared table
                const int id = -c - 1;
                if (id < nb) {
                    BorderAcc *tacc = root_acc(sx->HK[sx->HR[id]]);
                    atomicAdd(&tacc->count, d.cnt);
                    atomicMin(&tacc->xmin, x0 + (int)d.xmn);
                    atomicMin(&tacc->ymin, y0 + (int)d.ymn);
                    atomicMax(&tacc->xmax, x0 + (int)d.xmx);
                    atomicMax(&tacc->ymax, y0 + (int)d.ymx);
                    atomicAdd(&tacc->sum_x, (unsigned long long)d.sx + (unsigned long long)x0 * d.cnt);
                    atomicAdd(&tacc->sum_y, (unsigned long long)d.sy + (unsigned long long)y0 * d.cnt);
                }
            }
        };
        Agg A{0x7FFFFFFF, 0u, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u, 0u};
        Agg B = A;
        const bool has_pre = mL && (m & 1u) && base >= 1;
        const uint32_t pre = has_pre ? (m & ~(m + 1u)) : 0u;   // run continuing from the word before
        const int xw = 32 * w, ys = s * HS;
        // statistics of the pixels of this word's rows under `mask`
        auto piece = [&](uint32_t mask, unsigned &cnt, unsigned &xmn, unsigned &ymn,
                         unsigned &xmx, unsigned &ymx, unsigned &sxl, unsigned &syl) {
            const uint32_t tt = rows[0] & mask, bb = HS == 2 ? (rows[HS - 1] & mask) : 0u;
            const uint32_t any = tt | bb;
            const int ct = __popc(tt), cb = __popc(bb);
            cnt = (unsigned)(ct + cb);
            sxl = (unsigned)(xw * (ct + cb) + bit_position_sum(tt) + bit_position_sum(bb));
            syl = (unsigned)(ys * ct + (ys + 1) * cb);
            xmn = (unsigned)(xw + __ffs(any) - 1);
            xmx = (unsigned)(xw + 31 - __clz(any));
            ymn = ct ? ys : ys + 1;
            ymx = cb ? ys + 1 : ys;
        };
        // component of piece n (a segment rank): >= 0 inside the tile,
        // < 0: -(1 + aggregate index) of a border root
        auto comp_of = [&](int n) {
            const unsigned cv = sx->C[n];
            if (!(cv & kSlotBorder)) return (int)cv;
            const int j = (int)(cv & (kSlotBorder - 1u));
            return -1 - (int)sx->HJ[j < nb ? j : 0];
        };
        // First pass, cheap and nearly uniform across the warp: the component
        // of every piece; B takes the first crossing one, and the start bits
        // of the other components' pieces (bit 0 for the piece continuing
        // from the word before) are set aside.
        uint32_t other = 0u;
        if (has_pre) {
            const int c = comp_of(base - 1);
            if (c < 0) B.c = c;
            else other |= 1u;
        }
        {
            int n = base;
            for (uint32_t rem = st; rem; rem &= rem - 1, ++n) {
                const uint32_t bit = rem & (0u - rem);
                if (n >= total) { other |= bit; continue; }
                const int c = comp_of(n);
                if (c < 0 && B.c == 0x7FFFFFFF) B.c = c;
                if (c != B.c) other |= bit;
            }
        }
        // Second pass, over the other pieces only: their statistics, added
        // run by run of one component; B's pixels are the word's others.
        uint32_t omask = 0u;
        for (uint32_t rem = other; rem; rem &= rem - 1) {
            const int i = __ffs(rem) - 1;
            int n;
            uint32_t mask;
            if (i == 0 && has_pre) {
                n = base - 1;
                mask = pre;
            } else {
                n = base + __popc(st & ((1u << i) - 1u));
                const uint32_t z = ~m & (0xFFFFFFFFu << i);
                const int end = z ? __ffs(z) - 1 : 32;
                mask = __funnelshift_lc(0xFFFFFFFFu, 0u, (unsigned)end) & (0xFFFFFFFFu << i);
            }
            omask |= mask;
            if (n >= total) continue;
            const int c = comp_of(n);
            unsigned cnt, xmn, ymn, xmx, ymx, sxl, syl;
            piece(mask, cnt, xmn, ymn, xmx, ymx, sxl, syl);
            if (c != A.c) {
                if (A.c != 0x7FFFFFFF) flush(A);
                A = Agg{c, 0u, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u, 0u};
            }
            add_to(A, cnt, xmn, ymn, xmx, ymx, sxl, syl);
        }
        const uint32_t bmask = B.c != 0x7FFFFFFF ? (m & ~omask) : 0u;
        if (bmask) piece(bmask, B.cnt, B.xmn, B.ymn, B.xmx, B.ymx, B.sx, B.sy);
        if (A.c != 0x7FFFFFFF) flush(A);
        {
            const bool hb = B.c != 0x7FFFFFFF;
            const unsigned am = __ballot_sync(0xFFFFFFFFu, hb);
            if (hb) {
                const unsigned gm = __match_any_sync(am, B.c);
                B.cnt = __reduce_add_sync(gm, B.cnt);
                B.sx = __reduce_add_sync(gm, B.sx);
                B.sy = __reduce_add_sync(gm, B.sy);
                B.xmn = __reduce_min_sync(gm, B.xmn);
                B.ymn = __reduce_min_sync(gm, B.ymn);
                B.xmx = __reduce_max_sync(gm, B.xmx);
                B.ymx = __reduce_max_sync(gm, B.ymx);
                if ((tid & 31) == __ffs(gm) - 1) flush(B);
            }
        }
        __syncthreads();
        for (int l = tid; l < min(nloc, kStatLocal); l += kThreads) {
            if ((long long)ob + l >= a.max_comps) continue;
            const unsigned *e = sx->LA[l];
            CompRec *rc = recs + ob + l;
            const int cnt = (int)e[0];
            rc->count = cnt;
            rc->xmin = x0 + (int)e[1];
            rc->ymin = y0 + (int)e[2];
            rc->xmax = x0 + (int)e[3];
            rc->ymax = y0 + (int)e[4];
            rc->sum_x = (long long)e[5] + (long long)x0 * cnt;
            rc->sum_y = (long long)e[6] + (long long)y0 * cnt;
        }
        for (int h = tid; h < kStatHash; h += kThreads) {
            const uint32_t r = sx->HK[h];
            if (r == kNoSite || sx->HV[h] >= kStatBorder) continue;
            const unsigned *e = sx->BA[sx->HV[h]];
            if (e[0] == 0u) continue;
            BorderAcc *t = root_acc(r);
            atomicAdd(&t->count, e[0]);
            atomicMin(&t->xmin, x0 + (int)e[1]);
            atomicMin(&t->ymin, y0 + (int)e[2]);
            atomicMax(&t->xmax, x0 + (int)e[3]);
            atomicMax(&t->ymax, y0 + (int)e[4]);
            atomicAdd(&t->sum_x, (unsigned long long)e[5] + (unsigned long long)x0 * e[0]);
            atomicAdd(&t->sum_y, (unsigned long long)e[6] + (unsigned long long)y0 * e[0]);
        }
    }

    const int ncols = min(TW, g.W - x0);   // valid columns of this tile
    const int nrows = min(TH, g.H - y0);
    if (a.out_aligned16 && (ncols & 3) == 0) {
        // chunk = 4 pixels; a row has TW/4 chunks
        constexpr int CPR = TW / 4;
        for (int id = tid; id < TH * CPR; id += kThreads) {
            const int r = id / CPR, q = id % CPR;
            const int c0 = 4 * q;
            if (r >= nrows || c0 >= ncols) continue;
            const int wq = c0 >> 5, b0 = c0 & 31;
            const int o = (r / HS) * NW + wq;
            const uint32_t rb = sm.rows[r * NW + wq];
            const uint32_t sq = sm.st[o];
            int cur = sm.base[o] + __popc(sq & le_mask(b0)) - 1;
            int32_t *out = a.labels + (size_t)(y0 + r) * g.W + x0 + c0;
            int v[4] = {0, 0, 0, 0};
            if (a.merge_out) {   // keep the pixels this pass does not label
                const int4 keep = *reinterpret_cast<const int4 *>(out);
                v[0] = keep.x; v[1] = keep.y; v[2] = keep.z; v[3] = keep.w;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e > 0) cur += (sq >> (b0 + e)) & 1u;
                if ((rb >> (b0 + e)) & 1u) v[e] = S[cur < 0 ? 0 : cur];
            }
            __stcs(reinterpret_cast<int4 *>(out), make_int4(v[0], v[1], v[2], v[3]));
        }
    } else {
        // rows not 16-byte aligned (W % 4 != 0 or an unaligned label pointer):
        // one label per thread and step, 32 lanes writing 128 consecutive bytes
        for (int id = tid; id < TH * TW; id += kThreads) {
            const int r = id / TW, c = id % TW;
            if (r >= nrows || c >= ncols) continue;
            const int wq = c >> 5, b = c & 31;
            const int o = (r / HS) * NW + wq;
            const uint32_t rb = sm.rows[r * NW + wq];
            const uint32_t sq = sm.st[o];
            const int cur = sm.base[o] + __popc(sq & le_mask(b)) - 1;
            int32_t *out = a.labels + (size_t)(y0 + r) * g.W + x0 + c;
            if ((rb >> b) & 1u) *out = S[cur < 0 ? 0 : cur];
            else if (!a.merge_out) *out = 0;
        }
    }
}

}  // namespace ccl
