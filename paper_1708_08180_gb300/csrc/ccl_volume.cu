// ccl_volume.cu -- labelling of 3-D volumes (the "2D/3D grid" of §I) with the
// paper's three phases one dimension up: tiles become bricks, tile seams become
// brick faces.
//   * A strip is SY x SZ neighbouring rows (one row at 6-connectivity, two rows
//     along y at 18, 2 x 2 rows at 26), read as one 32-voxel word per row.
//     Every run of ones of the OR of a strip's rows is connected (its voxels at
//     x and x + 1 are neighbours whatever their rows), so the runs of the OR,
//     "segments", are the union-find nodes.  A brick is one word along x by
//     16 x 16 strips; thread t of a block owns strip (t % 16, t / 16).
//   * local merge (Kernel 1, §II-A): a block joins the segments of its brick in
//     shared memory, each strip with its earlier neighbour strips through the
//     rows that face each other: contacts listed per segment (or per overlap
//     run where x must match), first contacts as parent links, the other
//     contacts queued and unioned by the whole block; it also writes the
//     brick's rows and each strip's x-face records to the brick's workspace;
//   * boundary analysis (Kernel 2, §II-B): threads over the strips that meet a
//     brick face union the segments that touch across it, in a global forest
//     over the bricks' border roots (one kernel for the x faces, from the
//     records; one for y and z, from the rows), each block unioning a pair of
//     border roots once;
//   * link (§II-C): a block per brick copies its rows and segment labels to
//     shared memory, resolves its border roots and writes the final labels,
//     eight voxels per lane in one 32-byte store, a warp covering eight rows.
// The result is the canonical labelling: 0 for background, 1 + the smallest
// voxel index (z*H + y)*W + x of the component.
#include "ccl_core.cuh"
#include "ccl_internal.h"

namespace ccl {
namespace vol {

constexpr int kStrips = 16;   // strips per brick along y and along z
static_assert(kStrips * kStrips == kThreads, "one thread per strip");
constexpr int kNodes = kThreads * 16;   // at most 16 segments in a 32-voxel word
constexpr int kNodeBits = 12;           // node index inside a brick
constexpr int kNodeMask = (1 << kNodeBits) - 1;
static_assert(kNodes == 1 << kNodeBits, "node index width");
// Border roots per brick: every one owns a segment of a strip on a y or z face
// (60 strips of at most 16 segments) or a segment touching an x face (196
// inner strips, at most 2 each): at most 1352.
constexpr int kSlots = 2048;
constexpr int kSlotBits = 11;
constexpr int kBrickBits = 22;          // global node id: key << 33 | brick << 11 | slot
constexpr long long kMaxBricks = 1ll << kBrickBits;
static_assert(kSlotBits + kBrickBits == 33, "31-bit key in the top bits of a node id");
// Per-brick workspace, in ints from the brick's base:
//   [0] border roots, [1] segments;
//   [kOffBase, kOffSt)   rank of each strip's first segment (uint16 per strip);
//   [kOffSt, kOffLab)    segment starts of each strip (the runs of its OR);
//   [kOffLab, kOffKey)   label of each segment: 1 + the voxel index of its
//                        root's smallest voxel, or -(slot + 1) for a border root;
//   [kOffKey, kOffSeg)   key (smallest voxel index) of each border root;
//   [kOffSeg, kOffXR)    OR of each strip's rows;
//   [kOffXR, kOffXL)     x-face record of each strip's segment at x = 32 bx
//                        (bricks with bx > 0), an int2: {slot | rows << 16,
//                        key} of its root, rows = the strip's rows holding
//                        that voxel (0: no such segment);
//   [kOffXL, kOffRows)   the same for the segment at x = 32 bx + 31 (bricks
//                        with a brick to their right);
//   [kOffRows, kOffUni)  the brick's rows as bits, row rr of every strip
//                        together (R x 256 words), so that the later kernels
//                        read them in whole 16-byte pieces;
//   [kOffUni, ...)       per strip (18 and 26), the border slot of the root all
//                        its segments share, or -1 (no segment, several roots,
//                        not a face strip).
constexpr int kOffBase = 4;
constexpr int kOffSt = kOffBase + kThreads / 2;
constexpr int kOffLab = kOffSt + kThreads;
constexpr int kOffKey = kOffLab + kNodes;
constexpr int kOffSeg = kOffKey + kSlots;
constexpr int kOffXR = kOffSeg + kThreads;
constexpr int kOffXL = kOffXR + 2 * kThreads;
constexpr int kOffRows = kOffXL + 2 * kThreads;
constexpr int kOffUni = kOffRows + 4 * kThreads;
constexpr int kBrickInts = (kOffUni + kThreads + 63) & ~63;   // 256-byte multiple
static_assert(kOffLab % 4 == 0, "16-byte aligned segment labels");
static_assert(kOffXR % 2 == 0 && kOffXL % 2 == 0, "8-byte aligned x-face records");
static_assert(kOffBase % 4 == 0 && kOffSt % 4 == 0 && kOffRows % 4 == 0,
              "16-byte aligned strip arrays");

// Strip shape: every pair of voxels of the strip's rows whose x differ by at
// most one is a neighbour pair (|dy| + |dz| <= 1 at 18, any at 26).
template <int CONN> struct Strip {
    static constexpr int SY = CONN == 6 ? 1 : 2;
    static constexpr int SZ = CONN == 26 ? 2 : 1;
    static constexpr int R = SY * SZ;   // row rr = k * SY + j: j along y, k along z
};
inline int strip_sy(int conn) { return conn == 6 ? 1 : 2; }
inline int strip_sz(int conn) { return conn == 26 ? 2 : 1; }

struct Geom3 {
    int D, H, W;
    int sy, sz;     // strip rows along y and z
    int nwg;        // 32-voxel words per row = bricks along x
    int nsy, nsz;   // strips along y and z
    int nby, nbz;   // bricks along y and z
    long long nbricks;
};

inline Geom3 make_geom3(int D, int H, int W, int conn) {
    Geom3 g;
    g.D = D;
    g.H = H;
    g.W = W;
    g.sy = strip_sy(conn);
    g.sz = strip_sz(conn);
    g.nwg = (int)(((long long)W + 31) / 32);
    g.nsy = (H + g.sy - 1) / g.sy;
    g.nsz = (D + g.sz - 1) / g.sz;
    g.nby = (g.nsy + kStrips - 1) / kStrips;
    g.nbz = (g.nsz + kStrips - 1) / kStrips;
    g.nbricks = (long long)g.nwg * g.nby * g.nbz;
    return g;
}

inline bool valid_conn3(int c) { return c == 6 || c == 18 || c == 26; }

inline bool dims_ok(int D, int H, int W, int conn) {
    if (D < 1 || H < 1 || W < 1) return false;
    if ((long long)D * H > 2147483646LL / W) return false;   // 1 + index fits int32
    return make_geom3(D, H, W, conn).nbricks <= kMaxBricks;
}

inline size_t bricks_bytes3(const Geom3 &g) { return (size_t)g.nbricks * kBrickInts * 4u; }
inline size_t par_bytes3(const Geom3 &g) { return (size_t)g.nbricks * kSlots * sizeof(gnode); }

struct VolArgs {
    const uint8_t *vol;
    int32_t *labels;
    int *bws;          // per-brick workspace, kBrickInts ints per brick
    gnode *par;        // global forest: kSlots parents per brick
    Geom3 g;
    int aligned16;     // volume rows start on 16-byte boundaries (W % 16 == 0)
    int out_aligned16; // label rows start on 16-byte boundaries (W % 4 == 0)
    int out_aligned32; // label rows start on 32-byte boundaries (W % 8 == 0)
};

struct Forest3 {
    gnode *base;
    __device__ __forceinline__ gnode *par(gnode n) const {
        return base + (n & ((1ull << (kBrickBits + kSlotBits)) - 1ull));
    }
};

__device__ __forceinline__ gnode node3(int key, long long brick, int slot) {
    return ((gnode)(uint32_t)key << (kBrickBits + kSlotBits)) | ((gnode)brick << kSlotBits) |
           (gnode)slot;
}

// Pairs of neighbouring strips, the other strip earlier in the brick: offset
// (dz, dy) in strips, the rows of each strip that face the other (bit rr of a
// mask = row rr), and the x reach dil: a voxel of one row set and a voxel of
// the other are neighbours exactly when their x differ by at most dil.
struct StripPair {
    int dz, dy, ma, mb, dil;
};

template <int CONN> __host__ __device__ constexpr int n_pairs() {
    return CONN == 6 ? 2 : CONN == 18 ? 6 : 4;
}

template <int CONN> __device__ __forceinline__ StripPair strip_pair(int k) {
    if (CONN == 6) return k == 0 ? StripPair{0, -1, 1, 1, 0} : StripPair{-1, 0, 1, 1, 0};
    if (CONN == 18) {   // rows: 0 = even y, 1 = odd y
        switch (k) {
            case 0: return {0, -1, 1, 2, 1};    // strip below in y: facing rows, x +- 1
            case 1: return {-1, 0, 3, 3, 0};    // strip below in z, same x: any rows
            case 2: return {-1, 0, 1, 1, 1};    // strip below in z, same y: x +- 1
            case 3: return {-1, 0, 2, 2, 1};
            case 4: return {-1, -1, 1, 2, 0};   // diagonal strips: facing rows, same x
            default: return {-1, 1, 2, 1, 0};
        }
    }
    switch (k) {        // 26, rows rr = zz * 2 + yy
        case 0: return {0, -1, 1 | 4, 2 | 8, 1};
        case 1: return {-1, 0, 1 | 2, 4 | 8, 1};
        case 2: return {-1, -1, 1, 8, 1};
        default: return {-1, 1, 2, 4, 1};
    }
}

// Whether the voxel at (x - 1, y + dy, z + dz) is a neighbour of (x, y, z).
template <int CONN> __host__ __device__ constexpr bool x_pair(int dy, int dz) {
    return CONN == 26 || (CONN == 18 && (dy != 0) + (dz != 0) <= 1) ||
           (CONN == 6 && dy == 0 && dz == 0);
}

// Rows r2 of the strip at offset (dsy, dsz) (in strips) whose voxel at x - 1
// is a neighbour of the voxel at x of row rr of a strip.
template <int CONN> __host__ __device__ constexpr uint32_t x_rows(int dsy, int dsz, int rr) {
    constexpr int SY = CONN == 6 ? 1 : 2, SZ = CONN == 26 ? 2 : 1;
    uint32_t m = 0;
    for (int r2 = 0; r2 < SY * SZ; ++r2) {
        const int dy = dsy * SY + r2 % SY - rr % SY, dz = dsz * SZ + r2 / SY - rr / SY;
        if (dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1 && x_pair<CONN>(dy, dz)) m |= 1u << r2;
    }
    return m;
}

// bits of the run of ones of a that starts at bit p
__device__ __forceinline__ uint32_t run_at(uint32_t a, int p) {
    const uint32_t rest = ~(a >> p);   // zeros of a from bit p on (ones past bit 31 - p)
    const int len = rest ? __ffs(rest) - 1 : 32;
    return (len >= 32 ? 0xFFFFFFFFu : ((1u << len) - 1u)) << p;
}

// Rank of the segment holding bit u of a strip whose segment starts are st and
// whose first segment has rank base.
__device__ __forceinline__ int seg_rank3(int base, uint32_t st, int u) {
    return base + __popc(st & le_mask(u)) - 1;
}

// Lowest set bit of v among bits u - 1, u and u + 1 (one of them is set).
__device__ __forceinline__ int low3(uint32_t v, int u) {
    return u - 2 + __ffs(__funnelshift_r(v << 1, v >> 31, u) & 7u);
}

// Contacts of two neighbouring strips A and B at the level of their segments
// (the runs of each strip's OR).  Facing rows fa, fb, x reach dil.  When x must
// match (dil = 0), two segments touch exactly when they overlap, every run of
// fa & fb lies in one segment of each strip, and so the runs of fa & fb, one
// contact each at the run's first voxel, are the touching pairs (fewer than
// the picks below when the rows are sparse).  Otherwise, for every
// segment of A that touches B, its pick is the segment of B holding the lowest
// B voxel it touches; that voxel lies within one of the segment's lowest
// touching voxel, which the carry of (segA & ~X) + stA marks (X = the voxels
// of fa that touch fb).  Likewise for every segment of B.  Segments of a strip
// are separated by empty voxels and touch only within dil <= 1, so two touching
// pairs never cross (A left of A' and B right of B'); hence if neither A nor B
// picks the other, their picks would form a crossing pair, and the picks are
// exactly the touching pairs, with repeats.  Pairs in increasing position
// order are non-decreasing in both segments, so every repeat follows its
// first occurrence directly.  f(u, v) gets voxel u of A and v of B.
template <class F>
__device__ __forceinline__ void segment_contacts(uint32_t segA, uint32_t stA, uint32_t fa,
                                                 uint32_t segB, uint32_t stB, uint32_t fb,
                                                 int dil, F &&f) {
    if (!dil) {
        const uint32_t o = fa & fb;
        for (uint32_t e = o & ~(o << 1); e; e &= e - 1) {
            const int u = __ffs(e) - 1;
            f(u, u);
        }
        return;
    }
    const uint32_t X = fa & (fb | (fb << 1) | (fb >> 1));
    const uint32_t Y = fb & (fa | (fa << 1) | (fa >> 1));
    const uint32_t pa = ((segA & ~X) + stA) & X;
    const uint32_t pb = ((segB & ~Y) + stB) & Y;
    for (uint32_t e = pa | pb; e; e &= e - 1) {
        const int u = __ffs(e) - 1;
        if ((pa >> u) & 1u) f(u, low3(fb, u));
        if ((pb >> u) & 1u) f(low3(fa, u), u);
    }
}

// Shared-memory union-find over segments.  P[n] = key(parent) << 12 | parent,
// where key is the brick-local index of a segment's smallest voxel, so the
// smaller packed value is the smaller key.  A root holds its own packed id;
// links go from the larger key to the smaller by an atomic minimum, and a node
// linked elsewhere meanwhile only has its parent lowered: the union goes on
// with the parent it had (no retry storm when many threads join one set).
__device__ __forceinline__ int pfind(volatile int *P, int x, int &budget, int *err) {
    for (;;) {
        if (--budget < 0) { atomicOr(err, kErrSmemFind); return x; }
        const int p = P[x] & kNodeMask;
        if (p == x) return x;
        const int gp = P[p];
        if ((gp & kNodeMask) == p) return p;
        P[x] = gp;   // path halving: gp is an ancestor of x
        x = gp & kNodeMask;
    }
}

__device__ __forceinline__ void punion(int *P, const uint16_t *K, int a, int b, int &budget,
                                       int *err) {
    volatile int *vP = P;
    for (;;) {
        a = pfind(vP, a, budget, err);
        b = pfind(vP, b, budget, err);
        if (a == b) return;
        if (budget < 0) { atomicOr(err, kErrSmemUnion); return; }
        int pa = ((int)K[a] << kNodeBits) | a, pb = ((int)K[b] << kNodeBits) | b;
        if (pa > pb) {   // link the root with the larger key, b, under a
            const int tp = pa; pa = pb; pb = tp;
            b = a;
        }
        const int old = atomicMin(&P[b], pa);
        if (old == pb) return;
        a = pa & kNodeMask;
        b = old & kNodeMask;
    }
}

// Contact queue entries beyond the unused end of P (sized so that a Bernoulli
// 0.5 volume needs one pass; a fuller queue takes further passes).
template <int CONN> __host__ __device__ constexpr int queue_extra() {
    return CONN == 26 ? 2816 : CONN == 18 ? 3328 : 2048;
}

// Pairs whose earlier strip's segments all have strictly smaller keys (every
// pair but 26-connectivity's strip below in y, whose rows share z with ours).
template <int CONN> __host__ __device__ constexpr bool key_monotone(int k) {
    return CONN != 26 || k != 0;
}

// Whether the merge records each face strip's single border slot (most face
// strips have one at 18 and 26; about 40 % at 6 in a Bernoulli 0.5 volume, too
// few to pay for the record).
template <int CONN> __host__ __device__ constexpr bool uniform_slots() { return CONN != 6; }

// 18-connectivity: the same-row x +- 1 pairs of the strip below in z add only
// contacts of segments that do not overlap (overlapping ones meet in pair 1).
template <int CONN> __host__ __device__ constexpr bool overlap_joined(int k) {
    return CONN == 18 && (k == 2 || k == 3);
}

// The contacts such a pair adds: a voxel u of A's facing row outside every
// segment of B and a voxel v = u +- 1 of B's facing row outside every segment
// of A.  Any other contact of the pair has u or v inside a segment of the
// other strip, hence its two segments overlap (adjacent bits lie in one
// segment) and pair 1 joins them.  f(u, v) as in segment_contacts.
template <class F>
__device__ __forceinline__ void diagonal_contacts(uint32_t segA, uint32_t fa, uint32_t segB,
                                                  uint32_t fb, F &&f) {
    const uint32_t g = fb & ~segA;
    const uint32_t gl = g << 1, gr = g >> 1;   // bit u: g holds u - 1, u + 1
    for (uint32_t e = fa & ~segB & (gl | gr); e; e &= e - 1) {
        const int u = __ffs(e) - 1;
        if ((gl >> u) & 1u) f(u, u - 1);
        if ((gr >> u) & 1u) f(u, u + 1);
    }
}

template <int R, int QX> struct SmemVolMerge {
    int P[kNodes];                // packed parent of each segment; [total, kNodes): queue
    uint16_t K[kNodes];           // brick-local index of the segment's smallest voxel
    uint32_t rows[R][kThreads];   // each strip's rows
    uint32_t seg[kThreads];       // OR of each strip's rows
    uint32_t st[kThreads];        // segment starts of each strip
    int base[kThreads];           // rank of each strip's first segment
    uint32_t flag[kNodes / 32];   // roots whose component reaches a brick face
    int fbase[kNodes / 32];       // slot of the first flagged root of each flag word
    int warp_sums[kThreads / 32];
    int nq;                       // queued contacts
    uint32_t Q2[QX];              // queue entries past the unused end of P
};

__device__ __forceinline__ void brick_coords(const Geom3 &g, long long brick, int &bx, int &by,
                                             int &bz) {
    bx = (int)(brick % g.nwg);
    const long long q = brick / g.nwg;
    by = (int)(q % g.nby);
    bz = (int)(q / g.nby);
}

// ---------------------------------------------------------------------------
// Kernel 1: local merge of one brick.
template <int CONN>
__global__ void __launch_bounds__(kThreads, 5) kv_merge(VolArgs a, int *err) {
    constexpr int SY = Strip<CONN>::SY, SZ = Strip<CONN>::SZ, R = Strip<CONN>::R;
    constexpr int BYR = kStrips * SY;   // rows of a brick along y
    __shared__ SmemVolMerge<R, queue_extra<CONN>()> sm;
    const Geom3 &g = a.g;
    const int t = threadIdx.x;
    const long long brick = blockIdx.x;
    int bx, by, bz;
    brick_coords(g, brick, bx, by, bz);
    const int sy = t % kStrips, sz = t / kStrips;
    const int x0 = 32 * bx;
    const int gsy = by * kStrips + sy, gsz = bz * kStrips + sz;
    const uint8_t *vol_end = a.vol + (size_t)g.D * g.H * g.W;
    uint32_t rows[R];
    uint32_t seg = 0;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const int y = gsy * SY + rr % SY, z = gsz * SZ + rr / SY;
        rows[rr] = (y < g.H && z < g.D)
                       ? load_row_bits(a.vol, vol_end, z * g.H + y, x0, g.W, a.aligned16 != 0)
                       : 0u;
        sm.rows[rr][t] = rows[rr];
        seg |= rows[rr];
    }
    const uint32_t st = seg & ~(seg << 1);
    sm.st[t] = st;
    sm.seg[t] = seg;
    if (t == 0) sm.nq = 0;
    int total;
    const int base = block_excl_scan(__popc(st), sm.warp_sums, total);   // syncs
    sm.base[t] = base;
    {   // key of each segment: its first voxel in (z, y, x) order
        int n = base;
        for (uint32_t s = st; s; s &= s - 1, ++n) {
            const uint32_t m = run_at(seg, __ffs(s) - 1);
            int key = 0;
#pragma unroll
            for (int rr = R - 1; rr >= 0; --rr) {
                const uint32_t hit = rows[rr] & m;
                if (hit) {
                    const int ly = sy * SY + rr % SY, lz = sz * SZ + rr / SY;
                    key = (lz * BYR + ly) * 32 + __ffs(hit) - 1;
                }
            }
            sm.K[n] = (uint16_t)key;
            sm.P[n] = (key << kNodeBits) | n;
        }
    }
    for (int k = t; k < kNodes / 32; k += kThreads) sm.flag[k] = 0u;
    __syncthreads();

    // Unions with the earlier neighbour strips of the brick.  Every thread
    // lists the contacts of its strip with each earlier neighbour strip
    // (segment_contacts).  A segment's first contact with a strip of smaller
    // keys is its parent link (a plain store: only this thread writes the
    // parents of its segments here), which makes a forest whose roots are the
    // smallest keys of their trees.  The other contacts go to a queue (the
    // unused end of P, then Q2); after the forest is flattened, the whole
    // block takes them in turn, one lock-free union each.  A contact that
    // finds the queue full is listed again by a further pass: a thread's
    // queued contacts are always a prefix of its list (the queue counter only
    // grows), so each pass skips the ones queued before.
    uint32_t *Q = reinterpret_cast<uint32_t *>(sm.P + total);
    const int qcap1 = kNodes - total;
    const int qcap = qcap1 + queue_extra<CONN>();
    int budget = kSmemHopBudget;
    int skip = 0;   // this thread's contacts queued by earlier passes
    for (int pass = 0;; ++pass) {
        int c = 0;
        if (seg) {
            uint32_t parented = 0;   // own segments (bit = rank - base) with a parent link
            int la = -1, lb = -1;
#pragma unroll
            for (int kk = 0; kk < n_pairs<CONN>(); ++kk) {
                const int k = (kk + 1) % n_pairs<CONN>();   // pair 0 last
                const StripPair sp = strip_pair<CONN>(k);
                const int sy2 = sy + sp.dy, sz2 = sz + sp.dz;
                if (sz2 < 0 || sy2 < 0 || sy2 >= kStrips) continue;
                const int t2 = sz2 * kStrips + sy2;
                uint32_t fa = 0, fb = 0;
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    if ((sp.ma >> rr) & 1) fa |= rows[rr];
                    if ((sp.mb >> rr) & 1) fb |= sm.rows[rr][t2];
                }
                if (!fa || !fb) continue;
                const uint32_t segB = sm.seg[t2], stB = sm.st[t2];
                const int baseB = sm.base[t2];
                auto contact = [&](int u, int v) {
                    const int ia = seg_rank3(base, st, u), jb = seg_rank3(baseB, stB, v);
                    if (ia == la && jb == lb) return;
                    la = ia;
                    lb = jb;
                    if (key_monotone<CONN>(k)) {
                        const uint32_t bit = 1u << (ia - base);
                        if (!(parented & bit)) {
                            parented |= bit;
                            if (pass == 0) sm.P[ia] = ((int)sm.K[jb] << kNodeBits) | jb;
                            return;
                        }
                    }
                    if (c++ < skip) return;
                    const int q = atomicAdd(&sm.nq, 1);
                    if (q < qcap) {
                        const uint32_t ev = (uint32_t)ia | ((uint32_t)jb << 16);
                        if (q < qcap1) Q[q] = ev;
                        else sm.Q2[q - qcap1] = ev;
                        ++skip;
                    }
                };
                if (overlap_joined<CONN>(k)) diagonal_contacts(seg, fa, segB, fb, contact);
                else segment_contacts(seg, st, fa, segB, stB, fb, sp.dil, contact);
            }
        }
        __syncthreads();
        if (pass == 0) {   // flatten the forest of parent links
            for (int round = 0; round < 64; ++round) {
                int changed = 0;
                for (int n = t; n < total; n += kThreads) {
                    const int p = sm.P[n];
                    const int gp = sm.P[p & kNodeMask];
                    if (gp != p) { sm.P[n] = gp; changed = 1; }
                }
                if (!__syncthreads_or(changed)) break;
            }
        }
        const int nq_all = sm.nq;
        const int nq = min(nq_all, qcap);
        for (int i = t; i < nq; i += kThreads) {
            const uint32_t e = i < qcap1 ? Q[i] : sm.Q2[i - qcap1];
            punion(sm.P, sm.K, (int)(e & 0xFFFFu), (int)(e >> 16), budget, err);
        }
        __syncthreads();
        if (nq_all <= qcap) break;
        if (t == 0) sm.nq = 0;
        __syncthreads();
    }
    // every segment points at its root: read-only walks first (the forest no
    // longer changes), then, after a barrier, the stores, so that no walk sees
    // a half-rewritten parent
    constexpr int kPer = kNodes / kThreads;
    int roots[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        int r = t + i * kThreads;
        if (r < total) {
            for (;;) {
                if (--budget < 0) { atomicOr(err, kErrSmemFind); break; }
                const int p = sm.P[r] & kNodeMask;
                if (p == r) break;
                r = p;
            }
        }
        roots[i] = r;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (t + i * kThreads < total) sm.P[t + i * kThreads] = roots[i];   // plain index
    __syncthreads();

    // roots of segments on a face shared with another brick
    const bool yzface = (sy == 0 && by > 0) || (sy == kStrips - 1 && by + 1 < g.nby) ||
                        (sz == 0 && bz > 0) || (sz == kStrips - 1 && bz + 1 < g.nbz);
    {
        int n = base;
        for (uint32_t s = st; s; s &= s - 1, ++n) {
            const int p = __ffs(s) - 1;
            const bool border = yzface || (p == 0 && bx > 0) ||
                                ((run_at(seg, p) >> 31) && bx + 1 < g.nwg);
            if (border) {
                const int r = sm.P[n];
                const uint32_t bit = 1u << (r & 31);
                if (!(sm.flag[r >> 5] & bit)) atomicOr(&sm.flag[r >> 5], bit);
            }
        }
    }
    __syncthreads();
    int nb;
    {
        const int c = t < kNodes / 32 ? __popc(sm.flag[t]) : 0;
        const int fb = block_excl_scan(c, sm.warp_sums, nb);   // syncs
        if (t < kNodes / 32) sm.fbase[t] = fb;
    }
    __syncthreads();

    int *bw = a.bws + (size_t)brick * kBrickInts;
    if (t == 0) {
        bw[0] = nb < kSlots ? nb : kSlots;
        bw[1] = total;
        if (nb > kSlots) atomicOr(err, kErrBorderCap);
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr) bw[kOffRows + rr * kThreads + t] = (int)rows[rr];
    reinterpret_cast<uint16_t *>(bw + kOffBase)[t] = (uint16_t)base;
    bw[kOffSt + t] = (int)st;
    bw[kOffSeg + t] = (int)seg;
    const long long HW = (long long)g.H * g.W;
    auto gkey = [&](int k) {   // volume index of brick-local voxel index k
        const int lz = k / (32 * BYR), ly = (k / 32) % BYR;
        return (int)((long long)(bz * kStrips * SZ + lz) * HW + (long long)(by * BYR + ly) * g.W +
                     x0 + (k & 31));
    };
    auto slot_of = [&](int r) {   // border slot of flagged root r
        return sm.fbase[r >> 5] + __popc(sm.flag[r >> 5] & ((1u << (r & 31)) - 1u));
    };
    // x-face records: the roots of the segments at the brick's first and last x
    auto xrec = [&](int bit, int n) {
        uint32_t m = 0;
#pragma unroll
        for (int rr = 0; rr < R; ++rr) m |= ((rows[rr] >> bit) & 1u) << rr;
        if (!m) return make_int2(0, 0);
        const int r = sm.P[n], slot = slot_of(r);
        return slot < kSlots ? make_int2(slot | (int)(m << 16), gkey(sm.K[r])) : make_int2(0, 0);
    };
    if (bx > 0) reinterpret_cast<int2 *>(bw + kOffXR)[t] = xrec(0, base);
    if (bx + 1 < g.nwg) reinterpret_cast<int2 *>(bw + kOffXL)[t] = xrec(31, base + __popc(st) - 1);
    if (uniform_slots<CONN>()) {   // a face strip's single border slot, if it has one
        int uni = -1;
        if (seg && yzface) {
            const int r0 = sm.P[base];
            bool same = true;
            for (int n = base + 1; n < base + __popc(st); ++n) same &= sm.P[n] == r0;
            if (same && ((sm.flag[r0 >> 5] >> (r0 & 31)) & 1u)) {
                const int slot = slot_of(r0);
                if (slot < kSlots) uni = slot;
            }
        }
        bw[kOffUni + t] = uni;
    }
    for (int n = t; n < total; n += kThreads) {
        const int r = sm.P[n];
        const uint32_t fw = sm.flag[r >> 5];
        const int key = gkey(sm.K[r]);
        int v;
        if ((fw >> (r & 31)) & 1u) {
            const int slot = slot_of(r);
            v = -(slot + 1);
            if (r == n && slot < kSlots) {   // the root publishes its slot
                bw[kOffKey + slot] = key;
                a.par[(size_t)brick * kSlots + slot] = node3(key, brick, slot);
            }
        } else {
            v = 1 + key;
        }
        bw[kOffLab + n] = v;
    }
}

// The face kernels read what the local merge wrote (brick rows, strip words,
// segment labels, keys, x-face records) through L1: a kernel boundary separates the
// writes from these reads and nothing changes them meanwhile.  Only the
// global forest, which the unions change, is read from L2 (in gfind/gunion).

// Global node of border slot `slot` of a brick, from the key it published.
__device__ __forceinline__ gnode slot_node(const int *bw, long long brick, int slot) {
    return node3(__ldg(bw + kOffKey + slot), brick, slot);
}

// A block's set of the border-root pairs it has unioned, so that each pair is
// unioned once per block (faces repeat the same few pairs of large local
// components many times).  Open addressing over 48-bit keys: brick << 26 |
// slot << 15 | neighbour-brick code << 11 | slot of the other root.
constexpr int kPairSet = 2048;
constexpr unsigned long long kPairEmpty = ~0ull;

__device__ __forceinline__ void pair_set_clear(unsigned long long *set) {
    for (int i = threadIdx.x; i < kPairSet; i += blockDim.x) set[i] = kPairEmpty;
}

// Whether `key` was not in the set (it is now): the caller unions the pair.
__device__ __forceinline__ bool pair_set_add(unsigned long long *set, unsigned long long key) {
    unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 53) & (kPairSet - 1);
    for (int probe = 0; probe < 16; ++probe) {
        const unsigned long long v = *reinterpret_cast<volatile unsigned long long *>(set + h);
        if (v == key) return false;
        if (v == kPairEmpty) {
            const unsigned long long old = atomicCAS(set + h, kPairEmpty, key);
            if (old == kPairEmpty) return true;
            if (old == key) return false;
        }
        h = (h + 1) & (kPairSet - 1);
    }
    return true;   // crowded: union it anyway
}

// Code of brick b2 relative to b, b2 = b + dx + dy * nwg + dz * nwg * nby with
// dx, dy, dz in {-1, 0, 1}.
__device__ __forceinline__ unsigned long long pair_key(long long b, int s, int dx, int dy, int dz,
                                                       int s2) {
    const int code = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);   // < 27
    return ((unsigned long long)b << 27) | ((unsigned long long)s << 16) |
           ((unsigned long long)code << 11) | (unsigned long long)s2;
}

// ---------------------------------------------------------------------------
// Kernel 2a: unions across x faces.  Item i = (word w >= 1, strip): the
// segment at voxel 32w of the strip (x-face record of brick w) and, for each of
// the 3 x 3 strips around it, the segment at x = 32w - 1 (record of brick
// w - 1) when one of its rows holds a neighbour of a voxel 32w of the strip's
// rows.  Items run strip-fastest, so a block covers neighbouring strips of one
// face, whose records mostly name the same few roots: each pair of border
// roots is unioned once per block (pair_set_add), and a lane skips a
// neighbour whose root it has just unioned.
template <int CONN>
__global__ void __launch_bounds__(256) kv_xfaces(VolArgs a, long long items, int *err) {
    constexpr int R = Strip<CONN>::R;
    __shared__ unsigned long long pairs[kPairSet];
    pair_set_clear(pairs);
    __syncthreads();
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= items) return;
    const Geom3 &g = a.g;
    const long long ns = (long long)g.nsy * g.nsz;
    const int w = 1 + (int)(i / ns);
    const long long sidx = i % ns;
    const int gsy = (int)(sidx % g.nsy), gsz = (int)(sidx / g.nsy);
    const long long brick = ((long long)(gsz / kStrips) * g.nby + gsy / kStrips) * g.nwg + w;
    const int2 xr = __ldg(reinterpret_cast<const int2 *>(a.bws + (size_t)brick * kBrickInts +
                                                          kOffXR) +
                           (gsz % kStrips) * kStrips + gsy % kStrips);
    const uint32_t m = (uint32_t)xr.x >> 16;
    if (!m) return;
    const int slot = xr.x & 0xFFFF;
    const gnode self = node3(xr.y, brick, slot);
    const Forest3 F{a.par};
    int budget = kGlobHopBudget;
    gnode last = kNoNode;
#pragma unroll
    for (int dsz = -1; dsz <= 1; ++dsz)
#pragma unroll
        for (int dsy = -1; dsy <= 1; ++dsy) {
            uint32_t near = 0;   // rows of the other strip that can hold a neighbour
#pragma unroll
            for (int rr = 0; rr < R; ++rr)
                if ((m >> rr) & 1u) near |= x_rows<CONN>(dsy, dsz, rr);
            if (!near) continue;
            const int gsy2 = gsy + dsy, gsz2 = gsz + dsz;
            if (gsy2 < 0 || gsy2 >= g.nsy || gsz2 < 0 || gsz2 >= g.nsz) continue;
            const int dby = gsy2 / kStrips - gsy / kStrips, dbz = gsz2 / kStrips - gsz / kStrips;
            const long long b2 = brick - 1 + ((long long)dbz * g.nby + dby) * g.nwg;
            const int2 xl = __ldg(reinterpret_cast<const int2 *>(a.bws + (size_t)b2 * kBrickInts +
                                                                  kOffXL) +
                                   (gsz2 % kStrips) * kStrips + gsy2 % kStrips);
            if (!(((uint32_t)xl.x >> 16) & near)) continue;
            const int slot2 = xl.x & 0xFFFF;
            const gnode other = node3(xl.y, b2, slot2);
            if (other == last) continue;
            last = other;
            if (!pair_set_add(pairs, pair_key(brick, slot, -1, dby, dbz, slot2))) continue;
            gunion(F, self, other, budget, err);
        }
}

// Strips that may pair with a strip of another brick along y or z: strip y
// index % 16 in {0, 15}, or strip z index a positive multiple of 16.  Face
// strip f in raster order of (strip z, strip y) -> (strip z, strip y), for a
// grid of nsz x nsy strips.
__host__ __device__ __forceinline__ int face_ys(int nsy) {
    return (nsy + kStrips - 1) / kStrips + nsy / kStrips;
}
__host__ __device__ __forceinline__ long long face_strips(int nsz, int nsy) {
    const long long full = (nsz - 1) / kStrips;   // z = 16, 32, ... below nsz
    return full * nsy + (nsz - full) * face_ys(nsy);
}
__device__ __forceinline__ void face_strip(long long f, int nsy, int &z, int &y) {
    const int ny = face_ys(nsy);
    int yi;
    if (f < (long long)kStrips * ny) {
        z = (int)(f / ny);
        yi = (int)(f % ny);
    } else {
        const long long f2 = f - (long long)kStrips * ny;
        const long long per = (long long)nsy + (kStrips - 1) * (long long)ny;
        const long long grp = 1 + f2 / per;
        long long r = f2 % per;
        if (r < nsy) {
            z = (int)(kStrips * grp);
            y = (int)r;
            return;
        }
        r -= nsy;
        z = (int)(kStrips * grp + 1 + r / ny);
        yi = (int)(r % ny);
    }
    y = kStrips * (yi / 2) + ((yi & 1) ? kStrips - 1 : 0);
}

// ---------------------------------------------------------------------------
// Kernel 2b: unions across y and z faces.  Item = (word, face strip, strip pair
// k), k fastest: the contacts of the strip and of its k-th earlier neighbour
// strip, when that strip lies in another brick, one per segment of either strip
// (segment_contacts).  A contact is unioned unless the lane has just unioned
// the same two border roots or the block has (pair_set_add).  When all
// segments of both strips share one root each (the merge records that per
// strip), the item needs only to know whether the strips touch.
template <int CONN>
__global__ void __launch_bounds__(256) kv_yzfaces(VolArgs a, long long items, int *err) {
    constexpr int R = Strip<CONN>::R;
    __shared__ unsigned long long pairs[kPairSet];
    pair_set_clear(pairs);
    __syncthreads();
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= items) return;
    const Geom3 &g = a.g;
    const long long nfk = items / g.nwg;   // face strips x pairs
    const int w = (int)(i / nfk);
    const long long fk = i % nfk;
    const int k = (int)(fk % n_pairs<CONN>());
    const StripPair sp = strip_pair<CONN>(k);
    int gsy, gsz;
    face_strip(fk / n_pairs<CONN>(), g.nsy, gsz, gsy);
    const int gsy2 = gsy + sp.dy, gsz2 = gsz + sp.dz;
    if (gsy2 < 0 || gsy2 >= g.nsy || gsz2 < 0) return;
    if (gsy2 / kStrips == gsy / kStrips && gsz2 / kStrips == gsz / kStrips) return;
    const long long ba = ((long long)(gsz / kStrips) * g.nby + gsy / kStrips) * g.nwg + w;
    const long long bb = ((long long)(gsz2 / kStrips) * g.nby + gsy2 / kStrips) * g.nwg + w;
    const int ta = (gsz % kStrips) * kStrips + gsy % kStrips;
    const int tb = (gsz2 % kStrips) * kStrips + gsy2 % kStrips;
    const int *bwa = a.bws + (size_t)ba * kBrickInts, *bwb = a.bws + (size_t)bb * kBrickInts;
    const int ua = uniform_slots<CONN>() ? __ldg(bwa + kOffUni + ta) : -1;
    const int ub = uniform_slots<CONN>() ? __ldg(bwb + kOffUni + tb) : -1;
    uint32_t fa = 0, fb = 0;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        if ((sp.ma >> rr) & 1) fa |= (uint32_t)__ldg(bwa + kOffRows + rr * kThreads + ta);
        if ((sp.mb >> rr) & 1) fb |= (uint32_t)__ldg(bwb + kOffRows + rr * kThreads + tb);
    }
    if (!fa || !fb) return;
    const int dyb = gsy2 / kStrips - gsy / kStrips, dzb = gsz2 / kStrips - gsz / kStrips;
    const Forest3 F{a.par};
    int budget = kGlobHopBudget;
    if (ua >= 0 && ub >= 0) {   // every contact joins the same two border roots: is there one?
        const uint32_t touch = sp.dil ? fa & (fb | (fb << 1) | (fb >> 1)) : fa & fb;
        if (touch && pair_set_add(pairs, pair_key(ba, ua, 0, dyb, dzb, ub)))
            gunion(F, slot_node(bwa, ba, ua), slot_node(bwb, bb, ub), budget, err);
        return;
    }
    const uint32_t sega = (uint32_t)__ldg(bwa + kOffSeg + ta), sta = (uint32_t)__ldg(bwa + kOffSt + ta);
    const uint32_t segb = (uint32_t)__ldg(bwb + kOffSeg + tb), stb = (uint32_t)__ldg(bwb + kOffSt + tb);
    const int basea = __ldg(reinterpret_cast<const uint16_t *>(bwa + kOffBase) + ta);
    const int baseb = __ldg(reinterpret_cast<const uint16_t *>(bwb + kOffBase) + tb);
    int last_sa = -1, last_sb = -1;
    bool bad = false;
    // the border slot of the segment holding voxel x of a strip (its single
    // slot when the strip has one), or -1 after flagging a missing slot
    auto slot_at = [&](int uni, const int *bw, int base, uint32_t st, int x) {
        if (uni >= 0) return uni;
        const int n = seg_rank3(base, st, x);
        const int v = (n >= 0 && n < kNodes) ? __ldg(bw + kOffLab + n) : 0;
        if (v >= 0 || -v - 1 >= kSlots) return -1;
        return -v - 1;
    };
    auto contact = [&](int u, int v) {
        if (bad) return;
        const int sa = slot_at(ua, bwa, basea, sta, u), sb = slot_at(ub, bwb, baseb, stb, v);
        if (sa < 0 || sb < 0) {
            atomicOr(err, kErrResolve);
            bad = true;
            return;
        }
        if (sa == last_sa && sb == last_sb) return;
        last_sa = sa;
        last_sb = sb;
        if (!pair_set_add(pairs, pair_key(ba, sa, 0, dyb, dzb, sb))) return;
        gunion(F, slot_node(bwa, ba, sa), slot_node(bwb, bb, sb), budget, err);
    };
    if (overlap_joined<CONN>(k)) diagonal_contacts(sega, fa, segb, fb, contact);
    else segment_contacts(sega, sta, fa, segb, stb, fb, sp.dil, contact);
}

// ---------------------------------------------------------------------------
// Kernel 3: link.  Resolve the brick's border roots to 1 + the key of their
// global root and write every voxel's label.
template <int R> struct SmemVolLink {
    __align__(16) int S[kNodes];   // label of each segment
    uint32_t rows[R][kThreads];    // the brick's rows, as in its workspace
    uint32_t st[kThreads];
    uint16_t base[kThreads];
    int Rt[kSlots];                // final label of each border root
};

template <int CONN>
__global__ void __launch_bounds__(kThreads) kv_link(VolArgs a, int *err) {
    constexpr int SY = Strip<CONN>::SY, SZ = Strip<CONN>::SZ, R = Strip<CONN>::R;
    constexpr int BYR = kStrips * SY;
    __shared__ SmemVolLink<R> sm;
    const Geom3 &g = a.g;
    const int t = threadIdx.x;
    const long long brick = blockIdx.x;
    int bx, by, bz;
    brick_coords(g, brick, bx, by, bz);
    const int *bw = a.bws + (size_t)brick * kBrickInts;
    const int nb = min(__ldcg(bw), kSlots);
    const int nn = min(__ldcg(bw + 1), kNodes);
    // the brick's rows, segment starts and ranks, and its segment labels, to
    // shared memory 16 bytes at a time (every source is 16-byte aligned; the
    // label count rounded up stays inside the brick's workspace)
    {
        auto copy16 = [&](void *dst, const int *src) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
        };
        constexpr int kRowChunks = R * kThreads / 4, kStChunks = kThreads / 4;
        constexpr int kBaseChunks = kThreads / 8;
        const int nchunks = kRowChunks + kStChunks + kBaseChunks + (nn + 3) / 4;
        for (int c = t; c < nchunks; c += kThreads) {
            if (c < kRowChunks) {
                copy16(&sm.rows[0][0] + 4 * c, bw + kOffRows + 4 * c);
            } else if (c < kRowChunks + kStChunks) {
                const int k = c - kRowChunks;
                copy16(&sm.st[4 * k], bw + kOffSt + 4 * k);
            } else if (c < kRowChunks + kStChunks + kBaseChunks) {
                const int k = c - kRowChunks - kStChunks;
                copy16(&sm.base[8 * k], bw + kOffBase + 4 * k);
            } else {
                const int k = c - kRowChunks - kStChunks - kBaseChunks;
                copy16(&sm.S[4 * k], bw + kOffLab + 4 * k);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    {
        const gnode *par = a.par + (size_t)brick * kSlots;
        const Forest3 F{a.par};
        int budget = kGlobHopBudget;
        for (int j = t; j < nb; j += kThreads) {
            gnode r = __ldcg(par + j);
            for (;;) {
                if (--budget < 0) { atomicOr(err, kErrGlobFind); break; }
                const gnode p = __ldcg(F.par(r));
                if (p == r) break;
                r = p;
            }
            sm.Rt[j] = 1 + (int)(r >> (kBrickBits + kSlotBits));
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int n = t; n < nn; n += kThreads) {
        const int v = sm.S[n];
        if (v < 0) {
            const int j = -v - 1;
            if (j < nb) {
                sm.S[n] = sm.Rt[j];
            } else {
                sm.S[n] = 0;
                atomicOr(err, kErrBorderCap);
            }
        }
    }
    __syncthreads();
    // the brick's rows in raster order, 4 eight-voxel chunks each: a warp
    // stores eight whole 128-byte rows, one 32-byte store per lane where rows
    // are 32-byte aligned.  Thread t keeps chunk t % 4 of one row along y
    // through the brick's layers along z, 64 / BYR layers apart.
    const int x0 = 32 * bx;
    const int c = t & 3, q0 = t >> 2;
    const int ly = q0 % BYR, y = by * BYR + ly, xs = x0 + 8 * c;
    if (y >= g.H || xs >= g.W) return;
    constexpr int kDz = (kThreads / 4) / BYR;   // layers between a thread's rows
    static_assert(kDz * BYR == kThreads / 4, "whole layers per pass");
    const int sy_ = ly / SY, ry = ly % SY, bit0 = 8 * c;
    const uint32_t below = (1u << bit0) - 1u;   // bits under the chunk
    const int mode = (a.out_aligned32 && xs + 7 < g.W) ? 2 : (a.out_aligned16 && xs + 7 < g.W) ? 1 : 0;
    const int z0 = bz * kStrips * SZ;
    for (int lz = q0 / BYR; lz < kStrips * SZ && z0 + lz < g.D; lz += kDz) {
        const int ts = (lz / SZ) * kStrips + sy_, rr = (lz % SZ) * SY + ry;
        const uint32_t rb = sm.rows[rr][ts] >> bit0;
        int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (rb & 0xFFu) {
            const uint32_t sq = sm.st[ts] >> bit0;
            int n = sm.base[ts] + __popc(sm.st[ts] & below) - 1;   // rank before the chunk
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                n += (sq >> e) & 1u;
                if ((rb >> e) & 1u) v[e] = sm.S[min((unsigned)n, (unsigned)kNodes - 1u)];
            }
        }
        int32_t *out = a.labels + ((size_t)(z0 + lz) * g.H + y) * g.W + xs;
        if (mode == 2) {
            asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(out),
                         "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                         "r"(v[6]), "r"(v[7])
                         : "memory");
        } else if (mode == 1) {
            __stcs(reinterpret_cast<int4 *>(out), make_int4(v[0], v[1], v[2], v[3]));
            __stcs(reinterpret_cast<int4 *>(out) + 1, make_int4(v[4], v[5], v[6], v[7]));
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (xs + e < g.W) out[e] = v[e];
        }
    }
}

template <int CONN>
static void launch_volume(const VolArgs &a, int *err, cudaStream_t stream) {
    const Geom3 &g = a.g;
    const unsigned nbricks = (unsigned)g.nbricks;
    kv_merge<CONN><<<nbricks, kThreads, 0, stream>>>(a, err);
    if (g.nwg > 1) {
        const long long items = (long long)g.nsy * g.nsz * (g.nwg - 1);
        kv_xfaces<CONN><<<(unsigned)((items + 255) / 256), 256, 0, stream>>>(a, items, err);
    }
    const long long yz = face_strips(g.nsz, g.nsy) * n_pairs<CONN>() * g.nwg;
    kv_yzfaces<CONN><<<(unsigned)((yz + 255) / 256), 256, 0, stream>>>(a, yz, err);
    kv_link<CONN><<<nbricks, kThreads, 0, stream>>>(a, err);
}

}  // namespace vol
}  // namespace ccl

extern "C" size_t ccl_workspace_bytes3d(int depth, int height, int width, int connectivity) {
    using namespace ccl::vol;
    if (!valid_conn3(connectivity) || !dims_ok(depth, height, width, connectivity)) return 0;
    const Geom3 g = make_geom3(depth, height, width, connectivity);
    return bricks_bytes3(g) + par_bytes3(g);
}

extern "C" ccl_status ccl_label3d(const uint8_t *d_vol, int32_t *d_labels, int depth, int height,
                                  int width, int connectivity, void *d_ws, size_t ws_bytes,
                                  ccl_stream stream) {
    using namespace ccl::vol;
    if (!d_vol || !d_labels || !valid_conn3(connectivity) ||
        !dims_ok(depth, height, width, connectivity))
        return CCL_ERR_INVALID_ARG;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t need = ccl_workspace_bytes3d(depth, height, width, connectivity);
    ccl_status st = CCL_OK;
    if (!d_ws) {
        d_ws = ccl::library_workspace(s, need, &st);
        if (st != CCL_OK) return st;
    } else if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        return CCL_ERR_INVALID_ARG;
    }
    int *err = ccl::device_error_word();
    if (!err) return CCL_ERR_CUDA;
    VolArgs a;
    a.g = make_geom3(depth, height, width, connectivity);
    a.vol = d_vol;
    a.labels = d_labels;
    a.bws = static_cast<int *>(d_ws);
    a.par = reinterpret_cast<ccl::gnode *>(static_cast<char *>(d_ws) + bricks_bytes3(a.g));
    a.aligned16 = (width % 16 == 0) && (reinterpret_cast<uintptr_t>(d_vol) % 16 == 0);
    a.out_aligned16 = (width % 4 == 0) && (reinterpret_cast<uintptr_t>(d_labels) % 16 == 0);
    a.out_aligned32 = (width % 8 == 0) && (reinterpret_cast<uintptr_t>(d_labels) % 32 == 0);
    switch (connectivity) {
        case 6: launch_volume<6>(a, err, s); break;
        case 18: launch_volume<18>(a, err, s); break;
        default: launch_volume<26>(a, err, s); break;
    }
    if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}
