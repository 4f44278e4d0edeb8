// ccl_volume.cu -- labelling of 3-D volumes (the "2D/3D grid" of §I) with the
// paper's three phases one dimension up: tiles become bricks, tile seams become
// brick faces.
//   * local merge (Kernel 1, §II-A): a block labels one brick of 32 x 16 x 16
//     voxels in shared memory; thread t owns one 32-voxel row (a bit word) and
//     the union-find nodes are the runs of ones in the rows;
//   * boundary analysis (Kernel 2, §II-B): threads over the rows that meet a
//     brick face union the runs that touch across it, in a global forest over
//     the bricks' border roots (one kernel for the x faces, one for y and z);
//   * link (§II-C): a block per brick resolves its border roots and writes the
//     final labels, four voxels per 16-byte store, a warp covering four rows.
// The result is the canonical labelling: 0 for background, 1 + the smallest
// voxel index (z*H + y)*W + x of the component.
#include "ccl_core.cuh"
#include "ccl_internal.h"

namespace ccl {
namespace vol {

// Brick = one 32-voxel word along x, kBY rows along y, kBZ slices along z;
// thread t of a block owns row (ly, lz) = (t % kBY, t / kBY).
constexpr int kBY = 16, kBZ = 16;
static_assert(kBY * kBZ == kThreads, "one thread per brick row");
constexpr int kNodes = kThreads * 16;   // at most 16 runs in a 32-voxel word
// Border roots per brick: every one owns a run on a y or z face (60 rows of at
// most 16 runs) or a run touching an x face (196 inner rows, at most 2 runs
// each): at most 1352.
constexpr int kSlots = 2048;
constexpr int kSlotBits = 11;
constexpr int kBrickBits = 22;          // global node id: key << 33 | brick << 11 | slot
constexpr long long kMaxBricks = 1ll << kBrickBits;
static_assert(kSlotBits + kBrickBits == 33, "31-bit key in the top bits of a node id");
// Per-brick workspace, in ints from the brick's base:
//   [0] border roots, [1] run nodes;
//   [kOffBase, kOffLab)  rank of each row's first run node (uint16 per row);
//   [kOffLab, kOffKey)   label of each run node: 1 + the voxel index of its
//                        root's first voxel, or -(slot + 1) for a border root;
//   [kOffKey, ...)       key (smallest voxel index) of each border root.
constexpr int kOffBase = 4;
constexpr int kOffLab = kOffBase + kThreads / 2;   // 16-byte aligned
constexpr int kOffKey = kOffLab + kNodes;
constexpr int kBrickInts = (kOffKey + kSlots + 63) & ~63;   // 256-byte multiple
static_assert(kOffLab % 4 == 0, "16-byte aligned node labels");

struct Geom3 {
    int D, H, W;
    int nwg;        // 32-voxel words per row = bricks along x
    int nby, nbz;   // bricks along y and z
    long long nbricks;
};

inline Geom3 make_geom3(int D, int H, int W) {
    Geom3 g;
    g.D = D;
    g.H = H;
    g.W = W;
    g.nwg = (int)(((long long)W + 31) / 32);
    g.nby = (H + kBY - 1) / kBY;
    g.nbz = (D + kBZ - 1) / kBZ;
    g.nbricks = (long long)g.nwg * g.nby * g.nbz;
    return g;
}

inline bool dims_ok(int D, int H, int W) {
    if (D < 1 || H < 1 || W < 1) return false;
    if ((long long)D * H > 2147483646LL / W) return false;   // 1 + index fits int32
    return make_geom3(D, H, W).nbricks <= kMaxBricks;
}

inline bool valid_conn3(int c) { return c == 6 || c == 18 || c == 26; }

inline size_t bits_bytes3(const Geom3 &g) {
    return ((size_t)g.D * g.H * g.nwg * 4u + 255u) & ~(size_t)255u;
}
inline size_t bricks_bytes3(const Geom3 &g) { return (size_t)g.nbricks * kBrickInts * 4u; }
inline size_t par_bytes3(const Geom3 &g) { return (size_t)g.nbricks * kSlots * sizeof(gnode); }

struct VolArgs {
    const uint8_t *vol;
    int32_t *labels;
    uint32_t *bits;    // D*H rows x nwg words (bit k of word w = voxel 32w + k)
    int *bws;          // per-brick workspace, kBrickInts ints per brick
    gnode *par;        // global forest: kSlots parents per brick
    Geom3 g;
    int aligned16;     // volume rows start on 16-byte boundaries (W % 16 == 0)
    int out_aligned16; // label rows start on 16-byte boundaries (W % 4 == 0)
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

// Row pairs inside the neighbourhood: the k-th offset (dz, dy) from a row to an
// earlier row, and whether voxels of the two rows may differ by one in x.
//   6:  (0,-1) (-1,0), same x only
//   18: (0,-1) (-1,0) with x +-1; (-1,-1) (-1,+1) same x only
//   26: all four with x +-1
template <int CONN> struct RowPairs {
    static constexpr int n = CONN == 6 ? 2 : 4;
    __device__ static __forceinline__ int at(int k, int &dz, int &dy) {
        dz = k == 0 ? 0 : -1;
        dy = k == 0 ? -1 : k == 1 ? 0 : k == 2 ? -1 : 1;
        return CONN == 26 ? 1 : CONN == 18 ? (k < 2 ? 1 : 0) : 0;
    }
};

// Whether the voxel at (x - 1, y + dy, z + dz) is a neighbour of (x, y, z).
template <int CONN> __device__ __forceinline__ bool x_pair(int dy, int dz) {
    const int s = (dy != 0) + (dz != 0);
    return CONN == 26 || (CONN == 18 && s <= 1) || (CONN == 6 && s == 0);
}

// bits of the run of ones of a that starts at bit p
__device__ __forceinline__ uint32_t run_at(uint32_t a, int p) {
    const uint32_t rest = ~(a >> p);   // zeros of a from bit p on (ones past bit 31 - p)
    const int len = rest ? __ffs(rest) - 1 : 32;
    return (len >= 32 ? 0xFFFFFFFFu : ((1u << len) - 1u)) << p;
}

// Touching run pairs of two rows a and b (words at the same x): voxels x and
// x' touch when |x - x'| <= dil.  Each run of a is paired with the run of b
// holding the lowest b-voxel it touches, and each run of b with the run of a
// holding the lowest a-voxel it touches.  These pairs connect all mutually
// touching runs: if neither rule picks a touching pair (A, B), then A's pick
// B' lies left of B and B's pick A' left of A, A' touches B' (the intervals
// interleave), and induction on the position links A' with B'.
// f(i, j): the i-th run of a and the j-th run of b.
template <class F>
__device__ __forceinline__ void touching_runs(uint32_t a, uint32_t b, int dil, F &&f) {
    const uint32_t sa = a & ~(a << 1), sb = b & ~(b << 1);
    int i = 0;
    for (uint32_t s = sa; s; s &= s - 1, ++i) {
        const uint32_t run = run_at(a, __ffs(s) - 1);
        const uint32_t hit = b & (dil ? (run | (run << 1) | (run >> 1)) : run);
        if (hit) f(i, __popc(sb & le_mask(__ffs(hit) - 1)) - 1);
    }
    int j = 0;
    for (uint32_t s = sb; s; s &= s - 1, ++j) {
        const uint32_t run = run_at(b, __ffs(s) - 1);
        const uint32_t hit = a & (dil ? (run | (run << 1) | (run >> 1)) : run);
        if (hit) f(__popc(sa & le_mask(__ffs(hit) - 1)) - 1, j);
    }
}

// Shared-memory union of run nodes; node order is key order (row-major inside
// the brick), so the larger root is linked under the smaller and every root is
// its set's smallest voxel.  The link is an atomic minimum on the larger
// root's parent: if that node was linked elsewhere meanwhile, the minimum
// still only lowers its parent, and the union goes on with the parent it had
// (no retry storm when many threads join the same set at once).
__device__ __forceinline__ void union_nodes(pnode *P, int a, int b, int &budget, int *err) {
    volatile pnode *vP = P;
    for (;;) {
        a = sfind(vP, a, budget, err);
        b = sfind(vP, b, budget, err);
        if (a == b) return;
        if (budget < 0) { atomicOr(err, kErrSmemUnion); return; }
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(&P[b], (pnode)a);
        if (old == b) return;
        b = old;
    }
}

struct SmemVolMerge {
    pnode P[kNodes];              // parent of each run node
    uint16_t K[kNodes];           // brick-local index (t * 32 + x) of the node's first voxel
    uint32_t bits[kThreads];      // each row's word
    int base[kThreads];           // rank of each row's first node
    uint32_t flag[kNodes / 32];   // roots whose component reaches a brick face
    int fbase[kNodes / 32];       // slot of the first flagged root of each flag word
    int warp_sums[kThreads / 32];
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
__global__ void __launch_bounds__(kThreads) kv_merge(VolArgs a, int *err) {
    __shared__ SmemVolMerge sm;
    const Geom3 &g = a.g;
    const int t = threadIdx.x;
    const long long brick = blockIdx.x;
    int bx, by, bz;
    brick_coords(g, brick, bx, by, bz);
    const int ly = t % kBY, lz = t / kBY;
    const int x0 = 32 * bx, y = by * kBY + ly, z = bz * kBZ + lz;
    const bool in = y < g.H && z < g.D;
    const int row = in ? z * g.H + y : 0;
    const uint8_t *vol_end = a.vol + (size_t)g.D * g.H * g.W;
    const uint32_t bits = in ? load_row_bits(a.vol, vol_end, row, x0, g.W, a.aligned16 != 0) : 0u;
    const uint32_t st = bits & ~(bits << 1);
    sm.bits[t] = bits;
    int total;
    const int base = block_excl_scan(__popc(st), sm.warp_sums, total);   // syncs: bits visible
    sm.base[t] = base;
    {
        int n = base;
        for (uint32_t s = st; s; s &= s - 1, ++n) {
            sm.P[n] = n;
            sm.K[n] = (uint16_t)(t * 32 + __ffs(s) - 1);
        }
    }
    for (int k = t; k < kNodes / 32; k += kThreads) sm.flag[k] = 0u;
    __syncthreads();

    // unions with the earlier rows of the brick
    int budget = kSmemHopBudget;
    if (bits) {
#pragma unroll
        for (int k = 0; k < RowPairs<CONN>::n; ++k) {
            int dz, dy;
            const int dil = RowPairs<CONN>::at(k, dz, dy);
            const int lz2 = lz + dz, ly2 = ly + dy;
            if (lz2 < 0 || ly2 < 0 || ly2 >= kBY) continue;
            const int t2 = lz2 * kBY + ly2;
            const uint32_t b = sm.bits[t2];
            if (!b) continue;
            const int base2 = sm.base[t2];
            touching_runs(bits, b, dil, [&](int i, int j) {
                union_nodes(sm.P, base + i, base2 + j, budget, err);
            });
        }
    }
    __syncthreads();
    // every node points at its root
    for (int n = t; n < total; n += kThreads) sm.P[n] = sfind(sm.P, n, budget, err);
    __syncthreads();

    // roots of runs on a face shared with another brick
    const bool yzface = (ly == 0 && by > 0) || (ly == kBY - 1 && by + 1 < g.nby) ||
                        (lz == 0 && bz > 0) || (lz == kBZ - 1 && bz + 1 < g.nbz);
    {
        int n = base;
        for (uint32_t s = st; s; s &= s - 1, ++n) {
            const int p = __ffs(s) - 1;
            const bool border = yzface || (p == 0 && bx > 0) ||
                                ((run_at(bits, p) >> 31) && bx + 1 < g.nwg);
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
    if (in) a.bits[(size_t)row * g.nwg + bx] = bits;
    reinterpret_cast<uint16_t *>(bw + kOffBase)[t] = (uint16_t)base;
    const long long HW = (long long)g.H * g.W;
    for (int n = t; n < total; n += kThreads) {
        const int r = sm.P[n];
        const uint32_t fw = sm.flag[r >> 5];
        const int k = sm.K[r];
        const int key = (int)((long long)(bz * kBZ + (k >> 9)) * HW +
                              (long long)(by * kBY + ((k >> 5) & (kBY - 1))) * g.W + x0 + (k & 31));
        int v;
        if ((fw >> (r & 31)) & 1u) {
            const int slot = sm.fbase[r >> 5] + __popc(fw & ((1u << (r & 31)) - 1u));
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

// The brick and border slot of the j-th run of row (y, z) in word w (a run on
// a brick face, so its root holds a slot).
__device__ __forceinline__ bool run_slot(const VolArgs &a, int w, int y, int z, int j,
                                         long long &brick, int &slot, int *err) {
    const Geom3 &g = a.g;
    brick = ((long long)(z / kBZ) * g.nby + y / kBY) * g.nwg + w;
    const int t = (z % kBZ) * kBY + (y % kBY);
    const int *bw = a.bws + (size_t)brick * kBrickInts;
    const int n = __ldcg(reinterpret_cast<const uint16_t *>(bw + kOffBase) + t) + j;
    const int v = n < kNodes ? __ldcg(bw + kOffLab + n) : 0;
    if (v >= 0 || -v - 1 >= kSlots) { atomicOr(err, kErrResolve); return false; }
    slot = -v - 1;
    return true;
}

__device__ __forceinline__ gnode slot_node(const VolArgs &a, long long brick, int slot) {
    return node3(__ldcg(a.bws + (size_t)brick * kBrickInts + kOffKey + slot), brick, slot);
}

// ---------------------------------------------------------------------------
// Kernel 2a: unions across x faces.  Item i = (row, word w >= 1): voxel 32w of
// the row and its neighbours at x = 32w - 1 (the last run of a row of brick
// w - 1).  Neighbour runs of one border root are unioned once.
template <int CONN>
__global__ void __launch_bounds__(256) kv_xfaces(VolArgs a, long long items, int *err) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= items) return;
    const Geom3 &g = a.g;
    const int nw1 = g.nwg - 1;
    const int w = 1 + (int)(i % nw1);
    const long long row = i / nw1;
    const uint32_t m = __ldcg(a.bits + row * g.nwg + w);
    if (!(m & 1u)) return;
    const int y = (int)(row % g.H), z = (int)(row / g.H);
    const Forest3 F{a.par};
    int budget = kGlobHopBudget;
    gnode self = kNoNode;
    long long last_brick = -1;
    int last_slot = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            if (!x_pair<CONN>(dy, dz)) continue;
            const int y2 = y + dy, z2 = z + dz;
            if (y2 < 0 || y2 >= g.H || z2 < 0 || z2 >= g.D) continue;
            const uint32_t b = __ldcg(a.bits + ((size_t)z2 * g.H + y2) * g.nwg + (w - 1));
            if (!(b >> 31)) continue;
            long long ob;
            int os;
            if (!run_slot(a, w - 1, y2, z2, __popc(b & ~(b << 1)) - 1, ob, os, err)) return;
            if (ob == last_brick && os == last_slot) continue;
            last_brick = ob;
            last_slot = os;
            if (self == kNoNode) {
                long long sb;
                int ss;
                if (!run_slot(a, w, y, z, 0, sb, ss, err)) return;
                self = slot_node(a, sb, ss);
            }
            gunion(F, self, slot_node(a, ob, os), budget, err);
        }
}

// Rows that may pair with a row of another brick along y or z: y % kBY in
// {0, kBY - 1}, or z a multiple of kBZ (z > 0).  Face row f in raster order of
// (z, y) -> (z, y).
__host__ __device__ __forceinline__ int face_ys(int H) {
    return (H + kBY - 1) / kBY + H / kBY;
}
__host__ __device__ __forceinline__ long long face_rows(int D, int H) {
    const long long full = (D - 1) / kBZ;   // slices z = kBZ, 2 kBZ, ... below D
    return full * H + (D - full) * face_ys(H);
}
__device__ __forceinline__ void face_row(long long f, int H, int &z, int &y) {
    const int ny = face_ys(H);
    int yi;
    if (f < (long long)kBZ * ny) {
        z = (int)(f / ny);
        yi = (int)(f % ny);
    } else {
        const long long f2 = f - (long long)kBZ * ny;
        const long long per = (long long)H + (kBZ - 1) * (long long)ny;
        const long long grp = 1 + f2 / per;
        long long r = f2 % per;
        if (r < H) {
            z = (int)(kBZ * grp);
            y = (int)r;
            return;
        }
        r -= H;
        z = (int)(kBZ * grp + 1 + r / ny);
        yi = (int)(r % ny);
    }
    y = kBY * (yi / 2) + ((yi & 1) ? kBY - 1 : 0);
}

// ---------------------------------------------------------------------------
// Kernel 2b: unions across y and z faces.  Item = (face row, row pair k, word):
// the touching runs of the row and of its k-th earlier neighbour row, when that
// row lies in another brick.  Consecutive pairs of the same two border roots
// are unioned once.
template <int CONN>
__global__ void __launch_bounds__(256) kv_yzfaces(VolArgs a, long long items, int *err) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= items) return;
    const Geom3 &g = a.g;
    const int w = (int)(i % g.nwg);
    const long long fk = i / g.nwg;
    const int k = (int)(fk % RowPairs<CONN>::n);
    int y, z;
    face_row(fk / RowPairs<CONN>::n, g.H, z, y);
    int dz, dy;
    const int dil = RowPairs<CONN>::at(k, dz, dy);
    const int y2 = y + dy, z2 = z + dz;
    if (y2 < 0 || y2 >= g.H || z2 < 0) return;
    if (y2 / kBY == y / kBY && z2 / kBZ == z / kBZ) return;   // same brick: merged locally
    const uint32_t m = __ldcg(a.bits + ((size_t)z * g.H + y) * g.nwg + w);
    if (!m) return;
    const uint32_t b = __ldcg(a.bits + ((size_t)z2 * g.H + y2) * g.nwg + w);
    if (!b) return;
    const Forest3 F{a.par};
    int budget = kGlobHopBudget;
    int last_sa = -1, last_sb = -1;
    bool bad = false;
    touching_runs(m, b, dil, [&](int ia, int jb) {
        long long pa, pb;
        int sa, sb;
        if (bad) return;
        if (!run_slot(a, w, y, z, ia, pa, sa, err) || !run_slot(a, w, y2, z2, jb, pb, sb, err)) {
            bad = true;
            return;
        }
        if (sa == last_sa && sb == last_sb) return;
        last_sa = sa;
        last_sb = sb;
        gunion(F, slot_node(a, pa, sa), slot_node(a, pb, sb), budget, err);
    });
}

// ---------------------------------------------------------------------------
// Kernel 3: link.  Resolve the brick's border roots to 1 + the key of their
// global root and write every voxel's label.
struct SmemVolLink {
    __align__(16) int S[kNodes];   // label of each run node
    int R[kSlots];                 // final label of each border root
    uint32_t bits[kThreads];
    uint32_t st[kThreads];
    int base[kThreads];
};

__global__ void __launch_bounds__(kThreads) kv_link(VolArgs a, int *err) {
    __shared__ SmemVolLink sm;
    const Geom3 &g = a.g;
    const int t = threadIdx.x;
    const long long brick = blockIdx.x;
    int bx, by, bz;
    brick_coords(g, brick, bx, by, bz);
    const int *bw = a.bws + (size_t)brick * kBrickInts;
    const int nb = min(__ldcg(bw), kSlots);
    const int nn = min(__ldcg(bw + 1), kNodes);
    // node labels to shared memory, 16 bytes at a time (the source is 16-byte
    // aligned and rounding the count up stays inside the brick's workspace)
    for (int c = t; c < (nn + 3) / 4; c += kThreads) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&sm.S[4 * c]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                     "l"(bw + kOffLab + 4 * c) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    {
        const int ly = t % kBY, lz = t / kBY;
        const int y = by * kBY + ly, z = bz * kBZ + lz;
        const uint32_t bits =
            (y < g.H && z < g.D) ? __ldcg(a.bits + ((size_t)z * g.H + y) * g.nwg + bx) : 0u;
        sm.bits[t] = bits;
        sm.st[t] = bits & ~(bits << 1);
        sm.base[t] = __ldcg(reinterpret_cast<const uint16_t *>(bw + kOffBase) + t);
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
            sm.R[j] = 1 + (int)(r >> (kBrickBits + kSlotBits));
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int n = t; n < nn; n += kThreads) {
        const int v = sm.S[n];
        if (v < 0) {
            const int j = -v - 1;
            if (j < nb) {
                sm.S[n] = sm.R[j];
            } else {
                sm.S[n] = 0;
                atomicOr(err, kErrBorderCap);
            }
        }
    }
    __syncthreads();
    // 8 four-voxel chunks per row: a warp stores four whole 128-byte rows
    const int x0 = 32 * bx;
    for (int k = 0; k < 8; ++k) {
        const int idx = k * kThreads + t;
        const int tr = idx >> 3, c = idx & 7;
        const int y = by * kBY + tr % kBY, z = bz * kBZ + tr / kBY;
        const int xs = x0 + 4 * c;
        if (y >= g.H || z >= g.D || xs >= g.W) continue;
        const uint32_t rb = sm.bits[tr], sq = sm.st[tr];
        const int b0 = sm.base[tr];
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int bit = 4 * c + e;
            int n = b0 + __popc(sq & le_mask(bit)) - 1;
            n = n < 0 ? 0 : (n < kNodes ? n : kNodes - 1);
            v[e] = ((rb >> bit) & 1u) ? sm.S[n] : 0;
        }
        int32_t *out = a.labels + ((size_t)z * g.H + y) * g.W + xs;
        if (a.out_aligned16 && xs + 3 < g.W) {
            __stcs(reinterpret_cast<int4 *>(out), make_int4(v[0], v[1], v[2], v[3]));
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
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
        const long long items = (long long)g.D * g.H * (g.nwg - 1);
        kv_xfaces<CONN><<<(unsigned)((items + 255) / 256), 256, 0, stream>>>(a, items, err);
    }
    const long long yz = face_rows(g.D, g.H) * RowPairs<CONN>::n * g.nwg;
    kv_yzfaces<CONN><<<(unsigned)((yz + 255) / 256), 256, 0, stream>>>(a, yz, err);
    kv_link<<<nbricks, kThreads, 0, stream>>>(a, err);
}

}  // namespace vol
}  // namespace ccl

extern "C" size_t ccl_workspace_bytes3d(int depth, int height, int width, int connectivity) {
    using namespace ccl::vol;
    if (!valid_conn3(connectivity) || !dims_ok(depth, height, width)) return 0;
    const Geom3 g = make_geom3(depth, height, width);
    return bits_bytes3(g) + bricks_bytes3(g) + par_bytes3(g);
}

extern "C" ccl_status ccl_label3d(const uint8_t *d_vol, int32_t *d_labels, int depth, int height,
                                  int width, int connectivity, void *d_ws, size_t ws_bytes,
                                  ccl_stream stream) {
    using namespace ccl::vol;
    if (!d_vol || !d_labels || !valid_conn3(connectivity) || !dims_ok(depth, height, width))
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
    a.g = make_geom3(depth, height, width);
    a.vol = d_vol;
    a.labels = d_labels;
    a.bits = static_cast<uint32_t *>(d_ws);
    a.bws = reinterpret_cast<int *>(static_cast<char *>(d_ws) + bits_bytes3(a.g));
    a.par = reinterpret_cast<ccl::gnode *>(static_cast<char *>(d_ws) + bits_bytes3(a.g) +
                                           bricks_bytes3(a.g));
    a.aligned16 = (width % 16 == 0) && (reinterpret_cast<uintptr_t>(d_vol) % 16 == 0);
    a.out_aligned16 = (width % 4 == 0) && (reinterpret_cast<uintptr_t>(d_labels) % 16 == 0);
    switch (connectivity) {
        case 6: launch_volume<6>(a, err, s); break;
        case 18: launch_volume<18>(a, err, s); break;
        default: launch_volume<26>(a, err, s); break;
    }
    if (cudaGetLastError() != cudaSuccess) return CCL_ERR_CUDA;
    return CCL_OK;
}
