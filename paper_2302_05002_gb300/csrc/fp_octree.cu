// fp_octree.cu -- local octrees of the chunks, the stitch above them and the
// level-of-detail selection (paper Sec. 4.4, Fig. "octree"; "shallow octree",
// Abstract).
//
// Definitions (exact-integer reading):
//   * node (L, k) exists iff it holds a point and (L == 0 or its parent holds
//     more than C points and lies above max_level); it is a leaf iff it holds
//     at most C points or L == max_level;
//   * an inner node at level L keeps, per occupied level-(L+s) cell among its
//     children's remaining points, the smallest original index (deepest first).
// Closed form used here: with lambda(p) the shallowest level at which p has the
// smallest index of its cell, p is kept by its ancestor at level
// min(max(0, lambda(p) - s), leaf level of p).  Every cell at a level >= s >= g
// lies inside one level-g cell, hence inside one chunk, so lambda is decided
// per level-g cell.  Inside a chunk the distributed order is index order.
//
// Steps:
//   1. group the distributed points by level-g cell (records (key21, j) with j
//      the position in the chunk array, i.e. index order; any order inside a
//      cell);
//   2. cells with more than kPieceMax points are key-sorted and cut into
//      node-aligned pieces of at most kPieceMax points (split tree, one warp per
//      open node); the split tree also gives the nodes between level g and the
//      pieces, and which piece minimum is the minimum of which coarser node;
//   3. one CTA per window of pieces: sort by key in shared memory, all nearest
//      smaller values of the index along the key order give each point's
//      lambda, deep subtrees inside pieces are split by binary search, and each
//      point gets its owner level and leaf level;
//   4. node records (levels <= g from the count pyramid, deeper ones from steps
//      2-3) are sorted into preorder; ids are resolved per point;
//   5. the points are scattered stably by leaf id (leaf-grouped output) and,
//      in fp_subsample, by owner id (final output); owner segments of nodes
//      above the chunks (the stitch) are re-sorted by original index.
#include "fp_seg.cuh"

namespace fp {

constexpr int kPieceMax = 1024;                 // largest piece handled in shared memory
constexpr int kRoundLevels = 3;                 // levels a split round groups the open nodes' records by
constexpr int kWindow = 1024;                   // pieces starting in one window form a unit
constexpr int kUnitCap = kPieceMax + kWindow;   // records of one unit
constexpr int kUnitNT = 512;
constexpr int kUnitWarps = kUnitNT / 32;
constexpr uint8_t kInner = 0xFF;                // hierarchy still inner at this level
constexpr uint8_t kEmpty = 0xFE;

struct NodeRec {   // a node before preorder numbering
    uint64_t key;
    uint32_t count, leaf_first;
    uint8_t level, is_leaf, pad[6];
};
static_assert(sizeof(NodeRec) == 24, "NodeRec layout");

struct Piece {
    uint32_t begin, count;   // record range in the cell-grouped arrays
    uint8_t q, hier, A, dup; // level, leaf level or kInner, first-min level of its minimum, oversized
    uint8_t srt;             // its records are in key order down to this level
    uint8_t pad[3];
};
static_assert(sizeof(Piece) == 16, "Piece layout");

struct OpenNode {
    uint64_t key;
    uint32_t begin, count;
    uint8_t q, hier, A, pad;
    uint32_t rb;          // its ancestor-or-self in the open list the current round started from
    uint32_t pad2, pad3;
};
static_assert(sizeof(OpenNode) == 32, "OpenNode layout");

// A record of the cell-grouped arrays in one 16-byte word, so that a record is
// moved by one load and one store: Morton key (level 21) in x | y << 32, its
// position j in the chunk array in z; w is the counting slot in the split
// rounds' copy and 0 elsewhere.
FP_DEV uint4 rec_make(uint64_t key, uint32_t j, uint32_t w)
{
    return make_uint4((uint32_t)key, (uint32_t)(key >> 32), j, w);
}
FP_DEV uint64_t rec_key(const uint4& r) { return (uint64_t)r.x | ((uint64_t)r.y << 32); }
FP_DEV uint64_t rec_key_at(const uint4* rec, uint64_t i) { return *reinterpret_cast<const uint64_t*>(rec + i); }
FP_DEV uint32_t rec_j_at(const uint4* rec, uint64_t i) { return reinterpret_cast<const uint32_t*>(rec + i)[2]; }

struct OctCtx {   // device pointers of one fp_build_chunk_octree call
    const uint32_t* counts;    // points per level-g cell: the hierarchy
    const uint32_t* rcounts;   // records per level-g cell: the points at hand (a chunk group's, or all)
    uint32_t leaf_base;        // position of the first record in the whole distributed array
    const uint32_t* pyr;
    const uint32_t* cstart;
    uint8_t* cell_leaf;
    uint4* rec;           // cell-grouped records (rec_key, rec_j)
    Piece* pieces;
    uint32_t* npieces;
    uint32_t piece_cap;
    uint32_t* dups;       // pieces of more than kPieceMax points (equal keys to the deepest level)
    uint32_t* ndups;
    NodeRec* nrec;
    uint32_t* nnode;
    uint32_t node_cap_ws;
    uint32_t* codes;      // per record position j: code_make(LOD owner level, leaf level, level-g cell)
    uint32_t open_cap;
    int g, s, lmax, dl;
    uint64_t C;
    uint64_t n;           // records (bound of record positions j and of record indices)
    uint32_t* err;
};

// code of record position jj (owner level, leaf level and the level-g cell of
// its key21), checked against the record count (an inconsistent grouping must
// not turn into a stray store)
FP_DEV void put_code(const OctCtx& c, uint32_t jj, int K, int leafl, uint64_t key21)
{
    if (jj < c.n) c.codes[jj] = code_make(K, leafl, (uint32_t)(key21 >> (3 * (kKeyLevels - c.g))));
    else raise(c.err, FP_ERR_CAPACITY, 17);
}

// record i of the cell-grouped array, checked likewise (a zero record beyond it)
FP_DEV uint4 get_rec(const OctCtx& c, uint64_t i)
{
    if (i < c.n) return c.rec[i];
    raise(c.err, FP_ERR_CAPACITY, 18);
    return make_uint4(0u, 0u, 0u, 0u);
}

FP_DEV uint32_t pyr_at(const uint32_t* pyr, const uint32_t* counts, int g, int l, uint64_t key)
{
    return l == g ? counts[key] : pyr[((1ull << (3 * l)) - 1) / 7 + key];
}

__global__ void k_pyr_level(const uint32_t* __restrict__ child, uint32_t* __restrict__ parent, uint64_t np)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    // level offsets (8^l - 1) / 7 are only 4-byte aligned: scalar loads
    const uint32_t* c = child + 8 * k;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += c[q];
    parent[k] = s;
}

FP_DEV void emit_node(const OctCtx& c, uint64_t key, int level, uint32_t count, uint32_t leaf_first, bool leaf)
{
    uint32_t id = atomicAdd(c.nnode, 1u);
    if (id >= c.node_cap_ws) { raise(c.err, FP_ERR_CAPACITY, 1); return; }
    NodeRec r;
    r.key = key;
    r.count = count;
    r.leaf_first = leaf_first + c.leaf_base;
    r.level = (uint8_t)level;
    r.is_leaf = leaf ? 1 : 0;
    for (int q = 0; q < 6; ++q) r.pad[q] = 0;
    c.nrec[id] = r;
}

FP_DEV void emit_piece(const OctCtx& c, uint32_t begin, uint32_t count, int q, uint8_t hier, uint8_t A, int srt)
{
    uint32_t id = atomicAdd(c.npieces, 1u);
    if (id >= c.piece_cap) { raise(c.err, FP_ERR_CAPACITY, 2); return; }
    Piece p;
    p.begin = begin;
    p.count = count;
    p.q = (uint8_t)q;
    p.hier = hier;
    p.A = A;
    p.dup = count > (uint32_t)kPieceMax ? 1 : 0;
    p.srt = (uint8_t)srt;
    p.pad[0] = p.pad[1] = p.pad[2] = 0;
    c.pieces[id] = p;
    if (p.dup) {
        const uint32_t k = atomicAdd(c.ndups, 1u);
        if (k < c.piece_cap) c.dups[k] = id;
    }
}

// ---------------------------------------------------------------- cells
// Records (key21, j) grouped by level-g cell, j = position in the chunk array:
// cell m's records fill [cstart[m], cstart[m] + rcounts[m]) in any order --
// every later step is independent of the order inside a cell (minima are
// reductions, keys are sorted where their order matters).  One pass over the
// points; the lanes of a warp that share a cell take their slots with one
// atomic on the cell's cursor, which starts at cstart[m].  The points arrive
// chunk by chunk, so the cells in use at any time are consecutive: cursors sit
// at bit-reversed cell ids, which spreads those atomics over the whole array
// (and every L2 slice).  A cursor that does not end at cstart[m + 1] means the
// count grid was not the grid of these points (reported by k_cell_check).
FP_DEV uint32_t cursor_slot(uint32_t m, int g) { return __brev(m) >> (32 - 3 * g); }

__global__ void k_cell_cursor_init(const uint32_t* __restrict__ cstart, uint64_t cells, uint32_t* cursor, int g)
{
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < cells; m += (uint64_t)gridDim.x * blockDim.x)
        cursor[cursor_slot((uint32_t)m, g)] = cstart[m];
}

__global__ void __launch_bounds__(256) k_cell_scatter(const int4* __restrict__ pts, uint64_t n, const fp_cube* cube_p,
                                                      uint32_t* cursor, uint4* __restrict__ rec, int g,
                                                      uint32_t* err)
{
    const CubeDev cube = load_cube(cube_p);
    const int lane = threadIdx.x & 31;
    const int sh = 3 * (kKeyLevels - g);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {   // warp-uniform trip count
        const uint64_t i = i0 + threadIdx.x;
        uint64_t k = 0;
        uint32_t m = kNone;
        if (i < n) {
            const int4 q = __ldg(pts + i);
            k = key21(q.x, q.y, q.z, cube);
            m = (uint32_t)(k >> sh);
        }
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, m);
        const int leader = __ffs(peers) - 1;
        uint32_t at = 0;
        if (lane == leader && m != kNone) at = atomicAdd(&cursor[cursor_slot(m, g)], (uint32_t)__popc(peers));
        at = __shfl_sync(0xFFFFFFFFu, at, leader) + (uint32_t)__popc(peers & lanemask_lt());
        if (m != kNone) {
            if (at >= n) { raise(err, FP_ERR_CAPACITY, 3); continue; }   // a count grid of other points
            rec[at] = rec_make(k, (uint32_t)i, 0u);
        }
    }
}

__global__ void k_cell_check(const uint32_t* __restrict__ cstart, uint64_t cells, const uint32_t* cursor, int g,
                             uint32_t* err)
{
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < cells; m += (uint64_t)gridDim.x * blockDim.x)
        if (cursor[cursor_slot((uint32_t)m, g)] != cstart[m + 1]) raise(err, FP_ERR_CAPACITY, 4);
}

// Per level-g cell: leaf level if the hierarchy ends at or above g, kInner if
// the cell node is inner, kEmpty for an empty cell.  Nonempty cells with at
// most kPieceMax points become pieces; larger ones open the split tree.
__global__ void k_cell_setup(OctCtx c, OpenNode* open0, uint32_t* nopen0)
{
    uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t cells = 1ull << (3 * c.g);
    if (m >= cells) return;
    uint32_t cnt = c.rcounts[m];
    if (cnt == 0) { c.cell_leaf[m] = kEmpty; return; }
    uint8_t hier = kInner;
    for (int l = 0; l <= c.g; ++l) {
        uint32_t v = pyr_at(c.pyr, c.counts, c.g, l, m >> (3 * (c.g - l)));
        if (v <= c.C || l == c.lmax) { hier = (uint8_t)l; break; }
    }
    c.cell_leaf[m] = hier;
    if (cnt <= (uint32_t)kPieceMax) {
        emit_piece(c, c.cstart[m], cnt, c.g, hier, (uint8_t)c.g, c.g);
    } else {
        uint32_t id = atomicAdd(nopen0, 1u);
        if (id >= c.open_cap) { raise(c.err, FP_ERR_CAPACITY, 5); return; }
        OpenNode o;
        o.key = m;
        o.begin = c.cstart[m];
        o.count = cnt;
        o.q = (uint8_t)c.g;
        o.hier = hier;
        o.A = (uint8_t)c.g;
        o.pad = 0;
        o.rb = o.pad2 = o.pad3 = 0;
        open0[id] = o;
    }
}

// nodes at levels <= g, from the count pyramid
__global__ void k_nodes_upper(OctCtx c)
{
    uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int L = 0;
    uint64_t base = 0;
    while (L <= c.g && f >= base + (1ull << (3 * L))) { base += 1ull << (3 * L); ++L; }
    if (L > c.g) return;
    uint64_t k = f - base;
    uint32_t cnt = pyr_at(c.pyr, c.counts, c.g, L, k);
    if (cnt == 0) return;
    for (int a = 0; a < L; ++a) {   // every ancestor must be inner
        uint32_t v = pyr_at(c.pyr, c.counts, c.g, a, k >> (3 * (L - a)));
        if (v <= c.C || a >= c.lmax) return;
    }
    bool leaf = cnt <= c.C || L == c.lmax;
    emit_node(c, k, L, cnt, c.cstart[k << (3 * (c.g - L))], leaf);
}

// ------------------------------------------------------- big cells: rounds
// position p of the records of the open nodes, copied out one node after another
FP_DEV uint32_t big_of(const uint32_t* bigstart, uint32_t nb, uint32_t p)
{
    uint32_t a = 0, b = nb;
    while (a < b) { uint32_t m = (a + b) >> 1; if (bigstart[m] <= p) a = m + 1; else b = m; }
    return a - 1;
}

// records of each open node; a round's records are copied out compactly (bigstart)
__global__ void k_open_counts(const OpenNode* open0, const uint32_t* nopen0, uint32_t* cnt_out, uint32_t cap,
                              const uint64_t* d_skip, uint64_t skip_min)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    const bool skip = d_skip && *d_skip > skip_min;
    cnt_out[i] = i < *nopen0 && !skip ? open0[i].count : 0;
}

// Counting slots of a round are digit-major (slot = d * cap + node): the cells
// of one node, used together, lie far apart in the array (and in L2 slices).
__global__ void k_round_zero(const uint32_t* nopen, uint32_t cap, int nd, uint32_t* cnt, uint32_t* smin)
{
    const uint32_t nb = min(*nopen, cap);
    const uint64_t tot = (uint64_t)nb * nd;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < tot; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t slot = (x / nb) * cap + x % nb;
        cnt[slot] = 0;
        smin[slot] = kNone;
    }
}

// copy of the open nodes' records (key, j) and their slot (node, cell of the
// round's depth), counted per slot with one atomic per slot and warp, and the
// smallest index of every slot (the splits of the round take their children's
// minima from these)
__global__ void k_round_copy(const OpenNode* open, const uint32_t* nopen, uint32_t cap, const uint32_t* bigstart,
                             const uint32_t* total, const uint4* __restrict__ rec, uint4* __restrict__ trec, int sh,
                             uint32_t dmask, uint32_t* cnt, uint32_t* smin)
{
    const uint32_t nb = min(*nopen, cap), T = *total;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t p0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); p0 < T; p0 += stride) {   // warp-uniform
        const uint32_t p = p0 + lane;
        uint32_t slot = kNone, jv = kNone;
        if (p < T) {
            const uint32_t b = big_of(bigstart, nb, p);
            const uint32_t src = open[b].begin + (p - bigstart[b]);
            const uint4 r = rec[src];
            slot = (uint32_t)((rec_key(r) >> sh) & dmask) * cap + b;
            jv = r.z;
            trec[p] = make_uint4(r.x, r.y, r.z, slot);
        }
        // a warp whose neighbouring lanes hold distinct slots adds per lane (no match,
        // no reduction over each slot's lanes); otherwise equal slots are merged first
        const uint32_t snext = __shfl_down_sync(0xFFFFFFFFu, slot, 1);   // (lane 31: its own)
        if (__any_sync(0xFFFFFFFFu, lane < 31 && slot != kNone && slot == snext)) {
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, slot);
            if (slot != kNone) {   // every lane of a slot's group takes part in its reduction
                const uint32_t m = __reduce_min_sync(peers, jv);
                if (lane == __ffs(peers) - 1) {
                    atomicAdd(&cnt[slot], (uint32_t)__popc(peers));
                    atomicMin(&smin[slot], m);
                }
            }
        } else if (slot != kNone) {
            atomicAdd(&cnt[slot], 1u);
            atomicMin(&smin[slot], jv);
        }
    }
}

// counts -> absolute starts: node b's cells in digit order from open[b].begin (one warp per node)
__global__ void k_round_bases(const OpenNode* open, const uint32_t* nopen, uint32_t cap, int nd, uint32_t* cnt)
{
    const uint32_t nb = min(*nopen, cap);
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int per = (nd + 31) / 32;   // <= 16
    for (uint32_t b = warp; b < nb; b += nwarps) {
        uint32_t v[16];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int d = lane * per + q;
            v[q] = q < per && d < nd ? cnt[(uint64_t)d * cap + b] : 0u;
            sum += v[q];
        }
        uint32_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = open[b].begin + (x - sum);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int d = lane * per + q;
            if (q < per && d < nd) {
                cnt[(uint64_t)d * cap + b] = run;
                run += v[q];
            }
        }
    }
}

// the copied records back into their nodes' ranges, grouped by slot (any order inside a slot)
__global__ void k_round_scatter(const uint32_t* total, const uint4* __restrict__ trec, uint32_t* cnt,
                                uint4* __restrict__ rec, uint64_t n, uint32_t* err)
{
    const uint32_t T = *total;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t p0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); p0 < T; p0 += stride) {   // warp-uniform
        const uint32_t p = p0 + lane;
        const uint4 r = p < T ? trec[p] : make_uint4(0u, 0u, 0u, kNone);
        const uint32_t slot = r.w;
        // as in k_round_copy: one slot per lane when neighbouring lanes differ
        const uint32_t snext = __shfl_down_sync(0xFFFFFFFFu, slot, 1);   // (lane 31: its own)
        uint32_t at = 0;
        if (__any_sync(0xFFFFFFFFu, lane < 31 && slot != kNone && slot == snext)) {
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, slot);
            const int leader = __ffs(peers) - 1;
            if (slot != kNone && lane == leader) at = atomicAdd(&cnt[slot], (uint32_t)__popc(peers));
            at = __shfl_sync(0xFFFFFFFFu, at, leader) + (uint32_t)__popc(peers & lanemask_lt());
        } else if (slot != kNone) {
            at = atomicAdd(&cnt[slot], 1u);
        }
        if (slot == kNone) continue;
        if (at >= n) { raise(err, FP_ERR_CAPACITY, 6); continue; }
        rec[at] = make_uint4(r.x, r.y, r.z, 0u);
    }
}

// --------------------------------------------------- big cells: split tree
// One warp per open node at level q: child ranges by binary search on the
// key-sorted records, smallest index of every child, hierarchy status, first-min
// level; children that are still too large stay open, the others become pieces.
__global__ void k_split(OctCtx c, const OpenNode* cur, const uint32_t* ncur, OpenNode* nxt, uint32_t* nnxt,
                        uint32_t open_cap, int srt, const uint32_t* smin, int q0)
{
    const uint32_t nc = *ncur;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t w = warp; w < nc; w += nwarps) {
        const OpenNode o = cur[w];
        const uint32_t rb = o.q == q0 ? w : o.rb;   // slot column of the round (q0: the round's first level)
        const int q1 = o.q + 1;
        const int sh = 3 * (kKeyLevels - q1);
        // lane d (0..8): first record whose child digit is >= d
        uint32_t lo = o.begin + o.count;
        if (lane <= 8) {
            uint32_t a = o.begin, b = o.begin + o.count;
            while (a < b) {
                uint32_t mid = (a + b) >> 1;
                if ((int)((rec_key_at(c.rec, mid) >> sh) & 7) < lane) a = mid + 1;
                else b = mid;
            }
            lo = a;
        }
        // smallest index of every child, and of the node (the smallest of those):
        // from the round's per-slot minima -- child d covers the slots whose
        // digits below q0 start with the node's digits below q0, then d
        // (8^(srt - q1) of them)
        uint32_t mjd[8];
        uint32_t pmin = 0xFFFFFFFFu;
        const int span = 3 * (srt - q1);
        const uint32_t pre = (uint32_t)(o.key & ((1ull << (3 * (o.q - q0))) - 1));
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const uint32_t d0 = ((pre << 3) | (uint32_t)d) << span;
            uint32_t mj = 0xFFFFFFFFu;
            for (uint32_t t = lane; t < (1u << span); t += 32) mj = min(mj, smin[(uint64_t)(d0 + t) * open_cap + rb]);
            for (int off = 16; off > 0; off >>= 1) mj = min(mj, __shfl_xor_sync(0xFFFFFFFFu, mj, off));
            mjd[d] = mj;
            pmin = min(pmin, mj);
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            uint32_t cb = __shfl_sync(0xFFFFFFFFu, lo, d);
            uint32_t ce = __shfl_sync(0xFFFFFFFFu, lo, d + 1);
            uint32_t cn = ce - cb;
            if (cn == 0) continue;
            const uint32_t mj = mjd[d];
            if (lane == 0) {
                uint64_t key = (o.key << 3) | (uint64_t)d;
                uint8_t hier;
                if (o.hier != kInner) hier = o.hier;
                else hier = (cn <= c.C || q1 == c.lmax) ? (uint8_t)q1 : kInner;
                // the child's minimum is the parent's minimum: it keeps the parent's first-min level
                uint8_t A = mj == pmin ? o.A : (uint8_t)q1;
                if (o.hier == kInner) emit_node(c, key, q1, cn, cb, hier != kInner);
                uint32_t id = 0;
                const bool open_child = cn > (uint32_t)kPieceMax && q1 < c.dl;
                if (open_child) id = atomicAdd(nnxt, 1u);
                if (open_child && id >= open_cap) {
                    raise(c.err, FP_ERR_CAPACITY, 7);
                } else if (open_child) {
                    OpenNode ch;
                    ch.key = key;
                    ch.begin = cb;
                    ch.count = cn;
                    ch.q = (uint8_t)q1;
                    ch.hier = hier;
                    ch.A = A;
                    ch.pad = 0;
                    ch.rb = rb;
                    ch.pad2 = ch.pad3 = 0;
                    nxt[id] = ch;
                } else {
                    emit_piece(c, cb, cn, q1, hier, A, srt);
                }
            }
        }
    }
}

// ------------------------------------------------------------ units
struct UnitSmem {
    uint64_t key[kUnitCap];
    uint64_t key2[kUnitCap];
    uint32_t j[kUnitCap];       // by local index
    uint32_t mt[kUnitCap];      // min-tree over hj: internal nodes 1..P-1 (the leaves are hj itself)
    uint16_t v[kUnitCap];       // local index by sorted position
    uint16_t v2[kUnitCap];
    uint16_t piece[kUnitCap];   // piece of a local index
    uint8_t cl[kUnitCap];       // by run: common level with the nearest smaller index on the left (255: none)
    uint8_t cr[kUnitCap];       // ... on the right
    uint32_t hj[kUnitCap];      // by run: smallest index of the run
    uint16_t hid[kUnitCap];     // by sorted position: run number
    uint8_t leaf[kUnitCap];     // leaf level by sorted position (pieces with a deep subtree)
    uint32_t pbeg[kWindow + 1];
    uint16_t pcnt[kWindow + 1]; // 0 for an oversized piece (handled elsewhere)
    uint16_t psrt[kWindow + 1]; // start of each piece in the unit (load order = sorted order)
    uint8_t pq[kWindow + 1], phier[kWindow + 1], pA[kWindow + 1], pkind[kWindow + 1];
    uint16_t pn[kWindow + 1];   // points of the piece (0 for an oversized one)
    uint16_t ptab[kWindow + 1]; // table pieces: first entry of the piece's level tables
    uint16_t pfst[kWindow + 1]; // table pieces: start of the piece's records in the table phase
    uint8_t pD[kWindow + 1];    // table pieces: levels below the piece that decide lambda
    uint32_t pmin[kWindow + 1]; // table pieces: smallest index of the piece
    uint16_t whist[kUnitWarps][256];
    uint32_t scan[64];
    uint64_t wmin[kUnitWarps], wmax[kUnitWarps];
    unsigned long long kmin, kmax;
    uint32_t np, cnt, p0, dl, nh, smin, fcnt, tabn;
};

// two units per SM: 228 KB of shared memory, 1 KB of it reserved per CTA
static_assert(sizeof(UnitSmem) <= 113 * 1024, "UnitSmem must leave room for two CTAs per SM");

// Table pieces.  A piece whose node is not inner needs lambda only at the
// levels q+1 .. dl of the piece (coarser: the piece minimum's rule; deeper: the
// leaf).  When there are at most kTabLevels of them, one direct-mapped table
// per level (8^d entries at q+d) takes the smallest index of every occupied
// cell by shared-memory atomicMin, and lambda of a record is the shallowest of
// those levels at which it is its cell's minimum -- no sort and no
// nearest-smaller search.  The tables overlay the arrays of the general path
// (key .. v2), which runs after them.
constexpr int kTabLevels = 4;
constexpr int kTabCap = (int)((offsetof(UnitSmem, piece) - offsetof(UnitSmem, key)) / sizeof(uint32_t));
static_assert(kTabCap >= 3 * 4680, "tables of three pieces of four levels");
FP_DEV uint32_t tab_size(int D) { return D <= 0 ? 0u : (uint32_t)(((1u << (3 * (D + 1))) - 8u) / 7u); }

// stable LSD pass over the unit's records by 8 key bits at `shift`
FP_DEV void unit_sort_pass(UnitSmem& S, const uint64_t* kin, const uint16_t* vin, uint64_t* kout, uint16_t* vout,
                           int cnt, int shift)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int per_warp = kUnitCap / kUnitWarps;   // records per warp
    for (int q = threadIdx.x; q < kUnitWarps * 256; q += kUnitNT) (&S.whist[0][0])[q] = 0;
    __syncthreads();
    uint32_t pack[per_warp / 32];
#pragma unroll
    for (int r = 0; r < per_warp / 32; ++r) {
        int p = warp * per_warp + r * 32 + lane;
        uint32_t d = p < cnt ? (uint32_t)(kin[p] >> shift) & 255u : 0xFFFFu;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d != 0xFFFFu) {
            old = S.whist[warp][d];
            S.whist[warp][d] = (uint16_t)(old + __popc(peers));
        }
        old = __shfl_sync(0xFFFFFFFFu, old, leader);
        pack[r] = d | ((old + __popc(peers & lanemask_lt())) << 16);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over (digit, warp): the first 256 threads own one digit each
    uint32_t tot_d = 0;
    if (threadIdx.x < 256) {
        for (int w = 0; w < kUnitWarps; ++w) {
            uint32_t v = S.whist[w][threadIdx.x];
            S.whist[w][threadIdx.x] = (uint16_t)tot_d;
            tot_d += v;
        }
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<kUnitNT, uint32_t>(threadIdx.x < 256 ? tot_d : 0u, S.scan, tot);
    if (threadIdx.x < 256)
        for (int w = 0; w < kUnitWarps; ++w) S.whist[w][threadIdx.x] = (uint16_t)(S.whist[w][threadIdx.x] + ex);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < per_warp / 32; ++r) {
        int p = warp * per_warp + r * 32 + lane;
        if (p < cnt) {
            uint32_t d = pack[r] & 0xFFFFu;
            uint32_t pos = S.whist[warp][d] + (pack[r] >> 16);
            kout[pos] = kin[p];
            vout[pos] = vin[p];
        }
    }
    __syncthreads();
}

// last piece whose start is <= r (pieces of zero length share starts)
FP_DEV int piece_of(const UnitSmem& S, int np, int r)
{
    int a = 0, b = np;
    while (a < b) {
        int m = (a + b) >> 1;
        if ((int)S.psrt[m] <= r) a = m + 1;
        else b = m;
    }
    return a - 1;
}

// last piece whose table-phase start is <= r
FP_DEV int piece_of_tab(const UnitSmem& S, int np, int r)
{
    int a = 0, b = np;
    while (a < b) {
        int m = (a + b) >> 1;
        if ((int)S.pfst[m] <= r) a = m + 1;
        else b = m;
    }
    return a - 1;
}

// One CTA per window of kWindow record positions: the pieces starting in it.
// Per unit:
//   sort the records by key (stable, 8-bit LSD passes in shared memory);
//   nearest smaller index on each side along the key order (min-tree walks
//   over one representative per run of equal keys).  The deeper of the levels
//   shared with those two neighbours, plus one, is lambda unless the record is
//   the minimum of its piece, whose lambda comes from the split tree;
//   deep subtrees of inner pieces by binary search on the sorted keys.
// first piece of every unit: lower bound of the unit's window start over the sorted piece begins
__global__ void k_unit_ranges(const uint64_t* piece_begin_sorted, const uint32_t* npieces, uint32_t cap,
                              uint64_t nunits, uint32_t* unit_p0)
{
    uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > nunits) return;
    const uint32_t np_all = *npieces < cap ? *npieces : cap;
    const uint64_t w = u * kWindow;
    uint32_t a = 0, b = np_all;
    while (a < b) { uint32_t m = (a + b) >> 1; if (piece_begin_sorted[m] < w) a = m + 1; else b = m; }
    unit_p0[u] = a;
}

// Per-window piece descriptors, one warp per window, ahead of k_units (which
// then reads them with one load per piece instead of waiting, every warp of a
// CTA, on the piece loads and two block scans).  Pieces in window order:
//   kind 0: one point; 1: 2..32 points, not inner; 2: general path (larger, or
//   inner); 3: more than kPieceMax equal keys (k_dup_pieces); 4: table path --
//   a kind-2 piece, not inner, whose lambda is decided within kTabLevels levels,
//   while the tables of the candidates up to it fit in kTabCap entries.
// pdesc[p] = {begin, pn | psrt << 16, pcnt | pfst << 16, ptab | q << 16 | hier << 24},
// pdesc2[p] = A | kind << 8 | D << 16 (p = window's first piece + index);
// uhead[u] = {first piece, pieces, general records | table records << 16,
//             table entries | deepest needed level << 16 | smallest sorted level << 24}.
__global__ void __launch_bounds__(256) k_unit_desc(OctCtx c, const uint32_t* unit_p0, const uint32_t* piece_order,
                                                   uint64_t nunits, uint4* pdesc, uint32_t* pdesc2, uint4* uhead)
{
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    constexpr uint32_t kSat = (uint32_t)kTabCap + 1u;   // table prefixes saturate here (past it nothing fits)
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nunits; u += nw) {
        const uint32_t p0 = unit_p0[u], np = unit_p0[u + 1] - p0;
        uint32_t tcarry = 0, rcarry = 0, dmax = 0, smin = 255;
        for (uint32_t b0 = 0; b0 < np; b0 += 32) {   // warp-uniform
            const uint32_t pi = b0 + lane;
            const bool valid = pi < np;
            Piece p{};
            if (valid) p = c.pieces[piece_order[p0 + pi]];
            uint32_t kind = 0, tz = 0, D = 0;
            bool cand = false;
            if (valid) {
                const bool large = !p.dup && (p.count > 32 || p.hier == kInner);
                kind = p.dup ? 3u : (large ? 2u : (p.count == 1 ? 0u : 1u));
                if (large && p.hier != kInner) {
                    const int Dv = min(kKeyLevels, c.s + (int)p.hier - 1) - (int)p.q;
                    if (Dv <= kTabLevels) { cand = true; tz = tab_size(Dv); D = (uint32_t)max(Dv, 0); }
                }
            }
            uint32_t inc = tz;   // saturating inclusive scan of the candidates' table sizes
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc = min(inc + y, kSat);
            }
            uint32_t tex = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
            tex = min(tcarry + (lane ? tex : 0u), kSat);
            uint32_t cn = 0, fn = 0, ptab = 0;
            if (valid && kind == 2) {
                if (cand && tex + tz <= (uint32_t)kTabCap) {
                    kind = 4;
                    ptab = tex;
                    fn = p.count;
                } else {
                    cn = p.count;
                    const uint32_t d = p.hier == kInner ? (uint32_t)c.dl
                                                        : (uint32_t)min(kKeyLevels, c.s + (int)p.hier - 1);
                    dmax = max(dmax, d);
                    smin = min(smin, (uint32_t)p.srt);
                }
            }
            uint32_t inc2 = cn | (fn << 16);   // records of both paths, in window order
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc2, o);
                if (lane >= o) inc2 += y;
            }
            uint32_t ex = __shfl_up_sync(0xFFFFFFFFu, inc2, 1);
            ex = rcarry + (lane ? ex : 0u);
            if (valid) {
                const uint32_t pn = p.dup ? 0u : p.count;
                pdesc[p0 + pi] = make_uint4(p.begin, pn | (ex << 16), cn | ((ex >> 16) << 16),
                                            ptab | ((uint32_t)p.q << 16) | ((uint32_t)p.hier << 24));
                pdesc2[p0 + pi] = (uint32_t)p.A | (kind << 8) | (D << 16);
            }
            tcarry = min(tcarry + __shfl_sync(0xFFFFFFFFu, inc, 31), kSat);
            rcarry += __shfl_sync(0xFFFFFFFFu, inc2, 31);
        }
        dmax = __reduce_max_sync(0xFFFFFFFFu, dmax);
        smin = __reduce_min_sync(0xFFFFFFFFu, smin);
        if (lane == 0)
            uhead[u] = make_uint4(p0, np, rcarry, min(tcarry, (uint32_t)kTabCap) | (dmax << 16) | (smin << 24));
    }
}

__global__ void __launch_bounds__(kUnitNT, 2) k_units(OctCtx c, const uint4* uhead, const uint4* pdesc,
                                                      const uint32_t* pdesc2, uint64_t n)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    UnitSmem& S = *reinterpret_cast<UnitSmem*>(smem_raw);
    const uint64_t nunits = (n + kWindow - 1) / kWindow;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 hn = blockIdx.x < nunits ? uhead[blockIdx.x] : make_uint4(0, 0, 0, 0);
    for (uint64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        // piece descriptors of the window (k_unit_desc); the next window's
        // header is in flight while this one is worked on
        {
            const uint4 h = hn;
            if (u + gridDim.x < nunits) hn = uhead[u + gridDim.x];
            if (threadIdx.x == 0) {
                S.p0 = h.x;
                S.np = h.y;
                S.cnt = h.z & 0xFFFFu;
                S.fcnt = h.z >> 16;
                S.tabn = h.w & 0xFFFFu;
                S.dl = (h.w >> 16) & 0xFFu;
                S.smin = h.w >> 24;
            }
            for (int pi = threadIdx.x; pi < (int)h.y; pi += kUnitNT) {
                const uint4 d = pdesc[h.x + pi];
                const uint32_t d2 = pdesc2[h.x + pi];
                S.pbeg[pi] = d.x;
                S.pn[pi] = (uint16_t)(d.y & 0xFFFFu);
                S.psrt[pi] = (uint16_t)(d.y >> 16);
                S.pcnt[pi] = (uint16_t)(d.z & 0xFFFFu);
                S.pfst[pi] = (uint16_t)(d.z >> 16);
                S.ptab[pi] = (uint16_t)(d.w & 0xFFFFu);
                S.pq[pi] = (uint8_t)(d.w >> 16);
                S.phier[pi] = (uint8_t)(d.w >> 24);
                S.pA[pi] = (uint8_t)d2;
                S.pkind[pi] = (uint8_t)(d2 >> 8);
                S.pD[pi] = (uint8_t)(d2 >> 16);
            }
        }
        __syncthreads();
        const int np = (int)S.np;
        // ---- pieces of one point: the point is its piece's minimum
        for (int pi = threadIdx.x; pi < np; pi += kUnitNT) {
            if (S.pkind[pi] != 0) continue;
            const uint4 rr = get_rec(c, S.pbeg[pi]);
            const int leafl = S.phier[pi];
            int K = (int)S.pA[pi] - c.s;
            K = K < 0 ? 0 : (K > leafl ? leafl : K);
            put_code(c, rr.z, K, leafl, rec_key(rr));
        }
        // ---- pieces of 2..32 points: lambda from the deepest level shared with any
        // point of smaller index in the piece (all pairs, by shuffles); a warp
        // loads the records of kSmallB of its pieces before working on them
        constexpr int kSmallB = 4;
        for (int pb = warp; pb < np; pb += kUnitWarps * kSmallB) {
            uint64_t kb[kSmallB];
            uint32_t jb[kSmallB];
            int nb[kSmallB];
#pragma unroll
            for (int t = 0; t < kSmallB; ++t) {
                const int pi = pb + t * kUnitWarps;
                nb[t] = pi < np && S.pkind[pi] == 1 ? (int)S.pn[pi] : 0;
                kb[t] = 0;
                jb[t] = 0xFFFFFFFFu;
                if (lane < nb[t]) {
                    const uint4 r = get_rec(c, S.pbeg[pi] + lane);
                    kb[t] = rec_key(r);
                    jb[t] = r.z;
                }
            }
#pragma unroll
            for (int t = 0; t < kSmallB; ++t) {
                const int cnum = nb[t];   // warp-uniform
                if (cnum == 0) continue;
                const int pi = pb + t * kUnitWarps;
                const uint64_t k = kb[t];
                const uint32_t jj = jb[t];
                int lm = -1;
                for (int q = 0; q < cnum; ++q) {
                    const uint64_t kt = __shfl_sync(0xFFFFFFFFu, k, q);
                    const uint32_t jt = __shfl_sync(0xFFFFFFFFu, jj, q);
                    if (jt < jj) lm = max(lm, common_level(k, kt));
                }
                if (lane < cnum) {
                    const int q0 = S.pq[pi];
                    const int lambda = lm < q0 ? (int)S.pA[pi] : lm + 1;
                    const int leafl = S.phier[pi];
                    int K = lambda - c.s;
                    K = K < 0 ? 0 : (K > leafl ? leafl : K);
                    put_code(c, jj, K, leafl, k);
                }
            }
        }
        // ---- table pieces: per-level smallest index of every occupied cell
        if (S.fcnt) {
            const int fcnt = (int)S.fcnt;
            uint32_t* tab = reinterpret_cast<uint32_t*>(S.key);
            const int tabn4 = (int)((S.tabn + 3u) >> 2);
            for (int x = threadIdx.x; x < tabn4; x += kUnitNT)
                reinterpret_cast<uint4*>(tab)[x] = make_uint4(kNone, kNone, kNone, kNone);
            for (int pi = threadIdx.x; pi < np; pi += kUnitNT)
                if (S.pkind[pi] == 4) S.pmin[pi] = kNone;
            constexpr int kPer = kUnitCap / kUnitNT;
            uint32_t gi[kPer], jq[kPer];
            uint64_t kq[kPer];
            int pp[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int r = threadIdx.x + q * kUnitNT;
                pp[q] = -1;
                gi[q] = 0;
                if (r < fcnt) {
                    pp[q] = piece_of_tab(S, np, r);
                    gi[q] = S.pbeg[pp[q]] + (uint32_t)(r - S.pfst[pp[q]]);
                }
            }
#pragma unroll
            for (int q = 0; q < kPer; ++q)   // all loads in flight together
                if (pp[q] >= 0) {
                    const uint4 r = get_rec(c, gi[q]);
                    kq[q] = rec_key(r);
                    jq[q] = r.z;
                }
            __syncthreads();   // tables cleared
            // deepest level first: a record that finds a smaller index in its cell
            // stops (that index lies in every coarser cell too); a cell's minimum
            // never does, so every cell ends with its minimum
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                if (pp[q] < 0) continue;
                const int pi = pp[q], D = S.pD[pi], q0 = S.pq[pi];
                const uint32_t jv = jq[q];
                bool least = true;
                for (int d = D; d >= 1 && least; --d) {
                    const uint32_t idx = (uint32_t)(kq[q] >> (3 * (kKeyLevels - q0 - d))) & ((1u << (3 * d)) - 1u);
                    uint32_t* t = &tab[S.ptab[pi] + tab_size(d - 1) + idx];
                    if (*t < jv) least = false;
                    else atomicMin(t, jv);
                }
                if (least && S.pmin[pi] > jv) atomicMin(&S.pmin[pi], jv);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                if (pp[q] < 0) continue;
                const int pi = pp[q], D = S.pD[pi], q0 = S.pq[pi];
                int lambda = kKeyLevels + 1;   // never its cell's minimum down to the piece's depth
                if (jq[q] == S.pmin[pi]) {
                    lambda = S.pA[pi];           // the piece minimum: from the split tree
                } else {
                    uint32_t off = S.ptab[pi];
                    for (int d = 1; d <= D; ++d) {
                        const uint32_t idx =
                            (uint32_t)(kq[q] >> (3 * (kKeyLevels - q0 - d))) & ((1u << (3 * d)) - 1u);
                        if (tab[off + idx] == jq[q]) { lambda = q0 + d; break; }
                        off += 1u << (3 * d);
                    }
                }
                const int leafl = S.phier[pi];
                int K = lambda - c.s;
                K = K < 0 ? 0 : (K > leafl ? leafl : K);
                put_code(c, jq[q], K, leafl, kq[q]);
            }
            __syncthreads();   // the tables overlay the general path's arrays
        }
        const int cnt = (int)S.cnt;
        if (cnt == 0) { __syncthreads(); continue; }
        // records; local index = position in load order
        {
            uint64_t mn = ~0ull, mx = 0;
            constexpr int kPer = kUnitCap / kUnitNT;   // records per thread
            uint32_t gi[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int r = threadIdx.x + q * kUnitNT;
                gi[q] = 0;
                if (r < cnt) {
                    const int pi = piece_of(S, np, r);
                    gi[q] = S.pbeg[pi] + (uint32_t)(r - S.psrt[pi]);
                    S.v[r] = (uint16_t)r;
                    S.piece[r] = (uint16_t)pi;
                }
            }
            uint64_t kq[kPer];
            uint32_t jq[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q)   // all loads in flight together
                if ((int)threadIdx.x + q * kUnitNT < cnt) {
                    const uint4 r = get_rec(c, gi[q]);
                    kq[q] = rec_key(r);
                    jq[q] = r.z;
                }
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int r = threadIdx.x + q * kUnitNT;
                if (r < cnt) {
                    S.key[r] = kq[q];
                    S.j[r] = jq[q];
                    mn = min(mn, kq[q]);
                    mx = max(mx, kq[q]);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, (uint64_t)__shfl_xor_sync(0xFFFFFFFFu, (unsigned long long)mn, o));
                mx = max(mx, (uint64_t)__shfl_xor_sync(0xFFFFFFFFu, (unsigned long long)mx, o));
            }
            if (lane == 0) { S.wmin[warp] = mn; S.wmax[warp] = mx; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < kUnitWarps; ++w) { mn = min(mn, S.wmin[w]); mx = max(mx, S.wmax[w]); }
                mn = min(mn, S.wmin[0]); mx = max(mx, S.wmax[0]);
                S.kmin = mn;
                S.kmax = mx;
            }
        }
        __syncthreads();
        {
            const int dl_unit = (int)S.dl;
            const int clev = common_level(S.kmin, S.kmax);
            // records already in key order down to the needed depth (every large
            // piece sorted that deep; pieces lie in key order) need no sort
            const int hi_bit = (int)S.smin >= max(dl_unit, clev) ? 0 : 3 * (kKeyLevels - clev);
            const int lo_bit = 3 * (kKeyLevels - max(dl_unit, clev));
            bool in_key = true;
            for (int sh = lo_bit; sh < hi_bit; sh += 8) {
                if (in_key) unit_sort_pass(S, S.key, S.v, S.key2, S.v2, cnt, sh);
                else unit_sort_pass(S, S.key2, S.v2, S.key, S.v, cnt, sh);
                in_key = !in_key;
            }
            if (!in_key) {
                for (int r = threadIdx.x; r < cnt; r += kUnitNT) { S.key[r] = S.key2[r]; S.v[r] = S.v2[r]; }
            }
        }
        __syncthreads();
        // ---- runs: records equal down to the sorted depth share every cell down
        // to that depth, so only the smallest index of a run can be the minimum of
        // any of those cells and the others inherit "never" (lambda beyond the
        // depth).  The search below runs over one representative per run: the
        // run's smallest index, with the run's key.
        int lo_bit_u = 0;
        {
            const int dl_unit = (int)S.dl;
            const int clev = common_level(S.kmin, S.kmax);
            lo_bit_u = 3 * (kKeyLevels - max(dl_unit, clev));
        }
        {
            constexpr int per_h = kUnitCap / kUnitNT;   // records per thread, contiguous
            const int h0 = threadIdx.x * per_h;
            uint32_t flags = 0, cntf = 0;
            for (int q = 0; q < per_h; ++q) {
                const int r = h0 + q;
                bool head = false;
                if (r < cnt) head = r == 0 || ((S.key[r] ^ S.key[r - 1]) >> lo_bit_u) != 0;
                flags |= (uint32_t)head << q;
                cntf += head;
            }
            uint32_t tot;
            const uint32_t ex0 = block_exclusive_scan<kUnitNT, uint32_t>(cntf, S.scan, tot);
            for (uint32_t x = threadIdx.x; x < tot; x += kUnitNT) S.hj[x] = 0xFFFFFFFFu;
            __syncthreads();
            int run = (int)ex0 - 1;   // run of the record before this thread's block
            uint32_t mn = 0xFFFFFFFFu;
            for (int q = 0; q < per_h; ++q) {
                const int r = h0 + q;
                if (r >= cnt) break;
                if ((flags >> q) & 1u) {
                    if (run >= 0 && mn != 0xFFFFFFFFu) atomicMin(&S.hj[run], mn);
                    ++run;
                    mn = 0xFFFFFFFFu;
                    S.key2[run] = S.key[r];
                }
                S.hid[r] = (uint16_t)run;
                mn = min(mn, S.j[S.v[r]]);
            }
            if (run >= 0 && mn != 0xFFFFFFFFu) atomicMin(&S.hj[run], mn);
            if (threadIdx.x == 0) S.nh = tot;
        }
        __syncthreads();
        const int nh = (int)S.nh;
        // ---- nearest smaller index on each side of every representative, by a
        // min-tree over hj (the leaves are hj itself, padded to a power of two
        // P >= 32): climb to the first sibling subtree that holds a smaller
        // index, then descend into it towards the near side.  The five levels
        // above the leaves are built per warp with shuffles, the rest by one
        // warp.  The level shared with that neighbour is the deepest level at
        // which the representative is not its cell's minimum on that side (keys
        // are sorted, so nearer records share at least as many levels).
        int P = 32;
        while (P < nh) P <<= 1;
        for (int b = warp; b < (P >> 5); b += kUnitWarps) {
            const int i = (b << 5) + lane;
            uint32_t v = i < nh ? S.hj[i] : 0xFFFFFFFFu;
#pragma unroll
            for (int t = 1; t <= 5; ++t) {
                v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, 1 << (t - 1)));
                if ((lane & ((1 << t) - 1)) == 0) S.mt[(P + i) >> t] = v;
            }
        }
        __syncthreads();
        if (warp == 0) {
            for (int m = P >> 6; m >= 1; m >>= 1) {
                for (int k = m + lane; k < 2 * m; k += 32) S.mt[k] = min(S.mt[2 * k], S.mt[2 * k + 1]);
                __syncwarp();
            }
        }
        __syncthreads();
        auto tv = [&](int k) -> uint32_t {
            return k >= P ? (k - P < nh ? S.hj[k - P] : 0xFFFFFFFFu) : S.mt[k];
        };
        for (int r = threadIdx.x; r < nh; r += kUnitNT) {
            const uint32_t jr = S.hj[r];
            const uint64_t kr = S.key2[r];
            int left = -1, right = -1;
            for (int k = P + r; k > 1; k >>= 1) {
                if ((k & 1) && tv(k - 1) < jr) {
                    k = k - 1;
                    while (k < P) k = tv(2 * k + 1) < jr ? 2 * k + 1 : 2 * k;
                    left = k - P;
                    break;
                }
            }
            for (int k = P + r; k > 1; k >>= 1) {
                if (!(k & 1) && tv(k + 1) < jr) {
                    k = k + 1;
                    while (k < P) k = tv(2 * k) < jr ? 2 * k : 2 * k + 1;
                    right = k - P;
                    break;
                }
            }
            S.cl[r] = left >= 0 ? (uint8_t)common_level(kr, S.key2[left]) : (uint8_t)255;
            S.cr[r] = right >= 0 ? (uint8_t)common_level(kr, S.key2[right]) : (uint8_t)255;
        }
        __syncthreads();
        // ---- deep subtrees inside pieces whose node is still inner: one warp per piece
        for (int pi = warp; pi < np; pi += kUnitWarps) {
            if (S.phier[pi] != kInner || S.pcnt[pi] == 0) continue;
            const int ps0 = S.psrt[pi], pn = S.pcnt[pi];
            int st_b[8 * 22], st_e[8 * 22], st_l[8 * 22];   // used by lane 0 only
            int sp = 0;
            if (lane == 0) { st_b[0] = ps0; st_e[0] = ps0 + pn; st_l[0] = S.pq[pi]; sp = 1; }
            for (;;) {
                int nb_ = 0, ne_ = 0, L = 0, more = 0;
                if (lane == 0 && sp > 0) { --sp; nb_ = st_b[sp]; ne_ = st_e[sp]; L = st_l[sp]; more = 1; }
                more = __shfl_sync(0xFFFFFFFFu, more, 0);
                if (!more) break;
                nb_ = __shfl_sync(0xFFFFFFFFu, nb_, 0);
                ne_ = __shfl_sync(0xFFFFFFFFu, ne_, 0);
                L = __shfl_sync(0xFFFFFFFFu, L, 0);
                const int L1 = L + 1;
                const int sh = 3 * (kKeyLevels - L1);
                int lo = ne_;
                if (lane <= 8) {   // lane d: first position whose child digit is >= d
                    int a2 = nb_, b2 = ne_;
                    while (a2 < b2) {
                        int mid = (a2 + b2) >> 1;
                        if ((int)((S.key[mid] >> sh) & 7) < lane) a2 = mid + 1;
                        else b2 = mid;
                    }
                    lo = a2;
                }
                for (int d = 0; d < 8; ++d) {
                    const int cb = __shfl_sync(0xFFFFFFFFu, lo, d);
                    const int ce = __shfl_sync(0xFFFFFFFFu, lo, d + 1);
                    const int cn = ce - cb;
                    if (cn <= 0) continue;
                    const bool leaf = (uint64_t)cn <= c.C || L1 == c.lmax;
                    if (lane == 0) {
                        emit_node(c, S.key[cb] >> sh, L1, (uint32_t)cn, S.pbeg[pi] + (uint32_t)(cb - ps0), leaf);
                        if (!leaf && sp < 8 * 22) { st_b[sp] = cb; st_e[sp] = ce; st_l[sp] = L1; ++sp; }
                    }
                    if (leaf)
                        for (int r = cb + lane; r < ce; r += 32) S.leaf[r] = (uint8_t)L1;
                }
            }
        }
        __syncthreads();
        // ---- owner level and leaf level of every record
        for (int r = threadIdx.x; r < cnt; r += kUnitNT) {
            const int vv = S.v[r];
            const int pi = S.piece[vv];
            const int h = S.hid[r];
            int lm = kKeyLevels;   // not its run's minimum: shares the sorted depth with a smaller index
            if (S.j[vv] == S.hj[h]) {
                const int ql = S.cl[h] == 255 ? -1 : (int)S.cl[h];
                const int qr = S.cr[h] == 255 ? -1 : (int)S.cr[h];
                lm = max(ql, qr);
            }
            const int q = S.pq[pi];
            const int lambda = lm < q ? (int)S.pA[pi] : lm + 1;   // the piece minimum: from the split tree
            const int leafl = S.phier[pi] == kInner ? (int)S.leaf[r] : (int)S.phier[pi];
            int K = lambda - c.s;
            if (K < 0) K = 0;
            if (K > leafl) K = leafl;
            const uint32_t jj = S.j[vv];
            put_code(c, jj, K, leafl, S.key[r]);
        }
        __syncthreads();
    }
}

// oversized pieces (more than kPieceMax identical keys down to the deepest
// needed level): only their first record, the smallest index, can be a minimum
__global__ void __launch_bounds__(256) k_dup_pieces(OctCtx c)
{
    __shared__ uint32_t s_min[8];
    const uint32_t nd = *c.ndups < c.piece_cap ? *c.ndups : c.piece_cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t k = blockIdx.x; k < nd; k += gridDim.x) {
        const Piece p = c.pieces[c.dups[k]];
        const int leafl = p.hier == kInner ? c.lmax : (int)p.hier;
        uint32_t mn = kNone;
        for (uint32_t r = threadIdx.x; r < p.count; r += blockDim.x) mn = min(mn, get_rec(c, (uint64_t)p.begin + r).z);
        mn = __reduce_min_sync(0xFFFFFFFFu, mn);
        if (lane == 0) s_min[warp] = mn;
        __syncthreads();
        mn = s_min[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mn = min(mn, s_min[w]);
        for (uint32_t r = threadIdx.x; r < p.count; r += blockDim.x) {
            const uint4 rr = get_rec(c, (uint64_t)p.begin + r);
            const uint32_t jj = rr.z;
            int K = leafl;
            if (jj == mn) {
                K = (int)p.A - c.s;
                if (K < 0) K = 0;
                if (K > leafl) K = leafl;
            }
            put_code(c, jj, K, leafl, rec_key(rr));
        }
        __syncthreads();
    }
}

__global__ void k_piece_keys(const Piece* pieces, const uint32_t* npieces, uint32_t cap, uint64_t* keys)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t np = *npieces < cap ? *npieces : cap;
    if (i < np) keys[i] = pieces[i].begin;
}

__global__ void k_clamp(uint32_t* v, uint32_t cap)
{
    if (*v > cap) *v = cap;
}

// ------------------------------------------------------------ node table
__global__ void k_node_keys(const NodeRec* nrec, const uint32_t* nnode, uint64_t* start, uint32_t* level, int lmax)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *nnode) return;
    NodeRec r = nrec[i];
    start[i] = r.key << (3 * (lmax - r.level));
    level[i] = r.level;
}

// preorder id of node (level, start); kNone when absent
FP_DEV uint32_t node_lookup(const uint64_t* sorted_start, const uint8_t* sorted_level, uint32_t M, uint64_t start,
                            int level)
{
    uint32_t a = 0, b = M;
    while (a < b) {
        uint32_t m = (a + b) >> 1;
        if (sorted_start[m] < start) a = m + 1;
        else b = m;
    }
    if (a >= M || sorted_start[a] != start || (int)sorted_level[a] > level) return kNone;
    uint32_t id = a + (uint32_t)(level - (int)sorted_level[a]);
    if (id >= M || sorted_start[id] != start || (int)sorted_level[id] != level) return kNone;
    return id;
}

// fp_node records in preorder; lookup structures for the id resolution
__global__ void k_node_write(const NodeRec* nrec, const uint32_t* nnode, const uint32_t* order,
                             const uint64_t* sorted_start, uint8_t* sorted_level, fp_node* nodes, uint32_t node_cap,
                             uint32_t* num_nodes, uint32_t* idxtab, uint32_t* leafw, int g, int lmax, uint32_t* err)
{
    const uint32_t M = *nnode;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *num_nodes = M;
        if (M > node_cap) raise(err, FP_ERR_CAPACITY, 8);
    }
    if (i >= M) return;
    NodeRec r = nrec[order[i]];
    sorted_level[i] = r.level;
    leafw[i] = r.is_leaf ? r.count : 0;
    if (r.level <= g) idxtab[((1ull << (3 * r.level)) - 1) / 7 + r.key] = i;
}

__global__ void k_node_fill(const NodeRec* nrec, const uint32_t* nnode, const uint32_t* order,
                            const uint64_t* sorted_start, const uint8_t* sorted_level, fp_node* nodes,
                            uint32_t node_cap, uint32_t* ndesc, int lmax)
{
    const uint32_t M = *nnode;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    NodeRec r = nrec[order[i]];
    fp_node o;
    o.key = r.key;
    o.first = 0;
    o.leaf_first = r.leaf_first;
    o.count = r.count;
    o.n_own = 0;
    uint64_t end = (r.key + 1) << (3 * (lmax - r.level));
    uint32_t a = i + 1, b = M;
    while (a < b) {
        uint32_t m = (a + b) >> 1;
        if (sorted_start[m] < end) a = m + 1;
        else b = m;
    }
    o.n_desc = a - i - 1;
    o.level = r.level;
    o.child_mask = 0;
    o.is_leaf = r.is_leaf;
    o.pad = 0;
    ndesc[i] = o.n_desc;
    if (i < node_cap) nodes[i] = o;
}

__global__ void k_node_children(const uint32_t* nnode, const uint64_t* sorted_start, const uint8_t* sorted_level,
                                fp_node* nodes, uint32_t node_cap, int lmax)
{
    const uint32_t M = *nnode;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M || i >= node_cap || sorted_level[i] == 0) return;
    const int L = sorted_level[i];
    const uint64_t key = sorted_start[i] >> (3 * (lmax - L));
    uint32_t p = node_lookup(sorted_start, sorted_level, M, (key >> 3) << (3 * (lmax - L + 1)), L - 1);
    if (p != kNone && p < node_cap) {
        // child_mask is byte 37 of the 40-byte record
        unsigned char* rec = reinterpret_cast<unsigned char*>(nodes + p);
        uint32_t* word = reinterpret_cast<uint32_t*>(rec + 36);
        atomicOr(word, (1u << (key & 7)) << 8);
    }
}

// owner and leaf ids of every distributed point; owned counts per node.
// A node at a level <= g is found from the level-g cell in the point's code
// (the id table of levels <= g); a node deeper than g lies in the subtree of its
// level-g ancestor, whose ids are consecutive in preorder: the search runs over
// that subtree only, with the point's key at max_level (32-bit for max_level
// <= 10) -- only then is the point itself read.  leafid (nullable): the leaf id.
// Owned counts are summed per tile of kResolveTile consecutive points in a
// shared-memory table keyed by node id (open addressing, bounded probes; a point
// that finds no slot adds to the global count directly), then flushed with one
// global atomic per node of the tile: consecutive points lie in one chunk, whose
// owners are few, and the nodes above the chunks (the root owns a point of every
// occupied level-s cell) are not hit by an atomic per point.
constexpr int kResolveNT = 256;
constexpr int kResolveIPT = 16;
constexpr int kResolveTile = kResolveNT * kResolveIPT;
constexpr int kOwnSlots = 1024;   // power of two
constexpr int kOwnProbes = 32;
constexpr int kResolveTabLevel = 4;   // node ids of the levels 0..4 in shared memory
constexpr int kResolveTab = ((1 << (3 * (kResolveTabLevel + 1))) - 1) / 7;

FP_DEV void own_add(uint32_t* keys, uint32_t* cnt, uint32_t* n_own, uint32_t id, uint32_t v)
{
    uint32_t h = (id * 2654435761u) & (kOwnSlots - 1);
    for (int q = 0; q < kOwnProbes; ++q) {
        uint32_t k = keys[h];
        if (k == kNone) {
            k = atomicCAS(&keys[h], kNone, id);
            if (k == kNone) k = id;
        }
        if (k == id) { atomicAdd(&cnt[h], v); return; }
        h = (h + 1) & (kOwnSlots - 1);
    }
    atomicAdd(&n_own[id], v);   // the table is crowded: straight to the global count
}

// id of the node at level L > g holding distributed point j (kNone when absent):
// by binary search among the descendants of its level-g cell's node, on the
// point's key at max_level
template <bool SMALL>
__device__ __noinline__ uint32_t deep_id(const fp_point* __restrict__ pts, uint64_t j, const CubeDev& cb, float scale_l,
                                         uint32_t cell, int L, const uint32_t* idxtab, const uint64_t* sorted_start,
                                         const uint8_t* sorted_level, const uint32_t* ndesc, uint32_t M, int g, int lmax)
{
    const uint32_t c0 = idxtab[((1ull << (3 * g)) - 1) / 7 + cell];
    if (L > lmax || c0 >= M) return kNone;
    const int4 p = ld_point(pts, j);
    const uint64_t kl = SMALL ? (uint64_t)key_small(p.x, p.y, p.z, cb, scale_l, lmax)
                              : key21(p.x, p.y, p.z, cb) >> (3 * (kKeyLevels - lmax));
    const uint64_t k = kl >> (3 * (lmax - L));
    const uint32_t rr =
        node_lookup(sorted_start + c0, sorted_level + c0, min(ndesc[c0] + 1, M - c0), k << (3 * (lmax - L)), L);
    return rr != kNone ? c0 + rr : kNone;
}

template <bool SMALL>
__global__ void __launch_bounds__(kResolveNT) k_resolve(const fp_point* __restrict__ pts, uint64_t n,
                                                        const fp_cube* cube, const uint32_t* codes,
                                                        const uint32_t* idxtab, const uint64_t* sorted_start,
                                                        const uint8_t* sorted_level, const uint32_t* ndesc,
                                                        const uint32_t* nnode, uint32_t* owner, uint32_t* leafid,
                                                        uint32_t* n_own, int g, int lmax, uint32_t* err)
{
    __shared__ uint32_t s_key[kOwnSlots], s_cnt[kOwnSlots];
    __shared__ uint32_t s_idx[kResolveTab];   // the node ids of the coarse levels' cells
    const CubeDev cb = load_cube(cube);
    const int tl = min(g, kResolveTabLevel);
    const uint32_t ntab = ((1u << (3 * (tl + 1))) - 1) / 7;
    for (uint32_t q = threadIdx.x; q < ntab; q += kResolveNT) s_idx[q] = idxtab[q];
    const float scale_l = SMALL ? scale_at(cb, lmax) : 0.f;
    const uint32_t M = *nnode;
    const int nt = leafid ? 2 : 1;
    const uint64_t ntiles = (n + kResolveTile - 1) / kResolveTile;
    for (int q = threadIdx.x; q < kOwnSlots; q += kResolveNT) { s_key[q] = kNone; s_cnt[q] = 0; }
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();   // the table is clear
        const uint64_t base = t * kResolveTile;
        uint32_t cw[kResolveIPT];
#pragma unroll
        for (int r = 0; r < kResolveIPT; ++r) {   // all loads in flight together
            const uint64_t j = base + (uint64_t)r * kResolveNT + threadIdx.x;
            cw[r] = j < n ? codes[j] : 0u;
        }
#pragma unroll 4
        for (int r = 0; r < kResolveIPT; ++r) {
            const uint64_t j = base + (uint64_t)r * kResolveNT + threadIdx.x;
            uint32_t oid = kNone;
            if (j < n) {
                const uint32_t cell = code_cell(cw[r]);
                const int ks[2] = {code_own(cw[r]), code_leaf(cw[r])};
                uint32_t ids[2] = {0u, 0u};
                for (int u = 0; u < nt; ++u) {
                    const int L = ks[u];
                    if (L <= tl)
                        ids[u] = s_idx[((1u << (3 * L)) - 1) / 7 + (cell >> (3 * (g - L)))];
                    else if (L <= g)
                        ids[u] = idxtab[((1ull << (3 * L)) - 1) / 7 + (cell >> (3 * (g - L)))];
                    else   // (kept out of the unrolled loop: its code is large and rarely run)
                        ids[u] = deep_id<SMALL>(pts, j, cb, scale_l, cell, L, idxtab, sorted_start, sorted_level,
                                                ndesc, M, g, lmax);
                }
                if (ids[0] >= M || ids[1] >= M) {   // never for a consistent tree
                    raise(err, FP_ERR_CAPACITY, 9);
                    ids[0] = ids[1] = 0;
                }
                owner[j] = ids[0];
                if (leafid) leafid[j] = ids[1];
                oid = ids[0];
            }
            if (oid != kNone) own_add(s_key, s_cnt, n_own, oid, 1u);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kOwnSlots; q += kResolveNT) {   // flush, and clear for the next tile
            const uint32_t k = s_key[q];
            if (k != kNone) {
                atomicAdd(&n_own[k], s_cnt[q]);
                s_key[q] = kNone;
                s_cnt[q] = 0;
            }
        }
    }
}

__global__ void k_write_nown(fp_node* nodes, const uint32_t* nnode, uint32_t node_cap, const uint32_t* n_own)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *nnode && i < node_cap) nodes[i].n_own = n_own[i];
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

__global__ void k_level_keys(const uint32_t* level, const uint32_t* nnode, uint64_t* keys)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *nnode) keys[i] = level[i];
}

__global__ void k_gather_u64(const uint64_t* src, const uint32_t* idx, const uint32_t* nn, uint64_t* dst)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *nn) dst[i] = src[idx[i]];
}

// ------------------------------------------------------------ host: octree
struct OctLayout {
    uint64_t cells, npyr, piece_cap, open_cap, node_cap;
};

static OctLayout oct_layout(uint64_t n, const fp_params& p)
{
    OctLayout L;
    L.cells = 1ull << (3 * p.grid_log2);
    L.npyr = (L.cells - 1) / 7;
    L.piece_cap = L.cells + 16 * (n / kPieceMax) + 4096;
    L.open_cap = n / kPieceMax + 1024;
    const uint64_t upper = (L.cells * 8 - 1) / 7;
    const uint64_t C = p.node_capacity ? p.node_capacity : 1;
    // every deep node is a child of an inner node, and an inner node holds more than C points:
    // at most n / C inner nodes per level, 8 children each
    uint64_t deep = 8 * (n / C + 1) * (uint64_t)(p.max_level - p.grid_log2 + 1) + 4096;
    if (deep > 2 * n + 4096) deep = 2 * n + 4096;
    L.node_cap = upper + deep;
    if (L.node_cap > 0xFFFFFFF0ull) L.node_cap = 0xFFFFFFF0ull;
    return L;
}

uint64_t node_capacity_bound(uint64_t n, const fp_params& p) { return oct_layout(n, p).node_cap; }

struct OctBufs {
    SortScratch sc;
    uint32_t* rcnt;        // counting slots of a split round: 8^3 per open node
    uint32_t* rmin;        // the smallest index of every slot
    uint4* trec;   // split rounds: the copied records with their slots
    int4* lt_pt;
    uint32_t *lt_val, *lt_k32;
    uint32_t *pyr, *cstart, *cursor;
    uint8_t* cell_leaf;
    uint4* rec;           // cell-grouped records (rec_key, rec_j)
    Piece* pieces;
    uint32_t* counters;   // [0] pieces, [1] pieces of equal keys, [3] node records
    uint32_t* dups;
    uint64_t *pk, *pk2, *pk3;
    uint32_t *pv, *pv2;
    OpenNode* open[2];
    uint32_t *ocount, *bigstart;
    NodeRec* nrec;
    uint64_t *nk, *nk2, *nk3, *nk4;
    uint32_t *nl, *nv2, *nv3;
    uint8_t* slevel;
    uint32_t *idxtab, *leafw, *nown;
    uint32_t* codes;
    uint32_t* leafid;
    uint32_t* unit_p0;
    uint4 *pdesc, *uhead;   // window descriptors (k_unit_desc)
    uint32_t* pdesc2;
    uint32_t* ndesc;
    SegScratch seg;
};

// one carve-up serves both the size query (base == nullptr) and the launch
static OctBufs oct_carve(const Workspace& ws, uint64_t n, const OctLayout& Ly)
{
    OctBufs B;
    const uint64_t N = n ? n : 1;
    B.sc = take_sort_scratch(ws, std::max<uint64_t>(N, std::max(Ly.node_cap, Ly.piece_cap)));
    B.rcnt = ws.take<uint32_t>(Ly.open_cap << (3 * kRoundLevels));
    B.rmin = ws.take<uint32_t>(Ly.open_cap << (3 * kRoundLevels));
    // aliased phase region: grouping temporaries, later the leaf scatter temporaries
    const size_t phase_base = ws.used;
    B.trec = ws.take<uint4>(N);
    const size_t phase_end = ws.used;
    ws.used = phase_base;
    B.lt_pt = ws.take<int4>(N); B.lt_val = ws.take<uint32_t>(N); B.lt_k32 = ws.take<uint32_t>(N);
    ws.used = std::max(phase_end, ws.used);
    B.pyr = ws.take<uint32_t>(Ly.npyr ? Ly.npyr : 1);
    B.cstart = ws.take<uint32_t>(Ly.cells + 1);
    B.cursor = ws.take<uint32_t>(Ly.cells);
    B.cell_leaf = ws.take<uint8_t>(Ly.cells);
    B.rec = ws.take<uint4>(N);
    B.pieces = ws.take<Piece>(Ly.piece_cap);
    B.counters = ws.take<uint32_t>(4);
    B.dups = ws.take<uint32_t>(Ly.piece_cap);
    B.pk = ws.take<uint64_t>(Ly.piece_cap); B.pk2 = ws.take<uint64_t>(Ly.piece_cap);
    B.pk3 = ws.take<uint64_t>(Ly.piece_cap);
    B.pv = ws.take<uint32_t>(Ly.piece_cap); B.pv2 = ws.take<uint32_t>(Ly.piece_cap);
    B.open[0] = ws.take<OpenNode>(Ly.open_cap); B.open[1] = ws.take<OpenNode>(Ly.open_cap);
    B.ocount = ws.take<uint32_t>(4);
    B.bigstart = ws.take<uint32_t>(Ly.open_cap + 1);
    B.nrec = ws.take<NodeRec>(Ly.node_cap);
    B.nk = ws.take<uint64_t>(Ly.node_cap); B.nk2 = ws.take<uint64_t>(Ly.node_cap);
    B.nk3 = ws.take<uint64_t>(Ly.node_cap); B.nk4 = ws.take<uint64_t>(Ly.node_cap);
    B.nl = ws.take<uint32_t>(Ly.node_cap); B.nv2 = ws.take<uint32_t>(Ly.node_cap);
    B.nv3 = ws.take<uint32_t>(Ly.node_cap);
    B.slevel = ws.take<uint8_t>(Ly.node_cap);
    B.idxtab = ws.take<uint32_t>(Ly.cells * 8 / 7 + 8);
    B.leafw = ws.take<uint32_t>(std::max<uint64_t>(Ly.node_cap, kScanMaxTiles));
    B.nown = ws.take<uint32_t>(Ly.node_cap);
    B.codes = ws.take<uint32_t>(N);
    B.leafid = ws.take<uint32_t>(N);
    B.unit_p0 = ws.take<uint32_t>((N + kWindow - 1) / kWindow + 2);
    B.pdesc = ws.take<uint4>(Ly.piece_cap);
    B.pdesc2 = ws.take<uint32_t>(Ly.piece_cap);
    B.uhead = ws.take<uint4>((N + kWindow - 1) / kWindow + 1);
    B.ndesc = ws.take<uint32_t>(Ly.node_cap);
    B.seg = take_seg_scratch(ws, N, Ly.cells, 1);
    return B;
}

size_t octree_ws_bytes(uint64_t n, const fp_params& p)
{
    Workspace dry;
    oct_carve(dry, n, oct_layout(n, p));
    return dry.used;
}

template <int DIG, bool CPT, bool CK64, bool CK32>
static cudaError_t run_sort(const SortScratch& sc, SortArgs a, int npass, const Workspace& ws, cudaStream_t st)
{
    for (int slot = 0; slot < npass; ++slot) {
        cudaError_t e = sort_run_pass<DIG, CPT, CK64, CK32>(sc, a, slot, ws.num_sms, st);
        if (e) return e;
    }
    return cudaSuccess;
}

// node records -> fp_node table in preorder, the level-g id table, sorted starts,
// levels and subtree sizes (the lookups of the id resolution)
struct NodeSortBufs {
    uint64_t *nk, *nk2, *nk3, *nk4;
    uint32_t *nl, *nv2, *nv3;
    uint8_t* slevel;
    uint32_t *idxtab, *leafw, *ndesc;
};

static cudaError_t node_table(const SortScratch& sc, const NodeRec* nrec, uint32_t* nnode, uint32_t ncap,
                              const NodeSortBufs& B, fp_node* nodes, uint32_t node_cap, uint32_t* num_nodes, int g,
                              int lmax, const Workspace& ws, cudaStream_t st)
{
    cudaError_t e;
    const unsigned gn = (ncap + 255) / 256;
    k_clamp<<<1, 1, 0, st>>>(nnode, ncap);
    k_node_keys<<<gn, 256, 0, st>>>(nrec, nnode, B.nk, B.nl, lmax);
    k_level_keys<<<gn, 256, 0, st>>>(B.nl, nnode, B.nk3);
    if ((e = sort_plan_keys(sc, B.nk3, ncap, nnode, 0, 5, st))) return e;
    SortArgs a{};
    a.b.k64_src = B.nk3; a.b.k64_tmp = B.nk2; a.b.k64_dst = B.nk4;
    a.b.val_src = nullptr; a.b.val_tmp = B.nv2; a.b.val_dst = B.nv3;
    a.n = ncap; a.d_n = nnode; a.err = ws.err;
    if ((e = run_sort<DIG_K64, false, true, false>(sc, a, sort_passes(5), ws, st))) return e;
    k_gather_u64<<<gn, 256, 0, st>>>(B.nk, B.nv3, nnode, B.nk3);
    if ((e = sort_plan_keys(sc, B.nk3, ncap, nnode, 0, (uint32_t)std::max(1, 3 * lmax), st))) return e;
    SortArgs b2{};
    b2.b.k64_src = B.nk3; b2.b.k64_tmp = B.nk2; b2.b.k64_dst = B.nk;   // nk <- sorted starts
    b2.b.val_src = B.nv3; b2.b.val_tmp = B.nv2; b2.b.val_dst = B.nl;   // nl <- record of preorder position
    b2.n = ncap; b2.d_n = nnode; b2.err = ws.err;
    if ((e = run_sort<DIG_K64, false, true, false>(sc, b2, sort_passes(3 * lmax), ws, st))) return e;
    k_node_write<<<gn, 256, 0, st>>>(nrec, nnode, B.nl, B.nk, B.slevel, nodes, node_cap, num_nodes, B.idxtab, B.leafw,
                                     g, lmax, ws.err);
    k_node_fill<<<gn, 256, 0, st>>>(nrec, nnode, B.nl, B.nk, B.slevel, nodes, node_cap, B.ndesc, lmax);
    k_node_children<<<gn, 256, 0, st>>>(nnode, B.nk, B.slevel, nodes, node_cap, lmax);
    return cudaGetLastError();
}

// append the node records of a chunk group to the caller's array
__global__ void k_append_nodes(const NodeRec* rec, const uint32_t* nrec, uint32_t cap_ws, NodeRec* out,
                               uint32_t* nout, uint32_t out_cap, uint32_t* err)
{
    const uint32_t M = min(*nrec, cap_ws), base = *nout;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
        if (base + i < out_cap) out[base + i] = rec[i];
        else raise(err, FP_ERR_CAPACITY, 10);
    }
}

__global__ void k_add_u32(uint32_t* a, const uint32_t* b, uint32_t cap_b) { *a += min(*b, cap_b); }

cudaError_t launch_octree(const fp_point* sorted, const uint32_t* perm, uint64_t n, const fp_cube* cube,
                          const fp_chunk* chunks, const uint32_t* num_chunks, const uint64_t* offsets,
                          const uint32_t* counts, const fp_params& prm, fp_node* nodes, uint32_t node_cap,
                          uint32_t* num_nodes, fp_point* leaf_pts, uint32_t* leaf_perm, uint32_t* owner,
                          const Workspace& ws, cudaStream_t st)
{
    return launch_octree_impl(sorted, perm, n, cube, chunks, num_chunks, offsets, counts, prm, nodes, node_cap,
                              num_nodes, leaf_pts, leaf_perm, owner, nullptr, ws, st);
}

cudaError_t launch_octree_impl(const fp_point* sorted, const uint32_t* perm, uint64_t n, const fp_cube* cube,
                               const fp_chunk* chunks, const uint32_t* num_chunks, const uint64_t* offsets,
                               const uint32_t* counts, const fp_params& prm, fp_node* nodes, uint32_t node_cap,
                               uint32_t* num_nodes, fp_point* leaf_pts, uint32_t* leaf_perm, uint32_t* owner,
                               const OctGroup* grp, const Workspace& ws, cudaStream_t st)
{
    cudaError_t e;
    if (n == 0) {
        if (!grp) k_set_u32<<<1, 1, 0, st>>>(num_nodes, 0);
        return cudaGetLastError();
    }
    const uint32_t* rcounts = grp ? grp->rec_counts : counts;
    const int g = (int)prm.grid_log2, s = (int)prm.sub_log2, lmax = (int)prm.max_level;
    const int dl = std::min(kKeyLevels, std::max(s + lmax - 1, g + 1));
    const OctLayout Ly = oct_layout(n, prm);
    const uint64_t N = n;
    const OctBufs B = oct_carve(ws, n, Ly);
    const SortScratch& sc = B.sc;
    uint32_t* npieces = B.counters;
    uint32_t* nnode = B.counters + 3;
    if ((e = cudaMemsetAsync(B.counters, 0, 4 * sizeof(uint32_t), st))) return e;
    if ((e = cudaMemsetAsync(B.ocount, 0, 4 * sizeof(uint32_t), st))) return e;

    // 1. pyramid and per-cell starts
    for (int l = g - 1; l >= 0; --l) {
        uint64_t np_ = 1ull << (3 * l);
        const uint32_t* child = l + 1 == g ? counts : B.pyr + ((1ull << (3 * (l + 1))) - 1) / 7;
        k_pyr_level<<<(unsigned)((np_ + 255) / 256), 256, 0, st>>>(child, B.pyr + (np_ - 1) / 7, np_);
    }
    if ((e = scan_exclusive<uint32_t, uint32_t>(rcounts, B.cstart, Ly.cells, nullptr, B.leafw, B.cstart + Ly.cells,
                                                (uint32_t*)nullptr, st)))
        return e;
    OctCtx c;
    c.counts = counts; c.rcounts = rcounts; c.leaf_base = grp ? grp->leaf_base : 0u;
    c.pyr = B.pyr; c.cstart = B.cstart; c.cell_leaf = B.cell_leaf;
    c.rec = B.rec; c.pieces = B.pieces; c.npieces = npieces; c.piece_cap = (uint32_t)Ly.piece_cap;
    c.dups = B.dups; c.ndups = B.counters + 1;
    c.nrec = B.nrec; c.nnode = nnode; c.node_cap_ws = (uint32_t)Ly.node_cap;
    c.codes = grp ? grp->codes : B.codes;
    c.open_cap = (uint32_t)Ly.open_cap;
    c.g = g; c.s = s; c.lmax = lmax; c.dl = dl; c.C = prm.node_capacity; c.n = N; c.err = ws.err;

    // 2. group by level-g cell: (key21, j) scattered by cell id
    {
        const int gcell = (int)std::max<uint64_t>(1, std::min<uint64_t>((Ly.cells + 255) / 256, ws.num_sms * 8ull));
        k_cell_cursor_init<<<gcell, 256, 0, st>>>(B.cstart, Ly.cells, B.cursor, g);
        const int gs = (int)std::max<uint64_t>(1, std::min<uint64_t>((N + 255) / 256, (uint64_t)ws.num_sms * 8));
        KTimerScope kt(FP_KERNEL_CELL_GROUP, st);
        k_cell_scatter<<<gs, 256, 0, st>>>(reinterpret_cast<const int4*>(sorted), N, cube, B.cursor, B.rec, g,
                                           ws.err);
        k_cell_check<<<gcell, 256, 0, st>>>(B.cstart, Ly.cells, B.cursor, g, ws.err);
    }
    // 3. cells: pieces, leaf levels, open big cells
    k_cell_setup<<<(unsigned)((Ly.cells + 255) / 256), 256, 0, st>>>(c, B.open[0], B.ocount);
    // 4. big cells: split tree.  Rounds of up to three levels: the records of
    // the open nodes are grouped by their cell three levels down (one counting
    // scatter: copy out with per-(node, cell) counts, starts, scatter back),
    // which puts them in key order down to that depth; then the splits of
    // those levels, whose children still too large stay open for the next round.
    {
        KTimerScope kt(FP_KERNEL_SPLIT_ROUNDS, st);
        const uint32_t cap = (uint32_t)Ly.open_cap;
        int gw = std::max(1, std::min(ws.num_sms * 16, (int)(((uint64_t)cap * 32 + 255) / 256)));
        const int gr = std::max(1, std::min(ws.num_sms * 8, (int)((N + 255) / 256)));
        int cur = 0;
        for (int q = g; q < dl;) {
            const int k = std::min(kRoundLevels, dl - q);
            const int nd = 1 << (3 * k);
            k_open_counts<<<(cap + 255) / 256, 256, 0, st>>>(B.open[cur], B.ocount + cur, B.bigstart, cap, nullptr, 0);
            if ((e = scan_exclusive<uint32_t, uint32_t>(B.bigstart, B.bigstart, cap, nullptr, B.leafw, B.ocount + 3,
                                                        (uint32_t*)nullptr, st)))
                return e;
            k_round_zero<<<gr, 256, 0, st>>>(B.ocount + cur, cap, nd, B.rcnt, B.rmin);
            k_round_copy<<<gr, 256, 0, st>>>(B.open[cur], B.ocount + cur, cap, B.bigstart, B.ocount + 3, B.rec,
                                             B.trec, 3 * (kKeyLevels - q - k), (uint32_t)(nd - 1), B.rcnt, B.rmin);
            k_round_bases<<<gw, 256, 0, st>>>(B.open[cur], B.ocount + cur, cap, nd, B.rcnt);
            k_round_scatter<<<gr, 256, 0, st>>>(B.ocount + 3, B.trec, B.rcnt, B.rec, N, ws.err);
            for (int l = q; l < q + k; ++l) {
                k_set_u32<<<1, 1, 0, st>>>(B.ocount + (1 - cur), 0);
                k_split<<<gw, 256, 0, st>>>(c, B.open[cur], B.ocount + cur, B.open[1 - cur], B.ocount + (1 - cur),
                                            cap, q + k, B.rmin, q);
                cur = 1 - cur;
            }
            q += k;
        }
    }
    // 5. nodes at levels <= g (a chunk group leaves them to the whole-cloud node table)
    if (!grp) {
        uint64_t total = (Ly.cells * 8 - 1) / 7;
        k_nodes_upper<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(c);
    }
    // 6. pieces in record order, then the units
    {
        const uint32_t pcap = (uint32_t)Ly.piece_cap;
        k_clamp<<<1, 1, 0, st>>>(npieces, pcap);
        k_piece_keys<<<(pcap + 255) / 256, 256, 0, st>>>(B.pieces, npieces, pcap, B.pk);
        int bits = 1;
        while ((1ull << bits) <= N) ++bits;
        if ((e = sort_plan_keys(sc, B.pk, pcap, npieces, 0, (uint32_t)bits, st))) return e;
        SortArgs a{};
        a.b.k64_src = B.pk; a.b.k64_tmp = B.pk2; a.b.k64_dst = B.pk3;
        a.b.val_src = nullptr; a.b.val_tmp = B.pv2; a.b.val_dst = B.pv;
        a.n = pcap; a.d_n = npieces; a.err = ws.err;
        if ((e = run_sort<DIG_K64, false, true, false>(sc, a, sort_passes(bits), ws, st))) return e;
        const size_t smem = sizeof(UnitSmem);
        if ((e = cudaFuncSetAttribute(k_units, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
        const uint64_t nunits = (N + kWindow - 1) / kWindow;
        k_unit_ranges<<<(unsigned)((nunits + 1 + 255) / 256), 256, 0, st>>>(B.pk3, npieces, pcap, nunits, B.unit_p0);
        const int gd =
            (int)std::max<uint64_t>(1, std::min<uint64_t>((nunits * 32 + 255) / 256, (uint64_t)ws.num_sms * 8));
        k_unit_desc<<<gd, 256, 0, st>>>(c, B.unit_p0, B.pv, nunits, B.pdesc, B.pdesc2, B.uhead);
        int grid = (int)std::min<uint64_t>(nunits, (uint64_t)ws.num_sms * 2);
        {
            KTimerScope kt(FP_KERNEL_UNITS, st);
            k_units<<<grid, kUnitNT, smem, st>>>(c, B.uhead, B.pdesc, B.pdesc2, N);
        }
        k_dup_pieces<<<ws.num_sms, 256, 0, st>>>(c);
    }
    if (grp) {   // a chunk group: its nodes below level g are appended to the caller's list
        const unsigned ga = (unsigned)std::max(1, std::min(ws.num_sms * 8, (int)((Ly.node_cap + 255) / 256)));
        k_append_nodes<<<ga, 256, 0, st>>>(B.nrec, nnode, (uint32_t)Ly.node_cap, grp->deep, grp->num_deep,
                                           grp->deep_cap, ws.err);
        k_add_u32<<<1, 1, 0, st>>>(grp->num_deep, nnode, (uint32_t)Ly.node_cap);
        return cudaGetLastError();
    }
    // 7. node table in preorder: stable sort by level, then by start at max_level resolution
    {
        NodeSortBufs nb{B.nk, B.nk2, B.nk3, B.nk4, B.nl, B.nv2, B.nv3, B.slevel, B.idxtab, B.leafw, B.ndesc};
        KTimerScope kt(FP_KERNEL_NODE_TABLE, st);
        if ((e = node_table(sc, B.nrec, nnode, (uint32_t)Ly.node_cap, nb, nodes, node_cap, num_nodes, g, lmax, ws, st)))
            return e;
        if ((e = cudaMemsetAsync(B.nown, 0, (size_t)Ly.node_cap * sizeof(uint32_t), st))) return e;
    }
    // 8. owner and leaf ids per distributed point, owned counts
    {
        const int grid = (int)std::max<uint64_t>(
            1, std::min<uint64_t>((N + kResolveTile - 1) / kResolveTile, (uint64_t)ws.num_sms * 8));
        auto kres = lmax <= 10 ? k_resolve<true> : k_resolve<false>;
        KTimerScope kt(FP_KERNEL_RESOLVE, st);
        kres<<<grid, kResolveNT, 0, st>>>(sorted, N, cube, B.codes, B.idxtab, B.nk, B.slevel, B.ndesc, nnode, owner,
                                   (leaf_pts || leaf_perm) ? B.leafid : nullptr,
                                   B.nown, g, lmax, ws.err);
        k_write_nown<<<(unsigned)((Ly.node_cap + 255) / 256), 256, 0, st>>>(nodes, nnode, node_cap, B.nown);
    }
    // 9. leaf-grouped points: stable scatter by leaf id, chunk by chunk (every
    // leaf lies in the subtree of its points' chunk); the whole-array sort by
    // leaf id runs instead, gated on the device, when a chunk does not fit
    if (leaf_pts || leaf_perm) {
        KTimerScope kt(FP_KERNEL_LEAF_SCATTER, st);
        SegCall sg{};
        sg.mode = SEG_LEAF;
        sg.nodes = nodes; sg.num_nodes = num_nodes; sg.node_cap = node_cap;
        sg.chunks = chunks; sg.num_chunks = num_chunks; sg.offsets = offsets;
        sg.pt_in = leaf_pts ? reinterpret_cast<const int4*>(sorted) : nullptr;
        sg.pt_out = reinterpret_cast<int4*>(leaf_pts);
        sg.val_in = perm; sg.val_out = leaf_perm;
        sg.id_in = B.leafid;
        sg.n = N;
        sg.first = reinterpret_cast<const uint64_t*>(nodes) + offsetof(fp_node, leaf_first) / sizeof(uint64_t);
        sg.first_stride = sizeof(fp_node) / sizeof(uint64_t);
        if ((e = seg_scatter(B.seg, sg, ws, st))) return e;
        if ((e = sort_plan_weights(sc, B.leafw, nullptr, nnode, Ly.node_cap, 0, st))) return e;
        SortArgs a{};
        a.b.pt_src = reinterpret_cast<const int4*>(sorted);
        a.b.pt_tmp = B.lt_pt;
        a.b.pt_dst = reinterpret_cast<int4*>(leaf_pts);
        a.b.val_src = perm; a.b.val_tmp = B.lt_val; a.b.val_dst = leaf_perm;
        a.b.k32_src = B.leafid; a.b.k32_tmp = B.lt_k32; a.b.k32_dst = nullptr;
        a.n = N; a.d_n = B.seg.cnt + 5; a.err = ws.err;
        const int np = sort_passes(count_bits(Ly.node_cap));   // leaf ids below node_cap
        if (leaf_pts) e = run_sort<DIG_K32, true, false, true>(sc, a, np, ws, st);
        else e = run_sort<DIG_K32, false, false, true>(sc, a, np, ws, st);
        if (e) return e;
    }
    return cudaGetLastError();
}

// ------------------------------------------- whole-cloud tables (chunk groups)
__global__ void k_copy_u32(uint32_t* dst, const uint32_t* src) { *dst = *src; }

struct NodesBufs {
    SortScratch sc;
    uint32_t *pyr, *cstart;
    NodeSortBufs nb;
};

static NodesBufs nodes_carve(const Workspace& ws, const fp_params& p, uint64_t rec_cap)
{
    NodesBufs B;
    const uint64_t cells = 1ull << (3 * p.grid_log2);
    const uint64_t R = rec_cap ? rec_cap : 1;
    B.sc = take_sort_scratch(ws, R);
    B.pyr = ws.take<uint32_t>((cells - 1) / 7 ? (cells - 1) / 7 : 1);
    B.cstart = ws.take<uint32_t>(cells + 1);
    B.nb.nk2 = ws.take<uint64_t>(R); B.nb.nk3 = ws.take<uint64_t>(R); B.nb.nk4 = ws.take<uint64_t>(R);
    B.nb.nl = ws.take<uint32_t>(R); B.nb.nv2 = ws.take<uint32_t>(R); B.nb.nv3 = ws.take<uint32_t>(R);
    B.nb.leafw = ws.take<uint32_t>(std::max<uint64_t>(R, kScanMaxTiles));
    return B;
}

size_t nodes_ws_bytes(const fp_params& p, uint64_t rec_cap)
{
    Workspace dry;
    nodes_carve(dry, p, rec_cap);
    return dry.used;
}

uint64_t upper_node_bound(const fp_params& p) { return ((1ull << (3 * p.grid_log2)) * 8 - 1) / 7; }

cudaError_t launch_octree_nodes(const uint32_t* counts, const fp_params& prm, NodeRec* recs, uint64_t rec_cap,
                                const uint32_t* num_deep, fp_node* nodes, uint32_t node_cap, uint32_t* num_nodes,
                                const NodeTables& T, const Workspace& ws, cudaStream_t st)
{
    cudaError_t e;
    const int g = (int)prm.grid_log2, lmax = (int)prm.max_level;
    const uint64_t cells = 1ull << (3 * g);
    const NodesBufs B = nodes_carve(ws, prm, rec_cap);
    for (int l = g - 1; l >= 0; --l) {
        uint64_t np_ = 1ull << (3 * l);
        const uint32_t* child = l + 1 == g ? counts : B.pyr + ((1ull << (3 * (l + 1))) - 1) / 7;
        k_pyr_level<<<(unsigned)((np_ + 255) / 256), 256, 0, st>>>(child, B.pyr + (np_ - 1) / 7, np_);
    }
    if ((e = scan_exclusive<uint32_t, uint32_t>(counts, B.cstart, cells, nullptr, B.nb.leafw, B.cstart + cells,
                                                (uint32_t*)nullptr, st)))
        return e;
    k_copy_u32<<<1, 1, 0, st>>>(T.nnode, num_deep);
    OctCtx c{};
    c.counts = counts; c.rcounts = counts; c.leaf_base = 0;
    c.pyr = B.pyr; c.cstart = B.cstart; c.nrec = recs; c.nnode = T.nnode; c.node_cap_ws = (uint32_t)rec_cap;
    c.g = g; c.s = (int)prm.sub_log2; c.lmax = lmax; c.C = prm.node_capacity; c.err = ws.err;
    k_nodes_upper<<<(unsigned)((upper_node_bound(prm) + 255) / 256), 256, 0, st>>>(c);
    NodeSortBufs nb = B.nb;
    nb.nk = T.starts; nb.slevel = T.slevel; nb.idxtab = T.idxtab; nb.ndesc = T.ndesc;
    if ((e = node_table(B.sc, recs, T.nnode, (uint32_t)rec_cap, nb, nodes, node_cap, num_nodes, g, lmax, ws, st)))
        return e;
    return cudaMemsetAsync(T.nown, 0, rec_cap * sizeof(uint32_t), st);
}

cudaError_t launch_octree_resolve(const fp_point* pts, uint64_t n, const fp_cube* cube, const uint32_t* codes,
                                  const NodeTables& T, const fp_params& prm,
                                  uint32_t* owner, const Workspace& ws, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>((n + kResolveTile - 1) / kResolveTile, (uint64_t)ws.num_sms * 8));
    auto kres = prm.max_level <= 10 ? k_resolve<true> : k_resolve<false>;
    kres<<<grid, kResolveNT, 0, st>>>(pts, n, cube, codes, T.idxtab, T.starts, T.slevel, T.ndesc, T.nnode, owner, nullptr,
                               T.nown, (int)prm.grid_log2, (int)prm.max_level, ws.err);
    return cudaGetLastError();
}

// n_own of every node from the owned counts, then first = exclusive prefix of n_own
cudaError_t launch_node_first(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const uint32_t* nown,
                              uint64_t* first, uint32_t* nm, uint64_t* tiles64, cudaStream_t st);

// ------------------------------------------------------------ subsample
__global__ void k_nown_in(const fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, uint32_t* nown)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t M = *num_nodes < node_cap ? *num_nodes : node_cap;
    if (i < M) nown[i] = nodes[i].n_own;
}

__global__ void k_first_out(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const uint64_t* first)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t M = *num_nodes < node_cap ? *num_nodes : node_cap;
    if (i < M) nodes[i].first = first[i];
}

// owner segments whose original indices are not ascending (owners above the chunks)
__global__ void k_mark_unsorted(const uint32_t* fown, const uint32_t* fperm, uint64_t n, const uint32_t* d_n,
                                uint32_t* mark, const uint32_t* nm)
{
    const uint32_t M = *nm;
    if (*d_n < n) n = *d_n;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f + 1 < n; f += stride)
        if (fown[f] == fown[f + 1] && fperm[f] > fperm[f + 1] && fown[f] < M) mark[fown[f]] = 1;
}

__global__ void k_clamp_copy(const uint32_t* v, uint32_t cap, uint32_t* out) { *out = *v < cap ? *v : cap; }

__global__ void k_stitch_list(const uint32_t* mark, const uint32_t* mrank, const uint32_t* num_nodes,
                              uint32_t node_cap, uint32_t* mlist, const uint32_t* nown, uint32_t* mown)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t M = *num_nodes < node_cap ? *num_nodes : node_cap;
    if (i < M && mark[i]) {
        mlist[mrank[i]] = i;
        mown[mrank[i]] = nown[i];
    }
}

// keys (rank << 32 | original index) of the points of marked nodes, value = final position;
// one thread per stitch record, its node found by binary search over the segment offsets
__global__ void k_stitch_keys(const uint32_t* mlist, const uint32_t* nmarked, const uint32_t* soff,
                              const uint32_t* nstitch, const uint64_t* first, const uint32_t* fperm, uint64_t* key,
                              uint32_t* val)
{
    const uint32_t nm = *nmarked, S = *nstitch;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < S; t += gridDim.x * blockDim.x) {
        uint32_t a = 0, b = nm;
        while (a < b) { uint32_t m = (a + b) >> 1; if (soff[m] <= t) a = m + 1; else b = m; }
        const uint32_t r = a - 1;
        const uint64_t f = first[mlist[r]] + (t - soff[r]);
        key[t] = ((uint64_t)r << 32) | fperm[f];
        val[t] = (uint32_t)f;
    }
}

__global__ void k_stitch_gather(const uint32_t* nstitch, const uint32_t* val, const int4* fin, const uint32_t* fperm,
                                int4* tpt, uint32_t* tperm)
{
    const uint32_t S = *nstitch;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < S; t += gridDim.x * blockDim.x) {
        tpt[t] = fin[val[t]];
        tperm[t] = fperm[val[t]];
    }
}

__global__ void k_stitch_put(const uint32_t* nstitch, const uint64_t* key, const uint32_t* mlist, const uint32_t* soff,
                             const uint64_t* first, const int4* tpt, const uint32_t* tperm, int4* fin, uint32_t* fperm)
{
    const uint32_t S = *nstitch;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < S; t += gridDim.x * blockDim.x) {
        uint32_t r = (uint32_t)(key[t] >> 32);
        uint64_t f = first[mlist[r]] + (t - soff[r]);
        fin[f] = tpt[t];
        fperm[f] = tperm[t];
    }
}

// stitch records staged by the segmented scatter: a node above the chunks keeps
// all of its points through the staging area, the others none of theirs
__global__ void k_stitch_counts(const uint8_t* inside, const uint32_t* nown, const uint32_t* nm, uint32_t* scnt,
                                uint32_t cap)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    scnt[i] = i < *nm && !inside[i] ? nown[i] : 0u;
}

// sorted staging record t = (rank of node X, original index): final position
// first[X] + rank inside X
__global__ void k_stitch_place(const uint32_t* nstaged, const uint64_t* key, const uint32_t* src, int shift,
                               const uint32_t* list, const uint32_t* nlist, const uint32_t* nm, const uint32_t* soff,
                               const uint64_t* first, const int4* pts, const uint32_t* perm, uint64_t n, int4* fin,
                               uint32_t* fperm, uint32_t* err)
{
    const uint32_t S = *nstaged, M = *nm, R = *nlist;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < S; t += gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(key[t] >> shift);
        const uint32_t X = r < R ? list[r] : M;
        const uint32_t j = src[t];
        const uint64_t f = X < M ? first[X] + (t - soff[X]) : n;
        if (f >= n || j >= n) { raise(err, FP_ERR_CAPACITY, 11); continue; }
        fin[f] = __ldg(pts + j);
        fperm[f] = perm[j];
    }
}

cudaError_t launch_node_first(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const uint32_t* nown,
                              uint64_t* first, uint32_t* nm, uint64_t* tiles64, cudaStream_t st)
{
    const unsigned gM = (node_cap + 255) / 256;
    k_write_nown<<<gM, 256, 0, st>>>(nodes, num_nodes, node_cap, nown);
    k_clamp_copy<<<1, 1, 0, st>>>(num_nodes, node_cap, nm);
    cudaError_t e = scan_exclusive<uint32_t, uint64_t>(nown, first, node_cap, nm, tiles64, (uint64_t*)nullptr,
                                                       (uint64_t*)nullptr, st);
    if (e) return e;
    k_first_out<<<gM, 256, 0, st>>>(nodes, num_nodes, node_cap, first);
    return cudaGetLastError();
}

static const uint64_t kMaxScanNodes = (uint64_t)kScanTile * kScanMaxTiles;

struct SubBufs {
    SortScratch sc;
    uint32_t *nown, *mark, *mrank, *mlist, *mown, *soff, *cnt;
    uint32_t *srank, *slist;   // staging: rank of a node outside every chunk subtree, and back
    uint64_t* first;
    int4* t_pt;
    uint32_t *t_val, *t_k32, *fown;
    uint64_t *s_key, *s_key2, *s_key3;
    uint32_t *s_val, *s_val2, *s_val3;
    int4* s_pt;
    uint32_t* s_perm;
    uint64_t* tiles64;
    uint32_t* tiles32;
    uint32_t* scnt;
    SegScratch seg;
};

// chunks of a cloud of n points: at most n, and at most 8^7 count-grid cells
static uint64_t chunk_bound(uint64_t n) { return std::min<uint64_t>(n ? n : 1, 1ull << 21); }

static SubBufs sub_carve(const Workspace& ws, uint64_t n, uint64_t M)
{
    SubBufs B;
    const uint64_t N = n ? n : 1;
    B.sc = take_sort_scratch(ws, N);
    B.nown = ws.take<uint32_t>(M); B.first = ws.take<uint64_t>(M + 1);
    B.mark = ws.take<uint32_t>(M); B.mrank = ws.take<uint32_t>(M); B.mlist = ws.take<uint32_t>(M);
    B.mown = ws.take<uint32_t>(M); B.soff = ws.take<uint32_t>(M + 1); B.cnt = ws.take<uint32_t>(8);
    B.srank = ws.take<uint32_t>(M); B.slist = ws.take<uint32_t>(M);
    // One region serves three sets of per-point buffers that are never live
    // together: the whole-array path's sort temporaries and owner copy (dead
    // once its unsorted segments are marked), the stitch records and their
    // sort buffers, and the stitch's gathered points (written over the sort's
    // source and temporary, both dead after the sort).
    const size_t region = ws.used;
    B.t_pt = ws.take<int4>(N); B.t_val = ws.take<uint32_t>(N); B.t_k32 = ws.take<uint32_t>(N);
    B.fown = ws.take<uint32_t>(N);
    const size_t end_t = ws.used;
    ws.used = region;
    B.s_key = ws.take<uint64_t>(N); B.s_val = ws.take<uint32_t>(N);
    B.s_key2 = ws.take<uint64_t>(N); B.s_val2 = ws.take<uint32_t>(N);
    const size_t end_src = ws.used;
    B.s_key3 = ws.take<uint64_t>(N); B.s_val3 = ws.take<uint32_t>(N);
    const size_t end_s = ws.used;
    ws.used = region;
    B.s_pt = ws.take<int4>(N); B.s_perm = ws.take<uint32_t>(N);
    if (ws.used > end_src) {   // (20 bytes per point fit in 24 unless rounding says otherwise: then after)
        ws.used = end_s;
        B.s_pt = ws.take<int4>(N); B.s_perm = ws.take<uint32_t>(N);
    }
    ws.used = std::max(std::max(end_t, end_s), ws.used);
    B.tiles64 = ws.take<uint64_t>(kScanMaxTiles); B.tiles32 = ws.take<uint32_t>(kScanMaxTiles);
    B.scnt = ws.take<uint32_t>(M + 1);
    B.seg = take_seg_scratch(ws, N, chunk_bound(n), M);
    return B;
}

size_t subsample_ws_bytes(uint64_t n, uint64_t node_cap)
{
    Workspace dry;
    sub_carve(dry, n, std::max<uint64_t>(node_cap, 1));
    return dry.used;
}

cudaError_t launch_subsample(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const fp_point* sorted,
                             const uint32_t* perm, const uint32_t* owner, uint64_t n, const fp_chunk* chunks,
                             const uint32_t* num_chunks, const uint64_t* offsets, fp_point* final_pts,
                             uint32_t* final_perm, const Workspace& ws, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    if (node_cap > kMaxScanNodes) return cudaErrorInvalidValue;
    cudaError_t e;
    const uint64_t N = n;
    const uint32_t M = node_cap;
    const SubBufs B = sub_carve(ws, n, M);
    const SortScratch& sc = B.sc;
    uint32_t *nown = B.nown, *mark = B.mark, *mrank = B.mrank, *mlist = B.mlist, *mown = B.mown, *soff = B.soff;
    uint32_t* cnt = B.cnt;
    uint64_t* first = B.first;
    const unsigned gM = (M + 255) / 256;
    const unsigned gN = (unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)ws.num_sms * 16);

    uint32_t* nm = cnt + 2;   // node count clamped to the capacity
    uint32_t* nstaged = cnt + 3;
    k_clamp_copy<<<1, 1, 0, st>>>(num_nodes, node_cap, nm);
    k_nown_in<<<gM, 256, 0, st>>>(nodes, num_nodes, node_cap, nown);
    if ((e = scan_exclusive<uint32_t, uint64_t>(nown, first, M, nm, B.tiles64, (uint64_t*)nullptr,
                                                (uint64_t*)nullptr, st)))
        return e;
    k_first_out<<<gM, 256, 0, st>>>(nodes, num_nodes, node_cap, first);

    // 1. stable scatter by owner id, chunk by chunk; owners above the chunk are staged
    int pbits = 1;
    while ((1ull << pbits) < N) ++pbits;   // original indices are below 2^pbits
    SegCall sg{};
    sg.mode = SEG_OWNER;
    sg.nodes = nodes; sg.num_nodes = num_nodes; sg.node_cap = node_cap;
    sg.chunks = chunks; sg.num_chunks = num_chunks; sg.offsets = offsets;
    sg.pt_in = reinterpret_cast<const int4*>(sorted); sg.pt_out = reinterpret_cast<int4*>(final_pts);
    sg.val_in = perm; sg.val_out = final_perm;
    sg.id_in = owner;
    sg.n = N;
    sg.first = first; sg.first_stride = 1;
    sg.st_key = B.s_key; sg.st_src = B.s_val; sg.st_count = nstaged; sg.st_shift = pbits;
    uint32_t* nrank = cnt + 4;   // nodes outside every chunk subtree
    sg.st_rank = B.srank; sg.st_list = B.slist; sg.st_nrank = nrank; sg.st_tiles = B.tiles32;
    {
        KTimerScope kt(FP_KERNEL_OWNER_SCATTER, st);
        if ((e = seg_scatter(B.seg, sg, ws, st))) return e;
    }
    // 2. the stitch: staged records sorted by (node, original index), then placed
    KTimerScope kt_stitch(FP_KERNEL_STITCH, st);
    k_stitch_counts<<<gM, 256, 0, st>>>(B.seg.inside, nown, nm, B.scnt, M);
    if ((e = scan_exclusive<uint32_t, uint32_t>(B.scnt, soff, M, nm, B.tiles32, (uint32_t*)nullptr,
                                                (uint32_t*)nullptr, st)))
        return e;
    if ((e = sort_plan_keys(sc, B.s_key, N, nstaged, 0, (uint32_t)pbits, st, nrank))) return e;
    {
        SortArgs b{};
        b.b.k64_src = B.s_key; b.b.k64_tmp = B.s_key2; b.b.k64_dst = B.s_key3;
        b.b.val_src = B.s_val; b.b.val_tmp = B.s_val2; b.b.val_dst = B.s_val3;
        b.n = N; b.d_n = nstaged; b.err = ws.err;
        const int np = sort_passes(pbits + count_bits(M));   // node ids below M above the index bits
        for (int slot = 0; slot < np; ++slot)
            if ((e = sort_run_pass<DIG_K64, false, true, false>(sc, b, slot, ws.num_sms, st))) return e;
    }
    k_stitch_place<<<gN, 256, 0, st>>>(nstaged, B.s_key3, B.s_val3, pbits, B.slist, nrank, nm, soff, first,
                                       reinterpret_cast<const int4*>(sorted), perm, N,
                                       reinterpret_cast<int4*>(final_pts), final_perm, ws.err);
    ktimer_mark(FP_KERNEL_STITCH, false, st);   // the gated whole-array path below is not timed with it
    kt_stitch.id = FP_KERNEL_NONE;

    // whole-array path (runs with seg cnt[5] = n records when a chunk did not fit, else on none):
    // stable scatter by owner id, then the owner segments spanning several chunks re-sorted
    const uint32_t* gate = B.seg.cnt + 5;
    if ((e = sort_plan_weights(sc, nown, nullptr, nm, M, 0, st))) return e;
    SortArgs a{};
    a.b.pt_src = reinterpret_cast<const int4*>(sorted); a.b.pt_tmp = B.t_pt;
    a.b.pt_dst = reinterpret_cast<int4*>(final_pts);
    a.b.val_src = perm; a.b.val_tmp = B.t_val; a.b.val_dst = final_perm;
    a.b.k32_src = owner; a.b.k32_tmp = B.t_k32; a.b.k32_dst = B.fown;
    a.n = N; a.d_n = gate; a.err = ws.err;
    for (int slot = 0; slot < sort_passes(count_bits(M)); ++slot)
        if ((e = sort_run_pass<DIG_K32, true, false, true>(sc, a, slot, ws.num_sms, st))) return e;
    if ((e = cudaMemsetAsync(mark, 0, (size_t)M * 4, st))) return e;
    if ((e = cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), st))) return e;
    k_mark_unsorted<<<gN, 256, 0, st>>>(B.fown, final_perm, N, gate, mark, nm);
    if ((e = scan_exclusive<uint32_t, uint32_t>(mark, mrank, M, nm, B.tiles32, cnt, (uint32_t*)nullptr, st)))
        return e;
    k_stitch_list<<<gM, 256, 0, st>>>(mark, mrank, num_nodes, node_cap, mlist, nown, mown);
    if ((e = scan_exclusive<uint32_t, uint32_t>(mown, soff, M, cnt, B.tiles32, cnt + 1, (uint32_t*)nullptr, st)))
        return e;
    k_stitch_keys<<<ws.num_sms * 8, 256, 0, st>>>(mlist, cnt, soff, cnt + 1, first, final_perm, B.s_key, B.s_val);
    int rank_bits = 1;
    while ((1ull << rank_bits) < M) ++rank_bits;
    if ((e = sort_plan_keys(sc, B.s_key, N, cnt + 1, 0, (uint32_t)(32 + rank_bits), st))) return e;
    SortArgs b{};
    b.b.k64_src = B.s_key; b.b.k64_tmp = B.s_key2; b.b.k64_dst = B.s_key3;
    b.b.val_src = B.s_val; b.b.val_tmp = B.s_val2; b.b.val_dst = B.s_val3;
    b.n = N; b.d_n = cnt + 1; b.err = ws.err;
    for (int slot = 0; slot < sort_passes(32 + rank_bits); ++slot)
        if ((e = sort_run_pass<DIG_K64, false, true, false>(sc, b, slot, ws.num_sms, st))) return e;
    k_stitch_gather<<<gN, 256, 0, st>>>(cnt + 1, B.s_val3,
                                                                  reinterpret_cast<const int4*>(final_pts),
                                                                  final_perm, B.s_pt, B.s_perm);
    k_stitch_put<<<gN, 256, 0, st>>>(cnt + 1, B.s_key3, mlist, soff, first, B.s_pt,
                                                               B.s_perm, reinterpret_cast<int4*>(final_pts),
                                                               final_perm);
    return cudaGetLastError();
}

}  // namespace fp
