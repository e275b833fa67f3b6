// fp_seg.cuh -- single-pass stable scatter of the chunk array by node id, chunk
// by chunk: the leaf grouping of fp_build_chunk_octree and the owner layout of
// fp_subsample (Sec. 4.4: every chunk's local octree is a subtree of the global
// one).
//
// Inside a chunk the distributed order is index order, and every leaf of a
// chunk's points, and every owner below the chunk, lies in the subtree of the
// chunk's node, whose ids are consecutive in preorder.  So the scatter runs
// chunk by chunk with digit = node id - id of the chunk's node: tiles never
// straddle chunks, the decoupled look-back stops at the chunk's first tile, and
// the bucket bases come from the node table -- no histogram or plan passes.
// Points owned by a node above their chunk (the stitch, owner layout only) take
// the last digit and go to a staging area, merged across chunks afterwards.
//
// Two widths: chunks of at most 256 digits run on the 8-bit variant (two CTAs
// per SM), chunks of up to 2048 on the 11-bit one; a chunk with more sets the
// fail word and the caller's whole-array sort runs instead.
#pragma once
#include <cstddef>
#include "fp_sort.cuh"

namespace fp {

static_assert(sizeof(fp_node) == 40 && offsetof(fp_node, leaf_first) % 8 == 0, "fp_node layout");

constexpr int kSegSmallBits = 8;
// earlier tiles' words one look-back round trip reads per digit (16 measured
// no faster than 8 on the 10^9-point distribution)
constexpr int kSegLookBatch = 8;
constexpr int kSegMaxBits = 11;

struct SegTile {
    uint32_t chunk, index;   // chunk, and tile number inside the chunk
};

struct SegArgs {
    const int4* pt_in;                    // nullable: points not carried
    int4* pt_out;
    const uint32_t* val_in;               // original index of every record
    uint32_t* val_out;                    // nullable
    const uint32_t* id_in;                // node id of every record
    const uint64_t* offsets;              // chunk c = records [offsets[c], offsets[c + 1])
    const uint32_t* seg_lo;               // id of the chunk's node
    const uint32_t* seg_nb;               // digits of the chunk
    const SegTile* tiles;                 // this variant's tiles, each chunk's in order
    const uint32_t* d_ntiles;
    uint64_t ntiles_max;
    const uint64_t* first;                // output start of node id: first[id * first_stride]
    uint32_t first_stride;
    uint32_t* status;                     // [row][1 << MAXB], row = tile start / kSortTile
    uint32_t* counter;
    int stitch;                           // nonzero: the chunk's last digit is the staging digit
    uint64_t* st_key;                     // (node << st_shift) | original index, node = st_rank[id] or id
    const uint32_t* st_rank;              // nullable: rank of a node among those outside every chunk subtree
    uint32_t* st_src;                     // position in the chunk array
    uint32_t* st_count;
    uint64_t st_cap;
    int st_shift;
    uint64_t n;                           // bound of the output positions

    const uint32_t* d_fail;
    uint32_t* err;

    // distribution (DIST): the digit is the chunk of the point's level-g cell
    const fp_cube* cube;
    const uint32_t* lut;
    const uint32_t* cells;                // nullable: the level-g cell of every point (else computed)
    int g;
};

template <bool CPT, int MAXB, bool DIST = false>
struct SegSmem {
    using dig_t = typename std::conditional<(MAXB <= 8), uint8_t, uint16_t>::type;
    static constexpr size_t pt = CPT ? sizeof(int4) * kSortTile : 0;
    static constexpr size_t gbase = sizeof(uint64_t) * (1 << MAXB);
    static constexpr size_t val = sizeof(uint32_t) * kSortTile;
    static constexpr size_t cnt = sizeof(uint32_t) * (1 << MAXB);
    static constexpr size_t off = sizeof(uint32_t) * (1 << MAXB);
    static constexpr size_t pos = DIST ? 0 : sizeof(uint16_t) * kSortTile;   // tile position of a staged record
    static constexpr size_t dig = sizeof(dig_t) * kSortTile;
    static constexpr size_t whist = sizeof(uint16_t) * kSortWarps * (1 << MAXB);
    static constexpr size_t misc = 4 * (1 + kSortWarps + 15);
    static constexpr size_t tiles = 4 * 2;   // current and next tile id
    static constexpr size_t total = pt + gbase + val + cnt + off + pos + dig + whist + misc + tiles;
};

// two CTAs per SM while the shared memory allows it (8-bit digits; 9-bit
// digits without the staging positions, i.e. in the distribution)
template <bool CPT, int MAXB, bool DIST>
constexpr int seg_ctas() { return SegSmem<CPT, MAXB, DIST>::total <= 113 * 1024 ? 2 : 1; }

template <bool CPT, int MAXB, bool DIST = false>
__global__ void __launch_bounds__(kSortNT, (seg_ctas<CPT, MAXB, DIST>())) k_seg_pass(SegArgs a)
{
    if (*a.d_fail) return;
    CubeDev cube;
    float scale_g = 0.f;
    if (DIST && !a.cells) {
        cube = load_cube(a.cube);
        scale_g = scale_at(cube, a.g);
    }
    using SM = SegSmem<CPT, MAXB, DIST>;
    using dig_t = typename SM::dig_t;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    int4* s_pt = reinterpret_cast<int4*>(sp); sp += SM::pt;
    uint64_t* s_gbase = reinterpret_cast<uint64_t*>(sp); sp += SM::gbase;
    uint32_t* s_val = reinterpret_cast<uint32_t*>(sp); sp += SM::val;
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(sp); sp += SM::cnt;
    uint32_t* s_off = reinterpret_cast<uint32_t*>(sp); sp += SM::off;
    uint16_t* s_pos = reinterpret_cast<uint16_t*>(sp); sp += SM::pos;
    dig_t* s_dig = reinterpret_cast<dig_t*>(sp); sp += SM::dig;
    uint16_t* s_whist = reinterpret_cast<uint16_t*>(sp); sp += SM::whist;
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(sp); sp += SM::misc;
    uint32_t* s_tile = reinterpret_cast<uint32_t*>(sp);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t ntiles = min((uint64_t)*a.d_ntiles, a.ntiles_max);
    constexpr int kStride = 1 << MAXB;

    // the next tile is claimed while the current one is worked on (tiles only
    // wait on earlier tiles of their chunk, so a reserved tile cannot deadlock)
    if (threadIdx.x == 0) s_tile[0] = atomicAdd(a.counter, 1u);
    for (int it = 0;; ++it) {
        __syncthreads();
        const uint64_t tile = s_tile[it & 1];
        if (tile >= ntiles) break;
        if (threadIdx.x == 0) s_tile[(it + 1) & 1] = atomicAdd(a.counter, 1u);
        const SegTile td = a.tiles[tile];
        const uint32_t lo = a.seg_lo[td.chunk];
        const int nb = (int)a.seg_nb[td.chunk];   // 1 .. 1 << MAXB (checked by the setup)
        const uint64_t cend = a.offsets[td.chunk + 1];
        const uint64_t base = a.offsets[td.chunk] + (uint64_t)td.index * kSortTile;
        const int tn = (int)(cend - base < (uint64_t)kSortTile ? cend - base : (uint64_t)kSortTile);
        const bool last = base + (uint64_t)tn >= cend;   // no later tile of the chunk reads this one
        const uint64_t row = base / kSortTile;            // tiles that are not last are full: rows are distinct
        const int sdig = a.stitch ? nb - 1 : nb;          // staging digit (nb: none)
        for (int q = threadIdx.x; q < kSortWarps * nb; q += kSortNT) s_whist[q] = 0;
        __syncthreads();
        uint16_t* wh = s_whist + warp * nb;

        // ---- digits (all loads issued first), then in-warp stable ranks
        uint32_t dg[kSortIPT];
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const int p = warp * (kSortIPT * 32) + r * 32 + lane;
            if (DIST) {
                uint32_t cell = 0;
                if (p < tn) {
                    if (a.cells) {
                        cell = __ldg(a.cells + base + p);
                        if (cell >> (3 * a.g)) { raise(a.err, FP_ERR_CAPACITY, 19); cell = 0; }   // not a cell of the grid
                    } else {
                        const int4 q = __ldg(a.pt_in + base + p);
                        cell = key_small(q.x, q.y, q.z, cube, scale_g, a.g);
                    }
                }
                dg[r] = cell;
            } else {
                dg[r] = p < tn ? a.id_in[base + p] - lo : 0xFFFFFFFFu;
            }
        }
        if (DIST) {   // cell -> chunk, all gathers in flight together
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const int p = warp * (kSortIPT * 32) + r * 32 + lane;
                dg[r] = p < tn ? a.lut[dg[r]] - lo : 0xFFFFFFFFu;
            }
        }
        uint32_t pack[kSortIPT];
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const int p = warp * (kSortIPT * 32) + r * 32 + lane;
            uint32_t d = 0xFFFFu;
            if (p < tn) {
                d = dg[r];
                if (d >= (uint32_t)sdig) {
                    if (!a.stitch) raise(a.err, FP_ERR_CAPACITY, 13);   // a leaf outside the chunk's subtree
                    d = (uint32_t)(nb - 1);
                }
            }
            uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader && d != 0xFFFFu) {
                old = wh[d];
                wh[d] = (uint16_t)(old + __popc(peers));
            }
            old = __shfl_sync(0xFFFFFFFFu, old, leader);
            pack[r] = d | ((old + __popc(peers & lanemask_lt())) << 16);
            __syncwarp();
        }
        __syncthreads();
        // ---- per-digit totals, per-warp exclusive prefixes; publish aggregates
        for (int d = threadIdx.x; d < nb; d += kSortNT) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t v = s_whist[w * nb + d];
                s_whist[w * nb + d] = (uint16_t)s;
                s += v;
            }
            s_cnt[d] = s;
            if (!last && d != sdig) a.status[row * kStride + d] = (td.index == 0 ? kStFlagInc : kStFlagAgg) | s;
        }
        __syncthreads();
        {
            const int per = (nb + kSortNT - 1) / kSortNT;
            const int d0 = threadIdx.x * per;
            uint32_t s = 0;
            for (int q = 0; q < per; ++q)
                if (d0 + q < nb) s += s_cnt[d0 + q];
            uint32_t tot;
            uint32_t ex = block_exclusive_scan<kSortNT, uint32_t>(s, s_misc + 1, tot);
            for (int q = 0; q < per; ++q)
                if (d0 + q < nb) { s_off[d0 + q] = ex; ex += s_cnt[d0 + q]; }
        }
        __syncthreads();
        // ---- stage the records in digit order
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const int p = warp * (kSortIPT * 32) + r * 32 + lane;
            if (p < tn) {
                const uint32_t d = pack[r] & 0xFFFFu;
                const uint32_t lp = s_off[d] + s_whist[warp * nb + d] + (pack[r] >> 16);
                const uint64_t i = base + p;
                if (CPT) s_pt[lp] = __ldg(a.pt_in + i);
                s_val[lp] = DIST ? (uint32_t)i : a.val_in[i];
                if (!DIST) s_pos[lp] = (uint16_t)p;
                s_dig[lp] = (dig_t)d;
            }
        }
        // ---- look-back over the chunk's earlier tiles; staging slots for the stitch digit
        for (int d = threadIdx.x; d < nb; d += kSortNT) {
            if (d == sdig) {
                const uint32_t k = s_cnt[d];
                const uint32_t at = k ? atomicAdd(a.st_count, k) : 0u;
                s_gbase[d] = (uint64_t)at - s_off[d];
                continue;
            }
            uint32_t excl = 0;
            if (td.index > 0) {
                auto word = [&](int64_t t) { return &a.status[(uint64_t)t * kStride + d]; };
                excl = look_back<decltype(word), kSegLookBatch>(word, (int64_t)row - 1,
                                                                (int64_t)row - (int64_t)td.index, a.err);
                if (!last) atomicExch(&a.status[row * kStride + d], kStFlagInc | (excl + s_cnt[d]));
            }
            s_gbase[d] = a.first[(uint64_t)(lo + d) * a.first_stride] + excl - s_off[d];
        }
        __syncthreads();
        // ---- coalesced writes of each digit run
        for (int q = threadIdx.x; q < tn; q += kSortNT) {
            const int d = s_dig[q];
            const uint64_t o = s_gbase[d] + q;
            if (d == sdig) {
                if (o >= a.st_cap) { raise(a.err, FP_ERR_CAPACITY, 14); continue; }
                const uint64_t src = base + s_pos[q];
                const uint32_t id = a.id_in[src];
                a.st_key[o] = ((uint64_t)(a.st_rank ? a.st_rank[id] : id) << a.st_shift) | s_val[q];
                a.st_src[o] = (uint32_t)src;
            } else {
                if (o >= a.n) { raise(a.err, FP_ERR_CAPACITY, 15); continue; }   // inconsistent node table
                if (CPT) a.pt_out[o] = s_pt[q];
                if (a.val_out) a.val_out[o] = s_val[q];
            }
        }
        __syncthreads();
    }
}

// ---- host side
struct SegScratch {
    uint32_t* lo;          // [kmax]
    uint32_t* nb;          // [kmax]
    SegTile* tiles[2];     // [tiles_max] per variant
    uint32_t* status[2];   // [rows][256] and [rows][2048]
    uint32_t* cnt;         // [0..1] tiles per variant, [2] fail, [3..4] tile counters, [5] gated record count
    uint8_t* inside;       // [node_cap] owner layout: node lies in a chunk's subtree
    uint64_t kmax, tiles_max, rows, node_cap;
};
SegScratch take_seg_scratch(const Workspace& ws, uint64_t n, uint64_t kmax, uint64_t node_cap);

enum SegMode { SEG_LEAF = 0, SEG_OWNER = 1 };

struct SegCall {
    SegMode mode;
    const fp_node* nodes; const uint32_t* num_nodes; uint32_t node_cap;
    const fp_chunk* chunks; const uint32_t* num_chunks; const uint64_t* offsets;
    const int4* pt_in; int4* pt_out;
    const uint32_t* val_in; uint32_t* val_out;
    const uint32_t* id_in;
    uint64_t n;
    uint64_t out_n;       // bound of the output positions (0: n)
    const uint64_t* first; uint32_t first_stride;
    // owner layout: staging
    uint64_t* st_key; uint32_t* st_src; uint32_t* st_count; int st_shift;
    // owner layout, nullable: staging keys by rank among the nodes outside every
    // chunk subtree (in node order, so the sorted order is that of node ids):
    // st_rank[node] (node_cap), st_list[rank] = node, *st_nrank = their number;
    // st_tiles: scan scratch (kScanMaxTiles)
    uint32_t *st_rank, *st_list, *st_nrank, *st_tiles;
};

// Distribution of n points into chunks without the radix passes: with the
// cells and a 16-byte aligned scratch of n chunk ids given, 1..512 chunks take
// the counting pass and the double-buffered sweep (fp_seg.cu); else 257..512
// chunks the 9-bit segmented sweep; 513..2048 chunks the 11-bit one (digit =
// chunk of the point's cell, bucket bases = the chunk offsets).  *run_sort is
// set to 1 when the count is outside these ranges (the radix passes run
// instead), 0 when one of them ran.
size_t dist_wide_bytes(uint64_t n);
cudaError_t dist_wide(const int4* pts, uint64_t n, const fp_cube* cube, int g, const uint32_t* lut,
                      const uint64_t* offsets, const uint32_t* num_chunks, int4* out, uint32_t* perm,
                      uint32_t* run_sort, const Workspace& ws, cudaStream_t st, const uint32_t* cells = nullptr,
                      uint16_t* chunk_tmp = nullptr);

// Setup (chunk node ids, digits, tiles), status reset, both pass variants.
// Afterwards cnt[2] != 0 means a chunk did not fit (the caller's whole-array
// path must run; it is gated on cnt[5] = n in that case, 0 otherwise).
cudaError_t seg_scatter(const SegScratch& sc, const SegCall& call, const Workspace& ws, cudaStream_t st);

}  // namespace fp
