// fp_seg.cu -- setup and launch of the chunk-segmented scatter (fp_seg.cuh).
#include "fp_seg.cuh"

namespace fp {

// Node id of (key, level) in a preorder node table, kNone if absent.  Preorder
// is lexicographic in (key << 3 (21 - level), level): a node's cell starts at
// its first descendant's, and the ancestor comes first.
FP_DEV uint32_t find_node(const fp_node* nodes, uint32_t M, uint64_t key, uint32_t level)
{
    const uint64_t K = key << (3 * (kKeyLevels - level));
    uint32_t a = 0, b = M;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        const uint32_t lm = nodes[m].level;
        const uint64_t km = nodes[m].key << (3 * (kKeyLevels - lm));
        if (km < K || (km == K && lm < level)) a = m + 1;
        else b = m;
    }
    if (a < M && nodes[a].level == level && nodes[a].key == key) return a;
    return kNone;
}

// Per chunk: its node, digits, and its tiles appended to the variant's list.
__global__ void k_seg_setup(int mode, const fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap,
                            const fp_chunk* chunks, const uint32_t* num_chunks, const uint64_t* offsets,
                            uint64_t kmax, uint64_t n, uint32_t* seg_lo, uint32_t* seg_nb, SegTile* t0,
                            SegTile* t1, uint64_t tiles_max, uint32_t* cnt, uint8_t* inside, uint32_t* err)
{
    const uint64_t K = min((uint64_t)*num_chunks, kmax);
    const uint32_t M = min(*num_nodes, node_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (*num_chunks > kmax || offsets[K] != n)) atomicOr(&cnt[2], 1u);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < K; c += stride) {
        const uint64_t beg = offsets[c], end = offsets[c + 1], cn = end - beg;
        seg_lo[c] = 0;
        seg_nb[c] = 1;
        if (end > n || end < beg) { atomicOr(&cnt[2], 1u); continue; }   // offsets not a partition of [0, n)
        if (cn == 0) continue;
        const fp_chunk ch = chunks[c];
        const uint32_t id = find_node(nodes, M, ch.key, ch.level);
        if (id == kNone) { atomicOr(&cnt[2], 1u); continue; }   // not in the table: the whole-array path runs
        const uint32_t nd = nodes[id].n_desc;
        if ((uint64_t)id + nd >= M) { atomicOr(&cnt[2], 1u); continue; }
        const uint64_t nb = (uint64_t)nd + (mode == SEG_OWNER ? 2 : 1);
        if (nb > (1u << kSegMaxBits)) { atomicOr(&cnt[2], 1u); continue; }
        const int v = nb <= (1u << kSegSmallBits) ? 0 : 1;
        const uint32_t ntl = (uint32_t)((cn + kSortTile - 1) / kSortTile);
        const uint32_t at = atomicAdd(&cnt[v], ntl);
        if ((uint64_t)at + ntl > tiles_max) {
            raise(err, FP_ERR_CAPACITY, 12);
            atomicOr(&cnt[2], 1u);
            continue;
        }
        SegTile* tl = v ? t1 : t0;
        for (uint32_t i = 0; i < ntl; ++i) tl[at + i] = SegTile{(uint32_t)c, i};
        seg_lo[c] = id;
        seg_nb[c] = (uint32_t)nb;
        if (inside)
            for (uint32_t x = 0; x <= nd && id + x < M; ++x) inside[id + x] = 1;
    }
}

// owner layout: 1 for a node outside every chunk subtree (then its rank, by the scan)
__global__ void k_outside_flags(const uint8_t* inside, const uint32_t* num_nodes, uint32_t cap, uint32_t* flag)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap) flag[i] = i < min(*num_nodes, cap) && !inside[i] ? 1u : 0u;
}

__global__ void k_outside_list(const uint8_t* inside, const uint32_t* num_nodes, uint32_t cap, const uint32_t* rank,
                               uint32_t* list)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < min(*num_nodes, cap) && !inside[i]) list[rank[i]] = i;
}

// clear the status words that later tiles of the same chunk will read
template <int MAXB>
__global__ void k_seg_zero(const SegTile* tiles, const uint32_t* d_ntiles, uint64_t tiles_max,
                           const uint64_t* offsets, const uint32_t* seg_nb, uint32_t* status, const uint32_t* fail)
{
    if (*fail) return;
    const uint64_t T = min((uint64_t)*d_ntiles, tiles_max);
    for (uint64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const SegTile td = tiles[t];
        const uint64_t base = offsets[td.chunk] + (uint64_t)td.index * kSortTile;
        if (base + kSortTile >= offsets[td.chunk + 1]) continue;   // the chunk's last tile publishes nothing
        const uint64_t row = base / kSortTile;
        const int nb = (int)seg_nb[td.chunk];
        for (int d = threadIdx.x; d < nb; d += blockDim.x) status[(row << MAXB) + d] = 0;
    }
}

// record count of the whole-array path: n when a chunk did not fit, else 0
__global__ void k_seg_gate(uint32_t* cnt, uint32_t n) { cnt[5] = cnt[2] ? n : 0u; }

SegScratch take_seg_scratch(const Workspace& ws, uint64_t n, uint64_t kmax, uint64_t node_cap)
{
    SegScratch s;
    s.kmax = kmax ? kmax : 1;
    s.rows = n / kSortTile + 1;
    s.tiles_max = n / kSortTile + s.kmax + 1;
    s.node_cap = node_cap ? node_cap : 1;
    s.lo = ws.take<uint32_t>(s.kmax);
    s.nb = ws.take<uint32_t>(s.kmax);
    s.tiles[0] = ws.take<SegTile>(s.tiles_max);
    s.tiles[1] = ws.take<SegTile>(s.tiles_max);
    s.status[0] = ws.take<uint32_t>(s.rows << kSegSmallBits);
    s.status[1] = ws.take<uint32_t>(s.rows << kSegMaxBits);
    s.cnt = ws.take<uint32_t>(8);
    s.inside = ws.take<uint8_t>(s.node_cap);
    return s;
}

template <bool CPT, int MAXB>
static cudaError_t seg_launch(SegArgs a, const SegScratch& sc, int v, int num_sms, cudaStream_t st)
{
    using SM = SegSmem<CPT, MAXB>;
    auto kern = k_seg_pass<CPT, MAXB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::total);
    if (e) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSortNT, SM::total))) return e;
    if (per_sm < 1) per_sm = 1;
    a.tiles = sc.tiles[v];
    a.d_ntiles = sc.cnt + v;
    a.ntiles_max = sc.tiles_max;
    a.status = sc.status[v];
    a.counter = sc.cnt + 3 + v;
    const int grid = (int)std::min<uint64_t>(sc.tiles_max, (uint64_t)num_sms * per_sm);
    kern<<<grid, kSortNT, SM::total, st>>>(a);
    return cudaGetLastError();
}

// ---- the distribution with each point's cell given, up to 4096 chunks, in four
// launches and without any wait between blocks (the sweep below for up to 512
// chunks, k_dist_sweep_wide further down for 513 .. 4096):
//   k_dist_table: per node of level L = min(g, 5), its chunk when every
//     occupied cell of the node lies in that one chunk (else none) -- a 64 KB
//     table that spares most points the gather of the cell -> chunk table;
//   k_dist_count: one block per group of kDistGroup consecutive tiles writes
//     every point's chunk, and per tile the points of each chunk in the group's
//     earlier tiles, and per group its totals;
//   k_dist_colscan: per chunk, the exclusive prefix of the group totals plus the
//     chunk's offset -- each group's output start in every chunk;
//   k_dist_sweep: one CTA of 1024 threads per SM; tiles taken in order from a
//     counter.  The points and chunks of the next tile arrive by bulk copy in
//     the second buffer while the current tile is worked on; a tile stages only
//     (tile position, chunk) per output slot, and its write phase reads every
//     point from the tile buffer.  A tile's run of chunk d starts at its group's
//     start in d plus the points of d in the group's earlier tiles.
constexpr int kDistNT = 1024;
constexpr int kDistIPT = kSortTile / kDistNT;
constexpr int kDistWarps = kDistNT / 32;
constexpr int kDistBits = 9;
constexpr int kDistDig = 1 << kDistBits;
constexpr int kDistWideBits = 12;               // the wide sweep: 513 .. 4096 chunks
constexpr int kDistWideDig = 1 << kDistWideBits;
constexpr int kDistGroup = 64;                  // tiles per block of k_dist_count
constexpr int kDistCountNT = 512;               // thread d of k_dist_count owns chunks d, d + 512, ...
constexpr int kDistCountIPT = kSortTile / kDistCountNT;
constexpr int kDistTabLevel = 5;                // level of the node -> chunk table
constexpr uint16_t kDistSplit = 0xFFFFu;        // the node's points lie in several chunks

struct DistSweepArgs {
    const int4* pts;
    const uint32_t* cells;      // level-g cell of every point
    const uint32_t* lut;        // cell -> chunk (kNone: empty cell)
    const uint64_t* offsets;    // chunk c = output positions [offsets[c], offsets[c + 1])
    int4* out;
    uint32_t* perm;             // nullable
    uint16_t* tab;              // [8^tl]: chunk of a level-tl node, or kDistSplit
    uint16_t* chunk;            // chunk of every point, 16-byte aligned
    uint32_t* before;           // [tile][DIG]: points of the chunk in the group's earlier tiles
    uint32_t* gstart;           // [group][DIG]: group totals, then the group's start in the chunk
    uint32_t* counter;
    const uint32_t* d_ntiles;   // tiles of this sweep (0: another path runs)
    uint64_t ntiles_max;
    const uint32_t* nb;         // chunks (1 .. DIG, the sweep's width)
    uint64_t n;
    uint32_t ncell;             // cells of the grid (bound of a cell id)
    int g, tl;                  // grid level, table level (tl <= g)
    uint32_t* err;
};

// one warp per level-tl node: the chunks of its occupied cells (built for both
// sweeps, whichever of them runs)
__global__ void k_dist_table(DistSweepArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= (1u << (3 * a.tl))) return;
    const uint32_t span = 1u << (3 * (a.g - a.tl)), lo = k * span;
    uint32_t cmin = kNone, cmax = 0;
    for (uint32_t q = lane; q < span; q += 32) {
        const uint32_t c = __ldg(a.lut + lo + q);
        if (c != kNone) { cmin = min(cmin, c); cmax = max(cmax, c); }
    }
    cmin = __reduce_min_sync(0xFFFFFFFFu, cmin);
    cmax = __reduce_max_sync(0xFFFFFFFFu, cmax);
    if (lane == 0) a.tab[k] = (cmin == cmax && cmin < (uint32_t)kDistWideDig) ? (uint16_t)cmin : kDistSplit;
}

template <int DIG>
__global__ void __launch_bounds__(kDistCountNT) k_dist_count(DistSweepArgs a)
{
    constexpr int kOwn = DIG / kDistCountNT;   // chunks per thread
    extern __shared__ __align__(16) uint16_t dist_tab[];   // 8^tl entries
    __shared__ uint32_t h[DIG];
    const uint64_t ntiles = min((uint64_t)*a.d_ntiles, a.ntiles_max);
    if (ntiles == 0) return;
    const uint64_t ngroups = (ntiles + kDistGroup - 1) / kDistGroup;
    const uint32_t nb = min(*a.nb, (uint32_t)DIG);
    const uint32_t d = threadIdx.x;
    const int tsh = 3 * (a.g - a.tl);
    {
        const uint32_t nt4 = (1u << (3 * a.tl)) / 8;   // uint4 words of the table (8^tl >= 8 when tl >= 1)
        if (a.tl >= 1) {
            for (uint32_t q = d; q < nt4; q += kDistCountNT)
                reinterpret_cast<uint4*>(dist_tab)[q] = __ldg(reinterpret_cast<const uint4*>(a.tab) + q);
        } else if (d == 0) {
            dist_tab[0] = a.tab[0];
        }
    }
    for (uint64_t gi = blockIdx.x; gi < ngroups; gi += gridDim.x) {
        const uint64_t t0 = gi * kDistGroup, t1 = min(ntiles, t0 + kDistGroup);
        uint32_t run[kOwn];
#pragma unroll
        for (int o = 0; o < kOwn; ++o) { run[o] = 0; h[d + o * kDistCountNT] = 0; }
        // the cells of the next tile are loaded while the current one is counted
        uint32_t c[kDistCountIPT];
        auto load = [&](uint64_t t) {
            const uint64_t base = t * kSortTile;
#pragma unroll
            for (int r = 0; r < kDistCountIPT; ++r) {
                const uint64_t i = base + (uint64_t)r * kDistCountNT + d;
                c[r] = i < a.n ? __ldg(a.cells + i) : kNone;
            }
        };
        load(t0);
        __syncthreads();   // (also: the table is in shared memory)
        for (uint64_t t = t0; t < t1; ++t) {
            uint32_t k[kDistCountIPT];
#pragma unroll
            for (int r = 0; r < kDistCountIPT; ++r) {
                k[r] = c[r];
                if (k[r] != kNone && k[r] >= a.ncell) { raise(a.err, FP_ERR_CAPACITY, 19); k[r] = 0; }
            }
            if (t + 1 < t1) load(t + 1);
#pragma unroll
            for (int r = 0; r < kDistCountIPT; ++r)   // the table, else the gather
                if (k[r] != kNone) {
                    const uint16_t v = dist_tab[k[r] >> tsh];
                    k[r] = v != kDistSplit ? (uint32_t)v : __ldg(a.lut + k[r]);
                }
            const uint64_t base = t * kSortTile;
#pragma unroll
            for (int r = 0; r < kDistCountIPT; ++r)
                if (k[r] != kNone) {
                    if (k[r] >= nb) { raise(a.err, FP_ERR_CAPACITY, 13); k[r] = nb - 1; }   // not a chunk
                    a.chunk[base + (uint64_t)r * kDistCountNT + d] = (uint16_t)k[r];
                    atomicAdd(&h[k[r]], 1u);
                }
            __syncthreads();
#pragma unroll
            for (int o = 0; o < kOwn; ++o) {
                const uint32_t cd = d + o * kDistCountNT;
                if (cd < nb) {
                    a.before[t * DIG + cd] = run[o];
                    run[o] += h[cd];
                }
                h[cd] = 0;
            }
            __syncthreads();
        }
#pragma unroll
        for (int o = 0; o < kOwn; ++o)
            if (d + o * kDistCountNT < nb) a.gstart[gi * DIG + d + o * kDistCountNT] = run[o];
    }
}

// one warp per chunk: exclusive prefix of the group totals, plus the chunk's offset
template <int DIG>
__global__ void k_dist_colscan(DistSweepArgs a)
{
    const uint64_t ntiles = min((uint64_t)*a.d_ntiles, a.ntiles_max);
    const uint64_t ngroups = (ntiles + kDistGroup - 1) / kDistGroup;
    const uint32_t nb = min(*a.nb, (uint32_t)DIG);
    const int lane = threadIdx.x & 31;
    const uint32_t d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (d >= nb || ngroups == 0) return;
    uint32_t run = (uint32_t)a.offsets[d];
    for (uint64_t g0 = 0; g0 < ngroups; g0 += 32) {
        const uint64_t gi = g0 + lane;
        const uint32_t v = gi < ngroups ? a.gstart[gi * DIG + d] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (gi < ngroups) a.gstart[gi * DIG + d] = run + x - v;
        run += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
}

struct DistSmem {
    int4 raw[2][kSortTile];                 // the tile's points, as stored
    uint16_t chk[2][kSortTile];             // and their chunks
    uint32_t slot[kSortTile];               // by output slot: tile position | chunk << 16
    uint16_t whist[kDistWarps][kDistDig];   // per-warp counts, then exclusive prefixes over the warps
    uint32_t gbase[kDistDig];               // output position of slot 0 of every chunk's run
    uint32_t cnt[kDistDig];
    uint32_t scan[kDistWarps];
    uint32_t tile[2];
    uint64_t bar[2];
};

__global__ void __launch_bounds__(kDistNT, 1) k_dist_sweep(DistSweepArgs a)
{
    extern __shared__ __align__(128) unsigned char dist_smem[];
    DistSmem& S = *reinterpret_cast<DistSmem*>(dist_smem);
    const uint64_t ntiles = min((uint64_t)*a.d_ntiles, a.ntiles_max);
    if (ntiles == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t n = a.n;
    const int nb = (int)min(*a.nb, (uint32_t)kDistDig);
    // a full tile by bulk copy into buffer b (thread 0); a partial one is loaded by the threads
    auto issue = [&](uint64_t t, int b) {
        const uint64_t base = t * kSortTile;
        if (base + kSortTile > n) return;
        fence_async_smem();
        mbar_expect_tx(&S.bar[b], kSortTile * (uint32_t)(sizeof(int4) + sizeof(uint16_t)));
        bulk_g2s(S.raw[b], a.pts + base, kSortTile * (uint32_t)sizeof(int4), &S.bar[b]);
        bulk_g2s(S.chk[b], a.chunk + base, kSortTile * (uint32_t)sizeof(uint16_t), &S.bar[b]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        const uint32_t t0 = atomicAdd(a.counter, 1u);
        S.tile[0] = t0;
        if (t0 < ntiles) issue(t0, 0);
    }
    __syncthreads();
    uint32_t phase = 0;   // bit b: parity of buffer b's next completion
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const uint64_t tile = S.tile[b];
        if (tile >= ntiles) break;
        // the next tile is claimed now and its copy issued after the ranking,
        // so that no warp waits on the claim's round trip
        uint32_t nx = 0;
        if (threadIdx.x == 0) nx = atomicAdd(a.counter, 1u);
        // this tile's start in every chunk, in flight during the ranking
        uint32_t start = 0;
        if (threadIdx.x < (unsigned)nb)
            start = __ldg(a.gstart + (tile / kDistGroup) * kDistDig + threadIdx.x) +
                    __ldg(a.before + tile * kDistDig + threadIdx.x);
        const uint64_t base = tile * kSortTile;
        const int tn = (int)(n - base < (uint64_t)kSortTile ? n - base : (uint64_t)kSortTile);
        if (tn == kSortTile) {
            if (!mbar_wait(&S.bar[b], (phase >> b) & 1u)) {
                raise(a.err, FP_ERR_TIMEOUT);
                mbar_wait(&S.bar[b], (phase >> b) & 1u);   // the copy in flight, once more (bounded)
            }
            phase ^= 1u << b;
        } else {
            for (int p = threadIdx.x; p < tn; p += kDistNT) {
                S.raw[b][p] = __ldg(a.pts + base + p);
                S.chk[b][p] = a.chunk[base + p];
            }
        }
        for (int q = threadIdx.x; q < kDistWarps * kDistDig / 8; q += kDistNT)
            reinterpret_cast<uint4*>(&S.whist[0][0])[q] = make_uint4(0, 0, 0, 0);
        __syncthreads();

        // ---- in-warp stable ranks of the chunks (checked below nb by k_dist_count)
        uint32_t pack[kDistIPT];
#pragma unroll
        for (int r = 0; r < kDistIPT; ++r) {
            const int p = warp * (kDistIPT * 32) + r * 32 + lane;
            uint32_t d = p < tn ? (uint32_t)S.chk[b][p] : 0xFFFFu;
            if (d != 0xFFFFu && d >= (uint32_t)nb) d = (uint32_t)(nb - 1);
            const uint32_t peers = match_bits<kDistBits>(d, d != 0xFFFFu);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (lane == leader && d != 0xFFFFu) {
                old = S.whist[warp][d];
                S.whist[warp][d] = (uint16_t)(old + __popc(peers));
            }
            old = __shfl_sync(0xFFFFFFFFu, old, leader);
            pack[r] = d | ((old + __popc(peers & lanemask_lt())) << 16);
            __syncwarp();
        }
        if (threadIdx.x == 0) {   // buffer b ^ 1 was released by the last tile's closing barrier
            S.tile[b ^ 1] = nx;
            if (nx < ntiles) issue(nx, b ^ 1);
        }
        __syncthreads();
        // ---- per-chunk totals and per-warp exclusive prefixes
        for (int d = threadIdx.x; d < nb; d += kDistNT) {
            uint32_t s = 0;
#pragma unroll 8
            for (int w = 0; w < kDistWarps; ++w) {
                const uint32_t v = S.whist[w][d];
                S.whist[w][d] = (uint16_t)s;
                s += v;
            }
            S.cnt[d] = s;
        }
        __syncthreads();
        {   // first slot of every chunk's run; output position of its slot 0
            uint32_t tot;
            const uint32_t c = threadIdx.x < (unsigned)nb ? S.cnt[threadIdx.x] : 0u;
            const uint32_t ex = block_exclusive_scan<kDistNT, uint32_t>(c, S.scan, tot);
            if (threadIdx.x < (unsigned)nb) {
                S.gbase[threadIdx.x] = start - ex;
                S.cnt[threadIdx.x] = ex;
            }
        }
        __syncthreads();
        // ---- staging entries
#pragma unroll
        for (int r = 0; r < kDistIPT; ++r) {
            const int p = warp * (kDistIPT * 32) + r * 32 + lane;
            if (p < tn) {
                const uint32_t d = pack[r] & 0xFFFFu;
                S.slot[S.cnt[d] + S.whist[warp][d] + (pack[r] >> 16)] = (uint32_t)p | (d << 16);
            }
        }
        __syncthreads();
        // ---- coalesced writes of every chunk's run
        for (int q = threadIdx.x; q < tn; q += kDistNT) {
            const uint32_t v = S.slot[q];
            const uint32_t p = v & 0xFFFFu;
            const uint64_t o = (uint32_t)(S.gbase[v >> 16] + (uint32_t)q);   // positions are below 2^30
            if (o >= n) { raise(a.err, FP_ERR_CAPACITY, 15); continue; }   // offsets not those of these points
            a.out[o] = S.raw[b][p];
            if (a.perm) a.perm[o] = (uint32_t)(base + p);
        }
        __syncthreads();
    }
}

// The wide sweep: 513 .. 4096 chunks, 12-bit chunk ids.  Per-warp histograms of
// 4096 chunks would not fit beside the double-buffered tile, so a tile ranks its
// points by a stable two-pass sort of (chunk, position) in shared memory (6-bit
// digits, ballot-matched per warp); every chunk present takes its output start
// once (its group's start plus the points of the chunk in the group's earlier
// tiles) and each point the start plus its place in the chunk's run.
constexpr int kWideRadix = 6;
constexpr int kWideBins = 1 << kWideRadix;

struct WideSmem {
    int4 raw[2][kSortTile];                  // the tile's points, as stored
    uint16_t chk[2][kSortTile];              // and their chunks
    uint32_t s0[kSortTile];                  // chunk << 12 | position, after the first pass
    uint32_t s1[kSortTile];                  // the same, sorted by chunk (then position)
    uint16_t whist[kDistWarps][kWideBins];   // per-warp digit counts, then their prefixes
    uint32_t off[kWideBins];                 // first slot of every digit
    uint16_t rstart[kDistWideDig];           // first slot of every chunk present
    uint32_t startv[kDistWideDig];           // output position of the tile's first point of every chunk present
    uint32_t scan[kDistWarps];
    uint32_t tile[2];
    uint64_t bar[2];
};

// one stable pass of the tile's (chunk << 12 | position) words by 6 chunk bits at `shift`;
// pass 0 builds the words from the chunks in buffer b, later passes read `src`
FP_DEV void wide_pass(WideSmem& S, int b, const uint32_t* src, uint32_t* dst, int tn, int shift, bool first)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < kDistWarps * kWideBins / 2; q += kDistNT)
        reinterpret_cast<uint32_t*>(&S.whist[0][0])[q] = 0u;
    __syncthreads();
    uint32_t v[kDistIPT], pack[kDistIPT];
#pragma unroll
    for (int r = 0; r < kDistIPT; ++r) {
        const int p = warp * (kDistIPT * 32) + r * 32 + lane;
        const bool valid = p < tn;
        v[r] = 0;
        if (valid) v[r] = first ? ((uint32_t)S.chk[b][p] << 12) | (uint32_t)p : src[p];
        const uint32_t d = valid ? (v[r] >> (12 + shift)) & (kWideBins - 1) : 0u;
        const uint32_t peers = match_bits<kWideRadix>(d, valid);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && valid) {
            old = S.whist[warp][d];
            S.whist[warp][d] = (uint16_t)(old + __popc(peers));
        }
        old = __shfl_sync(0xFFFFFFFFu, old, leader < 0 ? 0 : leader);
        pack[r] = valid ? (d | ((old + __popc(peers & lanemask_lt())) << 16)) : 0xFFFFFFFFu;
        __syncwarp();
    }
    __syncthreads();
    uint32_t tot_d = 0;
    if (threadIdx.x < kWideBins) {   // prefix over the warps of every digit
        for (int w = 0; w < kDistWarps; ++w) {
            const uint32_t x = S.whist[w][threadIdx.x];
            S.whist[w][threadIdx.x] = (uint16_t)tot_d;
            tot_d += x;
        }
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<kDistNT, uint32_t>(threadIdx.x < kWideBins ? tot_d : 0u, S.scan, tot);
    if (threadIdx.x < kWideBins) S.off[threadIdx.x] = ex;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kDistIPT; ++r) {
        if (pack[r] == 0xFFFFFFFFu) continue;
        const uint32_t d = pack[r] & 0xFFFFu;
        dst[S.off[d] + S.whist[warp][d] + (pack[r] >> 16)] = v[r];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDistNT, 1) k_dist_sweep_wide(DistSweepArgs a)
{
    extern __shared__ __align__(128) unsigned char wide_smem[];
    WideSmem& S = *reinterpret_cast<WideSmem*>(wide_smem);
    const uint64_t ntiles = min((uint64_t)*a.d_ntiles, a.ntiles_max);
    if (ntiles == 0) return;
    const uint64_t n = a.n;
    const uint32_t nb = min(*a.nb, (uint32_t)kDistWideDig);
    auto issue = [&](uint64_t t, int b) {
        const uint64_t base = t * kSortTile;
        if (base + kSortTile > n) return;
        fence_async_smem();
        mbar_expect_tx(&S.bar[b], kSortTile * (uint32_t)(sizeof(int4) + sizeof(uint16_t)));
        bulk_g2s(S.raw[b], a.pts + base, kSortTile * (uint32_t)sizeof(int4), &S.bar[b]);
        bulk_g2s(S.chk[b], a.chunk + base, kSortTile * (uint32_t)sizeof(uint16_t), &S.bar[b]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        const uint32_t t0 = atomicAdd(a.counter, 1u);
        S.tile[0] = t0;
        if (t0 < ntiles) issue(t0, 0);
    }
    __syncthreads();
    uint32_t phase = 0;   // bit b: parity of buffer b's next completion
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const uint64_t tile = S.tile[b];
        if (tile >= ntiles) break;
        uint32_t nx = 0;
        if (threadIdx.x == 0) nx = atomicAdd(a.counter, 1u);
        const uint64_t base = tile * kSortTile;
        const int tn = (int)(n - base < (uint64_t)kSortTile ? n - base : (uint64_t)kSortTile);
        if (tn == kSortTile) {
            if (!mbar_wait(&S.bar[b], (phase >> b) & 1u)) {
                raise(a.err, FP_ERR_TIMEOUT);
                mbar_wait(&S.bar[b], (phase >> b) & 1u);   // the copy in flight, once more (bounded)
            }
            phase ^= 1u << b;
        } else {
            for (int p = threadIdx.x; p < tn; p += kDistNT) {
                S.raw[b][p] = __ldg(a.pts + base + p);
                S.chk[b][p] = a.chunk[base + p];
            }
        }
        // (the first pass's barrier also publishes the partial tile's loads)
        wide_pass(S, b, nullptr, S.s0, tn, 0, true);
        if (threadIdx.x == 0) {   // buffer b ^ 1 was released by the last tile's closing barrier
            S.tile[b ^ 1] = nx;
            if (nx < ntiles) issue(nx, b ^ 1);
        }
        wide_pass(S, b, S.s0, S.s1, tn, kWideRadix, false);
        // ---- every chunk present: its first slot and its output start
        const uint64_t g = tile / kDistGroup;
        for (int q = threadIdx.x; q < tn; q += kDistNT) {
            const uint32_t c = S.s1[q] >> 12;
            if (q == 0 || (S.s1[q - 1] >> 12) != c) {
                if (c >= nb) { raise(a.err, FP_ERR_CAPACITY, 13); continue; }   // not a chunk
                S.rstart[c] = (uint16_t)q;
                S.startv[c] = __ldg(a.gstart + g * kDistWideDig + c) + __ldg(a.before + tile * kDistWideDig + c);
            }
        }
        __syncthreads();
        // ---- writes: every chunk's run in position order
        for (int q = threadIdx.x; q < tn; q += kDistNT) {
            const uint32_t v = S.s1[q];
            const uint32_t c = v >> 12, p = v & 0xFFFu;
            if (c >= nb) continue;
            const uint64_t o = (uint64_t)S.startv[c] + (uint64_t)(q - S.rstart[c]);
            if (o >= n) { raise(a.err, FP_ERR_CAPACITY, 15); continue; }   // offsets not those of these points
            a.out[o] = S.raw[b][p];
            if (a.perm) a.perm[o] = (uint32_t)(base + p);
        }
        __syncthreads();
    }
}

// ------------------------------------------------ distribution in one sweep
// one segment [0, n) with K digits when k_lo < K <= 2048 (k_lo: 256, or 0 when
// the cells are given and the double-buffered sweep takes the small counts
// too): its tiles, the segment bounds, and the flag that gates the radix passes
constexpr int kDistMidBits = 9;   // up to 512 chunks: two CTAs per SM
static_assert(kDistMidBits == kDistBits, "the sweep with the cells given is the 9-bit variant");

__global__ void k_dist_setup(const uint32_t* num_chunks, uint64_t n, uint32_t k_lo, uint32_t k_hi, uint64_t* seg_off,
                             uint32_t* seg_lo, uint32_t* seg_nb, SegTile* tiles, uint32_t* cnt, uint32_t* run_sort)
{
    const uint32_t K = *num_chunks;
    const bool wide = K > k_lo && K <= k_hi;
    const uint64_t ntl = wide ? (n + kSortTile - 1) / kSortTile : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntl; t += stride)
        tiles[t] = SegTile{0u, (uint32_t)t};
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const bool mid = K <= (1u << kDistMidBits);
        seg_off[0] = 0;
        seg_off[1] = n;
        seg_lo[0] = 0;
        seg_nb[0] = wide ? K : 1u;
        cnt[0] = mid ? (uint32_t)ntl : 0u;   // tiles of the 9-bit pass
        cnt[3] = mid ? 0u : (uint32_t)ntl;   // tiles of the 11-bit pass (the wide sweep with the cells)
        cnt[1] = cnt[4] = 0;                 // tile counters
        cnt[2] = 0;                          // fail word (never set here)
        *run_sort = wide ? 0u : 1u;
    }
}

struct DistScratch {
    uint64_t* seg_off;
    uint32_t *lo, *nb, *cnt, *status, *gstart;
    uint16_t* tab;
    SegTile* tiles;
    uint64_t ntiles;
};

static DistScratch dist_carve(const Workspace& ws, uint64_t n)
{
    DistScratch d;
    d.ntiles = (n + kSortTile - 1) / kSortTile;
    const uint64_t T = d.ntiles ? d.ntiles : 1;
    d.seg_off = ws.take<uint64_t>(2);
    d.lo = ws.take<uint32_t>(1);
    d.nb = ws.take<uint32_t>(1);
    d.cnt = ws.take<uint32_t>(8);
    d.tiles = ws.take<SegTile>(T);
    d.status = ws.take<uint32_t>(T << kDistWideBits);   // (also the wide sweep's per-tile starts)
    d.gstart = ws.take<uint32_t>(((T + kDistGroup - 1) / kDistGroup) << kDistWideBits);
    d.tab = ws.take<uint16_t>(1u << (3 * kDistTabLevel));
    return d;
}

template <int MAXB>
static cudaError_t dist_launch(const SegArgs& a, uint64_t ntiles, int num_sms, cudaStream_t st)
{
    using SM = SegSmem<true, MAXB, true>;
    auto kern = k_seg_pass<true, MAXB, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::total);
    if (e) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSortNT, SM::total))) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)num_sms * per_sm));
    kern<<<grid, kSortNT, SM::total, st>>>(a);
    return cudaGetLastError();
}

size_t dist_wide_bytes(uint64_t n)
{
    Workspace dry;
    dist_carve(dry, n);
    return dry.used;
}

cudaError_t dist_wide(const int4* pts, uint64_t n, const fp_cube* cube, int g, const uint32_t* lut,
                      const uint64_t* offsets, const uint32_t* num_chunks, int4* out, uint32_t* perm,
                      uint32_t* run_sort, const Workspace& ws, cudaStream_t st, const uint32_t* cells,
                      uint16_t* chunk_tmp)
{
    const DistScratch d = dist_carve(ws, n);
    // the cells given and a scratch array for every point's chunk: up to 4096
    // chunks take the counting pass and a double-buffered sweep
    const bool sweep = cells && chunk_tmp && ((uintptr_t)chunk_tmp & 15) == 0 && ((uintptr_t)pts & 15) == 0;
    const int gs = (int)std::max<uint64_t>(1, std::min<uint64_t>((d.ntiles + 255) / 256, (uint64_t)ws.num_sms * 4));
    k_dist_setup<<<gs, 256, 0, st>>>(num_chunks, n, sweep ? 0u : (1u << kSegSmallBits),
                                     sweep ? (uint32_t)kDistWideDig : (1u << kSegMaxBits), d.seg_off, d.lo, d.nb,
                                     d.tiles, d.cnt, run_sort);
    cudaError_t e;
    if (sweep) {
        DistSweepArgs b{};
        b.pts = pts; b.cells = cells; b.lut = lut; b.offsets = offsets;
        b.out = out; b.perm = perm; b.tab = d.tab; b.chunk = chunk_tmp;
        b.before = d.status; b.gstart = d.gstart;
        b.ntiles_max = d.ntiles; b.nb = d.nb;
        b.n = n; b.ncell = 1u << (3 * g); b.g = g; b.tl = std::min(g, kDistTabLevel); b.err = ws.err;
        const uint32_t nodes = 1u << (3 * b.tl);
        k_dist_table<<<(nodes * 32 + 255) / 256, 256, 0, st>>>(b);
        const uint64_t ngroups = (d.ntiles + kDistGroup - 1) / kDistGroup;
        const int tsm = (int)(nodes * sizeof(uint16_t) < 16 ? 16 : nodes * sizeof(uint16_t));
        const int gc = (int)std::max<uint64_t>(1, std::min<uint64_t>(ngroups, (uint64_t)ws.num_sms * 3));
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(d.ntiles, (uint64_t)ws.num_sms));
        // up to 512 chunks: per-warp histograms in the sweep (tiles cnt[0], counter cnt[1])
        b.d_ntiles = d.cnt; b.counter = d.cnt + 1;
        if ((e = cudaFuncSetAttribute(k_dist_count<kDistDig>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm)))
            return e;
        k_dist_count<kDistDig><<<gc, kDistCountNT, tsm, st>>>(b);
        k_dist_colscan<kDistDig><<<kDistDig * 32 / 256, 256, 0, st>>>(b);
        const int smem = (int)sizeof(DistSmem);
        if ((e = cudaFuncSetAttribute(k_dist_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
        k_dist_sweep<<<grid, kDistNT, smem, st>>>(b);
        // 513 .. 4096 chunks: the tile's ranks by a two-pass sort (tiles cnt[3], counter cnt[4])
        b.d_ntiles = d.cnt + 3; b.counter = d.cnt + 4;
        if ((e = cudaFuncSetAttribute(k_dist_count<kDistWideDig>, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm)))
            return e;
        k_dist_count<kDistWideDig><<<gc, kDistCountNT, tsm, st>>>(b);
        k_dist_colscan<kDistWideDig><<<kDistWideDig * 32 / 256, 256, 0, st>>>(b);
        const int wsm = (int)sizeof(WideSmem);
        if ((e = cudaFuncSetAttribute(k_dist_sweep_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, wsm))) return e;
        k_dist_sweep_wide<<<grid, kDistNT, wsm, st>>>(b);
        return cudaGetLastError();
    }
    const int gz = std::max(1, ws.num_sms * 8);
    k_seg_zero<kDistMidBits><<<gz, 256, 0, st>>>(d.tiles, d.cnt, d.ntiles, d.seg_off, d.nb, d.status, d.cnt + 2);
    k_seg_zero<kSegMaxBits><<<gz, 256, 0, st>>>(d.tiles, d.cnt + 3, d.ntiles, d.seg_off, d.nb, d.status, d.cnt + 2);
    SegArgs a{};
    a.pt_in = pts; a.pt_out = out;
    a.val_in = nullptr; a.val_out = perm;
    a.offsets = d.seg_off;
    a.seg_lo = d.lo; a.seg_nb = d.nb;
    a.tiles = d.tiles; a.d_ntiles = d.cnt; a.ntiles_max = d.ntiles;
    a.first = offsets; a.first_stride = 1;
    a.status = d.status; a.counter = d.cnt + 1;
    a.stitch = 0;
    a.n = n;
    a.d_fail = d.cnt + 2;
    a.err = ws.err;
    a.cube = cube; a.lut = lut; a.cells = cells; a.g = g;
    if ((e = dist_launch<kDistMidBits>(a, d.ntiles, ws.num_sms, st))) return e;
    a.d_ntiles = d.cnt + 3; a.counter = d.cnt + 4;
    return dist_launch<kSegMaxBits>(a, d.ntiles, ws.num_sms, st);
}

cudaError_t seg_scatter(const SegScratch& sc, const SegCall& c, const Workspace& ws, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(sc.cnt, 0, 8 * sizeof(uint32_t), st))) return e;
    const bool owner = c.mode == SEG_OWNER;
    if (owner) {
        if ((e = cudaMemsetAsync(sc.inside, 0, sc.node_cap, st))) return e;
        if ((e = cudaMemsetAsync(c.st_count, 0, sizeof(uint32_t), st))) return e;
    }
    const int gk = (int)std::max<uint64_t>(1, std::min<uint64_t>((sc.kmax + 255) / 256, (uint64_t)ws.num_sms * 8));
    k_seg_setup<<<gk, 256, 0, st>>>((int)c.mode, c.nodes, c.num_nodes, c.node_cap, c.chunks, c.num_chunks,
                                    c.offsets, sc.kmax, c.n, sc.lo, sc.nb, sc.tiles[0], sc.tiles[1], sc.tiles_max, sc.cnt,
                                    owner ? sc.inside : nullptr, ws.err);
    if (owner && c.st_rank) {
        const unsigned gn = (c.node_cap + 255) / 256;
        k_outside_flags<<<gn, 256, 0, st>>>(sc.inside, c.num_nodes, c.node_cap, c.st_rank);
        if ((e = scan_exclusive<uint32_t, uint32_t>(c.st_rank, c.st_rank, c.node_cap, nullptr, c.st_tiles, c.st_nrank,
                                                    (uint32_t*)nullptr, st)))
            return e;
        k_outside_list<<<gn, 256, 0, st>>>(sc.inside, c.num_nodes, c.node_cap, c.st_rank, c.st_list);
    }
    const int gz = std::max(1, ws.num_sms * 8);
    k_seg_zero<kSegSmallBits><<<gz, 256, 0, st>>>(sc.tiles[0], sc.cnt + 0, sc.tiles_max, c.offsets, sc.nb,
                                                   sc.status[0], sc.cnt + 2);
    k_seg_zero<kSegMaxBits><<<gz, 256, 0, st>>>(sc.tiles[1], sc.cnt + 1, sc.tiles_max, c.offsets, sc.nb,
                                                 sc.status[1], sc.cnt + 2);
    SegArgs a{};
    a.pt_in = c.pt_in; a.pt_out = c.pt_out;
    a.val_in = c.val_in; a.val_out = c.val_out;
    a.id_in = c.id_in;
    a.offsets = c.offsets;
    a.seg_lo = sc.lo; a.seg_nb = sc.nb;
    a.first = c.first; a.first_stride = c.first_stride;
    a.stitch = owner ? 1 : 0;
    a.st_key = c.st_key; a.st_src = c.st_src; a.st_count = c.st_count; a.st_cap = c.n; a.st_shift = c.st_shift;
    a.st_rank = owner ? c.st_rank : nullptr;
    a.n = c.out_n ? c.out_n : c.n;
    a.d_fail = sc.cnt + 2;
    a.err = ws.err;
    const bool cpt = c.pt_in && c.pt_out;
    if (cpt) {
        if ((e = seg_launch<true, kSegSmallBits>(a, sc, 0, ws.num_sms, st))) return e;
        if ((e = seg_launch<true, kSegMaxBits>(a, sc, 1, ws.num_sms, st))) return e;
    } else {
        if ((e = seg_launch<false, kSegSmallBits>(a, sc, 0, ws.num_sms, st))) return e;
        if ((e = seg_launch<false, kSegMaxBits>(a, sc, 1, ws.num_sms, st))) return e;
    }
    k_seg_gate<<<1, 1, 0, st>>>(sc.cnt, (uint32_t)c.n);
    return cudaGetLastError();
}

}  // namespace fp
