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

// ------------------------------------------------ distribution in one sweep
// one segment [0, n) with K digits when 256 < K <= 2048: its tiles, the
// segment bounds, and the flag that gates the radix passes
constexpr int kDistMidBits = 9;   // up to 512 chunks: two CTAs per SM

__global__ void k_dist_setup(const uint32_t* num_chunks, uint64_t n, uint64_t* seg_off, uint32_t* seg_lo,
                             uint32_t* seg_nb, SegTile* tiles, uint32_t* cnt, uint32_t* run_sort)
{
    const uint32_t K = *num_chunks;
    const bool wide = K > (1u << kSegSmallBits) && K <= (1u << kSegMaxBits);
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
        cnt[3] = mid ? 0u : (uint32_t)ntl;   // tiles of the 11-bit pass
        cnt[1] = cnt[4] = 0;                 // tile counters
        cnt[2] = 0;                          // fail word (never set here)
        *run_sort = wide ? 0u : 1u;
    }
}

struct DistScratch {
    uint64_t* seg_off;
    uint32_t *lo, *nb, *cnt, *status;
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
    d.status = ws.take<uint32_t>(T << kSegMaxBits);
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
                      uint32_t* run_sort, const Workspace& ws, cudaStream_t st, const uint32_t* cells)
{
    const DistScratch d = dist_carve(ws, n);
    const int gs = (int)std::max<uint64_t>(1, std::min<uint64_t>((d.ntiles + 255) / 256, (uint64_t)ws.num_sms * 4));
    k_dist_setup<<<gs, 256, 0, st>>>(num_chunks, n, d.seg_off, d.lo, d.nb, d.tiles, d.cnt, run_sort);
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
    cudaError_t e;
    a.d_ntiles = d.cnt; a.counter = d.cnt + 1;
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
