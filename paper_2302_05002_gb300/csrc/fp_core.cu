// fp_core.cu -- bounds, preview decimation, count grid and chunk merge.
//
//   k_bounds_decimate  one pass over the cloud: per-axis min/max (Sec. 4.4) and,
//                      optionally, the preview compaction (Sec. 3 / Sec. 4.2):
//                      index i is kept iff splitmix64(first + i) % m == 0.  Kept
//                      points keep ascending index order through a single-pass
//                      scan with decoupled look-back across tiles.  With the
//                      bounds (the main path, k_bounds_bulk) each tile arrives
//                      in shared memory by one bulk copy issued when the tile is
//                      claimed, in flight during the ranking and look-back.
//   k_count            count grid: one level-g Morton key per point, warp-
//                      aggregated atomics into an L2-resident 8^g histogram.
//   k_pyramid / k_chunk_mark / k_chunk_write
//                      bottom-up sums of the grid and the chunk rule of Fig.
//                      "octree" (maximal nodes with 0 < count <= T, plus
//                      overflowing finest cells), listed in Morton preorder.
#include "fp_internal.cuh"

namespace fp {

// ----------------------------------------------------------------- bounds
constexpr int kBdNT = 256;
constexpr int kBdIPT = 8;
constexpr int kBdTile = kBdNT * kBdIPT;   // 2048 points per tile

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

// keep rule of the compaction: none, index hash modulo m (the uniform
// preview), or the smallest index hash of the point's cell (the spatial one)
enum KeepRule { KEEP_NONE = 0, KEEP_MODULUS = 1, KEEP_CELL_MIN = 2 };

FP_DEV bool keep_modulus(uint64_t first, uint64_t i, uint32_t modulus)
{
    const uint64_t h = splitmix64(first + i);
    return (modulus & (modulus - 1)) == 0 ? (h & ((uint64_t)modulus - 1)) == 0 : (h % modulus) == 0;
}

template <bool BOUNDS, int KEEP>
__global__ void __launch_bounds__(kBdNT) k_bounds_decimate(const fp_point* __restrict__ pts, uint64_t n,
                                                           uint64_t first, uint32_t modulus, fp_point* __restrict__ out,
                                                           uint64_t out_cap, uint64_t* __restrict__ out_count,
                                                           int32_t* __restrict__ partial, uint64_t* tile_status,
                                                           uint32_t* tile_counter, uint64_t ntiles, uint32_t* err,
                                                           const uint64_t* __restrict__ cell_min,
                                                           const fp_cube* cube_p, int level)
{
    constexpr bool DECIM = KEEP != KEEP_NONE;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_cnt[kBdIPT][kBdNT / 32];
    __shared__ uint64_t s_base;
    __shared__ int32_t s_red[6][kBdNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool pow2 = (modulus & (modulus - 1)) == 0;
    const uint64_t mmask = (uint64_t)modulus - 1;

    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    int32_t hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    CubeDev cube;
    if (KEEP == KEEP_CELL_MIN) cube = load_cube(cube_p);
    const int csh = 3 * (kKeyLevels - level);

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
        __syncthreads();
        const uint64_t tile = s_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        const uint64_t base = tile * kBdTile;

        uint32_t keepmask = 0;   // bit r: item r of this thread kept
        if (DECIM) {
            // the keep decisions first (the uniform rule needs the index only), then publish
#pragma unroll
            for (int r = 0; r < kBdIPT; ++r) {
                uint64_t i = base + (uint64_t)r * kBdNT + threadIdx.x;
                bool k = false;
                if (i < n) {
                    uint64_t h = splitmix64(first + i);
                    if (KEEP == KEEP_MODULUS) {
                        k = pow2 ? (h & mmask) == 0 : (h % modulus) == 0;
                    } else {
                        const int4 q = ld_point(pts, i);
                        k = cell_min[key21(q.x, q.y, q.z, cube) >> csh] == h;
                    }
                }
                uint32_t bal = __ballot_sync(0xFFFFFFFFu, k);
                if (lane == 0) s_cnt[r][warp] = __popc(bal);
                keepmask |= (uint32_t)k << r;
            }
            __syncthreads();
            // exclusive scan over (r, warp) order = index order
            if (threadIdx.x < 32) {
                uint32_t v[kBdIPT * (kBdNT / 32) / 32];   // 2 entries per lane
                uint32_t s = 0;
                constexpr int per = kBdIPT * (kBdNT / 32) / 32;
#pragma unroll
                for (int q = 0; q < per; ++q) {
                    int e = lane * per + q;
                    v[q] = s_cnt[e / (kBdNT / 32)][e % (kBdNT / 32)];
                    s += v[q];
                }
                uint32_t x = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if (lane >= o) x += y;
                }
                uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
                uint32_t ex = x - s;
#pragma unroll
                for (int q = 0; q < per; ++q) {
                    int e = lane * per + q;
                    s_cnt[e / (kBdNT / 32)][e % (kBdNT / 32)] = ex;
                    ex += v[q];
                }
                // decoupled look-back for the tile's global offset
                if (lane == 0) {
                    uint64_t excl = 0;
                    if (tile == 0) {
                        atomicExch((unsigned long long*)&tile_status[0], (unsigned long long)(kFlagInc | total));
                    } else {
                        atomicExch((unsigned long long*)&tile_status[tile], (unsigned long long)(kFlagAgg | total));
                        int64_t t = (int64_t)tile - 1;
                        uint32_t spins = 0;
                        while (t >= 0) {
                            uint64_t s2 = ld_volatile64(&tile_status[t]);
                            if ((s2 >> 62) == 0) {
                                if (++spins > kSpinLimit) { raise(err, FP_ERR_TIMEOUT); break; }
                                continue;
                            }
                            excl += s2 & kValMask;
                            if ((s2 >> 62) == 2) break;
                            --t;
                        }
                        atomicExch((unsigned long long*)&tile_status[tile],
                                   (unsigned long long)(kFlagInc | (excl + total)));
                    }
                    s_base = excl;
                    if (tile == ntiles - 1) {
                        *out_count = excl + total;
                        if (excl + total > out_cap) raise(err, FP_ERR_CAPACITY, 0);
                    }
                }
            }
            __syncthreads();
        }

        if (BOUNDS) {
#pragma unroll 4
            for (int r = 0; r < kBdIPT; ++r) {
                uint64_t i = base + (uint64_t)r * kBdNT + threadIdx.x;
                if (i < n) {
                    int4 p = ld_point_cs(pts, i);
                    lo[0] = min(lo[0], p.x); hi[0] = max(hi[0], p.x);
                    lo[1] = min(lo[1], p.y); hi[1] = max(hi[1], p.y);
                    lo[2] = min(lo[2], p.z); hi[2] = max(hi[2], p.z);
                }
            }
        }
        if (DECIM) {
            // second sweep for the writes (ballots need converged warps)
#pragma unroll 4
            for (int r = 0; r < kBdIPT; ++r) {
                bool kept = (keepmask >> r) & 1u;
                uint32_t bal = __ballot_sync(0xFFFFFFFFu, kept);
                if (kept) {
                    uint64_t i = base + (uint64_t)r * kBdNT + threadIdx.x;
                    uint64_t pos = s_base + s_cnt[r][warp] + __popc(bal & lanemask_lt());
                    if (pos < out_cap) st_point(out, pos, ld_point(pts, i));
                }
            }
        }
        __syncthreads();
    }

    if (BOUNDS) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            for (int o = 16; o > 0; o >>= 1) {
                lo[a] = min(lo[a], __shfl_xor_sync(0xFFFFFFFFu, lo[a], o));
                hi[a] = max(hi[a], __shfl_xor_sync(0xFFFFFFFFu, hi[a], o));
            }
        }
        if (lane == 0) {
            for (int a = 0; a < 3; ++a) { s_red[a][warp] = lo[a]; s_red[3 + a][warp] = hi[a]; }
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            int a = threadIdx.x;
            int32_t v = s_red[a][0];
            for (int w = 1; w < kBdNT / 32; ++w) v = a < 3 ? min(v, s_red[a][w]) : max(v, s_red[a][w]);
            partial[blockIdx.x * 6 + a] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_bounds_final(const int32_t* partial, int nblocks, uint64_t n,
                                                      fp_cube* cube)
{
    __shared__ int32_t s_red[6][8];
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], partial[b * 6 + a]);
            hi[a] = max(hi[a], partial[b * 6 + 3 + a]);
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(0xFFFFFFFFu, lo[a]);
        hi[a] = __reduce_max_sync(0xFFFFFFFFu, hi[a]);
        if (lane == 0) { s_red[a][warp] = lo[a]; s_red[3 + a][warp] = hi[a]; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    fp_cube c;
    for (int a = 0; a < 3; ++a) { c.o[a] = 0; c.mx[a] = 0; }
    c.S = 0;
    if (n > 0) {
        uint64_t ext = 0;
        for (int a = 0; a < 3; ++a) {
            int32_t l = s_red[a][0], h = s_red[3 + a][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { l = min(l, s_red[a][w]); h = max(h, s_red[3 + a][w]); }
            c.o[a] = l;
            c.mx[a] = h;
            uint64_t e = (uint64_t)((int64_t)h - (int64_t)l);
            ext = e > ext ? e : ext;
        }
        c.S = ext + 1;
    }
    *cube = c;
}

__global__ void k_zero_count(uint64_t* out_count) { *out_count = 0; }

// a[*idx] = *val  (writes the grand total behind a device-sized prefix array)
__global__ void k_put_at(uint64_t* a, const uint32_t* idx, const uint64_t* val) { a[*idx] = *val; }

// ----------------------------------------------------------------- count
// Each block also keeps a small direct-mapped table of cells in shared memory:
// the first cell to reach a slot owns it for the block's lifetime and its hits
// are added there, flushed to the grid at the end.  Clouds with dense spots
// (scanner surroundings) send most of their hits to a few cells; those end up
// in the tables and stop contending for the same global counters.
constexpr int kCountSlots = 1024;

// cells (nullable): the level-g Morton cell of every point, for fp_distribute_cells
template <bool AGG>
__global__ void __launch_bounds__(256) k_count(const fp_point* __restrict__ pts, uint64_t n,
                                               const fp_cube* __restrict__ cube, int g, uint32_t* __restrict__ counts,
                                               uint32_t* __restrict__ cells)
{
    __shared__ uint32_t s_tag[kCountSlots], s_cnt[kCountSlots];
    for (int q = threadIdx.x; q < kCountSlots; q += blockDim.x) { s_tag[q] = kNone; s_cnt[q] = 0; }
    __syncthreads();
    const CubeDev c = load_cube(cube);
    const float sg = scale_at(c, g);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride * 4) {
        uint32_t key[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint64_t i = i0 + u * stride + threadIdx.x;
            key[u] = kNone;
            if (i < n) {
                int4 p = ld_point_cs(pts, i);
                key[u] = key_small(p.x, p.y, p.z, c, sg, g);
                if (cells) cells[i] = key[u];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // a warp whose neighbouring lanes never share a cell (spread-out
            // points) adds directly; otherwise its equal cells are merged first
            const uint32_t knext = __shfl_down_sync(0xFFFFFFFFu, key[u], 1);   // (lane 31: its own)
            const bool twin = lane < 31 && key[u] != kNone && key[u] == knext;
            if (AGG && __any_sync(0xFFFFFFFFu, twin)) {
                uint32_t peers = __match_any_sync(0xFFFFFFFFu, key[u]);
                if (key[u] != kNone && lane == __ffs(peers) - 1) {
                    const uint32_t slot = (key[u] * 2654435761u) >> 22;   // 10-bit multiplicative hash
                    uint32_t t = s_tag[slot];
                    if (t == kNone) t = atomicCAS(&s_tag[slot], kNone, key[u]) == kNone ? key[u] : s_tag[slot];
                    if (t == key[u]) atomicAdd(&s_cnt[slot], (uint32_t)__popc(peers));
                    else atomicAdd(&counts[key[u]], (uint32_t)__popc(peers));
                }
            } else if (key[u] != kNone) {
                atomicAdd(&counts[key[u]], 1u);
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kCountSlots; q += blockDim.x)
        if (s_cnt[q]) atomicAdd(&counts[s_tag[q]], s_cnt[q]);
}

// ----------------------------------------------------------------- merge
// pyramid[level l] at offset (8^l - 1) / 7 for l < g; level g is the count grid
__global__ void k_pyramid_level(const uint32_t* __restrict__ child, uint32_t* __restrict__ parent, uint64_t nparent)
{
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nparent) return;
    // level offsets (8^l - 1) / 7 are only 4-byte aligned: scalar loads
    const uint32_t* c = child + 8 * k;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += c[q];
    parent[k] = s;
}

FP_DEV uint32_t pyr_count(const uint32_t* pyr, const uint32_t* counts, int g, int l, uint64_t key)
{
    return l == g ? counts[key] : pyr[((1ull << (3 * l)) - 1) / 7 + key];
}

// block node of cell m: shallowest ancestor-or-self with count <= T, or the cell
FP_DEV void block_of(const uint32_t* pyr, const uint32_t* counts, int g, uint64_t T, uint64_t m, int& lvl,
                     uint32_t& cnt)
{
    for (int l = 0; l <= g; ++l) {
        uint32_t c = pyr_count(pyr, counts, g, l, m >> (3 * (g - l)));
        if (c <= T || l == g) { lvl = l; cnt = c; return; }
    }
}

__global__ void k_chunk_mark(const uint32_t* __restrict__ pyr, const uint32_t* __restrict__ counts, int g,
                             uint64_t T, uint32_t* __restrict__ start)
{
    uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (1ull << (3 * g))) return;
    int l;
    uint32_t c;
    block_of(pyr, counts, g, T, m, l, c);
    uint64_t align = (1ull << (3 * (g - l))) - 1;
    start[m] = (c > 0 && (m & align) == 0) ? 1u : 0u;
}

__global__ void k_chunk_write(const uint32_t* __restrict__ pyr, const uint32_t* __restrict__ counts, int g,
                              uint64_t T, const uint32_t* __restrict__ start, const uint32_t* __restrict__ excl,
                              fp_chunk* __restrict__ chunks, uint32_t* __restrict__ lut, uint32_t* __restrict__ ccount)
{
    uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (1ull << (3 * g))) return;
    uint32_t id = excl[m] + start[m] - 1;   // chunk holding cell m when the cell is in a chunk
    if (start[m]) {
        int l;
        uint32_t c;
        block_of(pyr, counts, g, T, m, l, c);
        fp_chunk ch;
        ch.key = m >> (3 * (g - l));
        ch.count = c;
        ch.level = (uint32_t)l;
        chunks[id] = ch;
        ccount[id] = c;
    }
    lut[m] = counts[m] > 0 ? id : kNone;
}

// The bounds + preview pass of the main path: the tile's 32 KB of points are
// brought into shared memory by one bulk copy (cp.async.bulk, completion on an
// mbarrier) issued when the tile is claimed, so the copy is in flight while the
// keep flags are ranked and the tile's output offset is found by decoupled
// look-back; extents and kept points are then read from shared memory.  Few
// registers and 32 KB of shared memory per block: six blocks per SM, each with
// a whole tile in flight (2048-point tiles measured faster than 4096 and 1024).
// A second buffer per block, with the next tile claimed ahead, is slower: the
// claimed tile publishes its keep count only when its block reaches it, and
// every later tile's look-back waits for that.  Waits are bounded
// (FP_ERR_TIMEOUT).
constexpr size_t kBdBulkSmem = sizeof(int4) * kBdTile;

template <bool DECIM>
__global__ void __launch_bounds__(kBdNT) k_bounds_bulk(const fp_point* __restrict__ pts, uint64_t n, uint64_t first,
                                                       uint32_t modulus, fp_point* __restrict__ out, uint64_t out_cap,
                                                       uint64_t* __restrict__ out_count, int32_t* __restrict__ partial,
                                                       uint64_t* tile_status, uint32_t* tile_counter, uint64_t ntiles,
                                                       uint32_t* err)
{
    extern __shared__ __align__(128) int4 s_pts[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_cnt[kBdIPT][kBdNT / 32];
    __shared__ uint64_t s_base;
    __shared__ int32_t s_red[6][kBdNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    int32_t hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    uint32_t nwait = 0;
    for (;;) {
        __syncthreads();   // the previous tile's reads of s_pts are done
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(tile_counter, 1u);
            s_tile = t;
            if (t < ntiles) {
                const uint64_t b = (uint64_t)t * kBdTile;
                const uint32_t bytes = (uint32_t)(sizeof(int4) * min((uint64_t)kBdTile, n - b));
                fence_async_smem();
                mbar_expect_tx(&s_bar, bytes);
                bulk_g2s(s_pts, reinterpret_cast<const int4*>(pts) + b, bytes, &s_bar);
            }
        }
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint64_t base = tile * kBdTile;

        uint32_t keepmask = 0;
        if (DECIM) {
#pragma unroll
            for (int r = 0; r < kBdIPT; ++r) {
                const uint64_t i = base + (uint64_t)r * kBdNT + threadIdx.x;
                const bool k = i < n && keep_modulus(first, i, modulus);
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, k);
                if (lane == 0) s_cnt[r][warp] = __popc(bal);
                keepmask |= (uint32_t)k << r;
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                constexpr int per = kBdIPT * (kBdNT / 32) / 32;
                uint32_t v[per];
                uint32_t s = 0;
#pragma unroll
                for (int q = 0; q < per; ++q) {
                    const int e = lane * per + q;
                    v[q] = s_cnt[e / (kBdNT / 32)][e % (kBdNT / 32)];
                    s += v[q];
                }
                uint32_t x = s;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if (lane >= o) x += y;
                }
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
                uint32_t ex = x - s;
#pragma unroll
                for (int q = 0; q < per; ++q) {
                    const int e = lane * per + q;
                    s_cnt[e / (kBdNT / 32)][e % (kBdNT / 32)] = ex;
                    ex += v[q];
                }
                // decoupled look-back by the whole warp: 32 earlier tiles' words per
                // round trip; the sum runs back to the nearest inclusive prefix, and
                // stops (and reads again) at the nearest word not yet published
                uint64_t excl = 0;
                if (tile == 0) {
                    if (lane == 0)
                        atomicExch((unsigned long long*)&tile_status[0], (unsigned long long)(kFlagInc | total));
                } else {
                    if (lane == 0)
                        atomicExch((unsigned long long*)&tile_status[tile], (unsigned long long)(kFlagAgg | total));
                    int64_t t = (int64_t)tile - 1;
                    uint32_t spins = 0;
                    while (t >= 0) {
                        const int64_t q = t - lane;
                        const uint64_t w = q >= 0 ? ld_volatile64(&tile_status[q]) : kFlagInc;
                        const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (w >> 62) == 2);
                        const uint32_t none = __ballot_sync(0xFFFFFFFFu, (w >> 62) == 0);
                        const int fi = inc ? __ffs(inc) - 1 : 32, fn = none ? __ffs(none) - 1 : 32;
                        // lanes [0, take) are summed: up to the first unpublished word, or
                        // through the first inclusive prefix, or all 32 aggregates
                        const int take = fn < fi ? fn : (fi < 32 ? fi + 1 : 32);
                        uint64_t v = lane < take ? (w & kValMask) : 0;
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                        excl += v;
                        if (fi < fn) break;   // reached an inclusive prefix
                        if (take == 0 && ++spins > kSpinLimit) {
                            if (lane == 0) raise(err, FP_ERR_TIMEOUT);
                            break;
                        }
                        t -= take;
                    }
                    if (lane == 0)
                        atomicExch((unsigned long long*)&tile_status[tile],
                                   (unsigned long long)(kFlagInc | (excl + total)));
                }
                if (lane == 0) {
                    s_base = excl;
                    if (tile == ntiles - 1) {
                        *out_count = excl + total;
                        if (excl + total > out_cap) raise(err, FP_ERR_CAPACITY, 0);
                    }
                }
            }
        }
        // the tile's points have landed (bounded wait; on a time-out the copy is
        // given a second bounded wait to land before the block leaves)
        const bool ok = mbar_wait(&s_bar, nwait & 1);
        ++nwait;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) raise(err, FP_ERR_TIMEOUT);
            mbar_wait(&s_bar, (nwait - 1) & 1);
            break;
        }
#pragma unroll 4
        for (int r = 0; r < kBdIPT; ++r) {
            const uint64_t i = base + (uint64_t)r * kBdNT + threadIdx.x;
            if (i < n) {
                const int4 p = s_pts[r * kBdNT + threadIdx.x];
                lo[0] = min(lo[0], p.x); hi[0] = max(hi[0], p.x);
                lo[1] = min(lo[1], p.y); hi[1] = max(hi[1], p.y);
                lo[2] = min(lo[2], p.z); hi[2] = max(hi[2], p.z);
            }
        }
        if (DECIM) {
#pragma unroll 4
            for (int r = 0; r < kBdIPT; ++r) {
                const bool kept = (keepmask >> r) & 1u;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, kept);
                if (kept) {
                    const uint64_t pos = s_base + s_cnt[r][warp] + __popc(bal & lanemask_lt());
                    if (pos < out_cap) st_point(out, pos, s_pts[r * kBdNT + threadIdx.x]);
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(0xFFFFFFFFu, lo[a]);
        hi[a] = __reduce_max_sync(0xFFFFFFFFu, hi[a]);
    }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { s_red[a][warp] = lo[a]; s_red[3 + a][warp] = hi[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        int32_t v = s_red[a][0];
        for (int w = 1; w < kBdNT / 32; ++w) v = a < 3 ? min(v, s_red[a][w]) : max(v, s_red[a][w]);
        partial[blockIdx.x * 6 + a] = v;
    }
}

// ----------------------------------------------------------------- host side
// the carve of launch_bounds_decimate: block partials (grid <= 8 per SM), one
// look-back word per tile, the tile counter
size_t bounds_ws_bytes(uint64_t n, int num_sms)
{
    const size_t nt = (size_t)((n + kBdTile - 1) / kBdTile);
    return Workspace::bytes_for({6 * 4 * (size_t)num_sms * 8, 8 * (nt ? nt : 1), 4 * sizeof(uint32_t)});
}

cudaError_t launch_bounds_decimate(const fp_point* pts, uint64_t n, fp_cube* cube, bool bounds, bool decim,
                                   uint64_t first, uint32_t modulus, fp_point* out, uint64_t out_cap,
                                   uint64_t* out_count, const Workspace& ws, cudaStream_t st)
{
    uint64_t ntiles = (n + kBdTile - 1) / kBdTile;
    int grid = (int)std::min<uint64_t>(ntiles ? ntiles : 1, (uint64_t)ws.num_sms * 8);
    int32_t* partial = ws.take<int32_t>(6 * (size_t)grid);
    uint64_t* status = ws.take<uint64_t>(ntiles ? ntiles : 1);
    uint32_t* counter = ws.take<uint32_t>(4);
    cudaError_t e = cudaMemsetAsync(counter, 0, 4 * sizeof(uint32_t), st);
    if (e) return e;
    if (decim && ntiles) {
        e = cudaMemsetAsync(status, 0, ntiles * sizeof(uint64_t), st);
        if (e) return e;
    }
    if (decim && n == 0) k_zero_count<<<1, 1, 0, st>>>(out_count);
    if (n) {
        KTimerScope kt(FP_KERNEL_BOUNDS_DECIMATE, st);
        if (bounds) {   // points by bulk copy into shared memory
            auto kern = decim ? k_bounds_bulk<true> : k_bounds_bulk<false>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBdBulkSmem)))
                return e;
            kern<<<grid, kBdNT, kBdBulkSmem, st>>>(pts, n, first, modulus, out, out_cap, out_count, partial, status,
                                                  counter, ntiles, ws.err);
        } else
            k_bounds_decimate<false, KEEP_MODULUS><<<grid, kBdNT, 0, st>>>(
                pts, n, first, modulus, out, out_cap, out_count, partial, status, counter, ntiles, ws.err, nullptr,
                nullptr, 0);
    }
    if (bounds) k_bounds_final<<<1, 256, 0, st>>>(partial, n ? grid : 0, n, cube);
    return cudaGetLastError();
}

// ----------------------------------------------------- spatial preview
// Spatially constrained random sampler (the alternative preview the paper
// proposes for clouds whose file order makes the uniform one uneven, Sec. 6):
// of the points of every occupied cell of the 2^level grid, the one with the
// smallest splitmix64(first + i) is kept (a uniformly random point of the cell,
// the same on every run).  Pass 1 takes each cell's smallest hash; pass 2 is
// the preview compaction with "hash == its cell's smallest" as the keep rule.
__global__ void __launch_bounds__(256) k_cell_min_hash(const fp_point* __restrict__ pts, uint64_t n, uint64_t first,
                                                       const fp_cube* cube_p, int level,
                                                       unsigned long long* cell_min)
{
    const CubeDev cube = load_cube(cube_p);
    const int csh = 3 * (kKeyLevels - level);
    // a cell's running minimum only falls: a hash not below any value read for
    // it (however stale) cannot be the minimum, and the atomic is skipped --
    // in a cell of c points in random order about ln c atomics remain
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int4 q = ld_point_cs(pts, i);
        unsigned long long* slot = &cell_min[key21(q.x, q.y, q.z, cube) >> csh];
        const unsigned long long h = splitmix64(first + i);
        if (h < __ldcg(slot)) atomicMin(slot, h);
    }
}

size_t spatial_ws_bytes(uint64_t n, int level, int num_sms)
{
    return Workspace::bytes_for({sizeof(uint64_t) << (3 * level)}) + bounds_ws_bytes(n, num_sms);
}

cudaError_t launch_preview_spatial(const fp_point* pts, uint64_t n, const fp_cube* cube, int level, uint64_t first,
                                   fp_point* out, uint64_t out_cap, uint64_t* out_count, const Workspace& ws,
                                   cudaStream_t st)
{
    const uint64_t cells = 1ull << (3 * level);
    uint64_t* cell_min = ws.take<uint64_t>(cells);
    uint64_t ntiles = (n + kBdTile - 1) / kBdTile;
    int grid = (int)std::min<uint64_t>(ntiles ? ntiles : 1, (uint64_t)ws.num_sms * 8);
    int32_t* partial = ws.take<int32_t>(6 * (size_t)grid);
    uint64_t* status = ws.take<uint64_t>(ntiles ? ntiles : 1);
    uint32_t* counter = ws.take<uint32_t>(4);
    cudaError_t e;
    if ((e = cudaMemsetAsync(counter, 0, 4 * sizeof(uint32_t), st))) return e;
    if (n == 0) {
        k_zero_count<<<1, 1, 0, st>>>(out_count);
        return cudaGetLastError();
    }
    if ((e = cudaMemsetAsync(status, 0, ntiles * sizeof(uint64_t), st))) return e;
    if ((e = cudaMemsetAsync(cell_min, 0xFF, cells * sizeof(uint64_t), st))) return e;
    const int gm = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)ws.num_sms * 8);
    k_cell_min_hash<<<gm, 256, 0, st>>>(pts, n, first, cube, level, reinterpret_cast<unsigned long long*>(cell_min));
    k_bounds_decimate<false, KEEP_CELL_MIN><<<grid, kBdNT, 0, st>>>(pts, n, first, 1, out, out_cap, out_count, partial,
                                                                    status, counter, ntiles, ws.err, cell_min, cube,
                                                                    level);
    return cudaGetLastError();
}

cudaError_t launch_count(const fp_point* pts, uint64_t n, const fp_cube* cube, int g, uint32_t* counts,
                         bool accumulate, uint32_t* cells, const Workspace& ws, cudaStream_t st)
{
    const uint64_t ncell = 1ull << (3 * g);
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(counts, 0, ncell * sizeof(uint32_t), st);
        if (e) return e;
    }
    if (n == 0) return cudaSuccess;
    uint64_t want = (n + 1023) / 1024;
    int grid = (int)std::min<uint64_t>(want, (uint64_t)ws.num_sms * 8);
    KTimerScope kt(FP_KERNEL_COUNT, st);
    k_count<true><<<grid, 256, 0, st>>>(pts, n, cube, g, counts, cells);
    return cudaGetLastError();
}

size_t merge_ws_bytes(int g)
{
    uint64_t cells = 1ull << (3 * g);
    uint64_t pyr = ((1ull << (3 * g)) - 1) / 7;
    return Workspace::bytes_for({pyr * 4, cells * 4, cells * 4, cells * 4, (size_t)kScanMaxTiles * 8,
                                 (size_t)kScanMaxTiles * 8, 8});
}

cudaError_t launch_merge(const uint32_t* counts, int g, uint64_t T, fp_chunk* chunks, uint32_t* num_chunks,
                         uint32_t* lut, uint64_t* offsets, const Workspace& ws, cudaStream_t st)
{
    uint64_t cells = 1ull << (3 * g);
    uint64_t npyr = ((1ull << (3 * g)) - 1) / 7;
    uint32_t* pyr = ws.take<uint32_t>(npyr ? npyr : 1);
    uint32_t* start = ws.take<uint32_t>(cells);
    uint32_t* excl = ws.take<uint32_t>(cells);
    uint32_t* ccount = ws.take<uint32_t>(cells);
    uint32_t* tiles32 = ws.take<uint32_t>(kScanMaxTiles);
    uint64_t* tiles64 = ws.take<uint64_t>(kScanMaxTiles);
    for (int l = g - 1; l >= 0; --l) {
        uint64_t np = 1ull << (3 * l);
        const uint32_t* child = l + 1 == g ? counts : pyr + ((1ull << (3 * (l + 1))) - 1) / 7;
        uint32_t* parent = pyr + (np - 1) / 7;
        k_pyramid_level<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(child, parent, np);
    }
    unsigned gb = (unsigned)((cells + 255) / 256);
    k_chunk_mark<<<gb, 256, 0, st>>>(pyr, counts, g, T, start);
    cudaError_t e = scan_exclusive<uint32_t, uint32_t>(start, excl, cells, nullptr, tiles32, num_chunks,
                                                       (uint32_t*)nullptr, st);
    if (e) return e;
    k_chunk_write<<<gb, 256, 0, st>>>(pyr, counts, g, T, start, excl, chunks, lut, ccount);
    // offsets[0..K] = exclusive prefix of chunk counts; offsets[K] = total
    uint64_t* total = ws.take<uint64_t>(1);
    e = scan_exclusive<uint32_t, uint64_t>(ccount, offsets, cells, num_chunks, tiles64, total, (uint64_t*)nullptr, st);
    if (e) return e;
    k_put_at<<<1, 1, 0, st>>>(offsets, num_chunks, total);
    return cudaGetLastError();
}

}  // namespace fp
