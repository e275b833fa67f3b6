// fp_build_batched: many clouds per call.  Every cloud runs the plain entry
// points in order (bounds + preview, count, merge, distribute, chunk octrees,
// subsample) on one of a set of library-owned streams ("lanes") forked from
// and joined back into the caller's stream with events, so that the many small
// launches of small clouds overlap and the whole batch is one unit for CUDA
// graph capture.  Optionally (fp_build_batched_ex, fused_first) the bounds +
// preview pass and the count pass of up to 256 clouds run as one launch each
// over the work items of all of them, before the lanes fork.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>
#include "fp_internal.cuh"

namespace fp {

fp_status check_params(const fp_params* p);

namespace {

struct Lanes {
    bool ready = false;
    cudaStream_t s[FP_MAX_LANES];
    cudaEvent_t join[FP_MAX_LANES];
    cudaEvent_t fork;
};

std::mutex g_lane_mu;
Lanes g_lanes[64];

fp_status lanes_of_device(Lanes*& out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FP_ERR_CUDA;
    Lanes& L = g_lanes[dev];
    if (!L.ready) {
        for (int i = 0; i < FP_MAX_LANES; ++i) {
            if (cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking) != cudaSuccess) return FP_ERR_CUDA;
            if (cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming) != cudaSuccess) return FP_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess) return FP_ERR_CUDA;
        L.ready = true;
    }
    out = &L;
    return FP_OK;
}

// ------------------------------------------------ fused first passes
// The bounds + preview pass and the count pass of every cloud of a batch in one
// launch each (work items of all clouds, claimed in order from one counter),
// instead of a few small launches per cloud.  Up to kFusedMax clouds per
// launch; their descriptors travel in the kernel parameters, so the launch
// needs no copy of host memory and captures into a CUDA graph as it is.
constexpr int kFusedMax = 256;
constexpr int kFbNT = 256;
constexpr int kFbIPT = 16;
constexpr int kFbTile = kFbNT * kFbIPT;   // 4096 points per preview tile (the layout does not depend on it)
constexpr int kFcTiles = 16;              // count work item: 16 tiles (65,536 points)

struct FusedCloud {
    const int4* pts;
    uint64_t n;
    fp_cube* cube;
    int4* prev;
    uint64_t prev_cap;
    uint64_t* prev_cnt;
    uint32_t* counts;
    uint32_t modulus, g;
};

struct FusedArgs {
    uint32_t ncloud, pad;
    uint64_t tile0[kFusedMax + 1];   // first preview tile of every cloud; tile0[ncloud] = all tiles
    uint64_t item0[kFusedMax + 1];   // first count item of every cloud
    FusedCloud c[kFusedMax];
};
static_assert(sizeof(FusedArgs) <= 32000, "fused descriptors must fit the kernel parameters");

// cloud of work item t: last c with first[c] <= t (first[] ascending)
FP_DEV uint32_t fused_cloud(const uint64_t* first, uint32_t ncloud, uint64_t t)
{
    uint32_t a = 0, b = ncloud;
    while (b - a > 1) {
        const uint32_t m = (a + b) >> 1;
        if (first[m] <= t) a = m;
        else b = m;
    }
    return a;
}

// zero every count grid and preview count, open every cube's extents
__global__ void k_fused_init(const __grid_constant__ FusedArgs a)
{
    for (uint32_t c = blockIdx.x; c < a.ncloud; c += gridDim.x) {
        const FusedCloud& d = a.c[c];
        const uint64_t cells = 1ull << (3 * d.g);
        for (uint64_t m = threadIdx.x; m < cells; m += blockDim.x) d.counts[m] = 0;
        if (threadIdx.x == 0) {
            *d.prev_cnt = 0;
            for (int k = 0; k < 3; ++k) { d.cube->o[k] = INT32_MAX; d.cube->mx[k] = INT32_MIN; }
            d.cube->S = 0;
        }
    }
}

// bounds + preview of every tile of every cloud: per-axis extents folded into
// the cloud's cube by atomics; kept points compacted in index order by a
// decoupled look-back that stops at the cloud's first tile
__global__ void __launch_bounds__(kFbNT, 2) k_fused_bounds_decimate(const __grid_constant__ FusedArgs a,
                                                                    uint64_t* status, uint32_t* counter,
                                                                    uint32_t* err)
{
    __shared__ uint32_t s_item[2];
    __shared__ uint32_t s_cnt[kFbIPT][kFbNT / 32];
    __shared__ uint64_t s_base;
    __shared__ int32_t s_red[6][kFbNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t ntiles = a.tile0[a.ncloud];
    for (;;) {
        if (threadIdx.x == 0) {
            const uint64_t t = atomicAdd(counter, 1u);
            s_item[0] = (uint32_t)t;
            s_item[1] = t < ntiles ? fused_cloud(a.tile0, a.ncloud, t) : 0u;
        }
        __syncthreads();
        const uint64_t t = s_item[0];
        const uint32_t c = s_item[1];
        __syncthreads();
        if (t >= ntiles) break;
        const FusedCloud& d = a.c[c];
        const uint64_t t0 = a.tile0[c], tl = t - t0, nt = a.tile0[c + 1] - t0;
        constexpr uint64_t kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kValMask = (1ull << 62) - 1;
        const uint64_t base = tl * kFbTile;
        int4 pv[kFbIPT];
#pragma unroll
        for (int r = 0; r < kFbIPT; ++r) {   // all loads in flight together
            const uint64_t i = base + (uint64_t)r * kFbNT + threadIdx.x;
            pv[r] = i < d.n ? ld_point_cs(reinterpret_cast<const fp_point*>(d.pts), i) : make_int4(0, 0, 0, 0);
        }
        uint32_t keepmask = 0;
#pragma unroll
        for (int r = 0; r < kFbIPT; ++r) {
            const uint64_t i = base + (uint64_t)r * kFbNT + threadIdx.x;
            bool k = false;
            if (i < d.n) {
                const uint64_t h = splitmix64(i);
                k = (d.modulus & (d.modulus - 1)) == 0 ? (h & ((uint64_t)d.modulus - 1)) == 0 : (h % d.modulus) == 0;
            }
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, k);
            if (lane == 0) s_cnt[r][warp] = __popc(bal);
            keepmask |= (uint32_t)k << r;
        }
        // extents of the tile, folded into the cloud's cube
        int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
#pragma unroll
        for (int r = 0; r < kFbIPT; ++r) {
            const uint64_t i = base + (uint64_t)r * kFbNT + threadIdx.x;
            if (i < d.n) {
                lo[0] = min(lo[0], pv[r].x); hi[0] = max(hi[0], pv[r].x);
                lo[1] = min(lo[1], pv[r].y); hi[1] = max(hi[1], pv[r].y);
                lo[2] = min(lo[2], pv[r].z); hi[2] = max(hi[2], pv[r].z);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = __reduce_min_sync(0xFFFFFFFFu, lo[k]);
            hi[k] = __reduce_max_sync(0xFFFFFFFFu, hi[k]);
        }
        if (lane == 0)
            for (int k = 0; k < 3; ++k) { s_red[k][warp] = lo[k]; s_red[3 + k][warp] = hi[k]; }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int k = threadIdx.x;
            int32_t v = s_red[k][0];
            for (int w = 1; w < kFbNT / 32; ++w) v = k < 3 ? min(v, s_red[k][w]) : max(v, s_red[k][w]);
            if (k < 3) atomicMin(&d.cube->o[k], v);
            else atomicMax(&d.cube->mx[k - 3], v);
        }
        // exclusive scan of the keep counts over (r, warp) order = index order, then the look-back
        if (threadIdx.x < 32) {
            constexpr int per = kFbIPT * (kFbNT / 32) / 32;
            uint32_t v[per];
            uint32_t s = 0;
#pragma unroll
            for (int q = 0; q < per; ++q) {
                const int e = lane * per + q;
                v[q] = s_cnt[e / (kFbNT / 32)][e % (kFbNT / 32)];
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
                s_cnt[e / (kFbNT / 32)][e % (kFbNT / 32)] = ex;
                ex += v[q];
            }
            if (lane == 0) {
                uint64_t excl = 0;
                if (tl == 0) {
                    atomicExch((unsigned long long*)&status[t], (unsigned long long)(kFlagInc | total));
                } else {
                    atomicExch((unsigned long long*)&status[t], (unsigned long long)(kFlagAgg | total));
                    int64_t q = (int64_t)t - 1;
                    uint32_t spins = 0;
                    while (q >= (int64_t)t0) {
                        const uint64_t s2 = ld_volatile64(&status[q]);
                        if ((s2 >> 62) == 0) {
                            if (++spins > kSpinLimit) { raise(err, FP_ERR_TIMEOUT); break; }
                            continue;
                        }
                        excl += s2 & kValMask;
                        if ((s2 >> 62) == 2) break;
                        --q;
                    }
                    atomicExch((unsigned long long*)&status[t], (unsigned long long)(kFlagInc | (excl + total)));
                }
                s_base = excl;
                if (tl == nt - 1) {
                    *d.prev_cnt = excl + total;
                    if (excl + total > d.prev_cap) raise(err, FP_ERR_CAPACITY, 0);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kFbIPT; ++r) {
            const bool kept = (keepmask >> r) & 1u;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, kept);
            if (kept) {
                const uint64_t pos = s_base + s_cnt[r][warp] + __popc(bal & lanemask_lt());
                if (pos < d.prev_cap) d.prev[pos] = pv[r];
            }
        }
        __syncthreads();
    }
}

// cube side of every cloud from its extents (S = 0 for an empty cloud)
__global__ void k_fused_cube(const __grid_constant__ FusedArgs a)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ncloud; c += gridDim.x * blockDim.x) {
        fp_cube* cb = a.c[c].cube;
        if (a.c[c].n == 0) {
            for (int k = 0; k < 3; ++k) { cb->o[k] = 0; cb->mx[k] = 0; }
            cb->S = 0;
            continue;
        }
        uint64_t ext = 0;
        for (int k = 0; k < 3; ++k) {
            const uint64_t e = (uint64_t)((int64_t)cb->mx[k] - (int64_t)cb->o[k]);
            ext = e > ext ? e : ext;
        }
        cb->S = ext + 1;
    }
}

// count grids of every cloud: work items of kFcTiles tiles of one cloud;
// warp-aggregated atomics, and a per-block table of SLOTS hot cells flushed
// after every item (SLOTS == 0: no table)
template <int NT, int SLOTS>
__global__ void __launch_bounds__(NT) k_fused_count(const __grid_constant__ FusedArgs a, uint32_t* counter)
{
    __shared__ uint32_t s_tag[SLOTS > 0 ? SLOTS : 1], s_cnt[SLOTS > 0 ? SLOTS : 1];
    __shared__ uint32_t s_item[2];
    const int lane = threadIdx.x & 31;
    const uint64_t nitems = a.item0[a.ncloud];
    for (;;) {
        if (threadIdx.x == 0) {
            const uint64_t t = atomicAdd(counter, 1u);
            s_item[0] = (uint32_t)t;
            s_item[1] = t < nitems ? fused_cloud(a.item0, a.ncloud, t) : 0u;
        }
        for (int q = threadIdx.x; q < SLOTS; q += NT) { s_tag[q] = kNone; s_cnt[q] = 0; }
        __syncthreads();
        const uint64_t t = s_item[0];
        const uint32_t c = s_item[1];
        __syncthreads();
        if (t >= nitems) break;
        const FusedCloud& d = a.c[c];
        const CubeDev cube = load_cube(d.cube);
        const int g = (int)d.g;
        const float sg = scale_at(cube, g);
        const uint64_t b0 = (t - a.item0[c]) * (uint64_t)(kFcTiles * kFbTile);
        const uint64_t b1 = min(d.n, b0 + (uint64_t)(kFcTiles * kFbTile));
        for (uint64_t i0 = b0; i0 < b1; i0 += 4 * NT) {   // block-uniform
            uint32_t key[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + (uint64_t)u * NT + threadIdx.x;
                key[u] = kNone;
                if (i < b1) {
                    const int4 p = ld_point_cs(reinterpret_cast<const fp_point*>(d.pts), i);
                    key[u] = key_small(p.x, p.y, p.z, cube, sg, g);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key[u]);
                if (key[u] == kNone || lane != __ffs(peers) - 1) continue;
                if (SLOTS > 0) {
                    constexpr int kLog2 = SLOTS >= 4096 ? 12 : (SLOTS >= 1024 ? 10 : 1);
                    const uint32_t slot = (key[u] * 2654435761u) >> (32 - kLog2);
                    uint32_t tg = s_tag[slot];
                    if (tg == kNone) tg = atomicCAS(&s_tag[slot], kNone, key[u]) == kNone ? key[u] : s_tag[slot];
                    if (tg == key[u]) { atomicAdd(&s_cnt[slot], (uint32_t)__popc(peers)); continue; }
                }
                atomicAdd(&d.counts[key[u]], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < SLOTS; q += NT)
            if (s_cnt[q]) atomicAdd(&d.counts[s_tag[q]], s_cnt[q]);
        __syncthreads();
    }
}

bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// workspace one cloud needs: the largest of its stages
size_t cloud_ws(const fp_cloud_desc& c)
{
    size_t w = 0;
    for (fp_stage st : {FP_STAGE_BOUNDS_DECIMATE, FP_STAGE_COUNT, FP_STAGE_MERGE, FP_STAGE_DISTRIBUTE, FP_STAGE_OCTREE,
                        FP_STAGE_SUBSAMPLE})
        w = std::max(w, fp_workspace_size(st, c.n, &c.prm));
    return (w + 255) / 256 * 256;
}

// lane of every cloud: largest first, each to the lane with the fewest points (ties: lowest lane)
std::vector<int> assign(const fp_cloud_desc* c, uint32_t ncloud, uint32_t nlanes)
{
    std::vector<uint32_t> order(ncloud);
    for (uint32_t i = 0; i < ncloud; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return c[a].n > c[b].n; });
    std::vector<uint64_t> load(nlanes, 0);
    std::vector<int> lane(ncloud, 0);
    for (uint32_t k : order) {
        uint32_t best = 0;
        for (uint32_t l = 1; l < nlanes; ++l)
            if (load[l] < load[best]) best = l;
        lane[k] = (int)best;
        load[best] += c[k].n + 1;
    }
    return lane;
}

fp_status check_cloud(const fp_cloud_desc& c)
{
    fp_status s = check_params(&c.prm);
    if (s != FP_OK) return s;
    if (c.n >= (1ull << 30)) return FP_ERR_TOO_LARGE;
    if (!c.d_cube || !c.d_preview_count || !c.d_counts || !c.d_chunks || !c.d_num_chunks || !c.d_lut ||
        !c.d_offsets || !c.d_num_nodes || (c.node_cap && !c.d_nodes))
        return FP_ERR_INVALID;
    if (c.n && (!c.d_pts || !c.d_dist || !c.d_perm || !c.d_owner || !c.d_final || !c.d_final_perm ||
                (c.preview_cap && !c.d_preview)))
        return FP_ERR_INVALID;
    if (c.n && c.d_pts == c.d_dist) return FP_ERR_INVALID;
    if (c.n && (!aligned(c.d_pts) || !aligned(c.d_dist) || !aligned(c.d_final))) return FP_ERR_ALIGN;
    if ((c.d_preview && !aligned(c.d_preview)) || (c.d_leaf_pts && !aligned(c.d_leaf_pts))) return FP_ERR_ALIGN;
    if (c.node_cap > (1u << 23)) return FP_ERR_UNSUPPORTED;
    return FP_OK;
}

// the plain calls, in order, on one stream (first_done: bounds + preview and
// count already done by the fused launches)
fp_status run_cloud(const fp_cloud_desc& c, char* ws, size_t ws_bytes, cudaStream_t st, bool first_done)
{
    fp_status s;
    const uint32_t g = c.prm.grid_log2;
    if (!first_done) {
        if ((s = fp_bounds_decimate(c.d_pts, c.n, c.d_cube, 0, c.prm.decim_modulus, c.d_preview, c.preview_cap,
                                    c.d_preview_count, ws, ws_bytes, st)))
            return s;
        if ((s = fp_count(c.d_pts, c.n, c.d_cube, g, c.d_counts, 0, ws, ws_bytes, st))) return s;
    }
    if ((s = fp_merge_chunks(c.d_counts, g, c.prm.chunk_threshold, c.d_chunks, c.d_num_chunks, c.d_lut, c.d_offsets,
                             ws, ws_bytes, st)))
        return s;
    if ((s = fp_distribute(c.d_pts, c.n, c.d_cube, g, c.d_lut, c.d_offsets, c.d_num_chunks, c.d_dist, c.d_perm, ws,
                           ws_bytes, st)))
        return s;
    if ((s = fp_build_chunk_octree(c.d_dist, c.d_perm, c.n, c.d_cube, c.d_chunks, c.d_num_chunks, c.d_offsets,
                                   c.d_counts, &c.prm, c.d_nodes, c.node_cap, c.d_num_nodes, c.d_leaf_pts,
                                   c.d_leaf_perm, c.d_owner, ws, ws_bytes, st)))
        return s;
    return fp_subsample(c.d_nodes, c.d_num_nodes, c.node_cap, c.d_dist, c.d_perm, c.d_owner, c.n, c.d_chunks,
                        c.d_num_chunks, c.d_offsets, c.d_final, c.d_final_perm, ws, ws_bytes, st);
}

// workspace of the fused first passes: one look-back word per preview tile of
// the largest group of kFusedMax clouds, and two work counters
size_t fused_ws(const fp_cloud_desc* c, uint32_t ncloud)
{
    uint64_t most = 0;
    for (uint32_t g0 = 0; g0 < ncloud; g0 += kFusedMax) {
        uint64_t t = 0;
        for (uint32_t i = g0; i < std::min<uint32_t>(ncloud, g0 + kFusedMax); ++i) t += (c[i].n + kFbTile - 1) / kFbTile;
        most = std::max(most, t);
    }
    return Workspace::bytes_for({8 * (size_t)(most ? most : 1), 16});
}

template <int NT, int SLOTS>
cudaError_t launch_fused_count(const FusedArgs& a, uint32_t* counter, int num_sms, cudaStream_t st)
{
    const uint64_t items = a.item0[a.ncloud];
    const int per_sm = NT == 256 ? 8 : 4;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(items, (uint64_t)num_sms * per_sm));
    k_fused_count<NT, SLOTS><<<grid, NT, 0, st>>>(a, counter);
    return cudaGetLastError();
}

// bounds + preview and count of clouds [g0, g1) in one launch each
fp_status fused_first(const fp_cloud_desc* c, uint32_t g0, uint32_t g1, const fp_batch_opts& o, char* ws,
                      int num_sms, uint32_t* err, cudaStream_t st)
{
    static FusedArgs a;   // host staging of the kernel parameters (copied at launch)
    std::memset(&a, 0, sizeof(a));
    a.ncloud = g1 - g0;
    uint64_t tiles = 0, items = 0;
    for (uint32_t i = g0; i < g1; ++i) {
        const fp_cloud_desc& d = c[i];
        FusedCloud& f = a.c[i - g0];
        f.pts = reinterpret_cast<const int4*>(d.d_pts);
        f.n = d.n;
        f.cube = d.d_cube;
        f.prev = reinterpret_cast<int4*>(d.d_preview);
        f.prev_cap = d.d_preview ? d.preview_cap : 0;
        f.prev_cnt = d.d_preview_count;
        f.counts = d.d_counts;
        f.modulus = d.prm.decim_modulus;
        f.g = d.prm.grid_log2;
        a.tile0[i - g0] = tiles;
        a.item0[i - g0] = items;
        tiles += (d.n + kFbTile - 1) / kFbTile;
        items += (d.n + (uint64_t)kFcTiles * kFbTile - 1) / ((uint64_t)kFcTiles * kFbTile);
    }
    a.tile0[a.ncloud] = tiles;
    a.item0[a.ncloud] = items;
    Workspace w;
    w.base = ws;
    uint64_t* status = w.take<uint64_t>(tiles ? tiles : 1);
    uint32_t* counter = w.take<uint32_t>(4);
    if (cudaMemsetAsync(status, 0, 8 * (tiles ? tiles : 1), st) != cudaSuccess) return FP_ERR_CUDA;
    if (cudaMemsetAsync(counter, 0, 16, st) != cudaSuccess) return FP_ERR_CUDA;
    k_fused_init<<<(int)std::min<uint32_t>(a.ncloud, 1024u), 256, 0, st>>>(a);
    if (tiles) {
        const int gb = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)num_sms * 2));
        k_fused_bounds_decimate<<<gb, kFbNT, 0, st>>>(a, status, counter, err);
    }
    k_fused_cube<<<1, 256, 0, st>>>(a);
    if (items) {
        cudaError_t e;
        const int slots = o.count_slots;
        if (o.count_threads == 512)
            e = slots == 0 ? launch_fused_count<512, 0>(a, counter + 1, num_sms, st)
                : slots == 4096 ? launch_fused_count<512, 4096>(a, counter + 1, num_sms, st)
                                : launch_fused_count<512, 1024>(a, counter + 1, num_sms, st);
        else
            e = slots == 0 ? launch_fused_count<256, 0>(a, counter + 1, num_sms, st)
                : slots == 4096 ? launch_fused_count<256, 4096>(a, counter + 1, num_sms, st)
                                : launch_fused_count<256, 1024>(a, counter + 1, num_sms, st);
        if (e) return FP_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

bool opts_ok(const fp_batch_opts* o)
{
    return o && o->nlanes >= 1 && o->nlanes <= FP_MAX_LANES && (o->count_threads == 256 || o->count_threads == 512) &&
           (o->count_slots == 0 || o->count_slots == 1024 || o->count_slots == 4096);
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

size_t fp_batch_workspace_size_ex(const fp_cloud_desc* h_clouds, uint32_t ncloud, const fp_batch_opts* opts)
{
    if (!h_clouds || !opts_ok(opts)) return 0;
    const uint32_t nlanes = opts->nlanes;
    std::vector<int> lane = assign(h_clouds, ncloud, nlanes);
    std::vector<size_t> need(nlanes, 0);
    for (uint32_t i = 0; i < ncloud; ++i) need[lane[i]] = std::max(need[lane[i]], cloud_ws(h_clouds[i]));
    size_t t = opts->fused_first ? fused_ws(h_clouds, ncloud) : 0;
    for (size_t w : need) t += w;
    return t;
}

size_t fp_batch_workspace_size(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes)
{
    const fp_batch_opts o{nlanes, 0u, 256u, 1024u};
    return fp_batch_workspace_size_ex(h_clouds, ncloud, &o);
}

fp_status fp_build_batched_ex(const fp_cloud_desc* h_clouds, uint32_t ncloud, const fp_batch_opts* opts,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if ((ncloud && !h_clouds) || !opts_ok(opts)) return FP_ERR_INVALID;
    for (uint32_t i = 0; i < ncloud; ++i) {
        fp_status s = check_cloud(h_clouds[i]);
        if (s != FP_OK) return s;
    }
    if (ncloud == 0) return FP_OK;
    const uint32_t nlanes = opts->nlanes;
    const size_t need_total = fp_batch_workspace_size_ex(h_clouds, ncloud, opts);
    if (need_total && (!d_ws || ws_bytes < need_total)) return FP_ERR_WORKSPACE;
    std::vector<int> lane = assign(h_clouds, ncloud, nlanes);
    std::vector<size_t> need(nlanes, 0), base(nlanes, 0);
    for (uint32_t i = 0; i < ncloud; ++i) need[lane[i]] = std::max(need[lane[i]], cloud_ws(h_clouds[i]));
    const size_t f0 = opts->fused_first ? fused_ws(h_clouds, ncloud) : 0;
    base[0] = f0;
    for (uint32_t l = 1; l < nlanes; ++l) base[l] = base[l - 1] + need[l - 1];

    std::lock_guard<std::mutex> lk(g_lane_mu);
    Lanes* L = nullptr;
    fp_status s = lanes_of_device(L);
    if (s != FP_OK) return s;
    if (opts->fused_first) {   // on the caller's stream, before the lanes fork
        Workspace w;
        if ((s = make_workspace(d_ws, ws_bytes, 0, w)) != FP_OK) return s;
        for (uint32_t g0 = 0; g0 < ncloud; g0 += kFusedMax)
            if ((s = fused_first(h_clouds, g0, std::min<uint32_t>(ncloud, g0 + kFusedMax), *opts,
                                 static_cast<char*>(d_ws), w.num_sms, w.err, stream)) != FP_OK)
                return s;
    }
    if (cudaEventRecord(L->fork, stream) != cudaSuccess) return FP_ERR_CUDA;
    for (uint32_t l = 0; l < nlanes; ++l)
        if (cudaStreamWaitEvent(L->s[l], L->fork, 0) != cudaSuccess) return FP_ERR_CUDA;
    // clouds in descriptor order within each lane
    fp_status first_err = FP_OK;
    for (uint32_t i = 0; i < ncloud && first_err == FP_OK; ++i) {
        const int l = lane[i];
        first_err = run_cloud(h_clouds[i], static_cast<char*>(d_ws) + base[l], need[l], L->s[l],
                              opts->fused_first != 0);
    }
    // join every lane, also after an error, so the caller's stream never runs ahead of enqueued work
    for (uint32_t l = 0; l < nlanes; ++l) {
        if (cudaEventRecord(L->join[l], L->s[l]) != cudaSuccess) return FP_ERR_CUDA;
        if (cudaStreamWaitEvent(stream, L->join[l], 0) != cudaSuccess) return FP_ERR_CUDA;
    }
    return first_err;
}

fp_status fp_build_batched(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes, void* d_ws,
                           size_t ws_bytes, cudaStream_t stream)
{
    if (nlanes < 1 || nlanes > FP_MAX_LANES) return FP_ERR_INVALID;
    const fp_batch_opts o{nlanes, 0u, 256u, 1024u};
    return fp_build_batched_ex(h_clouds, ncloud, &o, d_ws, ws_bytes, stream);
}

}  // extern "C"
