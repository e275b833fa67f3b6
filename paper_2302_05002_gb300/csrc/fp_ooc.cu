// fp_ooc.cu -- fp_build_ooc: the out-of-core build of one cloud held in pinned
// host memory, every device buffer inside a caller-given arena (the budget).
//
// The level-of-detail owner and the leaf of a point depend only on the points
// of its level-g cell and on the count pyramid above it (owner levels at or
// above g collapse to the root since g <= s), and chunks are unions of whole
// level-g cells.  So the cloud is cut into groups of consecutive chunks that
// fit the arena; every group's local octrees run on the device against the
// whole cloud's count grid, the node table of the whole cloud is assembled
// from the count pyramid and the groups' deeper nodes, and the final layout is
// written group by group -- points kept by nodes above the chunks (count > T,
// level < g) are staged and merged across groups by one device sort.
//
// Passes over the host points (pieces of piece_points, double-buffered copies
// on a side stream): bounds + preview, counts, and the distribution into the
// host store (each piece scattered by chunk at per-chunk cursors); then the
// groups are read back from the store -- unless the arena holds the whole
// distributed cloud next to a group as large as the largest chunk, in which
// case pass 3 also writes it to the device and the group passes read it there
// (a cloud up to about half the arena in size crosses the link three times
// fewer); when the arena also holds a raw copy of the cloud, pass 1 leaves it
// there and passes 2 and 3 read it on the device.  The pinned host scratch is the out-of-core store between passes:
// the distributed points and original indices of every group, the two levels
// and the owner of every point, and the staged records.
#include <algorithm>
#include <vector>
#include "fp_sort.cuh"

namespace fp {

fp_status check_params(const fp_params* p);
size_t bounds_ws_bytes(uint64_t n, int num_sms);
fp_status make_workspace(void* base, size_t bytes, size_t need, Workspace& ws);
size_t merge_ws_bytes(int g);

namespace {

constexpr uint64_t kMaxPiece = 1ull << 23;   // the flag scan covers 8M entries

// ------------------------------------------------------------------ kernels
__global__ void k_cube_fold(fp_cube* acc, const fp_cube* piece, int first)
{
    fp_cube a = *acc;
    const fp_cube p = *piece;
    if (first) {
        a = p;
    } else {
        for (int k = 0; k < 3; ++k) {
            a.o[k] = min(a.o[k], p.o[k]);
            a.mx[k] = max(a.mx[k], p.mx[k]);
        }
    }
    uint64_t S = 0;
    for (int k = 0; k < 3; ++k) S = max(S, (uint64_t)((int64_t)a.mx[k] - (int64_t)a.o[k]) + 1);
    a.S = S;
    *acc = a;
}

// the kept points of a piece appended to the host preview (index order is piece order)
__global__ void k_preview_append(const int4* prev, const uint64_t* cnt, int4* out, uint64_t cap, const uint64_t* run,
                                 uint32_t* err)
{
    const uint64_t c = *cnt, r = *run;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (uint64_t)gridDim.x * blockDim.x) {
        if (r + i < cap) out[r + i] = prev[i];
        else if (r + i == cap) raise(err, FP_ERR_CAPACITY);
    }
}

__global__ void k_add_u64(uint64_t* run, const uint64_t* cnt) { *run += *cnt; }

// points of a piece per chunk (warp-aggregated)
__global__ void k_piece_hist(const fp_point* pts, uint64_t n, const fp_cube* cube, int g, const uint32_t* lut,
                             uint32_t* pcnt)
{
    const CubeDev c = load_cube(cube);
    const float sg = scale_at(c, g);
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        uint32_t ch = 0xFFFFFFFFu;
        if (i < n) {
            const int4 p = ld_point(pts, i);
            ch = __ldg(lut + key_small(p.x, p.y, p.z, c, sg, g));
        }
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, ch);
        if (ch != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&pcnt[ch], (uint32_t)__popc(peers));
    }
}

// a piece scattered stably by chunk: its run of chunk c lands at the chunk's cursor
// in the whole cloud's distributed order (the host store, or the device when the
// cloud stays resident)
__global__ void k_piece_scatter(const int4* dpts, const uint32_t* dperm, uint64_t n, const fp_cube* cube, int g,
                                const uint32_t* lut, const uint64_t* poff, const uint64_t* ccur, uint64_t base,
                                int4* h_pts, uint32_t* h_perm, int4* d_pts, uint32_t* d_perm, uint64_t n_all,
                                uint32_t* err)
{
    const CubeDev c = load_cube(cube);
    const float sg = scale_at(c, g);
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const int4 p = dpts[q];
        const uint32_t ch = __ldg(lut + key_small(p.x, p.y, p.z, c, sg, g));
        const uint64_t dest = ccur[ch] + (q - poff[ch]);
        if (dest >= n_all) { raise(err, FP_ERR_CAPACITY); continue; }
        if (h_pts) {
            h_pts[dest] = p;
            h_perm[dest] = (uint32_t)(base + dperm[q]);
        }
        if (d_pts) {   // the resident copy on the device
            d_pts[dest] = p;
            d_perm[dest] = (uint32_t)(base + dperm[q]);
        }
    }
}

__global__ void k_cursor_init(const uint64_t* offsets, uint32_t K, uint64_t* ccur)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) ccur[c] = offsets[c];
}

__global__ void k_cursor_advance(uint64_t* ccur, const uint32_t* pcnt, uint32_t K)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) ccur[c] += pcnt[c];
}

// the group's points per cell (0 outside), chunk of a cell relative to c0, chunk offsets relative to the group
__global__ void k_group_tables(const uint32_t* counts, const uint32_t* lut, uint64_t cells, uint32_t c0, uint32_t c1,
                               uint32_t* rcounts, uint32_t* lut_local)
{
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < cells;
         m += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t ch = lut[m];
        const bool in = ch >= c0 && ch < c1;
        rcounts[m] = in ? counts[m] : 0u;
        lut_local[m] = in ? ch - c0 : 0xFFFFFFFFu;
    }
}

__global__ void k_group_offsets(const uint64_t* offsets, uint32_t c0, uint32_t k, uint64_t* off_local, uint32_t* kdev)
{
    const uint64_t b = offsets[c0];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= k; i += gridDim.x * blockDim.x)
        off_local[i] = offsets[c0 + i] - b;
    if (blockIdx.x == 0 && threadIdx.x == 0) *kdev = k;
}

__global__ void k_owner_keys(const uint32_t* owner, uint64_t n, uint64_t* key)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        key[i] = owner[i];
}

// first position of every key run of a sorted array: soff[key >> shift] = t
__global__ void k_run_starts(const uint64_t* key, uint64_t S, int shift, uint32_t* soff, uint32_t cap)
{
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < S; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t X = key[t] >> shift;
        if ((t == 0 || (key[t - 1] >> shift) != X) && X < cap) soff[X] = (uint32_t)t;
    }
}

// A group's points sorted by owner: points of nodes inside the group's chunks go
// to their final positions (index order inside an owner is the distributed
// order); points of nodes above the chunks are staged with key (owner, index)
// and their position in the store of group points.
__global__ void k_group_place(const uint64_t* key, const uint32_t* src, uint64_t n, const uint32_t* soff,
                              const fp_node* nodes, uint32_t M, uint64_t T, int g, const uint64_t* first,
                              const int4* pts, const uint32_t* perm, uint64_t group_base, int4* h_final,
                              uint32_t* h_final_perm, uint64_t n_all, uint64_t* h_st_key, uint32_t* h_st_src,
                              int4* h_st_pt, uint64_t* st_run, uint64_t st_cap, int pbits, uint32_t* err)
{
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t X = (uint32_t)key[t];
        const uint32_t j = src[t];
        if (X >= M) { raise(err, FP_ERR_CAPACITY); continue; }
        const bool above = nodes[X].count > T && (int)nodes[X].level < g;
        if (!above) {
            const uint64_t f = first[X] + (t - soff[X]);
            if (f >= n_all) { raise(err, FP_ERR_CAPACITY); continue; }
            h_final[f] = pts[j];
            h_final_perm[f] = perm[j];
        } else {
            const uint64_t o = atomicAdd((unsigned long long*)st_run, 1ull);
            if (o >= st_cap) { raise(err, FP_ERR_CAPACITY); continue; }
            h_st_key[o] = ((uint64_t)X << pbits) | perm[j];
            h_st_src[o] = (uint32_t)(group_base + j);
            if (h_st_pt) h_st_pt[o] = pts[j];   // the point itself (no host store of the cloud)
        }
    }
}

// staged records sorted by (owner, index): position first[owner] + rank.  The
// point comes from the host store, or (staged_pts) from its staged copy, the
// index from the key.
__global__ void k_stitch_final(const uint64_t* key, const uint32_t* val, uint64_t S, int pbits, const uint32_t* soff,
                               const uint64_t* first, const uint32_t* h_st_src, const int4* h_pts,
                               const uint32_t* h_perm, int staged_pts, int4* h_final, uint32_t* h_final_perm,
                               uint64_t n_all, uint32_t M, uint32_t* err)
{
    const uint64_t imask = (1ull << pbits) - 1;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < S; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t X = key[t] >> pbits;
        if (X >= M) { raise(err, FP_ERR_CAPACITY); continue; }
        const uint64_t f = first[X] + (t - soff[X]);
        const uint32_t j = staged_pts ? val[t] : h_st_src[val[t]];
        if (f >= n_all || j >= n_all) { raise(err, FP_ERR_CAPACITY); continue; }
        h_final[f] = h_pts[j];
        h_final_perm[f] = staged_pts ? (uint32_t)(key[t] & imask) : h_perm[j];
    }
}

// ------------------------------------------------------------------ layout
struct HostStore {
    int4* pts;          // n: the distributed points, group after group
    uint32_t* perm;     // n: their original indices
    uint32_t* codes;    // n: owner level, leaf level, level-g cell (code_make)
    uint32_t* owner;    // n: owner id
    uint64_t* st_key;   // n: staged (owner, index)
    uint32_t* st_src;   // n: staged record's position in pts
};

HostStore host_carve(void* base, uint64_t n)
{
    Workspace w;
    w.base = static_cast<char*>(base);
    const uint64_t N = n ? n : 1;
    HostStore h;
    h.pts = w.take<int4>(N);
    h.perm = w.take<uint32_t>(N);
    h.codes = w.take<uint32_t>(N);
    h.owner = w.take<uint32_t>(N);
    h.st_key = w.take<uint64_t>(N);
    h.st_src = w.take<uint32_t>(N);
    return h;
}

size_t host_bytes(uint64_t n)
{   // the pieces host_carve takes, in its order
    const uint64_t N = n ? n : 1;
    return Workspace::bytes_for({16 * N, 4 * N, 4 * N, 4 * N, 8 * N, 4 * N});
}

uint64_t preview_piece_cap(uint64_t p, uint32_t m)
{   // a sum of p Bernoulli(1/m) draws: far below this bound
    if (m <= 2) return p;
    uint64_t mean = p / m;
    uint64_t sd = 1;
    while (sd * sd < mean) ++sd;
    return std::min<uint64_t>(p, mean + 64 + 32 * sd);
}

struct Fixed {   // device buffers kept for the whole build
    fp_cube *cube, *piece_cube;
    uint32_t *counts, *lut, *num_chunks;
    fp_chunk* chunks;
    uint64_t *offsets, *prev_run, *prev_cnt, *st_run;
    int4* piece[2];
    int4* prev_buf;
    int4* dpiece;        // a piece scattered by chunk
    uint32_t *dperm, *pcnt;
    uint64_t *poff, *ccur;
    NodeRec* recs;
    fp_node* nodes;
    uint32_t *num_deep, *num_nodes, *nm, *soff;
    uint64_t *first, *tiles64;
    NodeTables T;
    uint32_t *rcounts, *lut_local, *kdev;
    uint64_t* off_local;
};

Fixed fixed_carve(const Workspace& w, uint64_t P, const fp_params& p, uint64_t node_cap, int num_sms)
{
    Fixed F;
    const uint64_t cells = 1ull << (3 * p.grid_log2);
    F.cube = w.take<fp_cube>(1);
    F.piece_cube = w.take<fp_cube>(1);
    F.counts = w.take<uint32_t>(cells);
    F.lut = w.take<uint32_t>(cells);
    F.num_chunks = w.take<uint32_t>(1);
    F.chunks = w.take<fp_chunk>(cells);
    F.offsets = w.take<uint64_t>(cells + 1);
    F.prev_run = w.take<uint64_t>(1);
    F.prev_cnt = w.take<uint64_t>(1);
    F.st_run = w.take<uint64_t>(1);
    F.piece[0] = w.take<int4>(P);
    F.piece[1] = w.take<int4>(P);
    F.prev_buf = w.take<int4>(preview_piece_cap(P, p.decim_modulus) + 1);
    F.dpiece = w.take<int4>(P);
    F.dperm = w.take<uint32_t>(P);
    F.pcnt = w.take<uint32_t>(cells);
    F.poff = w.take<uint64_t>(cells + 1);
    F.ccur = w.take<uint64_t>(cells);
    F.recs = reinterpret_cast<NodeRec*>(w.take<unsigned char>(kNodeRecBytes * node_cap));
    F.nodes = w.take<fp_node>(node_cap);
    F.num_deep = w.take<uint32_t>(1);
    F.num_nodes = w.take<uint32_t>(1);
    F.nm = w.take<uint32_t>(1);
    F.soff = w.take<uint32_t>(node_cap);
    F.first = w.take<uint64_t>(node_cap + 1);
    F.tiles64 = w.take<uint64_t>(kScanMaxTiles);
    F.T.idxtab = w.take<uint32_t>(cells * 8 / 7 + 8);
    F.T.starts = w.take<uint64_t>(node_cap);
    F.T.slevel = w.take<uint8_t>(node_cap);
    F.T.ndesc = w.take<uint32_t>(node_cap);
    F.T.nown = w.take<uint32_t>(node_cap);
    F.T.nnode = w.take<uint32_t>(1);
    F.rcounts = w.take<uint32_t>(cells);
    F.lut_local = w.take<uint32_t>(cells);
    F.kdev = w.take<uint32_t>(1);
    F.off_local = w.take<uint64_t>(cells + 1);
    (void)num_sms;
    return F;
}

struct Group {   // device buffers of one chunk group (G points), reused group after group
    char* region;   // the start of the group region
    int4* pts;
    uint32_t *perm, *owner;
    uint32_t* codes;
    uint64_t *key, *key2, *key3;
    uint32_t *val2, *val3;
    char* ws;      // stage workspace
    size_t ws_bytes;
};

size_t stage_ws(uint64_t G, uint64_t P, const fp_params& p, uint64_t node_cap, int num_sms)
{
    size_t w = std::max(distribute_ws_bytes(P, (int)p.grid_log2), octree_ws_bytes(G, p));
    w = std::max(w, bounds_ws_bytes(P, num_sms));
    w = std::max(w, merge_ws_bytes((int)p.grid_log2));
    w = std::max(w, nodes_ws_bytes(p, node_cap));
    w = std::max(w, sort_scratch_bytes(G));
    return w;
}

// resident: the group's points and indices are a slice of the resident
// distributed cloud (set per group), not carved here
Group group_carve(const Workspace& w, uint64_t G, uint64_t P, const fp_params& p, uint64_t node_cap, int num_sms,
                  bool resident = false)
{
    Group g;
    const uint64_t N = G ? G : 1;
    g.region = w.base + w.used;
    g.pts = resident ? nullptr : w.take<int4>(N);
    g.perm = resident ? nullptr : w.take<uint32_t>(N);
    g.owner = w.take<uint32_t>(N);
    g.codes = w.take<uint32_t>(N);
    g.key = w.take<uint64_t>(N);
    g.key2 = w.take<uint64_t>(N);
    g.key3 = w.take<uint64_t>(N);
    g.val2 = w.take<uint32_t>(N);
    g.val3 = w.take<uint32_t>(N);
    g.ws_bytes = stage_ws(G, P, p, node_cap, num_sms);
    g.ws = w.take<char>(g.ws_bytes);
    return g;
}

size_t fixed_bytes(uint64_t P, const fp_params& p, uint64_t node_cap)
{
    Workspace dry;
    fixed_carve(dry, P, p, node_cap, 152);
    return dry.used;
}

size_t group_bytes(uint64_t G, uint64_t P, const fp_params& p, uint64_t node_cap, int num_sms, bool resident = false)
{
    Workspace dry;
    group_carve(dry, G, P, p, node_cap, num_sms, resident);
    return dry.used;
}

// the distributed cloud and its original indices kept in the arena
size_t resident_bytes(uint64_t n) { return Workspace::bytes_for({16 * (n ? n : 1), 4 * (n ? n : 1)}); }

// the largest group (points) that fits next to the fixed buffers (and the
// resident cloud)
uint64_t group_cap_for(size_t arena, uint64_t n, uint64_t P, const fp_params& p, uint64_t node_cap, int num_sms,
                       bool resident = false)
{
    const size_t fixed = fixed_bytes(P, p, node_cap) + (resident ? resident_bytes(n) : 0);
    if (arena <= fixed) return 0;
    uint64_t lo = 0, hi = std::max<uint64_t>(n, 1);
    while (lo < hi) {
        const uint64_t mid = (lo + hi + 1) / 2;
        if (fixed + group_bytes(mid, P, p, node_cap, num_sms, resident) <= arena) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct Piecer {   // double-buffered host -> device copies of the pieces on a side stream
    cudaStream_t cs = nullptr, st = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    const fp_point* h = nullptr;
    uint64_t n = 0, P = 0;
    int4* buf[2] = {nullptr, nullptr};
    int4* raw = nullptr;   // set: piece k lands at raw + k P (a device copy of the whole cloud)

    cudaError_t init(cudaStream_t stream, const fp_point* hp, uint64_t nn, uint64_t pp, int4* b0, int4* b1)
    {
        st = stream; h = hp; n = nn; P = pp; buf[0] = b0; buf[1] = b1;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && !e; ++b) {
            if ((e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming))) break;
            e = cudaEventCreateWithFlags(&consumed[b], cudaEventDisableTiming);
            if (!e) e = cudaEventRecord(consumed[b], st);
        }
        return e;
    }
    uint64_t pieces() const { return (n + P - 1) / P; }
    int4* dst(uint64_t k) const { return raw ? raw + k * P : buf[k & 1]; }
    uint64_t size(uint64_t k) const { return std::min(P, n - k * P); }
    // enqueue the copy of piece k (after the work that read its buffer), compute stream waits for it
    cudaError_t fetch(uint64_t k)
    {
        const int b = (int)(k & 1);
        cudaError_t e;
        if ((e = cudaStreamWaitEvent(cs, consumed[b], 0))) return e;
        if ((e = cudaMemcpyAsync(dst(k), h + k * P, size(k) * sizeof(fp_point), cudaMemcpyHostToDevice, cs))) return e;
        if ((e = cudaEventRecord(copied[b], cs))) return e;
        return cudaStreamWaitEvent(st, copied[b], 0);
    }
    cudaError_t done(uint64_t k) { return cudaEventRecord(consumed[k & 1], st); }
    // a pass over the device copy made by an earlier pass (raw set): no copies
    template <typename F>
    cudaError_t pass_raw(F body)
    {
        cudaError_t e;
        for (uint64_t k = 0; k < pieces(); ++k)
            if ((e = body(k, reinterpret_cast<const fp_point*>(raw + k * P), size(k)))) return e;
        return cudaSuccess;
    }
    // pass over all pieces: body(k, device pointer, size) enqueues the work on st
    template <typename F>
    cudaError_t pass(F body)
    {
        const uint64_t np = pieces();
        cudaError_t e;
        if (np && (e = fetch(0))) return e;
        for (uint64_t k = 0; k < np; ++k) {
            if (k + 1 < np && (e = fetch(k + 1))) return e;   // the next copy overlaps this piece's work
            if ((e = body(k, reinterpret_cast<const fp_point*>(dst(k)), size(k)))) return e;
            if ((e = done(k))) return e;
        }
        return cudaSuccess;
    }
    void release()
    {
        if (cs) cudaStreamSynchronize(cs);
        for (int b = 0; b < 2; ++b) {
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (consumed[b]) cudaEventDestroy(consumed[b]);
        }
        if (cs) cudaStreamDestroy(cs);
    }
};

fp_status cu(cudaError_t e) { return e == cudaSuccess ? FP_OK : FP_ERR_CUDA; }

inline unsigned grid_for(uint64_t n, int num_sms) { return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms * 16)); }

fp_status build(const fp_point* h_pts, uint64_t n, const fp_params& prm, uint64_t P, uint64_t group_points,
                void* d_arena, size_t arena_bytes,
                void* h_scratch, fp_cube* h_cube, fp_point* h_preview, uint64_t preview_cap,
                uint64_t* h_preview_count, fp_node* h_nodes, uint32_t node_cap, uint32_t* h_num_nodes,
                fp_point* h_final, uint32_t* h_final_perm, void (*preview_done)(void*), void* user, cudaStream_t st,
                Piecer& io)
{
    Workspace base;
    fp_status s = make_workspace(d_arena, arena_bytes, 0, base);
    if (s != FP_OK) return s;
    const int g = (int)prm.grid_log2;
    const uint64_t cells = 1ull << (3 * g);
    uint64_t G = group_cap_for(arena_bytes, n, P, prm, node_cap, base.num_sms);
    if (group_points) G = std::min(G, group_points);
    if (G == 0) return FP_ERR_WORKSPACE;
    Workspace w = base;
    const Fixed F = fixed_carve(w, P, prm, node_cap, base.num_sms);
    const size_t after_fixed = w.used;
    Group B = group_carve(w, G, P, prm, node_cap, base.num_sms);
    Workspace ws = base;   // stage workspace view
    ws.base = B.ws;
    ws.bytes = B.ws_bytes;
    ws.used = 0;
    const HostStore H = host_carve(h_scratch, n);
    cudaError_t e;
    if ((e = io.init(st, h_pts, n, P, F.piece[0], F.piece[1]))) return FP_ERR_CUDA;
    // When the arena also holds a copy of the raw cloud behind the space of the
    // resident distributed cloud (16 + 20 bytes per point, and the passes'
    // stage workspace after them), pass 1 copies every piece there and passes 2
    // and 3 read it on the device instead of crossing the link again.
    int4* raw = nullptr;
    {
        const size_t ws13 = std::max({bounds_ws_bytes(P, base.num_sms), merge_ws_bytes(g),
                                      distribute_ws_bytes(P, g)});
        const size_t raw_bytes = Workspace::bytes_for({16 * (n ? n : 1)});
        if (after_fixed + resident_bytes(n) + raw_bytes + ws13 <= arena_bytes) {
            Workspace wr = base;
            wr.used = after_fixed + resident_bytes(n);
            raw = wr.take<int4>(n ? n : 1);
            ws.base = base.base + wr.used;
            ws.bytes = ws13;
            ws.used = 0;
            io.raw = raw;
        }
    }

    // ---- pass 1: bounds and preview
    if ((e = cudaMemsetAsync(F.prev_run, 0, sizeof(uint64_t), st))) return cu(e);
    const uint64_t pcap = preview_piece_cap(P, prm.decim_modulus);
    e = io.pass([&](uint64_t k, const fp_point* p, uint64_t np) -> cudaError_t {
        ws.used = 0;
        cudaError_t x = launch_bounds_decimate(p, np, F.piece_cube, true, true, k * P, prm.decim_modulus,
                                               reinterpret_cast<fp_point*>(F.prev_buf), pcap, F.prev_cnt, ws, st);
        if (x) return x;
        k_cube_fold<<<1, 1, 0, st>>>(F.cube, F.piece_cube, k == 0);
        k_preview_append<<<grid_for(pcap, ws.num_sms), 256, 0, st>>>(F.prev_buf, F.prev_cnt,
                                                                     reinterpret_cast<int4*>(h_preview), preview_cap,
                                                                     F.prev_run, base.err);
        k_add_u64<<<1, 1, 0, st>>>(F.prev_run, F.prev_cnt);
        return cudaGetLastError();
    });
    if (e) return cu(e);
    if ((e = cudaMemcpyAsync(h_cube, F.cube, sizeof(fp_cube), cudaMemcpyDeviceToHost, st))) return cu(e);
    if ((e = cudaMemcpyAsync(h_preview_count, F.prev_run, sizeof(uint64_t), cudaMemcpyDeviceToHost, st))) return cu(e);
    if (preview_done && (e = cudaLaunchHostFunc(st, preview_done, user))) return cu(e);

    // ---- pass 2: counts; chunks
    auto count_piece = [&](uint64_t k, const fp_point* p, uint64_t np) -> cudaError_t {
        ws.used = 0;
        return launch_count(p, np, F.cube, g, F.counts, k > 0, nullptr, ws, st);
    };
    e = raw ? io.pass_raw(count_piece) : io.pass(count_piece);
    if (e) return cu(e);
    ws.used = 0;
    if ((e = launch_merge(F.counts, g, prm.chunk_threshold, F.chunks, F.num_chunks, F.lut, F.offsets, ws, st)))
        return cu(e);
    uint32_t K = 0;
    if ((e = cudaMemcpyAsync(&K, F.num_chunks, sizeof(K), cudaMemcpyDeviceToHost, st))) return cu(e);
    if ((e = cudaStreamSynchronize(st))) return cu(e);
    std::vector<uint64_t> off(K + 1);
    if ((e = cudaMemcpyAsync(off.data(), F.offsets, (K + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st)))
        return cu(e);
    if ((e = cudaStreamSynchronize(st))) return cu(e);
    if (off[K] != n) return FP_ERR_INVALID;
    // When the arena holds the distributed cloud (points and indices) next to the
    // fixed buffers and a group as large as the largest chunk, the cloud stays
    // on the device after pass 3: the group passes read it in place instead of
    // copying it back from the host store three times.
    uint64_t biggest = 0;
    for (uint32_t c = 0; c < K; ++c) biggest = std::max(biggest, off[c + 1] - off[c]);
    int4* res_pts = nullptr;
    uint32_t* res_perm = nullptr;
    {
        uint64_t Gr = group_cap_for(arena_bytes, n, P, prm, node_cap, base.num_sms, true);
        if (group_points) Gr = std::min(Gr, group_points);
        if (Gr >= biggest && Gr > 0) {
            Workspace wr = base;
            wr.used = after_fixed;
            res_pts = wr.take<int4>(n ? n : 1);
            res_perm = wr.take<uint32_t>(n ? n : 1);
            G = Gr;
            B = group_carve(wr, G, P, prm, node_cap, base.num_sms, true);
        }
    }
    const bool resident = res_pts != nullptr;
    if (raw && !resident) {   // the non-resident group region covers the raw copy: pass 3 streams again
        raw = nullptr;
        io.raw = nullptr;
    }
    if (!raw) {   // pass 3's stage workspace: the group's (the raw copy keeps its own until pass 3 is done)
        ws.base = B.ws;
        ws.bytes = B.ws_bytes;
        ws.used = 0;
    }

    // consecutive chunks while they fit a group
    std::vector<std::pair<uint32_t, uint32_t>> groups;
    for (uint32_t c0 = 0; c0 < K;) {
        uint32_t c1 = c0 + 1;
        if (off[c1] - off[c0] > G) return FP_ERR_WORKSPACE;   // one chunk larger than the arena allows
        while (c1 < K && off[c1 + 1] - off[c0] <= G) ++c1;
        groups.push_back({c0, c1});
        c0 = c1;
    }

    // ---- pass 3: the whole cloud in distributed order into the host store.  Each
    // piece is scattered stably by chunk on the device; its run of every chunk
    // lands after the earlier pieces' points of that chunk (a cursor per chunk).
    const unsigned gK = grid_for(K, base.num_sms);
    k_cursor_init<<<gK, 256, 0, st>>>(F.offsets, K, F.ccur);
    auto distribute_piece = [&](uint64_t k, const fp_point* p, uint64_t np) -> cudaError_t {
        cudaError_t x;
        if ((x = cudaMemsetAsync(F.pcnt, 0, (size_t)K * sizeof(uint32_t), st))) return x;
        k_piece_hist<<<grid_for(np, base.num_sms), 256, 0, st>>>(p, np, F.cube, g, F.lut, F.pcnt);
        if ((x = scan_exclusive<uint32_t, uint64_t>(F.pcnt, F.poff, K, nullptr, F.tiles64, F.poff + K,
                                                    (uint64_t*)nullptr, st)))
            return x;
        ws.used = 0;
        if ((x = launch_distribute(p, np, F.cube, g, F.lut, F.poff, F.num_chunks, reinterpret_cast<fp_point*>(F.dpiece),
                                   F.dperm, ws, st)))
            return x;
        k_piece_scatter<<<grid_for(np, base.num_sms), 256, 0, st>>>(F.dpiece, F.dperm, np, F.cube, g, F.lut, F.poff,
                                                                    F.ccur, k * P, resident ? nullptr : H.pts,
                                                                    resident ? nullptr : H.perm, res_pts, res_perm, n,
                                                                    base.err);
        k_cursor_advance<<<gK, 256, 0, st>>>(F.ccur, F.pcnt, K);
        return cudaGetLastError();
    };
    e = raw ? io.pass_raw(distribute_piece) : io.pass(distribute_piece);
    if (e) return cu(e);
    ws.base = B.ws;   // the raw copy is dead from here on
    ws.bytes = B.ws_bytes;
    ws.used = 0;

    // ---- per group: its points from the store; levels and nodes below level g
    if ((e = cudaMemsetAsync(F.num_deep, 0, sizeof(uint32_t), st))) return cu(e);
    const unsigned gc = grid_for(cells, base.num_sms);
    for (auto [c0, c1] : groups) {
        const uint64_t b0 = off[c0], ng = off[c1] - off[c0];
        k_group_tables<<<gc, 256, 0, st>>>(F.counts, F.lut, cells, c0, c1, F.rcounts, F.lut_local);
        k_group_offsets<<<gc, 256, 0, st>>>(F.offsets, c0, c1 - c0, F.off_local, F.kdev);
        if (resident) {
            B.pts = res_pts + b0;
            B.perm = res_perm + b0;
        } else {
            if ((e = cudaMemcpyAsync(B.pts, H.pts + b0, ng * 16, cudaMemcpyHostToDevice, st))) return cu(e);
            if ((e = cudaMemcpyAsync(B.perm, H.perm + b0, ng * 4, cudaMemcpyHostToDevice, st))) return cu(e);
        }
        OctGroup grp{F.rcounts, (uint32_t)b0, B.codes, F.recs, node_cap, F.num_deep};
        ws.used = 0;
        if ((e = launch_octree_impl(reinterpret_cast<const fp_point*>(B.pts), B.perm, ng, F.cube, F.chunks + c0,
                                    F.kdev, F.off_local, F.counts, prm, nullptr, 0, nullptr, nullptr, nullptr,
                                    nullptr, &grp, ws, st)))
            return cu(e);
        if ((e = cudaMemcpyAsync(H.codes + b0, B.codes, ng * 4, cudaMemcpyDeviceToHost, st))) return cu(e);
    }

    // ---- node table of the whole cloud
    ws.used = 0;
    if ((e = launch_octree_nodes(F.counts, prm, F.recs, node_cap, F.num_deep, F.nodes, node_cap, F.num_nodes, F.T, ws,
                                 st)))
        return cu(e);

    // ---- pass 4 per group: owner ids, owned counts
    for (auto [c0, c1] : groups) {
        const uint64_t b0 = off[c0], ng = off[c1] - off[c0];
        if (resident) B.pts = res_pts + b0;
        else if ((e = cudaMemcpyAsync(B.pts, H.pts + b0, ng * 16, cudaMemcpyHostToDevice, st))) return cu(e);
        if ((e = cudaMemcpyAsync(B.codes, H.codes + b0, ng * 4, cudaMemcpyHostToDevice, st))) return cu(e);
        if ((e = launch_octree_resolve(reinterpret_cast<const fp_point*>(B.pts), ng, F.cube, B.codes, F.T, prm,
                                       B.owner, ws, st)))
            return cu(e);
        if ((e = cudaMemcpyAsync(H.owner + b0, B.owner, ng * 4, cudaMemcpyDeviceToHost, st))) return cu(e);
    }
    if ((e = launch_node_first(F.nodes, F.num_nodes, node_cap, F.T.nown, F.first, F.nm, F.tiles64, st))) return cu(e);
    uint32_t M = 0;
    if ((e = cudaMemcpyAsync(&M, F.num_nodes, sizeof(M), cudaMemcpyDeviceToHost, st))) return cu(e);
    if ((e = cudaStreamSynchronize(st))) return cu(e);
    if (M > node_cap) return FP_ERR_INVALID;
    int pbits = 1;
    while ((1ull << pbits) < n) ++pbits;
    int mbits = 1;
    while ((1ull << mbits) < M) ++mbits;

    // ---- pass 5 per group: final positions of points kept inside the chunks; the rest staged
    if ((e = cudaMemsetAsync(F.st_run, 0, sizeof(uint64_t), st))) return cu(e);
    ws.used = 0;
    const SortScratch sc = take_sort_scratch(ws, G);
    const size_t ws_after_sc = ws.used;
    for (auto [c0, c1] : groups) {
        const uint64_t b0 = off[c0], ng = off[c1] - off[c0];
        if (resident) {
            B.pts = res_pts + b0;
            B.perm = res_perm + b0;
        } else {
            if ((e = cudaMemcpyAsync(B.pts, H.pts + b0, ng * 16, cudaMemcpyHostToDevice, st))) return cu(e);
            if ((e = cudaMemcpyAsync(B.perm, H.perm + b0, ng * 4, cudaMemcpyHostToDevice, st))) return cu(e);
        }
        if ((e = cudaMemcpyAsync(B.owner, H.owner + b0, ng * 4, cudaMemcpyHostToDevice, st))) return cu(e);
        k_owner_keys<<<grid_for(ng, base.num_sms), 256, 0, st>>>(B.owner, ng, B.key);
        ws.used = ws_after_sc;
        if ((e = sort_plan_keys(sc, B.key, ng, nullptr, 0, (uint32_t)mbits, st))) return cu(e);
        SortArgs a{};
        a.b.k64_src = B.key; a.b.k64_tmp = B.key2; a.b.k64_dst = B.key3;
        a.b.val_src = nullptr; a.b.val_tmp = B.val2; a.b.val_dst = B.val3;
        a.n = ng; a.err = base.err;
        for (int slot = 0; slot < sort_passes(mbits); ++slot)
            if ((e = sort_run_pass<DIG_K64, false, true, false>(sc, a, slot, base.num_sms, st))) return cu(e);
        k_run_starts<<<grid_for(ng, base.num_sms), 256, 0, st>>>(B.key3, ng, 0, F.soff, M);
        k_group_place<<<grid_for(ng, base.num_sms), 256, 0, st>>>(
            B.key3, B.val3, ng, F.soff, F.nodes, M, prm.chunk_threshold, g, F.first, B.pts, B.perm, b0,
            reinterpret_cast<int4*>(h_final), h_final_perm, n, H.st_key, H.st_src, resident ? H.pts : nullptr,
            F.st_run, n, pbits, base.err);
        if ((e = cudaGetLastError())) return cu(e);
    }

    // ---- the staged points: sorted by (owner, index), placed after their owners' earlier points
    uint64_t S = 0;
    if ((e = cudaMemcpyAsync(&S, F.st_run, sizeof(S), cudaMemcpyDeviceToHost, st))) return cu(e);
    if ((e = cudaStreamSynchronize(st))) return cu(e);
    if (S) {   // the sort of the staged records reuses the whole group region
        Workspace wf = base;
        // (the resident cloud is dead by now: the staged points were copied out with their records)
        wf.base = resident ? reinterpret_cast<char*>(res_pts) : B.region;
        wf.bytes = group_bytes(G, P, prm, node_cap, base.num_sms, resident) + (resident ? resident_bytes(n) : 0);
        wf.used = 0;
        uint64_t* k1 = wf.take<uint64_t>(S);
        uint64_t* k2 = wf.take<uint64_t>(S);
        uint64_t* k3 = wf.take<uint64_t>(S);
        uint32_t* v2 = wf.take<uint32_t>(S);
        uint32_t* v3 = wf.take<uint32_t>(S);
        const SortScratch sf = take_sort_scratch(wf, S);
        if (wf.used > wf.bytes) return FP_ERR_WORKSPACE;
        if ((e = cudaMemcpyAsync(k1, H.st_key, S * 8, cudaMemcpyHostToDevice, st))) return cu(e);
        if ((e = sort_plan_keys(sf, k1, S, nullptr, 0, (uint32_t)(pbits + mbits), st))) return cu(e);
        SortArgs a{};
        a.b.k64_src = k1; a.b.k64_tmp = k2; a.b.k64_dst = k3;
        a.b.val_src = nullptr; a.b.val_tmp = v2; a.b.val_dst = v3;
        a.n = S; a.err = base.err;
        for (int slot = 0; slot < sort_passes(pbits + mbits); ++slot)
            if ((e = sort_run_pass<DIG_K64, false, true, false>(sf, a, slot, base.num_sms, st))) return cu(e);
        k_run_starts<<<grid_for(S, base.num_sms), 256, 0, st>>>(k3, S, pbits, F.soff, M);
        k_stitch_final<<<grid_for(S, base.num_sms), 256, 0, st>>>(k3, v3, S, pbits, F.soff, F.first, H.st_src, H.pts,
                                                                  H.perm, resident ? 1 : 0,
                                                                  reinterpret_cast<int4*>(h_final),
                                                                  h_final_perm, n, M, base.err);
        if ((e = cudaGetLastError())) return cu(e);
    }
    if ((e = cudaMemcpyAsync(h_nodes, F.nodes, (size_t)M * sizeof(fp_node), cudaMemcpyDeviceToHost, st))) return cu(e);
    if ((e = cudaMemcpyAsync(h_num_nodes, F.num_nodes, sizeof(uint32_t), cudaMemcpyDeviceToHost, st))) return cu(e);
    return cu(cudaStreamSynchronize(st));
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

size_t fp_ooc_host_bytes(uint64_t n, const fp_params* prm)
{
    if (!prm || check_params(prm) != FP_OK) return 0;
    return host_bytes(n);
}

size_t fp_ooc_arena_min(uint64_t n, const fp_params* prm, uint64_t piece_points)
{
    if (!prm || check_params(prm) != FP_OK) return 0;
    const uint64_t P = piece_points ? std::min(piece_points, kMaxPiece) : kMaxPiece;
    const uint64_t ncap = node_capacity_bound(n, *prm);
    // the fixed buffers and a group of 2^20 points (or the whole cloud)
    return fixed_bytes(P, *prm, ncap) + group_bytes(std::min<uint64_t>(std::max<uint64_t>(n, 1), 1ull << 20), P, *prm,
                                                    ncap, 152);
}

fp_status fp_build_ooc(const fp_point* h_pts, uint64_t n, const fp_params* h_prm, uint64_t piece_points,
                       uint64_t group_points, void* d_arena, size_t arena_bytes, void* h_scratch,
                       size_t scratch_bytes, fp_cube* h_cube,
                       fp_point* h_preview, uint64_t preview_cap, uint64_t* h_preview_count, fp_node* h_nodes,
                       uint32_t node_cap, uint32_t* h_num_nodes, fp_point* h_final, uint32_t* h_final_perm,
                       void (*preview_done)(void*), void* user, cudaStream_t stream)
{
    fp_status s = check_params(h_prm);
    if (s != FP_OK) return s;
    if (n == 0 || !h_pts || !d_arena || !h_scratch || !h_cube || !h_preview_count || !h_nodes || !h_num_nodes ||
        !h_final || !h_final_perm || (preview_cap && !h_preview))
        return FP_ERR_INVALID;
    if (n >= (1ull << 30)) return FP_ERR_TOO_LARGE;
    if ((reinterpret_cast<uintptr_t>(h_pts) | reinterpret_cast<uintptr_t>(h_final) |
         reinterpret_cast<uintptr_t>(h_preview) | reinterpret_cast<uintptr_t>(d_arena) |
         reinterpret_cast<uintptr_t>(h_scratch)) & 15u)
        return FP_ERR_ALIGN;
    if (scratch_bytes < host_bytes(n)) return FP_ERR_WORKSPACE;
    if (node_cap < node_capacity_bound(n, *h_prm) || node_cap > (1u << 23)) return FP_ERR_UNSUPPORTED;
    const uint64_t P = piece_points ? std::min(piece_points, kMaxPiece) : kMaxPiece;
    Piecer io;
    s = build(h_pts, n, *h_prm, P, group_points, d_arena, arena_bytes, h_scratch, h_cube, h_preview, preview_cap, h_preview_count,
              h_nodes, node_cap, h_num_nodes, h_final, h_final_perm, preview_done, user, stream, io);
    io.release();
    // nothing of the build may still run once the caller gets the arena back
    if (cudaStreamSynchronize(stream) != cudaSuccess && s == FP_OK) s = FP_ERR_CUDA;
    return s;
}

}  // extern "C"
