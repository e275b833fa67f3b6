// fp_sort.cu -- plans of the stable bucket-scatter passes and fp_distribute.
//
// fp_distribute (Sec. 4.4: the cloud is "sorted into a number of chunks", each
// a node of the global tree, Fig. "octree") is a stable scatter of the points by
// chunk id.  The bucket of every point is looked up from its level-g cell
// (lut); the bucket bases are the chunk offsets, so with at most 1024 chunks a
// single pass reads each point once and writes it once.  More chunks take two
// or three least-significant-digit-first passes, chosen on the device.
#include "fp_seg.cuh"

namespace fp {

// Passes and digit width for a key of `need` bits (at most 64): the fewest
// passes of at most 8 bits, the bits spread evenly over them.
FP_DEV void plan_shape(uint64_t nw, uint32_t fixed_bits, uint32_t& npass, uint32_t& bits)
{
    uint32_t need = fixed_bits;
    if (!need) {
        need = 1;
        while (need < 64 && (nw - 1) >> need) ++need;
        if (nw <= 1) need = 1;
    }
    if (need > 64) need = 64;
    npass = (need + kSortMaxBits - 1) / kSortMaxBits;
    if (npass < 1) npass = 1;
    bits = (need + npass - 1) / npass;
    if (bits < 1) bits = 1;
}

// bits of the largest value below *d (at least 1)
FP_DEV uint32_t bits_of_count(uint32_t v)
{
    uint32_t b = 1;
    while (b < 32 && ((v ? v - 1 : 0) >> b)) ++b;
    return b;
}

__global__ void k_sort_zero(uint32_t* status, uint32_t* counter, uint64_t n, const uint32_t* d_n, const SortPlan* plan,
                            int slot)
{   // n is the record bound of the pass: zeroing every tile it may use is a superset
    if (slot >= (int)plan->npass) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    if (d_n && *d_n < n) n = *d_n;
    uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint64_t words = ntiles << plan->bits;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint4* s4 = reinterpret_cast<uint4*>(status);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words / 4; i += stride)
        s4[i] = make_uint4(0, 0, 0, 0);
    for (uint64_t i = words / 4 * 4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride)
        status[i] = 0;
}

__global__ void k_plan_hist_weights(const uint32_t* weights, const uint64_t* offsets, const uint32_t* d_nw,
                                    uint64_t nw_max, uint32_t* hist)
{
    __shared__ uint32_t sh[kSortMaxPass << kSortMaxBits];
    uint64_t nw = d_nw ? *d_nw : nw_max;
    uint32_t npass, bits;
    plan_shape(nw, 0, npass, bits);
    const uint32_t mask = (1u << bits) - 1;
    for (int q = threadIdx.x; q < (kSortMaxPass << kSortMaxBits); q += blockDim.x) sh[q] = 0;
    __syncthreads();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; id < nw; id += stride) {
        uint32_t w = weights ? weights[id] : (uint32_t)(offsets[id + 1] - offsets[id]);
        if (!w) continue;
        for (uint32_t k = 0; k < npass; ++k)
            atomicAdd(&sh[(k << kSortMaxBits) + ((id >> (k * bits)) & mask)], w);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (kSortMaxPass << kSortMaxBits); q += blockDim.x)
        if (sh[q]) atomicAdd(&hist[q], sh[q]);
}

__global__ void k_plan_hist_keys(const uint64_t* keys, uint64_t n, const uint32_t* d_n, uint32_t shift0,
                                 uint32_t total_bits, uint32_t* hist, const uint32_t* d_rank_n)
{
    if (d_n && *d_n < n) n = *d_n;
    if (d_rank_n) total_bits += bits_of_count(*d_rank_n);
    __shared__ uint32_t sh[kSortMaxPass << kSortMaxBits];
    uint32_t npass, bits;
    plan_shape(0, total_bits, npass, bits);
    const uint32_t mask = (1u << bits) - 1;
    for (int q = threadIdx.x; q < (kSortMaxPass << kSortMaxBits); q += blockDim.x) sh[q] = 0;
    __syncthreads();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t k = keys[i] >> shift0;
        for (uint32_t p = 0; p < npass; ++p) atomicAdd(&sh[(p << kSortMaxBits) + ((k >> (p * bits)) & mask)], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (kSortMaxPass << kSortMaxBits); q += blockDim.x)
        if (sh[q]) atomicAdd(&hist[q], sh[q]);
}

__global__ void __launch_bounds__(1024) k_plan_finalize(const uint32_t* d_nw, uint64_t nw_max, uint32_t fixed_bits,
                                                        uint32_t shift0, const uint32_t* hist, SortPlan* plan,
                                                        uint64_t* bases, const uint32_t* d_rank_n)
{
    __shared__ uint64_t warp_s[32];
    if (d_rank_n) fixed_bits += bits_of_count(*d_rank_n);
    uint64_t nw = d_nw ? *d_nw : nw_max;
    uint32_t npass, bits;
    plan_shape(nw, fixed_bits, npass, bits);
    const int nb = 1 << bits;
    for (uint32_t k = 0; k < npass; ++k) {
        const int d = 2 * threadIdx.x;   // two digits per thread
        uint64_t v0 = d < nb ? hist[(k << kSortMaxBits) + d] : 0;
        uint64_t v1 = d + 1 < nb ? hist[(k << kSortMaxBits) + d + 1] : 0;
        uint64_t tot;
        uint64_t ex = block_exclusive_scan<1024, uint64_t>(v0 + v1, warp_s, tot);
        if (d < nb) bases[((size_t)k << kSortMaxBits) + d] = ex;
        if (d + 1 < nb) bases[((size_t)k << kSortMaxBits) + d + 1] = ex + v0;
    }
    if (threadIdx.x == 0) {
        SortPlan p;
        p.npass = npass;
        p.bits = bits;
        p.shift0 = shift0;
        p.pad = 0;
        *plan = p;
    }
}

size_t sort_scratch_bytes(uint64_t n)
{
    uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return Workspace::bytes_for({sizeof(SortPlan), sizeof(uint64_t) * (kSortMaxPass << kSortMaxBits),
                                 sizeof(uint32_t) * (kSortMaxPass << kSortMaxBits),
                                 sizeof(uint32_t) * (size_t)(ntiles ? ntiles : 1) * (1 << kSortMaxBits),
                                 sizeof(uint32_t) * 8});
}

SortScratch take_sort_scratch(const Workspace& ws, uint64_t n)
{
    uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
    SortScratch s;
    s.plan = ws.take<SortPlan>(1);
    s.bases = ws.take<uint64_t>(kSortMaxPass << kSortMaxBits);
    s.hist = ws.take<uint32_t>(kSortMaxPass << kSortMaxBits);
    s.status = ws.take<uint32_t>((size_t)(ntiles ? ntiles : 1) * (1 << kSortMaxBits));
    s.counter = ws.take<uint32_t>(8);
    return s;
}

cudaError_t sort_plan_weights(const SortScratch& sc, const uint32_t* weights, const uint64_t* offsets,
                              const uint32_t* d_nw, uint64_t nw_max, uint32_t shift0, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * (kSortMaxPass << kSortMaxBits), st);
    if (e) return e;
    int grid = (int)std::min<uint64_t>((nw_max + 1023) / 1024 ? (nw_max + 1023) / 1024 : 1, 512);
    k_plan_hist_weights<<<grid, 1024, 0, st>>>(weights, offsets, d_nw, nw_max, sc.hist);
    k_plan_finalize<<<1, 1024, 0, st>>>(d_nw, nw_max, 0, shift0, sc.hist, sc.plan, sc.bases, nullptr);
    return cudaGetLastError();
}

cudaError_t sort_plan_keys(const SortScratch& sc, const uint64_t* keys, uint64_t n, const uint32_t* d_n,
                           uint32_t shift0, uint32_t total_bits, cudaStream_t st, const uint32_t* d_rank_n)
{
    cudaError_t e = cudaMemsetAsync(sc.hist, 0, sizeof(uint32_t) * (kSortMaxPass << kSortMaxBits), st);
    if (e) return e;
    int grid = (int)std::min<uint64_t>((n + 4095) / 4096 ? (n + 4095) / 4096 : 1, 1024);
    k_plan_hist_keys<<<grid, 1024, 0, st>>>(keys, n, d_n, shift0, total_bits, sc.hist, d_rank_n);
    k_plan_finalize<<<1, 1024, 0, st>>>(nullptr, 0, total_bits, shift0, sc.hist, sc.plan, sc.bases, d_rank_n);
    return cudaGetLastError();
}

// ------------------------------------------------------------- distribute
size_t distribute_ws_bytes(uint64_t n, int g)
{
    (void)g;
    return sort_scratch_bytes(n) + Workspace::bytes_for({16 * (size_t)n, 4 * (size_t)n, sizeof(uint32_t)}) +
           dist_wide_bytes(n);
}

cudaError_t launch_distribute(const fp_point* pts, uint64_t n, const fp_cube* cube, int g, const uint32_t* lut,
                              const uint64_t* offsets, const uint32_t* num_chunks, fp_point* out, uint32_t* perm,
                              const Workspace& ws, cudaStream_t st, const uint32_t* cells)
{
    if (n == 0) return cudaSuccess;
    SortScratch sc = take_sort_scratch(ws, n);
    int4* pt_tmp = ws.take<int4>(n);
    uint32_t* val_tmp = ws.take<uint32_t>(n);
    uint32_t* run_sort = ws.take<uint32_t>(1);
    Workspace rest = ws;
    KTimerScope kt(FP_KERNEL_DISTRIBUTE, st);
    // With the cells given (16-byte aligned), up to 4096 chunks: the count, scan
    // and double-buffered sweep (every point's chunk kept in val_tmp, which the
    // radix passes below then do not use).  Otherwise 257..2048 chunks: one sweep
    // with chunk digits (no plan, bases = offsets).  Else the radix passes below
    // (one pass up to 256 chunks), which compute the cells from the points.
    cudaError_t e = dist_wide(reinterpret_cast<const int4*>(pts), n, cube, g, lut, offsets, num_chunks,
                              reinterpret_cast<int4*>(out), perm, run_sort, rest, st, cells,
                              reinterpret_cast<uint16_t*>(val_tmp));
    if (e) return e;
    // bucket weights = chunk counts (offsets[c+1] - offsets[c])
    if ((e = sort_plan_weights(sc, nullptr, offsets, num_chunks, 1ull << (3 * g), 0, st))) return e;
    SortArgs a{};
    a.b.pt_src = reinterpret_cast<const int4*>(pts);
    a.b.pt_tmp = pt_tmp;
    a.b.pt_dst = reinterpret_cast<int4*>(out);
    a.b.val_src = nullptr;   // value = original index
    a.b.val_tmp = perm ? val_tmp : nullptr;
    a.b.val_dst = perm;
    a.n = n;
    a.cube = cube;
    a.lut = lut;
    a.g = g;
    a.err = ws.err;
    a.run_if = run_sort;
    const int npass = sort_passes(count_bits(1ull << (3 * g)));   // chunk ids below 8^g
    for (int slot = 0; slot < npass; ++slot) {
        e = sort_run_pass<DIG_CHUNK, true, false, false>(sc, a, slot, ws.num_sms, st);
        if (e) return e;
    }
    return cudaSuccess;
}

}  // namespace fp
