// fp_sort.cuh -- stable bucket scatter ("one sweep" LSD radix pass) used by the
// chunk distribution (Sec. 4.4, "sorted into chunks") and by the octree stages.
//
// One pass moves n records to out[base[d] + (records of digit d before it)],
// i.e. a stable scatter by one digit d of a key.  Tiles of 4096 records are
// claimed in order; each tile
//   1. computes the digits and ranks every record among the equal digits of its
//      own warp (match_any), warps own contiguous 256-record slices,
//   2. publishes its digit histogram, then looks back over earlier tiles for the
//      per-digit exclusive prefix (decoupled look-back, bounded spin),
//   3. stages the records in shared memory in digit order and writes each digit
//      run contiguously (coalesced).
// Several passes (least significant digit first) sort by a wider key.  The
// number of passes and the digit width are read from a device-side plan, so a
// whole multi-pass sort can be enqueued without knowing the key range on the
// host: surplus pass slots return at once, and slot k reads from the source,
// or the temporaries, and writes to the destination when it is the last pass.
#pragma once
#include "fp_internal.cuh"

namespace fp {

constexpr int kSortNT = 512;
constexpr int kSortIPT = 8;
constexpr int kSortWarps = kSortNT / 32;
constexpr int kSortTile = kSortNT * kSortIPT;   // 4096
constexpr int kSortMaxBits = 8;                 // at most 256 buckets per pass
constexpr int kSortMaxPass = 8;                 // keys of up to 64 bits
constexpr uint32_t kStFlagAgg = 1u << 30;
constexpr uint32_t kStFlagInc = 2u << 30;
constexpr uint32_t kStMask = (1u << 30) - 1;

enum DigitSource { DIG_K64 = 0, DIG_K32 = 1, DIG_CHUNK = 2 };

// Decoupled look-back of one digit: the sum of the counts of tiles t, t-1, ...
// down to the nearest one that published an inclusive prefix (tile t_first
// always does).  The status words of kLookBatch earlier tiles are read at once,
// so a walk over many tiles that published only their own counts costs one
// round trip per kLookBatch of them; reading stops at the first word not yet
// published and resumes there (bounded: FP_ERR_TIMEOUT after kSpinLimit rounds).
constexpr int kLookBatch = 8;
template <typename Word, int BATCH = kLookBatch>
FP_DEV uint32_t look_back(Word word, int64_t t, int64_t t_first, uint32_t* err, uint32_t limit = kSpinLimit)
{
    uint32_t excl = 0, spins = 0;
    while (t >= t_first) {
        uint32_t sv[BATCH];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) sv[k] = t - k >= t_first ? ld_volatile(word(t - k)) : 0u;
        int adv = 0;
        bool stop = false;
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            if (stop || t - k < t_first) { stop = true; continue; }
            const uint32_t f = sv[k] & ~kStMask;
            if (f == 0) { stop = true; continue; }   // not published yet: read again from here
            excl += sv[k] & kStMask;
            if (f == kStFlagInc) return excl;
            ++adv;
        }
        if (adv == 0 && ++spins > limit) {
            raise(err, FP_ERR_TIMEOUT);
            return excl;
        }
        t -= adv;
    }
    return excl;
}

struct SortPlan {
    uint32_t npass;    // passes to run (1..kSortMaxPass)
    uint32_t bits;     // digit width of every pass
    uint32_t shift0;   // key bit of digit 0
    uint32_t pad;
};

// Buffers of one multi-pass sort.  Null pointers mean "field not present".
// Passes ping-pong between dst and one temporary so that the last pass lands
// in dst: pass k writes dst when (npass - 1 - k) is even, tmp otherwise.
struct SortBufs {
    const int4* pt_src; int4* pt_tmp; int4* pt_dst;
    const uint32_t* val_src; uint32_t* val_tmp; uint32_t* val_dst;   // val_src null: value = index
    const uint64_t* k64_src; uint64_t* k64_tmp; uint64_t* k64_dst;
    const uint32_t* k32_src; uint32_t* k32_tmp; uint32_t* k32_dst;
};

struct SortArgs {
    SortBufs b;
    uint64_t n;               // records (upper bound when d_n is set)
    const uint32_t* d_n;      // device-side record count (nullable)
    const SortPlan* plan;
    const uint64_t* bases;    // [kSortMaxPass][1 << kSortMaxBits]
    uint32_t* status;         // [tiles][1 << bits]
    uint32_t* counter;        // tile counter of the pass
    // digit from points
    const fp_cube* cube;
    const uint32_t* lut;      // DIG_CHUNK: cell -> chunk
    int g;
    const uint32_t* run_if;   // nullable: the pass runs only when *run_if != 0
    int bulk;                 // 64-bit key layout with 16-byte aligned arrays: tiles arrive by bulk copy
    uint32_t withhold;        // test hook of the bounded waits: this tile publishes nothing (0xFFFFFFFF: none)
    uint32_t spin_limit;      // rounds of the look-back before FP_ERR_TIMEOUT
    uint32_t* err;
};

template <typename T>
FP_DEV T* pick_dst(int slot, int npass, T* dst, T* tmp) { return ((npass - 1 - slot) & 1) ? tmp : dst; }
template <typename T>
FP_DEV const T* pick_src(int slot, int npass, const T* src, T* dst, T* tmp)
{
    return slot == 0 ? src : pick_dst(slot - 1, npass, dst, tmp);
}

// Digits of at most 8 bits keep the per-warp histograms, the digit scan and the
// look-back small enough for two CTAs per SM; wider digits measured several
// times slower per pass than two 8-bit passes.
// The 64-bit key layout (optionally with values) streams each full tile into
// shared memory with bulk copies; the next tile's copy is issued as soon as the
// current tile has been staged, so it overlaps the look-back and the writes.
template <int DIG, bool CPT, bool CK64, bool CK32>
constexpr bool sort_bulk_layout() { return DIG == DIG_K64 && CK64 && !CPT && !CK32; }

template <int DIG, bool CPT, bool CK64, bool CK32>
struct SortSmem {
    using dig_t = uint8_t;
    static constexpr bool BULK = sort_bulk_layout<DIG, CPT, CK64, CK32>();
    static constexpr size_t raw_k = BULK ? sizeof(uint64_t) * kSortTile : 0;   // first: 16-byte aligned
    static constexpr size_t raw_v = BULK ? sizeof(uint32_t) * kSortTile : 0;
    static constexpr size_t bar = BULK ? 16 : 0;
    static constexpr size_t pt = CPT ? sizeof(int4) * kSortTile : 0;
    static constexpr size_t k64 = CK64 ? sizeof(uint64_t) * kSortTile : 0;
    static constexpr size_t val = sizeof(uint32_t) * kSortTile;
    static constexpr size_t k32 = CK32 ? sizeof(uint32_t) * kSortTile : 0;
    static constexpr size_t dig = sizeof(dig_t) * kSortTile;
    static constexpr size_t whist = sizeof(uint16_t) * kSortWarps * (1 << kSortMaxBits);
    static constexpr size_t gbase = sizeof(uint64_t) * (1 << kSortMaxBits);
    static constexpr size_t cnt = sizeof(uint32_t) * (1 << kSortMaxBits);
    static constexpr size_t off = sizeof(uint32_t) * (1 << kSortMaxBits);
    static constexpr size_t misc = 4 * (1 + kSortWarps + 15);   // block-scan scratch
    static constexpr size_t tiles = 4 * 2;                       // current and next tile id
    static constexpr size_t total =
        raw_k + raw_v + bar + pt + k64 + val + k32 + dig + whist + gbase + cnt + off + misc + tiles;
    // two CTAs per SM: 228 KB of shared memory, 1 KB of it reserved per CTA
    static_assert(!BULK || total <= 113 * 1024, "bulk layout must leave room for two CTAs per SM");
};

template <int DIG, bool CPT, bool CK64, bool CK32>
__global__ void __launch_bounds__(kSortNT, 2) k_sort_pass(SortArgs a, int slot)
{
    const SortPlan plan = *a.plan;
    if (slot >= (int)plan.npass || (a.run_if && !*a.run_if)) return;
    using SM = SortSmem<DIG, CPT, CK64, CK32>;
    using dig_t = typename SM::dig_t;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* sp = smem;
    uint64_t* raw_k = reinterpret_cast<uint64_t*>(sp); sp += SM::raw_k;
    uint32_t* raw_v = reinterpret_cast<uint32_t*>(sp); sp += SM::raw_v;
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(sp); sp += SM::bar;
    int4* s_pt = reinterpret_cast<int4*>(sp); sp += SM::pt;
    uint64_t* s_k64 = reinterpret_cast<uint64_t*>(sp); sp += SM::k64;
    uint64_t* s_gbase = reinterpret_cast<uint64_t*>(sp); sp += SM::gbase;
    uint32_t* s_val = reinterpret_cast<uint32_t*>(sp); sp += SM::val;
    uint32_t* s_k32 = reinterpret_cast<uint32_t*>(sp); sp += SM::k32;
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(sp); sp += SM::cnt;
    uint32_t* s_off = reinterpret_cast<uint32_t*>(sp); sp += SM::off;
    dig_t* s_dig = reinterpret_cast<dig_t*>(sp); sp += SM::dig;
    uint16_t* s_whist = reinterpret_cast<uint16_t*>(sp); sp += SM::whist;
    uint32_t* s_misc = reinterpret_cast<uint32_t*>(sp); sp += SM::misc;   // [1..] scan scratch
    uint32_t* s_tile = reinterpret_cast<uint32_t*>(sp);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bits = (int)plan.bits;
    const int nb = 1 << bits;
    const uint32_t dmask = (uint32_t)nb - 1;
    const int shift = (int)(plan.shift0 + slot * plan.bits);
    const uint64_t n = a.d_n ? min((uint64_t)*a.d_n, a.n) : a.n;
    const uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int npass = (int)plan.npass;

    const int4* in_pt = pick_src(slot, npass, a.b.pt_src, a.b.pt_dst, a.b.pt_tmp);
    const uint32_t* in_val = pick_src(slot, npass, a.b.val_src, a.b.val_dst, a.b.val_tmp);
    const uint64_t* in_k64 = pick_src(slot, npass, a.b.k64_src, a.b.k64_dst, a.b.k64_tmp);
    const uint32_t* in_k32 = pick_src(slot, npass, a.b.k32_src, a.b.k32_dst, a.b.k32_tmp);
    int4* out_pt = pick_dst(slot, npass, a.b.pt_dst, a.b.pt_tmp);
    uint32_t* out_val = pick_dst(slot, npass, a.b.val_dst, a.b.val_tmp);
    uint64_t* out_k64 = pick_dst(slot, npass, a.b.k64_dst, a.b.k64_tmp);
    uint32_t* out_k32 = pick_dst(slot, npass, a.b.k32_dst, a.b.k32_tmp);
    const uint64_t* bases = a.bases + (size_t)slot * (1 << kSortMaxBits);

    CubeDev cube;
    if (DIG == DIG_CHUNK) cube = load_cube(a.cube);
    const float scale_g = DIG == DIG_CHUNK ? scale_at(cube, a.g) : 0.f;

    const bool use_bulk = SM::BULK && a.bulk;
    const bool has_val = in_val != nullptr;
    const uint32_t tx_bytes = (uint32_t)(sizeof(uint64_t) * kSortTile + (has_val ? sizeof(uint32_t) * kSortTile : 0));
    auto issue = [&](uint64_t t) {   // thread 0: bulk copy of full tile t, if any
        if (t >= ntiles || (t + 1) * kSortTile > n) return;
        fence_async_smem();
        mbar_expect_tx(s_bar, tx_bytes);
        bulk_g2s(raw_k, in_k64 + t * kSortTile, (uint32_t)(sizeof(uint64_t) * kSortTile), s_bar);
        if (has_val) bulk_g2s(raw_v, in_val + t * kSortTile, (uint32_t)(sizeof(uint32_t) * kSortTile), s_bar);
    };
    uint32_t nwait = 0;   // bulk tiles waited for: the mbarrier's phase parity

    // Tiles are claimed in order through the counter; each CTA claims its next
    // tile while it works on the current one (a claimed tile only waits on
    // smaller ones, so holding one in reserve cannot deadlock the look-back).
    if (threadIdx.x == 0) {
        if (use_bulk) mbar_init(s_bar, 1);
        s_tile[0] = atomicAdd(a.counter, 1u);
        if (use_bulk) issue(s_tile[0]);
    }
    for (int it = 0;; ++it) {
        // zero the per-warp histograms of this tile
        for (int q = threadIdx.x; q < kSortWarps * nb / 8; q += kSortNT)
            reinterpret_cast<uint4*>(s_whist)[q] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        const uint64_t tile = s_tile[it & 1];
        if (tile >= ntiles) break;
        if (threadIdx.x == 0) s_tile[(it + 1) & 1] = atomicAdd(a.counter, 1u);
        const uint64_t base = tile * kSortTile;
        const int tn = (int)(n - base < (uint64_t)kSortTile ? n - base : (uint64_t)kSortTile);
        uint16_t* wh = s_whist + warp * nb;
        if (use_bulk) {
            if (tn == kSortTile) {   // this tile's bulk copy was issued a tile ago (or in the prologue)
                const bool ok = mbar_wait(s_bar, nwait & 1);
                ++nwait;
                if (__syncthreads_or(!ok)) {
                    if (threadIdx.x == 0) raise(a.err, FP_ERR_TIMEOUT);
                    mbar_wait(s_bar, (nwait - 1) & 1);   // bounded: let the copy land before leaving
                    break;
                }
            } else {                 // the ragged last tile: plain loads
                for (int p = threadIdx.x; p < tn; p += kSortNT) {
                    raw_k[p] = in_k64[base + p];
                    if (has_val) raw_v[p] = in_val[base + p];
                }
                __syncthreads();
            }
        }

        // ---- phase 1: digits (all loads issued first), then in-warp stable ranks
        uint32_t dg[kSortIPT];
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const int p = warp * (kSortIPT * 32) + r * 32 + lane;
            uint32_t d = 0xFFFFu;
            if (p < tn) {
                const uint64_t i = base + p;
                if (DIG == DIG_K64) d = (uint32_t)((use_bulk ? raw_k[p] : in_k64[i]) >> shift) & dmask;
                else if (DIG == DIG_K32) d = (in_k32[i] >> shift) & dmask;
                else {
                    int4 q = __ldg(in_pt + i);
                    d = key_small(q.x, q.y, q.z, cube, scale_g, a.g);   // cell; its chunk below
                }
            }
            dg[r] = d;
        }
        if (DIG == DIG_CHUNK) {
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r)
                if (warp * (kSortIPT * 32) + r * 32 + lane < tn) dg[r] = (__ldg(a.lut + dg[r]) >> shift) & dmask;
        }
        uint32_t pack[kSortIPT];
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const uint32_t d = dg[r];
            const uint32_t peers = match_bits<kSortMaxBits>(d, d != 0xFFFFu);
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

        // ---- per-digit totals, per-warp exclusive prefixes, publish aggregates
        for (int d = threadIdx.x; d < nb; d += kSortNT) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t v = s_whist[w * nb + d];
                s_whist[w * nb + d] = (uint16_t)s;
                s += v;
            }
            s_cnt[d] = s;
            if (tile != a.withhold) a.status[tile * nb + d] = (tile == 0 ? kStFlagInc : kStFlagAgg) | s;
        }
        __syncthreads();
        // exclusive scan of s_cnt over digits -> s_off (each thread a run of digits)
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

        // ---- phase 2: stage records in digit order
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const int p = warp * (kSortIPT * 32) + r * 32 + lane;
            if (p < tn) {
                const uint32_t d = pack[r] & 0xFFFFu;
                const uint32_t lp = s_off[d] + s_whist[warp * nb + d] + (pack[r] >> 16);
                const uint64_t i = base + p;
                if (CPT) s_pt[lp] = __ldg(in_pt + i);
                if (CK64) s_k64[lp] = use_bulk ? raw_k[p] : in_k64[i];
                if (CK32) s_k32[lp] = in_k32[i];
                s_val[lp] = has_val ? (use_bulk ? raw_v[p] : in_val[i]) : (uint32_t)i;
                s_dig[lp] = (dig_t)d;
            }
        }
        if (use_bulk) {   // the raw tile is consumed: start the next one
            __syncthreads();
            if (threadIdx.x == 0) issue(s_tile[(it + 1) & 1]);
        }

        // ---- look-back: exclusive prefix of every digit over earlier tiles
        for (int d = threadIdx.x; d < nb; d += kSortNT) {
            uint32_t excl = 0;
            if (tile > 0) {
                auto word = [&](int64_t t) { return &a.status[(uint64_t)t * nb + d]; };
                excl = look_back<decltype(word), kLookBatch>(word, (int64_t)tile - 1, 0, a.err, a.spin_limit);
                if (tile != a.withhold) atomicExch(&a.status[tile * nb + d], kStFlagInc | (excl + s_cnt[d]));
            }
            s_gbase[d] = bases[d] + excl - s_off[d];
        }
        __syncthreads();

        // ---- phase 3: coalesced writes of each digit run
        for (int q = threadIdx.x; q < tn; q += kSortNT) {
            const uint64_t o = s_gbase[s_dig[q]] + q;
            if (o >= n) { raise(a.err, FP_ERR_CAPACITY, 16); continue; }   // inconsistent bucket totals
            if (CPT) out_pt[o] = s_pt[q];
            if (CK64) out_k64[o] = s_k64[q];
            if (CK32 && out_k32) out_k32[o] = s_k32[q];
            if (out_val) out_val[o] = s_val[q];
        }
        __syncthreads();
    }
}

// zero the status words and the tile counter of one pass slot
__global__ void k_sort_zero(uint32_t* status, uint32_t* counter, uint64_t n, const uint32_t* d_n, const SortPlan* plan,
                            int slot);

// Plan from per-id weights (ids 0..*d_nw-1, or nw_max when d_nw is null; the id
// is the key above bit shift0):
// digit histograms of every pass -> bucket bases.  hist: kSortMaxPass << kSortMaxBits u32, zeroed by the caller.
__global__ void k_plan_hist_weights(const uint32_t* weights, const uint64_t* offsets, const uint32_t* d_nw,
                                    uint64_t nw_max, uint32_t* hist);
__global__ void k_plan_finalize(const uint32_t* d_nw, uint64_t nw_max, uint32_t fixed_bits, uint32_t shift0,
                                const uint32_t* hist, SortPlan* plan, uint64_t* bases, const uint32_t* d_rank_n);
// Plan of a fixed-width key sort: digits of bits [shift0, shift0 + total_bits) of k64 keys.
__global__ void k_plan_hist_keys(const uint64_t* keys, uint64_t n, const uint32_t* d_n, uint32_t shift0,
                                 uint32_t total_bits, uint32_t* hist, const uint32_t* d_rank_n);

// host helpers
// Launch bound of a sort: the device plan of keys with `bits` significant bits
// takes ceil(bits / kSortMaxBits) passes (ids below nw: count_bits(nw) bits);
// the passes past the plan exit at once, so launching this many suffices.
inline int sort_passes(uint64_t bits)
{
    bits = bits < 1 ? 1 : (bits > 64 ? 64 : bits);
    return (int)((bits + kSortMaxBits - 1) / kSortMaxBits);
}
inline uint32_t count_bits(uint64_t v)   // bits of v - 1, at least 1, as the device plan counts them
{
    uint32_t b = 1;
    while (b < 64 && ((v ? v - 1 : 0) >> b)) ++b;
    return b;
}
struct SortScratch {
    SortPlan* plan;
    uint64_t* bases;
    uint32_t* hist;
    uint32_t* status;
    uint32_t* counter;
};
size_t sort_scratch_bytes(uint64_t n);
SortScratch take_sort_scratch(const Workspace& ws, uint64_t n);

// plan from weights of ids; then run the passes of the given kind
cudaError_t sort_plan_weights(const SortScratch& sc, const uint32_t* weights, const uint64_t* offsets,
                              const uint32_t* d_nw, uint64_t nw_max, uint32_t shift0, cudaStream_t st);
// total_bits of key above shift0, plus the bit width of *d_rank_n when given
cudaError_t sort_plan_keys(const SortScratch& sc, const uint64_t* keys, uint64_t n, const uint32_t* d_n,
                           uint32_t shift0, uint32_t total_bits, cudaStream_t st,
                           const uint32_t* d_rank_n = nullptr);

template <int DIG, bool CPT, bool CK64, bool CK32>
cudaError_t sort_launch(const SortArgs& a, int slot, int num_sms, cudaStream_t st)
{
    using SM = SortSmem<DIG, CPT, CK64, CK32>;
    auto kern = k_sort_pass<DIG, CPT, CK64, CK32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::total);
    if (e) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSortNT, SM::total);
    if (e) return e;
    if (per_sm < 1) per_sm = 1;
    uint64_t ntiles = (a.n + kSortTile - 1) / kSortTile;
    int grid = (int)std::min<uint64_t>(ntiles ? ntiles : 1, (uint64_t)num_sms * per_sm);
    kern<<<grid, kSortNT, SM::total, st>>>(a, slot);
    return cudaGetLastError();
}

template <int DIG, bool CPT, bool CK64, bool CK32>
cudaError_t sort_run_pass(const SortScratch& sc, const SortArgs& a0, int slot, int num_sms, cudaStream_t st)
{
    cudaError_t e;
    SortArgs a = a0;
    debug_wait_config(&a.withhold, &a.spin_limit);
    a.plan = sc.plan;
    a.bases = sc.bases;
    a.status = sc.status;
    a.counter = sc.counter + slot;
    uint64_t ntiles = (a.n + kSortTile - 1) / kSortTile;
    k_sort_zero<<<std::max(1, std::min(num_sms * 4, (int)((ntiles * (1 << kSortMaxBits) + 1023) / 1024))), 256, 0,
                  st>>>(sc.status, sc.counter + slot, a.n, a.d_n, sc.plan, slot);
    if ((e = cudaGetLastError())) return e;
    if (sort_bulk_layout<DIG, CPT, CK64, CK32>()) {
        auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
        a.bulk = al(a.b.k64_src) && al(a.b.k64_tmp) && al(a.b.k64_dst) && al(a.b.val_src) && al(a.b.val_tmp) &&
                 al(a.b.val_dst);
    }
    return sort_launch<DIG, CPT, CK64, CK32>(a, slot, num_sms, st);
}

}  // namespace fp
