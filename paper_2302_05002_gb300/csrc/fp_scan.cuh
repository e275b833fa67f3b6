// fp_scan.cuh -- device-wide exclusive scan for arrays of up to 8M entries whose
// length may live on the device (three launches: tile sums, one-block scan of
// the tile sums, tile scan plus carry).  Used for the count grid (8^g cells),
// chunk offsets and per-cell node counts.
#pragma once
#include "fp_common.cuh"

namespace fp {

constexpr int kScanNT = 256;
constexpr int kScanIPT = 16;
constexpr int kScanTile = kScanNT * kScanIPT;      // 4096
constexpr int kScanMaxTiles = 2048;                // n <= 8M

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanNT) k_scan_tile_sums(const Tin* in, uint64_t n_max, const uint32_t* d_n,
                                                            Tout* tile_sums)
{
    uint64_t n = d_n ? *d_n : n_max;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    Tout s = 0;
    if (base < n) {
        for (int r = 0; r < kScanIPT; ++r) {
            uint64_t i = base + (uint64_t)r * kScanNT + threadIdx.x;
            if (i < n) s += (Tout)in[i];
        }
    }
    __shared__ Tout warp_s[kScanNT / 32];
    Tout tot;
    block_exclusive_scan<kScanNT, Tout>(s, warp_s, tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// one block of 1024 threads scans up to 2048 tile sums in place (exclusive);
// *total receives the grand total when not null
template <typename Tout>
__global__ void __launch_bounds__(1024) k_scan_top(Tout* tile_sums, int ntiles, Tout* total, Tout* total2)
{
    __shared__ Tout warp_s[32];
    int t = threadIdx.x;
    Tout a = 2 * t < ntiles ? tile_sums[2 * t] : Tout(0);
    Tout b = 2 * t + 1 < ntiles ? tile_sums[2 * t + 1] : Tout(0);
    Tout tot;
    Tout ex = block_exclusive_scan<1024, Tout>(a + b, warp_s, tot);
    if (2 * t < ntiles) tile_sums[2 * t] = ex;
    if (2 * t + 1 < ntiles) tile_sums[2 * t + 1] = ex + a;
    if (t == 0) {
        if (total) *total = tot;
        if (total2) *total2 = tot;
    }
}

// out[i] = exclusive prefix; in and out may alias
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanNT) k_scan_apply(const Tin* in, Tout* out, uint64_t n_max, const uint32_t* d_n,
                                                        const Tout* tile_sums)
{
    uint64_t n = d_n ? *d_n : n_max;
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    if (base >= n) return;
    // each thread owns kScanIPT consecutive entries
    Tout v[kScanIPT];
    Tout s = 0;
    uint64_t b0 = base + (uint64_t)threadIdx.x * kScanIPT;
#pragma unroll
    for (int r = 0; r < kScanIPT; ++r) {
        uint64_t i = b0 + r;
        v[r] = i < n ? (Tout)in[i] : Tout(0);
        s += v[r];
    }
    __shared__ Tout warp_s[kScanNT / 32];
    Tout tot;
    Tout ex = block_exclusive_scan<kScanNT, Tout>(s, warp_s, tot) + tile_sums[blockIdx.x];
#pragma unroll
    for (int r = 0; r < kScanIPT; ++r) {
        uint64_t i = b0 + r;
        if (i < n) out[i] = ex;
        ex += v[r];
    }
}

// Exclusive scan of in[0..n) into out[0..n) where n = *d_n (or n_max when
// d_n is null); n_max <= 8M bounds the grid.  tile_sums: kScanMaxTiles entries.
// *d_total / *d_total2 (nullable) receive the sum.
template <typename Tin, typename Tout>
inline cudaError_t scan_exclusive(const Tin* in, Tout* out, uint64_t n_max, const uint32_t* d_n, Tout* tile_sums,
                                  Tout* d_total, Tout* d_total2, cudaStream_t st)
{
    int ntiles = (int)((n_max + kScanTile - 1) / kScanTile);
    if (ntiles < 1) ntiles = 1;
    if (ntiles > kScanMaxTiles) return cudaErrorInvalidValue;
    k_scan_tile_sums<Tin, Tout><<<ntiles, kScanNT, 0, st>>>(in, n_max, d_n, tile_sums);
    k_scan_top<Tout><<<1, 1024, 0, st>>>(tile_sums, ntiles, d_total, d_total2);
    k_scan_apply<Tin, Tout><<<ntiles, kScanNT, 0, st>>>(in, out, n_max, d_n, tile_sums);
    return cudaGetLastError();
}

}  // namespace fp
