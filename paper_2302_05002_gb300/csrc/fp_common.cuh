// fp_common.cuh -- device helpers shared by the kernels of libfastpoints.
//
// Cell arithmetic (paper Sec. 4.4; exact-integer reading): for axis a,
//   c_a(l) = floor((p_a - o_a) * 2^l / S),   0 <= p_a - o_a < 2^32,  1 <= S <= 2^32.
// It is evaluated once at l = 21 and shifted for coarser levels (floor of a
// floor: c(l) = c(21) >> (21 - l)).  The level-21 quotient is first estimated in
// fp32 (relative error < 2^-22, so the estimate is within 1 of the true floor
// for quotients below 2^21) and then corrected exactly with one 64-bit
// remainder test.  The Morton key interleaves one bit per axis per level with
// the x bit most significant inside every 3-bit digit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/fastpoints.h"

#define FP_DEV __device__ __forceinline__

namespace fp {

constexpr int kKeyLevels = 21;          // deepest level of the 63-bit key
constexpr uint32_t kNone = 0xFFFFFFFFu;

// Sticky per-device error word (passed to every kernel); bit (1u << fp_status)
// marks each kind of fault.
// err[0]: status bits (1 << status); err[1]: the check sites that fired (one
// bit per site, for diagnosing which capacity or consistency check failed)
FP_DEV void raise(uint32_t* err, fp_status s, int site = -1)
{
    atomicOr(err, 1u << (unsigned)s);
    if (site >= 0) atomicOr(err + 1, 1u << (unsigned)site);
}

// ------------------------------------------------------------------ cube
struct CubeDev {
    int32_t o[3];
    uint64_t S;
    float scale21;   // 2^21 / S in fp32
};

FP_DEV CubeDev load_cube(const fp_cube* c)
{
    CubeDev d;
    d.o[0] = c->o[0]; d.o[1] = c->o[1]; d.o[2] = c->o[2];
    d.S = c->S;
    d.scale21 = d.S ? 2097152.0f / (float)d.S : 0.f;
    return d;
}

// floor(d * 2^l / S) for d = p - o, 0 <= d < S <= 2^32, l <= 21; scale = 2^l / S
// in fp32.  d fits 32 bits, q * S is a 32 x 32 -> 64-bit product (S = 2^32 is
// the one value with a high word).
FP_DEV uint32_t cell_at(int32_t p, int32_t o, uint64_t S, float scale, int l)
{
    const uint32_t d = (uint32_t)((int64_t)p - (int64_t)o);
    int32_t q = (int32_t)((float)d * scale);
    if (q < 0) q = 0;
    const uint64_t num = (uint64_t)d << l;
    const uint64_t qs = (uint64_t)(uint32_t)q * (uint32_t)S + ((uint64_t)((uint32_t)q * (uint32_t)(S >> 32)) << 32);
    if (num < qs) --q;
    else if (num - qs >= S) ++q;
    return (uint32_t)q;
}

FP_DEV uint32_t cell21(int32_t p, int32_t o, uint64_t S, float scale21) { return cell_at(p, o, S, scale21, 21); }

FP_DEV uint32_t spread3_10(uint32_t x)   // 10 bits -> bits 0, 3, ..., 27
{
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

FP_DEV uint64_t spread3(uint32_t v)   // 21 bits -> bits 0, 3, ..., 60
{
    return (uint64_t)spread3_10(v) | ((uint64_t)spread3_10(v >> 10) << 30) | ((uint64_t)((v >> 20) & 1u) << 60);
}

// 63-bit Morton key of the level-21 cell of a point
FP_DEV uint64_t key21(int32_t x, int32_t y, int32_t z, const CubeDev& c)
{
    uint32_t cx = cell21(x, c.o[0], c.S, c.scale21);
    uint32_t cy = cell21(y, c.o[1], c.S, c.scale21);
    uint32_t cz = cell21(z, c.o[2], c.S, c.scale21);
    return (spread3(cx) << 2) | (spread3(cy) << 1) | spread3(cz);
}

// fp32 2^l / S from the cube's 2^21 / S (scaling by a power of two is exact)
FP_DEV float scale_at(const CubeDev& c, int l) { return c.scale21 * __int_as_float((127 + l - 21) << 23); }

// Morton key of the level-l cell of a point, l <= 10 (equal to key21 >> 3 (21 - l))
FP_DEV uint32_t key_small(int32_t x, int32_t y, int32_t z, const CubeDev& c, float scale, int l)
{
    return (spread3_10(cell_at(x, c.o[0], c.S, scale, l)) << 2) | (spread3_10(cell_at(y, c.o[1], c.S, scale, l)) << 1) |
           spread3_10(cell_at(z, c.o[2], c.S, scale, l));
}

FP_DEV uint64_t key_at(uint64_t k21, int level) { return k21 >> (3 * (kKeyLevels - level)); }

// per-point code of the octree stage: LOD owner level (5 bits), leaf level (5
// bits) and the Morton key of the point's level-g cell (3 g <= 21 bits)
FP_DEV uint32_t code_make(int own, int leaf, uint32_t cell)
{
    return (uint32_t)own | ((uint32_t)leaf << 5) | (cell << 10);
}
FP_DEV int code_own(uint32_t c) { return (int)(c & 31u); }
FP_DEV int code_leaf(uint32_t c) { return (int)((c >> 5) & 31u); }
FP_DEV uint32_t code_cell(uint32_t c) { return c >> 10; }

// level of the deepest cell two level-21 keys share (-1: not even the root? no: >= 0)
FP_DEV int common_level(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return kKeyLevels;
    int lz = __clzll((long long)x) - 1;   // bit 63 is always 0
    return lz / 3;
}

// ------------------------------------------------------------------ hash
// first output of a splitmix64 generator seeded with v (Steele, Lea, Flood 2014)
FP_DEV uint64_t splitmix64(uint64_t v)
{
    uint64_t z = v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------------ memory
FP_DEV int4 ld_point(const fp_point* p, uint64_t i) { return __ldg(reinterpret_cast<const int4*>(p) + i); }
FP_DEV int4 ld_point_cs(const fp_point* p, uint64_t i)
{
    return __ldcs(reinterpret_cast<const int4*>(p) + i);
}
FP_DEV void st_point(fp_point* p, uint64_t i, int4 v) { reinterpret_cast<int4*>(p)[i] = v; }

FP_DEV uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp holding the same BITS-bit value v as this lane, among the
// lanes with `valid` set (one ballot per bit: the cost does not grow with the
// number of distinct values in the warp).  All 32 lanes take part.
template <int BITS>
FP_DEV uint32_t match_bits(uint32_t v, bool valid)
{
    uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (v >> b) & 1u;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// volatile load for inter-block flags
FP_DEV uint32_t ld_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// ---- bulk copies global -> shared memory completing on an mbarrier (TMA,
// one-dimensional form: 16-byte aligned addresses, size a multiple of 16)
FP_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
FP_DEV void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// orders this CTA's earlier shared-memory accesses before later bulk copies into it
FP_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
FP_DEV void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
FP_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
FP_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before a wait counts as timed out
FP_DEV bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
FP_DEV uint64_t ld_volatile64(const uint64_t* p) { return *(const volatile uint64_t*)p; }

// ------------------------------------------------------------------ block scan
// Exclusive scan of one value per thread over a block of NT threads (NT % 32 == 0).
template <int NT, typename T>
FP_DEV T block_exclusive_scan(T v, T* smem_warp /* NT/32 entries */, T& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? smem_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) smem_warp[lane] = w;
    }
    __syncthreads();
    total = smem_warp[NT / 32 - 1];
    T before = warp ? smem_warp[warp - 1] : T(0);
    __syncthreads();
    return before + x - v;
}

// Bounded spin: number of polls before an inter-block wait gives up.
constexpr uint32_t kSpinLimit = 1u << 24;

}  // namespace fp
