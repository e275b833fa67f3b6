// fp_render.cu -- the renderer's side of the octree, headless (Sec. 4.5):
// which nodes a camera draws, and the points of those nodes rasterised into a
// device framebuffer.
//
// Selection: a node is drawn when its box is not outside the view frustum and
// every ancestor was refined; a node is refined when it is drawn, is not a
// leaf, and its box covers more than min_node_px pixels on screen (a box that
// reaches behind the camera plane counts as infinitely large).  So each drawn
// node contributes its own level-of-detail sample, and finer nodes are drawn
// only where the coarser ones are large on screen.  In preorder a node's
// subtree is the range [i, i + n_desc]: a node that is not refined excludes
// that range (difference array + scan), then the drawn nodes are compacted.
//
// Rasterisation: each point of a drawn node is projected by the 4x4 matrix;
// the nearest one per pixel wins through a 64-bit atomicMin on
// (depth bits << 32 | colour), depth = clip z / w in [0, 1].
//
// All floating point is fp32 with the fused multiply-adds, divisions and
// roundings spelled out, so that the CPU restatement reproduces every
// projection, pixel and visibility decision bit for bit.
#include "fp_internal.cuh"

namespace fp {

namespace {

struct CamDev {
    float m[16];
    float W, H, minpx;
    uint32_t w, h;
};

CamDev cam_dev(const fp_camera& c)
{
    CamDev d;
    for (int i = 0; i < 16; ++i) d.m[i] = c.m[i];
    d.W = (float)c.width;
    d.H = (float)c.height;
    d.minpx = c.min_node_px;
    d.w = c.width;
    d.h = c.height;
    return d;
}

struct Clip {
    float x, y, z, w;
};

// clip = m * (x, y, z, 1), each row as fma(m0, x, fma(m1, y, fma(m2, z, m3)))
FP_DEV Clip clip_of(const CamDev& c, float x, float y, float z)
{
    Clip r;
    r.x = __fmaf_rn(c.m[0], x, __fmaf_rn(c.m[1], y, __fmaf_rn(c.m[2], z, c.m[3])));
    r.y = __fmaf_rn(c.m[4], x, __fmaf_rn(c.m[5], y, __fmaf_rn(c.m[6], z, c.m[7])));
    r.z = __fmaf_rn(c.m[8], x, __fmaf_rn(c.m[9], y, __fmaf_rn(c.m[10], z, c.m[11])));
    r.w = __fmaf_rn(c.m[12], x, __fmaf_rn(c.m[13], y, __fmaf_rn(c.m[14], z, c.m[15])));
    return r;
}

// screen x (or y) of a normalised device coordinate: fma(n, 0.5, 0.5) * W
FP_DEV float screen(float n, float W) { return __fmul_rn(__fmaf_rn(n, 0.5f, 0.5f), W); }

// integer bounds of the points of node (level, key): lo_a = o_a + ceil(c S / 2^L),
// hi_a = o_a + ceil((c + 1) S / 2^L) - 1, exact in 64 bits (c S < 2^53)
FP_DEV void node_box(const fp_cube& cb, int L, uint64_t key, float lo[3], float hi[3])
{
    uint64_t c[3] = {0, 0, 0};
    for (int b = 0; b < L; ++b) {
        c[0] |= ((key >> (3 * b + 2)) & 1ull) << b;
        c[1] |= ((key >> (3 * b + 1)) & 1ull) << b;
        c[2] |= ((key >> (3 * b)) & 1ull) << b;
    }
    const uint64_t r = (1ull << L) - 1;
    for (int a = 0; a < 3; ++a) {
        const int64_t l = (int64_t)cb.o[a] + (int64_t)((c[a] * cb.S + r) >> L);
        const int64_t h = (int64_t)cb.o[a] + (int64_t)(((c[a] + 1) * cb.S + r) >> L) - 1;
        lo[a] = __ll2float_rn(l);
        hi[a] = __ll2float_rn(h);
    }
}

__global__ void __launch_bounds__(256) k_render_flags(const fp_node* __restrict__ nodes, const uint32_t* d_num,
                                                      uint32_t cap, const fp_cube* cube_p, CamDev cam,
                                                      uint8_t* __restrict__ vis, uint32_t* diff)
{
    const uint32_t M = *d_num < cap ? *d_num : cap;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const fp_node nd = nodes[i];
    const fp_cube cb = *cube_p;
    float lo[3], hi[3];
    node_box(cb, nd.level, nd.key, lo, hi);
    bool all_l = true, all_r = true, all_b = true, all_t = true, all_n = true, all_f = true, behind = false;
    bool any = false;
    float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
    for (int k = 0; k < 8; ++k) {
        const Clip c = clip_of(cam, (k & 4) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 1) ? hi[2] : lo[2]);
        all_l &= c.x < -c.w;
        all_r &= c.x > c.w;
        all_b &= c.y < -c.w;
        all_t &= c.y > c.w;
        all_n &= c.z < 0.f;
        all_f &= c.z > c.w;
        if (c.w <= 0.f) {
            behind = true;
        } else {
            const float sx = screen(__fdiv_rn(c.x, c.w), cam.W), sy = screen(__fdiv_rn(c.y, c.w), cam.H);
            if (!any || sx < x0) x0 = sx;
            if (!any || sx > x1) x1 = sx;
            if (!any || sy < y0) y0 = sy;
            if (!any || sy > y1) y1 = sy;
            any = true;
        }
    }
    const bool visible = !(all_l || all_r || all_b || all_t || all_n || all_f);
    const float ex = __fsub_rn(x1, x0), ey = __fsub_rn(y1, y0);
    const float size = ex > ey ? ex : ey;
    const bool refine = visible && !nd.is_leaf && (behind || size > cam.minpx);
    vis[i] = visible ? 1 : 0;
    if (!refine && nd.n_desc && nd.n_desc < M - i) {   // the subtree below is not drawn
        atomicAdd(&diff[i + 1], 1u);
        atomicAdd(&diff[i + nd.n_desc + 1], 0xFFFFFFFFu);
    }
}

__global__ void k_min_u32(const uint32_t* a, uint32_t cap, uint32_t* out) { *out = *a < cap ? *a : cap; }

__global__ void k_render_mark(const uint8_t* vis, const uint32_t* diff, const uint32_t* ex, const uint32_t* d_num,
                              uint32_t cap, uint32_t* sel)
{
    const uint32_t M = *d_num < cap ? *d_num : cap;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) sel[i] = vis[i] && ex[i] + diff[i] == 0u ? 1u : 0u;
}

__global__ void k_render_write(const fp_node* __restrict__ nodes, const uint32_t* sel, const uint32_t* pos,
                               const uint32_t* d_num, uint32_t cap, uint32_t* ids, uint32_t* own)
{
    const uint32_t M = *d_num < cap ? *d_num : cap;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && sel[i]) {
        ids[pos[i]] = i;
        if (own) own[pos[i]] = nodes[i].n_own;
    }
}

__global__ void k_gather_own(const fp_node* __restrict__ nodes, const uint32_t* ids, const uint32_t* d_nsel,
                             uint32_t cap, uint32_t* own)
{
    const uint32_t S = *d_nsel < cap ? *d_nsel : cap;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < S) own[k] = nodes[ids[k]].n_own;
}

// one thread per point of the drawn nodes; its node by binary search over the
// drawn nodes' point starts (the last start <= p: empty nodes share starts)
__global__ void __launch_bounds__(256) k_raster(const fp_node* __restrict__ nodes, const uint32_t* __restrict__ ids,
                                                const uint64_t* __restrict__ pstart, const uint32_t* d_nsel,
                                                uint32_t cap, const uint64_t* d_total, const int4* __restrict__ fin,
                                                uint64_t n, CamDev cam, unsigned long long* fb)
{
    const uint32_t S = *d_nsel < cap ? *d_nsel : cap;
    const uint64_t P = *d_total;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = 0, b = S;
        while (a < b) {
            const uint32_t m = (a + b) >> 1;
            if (pstart[m] <= p) a = m + 1;
            else b = m;
        }
        const uint32_t k = a - 1;
        const uint64_t at = nodes[ids[k]].first + (p - pstart[k]);
        if (at >= n) continue;   // a node table of another point array
        const int4 q = __ldg(fin + at);
        const Clip c = clip_of(cam, __int2float_rn(q.x), __int2float_rn(q.y), __int2float_rn(q.z));
        if (!(c.w > 0.f) || c.x < -c.w || c.x > c.w || c.y < -c.w || c.y > c.w || c.z < 0.f || c.z > c.w) continue;
        const float sx = screen(__fdiv_rn(c.x, c.w), cam.W), sy = screen(__fdiv_rn(c.y, c.w), cam.H);
        const uint32_t px = min((uint32_t)floorf(sx), cam.w - 1), py = min((uint32_t)floorf(sy), cam.h - 1);
        const float depth = __fadd_rn(__fdiv_rn(c.z, c.w), 0.f);   // -0 -> +0
        const unsigned long long v = ((unsigned long long)__float_as_uint(depth) << 32) | (uint32_t)q.w;
        unsigned long long* px_word = &fb[(uint64_t)py * cam.w + px];
        if (v < __ldcg(px_word)) atomicMin(px_word, v);   // a pixel's value only falls: skip the hopeless

    }
}

}  // namespace

struct RenderBufs {
    uint8_t* vis;
    uint32_t *diff, *ex, *sel, *pos, *own, *tiles32, *num;
    uint64_t *pstart, *tiles64, *total;
};

static RenderBufs render_carve(const Workspace& ws, uint32_t cap)
{
    RenderBufs B;
    const uint64_t M = cap ? cap : 1;
    B.vis = ws.take<uint8_t>(M);
    B.diff = ws.take<uint32_t>(M + 1);
    B.ex = ws.take<uint32_t>(M + 1);
    B.sel = ws.take<uint32_t>(M);
    B.pos = ws.take<uint32_t>(M);
    B.own = ws.take<uint32_t>(M);
    B.tiles32 = ws.take<uint32_t>(kScanMaxTiles);
    B.num = ws.take<uint32_t>(2);
    B.pstart = ws.take<uint64_t>(M);
    B.tiles64 = ws.take<uint64_t>(kScanMaxTiles);
    B.total = ws.take<uint64_t>(1);
    return B;
}

size_t render_ws_bytes(uint32_t cap)
{
    Workspace dry;
    render_carve(dry, cap);
    return dry.used;
}

cudaError_t launch_select_nodes(const fp_node* nodes, const uint32_t* num_nodes, uint32_t cap, const fp_cube* cube,
                                const fp_camera& cam, uint32_t* ids, uint32_t* num_sel, uint64_t* num_points,
                                const Workspace& ws, cudaStream_t st)
{
    const RenderBufs B = render_carve(ws, cap);
    cudaError_t e;
    if ((e = cudaMemsetAsync(B.diff, 0, ((size_t)cap + 1) * sizeof(uint32_t), st))) return e;
    const unsigned grid = (cap + 255) / 256 ? (cap + 255) / 256 : 1;
    k_min_u32<<<1, 1, 0, st>>>(num_nodes, cap, B.num);   // the nodes at hand: at most cap
    k_render_flags<<<grid, 256, 0, st>>>(nodes, B.num, cap, cube, cam_dev(cam), B.vis, B.diff);
    if ((e = scan_exclusive<uint32_t, uint32_t>(B.diff, B.ex, cap, B.num, B.tiles32, (uint32_t*)nullptr,
                                                (uint32_t*)nullptr, st)))
        return e;
    k_render_mark<<<grid, 256, 0, st>>>(B.vis, B.diff, B.ex, B.num, cap, B.sel);
    if ((e = scan_exclusive<uint32_t, uint32_t>(B.sel, B.pos, cap, B.num, B.tiles32, num_sel, (uint32_t*)nullptr,
                                                st)))
        return e;
    k_render_write<<<grid, 256, 0, st>>>(nodes, B.sel, B.pos, B.num, cap, ids, B.own);
    if ((e = scan_exclusive<uint32_t, uint64_t>(B.own, B.pstart, cap, num_sel, B.tiles64, num_points,
                                                (uint64_t*)nullptr, st)))
        return e;
    return cudaGetLastError();
}

cudaError_t launch_rasterize(const fp_node* nodes, const uint32_t* ids, const uint32_t* num_sel, uint32_t cap,
                             const fp_point* fin, uint64_t n, const fp_camera& cam, unsigned long long* fb,
                             const Workspace& ws, int num_sms, cudaStream_t st)
{
    const RenderBufs B = render_carve(ws, cap);
    cudaError_t e;
    if ((e = cudaMemsetAsync(fb, 0xFF, (size_t)cam.width * cam.height * sizeof(unsigned long long), st))) return e;
    const unsigned grid = (cap + 255) / 256 ? (cap + 255) / 256 : 1;
    k_min_u32<<<1, 1, 0, st>>>(num_sel, cap, B.num);
    k_gather_own<<<grid, 256, 0, st>>>(nodes, ids, B.num, cap, B.own);
    if ((e = scan_exclusive<uint32_t, uint64_t>(B.own, B.pstart, cap, B.num, B.tiles64, B.total, (uint64_t*)nullptr,
                                                st)))
        return e;
    k_raster<<<num_sms * 8, 256, 0, st>>>(nodes, ids, B.pstart, B.num, cap, B.total,
                                          reinterpret_cast<const int4*>(fin), n, cam_dev(cam), fb);
    return cudaGetLastError();
}

}  // namespace fp
