// fp_api.cu -- the extern "C" entry points declared in include/fastpoints.h:
// argument checks, workspace carve-up and launch order.  Each entry point cites
// the paper section of the stage it runs; the kernels live in fp_core.cu,
// fp_sort.cu and fp_octree.cu.
#include <atomic>
#include <cstring>
#include <mutex>
#include "fp_internal.cuh"

namespace fp {

// the bounded-wait test hook (fp_debug_withhold_publish)
static std::atomic<uint32_t> g_dbg_withhold{0xFFFFFFFFu};
static std::atomic<uint32_t> g_dbg_limit{kSpinLimit};

void debug_wait_config(uint32_t* withhold_tile, uint32_t* spin_limit)
{
    *withhold_tile = g_dbg_withhold.load(std::memory_order_acquire);
    *spin_limit = g_dbg_limit.load(std::memory_order_acquire);
}

// armed kernel of fp_time_kernel and the caller's events
static std::atomic<int> g_kt_id{0};
static cudaEvent_t g_kt_ev[2] = {nullptr, nullptr};

void ktimer_mark(fp_kernel id, bool begin, cudaStream_t st)
{
    if (g_kt_id.load(std::memory_order_acquire) != (int)id || id == FP_KERNEL_NONE) return;
    cudaEventRecord(g_kt_ev[begin ? 0 : 1], st);
}

// sticky error word of each device; kernels receive its address
static __device__ uint32_t g_error_word[2] = {0, 0};   // status bits, check sites

struct DeviceInfo {
    bool ready = false;
    int num_sms = 0;
    uint32_t* err = nullptr;
};

static std::mutex g_mu;
static DeviceInfo g_dev[64];

// Per-device set-up (SM count, device address of the error word).  Runs on the
// first call made with each device current.
static fp_status device_info(DeviceInfo& out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo& d = g_dev[dev];
    if (!d.ready) {
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FP_ERR_CUDA;
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return FP_ERR_CUDA;
        d.err = static_cast<uint32_t*>(p);
        d.ready = true;
    }
    out = d;
    return FP_OK;
}

static fp_status make_ws(void* base, size_t bytes, size_t need, Workspace& ws)
{
    if (need > 0 && (base == nullptr || bytes < need)) return FP_ERR_WORKSPACE;
    DeviceInfo d;
    fp_status s = device_info(d);
    if (s != FP_OK) return s;
    ws.base = static_cast<char*>(base);
    ws.bytes = bytes;
    ws.used = 0;
    ws.num_sms = d.num_sms;
    ws.err = d.err;
    return FP_OK;
}

static fp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FP_OK : FP_ERR_CUDA; }

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr uint64_t kMaxPoints = 1ull << 30;

fp_status check_params(const fp_params* p)
{
    if (!p) return FP_ERR_INVALID;
    if (p->grid_log2 < 1 || p->grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    if (p->sub_log2 < p->grid_log2) return FP_ERR_UNSUPPORTED;
    if (p->max_level < p->grid_log2 || p->max_level + p->sub_log2 > 22) return FP_ERR_UNSUPPORTED;
    if (p->node_capacity < 1 || p->chunk_threshold < p->node_capacity) return FP_ERR_UNSUPPORTED;
    if (p->decim_modulus < 1) return FP_ERR_UNSUPPORTED;
    return FP_OK;
}

// workspace view over a caller-provided (or library-held) buffer
fp_status make_workspace(void* base, size_t bytes, size_t need, Workspace& ws) { return make_ws(base, bytes, need, ws); }

}  // namespace fp

using namespace fp;

extern "C" {

const char* fp_status_string(fp_status s)
{
    switch (s) {
    case FP_OK: return "ok";
    case FP_ERR_INVALID: return "invalid argument";
    case FP_ERR_ALIGN: return "point array not 16-byte aligned";
    case FP_ERR_TOO_LARGE: return "too many points (n >= 2^30)";
    case FP_ERR_NOMEM: return "out of memory";
    case FP_ERR_WORKSPACE: return "workspace too small";
    case FP_ERR_TIMEOUT: return "bounded device wait ran out";
    case FP_ERR_CUDA: return "CUDA error";
    case FP_ERR_UNSUPPORTED: return "unsupported parameters";
    case FP_ERR_CAPACITY: return "output capacity exceeded";
    case FP_ERR_IO: return "file read or write failed";
    }
    return "unknown status";
}

size_t fp_workspace_size(fp_stage stage, uint64_t n, const fp_params* prm)
{
    int sms = 152;
    {
        DeviceInfo d;
        if (device_info(d) == FP_OK) sms = d.num_sms;
    }
    int g = prm ? (int)prm->grid_log2 : 7;
    if (g < 1 || g > 7) g = 7;
    switch (stage) {
    case FP_STAGE_BOUNDS:
    case FP_STAGE_DECIMATE:
    case FP_STAGE_BOUNDS_DECIMATE: return bounds_ws_bytes(n, sms);
    case FP_STAGE_COUNT: return 0;
    case FP_STAGE_MERGE: return merge_ws_bytes(g);
    case FP_STAGE_DISTRIBUTE: return distribute_ws_bytes(n, g);
    case FP_STAGE_OCTREE: return prm ? octree_ws_bytes(n, *prm) : 0;
    case FP_STAGE_SUBSAMPLE: return prm ? subsample_ws_bytes(n, node_capacity_bound(n, *prm)) : 0;
    case FP_STAGE_PREVIEW_SPATIAL: return spatial_ws_bytes(n, g, sms);
    }
    return 0;
}

uint32_t fp_node_capacity_bound(uint64_t n, const fp_params* prm)
{
    if (!prm || check_params(prm) != FP_OK) return 0;
    uint64_t b = node_capacity_bound(n, *prm);
    return b > 0xFFFFFFF0ull ? 0xFFFFFFF0u : (uint32_t)b;
}

fp_status fp_debug_withhold_publish(uint32_t tile, uint32_t spin_limit)
{
    if (tile != 0xFFFFFFFFu && spin_limit == 0) return FP_ERR_INVALID;
    g_dbg_limit.store(tile == 0xFFFFFFFFu ? kSpinLimit : spin_limit, std::memory_order_release);
    g_dbg_withhold.store(tile, std::memory_order_release);
    return FP_OK;
}

fp_status fp_time_kernel(fp_kernel k, cudaEvent_t start, cudaEvent_t stop)
{
    if ((int)k < (int)FP_KERNEL_NONE || (int)k > (int)FP_KERNEL_STITCH) return FP_ERR_INVALID;
    if (k != FP_KERNEL_NONE && (!start || !stop)) return FP_ERR_INVALID;
    g_kt_id.store(0, std::memory_order_release);
    g_kt_ev[0] = start;
    g_kt_ev[1] = stop;
    g_kt_id.store((int)k, std::memory_order_release);
    return FP_OK;
}

fp_status fp_get_device_error_sites(cudaStream_t stream, uint32_t* h_sites)
{
    if (!h_sites) return FP_ERR_INVALID;
    DeviceInfo d;
    fp_status s = device_info(d);
    if (s != FP_OK) return s;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, d.err + 1, sizeof(v), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return FP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FP_ERR_CUDA;
    *h_sites = v;
    return FP_OK;
}

fp_status fp_get_device_error(cudaStream_t stream, uint32_t* h_bits, int clear)
{
    if (!h_bits) return FP_ERR_INVALID;
    DeviceInfo d;
    fp_status s = device_info(d);
    if (s != FP_OK) return s;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, d.err, sizeof(v), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return FP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FP_ERR_CUDA;
    if (clear) {
        if (cudaMemsetAsync(d.err, 0, 2 * sizeof(uint32_t), stream) != cudaSuccess) return FP_ERR_CUDA;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return FP_ERR_CUDA;
    }
    *h_bits = v;
    return FP_OK;
}

// Sec. 4.4: extent of the cloud
fp_status fp_bounds(const fp_point* d_pts, uint64_t n, fp_cube* d_cube, void* d_ws, size_t ws_bytes,
                    cudaStream_t stream)
{
    if (!d_cube || (n && !d_pts)) return FP_ERR_INVALID;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && !aligned16(d_pts)) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_BOUNDS, n, nullptr), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_bounds_decimate(d_pts, n, d_cube, true, false, 0, 1, nullptr, 0, nullptr, ws, stream));
}

size_t fp_render_workspace_size(uint32_t node_cap) { return render_ws_bytes(node_cap); }

static bool camera_ok(const fp_camera* c)
{
    return c && c->width >= 1 && c->height >= 1 && c->width <= 16384 && c->height <= 16384;
}

// Sec. 4.5: the traversal that picks the nodes to draw
fp_status fp_select_nodes(const fp_node* d_nodes, const uint32_t* d_num_nodes, uint32_t node_cap,
                          const fp_cube* d_cube, const fp_camera* h_cam, uint32_t* d_selected,
                          uint32_t* d_num_selected, uint64_t* d_num_points, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream)
{
    if (!d_num_nodes || !d_cube || !d_num_selected || !d_num_points || !camera_ok(h_cam) ||
        (node_cap && (!d_nodes || !d_selected)))
        return FP_ERR_INVALID;
    if (node_cap > (1u << 23)) return FP_ERR_UNSUPPORTED;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, render_ws_bytes(node_cap), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_select_nodes(d_nodes, d_num_nodes, node_cap, d_cube, *h_cam, d_selected,
                                           d_num_selected, d_num_points, ws, stream));
}

// Sec. 4.5: the selected nodes' points drawn, nearest per pixel
fp_status fp_rasterize(const fp_node* d_nodes, const uint32_t* d_selected, const uint32_t* d_num_selected,
                       uint32_t node_cap, const fp_point* d_final, uint64_t n, const fp_camera* h_cam,
                       uint64_t* d_framebuffer, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_num_selected || !d_framebuffer || !camera_ok(h_cam) || (node_cap && (!d_nodes || !d_selected || !d_final)))
        return FP_ERR_INVALID;
    if (node_cap > (1u << 23)) return FP_ERR_UNSUPPORTED;
    if (d_final && !aligned16(d_final)) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, render_ws_bytes(node_cap), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_rasterize(d_nodes, d_selected, d_num_selected, node_cap, d_final, n, *h_cam,
                                        reinterpret_cast<unsigned long long*>(d_framebuffer), ws, ws.num_sms, stream));
}

uint32_t fp_preview_modulus(uint64_t n, uint64_t target)
{
    if (target == 0 || n <= target) return 1;
    const uint64_t m = (n + target - 1) / target;
    return m > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)m;
}

// Sec. 6 (future work): spatially constrained random preview
fp_status fp_preview_spatial(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t level,
                             uint64_t first_index, fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count,
                             void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_out_count || !d_cube || (n && (!d_pts || (out_cap && !d_out)))) return FP_ERR_INVALID;
    if (level < 1 || level > 7) return FP_ERR_UNSUPPORTED;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if ((n && !aligned16(d_pts)) || (d_out && !aligned16(d_out))) return FP_ERR_ALIGN;
    fp_params p{};
    p.grid_log2 = level;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_PREVIEW_SPATIAL, n, &p), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_preview_spatial(d_pts, n, d_cube, (int)level, first_index, d_out, out_cap, d_out_count,
                                              ws, stream));
}

// Sec. 3 / Sec. 4.2: uniform preview, made index-deterministic by a hash
fp_status fp_decimate(const fp_point* d_pts, uint64_t n, uint64_t first_index, uint32_t modulus, fp_point* d_out,
                      uint64_t out_cap, uint64_t* d_out_count, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_out_count || (n && (!d_pts || (out_cap && !d_out))) || modulus < 1) return FP_ERR_INVALID;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if ((n && !aligned16(d_pts)) || (d_out && !aligned16(d_out))) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_DECIMATE, n, nullptr), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_bounds_decimate(d_pts, n, nullptr, false, true, first_index, modulus, d_out, out_cap,
                                              d_out_count, ws, stream));
}

fp_status fp_bounds_decimate(const fp_point* d_pts, uint64_t n, fp_cube* d_cube, uint64_t first_index,
                             uint32_t modulus, fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count, void* d_ws,
                             size_t ws_bytes, cudaStream_t stream)
{
    if (!d_cube || !d_out_count || (n && (!d_pts || (out_cap && !d_out))) || modulus < 1) return FP_ERR_INVALID;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if ((n && !aligned16(d_pts)) || (d_out && !aligned16(d_out))) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_BOUNDS_DECIMATE, n, nullptr), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_bounds_decimate(d_pts, n, d_cube, true, true, first_index, modulus, d_out, out_cap,
                                              d_out_count, ws, stream));
}

// Sec. 4.4: points per cell of the chunking grid
fp_status fp_count(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2, uint32_t* d_counts,
                   int accumulate, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_cube || !d_counts || (n && !d_pts)) return FP_ERR_INVALID;
    if (grid_log2 < 1 || grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && !aligned16(d_pts)) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, 0, ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_count(d_pts, n, d_cube, (int)grid_log2, d_counts, accumulate != 0, nullptr, ws, stream));
}

fp_status fp_count_cells(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2,
                         uint32_t* d_counts, int accumulate, uint32_t* d_cells, void* d_ws, size_t ws_bytes,
                         cudaStream_t stream)
{
    if (!d_cube || !d_counts || (n && (!d_pts || !d_cells))) return FP_ERR_INVALID;
    if (grid_log2 < 1 || grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && !aligned16(d_pts)) return FP_ERR_ALIGN;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, 0, ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_count(d_pts, n, d_cube, (int)grid_log2, d_counts, accumulate != 0, d_cells, ws, stream));
}

// Fig. "octree": chunks are nodes of the global tree holding at most T points
fp_status fp_merge_chunks(const uint32_t* d_counts, uint32_t grid_log2, uint64_t threshold, fp_chunk* d_chunks,
                          uint32_t* d_num_chunks, uint32_t* d_lut, uint64_t* d_offsets, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream)
{
    if (!d_counts || !d_chunks || !d_num_chunks || !d_lut || !d_offsets || threshold < 1) return FP_ERR_INVALID;
    if (grid_log2 < 1 || grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    Workspace ws;
    fp_params p{};
    p.grid_log2 = grid_log2;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_MERGE, 0, &p), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_merge(d_counts, (int)grid_log2, threshold, d_chunks, d_num_chunks, d_lut, d_offsets, ws,
                                    stream));
}

// Sec. 4.4: stable scatter of the points into their chunks
fp_status fp_distribute(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2,
                        const uint32_t* d_lut, const uint64_t* d_offsets, const uint32_t* d_num_chunks,
                        fp_point* d_out, uint32_t* d_perm, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_cube || !d_lut || !d_offsets || !d_num_chunks || (n && (!d_pts || !d_out))) return FP_ERR_INVALID;
    if (grid_log2 < 1 || grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && (!aligned16(d_pts) || !aligned16(d_out))) return FP_ERR_ALIGN;
    if (n && d_pts == d_out) return FP_ERR_INVALID;
    Workspace ws;
    fp_params p{};
    p.grid_log2 = grid_log2;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_DISTRIBUTE, n, &p), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_distribute(d_pts, n, d_cube, (int)grid_log2, d_lut, d_offsets, d_num_chunks, d_out,
                                         d_perm, ws, stream));
}

fp_status fp_distribute_cells(const fp_point* d_pts, const uint32_t* d_cells, uint64_t n, const fp_cube* d_cube,
                              uint32_t grid_log2, const uint32_t* d_lut, const uint64_t* d_offsets,
                              const uint32_t* d_num_chunks, fp_point* d_out, uint32_t* d_perm, void* d_ws,
                              size_t ws_bytes, cudaStream_t stream)
{
    if (!d_cube || !d_lut || !d_offsets || !d_num_chunks || (n && (!d_pts || !d_out || !d_cells)))
        return FP_ERR_INVALID;
    if (grid_log2 < 1 || grid_log2 > 7) return FP_ERR_UNSUPPORTED;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && (!aligned16(d_pts) || !aligned16(d_out))) return FP_ERR_ALIGN;
    if (n && d_pts == d_out) return FP_ERR_INVALID;
    Workspace ws;
    fp_params p{};
    p.grid_log2 = grid_log2;
    fp_status s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_DISTRIBUTE, n, &p), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_distribute(d_pts, n, d_cube, (int)grid_log2, d_lut, d_offsets, d_num_chunks, d_out,
                                         d_perm, ws, stream, d_cells));
}

// Sec. 4.4 / Fig. "octree": local octrees of the chunks, stitched, and LOD selection
fp_status fp_build_chunk_octree(const fp_point* d_sorted, const uint32_t* d_perm, uint64_t n, const fp_cube* d_cube,
                                const fp_chunk* d_chunks, const uint32_t* d_num_chunks, const uint64_t* d_offsets,
                                const uint32_t* d_counts, const fp_params* h_prm, fp_node* d_nodes,
                                uint32_t node_cap, uint32_t* d_num_nodes, fp_point* d_leaf_pts,
                                uint32_t* d_leaf_perm, uint32_t* d_owner, void* d_ws, size_t ws_bytes,
                                cudaStream_t stream)
{
    fp_status s = check_params(h_prm);
    if (s != FP_OK) return s;
    if (!d_cube || !d_chunks || !d_num_chunks || !d_offsets || !d_counts || !d_num_nodes || (node_cap && !d_nodes) ||
        (n && (!d_sorted || !d_perm || !d_owner)))
        return FP_ERR_INVALID;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if ((n && !aligned16(d_sorted)) || (d_leaf_pts && !aligned16(d_leaf_pts))) return FP_ERR_ALIGN;
    Workspace ws;
    s = make_ws(d_ws, ws_bytes, fp_workspace_size(FP_STAGE_OCTREE, n, h_prm), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_octree(d_sorted, d_perm, n, d_cube, d_chunks, d_num_chunks, d_offsets, d_counts, *h_prm,
                                     d_nodes, node_cap, d_num_nodes, d_leaf_pts, d_leaf_perm, d_owner, ws, stream));
}

// Sec. 4.4: final layout, points of nodes above the chunks merged across chunks
fp_status fp_subsample(fp_node* d_nodes, const uint32_t* d_num_nodes, uint32_t node_cap, const fp_point* d_sorted,
                       const uint32_t* d_perm, const uint32_t* d_owner, uint64_t n, const fp_chunk* d_chunks,
                       const uint32_t* d_num_chunks, const uint64_t* d_offsets, fp_point* d_final,
                       uint32_t* d_final_perm, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!d_num_nodes || (node_cap && !d_nodes) ||
        (n && (!d_sorted || !d_perm || !d_owner || !d_chunks || !d_num_chunks || !d_offsets || !d_final ||
               !d_final_perm)))
        return FP_ERR_INVALID;
    if (n >= kMaxPoints) return FP_ERR_TOO_LARGE;
    if (n && (!aligned16(d_sorted) || !aligned16(d_final))) return FP_ERR_ALIGN;
    if (node_cap > (1u << 23)) return FP_ERR_UNSUPPORTED;
    Workspace ws;
    fp_status s = make_ws(d_ws, ws_bytes, subsample_ws_bytes(n, node_cap), ws);
    if (s != FP_OK) return s;
    return cuda_status(launch_subsample(d_nodes, d_num_nodes, node_cap, d_sorted, d_perm, d_owner, n, d_chunks,
                                        d_num_chunks, d_offsets, d_final, d_final_perm, ws, stream));
}

}  // extern "C"
