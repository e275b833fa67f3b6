// fp_batch.cu -- fp_build_batched: many clouds per call.  Every cloud runs the
// plain entry points in order (bounds + preview, count, merge, distribute,
// chunk octrees, subsample) on one of a set of library-owned streams ("lanes")
// forked from and joined back into the caller's stream with events, so that the
// many small launches of small clouds overlap and the whole batch is one unit
// for CUDA graph capture.
#include <algorithm>
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

// the plain calls, in order, on one stream
fp_status run_cloud(const fp_cloud_desc& c, char* ws, size_t ws_bytes, cudaStream_t st)
{
    fp_status s;
    const uint32_t g = c.prm.grid_log2;
    if ((s = fp_bounds_decimate(c.d_pts, c.n, c.d_cube, 0, c.prm.decim_modulus, c.d_preview, c.preview_cap,
                                c.d_preview_count, ws, ws_bytes, st)))
        return s;
    if ((s = fp_count(c.d_pts, c.n, c.d_cube, g, c.d_counts, 0, ws, ws_bytes, st))) return s;
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

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

size_t fp_batch_workspace_size(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes)
{
    if (!h_clouds || nlanes < 1 || nlanes > FP_MAX_LANES) return 0;
    std::vector<int> lane = assign(h_clouds, ncloud, nlanes);
    std::vector<size_t> need(nlanes, 0);
    for (uint32_t i = 0; i < ncloud; ++i) need[lane[i]] = std::max(need[lane[i]], cloud_ws(h_clouds[i]));
    size_t t = 0;
    for (size_t w : need) t += w;
    return t;
}

fp_status fp_build_batched(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes, void* d_ws,
                           size_t ws_bytes, cudaStream_t stream)
{
    if ((ncloud && !h_clouds) || nlanes < 1 || nlanes > FP_MAX_LANES) return FP_ERR_INVALID;
    for (uint32_t i = 0; i < ncloud; ++i) {
        fp_status s = check_cloud(h_clouds[i]);
        if (s != FP_OK) return s;
    }
    if (ncloud == 0) return FP_OK;
    const size_t need_total = fp_batch_workspace_size(h_clouds, ncloud, nlanes);
    if (need_total && (!d_ws || ws_bytes < need_total)) return FP_ERR_WORKSPACE;
    std::vector<int> lane = assign(h_clouds, ncloud, nlanes);
    std::vector<size_t> need(nlanes, 0), base(nlanes, 0);
    for (uint32_t i = 0; i < ncloud; ++i) need[lane[i]] = std::max(need[lane[i]], cloud_ws(h_clouds[i]));
    for (uint32_t l = 1; l < nlanes; ++l) base[l] = base[l - 1] + need[l - 1];

    std::lock_guard<std::mutex> lk(g_lane_mu);
    Lanes* L = nullptr;
    fp_status s = lanes_of_device(L);
    if (s != FP_OK) return s;
    if (cudaEventRecord(L->fork, stream) != cudaSuccess) return FP_ERR_CUDA;
    for (uint32_t l = 0; l < nlanes; ++l)
        if (cudaStreamWaitEvent(L->s[l], L->fork, 0) != cudaSuccess) return FP_ERR_CUDA;
    // clouds in descriptor order within each lane
    fp_status first_err = FP_OK;
    for (uint32_t i = 0; i < ncloud && first_err == FP_OK; ++i) {
        const int l = lane[i];
        first_err = run_cloud(h_clouds[i], static_cast<char*>(d_ws) + base[l], need[l], L->s[l]);
    }
    // join every lane, also after an error, so the caller's stream never runs ahead of enqueued work
    for (uint32_t l = 0; l < nlanes; ++l) {
        if (cudaEventRecord(L->join[l], L->s[l]) != cudaSuccess) return FP_ERR_CUDA;
        if (cudaStreamWaitEvent(stream, L->join[l], 0) != cudaSuccess) return FP_ERR_CUDA;
    }
    return first_err;
}

}  // extern "C"
