// fp_internal.cuh -- host-side helpers shared by the translation units of
// libfastpoints: the workspace carve-up and the launch functions each unit
// exports to fp_api.cu.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include "fp_common.cuh"
#include "fp_scan.cuh"

namespace fp {

// Bump allocator over the caller's workspace; every piece is 256-byte aligned.
struct Workspace {
    char* base = nullptr;
    size_t bytes = 0;
    mutable size_t used = 0;
    int num_sms = 152;
    uint32_t* err = nullptr;   // device error word

    static constexpr size_t kAlign = 256;
    static size_t round(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
    static size_t bytes_for(std::initializer_list<size_t> parts)
    {
        size_t t = 0;
        for (size_t p : parts) t += round(p ? p : 1);
        return t;
    }
    template <typename T>
    T* take(size_t count) const
    {
        size_t b = round(count * sizeof(T) ? count * sizeof(T) : 1);
        char* p = base + used;
        used += b;
        return reinterpret_cast<T*>(p);
    }
};

// fp_api.cu
fp_status make_workspace(void* base, size_t bytes, size_t need, Workspace& ws);
// test hook of the bounded waits (fp_debug_withhold_publish): the tile whose
// publish the look-back passes withhold (0xFFFFFFFF: none) and their spin limit
void debug_wait_config(uint32_t* withhold_tile, uint32_t* spin_limit);
// kernel timing (fp_time_kernel): records the armed events around the launches of kernel `id`
void ktimer_mark(fp_kernel id, bool begin, cudaStream_t st);
struct KTimerScope {
    fp_kernel id;
    cudaStream_t st;
    KTimerScope(fp_kernel k, cudaStream_t s) : id(k), st(s) { ktimer_mark(id, true, st); }
    ~KTimerScope() { ktimer_mark(id, false, st); }
};

// fp_core.cu
cudaError_t launch_bounds_decimate(const fp_point* pts, uint64_t n, fp_cube* cube, bool bounds, bool decim,
                                   uint64_t first, uint32_t modulus, fp_point* out, uint64_t out_cap,
                                   uint64_t* out_count, const Workspace& ws, cudaStream_t st);
size_t bounds_ws_bytes(uint64_t n, int num_sms);

// fp_render.cu
size_t render_ws_bytes(uint32_t cap);
cudaError_t launch_select_nodes(const fp_node* nodes, const uint32_t* num_nodes, uint32_t cap, const fp_cube* cube,
                                const fp_camera& cam, uint32_t* ids, uint32_t* num_sel, uint64_t* num_points,
                                const Workspace& ws, cudaStream_t st);
cudaError_t launch_rasterize(const fp_node* nodes, const uint32_t* ids, const uint32_t* num_sel, uint32_t cap,
                             const fp_point* fin, uint64_t n, const fp_camera& cam, unsigned long long* fb,
                             const Workspace& ws, int num_sms, cudaStream_t st);
size_t spatial_ws_bytes(uint64_t n, int level, int num_sms);
cudaError_t launch_preview_spatial(const fp_point* pts, uint64_t n, const fp_cube* cube, int level, uint64_t first,
                                   fp_point* out, uint64_t out_cap, uint64_t* out_count, const Workspace& ws,
                                   cudaStream_t st);
cudaError_t launch_count(const fp_point* pts, uint64_t n, const fp_cube* cube, int g, uint32_t* counts,
                         bool accumulate, uint32_t* cells, const Workspace& ws, cudaStream_t st);
size_t merge_ws_bytes(int g);
cudaError_t launch_merge(const uint32_t* counts, int g, uint64_t T, fp_chunk* chunks, uint32_t* num_chunks,
                         uint32_t* lut, uint64_t* offsets, const Workspace& ws, cudaStream_t st);

// fp_sort.cu
size_t distribute_ws_bytes(uint64_t n, int g);
cudaError_t launch_distribute(const fp_point* pts, uint64_t n, const fp_cube* cube, int g, const uint32_t* lut,
                              const uint64_t* offsets, const uint32_t* num_chunks, fp_point* out, uint32_t* perm,
                              const Workspace& ws, cudaStream_t st, const uint32_t* cells = nullptr);

// fp_octree.cu
size_t octree_ws_bytes(uint64_t n, const fp_params& p);
size_t subsample_ws_bytes(uint64_t n, uint64_t node_cap);
uint64_t node_capacity_bound(uint64_t n, const fp_params& p);
cudaError_t launch_octree(const fp_point* sorted, const uint32_t* perm, uint64_t n, const fp_cube* cube,
                          const fp_chunk* chunks, const uint32_t* num_chunks, const uint64_t* offsets,
                          const uint32_t* counts, const fp_params& prm, fp_node* nodes, uint32_t node_cap,
                          uint32_t* num_nodes, fp_point* leaf_pts, uint32_t* leaf_perm, uint32_t* owner,
                          const Workspace& ws, cudaStream_t st);
// chunk groups of an out-of-core build (fp_ooc.cu)
struct NodeRec;                      // a node before preorder numbering (fp_octree.cu)
constexpr size_t kNodeRecBytes = 24;
struct OctGroup {
    const uint32_t* rec_counts;      // the group's points per level-g cell (0 outside the group)
    uint32_t leaf_base;              // position of the group's first point in the whole distributed array
    uint32_t* codes;                 // per group point: owner level, leaf level, level-g cell (code_make)
    NodeRec* deep;                   // nodes below level g, appended at *num_deep
    uint32_t deep_cap;
    uint32_t* num_deep;
};
cudaError_t launch_octree_impl(const fp_point* sorted, const uint32_t* perm, uint64_t n, const fp_cube* cube,
                               const fp_chunk* chunks, const uint32_t* num_chunks, const uint64_t* offsets,
                               const uint32_t* counts, const fp_params& prm, fp_node* nodes, uint32_t node_cap,
                               uint32_t* num_nodes, fp_point* leaf_pts, uint32_t* leaf_perm, uint32_t* owner,
                               const OctGroup* grp, const Workspace& ws, cudaStream_t st);
struct NodeTables {                  // lookups of the id resolution, kept between calls
    uint32_t* idxtab;                // node id of every (level <= g, key): (8^(g+1) - 1) / 7 + 8 entries
    uint64_t* starts;                // preorder position -> start key at max_level resolution
    uint8_t* slevel;                 // preorder position -> level
    uint32_t* ndesc;                 // preorder position -> subtree size - 1
    uint32_t* nown;                  // owned points per node (accumulated by the resolution)
    uint32_t* nnode;                 // node count
};
size_t nodes_ws_bytes(const fp_params& p, uint64_t rec_cap);
uint64_t upper_node_bound(const fp_params& p);
cudaError_t launch_octree_nodes(const uint32_t* counts, const fp_params& prm, NodeRec* recs, uint64_t rec_cap,
                                const uint32_t* num_deep, fp_node* nodes, uint32_t node_cap, uint32_t* num_nodes,
                                const NodeTables& T, const Workspace& ws, cudaStream_t st);
cudaError_t launch_octree_resolve(const fp_point* pts, uint64_t n, const fp_cube* cube, const uint32_t* codes,
                                  const NodeTables& T, const fp_params& prm,
                                  uint32_t* owner, const Workspace& ws, cudaStream_t st);
cudaError_t launch_node_first(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const uint32_t* nown,
                              uint64_t* first, uint32_t* nm, uint64_t* tiles64, cudaStream_t st);

cudaError_t launch_subsample(fp_node* nodes, const uint32_t* num_nodes, uint32_t node_cap, const fp_point* sorted,
                             const uint32_t* perm, const uint32_t* owner, uint64_t n, const fp_chunk* chunks,
                             const uint32_t* num_chunks, const uint64_t* offsets, fp_point* final_pts,
                             uint32_t* final_perm, const Workspace& ws, cudaStream_t st);

}  // namespace fp
