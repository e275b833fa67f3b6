/*
 * fastpoints.h -- C ABI of the GB300 (sm_103a) octree-construction library.
 *
 * The library builds, on one GPU, the structure FastPoints (arxiv 2302.05002)
 * needs before it can render a large unprocessed cloud: an immediate decimated
 * preview (Sec. 3, Sec. 4.2) and a shallow level-of-detail octree built by the
 * chunk -> index -> stitch method the paper adopts (Sec. 2.2, Sec. 4.4,
 * Fig. "octree").  The calls follow those stages:
 *
 *   fp_bounds              cube of the cloud                    (Sec. 4.4, extent)
 *   fp_decimate            hash-uniform preview                 (Sec. 3, Sec. 4.2)
 *   fp_preview_spatial     one random point per occupied cell   (Sec. 6, proposed sampler)
 *   fp_count               points per cell of the 2^g grid      (Sec. 4.4, "sorted into chunks")
 *   fp_merge_chunks        cells merged into chunks under T     (Fig. "octree": chunk = node of the tree)
 *   fp_distribute          stable scatter of points into chunks (Sec. 4.4, Fig. "octree")
 *   fp_build_chunk_octree  local octrees of all chunks, stitched,
 *                          and the LOD node that keeps each point (Sec. 4.4, Abstract "shallow octree")
 *   fp_subsample           final LOD layout of the points        (Sec. 4.4, "stitched into a global octree")
 *
 * Conventions (all calls):
 *   - Every pointer named d_* is device memory owned by the caller; h_* is host
 *     memory.  The library never allocates device memory: scratch space is the
 *     caller's workspace (d_ws, ws_bytes), sized by fp_workspace_size().
 *     Workspace contents need not be initialised and are not preserved.
 *   - Calls are asynchronous on `stream` and never synchronise the host.
 *     Counts produced on the device (number of chunks, nodes, preview points)
 *     are written to device memory.
 *   - Argument errors are detected on the host and returned at once; nothing is
 *     enqueued then.  Errors found on the device (an output capacity exceeded,
 *     a bounded wait that ran out) are OR-ed into a sticky per-device error word
 *     read with fp_get_device_error(); the affected outputs are then undefined.
 *   - n == 0 is valid and gives empty outputs.
 *   - Limits: n < 2^30; 1 <= grid_log2 <= 7; grid_log2 <= sub_log2;
 *     grid_log2 <= max_level; max_level + sub_log2 <= 22;
 *     1 <= node_capacity <= chunk_threshold; decim_modulus >= 1.
 *   - Point records must be 16-byte aligned.
 *   - Every kernel is CUDA for sm_103a; there is no CPU fallback.  Without a
 *     usable device the calls return FP_ERR_CUDA.
 *
 * Outputs are exact (integer arithmetic only) and identical from run to run.
 */
#ifndef FASTPOINTS_H
#define FASTPOINTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t;
typedef struct CUevent_st* cudaEvent_t;

/* One point: integer position and 8-bit colour, 16 bytes. */
typedef struct { int32_t x, y, z; uint8_t r, g, b, a; } fp_point;

/* Bounding cube: origin o = per-axis minimum, mx = per-axis maximum,
 * side S = max_a(mx_a - o_a) + 1 (1 <= S <= 2^32; S == 0 for an empty cloud). */
typedef struct { int32_t o[3]; int32_t mx[3]; uint64_t S; } fp_cube;

/* A chunk: node (level, Morton key at that level) of the count grid with its
 * number of points. */
typedef struct { uint64_t key; uint32_t count; uint32_t level; } fp_chunk;

/* A node of the octree, nodes stored in preorder (parent first, children in
 * Morton digit order).  Node i's subtree is nodes [i, i + n_desc].
 *   key        Morton key of the node's cell at `level` (3*level bits)
 *   first      start of the points the node keeps, in the final array
 *   leaf_first start of the subtree's points in the leaf-grouped array
 *   count      points in the subtree
 *   n_own      points the node keeps after LOD subsampling
 *   child_mask bit c set iff child with digit c exists (x bit = 4, y = 2, z = 1) */
typedef struct {
    uint64_t key, first, leaf_first;
    uint32_t count, n_own, n_desc;
    uint8_t level, child_mask, is_leaf, pad;
} fp_node;

/* Build parameters.
 *   grid_log2       g: count grid of 2^g cells per axis (the paper's chunking grid)
 *   sub_log2        s: an inner node at level L keeps one point per occupied
 *                   cell of the level-(L+s) grid (2^s cells per axis per node)
 *   max_level       deepest node level (root = 0)
 *   decim_modulus   preview keeps index i iff splitmix64(i) % decim_modulus == 0
 *   chunk_threshold T: most points in a chunk, unless it is one finest cell
 *   node_capacity   C: a node with more than C points is split (below max_level) */
typedef struct {
    uint32_t grid_log2, sub_log2, max_level, decim_modulus;
    uint64_t chunk_threshold, node_capacity;
} fp_params;

typedef enum {
    FP_OK = 0,
    FP_ERR_INVALID = 1,      /* a null pointer where one is required, or bad parameters */
    FP_ERR_ALIGN = 2,        /* a point array is not 16-byte aligned */
    FP_ERR_TOO_LARGE = 3,    /* n >= 2^30 */
    FP_ERR_NOMEM = 4,        /* reserved for callers' allocators */
    FP_ERR_WORKSPACE = 5,    /* ws_bytes smaller than fp_workspace_size() */
    FP_ERR_TIMEOUT = 6,      /* device word: a bounded inter-block wait ran out */
    FP_ERR_CUDA = 7,         /* a CUDA call failed (no device, launch error) */
    FP_ERR_UNSUPPORTED = 8,  /* parameters outside the limits above */
    FP_ERR_CAPACITY = 9,     /* device word: an output array was too small */
    FP_ERR_IO = 10           /* a file could not be opened, read or written */
} fp_status;

typedef enum {
    FP_STAGE_BOUNDS = 0,
    FP_STAGE_DECIMATE = 1,
    FP_STAGE_BOUNDS_DECIMATE = 2,
    FP_STAGE_COUNT = 3,
    FP_STAGE_MERGE = 4,
    FP_STAGE_DISTRIBUTE = 5,
    FP_STAGE_OCTREE = 6,
    FP_STAGE_SUBSAMPLE = 7,
    FP_STAGE_PREVIEW_SPATIAL = 8   /* prm->grid_log2 is the sampler's level (NULL: level 7) */
} fp_stage;

/* Bytes of workspace a stage needs for n points with these parameters
 * (prm may be NULL for the stages before the octree).  For FP_STAGE_SUBSAMPLE
 * the size assumes node_cap == fp_node_capacity_bound(n, prm). */
size_t fp_workspace_size(fp_stage stage, uint64_t n, const fp_params* prm);

/* An upper bound on the number of octree nodes of any cloud of n points under
 * these parameters: a node_cap for fp_build_chunk_octree / fp_subsample that can
 * never overflow (0 for invalid parameters). */
uint32_t fp_node_capacity_bound(uint64_t n, const fp_params* prm);

const char* fp_status_string(fp_status s);

/* Sticky device error word of the current device (bits (1u << status)); the
 * call synchronises `stream` and clears the word when `clear` is nonzero. */
fp_status fp_get_device_error(cudaStream_t stream, uint32_t* h_bits, int clear);

/* Which of the library's capacity and consistency checks raised FP_ERR_CAPACITY
 * since the device error word was last cleared: one bit per check site (an
 * output array too small, or inputs that contradict each other, such as a
 * count grid that is not the grid of the points).  For diagnosis; synchronises
 * `stream`; cleared together with the error word by fp_get_device_error(). */
fp_status fp_get_device_error_sites(cudaStream_t stream, uint32_t* h_sites);

/* Test hook of the bounded waits.  The radix passes (fp_distribute with more
 * than 2048 chunks, the sorts of the octree and subsample stages) find each
 * tile's output offsets by a decoupled look-back over the earlier tiles'
 * published counts; every such wait gives up after a bounded number of
 * rounds, raises FP_ERR_TIMEOUT in the device error word and lets the kernel
 * finish.  After fp_debug_withhold_publish(tile, spin_limit), tile `tile` of
 * every later radix pass publishes nothing and the waits give up after
 * spin_limit rounds, so the tile after it times out (its call's outputs are
 * then undefined).  tile = 0xFFFFFFFF restores normal operation (and the
 * default limit).  For tests only; process-wide; spin_limit >= 1. */
fp_status fp_debug_withhold_publish(uint32_t tile, uint32_t spin_limit);

/* Kernel timing for profiling.  The library's main kernels, by stage:
 *   FP_KERNEL_BOUNDS_DECIMATE  k_bounds_decimate (fp_bounds, fp_decimate, fp_bounds_decimate)
 *   FP_KERNEL_COUNT            k_count (fp_count)
 *   FP_KERNEL_DISTRIBUTE       the stable scatter of fp_distribute (every launch of it)
 *   FP_KERNEL_CELL_GROUP       k_cell_scatter: points grouped by count-grid cell (fp_build_chunk_octree)
 *   FP_KERNEL_SPLIT_ROUNDS     the split rounds of cells larger than one shared-memory piece
 *   FP_KERNEL_UNITS            k_units: LOD level and leaf level of every point
 *   FP_KERNEL_NODE_TABLE       node records sorted into preorder
 *   FP_KERNEL_RESOLVE          k_resolve: owner node and leaf node of every point
 *   FP_KERNEL_LEAF_SCATTER     the leaf-grouped layout (when requested)
 *   FP_KERNEL_OWNER_SCATTER    the final layout scatter of fp_subsample
 *   FP_KERNEL_STITCH           the merge of points kept above the chunks (sort and placement)
 * fp_time_kernel(k, start, stop) arms kernel k for the calling process: every
 * later call that launches it records `start` on its stream before the first
 * launch of k and `stop` after the last one (cudaEventElapsedTime then gives
 * the kernel's device time in that call).  k = FP_KERNEL_NONE disarms.  One
 * kernel is armed at a time; the events belong to the caller and must stay
 * valid while armed.  Not for use while several threads issue calls. */
typedef enum {
    FP_KERNEL_NONE = 0,
    FP_KERNEL_BOUNDS_DECIMATE = 1,
    FP_KERNEL_COUNT = 2,
    FP_KERNEL_DISTRIBUTE = 3,
    FP_KERNEL_CELL_GROUP = 4,
    FP_KERNEL_SPLIT_ROUNDS = 5,
    FP_KERNEL_UNITS = 6,
    FP_KERNEL_NODE_TABLE = 7,
    FP_KERNEL_RESOLVE = 8,
    FP_KERNEL_LEAF_SCATTER = 9,
    FP_KERNEL_OWNER_SCATTER = 10,
    FP_KERNEL_STITCH = 11
} fp_kernel;

fp_status fp_time_kernel(fp_kernel k, cudaEvent_t start, cudaEvent_t stop);

/* Cube of d_pts[0..n): per-axis min and max, S = largest extent + 1 (Sec. 4.4:
 * the converter first needs the extent of the cloud).  d_cube: one record. */
fp_status fp_bounds(const fp_point* d_pts, uint64_t n, fp_cube* d_cube,
                    void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Preview (Sec. 3 "uniformly downsampling", Sec. 4.2): keeps d_pts[i] iff
 * splitmix64(first_index + i) % modulus == 0, where splitmix64(v) is the first
 * output of a splitmix64 generator seeded with v; the kept points are written to
 * d_out in ascending i and their number to *d_out_count.  Points beyond out_cap
 * are not written (FP_ERR_CAPACITY in the device word).  first_index lets a
 * cloud streamed in pieces keep its global indices. */
fp_status fp_decimate(const fp_point* d_pts, uint64_t n, uint64_t first_index, uint32_t modulus,
                      fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count,
                      void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Modulus of a preview of about `target` points (Sec. 5: the preview is the
 * cloud downsampled to a fixed budget of points): max(1, ceil(n / target));
 * 1 when target is 0.  Pass it to fp_decimate / fp_bounds_decimate. */
uint32_t fp_preview_modulus(uint64_t n, uint64_t target);

/* Spatially constrained random preview (the sampler Sec. 6 proposes for clouds
 * whose file order makes the uniform preview uneven).  Of the points of every
 * occupied cell of the 2^level grid over *d_cube (cells as in fp_count,
 * 1 <= level <= 7), the one with the smallest splitmix64(first_index + i) is
 * kept; kept points are written to d_out in ascending index, their number to
 * *d_out_count (= the number of occupied cells; beyond out_cap they are not
 * written and FP_ERR_CAPACITY is raised in the device word).  Two passes over
 * the points; the workspace holds an 8^level table of 64-bit minima
 * (fp_workspace_size(FP_STAGE_PREVIEW_SPATIAL, n, prm) with prm->grid_log2 =
 * level).  The whole cloud must be in one call (the minimum is over the cloud). */
fp_status fp_preview_spatial(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t level,
                             uint64_t first_index, fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count,
                             void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* fp_bounds and fp_decimate in one pass over the points (one read of the cloud). */
fp_status fp_bounds_decimate(const fp_point* d_pts, uint64_t n, fp_cube* d_cube,
                             uint64_t first_index, uint32_t modulus,
                             fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count,
                             void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* fp_bounds_decimate without a workspace, for callers that cannot allocate
 * device memory (a host application whose device memory belongs to another
 * allocator or budget, or a real-time loop that must not wait on one).  The
 * paper has no counterpart: this is a deployment convenience.
 * Scratch: a 1 MiB array inside the library, held by every GPU that loads it
 * until the process exits; n <= 2^27 (134,217,728) points, larger n returns
 * FP_ERR_TOO_LARGE.  The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture.  Every call shares the one array (the scratch it needs is reset by
 * each call), so calls that overlap on the GPU -- on different streams, or from
 * different host threads -- race and must be serialised by the caller.  No
 * device memory is allocated or freed.  The array's device address (and the
 * device error word's) is looked up once per device and kept for the process:
 * do not use the library across a cudaDeviceReset() of that device.
 * Outputs as fp_bounds_decimate. */
fp_status fp_bounds_decimate_static(const fp_point* d_pts, uint64_t n, fp_cube* d_cube,
                                    uint64_t first_index, uint32_t modulus,
                                    fp_point* d_out, uint64_t out_cap, uint64_t* d_out_count,
                                    cudaStream_t stream);

/* Count grid (Sec. 4.4, the first step of sorting points into chunks):
 * d_counts[m] = number of points whose level-g cell has Morton key m, where the
 * cell of axis a is floor((p_a - o_a) * 2^g / S) in exact integer arithmetic and
 * the Morton key takes one bit per axis per level, x most significant.
 * d_counts has 8^g entries; it is zeroed first unless `accumulate` is nonzero
 * (pieces of one cloud, all with the same cube). */
fp_status fp_count(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2,
                   uint32_t* d_counts, int accumulate,
                   void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* fp_count that also writes d_cells[i] = the level-g Morton cell of point i (n
 * entries, required for n > 0): fp_distribute_cells then reads the cells
 * instead of computing them from the points again. */
fp_status fp_count_cells(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2,
                         uint32_t* d_counts, int accumulate, uint32_t* d_cells,
                         void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Chunks (Fig. "octree": each chunk is a node of the global tree): sums the count
 * grid up to the root; a chunk is a node with 0 < count <= threshold whose parent
 * holds more than threshold points (or the root itself), or a level-g cell holding
 * more than threshold points.  Chunks are listed in Morton preorder in d_chunks
 * (capacity 8^g), their number in *d_num_chunks, d_lut[m] = chunk of cell m
 * (0xFFFFFFFF for empty cells, 8^g entries), d_offsets[0..K] = exclusive prefix
 * sums of the chunk counts (capacity 8^g + 1). */
fp_status fp_merge_chunks(const uint32_t* d_counts, uint32_t grid_log2, uint64_t threshold,
                          fp_chunk* d_chunks, uint32_t* d_num_chunks, uint32_t* d_lut, uint64_t* d_offsets,
                          void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Stable scatter into chunks (Sec. 4.4 "sorted into a number of chunks"):
 * d_out[d_offsets[c] + r] = d_pts[i] where c is the chunk of point i and r the
 * number of points of chunk c with an index below i; d_perm (nullable) receives
 * i at the same position.  d_out must not alias d_pts. */
fp_status fp_distribute(const fp_point* d_pts, uint64_t n, const fp_cube* d_cube, uint32_t grid_log2,
                        const uint32_t* d_lut, const uint64_t* d_offsets, const uint32_t* d_num_chunks,
                        fp_point* d_out, uint32_t* d_perm,
                        void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* fp_distribute with the points' level-g cells given (d_cells from
 * fp_count_cells, same cube and grid_log2): the chunk of point i is
 * d_lut[d_cells[i]] instead of being computed from the point.  With d_cells
 * 16-byte aligned, up to 4096 chunks take a counting pass and a double-buffered
 * sweep (no wait between blocks); otherwise up to 2048 chunks the one-sweep
 * scatter; more chunks take the radix passes, which compute the cell.  Every
 * d_cells[i] must be below 8^grid_log2 (else FP_ERR_CAPACITY, outputs invalid).
 * Outputs identical to fp_distribute's. */
fp_status fp_distribute_cells(const fp_point* d_pts, const uint32_t* d_cells, uint64_t n, const fp_cube* d_cube,
                              uint32_t grid_log2, const uint32_t* d_lut, const uint64_t* d_offsets,
                              const uint32_t* d_num_chunks, fp_point* d_out, uint32_t* d_perm,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Local octrees of all chunks, stitched under the global nodes above them
 * (Sec. 4.4, Fig. "octree"), and the level-of-detail selection.
 * Input: the output of fp_distribute (d_sorted, d_perm) and of the earlier stages.
 * Hierarchy: a node at level L exists iff it holds a point and (L == 0 or its
 * parent holds more than node_capacity points and lies above max_level); it is
 * a leaf iff it holds at most node_capacity points or L == max_level.
 * Outputs:
 *   d_nodes[0..M), *d_num_nodes = M (nodes beyond node_cap are not written,
 *     FP_ERR_CAPACITY); every field but `first` is filled;
 *   d_leaf_pts / d_leaf_perm (n each, nullable): points grouped by leaf, leaves
 *     in preorder, ascending original index inside a leaf;
 *   d_owner[j] (n, u32): node that keeps distributed point j after LOD
 *     subsampling -- an inner node at level L keeps, of every occupied
 *     level-(L + sub_log2) cell, the point with the smallest original index
 *     among its children's remaining points (deepest nodes first); a point not
 *     taken by any ancestor stays in its leaf. */
fp_status fp_build_chunk_octree(const fp_point* d_sorted, const uint32_t* d_perm, uint64_t n,
                                const fp_cube* d_cube, const fp_chunk* d_chunks, const uint32_t* d_num_chunks,
                                const uint64_t* d_offsets, const uint32_t* d_counts, const fp_params* h_prm,
                                fp_node* d_nodes, uint32_t node_cap, uint32_t* d_num_nodes,
                                fp_point* d_leaf_pts, uint32_t* d_leaf_perm, uint32_t* d_owner,
                                void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Final level-of-detail layout: nodes in preorder, each node's kept points in
 * ascending original index (points kept by nodes above the chunks are merged
 * across chunks: the stitch).  Fills d_nodes[*].first and writes d_final /
 * d_final_perm (n each, required).  d_chunks / d_num_chunks / d_offsets are the
 * chunks the points were distributed into (fp_merge_chunks); the layout is
 * computed chunk by chunk.  node_cap <= 2^23; the workspace is sized for this
 * node_cap (fp_workspace_size(FP_STAGE_SUBSAMPLE) assumes the bound above). */
fp_status fp_subsample(fp_node* d_nodes, const uint32_t* d_num_nodes, uint32_t node_cap,
                       const fp_point* d_sorted, const uint32_t* d_perm, const uint32_t* d_owner, uint64_t n,
                       const fp_chunk* d_chunks, const uint32_t* d_num_chunks, const uint64_t* d_offsets,
                       fp_point* d_final, uint32_t* d_final_perm,
                       void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------- batches
 * Many clouds in one call.  The paper builds one cloud at a time; the batched
 * form runs every cloud's whole pipeline (the seven calls above, in order) on
 * one of nlanes library-owned streams forked from and joined back into
 * `stream`, so small clouds overlap on the device and the whole batch can be
 * captured into one CUDA graph (lanes are created on the first call with each
 * device current: make that first call outside a stream capture).  Each
 * cloud's outputs are bit-identical to the plain calls'.  Clouds go to lanes
 * largest first, each to the lane with the fewest points so far. */
typedef struct {
    const fp_point* d_pts;            /* input, 16-byte aligned */
    uint64_t n;
    fp_params prm;
    fp_cube* d_cube;                  /* outputs, sized as for the plain calls */
    fp_point* d_preview;
    uint64_t preview_cap;
    uint64_t* d_preview_count;
    uint32_t* d_counts;               /* 8^grid_log2 */
    fp_chunk* d_chunks;               /* 8^grid_log2 */
    uint32_t* d_num_chunks;
    uint32_t* d_lut;                  /* 8^grid_log2 */
    uint64_t* d_offsets;              /* 8^grid_log2 + 1 */
    fp_point* d_dist;                 /* n */
    uint32_t* d_perm;                 /* n */
    fp_node* d_nodes;                 /* node_cap = fp_node_capacity_bound(n, &prm) */
    uint32_t node_cap;
    uint32_t* d_num_nodes;
    fp_point* d_leaf_pts;             /* n, nullable */
    uint32_t* d_leaf_perm;            /* n, nullable */
    uint32_t* d_owner;                /* n */
    fp_point* d_final;                /* n */
    uint32_t* d_final_perm;           /* n */
} fp_cloud_desc;

#define FP_MAX_LANES 32

/* Workspace bytes of fp_build_batched for these clouds on nlanes lanes
 * (1 <= nlanes <= FP_MAX_LANES): each lane's largest per-cloud need. */
size_t fp_batch_workspace_size(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes);

/* Builds every cloud of h_clouds[0..ncloud) (host array of descriptors).  All
 * descriptors are checked before anything is enqueued; on an error nothing is. */
fp_status fp_build_batched(const fp_cloud_desc* h_clouds, uint32_t ncloud, uint32_t nlanes,
                           void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Options of a batched build; none of them changes any output bit.
 *   nlanes         library-owned streams the clouds' calls run on (1 .. FP_MAX_LANES)
 *   fused_first    nonzero: the bounds + preview pass and the count pass of every
 *                  cloud run as one launch each (groups of up to 256 clouds, their
 *                  descriptors passed in the kernel parameters), on `stream`
 *                  before the lanes fork; the remaining calls run on the lanes
 *   count_threads  256 or 512: block size of the fused count pass
 *   count_slots    0, 1024 or 4096: cells of the per-block shared-memory table the
 *                  fused count pass accumulates hot cells in (0: none) */
typedef struct {
    uint32_t nlanes, fused_first, count_threads, count_slots;
} fp_batch_opts;

size_t fp_batch_workspace_size_ex(const fp_cloud_desc* h_clouds, uint32_t ncloud, const fp_batch_opts* opts);
fp_status fp_build_batched_ex(const fp_cloud_desc* h_clouds, uint32_t ncloud, const fp_batch_opts* opts,
                              void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------- out of core
 * A cloud larger than the device memory it may use (Sec. 4.4: the converter
 * streams clouds that do not fit, chunk by chunk).  The points stay in pinned
 * host memory and are streamed in pieces of piece_points (<= 2^23) with
 * cudaMemcpyAsync on a side stream; every device buffer of the build lies in
 * d_arena (the budget); h_scratch (pinned, fp_ooc_host_bytes) holds the chunk
 * groups between passes.  Passes:
 * bounds + preview (preview_done(user) runs on a CUDA host-callback thread once
 * the preview and its count are in h_preview / *h_preview_count; nullable),
 * counts, chunks, then groups of consecutive chunks that fit the arena: each
 * group's local octrees (levels and nodes below the count grid), the node table
 * of the whole cloud, owners, and the final layout (points kept above the
 * chunks merged across groups by a device sort).  When the arena also holds
 * the distributed cloud (20 bytes per point) next to a group as large as the
 * largest chunk, the cloud stays on the device after the distribution pass and
 * is not read back from h_scratch.  The outputs equal the in-core calls'
 * (cube, preview, node table, final points and perm).
 * This call blocks the calling host thread until the build is done (it reads
 * the chunk list between passes); h_* outputs are pinned host memory. */
size_t fp_ooc_arena_min(uint64_t n, const fp_params* prm, uint64_t piece_points);
size_t fp_ooc_host_bytes(uint64_t n, const fp_params* prm);

/* group_points: largest chunk group in points (0: as large as the arena allows). */
fp_status fp_build_ooc(const fp_point* h_pts, uint64_t n, const fp_params* h_prm, uint64_t piece_points,
                       uint64_t group_points, void* d_arena, size_t arena_bytes, void* h_scratch, size_t scratch_bytes,
                       fp_cube* h_cube, fp_point* h_preview, uint64_t preview_cap, uint64_t* h_preview_count,
                       fp_node* h_nodes, uint32_t node_cap, uint32_t* h_num_nodes,
                       fp_point* h_final, uint32_t* h_final_perm,
                       void (*preview_done)(void*), void* user, cudaStream_t stream);

/* ------------------------------------------------------ octree file, cache
 * The stitched global octree written to one file and loaded back (Sec. 4.4:
 * the global octree is written to a file; Sec. 4.5: the renderer loads the
 * points of the nodes it draws on demand), and a digest of the input cloud
 * that keys a cache of built octrees (Sec. 3, Fig. "pipeline": a cloud whose
 * octree was built before is not built again).
 *
 * File layout (little-endian): fp_file_header at offset 0; the node table
 * (num_nodes fp_node records, preorder) at nodes_offset; the points in the
 * final layout (n fp_point records; node i's kept points are records
 * [first, first + n_own)) at points_offset; when flags has FP_FILE_HAS_PERM,
 * the original index of every final point (n uint32) at perm_offset.  Offsets
 * are multiples of 4096 except perm_offset (= points_offset + 16 n). */
#define FP_FILE_HAS_PERM 1u
typedef struct {
    char magic[8];                 /* "FPOCTREE" */
    uint32_t version, header_bytes;   /* 1, sizeof(fp_file_header) */
    fp_params prm;
    fp_cube cube;
    uint64_t n;
    uint32_t num_nodes, flags;
    uint64_t digest;               /* fp_cloud_digest of the input cloud (0: not recorded) */
    uint64_t nodes_offset, points_offset, perm_offset;
    uint64_t reserved[4];
} fp_file_header;

/* Digest of a cloud: n + sum over i of splitmix64(splitmix64(i) ^
 * splitmix64(x | y << 32) ^ splitmix64((z | rgba << 32) ^ 0x5851F42D4C957F2D))
 * (mod 2^64), with x, y, z, rgba the record's four 32-bit words as unsigned.
 * Depends on every point and on the order.  Written to *d_digest. */
fp_status fp_cloud_digest(const fp_point* d_pts, uint64_t n, uint64_t* d_digest, cudaStream_t stream);

/* Writes the octree of fp_build_chunk_octree + fp_subsample (device outputs)
 * to `path`: header, node table, final points, and the final permutation when
 * d_final_perm is not NULL.  h_staging: pinned host memory of staging_bytes
 * (>= 8 KiB; larger pieces overlap better), used in two halves so the device
 * copy of one piece overlaps the file write of the other.  Blocks the calling
 * thread until the file is closed.  FP_ERR_IO when the file cannot be written. */
fp_status fp_octree_save(const char* path, const fp_params* h_prm, const fp_cube* d_cube, const fp_node* d_nodes,
                         const uint32_t* d_num_nodes, const fp_point* d_final, const uint32_t* d_final_perm,
                         uint64_t n, uint64_t digest, void* h_staging, size_t staging_bytes, cudaStream_t stream);

/* Reads and checks the header (FP_ERR_INVALID: not an octree file of this version). */
fp_status fp_octree_read_header(const char* path, fp_file_header* h_hdr);

/* Loads into device memory the node table (d_nodes non-NULL; node_cap >=
 * num_nodes, else FP_ERR_CAPACITY) and final points [first, first + count)
 * (d_points non-NULL), with their original indices (d_perm non-NULL; the file
 * must hold them) -- a node's points are first = node.first, count = n_own.
 * Staging as for fp_octree_save.  Blocks until the data are on the device. */
fp_status fp_octree_load(const char* path, fp_node* d_nodes, uint32_t node_cap, fp_point* d_points,
                         uint32_t* d_perm, uint64_t first, uint64_t count, void* h_staging, size_t staging_bytes,
                         cudaStream_t stream);

/* ------------------------------------------------------ rendering, headless
 * The renderer's side of the octree (Sec. 4.5: a traversal picks the nodes the
 * camera needs, their points are drawn), into a device framebuffer instead of
 * a graphics API.
 *
 * Camera: m is a row-major 4x4 view-projection matrix; a position p maps to
 * clip = m (x, y, z, 1) with every row evaluated as
 * fmaf(m0, x, fmaf(m1, y, fmaf(m2, z, m3))) in fp32 (x, y, z the coordinates
 * rounded to fp32).  A point is inside when w > 0, -w <= x, y <= w and
 * 0 <= z <= w; its pixel is (floor(sx), floor(sy)) clamped to the image with
 * sx = fmaf(x / w, 0.5, 0.5) * width (sy likewise with y, height; IEEE
 * division), framebuffer index py * width + px; its depth is z / w + 0.
 *
 * Node box: the integer range of the points a node can hold, per axis
 * [o + ceil(c S / 2^L), o + ceil((c + 1) S / 2^L) - 1] for cell coordinate c at
 * level L.  A node is outside when all 8 box corners (as fp32) are beyond the
 * same clip plane (x < -w, x > w, y < -w, y > w, z < 0 or z > w).  Its screen
 * size is the larger of the x and y extents of the corners' sx, sy, infinite
 * when a corner has w <= 0.  A node is drawn when it is not outside and every
 * ancestor was refined; refined = drawn, not a leaf, size > min_node_px. */
typedef struct {
    float m[16];
    uint32_t width, height;   /* 1 .. 16384 */
    float min_node_px;
    uint32_t reserved;
} fp_camera;

/* Workspace of fp_select_nodes and fp_rasterize for a node table of node_cap entries. */
size_t fp_render_workspace_size(uint32_t node_cap);

/* The drawn nodes in preorder (ids into d_nodes) to d_selected (node_cap
 * entries), their number to *d_num_selected and their kept points in total to
 * *d_num_points.  node_cap <= 2^23. */
fp_status fp_select_nodes(const fp_node* d_nodes, const uint32_t* d_num_nodes, uint32_t node_cap,
                          const fp_cube* d_cube, const fp_camera* h_cam, uint32_t* d_selected,
                          uint32_t* d_num_selected, uint64_t* d_num_points, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream);

/* The kept points of the selected nodes (final layout of n points: node.first,
 * n_own) rasterised into d_framebuffer (width * height entries, set by the
 * call): every pixel holds the minimum over its points of
 * (depth bits << 32 | rgba), all ones where no point lands.  Records outside
 * [0, n) are skipped. */
fp_status fp_rasterize(const fp_node* d_nodes, const uint32_t* d_selected, const uint32_t* d_num_selected,
                       uint32_t node_cap, const fp_point* d_final, uint64_t n, const fp_camera* h_cam,
                       uint64_t* d_framebuffer, void* d_ws, size_t ws_bytes, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif
