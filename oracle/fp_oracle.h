/*
 * fp_oracle.h -- plain, slow, single-threaded CPU oracle for the FastPoints
 * octree-construction hot path (arxiv 2302.05002).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the record layouts
 * below are written out again here on purpose (the 16-byte point record is
 * the interchange format, nothing else is shared).
 *
 * The paper (Sec. 3, Sec. 4.4, Fig. "octree") delegates octree construction to a
 * chunk -> index -> stitch converter and gives no constants; every definition
 * implemented here is one exact-integer reading of it:
 *   cube      o_a = min p_a, S = max_a(max p_a - o_a) + 1                  (Sec. 4.4)
 *   cell      c_a(l) = floor((p_a - o_a) * 2^l / S), Morton x-major        (Sec. 4.4)
 *   preview   keep i  <=>  splitmix64(i) mod m == 0, ascending i            (Sec. 3, 4.2)
 *   chunks    maximal nodes with 0 < count <= T, plus overflowing cells     (Sec. 4.4, Fig. octree)
 *   hierarchy node exists iff count > 0 and parent count > C, parent level < Lmax
 *   LOD       each inner node at level L moves up, per occupied level-(L+s)
 *             cell among its children's current points, the smallest index  (Abstract "shallow octree")
 */
#ifndef FP_ORACLE_H
#define FP_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int32_t x, y, z; uint8_t r, g, b, a; } orc_point;      /* 16 B */
typedef struct { int32_t o[3]; int32_t mx[3]; uint64_t S; } orc_cube;   /* 32 B */
typedef struct { uint64_t key; uint32_t count; uint32_t level; } orc_chunk; /* 16 B */
typedef struct {
    uint64_t key, first, leaf_first;
    uint32_t count, n_own, n_desc;
    uint8_t level, child_mask, is_leaf, pad;
} orc_node;                                                              /* 40 B */
typedef struct {
    uint32_t grid_log2, sub_log2, max_level, decim_modulus;
    uint64_t chunk_threshold, node_capacity;
} orc_params;

/* first output of a splitmix64 generator whose state is seeded with i */
uint64_t orc_splitmix64(uint64_t i);

/* cube of n points; n == 0 gives an all-zero cube with S == 0 */
void orc_bounds(const orc_point* pts, uint64_t n, orc_cube* cube);

/* preview: copies pts[i] (i ascending) with splitmix64(first_index+i) % modulus == 0
 * into out (capacity n) and, if out_idx != NULL, first_index+i into out_idx; returns the count */
uint64_t orc_decimate(const orc_point* pts, uint64_t n, uint64_t first_index, uint32_t modulus,
                      orc_point* out, uint64_t* out_idx);

/* digest of a cloud: n + sum of one mixed word per point (mod 2^64) */
uint64_t orc_cloud_digest(const orc_point* pts, uint64_t n);

/* modulus of a preview of about `target` points: max(1, ceil(n / target)) */
uint32_t orc_preview_modulus(uint64_t n, uint64_t target);

/* one point per occupied level cell: the smallest splitmix64(first_index + i);
 * kept points in ascending index; returns their number (~0 on allocation failure) */
uint64_t orc_preview_spatial(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t level,
                             uint64_t first_index, orc_point* out, uint64_t* out_idx);

/* exact integer cell coordinate of one axis at level l (0 <= l <= 21) */
uint64_t orc_axis_cell(int32_t p, int32_t o, uint64_t S, uint32_t level);
/* Morton key of a cell at level l; x bit most significant inside each 3-bit digit */
uint64_t orc_morton(uint64_t cx, uint64_t cy, uint64_t cz, uint32_t level);
/* Morton key of the level-l cell that holds point p */
uint64_t orc_point_key(const orc_point* p, const orc_cube* cube, uint32_t level);

/* counts[8^g] (zeroed here) of points per level-g cell, Morton order */
void orc_count(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t g, uint32_t* counts);

/* chunks in Morton preorder (capacity 8^g), lut[8^g] (0xFFFFFFFF for empty cells),
 * offsets[K+1]; returns K */
uint32_t orc_merge(const uint32_t* counts, uint32_t g, uint64_t T,
                   orc_chunk* chunks, uint32_t* lut, uint64_t* offsets);

/* stable scatter of the points into their chunks; perm[j] = original index (nullable) */
void orc_distribute(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t g,
                    const uint32_t* lut, const uint64_t* offsets, orc_point* out, uint32_t* perm);

/* Hierarchy, leaf-grouped points and LOD of the whole cloud, straight from the
 * definitions.  pts are in original index order.  Node records are written if
 * M <= node_cap; the return value is M (or (uint32_t)-1 on allocation failure).
 * leaf_pts/leaf_perm (n each): leaves in preorder, ascending index inside a leaf.
 * final_pts/final_perm (n each): nodes in preorder, owned points ascending index.
 * lod_form 0 = bottom-up move simulation, 1 = closed form (first-min level). */
uint32_t orc_octree_lod(const orc_point* pts, uint64_t n, const orc_cube* cube, const orc_params* prm,
                        orc_node* nodes, uint32_t node_cap,
                        orc_point* leaf_pts, uint32_t* leaf_perm,
                        orc_point* final_pts, uint32_t* final_perm, int lod_form);

/* per-point closed-form quantities: lambda[i] (22 == never the minimum up to level 21),
 * leaf_level[i], owner_level[i]; returns 0 on success */
int orc_point_levels(const orc_point* pts, uint64_t n, const orc_cube* cube, const orc_params* prm,
                     uint8_t* lambda, uint8_t* leaf_level, uint8_t* owner_level);

/* ---- headless rendering (Sec. 4.5) */
typedef struct {
    float m[16];               /* row-major view-projection */
    uint32_t width, height;
    float min_node_px;
    uint32_t reserved;
} orc_camera;

/* drawn nodes (ids in preorder) to sel (capacity M); returns their number */
uint32_t orc_render_select(const orc_node* nodes, uint32_t M, const orc_cube* cube, const orc_camera* cam,
                           uint32_t* sel);

/* the kept points of the drawn nodes rasterised: fb[width * height] = min over the
 * pixel's points of (depth bits << 32 | rgba), all ones where none lands */
void orc_rasterize(const orc_node* nodes, const uint32_t* sel, uint32_t nsel, const orc_point* final_pts,
                   const orc_camera* cam, uint64_t* fb);

#ifdef __cplusplus
}
#endif
#endif
