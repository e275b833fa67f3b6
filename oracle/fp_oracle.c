/*
 * fp_oracle.c -- plain single-threaded CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Every function restates one definition of the octree-construction hot path
 * (paper Sec. 3, Sec. 4.2, Sec. 4.4 and Fig. "octree", in the exact-integer
 * readings listed in fp_oracle.h) in the most direct form: loops, qsort,
 * per-level work.
 * There is no blocking, fusion or reordering beyond what the definitions say.
 * Nothing here is shared with the CUDA library.
 */
#include "fp_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- hashing */
/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by the
 * golden-ratio increment, then the mix function with shifts 30/27/31.  The
 * preview keeps index i when this value is divisible by the modulus (Sec. 4.2,
 * "uniform downsampling", made index-deterministic). */
uint64_t orc_splitmix64(uint64_t i)
{
    uint64_t z = i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Digest of a cloud (the key of the cache of built octrees): n plus the sum,
 * modulo 2^64, of one mixed word per point built from its index and the two
 * 64-bit halves of its record. */
uint64_t orc_cloud_digest(const orc_point* pts, uint64_t n)
{
    uint64_t d = n;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        memcpy(w, &pts[i], sizeof(w));
        uint64_t a = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
        uint64_t b = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
        d += orc_splitmix64(orc_splitmix64(i) ^ orc_splitmix64(a) ^ orc_splitmix64(b ^ 0x5851F42D4C957F2Dull));
    }
    return d;
}

/* ----------------------------------------------------------------- bounds */
/* Sec. 4.4: the converter needs the cloud's extent.  Origin at the minimum
 * corner, cube side = largest axis extent + 1 so the maximum lies inside. */
void orc_bounds(const orc_point* pts, uint64_t n, orc_cube* cube)
{
    memset(cube, 0, sizeof(*cube));
    if (n == 0) return;
    int32_t lo[3] = {pts[0].x, pts[0].y, pts[0].z};
    int32_t hi[3] = {pts[0].x, pts[0].y, pts[0].z};
    for (uint64_t i = 1; i < n; ++i) {
        int32_t v[3] = {pts[i].x, pts[i].y, pts[i].z};
        for (int a = 0; a < 3; ++a) {
            if (v[a] < lo[a]) lo[a] = v[a];
            if (v[a] > hi[a]) hi[a] = v[a];
        }
    }
    uint64_t ext = 0;
    for (int a = 0; a < 3; ++a) {
        cube->o[a] = lo[a];
        cube->mx[a] = hi[a];
        uint64_t e = (uint64_t)((int64_t)hi[a] - (int64_t)lo[a]);
        if (e > ext) ext = e;
    }
    cube->S = ext + 1;
}

/* --------------------------------------------------------------- preview */
uint64_t orc_decimate(const orc_point* pts, uint64_t n, uint64_t first_index, uint32_t modulus,
                      orc_point* out, uint64_t* out_idx)
{
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (orc_splitmix64(first_index + i) % modulus == 0) {
            out[k] = pts[i];
            if (out_idx) out_idx[k] = first_index + i;
            ++k;
        }
    }
    return k;
}

/* Sec. 5 sizes the preview by a point budget (1,000,000 points): the modulus
 * is the smallest one whose expected preview fits, ceil(n / target). */
uint32_t orc_preview_modulus(uint64_t n, uint64_t target)
{
    if (target == 0 || n <= target) return 1;
    uint64_t m = n / target + (n % target != 0);
    return m > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)m;
}

/* ------------------------------------------------------------------ cells */
uint64_t orc_axis_cell(int32_t p, int32_t o, uint64_t S, uint32_t level)
{
    uint64_t d = (uint64_t)((int64_t)p - (int64_t)o);   /* 0 <= d < 2^32 */
    return (d << level) / S;                            /* < 2^53, exact */
}

uint64_t orc_morton(uint64_t cx, uint64_t cy, uint64_t cz, uint32_t level)
{
    uint64_t k = 0;
    for (int b = (int)level - 1; b >= 0; --b)
        k = (k << 3) | (((cx >> b) & 1u) << 2) | (((cy >> b) & 1u) << 1) | ((cz >> b) & 1u);
    return k;
}

uint64_t orc_point_key(const orc_point* p, const orc_cube* c, uint32_t level)
{
    return orc_morton(orc_axis_cell(p->x, c->o[0], c->S, level),
                      orc_axis_cell(p->y, c->o[1], c->S, level),
                      orc_axis_cell(p->z, c->o[2], c->S, level), level);
}

/* ------------------------------------------------------- spatial preview */
/* Sec. 6 proposes a spatially constrained random sampler for the preview.
 * Reading: a grid of 2^level cells per axis over the cube; in every occupied
 * cell the point whose index hash splitmix64(first_index + i) is smallest is
 * kept (a random point of the cell, fixed by the hash); kept points in
 * ascending index.  Written as: the smallest hash per cell, then a sweep that
 * keeps the points holding it. */
uint64_t orc_preview_spatial(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t level,
                             uint64_t first_index, orc_point* out, uint64_t* out_idx)
{
    uint64_t cells = 1ull << (3 * level);
    uint64_t* best = (uint64_t*)malloc(cells * sizeof(uint64_t));
    if (!best) return ~0ull;
    for (uint64_t c = 0; c < cells; ++c) best[c] = ~0ull;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t c = orc_point_key(&pts[i], cube, level);
        uint64_t h = orc_splitmix64(first_index + i);
        if (h < best[c]) best[c] = h;
    }
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (best[orc_point_key(&pts[i], cube, level)] == orc_splitmix64(first_index + i)) {
            out[k] = pts[i];
            if (out_idx) out_idx[k] = first_index + i;
            ++k;
        }
    }
    free(best);
    return k;
}

/* ------------------------------------------------------------------ count */
void orc_count(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t g, uint32_t* counts)
{
    uint64_t cells = 1ull << (3 * g);
    memset(counts, 0, cells * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i) counts[orc_point_key(&pts[i], cube, g)] += 1;
}

/* ------------------------------------------------------------------ merge */
typedef struct {
    uint64_t** lvl;     /* lvl[l][k] = points in node (l, k), l = 0..g */
    uint32_t g;
    uint64_t T;
    orc_chunk* chunks;
    uint32_t K;
} merge_ctx;

/* A chunk is a node of the count pyramid with 0 < count <= T whose parent
 * holds more than T points (or the root), or a level-g cell holding more than T
 * (it cannot be split further).  Visiting children in digit order lists the
 * chunks in Morton preorder. */
static void merge_visit(merge_ctx* m, uint32_t l, uint64_t k)
{
    uint64_t c = m->lvl[l][k];
    if (c == 0) return;
    if (c <= m->T || l == m->g) {
        orc_chunk* ch = &m->chunks[m->K++];
        ch->key = k;
        ch->count = (uint32_t)c;
        ch->level = l;
        return;
    }
    for (uint64_t j = 0; j < 8; ++j) merge_visit(m, l + 1, 8 * k + j);
}

uint32_t orc_merge(const uint32_t* counts, uint32_t g, uint64_t T,
                   orc_chunk* chunks, uint32_t* lut, uint64_t* offsets)
{
    uint64_t* lvl[32];
    for (uint32_t l = 0; l <= g; ++l) lvl[l] = (uint64_t*)calloc(1ull << (3 * l), sizeof(uint64_t));
    uint64_t cells = 1ull << (3 * g);
    for (uint64_t m = 0; m < cells; ++m) lvl[g][m] = counts[m];
    for (int l = (int)g - 1; l >= 0; --l)
        for (uint64_t k = 0; k < (1ull << (3 * l)); ++k) {
            uint64_t s = 0;
            for (uint64_t j = 0; j < 8; ++j) s += lvl[l + 1][8 * k + j];
            lvl[l][k] = s;
        }
    merge_ctx mc = {lvl, g, T, chunks, 0};
    merge_visit(&mc, 0, 0);
    for (uint64_t m = 0; m < cells; ++m) lut[m] = 0xFFFFFFFFu;
    offsets[0] = 0;
    for (uint32_t q = 0; q < mc.K; ++q) {
        uint32_t sh = 3 * (g - chunks[q].level);
        uint64_t b = chunks[q].key << sh, e = (chunks[q].key + 1) << sh;
        for (uint64_t m = b; m < e; ++m)
            if (counts[m] > 0) lut[m] = q;
        offsets[q + 1] = offsets[q] + chunks[q].count;
    }
    for (uint32_t l = 0; l <= g; ++l) free(lvl[l]);
    return mc.K;
}

/* ------------------------------------------------------------- distribute */
/* out[offsets[chunk(p)] + (points of that chunk with a smaller index)] = p */
void orc_distribute(const orc_point* pts, uint64_t n, const orc_cube* cube, uint32_t g,
                    const uint32_t* lut, const uint64_t* offsets, orc_point* out, uint32_t* perm)
{
    uint64_t cells = 1ull << (3 * g);
    /* number of chunks = largest id in the LUT + 1 */
    uint32_t K = 0;
    for (uint64_t m = 0; m < cells; ++m)
        if (lut[m] != 0xFFFFFFFFu && lut[m] + 1 > K) K = lut[m] + 1;
    uint64_t* cur = (uint64_t*)malloc((K + 1) * sizeof(uint64_t));
    for (uint32_t q = 0; q < K; ++q) cur[q] = offsets[q];
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t q = lut[orc_point_key(&pts[i], cube, g)];
        uint64_t j = cur[q]++;
        out[j] = pts[i];
        if (perm) perm[j] = (uint32_t)i;
    }
    free(cur);
}

/* ------------------------------------------------------------- hierarchy */
typedef struct {
    uint64_t key, leaf_first;
    uint32_t count, n_desc, parent;
    uint8_t level, child_mask, is_leaf;
    uint32_t child[8];
} onode;

typedef struct {
    const orc_point* pts;
    const orc_cube* cube;
    const orc_params* prm;
    onode* nd;
    uint32_t M, cap;
    uint32_t* leaf_of;      /* per point: id of its leaf */
    uint32_t* leaf_order;   /* point ids in leaf-grouped order */
    uint64_t n_leafed;
    uint32_t** list;        /* per leaf: its point ids (ascending) */
    uint64_t* list_len;
    int oom;
} tree_ctx;

static uint32_t new_node(tree_ctx* t)
{
    if (t->M == t->cap) {
        uint32_t nc = t->cap ? 2 * t->cap : 1024;
        onode* nn = (onode*)realloc(t->nd, (size_t)nc * sizeof(onode));
        uint32_t** nl = (uint32_t**)realloc(t->list, (size_t)nc * sizeof(uint32_t*));
        uint64_t* nlen = (uint64_t*)realloc(t->list_len, (size_t)nc * sizeof(uint64_t));
        if (!nn || !nl || !nlen) { t->oom = 1; return 0; }
        t->nd = nn; t->list = nl; t->list_len = nlen; t->cap = nc;
    }
    uint32_t id = t->M++;
    memset(&t->nd[id], 0, sizeof(onode));
    t->list[id] = NULL;
    t->list_len[id] = 0;
    return id;
}

/* Node (level, key) holding the points idx[0..cnt) (ascending).  It is a leaf
 * when it holds at most C points or sits at Lmax; otherwise its points are split
 * by the next Morton digit (stable) and every non-empty part is a child. */
static uint32_t build_node(tree_ctx* t, uint32_t parent, uint32_t level, uint64_t key,
                           uint32_t* idx, uint64_t cnt)
{
    uint32_t id = new_node(t);
    if (t->oom) return 0;
    onode* d = &t->nd[id];
    d->key = key;
    d->level = (uint8_t)level;
    d->count = (uint32_t)cnt;
    d->parent = parent;
    d->leaf_first = t->n_leafed;
    for (int c = 0; c < 8; ++c) d->child[c] = 0xFFFFFFFFu;
    if (cnt > t->prm->node_capacity && level < t->prm->max_level) {
        uint64_t bucket[8] = {0}, start[8];
        uint8_t* dig = (uint8_t*)malloc(cnt ? cnt : 1);
        uint32_t* tmp = (uint32_t*)malloc((cnt ? cnt : 1) * sizeof(uint32_t));
        for (uint64_t q = 0; q < cnt; ++q) {
            dig[q] = (uint8_t)(orc_point_key(&t->pts[idx[q]], t->cube, level + 1) & 7u);
            bucket[dig[q]]++;
        }
        uint64_t s = 0;
        for (int c = 0; c < 8; ++c) { start[c] = s; s += bucket[c]; }
        uint64_t pos[8];
        memcpy(pos, start, sizeof(pos));
        for (uint64_t q = 0; q < cnt; ++q) tmp[pos[dig[q]]++] = idx[q];
        free(dig);
        uint8_t mask = 0;
        for (int c = 0; c < 8; ++c) {
            if (bucket[c] == 0) continue;
            mask |= (uint8_t)(1u << c);
            uint32_t ch = build_node(t, id, level + 1, key * 8 + (uint64_t)c, tmp + start[c], bucket[c]);
            if (t->oom) { free(tmp); return 0; }
            t->nd[id].child[c] = ch;
        }
        free(tmp);
        t->nd[id].child_mask = mask;
        t->nd[id].is_leaf = 0;
    } else {
        d->is_leaf = 1;
        t->list[id] = (uint32_t*)malloc((cnt ? cnt : 1) * sizeof(uint32_t));
        memcpy(t->list[id], idx, cnt * sizeof(uint32_t));
        t->list_len[id] = cnt;
        for (uint64_t q = 0; q < cnt; ++q) {
            t->leaf_of[idx[q]] = id;
            t->leaf_order[t->n_leafed++] = idx[q];
        }
    }
    t->nd[id].n_desc = t->M - id - 1;
    return id;
}

/* ---------------------------------------------------- LOD: move simulation */
typedef struct { uint64_t cell; uint32_t idx; uint32_t child; } cand;

static int cand_cmp(const void* a, const void* b)
{
    const cand* x = (const cand*)a;
    const cand* y = (const cand*)b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static int u32_cmp(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Deepest first (reverse preorder): every inner node at level L takes, from the
 * current points of its children, the smallest index of each occupied
 * level-(L+s) cell and moves it up into itself. */
static int lod_simulate(tree_ctx* t)
{
    uint32_t s = t->prm->sub_log2;
    for (int64_t id = (int64_t)t->M - 1; id >= 0; --id) {
        onode* d = &t->nd[id];
        if (d->is_leaf) continue;
        uint64_t total = 0;
        for (int c = 0; c < 8; ++c)
            if (d->child[c] != 0xFFFFFFFFu) total += t->list_len[d->child[c]];
        cand* cs = (cand*)malloc((total ? total : 1) * sizeof(cand));
        if (!cs) return -1;
        uint64_t q = 0;
        for (int c = 0; c < 8; ++c) {
            uint32_t ch = d->child[c];
            if (ch == 0xFFFFFFFFu) continue;
            for (uint64_t r = 0; r < t->list_len[ch]; ++r) {
                cs[q].idx = t->list[ch][r];
                cs[q].cell = orc_point_key(&t->pts[cs[q].idx], t->cube, d->level + s);
                cs[q].child = ch;
                ++q;
            }
        }
        qsort(cs, total, sizeof(cand), cand_cmp);
        uint32_t* own = (uint32_t*)malloc((total ? total : 1) * sizeof(uint32_t));
        uint64_t n_own = 0;
        for (uint64_t r = 0; r < total; ++r)       /* first of each cell = its minimum */
            if (r == 0 || cs[r].cell != cs[r - 1].cell) own[n_own++] = cs[r].idx;
        /* remove the picked points from the children */
        qsort(own, n_own, sizeof(uint32_t), u32_cmp);
        for (int c = 0; c < 8; ++c) {
            uint32_t ch = d->child[c];
            if (ch == 0xFFFFFFFFu) continue;
            uint64_t w = 0;
            for (uint64_t r = 0; r < t->list_len[ch]; ++r) {
                uint32_t v = t->list[ch][r];
                if (!bsearch(&v, own, n_own, sizeof(uint32_t), u32_cmp)) t->list[ch][w++] = v;
            }
            t->list_len[ch] = w;
        }
        free(cs);
        t->list[id] = own;
        t->list_len[id] = n_own;
    }
    return 0;
}

/* ------------------------------------------------- LOD: closed form */
typedef struct { uint64_t key; uint32_t idx; } kidx;
static int kidx_cmp(const void* a, const void* b)
{
    const kidx* x = (const kidx*)a;
    const kidx* y = (const kidx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* lambda(p) = smallest level l (0..21) at which p has the smallest index of
 * its level-l cell over the whole cloud; 22 if it never does (an identical
 * point with a smaller index shares every cell). */
static int compute_lambda(const orc_point* pts, uint64_t n, const orc_cube* cube, uint8_t* lambda)
{
    kidx* a = (kidx*)malloc((n ? n : 1) * sizeof(kidx));
    if (!a) return -1;
    for (uint64_t i = 0; i < n; ++i) lambda[i] = 22;
    for (uint32_t l = 0; l <= 21; ++l) {
        for (uint64_t i = 0; i < n; ++i) { a[i].key = orc_point_key(&pts[i], cube, l); a[i].idx = (uint32_t)i; }
        qsort(a, n, sizeof(kidx), kidx_cmp);
        for (uint64_t r = 0; r < n; ++r)
            if ((r == 0 || a[r].key != a[r - 1].key) && lambda[a[r].idx] == 22) lambda[a[r].idx] = (uint8_t)l;
    }
    free(a);
    return 0;
}

/* owner level = min(max(0, lambda - s), leaf level); the owner is the node on the
 * point's path at that level.  Derivation: a node at level K on the
 * path takes p iff K < leaf level and p is the minimum of its level-(K+s) cell,
 * and being a minimum at level l implies being one at every deeper level. */
static int lod_closed(tree_ctx* t, uint64_t n)
{
    uint8_t* lambda = (uint8_t*)malloc(n ? n : 1);
    if (!lambda || compute_lambda(t->pts, n, t->cube, lambda)) { free(lambda); return -1; }
    uint32_t* owner = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    uint64_t* cnt = (uint64_t*)calloc(t->M ? t->M : 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t leaf = t->leaf_of[i];
        int lam = lambda[i];
        int lv = lam - (int)t->prm->sub_log2;
        if (lv < 0) lv = 0;
        if (lv > t->nd[leaf].level) lv = t->nd[leaf].level;
        uint32_t o = leaf;
        while (t->nd[o].level > lv) o = t->nd[o].parent;
        owner[i] = o;
        cnt[o]++;
    }
    for (uint32_t id = 0; id < t->M; ++id) {
        free(t->list[id]);
        t->list[id] = (uint32_t*)malloc((cnt[id] ? cnt[id] : 1) * sizeof(uint32_t));
        t->list_len[id] = 0;
    }
    for (uint64_t i = 0; i < n; ++i) {   /* ascending index inside each node */
        uint32_t o = owner[i];
        t->list[o][t->list_len[o]++] = (uint32_t)i;
    }
    free(cnt); free(owner); free(lambda);
    return 0;
}

/* ------------------------------------------------------------- the build */
static void tree_free(tree_ctx* t)
{
    if (t->list)
        for (uint32_t id = 0; id < t->M; ++id) free(t->list[id]);
    free(t->list); free(t->list_len); free(t->nd); free(t->leaf_of); free(t->leaf_order);
}

static int tree_build(tree_ctx* t, const orc_point* pts, uint64_t n, const orc_cube* cube, const orc_params* prm)
{
    memset(t, 0, sizeof(*t));
    t->pts = pts; t->cube = cube; t->prm = prm;
    t->leaf_of = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    t->leaf_order = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!t->leaf_of || !t->leaf_order) return -1;
    if (n == 0) return 0;
    uint32_t* idx = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    build_node(t, 0xFFFFFFFFu, 0, 0, idx, n);
    free(idx);
    return t->oom ? -1 : 0;
}

uint32_t orc_octree_lod(const orc_point* pts, uint64_t n, const orc_cube* cube, const orc_params* prm,
                        orc_node* nodes, uint32_t node_cap,
                        orc_point* leaf_pts, uint32_t* leaf_perm,
                        orc_point* final_pts, uint32_t* final_perm, int lod_form)
{
    tree_ctx t;
    if (tree_build(&t, pts, n, cube, prm)) { tree_free(&t); return 0xFFFFFFFFu; }
    uint32_t M = t.M;
    for (uint64_t q = 0; q < n; ++q) {
        if (leaf_pts) leaf_pts[q] = pts[t.leaf_order[q]];
        if (leaf_perm) leaf_perm[q] = t.leaf_order[q];
    }
    int rc = lod_form == 0 ? lod_simulate(&t) : lod_closed(&t, n);
    if (rc) { tree_free(&t); return 0xFFFFFFFFu; }
    uint64_t first = 0;
    for (uint32_t id = 0; id < M; ++id) {
        if (id < node_cap && nodes) {
            orc_node* o = &nodes[id];
            memset(o, 0, sizeof(*o));
            o->key = t.nd[id].key;
            o->first = first;
            o->leaf_first = t.nd[id].leaf_first;
            o->count = t.nd[id].count;
            o->n_own = (uint32_t)t.list_len[id];
            o->n_desc = t.nd[id].n_desc;
            o->level = t.nd[id].level;
            o->child_mask = t.nd[id].child_mask;
            o->is_leaf = t.nd[id].is_leaf;
        }
        /* lists are ascending: the simulation sorts each pick set, children
         * keep their ascending order when points leave them */
        for (uint64_t r = 0; r < t.list_len[id]; ++r) {
            if (final_pts) final_pts[first + r] = pts[t.list[id][r]];
            if (final_perm) final_perm[first + r] = t.list[id][r];
        }
        first += t.list_len[id];
    }
    tree_free(&t);
    return M;
}

int orc_point_levels(const orc_point* pts, uint64_t n, const orc_cube* cube, const orc_params* prm,
                     uint8_t* lambda, uint8_t* leaf_level, uint8_t* owner_level)
{
    tree_ctx t;
    if (tree_build(&t, pts, n, cube, prm)) { tree_free(&t); return -1; }
    if (compute_lambda(pts, n, cube, lambda)) { tree_free(&t); return -1; }
    for (uint64_t i = 0; i < n; ++i) {
        int ll = t.nd[t.leaf_of[i]].level;
        int lv = (int)lambda[i] - (int)prm->sub_log2;
        if (lv < 0) lv = 0;
        if (lv > ll) lv = ll;
        leaf_level[i] = (uint8_t)ll;
        owner_level[i] = (uint8_t)lv;
    }
    tree_free(&t);
    return 0;
}

/* ----------------------------------------------------- headless rendering */
/* Sec. 4.5: the renderer walks the octree, draws the nodes the camera needs
 * and the points of those nodes.  Restated with fp32 arithmetic in the order
 * the boundary documents: each clip row is fmaf(m0, x, fmaf(m1, y, fmaf(m2, z,
 * m3))); screen x = fmaf(x / w, 0.5, 0.5) * width.  (C float arithmetic is
 * IEEE single here; the library is built without contraction.) */
typedef struct { float x, y, z, w; } orc_clip;

static orc_clip clip_of(const orc_camera* c, float x, float y, float z)
{
    orc_clip r;
    r.x = fmaf(c->m[0], x, fmaf(c->m[1], y, fmaf(c->m[2], z, c->m[3])));
    r.y = fmaf(c->m[4], x, fmaf(c->m[5], y, fmaf(c->m[6], z, c->m[7])));
    r.z = fmaf(c->m[8], x, fmaf(c->m[9], y, fmaf(c->m[10], z, c->m[11])));
    r.w = fmaf(c->m[12], x, fmaf(c->m[13], y, fmaf(c->m[14], z, c->m[15])));
    return r;
}

static float screen(float ndc, float size)
{
    float t = fmaf(ndc, 0.5f, 0.5f);
    return t * size;
}

/* the integer range of the points node (L, key) can hold, per axis */
static void node_box(const orc_node* nd, const orc_cube* cb, float lo[3], float hi[3])
{
    uint64_t c[3] = {0, 0, 0};
    for (int b = 0; b < nd->level; ++b)
        for (int a = 0; a < 3; ++a) c[a] |= ((nd->key >> (3 * b + (2 - a))) & 1u) << b;
    uint64_t den = 1ull << nd->level;
    for (int a = 0; a < 3; ++a) {
        uint64_t first = (c[a] * cb->S + den - 1) / den;         /* ceil(c S / 2^L) */
        uint64_t next = ((c[a] + 1) * cb->S + den - 1) / den;    /* ceil((c + 1) S / 2^L) */
        lo[a] = (float)((int64_t)cb->o[a] + (int64_t)first);
        hi[a] = (float)((int64_t)cb->o[a] + (int64_t)next - 1);
    }
}

/* visible: not all corners beyond one clip plane; refine: visible, inner, and
 * the screen extent of the corners above min_node_px (or a corner behind) */
static void node_flags(const orc_node* nd, const orc_cube* cb, const orc_camera* cam, int* visible, int* refine)
{
    float lo[3], hi[3];
    node_box(nd, cb, lo, hi);
    int out[6] = {1, 1, 1, 1, 1, 1}, behind = 0, any = 0;
    float x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    for (int k = 0; k < 8; ++k) {
        orc_clip c = clip_of(cam, (k & 4) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 1) ? hi[2] : lo[2]);
        out[0] &= c.x < -c.w;
        out[1] &= c.x > c.w;
        out[2] &= c.y < -c.w;
        out[3] &= c.y > c.w;
        out[4] &= c.z < 0.f;
        out[5] &= c.z > c.w;
        if (c.w <= 0.f) { behind = 1; continue; }
        float sx = screen(c.x / c.w, (float)cam->width), sy = screen(c.y / c.w, (float)cam->height);
        if (!any || sx < x0) x0 = sx;
        if (!any || sx > x1) x1 = sx;
        if (!any || sy < y0) y0 = sy;
        if (!any || sy > y1) y1 = sy;
        any = 1;
    }
    *visible = !(out[0] || out[1] || out[2] || out[3] || out[4] || out[5]);
    float w = x1 - x0, h = y1 - y0;
    float size = w > h ? w : h;
    *refine = *visible && !nd->is_leaf && (behind || size > cam->min_node_px);
}

/* preorder walk: a node is drawn when visible and its parent refined */
static void select_visit(const orc_node* nodes, uint32_t i, const orc_cube* cb, const orc_camera* cam,
                         uint32_t* sel, uint32_t* ns)
{
    int visible, refine;
    node_flags(&nodes[i], cb, cam, &visible, &refine);
    if (visible) sel[(*ns)++] = i;
    if (!refine) return;
    for (uint32_t j = i + 1; j <= i + nodes[i].n_desc; j += nodes[j].n_desc + 1) select_visit(nodes, j, cb, cam, sel, ns);
}

uint32_t orc_render_select(const orc_node* nodes, uint32_t M, const orc_cube* cube, const orc_camera* cam,
                           uint32_t* sel)
{
    uint32_t ns = 0;
    if (M) select_visit(nodes, 0, cube, cam, sel, &ns);
    return ns;
}

void orc_rasterize(const orc_node* nodes, const uint32_t* sel, uint32_t nsel, const orc_point* final_pts,
                   const orc_camera* cam, uint64_t* fb)
{
    uint64_t npx = (uint64_t)cam->width * cam->height;
    for (uint64_t q = 0; q < npx; ++q) fb[q] = ~0ull;
    for (uint32_t k = 0; k < nsel; ++k) {
        const orc_node* nd = &nodes[sel[k]];
        for (uint64_t i = nd->first; i < nd->first + nd->n_own; ++i) {
            const orc_point* p = &final_pts[i];
            orc_clip c = clip_of(cam, (float)p->x, (float)p->y, (float)p->z);
            if (!(c.w > 0.f) || c.x < -c.w || c.x > c.w || c.y < -c.w || c.y > c.w || c.z < 0.f || c.z > c.w) continue;
            float sx = screen(c.x / c.w, (float)cam->width), sy = screen(c.y / c.w, (float)cam->height);
            uint32_t px = (uint32_t)floorf(sx), py = (uint32_t)floorf(sy);
            if (px > cam->width - 1) px = cam->width - 1;
            if (py > cam->height - 1) py = cam->height - 1;
            float depth = c.z / c.w + 0.0f;
            uint32_t dbits, rgba;
            memcpy(&dbits, &depth, 4);
            memcpy(&rgba, &p->r, 4);
            uint64_t v = ((uint64_t)dbits << 32) | rgba;
            uint64_t at = (uint64_t)py * cam->width + px;
            if (v < fb[at]) fb[at] = v;
        }
    }
}
