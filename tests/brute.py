"""Brute force of the hot path's definitions in pure Python integers, for
clouds of a few hundred points.  Written independently of the C oracle (no
shared code, different structure: dictionaries, recursion on point sets, the
LOD owner found by searching down each point's path).  It pins the oracle.
"""


def cube(pts):
    if not pts:
        return (0, 0, 0), (0, 0, 0), 0
    lo = tuple(min(p[a] for p in pts) for a in range(3))
    hi = tuple(max(p[a] for p in pts) for a in range(3))
    return lo, hi, max(hi[a] - lo[a] for a in range(3)) + 1


def cell(p, cb, level):
    """per-axis floor((p - o) * 2^level / S) with Python's exact integers"""
    o, _, S = cb
    return tuple(((p[a] - o[a]) * (1 << level)) // S for a in range(3))


def key(p, cb, level):
    c = cell(p, cb, level)
    k = 0
    for b in reversed(range(level)):
        k = k * 8 + ((c[0] >> b) & 1) * 4 + ((c[1] >> b) & 1) * 2 + ((c[2] >> b) & 1)
    return k


def splitmix64(i):
    M = (1 << 64) - 1
    z = (i + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def counts(pts, cb, g):
    out = {}
    for p in pts:
        k = key(p, cb, g)
        out[k] = out.get(k, 0) + 1
    return out


def chunks(cnt, g, T):
    """[(level, key, count)] in Morton preorder"""
    def node_count(level, k):
        sh = 3 * (g - level)
        return sum(v for m, v in cnt.items() if (m >> sh) == k)

    res = []

    def visit(level, k):
        c = node_count(level, k)
        if c == 0:
            return
        if c <= T or level == g:
            res.append((level, k, c))
            return
        for j in range(8):
            visit(level + 1, 8 * k + j)

    visit(0, 0)
    return res


def distribute(pts, cb, g, chs):
    def chunk_of(p):
        m = key(p, cb, g)
        for q, (level, k, _) in enumerate(chs):
            if (m >> (3 * (g - level))) == k:
                return q
        raise AssertionError("point outside every chunk")
    order = sorted(range(len(pts)), key=lambda i: (chunk_of(pts[i]), i))
    return order


def tree(pts, cb, C, Lmax):
    """nodes in preorder: dict(level, key, members (sorted list), leaf, children)"""
    nodes = []

    def make(level, k, members):
        me = dict(level=level, key=k, members=members, leaf=True, children=[])
        nodes.append(me)
        if len(members) > C and level < Lmax:
            me["leaf"] = False
            for j in range(8):
                sub = [i for i in members if key(pts[i], cb, level + 1) == 8 * k + j]
                if sub:
                    me["children"].append(make(level + 1, 8 * k + j, sub))
        return me

    if pts:
        make(0, 0, list(range(len(pts))))
    return nodes


def lod_owner_levels(pts, cb, nodes, s):
    """For each point: walk its path from the root; the first inner node at
    level K for which the point is the smallest index of its level-(K+s) cell
    owns it, else its leaf does."""
    leaf_level = {}
    for nd in nodes:
        if nd["leaf"]:
            for i in nd["members"]:
                leaf_level[i] = nd["level"]
    cell_min = {}
    for i, p in enumerate(pts):
        for l in range(22):
            kk = (l, key(p, cb, l))
            if kk not in cell_min or i < cell_min[kk]:
                cell_min[kk] = i
    owner = {}
    for i, p in enumerate(pts):
        owner[i] = leaf_level[i]
        for K in range(leaf_level[i]):
            if cell_min[(K + s, key(p, cb, K + s))] == i:
                owner[i] = K
                break
    return owner, leaf_level


def build(pts, g, s, Lmax, C, T):
    """Everything: returns a dict mirroring the oracle's outputs (as lists)."""
    cb = cube(pts)
    cnt = counts(pts, cb, g)
    chs = chunks(cnt, g, T)
    dist = distribute(pts, cb, g, chs)
    nodes = tree(pts, cb, C, Lmax)
    owner, leaf_level = lod_owner_levels(pts, cb, nodes, s)
    leaf_perm = [i for nd in nodes if nd["leaf"] for i in nd["members"]]
    final_perm, n_own = [], []
    for nd in nodes:
        own = sorted(i for i in nd["members"] if owner[i] == nd["level"])
        final_perm += own
        n_own.append(len(own))
    return dict(cube=cb, counts=cnt, chunks=chs, dist_perm=dist, nodes=nodes,
                leaf_perm=leaf_perm, final_perm=final_perm, n_own=n_own, owner_level=owner,
                leaf_level=leaf_level)
