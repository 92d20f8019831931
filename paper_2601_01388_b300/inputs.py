"""Seeded synthetic inputs: data graphs in CSR form and pattern edge lists.

This module holds no arithmetic of the counting method; it only builds the
inputs that both the CUDA library and the CPU oracle consume.  Graphs are
undirected and stored with both directions: int64 row offsets, int32 column ids,
rows sorted ascending, no duplicates, no self-loops (the setting of Sec. 2).

The paper's data sets (LiveJournal, UK-2002, Twitter, Friendster, gsh-2015;
Table 1) are not available here; R-MAT and Chung-Lu graphs of matching shape
stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# CSR construction
# --------------------------------------------------------------------------


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """Symmetrise, drop self-loops, deduplicate and sort: returns (off int64[n+1],
    cols int32[nnz])."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    keys = np.concatenate([src * n + dst, dst * n + src])
    del src, dst
    keys.sort()
    if len(keys):
        first = np.empty(len(keys), dtype=bool)
        first[0] = True
        np.not_equal(keys[1:], keys[:-1], out=first[1:])
        keys = keys[first]                      # sorted, deduplicated
    rows = keys // n
    cols = (keys - rows * n).astype(np.int32)
    del keys
    counts = np.bincount(rows, minlength=n)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off, cols


def relabel(off, cols, perm):
    """Apply the vertex bijection v -> perm[v] and rebuild a sorted CSR."""
    n = len(off) - 1
    deg = np.diff(off)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    return csr_from_edges(n, perm[rows], perm[cols.astype(np.int64)])


def edges_of(off, cols):
    """Undirected edge list (u < v) of a CSR graph."""
    n = len(off) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    c = cols.astype(np.int64)
    m = rows < c
    return rows[m], c[m]


# --------------------------------------------------------------------------
# Small deterministic graphs
# --------------------------------------------------------------------------


def complete_graph(n):
    a, b = np.triu_indices(n, 1)
    return csr_from_edges(n, a, b)


def cycle_graph(n):
    a = np.arange(n)
    return csr_from_edges(n, a, (a + 1) % n)


def path_graph(n):
    a = np.arange(n - 1)
    return csr_from_edges(n, a, a + 1)


def star_graph(leaves):
    return csr_from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1))


def gnp_graph(n, p, seed):
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x6E70]))
    a, b = np.triu_indices(n, 1)
    m = rng.random(len(a)) < p
    return csr_from_edges(n, a[m], b[m])


def random_tree(n, seed):
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x7472]))
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    return csr_from_edges(n, np.arange(1, n), parent)


def disjoint_union(*graphs):
    srcs, dsts, base = [], [], 0
    for off, cols in graphs:
        s, d = edges_of(off, cols)
        srcs.append(s + base)
        dsts.append(d + base)
        base += len(off) - 1
    return csr_from_edges(base, np.concatenate(srcs), np.concatenate(dsts))


# --------------------------------------------------------------------------
# R-MAT (Chakrabarti, Zhan & Faloutsos, SDM'04) and Chung-Lu power-law graphs
# --------------------------------------------------------------------------


def rmat_edges(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed=1,
               chunk=1 << 24):
    """ef * 2^scale directed edge draws; each picks one of four quadrants per level
    with probabilities (a, b, c, 1-a-b-c), no noise."""
    m = edge_factor << scale
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x524D4154]))
    ta = np.uint64(int(a * 2.0 ** 64))
    tab = np.uint64(int((a + b) * 2.0 ** 64))
    tabc = np.uint64(int(min(a + b + c, 1.0 - 2.0 ** -53) * 2.0 ** 64))
    src = np.empty(m, dtype=np.int64)
    dst = np.empty(m, dtype=np.int64)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.int64)
        d = np.zeros(hi - lo, dtype=np.int64)
        for level in range(scale):
            r = rng.bit_generator.random_raw(hi - lo)
            bit = np.int64(1) << np.int64(scale - 1 - level)
            down = r >= tab                     # quadrants c, d: source bit set
            right = ((r >= ta) & (r < tab)) | (r >= tabc)   # quadrants b, d
            s |= np.where(down, bit, 0)
            d |= np.where(right, bit, 0)
        src[lo:hi] = s
        dst[lo:hi] = d
    return src, dst


def rmat_graph(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed=1,
               permute=True):
    """R-MAT graph as sorted undirected CSR.  With ``permute`` the vertex ids go
    through a seeded random bijection (as Graph500 does) so that hubs are spread."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, a, b, c, seed)
    if permute:
        rng = np.random.Generator(np.random.Philox(key=[seed, 0x5045524D]))
        perm = rng.permutation(n).astype(np.int64)
        src = perm[src]
        dst = perm[dst]
    return csr_from_edges(n, src, dst)


def chung_lu_graph(n: int, gamma: float = 2.1, mean_degree: float = 32.0, seed=1):
    """Chung-Lu graph with expected degrees w_i proportional to (i + i0)^(-1/(gamma-1)),
    scaled to the requested mean; n*mean/2 endpoint pairs are drawn in proportion to w."""
    alpha = 1.0 / (gamma - 1.0)
    i0 = 1.0
    for _ in range(60):                      # choose i0 so that w_0 ~ sqrt(sum w)
        w = (np.arange(n) + i0) ** -alpha
        w *= mean_degree * n / w.sum()
        if w[0] <= math.sqrt(w.sum()):
            break
        i0 *= 2.0
    p = w / w.sum()
    cdf = np.cumsum(p)
    m = int(n * mean_degree / 2)
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x434C]))
    src = np.searchsorted(cdf, rng.random(m) * cdf[-1], side="right")
    dst = np.searchsorted(cdf, rng.random(m) * cdf[-1], side="right")
    src = np.minimum(src, n - 1)
    dst = np.minimum(dst, n - 1)
    perm = rng.permutation(n).astype(np.int64)
    return csr_from_edges(n, perm[src], perm[dst])


def dense_graph_rows(n: int, u0: int, u1: int):
    """Rows u0..u1-1 of dense_graph(n) as a boolean adjacency block ((u1-u0) x n).
    {u, v} (u != v) is an edge unless (u XOR v) & 7 == 0, (u + v) & 31 == 5,
    u & v & 0x300 == 0x300 or (u | v) & 0x1C00 == 0; every rule is symmetric in u
    and v, and u XOR u = 0 drops the diagonal.  About 80% of the pairs are edges; the
    last two rules split the vertices into degree classes by bits 8-12 of their id."""
    u = np.arange(u0, u1, dtype=np.int64)[:, None]
    w = np.arange(n, dtype=np.int64)[None, :]
    keep = (((u ^ w) & 7) != 0) & (((u + w) & 31) != 5)
    keep &= ((u & w & 0x300) != 0x300) & (((u | w) & 0x1C00) != 0)
    return keep


def dense_graph(n: int, rows_per_chunk: int = 256):
    """The dense, deterministic graph of dense_graph_rows as a sorted CSR, built in two
    passes over row blocks (counts, then columns).  With n = 54000 it has about 2.3e9
    directed entries, past the int32 range of CSR positions."""
    off = np.zeros(n + 1, dtype=np.int64)
    for u0 in range(0, n, rows_per_chunk):
        u1 = min(n, u0 + rows_per_chunk)
        off[u0 + 1:u1 + 1] = dense_graph_rows(n, u0, u1).sum(axis=1)
    np.cumsum(off, out=off)
    cols = np.empty(int(off[-1]), dtype=np.int32)
    for u0 in range(0, n, rows_per_chunk):
        u1 = min(n, u0 + rows_per_chunk)
        cols[off[u0]:off[u1]] = np.nonzero(dense_graph_rows(n, u0, u1))[1].astype(np.int32)
    return off, cols


# --------------------------------------------------------------------------
# Patterns (k vertices, undirected edge list)
# --------------------------------------------------------------------------


def clique(k):
    return k, [(i, j) for i in range(k) for j in range(i + 1, k)]


def cycle(k):
    return k, [(i, (i + 1) % k) if i < (i + 1) % k else ((i + 1) % k, i) for i in range(k)]


def path(k):
    return k, [(i, i + 1) for i in range(k - 1)]


def star(leaves):
    return leaves + 1, [(0, i) for i in range(1, leaves + 1)]


PATTERNS = {
    "edge": (2, [(0, 1)]),
    "triangle": clique(3),
    "4-cycle": cycle(4),
    "4-clique": clique(4),
    "5-cycle": cycle(5),
    # square 0-1-2-3 with a roof vertex 4 joined to 0 and 1
    "house": (5, [(0, 1), (1, 2), (2, 3), (0, 3), (0, 4), (1, 4)]),
    "5-clique": clique(5),
    "6-clique": clique(6),
    "7-cycle": cycle(7),
    "tailed-triangle": (4, [(0, 1), (1, 2), (0, 2), (2, 3)]),
    "diamond": (4, [(0, 1), (1, 2), (2, 3), (0, 3), (0, 2)]),        # chordal 4-cycle
    "chordal-5-cycle": (5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4), (0, 2), (0, 3)]),
    "3-path": path(3),
    "4-path": path(4),
    "3-star": star(3),
    "4-star": star(4),
}


def random_connected_pattern(rng, kmin=3, kmax=8, p_extra=0.3):
    """A random connected pattern: a Pruefer-sequence tree on k vertices plus each
    remaining pair as an edge with probability p_extra."""
    k = int(rng.integers(kmin, kmax + 1))
    edges = set()
    if k == 2:
        edges.add((0, 1))
    else:
        seq = [int(x) for x in rng.integers(0, k, size=k - 2)]
        degree = [1] * k
        for x in seq:
            degree[x] += 1
        for x in seq:
            leaf = min(i for i in range(k) if degree[i] == 1)
            edges.add((min(leaf, x), max(leaf, x)))
            degree[leaf] -= 1
            degree[x] -= 1
        u, v = [i for i in range(k) if degree[i] == 1]
        edges.add((u, v))
    for i in range(k):
        for j in range(i + 1, k):
            if (i, j) not in edges and rng.random() < p_extra:
                edges.add((i, j))
    return k, sorted(edges)


def batch_queries(n=64, seed=1, log2_min=16, log2_max=26):
    """The 64-query batch: families clique/cycle/path/star of 3..7 vertices plus
    tailed triangle, diamond and chordal 5-cycle; budgets 2^(16+10u), u uniform."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x42415443]))
    fams = ["clique", "cycle", "path", "star", "tailed-triangle", "diamond", "chordal-5-cycle"]
    out = []
    for _ in range(n):
        f = fams[int(rng.integers(0, len(fams)))]
        size = int(rng.integers(3, 8))
        if f == "clique":
            pat = clique(size)
        elif f == "cycle":
            pat = cycle(size)
        elif f == "path":
            pat = path(size)
        elif f == "star":
            pat = star(size - 1)
        else:
            pat = PATTERNS[f]
        budget = int(2.0 ** (log2_min + (log2_max - log2_min) * rng.random()))
        out.append((f if f not in ("clique", "cycle", "path", "star") else f"{size}-{f}", pat, budget))
    return out
