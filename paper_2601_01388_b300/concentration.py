"""Pattern concentration (Sec. 6.3): the share of each connected k-vertex pattern
among all connected k-vertex patterns of a graph, from one estimate per pattern.

The sampler estimates non-induced counts (C(G,P) embeddings, C(G,P)/|Aut(P)|
subgraphs).  Concentrations are those subgraph counts normalised by their total
over the connected patterns of the size.  Induced counts, which random-walk
methods estimate, follow from the non-induced ones through the spanning-copy
matrix S: the k-vertex sets that induce Q contain S[P][Q] copies of P, so
N = S I with S unit upper triangular once patterns are ordered by edge count.

Host-side bookkeeping only: no step of the sampling runs here.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np


def _pairs(k):
    return [(i, j) for i in range(k) for j in range(i + 1, k)]


def _connected(k, edges):
    adj = [[] for _ in range(k)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen, stack = {0}, [0]
    while stack:
        for y in adj[stack.pop()]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == k


@lru_cache(maxsize=None)
def connected_patterns(k: int):
    """The connected graphs on k vertices up to isomorphism (1, 1, 2, 6, 21, 112 for
    k = 1..6), ordered by edge count, then by canonical edge mask.  The canonical
    form of an edge set is the smallest mask over all relabellings, the mask having
    bit t set when pair t of (0,1), (0,2), ..., (k-2,k-1) is an edge."""
    if not 1 <= k <= 6:
        raise ValueError("k must be in 1..6")
    pairs = _pairs(k)
    index = {p: t for t, p in enumerate(pairs)}
    masks = np.arange(1 << len(pairs), dtype=np.int64)
    best = masks.copy()
    for perm in itertools.permutations(range(k)):
        img = np.zeros_like(masks)
        for t, (a, b) in enumerate(pairs):
            x, y = perm[a], perm[b]
            img |= ((masks >> t) & 1) << index[(min(x, y), max(x, y))]
        np.minimum(best, img, out=best)
    out = []
    for m in np.unique(best).tolist():
        edges = [pairs[t] for t in range(len(pairs)) if m >> t & 1]
        if _connected(k, edges):
            out.append((len(edges), m, (k, edges)))
    out.sort()
    return tuple(p for _, _, p in out)


def _automorphisms(k, edges):
    es = {frozenset(e) for e in edges}
    return sum(1 for perm in itertools.permutations(range(k))
               if all(frozenset((perm[a], perm[b])) in es for a, b in edges))


def spanning_copies(p, q) -> int:
    """Edge subsets of q (on all of q's vertices) that form a copy of p: bijections
    V_p -> V_q mapping every edge of p onto an edge of q, divided by |Aut(p)|."""
    k, pe = p
    kq, qe = q
    if k != kq:
        raise ValueError("patterns of different sizes")
    qs = {frozenset(e) for e in qe}
    maps = sum(1 for perm in itertools.permutations(range(k))
               if all(frozenset((perm[a], perm[b])) in qs for a, b in pe))
    return maps // _automorphisms(k, pe)


@lru_cache(maxsize=None)
def spanning_matrix(k: int) -> np.ndarray:
    pats = connected_patterns(k)
    return np.array([[spanning_copies(p, q) for q in pats] for p in pats], dtype=np.int64)


def subgraph_counts(embeddings, k: int) -> np.ndarray:
    """Non-induced subgraph counts C(G,P)/|Aut(P)| from embedding estimates given in
    the order of connected_patterns(k)."""
    pats = connected_patterns(k)
    return np.asarray(embeddings, dtype=np.float64) / np.array([_automorphisms(*p) for p in pats], float)


def induced_counts(subgraphs, k: int) -> np.ndarray:
    """Induced counts I from non-induced subgraph counts N by back substitution in
    N = S I (S unit upper triangular)."""
    S = spanning_matrix(k).astype(np.float64)
    n = np.asarray(subgraphs, dtype=np.float64)
    out = np.zeros_like(n)
    for i in range(len(n) - 1, -1, -1):
        out[i] = n[i] - S[i, i + 1:] @ out[i + 1:]
    return out


def concentration(counts) -> np.ndarray:
    c = np.asarray(counts, dtype=np.float64)
    return c / c.sum()


def variation_distance(a, b) -> float:
    """Half the L1 distance between two concentration vectors (Sec. 6.3)."""
    return 0.5 * float(np.abs(np.asarray(a, float) - np.asarray(b, float)).sum())
