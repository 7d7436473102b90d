"""Plain CPU oracle of the physics-to-render dual-mesh mapping (§III-D.1, Eqs. 5-6).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's CPU-baseline leg may use this
module; it shares no code with the CUDA library.

The fine render mesh of a deformable body is its coarse simulation surface after L levels of Loop
subdivision.  Each level is linear in the vertex positions, so the whole subdivision is one sparse
matrix W = S^(L) ... S^(1) (Eq. 5), precomputed once, and the fine positions of every frame are
X_f = W X_c (Eq. 6).

One level of Loop subdivision (Loop 1987), on a triangle mesh:
  * every edge gets a new vertex: 3/8 (a + b) + 1/8 (c + d) for an interior edge (a, b) with opposite
    vertices c and d, (a + b) / 2 for a boundary edge;
  * every old vertex v of valence n moves to (1 - n beta) v + beta sum of its neighbours, with
    beta = (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n; a boundary vertex to 3/4 v + 1/8 (its two boundary
    neighbours);
  * every triangle (a, b, c) becomes four: (a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca).
New vertices are numbered after the old ones, in the order of the sorted unique edges.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def loop_beta(n: int) -> float:
    return (5.0 / 8.0 - (3.0 / 8.0 + 0.25 * math.cos(2.0 * math.pi / n)) ** 2) / n


def loop_level(tris: np.ndarray, n_verts: int):
    """One subdivision level: (S (n_new x n_verts) as CSR, the new triangles)."""
    tris = np.asarray(tris, dtype=np.int64)
    # edges with the opposite vertex of every triangle side
    edge_opp = {}
    for t in tris:
        for k in range(3):
            a, b, c = int(t[k]), int(t[(k + 1) % 3]), int(t[(k + 2) % 3])
            key = (min(a, b), max(a, b))
            edge_opp.setdefault(key, []).append(c)
    edges = sorted(edge_opp)
    edge_id = {e: n_verts + i for i, e in enumerate(edges)}
    n_new = n_verts + len(edges)
    rows, cols, vals = [], [], []
    # neighbours and boundary neighbours of the old vertices
    nbrs = [set() for _ in range(n_verts)]
    bnd = [[] for _ in range(n_verts)]
    for (a, b), opp in edge_opp.items():
        nbrs[a].add(b)
        nbrs[b].add(a)
        if len(opp) == 1:
            bnd[a].append(b)
            bnd[b].append(a)
    for v in range(n_verts):
        if bnd[v]:
            rows += [v, v, v]
            cols += [v, bnd[v][0], bnd[v][1]]
            vals += [0.75, 0.125, 0.125]
        elif nbrs[v]:
            n = len(nbrs[v])
            beta = loop_beta(n)
            rows.append(v); cols.append(v); vals.append(1.0 - n * beta)
            for u in sorted(nbrs[v]):
                rows.append(v); cols.append(u); vals.append(beta)
        else:  # a vertex of no triangle keeps its position
            rows.append(v); cols.append(v); vals.append(1.0)
    for (a, b) in edges:
        i = edge_id[(a, b)]
        opp = edge_opp[(a, b)]
        if len(opp) == 2:
            rows += [i, i, i, i]
            cols += [a, b, opp[0], opp[1]]
            vals += [0.375, 0.375, 0.125, 0.125]
        else:
            rows += [i, i]
            cols += [a, b]
            vals += [0.5, 0.5]
    S = sp.csr_matrix((vals, (rows, cols)), shape=(n_new, n_verts))
    S.sum_duplicates()
    new_tris = []
    for t in tris:
        a, b, c = (int(x) for x in t)
        ab, bc, ca = edge_id[(min(a, b), max(a, b))], edge_id[(min(b, c), max(b, c))], edge_id[(min(c, a), max(c, a))]
        new_tris += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    return S, np.asarray(new_tris, dtype=np.int64)


def subdivision_matrix(tris: np.ndarray, n_verts: int, levels: int):
    """W = S^(L) ... S^(1) (Eq. 5) and the fine triangles after `levels` levels."""
    W = sp.identity(n_verts, format="csr")
    t, n = np.asarray(tris, dtype=np.int64), n_verts
    for _ in range(levels):
        S, t = loop_level(t, n)
        W = (S @ W).tocsr()
        n = S.shape[0]
    W.sum_duplicates()
    W.sort_indices()
    return W, t


def fine_positions(W, Xc):
    """X_f = W X_c (Eq. 6)."""
    return W @ np.asarray(Xc, dtype=np.float64)
