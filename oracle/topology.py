"""Stencils of a consistently oriented manifold triangle mesh (oracle; test infrastructure only).

Edge-based stencil (Section 4.3, Figure "corotational_edge_based_hinge"): hinge edge 2-3 with wing
vertices 1 and 4; triangles T123 and T432 are the mesh's own triangles with their own orientation.

Triangle-centred stencil (Section 4.4-4.5, App. C Eq. 78): central triangle 1-2-3 and the vertex i+3 of
the neighbour across the edge opposite vertex i.

Boundary edges (Section 4.3 "Boundary conditions", Eq. 30-31, Eq. 58-61): the missing neighbour of a
boundary edge MN of triangle LMN is a virtual node L' = M + N - L (the point reflection of L through the
edge midpoint). Free boundary edges carry no edge stencil; clamped ones carry an edge stencil
L-M-N-L'. Triangle stencils keep the virtual node and record the edge's condition.

Reading (relabelling): a triangle stencil with at least one free boundary edge is rotated cyclically so
that its first free edge, in the order (1->2, 2->3, 3->1), becomes edge 1->2. The corotational x axis
(along x_12, App. A) then runs along that boundary, which is the frame in which the twist term is
dropped for the FVM hinge (Section 4.4, boundary conditions).
"""
from __future__ import annotations

import numpy as np

INTERIOR, FREE, CLAMPED = 0, 1, 2


def _directed_edges(tris):
    """Map directed edge (p, q) -> (triangle index, vertex opposite the edge)."""
    owner = {}
    for t, (a, b, c) in enumerate(np.asarray(tris).tolist()):
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            if (p, q) in owner:
                raise ValueError(f"edge {p}->{q} used twice: mesh is non-manifold or inconsistently oriented")
            owner[(p, q)] = (t, r)
    return owner


def build_stencils(tris, n_verts, clamped_edges=()):
    """Return the stencil sets of a mesh.

    Returns a dict with

    * ``edge``: int64 [E,4] vertex indices (x1, x2, x3, x4) of interior-edge stencils,
    * ``edge_clamped``: int64 [Ec,3] (L, M, N) for clamped boundary edges; the fourth node is virtual,
    * ``tri``: int64 [T,6] triangle stencils (relabelled), -1 marks a virtual neighbour,
    * ``tri_bc``: int8 [T,3] condition of hinge i (edge opposite vertex i): INTERIOR, FREE or CLAMPED,
    * ``tri_orig``: int64 [T] index of the source triangle.
    """
    tris = np.asarray(tris, dtype=np.int64)
    owner = _directed_edges(tris)
    clamped = set()
    for a, b in np.asarray(clamped_edges, dtype=np.int64).reshape(-1, 2).tolist():
        clamped.add((a, b))
        clamped.add((b, a))

    edge, edge_cl = [], []
    for (p, q), (t, r) in owner.items():
        twin = owner.get((q, p))
        if twin is not None:
            if p < q:
                edge.append((r, p, q, twin[1]))
        elif (p, q) in clamped:
            edge_cl.append((r, p, q))
    for a, b in clamped:
        if (a, b) in owner and (b, a) in owner:
            raise ValueError(f"clamped edge {a}-{b} is not a boundary edge")

    tri, tri_bc = [], []
    for t, (v1, v2, v3) in enumerate(tris.tolist()):
        def hinge(a, b):  # neighbour vertex across directed edge a->b, and its condition
            twin = owner.get((b, a))
            if twin is not None:
                return twin[1], INTERIOR
            return -1, (CLAMPED if (a, b) in clamped else FREE)

        verts = [v1, v2, v3]
        # relabel so that the first free edge (order 12, 23, 31) becomes edge 1->2
        for rot in range(3):
            a, b = verts[rot], verts[(rot + 1) % 3]
            if hinge(a, b)[1] == FREE:
                verts = verts[rot:] + verts[:rot]
                break
        v1, v2, v3 = verts
        n4, c4 = hinge(v2, v3)  # across the edge opposite vertex 1
        n5, c5 = hinge(v3, v1)  # opposite vertex 2
        n6, c6 = hinge(v1, v2)  # opposite vertex 3
        tri.append((v1, v2, v3, n4, n5, n6))
        tri_bc.append((c4, c5, c6))

    return {
        "edge": np.asarray(edge, dtype=np.int64).reshape(-1, 4),
        "edge_clamped": np.asarray(edge_cl, dtype=np.int64).reshape(-1, 3),
        "tri": np.asarray(tri, dtype=np.int64).reshape(-1, 6),
        "tri_bc": np.asarray(tri_bc, dtype=np.int8).reshape(-1, 3),
    }


HINGE_EDGE = ((1, 2), (2, 0), (0, 1))
"""Hinge i of a triangle stencil (0-based): the central edge (a_i -> b_i) opposite central vertex i; its
neighbour is vertex i+3 (App. C Eq. 78)."""


def stencil_positions(pos, tri, tri_bc=None):
    """Gather [T,6,3] positions of triangle stencils; virtual neighbours become M + N - L."""
    tri = np.asarray(tri)
    X = np.zeros(tri.shape + (3,))
    X[:, :3] = pos[tri[:, :3]]
    for i, (a, b) in enumerate(HINGE_EDGE):
        real = tri[:, 3 + i] >= 0
        X[real, 3 + i] = pos[tri[real, 3 + i]]
        virt = ~real
        X[virt, 3 + i] = X[virt, a] + X[virt, b] - X[virt, i]
    return X
