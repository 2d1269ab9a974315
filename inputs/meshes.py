"""Structured simplicial meshes of the unit square and the unit cube.

These are seeded-input generators shared by the oracle, the tests and the
benchmark. They hold mesh topology and coordinates only, none of the DPP
method's arithmetic.

Node numbering is lexicographic with x fastest. The DoF count of the
four-field P1 system on these meshes is (N+1)^2 * 6 in 2D and (N+1)^3 * 8 in
3D. These are the CG-VMS TRI and TET columns of the paper's h-size vs DoF
tables (Section 5.1, Table "2D h-size vs DoF"; Section 5.2, Table "h-size vs
DoF"). The Q1 meshes (QUAD, HEX: Table "ELE_level_discretization") have the
same nodes, so the same counts (the QUAD and HEX columns of those tables).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    dim: int
    coords: np.ndarray      # float64 [n_nodes, dim]
    cells: np.ndarray       # int32 [n_cells, dim+1] (simplices) or [n_cells, 2^dim] (Q1)
    bfacets: np.ndarray     # int32 [n_bfacets, dim] or [n_bfacets, 2^(dim-1)]: boundary facets
    n: int                  # cells per edge of the unit square / cube
    kind: str = "simplex"   # "simplex" (P1 triangles, tetrahedra) or "q1" (quads, hexahedra)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_bfacets(self) -> int:
        return int(self.bfacets.shape[0])

    @property
    def dofs_per_node(self) -> int:
        return 2 * self.dim + 2

    @property
    def n_dofs(self) -> int:
        return self.n_nodes * self.dofs_per_node


def boundary_facets(cells: np.ndarray, dim: int) -> np.ndarray:
    """Facets that belong to exactly one cell, each as its sorted node ids."""
    nv = dim + 1
    facets = []
    for drop in range(nv):
        keep = [v for v in range(nv) if v != drop]
        facets.append(cells[:, keep])
    f = np.sort(np.concatenate(facets, axis=0).astype(np.int64), axis=1)
    # Encode each sorted facet as one int64 key (node ids < 2^21).
    key = np.zeros(f.shape[0], dtype=np.int64)
    for c in range(dim):
        key = key * (1 << 21) + f[:, c]
    uniq, idx, counts = np.unique(key, return_index=True, return_counts=True)
    return f[idx[counts == 1]].astype(np.int32)


def unit_square_tri(n: int) -> Mesh:
    """N x N squares on [0,1]^2, each cut along the (i,j)->(i+1,j+1) diagonal."""
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    coords = np.stack([i.ravel() / n, j.ravel() / n], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    n00 = (ci + m * cj).ravel()
    n10 = n00 + 1
    n01 = n00 + m
    n11 = n00 + m + 1
    t1 = np.stack([n00, n10, n11], axis=1)
    t2 = np.stack([n00, n11, n01], axis=1)
    cells = np.empty((2 * n * n, 3), dtype=np.int32)
    cells[0::2] = t1
    cells[1::2] = t2
    return Mesh(2, coords, cells, boundary_facets(cells, 2), n)


def unit_cube_kuhn(n: int) -> Mesh:
    """N^3 cubes on [0,1]^3, each cut into the six Kuhn tetrahedra.

    Each tetrahedron is the monotone lattice path 0 -> e_s0 -> e_s0+e_s1 ->
    (1,1,1) for one permutation s of the three axes; all six share the
    main diagonal of the cube.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([i.ravel() / n, j.ravel() / n, k.ravel() / n], axis=1).astype(np.float64)
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = (ci + m * (cj + m * ck)).ravel()
    step = np.array([1, m, m * m], dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        v0 = base
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v2 + step[perm[2]]
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return Mesh(3, coords, cells, boundary_facets(cells, 3), n)


def disc_wheel(sectors: int, rings: int) -> Mesh:
    """Triangles of a regular polygon of radius 1: a centre node and `rings`
    concentric rings of `sectors` nodes. The centre lies in `sectors` cells,
    every other interior node in 6, so a large `sectors` gives one node with
    many more cells (and neighbours) than the structured meshes have.
    ``n`` of the returned mesh is `rings`.
    """
    if sectors < 3 or rings < 1:
        raise ValueError("need sectors >= 3 and rings >= 1")
    th = 2.0 * np.pi * np.arange(sectors) / sectors
    coords = [np.zeros((1, 2))]
    for r in range(1, rings + 1):
        coords.append(np.stack([r / rings * np.cos(th), r / rings * np.sin(th)], axis=1))
    coords = np.concatenate(coords).astype(np.float64)
    ring = lambda r, j: 1 + (r - 1) * sectors + (j % sectors)
    cells = []
    for j in range(sectors):
        cells.append((0, ring(1, j), ring(1, j + 1)))
    for r in range(1, rings):
        for j in range(sectors):
            a, b = ring(r, j), ring(r, j + 1)
            c, d = ring(r + 1, j), ring(r + 1, j + 1)
            cells.append((a, c, d))
            cells.append((a, d, b))
    cells = np.asarray(cells, dtype=np.int32)
    return Mesh(2, coords, cells, boundary_facets(cells, 2), rings)


def tensor_facets(dim: int):
    """Local vertex lists of the 2*dim facets of a tensor-ordered Q1 cell.

    Vertex v of the cell sits at the corner whose coordinate bits are
    (v & 1, (v >> 1) & 1, (v >> 2) & 1). The facet on side s of axis k holds
    the vertices with bit k equal to s, in increasing order. That order is
    itself the tensor order of the facet.
    """
    nv = 1 << dim
    return [[v for v in range(nv) if ((v >> k) & 1) == side]
            for k in range(dim) for side in (0, 1)]


def boundary_facets_q1(cells: np.ndarray, dim: int) -> np.ndarray:
    """Facets of tensor-ordered Q1 cells that belong to exactly one cell."""
    faces = np.concatenate([cells[:, f] for f in tensor_facets(dim)], axis=0).astype(np.int64)
    srt = np.sort(faces, axis=1)
    key = np.zeros(srt.shape[0], dtype=np.int64)
    for c in range(srt.shape[1]):
        key = key * (1 << 21) + srt[:, c]
    uniq, idx, counts = np.unique(key, return_index=True, return_counts=True)
    return faces[idx[counts == 1]].astype(np.int32)


def unit_square_quad(n: int) -> Mesh:
    """N x N squares on [0,1]^2 as Q1 cells (vertices in tensor order)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    i, j = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    coords = np.stack([i.ravel() / n, j.ravel() / n], axis=1).astype(np.float64)
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    n00 = (ci + m * cj).ravel()
    cells = np.stack([n00, n00 + 1, n00 + m, n00 + m + 1], axis=1).astype(np.int32)
    return Mesh(2, coords, cells, boundary_facets_q1(cells, 2), n, kind="q1")


def unit_cube_hex(n: int) -> Mesh:
    """N^3 cubes on [0,1]^3 as Q1 hexahedra (vertices in tensor order)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    m = n + 1
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([i.ravel() / n, j.ravel() / n, k.ravel() / n], axis=1).astype(np.float64)
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = (ci + m * (cj + m * ck)).ravel()
    offs = [(v & 1) + m * ((v >> 1) & 1) + m * m * ((v >> 2) & 1) for v in range(8)]
    cells = np.stack([base + o for o in offs], axis=1).astype(np.int32)
    return Mesh(3, coords, cells, boundary_facets_q1(cells, 3), n, kind="q1")


def unit_mesh(dim: int, n: int, kind: str = "simplex") -> Mesh:
    if kind == "q1":
        if dim == 2:
            return unit_square_quad(n)
        if dim == 3:
            return unit_cube_hex(n)
        raise ValueError("dim must be 2 or 3")
    if dim == 2:
        return unit_square_tri(n)
    if dim == 3:
        return unit_cube_kuhn(n)
    raise ValueError("dim must be 2 or 3")


def dof_count(dim: int, n: int) -> int:
    """Four-field P1 DoF count on the N-per-edge mesh (2d+2 DoF per node)."""
    return (n + 1) ** dim * (2 * dim + 2)
