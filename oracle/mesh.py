"""Topology of the structured hexahedral mesh (oracle; test infrastructure only).

Element (i,j,l) has index i + nx*(j + ny*l); its corner (s,t,u) in {0,1}^3 is
vertex (i+s, j+t, l+u), listed with s fastest. Faces normal to axis d are
indexed by their plane position along d and the cell position across it.

Multipliers (the space M of Example 2.2) live on interior faces only: a
Q_k Lagrange basis on the (k+1)^2 tensor Gauss-Legendre nodes of each face
(reading: the paper only asks for "a specified multiplier space", Sec. 5).
Global multiplier order: faces by normal axis (x, y, z), then face position
lexicographically (first index fastest), then face node (lower tangential axis
fastest).
"""
from __future__ import annotations

import numpy as np


class StructuredHexMesh:
    def __init__(self, nx, ny, nz, vertices):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.vertices = np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
        assert self.vertices.shape[0] == (nx + 1) * (ny + 1) * (nz + 1)
        self.n_elem = nx * ny * nz
        # number of faces normal to each axis: planes * cells across
        self.dims = (nx, ny, nz)
        self.n_faces_axis = []
        self.n_interior_faces_axis = []
        for d in range(3):
            across = [self.dims[a] for a in range(3) if a != d]
            self.n_faces_axis.append((self.dims[d] + 1) * across[0] * across[1])
            self.n_interior_faces_axis.append((self.dims[d] - 1) * across[0] * across[1])
        self.n_faces = sum(self.n_faces_axis)
        self.n_interior_faces = sum(self.n_interior_faces_axis)

    def elem_ijk(self, e):
        nx, ny = self.nx, self.ny
        return e % nx, (e // nx) % ny, e // (nx * ny)

    def element_vertices(self, e):
        i, j, l = self.elem_ijk(e)
        nx1, ny1 = self.nx + 1, self.ny + 1
        idx = []
        for u in (0, 1):
            for t in (0, 1):
                for s in (0, 1):
                    idx.append((i + s) + nx1 * ((j + t) + ny1 * (l + u)))
        return self.vertices[idx]

    def _face_pos(self, d, pos):
        """(axis, plane, a, b): plane index along d, a/b the cell indices across (lower axis first)."""
        plane = pos[d]
        a, b = [pos[x] for x in range(3) if x != d]
        return plane, a, b

    def face_id(self, d, pos):
        """Global face id (all faces, boundary included) of the axis-d face at grid position pos."""
        plane, a, b = self._face_pos(d, pos)
        across = [self.dims[x] for x in range(3) if x != d]
        off = sum(self.n_faces_axis[:d])
        return off + plane + (self.dims[d] + 1) * (a + across[0] * b)

    def interior_face_index(self, d, pos):
        """Index of an interior face among interior faces (the multiplier face order), or -1."""
        plane, a, b = self._face_pos(d, pos)
        if plane == 0 or plane == self.dims[d]:
            return -1
        across = [self.dims[x] for x in range(3) if x != d]
        off = sum(self.n_interior_faces_axis[:d])
        return off + (plane - 1) + (self.dims[d] - 1) * (a + across[0] * b)

    def element_faces(self, e):
        """For local faces x0,x1,y0,y1,z0,z1: (global face id, interior face index or -1)."""
        i, j, l = self.elem_ijk(e)
        out = []
        for f in range(6):
            d, side = f // 2, f % 2
            pos = [i, j, l]
            pos[d] += side
            out.append((self.face_id(d, pos), self.interior_face_index(d, pos)))
        return out
