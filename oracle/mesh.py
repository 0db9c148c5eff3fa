"""Structured Cartesian quad/hex mesh for the tensor-product DG space Q^k.

Section 3.1: mesh T_h, facets F_h, fixed facet normal and the traces
U^-/U^+.  Conventions (shared with the C interface only by documentation,
not by code):
  * d = 2 or 3; the vertical coordinate is the last one (y in 2-D, z in 3-D).
  * element index e = i_0 + n_0 (i_1 + n_1 i_2)      (first direction fastest)
  * node index within an element a = a_0 + (k+1)(a_1 + (k+1) a_2)
  * node coordinate x_j = i_j h_j + (1 + xi_{a_j}) h_j / 2 with the
    Gauss-Legendre points xi.
  * face (j, s): the element face with outward normal s e_j, s = +1 or -1;
    its (k+1)^(d-1) points are ordered by the remaining directions in
    increasing order, the first remaining direction fastest.
  * node z-levels: level index i_vert (k+1) + a_vert; face z-levels: i_vert.
"""
import itertools

import numpy as np

from .basis import gauss_legendre


class Mesh:
    def __init__(self, dim, n, L, order, periodic):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        if len(self.n) != dim or len(self.L) != dim or min(self.n) < 1:
            raise ValueError("bad mesh size")
        self.k = int(order)
        self.p1 = self.k + 1
        self.periodic = tuple(bool(p) for p in periodic)
        self.h = tuple(self.L[j] / self.n[j] for j in range(dim))
        self.xi, self.w = gauss_legendre(self.p1)
        self.Np = self.p1 ** dim
        self.Ne = int(np.prod(self.n))
        self.vert = dim - 1
        # node multi-indices, shape (Np, dim): first direction fastest
        self.node_multi = np.array(
            [tuple(reversed(t)) for t in itertools.product(range(self.p1), repeat=dim)],
            dtype=np.int64)
        # tensor weights W_a and element Jacobian |K| / 2^d
        self.W = np.prod(self.w[self.node_multi], axis=1)
        self.J = float(np.prod([hj / 2.0 for hj in self.h]))

    # ---- element indexing -------------------------------------------------
    def elem_multi(self, e):
        e = np.asarray(e, dtype=np.int64)
        out = []
        rem = e
        for j in range(self.dim):
            out.append(rem % self.n[j])
            rem = rem // self.n[j]
        return out

    def elem_index(self, multi):
        e = np.zeros_like(np.asarray(multi[0], dtype=np.int64))
        stride = 1
        for j in range(self.dim):
            e = e + np.asarray(multi[j], dtype=np.int64) * stride
            stride *= self.n[j]
        return e

    def neighbour(self, e, j, s):
        """Element across face (j, s) of e, or -1 where that face is a wall."""
        multi = self.elem_multi(e)
        ij = multi[j] + s
        if self.periodic[j]:
            ij = np.mod(ij, self.n[j])
            valid = np.ones_like(ij, dtype=bool)
        else:
            valid = (ij >= 0) & (ij < self.n[j])
            ij = np.clip(ij, 0, self.n[j] - 1)
        multi[j] = ij
        nb = self.elem_index(multi)
        return np.where(valid, nb, -1)

    # ---- geometry -----------------------------------------------------------
    def node_coords(self, elements=None):
        """List of d arrays (len(elements), Np) of physical node coordinates."""
        if elements is None:
            elements = np.arange(self.Ne)
        multi = self.elem_multi(elements)
        xs = []
        for j in range(self.dim):
            loc = (1.0 + self.xi[self.node_multi[:, j]]) * self.h[j] / 2.0
            xs.append(multi[j][:, None] * self.h[j] + loc[None, :])
        return xs

    def z_node_levels(self):
        nz = self.n[self.vert]
        hz = self.h[self.vert]
        iz = np.repeat(np.arange(nz), self.p1)
        a = np.tile(np.arange(self.p1), nz)
        return iz * hz + (1.0 + self.xi[a]) * hz / 2.0

    def z_face_levels(self):
        nz = self.n[self.vert]
        return np.arange(nz + 1) * self.h[self.vert]

    def node_level_index(self, elements=None):
        """(len(elements), Np) index into the node z-level table."""
        if elements is None:
            elements = np.arange(self.Ne)
        iz = self.elem_multi(elements)[self.vert]
        return iz[:, None] * self.p1 + self.node_multi[None, :, self.vert]

    # ---- faces ----------------------------------------------------------------
    def face_dirs(self, j):
        return [i for i in range(self.dim) if i != j]

    def face_points_multi(self, j):
        """(Nfp, d) multi-index of face points of a face normal to e_j (entry j unused)."""
        others = self.face_dirs(j)
        pts = []
        for t in itertools.product(range(self.p1), repeat=self.dim - 1):
            t = tuple(reversed(t))          # first remaining direction fastest
            m = [0] * self.dim
            for i, o in enumerate(others):
                m[o] = t[i]
            pts.append(m)
        return np.array(pts, dtype=np.int64)

    def face_weights(self, j):
        fp = self.face_points_multi(j)
        return np.prod(self.w[fp[:, self.face_dirs(j)]], axis=1)
