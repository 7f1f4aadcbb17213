"""Independent restatements of the grid's metric quantities, used by the pins.

These are written from the definitions of a finite-integration grid (edge
lengths, dual areas, dual volumes), not from the oracle's code, so that an
oracle whose update uses a different weighting fails the invariants that are
checked with them. Plain Python loops: small grids only.
"""
from __future__ import annotations

import numpy as np

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def coords(h):
    return np.concatenate([[0.0], np.cumsum(h)])


def dual(h, p):
    n = len(h)
    return (h[p - 1] / 2 if p > 0 else 0.0) + (h[p] / 2 if p < n else 0.0)


class Metric:
    def __init__(self, p):
        self.p = p
        self.h = [np.asarray(p.dx), np.asarray(p.dy), np.asarray(p.dz)]
        self.n = [p.nx, p.ny, p.nz]
        self.tab = p.material_table()

    def nid(self, n):
        return (n[2] * (self.n[1] + 1) + n[1]) * (self.n[0] + 1) + n[0]

    def mat(self, c):
        return int(self.p.mat[c[2], c[1], c[0]])

    def nodes(self):
        for k in range(self.n[2] + 1):
            for j in range(self.n[1] + 1):
                for i in range(self.n[0] + 1):
                    yield (i, j, k)

    def edge_tangent_to_wall(self, a, n):
        for b in range(3):
            if b == a:
                continue
            if n[b] == 0 and self.p.em_bc[2 * b] != 1:
                return True
            if n[b] == self.n[b] and self.p.em_bc[2 * b + 1] != 1:
                return True
        return False

    def edges(self, a, free_only=True):
        for n in self.nodes():
            if n[a] >= self.n[a]:
                continue
            if free_only and self.edge_tangent_to_wall(a, n):
                continue
            yield n

    def faces(self, a):
        b, c = (a + 1) % 3, (a + 2) % 3
        for n in self.nodes():
            if n[b] < self.n[b] and n[c] < self.n[c]:
                yield n

    def edge_integral(self, a, n, col):
        """integral of a voxel property over the edge's dual volume
        (edge length x the four quarter cross-sections of its voxels)"""
        b, c = (a + 1) % 3, (a + 2) % 3
        s = 0.0
        for db in (-1, 0):
            for dc in (-1, 0):
                cell = [0, 0, 0]
                cell[a], cell[b], cell[c] = n[a], n[b] + db, n[c] + dc
                if not (0 <= cell[b] < self.n[b] and 0 <= cell[c] < self.n[c]):
                    continue
                s += self.tab[self.mat(cell), col] * self.h[b][cell[b]] * self.h[c][cell[c]] / 4
        return s * self.h[a][n[a]]

    def edge_volume(self, a, n):
        b, c = (a + 1) % 3, (a + 2) % 3
        return self.h[a][n[a]] * dual(self.h[b], n[b]) * dual(self.h[c], n[c])

    def face_mu_volume(self, a, n):
        """mu_f * V_f: primal face area x dual length, mu_f the series mean"""
        b, c = (a + 1) % 3, (a + 2) % 3
        A = self.h[b][n[b]] * self.h[c][n[c]]
        lstar = dual(self.h[a], n[a])
        rel = 0.0
        for d in (-1, 0):
            cell = list(n)
            cell[a] = n[a] + d
            if 0 <= cell[a] < self.n[a]:
                rel += (self.h[a][cell[a]] / 2) / (MU0 * self.tab[self.mat(cell), 1])
        return A * lstar * lstar / rel

    def em_energy(self, E, H_old, H_new):
        """W = 1/2 sum eps_e V_e E^2 + 1/2 sum mu_f V_f H^{n-1/2} H^{n+1/2}"""
        w = 0.0
        for a in range(3):
            for n in self.edges(a):
                w += 0.5 * EPS0 * self.edge_integral(a, n, 0) * E[a][self.nid(n)] ** 2
            for n in self.faces(a):
                i = self.nid(n)
                w += 0.5 * self.face_mu_volume(a, n) * H_old[a][i] * H_new[a][i]
        return w

    def node_capacity(self):
        C = np.zeros((self.n[2] + 1) * (self.n[1] + 1) * (self.n[0] + 1))
        for k in range(self.n[2]):
            for j in range(self.n[1]):
                for i in range(self.n[0]):
                    V = self.h[0][i] * self.h[1][j] * self.h[2][k]
                    rc = self.tab[self.mat((i, j, k)), 6]
                    for dk in (0, 1):
                        for dj in (0, 1):
                            for di in (0, 1):
                                C[self.nid((i + di, j + dj, k + dk))] += rc * V / 8
        return C
