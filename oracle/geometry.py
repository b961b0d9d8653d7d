"""Horizontal grid factors of the oracle, derived from the raw grid (row A0).

The paper names the ICON discretisation only by citation (Sec. 4.1) and
describes the grid as the icosahedral RnBm grid (Sec. 5.1).  The readings
used here, all on a sphere of radius a, with unit position vectors:

* cell area A_c: spherical triangle area of the three vertices;
* primal edge length l_e: great-circle arc between the two edge vertices;
* dual edge length d_e: great-circle arc between the two cell circumcentres;
* dual area A_v: sum over the incident edges of the spherical triangles
  (vertex, circumcentre c0, circumcentre c1), so that sum A_v = 4 pi a^2;
* edge normal n_e: tangent at the edge midpoint, pointing from e2c[0] to
  e2c[1]; tangent t_e = r_e x n_e, so (n, t, r) is right-handed;
* divergence sign s_{c,e} = +1 if c = e2c[e][0] (n_e is outward), else -1;
* circulation sign t_{v,e} = +1 if t_e points towards v, -1 if away from v
  (counter-clockwise circulation around v seen from outside);
* edge->cell weights q_{c,e} = l_e h_{c,e} / (2 A_c), h = arc from the
  circumcentre to the edge midpoint, normalised to sum 1 per cell;
* cell->vertex weights r_{v,c}: area of the kite (vertex, edge midpoint,
  circumcentre, edge midpoint) that cell c contributes to the dual cell of
  v, normalised to sum 1 per vertex;
* cell->edge linear weights (r1, r0)/(r0 + r1), r_i = arc(circumcentre i,
  edge midpoint), along the dual edge (which crosses the edge at its midpoint);
* edge area A_e = l_e d_e;  Coriolis f_e = 2 Omega sin(lat_e).
"""
import numpy as np


def _norm(x):
    """Euclidean norm over the last axis."""
    return np.linalg.norm(x, axis=-1)


def arc(p, q):
    """Great-circle angle between unit vectors (radians)."""
    return np.arctan2(_norm(np.cross(p, q)), np.sum(p * q, axis=-1))


def tri_area(p, q, r):
    """Spherical excess of the triangle (p, q, r) on the unit sphere."""
    num = np.abs(np.sum(p * np.cross(q, r), axis=-1))
    den = 1.0 + np.sum(p * q, -1) + np.sum(q * r, -1) + np.sum(r * p, -1)
    return 2.0 * np.arctan2(num, den)


def project(v, x):
    """Project vectors v (..., 3) onto the tangent plane at unit x (..., 3)."""
    return v - np.sum(v * x, axis=-1, keepdims=True) * x


class Geometry:
    """The factors of the module docstring for one grid on a sphere of radius a (row A0)."""
    def __init__(self, grid, radius):
        """Derives every factor from the grid's tables and unit position vectors."""
        a = float(radius)
        self.a = a
        V, C, E = grid.vert_xyz, grid.cell_xyz, grid.edge_xyz
        self.V, self.C, self.E = V, C, E
        self.c2v = grid.c2v.astype(np.int64)
        self.c2e = grid.c2e.astype(np.int64)
        self.e2c = grid.e2c.astype(np.int64)
        self.e2v = grid.e2v.astype(np.int64)
        self.v2e = grid.v2e.astype(np.int64)
        self.v2c = grid.v2c.astype(np.int64)
        self.nc, self.ne, self.nv = C.shape[0], E.shape[0], V.shape[0]
        self.v2e_mask = self.v2e >= 0
        self.v2c_mask = self.v2c >= 0
        v2e = np.where(self.v2e_mask, self.v2e, 0)
        v2c = np.where(self.v2c_mask, self.v2c, 0)

        c0, c1 = self.e2c[:, 0], self.e2c[:, 1]
        self.cell_area = a * a * tri_area(V[self.c2v[:, 0]], V[self.c2v[:, 1]], V[self.c2v[:, 2]])
        self.edge_length = a * arc(V[self.e2v[:, 0]], V[self.e2v[:, 1]])
        self.dual_length = a * arc(C[c0], C[c1])
        self.dual_area = a * a * np.sum(
            np.where(self.v2e_mask, tri_area(V[:, None, :], C[c0[v2e]], C[c1[v2e]]), 0.0), axis=1)
        n = project(C[c1] - C[c0], E)
        self.normal = n / _norm(n)[:, None]
        self.tangent = np.cross(E, self.normal)
        self.edge_area = self.edge_length * self.dual_length
        self.dual_mid = C[c0] + C[c1]
        self.dual_mid /= _norm(self.dual_mid)[:, None]

        # signs
        self.c2e_sign = np.where(self.e2c[self.c2e, 0] == np.arange(self.nc)[:, None], 1.0, -1.0)
        tv = np.sum((V[:, None, :] - E[v2e]) * self.tangent[v2e], axis=-1)
        self.v2e_sign = np.where(self.v2e_mask, np.sign(tv), 0.0)
        te = np.sum((V[self.e2v] - E[:, None, :]) * self.tangent[:, None, :], axis=-1)
        self.e2v_sign = np.sign(te)            # [ne, 2]: +1 at the vertex t_e points to

        # neighbour cell across each cell edge
        other = np.where(self.e2c[self.c2e, 0] == np.arange(self.nc)[:, None],
                         self.e2c[self.c2e, 1], self.e2c[self.c2e, 0])
        self.c2e2c = other
        # vertices opposite the edge in c0 and c1 (diamond of the edge)
        self.e2c2v = np.zeros((self.ne, 4), dtype=np.int64)
        self.e2c2v[:, 0:2] = self.e2v
        for j, c in enumerate((c0, c1)):
            cv = self.c2v[c]
            opp = np.where((cv != self.e2v[:, 0:1]) & (cv != self.e2v[:, 1:2]), cv, -1).max(axis=1)
            self.e2c2v[:, 2 + j] = opp

        # edge -> cell interpolation weights
        h = a * arc(C[:, None, :], E[self.c2e])
        q = self.edge_length[self.c2e] * h / (2.0 * self.cell_area[:, None])
        self.e2c_weight = q / np.sum(q, axis=1, keepdims=True)

        # cell -> vertex weights: kite areas
        r = np.zeros((self.nv, 6))
        for j in range(6):
            c = v2c[:, j]
            cv = self.c2v[c]
            # the two other vertices of c are the far ends of the two edges of c at v
            others = [np.where(cv[:, i] == np.arange(self.nv), -1, cv[:, i]) for i in range(3)]
            o = np.stack(others, 1)
            o_sorted = np.sort(o, axis=1)[:, 1:]      # drop the -1
            m1 = V[o_sorted[:, 0]] + V
            m2 = V[o_sorted[:, 1]] + V
            m1 /= _norm(m1)[:, None]
            m2 /= _norm(m2)[:, None]
            kite = tri_area(V, m1, C[c]) + tri_area(V, C[c], m2)
            r[:, j] = np.where(self.v2c_mask[:, j], kite, 0.0)
        self.v2c_weight = r / np.sum(r, axis=1, keepdims=True)

        # cell -> edge-midpoint linear interpolation along the dual edge
        r0, r1 = arc(C[c0], E), arc(C[c1], E)
        self.e2c_lin = np.stack([r1 / (r0 + r1), r0 / (r0 + r1)], axis=1)

        # vertices of the diamond: dn = arc between the two opposite vertices
        self.vert_vert_length = a * arc(V[self.e2c2v[:, 2]], V[self.e2c2v[:, 3]])

    def coriolis(self, omega):
        """f_e = 2 omega sin(lat_e) at the edge midpoints."""
        return 2.0 * omega * self.E[:, 2]
