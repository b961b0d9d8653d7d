"""Icosahedral RnBm grid generator (paper Sec. 5.1: Sadourny root division of
the 20 icosahedron faces into n^2 triangles, then m recursive bisections).

Only n = 2 is built: splitting each icosahedron edge into two equal
great-circle arcs is the same as one bisection step, so RnBm = (m+1)
bisections of the icosahedron.  Output is raw connectivity and unit-sphere
coordinates, numbered for locality:

* cells in hierarchical (quadtree) order: the four children of a parent
  triangle are consecutive, so any run of cells is a compact patch;
* vertices and edges by first appearance when walking the cells in order.

Conventions (these are facts about the produced tables, relied on by the
consumers only through what the tables say):

* ``c2v[c]`` is counter-clockwise seen from outside the sphere;
* ``c2e[c][j]`` is the edge from ``c2v[c][j]`` to ``c2v[c][(j+1)%3]``;
* ``e2v[e] = (a, b)`` and ``e2c[e] = (c0, c1)`` where c0 walks a->b in its
  counter-clockwise order and c1 walks b->a;
* ``v2e``/``v2c`` list the 5 or 6 incident edges/cells counter-clockwise,
  padded with -1 for the 12 pentagon vertices;
* cell centres are spherical circumcentres, edge midpoints are normalised
  chord midpoints (the arc midpoints).
"""
from dataclasses import dataclass
import numpy as np


@dataclass
class Grid:
    root: int
    bisections: int
    vert_xyz: np.ndarray   # [nv, 3] float64 unit vectors
    cell_xyz: np.ndarray   # [nc, 3] circumcentres
    edge_xyz: np.ndarray   # [ne, 3] arc midpoints
    c2v: np.ndarray        # [nc, 3] int32
    c2e: np.ndarray        # [nc, 3] int32
    e2v: np.ndarray        # [ne, 2] int32
    e2c: np.ndarray        # [ne, 2] int32
    v2e: np.ndarray        # [nv, 6] int32, -1 padded
    v2c: np.ndarray        # [nv, 6] int32, -1 padded

    @property
    def n_cells(self):
        return self.c2v.shape[0]

    @property
    def n_edges(self):
        return self.e2v.shape[0]

    @property
    def n_verts(self):
        return self.vert_xyz.shape[0]

    @property
    def name(self):
        return f"R{self.root}B{self.bisections}"


def _normalize(x):
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def _icosahedron():
    p = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v = _normalize(v)
    # rotate so that vertex 0 sits on the north pole (as ICON grids do)
    z = v[0]
    x = _normalize(np.cross(z, v[1]))
    x = _normalize(v[1] - np.dot(v[1], z) * z)
    y = np.cross(z, x)
    rot = np.stack([x, y, z])            # rows: new axes
    v = v @ rot.T
    # orient every face counter-clockwise seen from outside
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def _bisect(verts, faces):
    """One bisection: every triangle (a,b,c) -> (a,ab,ca),(ab,b,bc),(ca,bc,c),(ab,bc,ca)."""
    nv = verts.shape[0]
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
    uniq, inv = np.unique(key, return_inverse=True)
    a, b = uniq // nv, uniq % nv
    mids = _normalize(verts[a] + verts[b])
    mid_id = nv + inv.reshape(3, -1).T       # [nf, 3]: ab, bc, ca
    ab, bc, ca = mid_id[:, 0], mid_id[:, 1], mid_id[:, 2]
    A, B, C = faces[:, 0], faces[:, 1], faces[:, 2]
    child = np.stack([np.stack([A, ab, ca], 1), np.stack([ab, B, bc], 1),
                      np.stack([ca, bc, C], 1), np.stack([ab, bc, ca], 1)], 1)
    return np.concatenate([verts, mids]), child.reshape(-1, 3)


def _ccw_sort(center, nbr_xyz, valid):
    """Order up to 6 neighbour points counter-clockwise around ``center``."""
    ref = np.where(np.abs(center[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]),
                   np.array([[1.0, 0.0, 0.0]]))
    e1 = _normalize(np.cross(ref, center))
    e2 = np.cross(center, e1)
    d = nbr_xyz - center[:, None, :]
    ang = np.arctan2(np.einsum("ijk,ik->ij", d, e2), np.einsum("ijk,ik->ij", d, e1))
    ang = np.where(valid, ang, np.inf)
    return np.argsort(ang, axis=1, kind="stable")


def make_grid(bisections: int, root: int = 2) -> Grid:
    """Build the R{root}B{bisections} grid (root must be 2)."""
    if root != 2:
        raise ValueError("only root division n=2 is supported")
    verts, faces = _icosahedron()
    for _ in range(bisections + 1):
        verts, faces = _bisect(verts, faces)
    nc = faces.shape[0]

    # renumber vertices by first appearance in cell order
    flat = faces.reshape(-1)
    _, first = np.unique(flat, return_index=True)
    order = np.argsort(first, kind="stable")
    old_ids = np.unique(flat)[order]
    new_of_old = np.empty(verts.shape[0], dtype=np.int64)
    new_of_old[old_ids] = np.arange(old_ids.size)
    verts = verts[old_ids]
    faces = new_of_old[faces]
    nv = verts.shape[0]

    # edges: half-edge j of cell c runs c2v[c][j] -> c2v[c][(j+1)%3]
    he_a = faces.reshape(-1)
    he_b = faces[:, [1, 2, 0]].reshape(-1)
    key = np.minimum(he_a, he_b) * nv + np.maximum(he_a, he_b)
    ukey, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    he_edge = rank[inv]                       # edge id of each half-edge
    ne = ukey.size
    c2e = he_edge.reshape(nc, 3)
    he_cell = np.repeat(np.arange(nc), 3)
    # the first appearance (in cell order) defines c0 and the direction a->b
    first_he = first[order]
    e2v = np.stack([he_a[first_he], he_b[first_he]], 1)
    e2c = np.full((ne, 2), -1, dtype=np.int64)
    e2c[:, 0] = he_cell[first_he]
    is_second = np.ones(he_edge.size, dtype=bool)
    is_second[first_he] = False
    e2c[he_edge[is_second], 1] = he_cell[is_second]
    assert (e2c >= 0).all()

    cell_xyz = _normalize(np.cross(verts[faces[:, 1]] - verts[faces[:, 0]],
                                   verts[faces[:, 2]] - verts[faces[:, 0]]))
    edge_xyz = _normalize(verts[e2v[:, 0]] + verts[e2v[:, 1]])

    # vertex -> cells and vertex -> edges, counter-clockwise, padded to 6
    def incidence(ids, owners, n):
        o = np.argsort(ids, kind="stable")
        s_ids, s_own = ids[o], owners[o]
        start = np.searchsorted(s_ids, np.arange(n))
        cnt = np.bincount(ids, minlength=n)
        slot = np.arange(ids.size) - start[s_ids]
        tab = np.full((n, 6), -1, dtype=np.int64)
        tab[s_ids, slot] = s_own
        return tab, cnt

    v2c, _ = incidence(faces.reshape(-1), np.repeat(np.arange(nc), 3), nv)
    v2e, _ = incidence(e2v.reshape(-1), np.repeat(np.arange(ne), 2), nv)
    for tab, pts in ((v2c, cell_xyz), (v2e, edge_xyz)):
        valid = tab >= 0
        xyz = pts[np.where(valid, tab, 0)]
        o = _ccw_sort(verts, xyz, valid)
        tab[:] = np.take_along_axis(tab, o, axis=1)

    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    return Grid(root=root, bisections=bisections, vert_xyz=f64(verts), cell_xyz=f64(cell_xyz),
                edge_xyz=f64(edge_xyz), c2v=i32(faces), c2e=i32(c2e), e2v=i32(e2v),
                e2c=i32(e2c), v2e=i32(v2e), v2c=i32(v2c))
