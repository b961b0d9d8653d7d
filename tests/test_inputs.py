"""Seeded input generators: icosahedral RnBm grid (paper Sec. 5.1), vertical
grid and the balanced JW-type jet."""
import numpy as np
import pytest

from icon_inputs import make_grid, make_vct, jw_type_state, sample_perturbation_centre
from icon_inputs.vertical import stretch_ratio
from icon_inputs.state import edge_normals, CONSTANTS


@pytest.mark.parametrize("b", [0, 1, 2, 3, 4])
def test_rnbm_counts_and_topology(b):
    # RnBm: 20 n^2 4^m triangles; closed triangulated sphere => E = 3F/2, V = E - F + 2
    g = make_grid(b)
    nc = 20 * 4 * 4 ** b
    assert g.n_cells == nc and g.n_edges == 3 * nc // 2 and g.n_verts == nc // 2 + 2
    assert g.n_verts - g.n_edges + g.n_cells == 2
    # exactly 12 five-valent vertices (the icosahedron's), all others six-valent
    assert np.sum(g.v2c[:, 5] < 0) == 12 and np.all(g.v2c[:, :5] >= 0)
    assert np.sum(g.v2e[:, 5] < 0) == 12
    # every edge: two distinct cells that both list it, two distinct vertices
    assert np.all(g.e2c[:, 0] != g.e2c[:, 1]) and np.all(g.e2v[:, 0] != g.e2v[:, 1])
    for j in range(2):
        assert np.all(np.any(g.c2e[g.e2c[:, j]] == np.arange(g.n_edges)[:, None], axis=1))
    # cells counter-clockwise seen from outside
    V = g.vert_xyz
    a, bb, c = V[g.c2v[:, 0]], V[g.c2v[:, 1]], V[g.c2v[:, 2]]
    assert np.all(np.einsum("ij,ij->i", np.cross(bb - a, c - a), a) > 0)
    # circumcentres are equidistant from the three vertices
    d = np.stack([np.einsum("ij,ij->i", g.cell_xyz, V[g.c2v[:, j]]) for j in range(3)], 1)
    assert np.max(np.abs(d - d[:, :1])) < 1e-14


def test_rnbm_matches_published_r2b2_counts():
    # R2B2: 1280 cells, 1920 edges, 642 vertices (the configuration names them)
    g = make_grid(2)
    assert (g.n_cells, g.n_edges, g.n_verts) == (1280, 1920, 642)


def test_vertical_grid():
    for nlev, r in ((30, 1.1662), (65, 1.0561), (90, 1.0349)):
        z = make_vct(nlev)
        assert z.size == nlev + 1 and z[0] == 30000.0 and z[-1] == 0.0
        assert np.all(np.diff(z) < 0)
        assert abs(z[-2] - 50.0) < 1e-9
        assert abs(stretch_ratio(nlev) - r) < 1e-4
        dz = -np.diff(z)[::-1]
        assert np.allclose(dz[1:] / dz[:-1], stretch_ratio(nlev), rtol=1e-9)


def test_jw_type_state_balance_and_symmetry():
    g = make_grid(2)
    z = make_vct(30)
    st = jw_type_state(g, z, amp=0.0)
    c = CONSTANTS
    # equation of state
    p = c["p00"] * st["exner"] ** (c["cpd"] / c["rd"])
    assert np.allclose(st["rho"], p / (c["rd"] * st["theta_v"] * st["exner"]), rtol=1e-13)
    # static stability: theta increases with height (k = 0 is the top)
    assert np.all(np.diff(st["theta_v"], axis=1) < 0)
    # hydrostatic to discretisation accuracy: c_pd theta dpi/dz ~ -g
    zm = 0.5 * (z[:-1] + z[1:])
    dpi = (st["exner"][:, :-1] - st["exner"][:, 1:]) / (zm[:-1] - zm[1:])
    th = 0.5 * (st["theta_v"][:, :-1] + st["theta_v"][:, 1:])
    assert np.max(np.abs(c["cpd"] * th * dpi / c["grav"] + 1.0)) < 0.02
    # westerly jet, ~30 m/s, zero at the ground
    lat_e = np.arcsin(g.edge_xyz[:, 2])
    east = np.cross([0, 0, 1.0], g.edge_xyz)
    east /= np.linalg.norm(east, axis=1, keepdims=True)
    u = st["vn"] / np.einsum("ij,ij->i", east, edge_normals(g))[:, None].clip(1e-300)
    proj = np.abs(np.einsum("ij,ij->i", east, edge_normals(g)))
    sel = proj > 0.5
    assert 25.0 < np.max(u[sel]) < 40.0
    assert np.max(np.abs(st["vn"][:, -1])) < 0.5
    assert np.all(u[sel & (np.abs(lat_e) < 0.05)][:, :] < 1.0)


def test_perturbation_centre_is_seeded():
    a = sample_perturbation_centre(0)
    assert a == sample_perturbation_centre(0) and a != sample_perturbation_centre(1)
    lon, lat = a
    assert 0 <= lon < 2 * np.pi and np.deg2rad(25) <= lat <= np.deg2rad(55)
    g = make_grid(3)  # fine enough to resolve the a/10 e-folding radius
    z = make_vct(30)
    s0, s1 = jw_type_state(g, z, seed=0), jw_type_state(g, z, seed=0, amp=0.0)
    du = s0["vn"] - s1["vn"]
    assert 0.5 < np.max(np.abs(du)) <= 1.0


def test_edge_normals_are_unit_tangents_from_the_first_cell_to_the_second():
    from icon_inputs.state import edge_normals
    g = make_grid(2)
    n = edge_normals(g)
    assert np.max(np.abs(np.linalg.norm(n, axis=1) - 1.0)) < 1e-14
    assert np.max(np.abs(np.einsum("ij,ij->i", n, g.edge_xyz))) < 1e-14
    d = g.cell_xyz[g.e2c[:, 1]] - g.cell_xyz[g.e2c[:, 0]]
    assert np.all(np.einsum("ij,ij->i", n, d) > 0)


def test_perturbation_is_an_eastward_bump_of_the_given_amplitude():
    """The seeded bump adds amp exp(-(r/(a/10))^2) to the zonal wind: eastward,
    about amp at the edges nearest its centre, negligible far away."""
    from icon_inputs.state import edge_normals, gaussian_perturbation_centre
    g, z = make_grid(3), make_vct(10)
    dvn = jw_type_state(g, z, seed=4, amp=2.0)["vn"] - jw_type_state(g, z, seed=4, amp=0.0)["vn"]
    east = np.cross([0.0, 0.0, 1.0], g.edge_xyz)
    east /= np.linalg.norm(east, axis=1, keepdims=True)
    proj = np.einsum("ij,ij->i", east, edge_normals(g))
    du = dvn[:, 0] / np.where(np.abs(proj) > 0.5, proj, np.nan)      # zonal change where vn sees it
    xc = gaussian_perturbation_centre(4)
    r = np.arccos(np.clip(g.edge_xyz @ xc, -1.0, 1.0))
    near = (r < 0.02) & np.isfinite(du)
    assert near.any() and np.all(du[near] > 1.9) and np.all(du[near] <= 2.0 + 1e-12)
    far = r > 0.5
    assert np.max(np.abs(dvn[far])) < 1e-6


def test_jw_state_over_terrain_is_evaluated_at_each_columns_heights():
    """Over per-column heights the balanced jet of a cell is the one-column
    state at that cell's own heights; vn uses the mean of the adjacent cells'."""
    from icon_inputs import mountain_height, terrain_following_z
    grid, z = make_grid(2), make_vct(12)
    zz = terrain_following_z(z, mountain_height(grid.cell_xyz))
    st = jw_type_state(grid, zz, seed=3)
    c = int(np.argmax(zz[:, -1]))
    assert zz[c, -1] > 1000.0
    one = jw_type_state(grid, zz[c], seed=3)
    for k in ("rho", "exner", "theta_v"):
        assert np.array_equal(st[k][c], one[k][c])
    flat = jw_type_state(grid, z, seed=3)
    far = int(np.argmin(zz[:, -1]))
    assert zz[far, -1] < 1e-6 * 2000.0 or np.allclose(st["exner"][far], flat["exner"][far], rtol=1e-6)
    assert not np.allclose(st["exner"][c], flat["exner"][c], rtol=1e-3)
