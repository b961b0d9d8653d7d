"""Analytic initial states on the RnBm grid.

``jw_type_state`` is a self-derived balanced baroclinic jet in the spirit of
the Jablonowski-Williamson test (whose own formulas are not used here).  The
Exner pressure is prescribed analytically,

    pi(phi, z) = exp(-z/H) * (1 - eps(z) * G(phi)),      H = c_pd*T0/g,
    eps(z)     = eps0 * (z/z_j) * exp(1 - z/z_j),
    G(phi)     = 8/15 - 4*(cos^3(phi)/3 - cos^5(phi)/5),  G'(phi) = sin(phi) sin^2(2 phi),

theta_v follows from hydrostatic balance, c_pd*theta*dpi/dz = -g, the zonal
wind u from gradient-wind balance,
(tan(phi)/a) u^2 + f u = -(c_pd*theta/a) dpi/dphi  (the root that vanishes
with the pressure gradient), and rho from the equation of state
rho = p00 * pi**(c_vd/R_d) / (R_d*theta).  The jet is westerly in both
hemispheres, zero at the ground, the equator and the poles, and peaks near
45 degrees and z_j.  w = 0.

A seeded Gaussian zonal-wind bump, amplitude 1 m/s and e-folding radius a/10,
is added; its centre is drawn with numpy's PCG64 from the seed: longitude
uniform in [0, 2pi), latitude uniform in [25, 55] degrees north.
"""
import numpy as np

CONSTANTS = dict(
    grav=9.80665, rd=287.04, cpd=1004.64, p00=1.0e5, omega=7.29212e-5,
    radius=6.371229e6,
)
CONSTANTS["cvd"] = CONSTANTS["cpd"] - CONSTANTS["rd"]

JW_DEFAULTS = dict(T0=250.0, eps0=0.12, z_jet=11000.0)


def _normalize(x):
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def _lat(xyz):
    return np.arcsin(np.clip(xyz[..., 2], -1.0, 1.0))


def _east(xyz):
    return _normalize(np.cross(np.array([0.0, 0.0, 1.0]), xyz))


def edge_normals(grid):
    """Unit normal at each edge midpoint, pointing from e2c[:,0] to e2c[:,1]."""
    x = grid.edge_xyz
    d = grid.cell_xyz[grid.e2c[:, 1]] - grid.cell_xyz[grid.e2c[:, 0]]
    d = d - np.einsum("ij,ij->i", d, x)[:, None] * x
    return _normalize(d)


def _jw_fields(phi, z, c, T0, eps0, z_jet):
    g, cpd, a, om = c["grav"], c["cpd"], c["radius"], c["omega"]
    H = cpd * T0 / g
    ez = np.exp(-z / H)
    s = z / z_jet
    eps = eps0 * s * np.exp(1.0 - s)
    deps = eps0 / z_jet * (1.0 - s) * np.exp(1.0 - s)
    cp = np.cos(phi)
    G = 8.0 / 15.0 - 4.0 * (cp ** 3 / 3.0 - cp ** 5 / 5.0)
    dG = np.sin(phi) * np.sin(2.0 * phi) ** 2
    pi = ez * (1.0 - eps * G)
    dpi_dz = ez * (-(1.0 - eps * G) / H - deps * G)
    theta = -g / (cpd * dpi_dz)
    dpi_dphi = -ez * eps * dG
    # gradient wind, written for |phi| (the state is symmetric about the equator)
    ap = np.abs(phi)
    P = -(cpd * theta / a) * dpi_dphi * np.sign(phi)
    f = 2.0 * om * np.sin(ap)
    den = f + np.sqrt(np.maximum(f * f + 4.0 * np.tan(ap) / a * P, 0.0))
    u = np.where(den > 0.0, 2.0 * P / np.where(den > 0.0, den, 1.0), 0.0)
    return pi, theta, u


def sample_perturbation_centre(seed: int):
    """(lon, lat) in radians of the Gaussian bump, drawn with PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lon = rng.uniform(0.0, 2.0 * np.pi)
    lat = np.deg2rad(rng.uniform(25.0, 55.0))
    return lon, lat


def gaussian_perturbation_centre(seed: int):
    lon, lat = sample_perturbation_centre(seed)
    return np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])


def jw_type_state(grid, z_ifc, seed=0, amp=1.0, constants=None, **jw):
    """Prognostic state dict (vn, w, rho, exner, theta_v), level-contiguous float64.

    Shapes: vn [ne, nlev], w [nc, nlev+1], rho/exner/theta_v [nc, nlev].
    ``amp`` = 0 gives the unperturbed balanced jet.  z_ifc is one column of
    half-level heights [nlev+1], or one per cell [nc, nlev+1] (terrain): the
    fields are then evaluated at each cell's full-level heights, and vn at the
    mean of the two adjacent cells' heights.
    """
    c = dict(CONSTANTS if constants is None else constants)
    p = dict(JW_DEFAULTS)
    p.update(jw)
    z_ifc = np.asarray(z_ifc, dtype=np.float64)
    if z_ifc.ndim == 1:
        z_mc = 0.5 * (z_ifc[:-1] + z_ifc[1:])
        zc = ze = z_mc[None, :]
    else:
        zc = 0.5 * (z_ifc[:, :-1] + z_ifc[:, 1:])
        ze = 0.5 * (zc[grid.e2c[:, 0]] + zc[grid.e2c[:, 1]])
    nlev = zc.shape[1]
    phi_c = _lat(grid.cell_xyz)[:, None]
    pi_c, th_c, _ = _jw_fields(phi_c, zc, c, p["T0"], p["eps0"], p["z_jet"])
    rho_c = c["p00"] * pi_c ** (c["cvd"] / c["rd"]) / (c["rd"] * th_c)

    xe = grid.edge_xyz
    phi_e = _lat(xe)[:, None]
    _, _, u_e = _jw_fields(phi_e, ze, c, p["T0"], p["eps0"], p["z_jet"])
    if amp != 0.0:
        xc = gaussian_perturbation_centre(seed)
        r = c["radius"] * np.arctan2(np.linalg.norm(np.cross(xe, xc), axis=1), xe @ xc)
        u_e = u_e + amp * np.exp(-(r / (c["radius"] / 10.0)) ** 2)[:, None]
    proj = np.einsum("ij,ij->i", _east(xe), edge_normals(grid))
    vn = u_e * proj[:, None]
    w = np.zeros((grid.n_cells, nlev + 1))
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    return dict(vn=f64(vn), w=f64(w), rho=f64(rho_c), exner=f64(pi_c), theta_v=f64(th_c))
