"""Topography and terrain-following half-level heights (inputs, as an ICON
external-parameter file and vertical coordinate table would give them).

* Gaussian mountain of height h0 and e-folding radius d (great-circle distance
  r from its centre): h = h0 exp(-(r/d)^2), at cell centres.
* Basic terrain-following coordinate: every half level of the flat table
  z_flat (top first, z_flat[nlev] = 0) is lifted by the local ground height
  and the lift decays linearly to zero at the model top,
  z_ifc[c, k] = z_flat[k] + h_c (1 - z_flat[k] / z_flat[0]).
"""
import numpy as np

EARTH_RADIUS = 6.371229e6


def mountain_height(cell_xyz, h0=2000.0, d=1.5e6, lon_deg=90.0, lat_deg=30.0, radius=EARTH_RADIUS):
    """Ground height [nc] of a Gaussian mountain at the cell centres (unit vectors)."""
    lon, lat = np.deg2rad(lon_deg), np.deg2rad(lat_deg)
    centre = np.array([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])
    r = radius * np.arccos(np.clip(cell_xyz @ centre, -1.0, 1.0))
    return h0 * np.exp(-(r / d) ** 2)


def terrain_following_z(z_flat, h):
    """Half-level heights [nc, nlev+1] (top first) over ground heights h [nc]."""
    z_flat = np.asarray(z_flat, dtype=np.float64)
    lift = 1.0 - z_flat / z_flat[0]
    return np.ascontiguousarray(z_flat[None, :] + h[:, None] * lift[None, :])
