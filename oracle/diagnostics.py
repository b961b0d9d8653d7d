"""Diagnostics of a state (outside the step; the paper defines none):
surface pressure, 850 hPa temperature, total mass, area-weighted RMS.

Readings:
* ps: exner at the ground extrapolated hydrostatically from the lowest full
  level with its theta_v, exner_sfc = exner + g (z_mc - z_sfc) / (cpd theta_v),
  z_sfc the ground height of the column (0 over flat ground), and
  ps = p00 exner_sfc^(cpd/rd);
* T850: T = theta_v exner at full levels, p = p00 exner^(cpd/rd); linear
  interpolation in ln p between the two levels around 850 hPa (the lowest
  level's T when the whole column is above 850 hPa);
* mass: sum over cells of A_c sum_k rho dz_k (each column's own dz over terrain);
* RMS of a difference: sqrt(sum A_c d^2 / sum A_c).
"""
import numpy as np


def surface_pressure(dycore, exner, theta_v):
    """Diagnostics outside the step; a reading, the paper defines none (its results, Sec. 5, are ICON
    runs)."""
    p, v = dycore.p, dycore.v
    dz_low = v.z_mc[..., -1] - v.z_ifc[..., -1]     # lowest full level above the ground
    ex_sfc = exner[:, -1] + p.grav * dz_low / (p.cpd * theta_v[:, -1])
    return p.p00 * ex_sfc ** (p.cpd / p.rd)


def temperature_850(dycore, exner, theta_v, p_target=85000.0):
    """Diagnostics outside the step; a reading, the paper defines none (its results, Sec. 5, are ICON
    runs)."""
    p = dycore.p
    pres = p.p00 * exner ** (p.cpd / p.rd)
    temp = theta_v * exner
    nc, nlev = exner.shape
    out = np.empty(nc)
    for c in range(nc):
        out[c] = temp[c, -1]
        for k in range(nlev - 1, 0, -1):   # from the ground up: k below, k-1 above
            if pres[c, k] >= p_target > pres[c, k - 1]:
                x = (np.log(p_target) - np.log(pres[c, k])) / (np.log(pres[c, k - 1]) - np.log(pres[c, k]))
                out[c] = temp[c, k] + x * (temp[c, k - 1] - temp[c, k])
                break
    return out


def total_mass(dycore, rho):
    """Diagnostics outside the step; a reading, the paper defines none (its results, Sec. 5, are ICON
    runs)."""
    dz = dycore.v.dz
    return float(np.sum(dycore.g.cell_area[:, None] * rho * (dz if dz.ndim == 2 else dz[None, :])))


def area_rms(dycore, diff):
    """Diagnostics outside the step; a reading, the paper defines none (its results, Sec. 5, are ICON
    runs)."""
    a = dycore.g.cell_area
    return float(np.sqrt(np.sum(a * diff ** 2) / np.sum(a)))
