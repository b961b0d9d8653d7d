"""Vertical metrics and reference state of the oracle (row A0).

Level order: k = 0 is the model top.  Full levels k = 0..nlev-1 lie between
half levels k (above) and k+1 (below); half levels run k = 0..nlev with
k = nlev the (flat) ground.  Readings (the paper gives no formula, Sec. 4.1):

* full-level height z_mc[k] = (z_ifc[k] + z_ifc[k+1]) / 2,
  layer thickness dz[k] = z_ifc[k] - z_ifc[k+1];
* interior half level k = 1..nlev-1: dzh[k] = z_mc[k-1] - z_mc[k], and a
  field X is interpolated linearly in z,
  X_ic[k] = wgt[k] X[k-1] + (1 - wgt[k]) X[k],
  wgt[k] = (z_ifc[k] - z_mc[k]) / (z_mc[k-1] - z_mc[k]);
* reference state, horizontally uniform: theta_ref(z) = T0 exp(z / H),
  H = c_pd T0 / g, at full levels; exner_ref at the lowest full level is
  exp(-z_mc / H) and is integrated upward in exact discrete hydrostatic
  balance, c_pd theta_ref_ic[k] (exner_ref[k-1] - exner_ref[k]) / dzh[k] = -g,
  with theta_ref_ic the interpolation above; d_exner_ref/dz at half levels
  is (exner_ref[k-1] - exner_ref[k]) / dzh[k];
* Rayleigh damping of w at half levels above damp_height z_d:
  w <- w / (1 + dt tau^-1 sin^2(pi/2 (z - z_d) / (z_top - z_d))).
Values at the top and ground half levels that the scheme never uses are NaN.
"""
import numpy as np


class VerticalGrid:
    """Row A0: vertical metrics and reference state, readings stated in this module's docstring."""
    def __init__(self, z_ifc, params):
        """Row A0: vertical metrics and reference state, readings stated in this module's docstring."""
        z_ifc = np.asarray(z_ifc, dtype=np.float64)
        self.nlev = nlev = z_ifc.size - 1
        self.z_ifc = z_ifc
        self.z_mc = 0.5 * (z_ifc[:-1] + z_ifc[1:])
        self.dz = z_ifc[:-1] - z_ifc[1:]
        self.dzh = np.full(nlev + 1, np.nan)
        self.wgt = np.full(nlev + 1, np.nan)
        for k in range(1, nlev):
            self.dzh[k] = self.z_mc[k - 1] - self.z_mc[k]
            self.wgt[k] = (z_ifc[k] - self.z_mc[k]) / (self.z_mc[k - 1] - self.z_mc[k])

        p = params
        T0 = p.ref_T0
        H = p.cpd * T0 / p.grav
        self.theta_ref = T0 * np.exp(self.z_mc / H)
        self.exner_ref = np.empty(nlev)
        self.exner_ref[nlev - 1] = np.exp(-self.z_mc[nlev - 1] / H)
        for k in range(nlev - 1, 0, -1):
            th_ic = self.wgt[k] * self.theta_ref[k - 1] + (1.0 - self.wgt[k]) * self.theta_ref[k]
            self.exner_ref[k - 1] = self.exner_ref[k] - p.grav * self.dzh[k] / (p.cpd * th_ic)
        self.dexner_ref_ic = np.full(nlev + 1, np.nan)
        for k in range(1, nlev):
            self.dexner_ref_ic[k] = (self.exner_ref[k - 1] - self.exner_ref[k]) / self.dzh[k]

    def interp_ic(self, x):
        """Interior half-level values [..., nlev+1] of full-level x [..., nlev]; ends NaN.
        Row A0: vertical metrics and reference state, readings stated in this module's docstring."""
        out = np.full(x.shape[:-1] + (self.nlev + 1,), np.nan)
        for k in range(1, self.nlev):
            out[..., k] = self.wgt[k] * x[..., k - 1] + (1.0 - self.wgt[k]) * x[..., k]
        return out

    def rayleigh_factor(self, dt, params):
        """dt * tau^-1 * sin^2(...) at half levels (0 below damp_height and when off).
        Row A0: vertical metrics and reference state, readings stated in this module's docstring."""
        p = params
        z = self.z_ifc
        top = z[0]
        f = np.zeros(self.nlev + 1)
        if p.rayleigh_coeff > 0.0:
            above = z > p.damp_height
            f[above] = dt * p.rayleigh_coeff * np.sin(
                0.5 * np.pi * (z[above] - p.damp_height) / (top - p.damp_height)) ** 2
        return f
