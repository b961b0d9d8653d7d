"""Terrain-following extension of the oracle (test infrastructure: only tests,
the smoke check and the benchmark's CPU baseline use ``oracle/``).

The paper runs ICON's dycore over real topography (Sec. 4.1, Sec. 5) and
states none of its formulas; the terms below are the terrain parts of rows
A0 (slopes), A1-A4 (contravariant correction), A6 (pressure-gradient chain
rule) and A7 (kinematic ground condition) of an ICON-type scheme, read on the
same grid and operators as the flat oracle (``dycore.py``), which this class
extends.  Over flat ground every term below vanishes exactly and the class
reproduces the flat oracle to rounding.

Readings:

* Half-level heights z_ifc [nc, nlev+1] per column (top first, the top flat).
  Per column: z_mc, dz, dzh, the interpolation weights and the reference
  state, all as in the flat oracle; at edges, heights are the mean of the two
  cells' and give dz_e and the edge interpolation weights.
* Slopes at edges: dz/dn = (z_c1 - z_c0)/d_e on half and full levels; dz/dt
  from the vertex heights (kite-weighted cell->vertex average, formed as
  offsets from one adjacent cell so that equal heights give an exactly flat
  vertex) along t_e.
* Contravariant correction at half levels: w_concorr = edge->cell average of
  vn_ie dz/dn + vt_ie dz/dt (vn_ie, vt_ie extrapolated to the ground as the
  lowest full level); the vertical advection in velocity advection uses the
  contravariant velocity w_con = w - w_concorr as the advecting velocity.
* Horizontal pressure gradient along the true horizontal:
  cpd theta_e [d pr/dn - (dz_mc/dn) (d pr/dz)_e], (d pr/dz)_e the mean of the
  two cells' centred (one-sided at top and bottom) vertical differences of
  the extrapolated exner perturbation; the reference part of exner is a
  function of height only and exerts no horizontal force.
* Horizontal mass and theta fluxes carry the edge layer thickness:
  div_m = (1/dz_c) div(rho_e vn dz_e), so the mass sum_c,k A_c dz_c rho is
  conserved exactly.
* Column solve in w_con: the vertical fluxes are rho_ic w_con; w_con = 0 at the
  top and the ground, so the tridiagonal system is the flat one with
  w*_con = w* - w_concorr; w = w_con + w_concorr afterwards, which sets the
  ground value w = w_concorr (kinematic condition).  The predictor uses the
  w_concorr of the "now" winds, the corrector that of the predicted winds.
  Rayleigh damping scales w_con.
* Diffusion along model levels as in the flat oracle (the truly horizontal
  diffusion of steep terrain is not part of this reading); it leaves the ground
  value of w unchanged.

Steep terrain (the paper's diffusion raises its coefficients for strong
near-surface temperature gradients, Sec. 4.1; its dycore runs over real,
steep orography), two options of DycoreParams:

* steep_hpg: at an edge full level whose two cells' levels are offset by more
  than half a layer -- the level of a neighbour column nearest to the edge's
  height z_e (the mean of the two cells' full-level heights) is not the same
  level -- the pressure gradient is taken at constant height: each cell's
  extrapolated exner perturbation is interpolated to z_e by the quadratic
  through the three consecutive levels of that column nearest to z_e
  (Lagrange weights), and hpg = cpd theta_e (pi_c1(z_e) - pi_c0(z_e)) / d_e.
  Elsewhere the chain-rule form above.
* hdiff_tenh_fac > 0: the enhanced near-surface temperature diffusion of the
  flat oracle's diffusion (dycore.py), here along the terrain-following levels.
"""
import numpy as np

from .dycore import Dycore, thomas
from .geometry import Geometry
from .params import DycoreParams


class TerrainColumns:
    """Per-column vertical metrics and reference state (row A0 with topography);
    cell arrays [nc, ...], edge arrays [ne, ...]."""

    def __init__(self, z_ifc, g: Geometry, p: DycoreParams):
        """Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        z = np.ascontiguousarray(z_ifc, dtype=np.float64)
        nc = z.shape[0]
        self.nlev = nlev = z.shape[1] - 1
        self.z_ifc = z
        self.z_mc = 0.5 * (z[:, :-1] + z[:, 1:])
        self.dz = z[:, :-1] - z[:, 1:]
        self.dzh = np.full((nc, nlev + 1), np.nan)
        self.wgt = np.full((nc, nlev + 1), np.nan)
        for k in range(1, nlev):
            self.dzh[:, k] = self.z_mc[:, k - 1] - self.z_mc[:, k]
            self.wgt[:, k] = (z[:, k] - self.z_mc[:, k]) / (self.z_mc[:, k - 1] - self.z_mc[:, k])
        # reference state, per column, in discrete hydrostatic balance
        T0 = p.ref_T0
        H = p.cpd * T0 / p.grav
        self.theta_ref = T0 * np.exp(self.z_mc / H)
        self.exner_ref = np.empty((nc, nlev))
        self.exner_ref[:, nlev - 1] = np.exp(-self.z_mc[:, nlev - 1] / H)
        for k in range(nlev - 1, 0, -1):
            th_ic = self.wgt[:, k] * self.theta_ref[:, k - 1] + (1.0 - self.wgt[:, k]) * self.theta_ref[:, k]
            self.exner_ref[:, k - 1] = self.exner_ref[:, k] - p.grav * self.dzh[:, k] / (p.cpd * th_ic)
        self.dexner_ref_ic = np.full((nc, nlev + 1), np.nan)
        for k in range(1, nlev):
            self.dexner_ref_ic[:, k] = (self.exner_ref[:, k - 1] - self.exner_ref[:, k]) / self.dzh[:, k]
        # edges: mean heights of the two cells
        c0, c1 = g.e2c[:, 0], g.e2c[:, 1]
        ze = 0.5 * (z[c0] + z[c1])
        ze_mc = 0.5 * (ze[:, :-1] + ze[:, 1:])
        self.dz_e = ze[:, :-1] - ze[:, 1:]
        self.wgt_e = np.full((g.ne, nlev + 1), np.nan)
        for k in range(1, nlev):
            self.wgt_e[:, k] = (ze[:, k] - ze_mc[:, k]) / (ze_mc[:, k - 1] - ze_mc[:, k])
        # normal slopes on half and full levels
        self.ddxn_ifc = (z[c1] - z[c0]) / g.dual_length[:, None]
        self.ddxn_mc = (self.z_mc[c1] - self.z_mc[c0]) / g.dual_length[:, None]
        self.steep = self.constant_height_stencil(g)

    def constant_height_stencil(self, g):
        """For every edge full level: the steep flag and, per adjacent cell s,
        the first of the three consecutive levels nearest to the edge height
        z_e and the Lagrange weights of z_e on them (steep_hpg option).
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        nlev = self.nlev
        c0, c1 = g.e2c[:, 0], g.e2c[:, 1]
        z_e = 0.5 * (self.z_mc[c0] + self.z_mc[c1])
        out = {"flag": np.zeros(z_e.shape, dtype=bool)}
        levels = np.arange(nlev)[None, :]
        for s, c in enumerate((c0, c1)):
            zc = self.z_mc[c]
            nearest = np.empty(z_e.shape, dtype=np.int64)
            for k in range(nlev):
                nearest[:, k] = np.argmin(np.abs(zc - z_e[:, k:k + 1]), axis=1)
            k0 = np.clip(nearest - 1, 0, nlev - 3)
            zz = [np.take_along_axis(zc, k0 + j, axis=1) for j in range(3)]
            L = []
            for j in range(3):
                a, b = [zz[i] for i in range(3) if i != j]
                L.append((z_e - a) * (z_e - b) / ((zz[j] - a) * (zz[j] - b)))
            out["k0_%d" % s] = k0
            out["w_%d" % s] = np.stack(L, axis=-1)
            out["flag"] |= nearest != levels
        out["z_e"] = z_e
        return out

    def interp_ic(self, x):
        """Interior half-level values [nc, nlev+1] of a cell field; ends NaN.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        out = np.full((x.shape[0], self.nlev + 1), np.nan)
        for k in range(1, self.nlev):
            out[:, k] = self.wgt[:, k] * x[:, k - 1] + (1.0 - self.wgt[:, k]) * x[:, k]
        return out

    def interp_ic_e(self, x):
        """Interior half-level values [ne, nlev+1] of an edge field; ends NaN.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        out = np.full((x.shape[0], self.nlev + 1), np.nan)
        for k in range(1, self.nlev):
            out[:, k] = self.wgt_e[:, k] * x[:, k - 1] + (1.0 - self.wgt_e[:, k]) * x[:, k]
        return out

    def rayleigh_factor(self, dt, p):
        """dt tau^-1 sin^2(pi/2 (z - z_d)/(z_top - z_d)) at every column's half levels.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        z = self.z_ifc
        f = np.zeros_like(z)
        if p.rayleigh_coeff > 0.0:
            top = z[:, 0:1]
            s = np.sin(0.5 * np.pi * (z - p.damp_height) / (top - p.damp_height)) ** 2
            f = np.where(z > p.damp_height, dt * p.rayleigh_coeff * s, 0.0)
        return f


class TerrainDycore(Dycore):
    """The oracle dycore over half-level heights z_ifc [nc, nlev+1].
    Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""

    def __init__(self, grid, z_ifc, params: DycoreParams = None):
        """Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        self.p = params if params is not None else DycoreParams()
        self.g = Geometry(grid, self.p.radius)
        self.v = TerrainColumns(z_ifc, self.g, self.p)
        self.f_e = self.g.coriolis(self.p.omega)
        # tangential slopes on half levels from the vertex heights; each vertex
        # height is one adjacent cell's height plus the weighted offsets of all
        # of them (the cell->vertex average, exactly flat where the heights agree)
        g, z = self.g, self.v.z_ifc
        first = z[g.v2c[:, 0]]
        z_v = first.copy()
        for j in range(6):
            c = np.where(g.v2c_mask[:, j], g.v2c[:, j], 0)
            z_v += g.v2c_weight[:, j][:, None] * (z[c] - first)
        self.ddxt_ifc = self.grad_t(z_v)

    # ---------------------------------------------------------------- A1-A4
    def half_level_winds(self, vn, vt):
        """vn and vt at half levels [ne, nlev+1]: interpolated inside, the top
        and lowest full-level values at the top and the ground.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        nlev = self.v.nlev
        vn_ie, vt_ie = self.v.interp_ic_e(vn), self.v.interp_ic_e(vt)
        vn_ie[:, 0], vn_ie[:, nlev] = vn[:, 0], vn[:, nlev - 1]
        vt_ie[:, 0], vt_ie[:, nlev] = vt[:, 0], vt[:, nlev - 1]
        return vn_ie, vt_ie

    def tangential_wind(self, vn):
        """Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        g = self.g
        uc = self.perot_cell(vn)
        return 0.5 * np.einsum("ekx,ex->ek", uc[g.e2c[:, 0]] + uc[g.e2c[:, 1]], g.tangent)

    def w_concorr(self, vn):
        """Contravariant correction [nc, nlev+1] of the winds vn: the vertical
        velocity of a parcel that follows the coordinate surface.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        vn_ie, vt_ie = self.half_level_winds(vn, self.tangential_wind(vn))
        return self.edge_to_cell(vn_ie * self.v.ddxn_ifc + vt_ie * self.ddxt_ifc)

    def velocity_tendencies(self, vn, w):
        """As the flat oracle, with the contravariant velocity w - w_concorr as
        the advecting vertical velocity and edge layer thicknesses.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        g, v = self.g, self.v
        nlev = v.nlev
        c0, c1 = g.e2c[:, 0], g.e2c[:, 1]
        vt = self.tangential_wind(vn)
        vn_ie, vt_ie = self.half_level_winds(vn, vt)
        w_con = w - self.edge_to_cell(vn_ie * v.ddxn_ifc + vt_ie * self.ddxt_ifc)
        ekin_e = 0.5 * (vn * vn + vt * vt)
        ekin_c = self.edge_to_cell(ekin_e)
        w_full = 0.5 * (w[:, :-1] + w[:, 1:])
        wcon_full = 0.5 * (w_con[:, :-1] + w_con[:, 1:])
        zeta_v = self.curl(vn)
        w_v = self.cell_to_vert(w)
        zeta_e = 0.5 * (zeta_v[g.e2v[:, 0]] + zeta_v[g.e2v[:, 1]])
        wbar_e = 0.5 * (wcon_full[c0] + wcon_full[c1])
        dvn_dz = (vn_ie[:, :-1] - vn_ie[:, 1:]) / v.dz_e
        ddt_vn = (-self.grad_n(ekin_c) + (zeta_e + self.f_e[:, None]) * vt
                  - wbar_e * dvn_dz)
        hadv_w_e = np.zeros((g.ne, nlev + 1))
        kk = slice(1, nlev)
        hadv_w_e[:, kk] = (vn_ie[:, kk] * self.grad_n(w)[:, kk]
                           + vt_ie[:, kk] * self.grad_t(w_v)[:, kk])
        ddt_w = np.zeros((g.nc, nlev + 1))
        hadv_w_c = self.edge_to_cell(hadv_w_e)
        for k in range(1, nlev):
            ddt_w[:, k] = (-hadv_w_c[:, k]
                           - w_con[:, k] * (w_full[:, k - 1] - w_full[:, k]) / v.dzh[:, k])
        return ddt_vn, ddt_w, vt

    # ---------------------------------------------------------------- A6
    def horizontal_pressure_gradient(self, pr_ex, theta_e):
        """cpd theta_e [d pr/dn - (dz_mc/dn) (d pr/dz)_e] along the true horizontal.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        g, v = self.g, self.v
        zm = v.z_mc
        dpdz = np.empty_like(pr_ex)
        dpdz[:, 1:-1] = (pr_ex[:, :-2] - pr_ex[:, 2:]) / (zm[:, :-2] - zm[:, 2:])
        dpdz[:, 0] = (pr_ex[:, 0] - pr_ex[:, 1]) / (zm[:, 0] - zm[:, 1])
        dpdz[:, -1] = (pr_ex[:, -2] - pr_ex[:, -1]) / (zm[:, -2] - zm[:, -1])
        dpdz_e = 0.5 * (dpdz[g.e2c[:, 0]] + dpdz[g.e2c[:, 1]])
        hpg = self.p.cpd * theta_e * (self.grad_n(pr_ex) - v.ddxn_mc * dpdz_e)
        if self.p.steep_hpg:
            st = v.steep
            at_z = []
            tot = pr_ex + v.exner_ref          # the total exner is smooth in height
            for s in (0, 1):
                col = tot[g.e2c[:, s]]
                k0, w = st["k0_%d" % s], st["w_%d" % s]
                at_z.append(sum(w[..., j] * np.take_along_axis(col, k0 + j, axis=1) for j in range(3)))
            flat_z = self.p.cpd * theta_e * (at_z[1] - at_z[0]) / g.dual_length[:, None]
            hpg = np.where(st["flag"], flat_z, hpg)
        return hpg

    def layer_div(self, F):
        """Flux divergence per unit volume of a layer: (1/dz_c) div(F dz_e).
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        return self.div(F * self.v.dz_e) / self.v.dz

    # ---------------------------------------------------------------- A7
    def vertical_solve(self, now, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w_expl, dt, w_concorr=None):
        """The flat column solve in the contravariant velocity w_con = w - w_concorr
        (zero at the top and the ground), with per-column metrics.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        p, v = self.p, self.v
        nlev = v.nlev
        beta = p.vwind_impl_wgt
        rho, exner, theta, w = now["rho"], now["exner"], now["theta_v"], now["w"]
        nc = rho.shape[0]
        wc = np.zeros((nc, nlev + 1)) if w_concorr is None else w_concorr
        pr = exner - v.exner_ref
        zb = dt * (p.rd / p.cvd) * exner / (rho * theta * v.dz)
        rho_ic0 = np.zeros((nc, nlev + 1))
        rt_ic0 = np.zeros((nc, nlev + 1))
        rho_ic0[:, 1:nlev] = rho_ic[:, 1:nlev]
        rt_ic0[:, 1:nlev] = rho_ic[:, 1:nlev] * theta_ic[:, 1:nlev]
        alpha = beta * rt_ic0
        w_con = w - wc
        w_con[:, 0] = 0.0
        w_con[:, nlev] = 0.0
        fw = rho_ic0 * w_con
        gw = rt_ic0 * w_con
        rho_star = rho - dt * div_m - dt * (1.0 - beta) * (fw[:, :-1] - fw[:, 1:]) / v.dz
        pr_star = pr - zb * (v.dz * div_t + (1.0 - beta) * (gw[:, :-1] - gw[:, 1:]))
        w_star = np.zeros((nc, nlev + 1))
        for k in range(1, nlev):
            w_star[:, k] = w[:, k] + dt * ddt_w_expl[:, k] - dt * p.cpd * (
                (1.0 - beta) * theta_ic[:, k] * (pr[:, k - 1] - pr[:, k]) / v.dzh[:, k]
                + thp_ic[:, k] * v.dexner_ref_ic[:, k])
        a = np.zeros((nc, nlev + 1))
        b = np.ones((nc, nlev + 1))
        c = np.zeros((nc, nlev + 1))
        r = np.zeros((nc, nlev + 1))
        for k in range(1, nlev):
            gam = dt * p.cpd * beta * theta_ic[:, k] / v.dzh[:, k]
            a[:, k] = -gam * zb[:, k - 1] * alpha[:, k - 1]
            b[:, k] = 1.0 + gam * alpha[:, k] * (zb[:, k - 1] + zb[:, k])
            c[:, k] = -gam * zb[:, k] * alpha[:, k + 1]
            r[:, k] = (w_star[:, k] - wc[:, k]) - gam * (pr_star[:, k - 1] - pr_star[:, k])
        wcon_new = np.zeros((nc, nlev + 1))
        wcon_new[:, 1:nlev] = thomas(a[:, 1:nlev], b[:, 1:nlev], c[:, 1:nlev], r[:, 1:nlev])
        wcon_new = wcon_new / (1.0 + v.rayleigh_factor(dt, p))
        fwn = rho_ic0 * wcon_new
        gwn = alpha * wcon_new
        rho_new = rho_star - dt * beta * (fwn[:, :-1] - fwn[:, 1:]) / v.dz
        pr_new = pr_star - zb * (gwn[:, :-1] - gwn[:, 1:])
        theta_new = theta * (rho / rho_new) * (1.0 + (p.cvd / p.rd) * (pr_new - pr) / exner)
        return dict(w=wcon_new + wc, rho=rho_new, exner=v.exner_ref + pr_new, theta_v=theta_new)

    # ---------------------------------------------------------------- substep
    def substep(self, st):
        """The flat substep (predictor, corrector) with the terrain terms above.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        p, v = self.p, self.v
        dt = p.dtime / p.ndyn_substeps
        vn, w = st["vn"], st["w"]
        rho, exner, theta = st["rho"], st["exner"], st["theta_v"]
        # predictor
        ddt_vn_now, ddt_w_now, vt = self.velocity_tendencies(vn, w)
        wc_now = self.w_concorr(vn)
        pr = exner - v.exner_ref
        pr_ex = self.extrapolate_exner(pr, st["exner_pr"])
        exner_pr_new = pr.copy()
        rho_e = self.upwind_edge_values(rho, vn, vt, dt)
        theta_e = self.upwind_edge_values(theta, vn, vt, dt)
        hpg = self.horizontal_pressure_gradient(pr_ex, theta_e)
        vn_pred = vn + dt * (ddt_vn_now - hpg)
        rho_ic = v.interp_ic(rho)
        theta_ic = v.interp_ic(theta)
        thp_ic = v.interp_ic(theta - v.theta_ref)
        vn_flx = self.flux_velocity(vn_pred)
        div_m = self.layer_div(rho_e * vn_flx)
        div_t = self.layer_div(rho_e * theta_e * vn_flx)
        pred = self.vertical_solve(st, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w_now, dt, wc_now)
        # corrector
        ddt_vn_pred, ddt_w_pred, _ = self.velocity_tendencies(vn_pred, pred["w"])
        wc_pred = self.w_concorr(vn_pred)
        dd = self.lap_cell(self.div(vn_pred))
        mean_area = np.mean(self.g.cell_area)
        vn_new = vn + dt * (p.wgt_nnow_vel * ddt_vn_now + p.wgt_nnew_vel * ddt_vn_pred - hpg) \
            - p.divdamp_fac * mean_area * mean_area * self.grad_n(dd)
        rho_avg = p.wgt_nnow_rth * rho + p.wgt_nnew_rth * pred["rho"]
        th_avg = p.wgt_nnow_rth * theta + p.wgt_nnew_rth * pred["theta_v"]
        rho_ic = v.interp_ic(rho_avg)
        theta_ic = v.interp_ic(th_avg)
        thp_ic = v.interp_ic(th_avg - v.theta_ref)
        vn_flx = self.flux_velocity(vn_new)
        div_m = self.layer_div(rho_e * vn_flx)
        div_t = self.layer_div(rho_e * theta_e * vn_flx)
        ddt_w = p.wgt_nnow_vel * ddt_w_now + p.wgt_nnew_vel * ddt_w_pred
        new = self.vertical_solve(st, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w, dt, wc_pred)
        new["vn"] = vn_new
        new["exner_pr"] = exner_pr_new
        return new

    # ---------------------------------------------------------------- A10
    def diffusion(self, st):
        """The flat diffusion along model levels (with the enhanced near-surface
        temperature diffusion when hdiff_tenh_fac > 0); the ground value of w
        (the kinematic condition) is left as it is.
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        out = super().diffusion(st)
        out["w"][:, self.v.nlev] = st["w"][:, self.v.nlev]
        return out

    def initial_exner_pr(self, exner):
        """Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        return exner - self.v.exner_ref

    def reference_state(self):
        """Per-column reference profiles (theta_ref, exner_ref) [nc, nlev].
        Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        return self.v.theta_ref.copy(), self.v.exner_ref.copy()

    def total_mass(self, rho):
        """Terrain reading of rows A0-A7 (Sec. 4.1), stated in the module docstring."""
        return float(np.sum(self.g.cell_area[:, None] * rho * self.v.dz))
