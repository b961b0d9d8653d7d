"""One time step of the ICON-type nonhydrostatic dynamical core (oracle).

Structure (paper Sec. 4.1 and Fig. 1, Sec. 5.1): a step is ``ndyn_substeps``
dynamical substeps followed by one diffusion call.  Each substep is a
predictor and a corrector.  Each of the two starts with the advective
tendencies (velocity advection); the horizontal momentum equation is then
updated with pressure-gradient and advection terms, divergence damping acts
in the corrector only, and w and the thermodynamic state are advanced by a
vertically implicit solver.  Diffusion (Smagorinsky plus fourth-order
background) acts on vn, w and theta_v/exner once per step.

All formulas below are readings of an ICON-type scheme (the paper states
none); the layout is level-contiguous, X[h, k], k = 0 at the model top.

Prognostic state: vn [ne, nlev], w [nc, nlev+1], rho, exner, theta_v
[nc, nlev], and the exner perturbation of the previous substep exner_pr
[nc, nlev] (exner extrapolation history).  With flat ground the
contravariant vertical wind equals w and w = 0 at the top and the ground.
"""
import numpy as np

from .geometry import Geometry, project
from .params import DycoreParams
from .vertical import VerticalGrid


class Dycore:
    """The dycore step of Sec. 4.1 (rows A0-A10) as an ICON-type reading."""
    def __init__(self, grid, z_ifc, params: DycoreParams = None):
        """Row A0 set-up: geometry, vertical metrics, Coriolis parameter."""
        self.p = params if params is not None else DycoreParams()
        self.g = Geometry(grid, self.p.radius)
        self.v = VerticalGrid(z_ifc, self.p)
        self.f_e = self.g.coriolis(self.p.omega)

    # ------------------------------------------------------------------
    # discrete operators (row A0 readings, see geometry.py)
    # ------------------------------------------------------------------
    def div(self, F):
        """Cell divergence (1/A_c) sum_e s_{c,e} l_e F_e of an edge field [ne, K].
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        out = np.zeros((g.nc, F.shape[1]))
        for j in range(3):
            e = g.c2e[:, j]
            out += (g.c2e_sign[:, j] * g.edge_length[e])[:, None] * F[e]
        return out / g.cell_area[:, None]

    def curl(self, F):
        """Vertex circulation (1/A_v) sum_e t_{v,e} d_e F_e of an edge field.
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        out = np.zeros((g.nv, F.shape[1]))
        for j in range(6):
            e = np.where(g.v2e_mask[:, j], g.v2e[:, j], 0)
            out += (g.v2e_sign[:, j] * g.dual_length[e])[:, None] * F[e]
        return out / g.dual_area[:, None]

    def grad_n(self, X):
        """Edge-normal gradient (X_c1 - X_c0) / d_e of a cell field.
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        return (X[g.e2c[:, 1]] - X[g.e2c[:, 0]]) / g.dual_length[:, None]

    def grad_t(self, Y):
        """Edge-tangential gradient of a vertex field: (Y at the vertex t_e points to
        minus Y at the other) / l_e.
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        return (g.e2v_sign[:, 0:1] * Y[g.e2v[:, 0]] + g.e2v_sign[:, 1:2] * Y[g.e2v[:, 1]]) \
            / g.edge_length[:, None]

    def edge_to_cell(self, F):
        """sum_e q_{c,e} F_e (area-weighted edge->cell average).
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        out = np.zeros((g.nc, F.shape[1]))
        for j in range(3):
            out += g.e2c_weight[:, j][:, None] * F[g.c2e[:, j]]
        return out

    def cell_to_vert(self, X):
        """Kite-area weighted cell->vertex average; row A0 operator, a reading of the ICON
        discretisation Sec. 4.1 cites."""
        g = self.g
        out = np.zeros((g.nv, X.shape[1]))
        for j in range(6):
            c = np.where(g.v2c_mask[:, j], g.v2c[:, j], 0)
            out += g.v2c_weight[:, j][:, None] * X[c]
        return out

    def lap_cell(self, X):
        """Cell Laplacian (1/A_c) sum_e l_e (X_nbr - X_c) / d_e.
        Row A0 operator, a reading of the ICON discretisation Sec. 4.1 cites."""
        g = self.g
        out = np.zeros_like(X)
        for j in range(3):
            e = g.c2e[:, j]
            out += (g.edge_length[e] / g.dual_length[e])[:, None] * (X[g.c2e2c[:, j]] - X)
        return out / g.cell_area[:, None]

    def lap_vec(self, F):
        """Vector Laplacian of an edge-normal field: grad_n(div F) - grad_t(curl F).
        Rows A8/A10 (diffusion), a reading of the ICON discretisation Sec. 4.1 cites."""
        return self.grad_n(self.div(F)) - self.grad_t(self.curl(F))

    def perot_cell(self, vn):
        """Cell velocity vector [nc, K, 3]: (1/A_c) sum_e s l_e vn_e (x_e - x_c),
        projected on the tangent plane at the cell centre (Perot reconstruction).
        Row A1 reconstruction, a reading (ICON's own is not given, Sec. 4.1)."""
        g = self.g
        u = np.zeros((g.nc, vn.shape[1], 3))
        for j in range(3):
            e = g.c2e[:, j]
            coef = g.c2e_sign[:, j] * g.edge_length[e] / g.cell_area
            dx = g.a * (g.E[e] - g.C)
            u += coef[:, None, None] * vn[e][:, :, None] * dx[:, None, :]
        return project(u, g.C[:, None, :])

    def vertex_velocity(self, vn):
        """Vertex velocity vector [nv, K, 3] from the dual-cell circulation:
        u_v = r_v x (1/A_v) sum_e t_{v,e} d_e vn_e (m_e - x_v), m_e the dual-edge
        midpoint; exact for uniform flow on a plane.
        Row A10 (Smagorinsky deformation), a reading (Sec. 4.1)."""
        g = self.g
        s = np.zeros((g.nv, vn.shape[1], 3))
        for j in range(6):
            e = np.where(g.v2e_mask[:, j], g.v2e[:, j], 0)
            coef = g.v2e_sign[:, j] * g.dual_length[e] / g.dual_area
            dx = g.a * (g.dual_mid[e] - g.V)
            s += coef[:, None, None] * vn[e][:, :, None] * dx[:, None, :]
        s = project(s, g.V[:, None, :])
        return np.cross(np.broadcast_to(g.V[:, None, :], s.shape), s)

    def grad_cell(self, X):
        """Green-Gauss cell gradient [nc, K, 3]:
        (1/A_c) sum_e s l_e n_e (X_e - X_c), projected on the tangent plane, with X_e
        the linear interpolation along the dual edge to the edge midpoint,
        X_e = (r1 X_c0 + r0 X_c1)/(r0 + r1), r_i = arc(x_ci, x_e).  Subtracting X_c
        changes nothing on a plane (sum_e s l n_e = 0 around a closed polygon) and
        makes the gradient of a constant exactly zero on the sphere, where the
        edge normals lie in different tangent planes.
        Row A5/A6 (upwind reconstruction), a reading (Sec. 4.1)."""
        g = self.g
        out = np.zeros(X.shape + (3,))
        for j in range(3):
            e = g.c2e[:, j]
            coef = g.c2e_sign[:, j] * g.edge_length[e] / g.cell_area
            w_self = np.where(g.e2c[e, 0] == np.arange(g.nc), g.e2c_lin[e, 0], g.e2c_lin[e, 1])
            dxe = (1.0 - w_self)[:, None] * (X[g.c2e2c[:, j]] - X)
            out += coef[:, None, None] * dxe[:, :, None] * g.normal[e][:, None, :]
        return project(out, g.C[:, None, :])

    # ------------------------------------------------------------------
    # velocity advection (rows A1-A4)
    # ------------------------------------------------------------------
    def velocity_tendencies(self, vn, w):
        """Advective tendencies of vn and w (Sec. 4.1: each predictor and corrector
        starts with them).  Returns ddt_vn [ne, nlev] and ddt_w [nc, nlev+1].

        ddt_vn = -dK/dn + (zeta_e + f_e) vt - wbar_e dvn/dz
        ddt_w  = -(v . grad w)_cell - w dw/dz
        """
        g, v = self.g, self.v
        nlev = v.nlev
        c0, c1 = g.e2c[:, 0], g.e2c[:, 1]
        # A1: tangential wind, half-level vn and vt, kinetic energy at edges
        uc = self.perot_cell(vn)
        vt = 0.5 * np.einsum("ekx,ex->ek", uc[c0] + uc[c1], g.tangent)
        vn_ie = v.interp_ic(vn)
        vn_ie[:, 0] = vn[:, 0]
        vn_ie[:, nlev] = vn[:, nlev - 1]
        vt_ie = v.interp_ic(vt)
        ekin_e = 0.5 * (vn * vn + vt * vt)
        # A2: cell kinetic energy, full-level w, vertex vorticity and w
        ekin_c = self.edge_to_cell(ekin_e)
        w_full = 0.5 * (w[:, :-1] + w[:, 1:])
        zeta_v = self.curl(vn)
        w_v = self.cell_to_vert(w)
        # A3: vn tendency
        zeta_e = 0.5 * (zeta_v[g.e2v[:, 0]] + zeta_v[g.e2v[:, 1]])
        wbar_e = 0.5 * (w_full[c0] + w_full[c1])
        dvn_dz = (vn_ie[:, :-1] - vn_ie[:, 1:]) / v.dz[None, :]
        ddt_vn = (-self.grad_n(ekin_c) + (zeta_e + self.f_e[:, None]) * vt
                  - wbar_e * dvn_dz)
        # horizontal advection of w at edges, interior half levels
        hadv_w_e = np.zeros((g.ne, nlev + 1))
        kk = slice(1, nlev)
        hadv_w_e[:, kk] = (vn_ie[:, kk] * self.grad_n(w)[:, kk]
                           + vt_ie[:, kk] * self.grad_t(w_v)[:, kk])
        # A4: w tendency at interior half levels; 0 at the top and the ground
        ddt_w = np.zeros((g.nc, nlev + 1))
        hadv_w_c = self.edge_to_cell(hadv_w_e)
        for k in range(1, nlev):
            ddt_w[:, k] = (-hadv_w_c[:, k]
                           - w[:, k] * (w_full[:, k - 1] - w_full[:, k]) / v.dzh[k])
        return ddt_vn, ddt_w, vt

    # ------------------------------------------------------------------
    # vertically implicit solve (row A7)
    # ------------------------------------------------------------------
    def vertical_solve(self, now, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w_expl, dt):
        """Column solve of one predictor or corrector pass.

        Equations, for full levels k (dz_k) and interior half levels k (dzh_k),
        beta = vwind_impl_wgt, pr = exner - exner_ref:

          rho_new_k = rho_k - dt div_m_k - dt/dz_k [ (1-beta)(Fw_k - Fw_k+1)
                                                      + beta (Fw'_k - Fw'_k+1) ],  Fw = rho_ic w
          pr_new_k  = pr_k - zb_k [ dz_k div_t_k + (1-beta)(Gw_k - Gw_k+1)
                                     + beta (Gw'_k - Gw'_k+1) ],                   Gw = rho_ic theta_ic w
          w'_k      = w_k + dt ddt_w_k
                      - dt c_pd [ theta_ic_k ((1-beta) dpr^n_k + beta dpr'_k) / dzh_k
                                  + theta'_ic_k dexner_ref_k ]
        with zb_k = dt (R_d/c_vd) exner_k / (rho_k theta_k dz_k), primes = new
        values, dpr_k = pr_{k-1} - pr_k, w = 0 at the top and the ground.
        Eliminating pr_new gives a tridiagonal system in w' (Thomas algorithm,
        top to bottom, no pivoting); Rayleigh damping then scales w', and
        rho and pr follow by back-substitution.  theta_v comes from the
        linearised equation of state,
          theta_new = theta (rho / rho_new) (1 + (c_vd/R_d)(pr_new - pr) / exner).
        Row A7, Sec. 4.1: the vertically implicit solver of solve_nonhydro."""
        p, v = self.p, self.v
        nlev = v.nlev
        beta = p.vwind_impl_wgt
        rho, exner, theta, w = now["rho"], now["exner"], now["theta_v"], now["w"]
        pr = exner - v.exner_ref[None, :]
        zb = dt * (p.rd / p.cvd) * exner / (rho * theta * v.dz[None, :])
        nc = rho.shape[0]
        # half-level products, zero at top and ground (w = 0 there)
        rho_ic0 = np.zeros((nc, nlev + 1))
        rt_ic0 = np.zeros((nc, nlev + 1))
        rho_ic0[:, 1:nlev] = rho_ic[:, 1:nlev]
        rt_ic0[:, 1:nlev] = rho_ic[:, 1:nlev] * theta_ic[:, 1:nlev]
        alpha = beta * rt_ic0
        # explicit parts
        fw = rho_ic0 * w
        gw = rt_ic0 * w
        rho_star = rho - dt * div_m - dt * (1.0 - beta) * (fw[:, :-1] - fw[:, 1:]) / v.dz[None, :]
        pr_star = pr - zb * (v.dz[None, :] * div_t + (1.0 - beta) * (gw[:, :-1] - gw[:, 1:]))
        w_star = np.zeros((nc, nlev + 1))
        for k in range(1, nlev):
            w_star[:, k] = w[:, k] + dt * ddt_w_expl[:, k] - dt * p.cpd * (
                (1.0 - beta) * theta_ic[:, k] * (pr[:, k - 1] - pr[:, k]) / v.dzh[k]
                + thp_ic[:, k] * v.dexner_ref_ic[k])
        # tridiagonal system for w at k = 1..nlev-1
        a = np.zeros((nc, nlev + 1))
        b = np.ones((nc, nlev + 1))
        c = np.zeros((nc, nlev + 1))
        r = np.zeros((nc, nlev + 1))
        for k in range(1, nlev):
            gam = dt * p.cpd * beta * theta_ic[:, k] / v.dzh[k]
            a[:, k] = -gam * zb[:, k - 1] * alpha[:, k - 1]
            b[:, k] = 1.0 + gam * alpha[:, k] * (zb[:, k - 1] + zb[:, k])
            c[:, k] = -gam * zb[:, k] * alpha[:, k + 1]
            r[:, k] = w_star[:, k] - gam * (pr_star[:, k - 1] - pr_star[:, k])
        w_new = thomas(a[:, 1:nlev], b[:, 1:nlev], c[:, 1:nlev], r[:, 1:nlev])
        w_full_new = np.zeros((nc, nlev + 1))
        w_full_new[:, 1:nlev] = w_new
        # Rayleigh damping of w in the upper layers
        rf = v.rayleigh_factor(dt, p)
        w_full_new = w_full_new / (1.0 + rf[None, :])
        # back-substitution
        fwn = rho_ic0 * w_full_new
        gwn = alpha * w_full_new
        rho_new = rho_star - dt * beta * (fwn[:, :-1] - fwn[:, 1:]) / v.dz[None, :]
        pr_new = pr_star - zb * (gwn[:, :-1] - gwn[:, 1:])
        exner_new = v.exner_ref[None, :] + pr_new
        theta_new = theta * (rho / rho_new) * (1.0 + (p.cvd / p.rd) * (pr_new - pr) / exner)
        return dict(w=w_full_new, rho=rho_new, exner=exner_new, theta_v=theta_new)

    def flux_velocity(self, vn):
        """Velocity of the horizontal mass and theta fluxes:
        vn + divflux_fac * Abar * grad_n(div vn), Abar the mean cell area.

        A reading: a rhombus average of vn that is exact for uniform flow reduces
        to vn plus a multiple of grad_n(div vn); this form damps the divergent
        grid-scale (acoustic) modes in the continuity equations only, keeps the
        fluxes edge-based (mass stays conserved exactly) and changes smooth flow
        at second order.  It lowers the largest eigenvalue of the discrete
        acoustic operator grad(div(.)) so that the forward-backward substep
        stays stable at horizontal acoustic Courant numbers near 0.7."""
        p = self.p
        if p.divflux_fac == 0.0:
            return vn
        am = np.mean(self.g.cell_area)
        return vn + p.divflux_fac * am * self.grad_n(self.div(vn))

    # ------------------------------------------------------------------
    # predictor pieces (rows A5, A6)
    # ------------------------------------------------------------------
    def extrapolate_exner(self, pr, pr_old):
        """Exner perturbation extrapolated linearly in time from the substeps
        n-1 and n to n + gamma, gamma = exner_exfac:
        (1 + gamma) pr - gamma pr_old.
        Row A5, a reading of the predictor in Sec. 4.1."""
        gam = self.p.exner_exfac
        return (1.0 + gam) * pr - gam * pr_old

    def upwind_edge_values(self, X, vn, vt, dt):
        """Edge values [ne, K] of the cell field X taken from the upwind cell
        (c0 where vn >= 0, else c1) at the back-trajectory point of the edge
        midpoint over dt/2: X_up + grad X_up . (a x_e - (dt/2) v_e - a x_up),
        v_e = vn n + vt t, grad the Green-Gauss cell gradient.
        Row A6, a reading of the predictor in Sec. 4.1."""
        g = self.g
        c0, c1 = g.e2c[:, 0], g.e2c[:, 1]
        grad = self.grad_cell(X)
        up = np.where(vn >= 0.0, c0[:, None], c1[:, None])         # [ne, K]
        disp = (g.a * (g.E[:, None, :] - g.C[up])
                - 0.5 * dt * (vn[:, :, None] * g.normal[:, None, :]
                              + vt[:, :, None] * g.tangent[:, None, :]))
        kidx = np.arange(X.shape[1])[None, :]
        return X[up, kidx] + np.sum(grad[up, kidx] * disp, axis=-1)

    # ------------------------------------------------------------------
    # one dynamical substep: predictor + corrector (rows A5-A9, A7)
    # ------------------------------------------------------------------
    def substep(self, st):
        """Advance the state dict by one substep dt_s = dtime / ndyn_substeps.
        Returns the new state (vn, w, rho, exner, theta_v, exner_pr).
        Rows A5-A9 and A7, Sec. 4.1: one predictor-corrector substep."""
        p, g, v = self.p, self.g, self.v
        dt = p.dtime / p.ndyn_substeps
        vn, w = st["vn"], st["w"]
        rho, exner, theta = st["rho"], st["exner"], st["theta_v"]

        # ---------------- predictor ----------------
        ddt_vn_now, ddt_w_now, vt = self.velocity_tendencies(vn, w)
        # A5: exner perturbation, extrapolated in time; history update
        pr = exner - v.exner_ref[None, :]
        pr_ex = self.extrapolate_exner(pr, st["exner_pr"])
        exner_pr_new = pr.copy()
        # A6: upwind rho and theta_v at edges from a back trajectory over dt/2
        rho_e = self.upwind_edge_values(rho, vn, vt, dt)
        theta_e = self.upwind_edge_values(theta, vn, vt, dt)
        # horizontal pressure gradient term, kept for the corrector
        hpg = p.cpd * theta_e * self.grad_n(pr_ex)
        vn_pred = vn + dt * (ddt_vn_now - hpg)
        # A7 (predictor): fluxes with the predicted vn, half levels from "now"
        rho_ic = v.interp_ic(rho)
        theta_ic = v.interp_ic(theta)
        thp_ic = v.interp_ic(theta - v.theta_ref[None, :])
        vn_flx = self.flux_velocity(vn_pred)
        div_m = self.div(rho_e * vn_flx)
        div_t = self.div(rho_e * theta_e * vn_flx)
        pred = self.vertical_solve(st, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w_now, dt)

        # ---------------- corrector ----------------
        ddt_vn_pred, ddt_w_pred, _ = self.velocity_tendencies(vn_pred, pred["w"])
        # A8: fourth-order divergence damping on the predicted vn
        dd = self.lap_cell(self.div(vn_pred))
        mean_area = np.mean(g.cell_area)
        # A9: vn corrector
        vn_new = vn + dt * (p.wgt_nnow_vel * ddt_vn_now + p.wgt_nnew_vel * ddt_vn_pred - hpg) \
            - p.divdamp_fac * mean_area * mean_area * self.grad_n(dd)
        # A7 (corrector): time-averaged rho, theta for the half-level values
        rho_avg = p.wgt_nnow_rth * rho + p.wgt_nnew_rth * pred["rho"]
        th_avg = p.wgt_nnow_rth * theta + p.wgt_nnew_rth * pred["theta_v"]
        rho_ic = v.interp_ic(rho_avg)
        theta_ic = v.interp_ic(th_avg)
        thp_ic = v.interp_ic(th_avg - v.theta_ref[None, :])
        vn_flx = self.flux_velocity(vn_new)
        div_m = self.div(rho_e * vn_flx)
        div_t = self.div(rho_e * theta_e * vn_flx)
        ddt_w = p.wgt_nnow_vel * ddt_w_now + p.wgt_nnew_vel * ddt_w_pred
        new = self.vertical_solve(st, rho_ic, theta_ic, thp_ic, div_m, div_t, ddt_w, dt)
        new["vn"] = vn_new
        new["exner_pr"] = exner_pr_new
        return new

    # ------------------------------------------------------------------
    # diffusion (row A10)
    # ------------------------------------------------------------------
    def smagorinsky(self, vn):
        """nu_e = c_s A_e |D|, |D| = sqrt(tension^2 + shear^2) from the velocity
        vectors at the four vertices of the edge's diamond.
        Row A10, Sec. 4.1 (horizontal diffusion), a reading."""
        g = self.g
        uv = self.vertex_velocity(vn)
        sgn0 = g.e2v_sign[:, 0]
        # vertex that t_e points to (v_t+) and away from (v_t-)
        vtp = np.where(sgn0 > 0, g.e2v[:, 0], g.e2v[:, 1])
        vtm = np.where(sgn0 > 0, g.e2v[:, 1], g.e2v[:, 0])
        vnm, vnp = g.e2c2v[:, 2], g.e2c2v[:, 3]     # opposite vertex in c0 (behind), c1 (ahead)
        n, t = g.normal[:, None, :], g.tangent[:, None, :]
        du_t = uv[vtp] - uv[vtm]
        du_n = uv[vnp] - uv[vnm]
        l, dn = g.edge_length[:, None], g.vert_vert_length[:, None]
        tension = np.sum(du_n * n, -1) / dn - np.sum(du_t * t, -1) / l
        shear = np.sum(du_t * n, -1) / l + np.sum(du_n * t, -1) / dn
        return self.p.hdiff_smag_fac * g.edge_area[:, None] * np.sqrt(tension ** 2 + shear ** 2)

    def diffusion(self, st):
        """Horizontal diffusion over the full time step dtime:
          vn <- vn + dt nu_e lap(vn) - k4 A_e^2 lap(lap(vn))
          w  <- w - k4w A_c^2 lapc(lapc(w))          (interior half levels)
          theta <- theta + dt (1/A_c) sum_e l_e nu_e (theta_nbr - theta_c)/d_e
          exner <- exner (1 + (R_d/c_vd)(theta_new - theta)/theta)
        with, for theta only and when hdiff_tenh_fac > 0, nu_e raised by
        hdiff_tenh_fac A_e / dt max(e_c0, e_c1) (enhanced_edge_factor).
        Row A10, Sec. 4.1 (nh_diffusion), a reading."""
        p, g, v = self.p, self.g, self.v
        dt = p.dtime
        vn, w, theta, exner = st["vn"], st["w"], st["theta_v"], st["exner"]
        nu = self.smagorinsky(vn)
        lap = self.lap_vec(vn)
        lap2 = self.lap_vec(lap)
        vn_new = vn + dt * nu * lap - p.hdiff_k4 * (g.edge_area ** 2)[:, None] * lap2
        lw = self.lap_cell(w)
        lw2 = self.lap_cell(lw)
        w_new = w - p.hdiff_w_k4 * (g.cell_area ** 2)[:, None] * lw2
        w_new[:, 0] = 0.0
        w_new[:, v.nlev] = 0.0
        out = dict(st)
        out["vn"], out["w"] = vn_new, w_new
        if p.hdiff_temp:
            if p.hdiff_tenh_fac > 0.0:   # enhanced near-surface temperature diffusion
                nu = nu + p.hdiff_tenh_fac * g.edge_area[:, None] / dt * self.enhanced_edge_factor(theta)
            flux = np.zeros_like(theta)
            for j in range(3):
                e = g.c2e[:, j]
                flux += (g.edge_length[e] / g.dual_length[e])[:, None] * nu[e] \
                    * (theta[g.c2e2c[:, j]] - theta)
            th_new = theta + dt * flux / g.cell_area[:, None]
            out["theta_v"] = th_new
            out["exner"] = exner * (1.0 + (p.rd / p.cvd) * (th_new - theta) / theta)
        return out

    def enhanced_edge_factor(self, theta):
        """max(e_c0, e_c1) per edge and level: e_c = min(1, (|theta_c - mean of
        its three neighbours| - thresh) / thresh) in the lowest
        hdiff_tenh_levels levels where above the threshold, else 0.
        Row A10, the diffusion's increased coefficients for strong near-surface
        temperature gradients (Sec. 4.1), a reading."""
        p, g = self.p, self.g
        nbr = (theta[g.c2e2c[:, 0]] + theta[g.c2e2c[:, 1]] + theta[g.c2e2c[:, 2]]) / 3.0
        ex = np.clip((np.abs(theta - nbr) - p.hdiff_tenh_thresh) / p.hdiff_tenh_thresh, 0.0, 1.0)
        ex[:, :max(0, theta.shape[1] - p.hdiff_tenh_levels)] = 0.0
        return np.maximum(ex[g.e2c[:, 0]], ex[g.e2c[:, 1]])

    # ------------------------------------------------------------------
    def step(self, st):
        """One full time step: ndyn_substeps substeps, then diffusion.
        Sec. 4.1 and Sec. 5.1: ndyn_substeps substeps per diffusion call."""
        for _ in range(self.p.ndyn_substeps):
            st = self.substep(st)
        return self.diffusion(st)

    def initial_exner_pr(self, exner):
        """exner - exner_ref: the extrapolation history at a cold start.
        Row A5, a reading."""
        return exner - self.v.exner_ref[None, :]

    def reference_state(self):
        """Row A0: the reference profiles (theta_ref, exner_ref), a reading."""
        return self.v.theta_ref.copy(), self.v.exner_ref.copy()


def thomas(a, b, c, r):
    """Solve a_k x_{k-1} + b_k x_k + c_k x_{k+1} = r_k (k = 0..n-1, a_0 and c_{n-1}
    unused) per row, forward elimination then back-substitution, no pivoting.
    Row A7: the tridiagonal solve of the vertically implicit scheme (Sec. 4.1), Thomas algorithm."""
    n = b.shape[1]
    cp = np.zeros_like(b)
    rp = np.zeros_like(b)
    cp[:, 0] = c[:, 0] / b[:, 0]
    rp[:, 0] = r[:, 0] / b[:, 0]
    for k in range(1, n):
        m = b[:, k] - a[:, k] * cp[:, k - 1]
        cp[:, k] = c[:, k] / m
        rp[:, k] = (r[:, k] - a[:, k] * rp[:, k - 1]) / m
    x = np.zeros_like(b)
    x[:, n - 1] = rp[:, n - 1]
    for k in range(n - 2, -1, -1):
        x[:, k] = rp[:, k] - cp[:, k] * x[:, k + 1]
    return x
