"""Scheme parameters of the oracle.

Values are ICON-like defaults (the paper gives none, Sec. 4.1):
implicit weight beta = 0.65, velocity-tendency weights 0.25/0.75 (now/new),
rho/theta time weights 0.6/0.4 in the corrector, exner extrapolation 1/3,
fourth-order divergence damping 0.0025, mass-flux divergence filter 0.07,
Smagorinsky factor 0.015,
fourth-order background diffusion A^2/288.
"""
from dataclasses import dataclass


@dataclass
class DycoreParams:
    """Parameters of the step (Sec. 4.1 names their roles, not their values; ICON-like readings)."""
    dtime: float = 1800.0
    ndyn_substeps: int = 5
    # physical constants (dry, shallow atmosphere)
    grav: float = 9.80665
    rd: float = 287.04
    cpd: float = 1004.64
    p00: float = 1.0e5
    omega: float = 7.29212e-5
    radius: float = 6.371229e6
    # solve_nonhydro
    vwind_impl_wgt: float = 0.65
    wgt_nnow_vel: float = 0.25
    wgt_nnew_vel: float = 0.75
    wgt_nnow_rth: float = 0.6
    wgt_nnew_rth: float = 0.4
    exner_exfac: float = 1.0 / 3.0
    divdamp_fac: float = 0.0025
    # divergence filter of the mass-flux velocity, vn + divflux_fac * Abar * grad_n(div vn)
    divflux_fac: float = 0.07
    # Rayleigh damping of w above damp_height (coefficient 0 switches it off)
    rayleigh_coeff: float = 0.0
    damp_height: float = 20000.0
    # diffusion
    hdiff_smag_fac: float = 0.015
    hdiff_k4: float = 1.0 / 288.0
    hdiff_w_k4: float = 1.0 / 288.0
    hdiff_temp: bool = True
    # reference state theta_ref(z) = T0 * exp(z / H), H = cpd * T0 / grav
    ref_T0: float = 250.0
    # steep terrain (terrain-following heights only): the horizontal pressure
    # gradient at constant height where the levels of the two cells of an edge
    # are offset by more than half a layer (steep_hpg), and enhanced
    # temperature diffusion where the lowest levels hold strong horizontal
    # temperature differences (factor 0 switches it off)
    steep_hpg: bool = False
    hdiff_tenh_fac: float = 0.0
    hdiff_tenh_thresh: float = 5.0
    hdiff_tenh_levels: int = 5

    @property
    def cvd(self):
        """Parameters of the step (Sec. 4.1 names their roles, not their values; ICON-like readings)."""
        return self.cpd - self.rd
