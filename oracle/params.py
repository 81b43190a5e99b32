"""Oracle-side parameter helper: physical inputs -> lattice parameters.

TEST INFRASTRUCTURE (see oracle/__init__.py).  Written independently of the
library's own helper; a CPU test checks that both agree.

Relations used:
  * nu = cs2 (1/omega - 1/2), Eq. (effective-viscosity)  -> omega_l from the
    viscosity ratio.
  * kappa_I = 3 C_d / (4 d), Clift-Grace-Weber, Sec. 3.3.
  * c/tau = g / g_hat, Eq. (scaling-grav-acceleration); c*tau = kappa_hat /
    kappa_I, Eq. (scaling-kappaI); c = sqrt((c/tau)(c tau)), Eq.
    (lattice-speed).  Given c, kappa_hat = kappa_I * c^2 * g_hat / g.
  * M_ex, Eq. (Mex), with Lambda of Eq. (Lambda).
"""
import math

CS2 = 1.0 / 3.0


def omega_from_nu(nu):
    return 1.0 / (nu / CS2 + 0.5)


def nu_from_omega(omega):
    return CS2 * (1.0 / omega - 0.5)


def kappa_cgw(C_d, d):
    return 3.0 * C_d / (4.0 * d)


def similarity(g, g_hat, kappa, kappa_hat):
    c_over_tau = g / g_hat
    c_tau = kappa_hat / kappa
    return c_over_tau, c_tau, math.sqrt(c_over_tau * c_tau)


def kappa_hat_from_c(kappa, c, g, g_hat):
    c_tau = c * c / (g / g_hat)
    return kappa * c_tau


def Lambda(alpha_g, R):
    a_l = 1.0 - alpha_g
    return alpha_g * a_l * (alpha_g + a_l * R)


def M_ex(kappa, alpha_g, u_g, u_l, R, g):
    return kappa * Lambda(alpha_g, R) * abs(u_g - u_l) ** 2 / alpha_g / ((R - 1.0) * g)


def lattice_params(physics):
    """Lattice-unit parameter dict from a workload's physics block."""
    ph = dict(physics)
    out = {k: v for k, v in ph.items() if k in (
        "R", "omega_g", "omega_alpha", "psi_g", "psi_l", "drag_model", "g_hat", "g_axis", "gamma",
        "n_gamma", "spalding_mode", "alpha_floor", "bc_lo", "bc_hi", "inlet_lo", "inlet_hi",
        "in_alpha", "in_ug", "in_ul", "ramp_nt", "inlet_ul_mode")}
    nu_g = nu_from_omega(ph["omega_g"])
    out["omega_l"] = omega_from_nu(nu_g / ph["nu_ratio_g_over_l"])
    kap = kappa_cgw(ph["C_d"], ph["d_m"])
    kh = kappa_hat_from_c(kap, ph["c_lattice"], ph["g_phys"], ph["g_hat"])
    out["kappa_I"] = kh
    out["kappa_W"] = kh if ph.get("wall_friction") else 0.0
    return out


def diffusive_scaling(base, eps):
    """Lattice parameters at mesh spacing eps = lambda/L under the diffusive
    scaling of Sec. 2.1.2 (time step tau/T = eps^2): the relaxation rates stay
    (lattice viscosities and the alpha diffusivity are the continuum ones),
    g_hat = eps^3 g and K_hat_I = eps K_I (so kappa_hat_I, kappa_hat_W scale
    with eps).  `base` holds the continuum values under the same keys
    (g_hat = g, kappa_I = K_I, kappa_W = K_W)."""
    p = dict(base)
    p["g_hat"] = base.get("g_hat", 0.0) * eps ** 3
    p["kappa_I"] = base.get("kappa_I", 0.0) * eps
    p["kappa_W"] = base.get("kappa_W", 0.0) * eps
    return p
