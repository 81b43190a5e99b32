"""Physical inputs -> lattice parameters (Sec. 3.3 similarity, Eq.
(effective-viscosity)), for building ``lbm_params`` dicts from a workload.

  nu = cs2 (1/omega - 1/2)                      Eq. (effective-viscosity)
  c/tau = g / g_hat, c tau = kappa_hat/kappa    Eqs. (scaling-grav-acceleration), (scaling-kappaI)
  kappa_I = 3 C_d / (4 d)                       Clift-Grace-Weber, Sec. 3.3
Given the lattice speed c, kappa_hat = kappa * c^2 / (g / g_hat).
"""

_CS2 = 1.0 / 3.0
_KEYS = ("R", "omega_g", "omega_alpha", "psi_g", "psi_l", "drag_model", "g_hat", "g_axis", "gamma", "n_gamma",
         "spalding_mode", "alpha_floor", "bc_lo", "bc_hi", "inlet_lo", "inlet_hi", "in_alpha", "in_ug", "in_ul",
         "ramp_nt", "inlet_ul_mode")


def omega_l_for_ratio(omega_g, nu_ratio_g_over_l):
    nu_l = _CS2 * (1.0 / omega_g - 0.5) / nu_ratio_g_over_l
    return 1.0 / (0.5 + nu_l / _CS2)


def kappa_hat(C_d, d, c, g, g_hat):
    kappa = 3.0 * C_d / (4.0 * d)
    return kappa * c * c * g_hat / g


def lattice_params(physics, precision=None, diag_every=0, drift_limit=0.0):
    out = {k: physics[k] for k in _KEYS if k in physics}
    out["omega_l"] = omega_l_for_ratio(physics["omega_g"], physics["nu_ratio_g_over_l"])
    kh = kappa_hat(physics["C_d"], physics["d_m"], physics["c_lattice"], physics["g_phys"], physics["g_hat"])
    out["kappa_I"] = kh
    out["kappa_W"] = kh if physics.get("wall_friction") else 0.0
    if precision is not None:
        out["precision"] = precision
    out["diag_every"] = diag_every
    out["drift_limit"] = drift_limit
    return out


def diffusive_scaling(base, eps):
    """Parameters at mesh spacing eps under the diffusive scaling of Sec.
    2.1.2 (tau/T = eps^2): relaxation rates unchanged, buoyancy eps^3, drag
    coefficients eps (the continuum values are given under the lattice keys)."""
    out = dict(base)
    for key, power in (("g_hat", 3), ("kappa_I", 1), ("kappa_W", 1)):
        out[key] = base.get(key, 0.0) * eps ** power
    return out
