"""Closed-form steady states of the 1D model (TEST INFRASTRUCTURE).

Sec. 3.1: with all gradients zero except a constant kinematic-pressure
gradient, Eqs. (lbm-mom-g1Danalytical) and (lbm-mom-l1Danalytical) hold.
Eliminating the pressure gradient gives Eq. (analytical); its special case
u_l = 0 gives Eq. (analytical0) and, for u_l < u_g, Eq. (analyticalsolution).
In a periodic column the pressure gradient is zero as well, which fixes u_g and
u_l separately (used by the homogeneous steady-state pin).
"""
import math


def ug0(K_I, alpha_g, R, g):
    """Eq. (analytical0): gas velocity of the bubble-column state u_l = 0."""
    return math.sqrt(alpha_g * (1.0 - alpha_g) * (R - 1.0) * g / K_I)


def ul_from_ug(ug, ug0_, r):
    """Eq. (analyticalsolution) with r = (K_W/K_I) alpha_g; r = 1 uses its limit."""
    if abs(1.0 - r) < 1e-14:
        return (ug - ug0_) * (1.0 + ug0_ / ug) / 2.0
    return (ug - math.sqrt(ug * ug - (1.0 - r) * (ug * ug - ug0_ * ug0_))) / (1.0 - r)


def ul_approx_r1(ug, ug0_):
    """Limit r -> 1 of Eq. (analyticalsolution)."""
    return (ug - ug0_) * (1.0 + ug0_ / ug) / 2.0


def periodic_homogeneous(K_I, K_W, alpha_g, R, g):
    """Uniform periodic column: zero pressure gradient in both momentum
    balances of Sec. 3.1 gives K_I (u_g-u_l)^2 = (R-1) g alpha_g and
    K_W u_l^2 = K_I (u_g-u_l)^2, i.e. (u_g, u_l)."""
    dv = math.sqrt((R - 1.0) * g * alpha_g / K_I)
    ul = math.sqrt((R - 1.0) * g * alpha_g / K_W) if K_W > 0 else float("inf")
    return ul + dv, ul
