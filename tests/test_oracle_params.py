"""Pins of the oracle's parameter and closed-form helpers against numbers the
paper prints (tests/golden/paper_printed_values.txt, Sec. 3.6)."""
import math
import os

import pytest

from oracle import analytic, params

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")


def golden():
    out = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            out[k.strip()] = float(v)
    return out


def test_test4_similarity_numbers():
    g = golden()
    kap = params.kappa_cgw(0.66, 0.002)
    assert kap == pytest.approx(g["test4_kappa_I"], rel=1e-12)
    cot, ct, c = params.similarity(9.81, 1.2e-9, kap, 1.45e-4)
    assert cot == pytest.approx(g["test4_c_over_tau"], rel=5e-3)
    assert ct == pytest.approx(g["test4_c_tau"], rel=5e-3)
    assert c == pytest.approx(g["test4_c"], rel=5e-3)
    ugh = 0.3 / c
    assert ugh == pytest.approx(g["test4_ug_hat_max"], rel=2e-2)
    assert ugh / 4 == pytest.approx(g["test4_ul_hat_max"], rel=2e-2)
    # M_ex with the physical reference values; R = 1000/1.2
    R = 1000.0 / 1.2
    assert params.M_ex(kap, 0.1, 0.3, 0.3 / 4, R, 9.81) == pytest.approx(g["test4_M_ex"], rel=5e-3)
    # Eq. (Mex-hat): the lattice-unit value equals the physical one
    kh = params.kappa_hat_from_c(kap, c, 9.81, 1.2e-9)
    assert kh == pytest.approx(1.45e-4, rel=1e-12)
    assert params.M_ex(kh, 0.1, ugh, ugh / 4, R, 1.2e-9) == pytest.approx(params.M_ex(kap, 0.1, 0.3, 0.075, R, 9.81), rel=1e-12)


def test_test1_analytic_numbers():
    g = golden()
    ag, ug = g["test1_ag_out"], g["test1_ug_out"]
    u0 = analytic.ug0(1e-2, ag, 2.0, 1e-6)
    assert u0 == pytest.approx(g["test1_ug0"], rel=1e-12)
    r = (1e-2 / 1e-2) * ag
    assert analytic.ul_from_ug(ug, u0, r) == pytest.approx(g["test1_ul_analytic"], rel=1e-12)
    assert analytic.ul_approx_r1(ug, u0) == pytest.approx(g["test1_ul_approx"], rel=1e-12)
    assert ag * ug + (1 - ag) * g["test1_ul_out"] == pytest.approx(g["test1_mixture_flux_out"], rel=1e-12)
    # inlet u_g^min of Eq. (analytical0bis) ~ 9.95e-4
    assert analytic.ug0(1e-2, g["test1_alpha_min"], 2.0, 1e-6) == pytest.approx(9.95e-4, rel=1e-3)


def test_analytic_limits():
    """Sec. 3.1: r = 0 gives u_l = u_g - u_g0; r -> 1 gives the printed limit."""
    ug, u0 = 8e-3, 2e-3
    assert analytic.ul_from_ug(ug, u0, 0.0) == pytest.approx(ug - u0, rel=1e-12)
    assert analytic.ul_from_ug(ug, u0, 1.0 - 1e-9) == pytest.approx(analytic.ul_approx_r1(ug, u0), rel=1e-6)
    # the solution satisfies Eq. (analytical3): r u_l^2 = (u_g - u_l)^2 - u_g0^2
    for r in (0.1, 0.5, 0.9):
        ul = analytic.ul_from_ug(ug, u0, r)
        assert r * ul * ul == pytest.approx((ug - ul) ** 2 - u0 ** 2, rel=1e-10)


def test_workload_parameters():
    """omega_l from the viscosity ratio (Eq. (effective-viscosity)) and kappa_hat
    for d = 1 mm at c = 69.2 (Eqs. (scaling-grav-acceleration), (scaling-kappaI))."""
    import lbm_inputs
    p = params.lattice_params(lbm_inputs.WORKLOADS["box2d"]["physics"])
    assert params.nu_from_omega(p["omega_g"]) / params.nu_from_omega(p["omega_l"]) == pytest.approx(20.0, rel=1e-12)
    assert p["omega_l"] == pytest.approx(120.0 / 67.0, rel=1e-14)
    assert p["kappa_I"] == pytest.approx(2.42e-4, rel=2e-3)
    assert p["kappa_W"] == 0.0
    p1 = params.lattice_params(lbm_inputs.WORKLOADS["column1d"]["physics"])
    assert p1["kappa_W"] == p1["kappa_I"]
