"""Pin the C oracle against the independent mpmath stepper (oracle/brute.py)
on tiny lattices: every population of every scheme after a few steps.

The two implementations differ in lattice construction, layout, loop order,
contraction code, streaming direction (push vs pull) and precision (FP64 vs
40 digits); cases cover all three lattices, walls, periodic axes, the inlet
strip of Table 1, the outlet of Table 2, both drag models, the D = 1 and
D >= 2 stress forms (psi != 0), the lag latch and every Spalding mode.
"""
import zlib

import numpy as np
import pytest

import lbm_inputs
import oracle
from oracle import brute

PER, WALL, INLET, OUTLET = 0, 1, 2, 3

CASES = {
    "d1q3_walls": dict(lat="D1Q3", dims=(5, 1, 1), p=dict(
        R=40.0, omega_g=0.7, omega_l=1.6, omega_alpha=1.4, psi_g=0.3, psi_l=-0.2, drag_model=1,
        kappa_I=2e-2, kappa_W=1e-2, g_hat=3e-4, g_axis=0, gamma=1.0, n_gamma=2, spalding_mode=2,
        bc_lo=(WALL, 0, 0), bc_hi=(WALL, 0, 0))),
    "d1q3_inout": dict(lat="D1Q3", dims=(5, 1, 1), p=dict(
        R=2.0, omega_g=0.6, omega_l=0.6, omega_alpha=1.7, drag_model=0, kappa_I=1e-2, kappa_W=1e-2,
        g_hat=1e-4, g_axis=0, n_gamma=1, spalding_mode=2, bc_lo=(INLET, 0, 0), bc_hi=(OUTLET, 0, 0),
        in_alpha=(0.01, 0.8), in_ug=(1e-3, 1e-2), in_ul=(0.0, 1e-3), ramp_nt=2, inlet_ul_mode=0)),
    "d2q9_strip": dict(lat="D2Q9", dims=(4, 3, 1), p=dict(
        R=100.0, omega_g=0.8, omega_l=1.5, omega_alpha=1.5, psi_g=0.2, psi_l=0.1, drag_model=1,
        kappa_I=5e-3, kappa_W=0.0, g_hat=1e-4, g_axis=1, gamma=0.7, n_gamma=2, spalding_mode=1,
        bc_lo=(PER, INLET, 0), bc_hi=(PER, WALL, 0), inlet_lo=1, inlet_hi=3,
        in_alpha=(0.05, 0.3), in_ug=(1e-3, 5e-3), ramp_nt=3, inlet_ul_mode=1)),
    "d2q9_outlet": dict(lat="D2Q9", dims=(3, 4, 1), p=dict(
        R=10.0, omega_g=1.1, omega_l=1.3, omega_alpha=1.2, drag_model=0, kappa_I=1e-2, kappa_W=3e-3,
        g_hat=1e-4, g_axis=1, n_gamma=1, spalding_mode=0, bc_lo=(WALL, WALL, 0), bc_hi=(WALL, OUTLET, 0))),
    "d3q19_mixed": dict(lat="D3Q19", dims=(3, 3, 3), p=dict(
        R=500.0, omega_g=0.6, omega_l=1.8, omega_alpha=1.5, drag_model=1, kappa_I=1e-3, kappa_W=0.0,
        g_hat=5e-6, g_axis=2, gamma=1.0, n_gamma=2, spalding_mode=2,
        bc_lo=(WALL, PER, WALL), bc_hi=(WALL, PER, WALL))),
}


def _fields(D, dims, seed):
    f = lbm_inputs.fields_random(D, dims[:D], seed=seed, alpha=(0.15, 0.85), u_amp=1e-2, pk_amp=1e-3)
    return f


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_matches_bruteforce(name):
    c = CASES[name]
    lat, dims = c["lat"], c["dims"]
    D = oracle.LATTICE_D[lat]
    p = dict(oracle.PARAM_DEFAULTS)
    p.update(c["p"])
    f = _fields(D, dims, seed=zlib.crc32(name.encode()) % 1000)
    o = oracle.Oracle(lat, dims, p)
    o.init(**f)
    b = brute.Brute(D, dims, p)
    b.init(f["alpha_g"], f["u_g"], f["u_l"], f["p_k"])
    v, _, _ = o.lattice_tables()
    for step in range(3):
        o.step(1)
        b.step(1)
        for s, name_s in enumerate(brute.SCHEMES):
            mine = o.pops(s)
            ref = b.pops(name_s)
            scale = max(abs(float(x)) for col in ref.values() for x in col)
            for q in range(o.Q):
                col = np.array([float(x) for x in ref[tuple(int(c) for c in v[q])]])
                err = np.abs(mine[q] - col).max()
                assert err <= 1e-14 * scale, (name, step, name_s, q, err)
