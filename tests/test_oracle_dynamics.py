"""Pins of the oracle's time step against properties the paper and the
mathematics fix (no GPU).

* Uniform equilibrium is a fixed point (no gradient, no force, no source).
* Homogeneous column (periodic, uniform alpha): the LBM moment of Eqs.
  (lbmg)/(lbml) gives u(t+1) = u(t) + G(t) exactly, and G reduces to buoyancy
  plus drag plus wall friction (Eqs. (Gg1D), (Gl1D)) up to O(G^2); the
  trajectory must follow an independently written forward-Euler recurrence,
  and the steady state must equal the closed form of Sec. 3.1 with zero
  pressure gradient.
* Conservation: BGK and bounce-back conserve sum(a_phi) exactly (Spalding
  modes 0/1), and sum(eps) changes by exactly sum(S'') per step (the forcing
  operator adds S'', Eq. (forcingoperator)).
* Mirror and transpose symmetry of the lattice.
* D2Q9 and D3Q19 runs invariant along the transverse axes reproduce the D1Q3
  run (App. A: D1Q3 is the projection of the higher lattices).
"""
import numpy as np
import pytest

import lbm_inputs
import oracle
from oracle import analytic

PER, WALL, INLET, OUTLET = 0, 1, 2, 3


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run(lat, dims, p, fields, n, threads=1):
    o = oracle.Oracle(lat, dims, p, threads=threads)
    o.init(**fields)
    o.step(n)
    return o


# ---------------------------------------------------------------- fixed point

@pytest.mark.parametrize("lat,dims,bc", [
    ("D1Q3", (7, 1, 1), (PER, PER, PER)),
    ("D2Q9", (6, 5, 1), (PER, PER, PER)),
    ("D3Q19", (4, 3, 5), (PER, PER, PER)),
])
def test_uniform_equilibrium_is_fixed_point(lat, dims, bc):
    D = oracle.LATTICE_D[lat]
    N = int(np.prod(dims))
    U = np.array([1.2e-3, -7e-4, 3e-4])[:D]
    # no wall friction: Eq. (wallmomentum1D) would decelerate a moving liquid
    p = dict(R=1000.0, omega_g=0.6, omega_l=1.79, omega_alpha=1.5, drag_model=1, kappa_I=2.4e-4,
             kappa_W=0.0, g_hat=0.0, gamma=1.0, n_gamma=3, bc_lo=bc, bc_hi=bc)
    f = dict(alpha_g=np.full(N, 0.3), u_g=np.tile(U[:, None], N), u_l=np.tile(U[:, None], N),
             p_k=np.full(N, 1.0 / 3.0))
    o = oracle.Oracle(lat, dims, p)
    o.init(**f)
    before = [o.pops(s) for s in range(6)]
    o.step(25)
    for s in range(6):  # fixed to rounding: a few ulps of O(1) values per step
        assert np.abs(o.pops(s) - before[s]).max() < 2e-14


def test_rest_state_with_walls_is_fixed_point():
    dims = (6, 5, 1)
    N = 30
    p = dict(R=5.0, omega_g=0.8, omega_l=1.2, drag_model=0, kappa_I=1e-2, bc_lo=(WALL, WALL, 0),
             bc_hi=(PER, WALL, 0))
    z = np.zeros((2, N))
    o = oracle.Oracle("D2Q9", dims, p)
    o.init(alpha_g=np.full(N, 0.4), u_g=z, u_l=z, p_k=np.full(N, 1 / 3))
    before = [o.pops(s) for s in range(6)]
    o.step(20)
    for s in range(6):
        assert np.abs(o.pops(s) - before[s]).max() < 2e-14


# ------------------------------------------------------- homogeneous column

def _euler(R, g, K_I, K_W, ag, n):
    """Forward Euler of the 0-D momentum balances of Sec. 3.1 (no gradients,
    periodic so no pressure gradient), unit time step."""
    al = 1.0 - ag
    ug = ul = 0.0
    out = []
    for _ in range(n):
        du = ul - ug
        dg = (R - 1.0) * g + K_I * abs(du) * du / ag
        dl = -K_I * abs(du) * du / (R * al) - K_W * abs(ul) * ul / (R * al)
        ug, ul = ug + dg, ul + dl
        out.append((ug, ul))
    return np.array(out)


@pytest.mark.parametrize("lat,dims,axis", [("D1Q3", (3, 1, 1), 0), ("D2Q9", (2, 3, 1), 1),
                                           ("D3Q19", (2, 2, 3), 2)])
@pytest.mark.parametrize("cgw", [False, True])
def test_homogeneous_trajectory_is_forward_euler(lat, dims, axis, cgw):
    D = oracle.LATTICE_D[lat]
    N = int(np.prod(dims))
    R, g, ag = 2.0, 1e-6, 0.3
    kap, kapW = (1e-2, 2e-2) if not cgw else (5e-3, 1e-2)
    lam = ag * (1 - ag) * (ag + (1 - ag) * R)
    K_I, K_W = (kap * lam, kapW * lam) if cgw else (kap, kapW)
    p = dict(R=R, omega_g=0.6, omega_l=0.9, omega_alpha=1.5, drag_model=1 if cgw else 0, kappa_I=kap,
             kappa_W=kapW, g_hat=g, g_axis=axis, gamma=0.0, n_gamma=1)
    z = np.zeros((D, N))
    o = oracle.Oracle(lat, dims, p)
    o.init(alpha_g=np.full(N, ag), u_g=z, u_l=z.copy(), p_k=np.full(N, 1 / 3))
    ref = _euler(R, g, K_I, K_W, ag, 3000)
    for k in (1, 10, 300, 3000):
        o.step(k - o.t)
        m = o.moments()
        ug, ul = m["u_g"][axis], m["u_l"][axis]
        assert np.ptp(ug) < 5e-15 and np.ptp(ul) < 5e-15
        # exact up to the O(G^2) stress/gradient coupling; u is a sum of O(1)
        # populations, so its absolute rounding floor is ~1e-16 per step
        assert abs(ug[0] - ref[k - 1, 0]) <= 1e-7 * abs(ref[k - 1, 0]) + 5e-15
        assert abs(ul[0] - ref[k - 1, 1]) <= 1e-7 * abs(ref[k - 1, 1]) + 5e-15
        others = [a for a in range(D) if a != axis]
        for a in others:
            assert np.abs(m["u_g"][a]).max() < 5e-15
        assert np.abs(m["alpha_g"] - ag).max() < 1e-13  # rounding over 3000 steps


@pytest.mark.parametrize("cgw", [False, True])
def test_homogeneous_steady_state_closed_form(cgw):
    R, g, ag = 2.0, 1e-6, 0.3
    kap, kapW = 1e-1, 2e-1  # stiff drag: > 40 e-folds of the slowest mode in 2e5 steps
    lam = ag * (1 - ag) * (ag + (1 - ag) * R)
    K_I, K_W = (kap * lam, kapW * lam) if cgw else (kap, kapW)
    p = dict(R=R, omega_g=0.6, omega_l=0.6, drag_model=1 if cgw else 0, kappa_I=kap, kappa_W=kapW,
             g_hat=g, g_axis=0, n_gamma=1)
    N = 2
    o = oracle.Oracle("D1Q3", (N, 1, 1), p)
    o.init(alpha_g=np.full(N, ag), u_g=np.zeros((1, N)), u_l=np.zeros((1, N)), p_k=np.full(N, 1 / 3))
    o.step(200000)
    m = o.moments()
    ug_ref, ul_ref = analytic.periodic_homogeneous(K_I, K_W, ag, R, g)
    assert abs(m["u_g"][0, 0] - ug_ref) < 1e-9 * ug_ref
    assert abs(m["u_l"][0, 0] - ul_ref) < 1e-9 * ul_ref


# ----------------------------------------------------------------- conservation

@pytest.mark.parametrize("lat,dims,bc_lo,bc_hi,axis", [
    ("D1Q3", (16, 1, 1), (WALL, 0, 0), (WALL, 0, 0), 0),
    ("D2Q9", (12, 10, 1), (PER, WALL, 0), (PER, WALL, 0), 1),
    ("D3Q19", (6, 5, 4), (WALL, WALL, PER), (WALL, WALL, PER), 2),
])
@pytest.mark.parametrize("mode", [0, 1])
def test_conservation(lat, dims, bc_lo, bc_hi, axis, mode):
    D = oracle.LATTICE_D[lat]
    p = dict(R=50.0, omega_g=0.7, omega_l=1.6, omega_alpha=1.4, drag_model=1, kappa_I=3e-3, kappa_W=1e-3,
             g_hat=2e-5, g_axis=axis, gamma=0.5, n_gamma=3, spalding_mode=mode, bc_lo=bc_lo, bc_hi=bc_hi)
    f = lbm_inputs.fields_random(D, dims, seed=21)
    o = oracle.Oracle(lat, dims, p)
    o.init(**f)
    a0 = o.diag()
    for _ in range(12):
        e_before = o.pops(0).sum(), o.pops(1).sum()
        o.step(1)
        h = o.held()
        e_after = o.pops(0).sum(), o.pops(1).sum()
        assert abs((e_after[0] - e_before[0]) - h["Spp_g"].sum()) < 1e-13 * o.N
        assert abs((e_after[1] - e_before[1]) - h["Spp_l"].sum()) < 1e-13 * o.N
    o.step(40)
    a1 = o.diag()
    assert abs(a1[0] - a0[0]) < 1e-13 * a0[0]
    assert abs(a1[1] - a0[1]) < 1e-13 * a0[1]
    assert a1[5] == 0


def test_spalding_sum_is_one():
    """alpha_g^B + alpha_l^B = 1 by construction (Eq. (spalding)); the raw sum
    stays close to 1 when the mixture flux is nearly divergence-free."""
    p = dict(R=10.0, omega_g=0.7, omega_l=1.2, drag_model=0, kappa_I=1e-2, g_hat=1e-5, g_axis=1,
             bc_lo=(PER, WALL, 0), bc_hi=(PER, WALL, 0), spalding_mode=2)
    o = run("D2Q9", (10, 12, 1), p, lbm_inputs.fields_random(2, (10, 12), seed=3, u_amp=1e-4), 200)
    m = o.moments()
    assert np.all((m["alpha_g"] >= 0) & (m["alpha_g"] <= 1))
    d = o.diag()
    assert d[3] / o.N < 1e-6


# -------------------------------------------------------------------- symmetry

def test_mirror_x_d2q9_with_inlet_strip():
    nx, ny = 10, 9
    p = dict(R=100.0, omega_g=0.6, omega_l=1.5, omega_alpha=1.5, drag_model=1, kappa_I=2e-3, g_hat=1e-5,
             g_axis=1, gamma=1.0, n_gamma=4, bc_lo=(PER, INLET, 0), bc_hi=(PER, WALL, 0), inlet_lo=3,
             inlet_hi=7, in_alpha=(0.05, 0.3), in_ug=(1e-3, 4e-3), ramp_nt=10, inlet_ul_mode=1)
    f = lbm_inputs.fields_random(2, (nx, ny), seed=8)
    idx = np.arange(nx * ny).reshape(ny, nx)
    mir = idx[:, ::-1].reshape(-1)
    fm = dict(alpha_g=f["alpha_g"][mir], p_k=f["p_k"][mir],
              u_g=np.stack([-f["u_g"][0][mir], f["u_g"][1][mir]]),
              u_l=np.stack([-f["u_l"][0][mir], f["u_l"][1][mir]]))
    a = run("D2Q9", (nx, ny, 1), p, f, 30).moments()
    b = run("D2Q9", (nx, ny, 1), p, fm, 30).moments()
    assert rel(b["alpha_g"], a["alpha_g"][mir]) < 1e-13
    assert rel(b["u_g"][0], -a["u_g"][0][mir]) < 1e-12
    assert rel(b["u_g"][1], a["u_g"][1][mir]) < 1e-12
    assert rel(b["u_l"][1], a["u_l"][1][mir]) < 1e-12
    assert rel(b["p_k"], a["p_k"][mir]) < 1e-14


def test_transpose_xy_d3q19():
    n, nz = 5, 4
    p = dict(R=30.0, omega_g=0.8, omega_l=1.4, omega_alpha=1.3, drag_model=1, kappa_I=2e-3, kappa_W=0.0,
             g_hat=1e-5, g_axis=2, gamma=1.0, n_gamma=2, bc_lo=(WALL, WALL, PER), bc_hi=(WALL, WALL, PER))
    f = lbm_inputs.fields_random(3, (n, n, nz), seed=9)
    idx = np.arange(n * n * nz).reshape(nz, n, n)
    tr = np.transpose(idx, (0, 2, 1)).reshape(-1)
    ft = dict(alpha_g=f["alpha_g"][tr], p_k=f["p_k"][tr],
              u_g=np.stack([f["u_g"][1][tr], f["u_g"][0][tr], f["u_g"][2][tr]]),
              u_l=np.stack([f["u_l"][1][tr], f["u_l"][0][tr], f["u_l"][2][tr]]))
    a = run("D3Q19", (n, n, nz), p, f, 15).moments()
    b = run("D3Q19", (n, n, nz), p, ft, 15).moments()
    assert rel(b["alpha_g"], a["alpha_g"][tr]) < 1e-13
    assert rel(b["u_g"][0], a["u_g"][1][tr]) < 1e-11
    assert rel(b["u_l"][2], a["u_l"][2][tr]) < 1e-11


# ------------------------------------------------------------------ projection

def _proj_case(bc):
    if bc == "walls":
        return dict(bc_lo=(WALL, PER, PER), bc_hi=(WALL, PER, PER))
    return dict(bc_lo=(INLET, PER, PER), bc_hi=(OUTLET, PER, PER), inlet_lo=0, inlet_hi=10 ** 6,
                in_alpha=(0.05, 0.6), in_ug=(1e-3, 6e-3), in_ul=(0.0, 1e-3), ramp_nt=20, inlet_ul_mode=0)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("bc", ["walls", "inout"])
def test_projection_onto_d1q3(lat, bc):
    nx = 12
    D = oracle.LATTICE_D[lat]
    dims = (nx, 3, 3 if D == 3 else 1)
    N = int(np.prod(dims))
    p = dict(R=200.0, omega_g=0.6, omega_l=1.7, omega_alpha=1.5, drag_model=1, kappa_I=1e-3, kappa_W=5e-4,
             g_hat=5e-6, g_axis=0, gamma=1.0, n_gamma=3, spalding_mode=2)
    p.update(_proj_case(bc))
    f1 = lbm_inputs.fields_random(1, (nx,), seed=4)
    rep = N // nx
    fD = dict(alpha_g=np.tile(f1["alpha_g"], rep), p_k=np.tile(f1["p_k"], rep),
              u_g=np.vstack([np.tile(f1["u_g"][0], rep)] + [np.zeros(N)] * (D - 1)),
              u_l=np.vstack([np.tile(f1["u_l"][0], rep)] + [np.zeros(N)] * (D - 1)))
    a = run("D1Q3", (nx, 1, 1), p, f1, 60).moments()
    b = run(lat, dims, p, fD, 60).moments()
    for k in ("alpha_g", "p_k"):
        assert rel(b[k].reshape(-1, nx), np.tile(a[k], (rep, 1))) < 1e-12, k
    # S = 1 - beta is a difference of O(1) sums: compare on the absolute scale
    for k in ("S_g", "S_l"):
        assert np.abs(b[k].reshape(-1, nx) - np.tile(a[k], (rep, 1))).max() < 1e-15, k
    for k in ("u_g", "u_l"):
        assert rel(b[k][0].reshape(-1, nx), np.tile(a[k][0], (rep, 1))) < 1e-12, k
        assert np.abs(b[k][1:]).max() < 1e-16


# ------------------------------------------------------------ rest state

@pytest.mark.parametrize("lat,dims", [("D1Q3", (16, 1, 1)), ("D2Q9", (8, 6, 1))])
def test_rest_state_with_alpha_wave(lat, dims):
    """At rest with uniform pressure eps_g != 1 (so phi != 1, Eq. (lbm-phi-l))
    the momentum populations are at equilibrium and, by Eq. (secondtensoreq),
    carry no stress: whatever alpha(x) does, both phases stay exactly at rest.
    With u = 0 and Spalding off, each f_alpha scheme is a plain linear BGK
    diffusion, reproduced here by an independent numpy recurrence."""
    D = oracle.LATTICE_D[lat]
    N = int(np.prod(dims))
    xs = np.arange(N) % dims[0]
    ys = (np.arange(N) // dims[0]) % dims[1]
    ag = 0.5 + 0.2 * np.sin(2 * np.pi * xs / dims[0]) + (0.1 * np.cos(2 * np.pi * ys / dims[1]) if D == 2 else 0)
    p = dict(R=2.0, omega_g=0.7, omega_l=1.3, omega_alpha=1.4, drag_model=1, kappa_I=1e-2, kappa_W=1e-2,
             g_hat=0.0, gamma=1.0, n_gamma=1, spalding_mode=0)
    z = np.zeros((D, N))
    o = oracle.Oracle(lat, dims, p)
    o.init(alpha_g=ag, u_g=z, u_l=z.copy(), p_k=np.full(N, 1 / 3 + 3e-3))
    g0, l0 = o.pops(0), o.pops(1)
    v, w, _ = o.lattice_tables()
    fa = w[:, None] * ag[None, :]
    shape = (dims[1], dims[0]) if D == 2 else (dims[0],)
    for _ in range(50):
        o.step(1)
        a = fa.sum(0)
        fa = fa + 1.4 * (w[:, None] * a[None, :] - fa)
        for q in range(o.Q):
            f2 = fa[q].reshape(shape)
            f2 = np.roll(f2, v[q][0], axis=-1)
            if D == 2:
                f2 = np.roll(f2, v[q][1], axis=0)
            fa[q] = f2.reshape(-1)
    m = o.moments()
    assert np.abs(m["u_g"]).max() < 1e-15 and np.abs(m["u_l"]).max() < 1e-15
    assert np.abs(o.pops(0) - g0).max() < 1e-15 and np.abs(o.pops(1) - l0).max() < 1e-15
    assert rel(o.pops(2).sum(0), fa.sum(0)) < 1e-13
