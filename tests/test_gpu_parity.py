"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Bars (relative L2 over a whole field, on alpha_g, u_g, u_l, p_k): 1e-12 for
FP64, 1e-5 for FP32, 1e-3 for FP16-stored deviations.  Sizes span several
tiles with ragged tails; cases cover all three lattices, walls, periodic axes,
the inlet strip (Table 1), the outlet (Table 2), both drag models, the lag
latch and the Spalding modes, plus edge cases (zero steps, odd step counts,
one-node-wide periodic axes).
"""
import zlib

import numpy as np
import pytest

import lbm_inputs
import oracle
import paper_2409_10399_gb300 as lbm
from oracle import params as oparams
from paper_2409_10399_gb300 import params as lparams

pytestmark = pytest.mark.gpu

PER, WALL, INLET, OUTLET = 0, 1, 2, 3
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16dev": 1e-3, "fp64dev": 1e-9, "fp16ab": 1e-3}
S_ATOL = {"fp64": 1e-14, "fp32": 1e-8, "fp16dev": 1e-5, "fp64dev": 1e-14, "fp16ab": 1e-5}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a)


def run_pair(lat, dims, p, fields, steps, prec, threads=8):
    D = lbm.LATTICE[lat]
    dims3 = tuple(dims) + (1,) * (3 - len(dims))
    o = oracle.Oracle(lat, dims3, p, threads=threads)
    o.init(**fields)
    o.step(steps)
    ref = o.moments()
    pg = dict(p)
    pg["precision"] = prec
    s = lbm.Simulation(lat, dims3, pg)
    s.init(**fields)
    s.step(steps)
    got = s.moments()
    return got, ref, s, o


def u_l_scale(ref, R):
    """Denominator of the liquid velocity's relative error: max(|u_l|, |u_g|/R)
    over the reference field.  The liquid's momentum receives the interphase
    force divided by R (Eq. (Gl), drag term of Eq. (interphasemomentum)), so a
    liquid brought nearly to rest (RMS 1e-9 in the test states, where the gas
    moves at 1e-4) carries, relative to the gas, the gas velocity's error
    scaled by 1/R; below |u_g|/R the liquid's own norm would measure rounding
    against a field the coupling does not resolve.  Wherever |u_l| >= |u_g|/R
    this is the plain per-phase relative error."""
    return max(np.linalg.norm(ref["u_l"]), np.linalg.norm(ref["u_g"]) / R)


def u_l_error(got, ref, R):
    return np.linalg.norm(np.asarray(got["u_l"]) - ref["u_l"]) / u_l_scale(ref, R)


def assert_parity(got, ref, prec, ctx="", R=1000.0, u_l=True):
    """Relative L2 per field: alpha_g, u_g, u_l (denominator u_l_scale) and
    p_k; S_g, S_l on the scale of max |S|.  u_l=False leaves the liquid
    velocity to a test of its own (the all-half store, see
    test_fp16dev_liquid_velocity)."""
    tol = TOL[prec]
    for k in ("alpha_g", "p_k", "u_g"):
        e = rel(got[k], ref[k])
        assert e <= tol, "%s %s rel L2 %.3e > %.1e" % (ctx, k, e, tol)
    if u_l:
        e = u_l_error(got, ref, R)
        assert e <= tol, "%s u_l rel L2 %.3e > %.1e (|u_l| %.2e, |u_g|/R %.2e)" % (
            ctx, e, tol, np.linalg.norm(ref["u_l"]), np.linalg.norm(ref["u_g"]) / R)
    # S = 1 - beta is a small difference: compare on the scale of max |S|
    for k in ("S_g", "S_l"):
        e = np.abs(got[k] - ref[k]).max()
        assert e <= max(S_ATOL[prec], tol * np.abs(ref[k]).max()), "%s %s max abs %.3e" % (ctx, k, e)


BASE = dict(R=1000.0, omega_g=0.6, omega_l=120.0 / 67.0, omega_alpha=1.5, drag_model=1, kappa_I=2.4e-4,
            kappa_W=0.0, g_hat=1e-6 / 999.0, gamma=1.0, n_gamma=7, spalding_mode=2, alpha_floor=1e-8)

CASES = {
    # 2D box, periodic x, walls y (ragged in both axes vs the 64x4 tile)
    "d2q9_walls": ("D2Q9", (70, 37), dict(BASE, g_axis=1, bc_lo=(PER, WALL, 0), bc_hi=(PER, WALL, 0)), 300),
    # 2D box with the bottom inlet strip of Table 1 and zero net volume flux
    "d2q9_strip": ("D2Q9", (72, 45), dict(BASE, g_axis=1, bc_lo=(PER, INLET, 0), bc_hi=(PER, WALL, 0),
                                          inlet_lo=20, inlet_hi=52, in_alpha=(0.01, 0.3), in_ug=(4.3e-4, 4.3e-3),
                                          ramp_nt=60, inlet_ul_mode=1), 250),
    # 2D with an outlet (Table 2) on the top face, walls on x, CONST drag, Spalding 1
    "d2q9_outlet": ("D2Q9", (33, 30), dict(BASE, R=20.0, drag_model=0, kappa_I=1e-2, kappa_W=2e-3, g_axis=1,
                                           g_hat=1e-5, spalding_mode=1, n_gamma=1,
                                           bc_lo=(WALL, WALL, 0), bc_hi=(WALL, OUTLET, 0)), 200),
    # 2D, gravity along x, inlet on x low face, strip in y, walls in y
    "d2q9_xinlet": ("D2Q9", (41, 22), dict(BASE, R=50.0, g_axis=0, g_hat=2e-6, bc_lo=(INLET, WALL, 0),
                                           bc_hi=(OUTLET, WALL, 0), inlet_lo=5, inlet_hi=17, in_alpha=(0.05, 0.4),
                                           in_ug=(1e-3, 4e-3), in_ul=(0.0, 5e-4), ramp_nt=30), 150),
    # 3D, walls on four sides, periodic z
    "d3q19_walls": ("D3Q19", (20, 18, 13), dict(BASE, g_axis=2, bc_lo=(WALL, WALL, PER), bc_hi=(WALL, WALL, PER)),
                    80),
    # 3D with an inlet strip on the bottom z face (tile shift along z)
    "d3q19_strip": ("D3Q19", (12, 10, 11), dict(BASE, g_axis=2, bc_lo=(PER, WALL, INLET), bc_hi=(PER, WALL, WALL),
                                                inlet_lo=3, inlet_hi=9, in_alpha=(0.02, 0.3), in_ug=(1e-3, 4e-3),
                                                ramp_nt=20, inlet_ul_mode=1), 60),
    # 1D column with wall friction, psi != 0 (1D stress form)
    "d1q3_walls": ("D1Q3", (300,), dict(BASE, kappa_W=2.4e-4, psi_g=0.2, psi_l=0.1, g_axis=0,
                                        bc_lo=(WALL, 0, 0), bc_hi=(WALL, 0, 0)), 500),
    # 1D open tube of Sec. 3.6 (Table 1 inlet, Table 2 outlet), ragged vs the 128 tile
    "d1q3_tube": ("D1Q3", (201,), dict(R=2.0, omega_g=0.6, omega_l=0.6, omega_alpha=1.9, drag_model=0,
                                       kappa_I=1e-2, kappa_W=1e-2, g_hat=1e-6, g_axis=0, n_gamma=1,
                                       bc_lo=(INLET, 0, 0), bc_hi=(OUTLET, 0, 0), in_alpha=(0.01, 0.8),
                                       in_ug=(1e-3, 1e-2), in_ul=(0.0, 1e-3), ramp_nt=200), 700),
}


def case_fields(lat, dims, seed):
    D = lbm.LATTICE[lat]
    return lbm_inputs.fields_random(D, dims, seed=seed, alpha=(0.05, 0.6), u_amp=2e-3, pk_amp=1e-5)


# Rounding differences grow with run length in these random-field states (a
# one-ulp perturbation of alpha moves the oracle's u by ~1e-10 after 1000
# steps), so FP32 runs are capped at 200 steps; the workload-length FP32 and
# FP16 errors are measured against the bitwise FP64 path instead.
FP32_STEPS = 200


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parity_cases(name, prec):
    lat, dims, p, steps = CASES[name]
    if prec == "fp32":
        steps = min(steps, FP32_STEPS)
    f = case_fields(lat, dims, seed=zlib.crc32(name.encode()) % 997)
    got, ref, _, _ = run_pair(lat, dims, p, f, steps, prec)
    assert_parity(got, ref, prec, name, R=p["R"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_reference_is_bitwise(name):
    """The FP64 path evaluates the paper's formulas in the order written, with
    no contraction, like the oracle: every field agrees exactly."""
    lat, dims, p, steps = CASES[name]
    f = case_fields(lat, dims, seed=zlib.crc32(name.encode()) % 997)
    got, ref, s, o = run_pair(lat, dims, p, f, steps, "fp64")
    for k in ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l"):
        assert np.array_equal(got[k], ref[k]), (name, k, np.abs(got[k] - ref[k]).max())
    for sch in range(6):
        assert np.array_equal(s.populations(sch), o.pops(sch)), (name, sch)


@pytest.mark.parametrize("name", sorted(CASES))
def test_parity_fp64dev(name):
    """The fast kernels' deviation arithmetic, in double.  Bar 1e-9: the
    oracle's own fields move by up to 1.6e-10 (relative L2 on u) when its
    input is perturbed by one ulp over these run lengths, so two FP64
    evaluations that round differently cannot agree better than that."""
    lat, dims, p, steps = CASES[name]
    f = case_fields(lat, dims, seed=zlib.crc32(name.encode()) % 997)
    got, ref, _, _ = run_pair(lat, dims, p, f, steps, "fp64dev")
    assert_parity(got, ref, "fp64dev", name, R=p["R"])


def _fp16_case(name, prec):
    lat, dims, p, steps = CASES[name]
    D = lbm.LATTICE[lat]
    d3 = tuple(dims) + (1,) * (3 - len(dims))
    f = lbm_inputs.fields_column3d(d3[0], d3[1], d3[2], seed=5, corr=2.0)
    f = dict(alpha_g=f["alpha_g"], p_k=f["p_k"], u_g=f["u_g"][:D], u_l=f["u_l"][:D])
    got, ref, _, _ = run_pair(lat, dims, p, f, min(steps, 100), prec)
    return got, ref, p


@pytest.mark.parametrize("name", ["d2q9_walls", "d3q19_walls", "d2q9_strip"])
def test_parity_fp16dev(name):
    """FP16 deviations on states of the 3D-column recipe (alpha = 0.05 +- 0.01,
    smooth; at rest), the regime the half store is meant for: alpha_g, u_g,
    p_k at the half store's bar."""
    got, ref, p = _fp16_case(name, "fp16dev")
    assert_parity(got, ref, "fp16dev", name, R=p["R"], u_l=False)


@pytest.mark.parametrize("name", ["d2q9_walls", "d3q19_walls"])
@pytest.mark.xfail(strict=True, reason="the all-half store keeps 11 significant bits of every f_l population, "
                                       "whose first moment is u_l: it resolves the liquid velocity to ~1e-3 of "
                                       "max(|u_l|, |u_g|/R) per step, not after 100 steps (FP16AB carries f_l "
                                       "in float and meets the bar, test_fp16ab_liquid_velocity)")
def test_fp16dev_liquid_velocity(name):
    got, ref, p = _fp16_case(name, "fp16dev")
    assert u_l_error(got, ref, p["R"]) <= TOL["fp16dev"]


@pytest.mark.parametrize("name", ["d2q9_walls", "d3q19_walls", "d2q9_strip"])
def test_fp16ab_liquid_velocity(name):
    """The same states with f_g, f_l in float and the alpha and beta schemes in
    half: every field, u_l included, at the half store's bar."""
    got, ref, p = _fp16_case(name, "fp16ab")
    assert_parity(got, ref, "fp16ab", name, R=p["R"])


@pytest.mark.parametrize("name", sorted(CASES))
def test_parity_fp16ab(name):
    """f_g, f_l in float and the alpha and beta schemes in half, on the random
    states of the FP32 cases (alpha 0.05..0.6), at the half store's bar."""
    lat, dims, p, steps = CASES[name]
    f = case_fields(lat, dims, seed=zlib.crc32(name.encode()) % 997)
    got, ref, _, _ = run_pair(lat, dims, p, f, min(steps, 100), "fp16ab")
    assert_parity(got, ref, "fp16ab", name, R=p["R"])


@pytest.mark.parametrize("steps", [0, 1, 2, 3])
def test_populations_and_parity_of_steps(steps):
    """Every population of every scheme after 0..3 steps (both AA parities)."""
    lat, dims, p, _ = CASES["d2q9_strip"]
    f = case_fields(lat, dims, seed=3)
    got, ref, s, o = run_pair(lat, dims, p, f, steps, "fp64")
    for sch in range(6):
        assert np.array_equal(s.populations(sch), o.pops(sch)), sch
    assert s.t == steps


def test_diagnostics_match_oracle():
    lat, dims, p, steps = CASES["d3q19_walls"]
    f = case_fields(lat, dims, seed=9)
    got, ref, s, o = run_pair(lat, dims, p, f, 31, "fp64")
    a, b = s.diag(), o.diag()
    for k in (0, 1, 2, 4):
        assert a[k] == pytest.approx(b[k], rel=1e-12)
    assert a[3] == pytest.approx(b[3], rel=1e-6, abs=1e-20)
    assert a[5] == b[5] == 0
    assert a[6] == pytest.approx(b[6], rel=1e-9, abs=1e-12)


def test_single_node_periodic_axis():
    p = dict(BASE, g_axis=0, bc_lo=(WALL, PER, 0), bc_hi=(WALL, PER, 0))
    f = case_fields("D2Q9", (40, 1), seed=2)
    got, ref, _, _ = run_pair("D2Q9", (40, 1), p, f, 50, "fp64")
    assert_parity(got, ref, "fp64", "ny=1")


def test_column1d_full_config_fp64():
    """The 1D column workload at full size: N = 512, 10,000 steps, FP64."""
    w = lbm_inputs.WORKLOADS["column1d"]
    f = lbm_inputs.fields_for("column1d")
    po = oparams.lattice_params(w["physics"])
    pl = lparams.lattice_params(w["physics"])
    o = oracle.Oracle("D1Q3", w["dims"], po)
    o.init(**f)
    o.step(w["steps"])
    ref = o.moments()
    s = lbm.Simulation("D1Q3", w["dims"], dict(pl, precision="fp64"))
    s.init(**f)
    s.step(w["steps"])
    assert_parity(s.moments(), ref, "fp64", "column1d")


def test_box2d_full_size_first_steps_fp32():
    """The 2D box at its full 512 x 2048 size and in the benchmark's launch
    configuration, a few steps against the oracle (multi-threaded)."""
    w = lbm_inputs.WORKLOADS["box2d"]
    f = lbm_inputs.fields_for("box2d")
    po = oparams.lattice_params(w["physics"])
    pl = lparams.lattice_params(w["physics"], precision="fp32")
    o = oracle.Oracle("D2Q9", w["dims"], po, threads=16)
    o.init(**f)
    o.step(5)
    s = lbm.Simulation("D2Q9", w["dims"], pl)
    s.init(**f)
    s.step(5)
    assert_parity(s.moments(), o.moments(), "fp32", "box2d full")


def test_column3d_full_size_against_fp64():
    """The 3D column at its full 256 x 256 x 512 size, in the launch
    configuration of its throughput study, against the FP64 reference path
    at the same size (bitwise equal to the oracle on the parity cases above;
    the oracle itself would need ~60 GB of host memory here): after 20 steps
    every form stays finite, alpha_g of the FP32 store agrees with FP64
    within the FP32 bar and that of the FP16 stores (every scheme half, and
    f_g, f_l float with f_alpha, f_beta half) within the FP16 bar, and so do
    their FP64 sums of the raw gas fraction a_g (with the workload's Spalding
    mode 2 that sum is not an exact invariant, Eq. (spalding2), but every
    form must move it alike).  The velocities are not compared here: 20 steps
    from rest leave them at ~1e-9, below what the FP16 stores resolve; the
    velocity bars hold at the workload's 5,000 steps (64 x 64 x 128,
    test_gpu_workloads) and on the parity cases above."""
    w = lbm_inputs.WORKLOADS["column3d"]
    f = lbm_inputs.fields_for("column3d")
    out, sums = {}, {}
    for prec in ("fp64", "fp32", "fp16dev", "fp16ab"):
        s = lbm.Simulation("D3Q19", w["dims"], lparams.lattice_params(w["physics"], precision=prec))
        s.init(**f)
        s.step(20)
        m = s.moments()
        d = s.diag()
        s.close()
        for k in ("alpha_g", "u_g", "u_l", "p_k"):
            assert np.isfinite(m[k]).all(), (prec, k)
        assert d[5] == 0
        sums[prec] = d[0]
        out[prec] = m["alpha_g"]
    for prec, tol in (("fp32", TOL["fp32"]), ("fp16dev", TOL["fp16dev"]), ("fp16ab", TOL["fp16ab"])):
        assert rel(out[prec], out["fp64"]) <= tol, (prec, rel(out[prec], out["fp64"]))
        assert abs(sums[prec] - sums["fp64"]) <= (1e-7 if prec == "fp32" else 1e-6) * sums["fp64"], (prec, sums)


def test_errors_are_reported():
    with pytest.raises(lbm.LBMError):
        lbm.Simulation("D2Q9", (8, 8), dict(BASE, omega_g=2.5))
    with pytest.raises(lbm.LBMError):  # inlet only on the low face of g_axis
        lbm.Simulation("D2Q9", (8, 8), dict(BASE, g_axis=1, bc_lo=(PER, WALL, 0), bc_hi=(PER, INLET, 0)))
    s = lbm.Simulation("D2Q9", (8, 8), BASE)
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == -7


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_results_independent_of_tile(prec):
    """The fused step gives identical fields for every legal tile (each node's
    arithmetic does not depend on the launch shape)."""
    lat, dims, p, _ = CASES["d2q9_strip"]
    f = case_fields(lat, dims, seed=4)
    outs = []
    for tile in [(64, 2, 1), (32, 4, 1), (16, 8, 1), (32, 2, 1)]:
        s = lbm.Simulation(lat, dims, dict(p, precision=prec))
        s.set_tile(*tile)
        assert s.tile == tile
        s.init(**f)
        s.step(41)
        outs.append(s.moments())
    for o in outs[1:]:
        for k in outs[0]:
            assert np.array_equal(o[k], outs[0][k]), k
    s = lbm.Simulation(lat, dims, dict(p, precision=prec))
    with pytest.raises(lbm.LBMError):
        s.set_tile(64, 1, 1)  # inlet face on y needs a tile of >= 2 along y
    with pytest.raises(lbm.LBMError):
        s.set_tile(48, 3, 1)  # not a multiple of 32 threads
    if prec == "fp32":
        with pytest.raises(lbm.LBMError):
            s.set_tile(64, 4, 1)  # the 2D float kernel is built for at most 128 threads


@pytest.mark.parametrize("name,prec,extra", [
    ("d2q9_walls", "fp32", dict(diag_every=20)),
    ("d2q9_walls", "fp16dev", dict(diag_every=0)),
    ("d3q19_walls", "fp32", dict(diag_every=6)),
    ("d1q3_walls", "fp64", dict(diag_every=35)),
    ("d2q9_walls", "fp32", dict(beta_stencil=1, diag_every=0)),
    ("d2q9_walls", "fp32", dict(diag_every=1)),
])
def test_graph_replay_is_bitwise_plain_launches(name, prec, extra):
    """lbm_step replays periods of lcm(2, n_gamma, diag_every) steps from a CUDA
    graph when the step arguments repeat (closed lattices): the fields are
    bitwise those of plain launches, over whole periods and ragged remainders,
    and the diagnostics agree.  A replayed period takes its diagnostics once,
    after its last step (diag_every = 1 gives 14 reductions per period
    launched one by one, one replayed), so the graph path launches fewer
    kernels when diagnostics are on and the same number when they are off."""
    lat, dims, p, _ = CASES[name]
    f = case_fields(lat, dims, seed=9)
    runs = []
    for graph in (True, False):
        s = lbm.Simulation(lat, dims, dict(p, precision=prec, **extra))
        s.set_graph(graph)
        s.init(**f)
        for n in (1, 3, 400, 29, 300):  # starts on and off period boundaries (periods 14..140)
            s.step(n)
        runs.append((s.moments(), s.diag(), s.launches, s.t))
    (mg, dg, lg, tg), (mp, dp, lp, tp) = runs
    assert tg == tp == 733
    assert lg == lp if extra.get("diag_every", 0) == 0 else lg < lp
    for k in mg:
        assert np.array_equal(mg[k], mp[k]), k
    assert np.array_equal(dg, dp)
