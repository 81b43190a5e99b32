"""Batched form: many independent lattices in one launch per step.

Instance i of a batch must equal a single-lattice run with the same sizes,
parameters and fields: the per-node arithmetic is the same source compiled
into a second kernel, where the compiler may fuse multiply-adds differently,
so the bar is the FP32 parity bar applied node by node (max difference <= 1e-5
of the field's scale after 31 steps; one-step differences are ~5e-8), with and without CUDA-graph
replay and for step counts that are not multiples of the graph period.  Within
the batched kernel the result is bitwise independent of the tile and of graph
replay.  Every instance of a ragged batch spanning R = 10..1000 is also
checked against the oracle."""
import numpy as np
import pytest

import lbm_inputs
import oracle
import paper_2409_10399_gb300 as lbm

pytestmark = pytest.mark.gpu

PER, WALL, INLET = 0, 1, 2


def _cases(prec="fp32"):
    out = []
    for i, (nx, ny, R, kap) in enumerate([(70, 37, 1000.0, 2.4e-4), (33, 60, 50.0, 1e-3), (128, 20, 10.0, 5e-3),
                                          (64, 64, 300.0, 1e-4), (9, 11, 1000.0, 2.4e-4)]):
        p = dict(R=R, omega_g=0.6, omega_l=120.0 / 67.0, omega_alpha=1.5, drag_model=1, kappa_I=kap,
                 g_hat=1e-6 / (R - 1.0), g_axis=1, gamma=1.0, n_gamma=7, spalding_mode=2, precision=prec,
                 bc_lo=(PER, WALL, 0), bc_hi=(PER, WALL, 0))
        f = lbm_inputs.fields_random(2, (nx, ny), seed=30 + i, alpha=(0.05, 0.6), u_amp=2e-3, pk_amp=1e-5)
        out.append(((nx, ny), p, f))
    return out


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("steps", [1, 31])
def test_batch_instances_equal_single_runs(graph, steps):
    cases = _cases()
    b = lbm.Batch("D2Q9", [c[0] for c in cases], [c[1] for c in cases])
    b.set_graph(graph)
    for i, c in enumerate(cases):
        b.init(i, **c[2])
    b.step(steps)
    assert b.t == steps
    for i, (dims, p, f) in enumerate(cases):
        s = lbm.Simulation("D2Q9", dims, p)
        s.init(**f)
        s.step(steps)
        got, ref = b.moments(i), s.moments()
        for k in ("alpha_g", "u_g", "u_l", "p_k"):
            scale = np.abs(ref[k] - (1 / 3 if k == "p_k" else 0)).max()
            assert np.abs(got[k] - ref[k]).max() <= 1e-5 * scale, (i, k, np.abs(got[k] - ref[k]).max(), scale)


def test_batch_tile_independent_and_graph_replays():
    cases = _cases()
    ref = None
    for tile in [(64, 2, 1), (32, 4, 1), (128, 1, 1)]:
        b = lbm.Batch("D2Q9", [c[0] for c in cases], [c[1] for c in cases])
        b.set_tile(*tile)
        assert b.tile == tile
        for i, c in enumerate(cases):
            b.init(i, **c[2])
        b.step(14)   # one graph period (lcm(2, n_gamma = 7))
        b.step(30)   # two replays and two direct launches
        m = [b.moments(i) for i in range(len(cases))]
        if ref is None:
            ref = m
        else:
            for a, r in zip(m, ref):
                for k in r:
                    assert np.array_equal(a[k], r[k])


def test_batch_instances_against_oracle():
    """Every instance of one ragged batch (sizes 9 x 11 to 128 x 20, R from 10
    to 1000, drag coefficients 1e-4 to 5e-3) against its own FP64 oracle run,
    per field at the FP32 bar (u_l on the scale of test_gpu_parity.u_l_scale)."""
    from test_gpu_parity import assert_parity
    cases = _cases()
    b = lbm.Batch("D2Q9", [d for d, _, _ in cases], [p for _, p, _ in cases])
    for i, (_, _, f) in enumerate(cases):
        b.init(i, **f)
    b.step(120)
    for i, (dims, p, f) in enumerate(cases):
        o = oracle.Oracle("D2Q9", dims + (1,), p, threads=8)
        o.init(**f)
        o.step(120)
        assert_parity(b.moments(i), o.moments(), "fp32", "batch instance %d" % i, R=p["R"])


def test_batch_rejects_inconsistent_instances():
    (d0, p0, _), (d1, p1, _) = _cases()[:2]
    with pytest.raises(lbm.LBMError):
        lbm.Batch("D2Q9", [d0, d1], [p0, dict(p1, n_gamma=3)])
    with pytest.raises(lbm.LBMError):
        lbm.Batch("D2Q9", [d0], [dict(p0, precision="fp64")])
    with pytest.raises(lbm.LBMError):
        lbm.Batch("D2Q9", [d0], [dict(p0, bc_lo=(PER, INLET, 0), inlet_lo=2, inlet_hi=6)])
