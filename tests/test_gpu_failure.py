"""Failure detection of lbm_step, driven from the host (no GPU fault).

With diag_every > 0 the step enqueues the FP64 diagnostics every that many
steps and checks, without blocking, the last ones it received:
- a non-finite population anywhere -> LBM_ENAN (-4);
- in a closed domain, sum(a_g) drifting by more than drift_limit relative to
  its initial value -> LBM_EDRIFT (-5);
both sticky: every later lbm_step returns LBM_ESTATE (-7) until lbm_init.
The non-finite state is planted in the initial fields (a NaN velocity at one
node), the drift by a limit below the rounding of the FP32 store.
"""
import numpy as np
import pytest

import lbm_inputs
import paper_2409_10399_gb300 as lbm

pytestmark = pytest.mark.gpu

PER, WALL = 0, 1
BASE = dict(R=1000.0, omega_g=0.6, omega_l=120.0 / 67.0, omega_alpha=1.5, drag_model=1, kappa_I=2.4e-4,
            g_hat=1e-6 / 999.0, g_axis=1, gamma=1.0, n_gamma=7, bc_lo=(PER, WALL, 0), bc_hi=(PER, WALL, 0),
            precision="fp32")
DIMS = (40, 30, 1)


def _fields(seed=5):
    return lbm_inputs.fields_random(2, DIMS[:2], seed=seed, alpha=(0.05, 0.6), u_amp=2e-3, pk_amp=1e-5)


def _step_until_error(s, max_calls=100):
    import torch
    for _ in range(max_calls):
        try:
            s.step(1)
        except lbm.LBMError as e:
            return e.code
        torch.cuda.synchronize()
    return None


@pytest.mark.parametrize("prec", ["fp32", "fp16dev", "fp64"])
def test_non_finite_state_is_reported_and_sticky(prec):
    f = _fields()
    f["u_g"][0, 17] = np.nan
    s = lbm.Simulation("D2Q9", DIMS, dict(BASE, precision=prec, diag_every=1))
    s.init(**f)
    assert _step_until_error(s) == -4
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == -7
    s.init(**_fields())          # a fresh init clears the sticky error
    s.step(20)
    assert np.isfinite(s.moments()["u_g"]).all()


def test_drift_beyond_limit_is_reported():
    s = lbm.Simulation("D2Q9", DIMS, dict(BASE, diag_every=1, drift_limit=1e-14))
    s.init(**_fields())
    assert _step_until_error(s) == -5
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == -7


def test_no_false_alarm_on_a_healthy_run():
    s = lbm.Simulation("D2Q9", DIMS, dict(BASE, diag_every=5, drift_limit=1e-3))
    s.init(**_fields())
    for _ in range(10):
        s.step(10)
    d = s.diag()
    assert d[5] == 0 and np.isfinite(d[:5]).all()


def test_non_finite_state_found_within_replayed_periods():
    """A state that turns non-finite only after many steps (a BGK lattice at
    omega = 1.99 started from velocities of 0.3, far above what the scheme
    can carry, which blows up), stepped a whole graph period per call
    (n_gamma = 7, diag_every = 7: period 14).  With graph replay the
    diagnostics are taken once per period, after its last step; both paths
    report LBM_ENAN, the replayed one at most one call after the one that
    launches every step, and the error is sticky."""
    import torch
    f = _fields(seed=6)
    r = np.random.default_rng(6)
    f["u_g"] = r.uniform(-0.3, 0.3, f["u_g"].shape)
    f["u_l"] = r.uniform(-0.3, 0.3, f["u_l"].shape)
    found = {}
    for graph in (False, True):
        s = lbm.Simulation("D2Q9", DIMS, dict(BASE, omega_g=1.99, omega_l=1.99, diag_every=7))
        s.set_graph(graph)
        s.init(**f)
        for call in range(300):
            try:
                s.step(14)
            except lbm.LBMError as e:
                assert e.code == -4, e
                found[graph] = call
                break
            torch.cuda.synchronize()
        else:
            pytest.fail("no LBM_ENAN in 300 periods (graph=%s)" % graph)
        with pytest.raises(lbm.LBMError) as e:
            s.step(14)
        assert e.value.code == -7
    assert found[False] >= 1  # the state was finite for the first period
    assert 0 <= found[True] - found[False] <= 1, found
