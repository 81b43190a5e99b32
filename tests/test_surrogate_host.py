"""Host logic of the surrogate study (no GPU): the inlet recipe's seeded
inlets, the nominal inflow of a trajectory, the window volumes and the
calibration of the volume check's expected inflow.

The calibration takes the expected change of sum(alpha_g) per window as k
times the trajectory's nominal inflow, k the ratio of the LBM's total change
to the total nominal inflow; its floor is the 99th percentile of the LBM's
own deviation from that, relative to the gas volume (what the check
bounds)."""
import numpy as np
import torch

import lbm_inputs
from paper_2409_10399_gb300 import surrogate as S


def test_surrogate_inlet_is_seeded_and_in_range():
    base = lbm_inputs.WORKLOADS["surrogate2d_inlet"]["physics"]
    assert lbm_inputs.surrogate_inlet(7) == lbm_inputs.surrogate_inlet(7)
    seen = set()
    for seed in range(200):
        ph = lbm_inputs.surrogate_inlet(seed)
        lo, hi = ph["inlet_lo"], ph["inlet_hi"]
        assert 0 <= lo and hi <= 256 and hi - lo == 64
        a, u = ph["in_alpha"], ph["in_ug"]
        assert a[0] == a[1] and 0.2 <= a[0] <= 0.4
        assert u[0] == u[1] and 0.5 * base["in_ug"][1] <= u[0] <= base["in_ug"][1]
        assert ph["ramp_nt"] == 0 and ph["bc_lo"][ph["g_axis"]] == lbm_inputs.INLET
        # everything but the inlet is the workload's physics
        assert {k: v for k, v in ph.items() if k not in ("inlet_lo", "inlet_hi", "in_alpha", "in_ug")} == \
            {k: v for k, v in base.items() if k not in ("inlet_lo", "inlet_hi", "in_alpha", "in_ug")}
        seen.add(lo)
    assert len(seen) > 50  # the position varies


def test_nominal_inflow():
    ph = lbm_inputs.surrogate_inlet(1234)
    want = 64 * (ph["inlet_hi"] - ph["inlet_lo"]) * ph["in_alpha"][1] * ph["in_ug"][1]
    assert S.inflow_per_window("inlet", 1234) == want
    assert np.array_equal(S.inflows(3, 1234, "inlet"),
                          [S.inflow_per_window("inlet", 1234 + i) for i in range(3)])
    w = lbm_inputs.WORKLOADS["surrogate2d_inlet"]["physics"]
    assert S.inflow_per_window("inlet") == 64 * 64 * w["in_alpha"][1] * w["in_ug"][1]
    assert S.inflow_per_window("plume") == 0.0 and not S.inflows(4, 0, "plume").any()


def test_window_volumes():
    r = np.random.default_rng(3)
    data = torch.from_numpy(r.uniform(0.0, 1.0, (2, 5, 6, 40)))
    dv, v = S.window_volumes(data)
    sums = data[:, :, 0].sum(dim=2).numpy()
    assert dv.shape == (2, 4) and v.shape == (2, 4)
    assert np.allclose(dv.numpy(), sums[:, 1:] - sums[:, :-1]) and np.allclose(v.numpy(), sums[:, :-1])
    # per trajectory expected inflow as a column
    dev = S.inflow_deviation(dv, v, torch.tensor([[0.5], [1.5]], dtype=torch.float64))
    assert np.allclose(dev.numpy(), np.abs(dv.numpy() - np.array([[0.5], [1.5]])) / v.numpy())


def test_calibration():
    r = np.random.default_rng(5)
    nom = np.repeat(r.uniform(2.0, 5.0, 10), 8)
    v = r.uniform(8000.0, 9000.0, nom.size)
    # exactly k x nominal: k recovered, no deviation, the check separates
    k, floor, summary = S.calibrate(1.7 * nom, v, nom, 1e-4)
    assert abs(k - 1.7) < 1e-12 and floor < 1e-15 and summary["check_separates_inflow"]
    # with scatter: k is the ratio of the totals, the floor the p99 of the relative deviation
    dv = 1.7 * nom + r.normal(0.0, 2.0, nom.size)
    k, floor, summary = S.calibrate(dv, v, nom, 1e-4)
    assert abs(k - dv.sum() / nom.sum()) < 1e-12
    assert abs(floor - np.quantile(np.abs(dv - k * nom) / v, 0.99)) < 1e-15
    assert not summary["check_separates_inflow"]
    assert summary["lbm_deviation_nominal"]["max"] == np.max(np.abs(dv - nom) / v)
    # a closed box: k = 1, the deviation is the LBM's own change
    dv0 = r.normal(0.0, 1e-3, nom.size)
    k, floor, summary = S.calibrate(dv0, v, np.zeros_like(nom), 1e-4)
    assert k == 1.0 and abs(floor - np.quantile(np.abs(dv0) / v, 0.99)) < 1e-18 and summary["check_separates_inflow"]
