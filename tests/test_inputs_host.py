"""The seeded input recipes (lbm_inputs) against their stated definitions:
shapes, ranges, seeding, the batched sweep's distributions, and the 3D
column's correlation length (white noise smoothed by a Gaussian of standard
deviation s nodes has autocorrelation exp(-d^2 / (4 s^2)) at lag d)."""
import numpy as np
import pytest

import lbm_inputs as I


def test_column1d_step_profile():
    f = I.fields_column1d(512, 1)
    a = f["alpha_g"]
    assert a.shape == (512,) and f["u_g"].shape == (1, 512) and not f["u_g"].any() and not f["u_l"].any()
    assert np.all(np.abs(a[:256] - 0.9) <= 1e-3) and np.all(np.abs(a[256:] - 0.1) <= 1e-3)
    assert np.all(f["p_k"] == I.CS2_PK)
    assert np.array_equal(a, I.fields_for("column1d")["alpha_g"])
    assert not np.array_equal(a, I.fields_column1d(512, 2)["alpha_g"])


def test_box2d_background_and_noise():
    f = I.fields_box2d(64, 256, 2)
    n = 64 * 256
    assert np.all(f["alpha_g"] == 0.01) and np.all(f["p_k"] == I.CS2_PK)
    for k in ("u_g", "u_l"):
        u = f[k]
        assert u.shape == (2, n) and np.abs(u).max() <= 4.3e-5
        assert abs(np.abs(u).mean() - 4.3e-5 / 2) < 4.3e-5 * 0.02  # U(-1, 1) * 1 % of 4.3e-3
    ph = I.WORKLOADS["box2d"]["physics"]
    assert (ph["inlet_lo"], ph["inlet_hi"]) == (192, 320) and ph["in_alpha"][1] == 0.3 and ph["ramp_nt"] == 1667


def test_column3d_smoothed_gas_fraction():
    # a periodic box of 16 correlation lengths, so that lags up to 2 s are
    # measured without the wrap-around's bias
    f = I.fields_column3d(128, 128, 128, seed=3)
    a = f["alpha_g"].reshape(128, 128, 128)
    assert abs(a.mean() - 0.05) < 1e-4 and abs(a.std() - 0.01) < 2e-4
    assert not f["u_g"].any() and f["u_g"].shape == (3, 128 ** 3)
    d = a - a.mean()
    for lag in (1, 8, 16):
        c = np.mean([np.mean(d * np.roll(d, lag, axis=ax)) for ax in range(3)]) / d.var()
        assert abs(c - np.exp(-lag * lag / (4 * 8.0 ** 2))) < 0.03, (lag, c)


def test_batch_sweep_distributions():
    sw = I.batch_sweep()
    assert len(sw) == 256 and sw == I.batch_sweep()
    nx = np.array([d[0] for d, _ in sw])
    R = np.array([ph["R"] for _, ph in sw])
    dm = np.array([ph["d_m"] for _, ph in sw])
    assert all(d[1] == 4 * d[0] and d[2] == 1 for d, _ in sw)
    assert nx.min() >= 64 and nx.max() <= 512 and 1.0e8 < (4 * nx * nx).sum() < 1.1e8
    assert R.min() >= 10.0 and R.max() <= 1000.0 and abs(np.log10(R).mean() - 2.0) < 0.15
    assert dm.min() >= 0.5e-3 and dm.max() <= 5e-3
    for _, ph in sw:
        assert ph["g_hat"] * (ph["R"] - 1.0) == pytest.approx(1e-6) and ph["gamma"] == 1.0 and ph["n_gamma"] == 200


def test_plumes_and_step_profile():
    p = I.fields_plumes(64, 128, 11)
    assert p["alpha_g"].min() >= 0.01 and p["alpha_g"].max() <= 0.6 and p["alpha_g"].max() > 0.1
    assert np.abs(p["u_g"]).max() <= 1e-5 and np.abs(p["u_l"]).max() <= 1e-5
    s = I.fields_step_profile(32, 128, 4)
    a = s["alpha_g"].reshape(128, 32)
    assert np.all(np.abs(a[:64] - 0.9) <= 1e-3) and np.all(np.abs(a[64:] - 0.1) <= 1e-3)
