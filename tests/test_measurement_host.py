"""Host arithmetic of the measurement (no GPU): the algorithmic bytes per
node update behind every roofline (each population read once and written
once, the three held fields read; the beta-stencil store with its c field),
SURVEY-style figures for the workloads (D2Q9 FP32 444 B, D3Q19 FP16 468 B,
the FP64 stores twice their FP32 size), the FP64 roofline, and the per-field
error metric of the forms (u_l over max(|u_l|, |u_g| / R))."""
import numpy as np
import pytest

import bench
from paper_2409_10399_gb300 import forms

Q = {"D1Q3": 3, "D2Q9": 9, "D3Q19": 19}
D = {"D1Q3": 1, "D2Q9": 2, "D3Q19": 3}


def _bytes(lat, prec):
    q = Q[lat]
    if prec == "fp16ab":  # f_g, f_l float; f_alpha, f_beta half; float held fields
        return 2 * q * 2 * 4 + 4 * q * 2 * 2 + 3 * 4
    store = {"fp64": 8, "fp32": 4, "fp16dev": 2}[prec]
    held = 8 if prec == "fp64" else 4
    return 6 * q * 2 * store + 3 * held


def test_algorithmic_bytes_per_node():
    for (lat, prec), b in forms.B6.items():
        assert b == _bytes(lat, prec), (lat, prec)
    assert forms.B6[("D2Q9", "fp32")] == 444 and forms.B6[("D3Q19", "fp16dev")] == 468
    assert forms.B6[("D2Q9", "fp64")] == 888 and forms.B6[("D3Q19", "fp64")] == 1848
    assert forms.B6[("D1Q3", "fp64")] == 312
    assert bench.bytes_per_node("D2Q9", "fp32") == 444
    # the beta-stencil store: 4 schemes' populations, the held fields, c read and written
    stored, bmin = forms.BSTENCIL[("D2Q9", "fp32")]
    assert stored == 4 * 9 * 2 * 4 + 12 + 2 * D["D2Q9"] * 4 * 2 and bmin == 4 * 9 * 2 * 4 + 12


def test_fp64_roofline_arithmetic():
    r = forms.fp64_roofline("D2Q9", 382.0, 1.1e12)
    assert r["ops_per_node"] == 1956 and r["achieved"] == pytest.approx(1956 * 382e6 / 1e12)
    assert r["frac"] == pytest.approx(1956 * 382e6 / 1.1e12) and r["peak"] == pytest.approx(1.1)
    assert forms.fp64_roofline("D4Q0", 1.0, 1e12)["frac"] is None


def test_error_metric():
    r = np.random.default_rng(1)
    ref = dict(alpha_g=r.uniform(0.1, 0.3, 50), u_g=r.normal(0, 1e-3, (2, 50)), u_l=r.normal(0, 1e-7, (2, 50)),
               p_k=1 / 3 + r.normal(0, 1e-5, 50))
    got = {k: v.copy() for k, v in ref.items()}
    got["u_l"] = got["u_l"] + 1e-8
    got["p_k"] = got["p_k"] + 1e-7
    e = forms.errors(got, ref, 1000.0)
    scale = max(np.linalg.norm(ref["u_l"]), np.linalg.norm(ref["u_g"]) / 1000.0)
    assert e["alpha_g"] == 0.0 and e["u_g"] == 0.0
    assert e["u_l"] == pytest.approx(np.linalg.norm(np.full((2, 50), 1e-8)) / scale)
    assert e["p_k"] == pytest.approx(np.linalg.norm(np.full(50, 1e-7)) / np.linalg.norm(ref["p_k"] - 1 / 3))
    # the liquid at rest: the gas velocity over R sets the scale
    ref["u_l"] = np.zeros((2, 50))
    got["u_l"] = np.full((2, 50), 1e-8)
    assert forms.errors(got, ref, 1000.0)["u_l"] == pytest.approx(
        np.linalg.norm(got["u_l"]) / (np.linalg.norm(ref["u_g"]) / 1000.0))


def test_speedups():
    res = {"forms": {"fp32": {"us_per_step": 80.0}, "fp16dev": {"us_per_step": 60.0}, "fp64": {"us_per_step": 2400.0}}}
    forms._speedups(res)
    f = res["forms"]
    assert f["fp16dev"]["speedup_vs_fp32"] == pytest.approx(80 / 60) and f["fp16dev"]["speedup_vs_fp64"] == 40.0
    assert f["fp32"]["speedup_vs_fp64"] == 30.0 and "speedup_vs_fp32" not in f["fp32"]
    assert "speedup_vs_fp64" not in f["fp64"]


def test_clock_sampler_parses_nvidia_smi_lines():
    """The clock record of the timed region (nvidia-smi CSV, no units): the
    median SM clock, the maximum, and every throttle reason seen active."""
    s = bench.ClockSampler(0)

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = _Proc()
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2050, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1980, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Active",
               "garbage", "0, N/A, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = s.stop()
    assert c == {"sm_mhz": 2050.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    empty = bench.ClockSampler(0)
    assert empty.stop() is None
