"""TEST #1 of Sec. 3.6 on the GPU (FP64 reference path, bitwise equal to the
oracle): the steady outlet state of the open tube against the values the
paper prints (tests/golden/paper_printed_values.txt), with the shortened ramp
and the bars of tests/test_oracle_test1.py."""
import os

import pytest

from paper_2409_10399_gb300 import validation

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")


def test_test1_outlet_on_gpu():
    g = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            g[k.strip()] = float(v)
    out = validation.run_test1(nt=200000, steps=1400000, omega_alpha=1.999)
    assert out["nonfinite"] == 0
    assert out["alpha_g"] == pytest.approx(g["test1_ag_out"], rel=5e-4)
    assert out["u_g"] == pytest.approx(g["test1_ug_out"], rel=5e-4)
    assert out["u_l"] == pytest.approx(g["test1_ul_out"], rel=5e-3)
    assert out["mixture_flux"] == pytest.approx(g["test1_mixture_flux_out"], rel=5e-4)
