"""Accuracy of the fast forms at the workloads' stated lengths, against the
FP64 path on the GPU (bitwise equal to the CPU oracle on every parity case;
the oracle itself would need hours at these sizes).

Per field, relative L2 after the stated step count: alpha_g, u_g, u_l (over
max(|u_l|, |u_g|/R), test_gpu_parity.u_l_scale) and, for FP32, p_k - 1/3.

- 2D bubble-column box (D2Q9 512 x 2048, FP32, inlet strip, R = 1000):
  20,000 steps, bar 1e-5 on every field.
- 3D column error configuration (D3Q19 64 x 64 x 128 of the 256 x 256 x 512
  recipe, R = 1000): 5,000 steps; FP32 at 1e-5 on alpha_g and u; FP16AB (f_g,
  f_l float, f_alpha, f_beta half) at the half store's 1e-3 on alpha_g, u_g,
  u_l; FP16DEV (every scheme half) at 1e-3 on alpha_g and u_g.
"""
import numpy as np
import pytest

import lbm_inputs
import paper_2409_10399_gb300 as lbm
from paper_2409_10399_gb300 import params as lparams
from test_gpu_parity import rel, u_l_scale

pytestmark = pytest.mark.gpu


def _run(name, dims, prec, steps, chunk=2000):
    w = lbm_inputs.WORKLOADS[name]
    s = lbm.Simulation(w["lattice"], dims, lparams.lattice_params(w["physics"], precision=prec))
    s.init(**lbm_inputs.fields_for(name, dims=dims))
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        s.step(k)
        done += k
    m, d = s.moments(), s.diag()
    s.close()
    assert d[5] == 0, (name, prec, "non-finite populations")
    return m


def _errors(got, ref, R):
    return dict(alpha_g=rel(got["alpha_g"], ref["alpha_g"]), u_g=rel(got["u_g"], ref["u_g"]),
                u_l=np.linalg.norm(got["u_l"] - ref["u_l"]) / u_l_scale(ref, R),
                p_k=rel(got["p_k"] - 1 / 3, ref["p_k"] - 1 / 3))


def test_box2d_fp32_at_20000_steps():
    w = lbm_inputs.WORKLOADS["box2d"]
    ref = _run("box2d", w["dims"], "fp64", w["steps"])
    got = _run("box2d", w["dims"], "fp32", w["steps"])
    e = _errors(got, ref, w["physics"]["R"])
    for k, v in e.items():
        assert v <= 1e-5, ("box2d fp32 20000 steps", k, e)


def test_column3d_error_configuration():
    w = lbm_inputs.WORKLOADS["column3d"]
    dims, steps, R = (64, 64, 128), w["steps"], w["physics"]["R"]
    ref = _run("column3d", dims, "fp64", steps)
    bars = {"fp32": (1e-5, ("alpha_g", "u_g", "u_l")), "fp16ab": (1e-3, ("alpha_g", "u_g", "u_l")),
            "fp16dev": (1e-3, ("alpha_g", "u_g"))}
    for prec, (tol, keys) in bars.items():
        e = _errors(_run("column3d", dims, prec, steps), ref, R)
        for k in keys:
            assert e[k] <= tol, ("column3d 64x64x128 5000 steps", prec, k, e)


def test_batch_sweep_fp32_at_10000_steps():
    """Three instances of the batched sweep (its smallest columns, R drawn
    log-uniform in [10, 1000]) advanced together through the batched kernel
    for the sweep's 10,000 steps, each against its own FP64 single-lattice
    run: every field within the FP32 bar."""
    sweep = lbm_inputs.batch_sweep()
    idx = sorted(range(len(sweep)), key=lambda i: sweep[i][0][0])[:3]
    dims = [sweep[i][0] for i in idx]
    pars = [lparams.lattice_params(sweep[i][1], precision="fp32") for i in idx]
    fields = [lbm_inputs.fields_step_profile(d[0], d[1], seed=4 + i) for d, i in zip(dims, idx)]
    b = lbm.Batch("D2Q9", dims, pars)
    for k, f in enumerate(fields):
        b.init(k, **f)
    steps = lbm_inputs.WORKLOADS["batch256"]["steps"]
    b.step(steps)
    for k, i in enumerate(idx):
        s = lbm.Simulation("D2Q9", dims[k], lparams.lattice_params(sweep[i][1], precision="fp64"))
        s.init(**fields[k])
        s.step(steps)
        e = _errors(b.moments(k), s.moments(), sweep[i][1]["R"])
        for key, v in e.items():
            assert v <= 1e-5, ("batch instance", i, dims[k], key, e)
