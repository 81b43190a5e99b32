"""Convergence order of the GPU paths under diffusive scaling (Sec. 2.1.2).

    python -m paper_2409_10399_gb300.convergence [--forms fp64,fp32,fp16dev]

Self-convergence on smooth periodic states (lbm_inputs.fields_smooth1d /
fields_smooth2d): mesh spacing eps = 1/n, time step eps^2 (T n^2 steps to
continuum time T), g_hat = eps^3 g, K_hat_I = eps K_I, rates fixed
(params.diffusive_scaling).  Successive resolutions are compared on the
coarser cell centres (the finer field averaged over 2 or 2 x 2 cells); the
order is log2 of the ratio of successive differences.  One JSON line per
(case, form) with the differences and orders of alpha_g, u_g, u_l
(continuum units u_hat/eps) and p_k - cs2 (units of eps^2).  The FP64
reference path converges at second order like the oracle; the fast forms
follow it until their rounding floor: at eps = 1/1024 the pressure deviation
is ~1e-6 of cs2, below FP16 resolution and near FP32's.
"""
import argparse
import json
import time

import numpy as np

import lbm_inputs
from . import Simulation
from . import params as lparams

CS2 = 1.0 / 3.0

CASES = {
    # 1D column: buoyancy along x and CGW drag (continuum g = 0.3, K_I = 5)
    "smooth1d": dict(lattice="D1Q3", ns=(32, 64, 128, 256, 512, 1024), T=1.0,
                     base=dict(R=10.0, omega_g=0.6, omega_l=0.6, omega_alpha=1.5, spalding_mode=2, g_axis=0,
                               g_hat=0.3, drag_model=1, kappa_I=5.0)),
    # 2D Taylor-Green start, buoyancy along y, CGW drag
    "smooth2d": dict(lattice="D2Q9", ns=(32, 64, 128, 256), T=1.0,
                     base=dict(R=10.0, omega_g=0.6, omega_l=0.6, omega_alpha=1.5, spalding_mode=2, g_axis=1,
                               g_hat=0.3, drag_model=1, kappa_I=5.0)),
}


def _run(case, n, form):
    import torch
    c = CASES[case]
    eps = 1.0 / n
    p = dict(lparams.diffusive_scaling(c["base"], eps), precision=form)
    if c["lattice"] == "D1Q3":
        dims, f = (n,), lbm_inputs.fields_smooth1d(n, eps)
    else:
        dims, f = (n, n), lbm_inputs.fields_smooth2d(n, eps)
    s = Simulation(c["lattice"], dims, p)
    s.init(**f)
    steps = int(round(c["T"] * n * n))
    done = 0
    while done < steps:
        k = min(100000, steps - done)
        s.step(k)
        done += k
    torch.cuda.synchronize()
    m = s.moments()
    s.close()
    return dict(alpha_g=m["alpha_g"], u_g=m["u_g"] / eps, u_l=m["u_l"] / eps, p_k=(m["p_k"] - CS2) / eps ** 2), steps


def _coarsen(v, D, n):
    if D == 1:
        return 0.5 * (v[..., 0::2] + v[..., 1::2])
    w = v.reshape(v.shape[:-1] + (n, n))
    w = 0.25 * (w[..., 0::2, 0::2] + w[..., 0::2, 1::2] + w[..., 1::2, 0::2] + w[..., 1::2, 1::2])
    return w.reshape(v.shape[:-1] + (-1,))


def study(case, form):
    c = CASES[case]
    D = 1 if c["lattice"] == "D1Q3" else 2
    t0 = time.time()
    res = [_run(case, n, form)[0] for n in c["ns"]]
    out = dict(case=case, lattice=c["lattice"], form=form, ns=list(c["ns"]), T=c["T"], diff={}, order={})
    for k in ("alpha_g", "u_g", "u_l", "p_k"):
        e = [float(np.sqrt(np.mean((res[i][k] - _coarsen(res[i + 1][k], D, c["ns"][i + 1])) ** 2)))
             for i in range(len(c["ns"]) - 1)]
        out["diff"][k] = e
        out["order"][k] = [float(np.log2(e[i] / e[i + 1])) if e[i + 1] > 0 else None for i in range(len(e) - 1)]
    out["wall_s"] = time.time() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--forms", default="fp64,fp32,fp16dev")
    ap.add_argument("--cases", default="smooth1d,smooth2d")
    args = ap.parse_args()
    for case in args.cases.split(","):
        for form in args.forms.split(","):
            print(json.dumps(study(case, form)), flush=True)


if __name__ == "__main__":
    main()
