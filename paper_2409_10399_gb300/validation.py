"""The paper's TEST #1 (Sec. 3.6) on the GPU: the 1D open tube with the inlet of
Table 1 and the outlet of Table 2, R = 2, g_hat = 1e-6, K_I = K_W = 1e-2,
nu = 1.1667 (omega = 0.6), N_x = 200, inlet ramp n_t and N_t steps, run with
the FP64 reference path; prints the outlet state next to the values the paper
prints.

    python -m paper_2409_10399_gb300.validation [--nt 500000] [--steps 6000000] [--omega-alpha 1.9997]

omega_alpha is not stated in the paper; 1.9997 is Eq. (diffusivity2) at
eps = 1/N_x with chi = 1 (the diffusive scaling drives it to 2).
"""
import argparse
import json
import math
import time

import numpy as np

from . import Simulation

PAPER = dict(u_g=0.008423711190781, u_l=0.003975027343349, alpha_g=0.949686618689092,
             mixture_flux=0.008199882864033)


def test1_params(nt, omega_alpha, precision="fp64"):
    R, g, K = 2.0, 1e-6, 1e-2
    ug_min = math.sqrt(0.01 * 0.99 * (R - 1.0) * g / K)  # Eq. (analytical0bis)
    return dict(R=R, omega_g=0.6, omega_l=0.6, omega_alpha=omega_alpha, drag_model=0, kappa_I=K, kappa_W=K,
                g_hat=g, g_axis=0, gamma=0.0, n_gamma=1, spalding_mode=2, bc_lo=(2, 0, 0), bc_hi=(3, 0, 0),
                in_alpha=(0.01, 0.8), in_ug=(ug_min, 1e-2), in_ul=(0.0, 1e-3), ramp_nt=nt, inlet_ul_mode=0,
                precision=precision), ug_min


def run_test1(nt, steps, omega_alpha, precision="fp64", chunk=100000):
    p, ug_min = test1_params(nt, omega_alpha, precision)
    N = 200
    s = Simulation("D1Q3", (N,), p)
    s.set_tile(32)
    s.init(alpha_g=np.full(N, 0.01), u_g=np.full((1, N), ug_min), u_l=np.zeros((1, N)), p_k=np.full(N, 1 / 3))
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        s.step(k)
        done += k
    m = s.moments()
    ag, ug, ul = float(m["alpha_g"][-1]), float(m["u_g"][0, -1]), float(m["u_l"][0, -1])
    return dict(alpha_g=ag, u_g=ug, u_l=ul, mixture_flux=ag * ug + (1 - ag) * ul, nonfinite=int(s.diag()[5]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nt", type=int, default=500000)
    ap.add_argument("--steps", type=int, default=6000000)
    ap.add_argument("--omega-alpha", type=float, default=2.0 / (1.0 + 2.0 * (1.0 / 200) ** 2 * 1.0 * 3.0))
    args = ap.parse_args()
    import torch
    t0 = time.time()
    out = run_test1(args.nt, args.steps, args.omega_alpha)
    torch.cuda.synchronize()
    out.update(study="TEST #1 (Sec. 3.6) on the GPU, FP64 reference path", nt=args.nt, steps=args.steps,
               omega_alpha=args.omega_alpha, wall_s=time.time() - t0,
               paper=PAPER, rel_vs_paper={k: out[k] / PAPER[k] - 1.0 for k in PAPER})
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
