"""Error and throughput of the precision forms on the workloads.

    python -m paper_2409_10399_gb300.accuracy [--study box2d|column3d|column1d|all|
                                                sensitivity|spalding|bstencil|column3d_small|
                                                fp64_launches]

For each study the same seeded state is advanced with the FP64 reference path
(bitwise equal to the CPU oracle on every case the tests cover) and with the
fast forms; the result reports, per form, the relative L2 error against FP64
on alpha_g, u_g, u_l (over max(|u_l|, |u_g|/R): the liquid receives the
interphase force divided by R) and p_k - 1/3, plus the device time per step
and MLUPS.  One JSON line per (study, form).
"""
import argparse
import json
import time

import numpy as np

import lbm_inputs
from . import LATTICE, Simulation
from . import params as lparams


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _rel_ul(got, ref, R):
    return float(np.linalg.norm(got["u_l"] - ref["u_l"]) /
                 max(np.linalg.norm(ref["u_l"]), np.linalg.norm(ref["u_g"]) / R))


def _run(lattice, dims, p, fields, steps, chunk=1000):
    import torch
    s = Simulation(lattice, dims, p)
    s.set_stream(torch.cuda.current_stream())
    s.init(**fields)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        s.step(n)
        done += n
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m = s.moments()
    d = s.diag()
    s.close()
    return m, ms / max(steps, 1), d


def study(name, steps=None, dims=None, forms=("fp32", "fp16dev"), spalding=None):
    w = lbm_inputs.WORKLOADS[name]
    dims = dims or w["dims"]
    steps = steps or w["steps"]
    f = lbm_inputs.fields_for(name, dims=dims)
    N = int(np.prod(dims))
    base = lparams.lattice_params(w["physics"])
    if spalding is not None:
        base["spalding_mode"] = spalding
    out = []
    ref, ms_ref, d_ref = _run(w["lattice"], dims, dict(base, precision="fp64"), f, steps)
    out.append(dict(study=name, dims=list(dims), steps=steps, form="fp64", spalding=base["spalding_mode"],
                    us_per_step=ms_ref * 1e3,
                    MLUPS=N / ms_ref / 1e3, nonfinite=int(d_ref[5])))
    u_ref = np.concatenate([ref["u_g"].ravel(), ref["u_l"].ravel()])
    for form in forms:
        got, ms, d = _run(w["lattice"], dims, dict(base, precision=form), f, steps)
        u = np.concatenate([got["u_g"].ravel(), got["u_l"].ravel()])
        out.append(dict(study=name, dims=list(dims), steps=steps, form=form, spalding=base["spalding_mode"],
                        us_per_step=ms * 1e3,
                        MLUPS=N / ms / 1e3, speedup_vs_fp64=ms_ref / ms,
                        err_alpha=_rel(got["alpha_g"], ref["alpha_g"]), err_u=_rel(u, u_ref),
                        err_u_g=_rel(got["u_g"], ref["u_g"]), err_u_l=_rel_ul(got, ref, base["R"]),
                        err_pk=_rel(got["p_k"] - 1 / 3, ref["p_k"] - 1 / 3), nonfinite=int(d[5])))
    return out


def sensitivity(name, rel_perturbation, steps=None, dims=None, seed=99):
    """How far the FP64 solution moves when the initial alpha_g is perturbed
    by +-rel_perturbation (random sign per node): the floor that any
    implementation rounding at that relative size faces after `steps`."""
    w = lbm_inputs.WORKLOADS[name]
    dims = dims or w["dims"]
    steps = steps or w["steps"]
    f = lbm_inputs.fields_for(name, dims=dims)
    g = dict(f)
    rng = np.random.default_rng(seed)
    g["alpha_g"] = f["alpha_g"] * (1.0 + rel_perturbation * rng.choice([-1.0, 1.0], f["alpha_g"].size))
    base = lparams.lattice_params(w["physics"], precision="fp64")
    a, _, _ = _run(w["lattice"], dims, base, f, steps)
    b, _, _ = _run(w["lattice"], dims, base, g, steps)
    ua = np.concatenate([a["u_g"].ravel(), a["u_l"].ravel()])
    ub = np.concatenate([b["u_g"].ravel(), b["u_l"].ravel()])
    return dict(study=name + "_sensitivity", dims=list(dims), steps=steps, rel_perturbation=rel_perturbation,
                err_alpha=_rel(b["alpha_g"], a["alpha_g"]), err_u=_rel(ub, ua),
                err_pk=_rel(b["p_k"] - 1 / 3, a["p_k"] - 1 / 3))


def throughput(name, form, steps=200, dims=None, beta_stencil=0, warm=20):
    """Device time per step of one form at the workload's full size."""
    w = lbm_inputs.WORKLOADS[name]
    dims = dims or w["dims"]
    f = lbm_inputs.fields_for(name, dims=dims)
    N = int(np.prod(dims))
    p = dict(lparams.lattice_params(w["physics"], precision=form), beta_stencil=beta_stencil)
    if warm:
        _run(w["lattice"], dims, p, f, warm)
    m, ms, d = _run(w["lattice"], dims, p, f, steps)
    return dict(study=name + "_throughput", dims=list(dims), steps=steps, form=form, beta_stencil=beta_stencil,
                us_per_step=ms * 1e3, MLUPS=N / ms / 1e3, nonfinite=int(d[5]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--study", default="all")
    ap.add_argument("--spalding", type=int, default=None, help="override the Spalding mode of the workloads")
    args = ap.parse_args()
    todo = []
    if args.study == "fp64_launches":
        # two launches of the FP64 reference step on each workload recipe at
        # a size one capture can hold (the FP64 operation counts of the
        # reference kernels are taken with ncu on these launches)
        todo.append(lambda: [throughput(n, "fp64", steps=2, dims=d, warm=0) for n, d in
                             (("column1d", (512, 1, 1)), ("box2d", (512, 256, 1)), ("column3d", (64, 64, 128)))])
    if args.study == "column3d_small":
        # D3Q19 at 128 x 128 x 256 (2 GB of store traffic per step): the
        # profiling case of the 3D kernels
        todo.append(lambda: [throughput("column3d", f, steps=20, dims=(128, 128, 256)) for f in ("fp16dev", "fp32")])
    if args.study == "bstencil":
        todo.append(lambda: [throughput(n, f, steps=400, beta_stencil=b) for n, f in
                             (("box2d", "fp32"), ("box2d", "fp16dev"), ("column3d", "fp16dev"), ("column3d", "fp32"))
                             for b in (0, 1)])
    if args.study == "spalding":
        todo.append(lambda: [r for m in (0, 1, 2) for r in study("box2d", steps=5000, forms=("fp32",), spalding=m)])
    if args.study in ("box2d", "all"):
        todo.append(lambda: study("box2d"))
    if args.study in ("column3d", "all"):
        todo.append(lambda: study("column3d", dims=(64, 64, 128)))
        todo.append(lambda: [throughput("column3d", "fp16dev"), throughput("column3d", "fp32")])
    if args.study in ("column1d", "all"):
        todo.append(lambda: study("column1d", forms=("fp32", "fp64dev")))
    if args.study in ("sensitivity", "all"):
        todo.append(lambda: [sensitivity("box2d", 2.0 ** -24), sensitivity("box2d", 2.0 ** -11),
                             sensitivity("column3d", 2.0 ** -24, dims=(64, 64, 128)),
                             sensitivity("column3d", 2.0 ** -11, dims=(64, 64, 128)),
                             sensitivity("column1d", 2.0 ** -24)])
    for job in todo:
        t0 = time.time()
        for line in job():
            line["wall_s"] = time.time() - t0
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
