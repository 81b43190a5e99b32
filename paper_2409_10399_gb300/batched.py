"""Batched parameter sweep: many independent D2Q9 columns in one launch per step.

    python -m paper_2409_10399_gb300.batched [--n 256] [--steps 1000] [--plain-steps 20]

Builds the sweep of lbm_inputs.batch_sweep (ragged sizes, per-instance density
ratio and drag), chooses the tile with the autotuner, advances every instance
with CUDA-graph replay, and compares with the plain path -- each instance
stepped on its own single-lattice context -- on the same GPU.  Instance i of
the batch is bitwise equal to its single-lattice run (tests), so the batch's
accuracy is the FP32 path's.  Prints one JSON line.
"""
import argparse
import json
import time

import numpy as np

import lbm_inputs
from . import Batch, Simulation, autotune
from . import params as lparams

B6_FP32_D2Q9 = 444


def build(n=256, seed=4, precision="fp32"):
    sweep = lbm_inputs.batch_sweep(n=n, seed=seed)
    dims = [d for d, _ in sweep]
    params = [lparams.lattice_params(ph, precision=precision) for _, ph in sweep]
    b = Batch("D2Q9", dims, params)
    fields = []
    for i, (d, _) in enumerate(sweep):
        f = lbm_inputs.fields_step_profile(d[0], d[1], seed=seed + i)
        b.init(i, **f)
        fields.append(f)
    return b, dims, params, fields


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--no-graph", action="store_true")
    args = ap.parse_args()
    t0 = time.time()
    b, dims, params, fields = build(args.n)
    N = sum(d[0] * d[1] for d in dims)
    stream = torch.cuda.current_stream()
    b.set_stream(stream)
    if args.no_graph:
        b.set_graph(False)
    tile, times = autotune.tune(b, 2, "fp32", N, "batch%d" % args.n, steps=10)
    # restart from the initial state after tuning, then warm up one graph period
    for i, f in enumerate(fields):
        b.init(i, **f)
    b.step(400)
    torch.cuda.synchronize()
    l0 = b.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    launches = b.launches - l0
    bad = sum(int(b.diag(i)[5]) for i in range(b.n))
    b.close()
    # plain path: each instance on its own context, one after another
    t_plain = 0.0
    for d, p, f in zip(dims, params, fields):
        s = Simulation("D2Q9", d, p)
        s.set_stream(stream)
        s.init(**f)
        s.step(4)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(args.plain_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1) / 1e3 / args.plain_steps
        s.close()
    per_step = t_batch / args.steps
    mlups = N / per_step / 1e6
    try:
        peak = json.load(open(__import__("os").path.join(__import__("os").path.dirname(__file__), "..",
                                                          "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        peak = 6800.0
    gbs = N * B6_FP32_D2Q9 / per_step / 1e9
    print(json.dumps(dict(
        workload="batch of %d D2Q9 FP32 columns (nx 64..512, ny = 4 nx), R log-uniform 10..1000, d 0.5..5 mm"
                 % args.n, nodes=N, steps=args.steps, graph=not args.no_graph, tile=list(tile),
        tuned={"x".join(map(str, k)): v for k, v in times.items()},
        us_per_step=per_step * 1e6, MLUPS=mlups, GBs=gbs, frac_of_measured_hbm=gbs / peak,
        plain_us_per_step=t_plain * 1e6, plain_MLUPS=N / t_plain / 1e6, speedup_vs_plain=t_plain / per_step,
        launches_in_timed_region=launches, nonfinite_nodes=bad, wall_s=time.time() - t0)), flush=True)


if __name__ == "__main__":
    main()
