"""Throughput and accuracy of the method's forms on their workloads, measured
live on the current GPU (CUDA events on the stream the library launches on).

    python -m paper_2409_10399_gb300.forms [--only box2d,column3d,batch,surrogate,column1d] [--quick]

Each form is timed at its workload's full size and compared with the plain
single-lattice paths on the same GPU: the FP32 fast path and the FP64
reference path (bitwise equal to the CPU oracle on every parity case).  The
accuracy it is run at is the relative L2 error against that FP64 path after
the workload's stated step count (or at the reduced size the workload names
for its error study), per field: alpha_g, u_g, u_l, p_k - 1/3.

- box2d (D2Q9 512 x 2048, inlet strip, 20,000 steps): FP32 (the benchmark
  form), FP16-dev, FP16AB, FP64, and the FP32 beta-stencil form (throughput,
  with its fractions of the HBM peak on B_min and on B_6 separately).
- column3d (D3Q19 256 x 256 x 512, 5,000 steps; errors at 64 x 64 x 128):
  FP16-dev (its form), FP16AB (f_g, f_l float), FP32, FP64.
- batch256 (256 ragged D2Q9 FP32 columns, 1.06e8 nodes): one launch per step
  under graph replay, against the same instances stepped one by one with the
  FP32 and FP64 single-lattice path; accuracy of one instance against its
  FP64 run after 10,000 steps.
- surrogate (D2Q9 256 x 1024, 2,115,920 parameters, one call = 64 LBM steps):
  speed of a call against 64 FP32 and FP64 LBM steps on the same state; its
  accuracy depends on training (the surrogate study), so none is claimed here.
- column1d (D1Q3 512, FP64, 10,000 steps): time per step, and FP64 FLOP/s
  against the GPU's FP64 peak measured here with a float64 matrix product.

The FP64 path is bound by FP64 arithmetic on this GPU, not by memory; its
roofline is FP64_OPS_PER_NODE (FP64 operations executed per node update,
dadd + dmul + 2 dfma, counted by ncu on the reference step kernel) over the
measured FP64 peak.
"""
import argparse
import json
import time

import numpy as np

import lbm_inputs
from . import Batch, Simulation, Surrogate
from . import params as lparams

# FP64 operations executed per node update by the FP64 reference step
# kernel (k_step_ref), counted with ncu as dadd + dmul + 2 dfma over the
# threads of a launch without the lag latch on the lattice's workload recipe
# (column1d 512, box2d at 512 x 256, column3d at 64 x 64 x 128), divided by the
# nodes.  The dfma come mostly from the IEEE division and square root
# sequences: the reference evaluates the paper's divisions literally.
FP64_OPS_PER_NODE = {"D1Q3": 710, "D2Q9": 1956, "D3Q19": 4219}
B6 = {("D2Q9", "fp32"): 444, ("D2Q9", "fp16dev"): 228, ("D2Q9", "fp64"): 888,
      ("D3Q19", "fp32"): 924, ("D3Q19", "fp16dev"): 468, ("D3Q19", "fp64"): 1848,
      ("D1Q3", "fp64"): 312, ("D1Q3", "fp32"): 156, ("D2Q9", "fp16ab"): 300, ("D3Q19", "fp16ab"): 620}


def _torch():
    import torch
    return torch


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def errors(got, ref, R):
    """Relative L2 per field of a run against the FP64 run of the same state;
    u_l over max(|u_l|, |u_g|/R), the scale the interphase force (divided by R
    on the liquid side, Eq. (Gl)) gives the liquid velocity."""
    ul = float(np.linalg.norm(got["u_l"] - ref["u_l"]) /
               max(np.linalg.norm(ref["u_l"]), np.linalg.norm(ref["u_g"]) / R))
    return dict(alpha_g=_rel(got["alpha_g"], ref["alpha_g"]), u_g=_rel(got["u_g"], ref["u_g"]), u_l=ul,
                p_k=_rel(got["p_k"] - 1 / 3, ref["p_k"] - 1 / 3))


def _sim(lat, dims, p, fields, stream):
    s = Simulation(lat, dims, p)
    s.set_stream(stream)
    s.init(**fields)
    return s


def time_steps(sim, n, stream, warm=5):
    """Seconds per step of `n` steps (after `warm` untimed ones), the GPU kept
    busy while the launches are queued so that no host gap is timed."""
    torch = _torch()
    sim.step(warm)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda._sleep(2_000_000)
    e0.record(stream)
    sim.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / n


def run(lat, dims, p, fields, steps, stream, chunk=2000):
    s = _sim(lat, dims, p, fields, stream)
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        s.step(k)
        done += k
    m = s.moments()
    d = s.diag()
    s.close()
    return m, d


def fp64_peak(n=4096, reps=5):
    """FP64 FLOP/s of a float64 matrix product (cuBLAS), best of `reps`."""
    torch = _torch()
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best


def _lattice_forms(name, lat, dims, forms, steps_time, stream):
    w = lbm_inputs.WORKLOADS[name]
    f = lbm_inputs.fields_for(name, dims=dims)
    N = int(np.prod(dims))
    out = {}
    for prec in forms:
        p = lparams.lattice_params(w["physics"], precision=prec)
        s = _sim(lat, dims, p, f, stream)
        n = steps_time if prec != "fp64" else max(4, steps_time // 10)
        sec = time_steps(s, n, stream)
        s.close()
        out[prec] = dict(us_per_step=sec * 1e6, MLUPS=N / sec / 1e6, bytes_per_node=B6.get((lat, prec)),
                         GBs=N * B6.get((lat, prec), 0) / sec / 1e9, timed_steps=n)
    return out


def box2d(stream, quick=False):
    """The bench workload's forms at full size, and FP32 / FP16 accuracy
    against FP64 after the stated 20,000 steps (quick: 2,000)."""
    w = lbm_inputs.WORKLOADS["box2d"]
    lat, dims = w["lattice"], w["dims"]
    res = dict(workload="box2d D2Q9 512x2048, R=1000, inlet strip", nodes=int(np.prod(dims)))
    res["forms"] = _lattice_forms("box2d", lat, dims, ("fp32", "fp16dev", "fp16ab", "fp64"), 400, stream)
    res["forms"]["fp32_bstencil"] = bstencil_form("box2d", lat, dims, "fp32", 400, stream)
    steps = 2000 if quick else w["steps"]
    f = lbm_inputs.fields_for("box2d")
    ref, _ = run(lat, dims, lparams.lattice_params(w["physics"], precision="fp64"), f, steps, stream)
    acc = {}
    for prec in ("fp32", "fp16dev", "fp16ab"):
        got, d = run(lat, dims, lparams.lattice_params(w["physics"], precision=prec), f, steps, stream)
        acc[prec] = dict(errors(got, ref, w["physics"]["R"]), nonfinite_nodes=int(d[5]))
    res["accuracy"] = dict(against="fp64 GPU path, same state", steps=steps, dims=list(dims), **acc)
    _speedups(res)
    return res


def column3d(stream, quick=False):
    w = lbm_inputs.WORKLOADS["column3d"]
    lat, dims = w["lattice"], w["dims"]
    res = dict(workload="column3d D3Q19 256x256x512, R=1000, walls x/y, periodic z", nodes=int(np.prod(dims)))
    res["forms"] = _lattice_forms("column3d", lat, dims, ("fp16dev", "fp16ab", "fp32", "fp64"), 50, stream)
    small = (64, 64, 128)
    steps = 500 if quick else w["steps"]
    f = lbm_inputs.fields_for("column3d", dims=small)
    ref, _ = run(lat, small, lparams.lattice_params(w["physics"], precision="fp64"), f, steps, stream)
    acc = {}
    for prec in ("fp16dev", "fp16ab", "fp32"):
        got, d = run(lat, small, lparams.lattice_params(w["physics"], precision=prec), f, steps, stream)
        acc[prec] = dict(errors(got, ref, w["physics"]["R"]), nonfinite_nodes=int(d[5]))
    res["accuracy"] = dict(against="fp64 GPU path, same state", steps=steps, dims=list(small), **acc)
    _speedups(res)
    return res


# Beta-stencil form (Eq. (lbmbeta) with beta = 1, the beta schemes replaced
# by the c field): bytes per node as stored (4 schemes' populations, the
# held fields, the 2 D values of c read and written) and B_min, the same
# without c; its fractions of the measured HBM peak are reported on B_min
# and on B_6 (the six-scheme store it stands for) separately.
BSTENCIL = {("D2Q9", "fp32"): (4 * 9 * 2 * 4 + 12 + 2 * 4 * 4, 300)}


def hbm_peak_gbs():
    """The measured copy bandwidth (MEASURED_PEAKS.json at the repository
    root), else the earlier GB300 measurement of 6,800 GB/s."""
    import os
    try:
        with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def bstencil_form(name, lat, dims, prec, steps_time, stream):
    w = lbm_inputs.WORKLOADS[name]
    f = lbm_inputs.fields_for(name, dims=dims)
    N = int(np.prod(dims))
    s = _sim(lat, dims, dict(lparams.lattice_params(w["physics"], precision=prec), beta_stencil=1), f, stream)
    sec = time_steps(s, steps_time, stream)
    s.close()
    stored, bmin = BSTENCIL[(lat, prec)]
    peak = hbm_peak_gbs()
    mlups = N / sec / 1e6
    return dict(us_per_step=sec * 1e6, MLUPS=mlups, bytes_per_node=stored, GBs=N * stored / sec / 1e9,
                timed_steps=steps_time, frac_of_peak_on_Bmin=mlups * 1e6 * bmin / 1e9 / peak,
                frac_of_peak_on_B6=mlups * 1e6 * B6[(lat, prec)] / 1e9 / peak, B_min=bmin, B_6=B6[(lat, prec)])


def _speedups(res):
    fm = res["forms"]
    for prec, r in fm.items():
        if prec != "fp32" and "fp32" in fm:
            r["speedup_vs_fp32"] = fm["fp32"]["us_per_step"] / r["us_per_step"]
        if prec != "fp64" and "fp64" in fm:
            r["speedup_vs_fp64"] = fm["fp64"]["us_per_step"] / r["us_per_step"]


def batch(stream, quick=False, n=256, seed=4):
    """The batched sweep against the same instances on the single-lattice path."""
    torch = _torch()
    sweep = lbm_inputs.batch_sweep(n=n, seed=seed)
    dims = [d for d, _ in sweep]
    N = sum(d[0] * d[1] for d in dims)
    res = dict(workload="batch of %d D2Q9 FP32 columns (nx 64..512, ny = 4 nx), R log-uniform 10..1000" % n,
               nodes=N)
    pars = [lparams.lattice_params(ph, precision="fp32") for _, ph in sweep]
    b = Batch("D2Q9", dims, pars)
    b.set_stream(stream)
    fields = [lbm_inputs.fields_step_profile(d[0], d[1], seed=seed + i) for i, d in enumerate(dims)]
    for i, f in enumerate(fields):
        b.init(i, **f)
    period = 200
    b.step(period)  # captures the period's graph
    torch.cuda.synchronize()
    steps = period if quick else 2 * period
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(2_000_000)
    l0 = b.launches
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3 / steps
    launches = b.launches - l0
    bad = sum(int(b.diag(i)[5]) for i in range(b.n))
    b.close()
    forms = {"batched_fp32": dict(us_per_step=t_b * 1e6, MLUPS=N / t_b / 1e6, GBs=N * 444 / t_b / 1e9,
                                  timed_steps=steps, launches_per_step=launches / steps, nonfinite_nodes=bad)}
    # plain single-lattice path: every instance on its own context in turn
    for prec, k in (("fp32", 20), ("fp64", 4)):
        tot = 0.0
        for d, ph, f in zip(dims, sweep, fields):
            p = lparams.lattice_params(ph[1], precision=prec)
            s = _sim("D2Q9", d, p, f, stream)
            tot += time_steps(s, k, stream, warm=2)
            s.close()
        forms["plain_" + prec] = dict(us_per_step=tot * 1e6, MLUPS=N / tot / 1e6, timed_steps_per_instance=k)
    for key in ("plain_fp32", "plain_fp64"):
        forms["batched_fp32"]["speedup_vs_" + key] = forms[key]["us_per_step"] / forms["batched_fp32"]["us_per_step"]
    res["forms"] = forms
    # accuracy: the first instance of the sweep through the batched kernel
    # against its FP64 run after the stated 10,000 steps (quick: 1,000)
    st = 1000 if quick else lbm_inputs.WORKLOADS["batch256"]["steps"]
    i = 0
    b1 = Batch("D2Q9", [dims[i]], [pars[i]])
    b1.set_stream(stream)
    b1.init(0, **fields[i])
    b1.step(st)
    got = b1.moments(0)
    b1.close()
    ref, _ = run("D2Q9", dims[i], lparams.lattice_params(sweep[i][1], precision="fp64"), fields[i], st, stream)
    res["accuracy"] = dict(against="fp64 GPU path, same state", steps=st, instance=i, dims=list(dims[i]),
                           R=sweep[i][1]["R"], batched_fp32=errors(got, ref, sweep[i][1]["R"]))
    return res


def surrogate(stream, reps=20):
    """One surrogate call (untrained weights: the cost does not depend on
    them) against 64 LBM steps of the same state on the plain paths."""
    torch = _torch()
    from . import surrogate as S
    nx, ny = 256, 1024
    st = S.trajectories(1, 1000, nx, ny, S.WINDOW)[0, 1].contiguous()
    m = Surrogate(nx, ny, 64, 32, 4)
    m.set_stream(stream)
    m.set_params(S.init_params(64, 32, 4))
    out = torch.empty_like(st)
    m.advance(st, out, max_drift=1e30)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(2_000_000)
    e0.record(stream)
    for _ in range(reps):
        m.advance(st, out, max_drift=1e30)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sur = e0.elapsed_time(e1) / 1e3 / reps
    m.close()
    res = dict(workload="surrogate: D2Q9 256x1024 inlet-box state, F-FNO C=64 K=32 L=4 (2,115,920 parameters), one call = "
                        "64 LBM steps", nodes=nx * ny, call_ms=t_sur * 1e3,
               tflops=S.model_flops(nx, ny, 64, 32, 4) / t_sur / 1e12)
    for prec in ("fp32", "fp64"):
        s = _sim("D2Q9", (nx, ny, 1), S._lbm_params(prec, seed=1000), S._views(st), stream)
        sec = time_steps(s, S.WINDOW if prec == "fp32" else 8, stream)
        s.close()
        res["lbm_%s_64_steps_ms" % prec] = sec * S.WINDOW * 1e3
        res["speedup_vs_" + prec] = sec * S.WINDOW / t_sur
    res["accuracy"] = "depends on training: held-out errors and hybrid runs of the trained model are in the " \
                      "surrogate study (python -m paper_2409_10399_gb300.surrogate)"
    return res


def column1d(stream, quick=False):
    """The FP64 1D column at full length: time per step (graph-replayed
    periods) and FP64 FLOP/s against the measured FP64 peak."""
    w = lbm_inputs.WORKLOADS["column1d"]
    lat, dims = w["lattice"], w["dims"]
    f = lbm_inputs.fields_for("column1d")
    N = dims[0]
    res = dict(workload="column1d D1Q3 512, FP64, walls, wall friction", nodes=N)
    steps = 2000 if quick else w["steps"]
    forms = {}
    for prec in ("fp64", "fp32"):
        s = _sim(lat, dims, lparams.lattice_params(w["physics"], precision=prec), f, stream)
        sec = time_steps(s, steps, stream, warm=400)
        s.close()
        forms[prec] = dict(us_per_step=sec * 1e6, steps_per_s=1.0 / sec, MLUPS=N / sec / 1e6, timed_steps=steps)
    forms["fp32"]["speedup_vs_fp64"] = forms["fp64"]["us_per_step"] / forms["fp32"]["us_per_step"]
    res["forms"] = forms
    return res


def fp64_roofline(lat, mlups, peak):
    ops = FP64_OPS_PER_NODE.get(lat)
    if ops is None:
        return dict(bound="fp64", ops_per_node=None, achieved=None, peak=peak / 1e12, unit="TFLOP/s", frac=None)
    ach = ops * mlups * 1e6
    return dict(bound="fp64", ops_per_node=ops, achieved=ach / 1e12, peak=peak / 1e12, unit="TFLOP/s",
                frac=ach / peak)


def all_forms(stream, only=None, quick=False, log=None):
    out = {}
    jobs = [("box2d", lambda: box2d(stream, quick)), ("column3d", lambda: column3d(stream, quick)),
            ("batch", lambda: batch(stream, quick)), ("surrogate", lambda: surrogate(stream)),
            ("column1d", lambda: column1d(stream, quick))]
    for name, fn in jobs:
        if only and name not in only:
            continue
        t0 = time.time()
        out[name] = fn()
        out[name]["wall_s"] = time.time() - t0
        if log:
            log(name, out[name])
        _torch().cuda.empty_cache()
    peak = fp64_peak()
    out["fp64_peak_tflops"] = peak / 1e12
    for name, lat in (("box2d", "D2Q9"), ("column3d", "D3Q19"), ("column1d", "D1Q3")):
        if name in out and "fp64" in out[name]["forms"]:
            out[name]["forms"]["fp64"]["roofline"] = fp64_roofline(lat, out[name]["forms"]["fp64"]["MLUPS"], peak)
    return out


def main():
    torch = _torch()
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="")
    ap.add_argument("--quick", action="store_true")
    args = ap.parse_args()
    stream = torch.cuda.current_stream()
    only = set(x for x in args.only.split(",") if x)
    res = all_forms(stream, only, args.quick, log=lambda n, r: print(json.dumps({n: r}), flush=True))
    print(json.dumps({"fp64_peak_tflops": res["fp64_peak_tflops"]}))


if __name__ == "__main__":
    main()
