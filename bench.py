#!/usr/bin/env python
"""Throughput of the fused six-scheme EE-LBM step on GB300 (MLUPS).

One "step" is one time step of the whole hot path (moments, sources,
coupling, stabilisers, drag, forces, six collisions, AA streaming with the
face rules) over the 2D bubble-column box: D2Q9, 512 x 2048 nodes, FP32 store
and arithmetic, R = 1000, CGW drag, bottom inlet strip.  The library also
enqueues its FP64 diagnostics after every DIAG_EVERY-th step; a timed run of K
steps after t0 warm-up steps contains floor((t0 + K)/DIAG_EVERY) -
floor(t0/DIAG_EVERY) of them (200 for the default 20,000 steps after 100; none
for 20 steps after 5), reported as `diag_passes_timed`; the kernel time of the
roofline comes from the timed region's segments without them.  The store
(466 MB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--no-cpu-baseline] [--no-forms] [--quick-forms]

Prints one JSON line.  Besides the benchmark's own keys it carries `forms`:
every other form of the method timed live on the same GPU at its workload's
full size (FP16-deviation and FP16AB stores, the beta-stencil form, FP64
reference path, the batched sweep, the learned surrogate, the 1D column),
each with its speedup over the plain FP32 and FP64 single-lattice paths and
the accuracy it is run at
(paper_2409_10399_gb300/forms.py).  Under torchrun (N > 1) every rank
advances its own replica (different seed), timing is the max over ranks and
`value` the aggregate; there is no data-path collective.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_inputs  # noqa: E402

WORKLOAD = "box2d"
DIAG_EVERY = 100
FALLBACK_HBM_GBS = 6800.0
STORE_BYTES = {"fp64": 8, "fp32": 4, "fp16dev": 2}
HELD_BYTES = {"fp64": 8, "fp32": 4, "fp16dev": 4}
Q_OF = {"D1Q3": 3, "D2Q9": 9, "D3Q19": 19}
KERNEL_SRC = os.path.join(ROOT, "paper_2409_10399_gb300", "csrc", "lbm_kernels.cuh")
# DRAM bytes (read + write) per launch of the box2d FP32 step kernel from one
# ncu capture, valid only for the kernel source it was taken on (the SHA-256
# prefix of lbm_kernels.cuh); otherwise the bench reports traffic null.
NCU_TRAFFIC = {"kernel_source_sha16": "b364f640c0f2b1e3", "bytes_per_launch": 408036352.0}


def bytes_per_node(lattice, prec):
    """Algorithmic bytes of one node update: every population read once and
    written once (6 schemes x Q), plus the three held fields read (their
    writes happen once every n_gamma steps and are not counted)."""
    return 6 * Q_OF[lattice] * 2 * STORE_BYTES[prec] + 3 * HELD_BYTES[prec]


def workload_desc(name):
    w = lbm_inputs.WORKLOADS[name]
    dims = w["dims"]
    return "%s %s %s %s, R=%g, 6 schemes, CGW drag, %s" % (
        name, w["lattice"], "x".join(str(d) for d in dims if d > 1), w["precision"].upper(),
        w["physics"]["R"], "inlet strip" if name == "box2d" else "closed")


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def ncu_traffic():
    """DRAM traffic per launch from the ncu capture of the current kernel
    source, else None."""
    return NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["kernel_source_sha16"] == kernel_hash() else None


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_max(x, dist=None, device="cpu"):
    """Max of a per-rank float over all ranks (the replica timing rule)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank, steps, world, t_max):
    """Whole-job throughput: every rank advances its own replica of
    `nodes_per_rank` nodes for `steps` steps; the job takes the slowest rank's
    time."""
    return world * nodes_per_rank * steps / t_max / 1e6


def replica_seed(base, rank):
    """Each rank's replica starts from its own seeded fields."""
    return base + rank


def _oracle_rate(threads, budget_s):
    """Node updates per second of the FP64 oracle, as it stands, on a 512 x 64
    strip of the box (same physics, inlet strip, walls) with `threads`
    OpenMP threads, for as many steps as fit in about `budget_s` seconds."""
    import oracle
    from oracle import params as oparams
    w = lbm_inputs.WORKLOADS[WORKLOAD]
    nx, ny = w["dims"][0], 64
    f = lbm_inputs.fields_box2d(nx, ny, seed=2)
    o = oracle.Oracle(w["lattice"], (nx, ny, 1), oparams.lattice_params(w["physics"]), threads=threads)
    o.init(**f)
    o.step(2)
    t0 = time.perf_counter()
    o.step(4)
    per = (time.perf_counter() - t0) / 4
    steps = max(4, int(budget_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt, nx, ny, steps


def cpu_baseline(budget_s=10.0):
    """The FP64 oracle on the host cores: all of them (the baseline value) and
    one thread, on the same bounded sample of the workload."""
    cores = os.cpu_count() or 1
    rate, nx, ny, steps = _oracle_rate(cores, budget_s)
    rate1, _, _, steps1 = _oracle_rate(1, budget_s)
    return {"value": rate / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%dx%d strip of the box (inlet strip, walls, same physics), %d steps at %d threads and %d "
                      "at 1, FP64 C, OpenMP" % (nx, ny, steps, cores, steps1),
            "single_thread_value": rate1 / 1e6, "cpu_model": cpu_model()}


def run_reference(args, rank, world):
    """CPU oracle arm: each step is one time step of a bounded sample of the
    same workload, sized so that the whole run ends in a few minutes."""
    if rank != 0:
        return
    import oracle
    from oracle import params as oparams
    w = lbm_inputs.WORKLOADS[WORKLOAD]
    nx = w["dims"][0]
    cores = os.cpu_count() or 1
    po = oparams.lattice_params(w["physics"])
    # calibrate the node-update rate, then size the strip for ~150 s in total
    f = lbm_inputs.fields_box2d(nx, 32, seed=2)
    o = oracle.Oracle(w["lattice"], (nx, 32, 1), po, threads=cores)
    o.init(**f)
    o.step(1)
    t0 = time.perf_counter()
    o.step(3)
    rate = nx * 32 * 3 / (time.perf_counter() - t0)
    total = args.steps + args.warmup
    ny = int(max(4, min(w["dims"][1], 150.0 * rate / max(total, 1) / nx)))
    f = lbm_inputs.fields_box2d(nx, ny, seed=2)
    o = oracle.Oracle(w["lattice"], (nx, ny, 1), po, threads=cores)
    o.init(**f)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = nx * ny * args.steps / dt / 1e6
    sample = "%dx%d strip of the box per step (inlet strip, walls, same physics), FP64 C oracle, OpenMP" % (nx, ny)
    line = {
        "impl": "reference", "metric": "MLUPS (all 6 schemes)", "value": value, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(WORKLOAD), "sampled_nodes": nx * ny},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_native(args, rank, world, local_rank):
    import torch
    import paper_2409_10399_gb300 as lbm
    from paper_2409_10399_gb300 import params as lparams

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = lbm_inputs.WORKLOADS[WORKLOAD]
    lat, dims, prec = w["lattice"], w["dims"], w["precision"]
    N = int(np.prod(dims))
    p = lparams.lattice_params(w["physics"], precision=prec, diag_every=DIAG_EVERY)
    fields = lbm_inputs.fields_for(WORKLOAD, seed=replica_seed(2, rank))
    stream = torch.cuda.current_stream()
    sim = lbm.Simulation(lat, dims, p)
    sim.set_stream(stream)
    sim.init(**fields)
    sim.step(args.warmup)
    torch.cuda.synchronize()

    K = args.steps
    # The timed region: exactly K steps on the library's stream between two
    # events.  The run is cut into segments at the steps after which the
    # library enqueues its diagnostics, with an event at every cut; the step
    # kernel's average launch duration is the time of the segments that hold
    # step kernels only, over their launches.  Before the start event a torch
    # sleep kernel keeps the GPU busy while the launches are queued, so no
    # host gap between launches is timed.
    t0_steps = sim.t
    cuts = sorted(set([0, K] + [k for k in range(K) if (t0_steps + k + 1) % DIAG_EVERY == 0] +
                      [k + 1 for k in range(K) if (t0_steps + k + 1) % DIAG_EVERY == 0]))
    cuts = [k for k in cuts if 0 <= k <= K]
    ev = [torch.cuda.Event(enable_timing=True) for _ in cuts]
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = sim.launches
    t0_wall = time.perf_counter()
    torch.cuda._sleep(2_000_000)
    ev[0].record(stream)
    for j in range(1, len(cuts)):
        sim.step(cuts[j] - cuts[j - 1])
        ev[j].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0_wall
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = sim.launches - l0
    t_total = ev[0].elapsed_time(ev[-1]) / 1e3
    pure_t, pure_n, diag_passes = 0.0, 0, 0
    for j in range(1, len(cuts)):
        n = cuts[j] - cuts[j - 1]
        has_diag = (t0_steps + cuts[j]) % DIAG_EVERY == 0
        diag_passes += int(has_diag)
        if not has_diag:
            pure_t += ev[j - 1].elapsed_time(ev[j]) / 1e3
            pure_n += n
    kern_s = pure_t / pure_n if pure_n else t_total / K
    t_total = reduce_max(t_total, dist, "cuda")
    diag = sim.diag()
    if diag[5] != 0:
        raise RuntimeError("non-finite populations after the timed run")

    # end to end through the C ABI with pinned host buffers: H2D of the
    # initial fields, K steps, D2H of all moments
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hf = {k: pin(v) for k, v in fields.items()}
    D = lbm.LATTICE[lat]
    hout = {k: pin(np.empty(s)) for k, s in (("alpha_g", N), ("u_g", (D, N)), ("u_l", (D, N)), ("p_k", N),
                                               ("S_g", N), ("S_l", N))}
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.init(**hf)
    sim.step(K)
    sim.moments(host_out=hout)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    t_e2e = reduce_max(t_e2e, dist, "cuda")
    h2d = sum(v.nbytes for v in hf.values())
    d2h = sum(v.nbytes for v in hout.values())

    if rank != 0:
        return
    value = aggregate_mlups(N, K, world, t_total)
    bpn = bytes_per_node(lat, prec)
    achieved = N * bpn / kern_s / 1e9
    peak, peak_kind = measured_peak()
    line = {
        "metric": "MLUPS (all 6 schemes)", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": t_total / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else ("f64" if prec == "fp64" else "f16-store/f32"),
        "data": "synthetic",
        "config": {"workload": workload_desc(WORKLOAD), "lattice": lat, "nodes": N, "precision": prec,
                   "diag_every": DIAG_EVERY, "l2": "store %.0f MB > 129 MB L2, no flush" % (N * (6 * Q_OF[lat] * STORE_BYTES[prec] + 3 * HELD_BYTES[prec]) / 1e6),
                   "parallelism": "replicas x%d" % world},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(), "kernel": "k_step<D2Q9,float,float>",
                     "bytes_per_node": bpn, "kernel_ms": kern_s * 1e3, "peak_source": peak_kind},
        "e2e": {"value": aggregate_mlups(N, K, world, t_e2e), "unit": "MLUPS", "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K},
        "gpu_launches": launches,
        "diag_passes_timed": diag_passes,
        "clocks": clk,
        "wall_s": wall,
    }
    sim.close()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_forms:
        from paper_2409_10399_gb300 import forms
        line["forms"] = forms.all_forms(stream, quick=args.quick_forms)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms (FP16, FP64, batch, surrogate)")
    ap.add_argument("--quick-forms", action="store_true", help="the forms' accuracy runs at a tenth of their steps")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
