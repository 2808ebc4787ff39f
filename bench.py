"""Benchmark of the Acc-FEM contact hot path on GB300 (one JSON line on stdout).

Workload (default): 600 mm robot, 300 two-node beam elements, in a 6 mm Catmull-Rom tube
(63,840 triangles); one step = one insertion sweep 0 -> 600 mm in 60 warm-started quasi-static
solves with seeded cable tensions U[0, 5] N.  Metric: solves per second of the plain FP64
single-instance path (every Newton iteration of every solve runs in the library's kernels).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

value  : device-resident inputs (tensions already in HBM), accfem_solve_resident per solve,
         timed with CUDA events on the stream the library launches on; L2 flushed between steps.
e2e    : the same sweeps through accfem_solve with host buffers (H2D of the inputs and D2H of the
         poses and contacts inside the timed region).
--impl reference : the CPU FP64 oracle on the host cores, each step a bounded sample of the sweep.
Multi-GPU (torchrun): independent replicas, one handle per rank, no data-path collective.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "solves/s (plain FP64 single-instance GPU path, 600 mm robot, 300 elements, insertion sweep)"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", type=int, default=0,
                    help="run the first N solves of the sweep once (for profilers) and exit")
    return ap.parse_args()


def workload():
    return wl.catmull_rom_workload(lumen_seed=1, tension_seed=2, n_steps=60)


def config_dict(w, extra=None):
    c = {"workload": "%s insertion sweep 0->600 mm, 60 warm-started solves" % w.name,
         "n_elements": int(w.robot.n_elements), "n_triangles": int(len(w.lumen.triangles)),
         "solves_per_step": int(len(w.insertions)), "tension_seed": 2, "lumen_seed": 1,
         "l2": "flushed between steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, max, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(w, budget_s):
    """The CPU oracle, as it stands, on the first solves of the sweep until budget_s elapses."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import solver
    m = solver.Model(w.robot, w.lumen)
    n = 0
    t0 = time.perf_counter()
    while n < len(w.insertions) and time.perf_counter() - t0 < budget_s:
        m.solve(w.tensions[n], w.insertions[n])
        n += 1
    dt = time.perf_counter() - t0
    return n, dt


def reference_arm(args, rank):
    if rank != 0:
        return 0
    w = workload()
    per_step = 6.0
    for _ in range(args.warmup):
        oracle_sample(w, per_step)
    times, solves = [], 0
    for _ in range(args.steps):
        n, dt = oracle_sample(w, per_step)
        times.append(dt)
        solves += n
    total = sum(times)
    value = solves / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "first solves of the 60-solve sweep (insertion 10 mm upward) for ~%.0f s per "
                                       "step; numpy FP64 oracle, single thread" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Algorithmic FP64 flops per unit (formulas in the design doc, roofline section):
#  element kernel, per element: B (7x12) from Tsinv and G, B E^T, K_l B E^T, the 78 tangent entries
#  and the 12 forces;
#  contact kernel, per launch with m rows and np active rows: the active W columns 6 m np, the
#  elimination of W_PP np^3 and the optimality check 2 m np.
ELEMENT_FLOPS = 2 * (216 + 252 + 168 + 546 + 84 + 120)
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clock x 2 flops x 2.07 GHz (the 1.25 TFLOP/s
# nominal FP64 rate of GB300; a DFMA throughput loop on this machine's GB300 reached 1.20 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def contact_flops(m, npa):
    return 6.0 * m * npa + float(npa) ** 3 + 2.0 * m * npa


def profile_run(args):
    """The first N solves of the sweep, once, on the library's stream (for ncu captures)."""
    import torch
    from paper_2503_06922_gb300 import accfem as af
    w = workload()
    h = af.AccFem(w.robot, w.lumen)
    for s in range(min(args.profile, len(w.insertions))):
        r = h.accfem_solve(w.tensions[s], w.insertions[s])
        print("solve %d status %d newton %d rows %d" % (s, r["status"], r["newton_iters"], r["n_contacts"]), flush=True)
    torch.cuda.synchronize()
    h.close()
    return 0


def ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2503_06922_gb300 import accfem as af
    w = workload()
    h = af.AccFem(w.robot, w.lumen)
    stream = torch.cuda.Stream()
    h.accfem_set_stream(stream.cuda_stream)
    tens_dev = torch.tensor(w.tensions, dtype=torch.float64, device="cuda")
    base = tens_dev.data_ptr()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    S = len(w.insertions)
    row_bytes = 8 * tens_dev.shape[1]

    def sweep_resident(lat=None):
        h.accfem_reset()
        bad = 0
        its = 0
        for s in range(S):
            if lat is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            st, it = h.accfem_solve_resident(base + s * row_bytes, float(w.insertions[s]))
            if lat is not None:
                e1.record(stream)
                lat.append((e0, e1))
            bad += st != af.OK
            its += it
        return bad, its

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sweep_resident()
            flush.fill_(1.0)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches0 = h.accfem_kernel_launches()
        lat = []
        total_ms = 0.0
        fails = 0
        iters = 0
        with ClockSampler(local_rank) as clk:
            for _ in range(args.steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(stream)
                b, it = sweep_resident(lat)
                t1.record(stream)
                t1.synchronize()
                total_ms += t0.elapsed_time(t1)
                fails += b
                iters += it
        torch.cuda.synchronize()
        launches = h.accfem_kernel_launches() - launches0
        solve_ms = np.array([a.elapsed_time(b) for a, b in lat])
        # ---- e2e: host buffers through accfem_solve, copies inside the timed region
        b0 = h.accfem_transfer_bytes()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_fail = 0
        for _ in range(args.steps):
            h.accfem_reset()
            for s in range(S):
                r = h.accfem_solve(w.tensions[s], w.insertions[s])
                e2e_fail += r["status"] != af.OK
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        b1 = h.accfem_transfer_bytes()
        h2d_step = (b1[0] - b0[0]) / args.steps + row_bytes * S
        d2h_step = (b1[1] - b0[1]) / args.steps
        # ---- kernels timed standalone on the resident final state (the last solve of the sweep)
        last = r
        m_last = int(last["n_contacts"])
        np_last = int(sum(1 for c in last["contacts"] if c["force"] > 0.0))
        el_us = h.accfem_time_kernel(af.KERNEL_ELEMENT, 50)
        co_us = h.accfem_time_kernel(af.KERNEL_COLLIDE, 20)
        ct_us = h.accfem_time_kernel(af.KERNEL_CONTACT, 20)
    # max over ranks
    t_max = total_ms
    e2e_max = e2e_s
    if dist:
        tt = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, e2e_max = float(tt[0]), float(tt[1])
    n_solves = S * args.steps * world
    value = n_solves / (t_max / 1000.0)
    e2e_value = n_solves / e2e_max
    nf = w.robot.n_elements
    el_achieved = ELEMENT_FLOPS * nf / (el_us * 1e-6) / 1e12
    achieved = contact_flops(m_last, np_last) / (ct_us * 1e-6) / 1e12
    peak = FP64_PEAK_TFLOPS
    if rank == 0:
        cpu_n, cpu_dt = oracle_sample(w, 15.0)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_dict(w, {"parallelism": "replicas" if world > 1 else "single instance"}),
                "latency_ms": {"p50": float(np.percentile(solve_ms, 50)), "p99": float(np.percentile(solve_ms, 99)),
                               "mean": float(solve_ms.mean())},
                "newton_iters_per_solve": iters / (S * args.steps), "failed_solves": int(fails),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d_step),
                        "d2h_bytes_per_step": int(d2h_step), "failed_solves": int(e2e_fail)},
                "gpu_launches": int(launches),
                "roofline": {"kernel": "contact_kernel (W columns + LCP active-set solve, m=%d rows, %d active)"
                                       % (m_last, np_last),
                             "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s FP64",
                             "frac": achieved / peak, "traffic": None, "launch_us": ct_us,
                             "note": "one-CTA latency-bound FP64 kernel; peak = FP64 rate derived from 152 SMs x "
                                     "2 DFMA/clk x 2.07 GHz (of derived)"},
                "kernel_us": {"element": el_us, "collide": co_us, "contact": ct_us},
                "element_roofline": {"achieved": el_achieved, "peak": peak, "unit": "TFLOP/s FP64",
                                     "frac": el_achieved / peak, "flops_per_element": ELEMENT_FLOPS},
                "clocks": clk.summary(),
                "cpu_baseline": {"value": cpu_n / cpu_dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": "first %d solves of the sweep (insertion 10..%d mm), %.1f s, numpy FP64 "
                                           "oracle, single thread" % (cpu_n, 10 * cpu_n, cpu_dt)}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    h.close()
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank)
    if args.profile:
        return profile_run(args)
    return ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
