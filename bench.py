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
MAX_CONTACTS = 4096         # constraint-row capacity of the benchmark handles
UNIT = "solves/s"


T_START = time.perf_counter()


def _measured_hbm_gbs():
    """HBM copy bandwidth measured on the GB300s (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


MEASURED_HBM_GBS = _measured_hbm_gbs()


def progress(msg):
    """Timestamped progress on stderr (the JSON line alone goes to stdout)."""
    print("[bench %7.1fs] %s" % (time.perf_counter() - T_START, msg), file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", type=int, default=0,
                    help="run the first N solves of the sweep once (for profilers) and exit")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="run N instances of the batched workload through their first steps (for profilers) and exit")
    ap.add_argument("--profile-steps", type=int, default=6, help="steps of --profile-batch")
    ap.add_argument("--profile-kernels", action="store_true",
                    help="run the sweep, then launch the factor group and the contact, element and collision kernels "
                         "twice each on its final state (for profilers) and exit")
    ap.add_argument("--segment", action="store_true", help="with --profile-kernels: segment contacts")
    ap.add_argument("--admm", action="store_true", help="with --profile-kernels: the ADMM contact solver")
    ap.add_argument("--primal", action="store_true",
                    help="with --profile-kernels: the primal ADMM contact solver (first 39 solves of the sweep)")
    ap.add_argument("--profile-phases", action="store_true",
                    help="run the batched workload, then its element, collision and assembly phases as bench times "
                         "them (for profilers) and exit")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched, served, tree-precision and frame-mode measurements")
    ap.add_argument("--frames-only", action="store_true", help="run the frame-mode measurement alone and exit")
    ap.add_argument("--serve-requests", type=int, default=1200, help="requests of each served request stream")
    return ap.parse_args()


def workload():
    return wl.catmull_rom_workload(lumen_seed=1, tension_seed=2, n_steps=60)


def replica_totals(total_ms, e2e_s, units_per_rank, world, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas (one handle per rank, no data-path collective):
    every rank processed units_per_rank solves; the job takes the slowest rank's time, the maximum
    over ranks of the device-timed and end-to-end times (one all_reduce on `device`).  Returns
    (t_max_ms, e2e_max_s, value, e2e_value) with value = all ranks' solves / t_max."""
    t_max, e2e_max = float(total_ms), float(e2e_s)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_max, e2e_max], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, e2e_max = float(tt[0]), float(tt[1])
    n = units_per_rank * world
    return t_max, e2e_max, n / (t_max / 1000.0), n / e2e_max


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


RECORD = os.path.join(ROOT, "oracle", "records", "catmull_rom_600mm_M300_sweep.npz")


BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _restore_env(saved):
    for v, x in saved.items():
        if x is None:
            os.environ.pop(v, None)
        else:
            os.environ[v] = x


def _oracle_iteration_worker(s, n_iters, record, q):
    """One worker of the CPU baseline (a fresh interpreter, spawned with one BLAS thread): the oracle,
    as it stands, starts solve s of the sweep from its own recorded state after solve s - 1 and runs
    n_iters Newton iterations; reports (s, seconds per iteration)."""
    from oracle import solver
    w = workload()
    rec = np.load(record)
    m = solver.Model(w.robot, w.lumen, solver.Options(max_newton_iters=n_iters, max_contacts=MAX_CONTACTS))
    if s > 0:
        m.state = (rec["pos"][s - 1].copy(), rec["rot"][s - 1].copy(), float(w.insertions[s - 1]))
    t0 = time.perf_counter()
    r = m.solve(w.tensions[s], w.insertions[s])
    q.put((s, (time.perf_counter() - t0) / max(r.newton_iters, 1)))


def oracle_sweep_baseline(procs=None, n_iters=1, offset=0.5, picks=None):
    """Throughput of the oracle over the whole 60-solve sweep on the host's cores, from a stratified
    sample: procs worker processes (spawned, one per core, one BLAS thread each) run at the same time,
    worker k timing n_iters Newton iterations of solve s_k = floor((k + offset) S / procs), started
    from the oracle's recorded state after the previous solve (oracle/record_sweep.py).  The seconds
    per iteration are interpolated over the sweep and weighted by the oracle's own iteration count of
    every solve (from the record): T = sum_s iters_s t(s) is the oracle's time for the whole sweep on
    one of procs busy cores, and procs independent sweeps give procs S / T solves/s.  Returns a dict
    or None when a worker did not report."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    if not os.path.exists(RECORD):
        return None
    rec = np.load(RECORD)
    S = len(rec["insertions"])
    if not np.all(rec["status"] == 0):
        return None
    if picks is None:
        picks = sorted({min(S - 1, int(math.floor((k + offset) * S / procs))) for k in range(procs)})
    ps = []
    # one BLAS thread per worker: a spawned interpreter reads these when it imports numpy
    saved = {v: os.environ.get(v) for v in BLAS_THREAD_VARS}
    try:
        os.environ.update({v: "1" for v in BLAS_THREAD_VARS})
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        t0 = time.perf_counter()
        ps = [ctx.Process(target=_oracle_iteration_worker, args=(s, n_iters, RECORD, q)) for s in picks]
        for p in ps:
            p.start()
        _restore_env(saved)
        res = {}
        while len(res) < len(ps):
            try:
                k, v = q.get(timeout=5.0)
                res[k] = v
            except Exception:
                if not any(p.is_alive() for p in ps) and q.empty():
                    raise RuntimeError("a CPU baseline worker exited without reporting")
        wall = time.perf_counter() - t0
    except Exception:
        _restore_env(saved)
        for p in ps:
            if p.is_alive():
                p.terminate()
        return None
    for p in ps:
        p.join(timeout=60)
    xs = np.array(sorted(res))
    t_it = np.interp(np.arange(S), xs, np.array([res[x] for x in xs]))
    T = float(np.sum(rec["newton_iters"] * t_it))
    return {"value": len(picks) * S / T, "cores": len(picks), "sweep_seconds_one_core": T,
            "sampled_solves": [int(x) for x in xs], "seconds_per_iteration": [float(res[x]) for x in xs],
            "wall_s": wall, "oracle_iters_per_solve": float(np.mean(rec["newton_iters"]))}


def reference_arm(args, rank):
    """The oracle as it stands on the host cores (the reference of this comparison): each step one
    stratified sample of the whole sweep (oracle_sweep_baseline, the sample points shifted from step
    to step); the line's value is the mean of the steps' estimates."""
    if rank != 0:
        return 0
    w = workload()
    for k in range(args.warmup):           # every step spawns fresh workers: warm the file cache only
        oracle_sweep_baseline(n_iters=1, picks=[0])
    vals, walls, last = [], [], None
    for k in range(args.steps):
        last = oracle_sweep_baseline(n_iters=2, offset=(k + 0.5) / max(args.steps, 1))
        if last is None:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle's sweep record is missing or a worker "
                                                                  "did not report"}), flush=True)
            return 0
        vals.append(last["value"])
        walls.append(last["wall_s"])
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(walls)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": "per step, %d worker processes (one per host core, one BLAS thread each) at "
                                       "once, each timing two Newton iterations of one solve of the 60-solve sweep "
                                       "(stratified over the sweep, shifted per step) from the oracle's recorded "
                                       "state; seconds per iteration interpolated over the sweep and weighted by the "
                                       "oracle's recorded iterations per solve (%.1f on average); numpy FP64 oracle"
                                       % (last["cores"], last["oracle_iters_per_solve"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Algorithmic FP64 flops per unit:
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


# Algorithmic FP64 flops of the factorisation and the multi-RHS solve of the block-tridiagonal
# system: a 6x6-block Cholesky costs about 560 flop per free node and the forward and backward solve
# about 230 flop per node per right-hand side column (the counts of a plain block Thomas
# factorisation, which the method needs; the cyclic reduction executes more, see factor_flops).
FACTOR_FLOPS_PER_NODE = 560.0
SOLVE_FLOPS_PER_NODE_COLUMN = 230.0


def factor_algorithmic_flops(nf, ncols):
    return FACTOR_FLOPS_PER_NODE * nf + SOLVE_FLOPS_PER_NODE_COLUMN * nf * ncols


def factor_flops(nf, ncols):
    """Executed FP64 flops of the block cyclic reduction factor + solve of nf 6x6-block nodes
    with ncols RHS columns, level by level as the kernels run it: an elimination is a 6x6 inverse
    (216 FMA) plus L = U P and R = U^T P (2 x 216 FMA); a kept-node update is D -= R U + L U^T and
    U <- -L U (3 x 216 FMA); per column, a kept node's forward step is 2 x 36 FMA, the root solve 36,
    an eliminated node's back substitution 3 x 36."""
    fma = 0
    s = 1
    n_elim = 0
    while s < nf:
        kept = (nf - 1) // (2 * s) + 1
        elim = (nf - s - 1) // (2 * s) + 1
        n_elim += elim
        fma += elim * 3 * 216 + kept * 3 * 216 + ncols * kept * 72
        s *= 2
    fma += 216 + ncols * 36 + ncols * n_elim * 108      # root inverse and solve, back substitution
    return 2.0 * fma


def profile_run(args):
    """The first N solves of the sweep, once, on the library's stream (for ncu captures)."""
    import torch
    from paper_2503_06922_gb300 import accfem as af
    w = workload()
    h = af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS)
    for s in range(min(args.profile, len(w.insertions))):
        r = h.accfem_solve(w.tensions[s], w.insertions[s])
        print("solve %d status %d newton %d rows %d" % (s, r["status"], r["newton_iters"], r["n_contacts"]), flush=True)
    torch.cuda.synchronize()
    h.close()
    return 0


MODES = (("fp64", 0), ("mixed", 1))      # name, accfem precision mode


def _one_launch_vs_sequential(af, b, hs, ws, seed=5):
    """The batching comparison of the 256-instance workload: one lock-step batched solve of every
    member (each a tension increment U[-0.2, 0.2] N per cable from its resident state, insertion
    unchanged) against the same solves issued one after another on the single-instance path
    (accfem_solve from the same start pose); both through the public API with host buffers.  Returns
    the times and the largest tip difference between the two."""
    rng = np.random.default_rng(seed)
    n = len(hs)
    saved = [h.accfem_get_state() for h in hs]
    ins = np.array([w.insertions[-1] for w in ws])
    ten = np.maximum(np.array([w.tensions[-1] for w in ws]) + rng.uniform(-0.2, 0.2, (n, 3)), 0.0)
    t0 = time.perf_counter()
    st, sts, res = b.accfem_batch_solve(ten, ins, results=True)
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    seq = [hs[i].accfem_solve(ten[i], ins[i], warm=saved[i]) for i in range(n)]
    t_seq = time.perf_counter() - t0
    tip = max(float(np.linalg.norm(res[i]["node_pos"][-1] - seq[i]["node_pos"][-1])) for i in range(n))
    return {"solves": n, "batched_s": t_batch, "sequential_s": t_seq, "speedup": t_seq / t_batch,
            "batched_failed": int(sum(x != af.OK for x in sts)),
            "sequential_failed": int(sum(r["status"] != af.OK for r in seq)),
            "max_tip_difference_m": tip}


# Algorithmic bytes per item of the batched phases (HBM roofline):
#  element, per element: the node frame it adds to the sweep (7 doubles, each node read by two
#  elements counted once), its stiffness constants (3 doubles) and its record (78 tangent entries and
#  12 forces): (7 + 3 + 90) x 8 = 800 B;
#  assembly, per free node: the element record it reads (90 doubles; each record serves two nodes,
#  counted once) and its block row written (6x6 diagonal block, 6x6 coupling, 6 residual values):
#  (90 + 36 + 36 + 6) x 8 = 1344 B.
PHASE_BYTES = {"element": 800.0, "assemble": 1344.0}
# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum) of the committed
# kernels on the same batch, first Newton iteration of all 256 members (profiles/batch256_phase_dram.md);
# None where no capture of the current kernel exists.
PHASE_DRAM_BYTES = {"element": 7.9e6 + 9.0e6, "collide": 165.1e6 + 4.2e6, "assemble": 172.7e6 + 699.0e6}
# DRAM traffic per launch of the factor group on the final state of the sweep, cold cache (ncu,
# profiles/factor_group_sweep600_M300_dram.md; assemble_rhs + 9 level + 9 back-substitution launches).
FACTOR_DRAM_BYTES = 7.476e6


def _batch_phase_rooflines(af, b, hs, ws, seed=6):
    """HBM fractions of the element, collision and assembly phases of the batch: every member starts one
    more solve (a tension increment from its resident state), the batch advances one Newton iteration,
    and each phase kernel is timed on the plan of the next iteration (all members still iterating, L2
    flushed before every launch); then the solves finish."""
    rng = np.random.default_rng(seed)
    for i, w in enumerate(ws):
        t = np.maximum(np.asarray(w.tensions[-1]) + rng.uniform(-0.2, 0.2, 3), 0.0)
        b.accfem_batch_begin(i, t, w.insertions[-1])
    st, left = b.accfem_batch_advance(1)
    out = {}
    peak = MEASURED_HBM_GBS
    for name, k in (("element", af.KERNEL_ELEMENT), ("collide", af.KERNEL_COLLIDE), ("assemble", af.KERNEL_ASSEMBLE)):
        s2, us, items = b.accfem_batch_time_phase(k, 5)
        if s2 != af.OK:
            out[name] = {"error": b.accfem_batch_last_error()}
            continue
        e = {"us_per_launch": us, "items": items, "members_iterating": left}
        if name in PHASE_BYTES:
            byt = PHASE_BYTES[name] * items
            e.update({"algorithmic_bytes": byt, "bytes_per_item": PHASE_BYTES[name],
                      "achieved_gbs": byt / (us * 1e-6) / 1e9, "peak_gbs": peak,
                      "frac": byt / (us * 1e-6) / 1e9 / peak})
        if PHASE_DRAM_BYTES.get(name) is not None:
            e["traffic"] = PHASE_DRAM_BYTES[name]
            e["dram_gbs"] = PHASE_DRAM_BYTES[name] / (us * 1e-6) / 1e9
        out[name] = e
    while left:
        st, left = b.accfem_batch_advance(200)
    out["note"] = "L2 flushed before each launch; peak = measured copy bandwidth (of measured)"
    return out


def batched_run(af, n_inst=256, chunk=8, seq_sample=16):
    """Uneven batched workload: n_inst instances (element counts log-uniform 50-2000, own lumens,
    target insertion U[0.3, 1] x 600 mm in ~10 mm warm-started steps), every step of every
    instance solved by continuous batching (a member begins its next step as soon as its previous
    one finished; chunk Newton iterations per launch), once with FP64 members and once with mixed
    precision members.  Compared with the plain FP64 single-instance path on every
    (n_inst / seq_sample)-th instance's full sweep, and, after each sweep, one lock-step solve of all
    members against the same solves issued sequentially on the plain path."""
    ws = wl.batch_workloads(n_instances=n_inst)
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS) for w in ws]
    total = sum(len(w.insertions) for w in ws)
    progress("batched: %d instances created, %d solves" % (n_inst, total))
    # every step of every instance as a request at time 0: the native server runs each member's
    # steps in order and admits a member's next step as soon as its previous one finished
    mem = np.concatenate([np.full(len(w.insertions), i) for i, w in enumerate(ws)])
    step = np.concatenate([np.arange(len(w.insertions)) for w in ws])
    ten = np.array([ws[i].tensions[k] for i, k in zip(mem, step)])
    ins = np.array([ws[i].insertions[k] for i, k in zip(mem, step)])
    out = {"workload": "%d uneven instances: elements log-uniform 50-2000, own Catmull-Rom lumens, target insertion "
                       "U[0.3,1] x 600 mm in ~10 mm warm-started steps (%d solves)" % (n_inst, total),
           "chunk_iters": chunk}
    for name, mode in MODES:
        for h in hs:
            h.accfem_reset()
            h.accfem_set_precision(mode)
        b = af.AccFemBatch(hs)
        # autotuning before the timed run, on work of the run's own size: every instance solves its
        # last step (full insertion) from the straight pose, two Newton iterations per launch, until
        # every variant has been timed twice; then the instances start over
        b.accfem_batch_autotune(2)
        last = np.array([len(w.insertions) - 1 for w in ws])
        sel = np.array([np.nonzero((mem == i) & (step == last[i]))[0][0] for i in range(len(ws))])
        for _ in range(4):
            b.accfem_batch_serve(np.zeros(len(sel)), mem[sel], ten[sel], ins[sel], chunk_iters=2)
            if b.accfem_batch_tuning()[0] >= 0:
                break
            for h in hs:
                h.accfem_reset()
        for h in hs:
            h.accfem_reset()
        l0 = b.accfem_batch_kernel_launches()
        res = b.accfem_batch_serve(np.zeros(total), mem, ten, ins, chunk_iters=chunk)
        dt = float(res["t_end"].max())
        variant, ms_pass = b.accfem_batch_tuning()
        launches = b.accfem_batch_kernel_launches() - l0
        lat = (res["t_end"] - res["t_begin"]) * 1e3
        fails = int(np.sum(res["status"] != af.OK))
        progress("batched %s: served in %.1f s, %d failed" % (name, dt, fails))
        one = _one_launch_vs_sequential(af, b, hs, ws)
        progress("batched %s: one launch of %d solves %.3f s, sequential %.3f s" % (name, n_inst, one["batched_s"],
                                                                                  one["sequential_s"]))
        phases = _batch_phase_rooflines(af, b, hs, ws) if name == "fp64" else None
        out[name] = {"solves_per_s": total / dt, "seconds": dt, "phase_roofline": phases,
                     "autotune": {"variant": variant, "grid_divisor": 2 ** (max(variant, 0) % 4),
                                  "element_warps_per_block": 2 << (max(variant, 0) // 4),
                                  "ms_per_iteration_by_variant": [float(x) for x in ms_pass]},
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                     "newton_iters_per_solve": float(np.mean(res["newton_iters"])), "failed_solves": fails,
                     "status_counts": {af.accfem_status_string(int(k)): int(v)
                                       for k, v in zip(*np.unique(res["status"], return_counts=True))},
                     "gpu_launches": int(launches), "one_launch_vs_sequential": one}
        b.close()
    for h in hs:
        h.accfem_set_precision(0)
    # plain path: full sweeps of a sample of the instances, one solve at a time
    sample = list(range(0, n_inst, max(1, n_inst // seq_sample)))
    t1 = time.perf_counter()
    cnt, seq_fail = 0, 0
    for i in sample:
        hs[i].accfem_reset()
        for s in range(len(ws[i].insertions)):
            r = hs[i].accfem_solve(ws[i].tensions[s], ws[i].insertions[s])
            cnt += 1
            seq_fail += r["status"] != af.OK
    seq_dt = time.perf_counter() - t1
    progress("batched: plain sample %d solves in %.1f s" % (cnt, seq_dt))
    for h in hs:
        h.close()
    plain = cnt / seq_dt
    out["plain_sequential"] = {"solves_per_s": plain, "solves": cnt, "failed_solves": int(seq_fail),
                               "sample": "full sweeps of instances %s" % sample[:4] + "... every %d-th" % (n_inst // seq_sample)}
    out["multiple_over_plain_fp64"] = {name: out[name]["solves_per_s"] / plain for name, _ in MODES}
    return out


def served_run(af, rates=(100.0, 200.0, 2000.0, 5000.0, 10000.0), requests=1200, seconds_min=6.0, n_scenes=16, chunk=4,
               plain_requests=300):
    """Serving: n_scenes resident scenes drawn as in the batched workload, each first swept to its
    target insertion; per rate a Poisson request stream (tension increments +-0.2 N per cable or
    insertion steps of +-0.5 mm) of `requests` requests, or of seconds_min seconds where that holds fewer
    requests (the rates below the server's capacity), served in real time by accfem_batch_serve, with FP64 scenes and with mixed-precision scenes.  The
    plain FP64 path serves the first plain_requests requests of the same stream one at a time
    (measured solve times, FIFO queue at the same arrival times)."""
    ws = wl.batch_workloads(n_instances=256, count=n_scenes)
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS) for w in ws]
    ps = [af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS) for w in ws]
    S = max(len(w.insertions) for w in ws)
    lengths = [w.robot.length for w in ws]
    streams = [(rate, 100 + k, min(requests / rate, seconds_min)) for k, rate in enumerate(rates)]

    def sweep_in(b):
        for s in range(S):
            mask = [1 if s < len(w.insertions) else 0 for w in ws]
            t = [w.tensions[min(s, len(w.insertions) - 1)] for w in ws]
            ins = [w.insertions[min(s, len(w.insertions) - 1)] for w in ws]
            b.accfem_batch_solve(t, ins, mask=mask, results=False)

    out = {}
    # plain FP64 path: the same scenes, swept in, then the first requests of each stream one at a time
    for i, w in enumerate(ws):
        for s in range(len(w.insertions)):
            ps[i].accfem_solve(w.tensions[s], w.insertions[s])
    ten0 = np.array([w.tensions[-1] for w in ws])
    ins0 = np.array([w.insertions[-1] for w in ws])
    plain = []
    for rate, seed, dur in streams:
        arr, sc, ten, ins = wl.serve_trace(ten0, ins0, lengths, rate, dur, seed=seed)
        npl = min(plain_requests, len(arr))
        svc = np.zeros(npl)
        for j in range(npl):
            t0 = time.perf_counter()
            ps[sc[j]].accfem_solve(ten[j], ins[j])
            svc[j] = time.perf_counter() - t0
        fin = np.zeros(npl)
        tprev = 0.0
        for j in range(npl):
            tprev = max(arr[j], tprev) + svc[j]
            fin[j] = tprev
        plat = (fin - arr[:npl]) * 1e3
        plain.append({"requests": int(npl), "capacity_solves_per_s": npl / svc.sum(),
                      "service_ms": {"p50": float(np.percentile(svc * 1e3, 50)), "p99": float(np.percentile(svc * 1e3, 99))},
                      "latency_ms": {"p50": float(np.percentile(plat, 50)), "p99": float(np.percentile(plat, 99))}})
        progress("served: plain path, rate %.0f, %d requests in %.1f s" % (rate, npl, svc.sum()))
        # every stream starts from the swept-in scenes: one solve of each at its final command
        for i, w in enumerate(ws):
            ps[i].accfem_solve(w.tensions[-1], w.insertions[-1])
    for name, mode in MODES:
        for h in hs:
            h.accfem_reset()
            h.accfem_set_precision(mode)
        b = af.AccFemBatch(hs)
        rows = []
        l0 = b.accfem_batch_kernel_launches()
        sweep_in(b)
        for (rate, seed, dur), pl in zip(streams, plain):
            # every stream starts from the swept-in scenes: one solve of each at its final command
            b.accfem_batch_solve([w.tensions[-1] for w in ws], [w.insertions[-1] for w in ws], results=False)
            arr, sc, ten, ins = wl.serve_trace(ten0, ins0, lengths, rate, dur, seed=seed)
            res = b.accfem_batch_serve(arr, sc, ten, ins, chunk_iters=chunk, hbm_cap_bytes=40 * 1024 ** 3)
            span = float(res["t_end"].max()) if len(arr) else 0.0
            lat = res["latency"] * 1e3
            p99 = float(np.percentile(lat, 99))
            sps = len(arr) / max(span, 1e-9)
            rows.append({"offered_req_per_s": rate, "requests": int(len(arr)), "stream_s": dur, "solves_per_s": sps,
                         "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": p99},
                         "newton_iters_per_solve": float(res["newton_iters"].mean()),
                         "failed_solves": int(np.sum(res["status"] != af.OK)),
                         "status_counts": {af.accfem_status_string(int(k)): int(v)
                                           for k, v in zip(*np.unique(res["status"], return_counts=True))},
                         "throughput_multiple_over_plain_fp64": sps / pl["capacity_solves_per_s"],
                         "p99_multiple_of_plain_fp64": p99 / pl["latency_ms"]["p99"]})
            progress("served %s: rate %.0f, %d requests, %.0f solves/s, p99 %.1f ms" % (name, rate, len(arr), sps, p99))
        out[name] = {"rates": rows, "gpu_launches": int(b.accfem_batch_kernel_launches() - l0)}
        b.close()
    for h in hs + ps:
        h.close()
    out["plain_fp64"] = [dict(p, offered_req_per_s=r[0]) for p, r in zip(plain, streams)]
    out["workload"] = ("%d scenes as in the batched workload, swept to their target insertion; per rate a Poisson "
                       "stream of %d requests or %.0f s (the shorter), tension increments U[-0.2,0.2] N per cable or "
                       "insertion steps +-0.5 mm; every stream starts from the swept-in scenes"
                       % (n_scenes, requests, seconds_min))
    out["chunk_iters"] = chunk
    out["hbm_cap_gb"] = 40
    out["multiples"] = ("throughput_multiple_over_plain_fp64 = served solves/s / plain FP64 capacity on the same "
                        "stream; p99_multiple_of_plain_fp64 = served p99 / plain FP64 p99 (FIFO, same arrivals)")
    return out


def same_rows(ca, cb, tol=1e-9):
    """Two contact sets agree: per node the same number of rows, and their closest points pair up
    within tol (rows of one node sorted by point)."""
    def group(cs):
        g = {}
        for c in cs:
            g.setdefault(c["node"], []).append(np.asarray(c["point"], dtype=np.float64))
        return {n: sorted(v, key=lambda x: tuple(x)) for n, v in g.items()}
    ga, gb = group(ca), group(cb)
    if set(ga) != set(gb):
        return False
    for n in ga:
        if len(ga[n]) != len(gb[n]):
            return False
        used = [False] * len(gb[n])
        for pa in ga[n]:
            k = next((j for j, pb in enumerate(gb[n]) if not used[j] and np.linalg.norm(pa - pb) <= tol), -1)
            if k < 0:
                return False
            used[k] = True
    return True


def tree_precision_run(af):
    """The precision configuration: 2000-element robot in the seeded 3-generation branching tube tree
    (~388k triangles), insertion swept to 0.9 x the shortest root-to-leaf path in ~10 mm steps, once in
    FP64 and once with the FP32 element tangent; every solve compared (no CPU oracle at this size: the
    FP64 GPU path, which matches the oracle on the smaller workloads, is the reference)."""
    w = wl.tree_workload()
    out = {}
    runs = {}
    for mode in (af.PRECISION_FP64, af.PRECISION_MIXED):
        h = af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS, max_contact_iters=5000)
        h.accfem_set_precision(mode)
        res, fb, t0 = [], 0, time.perf_counter()
        for s in range(len(w.insertions)):
            res.append(h.accfem_solve(w.tensions[s], w.insertions[s]))
            fb += h.accfem_solve_stats()[3]
        dt = time.perf_counter() - t0
        runs[mode] = res
        out["fp64" if mode == af.PRECISION_FP64 else "mixed"] = {
            "solves_per_s": len(res) / dt, "newton_iters_per_solve": float(np.mean([r["newton_iters"] for r in res])),
            "failed_solves": int(sum(r["status"] != af.OK for r in res)),
            "max_rows": int(max(r["n_contacts"] for r in res)), "fp64_tangent_fallbacks": int(fb),
            "per_solve": [[int(r["status"]), int(r["newton_iters"]), int(r["n_contacts"])] for r in res]}
        h.close()
    tip, ferr, same, both = 0.0, 0.0, 0, 0
    for r6, rm in zip(runs[af.PRECISION_FP64], runs[af.PRECISION_MIXED]):
        if r6["status"] != af.OK or rm["status"] != af.OK:
            continue
        both += 1
        tip = max(tip, float(np.linalg.norm(rm["node_pos"][-1] - r6["node_pos"][-1])))
        same += same_rows(rm["contacts"], r6["contacts"])
        f6, fm = {}, {}
        for c in r6["contacts"]:
            f6[c["node"]] = f6.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
        for c in rm["contacts"]:
            fm[c["node"]] = fm.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
        fmax = max([np.linalg.norm(v) for v in f6.values()] + [1e-300])
        for n in set(f6) | set(fm):
            ferr = max(ferr, float(np.linalg.norm(f6.get(n, 0.0) - fm.get(n, 0.0))) / fmax)
    out["workload"] = ("%s: 2000 elements, %d triangles, insertion to %.0f mm in %d steps (e2e through accfem_solve)"
                       % (w.name, len(w.lumen.triangles), 1e3 * w.insertions[-1], len(w.insertions)))
    out["mixed_vs_fp64"] = {"solves_compared": both, "max_tip_error_m": tip, "max_node_force_rel_error": ferr,
                            "identical_contact_sets": int(same)}
    progress("precision tree: fp64 %.1f, mixed %.1f solves/s, tip error %.2e m" %
             (out["fp64"]["solves_per_s"], out["mixed"]["solves_per_s"], tip))
    return out


def frames_run(af, node_counts=(100, 200, 300, 400), frames_per_step=5, solver=None):
    """The paper's per-timestep experiment (Sec. IV.A: computation time per timestep against the
    number of contacts, robots of 100, 200, 300 and 400 nodes) in frame mode, one linearisation of
    Eq. 20-23 per frame: the 600 mm robot with 99..399 elements in the benchmark's Catmull-Rom tube,
    insertion swept 0 -> 600 mm in 60 steps of frames_per_step frames each.  Per frame: the device
    time of one accfem_solve_resident call (CUDA events on the library's stream; graph launch,
    iteration and control read-back) and the rows active in its contact solve.  solver: the contact
    solver (default the active-set method); with the ADMM solvers, the ADMM iterations per frame."""
    import torch
    from dataclasses import replace
    w0 = workload()
    S = len(w0.insertions)
    tens = torch.tensor(w0.tensions, dtype=torch.float64, device="cuda")
    row_bytes = 8 * tens.shape[1]
    bins = ((0, 0), (1, 4), (5, 9), (10, 19), (20, 10 ** 6))
    out = {}
    for nn in node_counts:
        rob = replace(w0.robot, n_elements=nn - 1)
        h = af.AccFem(rob, w0.lumen, max_contacts=512)
        h.accfem_set_frame_mode(1)
        if solver is not None:
            h.accfem_set_contact_solver(solver)
        stream = torch.cuda.Stream()
        h.accfem_set_stream(stream.cuda_stream)
        recs = []
        with torch.cuda.stream(stream):
            for rep in range(2):                 # the first pass captures the graphs
                h.accfem_reset()
                for s in range(S):
                    for f in range(frames_per_step):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        st, it = h.accfem_solve_resident(tens.data_ptr() + s * row_bytes, float(w0.insertions[s]))
                        e1.record(stream)
                        e1.synchronize()
                        if rep == 1:
                            rows, working, active, _ = h.accfem_solve_stats()
                            recs.append((e0.elapsed_time(e1), active, rows, st, h.accfem_solve_admm_iterations()))
        h.close()
        ms = np.array([r[0] for r in recs])
        act = np.array([r[1] for r in recs])
        by = {}
        for lo, hi in bins:
            sel = (act >= lo) & (act <= hi)
            if sel.any():
                by["%d-%d" % (lo, hi) if hi < 10 ** 6 else "%d+" % lo] = {
                    "frames": int(sel.sum()), "ms_mean": float(ms[sel].mean()),
                    "admm_iters_mean": float(np.mean([recs[i][4] for i in np.nonzero(sel)[0]]))}
        out[str(nn)] = {"frames": len(recs), "ms_per_frame": float(ms.mean()), "ms_p50": float(np.percentile(ms, 50)),
                        "ms_p99": float(np.percentile(ms, 99)), "frames_per_s": float(1e3 / ms.mean()),
                        "max_active": int(act.max()), "max_rows": int(max(r[2] for r in recs)),
                        "failed": int(sum(r[3] != af.OK for r in recs)), "ms_by_active_contacts": by}
        progress("frames: %d nodes, %.3f ms per frame, up to %d active contacts" % (nn, ms.mean(), act.max()))
    out["workload"] = ("600 mm robot in %s, insertion 0->600 mm in %d steps x %d frames, one Newton iteration per "
                       "frame (frame mode)" % (w0.name, S, frames_per_step))
    return out


def config0_run(af, seeds=100):
    """The small plain configuration: the 120 mm, 20-element robot in the 5 mm bent tube, one tension
    triple U[0, 3] N per seed (seeds 0..99), insertion ramped 10 -> 100 mm in 10 warm-started solves
    per seed; FP64, device-resident tensions (accfem_solve_resident), CUDA events on the library's
    stream around each solve."""
    import torch
    ws = [wl.bent_tube_workload(s, n_steps=10) for s in range(seeds)]
    w0 = ws[0]
    h = af.AccFem(w0.robot, w0.lumen)
    stream = torch.cuda.Stream()
    h.accfem_set_stream(stream.cuda_stream)
    tens = torch.tensor(np.array([w.tensions[0] for w in ws]), dtype=torch.float64, device="cuda")
    row = 8 * tens.shape[1]
    recs = []
    with torch.cuda.stream(stream):
        for rep in range(2):                  # the first pass captures the Newton graphs
            recs = []
            for si, w in enumerate(ws):
                h.accfem_reset()
                for s in range(len(w.insertions)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st, it = h.accfem_solve_resident(tens.data_ptr() + si * row, float(w.insertions[s]))
                    e1.record(stream)
                    recs.append((e0, e1, st, it, s))
            torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b, _, _, _ in recs])
        final = np.array([r[4] == 9 for r in recs])
        h.accfem_reset()
        act = []
        for si, w in enumerate(ws[:20]):
            for s in range(len(w.insertions)):
                h.accfem_solve_resident(tens.data_ptr() + si * row, float(w.insertions[s]))
            act.append(h.accfem_solve_stats()[2])
    h.close()
    return {"workload": "%s in the 5 mm bent tube, tension seeds 0..%d (U[0,3] N), insertion 10 -> 100 mm in 10 "
                        "warm-started solves per seed" % (w0.name, seeds - 1),
            "solves": len(recs), "solves_per_s": len(recs) / (ms.sum() * 1e-3),
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "final_solve_latency_ms": {"p50": float(np.percentile(ms[final], 50)),
                                       "p99": float(np.percentile(ms[final], 99))},
            "newton_iters_per_solve": float(np.mean([r[3] for r in recs])),
            "failed_solves": int(sum(r[2] != af.OK for r in recs)),
            "active_contacts_at_100mm": {"min": int(min(act)), "max": int(max(act)), "seeds": len(act)}}


def profile_kernels_run(args):
    """The whole sweep in the device-side graph loop (kernels hidden from profilers), then, launched
    from the host on the final state of the sweep as bench times them, the factor group (assembly,
    reduction levels, back substitution) and the contact, element and collision kernels, twice each
    (for ncu captures)."""
    import torch
    from paper_2503_06922_gb300 import accfem as af
    w = workload()
    h = af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS)
    if args.segment:
        h.accfem_set_contact_model(af.CONTACT_SEGMENT)
    if args.admm:
        h.accfem_set_contact_solver(af.CONTACT_ADMM)
    if args.primal:
        h.accfem_set_contact_solver(af.CONTACT_PRIMAL_ADMM)
    n_solves = 39 if args.primal else len(w.insertions)   # the primal ADMM takes ~80 ms per solve
    for s in range(n_solves):
        h.accfem_solve(w.tensions[s], w.insertions[s])
    for name, k in (("factor group", af.KERNEL_FACTOR), ("contact", af.KERNEL_CONTACT), ("element", af.KERNEL_ELEMENT),
                    ("collide", af.KERNEL_COLLIDE)):
        print("%s: %.1f us per launch" % (name, h.accfem_time_kernel(k, 1)), flush=True)
    print("rows, working set, active: %s" % (h.accfem_solve_stats(),), flush=True)
    torch.cuda.synchronize()
    h.close()
    return 0


def profile_phases_run(args):
    """The batched workload (256 uneven instances, all steps, continuous batching in the graph loop);
    then a second batch over the same members with host-launched phase kernels (visible to
    profilers): every member begins a tension increment, one Newton iteration of all of them runs
    inside the NVTX range "iteration", and the element, collision and assembly phases are timed on
    the next iteration's plan as the bench's phase roofline does, inside the range "phases"."""
    import torch
    from paper_2503_06922_gb300 import accfem as af
    ws = wl.batch_workloads(n_instances=256)
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS) for w in ws]
    b = af.AccFemBatch(hs)
    mem = np.concatenate([np.full(len(w.insertions), i) for i, w in enumerate(ws)])
    step = np.concatenate([np.arange(len(w.insertions)) for w in ws])
    ten = np.array([ws[i].tensions[k] for i, k in zip(mem, step)])
    ins = np.array([ws[i].insertions[k] for i, k in zip(mem, step)])
    b.accfem_batch_serve(np.zeros(len(mem)), mem, ten, ins, chunk_iters=8)
    b.close()
    os.environ["ACCFEM_LAUNCH"] = "stream"
    b2 = af.AccFemBatch(hs)
    del os.environ["ACCFEM_LAUNCH"]
    rng = np.random.default_rng(7)
    for i, w in enumerate(ws):
        b2.accfem_batch_begin(i, np.maximum(np.asarray(w.tensions[-1]) + rng.uniform(-0.2, 0.2, 3), 0.0), w.insertions[-1])
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("iteration")
    st, left = b2.accfem_batch_advance(1)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print("one iteration of %d members, %d left" % (len(ws), left), flush=True)
    torch.cuda.nvtx.range_push("phases")
    out = {}
    for name, k in (("element", af.KERNEL_ELEMENT), ("collide", af.KERNEL_COLLIDE), ("assemble", af.KERNEL_ASSEMBLE)):
        st, us, items = b2.accfem_batch_time_phase(k, 3)
        out[name] = {"status": st, "us": us, "items": items}
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps(out), flush=True)
    while left:
        st, left = b2.accfem_batch_advance(200)
    b2.close()
    for h in hs:
        h.close()
    return 0


def profile_batch_run(args):
    """The first steps of the first N instances of the batched workload, in one batch (for ncu
    captures; with ACCFEM_LAUNCH=stream the phase kernels are launched from a host loop)."""
    import torch
    from paper_2503_06922_gb300 import accfem as af
    ws = wl.batch_workloads(n_instances=256, count=args.profile_batch)
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS) for w in ws]
    b = af.AccFemBatch(hs)
    for s in range(args.profile_steps):
        st, sts, _ = b.accfem_batch_solve([w.tensions[s] for w in ws], [w.insertions[s] for w in ws], results=False)
        print("step %d status %d launches %d" % (s, st, b.accfem_batch_kernel_launches()), flush=True)
    torch.cuda.synchronize()
    b.close()
    for h in hs:
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
    h = af.AccFem(w.robot, w.lumen, max_contacts=MAX_CONTACTS)
    stream = torch.cuda.Stream()
    h.accfem_set_stream(stream.cuda_stream)
    tens_dev = torch.tensor(w.tensions, dtype=torch.float64, device="cuda")
    base = tens_dev.data_ptr()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    S = len(w.insertions)
    row_bytes = 8 * tens_dev.shape[1]

    def sweep_resident(lat=None, admm=None):
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
            if admm is not None:
                admm.append(h.accfem_solve_admm_iterations())
            bad += st != af.OK
            its += it
        return bad, its

    progress("plain sweep: warm-up")
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
        progress("plain sweep: timed %d steps, %.1f ms/step, %d failed" % (args.steps, total_ms / args.steps, fails))
        # ---- e2e: host buffers through accfem_solve, copies inside the timed region
        b0 = h.accfem_transfer_bytes()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_fail = 0
        last_ok = 0
        fp64_runs = None
        for _ in range(args.steps):
            h.accfem_reset()
            fp64_runs = []
            for s in range(S):
                r = h.accfem_solve(w.tensions[s], w.insertions[s])
                e2e_fail += r["status"] != af.OK
                fp64_runs.append(r)
                if r["status"] == af.OK:
                    last_ok = s
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        b1 = h.accfem_transfer_bytes()
        h2d_step = (b1[0] - b0[0]) / args.steps + row_bytes * S
        d2h_step = (b1[1] - b0[1]) / args.steps
        # ---- kernels timed standalone on the resident state of the last converged solve of the sweep
        if r["status"] != af.OK:
            h.accfem_reset()
            for s in range(last_ok + 1):
                r = h.accfem_solve(w.tensions[s], w.insertions[s])
        last = r
        m_last, mc_last, np_last, _fb = h.accfem_solve_stats()
        nf_last = w.robot.n_elements - int(math.floor((w.robot.length - w.insertions[last_ok]) * w.robot.n_elements
                                                      / w.robot.length + 1e-6))
        # replayed from one CUDA graph (the kernels chained as in the Newton loop) for the rooflines;
        # host-issued launches beside them, for comparison
        el_us = h.accfem_time_kernel_graph(af.KERNEL_ELEMENT, 50)
        co_us = h.accfem_time_kernel_graph(af.KERNEL_COLLIDE, 20)
        ct_us = h.accfem_time_kernel_graph(af.KERNEL_CONTACT, 20)
        fa_us = h.accfem_time_kernel_graph(af.KERNEL_FACTOR, 20)
        host_us = {"element": h.accfem_time_kernel(af.KERNEL_ELEMENT, 50),
                   "collide": h.accfem_time_kernel(af.KERNEL_COLLIDE, 20),
                   "contact": h.accfem_time_kernel(af.KERNEL_CONTACT, 20),
                   "factor_group": h.accfem_time_kernel(af.KERNEL_FACTOR, 20)}
        # ---- the paper's contact scheme (OSQP's ADMM guess, then the exact polish): the same sweep,
        #      timed like `value`, and the contact kernel on the final state of the sweep
        progress("contact solver: ADMM sweep")
        h.accfem_set_contact_solver(af.CONTACT_ADMM)
        admm_ms, admm_fail, admm_iters, admm_inner = 0.0, 0, 0, []
        with torch.cuda.stream(stream):
            sweep_resident(admm=admm_inner)      # warm-up, and the ADMM iterations of every solve
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            admm_fail, admm_iters = sweep_resident()
            t1.record(stream)
            t1.synchronize()
            admm_ms = t0.elapsed_time(t1)
        admm_ct_us = h.accfem_time_kernel(af.KERNEL_CONTACT, 5)
        h.accfem_set_contact_solver(af.CONTACT_ACTIVE_SET)
        contact_admm = {"scheme": "OSQP ADMM on the contact-space QP over the working set (FP32 iterations, "
                                  "W + (sigma + rho) I inverted once), guess of the free rows polished by the "
                                  "exact FP64 active-set method",
                        "solves_per_s": S / (admm_ms * 1e-3), "ms_per_step": admm_ms,
                        "newton_iters_per_solve": admm_iters / S, "failed_solves": int(admm_fail),
                        "admm_iters_per_newton_iter": sum(admm_inner) / max(admm_iters, 1),
                        "contact_kernel_us_final_state": admm_ct_us, "active_set_contact_kernel_us": ct_us}
        progress("contact solver: ADMM %.1f solves/s, contact kernel %.0f us (active set %.0f us)"
                 % (contact_admm["solves_per_s"], admm_ct_us, ct_us))
        # ---- segment contacts (Eq. 3-7 at any point of an element): the same sweep, timed like `value`
        progress("segment contacts: sweep")
        h.accfem_set_contact_model(af.CONTACT_SEGMENT)
        with torch.cuda.stream(stream):
            sweep_resident()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            seg_fail, seg_iters = sweep_resident()
            t1.record(stream)
            t1.synchronize()
            seg_ms = t0.elapsed_time(t1)
        seg_rows = h.accfem_solve_stats()
        seg_coll_us = h.accfem_time_kernel(af.KERNEL_COLLIDE, 20)
        h.accfem_set_contact_model(af.CONTACT_NODE)
        segment_contacts = {"model": "contact points anywhere on an element's chord, displacement by N(xi) of Eq. 4-6 "
                                     "in the element frame; rows per element (chord against triangles)",
                            "solves_per_s": S / (seg_ms * 1e-3), "ms_per_step": seg_ms,
                            "newton_iters_per_solve": seg_iters / S, "failed_solves": int(seg_fail),
                            "rows_working_active_final": list(seg_rows[:3]), "collide_us_final_state": seg_coll_us}
        progress("segment contacts: %.1f solves/s, %d failed" % (segment_contacts["solves_per_s"], seg_fail))
        # ---- mixed precision: the same sweep with the FP32 element tangent, timed like `value`, and
        #      every solve compared with the FP64 solve of the same step
        progress("precision: mixed sweep")
        h.accfem_set_precision(af.PRECISION_MIXED)
        sweep_resident()
        mixed_ms, mixed_fail, mixed_iters = 0.0, 0, 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            b_, it_ = sweep_resident()
            t1.record(stream)
            t1.synchronize()
            mixed_ms += t0.elapsed_time(t1)
            mixed_fail += b_
            mixed_iters += it_
        h.accfem_reset()
        tip_err, force_err, same_sets, both_ok, fallbacks = 0.0, 0.0, 0, 0, 0
        for s in range(S):
            rm = h.accfem_solve(w.tensions[s], w.insertions[s])
            fallbacks += h.accfem_solve_stats()[3]
            r6 = fp64_runs[s]
            if rm["status"] != af.OK or r6["status"] != af.OK:
                continue
            both_ok += 1
            tip_err = max(tip_err, float(np.linalg.norm(rm["node_pos"][-1] - r6["node_pos"][-1])))
            same_sets += same_rows(rm["contacts"], r6["contacts"])
            fm, f6 = {}, {}
            for c in rm["contacts"]:
                fm[c["node"]] = fm.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
            for c in r6["contacts"]:
                f6[c["node"]] = f6.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"])
            fmax = max([np.linalg.norm(v) for v in f6.values()] + [1e-300])
            for n in set(fm) | set(f6):
                force_err = max(force_err, float(np.linalg.norm(fm.get(n, 0.0) - f6.get(n, 0.0))) / fmax)
        h.accfem_set_precision(af.PRECISION_FP64)
        precision = {"mode": "mixed: FP32 element tangent (FP32 operands and accumulation); FP64 element force, "
                             "residual, factor, contact Schur complement and contact solve",
                     "solves_per_s": S * args.steps / (mixed_ms / 1000.0),
                     "ms_per_step": mixed_ms / args.steps, "newton_iters_per_solve": mixed_iters / (S * args.steps),
                     "failed_solves": int(mixed_fail), "fp64_tangent_fallbacks": int(fallbacks),
                     "vs_fp64_gpu": {"solves_compared": both_ok, "max_tip_error_m": tip_err,
                                     "max_node_force_rel_error": force_err, "identical_contact_sets": int(same_sets)}}
        progress("precision: %.1f solves/s, tip error %.2e m" % (precision["solves_per_s"], tip_err))
    t_max, e2e_max, value, e2e_value = replica_totals(total_ms, e2e_s, S * args.steps, world, dist, "cuda")
    nf = w.robot.n_elements
    el_achieved = ELEMENT_FLOPS * nf / (el_us * 1e-6) / 1e12
    ct_achieved = contact_flops(mc_last, np_last) / (ct_us * 1e-6) / 1e12
    fa_flops = factor_algorithmic_flops(nf_last, 1 + mc_last)
    fa_exec = factor_flops(nf_last, 1 + mc_last)
    achieved = fa_flops / (fa_us * 1e-6) / 1e12
    peak = FP64_PEAK_TFLOPS
    extra = {}
    if rank == 0:
        extra["config0"] = config0_run(af)
        progress("config0: %.0f solves/s" % extra["config0"]["solves_per_s"])
    if rank == 0 and not args.no_extra:
        extra["batched"] = batched_run(af)
        extra["served"] = served_run(af, requests=args.serve_requests)
        extra["precision_tree"] = tree_precision_run(af)
        extra["frames"] = frames_run(af)
        # the paper's own solver of Eq. 23 (OSQP on the primal QP), frame by frame: its time per frame
        # against the number of contacts (the claim of Sec. IV.A)
        fp = frames_run(af, node_counts=(100, 300), frames_per_step=1, solver=af.CONTACT_PRIMAL_ADMM)
        fp["solver"] = ("OSQP's ADMM on the primal QP of Eq. 23 (K + sigma I + rho A^T A factored per frame by a "
                        "one-CTA block cyclic reduction, one 1-column solve per ADMM iteration), guess polished "
                        "exactly by the active-set method")
        extra["frames_primal_admm"] = fp
    if rank == 0:
        cpu = oracle_sweep_baseline(n_iters=2)
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
                "roofline": {"kernel": "assembly + block cyclic reduction factor and solve (assemble_rhs with the level-1 eliminations, "
                                       "bcr_level x levels, bcr_bwd x levels; nf=%d nodes, %d RHS columns)"
                                       % (nf_last, 1 + mc_last),
                             "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s FP64",
                             "frac": achieved / peak, "traffic": FACTOR_DRAM_BYTES, "launch_us": fa_us,
                             "launch_timing": "CUDA events around one replay of a CUDA graph holding 20 group "
                                              "launches in sequence, as the Newton loop chains them (%.1f us per "
                                              "group with host-issued launches)" % host_us["factor_group"],
                             "traffic_note": "ncu dram bytes per group launch at cold cache (the timed loop keeps "
                                             "the 11 MB working set in L2)",
                             "flops_per_launch": fa_flops, "executed_flops_per_launch": fa_exec,
                             "flops_rule": "560 flop per free node (6x6-block Cholesky) + 230 flop per node per RHS "
                                           "column (forward + backward solve); the reduction executes %.2fx that"
                                           % (fa_exec / fa_flops),
                             "note": "the dominant group by ncu share (bcr_level_kernel alone is the top kernel); "
                                     "latency-bound depth-2log2(nf) chain of launches; peak = FP64 rate derived "
                                     "from 152 SMs x 2 DFMA/clk x 2.07 GHz (of derived)"},
                "contact_roofline": {"kernel": "contact_kernel (W columns + LCP, %d rows, working set %d, %d active)"
                                               % (m_last, mc_last, np_last),
                                     "achieved": ct_achieved, "peak": peak, "unit": "TFLOP/s FP64",
                                     "frac": ct_achieved / peak},
                "kernel_us": {"element": el_us, "collide": co_us, "contact": ct_us, "factor_group": fa_us,
                              "timing": "graph-replayed launches on the final state of the sweep",
                              "host_launched": host_us},
                "element_roofline": {"achieved": el_achieved, "peak": peak, "unit": "TFLOP/s FP64",
                                     "frac": el_achieved / peak, "flops_per_element": ELEMENT_FLOPS},
                "clocks": clk.summary(),
                "cpu_baseline": None if cpu is None else {
                    "value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
                    "sample": "%d worker processes (one per host core, one BLAS thread each) at once, each timing 2 "
                              "Newton iterations of one solve of the 60-solve sweep (solves %s, stratified) from the "
                              "oracle's recorded state after the solve before; seconds per iteration interpolated "
                              "over the sweep and weighted by the oracle's recorded iterations per solve (%.1f on "
                              "average): the whole sweep takes %.0f s on one core; numpy FP64 oracle"
                              % (cpu["cores"], cpu["sampled_solves"], cpu["oracle_iters_per_solve"],
                                 cpu["sweep_seconds_one_core"]),
                    "seconds_per_iteration": cpu["seconds_per_iteration"]}}
        line["precision"] = precision
        line["contact_admm"] = contact_admm
        line["segment_contacts"] = segment_contacts
        line.update(extra)
        if "batched" in extra and "served" in extra:
            bt, sv = extra["batched"], extra["served"]
            line["target"] = {
                "statement": "served and batched mixed-precision solves; multiples over the plain single-instance "
                             "FP64 GPU path (accuracy against the oracle: tests/test_gpu_target.py)",
                "batched_mixed": {"solves_per_s": bt["mixed"]["solves_per_s"],
                                  "multiple_over_plain_fp64": bt["multiple_over_plain_fp64"]["mixed"],
                                  "failed_solves": bt["mixed"]["failed_solves"],
                                  "one_launch_of_256_speedup": bt["mixed"]["one_launch_vs_sequential"]["speedup"]},
                "served_mixed": [{k: r[k] for k in ("offered_req_per_s", "solves_per_s", "throughput_multiple_over_plain_fp64",
                                                    "p99_multiple_of_plain_fp64", "failed_solves")}
                                 | {"p99_ms": r["latency_ms"]["p99"]} for r in sv["mixed"]["rates"]]}
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
    if args.profile_batch:
        return profile_batch_run(args)
    if args.profile_kernels:
        return profile_kernels_run(args)
    if args.profile_phases:
        return profile_phases_run(args)
    if args.frames_only:
        from paper_2503_06922_gb300 import accfem as af
        af.load()
        print(json.dumps({"frames": frames_run(af)}), flush=True)
        return 0
    return ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
