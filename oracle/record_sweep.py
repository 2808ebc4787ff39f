"""Writes the oracle's record of the 600 mm insertion sweep (test and benchmark infrastructure).

The CPU baseline of the benchmark times the oracle on a stratified sample of that sweep: each sampled
solve starts from the oracle's own converged state of the solve before it.  This script runs the
oracle, alone, through the whole 60-solve sweep (300 elements, the 63,840-triangle Catmull-Rom tube,
lumen seed 1, tension seed 2, insertion 10 -> 600 mm) and stores, for every solve, the converged
poses, the status, the Newton iterations, the number of constraint rows and the seconds it took on
the machine that wrote it.  Nothing in it comes from the CUDA path.

    python -m oracle.record_sweep [--out PATH] [--resume] [--recount [--procs P]]

It takes hours on one core (the oracle tests every node against every triangle); --resume continues
a partial record.  --recount re-runs every solve of a complete record with the oracle as it stands,
each from the recorded state of the solve before it, in P worker processes, and replaces the
recorded status, Newton iterations, rows and seconds (the converged states do not depend on the
iteration's path, so the recorded states stay).
"""
import argparse
import os
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")      # one BLAS thread, read when numpy loads (workers inherit it)
import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MAX_CONTACTS = 4096      # constraint-row capacity, as the benchmark's handles (the sweep's end has ~330 rows)
DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "records", "catmull_rom_600mm_M300_sweep.npz")


def _recount_one(args):
    """Solve s of the sweep with the oracle as it stands, from the recorded state after solve s - 1."""
    path, s = args
    import workloads as wl
    from oracle import solver
    rec = np.load(path)
    w = wl.catmull_rom_workload(lumen_seed=1, tension_seed=2, n_steps=60)
    m = solver.Model(w.robot, w.lumen, solver.Options(max_contacts=MAX_CONTACTS))
    if s > 0:
        m.state = (rec["pos"][s - 1].copy(), rec["rot"][s - 1].copy(), float(w.insertions[s - 1]))
    t0 = time.perf_counter()
    r = m.solve(w.tensions[s], w.insertions[s])
    return s, r.status, r.newton_iters, len(r.contacts), time.perf_counter() - t0


def recount(path, procs):
    import multiprocessing as mp
    rec = dict(np.load(path))
    S = len(rec["insertions"])
    if not np.all(rec["status"] == 0):
        raise SystemExit("the record is not complete")
    ctx = mp.get_context("spawn")
    order = list(range(S - 1, -1, -1))            # the long solves first
    with ctx.Pool(procs) as pool:
        for s, st, it, rows, sec in pool.imap_unordered(_recount_one, [(path, s) for s in order]):
            rec["status"][s], rec["newton_iters"][s], rec["rows"][s], rec["seconds"][s] = st, it, rows, sec
            print("recount solve %d status %d newton %d rows %d %.1f s" % (s, st, it, rows, sec), flush=True)
    np.savez_compressed(path, **rec)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--recount", action="store_true")
    ap.add_argument("--procs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args(argv)
    if args.recount:
        recount(args.out, args.procs)
        return 0
    import workloads as wl
    from oracle import solver
    w = wl.catmull_rom_workload(lumen_seed=1, tension_seed=2, n_steps=60)
    m = solver.Model(w.robot, w.lumen, solver.Options(max_contacts=MAX_CONTACTS))
    S, N = len(w.insertions), w.robot.n_elements + 1
    rec = {"pos": np.zeros((S, N, 3)), "rot": np.zeros((S, N, 3, 3)), "status": np.full(S, -1, np.int32),
           "newton_iters": np.zeros(S, np.int32), "rows": np.zeros(S, np.int32), "seconds": np.zeros(S),
           "insertions": np.asarray(w.insertions, dtype=np.float64), "tensions": np.asarray(w.tensions, dtype=np.float64)}
    start = 0
    if args.resume and os.path.exists(args.out):
        old = np.load(args.out)
        bad = np.nonzero(old["status"] != 0)[0]           # resume at the first solve that is not OK
        done = int(bad[0]) if len(bad) else len(old["status"])
        for k in rec:
            rec[k][:done] = old[k][:done]
        start = done
        if start > 0:
            m.state = (rec["pos"][start - 1].copy(), rec["rot"][start - 1].copy(), float(w.insertions[start - 1]))
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    for s in range(start, S):
        t0 = time.perf_counter()
        r = m.solve(w.tensions[s], w.insertions[s])
        rec["seconds"][s] = time.perf_counter() - t0
        rec["pos"][s], rec["rot"][s] = m.state[0], m.state[1]
        rec["status"][s], rec["newton_iters"][s], rec["rows"][s] = r.status, r.newton_iters, len(r.contacts)
        np.savez_compressed(args.out, **rec)
        print("solve %d status %d newton %d rows %d %.1f s" % (s, r.status, r.newton_iters, len(r.contacts),
                                                                rec["seconds"][s]), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
