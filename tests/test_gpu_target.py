"""Served and batched solves in both arithmetic modes against the oracle.

The request server (accfem_batch_serve, continuous batching) and the batched solves run members in
FP64 or in mixed precision (FP32 element tangent, FP64 residual, factor, contact Schur complement
and contact solve).  Every answer must match the oracle solving the same per-scene sequence of
quasi-static steps: tip position within 1e-6 m, per-node net contact force within 1e-4 of the
scene's largest, and the same contact set (rows paired by node and closest point within 1e-9 m).
Each answer must also be the one the same sequence of solves gives alone, bit for bit."""
import numpy as np
import pytest

import workloads as wl
from oracle import solver

pytestmark = pytest.mark.gpu

TIP_TOL = 1e-6        # m
FORCE_RTOL = 1e-4     # of the largest per-node net contact force of the solve
POINT_TOL = 1e-9      # m, pairing of contact rows by closest point
N_START = 9           # quasi-static steps (insertion 10 -> 90 mm) that bring each scene to its resident state


@pytest.fixture(scope="module")
def af():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06922_gb300 import accfem
    import os
    if not os.path.exists(accfem.LIB_PATH):
        from paper_2503_06922_gb300 import build
        build.build()
    accfem.load()
    return accfem


def _node_forces(contacts):
    f = {}
    for c in contacts:
        f[c["node"]] = f.get(c["node"], 0.0) + c["force"] * np.asarray(c["normal"], dtype=np.float64)
    return f


def _same_set(ga, gb):
    """Per node the same number of rows, whose closest points pair up within POINT_TOL."""
    def group(cs):
        g = {}
        for c in cs:
            g.setdefault(c["node"], []).append(np.asarray(c["point"], dtype=np.float64))
        return g
    a, b = group(ga), group(gb)
    if set(a) != set(b):
        return False
    for n in a:
        if len(a[n]) != len(b[n]):
            return False
        used = [False] * len(b[n])
        for pa in a[n]:
            k = next((j for j, pb in enumerate(b[n]) if not used[j] and np.linalg.norm(pa - pb) <= POINT_TOL), -1)
            if k < 0:
                return False
            used[k] = True
    return True


def _check_vs_oracle(g, o, tag):
    assert g["status"] == 0 and o.status == solver.OK, (tag, g["status"], o.status)
    tip = float(np.linalg.norm(g["node_pos"][-1] - o.node_pos[-1]))
    assert tip <= TIP_TOL, (tag, tip)
    assert _same_set(g["contacts"], o.contacts), (tag, "contact sets differ")
    fg, fo = _node_forces(g["contacts"]), _node_forces(o.contacts)
    fmax = max([np.linalg.norm(v) for v in fo.values()] + [1e-300])
    for n in set(fg) | set(fo):
        err = np.linalg.norm(fg.get(n, np.zeros(3)) - fo.get(n, np.zeros(3)))
        assert err <= FORCE_RTOL * fmax, (tag, n, err / fmax)
    return tip


def _scenes():
    """Three bent-tube scenes (120 mm robot, 20 elements) with their own tension sequences."""
    return [wl.bent_tube_workload(s, n_steps=10) for s in (0, 7, 11)]


@pytest.fixture(scope="module")
def served_case():
    """The request stream and the oracle's answer to every request (scene by scene, in order)."""
    ws = _scenes()
    arr, sc, ten, ins = wl.serve_trace([w.tensions[N_START - 1] for w in ws], [w.insertions[N_START - 1] for w in ws],
                                       [w.robot.length for w in ws], rate=3000.0, duration=0.012, seed=23)
    ref = []
    oracle = {}
    for j, w in enumerate(ws):
        m = solver.Model(w.robot, w.lumen)
        for s in range(N_START):
            assert m.solve(w.tensions[s], w.insertions[s]).status == solver.OK
        oracle[j] = m
    for k in range(len(arr)):
        ref.append(oracle[int(sc[k])].solve(ten[k], ins[k]))
    return ws, arr, sc, ten, ins, ref


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_served_answers_match_oracle_and_alone(af, served_case, mode):
    """Continuous batching over three resident scenes: requests of different scenes overlap on the
    device.  Every served answer against the oracle, and against the same requests solved alone."""
    ws, arr, sc, ten, ins, ref = served_case
    prec = af.PRECISION_FP64 if mode == "fp64" else af.PRECISION_MIXED
    hs = [af.AccFem(w.robot, w.lumen) for w in ws]
    for h in hs:
        assert h.accfem_set_precision(prec) == af.OK
    b = af.AccFemBatch(hs)
    for s in range(N_START):
        st, _, _ = b.accfem_batch_solve([w.tensions[s] for w in ws], [w.insertions[s] for w in ws], results=False)
        assert st == af.OK
    assert len(arr) >= 24
    out = b.accfem_batch_serve(arr, sc, ten, ins, chunk_iters=3, full_results=True)
    assert out["call_status"] == af.OK
    # overlap: some request began while another scene's solve was still in flight
    assert any(out["t_begin"][k] < out["t_end"][j] and out["t_begin"][j] < out["t_end"][k] and sc[j] != sc[k]
               for k in range(len(arr)) for j in range(k))
    worst = 0.0
    for k in range(len(arr)):
        g = out["results"][k]
        assert np.array_equal(np.concatenate([g["node_pos"][-1], g["node_quat"][-1]]), out["tip"][k])
        worst = max(worst, _check_vs_oracle(g, ref[k], "%s request %d scene %d" % (mode, k, sc[k])))
    # the same requests, scene by scene, alone: the same bits
    for j, w in enumerate(ws):
        h = af.AccFem(w.robot, w.lumen)
        h.accfem_set_precision(prec)
        for s in range(N_START):
            h.accfem_solve(w.tensions[s], w.insertions[s])
        for k in np.nonzero(sc == j)[0]:
            r = h.accfem_solve(ten[k], ins[k])
            g = out["results"][k]
            assert r["status"] == g["status"] and r["newton_iters"] == g["newton_iters"], (j, k)
            assert np.array_equal(r["node_pos"], g["node_pos"]) and np.array_equal(r["node_quat"], g["node_quat"]), (j, k)
            assert [c["force"] for c in r["contacts"]] == [c["force"] for c in g["contacts"]], (j, k)
        h.close()
    b.close()
    for h in hs:
        h.close()
    print("%s served: %d requests, worst tip error vs oracle %.2e m" % (mode, len(arr), worst))


def test_batched_mixed_members_match_oracle_and_alone(af):
    """A lock-step batch of mixed-precision members of different sizes (the bent tube and three
    uneven instances of the batched workload, cut to their first steps): each member equals its mixed
    solve alone bit for bit, and the bent-tube member matches the oracle at every step."""
    ws = [wl.bent_tube_workload(0, n_steps=10)]
    for w in wl.batch_workloads(first=0, count=3):
        ws.append(wl.Workload(w.name, w.robot, w.lumen, w.insertions[:8], w.tensions[:8]))
    alone = []
    for w in ws:
        h = af.AccFem(w.robot, w.lumen, max_contacts=4096)
        h.accfem_set_precision(af.PRECISION_MIXED)
        alone.append([h.accfem_solve(w.tensions[s], w.insertions[s]) for s in range(len(w.insertions))])
        h.close()
    hs = [af.AccFem(w.robot, w.lumen, max_contacts=4096) for w in ws]
    for h in hs:
        h.accfem_set_precision(af.PRECISION_MIXED)
    b = af.AccFemBatch(hs)
    ref = solver.Model(ws[0].robot, ws[0].lumen)
    for s in range(max(len(w.insertions) for w in ws)):
        mask = [1 if s < len(w.insertions) else 0 for w in ws]
        t = [w.tensions[min(s, len(w.insertions) - 1)] for w in ws]
        ins = [w.insertions[min(s, len(w.insertions) - 1)] for w in ws]
        st, sts, res = b.accfem_batch_solve(t, ins, mask=mask)
        for i in range(len(ws)):
            if not mask[i]:
                continue
            a = alone[i][s]
            assert res[i]["status"] == a["status"] == af.OK, (i, s, res[i]["error"])
            assert res[i]["newton_iters"] == a["newton_iters"], (i, s)
            assert np.array_equal(res[i]["node_pos"], a["node_pos"]), (i, s)
            assert [c["force"] for c in res[i]["contacts"]] == [c["force"] for c in a["contacts"]], (i, s)
        if mask[0]:
            _check_vs_oracle(res[0], ref.solve(ws[0].tensions[s], ws[0].insertions[s]), "bent tube step %d" % s)
    b.close()
    for h in hs:
        h.close()
