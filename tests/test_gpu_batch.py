"""Batched solves (accfem_batch_*) through the C ABI.

A member of a batch runs the same kernel code on its own buffers as a solve alone, so its poses,
contact rows, forces and iteration counts must equal those of accfem_solve bit for bit, whatever
else is in flight; and, through that, match the oracle within the parity tolerance."""
import numpy as np
import pytest

import workloads as wl
from oracle import solver

pytestmark = pytest.mark.gpu


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


def _mixed_workloads():
    """Members of different sizes, lumens and loads: the bent tube (20 elements, two tension seeds),
    and three uneven instances of the batched workload cut to their first steps."""
    ws = [wl.bent_tube_workload(0, n_steps=10), wl.bent_tube_workload(7, n_steps=10)]
    for w in wl.batch_workloads(first=0, count=3):
        ws.append(wl.Workload(w.name, w.robot, w.lumen, w.insertions[:12], w.tensions[:12]))
    return ws


def _same(a, b, tag):
    assert a["status"] == b["status"], (tag, a["status"], b["status"], a["error"], b["error"])
    assert a["newton_iters"] == b["newton_iters"], (tag, a["newton_iters"], b["newton_iters"])
    assert a["contact_iters"] == b["contact_iters"], tag
    assert np.array_equal(a["node_pos"], b["node_pos"]), (tag, np.abs(a["node_pos"] - b["node_pos"]).max())
    assert np.array_equal(a["node_quat"], b["node_quat"]), tag
    assert a["n_contacts"] == b["n_contacts"], tag
    for ca, cb in zip(a["contacts"], b["contacts"]):
        assert ca["node"] == cb["node"] and ca["tri"] == cb["tri"], tag
        assert np.array_equal(ca["point"], cb["point"]) and np.array_equal(ca["normal"], cb["normal"]), tag
        assert ca["force"] == cb["force"], tag
    assert np.array_equal(a["base_reaction"], b["base_reaction"]), tag
    assert a["residual"] == b["residual"], tag


def _alone(af, ws):
    out = []
    for w in ws:
        h = af.AccFem(w.robot, w.lumen)
        out.append([h.accfem_solve(w.tensions[s], w.insertions[s]) for s in range(len(w.insertions))])
        h.close()
    return out


def test_batch_sweep_equals_solves_alone(af):
    """Lock-step sweep: step s of every member that still has one, in one batched solve."""
    ws = _mixed_workloads()
    alone = _alone(af, ws)
    hs = [af.AccFem(w.robot, w.lumen) for w in ws]
    b = af.AccFemBatch(hs)
    n_steps = max(len(w.insertions) for w in ws)
    for s in range(n_steps):
        mask = [1 if s < len(w.insertions) else 0 for w in ws]
        t = [w.tensions[min(s, len(w.insertions) - 1)] for w in ws]
        ins = [w.insertions[min(s, len(w.insertions) - 1)] for w in ws]
        st, sts, res = b.accfem_batch_solve(t, ins, mask=mask)
        for i in range(len(ws)):
            if mask[i]:
                _same(res[i], alone[i][s], "member %d step %d" % (i, s))
    assert any(r["n_contacts"] > 0 for r in res.values())
    b.close()
    for h in hs:
        h.close()


def test_autotuned_packing_keeps_results(af):
    """Autotuning takes the twelve variants (four grid divisors x three element mappings) in turn;
    every member still equals its solve alone."""
    ws = _mixed_workloads()
    alone = _alone(af, ws)
    hs = [af.AccFem(w.robot, w.lumen) for w in ws]
    b = af.AccFemBatch(hs)
    assert b.accfem_batch_autotune(0) == af.E_INVALID_ARG
    assert b.accfem_batch_autotune(1) == af.OK
    assert b.accfem_batch_tuning()[0] == -1
    for s in range(8):
        for i, w in enumerate(ws):
            assert b.accfem_batch_begin(i, w.tensions[s], w.insertions[s]) == af.OK
        left = 1
        while left:
            st, left = b.accfem_batch_advance(3)
            assert st == af.OK
        res = b.accfem_batch_results(list(range(len(ws))))
        for i in range(len(ws)):
            _same(res[i], alone[i][s], "member %d step %d" % (i, s))
    v, ms = b.accfem_batch_tuning()
    assert 0 <= v < 12 and len(ms) == 12 and np.all(ms > 0.0)
    b.close()
    for h in hs:
        h.close()


def test_continuous_admission_equals_alone(af):
    """Members start at different iterations of the others (continuous batching): each member
    begins its next step as soon as its previous one finished, advancing a few iterations at a
    time; results equal the solves alone."""
    ws = _mixed_workloads()
    alone = _alone(af, ws)
    hs = [af.AccFem(w.robot, w.lumen) for w in ws]
    b = af.AccFemBatch(hs)
    nxt = [0] * len(ws)
    # stagger: member i joins after i advances
    rounds = 0
    while True:
        for i, w in enumerate(ws):
            done, _, _ = b.accfem_batch_poll(i)
            if done and rounds >= i and nxt[i] < len(w.insertions):
                if nxt[i] > 0:
                    r = b.accfem_batch_results([i])[0]
                    _same(r, alone[i][nxt[i] - 1], "member %d step %d" % (i, nxt[i] - 1))
                assert b.accfem_batch_begin(i, w.tensions[nxt[i]], w.insertions[nxt[i]]) == af.OK
                nxt[i] += 1
        st, left = b.accfem_batch_advance(5)
        assert st == af.OK, b.accfem_batch_last_error()
        rounds += 1
        if left == 0 and all(nxt[i] == len(w.insertions) for i, w in enumerate(ws)):
            break
        assert rounds < 5000
    for i, w in enumerate(ws):
        r = b.accfem_batch_results([i])[0]
        _same(r, alone[i][-1], "member %d last step" % i)
    b.close()
    for h in hs:
        h.close()


def test_batch_member_matches_oracle(af):
    """The bent-tube member of a batch against the oracle (positions 1e-9 relative)."""
    w = wl.bent_tube_workload(0, n_steps=10)
    other = wl.bent_tube_workload(7, n_steps=10)
    hs = [af.AccFem(w.robot, w.lumen), af.AccFem(other.robot, other.lumen)]
    b = af.AccFemBatch(hs)
    ref = solver.Model(w.robot, w.lumen)
    for s in range(len(w.insertions)):
        st, sts, res = b.accfem_batch_solve([w.tensions[s], other.tensions[s]], [w.insertions[s], other.insertions[s]])
        o = ref.solve(w.tensions[s], w.insertions[s])
        assert sts[0] == af.OK and o.status == solver.OK
        err = np.abs(res[0]["node_pos"] - o.node_pos).max() / np.abs(o.node_pos).max()
        assert err <= 1e-9, (s, err)
        assert sorted(c["node"] for c in res[0]["contacts"]) == sorted(c["node"] for c in o.contacts), s
    b.close()
    for h in hs:
        h.close()


def test_mask_leaves_members_untouched_and_errors(af):
    w = wl.bent_tube_workload(0, n_steps=4)
    hs = [af.AccFem(w.robot, w.lumen) for _ in range(3)]
    b = af.AccFemBatch(hs)
    st, sts, res = b.accfem_batch_solve([w.tensions[0]] * 3, [w.insertions[0]] * 3)
    assert st == af.OK
    before = hs[1].accfem_get_state()
    st, sts, res = b.accfem_batch_solve([w.tensions[1]] * 3, [w.insertions[1]] * 3, mask=[1, 0, 1])
    assert st == af.OK and set(res) == {0, 2}
    after = hs[1].accfem_get_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert np.array_equal(res[0]["node_pos"], res[2]["node_pos"])
    # a member cannot be begun twice; results need a finished solve; bad indices are rejected
    assert b.accfem_batch_begin(0, w.tensions[2], w.insertions[2]) == af.OK
    assert b.accfem_batch_begin(0, w.tensions[2], w.insertions[2]) == af.E_INVALID_ARG
    assert b.accfem_batch_begin(5, w.tensions[2], w.insertions[2]) == af.E_INVALID_ARG
    assert b.accfem_batch_begin(1, w.tensions[2], 1.0) == af.E_INVALID_ARG
    st, left = b.accfem_batch_advance(200)
    assert st == af.OK and left == 0
    done, s0, it0 = b.accfem_batch_poll(0)
    assert done and s0 == af.OK and it0 > 0
    # an insertion with every node prescribed finishes without iterations
    assert b.accfem_batch_begin(2, w.tensions[0], 0.0) == af.OK
    st, left = b.accfem_batch_advance(10)
    assert st == af.OK and left == 0
    done, s2, it2 = b.accfem_batch_poll(2)
    assert done and s2 == af.OK and it2 == 0
    b.close()
    for h in hs:
        h.close()


def test_served_requests_equal_solves_alone(af):
    """Continuous-batching server: a request stream over three scenes (arrivals close enough that
    solves of different scenes overlap) gives, per request, the tip pose and iteration count of the
    same sequence of solves run alone; a scene left out by the memory cap is answered NOMEM."""
    ws = _mixed_workloads()[:3]
    hs = [af.AccFem(w.robot, w.lumen) for w in ws]
    b = af.AccFemBatch(hs)
    for s in range(3):
        b.accfem_batch_solve([w.tensions[s] for w in ws], [w.insertions[s] for w in ws])
    arr, sc, ten, ins = wl.serve_trace([w.tensions[2] for w in ws], [w.insertions[2] for w in ws],
                                       [w.robot.length for w in ws], rate=4000.0, duration=0.01, seed=11)
    assert len(arr) >= 20
    out = b.accfem_batch_serve(arr, sc, ten, ins, chunk_iters=3)
    assert out["call_status"] == af.OK
    assert np.all(out["t_end"] >= out["t_begin"]) and np.all(out["t_begin"] >= arr - 1e-9)
    # the same requests, scene by scene, alone
    for j, w in enumerate(ws):
        h = af.AccFem(w.robot, w.lumen)
        for s in range(3):
            h.accfem_solve(w.tensions[s], w.insertions[s])
        for k in np.nonzero(sc == j)[0]:
            r = h.accfem_solve(ten[k], ins[k])
            assert r["status"] == out["status"][k] and r["newton_iters"] == out["newton_iters"][k], (j, k)
            tip = np.concatenate([r["node_pos"][-1], r["node_quat"][-1]])
            assert np.array_equal(tip, out["tip"][k]), (j, k, np.abs(tip - out["tip"][k]).max())
            assert r["n_contacts"] == out["n_contacts"][k]
        h.close()
    # memory cap that admits nobody: every request answered NOMEM without a solve
    out2 = b.accfem_batch_serve(arr[:5], sc[:5], ten[:5], ins[:5], chunk_iters=3, hbm_cap_bytes=1)
    assert out2["call_status"] == af.OK and np.all(out2["status"] == af.E_NOMEM)
    b.close()
    for h in hs:
        h.close()
