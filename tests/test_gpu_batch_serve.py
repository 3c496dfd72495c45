"""Batched answers and the continuous-batching server: every query's answer
is bit for bit the answer it gets alone (and the alone answer is the
oracle's, see test_gpu_parity), whatever else runs with it."""
import numpy as np
import pytest
import torch

from tests.gpu_common import Setup, library

pytestmark = pytest.mark.gpu

# (n, s, seed) of a mixed batch on one parameter set (N = 2^10, t = 12289)
MIX = [(5000, 20, 1), (700, 3, 2), (12000, 40, 3), (1, 1, 4), (3000, 9, 5), (9000, 64, 6)]


@pytest.fixture(scope="module")
def mix():
    first = Setup("small", seed=MIX[0][2], n=MIX[0][0], s=MIX[0][1])
    sets = [first] + [Setup("small", seed=sd, n=n, s=s, ctx=first.ctx) for n, s, sd in MIX[1:]]
    alone = [st.answer().clone() for st in sets]
    torch.cuda.synchronize()
    return sets, alone


def _lane_ws(sets, lanes):
    ctx = sets[0].ctx
    need = [0] * lanes
    for i, st in enumerate(sets):
        nb = library().load().pdq_answer_workspace_bytes(ctx.h, st.plan)
        need[i % lanes] = max(need[i % lanes], nb)
    return [torch.empty(n, dtype=torch.uint8, device="cuda") for n in need]


@pytest.mark.parametrize("lanes", [1, 3])
def test_batch_equals_alone(mix, lanes):
    sets, alone = mix
    handles = [st.handle() for st in sets]
    sets[0].ctx.answer_batch(handles, _lane_ws(sets, lanes))
    torch.cuda.synchronize()
    for h, a in zip(handles, alone):
        assert torch.equal(h.out.view(a.shape), a)


def test_batch_captured_in_cuda_graph(mix):
    sets, alone = mix
    handles = [st.handle() for st in sets]
    ws = _lane_ws(sets, 3)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sets[0].ctx.answer_batch(handles, ws, stream=s)      # warm-up outside capture
    torch.cuda.synchronize()
    for h in handles:
        h.out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sets[0].ctx.answer_batch(handles, ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for h, a in zip(handles, alone):
        assert torch.equal(h.out.view(a.shape), a)
    for h in handles:
        h.out.zero_()
    g.replay()
    torch.cuda.synchronize()
    for h, a in zip(handles, alone):
        assert torch.equal(h.out.view(a.shape), a)


def test_server_results_equal_alone_in_a_mixed_stream(mix):
    pdq = library()
    sets, alone = mix
    # a second parameter set (N = 2^6, several record groups) in the same server
    other = Setup("grouped")
    other_alone = other.answer().clone()
    arena = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    srv = pdq.Server(arena, lanes=3)
    handles, tickets = [], []
    for rep in range(3):
        for st in sets + [other]:
            h = st.handle()
            handles.append((h, st))
            tickets.append(srv.submit(h))
    srv.drain()
    for t, (h, st) in zip(tickets, handles):
        info = srv.status(t)
        assert info.state == pdq.PDQ_REQ_DONE and info.status == 0
        assert info.t_submit_ns <= info.t_start_ns <= info.t_done_ns
        want = other_alone if st is other else alone[sets.index(st)]
        assert torch.equal(h.out.view(want.shape), want)
    srv.close()


def test_server_admission_limits(mix):
    pdq = library()
    sets, _ = mix
    big = max(sets, key=lambda st: pdq.load().pdq_answer_workspace_bytes(st.ctx.h, st.plan))
    need = pdq.load().pdq_answer_workspace_bytes(big.ctx.h, big.plan)
    arena = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    srv = pdq.Server(arena, lanes=1)
    with pytest.raises(pdq.PdqError) as e:
        srv.submit(big.handle())
    assert e.value.code == pdq.PDQ_E_NOMEM
    srv.close()
    # a full queue refuses further requests; the admitted ones still finish
    arena = torch.empty(need + (1 << 20), dtype=torch.uint8, device="cuda")
    srv = pdq.Server(arena, lanes=1, max_queue=1)
    tickets, refused = [], 0
    for _ in range(6):
        try:
            tickets.append(srv.submit(big.handle()))
        except pdq.PdqError as err:
            assert err.code == pdq.PDQ_E_BUSY
            refused += 1
    srv.drain()
    assert refused >= 1 and tickets
    for t in tickets:
        srv.wait(t)
    srv.close()


def test_server_waits_run_out_and_recover(mix):
    """A wait on a request still queued behind others runs out with
    PDQ_E_TIMEOUT (the request itself is unaffected), a drain with no time
    left does too, and a later wait returns the request's result, the same
    as alone."""
    pdq = library()
    sets, alone = mix
    ctx = sets[0].ctx
    need = max(pdq.load().pdq_answer_workspace_bytes(ctx.h, st.plan) for st in sets)
    arena = torch.empty(need + (1 << 20), dtype=torch.uint8, device="cuda")
    srv = pdq.Server(arena, lanes=1)
    handles = [(st.handle(), i) for _ in range(8) for i, st in enumerate(sets)]
    tickets = [srv.submit(h) for h, _ in handles]
    last = tickets[-1]
    with pytest.raises(pdq.PdqError) as e:
        srv.wait(last, timeout_ms=0)
    assert e.value.code == pdq.PDQ_E_TIMEOUT
    assert srv.status(last).state != pdq.PDQ_REQ_DONE
    with pytest.raises(pdq.PdqError) as e:
        srv.drain(timeout_ms=0)
    assert e.value.code == pdq.PDQ_E_TIMEOUT
    srv.wait(last)
    srv.drain()
    for t, (h, i) in zip(tickets, handles):
        assert srv.status(t).status == 0
        assert torch.equal(h.out.view(alone[i].shape), alone[i])
    srv.close()


def test_server_stacks_requests_of_one_shape(mix):
    """With stacking on, queued requests of one shape (other clients of the
    same database with the same record and match counts, each with its own
    keys) are answered together; every result is still the request's answer
    alone, and requests of other shapes in the same stream are unaffected."""
    pdq = library()
    sets, alone = mix
    base = sets[0]
    ctx, plan = base.ctx, base.plan
    clients = [Setup("small", seed=50 + i, n=MIX[0][0], s=MIX[0][1], ctx=ctx) for i in range(4)]

    def handle(st):
        out = ctx._u64(plan.n_out * ctx.ct_elems)
        return ctx.query(plan, st.v_cts, base.db, st.keys, base.galois, base.consts, out)

    want = [ctx.answer(plan, st.v_cts, base.db, st.keys, base.galois, base.consts).clone()
            for st in clients]
    # the server's streams do not order after this one: its arena must not be
    # memory that the answers above still use
    torch.cuda.synchronize()
    arena = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    srv = pdq.Server(arena, lanes=1)
    srv.set_stacking(8)
    subs = []
    for _ in range(3):
        for i, st in enumerate(clients):
            h = handle(st)
            subs.append((srv.submit(h), h, want[i]))
        for j, st in enumerate(sets):
            h = st.handle()
            subs.append((srv.submit(h), h, alone[j]))
    srv.drain()
    infos = [srv.status(t) for t, _, _ in subs]
    assert max(i.stacked for i in infos) > 1, "no requests were stacked"
    bad = [(k, info.stacked) for k, (info, (_, h, w)) in enumerate(zip(infos, subs))
           if not torch.equal(h.out.view(w.shape), w)]
    for info in infos:
        assert info.state == pdq.PDQ_REQ_DONE and info.status == 0 and info.stacked >= 1
    assert not bad, f"(request, stack size) differing from alone: {bad}"
    with pytest.raises(pdq.PdqError):
        srv.set_stacking(65)
    srv.close()
