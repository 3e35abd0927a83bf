"""Serving admission and host-side failures, with no GPU fault: the request
queue at capacity (DSES_ERR_QUEUE_FULL), a device allocation refused by the
engine's test hook (DSES_ERR_OOM; the context stays usable), and admission
under a device-memory budget below two requests' needs (requests wait, none
fails). Every completed registration is checked against the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_2502_00115_b300 import build, capi, synth

pytestmark = pytest.mark.gpu

f32 = lambda v: float(np.float32(v))


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = capi.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def tiny_set():
    """Four tiny problems (576 rotations each) with the oracle's registrations."""
    out = []
    for s in (21, 22, 23, 24):
        p = synth.tiny_problem(s, hopf_n=2)
        P = oracle.make_params(metric="trunc_l1", epsilon=f32(p.epsilon), tau=f32(p.tau),
                               t_half=[f32(v) for v in p.t_half], grid_cap=f32(2 * p.tau))
        out.append((p, oracle.register(p.X, p.Y, oracle.hopf_grid(2), P)))
    return out


def problems(ctx, tiny_set):
    pbs, targets = [], []
    for p, _ in tiny_set:
        t = ctx.create_target(p.Y, grid_cap=2 * p.tau)
        targets.append(t)
        pbs.append(ctx.problem(t, p.X, capi.hopf_grid(2),
                               capi.make_params(metric="trunc_l1", epsilon=p.epsilon, tau=p.tau, t_half=p.t_half)))
    return pbs, targets


def matches_oracle(r, ref):
    r = capi.result_dict(r) if not isinstance(r, dict) else r
    assert r["status"] == 0
    if r["rot_index"] == ref.rot_index:
        assert r["inliers"] == ref.inliers and r["votes"] == ref.votes
        np.testing.assert_allclose(r["t"], ref.t, atol=1e-6)
    else:  # a near-tie of the oracle's own costs
        assert abs(ref.costs[r["rot_index"]] - ref.costs[ref.rot_index]) <= 1e-4 * ref.costs[ref.rot_index] + 1e-6
    assert abs(r["cost"] - ref.costs[r["rot_index"]]) <= 1e-4 * abs(ref.costs[r["rot_index"]]) + 1.3e-4


def drain(ctx, tickets, deadline_s=120):
    out = {}
    deadline = time.time() + deadline_s
    while len(out) < len(tickets) and time.time() < deadline:
        for tk in tickets:
            if tk not in out:
                st, r = ctx.poll(tk)
                if st != capi.DSES_NOT_READY:
                    out[tk] = (st, r)
        time.sleep(0.002)
    assert len(out) == len(tickets)
    return out


def test_queue_full_is_reported_and_accepted_requests_complete(ctx, tiny_set):
    pbs, targets = problems(ctx, tiny_set)
    # a long request occupies the only batch slot; the queue holds one more
    big = synth.modelnet_like_problem(3, hopf_n=16)
    tb = ctx.create_target(big.Y, grid_cap=2 * big.tau)
    pbig = ctx.problem(tb, big.X, capi.hopf_grid(16),
                       capi.make_params(metric=big.metric, epsilon=big.epsilon, tau=big.tau, t_half=big.t_half))
    ctx.set_option("serve_max_batch", 1)
    ctx.set_option("serve_queue_cap", 1)
    try:
        accepted, full = [], 0
        st, tk = capi.dses_submit(ctx.h, pbig)
        assert st == capi.DSES_OK
        accepted.append((tk, None))
        for i, pb in enumerate(pbs):
            st, tk = capi.dses_submit(ctx.h, pb)
            if st == capi.DSES_ERR_QUEUE_FULL:
                full += 1
                assert "queue" in capi.dses_last_error(ctx.h)
            else:
                assert st == capi.DSES_OK
                accepted.append((tk, i))
        assert full >= 1  # at most one request waits while the long one holds the slot
        done = drain(ctx, [tk for tk, _ in accepted])
        for tk, i in accepted:
            st, r = done[tk]
            assert st == capi.DSES_OK
            if i is not None:
                matches_oracle(r, tiny_set[i][1])
    finally:
        ctx.set_option("serve_max_batch", 16)
        ctx.set_option("serve_queue_cap", 100000)
    # the context keeps serving
    tk = ctx.submit(pbs[0])
    st, r = drain(ctx, [tk])[tk]
    assert st == capi.DSES_OK
    matches_oracle(r, tiny_set[0][1])
    for t in targets + [tb]:
        ctx.destroy_target(t)


def test_refused_allocation_returns_oom_and_the_context_stays_usable(ctx, tiny_set):
    pbs, targets = problems(ctx, tiny_set)
    # blocking call
    ctx.set_option("fail_next_allocs", 1)
    st, r = capi.dses_register(ctx.h, pbs[0])
    assert st == capi.DSES_ERR_OOM and "fail_next_allocs" in capi.dses_last_error(ctx.h)
    assert ctx.get_option("fail_next_allocs") == 0
    matches_oracle(ctx.register(pbs[0]), tiny_set[0][1])
    # batch: the first problem's allocation is refused, the call reports OOM
    ctx.set_option("use_graphs", 0)
    try:
        ctx.set_option("fail_next_allocs", 1)
        st, rs = capi.dses_register_batch(ctx.h, pbs)
        assert st == capi.DSES_ERR_OOM
        for r, (p, ref) in zip(ctx.register_batch(pbs), tiny_set):
            matches_oracle(r, ref)
    finally:
        ctx.set_option("use_graphs", 1)
    # served: the first admitted request fails with OOM at poll, the rest complete
    ctx.set_option("fail_next_allocs", 1)
    tickets = [ctx.submit(pb) for pb in pbs]
    done = drain(ctx, tickets)
    statuses = [done[tk][0] for tk in tickets]
    assert statuses.count(capi.DSES_ERR_OOM) == 1 and statuses.count(capi.DSES_OK) == len(pbs) - 1
    for tk, (p, ref) in zip(tickets, tiny_set):
        st, r = done[tk]
        if st == capi.DSES_OK:
            matches_oracle(r, ref)
        else:
            assert r.status == capi.DSES_ERR_OOM and r.rot_index == -1
    for t in targets:
        ctx.destroy_target(t)


def test_memory_budget_below_two_requests_queues_them(ctx, tiny_set):
    pbs, targets = problems(ctx, tiny_set)
    for pb in pbs:  # warm every target's per-epsilon structures
        ctx.register(pb)
    ctx.set_option("serve_max_active", 0)
    ctx.set_option("serve_mem_budget", 1024)  # below any one request: one at a time
    try:
        tickets = [ctx.submit(pb) for pb in pbs]
        done = drain(ctx, tickets)
        assert ctx.get_option("serve_max_active") == 1
        for tk, (p, ref) in zip(tickets, tiny_set):
            st, r = done[tk]
            assert st == capi.DSES_OK
            matches_oracle(r, ref)
    finally:
        ctx.set_option("serve_mem_budget", 8 << 30)
    # with the default budget the same requests run together
    ctx.set_option("serve_max_active", 0)
    tickets = [ctx.submit(pb) for pb in pbs]
    done = drain(ctx, tickets)
    assert ctx.get_option("serve_max_active") >= 2
    for tk, (p, ref) in zip(tickets, tiny_set):
        matches_oracle(done[tk][1], ref)
    for t in targets:
        ctx.destroy_target(t)
