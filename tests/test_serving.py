"""Host logic of the serving scheduler (admission by memory, one request per graph per step,
release after the last step), with no device: the Server's library side is covered by the GPU
tests."""

import numpy as np
import pytest

from paper_2306_08967_gb300.serving import Request, Scheduler


def _req(rid, sid, k=3, t=0.0):
    z = np.zeros(k, np.int32)
    return Request(rid, sid, z, z + 1, np.ones(k, np.int8), t)


def test_admission_is_first_come_within_the_budget():
    s = Scheduler(budget_bytes=100)
    s.open(1, 40)
    s.open(2, 50)
    s.open(3, 30)          # fits beside 1 alone, but waits behind 2
    s.open(4, 5)
    assert s.admissions() == [1, 2]
    assert s.used == 90
    assert s.admissions() == []            # 3 needs 30, 10 left; 4 waits behind it
    with pytest.raises(ValueError):
        s.open(5, 101)                     # never fits
    with pytest.raises(ValueError):
        s.open(1, 10)                      # exists


def test_each_step_takes_the_oldest_request_of_each_resident_graph():
    s = Scheduler(budget_bytes=100, max_events=8)
    s.open(1, 10)
    s.open(2, 10)
    s.open(3, 90)                          # waits until 1 or 2 is freed
    for sid in s.admissions():
        s.admitted(sid)
    for rid, sid in enumerate([1, 1, 2, 3, 1]):
        s.submit(_req(rid, sid))
    with pytest.raises(ValueError):
        s.submit(_req(9, 1, k=9))          # more than max_events
    st, pick = s.next_step()
    assert st == 0 and {k: v.rid for k, v in pick.items()} == {1: 0, 2: 2}
    st, pick = s.next_step()
    assert st == 1 and {k: v.rid for k, v in pick.items()} == {1: 1}
    st, pick = s.next_step()
    assert st == 2 and {k: v.rid for k, v in pick.items()} == {1: 4}
    assert s.next_step() is None           # graph 3 is not resident: its request waits
    assert not s.idle()


def test_release_waits_for_the_last_step_and_frees_memory():
    s = Scheduler(budget_bytes=100)
    s.open(1, 60)
    s.open(2, 60)
    for sid in s.admissions():
        s.admitted(sid)
    assert s.resident() == [1]
    s.submit(_req(0, 1))
    s.submit(_req(1, 1))
    s.close(1)
    with pytest.raises(ValueError):
        s.submit(_req(2, 1))               # closing
    a = s.next_step(t=1.0)
    b = s.next_step(t=1.5)
    s.step_done(a[0], a[1], t=2.0)
    assert s.releases() == []                           # its second request still runs
    assert a[1][1].t_done == 2.0 and a[1][1].t_issue == 1.0
    s.step_done(b[0], b[1], t=3.0)
    assert s.releases() == [1] and s.releases() == []
    assert s.resident() == [] and s.admissions() == []   # memory not yet freed
    s.freed(1)
    assert s.admissions() == [2] and s.used == 60
    with pytest.raises(ValueError):
        s.freed(1)


def test_a_session_closed_while_empty_is_released_without_a_step():
    s = Scheduler(budget_bytes=10)
    s.open(1, 5)
    s.open(2, 5)
    s.open(3, 5)
    for sid in s.admissions():
        s.admitted(sid)
    s.submit(_req(0, 2))
    s.submit(_req(1, 3))                 # 3 waits for memory
    s.close(1)
    assert s.releases() == [1]           # it never took part in a step
    s.freed(1)
    assert s.admissions() == [3]
    s.admitted(3)
    assert s.backlog() == 2
    st = s.next_step()
    assert sorted(st[1]) == [2, 3]
    s.step_done(st[0], st[1], 1.0)
    assert s.idle() and s.backlog() == 0


def test_eviction_makes_room_with_the_least_recently_active_idle_graphs():
    s = Scheduler(budget_bytes=100)
    for sid in (1, 2, 3):
        s.open(sid, 30)
    for sid in s.admissions():
        s.admitted(sid)
    s.submit(_req(0, 1, t=5.0))
    s.submit(_req(1, 2, t=1.0))
    s.submit(_req(2, 3, t=3.0))
    st = s.next_step()
    s.step_done(st[0], st[1], 6.0)
    s.open(4, 50)                          # needs 50, 10 free: two idle graphs must go
    assert s.admissions() == []
    assert s.plan_evictions() == [2, 3]    # least recently active first
    s.evicting(2)
    s.evicting(3)
    assert s.plan_evictions() == []        # the memory on its way out is counted
    assert s.resident() == [1]
    s.evicted(2)
    s.evicted(3)
    assert s.used == 30 and s.admissions() == [4]
    # a request for an evicted graph queues it for readmission
    s.submit(_req(3, 2, t=7.0))
    assert s.sessions[2].state == "waiting" and list(s.waiting) == [2]
    assert s.sessions[2].evictions == 1


def test_busy_or_closing_graphs_are_not_evicted():
    s = Scheduler(budget_bytes=60)
    s.open(1, 30)
    s.open(2, 30)
    for sid in s.admissions():
        s.admitted(sid)
    s.submit(_req(0, 1))                   # 1 has a request waiting
    st = s.next_step()                     # and then running
    s.close(2)                             # 2 is closing
    s.open(3, 30)
    assert s.plan_evictions() == []
    s.step_done(st[0], st[1], 1.0)
    assert s.plan_evictions() == [1]       # now idle


def test_a_graph_that_closes_while_evicted_is_done_without_readmission():
    s = Scheduler(budget_bytes=30)
    s.open(1, 30)
    for sid in s.admissions():
        s.admitted(sid)
    s.open(2, 30)
    assert s.plan_evictions() == [1]
    s.evicting(1)
    s.evicted(1)
    s.close(1)
    assert s.releases() == [] and s.sessions[1].state == "freed"
    assert s.admissions() == [2]


def test_graphs_active_lately_are_not_evicted():
    s = Scheduler(budget_bytes=60, min_idle_s=2.0)
    s.open(1, 30)
    s.open(2, 30)
    for sid in s.admissions():
        s.admitted(sid)
    s.submit(_req(0, 1, t=10.0))
    s.submit(_req(1, 2, t=11.5))
    st = s.next_step()
    s.step_done(st[0], st[1], 11.6)
    s.open(3, 30)
    assert s.plan_evictions(t=11.7) == []        # both asked within the last 2 s
    assert s.plan_evictions(t=12.5) == [1]       # 1 has been idle for 2.5 s


@pytest.mark.parametrize("seed", range(6))
def test_random_traffic_keeps_the_scheduler_invariants(seed):
    # the Server's loop with the device replaced by delays: sessions open, ask and close at
    # random; steps finish in order after random delays, admissions and evictions take time.
    # Throughout: memory within the budget and equal to what the sessions on the device hold;
    # admissions first come; a step holds one request per resident graph; only idle graphs
    # are evicted; and in the end every request was served once, in its session's order.
    rng = np.random.default_rng(seed)
    budget = 100
    s = Scheduler(budget_bytes=budget, max_events=8, min_idle_s=float(rng.choice([0.0, 2.0])))
    on_device = ("admitting", "resident", "evicting", "released")
    submitted, served = {}, {}
    inflight, admitting, evicting, releasing = [], {}, [], []
    rid = nsid = 0
    admitted_order, waiting_order = [], []

    def check():
        assert 0 <= s.used <= budget
        assert s.used == sum(x.nbytes for x in s.sessions.values() if x.state in on_device)

    def turn(t, arrivals):
        nonlocal rid, nsid
        if arrivals:
            if rng.random() < 0.15 and nsid < 40:
                s.open(nsid, int(rng.integers(10, 61)), t)
                submitted[nsid] = []
                nsid += 1
            open_ = [x.sid for x in s.sessions.values() if not x.closing]
            for _ in range(int(rng.integers(0, 4))):
                if open_:
                    sid = int(rng.choice(open_))
                    s.submit(_req(rid, sid, k=int(rng.integers(1, 9)), t=t))
                    submitted[sid].append(rid)
                    rid += 1
            if open_ and rng.random() < 0.05:
                s.close(int(rng.choice(open_)))
        # steps finish in issue order
        while inflight and rng.random() < 0.6:
            st, reqs = inflight.pop(0)
            s.step_done(st, reqs, t)
        for sid in s.releases():
            releasing.append((sid, s.next_step_id - 1))
        for sid, last in list(releasing):
            if last <= s.done_upto:
                s.freed(sid)
                releasing.remove((sid, last))
        for sid, last in list(evicting):
            if last <= s.done_upto and rng.random() < 0.5:
                s.evicted(sid)
                evicting.remove((sid, last))
        for sid in s.plan_evictions(t):
            x = s.sessions[sid]
            assert x.state == "resident" and not x.queue and not x.closing and x.last_step <= s.done_upto
            s.evicting(sid)
            evicting.append((sid, s.next_step_id - 1))
        before = list(s.waiting)
        got = s.admissions(t)
        assert got == before[:len(got)]                 # first come, first admitted
        admitted_order.extend(got)
        waiting_order.extend(before[:len(got)])
        for sid in got:
            admitting[sid] = int(rng.integers(0, 3))
        for sid in list(admitting):
            if admitting[sid] == 0:
                s.admitted(sid)
                del admitting[sid]
            else:
                admitting[sid] -= 1
        if len(inflight) < 2:
            nxt = s.next_step(t)
            if nxt is not None:
                st, reqs = nxt
                for sid, r in reqs.items():
                    assert s.sessions[sid].state == "resident" and r.sid == sid
                    served.setdefault(sid, []).append(r.rid)
                inflight.append((st, reqs))
        check()

    t = 0.0
    for _ in range(600):
        t += float(rng.exponential(0.3))
        turn(t, arrivals=True)
    for sid in list(s.sessions):
        if not s.sessions[sid].closing:
            s.close(sid)
    for _ in range(5000):
        if all(x.state == "freed" for x in s.sessions.values()):
            break
        t += 0.3
        turn(t, arrivals=False)
    assert all(x.state == "freed" for x in s.sessions.values())
    assert s.used == 0 and not s.waiting and s.backlog() == 0
    for sid, rids in submitted.items():
        assert served.get(sid, []) == rids, sid         # each once, in arrival order
    assert sum(x.evictions for x in s.sessions.values()) > 0    # the traffic did make graphs leave
