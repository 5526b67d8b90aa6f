"""Host logic of the serving loop (no GPU): admission by budget in arrival
order, rejection of requests larger than the budget, row blocks that cover
every row exactly once and visit every running request each wave, budget
release on completion, and the one-at-a-time baseline model."""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_2503_09184_gb300.serving import Request, Scheduler, fifo_plain_model, request_bytes, serve

CT, EXT = 100, 10


def _req(rid, M, K, Nc, density=0.5, arrival=0.0, seed=0):
    rng = np.random.default_rng(seed + rid)
    A = rng.integers(1, 5, size=(M, K)) * (rng.random((M, K)) < density)
    B = rng.integers(-3, 4, size=(K, Nc))
    return Request(rid, A.astype(np.int64), B.astype(np.int64), arrival)


def test_request_bytes_formula():
    r = _req(0, 4, 6, 3)
    nnz = int((r.A != 0).sum())
    assert request_bytes(r, CT, EXT) == (nnz + 18) * (CT + EXT) + 12 * CT


def test_admission_fifo_by_budget_and_rejection():
    reqs = [_req(i, 4, 6, 3) for i in range(4)]
    big = _req(9, 40, 60, 30, density=1.0)
    s = Scheduler(budget_bytes=2 * max(request_bytes(r, CT, EXT) for r in reqs), wave_products=10, ct_bytes=CT,
                  ext_bytes=EXT)
    for r in reqs:
        s.arrive(r)
    s.arrive(big)
    assert big.state == "rejected"
    admitted = s.admit(0.0)
    assert [r.rid for r in admitted] == [0, 1]            # oldest first, while they fit
    assert s.used == sum(request_bytes(r, CT, EXT) for r in admitted) <= s.budget
    assert all(r.state == "queued" for r in reqs[2:])
    # finish request 0 entirely: its bytes return and request 2 is admitted
    while reqs[0].rows_done < reqs[0].rows:
        blocks = [b for b in s.next_wave() if b[0] is reqs[0]]
        s.complete(blocks, 1.0)
    assert reqs[0].state == "done" and reqs[0].finished == 1.0
    assert [r.rid for r in s.admit(2.0)] == [2]


@pytest.mark.parametrize("order", ["rr", "srpt", "auto", "hrrn"])
def test_waves_cover_rows_once_and_every_running_request_progresses(order):
    reqs = [_req(i, 5 + i, 6, 4, arrival=0.0) for i in range(3)]
    s = Scheduler(budget_bytes=10**9, wave_products=20, ct_bytes=CT, ext_bytes=EXT, order=order)
    for r in reqs:
        s.arrive(r)
    s.admit(0.0)
    seen = {r.rid: [] for r in reqs}
    waves = 0
    while not s.idle():
        blocks = s.next_wave(now=float(waves), rate=10.0)
        live = {r.rid for r in s.running if r.next_row < r.rows or any(b[0] is r for b in blocks)}
        assert {b[0].rid for b in blocks} == live          # every running request progresses
        for req, r0, r1 in blocks:
            assert r1 > r0
            seen[req.rid].extend(range(r0, r1))
        s.complete(blocks, float(waves))
        waves += 1
    for r in reqs:
        assert seen[r.rid] == list(range(r.rows))           # contiguous, each row once, in order
        assert r.state == "done"
    assert s.used == 0


def test_srpt_order_fills_waves_shortest_remaining_first():
    def dense(rid, M, K, Nc):
        return Request(rid, np.ones((M, K), dtype=np.int64), np.ones((K, Nc), dtype=np.int64))
    big, small, mid = dense(0, 8, 2, 4), dense(1, 2, 2, 4), dense(2, 4, 2, 4)  # 8 products a row
    s = Scheduler(budget_bytes=10**9, wave_products=40, ct_bytes=CT, ext_bytes=EXT, order="srpt")
    for r in (big, small, mid):
        s.arrive(r)
    s.admit(0.0)
    # small (16 left) whole, then mid (32 left) up to what leaves big one row
    w = {req.rid: (r0, r1) for req, r0, r1 in s.next_wave()}
    assert w == {1: (0, 2), 2: (0, 2), 0: (0, 1)}
    w = {req.rid: (r0, r1) for req, r0, r1 in s.next_wave()}
    assert w == {2: (2, 4), 0: (1, 4)}
    # every request keeps a row per wave, even when the shortest fill the wave
    s2 = Scheduler(budget_bytes=10**9, wave_products=8, ct_bytes=CT, ext_bytes=EXT, order="srpt")
    a, b = dense(3, 4, 2, 4), dense(4, 4, 2, 4)
    for r in (a, b):
        s2.arrive(r)
    s2.admit(0.0)
    assert sorted((req.rid, r1 - r0) for req, r0, r1 in s2.next_wave()) == [(3, 1), (4, 1)]
    try:
        Scheduler(1, 1, 1, 1, order="fifo")  # not a wave order
        raise AssertionError("unknown order accepted")
    except ValueError:
        pass


def test_auto_order_is_srpt_below_the_backlog_and_round_robin_above():
    def dense(rid, M, K, Nc):
        return Request(rid, np.ones((M, K), dtype=np.int64), np.ones((K, Nc), dtype=np.int64))

    def first_wave(backlog_waves):
        big, small = dense(0, 8, 2, 4), dense(1, 2, 2, 4)  # 64 and 16 products left
        s = Scheduler(10**9, 40, CT, EXT, order="auto", backlog_waves=backlog_waves)
        for r in (big, small):
            s.arrive(r)
        s.admit(0.0)
        return {req.rid: (r0, r1) for req, r0, r1 in s.next_wave()}

    # 80 products left: srpt when 2 waves of 40 may be queued, rr when one
    assert first_wave(2.0) == {1: (0, 2), 0: (0, 3)}
    assert first_wave(1.0) == {0: (0, 2), 1: (0, 2)}


def test_hrrn_order_is_srpt_without_waiting_and_ages_long_requests():
    def dense(rid, M, arrival):
        return Request(rid, np.ones((M, 2), dtype=np.int64), np.ones((2, 4), dtype=np.int64), arrival)

    def first_wave(order, now=None, rate=None, small_arrival=0.5):
        big, small = dense(0, 8, 0.0), dense(1, 2, small_arrival)  # 8 products a row: 64 and 16 left
        s = Scheduler(10**9, 40, CT, EXT, order=order)
        for r in (big, small):
            s.arrive(r)
        s.admit(0.0)
        return {req.rid: (r0, r1) for req, r0, r1 in s.next_wave(now=now, rate=rate)}

    # no clock or no rate yet: every ratio is 1, the order is srpt's
    assert first_wave("hrrn") == first_wave("srpt") == {1: (0, 2), 0: (0, 3)}
    assert first_wave("hrrn", now=5.0, rate=None) == first_wave("srpt")
    # soon after the arrivals the short request's ratio is higher:
    # big 1 + 1/64, small 1 + 0.5/16 (rate 1 product/s)
    assert first_wave("hrrn", now=1.0, rate=1.0) == {1: (0, 2), 0: (0, 3)}
    # the long request has waited 10 s, the short one 1 s:
    # big 1 + 10/64 = 1.16 > small 1 + 1/16 = 1.06, so big fills the wave
    # first and leaves the short request one row
    assert first_wave("hrrn", now=10.0, rate=1.0, small_arrival=9.0) == {0: (0, 4), 1: (0, 1)}
    # srpt ignores waiting
    assert first_wave("srpt", now=10.0, rate=1.0, small_arrival=9.0) == {1: (0, 2), 0: (0, 3)}


def test_fifo_plain_model_closed_form():
    reqs = [_req(i, 3, 4, 2, arrival=a) for i, a in enumerate([0.0, 0.5, 10.0])]
    m = fifo_plain_model(reqs, lambda r: 1.0)
    # starts 0, 1, 10; finishes 1, 2, 11
    assert np.allclose(m["latency_s"], [1.0, 1.5, 1.0])
    assert m["makespan_s"] == 11.0


class FakeExecutor:
    """stands in for the GPU: records which rows each wave covered."""

    def __init__(self):
        self.rows = {}
        self.admitted = []

    def admit(self, req):
        self.admitted.append(req.key)
        self.rows[req.key] = []

    def run_wave(self, blocks):
        n = 0
        for req, r0, r1 in blocks:
            self.rows[req.key].extend(range(r0, r1))
            n += int(req.row_products()[r0:r1].sum())
        return n

    def release(self, req):
        pass


@pytest.mark.parametrize("order", ["rr", "srpt", "auto", "hrrn"])
def test_serve_loop_with_fake_executor(order):
    reqs = [_req(i, 6, 8, 3, arrival=0.002 * i) for i in range(5)]
    one = max(request_bytes(r, CT, EXT) for r in reqs)
    ex = FakeExecutor()
    out = serve(reqs, ex, budget_bytes=2 * one, wave_products=8, ct_bytes=CT, ext_bytes=EXT, order=order)
    assert out["done"] == 5 and out["rejected"] == 0
    assert out["products"] == sum(r.products for r in reqs)
    assert ex.admitted == [(i, 0) for i in range(5)]
    for r in reqs:
        assert ex.rows[r.key] == list(range(r.rows))
        assert r.finished >= r.arrival
    assert out["p99_s"] >= out["p50_s"] >= 0.0


class FakeStoppableExecutor(FakeExecutor):
    """stands in for a GPU whose waves can be stopped: the first `stops`
    waits with an arrival ahead stop the wave when the arrival is due
    (having run none of its rows); each later wait completes the wave."""

    preempt = True

    def __init__(self, stops):
        super().__init__()
        self.stops_left = stops
        self.log = []
        self.rids = {}

    def start_wave(self, blocks):
        from paper_2503_09184_gb300.serving import Wave
        w = Wave(blocks, int(sum(int(req.row_products()[r0:r1].sum()) for req, r0, r1 in blocks)))
        w.tag = len(self.log)
        self.log.append(("start", w.tag))
        self.rids[w.tag] = {req.rid for req, _, _ in blocks}
        return w

    def finish_wave(self, w, within_s=None):
        if within_s is not None and self.stops_left > 0:
            time.sleep(within_s)  # the wave is stopped when the arrival is due
            self.stops_left -= 1
            self.log.append(("stop", w.tag))
            return False
        self.run_wave(w.blocks)
        self.log.append(("done", w.tag))
        return True

    def resume_wave(self, w):
        self.log.append(("resume", w.tag))


@pytest.mark.parametrize("order", ["rr", "hrrn"])
def test_serve_loop_stops_a_wave_for_an_arrival_and_resumes_it(order):
    reqs = [_req(i, 6, 8, 3, arrival=0.05 * i) for i in range(4)]
    one = max(request_bytes(r, CT, EXT) for r in reqs)
    ex = FakeStoppableExecutor(stops=2)
    out = serve(reqs, ex, budget_bytes=4 * one, wave_products=8, ct_bytes=CT, ext_bytes=EXT, order=order)
    assert out["done"] == 4 and out["products"] == sum(r.products for r in reqs)
    # every row of every request ran exactly once (a stopped wave's rows
    # complete after those of the wave that stopped it)
    for r in reqs:
        assert sorted(ex.rows[r.key]) == list(range(r.rows))
    # a stop is followed by a fresh wave run to completion, then the resume
    # of the stopped wave; no second wave is stopped while one is
    kinds = [k for k, _ in ex.log]
    assert kinds.count("stop") == 2
    for i, (k, w) in enumerate(ex.log):
        if k == "stop":
            assert ex.log[i + 1][0] == "start" and ex.log[i + 2][0] == "done"
            assert ex.log[i + 3] == ("resume", w)
            # the wave in between serves the newcomers alone
            assert not (ex.rids[ex.log[i + 1][1]] & ex.rids[w])
    # each stopped wave is completed exactly once
    done = [w for k, w in ex.log if k == "done"]
    assert len(done) == len(set(done))
    assert {w for k, w in ex.log if k == "stop"} <= set(done)


def test_over_budget_request_runs_as_column_tiles():
    big = _req(0, 6, 5, 9, density=0.8)
    small = _req(1, 3, 4, 2, arrival=0.0)
    nnz = int((big.A != 0).sum())
    # room for A and three columns of B and C, not for all nine
    budget = nnz * (CT + EXT) + 3 * (5 * (CT + EXT) + 6 * CT)
    assert request_bytes(big, CT, EXT) > budget
    s = Scheduler(budget_bytes=budget, wave_products=50, ct_bytes=CT, ext_bytes=EXT)
    s.arrive(big)
    s.arrive(small)
    tiles = [t for t in s.queue if t.parent is big]
    assert [t.col0 for t in tiles] == [0, 3, 6] and big.tiles_left == 3
    assert all(t.B.shape[1] == 3 and (t.B == big.B[:, t.col0:t.col0 + 3]).all() for t in tiles)
    assert all(request_bytes(t, CT, EXT) <= budget for t in tiles)
    from paper_2503_09184_gb300.serving import a_bytes, bc_bytes
    first = s.admit(0.0)
    assert first == [tiles[0]] and big.a_resident                 # A charged once, with the first tile
    assert s.used == a_bytes(big, CT, EXT) + bc_bytes(tiles[0], CT, EXT)
    t = 1.0
    while not s.idle():
        s.admit(t)
        assert s.used <= budget
        s.complete(s.next_wave(), t)
        t += 1.0
    assert big.state == "done" and big.tiles_left == 0 and small.state == "done"
    assert big.finished == max(x.finished for x in tiles)
    assert s.used == 0


def test_request_whose_left_operand_alone_exceeds_the_budget_is_rejected():
    big = _req(0, 8, 8, 2, density=1.0)
    s = Scheduler(budget_bytes=64 * (CT + EXT) - 1, wave_products=10, ct_bytes=CT, ext_bytes=EXT)
    s.arrive(big)
    assert big.state == "rejected" and not s.queue
