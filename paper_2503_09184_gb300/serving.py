"""Serving loop for encrypted sparse matmuls: continuous batching under an
HBM budget.

Requests (an encrypted sparse A times an encrypted dense B) arrive over time.
A request is admitted, in arrival order, once its ciphertexts fit the device
budget beside the requests already in flight; its operands are then
encrypted and lifted on the device and stay there until it completes.  A
request larger than the whole budget runs as column tiles (B and C split
by columns) that each fit beside its A, which is encrypted once and stays
resident until the last tile completes; one whose A alone does not fit is
rejected.  Work runs in waves: a
wave is one persistent launch (a batch plan) over row blocks of every
admitted request, up to a product budget, filled by a priority order
(highest response ratio first by default; shortest remaining work first and
round-robin shares are the alternatives), so requests that
arrive while others are on the GPU join the next wave and their products
overlap with those already running.  With preemption (GpuExecutor's
preempt) a request that arrives while a wave runs stops that wave at its
next output-entry boundary (the plan's stop word): the newcomer is admitted,
a wave over its rows runs, and the stopped wave resumes from its first entry
not taken.  Every output entry is computed by exactly one wave from its own
products, so a request's result is the same limb for limb alone and in any
mix, stopped or not.

`Scheduler` is the host-side policy (admission, row blocks, completion);
`GpuExecutor` carries it out through the C ABI.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    A: np.ndarray              # plaintext values of the sparse left operand (M x K)
    B: np.ndarray              # plaintext values of the dense right operand (K x Nc)
    arrival: float = 0.0       # seconds after the start of the run
    # column tile of a larger request: its first column there and the request
    col0: int = 0
    parent: "Request | None" = None
    # filled in by the scheduler
    state: str = "queued"      # queued, running, done, rejected
    admitted: float | None = None
    finished: float | None = None
    next_row: int = 0
    rows_done: int = 0
    tiles_left: int = 0
    a_resident: bool = False

    @property
    def key(self):
        return (self.rid, self.col0)

    @property
    def rows(self) -> int:
        return self.A.shape[0]

    def row_products(self) -> np.ndarray:
        """products of each output row: nonzeros of A's row times Nc."""
        return (self.A != 0).sum(axis=1).astype(np.int64) * self.B.shape[1]

    @property
    def products(self) -> int:
        return int(self.row_products().sum())


def a_bytes(req: Request, ct_bytes: int, ext_bytes: int) -> int:
    """device bytes of A: its nonzeros as ciphertexts plus lifted limbs."""
    return int((req.A != 0).sum()) * (ct_bytes + ext_bytes)


def bc_bytes(req: Request, ct_bytes: int, ext_bytes: int) -> int:
    """device bytes of B (ciphertexts plus lifted limbs) and C (ciphertexts)."""
    return req.B.size * (ct_bytes + ext_bytes) + req.A.shape[0] * req.B.shape[1] * ct_bytes


def request_bytes(req: Request, ct_bytes: int, ext_bytes: int) -> int:
    """device bytes a request holds while admitted: A's nonzeros and all of B
    as ciphertexts plus lifted limbs, and C as ciphertexts."""
    return a_bytes(req, ct_bytes, ext_bytes) + bc_bytes(req, ct_bytes, ext_bytes)


class Scheduler:
    """Admission by budget (FIFO, no overtaking) and row blocks per wave:
    order "rr" gives every running request an equal share of a wave in turn;
    "srpt" fills a wave shortest remaining work first (every running request
    still gets a row); "auto" takes srpt while the running requests' remaining
    work is at most backlog_waves waves and rr beyond (the median of
    shortest-first below overload, the tail of round-robin under it);
    "hrrn" (the default) fills a wave highest response ratio first (Brinch
    Hansen's highest-response-ratio-next): a request's ratio is 1 + its time since
    arrival over its remaining service time (remaining products at the
    loop's observed product rate), so with no waiting it is srpt, and a long
    request gains on newer short ones the longer it waits."""

    def __init__(self, budget_bytes: int, wave_products: int, ct_bytes: int, ext_bytes: int, order: str = "hrrn",
                 backlog_waves: float = 4.0):
        if order not in ("rr", "srpt", "auto", "hrrn"):
            raise ValueError(f"unknown wave order {order!r}")
        self.backlog_waves = backlog_waves
        self.order = order
        self.budget = budget_bytes
        self.wave_products = max(1, wave_products)
        self.ct_bytes, self.ext_bytes = ct_bytes, ext_bytes
        self.queue: deque[Request] = deque()
        self.running: list[Request] = []
        self.used = 0
        self._turn = 0

    def bytes_of(self, req: Request) -> int:
        """bytes admitting req adds: a tile adds its B and C blocks, plus its
        request's A if that is not resident yet."""
        if req.parent is None:
            return request_bytes(req, self.ct_bytes, self.ext_bytes)
        n = bc_bytes(req, self.ct_bytes, self.ext_bytes)
        return n if req.parent.a_resident else n + a_bytes(req.parent, self.ct_bytes, self.ext_bytes)

    def column_tiles(self, req: Request) -> list[Request]:
        """the widest column tiles (B[:, c0:c1] with C's columns) that fit the
        budget; [] if not even one column does."""
        nnz = int((req.A != 0).sum())
        K, M, Nc = req.B.shape[0], req.A.shape[0], req.B.shape[1]
        per_col = K * (self.ct_bytes + self.ext_bytes) + M * self.ct_bytes
        room = self.budget - nnz * (self.ct_bytes + self.ext_bytes)
        width = min(Nc, room // per_col) if room > 0 else 0
        if width < 1:
            return []
        return [Request(req.rid, req.A, req.B[:, c0:c0 + width], req.arrival, col0=c0, parent=req)
                for c0 in range(0, Nc, width)]

    def arrive(self, req: Request):
        if request_bytes(req, self.ct_bytes, self.ext_bytes) <= self.budget:
            self.queue.append(req)
            return
        tiles = self.column_tiles(req)
        if not tiles:
            req.state = "rejected"
            return
        req.tiles_left = len(tiles)
        self.queue.extend(tiles)

    def admit(self, now: float) -> list[Request]:
        """admit queued requests (or tiles), oldest first, while they fit."""
        out = []
        while self.queue and self.used + self.bytes_of(self.queue[0]) <= self.budget:
            req = self.queue.popleft()
            req.state, req.admitted = "running", now
            self.used += self.bytes_of(req)
            if req.parent is not None:
                if req.parent.admitted is None:
                    req.parent.state, req.parent.admitted = "running", now
                req.parent.a_resident = True
            self.running.append(req)
            out.append(req)
        return out

    def next_wave(self, only=None, now: float | None = None,
                  rate: float | None = None) -> list[tuple[Request, int, int]]:
        """row blocks (request, r0, r1) of the next wave: whole rows, taken in
        turn from every running request (starting one further each wave) until
        the wave's product budget is reached; every request with rows left
        gets at least one row.  only: take rows of these requests alone.
        now (seconds since the start) and rate (products per second of wave
        time so far) feed the response ratios of order "hrrn"; without them
        every ratio is 1 and the order is srpt's."""
        keep = None if only is None else {id(r) for r in only}
        live = [r for r in self.running if r.next_row < r.rows and (keep is None or id(r) in keep)]
        if not live:
            return []
        srpt = self.order in ("srpt", "hrrn")
        if self.order == "auto":
            backlog = sum(int(r.row_products()[r.next_row:].sum()) for r in live)
            srpt = backlog <= self.backlog_waves * self.wave_products
        if srpt:
            # a priority order (shortest remaining work first, or highest
            # response ratio first), each request taking what the wave has
            # left after one row for every request behind it
            def remaining(r):
                return int(r.row_products()[r.next_row:].sum())

            def ratio(r):
                if self.order != "hrrn" or now is None or not rate:
                    return 1.0
                return 1.0 + max(0.0, now - r.arrival) * rate / max(1, remaining(r))

            live.sort(key=lambda r: (-ratio(r), remaining(r), r.arrival, r.rid))
            left = self.wave_products
            blocks = []
            for n, req in enumerate(live):
                rp = req.row_products()
                r0 = r1 = req.next_row
                reserve = sum(int(q.row_products()[q.next_row]) for q in live[n + 1:])
                while r1 < req.rows and (r1 == r0 or rp[r1] <= left - reserve):
                    left -= int(rp[r1])
                    r1 += 1
                req.next_row = r1
                blocks.append((req, r0, r1))
            return blocks
        k = self._turn % len(live)
        live = live[k:] + live[:k]
        self._turn += 1
        share = max(1, self.wave_products // len(live))
        blocks = []
        for req in live:
            rp = req.row_products()
            r0 = r1 = req.next_row
            taken = 0
            while r1 < req.rows and (r1 == r0 or taken + rp[r1] <= share):
                taken += int(rp[r1])
                r1 += 1
            req.next_row = r1
            blocks.append((req, r0, r1))
        return blocks

    def complete(self, blocks, now: float) -> list[Request]:
        """mark the wave's rows done; returns the requests that finished."""
        done = []
        for req, r0, r1 in blocks:
            req.rows_done += r1 - r0
            if req.rows_done == req.rows and req.state == "running":
                req.state, req.finished = "done", now
                self.running.remove(req)
                done.append(req)
                if req.parent is None:
                    self.used -= request_bytes(req, self.ct_bytes, self.ext_bytes)
                    continue
                self.used -= bc_bytes(req, self.ct_bytes, self.ext_bytes)
                req.parent.tiles_left -= 1
                if req.parent.tiles_left == 0:
                    req.parent.state, req.parent.finished = "done", now
                    req.parent.a_resident = False
                    self.used -= a_bytes(req.parent, self.ct_bytes, self.ext_bytes)
                    done.append(req.parent)
        return done

    def idle(self) -> bool:
        return not self.queue and not self.running


@dataclasses.dataclass
class Wave:
    """one persistent launch over row blocks, possibly stopped and resumed"""
    blocks: list
    products: int
    entries: int = 0
    plan: int = 0
    work: object = None
    slot: int = 0
    events: list = dataclasses.field(default_factory=list)


class GpuExecutor:
    """Device side: encryption and lift on admission, one persistent batch
    plan per wave over CSR row blocks of A (and the matching rows of C).

    Matmul workspaces, each sized for the largest wave (wave_products
    products over as many output entries, up to max_blocks row blocks), are
    allocated once and reused: one, or two with preempt (a stopped wave keeps
    its plan and workspace while the wave that stopped it runs).  Their bytes
    (reserved_bytes) come out of the HBM budget before any request is
    admitted.  setup_s and kernel_s add up the waves' plan set-up (work-list
    build and upload) and their persistent launches."""

    def __init__(self, ctx, stream=None, lazy: bool = False, wave_products: int = 40000, max_blocks: int = 1024,
                 preempt: bool = False):
        """lazy: run the waves in the grouped accumulate-then-round mode
        (SFHE_EXEC_LAZY) instead of the per-product order.  preempt: waves
        can be stopped by a new arrival (the serving loop then runs a wave
        for the newcomer and resumes the stopped one)."""
        import torch
        from . import api, sfhe as S
        self.ctx, self.api, self.S, self.torch = ctx, api, S, torch
        self.flags = api.PERSISTENT | (api.LAZY if lazy else 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.mats = {}
        self.a_cache = {}
        self.admit_s = {}
        self.max_blocks = max_blocks
        self.preempt = preempt
        n = S.sfhe_matmul_workspace_bound(ctx.h, max_blocks, wave_products, wave_products, self.flags)
        self.works = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(2 if preempt else 1)]
        self.free = list(range(len(self.works)))
        self.reserved_bytes = n * len(self.works)
        if preempt:
            # the stop word (device) and its set value (pinned host), written
            # on a side stream while a wave runs
            self.stop = torch.zeros(1, dtype=torch.int32, device="cuda")
            self.one = torch.ones(1, dtype=torch.int32, pin_memory=True)
            self.side = torch.cuda.Stream()
        self.setup_s, self.kernel_s = 0.0, 0.0
        self.stops = 0

    def admit(self, req: Request):
        """encrypt and lift the request's operands on the device (the client's
        upload); a tile reuses its request's A.  The time it takes is kept in
        self.admit_s[rid]."""
        api = self.api
        t0 = time.perf_counter()
        if req.parent is not None and req.rid in self.a_cache:
            A = self.a_cache[req.rid]
        else:
            A = api.encrypt_matrix(self.ctx, req.A, "csr", 2 * req.rid + 1, stream=self.stream)
            if req.parent is not None:
                self.a_cache[req.rid] = A
        B = api.encrypt_matrix(self.ctx, req.B, "dense", 2 * req.rid + 2, stream=self.stream, col_offset=req.col0)
        C = api.result_matrix(self.ctx, req.A.shape[0], req.B.shape[1])
        self.stream.synchronize()
        self.admit_s[req.rid] = self.admit_s.get(req.rid, 0.0) + time.perf_counter() - t0
        self.mats[req.key] = (A, B, C)

    def _rows(self, req: Request, r0: int, r1: int):
        api, S = self.api, self.S
        A, B, C = self.mats[req.key]
        p0, p1 = int(A.row_ptr[r0]), int(A.row_ptr[r1])
        rp = np.ascontiguousarray(A.row_ptr[r0:r1 + 1] - p0, dtype=np.int32)
        ci = np.ascontiguousarray(A.col_idx[p0:p1], dtype=np.int32) if p1 > p0 else np.zeros(1, np.int32)
        q0, q1 = (p0, p1) if p1 > p0 else (0, 1)   # a block without nonzeros points at any stored ciphertext
        Ab = api.EncMatrix(r1 - r0, A.cols, S.SFHE_ENC_CSR, p1 - p0, row_ptr=rp, col_idx=ci,
                           ct=A.ct[q0:q1], ext=A.ext[q0:q1])
        Cb = api.EncMatrix(r1 - r0, C.cols, S.SFHE_ENC_DENSE, (r1 - r0) * C.cols,
                           ct=C.ct[r0 * C.cols:r1 * C.cols])
        return Ab, B, Cb

    def _launch(self, w: Wave, resume: bool):
        torch, S = self.torch, self.S
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        (S.sfhe_plan_resume if resume else S.sfhe_plan_execute)(w.plan, self.stream)
        e1.record(self.stream)
        w.events.append((e0, e1))

    def start_wave(self, blocks) -> Wave:
        """build the wave's plan and launch it (returns at once)."""
        api, S, torch = self.api, self.S, self.torch
        t0 = time.perf_counter()
        parts = [self._rows(req, r0, r1) for req, r0, r1 in blocks]
        As, Bs, Cs = [p[0] for p in parts], [p[1] for p in parts], [p[2] for p in parts]
        slot = self.free.pop(0)
        need = S.sfhe_matmul_workspace_size(self.ctx.h, [a.desc() for a in As], [b.desc() for b in Bs], self.flags)
        # a wave of unusually many empty rows may need more than the bound
        work = self.works[slot] if need <= self.works[slot].numel() else torch.empty(need, dtype=torch.uint8,
                                                                                     device="cuda")
        plan = S.sfhe_plan_create(self.ctx.h, [a.desc() for a in As], [b.desc() for b in Bs],
                                  [c.desc() for c in Cs], self.flags, work, self.stream)
        st = S.sfhe_plan_stats(plan)
        if self.preempt:
            S.sfhe_plan_set_stop(plan, self.stop)
        w = Wave(blocks, st["products"], st["entries"], plan, work, slot)
        self._launch(w, resume=False)
        self.setup_s += time.perf_counter() - t0
        return w

    def finish_wave(self, w: Wave, within_s: float | None = None) -> bool:
        """wait for the wave; if within_s (seconds) passes first, stop it at
        its next entry boundary.  True once every entry is done (the plan is
        released), False if it stopped short (resume_wave continues it)."""
        torch, S = self.torch, self.S
        deadline = None if within_s is None or not self.preempt else time.perf_counter() + within_s
        stopped = False
        while not w.events[-1][1].query():
            if deadline is not None and time.perf_counter() >= deadline:
                with torch.cuda.stream(self.side):
                    self.stop.copy_(self.one, non_blocking=True)
                stopped = True
                break
            time.sleep(0.0005)
        S.sfhe_matmul_check(w.work, self.stream)  # synchronises the stream
        e0, e1 = w.events[-1]
        self.kernel_s += e0.elapsed_time(e1) / 1e3
        if stopped:
            # the set value has landed before the word is cleared, and the
            # clearing precedes every later launch on the stream
            self.side.synchronize()
            with torch.cuda.stream(self.stream):
                self.stop.zero_()
            if S.sfhe_plan_progress(w.plan, self.stream) < w.entries:
                self.stops += 1
                return False
        S.sfhe_plan_destroy(w.plan)
        self.free.append(w.slot)
        return True

    def resume_wave(self, w: Wave):
        """launch a stopped wave's remaining entries (returns at once)."""
        self._launch(w, resume=True)

    def run_wave(self, blocks) -> int:
        """one persistent launch over the blocks, to completion; returns the
        products run."""
        w = self.start_wave(blocks)
        self.finish_wave(w)
        return w.products

    def result(self, req: Request, col0: int = 0):
        """C of a request, or of its column tile starting at col0."""
        return self.mats[(req.rid, col0)][2]

    def release(self, req: Request):
        """drop a finished request's (or tile's) device buffers; a request
        split into tiles also drops its shared A."""
        self.mats.pop(req.key, None)
        if req.tiles_left == 0 and req.parent is None:
            self.a_cache.pop(req.rid, None)


def serve(requests: list[Request], executor, budget_bytes: int, wave_products: int, ct_bytes: int,
          ext_bytes: int, keep_results: bool = False, clock=time.perf_counter, order: str = "hrrn") -> dict:
    """Run the requests (arrival times in seconds from now) through the
    continuous-batching loop on the wall clock.  Returns per-request
    latencies and totals; with keep_results the executor keeps every C.
    order: how waves share their products among running requests
    (Scheduler; highest response ratio first by default).

    An executor with start_wave / finish_wave / resume_wave (and preempt
    set) has a running wave stopped when the next request arrives: the
    arrival is admitted, a wave over the newcomers' rows runs to completion,
    and the stopped wave resumes (at most one wave is stopped at a time), so
    a short request that arrives behind long ones completes within about
    one entry's time plus its own work.  Without them every wave runs to
    completion (run_wave)."""
    # the executor's standing device memory (its matmul workspaces) is not
    # available to requests
    sched = Scheduler(budget_bytes - getattr(executor, "reserved_bytes", 0), wave_products, ct_bytes, ext_bytes,
                      order)
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    can_stop = hasattr(executor, "start_wave") and getattr(executor, "preempt", False)
    t0 = clock()
    waves, busy, products = 0, 0.0, 0
    suspended, resume_next = None, False
    newcomers = []   # requests (or tiles) admitted while a wave is stopped

    def completed(blocks):
        for req in sched.complete(blocks, clock() - t0):
            if not keep_results:
                executor.release(req)

    while pending or not sched.idle() or suspended is not None:
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            sched.arrive(pending.popleft())
        for req in sched.admit(clock() - t0):
            executor.admit(req)
            if suspended is not None:
                newcomers.append(req)
        rate = products / busy if busy > 0 else None
        if not can_stop:
            blocks = sched.next_wave(now=clock() - t0, rate=rate)
            if not blocks:
                if pending:   # nothing to run: wait for the next arrival
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
            w0 = clock()
            products += executor.run_wave(blocks)
            busy += clock() - w0
            waves += 1
            completed(blocks)
            continue
        # the next wave: the stopped one once the wave that stopped it is
        # done, else new rows (stoppable unless another wave is stopped)
        if suspended is not None and resume_next:
            wave, suspended, resume_next, stoppable = suspended, None, False, True
            executor.resume_wave(wave)
        else:
            blocks = sched.next_wave(only=newcomers if suspended is not None else None, now=clock() - t0,
                                     rate=rate)
            newcomers = []
            if blocks:
                wave = executor.start_wave(blocks)
                stoppable, resume_next = suspended is None, suspended is not None
            elif suspended is not None:
                wave, suspended, stoppable = suspended, None, True
                executor.resume_wave(wave)
            else:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
        within = max(0.0, pending[0].arrival - (clock() - t0)) if stoppable and pending else None
        w0 = clock()
        done = executor.finish_wave(wave, within)
        busy += clock() - w0
        if done:
            waves += 1
            products += wave.products
            completed(wave.blocks)
        else:
            suspended = wave
    end = clock() - t0
    done = [r for r in requests if r.state == "done"]
    lat = np.array([r.finished - r.arrival for r in done]) if done else np.zeros(0)
    return {
        "requests": len(requests), "done": len(done),
        "rejected": sum(1 for r in requests if r.state == "rejected"),
        "products": products, "waves": waves, "makespan_s": end, "busy_s": busy,
        "latency_s": lat,
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "ct_mults_per_s": products / end if end > 0 else None,
        "wave_setup_s": getattr(executor, "setup_s", None), "wave_kernel_s": getattr(executor, "kernel_s", None),
        "waves_stopped": getattr(executor, "stops", 0),
        "reserved_bytes": getattr(executor, "reserved_bytes", 0),
    }


def fifo_plain_model(requests: list[Request], service_s) -> dict:
    """One request at a time, in arrival order, each taking service_s(req)
    seconds: the latencies of the plain one-at-a-time server."""
    t, lat, products = 0.0, [], 0
    for req in sorted(requests, key=lambda r: r.arrival):
        start = max(t, req.arrival)
        t = start + service_s(req)
        lat.append(t - req.arrival)
        products += req.products
    lat = np.array(lat)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": t, "ct_mults_per_s": products / t if t > 0 else None, "latency_s": lat}
