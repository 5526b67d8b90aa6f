"""Preemption of persistent plans (the serving loop's continuous admission):
a launch stopped at an output-entry boundary by the plan's stop word, then
resumed, writes C limb for limb as one uninterrupted execution does; the
serving loop that stops waves for new arrivals keeps every request's result
identical to the request alone."""
from __future__ import annotations

import time

import pytest

import workloads as W
from gpu_common import gpu_ctx, gpu_modules

pytestmark = pytest.mark.gpu


def _coeff(api, ctx, M):
    return api.to_coeff(ctx, M.ct, M.rows * M.cols)


def _operands(api, ctx, M, K, Nc, s, seed):
    a, b = W.operands(W.MatmulShape(M, K, Nc, s, -16, 16, seed))
    return a, b, api.encrypt_matrix(ctx, a, "csr", 2 * seed + 1), api.encrypt_matrix(ctx, b, "dense", 2 * seed + 2)


def test_stop_word_set_before_the_launch_takes_no_entry_and_resume_completes():
    api, S = gpu_modules()
    import torch
    ctx = gpu_ctx(4096, 2, 11)
    a, b, A, B = _operands(api, ctx, 8, 16, 8, 0.5, 7)
    ref = api.matmul(ctx, A, B)
    plan = api.Plan(ctx, [A], [B])
    C = plan.Cs[0]
    C.ct.fill_(7)  # a marker that no written entry keeps
    stop = torch.ones(1, dtype=torch.int32, device="cuda")
    S.sfhe_plan_set_stop(plan.h, stop)
    plan.execute()
    assert S.sfhe_plan_progress(plan.h) == 0
    assert bool((C.ct == 7).all())
    stop.zero_()
    S.sfhe_plan_resume(plan.h)
    assert S.sfhe_plan_progress(plan.h) == plan.stats["entries"]
    assert (_coeff(api, ctx, C) == _coeff(api, ctx, ref)).all()
    want = ((a @ b + W.T_PLAIN // 2) % W.T_PLAIN) - W.T_PLAIN // 2
    assert (api.decrypt(ctx, C) == want).all()
    # a later execute starts again from the first entry
    C.ct.fill_(7)
    stop.fill_(1)
    plan.execute()
    assert S.sfhe_plan_progress(plan.h) == 0
    stop.zero_()
    plan.execute()
    assert S.sfhe_plan_progress(plan.h) == plan.stats["entries"]
    assert (_coeff(api, ctx, C) == _coeff(api, ctx, ref)).all()
    plan.close()


@pytest.mark.parametrize("delay_ms", [0.0, 2.0, 8.0])
def test_stop_while_running_then_resume_equals_one_execution(delay_ms):
    api, S = gpu_modules()
    import torch
    ctx = gpu_ctx(4096, 2, 12)
    _, _, A, B = _operands(api, ctx, 32, 32, 16, 0.5, 8)
    ref = api.matmul(ctx, A, B)
    plan = api.Plan(ctx, [A], [B])
    n = plan.stats["entries"]
    stop = torch.zeros(1, dtype=torch.int32, device="cuda")
    one = torch.ones(1, dtype=torch.int32, pin_memory=True)
    side = torch.cuda.Stream()
    S.sfhe_plan_set_stop(plan.h, stop)
    torch.cuda.synchronize()
    plan.execute()
    time.sleep(delay_ms / 1e3)
    with torch.cuda.stream(side):
        stop.copy_(one, non_blocking=True)
    done = S.sfhe_plan_progress(plan.h)
    side.synchronize()
    assert 0 <= done <= n
    stop.zero_()
    S.sfhe_plan_resume(plan.h)
    assert S.sfhe_plan_progress(plan.h) == n
    assert (_coeff(api, ctx, plan.Cs[0]) == _coeff(api, ctx, ref)).all()
    plan.close()


def test_stop_word_needs_a_plain_persistent_plan_and_resume_an_execution():
    api, S = gpu_modules()
    import torch
    ctx = gpu_ctx(4096, 2, 13)
    _, _, A, B = _operands(api, ctx, 4, 4, 4, 0.5, 9)
    stop = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan = api.Plan(ctx, [A], [B])
    assert S.sfhe_plan_progress(plan.h) == 0
    with pytest.raises(S.SfheError) as ex:
        S.sfhe_plan_resume(plan.h)  # nothing to resume yet
    assert ex.value.status == S.SFHE_EINVAL
    plan.close()
    for kw in ({"mode": "plain"}, {"graph": True}):
        plan = api.Plan(ctx, [A], [B], **kw)
        with pytest.raises(S.SfheError) as ex:
            S.sfhe_plan_set_stop(plan.h, stop)
        assert ex.value.status == S.SFHE_EINVAL
        plan.close()


def test_serving_with_waves_stopped_at_once_matches_requests_alone():
    """every wave that could be stopped is stopped as soon as it is waited
    on: new rows run in nested waves, stopped waves resume, and each
    request's C is still the one it gets alone"""
    api, S = gpu_modules()
    from paper_2503_09184_gb300 import serving as SV

    class EagerStop(SV.GpuExecutor):
        def finish_wave(self, w, within_s=None):
            return super().finish_wave(w, None if within_s is None else 0.0)

    ctx = gpu_ctx(4096, 2, 14)
    shapes = [(24, 16, 16, 0.5), (8, 8, 8, 0.3), (12, 16, 8, 0.7), (16, 8, 8, 0.5)]
    reqs = []
    for rid, (M, K, Nc, s) in enumerate(shapes):
        A, B = W.operands(W.MatmulShape(M, K, Nc, s, -16, 16, 200 + rid))
        reqs.append(SV.Request(rid, A, B, arrival=0.02 * rid))
    ct_b = 2 * ctx.L * ctx.N * 8
    ext_b = 2 * ctx.K * ctx.N * 4
    ex = EagerStop(ctx, wave_products=2048, preempt=True)
    budget = 4 * max(SV.request_bytes(r, ct_b, ext_b) for r in reqs) + ex.reserved_bytes
    out = SV.serve(reqs, ex, budget, wave_products=2048, ct_bytes=ct_b, ext_bytes=ext_b, keep_results=True)
    assert out["done"] == len(reqs)
    assert out["waves_stopped"] == ex.stops
    for r in reqs:
        A = api.encrypt_matrix(ctx, r.A, "csr", 2 * r.rid + 1)
        B = api.encrypt_matrix(ctx, r.B, "dense", 2 * r.rid + 2)
        C_alone = api.matmul(ctx, A, B)
        assert (_coeff(api, ctx, ex.result(r)) == _coeff(api, ctx, C_alone)).all(), r.rid
