"""Failure detection without a GPU fault: a bounded device wait that runs
out sets the status word, the host reads SFHE_ETIMEOUT through the same
check as after a persistent matmul, and the context stays usable (a matmul
afterwards is still bit-exact)."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_survives():
    import torch
    api, S = gpu_modules()
    work = torch.zeros(256, dtype=torch.uint8, device="cuda")
    S.sfhe_matmul_check(work)                       # clean status word
    S.sfhe_selftest_wait_bound(work, 1000)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_matmul_check(work)
    assert e.value.status == S.SFHE_ETIMEOUT
    with pytest.raises(S.SfheError) as e:
        S.sfhe_selftest_wait_bound(work, 0)
    assert e.value.status == S.SFHE_EINVAL
    ctx = gpu_ctx(4096, 2, 0)
    A = np.array([[3, 0, -7]], dtype=np.int64)
    B = np.array([[2], [5], [1]], dtype=np.int64)
    C = api.matmul(ctx, api.encrypt_matrix(ctx, A, "csr", 1), api.encrypt_matrix(ctx, B, "dense", 2))
    mm = O.OracleMatmul(oracle_ctx(4096, 2, 0), A, B, 1, 2)
    assert (coeff_of(api, ctx, C)[0] == mm.entry(O.encode(A, O.CSR), 0, 0)).all()


def test_wait_bounds_in_real_time():
    """The wait gives up on whichever bound comes first: a time bound of
    2 ms ends a wait of up to 2^30 attempts within a few milliseconds (the
    persistent kernel's own bound is one second or 2^26 attempts), and an
    attempt bound ends it without the time bound.  The measured time per
    attempt is printed (it depends on how long the hardware suspends a
    try_wait)."""
    import torch
    api, S = gpu_modules()
    work = torch.zeros(256, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S.sfhe_selftest_wait_bound(work, 1 << 30, 2000)
    e1.record()
    with pytest.raises(S.SfheError) as e:
        S.sfhe_matmul_check(work)
    assert e.value.status == S.SFHE_ETIMEOUT
    ms = e0.elapsed_time(e1)
    assert 1.9 <= ms < 100.0, ms
    for tries in (1 << 12, 1 << 16):
        work.zero_()
        e0.record()
        S.sfhe_selftest_wait_bound(work, tries, 1_000_000)
        e1.record()
        with pytest.raises(S.SfheError):
            S.sfhe_matmul_check(work)
        ms = e0.elapsed_time(e1)
        assert ms < 1000.0
        print(f"bounded wait: {tries} attempts in {ms:.3f} ms, {1e6 * ms / tries:.1f} ns per attempt")
    with pytest.raises(S.SfheError) as e:
        S.sfhe_selftest_wait_bound(work, 10, 0)
    assert e.value.status == S.SFHE_EINVAL
