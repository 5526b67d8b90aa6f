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
