"""sfhe_ct_mul_relin_static (static device scratch, no workspace argument)
against sfhe_ct_mul_relin with a caller-owned workspace: two calls in a row
on the same inputs, each identical in every limb to the workspace call.
Collected last so that it also runs after every other GPU test."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import gpu_ctx, gpu_modules

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 4)])
def test_static_scratch_matches_workspace_call(N, L):
    import torch
    api, S = gpu_modules()
    ctx = gpu_ctx(N, L, 1)
    M = api.encrypt_matrix(ctx, np.array([[7, -5, 300, -1]], dtype=np.int64), "dense", 31)
    need = ((3 * ctx.K * N * 4 + 255) // 256) * 256 + (3 * L + (L + 2) * L) * N * 8
    work = torch.empty(need, dtype=torch.uint8, device="cuda")
    for a, b in [(0, 1), (2, 3)]:
        ref = torch.empty((2, L, N), dtype=torch.int64, device="cuda")
        S.sfhe_ct_mul_relin(ctx.h, M.ext[a], M.ext[b], ref, work)
        want = api.to_numpy_u64(ref)
        for _ in range(2):
            out = torch.full((2, L, N), -1, dtype=torch.int64, device="cuda")
            S.sfhe_ct_mul_relin_static(ctx.h, M.ext[a], M.ext[b], out)
            assert (api.to_numpy_u64(out) == want).all()


def test_static_scratch_rejects_large_ring():
    """N = 16384, L = 8 needs 19.5 MB of scratch, more than the static array
    holds: rejected on the host before anything is launched."""
    import torch
    api, S = gpu_modules()
    ctx = gpu_ctx(16384, 8, 1)
    a = torch.zeros((2, ctx.K, ctx.N), dtype=torch.int32, device="cuda")
    out = torch.empty((2, ctx.L, ctx.N), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError, match="static scratch"):
        S.sfhe_ct_mul_relin_static(ctx.h, a, a, out)
