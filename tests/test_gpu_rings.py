"""Every ring the library implements (N in {4096, 8192, 16384}, L in
{2, 3, 4, 8}): a small sparse matmul through the persistent kernel and
through the plain path, every entry bit-exact against the oracle in every
limb, and the grouped mode against the oracle's grouped entries.  Each ring
runs its own kernel instances (tensor-base size K, staging layout, stage-S
interleave), so each is checked on its own."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O

pytestmark = pytest.mark.gpu
T = 65537
RINGS = [(N, L) for N in (4096, 8192, 16384) for L in (2, 3, 4, 8)]


@pytest.mark.parametrize("N,L", RINGS)
def test_ring_matmul_bit_exact(N, L):
    api, _ = gpu_modules()
    ctx = gpu_ctx(N, L, 5)
    octx = oracle_ctx(N, L, 5)
    # 2 x 3 times 3 x 2, one zero in A: entries of 1 to 3 products
    A = np.array([[4, 0, -7], [13, 2, 9]], dtype=np.int64)
    B = np.array([[3, -1], [16, 5], [-2, 8]], dtype=np.int64)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    enc = O.encode(A, O.CSR)
    entries = [(0, 1), (1, 0)] if N == 16384 else [(i, j) for i in range(2) for j in range(2)]
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    want = ((A @ B + T // 2) % T) - T // 2
    for mode in ("persistent", "plain", "lazy"):
        C = api.matmul(ctx, Ae, Be, mode=mode)
        got = coeff_of(api, ctx, C)
        group = ctx.lazy_group if mode == "lazy" else 1
        for i, j in entries:
            assert (got[i * 2 + j] == mm.entry(enc, i, j, group=group)).all(), (N, L, mode, i, j)
        assert (api.decrypt(ctx, C) == want).all(), (N, L, mode)
