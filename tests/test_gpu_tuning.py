"""The tiles the run-time tuner chooses between (stage-S tiles, and at
N = 8192 two code forms of the inverse NTT): every tile of every ring that
has several is bit-exact (against the oracle at N = 4096, L = 2; against the
plain per-product path, which the oracle checks, at N = 8192, L = 4 and
N = 16384, L = 8), and the tuner keeps the tile it timed fastest."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_modules, oracle_ctx
from oracle import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
T = 65537


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


def test_every_tile_against_the_oracle():
    api, S = gpu_modules()
    ctx = api.Context(4096, 2, seed=11)
    A = W.sparse_int_matrix(4, 6, 0.3, -16, 16, 61)
    A[2, :] = 0
    B = W.dense_int_matrix(6, 3, -16, 16, 62)
    mm = O.OracleMatmul(oracle_ctx(4096, 2, 11), A, B, 1, 2)
    enc = O.encode(A, O.CSR)
    want = {(i, j): mm.entry(enc, i, j) for i in range(4) for j in range(3)}
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    n = S.sfhe_ctx_tuning(ctx.h)["variants"]
    assert n == 3
    for v in range(n):
        S.sfhe_ctx_set_variant(ctx.h, v)
        got = coeff_of(api, ctx, api.matmul(ctx, Ae, Be))
        for (i, j), ct in want.items():
            assert (got[i * 3 + j] == ct).all(), (v, i, j)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_ctx_set_variant(ctx.h, n)
    assert e.value.status == S.SFHE_EINVAL
    ctx.close()


@pytest.mark.parametrize("N,L,shape", [(8192, 4, (3, 9, 2)), (16384, 8, (2, 4, 2))])
def test_every_tile_equals_the_plain_path(N, L, shape):
    api, S = gpu_modules()
    ctx = api.Context(N, L, seed=12)
    M, K, Nc = shape
    A = W.sparse_int_matrix(M, K, 0.3, -8, 8, 63)
    B = W.dense_int_matrix(K, Nc, -8, 8, 64)
    Ae = api.encrypt_matrix(ctx, A, "ell", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    ref = coeff_of(api, ctx, api.matmul(ctx, Ae, Be, mode="plain"))
    # one entry against the oracle too
    mm = O.OracleMatmul(oracle_ctx(N, L, 12), A, B, 1, 2)
    assert (ref[Nc - 1] == mm.entry(O.encode(A, O.CSR), 0, Nc - 1)).all()
    n = S.sfhe_ctx_tuning(ctx.h)["variants"]
    assert n == (5 if N == 8192 else 3)
    for v in range(n):
        S.sfhe_ctx_set_variant(ctx.h, v)
        C = api.matmul(ctx, Ae, Be)
        assert (coeff_of(api, ctx, C) == ref).all(), v
        assert (api.decrypt(ctx, C) == _centred(A @ B)).all(), v
    ctx.close()


def test_the_tuner_keeps_the_fastest_tile():
    api, S = gpu_modules()
    ctx = api.Context(8192, 4, seed=13)
    t0 = S.sfhe_ctx_tuning(ctx.h)
    assert t0["variant"] == -1 and t0["ms"] == [0.0] * 5
    A = W.sparse_int_matrix(8, 16, 0.5, -16, 16, 65)
    B = W.dense_int_matrix(16, 8, -16, 16, 66)
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    C = api.matmul(ctx, Ae, Be)
    t = S.sfhe_ctx_tuning(ctx.h)
    assert 0 <= t["variant"] < 5 and all(ms > 0 for ms in t["ms"])
    assert t["ms"][t["variant"]] == min(t["ms"])
    assert all(t["names"]) and len(set(t["names"])) == 5
    print("tuning at N = 8192, L = 4:", t)
    # the calibration wrote C of the first entries; the execution rewrote them
    plain = coeff_of(api, ctx, api.matmul(ctx, Ae, Be, mode="plain"))
    assert (coeff_of(api, ctx, C) == plain).all()
    # a ring without variants reports one and is never tuned
    ctx2 = api.Context(8192, 3, seed=13)
    assert S.sfhe_ctx_tuning(ctx2.h)["variants"] == 1
    ctx2.close()
    ctx.close()
