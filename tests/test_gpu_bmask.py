"""Naive sparse over both operands (Sec. 3.3.2: a product is skipped where
either operand's mask is set): the right operand MASK-encoded, the left in
each sparse encoding.  Every entry bit-exact against the oracle's
two-sided entries in every limb (per product and grouped), the product
count against its definition, entries left with no product equal to the
zero ciphertext, the dense loop still taking every k, and a full-size
64 x 64 x 64 case with both operands 50% zeros by decryption."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
T = 65537


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


def _two_sided_products(A, B):
    return int(((A != 0).astype(np.int64) @ (B != 0).astype(np.int64)).sum())


def _operands():
    A = np.array([[0, 4, 0, -7, 0, 0],
                  [13, 2, 9, 0, 0, 5],
                  [0, 0, 0, 0, 0, 0],
                  [1, -1, 2, -2, 3, -3]], dtype=np.int64)
    B = np.array([[3, 0, 2],
                  [0, 5, 1],
                  [-2, 8, 0],
                  [0, -4, 7],
                  [6, 0, 0],
                  [0, 1, -9]], dtype=np.int64)
    return A, B


@pytest.mark.parametrize("enc", ["mask", "csr", "ell"])
@pytest.mark.parametrize("mode", ["persistent", "plain", "lazy"])
def test_two_sided_bit_exact(enc, mode):
    api, S = gpu_modules()
    ctx = gpu_ctx(W.TINY_RING.N, W.TINY_RING.L, 3)
    octx = oracle_ctx(W.TINY_RING.N, W.TINY_RING.L, 3)
    A, B = _operands()
    bm = (B == 0).astype(np.uint8)
    Ae = api.encrypt_matrix(ctx, A, enc, 1)
    Be = api.encrypt_matrix(ctx, B, "mask", 2)
    plan = api.Plan(ctx, [Ae], [Be], mode=mode)
    assert plan.stats["products"] == _two_sided_products(A, B)
    plan.close()
    C = api.matmul(ctx, Ae, Be, mode=mode)
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    e = O.encode(A, O.ENCODINGS[enc])
    group = ctx.lazy_group if mode == "lazy" else 1
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            want = mm.entry(e, i, j, group=group, b_mask=bm)
            assert (got[i * B.shape[1] + j] == want).all(), (enc, mode, i, j)
    # entry (0, 0): A's nonzeros at k = 1, 3 meet zeros of B: no product at all
    assert not got[0].any()
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


def test_dense_loop_ignores_the_right_mask():
    api, S = gpu_modules()
    ctx = gpu_ctx(W.TINY_RING.N, W.TINY_RING.L, 3)
    octx = oracle_ctx(W.TINY_RING.N, W.TINY_RING.L, 3)
    A, B = _operands()
    Ae = api.encrypt_matrix(ctx, A, "dense", 1)
    Be = api.encrypt_matrix(ctx, B, "mask", 2)
    C = api.matmul(ctx, Ae, Be, dense=True)
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    e = O.encode(A, O.DENSE)
    for i, j in [(0, 0), (2, 1), (3, 2)]:
        assert (got[i * 3 + j] == mm.entry(e, i, j)).all(), (i, j)


def test_two_sided_full_size_decrypts():
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    A, B = W.operands(W.sweep(0.5))
    B = W.sparsify(B, 0.5, seed=77)
    assert 0.45 < (B == 0).mean() < 0.55
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "mask", 2)
    plan = api.Plan(ctx, [Ae], [Be])
    assert plan.stats["products"] == _two_sided_products(A, B)
    plan.execute()
    C = plan.Cs[0]
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()
    plan.close()
