"""The grouped accumulate-then-round mode (SFHE_EXEC_LAZY) against the
oracle's grouped entries, limb for limb: each output entry's products in
ascending k, in groups of G = sfhe_info.lazy_group, every group's exact
tensors summed, rounded once and relinearised once.  Covers the tiny shape
in every sparse encoding and the dense loop, entries split into several
groups (a partial last one), the N = 16384 path, the full sweep size by
decryption, and the flag's preconditions."""
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


def _lazy(api, ctx, A_vals, B_vals, enc):
    A = api.encrypt_matrix(ctx, A_vals, enc, 1)
    B = api.encrypt_matrix(ctx, B_vals, "dense", 2)
    return api.matmul(ctx, A, B, dense=(enc == "dense"), mode="lazy")


def _check_entries(api, ctx, octx, A_vals, B_vals, enc, entries=None):
    C = _lazy(api, ctx, A_vals, B_vals, enc)
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(octx, A_vals, B_vals, 1, 2)
    e = O.encode(A_vals, O.ENCODINGS[enc])
    Nc = B_vals.shape[1]
    for i, j in entries or [(i, j) for i in range(A_vals.shape[0]) for j in range(Nc)]:
        assert (got[i * Nc + j] == mm.entry(e, i, j, group=ctx.lazy_group)).all(), (enc, i, j)
    assert (api.decrypt(ctx, C) == _centred(A_vals @ B_vals)).all()


@pytest.mark.parametrize("enc", ["csr", "ell", "mask", "dense"])
def test_lazy_tiny_bit_exact(enc):
    api, _ = gpu_modules()
    ctx = gpu_ctx(W.TINY_RING.N, W.TINY_RING.L, 0)
    assert ctx.lazy_group > 8                     # one group holds a whole entry here
    A, B = W.operands(W.TINY)
    _check_entries(api, ctx, oracle_ctx(W.TINY_RING.N, W.TINY_RING.L, 0), A, B, enc)


def test_lazy_entries_split_into_groups():
    """N = 8192, four primes: G = 15, entries of about 31 products (groups of
    15, 15 and a partial last one)."""
    api, _ = gpu_modules()
    ctx = gpu_ctx(8192, 4, 1)
    assert 1 < ctx.lazy_group < 31
    A, B = W.operands(W.MatmulShape(2, 34, 2, 0.1, -16, 16, 21))
    assert (A != 0).sum(axis=1).min() > ctx.lazy_group
    _check_entries(api, ctx, oracle_ctx(8192, 4, 1), A, B, "csr")


def test_lazy_ring_16384_L8():
    api, _ = gpu_modules()
    ctx = gpu_ctx(16384, 8, 1)
    A, B = W.operands(W.MatmulShape(1, 5, 2, 0.0, -8, 8, 22))
    _check_entries(api, ctx, oracle_ctx(16384, 8, 1), A, B, "csr", entries=[(0, 1)])


def test_lazy_full_sweep_decrypts():
    api, _ = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    A, B = W.operands(W.sweep(0.5))
    C = _lazy(api, ctx, A, B, "csr")
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


def test_lazy_needs_persistent():
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 0)
    A = api.encrypt_matrix(ctx, np.array([[1, 2]]), "csr", 3)
    B = api.encrypt_matrix(ctx, np.array([[1], [2]]), "dense", 4)
    C = api.result_matrix(ctx, 1, 1)
    work = api.workspace(ctx, [A], [B], api.PERSISTENT)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_matmul_sparse_view(ctx.h, A.desc(), B.desc(), S.SFHE_ENC_CSR, C.desc(), api.PLAIN | api.LAZY, work)
    assert e.value.status == S.SFHE_EINVAL
