"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (persistent kernel): every entry through decryption
(= A B mod t), the three sparse encodings bit-identical to each other over
the whole matrix, and sampled entries (shortest and longest rows) bit-exact
against the oracle in every limb."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
T = W.T_PLAIN


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


def _row_extremes(A):
    nnz = (A != 0).sum(axis=1)
    rows = [i for i in range(A.shape[0]) if nnz[i] > 0]
    return min(rows, key=lambda i: nnz[i]), max(rows, key=lambda i: nnz[i])


def test_sweep_50_full_size(mods):
    """64x64x64 at 50% zeros, N = 8192, four primes: the benchmark's input."""
    import torch
    api, S = mods
    ring = W.SWEEP_RING
    A, B = W.operands(W.sweep(0.5))
    ctx = gpu_ctx(ring.N, ring.L, 0)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    res = {}
    for enc in ("csr", "mask", "ell"):
        Ae = api.encrypt_matrix(ctx, A, enc, 1)
        C = api.matmul(ctx, Ae, Be, mode="persistent")
        assert (api.decrypt(ctx, C) == _centred(A @ B)).all(), enc
        res[enc] = coeff_of(api, ctx, C)
        del Ae
        torch.cuda.empty_cache()
    assert (res["csr"] == res["mask"]).all() and (res["csr"] == res["ell"]).all()
    octx = oracle_ctx(ring.N, ring.L, 0)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    enc = O.encode(A, O.CSR)
    lo, hi = _row_extremes(A)
    for (i, j) in [(lo, 0), (hi, B.shape[1] - 1)]:
        assert (res["csr"][i * B.shape[1] + j] == mm.entry(enc, i, j)).all(), (i, j)


@pytest.mark.parametrize("s", [0.0, 0.1, 0.3, 0.7, 0.9, 0.99])
def test_sweep_sparsities_decrypt(mods, s):
    api, S = mods
    ring = W.SWEEP_RING
    A, B = W.operands(W.sweep(s))
    ctx = gpu_ctx(ring.N, ring.L, 0)
    Ae = api.encrypt_matrix(ctx, A, "ell", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    C = api.matmul(ctx, Ae, Be, mode="persistent")
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


def test_sweep_dense_loop_decrypts_equal(mods):
    api, S = mods
    ring = W.SWEEP_RING
    A, B = W.operands(W.sweep(0.5))
    ctx = gpu_ctx(ring.N, ring.L, 0)
    Ae = api.encrypt_matrix(ctx, A, "dense", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    C = api.matmul(ctx, Ae, Be, dense=True, mode="persistent")
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


@pytest.mark.parametrize("s", [0.5, 0.9])
def test_layer_shape(mods, s):
    """128x256 weights at s zeros times 256x16 activations, ints in [-8, 8]."""
    api, S = mods
    ring = W.LAYER_RING
    A, B = W.operands(W.layer(s))
    ctx = gpu_ctx(ring.N, ring.L, 0)
    Ae = api.encrypt_matrix(ctx, A, "csr", 21)
    Be = api.encrypt_matrix(ctx, B, "dense", 22)
    C = api.matmul(ctx, Ae, Be, mode="persistent")
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()
    if s == 0.9:
        octx = oracle_ctx(ring.N, ring.L, 0)
        mm = O.OracleMatmul(octx, A, B, 21, 22)
        lo, _ = _row_extremes(A)
        got = coeff_of(api, ctx, C, slice(lo * 16, lo * 16 + 1))
        assert (got[0] == mm.entry(O.encode(A, O.CSR), lo, 0)).all()


def test_mixed_ring_sampled(mods):
    """N = 16384, eight primes: the smallest matmul of the mixed workload,
    decrypted in full, one entry of its shortest row against the oracle."""
    api, S = mods
    ring = W.MIXED_RING
    shapes = W.mixed()
    shape = min(shapes, key=lambda m: m.M * m.K * m.Nc)
    A, B = W.operands(shape)
    ctx = gpu_ctx(ring.N, ring.L, 0)
    Ae = api.encrypt_matrix(ctx, A, "csr", 31)
    Be = api.encrypt_matrix(ctx, B, "dense", 32)
    C = api.matmul(ctx, Ae, Be, mode="persistent")
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()
    lo, _ = _row_extremes(A)
    if (A[lo] != 0).sum() <= 4:
        octx = oracle_ctx(ring.N, ring.L, 0)
        mm = O.OracleMatmul(octx, A, B, 31, 32)
        got = coeff_of(api, ctx, C, slice(lo * shape.Nc, lo * shape.Nc + 1))
        assert (got[0] == mm.entry(O.encode(A, O.CSR), lo, 0)).all()
