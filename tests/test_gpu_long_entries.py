"""Long output entries on the production kernel instances: the lazily
reduced sums of d0 and d1 are folded every 256 products, and the staged
N = 8192, L = 4 instance and the two-slot N = 16384, L = 8 instance run that
fold inside their own stage-S and round structure.  An entry of 300
products (one fold) is compared limb for limb with the oracle at N = 8192,
L = 4, and one of 320 products with the plain per-product path (which
reduces after every product) at N = 16384, L = 8.  Whole rows of the
64x64x64 sweep (50% zeros) are compared between the persistent and the
plain path."""
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


def _row(n, seed, lo=-16, hi=16):
    rng = np.random.default_rng(seed)
    vals = np.array([v for v in range(lo, hi + 1) if v != 0])
    return vals[rng.integers(0, len(vals), size=(1, n))].astype(np.int64)


def test_300_products_at_8192_4_against_the_oracle():
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 6)
    A = _row(300, 5)
    B = np.concatenate([_row(300, 6).T, _row(300, 7).T], axis=1)   # 300 x 2
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    C = api.matmul(ctx, Ae, Be, mode="persistent")
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(oracle_ctx(8192, 4, 6), A, B, 1, 2)
    assert (got[1] == mm.entry(O.encode(A, O.CSR), 0, 1)).all()
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


def test_320_products_at_16384_8_equal_the_plain_path():
    api, S = gpu_modules()
    ctx = gpu_ctx(16384, 8, 6)
    A = _row(320, 8, -8, 8)
    B = _row(320, 9, -8, 8).T.copy()
    Ae = api.encrypt_matrix(ctx, A, "ell", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    Cp = api.matmul(ctx, Ae, Be, mode="persistent")
    Cq = api.matmul(ctx, Ae, Be, mode="plain")
    assert (coeff_of(api, ctx, Cp) == coeff_of(api, ctx, Cq)).all()
    assert api.decrypt(ctx, Cp)[0, 0] == _centred(int((A @ B)[0, 0]))


def test_sweep_rows_persistent_equals_plain():
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    A, B = W.operands(W.sweep(0.5))
    rows = [0, 37]
    Ae = api.encrypt_matrix(ctx, A[rows], "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    Cp = coeff_of(api, ctx, api.matmul(ctx, Ae, Be, mode="persistent"))
    Cq = coeff_of(api, ctx, api.matmul(ctx, Ae, Be, mode="plain"))
    assert (Cp == Cq).all()
