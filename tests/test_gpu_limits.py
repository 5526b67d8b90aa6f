"""Entries at and past the persistent kernel's limit of 1024 products: the
sums of d0 and d1 stay lazily reduced and are folded back every 256
products, so an entry of 300 products crosses one fold (checked against
the oracle in every limb) and one of 1024 products crosses three (checked
limb for limb against the plain per-product path, which reduces after every
product, and by decryption); 1025 products are refused."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O

pytestmark = pytest.mark.gpu
T = 65537


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


def _row(n, seed):
    rng = np.random.default_rng(seed)
    vals = np.array([v for v in range(-16, 17) if v != 0])
    return vals[rng.integers(0, len(vals), size=(1, n))].astype(np.int64)


def test_entry_of_300_products_against_the_oracle():
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 4)
    A = _row(300, 1)
    B = _row(300, 2).T.copy()
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    C = api.matmul(ctx, Ae, Be, mode="persistent")
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(oracle_ctx(4096, 2, 4), A, B, 1, 2)
    assert (got[0] == mm.entry(O.encode(A, O.CSR), 0, 0)).all()
    assert api.decrypt(ctx, C)[0, 0] == _centred(int((A @ B)[0, 0]))


def test_entry_of_1024_products_equals_the_plain_path():
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 4)
    A = _row(1024, 3)
    B = _row(1024, 4).T.copy()
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    Cp = api.matmul(ctx, Ae, Be, mode="persistent")
    Cq = api.matmul(ctx, Ae, Be, mode="plain")
    assert (coeff_of(api, ctx, Cp) == coeff_of(api, ctx, Cq)).all()
    assert api.decrypt(ctx, Cp)[0, 0] == _centred(int((A @ B)[0, 0]))
    Cl = api.matmul(ctx, Ae, Be, mode="lazy")              # one group of 1024 at N = 4096
    assert api.decrypt(ctx, Cl)[0, 0] == _centred(int((A @ B)[0, 0]))


def test_entry_of_1025_products_is_refused():
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 4)
    A = _row(1025, 5)
    B = _row(1025, 6).T.copy()
    Ae = api.encrypt_matrix(ctx, A, "csr", 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2)
    with pytest.raises(S.SfheError) as e:
        api.matmul(ctx, Ae, Be, mode="persistent")
    assert e.value.status == S.SFHE_EUNSUPPORTED
