"""Shared fixtures of the GPU parity tests: build/load the CUDA library and
keep one GPU context and one oracle context per (N, L, seed)."""
from __future__ import annotations

import functools

import numpy as np
import pytest

from oracle import oracle as O


def gpu_modules():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_09184_gb300 import _build
    _build.build()
    from paper_2503_09184_gb300 import api, sfhe
    return api, sfhe


@functools.lru_cache(maxsize=None)
def gpu_ctx(N: int, L: int, seed: int):
    api, _ = gpu_modules()
    return api.Context(N, L, seed=seed)


@functools.lru_cache(maxsize=None)
def oracle_ctx(N: int, L: int, seed: int):
    return O.OracleCtx(N, L, seed=seed)


def coeff_of(api, ctx, M, idx=None) -> np.ndarray:
    """coefficient form [n][2][L][N] of M's ciphertexts (or a subset)."""
    ct = M.ct if idx is None else M.ct[idx]
    n = ct.shape[0]
    return api.to_coeff(ctx, ct.contiguous(), n)


def oracle_expected(octx, A, B, enc_name, entries, a_id, b_id, cache=None):
    """{(i, j): oracle ciphertext} for the listed entries."""
    mm = cache if cache is not None else O.OracleMatmul(octx, A, B, a_id, b_id)
    enc = O.encode(A, O.ENCODINGS[enc_name])
    return {(i, j): mm.entry(enc, i, j) for (i, j) in entries}, mm
