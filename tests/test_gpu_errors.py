"""Host-side validation of the C ABI (a GPU context is needed to reach it;
no kernel runs on bad input): workspaces that are too small, corrupted
CSR / ELLPACK arrays, bad Galois elements, aliasing, rotation keys of
another context and chunk sizes out of range each return their status."""
from __future__ import annotations


import numpy as np
import pytest

from gpu_common import gpu_ctx, gpu_modules

pytestmark = pytest.mark.gpu


def _status(S, fn, *args):
    with pytest.raises(S.SfheError) as e:
        fn(*args)
    return e.value.status


def test_small_workspaces_are_refused():
    import torch
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 0)
    A = api.encrypt_matrix(ctx, np.array([[1, 0, 2]]), "csr", 1)
    B = api.encrypt_matrix(ctx, np.array([[1], [2], [3]]), "dense", 2)
    C = api.result_matrix(ctx, 1, 1)
    tiny = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert _status(S, S.sfhe_matmul_sparse_view, ctx.h, A.desc(), B.desc(), S.SFHE_ENC_CSR, C.desc(), api.PERSISTENT,
                   tiny) == S.SFHE_ENOMEM
    ext = torch.empty((1, 2, ctx.K, ctx.N), dtype=torch.int32, device="cuda")
    assert _status(S, S.sfhe_lift, ctx.h, A.ct, 1, ext, tiny) == S.SFHE_ENOMEM
    g = S.sfhe_rotation_element(ctx.N, 1)
    key = torch.empty((ctx.L, 2, ctx.L, ctx.N), dtype=torch.int64, device="cuda")
    key_sh = torch.empty_like(key)
    S.sfhe_galois_keygen(ctx.h, g, key, key_sh)
    out = torch.empty_like(A.ct)
    assert _status(S, S.sfhe_rotate, ctx.h, A.ct, 1, g, key, key_sh, out, tiny) == S.SFHE_ENOMEM
    work = torch.empty(S.sfhe_rotate_workspace_size(ctx.h), dtype=torch.uint8, device="cuda")
    assert _status(S, S.sfhe_rotate, ctx.h, A.ct, 1, g, key, key_sh, A.ct, work) == S.SFHE_EINVAL   # aliasing
    assert _status(S, S.sfhe_rotate, ctx.h, A.ct, 1, g + 1, key, key_sh, out, work) == S.SFHE_EINVAL  # even g
    assert _status(S, S.sfhe_galois_keygen, ctx.h, 2 * ctx.N + 1, key, key_sh) == S.SFHE_EINVAL


def test_corrupted_structure_arrays_are_refused():
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 2, 0)
    A = api.encrypt_matrix(ctx, np.array([[1, 0, 2], [0, 3, 0]]), "csr", 1)
    B = api.encrypt_matrix(ctx, np.array([[1], [2], [3]]), "dense", 2)
    A.col_idx = A.col_idx.copy()
    A.col_idx[1] = 7                                    # column out of range
    assert _status(S, api.workspace, ctx, [A], [B], api.PERSISTENT) == S.SFHE_EINVAL
    A.col_idx[1] = 2
    A.row_ptr = A.row_ptr.copy()
    A.row_ptr[1], A.row_ptr[2] = 3, 2                   # not monotone
    assert _status(S, api.workspace, ctx, [A], [B], api.PERSISTENT) in (S.SFHE_EINVAL, S.SFHE_ESHAPE)
    E = api.encrypt_matrix(ctx, np.array([[1, 0, 2], [0, 3, 0]]), "ell", 3)
    E.ell_col = E.ell_col.copy()
    E.ell_col[0] = -2                                   # below the padding sentinel
    assert _status(S, api.workspace, ctx, [E], [B], api.PERSISTENT) == S.SFHE_EINVAL


def test_chunked_arguments_are_checked():
    import torch
    api, S = gpu_modules()
    ctx = gpu_ctx(4096, 3, 0)
    other = gpu_ctx(4096, 3, 1)
    assert _status(S, S.sfhe_rotkeys_create, ctx.h, 0) == S.SFHE_ESHAPE
    assert _status(S, S.sfhe_rotkeys_create, ctx.h, ctx.N) == S.SFHE_ESHAPE
    rk = api.RotationKeys(other, 2)
    A = api.encrypt_chunked(ctx, np.array([[1, 2], [3, 4]]), 2, 1)
    B = api.encrypt_chunked(ctx, np.array([[1, 0], [0, 1]]), 2, 2)
    C = torch.empty_like(A.ct)
    work = torch.empty(S.sfhe_matmul_chunked_workspace_size(ctx.h), dtype=torch.uint8, device="cuda")
    assert _status(S, S.sfhe_matmul_chunked, ctx.h, rk.h, 2, 2, 2, A.ct, B.ct, C, None, None,
                   work) == S.SFHE_EINVAL                       # keys of another context
    rk.close()
    rk = api.RotationKeys(ctx, 2)
    assert _status(S, S.sfhe_matmul_chunked, ctx.h, rk.h, 2, 2, 2, A.ct, B.ct, C, None, None,
                   work[:1024]) == S.SFHE_ENOMEM
    rk.close()
