"""Alg. 1 with chunk size c > 1 (Sec. 3.2) on the GPU against the oracle,
limb for limb: encryption of whole plaintext polynomials, Galois keys,
rotations, the slot-0 mask multiply (N = 4096, L = 2), and the chunked
matmul with and without the naive sparse skip (N = 4096, L = 3: the
rotations before the multiply switch keys without a special prime, adding
noise of order N q_j sigma that the multiply scales by about t N, which two
primes cannot hold); a larger chunked matmul by decryption."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O

pytestmark = pytest.mark.gpu
T = 65537
N, L, SEED = 4096, 2, 7


def _coeff(api, ctx, ct):
    n = ct.shape[0]
    return api.to_coeff(ctx, ct.contiguous(), n)


def _setup():
    api, S = gpu_modules()
    return api, S, gpu_ctx(N, L, SEED), oracle_ctx(N, L, SEED)


def _enc_slots(api, S, ctx, vals, mid):
    import torch
    polys = np.stack([S.sfhe_slots_encode(N, T, v) for v in vals])
    coords = np.array([[q, 0] for q in range(len(vals))], dtype=np.int32)
    ct = torch.empty((len(vals), 2, L, N), dtype=torch.int64, device="cuda")
    S.sfhe_encrypt_poly(ctx.h, polys, coords, mid, ct)
    return polys, ct


def test_poly_encryption_matches_oracle():
    import torch
    api, S, ctx, octx = _setup()
    vals = np.random.default_rng(1).integers(0, T, size=(2, N))
    polys, ct = _enc_slots(api, S, ctx, vals, 9)
    got = _coeff(api, ctx, ct)
    for q in range(2):
        assert (got[q] == octx.encrypt_poly(polys[q], 9, q, 0)).all(), q
    out = torch.empty((2, N), dtype=torch.int64, device="cuda")
    S.sfhe_decrypt_poly(ctx.h, ct, 2, out)
    assert (out.cpu().numpy() == polys).all()


@pytest.mark.parametrize("k", [1, -3])
def test_rotation_matches_oracle(k):
    import torch
    api, S, ctx, octx = _setup()
    g = S.sfhe_rotation_element(N, k)
    key = torch.empty((L, 2, L, N), dtype=torch.int64, device="cuda")
    key_sh = torch.empty_like(key)
    S.sfhe_galois_keygen(ctx.h, g, key, key_sh)
    okey = octx.galois_key(g)
    assert (api.to_coeff(ctx, key.contiguous(), L) == okey).all()   # L digits x (b, a): 2L polynomials
    vals = np.random.default_rng(2).integers(0, T, size=(1, N))
    polys, ct = _enc_slots(api, S, ctx, vals, 3)
    out = torch.empty_like(ct)
    work = torch.empty(S.sfhe_rotate_workspace_size(ctx.h), dtype=torch.uint8, device="cuda")
    S.sfhe_rotate(ctx.h, ct, 1, g, key, key_sh, out, work)
    want = octx.rotate(octx.encrypt_poly(polys[0], 3, 0, 0), g, okey)
    assert (_coeff(api, ctx, out)[0] == want).all()
    dec = torch.empty((1, N), dtype=torch.int64, device="cuda")
    S.sfhe_decrypt_poly(ctx.h, out, 1, dec)
    slots = S.sfhe_slots_decode(N, T, dec.cpu().numpy()[0])
    h = N // 2
    assert (slots == np.concatenate([np.roll(vals[0][:h], -k), np.roll(vals[0][h:], -k)])).all()


def test_mul_plain_matches_oracle():
    import torch
    api, S, ctx, octx = _setup()
    rng = np.random.default_rng(3)
    vals = rng.integers(0, T, size=(1, N))
    w = rng.integers(0, T, size=N)
    polys, ct = _enc_slots(api, S, ctx, vals, 4)
    pw = S.sfhe_slots_encode(N, T, w)
    pt = torch.empty((L, N), dtype=torch.int64, device="cuda")
    S.sfhe_plain_ntt(ctx.h, pw, pt)
    S.sfhe_mul_plain(ctx.h, ct, 1, pt)
    want = octx.mul_plain(octx.encrypt_poly(polys[0], 4, 0, 0), pw.astype(np.uint64))
    assert (_coeff(api, ctx, ct)[0] == want).all()


@pytest.mark.parametrize("chunk", [3, 4])
def test_chunked_matmul_matches_oracle(chunk):
    api, S = gpu_modules()
    ctx, octx = gpu_ctx(N, 3, SEED), oracle_ctx(N, 3, SEED)
    A = np.array([[3, 0, -7], [0, 5, 2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0]], dtype=np.int64)
    oc = O.OracleChunked(octx, A, B, chunk, 1, 2)
    Ae = api.encrypt_chunked(ctx, A, chunk, 1)
    Be = api.encrypt_chunked(ctx, B, chunk, 2)
    ga = _coeff(api, ctx, Ae.ct)
    assert all((ga[q] == oc.a_ct[q]).all() for q in range(Ae.nchunks))
    rk = api.RotationKeys(ctx, chunk)
    for skip in ((False, True) if chunk == 4 else (True,)):
        C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=skip)
        assert n == (int(((A != 0).astype(int) @ (B != 0).astype(int)).sum()) if skip else 12)
        got = _coeff(api, ctx, C.ct)
        want = oc.result(skip_zeros=skip)
        for q in range(C.nchunks):
            assert (got[q] == want[q]).all(), (chunk, skip, q)
        assert (api.decrypt_chunked(ctx, C) == A @ B).all()
    rk.close()


def test_chunked_matmul_batches_equal_the_terms_one_by_one():
    """the term-by-term product runs its terms in batches; over several
    batches (chunks receiving terms from two of them, every turn offset)
    each chunk is, limb for limb, what the terms give one after another
    through the single-ciphertext calls (turn, lift, multiply + relinearise,
    mask, turn back, add: each checked against the oracle above)"""
    import torch
    api, S = gpu_modules()
    Lc, ch = 3, 4
    ctx = gpu_ctx(N, Lc, SEED)
    rng = np.random.default_rng(9)
    A = rng.integers(-16, 17, size=(12, 20)) * (rng.random((12, 20)) < 0.5)
    B = rng.integers(-16, 17, size=(20, 10))
    Ae = api.encrypt_chunked(ctx, A, ch, 1)
    Be = api.encrypt_chunked(ctx, B, ch, 2)
    rk = api.RotationKeys(ctx, ch)
    C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=True)
    terms = [(i * 20 + k, k * 10 + j, i * 10 + j) for i in range(12) for j in range(10) for k in range(20)
             if A[i, k] != 0 and B[k, j] != 0]
    assert n == len(terms) > 2 * 456
    # the same terms one by one
    shape = (1, 2, Lc, N)
    keys = {}

    def turn(ct, k):
        if k == 0:
            return ct
        g = S.sfhe_rotation_element(N, k)
        if g not in keys:
            key = torch.empty((Lc, 2, Lc, N), dtype=torch.int64, device="cuda")
            key_sh = torch.empty_like(key)
            S.sfhe_galois_keygen(ctx.h, g, key, key_sh)
            keys[g] = (key, key_sh)
        out = torch.empty(shape, dtype=torch.int64, device="cuda")
        S.sfhe_rotate(ctx.h, ct, 1, g, *keys[g], out, rot_work)
        return out

    rot_work = torch.empty(S.sfhe_rotate_workspace_size(ctx.h), dtype=torch.uint8, device="cuda")
    lift_work = torch.empty(S.sfhe_lift_workspace_size(ctx.h, 1), dtype=torch.uint8, device="cuda")
    K_ = ctx.K
    mul_work = torch.empty(((3 * K_ * N * 4 + 255) // 256) * 256 + (3 * Lc + (Lc + 2) * Lc) * N * 8,
                           dtype=torch.uint8, device="cuda")

    def lifted(M, e):
        ct = turn(M.ct[e // ch:e // ch + 1].contiguous(), e % ch)
        ext = torch.empty((1, 2, K_, N), dtype=torch.int32, device="cuda")
        S.sfhe_lift(ctx.h, ct, 1, ext, lift_work)
        return ext

    ea = {e: lifted(Ae, e) for e in {t[0] for t in terms}}
    eb = {e: lifted(Be, e) for e in {t[1] for t in terms}}
    v = np.zeros(N, dtype=np.int64)
    v[0] = 1
    mask = torch.empty((Lc, N), dtype=torch.int64, device="cuda")
    S.sfhe_plain_ntt(ctx.h, S.sfhe_slots_encode(N, T, v), mask)
    ref = torch.zeros_like(C.ct)
    for a, b, r in terms:
        prod = torch.empty(shape, dtype=torch.int64, device="cuda")
        S.sfhe_ct_mul_relin(ctx.h, ea[a], eb[b], prod, mul_work)
        S.sfhe_mul_plain(ctx.h, prod, 1, mask)
        placed = turn(prod, -(r % ch))
        S.sfhe_add(ctx.h, ref[r // ch:r // ch + 1], placed.contiguous(), 1)
    assert torch.equal(C.ct, ref)
    want = ((A @ B + T // 2) % T) - T // 2
    assert (api.decrypt_chunked(ctx, C) == want).all()
    rk.close()


def test_chunked_matmul_without_terms():
    """every product skipped (A all zero under the mask): no terms, C zero in
    both placements"""
    api, S = gpu_modules()
    ctx = gpu_ctx(N, 3, SEED)
    A = np.zeros((3, 5), dtype=np.int64)
    B = np.arange(10, dtype=np.int64).reshape(5, 2)
    Ae = api.encrypt_chunked(ctx, A, 4, 1)
    Be = api.encrypt_chunked(ctx, B, 4, 2)
    rk = api.RotationKeys(ctx, 4)
    for fused in (False, True):
        C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=True, fused=fused)
        assert n == 0
        assert not C.ct.any()
        assert (api.decrypt_chunked(ctx, C) == 0).all()
    rk.close()


def test_chunked_matmul_8192_decrypts():
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    rng = np.random.default_rng(5)
    A = rng.integers(-16, 17, size=(6, 8)) * (rng.random((6, 8)) < 0.5)
    B = rng.integers(-16, 17, size=(8, 5))
    Ae = api.encrypt_chunked(ctx, A, 8, 11)
    Be = api.encrypt_chunked(ctx, B, 8, 12)
    rk = api.RotationKeys(ctx, 8)
    C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=True)
    assert n == int(((A != 0).astype(int) @ (B != 0).astype(int)).sum())
    want = ((A @ B + T // 2) % T) - T // 2
    assert (api.decrypt_chunked(ctx, C) == want).all()
    rk.close()


def test_chunked_fused_matches_oracle():
    """operand rotations once per element, inner sums on the persistent
    kernel, mask and result rotation per entry: limb for limb the oracle's
    fused order, decrypting to A B"""
    api, S = gpu_modules()
    ctx, octx = gpu_ctx(N, 3, SEED), oracle_ctx(N, 3, SEED)
    A = np.array([[3, 0, -7, 1], [0, 5, 2, 0], [4, 4, 0, -2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0], [1, 1]], dtype=np.int64)
    oc = O.OracleChunked(octx, A, B, 4, 1, 2)
    Ae = api.encrypt_chunked(ctx, A, 4, 1)
    Be = api.encrypt_chunked(ctx, B, 4, 2)
    rk = api.RotationKeys(ctx, 4)
    for skip in (False, True):
        C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=skip, fused=True)
        assert n == (int(((A != 0).astype(int) @ (B != 0).astype(int)).sum()) if skip else A.size * B.shape[1])
        got = _coeff(api, ctx, C.ct)
        want = oc.result(skip_zeros=skip, placement="entry")
        for q in range(C.nchunks):
            assert (got[q] == want[q]).all(), (skip, q)
        assert (api.decrypt_chunked(ctx, C) == A @ B).all()
    rk.close()


def test_chunked_fused_8192_decrypts():
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    rng = np.random.default_rng(6)
    A = rng.integers(-16, 17, size=(12, 16)) * (rng.random((12, 16)) < 0.5)
    B = rng.integers(-16, 17, size=(16, 10))
    Ae = api.encrypt_chunked(ctx, A, 8, 11)
    Be = api.encrypt_chunked(ctx, B, 8, 12)
    rk = api.RotationKeys(ctx, 8)
    C, n = api.matmul_chunked(ctx, Ae, Be, rk, skip_zeros=True, fused=True)
    assert n == int(((A != 0).astype(int) @ (B != 0).astype(int)).sum())
    want = ((A @ B + T // 2) % T) - T // 2
    assert (api.decrypt_chunked(ctx, C) == want).all()
    rk.close()


def test_rotation_batches_equal_single_rotations():
    """sfhe_rotate over several ciphertexts with a workspace for two at a
    time (batches of 2 and a partial one) equals rotating each alone"""
    import torch
    api, S, ctx, octx = _setup()
    g = S.sfhe_rotation_element(N, 2)
    key = torch.empty((L, 2, L, N), dtype=torch.int64, device="cuda")
    key_sh = torch.empty_like(key)
    S.sfhe_galois_keygen(ctx.h, g, key, key_sh)
    vals = np.random.default_rng(8).integers(0, T, size=(5, N))
    _, ct = _enc_slots(api, S, ctx, vals, 6)
    one = S.sfhe_rotate_workspace_size(ctx.h)
    out = torch.empty_like(ct)
    S.sfhe_rotate(ctx.h, ct, 5, g, key, key_sh, out, torch.empty(2 * one, dtype=torch.uint8, device="cuda"))
    w1 = torch.empty(one, dtype=torch.uint8, device="cuda")
    for q in range(5):
        single = torch.empty_like(ct[q:q + 1])
        S.sfhe_rotate(ctx.h, ct[q:q + 1].contiguous(), 1, g, key, key_sh, single, w1)
        assert torch.equal(single[0], out[q]), q
