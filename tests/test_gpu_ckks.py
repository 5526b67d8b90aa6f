"""The CKKS parameter set of Sec. 3.1 on the GPU against the CKKS oracle:
primes, encryption, the product with relinearisation, rescaling, rotations,
the mask product and the chunked matrix product of Alg. 1, every limb of
every ciphertext bit-exact (the arithmetic after encoding is exact modular
arithmetic; the encoding itself is floating point, so both sides encrypt the
same integer plaintexts, and the library's encoder is compared with the
oracle's within one unit per coefficient).  N = 64 carries the paper's prime
sizes and runs the whole chunked product; N = 8192 is the paper's ring."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import gpu_modules
from oracle import ckks as CK

pytestmark = pytest.mark.gpu


class Gpu:
    def __init__(self, S, torch, N, seed):
        self.S, self.torch, self.N = S, torch, N
        self.h = S.sfhe_ckks_ctx_create(N=N, seed=seed)
        self.q, self.P, self.scale = S.sfhe_ckks_ctx_primes(self.h, 4)
        self.L = 4
        n = max(S.sfhe_ckks_workspace_size(self.h) + 4 * self.L * N * 8 + (2 + 2 * self.L) * N * 8 * 4,
                S.sfhe_ckks_matmul_chunked_workspace_size(self.h))
        self.work = torch.empty(n, dtype=torch.uint8, device="cuda")

    def ct(self, n=1):
        return self.torch.zeros((n, 2, self.L, self.N), dtype=torch_int64(self.torch), device="cuda")

    def coeff(self, ct, level, n=1):
        out = self.ct(n)
        self.S.sfhe_ckks_to_coeff(self.h, ct, level, n, out)
        return out.cpu().numpy().view(np.uint64)

    def close(self):
        self.S.sfhe_ckks_ctx_destroy(self.h)


def torch_int64(torch):
    return torch.int64


def _encrypt(g, polys, mid, coords):
    ct = g.ct(len(polys))
    g.S.sfhe_ckks_encrypt(g.h, np.stack(polys), np.array(coords, dtype=np.int32).reshape(-1, 2), mid, ct)
    return ct


def _same(got, want, level, what):
    for c in range(2):
        for i in range(level + 1):
            assert (got[c, i] == want[c, i]).all(), (what, c, i)


@pytest.fixture(scope="module")
def small():
    api, S = gpu_modules()
    import torch
    g = Gpu(S, torch, 64, 21)
    ck = CK.OracleCkks(N=64, seed=21)
    yield g, ck
    g.close()


def test_primes_and_encoder(small):
    g, ck = small
    assert g.q == ck.q and g.P == ck.P and g.scale == 2.0 ** 40
    rng = np.random.default_rng(2)
    z = rng.uniform(-16, 16, 32)
    mine = g.S.sfhe_ckks_encode(g.h, 64, z, g.scale)
    ref = CK.encode(64, z, g.scale)
    assert np.max(np.abs(mine - ref)) <= 1
    coeff = np.array([[int(x) % q for x in ref] for q in ck.q], dtype=np.uint64)
    assert np.max(np.abs(g.S.sfhe_ckks_decode(g.h, coeff, 3, g.scale, 32) - CK.decode(64, ref, g.scale))) < 1e-9


def test_operations_limb_for_limb(small):
    g, ck = small
    S, torch = g.S, g.torch
    rng = np.random.default_rng(4)
    z1, z2 = rng.uniform(-8, 8, 32), rng.uniform(-8, 8, 32)
    m1, m2 = CK.encode(64, z1, ck.scale), CK.encode(64, z2, ck.scale)
    a = _encrypt(g, [m1], 5, [3, 4])
    b = _encrypt(g, [m2], 6, [0, 1])
    oa, ob = ck.encrypt(m1, 5, 3, 4), ck.encrypt(m2, 6, 0, 1)
    _same(g.coeff(a, 3)[0], oa, 3, "encrypt")
    x = g.ct()
    S.sfhe_ckks_mul_relin(g.h, a, b, 3, x, g.work)
    ox = ck.mul_relin(oa, ob, 3)
    _same(g.coeff(x, 3)[0], ox, 3, "mul_relin")
    S.sfhe_ckks_rescale(g.h, x, 3, 1, x, g.work)
    ox = ck.rescale(ox, 3)
    _same(g.coeff(x, 2)[0], ox, 2, "rescale")
    got = S.sfhe_ckks_decrypt(g.h, x, 2, 1, ck.scale ** 2 / ck.q[3], 32)[0]
    assert np.max(np.abs(got - z1 * z2)) < 1e-4
    rk = S.sfhe_ckks_rotkeys_create(g.h, 4)
    try:
        for k, lv in ((1, 3), (3, 3), (-2, 2)):
            src, osrc = (a, oa) if lv == 3 else (x, ox)
            r = g.ct()
            S.sfhe_ckks_rotate(g.h, rk, src, lv, k, r, g.work)
            _same(g.coeff(r, lv)[0], ck.rotate(osrc, lv, k), lv, f"rotate {k}")
    finally:
        S.sfhe_ckks_rotkeys_destroy(rk)
    mask = CK.encode(64, [1.0], float(ck.q[2]))
    pt = torch.zeros((4, 64), dtype=torch.int64, device="cuda")
    S.sfhe_ckks_plain_ntt(g.h, mask, 2, pt)
    S.sfhe_ckks_mul_plain(g.h, x, 2, 1, pt)
    _same(g.coeff(x, 2)[0], ck.mul_plain(ox, 2, mask), 2, "mul_plain")
    y = a.clone()
    S.sfhe_ckks_add(g.h, y, b, 3, 1)
    _same(g.coeff(y, 3)[0], ck.add_ct(oa.copy(), ob, 3), 3, "add")


@pytest.mark.parametrize("chunk,skip", [(1, False), (3, True), (4, False)])
def test_chunked_product_limb_for_limb(small, chunk, skip):
    g, ck = small
    S, torch = g.S, g.torch
    A = np.array([[3, 0, -7], [0, 5, 2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0]], dtype=np.int64)
    oc = CK.OracleCkksChunked(ck, A, B, chunk, 1, 2)
    want = oc.result(skip_zeros=skip)
    # the same chunks on the GPU: the oracle's plaintexts, the same stream objects
    def chunks(Mv, mid):
        flat = Mv.reshape(-1).astype(np.float64)
        polys = [CK.encode(64, flat[q * chunk:(q + 1) * chunk], ck.scale) for q in range(-(-flat.size // chunk))]
        return _encrypt(g, polys, mid, [[q, 0] for q in range(len(polys))])
    Ag, Bg = chunks(A, 1), chunks(B, 2)
    nC = -(-4 // chunk)
    C = g.ct(nC)
    rk = S.sfhe_ckks_rotkeys_create(g.h, chunk)
    try:
        az = (A == 0).astype(np.uint8).reshape(-1) if skip else None
        bz = (B == 0).astype(np.uint8).reshape(-1) if skip else None
        n, scale = S.sfhe_ckks_matmul_chunked(g.h, rk, 2, 3, 2, Ag, Bg, C, az, bz, g.work)
    finally:
        S.sfhe_ckks_rotkeys_destroy(rk)
    assert n == sum(len(v) for v in oc.product_sets(skip).values())
    assert scale == oc.result_scale
    got = g.coeff(C, 1, nC)
    for q in range(nC):
        _same(got[q], want[q], 1, f"chunk {q}")
    vals = S.sfhe_ckks_decrypt(g.h, C, 1, nC, scale, chunk).reshape(-1)[:4].reshape(2, 2)
    assert np.max(np.abs(vals - A @ B)) < 1e-3


@pytest.mark.parametrize("chunk,skip,shape", [(4, True, (8, 9, 7)), (5, False, (6, 7, 5))])
def test_chunked_product_many_batches_limb_for_limb(small, chunk, skip, shape):
    """products in several batches of the batched term-by-term product
    (64 products a batch), chunks touched by terms of several batches, every
    turn offset: each chunk limb for limb against the oracle's sequence"""
    g, ck = small
    S = g.S
    M, K, Nc = shape
    rng = np.random.default_rng(7 + chunk)
    A = rng.integers(-8, 9, (M, K))
    B = rng.integers(-8, 9, (K, Nc))
    if skip:
        A[rng.random((M, K)) < 0.4] = 0
        B[rng.random((K, Nc)) < 0.3] = 0
    oc = CK.OracleCkksChunked(ck, A, B, chunk, 1, 2)
    want = oc.result(skip_zeros=skip)
    assert sum(len(v) for v in oc.product_sets(skip).values()) > 2 * 64

    def chunks(Mv, mid):
        flat = Mv.reshape(-1).astype(np.float64)
        polys = [CK.encode(64, flat[q * chunk:(q + 1) * chunk], ck.scale) for q in range(-(-flat.size // chunk))]
        return _encrypt(g, polys, mid, [[q, 0] for q in range(len(polys))])
    Ag, Bg = chunks(A, 1), chunks(B, 2)
    nC = -(-(M * Nc) // chunk)
    C = g.ct(nC)
    rk = S.sfhe_ckks_rotkeys_create(g.h, chunk)
    try:
        az = (A == 0).astype(np.uint8).reshape(-1) if skip else None
        bz = (B == 0).astype(np.uint8).reshape(-1) if skip else None
        n, scale = S.sfhe_ckks_matmul_chunked(g.h, rk, M, K, Nc, Ag, Bg, C, az, bz, g.work)
    finally:
        S.sfhe_ckks_rotkeys_destroy(rk)
    assert n == sum(len(v) for v in oc.product_sets(skip).values())
    got = g.coeff(C, 1, nC)
    for q in range(nC):
        _same(got[q], want[q], 1, f"chunk {q}")
    vals = S.sfhe_ckks_decrypt(g.h, C, 1, nC, scale, chunk).reshape(-1)[:M * Nc].reshape(M, Nc)
    assert np.max(np.abs(vals - A @ B)) < 1e-2


def test_chunked_product_without_terms(small):
    """every product skipped: no terms, every chunk of C zero"""
    g, ck = small
    S = g.S
    A = np.zeros((2, 3), dtype=np.int64)
    B = np.ones((3, 2), dtype=np.int64)
    Ag = _encrypt(g, [CK.encode(64, [0.0] * 4, ck.scale)] * 2, 1, [[0, 0], [1, 0]])
    Bg = _encrypt(g, [CK.encode(64, [1.0] * 4, ck.scale)] * 2, 2, [[0, 0], [1, 0]])
    C = g.ct(1)
    C.fill_(5)
    rk = S.sfhe_ckks_rotkeys_create(g.h, 4)
    try:
        n, _ = S.sfhe_ckks_matmul_chunked(g.h, rk, 2, 3, 2, Ag, Bg, C, (A == 0).astype(np.uint8).reshape(-1),
                                          None, g.work)
    finally:
        S.sfhe_ckks_rotkeys_destroy(rk)
    assert n == 0
    assert not C.any()


def test_paper_ring_8192():
    """The paper's ring: encryption, the product with relinearisation and a
    rescale limb for limb against the oracle; the chunked product of a
    2 x 2 x 2 matmul at c = 4 decodes to A B."""
    api, S = gpu_modules()
    import torch
    g = Gpu(S, torch, 8192, 3)
    ck = CK.OracleCkks(N=8192, seed=3)
    try:
        assert g.q == ck.q and g.P == ck.P
        m1 = CK.encode(8192, [1.5, -2.0, 3.25], ck.scale)
        m2 = CK.encode(8192, [4.0, 0.5, -1.0], ck.scale)
        a, b = _encrypt(g, [m1], 1, [0, 0]), _encrypt(g, [m2], 2, [0, 0])
        oa, ob = ck.encrypt(m1, 1, 0, 0), ck.encrypt(m2, 2, 0, 0)
        _same(g.coeff(a, 3)[0], oa, 3, "encrypt")
        x = g.ct()
        S.sfhe_ckks_mul_relin(g.h, a, b, 3, x, g.work)
        S.sfhe_ckks_rescale(g.h, x, 3, 1, x, g.work)
        _same(g.coeff(x, 2)[0], ck.rescale(ck.mul_relin(oa, ob, 3), 3), 2, "mul_relin + rescale")
        got = S.sfhe_ckks_decrypt(g.h, x, 2, 1, ck.scale ** 2 / ck.q[3], 3)[0]
        assert np.max(np.abs(got - np.array([6.0, -1.0, -3.25]))) < 1e-3
        A = np.array([[3, -7], [5, 2]], dtype=np.int64)
        B = np.array([[2, -1], [6, 4]], dtype=np.int64)
        polysA = [S.sfhe_ckks_encode(g.h, 8192, A.reshape(-1).astype(float), g.scale)]
        polysB = [S.sfhe_ckks_encode(g.h, 8192, B.reshape(-1).astype(float), g.scale)]
        Ag, Bg = _encrypt(g, polysA, 1, [[0, 0]]), _encrypt(g, polysB, 2, [[0, 0]])
        C = g.ct(1)
        rk = S.sfhe_ckks_rotkeys_create(g.h, 4)
        try:
            n, scale = S.sfhe_ckks_matmul_chunked(g.h, rk, 2, 2, 2, Ag, Bg, C, None, None, g.work)
        finally:
            S.sfhe_ckks_rotkeys_destroy(rk)
        assert n == 8
        vals = S.sfhe_ckks_decrypt(g.h, C, 1, 1, scale, 4)[0].reshape(2, 2)
        assert np.max(np.abs(vals - A @ B)) < 1e-2
    finally:
        g.close()
