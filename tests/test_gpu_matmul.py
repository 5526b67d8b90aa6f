"""End-to-end parity of the encrypted matmul with the oracle: every entry
of C bit-exact in every limb, for the dense loop and the three sparse
encodings, through both the plain per-product path and the fused persistent
kernel; batches, graph replay and edge cases."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
T = 65537
ENCS = ["dense", "mask", "csr", "ell"]


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def _run(api, ctx, A_vals, B_vals, enc, mode, a_id, b_id):
    A = api.encrypt_matrix(ctx, A_vals, enc, a_id)
    B = api.encrypt_matrix(ctx, B_vals, "dense", b_id)
    C = api.matmul(ctx, A, B, dense=(enc == "dense"), mode=mode)
    return C


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


@pytest.fixture(scope="module")
def tiny(mods):
    """8x8 (50% zeros, seed 0) x 8x8, N = 4096, two primes: full C from the
    oracle for the dense loop and for the nonzero product set."""
    ring, shape = W.TINY_RING, W.TINY
    A, B = W.operands(shape)
    octx = oracle_ctx(ring.N, ring.L, 0)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    entries = [(i, j) for i in range(shape.M) for j in range(shape.Nc)]
    ref = {}
    for enc in ("dense", "csr"):
        e = O.encode(A, O.ENCODINGS[enc])
        ref[enc] = {ij: mm.entry(e, *ij) for ij in entries}
    return A, B, ref


@pytest.mark.parametrize("mode", ["persistent", "plain"])
@pytest.mark.parametrize("enc", ENCS)
def test_tiny_matmul_bit_exact(mods, tiny, enc, mode):
    api, S = mods
    A, B, ref = tiny
    ctx = gpu_ctx(W.TINY_RING.N, W.TINY_RING.L, 0)
    C = _run(api, ctx, A, B, enc, mode, 1, 2)
    got = coeff_of(api, ctx, C)
    want = ref["dense" if enc == "dense" else "csr"]
    for (i, j), ct in want.items():
        assert (got[i * B.shape[1] + j] == ct).all(), (enc, mode, i, j)
    assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


def test_sparse_encodings_identical_and_dense_decrypts_equal(mods):
    api, S = mods
    ctx = gpu_ctx(4096, 2, 0)
    A = W.sparse_int_matrix(6, 10, 0.7, -16, 16, 5)
    A[3, :] = 0
    B = W.dense_int_matrix(10, 5, -16, 16, 6)
    cts = {enc: coeff_of(api, ctx, _run(api, ctx, A, B, enc, "persistent", 3, 4)) for enc in ENCS}
    assert (cts["mask"] == cts["csr"]).all() and (cts["csr"] == cts["ell"]).all()
    # the all-zero row: no product touches it, its entries are the zero ciphertext
    assert not cts["csr"][3 * 5: 4 * 5].any()
    assert cts["dense"][3 * 5: 4 * 5].any()
    Cd = api.result_matrix(ctx, 6, 5)
    for enc in ENCS:
        C = _run(api, ctx, A, B, enc, "persistent", 3, 4)
        assert (api.decrypt(ctx, C) == _centred(A @ B)).all()


@pytest.mark.parametrize("N,L", [(8192, 4), (4096, 3)])
def test_persistent_equals_plain_and_oracle(mods, N, L):
    """The fused kernel relinearises once per entry (linearity of the NTT and
    of the key product); the plain path relinearises every product.  Both
    must give the same limbs, and the oracle's."""
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 2), oracle_ctx(N, L, 2)
    A = W.sparse_int_matrix(3, 4, 0.4, -16, 16, 8)
    A[0, :] = [1, 0, -3, 16]
    B = W.dense_int_matrix(4, 2, -16, 16, 9)
    Cp = coeff_of(api, ctx, _run(api, ctx, A, B, "csr", "persistent", 5, 6))
    Cq = coeff_of(api, ctx, _run(api, ctx, A, B, "csr", "plain", 5, 6))
    assert (Cp == Cq).all()
    mm = O.OracleMatmul(octx, A, B, 5, 6)
    enc = O.encode(A, O.CSR)
    for j in range(2):
        assert (Cp[j] == mm.entry(enc, 0, j)).all()


def test_ring_16384_L8_sampled_entry(mods):
    api, S = mods
    ctx, octx = gpu_ctx(16384, 8, 3), oracle_ctx(16384, 8, 3)
    A = np.array([[2, 0], [0, -5]], dtype=np.int64)
    B = np.array([[7, -1], [3, 8]], dtype=np.int64)
    C = _run(api, ctx, A, B, "ell", "persistent", 7, 8)
    assert (api.decrypt(ctx, C) == A @ B).all()
    got = coeff_of(api, ctx, C)
    mm = O.OracleMatmul(octx, A, B, 7, 8)
    assert (got[1] == mm.entry(O.encode(A, O.ELL), 0, 1)).all()


def test_batch_of_mixed_matmuls(mods):
    """Several matmuls of different shapes and encodings in one persistent
    launch give the same limbs as each run alone."""
    api, S = mods
    ctx = gpu_ctx(4096, 2, 0)
    specs = [(3, 5, 2, 0.5, "csr"), (4, 3, 3, 0.2, "ell"), (2, 6, 1, 0.9, "mask"), (1, 1, 1, 0.0, "dense")]
    As, Bs, alone = [], [], []
    for n, (M, K, Nc, s, enc) in enumerate(specs):
        Av = W.sparse_int_matrix(M, K, s, -8, 8, 20 + n)
        Bv = W.dense_int_matrix(K, Nc, -8, 8, 40 + n)
        A = api.encrypt_matrix(ctx, Av, enc, 100 + n)
        B = api.encrypt_matrix(ctx, Bv, "dense", 200 + n)
        As.append(A)
        Bs.append(B)
        alone.append((coeff_of(api, ctx, api.matmul(ctx, A, B)), Av @ Bv))
    Cs = api.matmul_batch(ctx, As, Bs)
    for C, (ref, plain) in zip(Cs, alone):
        assert (coeff_of(api, ctx, C) == ref).all()
        assert (api.decrypt(ctx, C) == plain).all()


def test_graph_plan_replays(mods):
    import torch
    api, S = mods
    ctx = gpu_ctx(4096, 2, 0)
    Av = W.sparse_int_matrix(5, 7, 0.5, -16, 16, 31)
    Bv = W.dense_int_matrix(7, 3, -16, 16, 32)
    A = api.encrypt_matrix(ctx, Av, "csr", 9)
    B = api.encrypt_matrix(ctx, Bv, "dense", 10)
    ref = coeff_of(api, ctx, api.matmul(ctx, A, B))
    plan = api.Plan(ctx, [A], [B], graph=True)
    assert plan.stats["launches"] == 1 and plan.stats["products"] == int((Av != 0).sum()) * 3
    for _ in range(3):
        plan.Cs[0].ct.zero_()
        plan.execute()
        torch.cuda.synchronize()
        assert (coeff_of(api, ctx, plan.Cs[0]) == ref).all()
    plan.close()


def test_edge_cases(mods):
    api, S = mods
    ctx = gpu_ctx(4096, 2, 0)
    # all-zero A: CSR / ELL store nothing and C is exactly zero; dense decrypts to 0
    Z = np.zeros((2, 3), dtype=np.int64)
    Bv = W.dense_int_matrix(3, 2, -16, 16, 50)
    for enc in ("csr", "ell", "mask"):
        C = _run(api, ctx, Z, Bv, enc, "persistent", 11, 12)
        assert not coeff_of(api, ctx, C).any()
    C = _run(api, ctx, Z, Bv, "dense", "persistent", 11, 12)
    assert (api.decrypt(ctx, C) == 0).all()
    # 1x1x1 and a product that wraps mod t
    C = _run(api, ctx, np.array([[300]]), np.array([[300]]), "csr", "plain", 13, 14)
    assert api.decrypt(ctx, C)[0, 0] == _centred(90000)
    # wrong encoding for the sparse call, mismatched shapes
    A = api.encrypt_matrix(ctx, np.array([[1, 2]]), "csr", 15)
    B = api.encrypt_matrix(ctx, np.array([[1], [2], [3]]), "dense", 16)
    with pytest.raises(S.SfheError) as e:
        api.matmul(ctx, A, B)
    assert e.value.status == S.SFHE_ESHAPE
    B2 = api.encrypt_matrix(ctx, np.array([[1], [2]]), "dense", 16)
    C = api.result_matrix(ctx, 1, 1)
    work = api.workspace(ctx, [A], [B2], api.PERSISTENT)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_matmul_sparse_view(ctx.h, A.desc(), B2.desc(), S.SFHE_ENC_ELL, C.desc(), api.PERSISTENT, work)
    assert e.value.status == S.SFHE_EINVAL
