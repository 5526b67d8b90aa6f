"""The library-owned matrix calls and the host-buffer matmul through the C
ABI, at the tiny configuration (8x8 at 50% zeros times 8x8, N = 4096, two
primes): the paper's problem statement as calls -- encrypted A and B with
their structure in, the encrypted product out.  Every ciphertext a handle
holds is compared limb for limb with the oracle's, and every product with
the oracle's entries or with the descriptor path (itself oracle-checked)."""
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


@pytest.fixture(scope="module")
def tiny(mods):
    ring = W.TINY_RING
    A, B = W.operands(W.TINY)
    A = A.copy()
    A[5, :] = 0                      # an all-zero row: its entries are the zero ciphertext
    octx = oracle_ctx(ring.N, ring.L, 0)
    mm = O.OracleMatmul(octx, A, B, 1, 2)
    return A, B, octx, mm


def _centred(x):
    return ((np.asarray(x) + T // 2) % T) - T // 2


def _export(S, ctx, M):
    info = S.sfhe_matrix_info(M)
    out = np.zeros((max(info["nct"], 1), 2, ctx.L, ctx.N), dtype=np.uint64)
    S.sfhe_matrix_export(M, out)
    return out[:info["nct"]]


def _idx(enc_name, e: "O.Encoded"):
    """the structure array sfhe_matrix_import takes for an encoding"""
    if enc_name == "dense":
        return None
    if enc_name == "mask":
        return e.mask.reshape(-1).astype(np.int32)
    if enc_name == "csr":
        return np.concatenate([e.row_ptr, e.col_idx]).astype(np.int32)
    return np.concatenate([[e.width], e.ell_col.reshape(-1)]).astype(np.int32)


def test_get_primes(mods):
    api, S = mods
    ctx = gpu_ctx(4096, 2, 0)
    q, p = S.sfhe_ctx_get_primes(ctx.h)
    assert q == O.ntt_primes(4096, 2) == ctx.q
    assert p == S.sfhe_select_primes(4096, 2)[1] == ctx.b


@pytest.mark.parametrize("enc", ENCS)
def test_encrypt_export_decrypt_and_matmul(mods, tiny, enc):
    """sfhe_matrix_encrypt stores exactly the oracle's ciphertexts of the
    encoding's stored elements; the matmul of handles gives the oracle's
    entries (sampled: rows 0, 3 and the zero row 5, every column) and the
    descriptor path's C everywhere; decryption is A B mod t."""
    api, S = mods
    A, B, octx, mm = tiny
    ctx = gpu_ctx(4096, 2, 0)
    e = O.encode(A, O.ENCODINGS[enc])
    Ah = S.sfhe_matrix_encrypt(ctx.h, A, S.ENCODINGS[enc], 1)
    Bh = S.sfhe_matrix_encrypt(ctx.h, B, S.SFHE_ENC_DENSE, 2)
    try:
        info = S.sfhe_matrix_info(Ah)
        assert info == {"rows": 8, "cols": 8, "encoding": S.ENCODINGS[enc], "nct": len(e.values)}
        got = _export(S, ctx, Ah)
        for t, (r, c) in enumerate(e.coords):
            assert (got[t] == mm.ct_a(r, c)).all(), (enc, t)
        dec = S.sfhe_matrix_decrypt(ctx.h, Ah)
        assert (dec == A).all()
        if enc == "dense":
            Ch = S.sfhe_matmul_dense(ctx.h, Ah, Bh)
        else:
            Ch = S.sfhe_matmul_sparse(ctx.h, Ah, Bh, S.ENCODINGS[enc])
        C = _export(S, ctx, Ch)
        assert C.shape[0] == 64
        ref_enc = O.encode(A, O.DENSE if enc == "dense" else O.CSR)
        for i in (0, 3, 5):
            for j in range(8):
                assert (C[i * 8 + j] == mm.entry(ref_enc, i, j)).all(), (enc, i, j)
        # the descriptor path on the same inputs, every entry
        Av = api.encrypt_matrix(ctx, A, enc, 1)
        Bv = api.encrypt_matrix(ctx, B, "dense", 2)
        Cv = api.matmul(ctx, Av, Bv, dense=(enc == "dense"))
        assert (C == coeff_of(api, ctx, Cv)).all()
        assert (S.sfhe_matrix_decrypt(ctx.h, Ch) == _centred(A @ B)).all()
        S.sfhe_matrix_destroy(Ch)
    finally:
        S.sfhe_matrix_destroy(Ah)
        S.sfhe_matrix_destroy(Bh)


@pytest.mark.parametrize("enc", ["mask", "csr", "ell"])
def test_import_of_oracle_ciphertexts(mods, tiny, enc):
    """sfhe_matrix_import of the oracle's own ciphertexts (coefficient form)
    with the encoding's structure array: exported back unchanged, and the
    sparse matmul of the imports gives the oracle's entries."""
    api, S = mods
    A, B, octx, mm = tiny
    ctx = gpu_ctx(4096, 2, 0)
    e = O.encode(A, O.ENCODINGS[enc])
    a_ct = np.stack([mm.ct_a(r, c) for r, c in e.coords]) if e.coords else np.zeros((0, 2, 2, 4096), np.uint64)
    b_ct = np.stack([mm.ct_b(k, j) for k in range(8) for j in range(8)])
    Ah = S.sfhe_matrix_import(ctx.h, a_ct, _idx(enc, e), 8, 8, S.ENCODINGS[enc])
    Bh = S.sfhe_matrix_import(ctx.h, b_ct, None, 8, 8, S.SFHE_ENC_DENSE)
    try:
        assert (_export(S, ctx, Ah) == a_ct).all()
        assert (_export(S, ctx, Bh) == b_ct).all()
        Ch = S.sfhe_matmul_sparse(ctx.h, Ah, Bh, S.ENCODINGS[enc])
        C = _export(S, ctx, Ch)
        csr = O.encode(A, O.CSR)
        for i in (0, 3, 5, 7):
            for j in (0, 4, 7):
                assert (C[i * 8 + j] == mm.entry(csr, i, j)).all(), (enc, i, j)
        assert (S.sfhe_matrix_decrypt(ctx.h, Ch) == _centred(A @ B)).all()
        S.sfhe_matrix_destroy(Ch)
    finally:
        S.sfhe_matrix_destroy(Ah)
        S.sfhe_matrix_destroy(Bh)


def test_import_rejects_bad_inputs(mods, tiny):
    api, S = mods
    A, B, octx, mm = tiny
    ctx = gpu_ctx(4096, 2, 0)
    b_ct = np.stack([mm.ct_b(k, j) for k in range(2) for j in range(2)])
    bad = b_ct.copy()
    bad[1, 0, 1, 17] = ctx.q[1]                        # a residue equal to its prime
    with pytest.raises(S.SfheError) as ex:
        S.sfhe_matrix_import(ctx.h, bad, None, 2, 2, S.SFHE_ENC_DENSE)
    assert ex.value.status == S.SFHE_EINVAL
    with pytest.raises(S.SfheError) as ex:           # CSR row pointers that go backwards
        S.sfhe_matrix_import(ctx.h, b_ct, np.array([0, 3, 2, 0, 1, 0], np.int32), 2, 2, S.SFHE_ENC_CSR)
    assert ex.value.status == S.SFHE_EINVAL
    with pytest.raises(S.SfheError) as ex:           # ELL width wider than the matrix
        S.sfhe_matrix_import(ctx.h, b_ct, np.array([3, 0, 1, -1, 0, 1, -1], np.int32), 2, 2, S.SFHE_ENC_ELL)
    assert ex.value.status == S.SFHE_EINVAL


def test_batch_chain_and_views(mods, tiny):
    """sfhe_matmul_batch equals the single calls; a handle's view runs in a
    caller-built plan with the same limbs; shape, encoding and context errors
    are reported before any launch."""
    import torch
    api, S = mods
    A, B, octx, mm = tiny
    ctx = gpu_ctx(4096, 2, 0)
    A2 = W.sparse_int_matrix(3, 8, 0.6, -4, 4, 77)
    hs = [S.sfhe_matrix_encrypt(ctx.h, A, S.SFHE_ENC_CSR, 1), S.sfhe_matrix_encrypt(ctx.h, B, S.SFHE_ENC_DENSE, 2),
          S.sfhe_matrix_encrypt(ctx.h, A2, S.SFHE_ENC_ELL, 3)]
    Ah, Bh, A2h = hs
    try:
        C1 = S.sfhe_matmul_sparse(ctx.h, Ah, Bh, S.SFHE_ENC_CSR)
        C2 = S.sfhe_matmul_sparse(ctx.h, A2h, Bh, S.SFHE_ENC_ELL)
        hs += [C1, C2]
        Cb = S.sfhe_matmul_batch(ctx.h, [Ah, A2h], [Bh, Bh], S.SFHE_EXEC_PERSISTENT)
        hs += Cb
        assert (_export(S, ctx, Cb[0]) == _export(S, ctx, C1)).all()
        assert (_export(S, ctx, Cb[1]) == _export(S, ctx, C2)).all()
        # views of handles in a plan
        Av, Bv = S.sfhe_matrix_view_of(Ah), S.sfhe_matrix_view_of(Bh)
        Cp = api.result_matrix(ctx, 8, 8)
        work = torch.empty(S.sfhe_matmul_workspace_size(ctx.h, [Av], [Bv], S.SFHE_EXEC_PERSISTENT),
                           dtype=torch.uint8, device="cuda")
        plan = S.sfhe_plan_create(ctx.h, [Av], [Bv], [Cp.desc()], S.SFHE_EXEC_PERSISTENT, work)
        S.sfhe_plan_execute(plan)
        torch.cuda.synchronize()
        S.sfhe_plan_destroy(plan)
        assert (coeff_of(api, ctx, Cp) == _export(S, ctx, C1)).all()
        # errors: shapes, a foreign context, the wrong encoding
        with pytest.raises(S.SfheError) as ex:
            S.sfhe_matmul_dense(ctx.h, A2h, A2h)
        assert ex.value.status == S.SFHE_ESHAPE
        with pytest.raises(S.SfheError) as ex:
            S.sfhe_matmul_sparse(ctx.h, Ah, Bh, S.SFHE_ENC_ELL)
        assert ex.value.status == S.SFHE_EINVAL
        other = gpu_ctx(4096, 2, 5)
        with pytest.raises(S.SfheError) as ex:
            S.sfhe_matmul_sparse(other.h, Ah, Bh, S.SFHE_ENC_CSR)
        assert ex.value.status == S.SFHE_EINVAL
    finally:
        for h in hs:
            S.sfhe_matrix_destroy(h)


def test_result_as_operand(mods):
    """A result handle used as the left operand of the next product is lifted
    on first use: (A x B) x D decrypts to the integer product of the three.
    Two multiplications in a row need L = 3 at N = 4096 (the noise of the
    first product's relinearisation, without a special prime, is about
    N q sigma; the second multiplies it by about t N)."""
    api, S = mods
    ctx = gpu_ctx(4096, 3, 0)
    A = W.sparse_int_matrix(3, 5, 0.5, -4, 4, 91)
    B = W.dense_int_matrix(5, 4, -4, 4, 92)
    D = W.sparse_int_matrix(4, 2, 0.3, -4, 4, 93)
    hs = [S.sfhe_matrix_encrypt(ctx.h, A, S.SFHE_ENC_CSR, 1), S.sfhe_matrix_encrypt(ctx.h, B, S.SFHE_ENC_DENSE, 2),
          S.sfhe_matrix_encrypt(ctx.h, D, S.SFHE_ENC_DENSE, 3)]
    try:
        hs.append(S.sfhe_matmul_sparse(ctx.h, hs[0], hs[1], S.SFHE_ENC_CSR))
        hs.append(S.sfhe_matmul_dense(ctx.h, hs[3], hs[2]))
        assert (S.sfhe_matrix_decrypt(ctx.h, hs[3]) == _centred(A @ B)).all()
        assert (S.sfhe_matrix_decrypt(ctx.h, hs[4]) == _centred(A @ B @ D)).all()
    finally:
        for h in hs:
            S.sfhe_matrix_destroy(h)


@pytest.mark.parametrize("flags_name,depth", [("PERSISTENT", 2), ("PERSISTENT", 1), ("PLAIN", 2)])
def test_host_plan_matches_device_path(mods, tiny, flags_name, depth):
    """sfhe_matmul_host: host ciphertexts in, host C out, three calls in a
    row (the pipelined buffer sets are reused), each C equal limb for limb
    to the device path's, which the oracle checks."""
    import torch
    api, S = mods
    A, B, octx, mm = tiny
    ctx = gpu_ctx(4096, 2, 0)
    Av = api.encrypt_matrix(ctx, A, "csr", 1)
    Bv = api.encrypt_matrix(ctx, B, "dense", 2)
    ref = api.matmul(ctx, Av, Bv)
    flags = getattr(S, "SFHE_EXEC_" + flags_name)
    hp = S.sfhe_host_plan_create(ctx.h, [Av.desc()], [Bv.desc()], flags, depth)
    try:
        st = S.sfhe_host_plan_stats(hp)
        ct_bytes = 2 * ctx.L * ctx.N * 8
        assert st["products"] == int((A != 0).sum()) * 8
        assert st["h2d_bytes"] == (Av.nct + Bv.nct) * ct_bytes and st["d2h_bytes"] == 64 * ct_bytes
        h_a = Av.ct.cpu().pin_memory()
        h_b = Bv.ct.cpu().pin_memory()
        outs = [torch.zeros(ref.ct.shape, dtype=torch.int64).pin_memory() for _ in range(3)]
        for o in outs:
            S.sfhe_matmul_host(hp, [h_a], [h_b], [o])
        torch.cuda.synchronize()
        want = ref.ct.cpu()
        for o in outs:
            assert (o == want).all()
    finally:
        S.sfhe_host_plan_destroy(hp)
    with pytest.raises(S.SfheError) as ex:
        S.sfhe_host_plan_create(ctx.h, [Av.desc()], [Bv.desc()], flags, 3)
    assert ex.value.status == S.SFHE_EINVAL
