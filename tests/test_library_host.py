"""CPU checks of the C ABI library: it loads, exports every entry point the
header declares, and its host-only helpers (prime selection, error table,
sparse encoders) agree with the oracle.  No GPU is touched."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_2503_09184_gb300 import _build, sfhe
    _build.build()
    return sfhe


def _declared_functions():
    hdr = open(os.path.join(ROOT, "include", "sfhe.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(sfhe_[a-z_0-9]+)\s*\(", hdr)))


def test_header_symbols_exported(S):
    import ctypes
    lib = ctypes.CDLL(S.LIB_PATH)
    declared = _declared_functions()
    assert len(declared) >= 29
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    assert sorted(S.exported_symbols()) == declared


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 4), (16384, 8), (4096, 3)])
def test_primes_match_oracle(S, N, L):
    """Ciphertext primes equal the oracle's; the tensor base holds the exact
    tensor of two ciphertexts with the stated margins (big integers)."""
    from oracle import oracle as O
    q, b = S.sfhe_select_primes(N, L)
    assert q == O.ntt_primes(N, L)
    assert all(O.is_prime(x) and x % (2 * N) == 1 and 2**29 < x < 2**30 for x in b)
    assert b == sorted(b, reverse=True) and len(set(b)) == len(b)
    # no candidate of the form k 2N + 1 between 2^30 and the last prime is skipped
    cand = [c for c in range(b[-1], 2**30, 2 * N) if O.is_prime(c)]
    assert sorted(cand, reverse=True) == b
    Q, B = 1, 1
    for x in q:
        Q *= x
    for x in b:
        B *= x
    assert B > 2 * N * Q * Q                # |tensor| < N Q^2 / 2: |x| / B < 1/4


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 4), (16384, 8), (4096, 3), (16384, 4)])
def test_bench_sizes_the_tensor_base_like_the_library(S, N, L):
    """bench.py's config block (the same for the GPU and the reference arm)
    sizes lifted operands with the library's tensor-base formula"""
    import math
    import bench
    assert bench.tensor_base_primes(int(math.log2(N)), L) == len(S.sfhe_select_primes(N, L)[1])


def test_cdt_matches_oracle_and_golden(S):
    from oracle import oracle as O
    path = os.path.join(ROOT, "tests", "golden", "cdt_sigma3.2.txt")
    golden = [int(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")]
    assert S.sfhe_cdt_table(3.2) == O.cdt(3.2) == golden


@pytest.mark.parametrize("enc", ["dense", "mask", "csr", "ell"])
def test_encoders_match_oracle(S, enc):
    from oracle import oracle as O
    from workloads import sparse_int_matrix
    A = sparse_int_matrix(7, 9, 0.6, -16, 16, 3)
    A[2, :] = 0
    f = S.sfhe_encode_fill(A, S.ENCODINGS[enc])
    ref = O.encode(A, O.ENCODINGS[enc])
    assert f["nct"] == len(ref.values)
    assert list(f["ct_values"]) == ref.values
    assert [tuple(x) for x in f["ct_coords"][: 2 * f["nct"]].reshape(-1, 2)] == ref.coords
    if enc == "mask":
        assert (f["mask"].reshape(A.shape) == ref.mask).all()
    if enc == "csr":
        assert list(f["row_ptr"]) == list(ref.row_ptr) and list(f["col_idx"][: f["nct"]]) == list(ref.col_idx)
    if enc == "ell":
        assert f["ell_width"] == ref.width
        assert (f["ell_col"][: f["nct"]].reshape(7, ref.width) == ref.ell_col).all()


def test_encoder_edge_cases(S):
    # all-zero matrix: CSR and ELL store nothing
    Z = np.zeros((3, 4), dtype=np.int64)
    assert S.sfhe_encode_count(Z, S.SFHE_ENC_CSR) == (0, 0)
    assert S.sfhe_encode_count(Z, S.SFHE_ENC_ELL) == (0, 0)
    assert S.sfhe_encode_count(Z, S.SFHE_ENC_DENSE) == (12, 0)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_encode_count(Z, 9)
    assert e.value.status == S.SFHE_EINVAL


def test_matrix_bytes_per_encoding(S):
    """sfhe_matrix_bytes (the per-scheme memory of Sec. 4.6): ciphertexts
    2 L N words of 8 bytes each, their lift 2 K N words of 4 bytes, and the
    structure arrays each encoding keeps; on a 50%-sparse matrix CSR and
    ELL hold fewer ciphertexts than the dense and mask encodings."""
    from workloads import sparse_int_matrix
    A = sparse_int_matrix(6, 10, 0.5, -16, 16, 4)
    A[3, :] = 0
    N, L = 8192, 4
    K = len(S.sfhe_select_primes(N, L)[1])
    nnz, width = int((A != 0).sum()), int((A != 0).sum(axis=1).max())
    want_nct = {"dense": 60, "mask": 60, "csr": nnz, "ell": 6 * width}
    want_meta = {"dense": 0, "mask": 60, "csr": (6 + 1 + nnz) * 4, "ell": 6 * width * 4}
    got = {}
    for enc, e in S.ENCODINGS.items():
        f = S.sfhe_encode_fill(A, e)
        M = S.sfhe_matrix_view(6, 10, e, f["nct"], f["ell_width"], None, None, None, None, None, None)
        got[enc] = S.sfhe_matrix_bytes(N, L, M)
        assert f["nct"] == want_nct[enc]
        assert got[enc] == {"ct": want_nct[enc] * 2 * L * N * 8, "ext": want_nct[enc] * 2 * K * N * 4,
                            "meta": want_meta[enc]}, enc
    assert got["csr"]["ct"] < got["ell"]["ct"] < got["dense"]["ct"] == got["mask"]["ct"]
    with pytest.raises(S.SfheError) as e:
        S.sfhe_matrix_bytes(1000, 4, S.sfhe_matrix_view(1, 1, 0, 1, 0, None, None, None, None, None, None))
    assert e.value.status == S.SFHE_EUNSUPPORTED


@pytest.mark.parametrize("N", [16, 4096])
def test_slot_codec_matches_oracle(S, N):
    """The library's slot encoding (a fast negacyclic transform mod t) and
    the oracle's (direct evaluation and interpolation) agree on random
    vectors both ways; rotation elements are 3^k mod 2N."""
    from oracle import oracle as O
    T = 65537
    v = np.random.default_rng(N).integers(-T // 2, T // 2, size=N)
    poly = S.sfhe_slots_encode(N, T, v)
    assert (poly == O.slots_encode(N, T, v).astype(np.int64)).all()
    assert (S.sfhe_slots_decode(N, T, poly) == v % T).all()
    assert (O.slots_decode(N, T, poly.astype(np.uint64)).astype(np.int64) == v % T).all()
    for k in (0, 1, 5, -1, -3, N // 2):
        assert S.sfhe_rotation_element(N, k) == O.rotation_element(N, k) == pow(3, k % (N // 2), 2 * N)
    with pytest.raises(S.SfheError) as e:
        S.sfhe_slots_encode(N, 65539, v)          # 65539 is not 1 mod 2N
    assert e.value.status == S.SFHE_EUNSUPPORTED
