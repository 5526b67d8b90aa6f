"""Python view of the plain CPU oracle (oracle/bfv_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py may import this module.  It shares no
code with the CUDA path (paper_2503_09184_gb300) and never imports it.

Layouts: a ciphertext is a uint64 array [2][L][N] in coefficient form with
canonical residues in [0, q_i) (c0 first, then c1).  Besides the
per-element form (value in the constant coefficient), OracleChunked runs
Alg. 1 over chunks of c values per ciphertext (Sec. 3.2: slots, rotations,
the slot-0 mask).

The encodings follow Sec. 3.3.2 of the paper ("Exploiting Unstructured
Sparsity in Fully Homomorphic Encrypted DNNs"):
  * naive dense (Alg. 1): every k of the shared dimension;
  * naive sparse: a plaintext mask B_ik = [A_ik == 0], products skipped where
    the mask is set; when the right operand carries its mask too, a product
    is skipped where either mask is set (the condition of Sec. 3.3.2 over
    both operands; `b_mask` below);
  * CSR: nonzeros of each row with a row-pointer array and a column array;
  * ELLPACK: each row holds j = max nonzeros-per-row slots, the nonzeros first
    and encrypted zero padding after, with a parallel column matrix.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build_oracle

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.or_is_prime.argtypes = [ctypes.c_uint64]
        L.or_is_prime.restype = ctypes.c_int
        L.or_ntt_primes.argtypes = [ctypes.c_int, ctypes.c_int, _u64p]
        L.or_psi.argtypes = [ctypes.c_uint64, ctypes.c_int]
        L.or_psi.restype = ctypes.c_uint64
        L.or_ntt_naive.argtypes = [ctypes.c_uint64, ctypes.c_int, _u64p, _u64p]
        L.or_intt_naive.argtypes = [ctypes.c_uint64, ctypes.c_int, _u64p, _u64p]
        L.or_negacyclic.argtypes = [ctypes.c_uint64, ctypes.c_int, _u64p, _u64p, _u64p]
        L.or_prng_word.argtypes = [ctypes.c_uint64] * 6
        L.or_prng_word.restype = ctypes.c_uint64
        L.or_cdt.argtypes = [ctypes.c_double, _u64p]
        L.or_ctx_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64]
        L.or_ctx_create.restype = ctypes.c_void_p
        L.or_ctx_free.argtypes = [ctypes.c_void_p]
        L.or_ctx_info.argtypes = [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 4 + [_u64p] * 3
        L.or_get_secret.argtypes = [ctypes.c_void_p, _i64p]
        L.or_get_rlk.argtypes = [ctypes.c_void_p, _u64p]
        L.or_get_cdt.argtypes = [ctypes.c_void_p, _u64p]
        L.or_get_delta.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_int]
        L.or_encrypt.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _u64p]
        L.or_encrypt.restype = ctypes.c_int
        L.or_decrypt.argtypes = [ctypes.c_void_p, _u64p, _i64p, ctypes.POINTER(ctypes.c_int)]
        L.or_tensor_scale.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p]
        L.or_tensor_scale_sum.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_u64p),
                                          ctypes.POINTER(_u64p), _u64p]
        L.or_tensor_scale_sum.restype = ctypes.c_int
        L.or_relin.argtypes = [ctypes.c_void_p, _u64p, _u64p]
        L.or_mul_relin.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p]
        L.or_add.argtypes = [ctypes.c_void_p, _u64p, _u64p]
        L.or_matmul_entries.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(_u64p), ctypes.POINTER(_u64p), _u64p, ctypes.c_int]
        L.or_matmul_entries_grouped.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(_u64p), ctypes.POINTER(_u64p), _u64p, ctypes.c_int,
                                                ctypes.c_int]
        L.or_matmul_entries_grouped.restype = ctypes.c_int
        L.or_num_threads.restype = ctypes.c_int
        L.or_slots_encode.argtypes = [ctypes.c_int, ctypes.c_uint64, _u64p, _u64p]
        L.or_slots_decode.argtypes = [ctypes.c_int, ctypes.c_uint64, _u64p, _u64p]
        L.or_encrypt_poly.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _u64p]
        L.or_encrypt_poly.restype = ctypes.c_int
        L.or_decrypt_poly.argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.POINTER(ctypes.c_int)]
        L.or_galois_key.argtypes = [ctypes.c_void_p, ctypes.c_uint64, _u64p]
        L.or_galois_key.restype = ctypes.c_int
        L.or_rotate.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64, _u64p, _u64p]
        L.or_mul_plain.argtypes = [ctypes.c_void_p, _u64p, _u64p, _u64p]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.uint64:
        return a.ctypes.data_as(_u64p)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_i64p)
    raise TypeError(a.dtype)


def is_prime(n: int) -> bool:
    return bool(lib().or_is_prime(n))


def ntt_primes(N: int, count: int) -> list[int]:
    out = np.zeros(count, dtype=np.uint64)
    if lib().or_ntt_primes(N, count, _p(out)) != 0:
        raise ValueError("not enough primes")
    return [int(x) for x in out]


def psi(q: int, N: int) -> int:
    return int(lib().or_psi(q, N))


def ntt_naive(q: int, a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_ntt_naive(q, a.size, _p(a), _p(out))
    return out


def intt_naive(q: int, a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_intt_naive(q, a.size, _p(a), _p(out))
    return out


def negacyclic(m: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().or_negacyclic(m, a.size, _p(a), _p(b), _p(out))
    return out


def prng_word(seed: int, domain: int, o0: int, o1: int, o2: int, idx: int) -> int:
    return int(lib().or_prng_word(seed, domain, o0, o1, o2, idx))


def cdt(sigma: float = 3.2) -> list[int]:
    T = np.zeros(20, dtype=np.uint64)
    lib().or_cdt(sigma, _p(T))
    return [int(x) for x in T]


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# slot packing (Sec. 3.2's chunks of c values per ciphertext)
# ---------------------------------------------------------------------------
def slots_encode(N: int, t: int, vals) -> np.ndarray:
    """plaintext polynomial [N] (coefficients in [0, t)) whose slots are vals
    (slot s = (row s // (N/2), column s % (N/2)); see or_slots_encode)."""
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.int64) % t, dtype=np.uint64)
    assert v.size == N
    out = np.zeros(N, dtype=np.uint64)
    if lib().or_slots_encode(N, t, _p(v), _p(out)):
        raise ValueError("t has no primitive 2N-th root of unity")
    return out


def slots_decode(N: int, t: int, poly) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(poly, dtype=np.uint64))
    out = np.zeros(N, dtype=np.uint64)
    if lib().or_slots_decode(N, t, _p(p), _p(out)):
        raise ValueError("t has no primitive 2N-th root of unity")
    return out


def rotation_element(N: int, k: int) -> int:
    """Galois element of a left rotation of each slot row by k (negative k:
    right): 3^(k mod N/2) mod 2N."""
    return pow(3, k % (N // 2), 2 * N)


class OracleCtx:
    """Keys and per-ciphertext operations of the oracle (coefficient form)."""

    def __init__(self, N: int, L: int, t: int = 65537, sigma: float = 3.2, seed: int = 0):
        self._h = lib().or_ctx_create(N, L, t, sigma, seed)
        if not self._h:
            raise ValueError("oracle context creation failed")
        n, l, nP, nA = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int())
        q = np.zeros(16, dtype=np.uint64)
        p = np.zeros(17, dtype=np.uint64)
        aux = np.zeros(48, dtype=np.uint64)
        lib().or_ctx_info(self._h, ctypes.byref(n), ctypes.byref(l), ctypes.byref(nP), ctypes.byref(nA),
                          _p(q), _p(p), _p(aux))
        self.N, self.L, self.t, self.seed, self.sigma = N, L, t, seed, sigma
        self.q = [int(x) for x in q[:L]]
        self.p = [int(x) for x in p[:nP.value]]
        self.aux = [int(x) for x in aux[:nA.value]]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_ctx_free(h)
            self._h = None

    @property
    def ct_shape(self):
        return (2, self.L, self.N)

    def secret(self) -> np.ndarray:
        s = np.zeros(self.N, dtype=np.int64)
        lib().or_get_secret(self._h, _p(s))
        return s

    def rlk(self) -> np.ndarray:
        """[L digit][2 (b, a)][L limb][N]"""
        out = np.zeros((self.L, 2, self.L, self.N), dtype=np.uint64)
        lib().or_get_rlk(self._h, _p(out))
        return out

    def cdt(self) -> list[int]:
        T = np.zeros(20, dtype=np.uint64)
        lib().or_get_cdt(self._h, _p(T))
        return [int(x) for x in T]

    def delta(self) -> int:
        w = np.zeros(18, dtype=np.uint64)
        lib().or_get_delta(self._h, _p(w), 18)
        return sum(int(x) << (64 * i) for i, x in enumerate(w))

    def encrypt(self, m: int, matrix_id: int, row: int, col: int) -> np.ndarray:
        ct = np.zeros(self.ct_shape, dtype=np.uint64)
        if lib().or_encrypt(self._h, int(m), matrix_id, row, col, _p(ct)) != 0:
            raise RuntimeError("sampling failed")
        return ct

    def decrypt(self, ct: np.ndarray) -> tuple[int, int]:
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        m = ctypes.c_int64()
        nb = ctypes.c_int()
        lib().or_decrypt(self._h, _p(ct), ctypes.byref(m), ctypes.byref(nb))
        return int(m.value), int(nb.value)

    def encrypt_poly(self, m, matrix_id: int, row: int, col: int) -> np.ndarray:
        """encryption of a plaintext polynomial m [N] (coefficients mod t)"""
        mm = np.ascontiguousarray(np.asarray(m, dtype=np.int64) % self.t, dtype=np.uint64)
        ct = np.zeros(self.ct_shape, dtype=np.uint64)
        if lib().or_encrypt_poly(self._h, _p(mm), matrix_id, row, col, _p(ct)) != 0:
            raise RuntimeError("sampling failed")
        return ct

    def decrypt_poly(self, ct: np.ndarray) -> tuple[np.ndarray, int]:
        """(message polynomial [N] in [0, t), noise bits)"""
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        m = np.zeros(self.N, dtype=np.uint64)
        nb = ctypes.c_int()
        lib().or_decrypt_poly(self._h, _p(ct), _p(m), ctypes.byref(nb))
        return m, int(nb.value)

    def galois_key(self, g: int) -> np.ndarray:
        """[L digit][2 (b, a)][L limb][N], coefficient form"""
        out = np.zeros((self.L, 2, self.L, self.N), dtype=np.uint64)
        if lib().or_galois_key(self._h, g, _p(out)) != 0:
            raise ValueError("g must be odd; or sampling failed")
        return out

    def rotate(self, ct: np.ndarray, g: int, key: np.ndarray) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        key = np.ascontiguousarray(key, dtype=np.uint64)
        out = np.zeros(self.ct_shape, dtype=np.uint64)
        lib().or_rotate(self._h, _p(ct), g, _p(key), _p(out))
        return out

    def mul_plain(self, ct: np.ndarray, pt) -> np.ndarray:
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        pt = np.ascontiguousarray(np.asarray(pt, dtype=np.uint64))
        out = np.zeros(self.ct_shape, dtype=np.uint64)
        lib().or_mul_plain(self._h, _p(ct), _p(pt), _p(out))
        return out

    def tensor_scale(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        """(d0, d1, d2) after the exact scale-and-round, [3][L][N]."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        d = np.zeros((3, self.L, self.N), dtype=np.uint64)
        lib().or_tensor_scale(self._h, _p(a), _p(b), _p(d))
        return d

    def tensor_scale_sum(self, a_list, b_list) -> np.ndarray:
        """(d0, d1, d2) = round(t (sum of the exact tensors of the pairs) / Q):
        one rounding for the whole sum (at most 1024 pairs)."""
        a_list = [np.ascontiguousarray(a, dtype=np.uint64) for a in a_list]
        b_list = [np.ascontiguousarray(b, dtype=np.uint64) for b in b_list]
        a_arr = (_u64p * len(a_list))(*[_p(a) for a in a_list])
        b_arr = (_u64p * len(b_list))(*[_p(b) for b in b_list])
        d = np.zeros((3, self.L, self.N), dtype=np.uint64)
        if lib().or_tensor_scale_sum(self._h, len(a_list), a_arr, b_arr, _p(d)):
            raise ValueError("between 1 and 1024 pairs")
        return d

    def relin(self, d: np.ndarray) -> np.ndarray:
        d = np.ascontiguousarray(d, dtype=np.uint64)
        out = np.zeros(self.ct_shape, dtype=np.uint64)
        lib().or_relin(self._h, _p(d), _p(out))
        return out

    def mul_relin(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.zeros(self.ct_shape, dtype=np.uint64)
        lib().or_mul_relin(self._h, _p(a), _p(b), _p(out))
        return out

    def add_(self, acc: np.ndarray, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.uint64)
        lib().or_add(self._h, _p(acc), _p(x))
        return acc

    def matmul_entries(self, entries, a_list, b_list, nthreads: int = 0, group: int = 1) -> np.ndarray:
        """Paper's multithreaded scheme (Sec. 3.4): entries = [(row, col, first, count)],
        products first..first+count-1 of the flat lists a_list / b_list; with
        group > 1 each run of `group` consecutive products is rounded once
        (grouped accumulate-then-round)."""
        ent = np.ascontiguousarray(np.asarray(entries, dtype=np.int32).reshape(-1, 4))
        a_arr = (_u64p * len(a_list))(*[_p(a) for a in a_list])
        b_arr = (_u64p * len(b_list))(*[_p(b) for b in b_list])
        out = np.zeros((ent.shape[0],) + self.ct_shape, dtype=np.uint64)
        if lib().or_matmul_entries_grouped(self._h, ent.shape[0], ent.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           a_arr, b_arr, _p(out), nthreads, group):
            raise ValueError("group between 1 and 1024")
        return out


# ---------------------------------------------------------------------------
# sparse encodings (Sec. 3.3.2) and the product sets they list
# ---------------------------------------------------------------------------
DENSE, MASK, CSR, ELL = 0, 1, 2, 3
ENCODINGS = {"dense": DENSE, "mask": MASK, "csr": CSR, "ell": ELL}


@dataclass
class Encoded:
    """Plaintext structure of an encoded left operand and the (row, col)
    coordinates of the element each stored ciphertext encrypts."""
    encoding: int
    rows: int
    cols: int
    values: list          # plaintext value of every stored ciphertext
    coords: list          # (row, col) stream coordinates of every stored ciphertext
    mask: np.ndarray | None = None       # naive sparse: 1 where A == 0
    row_ptr: np.ndarray | None = None    # CSR
    col_idx: np.ndarray | None = None    # CSR
    ell_col: np.ndarray | None = None    # ELLPACK, -1 marks padding
    width: int = 0                       # ELLPACK slots per row


def encode(A: np.ndarray, encoding: int) -> Encoded:
    A = np.asarray(A, dtype=np.int64)
    M, K = A.shape
    if encoding in (DENSE, MASK):
        coords = [(i, k) for i in range(M) for k in range(K)]
        vals = [int(A[i, k]) for i, k in coords]
        mask = (A == 0).astype(np.uint8) if encoding == MASK else None
        return Encoded(encoding, M, K, vals, coords, mask=mask)
    if encoding == CSR:
        row_ptr = [0]
        col_idx, vals, coords = [], [], []
        for i in range(M):
            for k in range(K):
                if A[i, k] != 0:
                    col_idx.append(k)
                    vals.append(int(A[i, k]))
                    coords.append((i, k))
            row_ptr.append(len(col_idx))
        return Encoded(encoding, M, K, vals, coords, row_ptr=np.array(row_ptr, dtype=np.int32),
                       col_idx=np.array(col_idx, dtype=np.int32))
    if encoding == ELL:
        width = max([int(np.count_nonzero(A[i])) for i in range(M)] + [0])
        ell_col = -np.ones((M, width), dtype=np.int32)
        vals, coords = [], []
        for i in range(M):
            nz = [k for k in range(K) if A[i, k] != 0]
            for s in range(width):
                if s < len(nz):
                    ell_col[i, s] = nz[s]
                    vals.append(int(A[i, nz[s]]))
                    coords.append((i, nz[s]))
                else:  # encrypted zero padding; its stream column is K + slot
                    vals.append(0)
                    coords.append((i, K + s))
        return Encoded(encoding, M, K, vals, coords, ell_col=ell_col, width=width)
    raise ValueError(encoding)


def product_set(enc: Encoded, i: int) -> list[tuple[int, int]]:
    """(stored ciphertext index, k) pairs Alg. 1's k-loop visits for row i."""
    if enc.encoding == DENSE:
        return [(i * enc.cols + k, k) for k in range(enc.cols)]
    if enc.encoding == MASK:
        return [(i * enc.cols + k, k) for k in range(enc.cols) if not enc.mask[i, k]]
    if enc.encoding == CSR:
        return [(t, int(enc.col_idx[t])) for t in range(enc.row_ptr[i], enc.row_ptr[i + 1])]
    if enc.encoding == ELL:
        return [(i * enc.width + s, int(enc.ell_col[i, s])) for s in range(enc.width) if enc.ell_col[i, s] >= 0]
    raise ValueError(enc.encoding)


def entry_products(enc: Encoded, i: int, j: int, b_mask: np.ndarray | None = None) -> list[tuple[int, int]]:
    """(stored ciphertext index, k) pairs entry (i, j) multiplies: row i's
    pairs as A's encoding lists them; with a right-operand mask
    (b_mask[k, j] = 1 where B[k][j] == 0), those whose B element is zero are
    skipped too.  The dense loop of Alg. 1 skips nothing."""
    ps = product_set(enc, i)
    if b_mask is None or enc.encoding == DENSE:
        return ps
    return [(t, k) for t, k in ps if not b_mask[k, j]]


class OracleMatmul:
    """Encrypts plaintext operands and evaluates entries of C = A x B.

    Ciphertexts are encrypted once per stream coordinate and reused, and each
    product Relin(A[i][k] x B[k][j]) is computed once and shared by every
    encoding that lists it (the encryption of an element depends only on its
    coordinates, so all encodings multiply the same ciphertexts)."""

    def __init__(self, ctx: OracleCtx, A: np.ndarray, B: np.ndarray, a_id: int, b_id: int):
        self.ctx, self.A, self.B, self.a_id, self.b_id = ctx, np.asarray(A), np.asarray(B), a_id, b_id
        self._ct = {}
        self._prod = {}

    def ct_a(self, row: int, col: int) -> np.ndarray:
        key = ("a", row, col)
        if key not in self._ct:
            v = int(self.A[row, col]) if col < self.A.shape[1] else 0
            self._ct[key] = self.ctx.encrypt(v, self.a_id, row, col)
        return self._ct[key]

    def ct_b(self, row: int, col: int) -> np.ndarray:
        key = ("b", row, col)
        if key not in self._ct:
            self._ct[key] = self.ctx.encrypt(int(self.B[row, col]), self.b_id, row, col)
        return self._ct[key]

    def product(self, i: int, k: int, j: int) -> np.ndarray:
        key = (i, k, j)
        if key not in self._prod:
            self._prod[key] = self.ctx.mul_relin(self.ct_a(i, k), self.ct_b(k, j))
        return self._prod[key]

    def entry(self, enc: Encoded, i: int, j: int, group: int = 1, b_mask: np.ndarray | None = None) -> np.ndarray:
        """C[i][j]: the trivial zero ciphertext plus every listed product (in
        ascending k; with b_mask, only k where B[k][j] is nonzero too); with
        group > 1, each run of `group` consecutive products is scaled and
        rounded once and relinearised once."""
        acc = np.zeros(self.ctx.ct_shape, dtype=np.uint64)
        ks = [k for _, k in entry_products(enc, i, j, b_mask)]
        if group == 1:
            for k in ks:
                self.ctx.add_(acc, self.product(i, k, j))
            return acc
        for p in range(0, len(ks), group):
            run = ks[p:p + group]
            d = self.ctx.tensor_scale_sum([self.ct_a(i, k) for k in run], [self.ct_b(k, j) for k in run])
            self.ctx.add_(acc, self.ctx.relin(d))
        return acc


class OracleChunked:
    """The encrypted matrix product over slot-packed chunks (Sec. 3.2).

    Storage: element e of a matrix's row-major order sits in slot e mod c of
    chunk ciphertext e // c (chunk q encrypted under the stream object
    (matrix id, q, 0)); the other slots hold 0.

    The result is defined per output entry (i, j).  Its product set P(i, j)
    is every k, or with skip_zeros the k where A[i][k] and B[k][j] are both
    nonzero (the naive sparse scheme's two masks, Sec. 3.3.2).  The operand
    of product k on the left is the chunk holding element e = i K + k turned
    left by e mod c, which brings A[i][k] into slot 0 (a Galois rotation; a
    turn by 0 is no operation), and likewise on the right with
    e = k Nc + j.  Their BFV product, relinearised (the exact scale-and-round
    of the BFV multiply stands where CKKS rescales), is the product's term.
    The entry's slot-0 value reaches its place, slot r mod c of chunk r // c
    with r = i Nc + j, by a plaintext product with the one-hot slot-0 mask
    and a turn right by r mod c; that placement is applied either to every
    term before the terms are added into the result chunk (placement
    "product", where Alg. 1 applies it) or once to the sum of the entry's
    terms (placement "entry": a different ciphertext with the same
    decryption, equal to the first wherever r mod c = 0 and the entry has at
    most one term).  Additions are exact and order-free."""

    def __init__(self, ctx: OracleCtx, A: np.ndarray, B: np.ndarray, c: int, a_id: int, b_id: int):
        self.ctx, self.A, self.B, self.c = ctx, np.asarray(A), np.asarray(B), c
        assert 1 <= c <= ctx.N // 2
        self.a_ct = self._chunks(self.A, a_id)
        self.b_ct = self._chunks(self.B, b_id)
        self._keys = {}
        onehot = np.zeros(ctx.N, dtype=np.int64)
        onehot[0] = 1
        self.mask = slots_encode(ctx.N, ctx.t, onehot)

    def _chunks(self, M: np.ndarray, mid: int) -> list:
        flat = M.reshape(-1)
        out = []
        for q in range(-(-flat.size // self.c)):
            v = np.zeros(self.ctx.N, dtype=np.int64)
            part = flat[q * self.c:(q + 1) * self.c]
            v[:part.size] = part
            out.append(self.ctx.encrypt_poly(slots_encode(self.ctx.N, self.ctx.t, v), mid, q, 0))
        return out

    def key(self, g: int) -> np.ndarray:
        if g not in self._keys:
            self._keys[g] = self.ctx.galois_key(g)
        return self._keys[g]

    def rot(self, ct: np.ndarray, k: int) -> np.ndarray:
        """ct turned left by k slots in each row (right for k < 0)"""
        if k % (self.ctx.N // 2) == 0:
            return ct
        g = rotation_element(self.ctx.N, k)
        return self.ctx.rotate(ct, g, self.key(g))

    def product_sets(self, skip_zeros: bool = False) -> dict:
        """{(i, j): [k, ...]} for every output entry"""
        M, Kd = self.A.shape
        Nc = self.B.shape[1]
        return {(i, j): [k for k in range(Kd) if not (skip_zeros and (self.A[i, k] == 0 or self.B[k, j] == 0))]
                for i in range(M) for j in range(Nc)}

    def slot0(self, chunks: list, e: int) -> np.ndarray:
        """element e of a chunked matrix brought into slot 0"""
        return self.rot(chunks[e // self.c], e % self.c)

    def term(self, i: int, k: int, j: int) -> np.ndarray:
        Kd, Nc = self.A.shape[1], self.B.shape[1]
        return self.ctx.mul_relin(self.slot0(self.a_ct, i * Kd + k), self.slot0(self.b_ct, k * Nc + j))

    def place(self, ct: np.ndarray, r: int) -> np.ndarray:
        """slot 0 of ct moved to slot r mod c, every other slot cleared"""
        return self.rot(self.ctx.mul_plain(ct, self.mask), -(r % self.c))

    def result(self, skip_zeros: bool = False, placement: str = "product") -> list:
        """the result chunks (list of ciphertexts, coefficient form)"""
        assert placement in ("product", "entry")
        M, Nc = self.A.shape[0], self.B.shape[1]
        R = [np.zeros(self.ctx.ct_shape, dtype=np.uint64) for _ in range(-(-(M * Nc) // self.c))]
        for (i, j), ks in self.product_sets(skip_zeros).items():
            r = i * Nc + j
            if placement == "product":
                for k in ks:
                    self.ctx.add_(R[r // self.c], self.place(self.term(i, k, j), r))
            else:
                e = np.zeros(self.ctx.ct_shape, dtype=np.uint64)
                for k in ks:
                    self.ctx.add_(e, self.term(i, k, j))
                self.ctx.add_(R[r // self.c], self.place(e, r))
        return R

    def decode(self, R: list) -> np.ndarray:
        """the result matrix from its chunks (centred mod t)"""
        M, Nc = self.A.shape[0], self.B.shape[1]
        vals = []
        for ct in R:
            m, _ = self.ctx.decrypt_poly(ct)
            vals.extend(int(x) for x in slots_decode(self.ctx.N, self.ctx.t, m)[:self.c])
        flat = np.array(vals[:M * Nc], dtype=np.int64)
        t = self.ctx.t
        return (((flat + t // 2) % t) - t // 2).reshape(M, Nc)
