"""CKKS over RNS with a special key-switching prime: the scheme and the
parameter set the paper runs (Sec. 3.1: ring degree 8192, a coefficient
modulus of 50, 40, 40, 40 and 40 bits, the last one the key-switching prime,
initial scale 2^40), and the chunked matrix product of Alg. 1 over it.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py may import this module.  It shares
no code with the CUDA path (paper_2503_09184_gb300) and never imports it;
its polynomial products are the C oracle's schoolbook negacyclic products.

Everything is in coefficient form with canonical residues:
  * primes (all 1 mod 2N): q_0 the largest below 2^50, q_1 .. q_3 the three
    largest below 2^40, the key-switching prime P the next one below 2^40
    (other bit sizes can be given for small test rings);
  * slots: slot j < N/2 of a real-coefficient polynomial m is m(zeta^(3^j)),
    zeta = exp(i pi / N) (slot N/2 + j, at the conjugate root, is its
    conjugate).  Encoding real values z at a scale D:
    m_k = round((2 D / N) sum_j z_j cos(pi 3^j k / N)); decoding:
    z_j = (1 / D) sum_k m_k cos(pi 3^j k / N);
  * secret: the ternary polynomial of the generator stream (seed, 1, 0, 0, 0)
    (the same draws as the BFV secret of oracle.py); errors: the rounded
    Gaussian of width 3.2 cut at 19 (the CDT of oracle.cdt);
  * encryption of an integer polynomial m: c = (-a s + e + m, a) mod every
    q_i, a uniform per prime from stream (seed, 11, id, row, col), slot
    i N + k; e from stream (seed, 12, id, row, col), slot k;
  * key switching of a polynomial d at level l (primes q_0 .. q_l) with a
    key for w: digits D_j = [d]_{q_j} in [0, q_j), j <= l;
    u = sum_j D_j k_j over q_0 .. q_l and P; the result round(u / P), limb by
    limb (u_i - [u_P]_centred) P^-1 mod q_i.  Key digit j:
    k_j = (-a_j s + e_j + P g_j w, a_j) with g_j = 1 mod q_j and 0 mod the
    other q_i (the CRT gadget of q_0 .. q_3), so P g_j w is P w in limb j and
    0 in every other limb and in P; a_j uniform from stream (seed, 9, g, j, 0)
    with slot t N + k for the t-th prime of q_0 .. q_3, P; e_j from stream
    (seed, 10, g, j, 0); g = 0 for w = s^2 (relinearisation), the Galois
    element for w = s(X^g);
  * multiply at level l: (a0 b0, a0 b1 + a1 b0) plus the key switch of
    a1 b1 with the relinearisation key;
  * rescale from level l: round(c / q_l) limb by limb,
    (c_i - [c_l]_centred) q_l^-1 mod q_i, i < l; the scale is divided by q_l;
  * rotation left by k: c(X^g), g = 3^k mod 2N, then c1(X^g) key-switched
    with the key for s(X^g);
  * decryption at level l: [c0 + c1 s]_{q_0 ... q_l}, centred, decoded at
    the ciphertext's scale.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import oracle as O

DOM_SECRET, DOM_KSK_A, DOM_KSK_E, DOM_ENC_A, DOM_ENC_E = 1, 9, 10, 11, 12
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _lib():
    L = O.lib()
    if not getattr(L, "_ckks_ready", False):
        L.or_ntt_primes_bits.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p]
        L.or_ntt_primes_bits.restype = ctypes.c_int
        L.or_sample_poly.argtypes = [ctypes.c_uint64] * 5 + [ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                                            ctypes.c_int, _u64p, _u64p]
        L.or_sample_poly.restype = ctypes.c_int
        L.or_mul_scalar.argtypes = [ctypes.c_uint64, ctypes.c_int, _u64p, ctypes.c_uint64, _u64p]
        L._ckks_ready = True
    return L


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


def primes_bits(N: int, bits: int, skip: int, count: int) -> list[int]:
    out = np.zeros(count, dtype=np.uint64)
    if _lib().or_ntt_primes_bits(N, bits, skip, count, _p(out)):
        raise ValueError("not enough primes")
    return [int(x) for x in out]


def slot_exponents(N: int) -> np.ndarray:
    """3^j mod 2N for the slots j < N/2"""
    e = np.zeros(N // 2, dtype=np.int64)
    x = 1
    for j in range(N // 2):
        e[j] = x
        x = x * 3 % (2 * N)
    return e


def encode(N: int, z, scale: float) -> np.ndarray:
    """the integer polynomial of real slot values z (fewer than N/2 values:
    the rest are 0), float64, the sum over j in ascending order"""
    zz = np.zeros(N // 2, dtype=np.float64)
    zv = np.asarray(z, dtype=np.float64)
    zz[:zv.size] = zv
    e = slot_exponents(N)
    cos_tab = np.cos(np.pi * np.arange(2 * N, dtype=np.float64) / N)
    m = np.zeros(N, dtype=np.int64)
    nz = np.nonzero(zz)[0]
    for k in range(N):
        acc = float(np.sum(zz[nz] * cos_tab[(e[nz] * k) % (2 * N)]))
        m[k] = int(round(2.0 * scale / N * acc))
    return m


def decode(N: int, m, scale: float) -> np.ndarray:
    """real slot values of an integer polynomial (m as Python ints or floats)"""
    e = slot_exponents(N)
    mf = np.array([float(x) for x in m], dtype=np.float64)
    cos_tab = np.cos(np.pi * np.arange(2 * N, dtype=np.float64) / N)
    k = np.arange(N, dtype=np.int64)
    return np.array([float(np.sum(mf * cos_tab[(e[j] * k) % (2 * N)])) for j in range(N // 2)]) / scale


def automorphism(m: np.ndarray, g: int, q: int) -> np.ndarray:
    """m(X^g) mod X^N + 1 for residues mod q (g odd)"""
    N = m.size
    out = np.zeros(N, dtype=np.uint64)
    for k in range(N):
        d = (g * k) % (2 * N)
        v = int(m[k])
        if d >= N:
            out[d - N] = (q - v) % q
        else:
            out[d] = v
    return out


class OracleCkks:
    """Keys and the operations of the scheme; ciphertexts are uint64 arrays
    [2][L][N] (limbs above the level are zero), coefficient form."""

    def __init__(self, N: int = 8192, bits=(50, 40, 40, 40), special_bits: int = 40, log_scale: int = 40,
                 seed: int = 0, sigma: float = 3.2):
        self.N, self.seed = N, seed
        self.L = len(bits)
        used: dict[int, int] = {}
        self.q = []
        for b in bits:
            self.q.append(primes_bits(N, b, used.get(b, 0), 1)[0])
            used[b] = used.get(b, 0) + 1
        self.P = primes_bits(N, special_bits, used.get(special_bits, 0), 1)[0]
        self.scale = float(2 ** log_scale)
        self.cdt = np.array(O.cdt(sigma), dtype=np.uint64)
        self.s = self._sample(DOM_SECRET, 0, 0, 0, 1, self.q[0], 0).astype(np.int64)
        self.s = np.where(self.s == self.q[0] - 1, -1, self.s)
        self._keys = {}

    # ---------------------------------------------------------- helpers ---
    def _sample(self, dom, o0, o1, o2, kind, q, limb) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint64)
        if _lib().or_sample_poly(self.seed, dom, o0, o1, o2, kind, q, limb, self.N, _p(self.cdt), _p(out)):
            raise RuntimeError("sampler ran out of words")
        return out

    def all_primes(self) -> list[int]:
        return self.q + [self.P]

    def mul(self, a: np.ndarray, b: np.ndarray, p: int) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint64)
        O.lib().or_negacyclic(p, self.N, _p(np.ascontiguousarray(a)), _p(np.ascontiguousarray(b)), _p(out))
        return out

    def scal(self, a: np.ndarray, c: int, p: int) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint64)
        _lib().or_mul_scalar(p, self.N, _p(np.ascontiguousarray(a)), c % p, _p(out))
        return out

    @staticmethod
    def add(a, b, p):
        return (a + b) % np.uint64(p) if p < 2 ** 63 else np.array([(int(x) + int(y)) % p for x, y in zip(a, b)],
                                                                   dtype=np.uint64)

    @staticmethod
    def sub(a, b, p):
        return np.where(a >= b, a - b, a + (np.uint64(p) - b)).astype(np.uint64)

    @staticmethod
    def residues(v: np.ndarray, p: int) -> np.ndarray:
        """signed integers to residues mod p"""
        return np.array([int(x) % p for x in v], dtype=np.uint64)

    @staticmethod
    def centred(a: np.ndarray, p: int) -> list[int]:
        return [int(x) - p if int(x) > p // 2 else int(x) for x in a]

    def zero_ct(self) -> np.ndarray:
        return np.zeros((2, self.L, self.N), dtype=np.uint64)

    # ------------------------------------------------------- encryption ---
    def secret_mod(self, p: int) -> np.ndarray:
        return self.residues(self.s, p)

    def encrypt(self, m, matrix_id: int, row: int, col: int) -> np.ndarray:
        """m: integer polynomial (N signed coefficients), at the top level"""
        ct = self.zero_ct()
        e = self._sample(DOM_ENC_E, matrix_id, row, col, 2, self.q[0], 0).astype(np.int64)
        e = np.where(e > self.q[0] // 2, e - np.int64(self.q[0]), e)
        me = [int(x) + int(y) for x, y in zip(m, e)]
        for i, q in enumerate(self.q):
            a = self._sample(DOM_ENC_A, matrix_id, row, col, 0, q, i)
            ct[1, i] = a
            ct[0, i] = self.sub(self.residues(np.array(me, dtype=object), q), self.mul(a, self.secret_mod(q), q), q)
        return ct

    def decrypt_poly(self, ct: np.ndarray, level: int) -> list[int]:
        """[c0 + c1 s]_{q_0 .. q_level}, centred, by CRT with Python integers"""
        Q = math.prod(self.q[:level + 1])
        acc = [0] * self.N
        for i in range(level + 1):
            q = self.q[i]
            v = self.add(ct[0, i], self.mul(ct[1, i], self.secret_mod(q), q), q)
            Qi = Q // q
            w = Qi * pow(Qi % q, -1, q)
            acc = [(x + int(y) * w) % Q for x, y in zip(acc, v)]
        return [x - Q if x > Q // 2 else x for x in acc]

    def decrypt(self, ct: np.ndarray, level: int, scale: float) -> np.ndarray:
        return decode(self.N, self.decrypt_poly(ct, level), scale)

    # ---------------------------------------------------- key switching ---
    def key(self, g: int) -> np.ndarray:
        """key digits [L][2][L + 1][N] for s^2 (g = 0) or s(X^g)"""
        if g in self._keys:
            return self._keys[g]
        if g == 0:
            w = [self.mul(self.secret_mod(p), self.secret_mod(p), p) for p in self.all_primes()]
        else:
            w = [automorphism(self.secret_mod(p), g, p) for p in self.all_primes()]
        K = np.zeros((self.L, 2, self.L + 1, self.N), dtype=np.uint64)
        for j in range(self.L):
            e = self._sample(DOM_KSK_E, g, j, 0, 2, self.q[0], 0).astype(np.int64)
            e = np.where(e > self.q[0] // 2, e - np.int64(self.q[0]), e)
            for t, p in enumerate(self.all_primes()):
                a = self._sample(DOM_KSK_A, g, j, 0, 0, p, t)
                b = self.sub(self.residues(e, p), self.mul(a, self.secret_mod(p), p), p)
                if t == j:
                    b = self.add(b, self.scal(w[t], self.P, p), p)
                K[j, 0, t], K[j, 1, t] = b, a
        self._keys[g] = K
        return K

    def keyswitch(self, d: np.ndarray, level: int, K: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """d: [L][N] residues of one polynomial (limbs 0 .. level); returns
        the two result polynomials [L][N] at the same level"""
        primes = self.q[:level + 1] + [self.P]
        tidx = list(range(level + 1)) + [self.L]
        u = np.zeros((2, level + 2, self.N), dtype=np.uint64)
        for j in range(level + 1):
            for n, (t, p) in enumerate(zip(tidx, primes)):
                Dj = (d[j] % np.uint64(p)) if p < self.q[j] else d[j]
                for c in range(2):
                    u[c, n] = self.add(u[c, n], self.mul(Dj, K[j, c, t], p), p)
        out = np.zeros((2, self.L, self.N), dtype=np.uint64)
        for c in range(2):
            uP = self.centred(u[c, level + 1], self.P)
            for i in range(level + 1):
                q = self.q[i]
                diff = self.sub(u[c, i], self.residues(np.array(uP, dtype=object), q), q)
                out[c, i] = self.scal(diff, pow(self.P, -1, q), q)
        return out[0], out[1]

    # -------------------------------------------------------- operations ---
    def mul_relin(self, a: np.ndarray, b: np.ndarray, level: int) -> np.ndarray:
        out = self.zero_ct()
        d2 = np.zeros((self.L, self.N), dtype=np.uint64)
        for i in range(level + 1):
            q = self.q[i]
            out[0, i] = self.mul(a[0, i], b[0, i], q)
            out[1, i] = self.add(self.mul(a[0, i], b[1, i], q), self.mul(a[1, i], b[0, i], q), q)
            d2[i] = self.mul(a[1, i], b[1, i], q)
        v0, v1 = self.keyswitch(d2, level, self.key(0))
        for i in range(level + 1):
            q = self.q[i]
            out[0, i] = self.add(out[0, i], v0[i], q)
            out[1, i] = self.add(out[1, i], v1[i], q)
        return out

    def rescale(self, ct: np.ndarray, level: int) -> np.ndarray:
        ql = self.q[level]
        out = self.zero_ct()
        for c in range(2):
            cl = self.centred(ct[c, level], ql)
            for i in range(level):
                q = self.q[i]
                diff = self.sub(ct[c, i], self.residues(np.array(cl, dtype=object), q), q)
                out[c, i] = self.scal(diff, pow(ql, -1, q), q)
        return out

    def rotate(self, ct: np.ndarray, level: int, k: int) -> np.ndarray:
        """slots turned left by k (right for k < 0); k = 0 is the identity"""
        if k % (self.N // 2) == 0:
            return ct
        g = O.rotation_element(self.N, k)
        c0 = np.zeros((self.L, self.N), dtype=np.uint64)
        c1 = np.zeros((self.L, self.N), dtype=np.uint64)
        for i in range(level + 1):
            c0[i] = automorphism(ct[0, i], g, self.q[i])
            c1[i] = automorphism(ct[1, i], g, self.q[i])
        v0, v1 = self.keyswitch(c1, level, self.key(g))
        out = self.zero_ct()
        for i in range(level + 1):
            out[0, i] = self.add(c0[i], v0[i], self.q[i])
            out[1, i] = v1[i]
        return out

    def mul_plain(self, ct: np.ndarray, level: int, m) -> np.ndarray:
        out = self.zero_ct()
        for i in range(level + 1):
            q = self.q[i]
            mm = self.residues(np.array([int(x) for x in m], dtype=object), q)
            for c in range(2):
                out[c, i] = self.mul(ct[c, i], mm, q)
        return out

    def add_ct(self, acc: np.ndarray, x: np.ndarray, level: int) -> np.ndarray:
        for i in range(level + 1):
            for c in range(2):
                acc[c, i] = self.add(acc[c, i], x[c, i], self.q[i])
        return acc


class OracleCkksChunked:
    """The chunked matrix product of Alg. 1 under CKKS, every term placed on
    its own (the placement Alg. 1 uses).  Chunk q of a matrix holds its
    row-major elements q c .. q c + c - 1 in slots 0 .. c-1, encoded at the
    scale D = 2^40 and encrypted at the top level (stream object (id, q, 0)).
    The term of product k of entry (i, j): the two chunks turned so that
    A[i][k] and B[k][j] sit in slot 0, multiplied and relinearised at the top
    level, rescaled by q_3; then the plaintext one-hot slot-0 mask, encoded
    at the scale q_2, multiplies it and a rescale by q_2 returns the scale to
    D^2 / q_3; the term is turned right by (i Nc + j) mod c and added into
    chunk (i Nc + j) // c of the result, at level 1.  Alg. 1 also
    relinearises after the mask product, which has nothing to relinearise
    with a plaintext.  With skip_zeros, products where A[i][k] or B[k][j] is
    zero are left out."""

    def __init__(self, ck: OracleCkks, A: np.ndarray, B: np.ndarray, c: int, a_id: int, b_id: int):
        assert ck.L == 4, "the term's two rescales take the chunks from level 3 to level 1"
        self.ck, self.A, self.B, self.c = ck, np.asarray(A), np.asarray(B), c
        self.top = ck.L - 1
        self.a_ct = self._chunks(self.A, a_id)
        self.b_ct = self._chunks(self.B, b_id)
        onehot = np.zeros(1)
        onehot[0] = 1.0
        self.mask = encode(ck.N, onehot, float(ck.q[self.top - 1]))
        self.result_scale = ck.scale * ck.scale / ck.q[self.top]

    def _chunks(self, M: np.ndarray, mid: int) -> list:
        flat = M.reshape(-1).astype(np.float64)
        return [self.ck.encrypt(encode(self.ck.N, flat[q * self.c:(q + 1) * self.c], self.ck.scale), mid, q, 0)
                for q in range(-(-flat.size // self.c))]

    def product_sets(self, skip_zeros: bool = False) -> dict:
        M, Kd = self.A.shape
        Nc = self.B.shape[1]
        return {(i, j): [k for k in range(Kd) if not (skip_zeros and (self.A[i, k] == 0 or self.B[k, j] == 0))]
                for i in range(M) for j in range(Nc)}

    def term(self, i: int, k: int, j: int) -> np.ndarray:
        ck, c, top = self.ck, self.c, self.top
        Kd, Nc = self.A.shape[1], self.B.shape[1]
        ea, eb = i * Kd + k, k * Nc + j
        a = ck.rotate(self.a_ct[ea // c], top, ea % c)
        b = ck.rotate(self.b_ct[eb // c], top, eb % c)
        return ck.rescale(ck.mul_relin(a, b, top), top)

    def place(self, x: np.ndarray, r: int) -> np.ndarray:
        ck, lv = self.ck, self.top - 1
        y = ck.rescale(ck.mul_plain(x, lv, self.mask), lv)
        return ck.rotate(y, lv - 1, -(r % self.c))

    def result(self, skip_zeros: bool = False) -> list:
        M, Nc = self.A.shape[0], self.B.shape[1]
        R = [self.ck.zero_ct() for _ in range(-(-(M * Nc) // self.c))]
        for (i, j), ks in self.product_sets(skip_zeros).items():
            r = i * Nc + j
            for k in ks:
                self.ck.add_ct(R[r // self.c], self.place(self.term(i, k, j), r), self.top - 2)
        return R

    def decode(self, R: list) -> np.ndarray:
        M, Nc = self.A.shape[0], self.B.shape[1]
        vals = []
        for ct in R:
            vals.extend(self.ck.decrypt(ct, self.top - 2, self.result_scale)[:self.c])
        return np.array(vals[:M * Nc]).reshape(M, Nc)
