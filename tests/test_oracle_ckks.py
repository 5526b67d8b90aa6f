"""Pins of the CKKS oracle (oracle/ckks.py) against what the mathematics
fixes: the prime lists by an independent scan; the slot encoding by
evaluating the polynomial at the complex roots directly; encryption,
key switching and rescaling by big-integer arithmetic over the whole
modulus; multiplication and rotation by their effect on the decoded slots;
the chunked product of Alg. 1 by the matrix product.  Small rings (N = 64)
carry the paper's prime sizes (50, 40, 40, 40 and a 40-bit key-switching
prime, scale 2^40) so that every step runs in seconds."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import ckks as CK
from oracle import oracle as O

N = 64


@pytest.fixture(scope="module")
def ck():
    return CK.OracleCkks(N=N, seed=21)


def _crt(limbs, primes):
    Q = math.prod(primes)
    acc = 0
    for v, q in zip(limbs, primes):
        Qi = Q // q
        acc = (acc + int(v) * Qi * pow(Qi % q, -1, q)) % Q
    return acc - Q if acc > Q // 2 else acc


def test_primes_by_an_independent_scan():
    sympy = pytest.importorskip("sympy")
    def scan(n, bits, count):
        out, k = [], (2 ** bits - 2) // (2 * n)
        while len(out) < count:
            if sympy.isprime(k * 2 * n + 1):
                out.append(k * 2 * n + 1)
            k -= 1
        return out

    for n in (64, 8192):
        q = CK.primes_bits(n, 50, 0, 1) + CK.primes_bits(n, 40, 0, 4)
        assert q == scan(n, 50, 1) + scan(n, 40, 4)
        if n == 64:
            ck = CK.OracleCkks(N=n)
            assert ck.q == q[:4] and ck.P == q[4]
    assert len(set(q)) == 5 and all(x % (2 * 8192) == 1 for x in q)


def test_encoding_against_direct_evaluation():
    """m(zeta^(3^j)) evaluated as a complex sum equals scale z_j (real, up
    to the rounding of the coefficients), for random values and for a
    constant, whose polynomial is the constant round(scale c)."""
    rng = np.random.default_rng(1)
    z = rng.uniform(-16, 16, size=N // 2)
    scale = 2.0 ** 30
    m = CK.encode(N, z, scale)
    zeta = np.exp(1j * np.pi / N)
    e = CK.slot_exponents(N)
    vals = np.array([np.sum(m * zeta ** ((e[j] * np.arange(N)) % (2 * N))) for j in range(N // 2)])
    assert np.max(np.abs(vals.real / scale - z)) < 1e-6
    assert np.max(np.abs(vals.imag / scale)) < 1e-6
    assert np.max(np.abs(CK.decode(N, m, scale) - z)) < 1e-6
    c = CK.encode(N, np.full(N // 2, 3.25), scale)
    assert c[0] == round(3.25 * scale) and not c[1:].any()


def test_encrypt_decrypt_error_is_small(ck):
    m = CK.encode(N, np.arange(N // 2) - 10.0, ck.scale)
    ct = ck.encrypt(m, 3, 1, 2)
    got = ck.decrypt_poly(ct, 3)
    assert max(abs(g - int(x)) for g, x in zip(got, m)) <= 19
    # the stream: c1 limb i is the uniform draw of slot i N + k mod q_i
    w = O.prng_word(ck.seed, CK.DOM_ENC_A, 3, 1, 2, (1 * N + 5) * 16)
    if w < (2 ** 64 // ck.q[1]) * ck.q[1]:
        assert int(ct[1, 1, 5]) == w % ck.q[1]


def test_keys_hold_the_gadget_relation(ck):
    """b_j + a_j s - e_j is P w in limb j and 0 in every other limb and in
    P (big integers over q_0 .. q_3 P: one small error, the same in every
    prime)."""
    K = ck.key(0)
    primes = ck.all_primes()
    s2 = [sum(int(ck.s[a]) * int(ck.s[(k - a) % N]) * (1 if a <= k else -1) for a in range(N)) for k in range(N)]
    for j in range(ck.L):
        for k in range(0, N, 7):
            lim = [(int(K[j, 0, t, k]) + sum(int(K[j, 1, t, a]) * int(ck.s[(k - a) % N]) * (1 if a <= k else -1)
                                             for a in range(N))) % p for t, p in enumerate(primes)]
            want_gadget = [((ck.P * s2[k]) % p if t == j else 0) for t, p in enumerate(primes)]
            err = [(x - g) % p for x, g, p in zip(lim, want_gadget, primes)]
            e = _crt(err, primes)
            assert abs(e) <= 19


def test_rescale_is_the_rounded_division(ck):
    m = CK.encode(N, np.linspace(-5, 5, N // 2), ck.scale)
    ct = ck.encrypt(m, 4, 0, 0)
    r = ck.rescale(ct, 3)
    for c in range(2):
        for k in range(0, N, 5):
            C = _crt([ct[c, i, k] for i in range(4)], ck.q)
            want = C // ck.q[3] + (1 if 2 * (C % ck.q[3]) > ck.q[3] else 0)   # nearest, Q odd: no ties
            for i in range(3):
                assert int(r[c, i, k]) == want % ck.q[i]


def test_keyswitch_by_big_integers(ck):
    """The key switch of d gives (v0, v1) with v0 + v1 s = d s^2 + e over
    q_0 .. q_l, e far below the primes (the rounded division by P)."""
    rng = np.random.default_rng(3)
    for level in (3, 1):
        d = np.zeros((4, N), dtype=np.uint64)
        for i in range(level + 1):
            d[i] = rng.integers(0, ck.q[i], size=N, dtype=np.uint64)
        v0, v1 = ck.keyswitch(d, level, ck.key(0))
        primes = ck.q[:level + 1]
        s2 = [sum(int(ck.s[a]) * int(ck.s[(k - a) % N]) * (1 if a <= k else -1) for a in range(N)) for k in range(N)]
        Dk = [_crt([d[i, k] for i in range(level + 1)], primes) for k in range(N)]
        for k in range(0, N, 9):
            lhs = [(int(v0[i, k]) + sum(int(v1[i, a]) * int(ck.s[(k - a) % N]) * (1 if a <= k else -1)
                                        for a in range(N))) % q for i, q in enumerate(primes)]
            rhs = sum(Dk[a] * s2[(k - a) % N] * (1 if a <= k else -1) for a in range(N))
            e = _crt([(x - rhs) % q for x, q in zip(lhs, primes)], primes)
            assert abs(e) < 2 ** 30, (level, k, e)


def test_multiply_and_rotate_act_on_the_slots(ck):
    rng = np.random.default_rng(5)
    z1, z2 = rng.uniform(-4, 4, N // 2), rng.uniform(-4, 4, N // 2)
    a = ck.encrypt(CK.encode(N, z1, ck.scale), 1, 0, 0)
    b = ck.encrypt(CK.encode(N, z2, ck.scale), 2, 0, 0)
    x = ck.rescale(ck.mul_relin(a, b, 3), 3)
    got = ck.decrypt(x, 2, ck.scale * ck.scale / ck.q[3])
    assert np.max(np.abs(got - z1 * z2)) < 1e-4
    for k in (1, 3, -2):
        r = ck.decrypt(ck.rotate(a, 3, k), 3, ck.scale)
        assert np.max(np.abs(r - np.roll(z1, -k))) < 1e-4, k


@pytest.mark.parametrize("chunk", [1, 3])
def test_chunked_product_decodes_to_the_matrix_product(ck, chunk):
    A = np.array([[3, 0, -7], [0, 5, 2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0]], dtype=np.int64)
    oc = CK.OracleCkksChunked(ck, A, B, chunk, 1, 2)
    for skip in (False, True):
        got = oc.decode(oc.result(skip_zeros=skip))
        assert np.max(np.abs(got - A @ B)) < 1e-3, (chunk, skip)
