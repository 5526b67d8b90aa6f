"""Pins of the CPU oracle against facts fixed outside it: number theory,
closed forms, distribution laws, and a textbook big-integer BFV (single
modulus Q, Python integers, no RNS) on tiny rings.

Each group names the oracle function it pins.  A plausible slip -- a dropped
tensor term, a wrong sign in the negacyclic wrap, a transposed operand, an
off-by-one in the rounding, a [0, Q) lift instead of a centred one -- fails at
least one test here.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import textbook as tb
from crafted import boundary_pair
from oracle import oracle as O

T = 65537


# ---------------------------------------------------------------- primes ---
def _trial_division(n: int) -> bool:
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def test_is_prime_small_range_and_pseudoprimes():
    """or_is_prime: trial division below 20000; strong pseudoprimes to the
    smallest bases and Carmichael numbers are composite; known primes."""
    for n in range(20000):
        assert O.is_prime(n) == _trial_division(n), n
    composites = [561, 1105, 1729, 2047, 3215031751, 2152302898747, 3474749660383,
                  341550071728321, 3825123056546413051, (2**32 + 1), 2**54 - 1]
    for n in composites:
        assert not O.is_prime(n), n
    for p in [2**31 - 1, 2**61 - 1, 18446744073709551557]:  # Mersenne primes, largest 64-bit prime
        assert O.is_prime(p), p


@pytest.mark.parametrize("N", [8, 16, 4096, 8192, 16384])
def test_ntt_primes_are_the_largest(N):
    """or_ntt_primes: primes, == 1 mod 2N, below 2^54, descending, and no such
    prime is skipped (every skipped candidate has a small factor or fails a
    Fermat test to base 2 and 3)."""
    ps = O.ntt_primes(N, 5)
    assert all(p < 2**54 and p % (2 * N) == 1 for p in ps)
    assert ps == sorted(ps, reverse=True)
    sympy = pytest.importorskip("sympy")
    for p in ps:
        assert sympy.isprime(p)
    cand = ((2**54 - 2) // (2 * N)) * 2 * N + 1
    found = []
    while len(found) < 5:
        if sympy.isprime(cand):
            found.append(cand)
        cand -= 2 * N
    assert found == ps


@pytest.mark.parametrize("q,N", [(97, 8), (193, 16), (257, 64), (7681, 256), (12289, 512)])
def test_psi_is_smallest_primitive_root(q, N):
    """or_psi: brute-force minimum of {x : x^N == -1 mod q}."""
    brute = min(x for x in range(1, q) if pow(x, N, q) == q - 1)
    assert O.psi(q, N) == brute


# ------------------------------------------------------------------- NTT ---
def _bitrev(x, logn):
    return int(format(x, f"0{logn}b")[::-1], 2)


@pytest.mark.parametrize("N", [8, 16, 32])
def test_ntt_definition_closed_forms(N):
    """or_ntt_naive: NTT(1) = all ones; NTT(X)[i] = psi^(2 bitrev(i) + 1), the
    evaluation points are N distinct roots of X^N + 1."""
    q = O.ntt_primes(N, 1)[0]
    logn = N.bit_length() - 1
    psi = O.psi(q, N)
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 1
    assert list(O.ntt_naive(q, one)) == [1] * N
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    pts = [int(v) for v in O.ntt_naive(q, x)]
    assert pts == [pow(psi, 2 * _bitrev(i, logn) + 1, q) for i in range(N)]
    assert len(set(pts)) == N and all(pow(p, N, q) == q - 1 for p in pts)


@pytest.mark.parametrize("N", [8, 32])
def test_ntt_convolution_theorem_and_roundtrip(N):
    """or_ntt_naive / or_intt_naive: NTT turns the negacyclic product
    (textbook, Python integers) into a pointwise product; INTT inverts it."""
    q = O.ntt_primes(N, 1)[0]
    rng = np.random.default_rng(N)
    a = [int(v) for v in rng.integers(0, q, N, dtype=np.uint64)]
    b = [int(v) for v in rng.integers(0, q, N, dtype=np.uint64)]
    ab = [v % q for v in tb.negacyclic(a, b)]
    A = O.ntt_naive(q, np.array(a, dtype=np.uint64))
    B = O.ntt_naive(q, np.array(b, dtype=np.uint64))
    AB = O.ntt_naive(q, np.array(ab, dtype=np.uint64))
    assert [int(x) for x in AB] == [int(x) * int(y) % q for x, y in zip(A, B)]
    assert [int(x) for x in O.intt_naive(q, A)] == a


# ------------------------------------------------------------ schoolbook ---
def test_negacyclic_matches_textbook_and_monomials():
    """or_negacyclic: Python big-int schoolbook; X^u X^v = +-X^((u+v) mod N)."""
    N = 32
    q = O.ntt_primes(N, 1)[0]
    rng = np.random.default_rng(1)
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    ref = [v % q for v in tb.negacyclic([int(x) for x in a], [int(x) for x in b])]
    assert [int(x) for x in O.negacyclic(q, a, b)] == ref
    for u, v in [(0, 0), (3, 5), (20, 20), (31, 1), (31, 31)]:
        xu = np.zeros(N, dtype=np.uint64)
        xv = np.zeros(N, dtype=np.uint64)
        xu[u] = 1
        xv[v] = 1
        out = O.negacyclic(q, xu, xv)
        exp = np.zeros(N, dtype=np.uint64)
        exp[(u + v) % N] = 1 if u + v < N else q - 1
        assert (out == exp).all()


# ------------------------------------------------------------------ PRNG ---
def test_prng_words_balanced():
    """or_prng_word: distinct words, each bit set about half the time
    (binomial, 6 sigma), streams of different objects differ."""
    w = [O.prng_word(7, 4, 1, 2, 3, i) for i in range(4096)]
    assert len(set(w)) == len(w)
    for bit in range(64):
        ones = sum((x >> bit) & 1 for x in w)
        assert abs(ones - 2048) < 6 * 32
    w2 = [O.prng_word(7, 4, 1, 2, 4, i) for i in range(64)]
    w3 = [O.prng_word(8, 4, 1, 2, 3, i) for i in range(64)]
    assert not set(w[:64]) & set(w2) and not set(w[:64]) & set(w3)


def test_cdt_matches_high_precision():
    """or_cdt: the double-precision table is within 2^12 of floor(CDF * 2^63)
    computed with 60 decimal digits; strictly increasing; last entry 2^63."""
    getcontext().prec = 60
    sigma = Decimal("3.2")
    rho = [(-(Decimal(k * k)) / (2 * sigma * sigma)).exp() for k in range(20)]
    S = rho[0] + 2 * sum(rho[1:])
    Tab = O.cdt(3.2)
    for k in range(19):
        exact = int((rho[0] + 2 * sum(rho[1:k + 1])) / S * (Decimal(2) ** 63))
        assert abs(Tab[k] - exact) <= 2**12, k
    assert Tab[19] == 2**63
    assert all(Tab[k] < Tab[k + 1] for k in range(19))


def test_golden_cdt_table():
    """The committed table (tests/golden/cdt_sigma3.2.txt) is the oracle's."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cdt_sigma3.2.txt")
    vals = [int(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")]
    assert vals == O.cdt(3.2)


# --------------------------------------------------------------- scheme ----
@pytest.fixture(scope="module")
def ctx16():
    return O.OracleCtx(16, 2, seed=11)


@pytest.fixture(scope="module")
def ctx16L3():
    return O.OracleCtx(16, 3, seed=12)


def _small(v: int, Q: int) -> int:
    return tb.centred(v, Q)


def test_secret_and_rlk_structure(ctx16L3):
    """Key generation: s ternary; b_j + a_j s - delta_ij s^2 is one small error
    polynomial e_j (|e_j| <= 19) seen identically in every limb."""
    c = ctx16L3
    s = [int(x) for x in c.secret()]
    assert set(s) <= {-1, 0, 1}
    s2 = tb.negacyclic(s, s)
    rlk = c.rlk()
    for j in range(c.L):
        errs = []
        for i, qi in enumerate(c.q):
            b = [int(x) for x in rlk[j, 0, i]]
            a = [int(x) for x in rlk[j, 1, i]]
            v = [(x + y) % qi for x, y in zip(b, tb.negacyclic(a, s))]
            if i == j:
                v = [(x - y) % qi for x, y in zip(v, s2)]
            e = [x - qi if x > qi // 2 else x for x in v]
            assert max(abs(x) for x in e) <= 19
            errs.append(e)
        assert all(e == errs[0] for e in errs)


def test_secret_ternary_frequencies():
    c = O.OracleCtx(4096, 1, seed=3)
    s = c.secret()
    counts = [int((s == v).sum()) for v in (-1, 0, 1)]
    for n in counts:  # binomial(4096, 1/3): sigma ~ 30
        assert abs(n - 4096 / 3) < 6 * 30.2


def test_encrypt_equation_and_fresh_noise():
    """or_encrypt: c0 + c1 s = Delta [m]_t X^0 + e (mod q_i) with the same
    small e in every limb; e is a rounded Gaussian of width 3.2: mean ~ 0,
    variance ~ 10.24, |e| <= 19, P(e=0) as the table gives; c1 uniform."""
    c = O.OracleCtx(256, 2, seed=21)
    Q = tb.prod(c.q)
    delta = Q // T
    assert c.delta() == delta
    s = [int(x) for x in c.secret()]
    allerr = []
    c1_vals = []
    for n, m in enumerate([0, 1, -1, 16, -16, 32768, -32768, 12345]):
        ct = c.encrypt(m, 3, n, 1)
        per_limb = []
        for i, qi in enumerate(c.q):
            c0 = [int(x) for x in ct[0, i]]
            c1 = [int(x) for x in ct[1, i]]
            c1_vals += c1
            v = [(x + y) % qi for x, y in zip(c0, tb.negacyclic(c1, s))]
            v[0] = (v[0] - delta * (m % T)) % qi
            per_limb.append([x - qi if x > qi // 2 else x for x in v])
        assert per_limb[0] == per_limb[1]
        allerr += per_limb[0]
    e = np.array(allerr, dtype=np.float64)
    assert np.abs(e).max() <= 19
    assert abs(e.mean()) < 6 * 3.2 / math.sqrt(len(e))
    assert abs(e.var() - 10.24) < 0.2 * 10.24
    rho = [math.exp(-k * k / 20.48) for k in range(20)]
    p0 = rho[0] / (rho[0] + 2 * sum(rho[1:]))
    n0 = int((e == 0).sum())
    assert abs(n0 - p0 * len(e)) < 6 * math.sqrt(len(e) * p0 * (1 - p0))
    # c1 uniform mod q_0 (both limbs pooled, normalised): 16 buckets, chi-square
    frac = np.array([v / c.q[0] for v in c1_vals[: len(c1_vals) // 2]])
    hist = np.histogram(frac, bins=16, range=(0, 1))[0]
    exp = len(frac) / 16
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 50  # 15 dof: p ~ 1e-5


@pytest.mark.parametrize("which", ["ctx16", "ctx16L3"])
def test_tensor_scale_matches_textbook(which, request):
    """or_tensor_scale: exact round(t x / Q) of the exact integer tensor."""
    c = request.getfixturevalue(which)
    a = c.encrypt(7, 1, 0, 0)
    b = c.encrypt(-9, 2, 0, 0)
    d = c.tensor_scale(a, b)
    ref = tb.tensor_scale(a, b, c.q, T)
    for p in range(3):
        assert (d[p] == tb.from_int_poly(ref[p], c.q)).all(), p


@pytest.mark.parametrize("which", ["ctx16", "ctx16L3"])
def test_tensor_scale_rounding_boundaries(which, request):
    """Coefficients on both rounding boundaries (t x / Q = n + 1/2 +- 1/(2Q))
    and on the centred-lift boundary ((Q-1)/2, (Q+1)/2)."""
    c = request.getfixturevalue(which)
    a, b = boundary_pair(c.q, T, c.N, seed=5)
    d = c.tensor_scale(a, b)
    ref = tb.tensor_scale(a, b, c.q, T)
    for p in range(3):
        assert (d[p] == tb.from_int_poly(ref[p], c.q)).all(), p
    # the lift boundary: (Q+1)/2 lifts to -(Q-1)/2, so d2 there is negative
    Q = tb.prod(c.q)
    b1 = tb.to_int_poly(b[1], c.q)
    d2 = tb.to_int_poly(d[2], c.q)
    for k in range(c.N):
        if b1[k] == (Q + 1) // 2:
            assert tb.centred(d2[k], Q) == -((T * (Q - 1) + Q) // (2 * Q))


@pytest.mark.parametrize("which", ["ctx16", "ctx16L3"])
def test_tensor_scale_sum_matches_textbook(which, request):
    """or_tensor_scale_sum: one exact rounding of the summed integer tensors
    (grouped accumulate-then-round), against big-integer arithmetic; with one
    pair it is or_tensor_scale."""
    c = request.getfixturevalue(which)
    pairs = [(c.encrypt(ma, 1, 0, k), c.encrypt(mb, 2, k, 0)) for k, (ma, mb) in enumerate([(7, -9), (16, 16), (-5, 3)])]
    d = c.tensor_scale_sum([p[0] for p in pairs], [p[1] for p in pairs])
    ref = tb.tensor_scale_sum(pairs, c.q, T)
    for p in range(3):
        assert (d[p] == tb.from_int_poly(ref[p], c.q)).all(), p
    assert (c.tensor_scale_sum([pairs[0][0]], [pairs[0][1]]) == c.tensor_scale(*pairs[0])).all()
    # a crafted pair on both rounding boundaries, summed with an ordinary one
    a, b = boundary_pair(c.q, T, c.N, seed=9)
    d = c.tensor_scale_sum([a, pairs[1][0]], [b, pairs[1][1]])
    ref = tb.tensor_scale_sum([(a, b), pairs[1]], c.q, T)
    for p in range(3):
        assert (d[p] == tb.from_int_poly(ref[p], c.q)).all(), p
    with pytest.raises(ValueError):
        c.tensor_scale_sum([a] * 1025, [b] * 1025)


def test_grouped_entries_decrypt_and_group_one_is_per_product(ctx16L3):
    """Entries computed with groups of 1 equal Alg. 1's per-product loop; larger
    groups give other ciphertexts with the same decryption (A B mod t) and
    each group's result is the textbook relinearisation of the summed tensor."""
    c = ctx16L3
    A = np.array([[3, 0, -7, 2, 5], [0, 0, 0, 0, 0], [16, -16, 1, 0, 9]], dtype=np.int64)
    B = np.array([[2, -1], [4, 0], [-3, 5], [7, 7], [1, -2]], dtype=np.int64)
    mm = O.OracleMatmul(c, A, B, 1, 2)
    enc = O.encode(A, O.CSR)
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            eager = mm.entry(enc, i, j)
            assert (mm.entry(enc, i, j, group=1) == eager).all()
            want = ((int(A[i] @ B[:, j]) + T // 2) % T) - T // 2
            for g in (2, 3, 8):
                lazy = mm.entry(enc, i, j, group=g)
                assert c.decrypt(lazy)[0] == want, (i, j, g)
    # one group holding all of row 0's products, against big integers
    ks = [k for k in range(A.shape[1]) if A[0, k]]
    pairs = [(mm.ct_a(0, k), mm.ct_b(k, 1)) for k in ks]
    ref = tb.relin(tb.tensor_scale_sum(pairs, c.q, T), c.rlk(), c.q)
    got = mm.entry(enc, 0, 1, group=len(ks))
    for p in range(2):
        assert (got[p] == tb.from_int_poly(ref[p], c.q)).all()


@pytest.mark.parametrize("which", ["ctx16", "ctx16L3"])
def test_mul_relin_matches_textbook(which, request):
    """or_relin / or_mul_relin: digits D_j = [d2]_{q_j}, c = (d0, d1) +
    sum_j D_j rlk_j, all in big-integer arithmetic mod Q."""
    c = request.getfixturevalue(which)
    a = c.encrypt(-3, 1, 2, 3)
    b = c.encrypt(11, 2, 3, 4)
    d = tb.tensor_scale(a, b, c.q, T)
    ref = tb.relin(d, c.rlk(), c.q)
    out = c.mul_relin(a, b)
    for p in range(2):
        assert (out[p] == tb.from_int_poly(ref[p], c.q)).all()


def test_relin_preserves_decryption(ctx16L3):
    """Gadget identity: sum_j D_j g_j == d2 (mod Q), so the relinearised
    ciphertext decrypts like d0 + d1 s + d2 s^2, to the product of the
    plaintexts."""
    c = ctx16L3
    Q = tb.prod(c.q)
    s = [int(x) for x in c.secret()]
    for ma, mb in [(3, 5), (-16, 16), (255, -255), (0, 9)]:
        a = c.encrypt(ma, 1, ma & 7, 0)
        b = c.encrypt(mb, 2, mb & 7, 0)
        d = c.tensor_scale(a, b)
        dint = [tb.to_int_poly(d[p], c.q) for p in range(3)]
        m3 = tb.decrypt3_int(dint, s, Q, T)
        # gadget: sum_j D_j (Q/q_j) [(Q/q_j)^-1]_{q_j} == d2 mod Q, coefficientwise
        for k in range(c.N):
            g = sum((dint[2][k] % qj) * (Q // qj) * pow(Q // qj, -1, qj) for qj in c.q)
            assert g % Q == dint[2][k]
        out = c.relin(d)
        m2 = tb.decrypt_int([tb.to_int_poly(out[p], c.q) for p in range(2)], s, Q, T)
        want = ((ma * mb + T // 2) % T) - T // 2
        assert m3[0] == want and m2[0] == want
        assert m2 == m3
        assert c.decrypt(out)[0] == want


def test_decrypt_matches_textbook(ctx16):
    c = ctx16
    Q = tb.prod(c.q)
    s = [int(x) for x in c.secret()]
    for m in [0, 1, -1, 32768, -32768, 65536, 70000]:
        ct = c.encrypt(m, 4, 0, m & 15)
        ref = tb.decrypt_int([tb.to_int_poly(ct[p], c.q) for p in range(2)], s, Q, T)
        got, bits = c.decrypt(ct)
        want = ((m + T // 2) % T) - T // 2
        assert got == ref[0] == want
        assert all(x == 0 for x in ref[1:])
        assert bits <= 5  # |e| <= 19


def test_noise_stays_below_decryption_bound():
    """Accumulating 16 products keeps the noise below Q / (2t)."""
    c = O.OracleCtx(64, 2, seed=9)
    Q = tb.prod(c.q)
    acc = np.zeros(c.ct_shape, dtype=np.uint64)
    total = 0
    for k in range(16):
        ma, mb = (k * 7) % 33 - 16, (k * 5) % 33 - 16
        total += ma * mb
        c.add_(acc, c.mul_relin(c.encrypt(ma, 1, 0, k), c.encrypt(mb, 2, k, 0)))
    m, bits = c.decrypt(acc)
    assert m == total
    assert 2**bits < Q // (2 * T)


# --------------------------------------------------------------- matmul ----
def _matmul_case(N=16, L=2, M=4, K=5, Nc=3, seed=0):
    c = O.OracleCtx(N, L, seed=seed)
    rng = np.random.default_rng(seed)
    A = rng.integers(-16, 17, size=(M, K))
    A[rng.random((M, K)) < 0.5] = 0
    A[1, :] = 0                      # an all-zero row: its entries are never touched
    B = rng.integers(-16, 17, size=(K, Nc))
    return c, A, B


def test_matmul_encodings_tiny():
    """Decryption equals A B mod t for every encoding; the three sparse
    encodings give bit-identical ciphertexts; all-zero rows of A give the
    exact zero ciphertext (no homomorphic op touches them)."""
    c, A, B = _matmul_case()
    mm = O.OracleMatmul(c, A, B, a_id=1, b_id=2)
    ref = A @ B
    C = {}
    for name, enc_id in O.ENCODINGS.items():
        enc = O.encode(A, enc_id)
        C[name] = [[mm.entry(enc, i, j) for j in range(B.shape[1])] for i in range(A.shape[0])]
        for i in range(A.shape[0]):
            for j in range(B.shape[1]):
                assert c.decrypt(C[name][i][j])[0] == ref[i, j]
    for i in range(A.shape[0]):
        for j in range(B.shape[1]):
            assert (C["mask"][i][j] == C["csr"][i][j]).all()
            assert (C["csr"][i][j] == C["ell"][i][j]).all()
            if i == 1:
                assert not C["csr"][i][j].any()
                assert C["dense"][i][j].any()   # dense multiplies encrypted zeros


def test_encoding_structures():
    """CSR row pointers / columns and ELLPACK width, columns and padding
    follow the definitions; every encoding lists the same nonzero products."""
    A = np.array([[0, 3, 0, 1], [0, 0, 0, 0], [5, 0, 0, 0], [1, 2, 3, 4]])
    csr = O.encode(A, O.CSR)
    assert list(csr.row_ptr) == [0, 2, 2, 3, 7]
    assert list(csr.col_idx) == [1, 3, 0, 0, 1, 2, 3]
    ell = O.encode(A, O.ELL)
    assert ell.width == 4
    assert ell.ell_col.tolist() == [[1, 3, -1, -1], [-1] * 4, [0, -1, -1, -1], [0, 1, 2, 3]]
    assert len(ell.values) == 16 and ell.coords[2] == (0, 6)   # padding slot 2 of row 0
    mask = O.encode(A, O.MASK)
    for i in range(4):
        ks = {k for _, k in O.product_set(csr, i)}
        assert ks == {k for _, k in O.product_set(ell, i)} == {k for _, k in O.product_set(mask, i)}
        assert ks == {k for k in range(4) if A[i, k] != 0}
        assert [k for _, k in O.product_set(O.encode(A, O.DENSE), i)] == [0, 1, 2, 3]


def test_two_sided_mask_skips_where_either_operand_is_zero():
    """Naive sparse over both operands (Sec. 3.3.2): entry (i, j) takes the k
    with A[i][k] != 0 and B[k][j] != 0 (checked against that definition);
    its ciphertext equals the one-sided entry of A with A[i][k] zeroed
    wherever B[k][j] is zero (the same encryptions, keyed by coordinates),
    it decrypts to (A B)[i][j] in per-product and grouped order, and it
    differs from the one-sided entry where a zero of B was skipped."""
    c, A, B = _matmul_case(M=3, K=6, Nc=3, seed=7)
    A[0, :] = [5, -3, 0, 7, 1, 2]
    B[[1, 3, 4], 0] = 0
    B[5, 2] = 0
    B[:, 1] = np.where(B[:, 1] == 0, 1, B[:, 1])       # column 1 without zeros
    bm = (B == 0).astype(np.uint8)
    assert bm[1, 0] and not bm[1, 1]                    # the mask is not symmetric in use
    mm = O.OracleMatmul(c, A, B, 1, 2)
    skipped = 0
    for name in ("mask", "csr", "ell"):
        enc = O.encode(A, O.ENCODINGS[name])
        for i in range(A.shape[0]):
            for j in range(B.shape[1]):
                ks = [k for _, k in O.entry_products(enc, i, j, bm)]
                assert ks == [k for k in range(A.shape[1]) if A[i, k] != 0 and B[k, j] != 0], (name, i, j)
                got = mm.entry(enc, i, j, b_mask=bm)
                A1 = A.copy()
                A1[i, B[:, j] == 0] = 0
                one = O.OracleMatmul(c, A1, B, 1, 2).entry(O.encode(A1, O.CSR), i, j)
                assert (got == one).all(), (name, i, j)
                want = ((int(A[i] @ B[:, j]) + T // 2) % T) - T // 2
                assert c.decrypt(got)[0] == want
                assert c.decrypt(mm.entry(enc, i, j, group=2, b_mask=bm))[0] == want
                full = mm.entry(enc, i, j)
                if len(ks) < len(O.product_set(enc, i)):
                    skipped += 1
                    assert not (got == full).all(), (name, i, j)
                else:
                    assert (got == full).all(), (name, i, j)
    assert skipped >= 3
    dense = O.encode(A, O.DENSE)
    assert O.entry_products(dense, 0, 0, bm) == O.product_set(dense, 0)   # Alg. 1 skips nothing


def test_paper_threading_scheme_matches_serial():
    """or_matmul_entries (one result entry per thread, (row*col) mod n) gives
    the same ciphertexts as the serial product loop."""
    c, A, B = _matmul_case(M=3, K=3, Nc=3, seed=4)
    mm = O.OracleMatmul(c, A, B, 1, 2)
    enc = O.encode(A, O.CSR)
    entries, alist, blist = [], [], []
    for i in range(3):
        for j in range(3):
            ps = O.product_set(enc, i)
            entries.append((i, j, len(alist), len(ps)))
            for _, k in ps:
                alist.append(mm.ct_a(i, k))
                blist.append(mm.ct_b(k, j))
    out = c.matmul_entries(entries, alist, blist, nthreads=3)
    for e, (i, j, _, _) in enumerate(entries):
        assert (out[e] == mm.entry(enc, i, j)).all()


def test_plaintext_wraps_mod_t():
    """Decryption is the integer product mod t (centred), also past t/2."""
    c = O.OracleCtx(16, 2, seed=2)
    a = c.encrypt(300, 1, 0, 0)
    b = c.encrypt(300, 2, 0, 0)
    assert c.decrypt(c.mul_relin(a, b))[0] == ((90000 + T // 2) % T) - T // 2


# ---------------------------------------------------- slot packing (N3) ----
def _rot_rows(v, k):
    """left rotation by k of each half of v (the two slot rows)"""
    h = len(v) // 2
    return np.concatenate([np.roll(v[:h], -k), np.roll(v[h:], -k)])


@pytest.mark.parametrize("N", [16, 32])
def test_slots_are_a_ring_isomorphism(N):
    """Slot encoding: decode(encode(v)) = v; a constant vector encodes to the
    constant polynomial; the negacyclic product of two encodings (big
    integers, mod t) decodes to the slot-wise product."""
    rng = np.random.default_rng(N)
    u = rng.integers(0, T, size=N)
    v = rng.integers(0, T, size=N)
    mu, mv = O.slots_encode(N, T, u), O.slots_encode(N, T, v)
    assert (O.slots_decode(N, T, mu) == u).all()
    const = O.slots_encode(N, T, np.full(N, 4242))
    assert int(const[0]) == 4242 and not const[1:].any()
    prod = [x % T for x in tb.negacyclic([int(x) for x in mu], [int(x) for x in mv])]
    assert [int(x) for x in O.slots_decode(N, T, prod)] == [int(a) * int(b) % T for a, b in zip(u, v)]


def test_poly_encryption_and_decryption(ctx16):
    """encrypt_poly of [m, 0, ..., 0] is the scalar encryption of m, limb
    for limb; decrypt_poly returns every coefficient of an encrypted
    polynomial with the noise of a fresh ciphertext."""
    c = ctx16
    for m in (0, 5, -7, 32768):
        poly = np.zeros(c.N, dtype=np.int64)
        poly[0] = m
        assert (c.encrypt_poly(poly, 3, 1, 2) == c.encrypt(m, 3, 1, 2)).all()
    poly = np.random.default_rng(1).integers(0, T, size=c.N)
    got, bits = c.decrypt_poly(c.encrypt_poly(poly, 4, 0, 0))
    assert (got == poly).all() and bits <= 5


@pytest.mark.parametrize("k", [1, 3, -1, -5])
def test_rotation_moves_slots(ctx16, k):
    """A key-switched automorphism X -> X^(3^k) rotates each slot row left
    by k (right for negative k); the Galois key is b_j + a_j s -
    delta_ij s(X^g) = one small error polynomial in every limb."""
    c = ctx16
    N = c.N
    g = O.rotation_element(N, k)
    key = c.galois_key(g)
    s = [int(x) for x in c.secret()]
    sg = [0] * N
    for i, x in enumerate(s):          # s(X^g) by the definition of X -> X^g
        d = i * g % (2 * N)
        if d < N:
            sg[d] += x
        else:
            sg[d - N] -= x
    for j in range(c.L):
        errs = []
        for i, qi in enumerate(c.q):
            b = [int(x) for x in key[j, 0, i]]
            a = [int(x) for x in key[j, 1, i]]
            e = [(x + y - (z if i == j else 0)) % qi for x, y, z in zip(b, tb.negacyclic(a, s), sg)]
            e = [x - qi if x > qi // 2 else x for x in e]
            assert max(abs(x) for x in e) <= 19
            errs.append(e)
        assert all(e == errs[0] for e in errs)
    v = np.random.default_rng(7).integers(0, T, size=N)
    ct = c.encrypt_poly(O.slots_encode(N, T, v), 5, 0, 0)
    m, bits = c.decrypt_poly(c.rotate(ct, g, key))
    assert (O.slots_decode(N, T, m) == _rot_rows(v, k)).all()
    assert 2**bits < tb.prod(c.q) // (2 * T)


def test_mul_plain_is_slotwise(ctx16):
    c = ctx16
    rng = np.random.default_rng(3)
    u, w = rng.integers(0, T, size=c.N), rng.integers(0, T, size=c.N)
    ct = c.encrypt_poly(O.slots_encode(c.N, T, u), 6, 0, 0)
    m, bits = c.decrypt_poly(c.mul_plain(ct, O.slots_encode(c.N, T, w)))
    assert [int(x) for x in O.slots_decode(c.N, T, m)] == [int(a) * int(b) % T for a, b in zip(u, w)]
    assert 2**bits < tb.prod(c.q) // (2 * T)


@pytest.mark.parametrize("chunk", [1, 3, 4])
def test_chunked_alg1_decrypts_to_the_product(chunk):
    """The chunked product with each term placed on its own (Alg. 1's
    placement): the result chunks decode to A B mod t, with and without the
    two-sided zero skip; skipping changes the ciphertexts (fewer products)
    but not the decryption."""
    c = O.OracleCtx(32, 3, seed=13)
    A = np.array([[3, 0, -7], [0, 5, 2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0]], dtype=np.int64)
    oc = O.OracleChunked(c, A, B, chunk, 1, 2)
    assert len(oc.a_ct) == -(-6 // chunk) and len(oc.b_ct) == -(-6 // chunk)
    full = oc.result()
    assert (oc.decode(full) == A @ B).all()
    skip = oc.result(skip_zeros=True)
    assert (oc.decode(skip) == A @ B).all()
    assert any(not (x == y).all() for x, y in zip(full, skip))


def test_chunked_fused_order_pins():
    """Placement on each entry's sum decrypts to A B mod t, and equals the
    per-term placement exactly for c = 1 (no turn to a result offset, and
    the mask product is exact and linear)."""
    c = O.OracleCtx(32, 3, seed=14)
    A = np.array([[3, 0, -7], [0, 5, 2]], dtype=np.int64)
    B = np.array([[2, -1], [0, 4], [6, 0]], dtype=np.int64)
    oc = O.OracleChunked(c, A, B, 4, 1, 2)
    assert (oc.decode(oc.result(placement="entry")) == A @ B).all()
    assert (oc.decode(oc.result(skip_zeros=True, placement="entry")) == A @ B).all()
    o1 = O.OracleChunked(c, A, B, 1, 1, 2)
    assert all((x == y).all() for x, y in zip(o1.result(), o1.result(placement="entry")))


def test_chunked_terms_and_placement_by_their_definition():
    """A product's term decrypts to A[i][k] B[k][j] mod t in slot 0 (both
    operands brought to slot 0 by their turns; the other slots hold the
    slot-wise products of the turned chunks), and place() leaves exactly that
    value in slot r mod c and zeros in every other slot."""
    c = O.OracleCtx(32, 3, seed=15)
    A = np.array([[3, -2, -7, 1], [4, 5, 2, -6]], dtype=np.int64)
    B = np.array([[2, -1, 3], [7, 4, -5], [6, 1, 2], [-3, 8, 1]], dtype=np.int64)
    oc = O.OracleChunked(c, A, B, 3, 1, 2)
    for i, k, j in [(0, 0, 0), (1, 2, 1), (1, 3, 2), (0, 1, 2)]:
        m, _ = c.decrypt_poly(oc.term(i, k, j))
        slots = [int(x) for x in O.slots_decode(c.N, T, m)]
        assert slots[0] == int(A[i, k] * B[k, j]) % T
        r = i * 3 + j
        m, _ = c.decrypt_poly(oc.place(oc.term(i, k, j), r))
        placed = [int(x) for x in O.slots_decode(c.N, T, m)]
        want = [0] * c.N
        want[r % 3] = int(A[i, k] * B[k, j]) % T
        assert placed == want, (i, k, j)
    sets = oc.product_sets(skip_zeros=True)
    assert sets[(0, 0)] == [0, 1, 2, 3] and all(len(v) == 4 for v in sets.values())
