"""Textbook BFV with Python integers: one big modulus Q, no RNS, no auxiliary
base, no NTT.  Used only to pin the oracle on tiny rings (test helper)."""
from __future__ import annotations

import numpy as np


def prod(xs):
    r = 1
    for x in xs:
        r *= x
    return r


def crt(limbs, q):
    """Integer in [0, Q) from residues (Gauss's construction)."""
    Q = prod(q)
    x = 0
    for r, qi in zip(limbs, q):
        Mi = Q // qi
        x += int(r) * Mi * pow(Mi, -1, qi)
    return x % Q


def to_int_poly(limbs: np.ndarray, q) -> list[int]:
    """[L][N] residues -> N integers in [0, Q)."""
    L, N = limbs.shape
    return [crt([limbs[i, k] for i in range(L)], q) for k in range(N)]


def from_int_poly(coeffs, q) -> np.ndarray:
    return np.array([[c % qi for c in coeffs] for qi in q], dtype=np.uint64)


def centred(x: int, M: int) -> int:
    x %= M
    return x - M if x > M // 2 else x


def negacyclic(a, b):
    N = len(a)
    out = [0] * N
    for i in range(N):
        if a[i] == 0:
            continue
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += a[i] * b[j]
            else:
                out[k - N] -= a[i] * b[j]
    return out


def tensor_scale(ct_a: np.ndarray, ct_b: np.ndarray, q, t: int) -> list[list[int]]:
    """round(t x / Q) mod Q for x0 = a0 b0, x1 = a0 b1 + a1 b0, x2 = a1 b1 over Z."""
    Q = prod(q)
    a0, a1 = ([centred(c, Q) for c in to_int_poly(ct_a[p], q)] for p in (0, 1))
    b0, b1 = ([centred(c, Q) for c in to_int_poly(ct_b[p], q)] for p in (0, 1))
    x0 = negacyclic(a0, b0)
    x1 = [u + v for u, v in zip(negacyclic(a0, b1), negacyclic(a1, b0))]
    x2 = negacyclic(a1, b1)
    # Python's // floors toward -infinity
    return [[((2 * t * x + Q) // (2 * Q)) % Q for x in xs] for xs in (x0, x1, x2)]


def tensor_scale_sum(pairs, q, t: int) -> list[list[int]]:
    """round(t (x(a_0, b_0) + ... ) / Q) mod Q: one rounding of the summed
    integer tensors."""
    Q = prod(q)
    N = pairs[0][0].shape[-1]
    X = [[0] * N for _ in range(3)]
    for ct_a, ct_b in pairs:
        a0, a1 = ([centred(c, Q) for c in to_int_poly(ct_a[p], q)] for p in (0, 1))
        b0, b1 = ([centred(c, Q) for c in to_int_poly(ct_b[p], q)] for p in (0, 1))
        x1 = [u + v for u, v in zip(negacyclic(a0, b1), negacyclic(a1, b0))]
        for p, xs in enumerate((negacyclic(a0, b0), x1, negacyclic(a1, b1))):
            X[p] = [u + v for u, v in zip(X[p], xs)]
    return [[((2 * t * x + Q) // (2 * Q)) % Q for x in xs] for xs in X]


def relin(d, rlk: np.ndarray, q) -> list[list[int]]:
    """c0 = d0 + sum_j D_j b_j, c1 = d1 + sum_j D_j a_j (mod Q), D_j = d2 mod q_j."""
    Q = prod(q)
    L = len(q)
    c0, c1 = list(d[0]), list(d[1])
    for j in range(L):
        Dj = [x % q[j] for x in d[2]]
        bj = to_int_poly(rlk[j, 0], q)
        aj = to_int_poly(rlk[j, 1], q)
        c0 = [(u + v) % Q for u, v in zip(c0, negacyclic(Dj, bj))]
        c1 = [(u + v) % Q for u, v in zip(c1, negacyclic(Dj, aj))]
    return [c0, c1]


def decrypt_int(ct_polys, s, Q: int, t: int) -> list[int]:
    """m = round(t [c0 + c1 s]_Q / Q) mod t, centred, every coefficient."""
    c0, c1 = ct_polys
    v = [(x + y) % Q for x, y in zip(c0, negacyclic(c1, list(s)))]
    ms = [((t * x + Q // 2) // Q) % t for x in v]
    return [m - t if m > t // 2 else m for m in ms]


def decrypt3_int(d, s, Q: int, t: int) -> list[int]:
    """Decryption of a three-component ciphertext: d0 + d1 s + d2 s^2."""
    s = list(s)
    s2 = negacyclic(s, s)
    v = [(x + y + z) % Q for x, y, z in zip(d[0], negacyclic(d[1], s), negacyclic(d[2], s2))]
    ms = [((t * x + Q // 2) // Q) % t for x in v]
    return [m - t if m > t // 2 else m for m in ms]
