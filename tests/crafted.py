"""Crafted ring elements on the rounding boundaries of the BFV multiply.

Both exact-rounding steps of the multiply have inputs whose rounding is
decided by a margin of 1/(2Q):
  * the centred lift of a coefficient c in [0, Q): c = (Q-1)/2 lifts to
    +(Q-1)/2, c = (Q+1)/2 to -(Q-1)/2;
  * round(t x / Q) for a tensor coefficient x with t x = (Q +- 1)/2 mod Q,
    i.e. t x / Q = n + 1/2 +- 1/(2Q).
With a0 = 1 and a1 = 1 (constant polynomials) the tensor is x0 = b0,
x1 = b0 + b1 (a0 b1 + a1 b0), x2 = b1, so every coefficient of b0 and b1 can
be placed on a boundary.  Test helper: builds residues only.
"""
from __future__ import annotations

import numpy as np

from textbook import from_int_poly, prod


def boundary_pair(q, t: int, N: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(a, b) coefficient-form [2][L][N] with a = (1, 1) and b on the boundaries."""
    rng = np.random.default_rng(seed)
    Q = prod(q)
    tinv = pow(t, -1, Q)
    one = [1] + [0] * (N - 1)
    a = np.stack([from_int_poly(one, q), from_int_poly(one, q)])
    b0, b1 = [], []
    for k in range(N):
        side = (Q + 1) // 2 if (k % 2 == 0) else (Q - 1) // 2
        x = (side * tinv) % Q                  # t x == side (mod Q)
        if k % 4 >= 2:
            x = Q - x                          # negative twin: t(-x) == -side
        b0.append(x)
        r = int(rng.integers(0, 4))
        if r == 0:
            b1.append((Q - 1) // 2)
        elif r == 1:
            b1.append((Q + 1) // 2)
        else:
            b1.append(x if r == 2 else int(rng.integers(0, 2**62)) % Q)
    b = np.stack([from_int_poly(b0, q), from_int_poly(b1, q)])
    return a, b
