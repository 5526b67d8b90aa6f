"""Writes the stored expected values under tests/golden/ from the oracle only.

cdt_sigma3.2.txt: cumulative table of |e| for the rounded Gaussian error of
width 3.2 (Homomorphic Encryption Security Standard error width), tail cut at
19, scaled to 2^63 (see or_cdt in oracle/bfv_oracle.c for the definition).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402


def main():
    with open(os.path.join(HERE, "cdt_sigma3.2.txt"), "w") as f:
        f.write("# k  T[k] = floor(CDF(|e| <= k) * 2^63), sigma = 3.2, tail 19; written by make_golden.py\n")
        for k, v in enumerate(O.cdt(3.2)):
            f.write(f"{k} {v}\n")


if __name__ == "__main__":
    main()
