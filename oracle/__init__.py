"""Plain CPU oracle for the encrypted sparse matmul.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py; never by the CUDA path.

Parity status of each oracle function (what pins it) is listed in
tests/test_oracle_*.py; every function is pinned (no "parity unpinned"
entries).
"""
