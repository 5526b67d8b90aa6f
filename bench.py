"""Benchmark of the encrypted sparse matmul on GB300.

Workload (default): A 64x64 with 50% Bernoulli unstructured zeros (ints in
[-16, 16], seed 1) times B 64x64 dense, one BFV ciphertext per element,
N = 8192, four 54-bit primes, t = 65537; A CSR-encoded.  A step is one pass
of the whole hot path over that input, as the library runs it:
  lift of A and B to Q u P, work-list build and upload, and the batched
  persistent kernel (tensor, exact scale-and-round, relinearisation,
  accumulation) over every nonzero product.
Encryption, key generation and decryption are setup and are not timed (the
paper times the matmul alone).  `value` = ciphertext products per second
with operands resident in HBM; `e2e` adds the host->device copy of the
operand ciphertexts and the device->host copy of C.  The plain per-product
path (four launches per product) is timed on a bounded sample of the same
workload and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ct-mults/s and encrypted matmul ms at 50% sparsity, batched vs plain, 1 GB300"
UNIT = "ct-mults/s"
SPARSITY = 0.5
ENCODING = "csr"
# The path is bound by the integer multiply pipe.  Work is counted in 32x32-bit
# multiplies (partial products) that the algorithm's modular arithmetic needs:
# a 30-bit Shoup or Barrett multiply 3, a 64-bit Shoup multiply 10 (mul.hi.u64
# 4 + two mul.lo.u64 3 each), a 64-bit Barrett reduction 7, a 30x54-bit split
# product 2.  Peak: 64 integer multiply-adds per clock per SM (Blackwell's
# integer multiply rate) x 152 SMs x the maximum SM clock.
IMAD_PER_CLK_PER_SM = 64
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-rows", type=int, default=2, help="rows of A timed through the plain path")
    ap.add_argument("--cpu-products", type=int, default=12, help="oracle products in the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default=None, help="M,K,Nc override (small profiling cases)")
    return ap.parse_args()


# --------------------------------------------------------- algorithmic work ---
def tensor_base_size(logN: int, L: int) -> int:
    """tensor-base primes K (as the library chooses them)."""
    return (10 * (logN + 108 * L + 1) + 298) // 299


def mults_per_product(N: int, L: int) -> int:
    """32-bit multiplies of one product: tensor over the K tensor-base primes
    (10 per coefficient and prime), 3K inverse NTTs (3 per butterfly), exact
    scale-and-round of the 3 polynomials (6K + 2KL + 9L per coefficient: the
    CRT digits, the overflow count, the fixed-point fraction, and the
    reconstruction mod every q_i)."""
    logN = int(math.log2(N))
    K = tensor_base_size(logN, L)
    tensor = 10 * K * N
    intt = 3 * K * (N // 2) * logN * 3
    scale = 3 * N * (6 * K + 2 * K * L + 9 * L)
    return tensor + intt + scale


def mults_per_entry(N: int, L: int) -> int:
    """per output entry with at least one product: L (L + 2) forward 64-bit
    NTTs of the accumulated sums (10 per butterfly, Barrett-reduced inputs),
    the key products (10 each) and the final reductions."""
    logN = int(math.log2(N))
    ntts = L * (L + 2) * ((N // 2) * logN * 10 + 7 * N)
    keyprod = 2 * L * L * N * 10
    final = 2 * L * N * 7
    return ntts + keyprod + final


def mults(products: int, entries: int, N: int, L: int) -> float:
    return products * mults_per_product(N, L) + entries * mults_per_entry(N, L)


# ------------------------------------------------------------------- clocks ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------- CPU oracle ---
def cpu_oracle_rate(ring, A, B, n_products: int, seed: int = 0) -> dict:
    """The oracle as it stands (OpenMP over the host cores) on a bounded
    sample: the first n_products nonzero products of row-major order."""
    from oracle import oracle as O
    octx = O.OracleCtx(ring.N, ring.L, seed=seed)
    pairs = [(i, k, j) for i in range(A.shape[0]) for k in range(A.shape[1]) if A[i, k] != 0
             for j in range(B.shape[1])][:n_products]
    ops = [(octx.encrypt(int(A[i, k]), 1, i, k), octx.encrypt(int(B[k, j]), 2, k, j)) for i, k, j in pairs]
    t0 = time.perf_counter()
    acc = np.zeros(octx.ct_shape, dtype=np.uint64)
    for a, b in ops:
        octx.add_(acc, octx.mul_relin(a, b))
    dt = time.perf_counter() - t0
    return {"value": len(ops) / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{len(ops)} ct x ct products (multiply + relinearise + add) of the same workload, "
                      f"schoolbook negacyclic products, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ring = W.SWEEP_RING
    A, B = W.operands(W.sweep(SPARSITY))
    from oracle import oracle as O
    octx = O.OracleCtx(ring.N, ring.L, seed=0)
    pairs = [(i, k, j) for i in range(A.shape[0]) for k in range(A.shape[1]) if A[i, k] != 0
             for j in range(B.shape[1])]
    per_step = 2
    need = (args.warmup + args.steps) * per_step
    ops = [(octx.encrypt(int(A[i, k]), 1, i, k), octx.encrypt(int(B[k, j]), 2, k, j)) for i, k, j in pairs[:need]]
    acc = np.zeros(octx.ct_shape, dtype=np.uint64)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for a, b in ops[s * per_step:(s + 1) * per_step]:
            octx.add_(acc, octx.mul_relin(a, b))
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "sweep-64x64x64-s0.5", "N": ring.N, "L": ring.L, "t": W.T_PLAIN,
                       "sparsity": SPARSITY, "encoding": ENCODING},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} products per step of the same workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------- main ---
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_09184_gb300 import api, sfhe as S

    ring = W.SWEEP_RING
    shape = W.sweep(SPARSITY)
    workload = "sweep-64x64x64-s0.5"
    if args.shape:
        M, K, Nc = (int(x) for x in args.shape.split(","))
        shape = W.MatmulShape(M, K, Nc, shape.sparsity, shape.lo, shape.hi, shape.seed)
        workload = f"sweep-{M}x{K}x{Nc}-s0.5"
    A_vals, B_vals = W.operands(shape)
    ctx = api.Context(ring.N, ring.L, seed=0)
    stream = torch.cuda.current_stream()

    # setup (untimed): encryption of the operands
    A = api.encrypt_matrix(ctx, A_vals, ENCODING, 1, lift=False)
    B = api.encrypt_matrix(ctx, B_vals, "dense", 2, lift=False)
    A.ext = api._dev_u32((A.nct, 2, ctx.K, ctx.N))
    B.ext = api._dev_u32((B.nct, 2, ctx.K, ctx.N))
    C = api.result_matrix(ctx, shape.M, shape.Nc)
    lift_ws = torch.empty(S.sfhe_lift_workspace_size(ctx.h, max(A.nct, B.nct)), dtype=torch.uint8, device="cuda")
    flags = api.PERSISTENT
    mm_ws = api.workspace(ctx, [A], [B], flags)
    ctx.check()

    def lift_all():
        S.sfhe_lift(ctx.h, A.ct, A.nct, A.ext, lift_ws, stream)
        S.sfhe_lift(ctx.h, B.ct, B.nct, B.ext, lift_ws, stream)

    kernel_ms = []

    def step(record: bool):
        lift_all()
        plan = S.sfhe_plan_create(ctx.h, [A.desc()], [B.desc()], [C.desc()], flags, mm_ws, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.sfhe_plan_execute(plan, stream)
        e1.record(stream)
        S.sfhe_plan_destroy(plan)
        if record:
            kernel_ms.append((e0, e1))
        return plan

    probe = S.sfhe_plan_create(ctx.h, [A.desc()], [B.desc()], [C.desc()], flags, mm_ws, stream)
    stats = S.sfhe_plan_stats(probe)
    S.sfhe_plan_destroy(probe)
    products, entries, ctas = stats["products"], stats["entries"], stats["ctas"]
    nonempty_entries = entries - sum(1 for i in range(shape.M) if not (A_vals[i] != 0).any()) * shape.Nc
    lift_launches = 3 * (math.ceil(A.nct / 256) + math.ceil(B.nct / 256))

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    kms = statistics.mean(a.elapsed_time(b) for a, b in kernel_ms)

    # correctness of the timed result: decrypt C and compare with A B mod t
    dec = api.decrypt(ctx, C)
    ref = ((A_vals @ B_vals + W.T_PLAIN // 2) % W.T_PLAIN) - W.T_PLAIN // 2
    correct = bool((dec == ref).all())

    # e2e: operands from pinned host memory, C back to pinned host memory
    hA = torch.empty(A.ct.shape, dtype=torch.int64, pin_memory=True)
    hB = torch.empty(B.ct.shape, dtype=torch.int64, pin_memory=True)
    hC = torch.empty(C.ct.shape, dtype=torch.int64, pin_memory=True)
    hA.copy_(A.ct)
    hB.copy_(B.ct)
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 3))
    for s in range(1 + e2e_steps):
        if s == 1:
            torch.cuda.synchronize()
            te0 = time.perf_counter()
        A.ct.copy_(hA, non_blocking=True)
        B.ct.copy_(hB, non_blocking=True)
        step(False)
        hC.copy_(C.ct, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = 1e3 * (time.perf_counter() - te0) / e2e_steps
    h2d = (hA.numel() + hB.numel()) * 8
    d2h = hC.numel() * 8

    # plain per-product path on a bounded sample: the first rows of A
    rows = list(range(min(args.plain_rows, shape.M)))
    A_rows = api.encrypt_matrix(ctx, A_vals[rows], ENCODING, 1)
    B.ext = B.ext  # lifted above
    C_rows = api.result_matrix(ctx, len(rows), shape.Nc)
    plain_ws = api.workspace(ctx, [A_rows], [B], api.PLAIN)
    pplan = S.sfhe_plan_create(ctx.h, [A_rows.desc()], [B.desc()], [C_rows.desc()], api.PLAIN, plain_ws, stream)
    pstats = S.sfhe_plan_stats(pplan)
    S.sfhe_plan_execute(pplan, stream)      # warm-up
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    S.sfhe_plan_execute(pplan, stream)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    S.sfhe_plan_destroy(pplan)
    plain_rate = pstats["products"] / (plain_ms / 1e3)
    # the plain and the persistent paths must agree limb for limb
    pers_rows = api.to_coeff(ctx, C.ct[: len(rows) * shape.Nc].contiguous(), len(rows) * shape.Nc)
    plain_rows = api.to_coeff(ctx, C_rows.ct, len(rows) * shape.Nc)
    plain_equal = bool((pers_rows == plain_rows).all())

    value = products * world / (ms / 1e3)
    work = mults(products, nonempty_entries, ring.N, ring.L)
    achieved = work / (kms / 1e3) / 1e12
    sm_clock = clk.get("sm_mhz") or SM_MAX_MHZ
    peak = SM_COUNT * IMAD_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload, "M": shape.M, "K": shape.K, "Nc": shape.Nc,
                   "sparsity": SPARSITY, "encoding": ENCODING, "N": ring.N, "L": ring.L, "t": W.T_PLAIN,
                   "products_per_step": products, "dense_products": shape.M * shape.K * shape.Nc,
                   "l2": f"inputs larger than L2 (lifted A and B: {(A.ext.numel() + B.ext.numel()) * A.ext.element_size() / 1e9:.1f} GB)",
                   "step": "lift A and B + work list + persistent matmul", "parallelism": f"replicas x{world}"},
        "matmul_ms": ms,
        "kernel_ms": kms,
        "correct": correct,
        "plain": {"value": plain_rate, "unit": UNIT, "products": pstats["products"],
                  "launches": pstats["launches"], "sample": f"rows {rows[0]}..{rows[-1]} of A, all columns",
                  "matmul_ms_extrapolated": products / plain_rate * 1e3, "bit_identical_to_batched": plain_equal},
        "speedup_batched_vs_plain": value / world / plain_rate,
        "e2e": {"value": products * world / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T int32-mul/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_matmul_persistent<13,4>",
                     "work_per_launch": work,
                     "peak_note": "152 SM x 64 int32 multiplies/clk x 2070 MHz (derived from unit counts and clock)",
                     "frac_at_measured_clock": achieved / (peak * sm_clock / SM_MAX_MHZ)},
        "gpu_launches": (lift_launches + 1) * args.steps,
        "clocks": clk,
        "persistent_ctas": ctas,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rate(ring, A_vals, B_vals, args.cpu_products)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
