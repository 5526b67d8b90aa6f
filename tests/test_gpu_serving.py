"""The serving loop on the GPU: requests that overlap in time (several
waves, budget-limited admission) give, limb for limb, the ciphertexts each
request gives alone, and decrypt to A B mod t."""
from __future__ import annotations

import pytest

import workloads as W
from gpu_common import gpu_ctx, gpu_modules

pytestmark = pytest.mark.gpu


def test_requests_alone_and_in_the_mix_are_identical():
    api, S = gpu_modules()
    from paper_2503_09184_gb300 import serving as SV
    ctx = gpu_ctx(4096, 2, 0)
    shapes = [(8, 8, 8, 0.5), (12, 8, 4, 0.3), (6, 16, 8, 0.7), (8, 8, 8, 0.9), (16, 4, 2, 0.5)]
    reqs = []
    for rid, (M, K, Nc, s) in enumerate(shapes):
        A, B = W.operands(W.MatmulShape(M, K, Nc, s, -16, 16, 100 + rid))
        reqs.append(SV.Request(rid, A, B, arrival=0.01 * rid))
    ct_b = 2 * ctx.L * ctx.N * 8
    ext_b = 2 * ctx.K * ctx.N * 4
    ex = SV.GpuExecutor(ctx, wave_products=96)
    # at most two or three requests in flight beside the executor's workspace
    budget = 2 * max(SV.request_bytes(r, ct_b, ext_b) for r in reqs) + ex.reserved_bytes
    out = SV.serve(reqs, ex, budget, wave_products=96, ct_bytes=ct_b, ext_bytes=ext_b, keep_results=True)
    assert out["reserved_bytes"] == ex.reserved_bytes > 0
    assert out["wave_kernel_s"] > 0 and out["wave_setup_s"] > 0
    assert out["done"] == len(reqs) and out["waves"] > len(reqs)
    for r in reqs:
        C_mix = ex.result(r)
        A = api.encrypt_matrix(ctx, r.A, "csr", 2 * r.rid + 1)
        B = api.encrypt_matrix(ctx, r.B, "dense", 2 * r.rid + 2)
        C_alone = api.matmul(ctx, A, B)
        n = r.A.shape[0] * r.B.shape[1]
        assert (api.to_coeff(ctx, C_mix.ct, n) == api.to_coeff(ctx, C_alone.ct, n)).all(), r.rid
        want = ((r.A @ r.B + W.T_PLAIN // 2) % W.T_PLAIN) - W.T_PLAIN // 2
        assert (api.decrypt(ctx, C_mix) == want).all()


def test_column_tiles_equal_the_untiled_request():
    """A request over the budget runs as column tiles; every tile's C equals
    the matching columns of the request run alone, limb for limb."""
    api, S = gpu_modules()
    from paper_2503_09184_gb300 import serving as SV
    ctx = gpu_ctx(4096, 2, 0)
    A, B = W.operands(W.MatmulShape(6, 8, 10, 0.4, -16, 16, 300))
    req = SV.Request(7, A, B, arrival=0.0)
    ct_b, ext_b = 2 * ctx.L * ctx.N * 8, 2 * ctx.K * ctx.N * 4
    nnz = int((A != 0).sum())
    ex = SV.GpuExecutor(ctx, wave_products=64)
    # four columns per tile beside A and the executor's workspace
    budget = nnz * (ct_b + ext_b) + 4 * (8 * (ct_b + ext_b) + 6 * ct_b) + ex.reserved_bytes
    out = SV.serve([req], ex, budget, wave_products=64, ct_bytes=ct_b, ext_bytes=ext_b, keep_results=True)
    assert out["done"] == 1 and req.state == "done"
    Ae = api.encrypt_matrix(ctx, A, "csr", 2 * req.rid + 1)
    Be = api.encrypt_matrix(ctx, B, "dense", 2 * req.rid + 2)
    whole = api.to_coeff(ctx, api.matmul(ctx, Ae, Be).ct, 60).reshape(6, 10, 2, ctx.L, ctx.N)
    for c0 in (0, 4, 8):
        w = min(4, 10 - c0)
        tile = api.to_coeff(ctx, ex.result(req, c0).ct, 6 * w).reshape(6, w, 2, ctx.L, ctx.N)
        assert (tile == whole[:, c0:c0 + w]).all(), c0
