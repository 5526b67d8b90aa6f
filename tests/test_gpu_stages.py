"""Stage-level parity of the CUDA path with the oracle, bit-exact in every
limb: generator words, keys, NTT form (ciphertext and tensor-base primes),
encryption, the exact centred lift to the tensor base, the tensor with its
exact scale-and-round (including inputs on both rounding boundaries),
relinearisation and decryption."""
from __future__ import annotations

import numpy as np
import pytest

import textbook as tb
from crafted import boundary_pair
from gpu_common import coeff_of, gpu_ctx, gpu_modules, oracle_ctx
from oracle import oracle as O

pytestmark = pytest.mark.gpu
T = 65537
RINGS = [(4096, 2), (4096, 3), (8192, 4)]


@pytest.fixture(scope="module")
def mods():
    return gpu_modules()


def test_generator_stream_equality(mods):
    import torch
    api, S = mods
    for (seed, dom, o) in [(0, 4, (1, 2, 3)), (7, 2, (3, 0, 0)), (2**63 + 5, 5, (9, 64, 71))]:
        out = torch.empty(300, dtype=torch.int64, device="cuda")
        S.sfhe_prng_words(seed, dom, *o, 1000, 300, out)
        got = api.to_numpy_u64(out)
        ref = [O.prng_word(seed, dom, *o, 1000 + i) for i in range(300)]
        assert [int(x) for x in got] == ref


@pytest.mark.parametrize("N,L", RINGS + [(16384, 8)])
def test_keys_match_oracle(mods, N, L):
    import torch
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    assert ctx.q == octx.q
    assert (S.sfhe_export_secret(ctx.h).astype(np.int64) == octx.secret()).all()
    rlk = torch.empty((L, 2, L, N), dtype=torch.int64, device="cuda")
    S.sfhe_export_relin_key(ctx.h, rlk)
    assert (api.to_numpy_u64(rlk) == octx.rlk()).all()


@pytest.mark.parametrize("N,L", [(4096, 2), (8192, 4), (16384, 8)])
def test_ntt_matches_definition(mods, N, L):
    """Forward NTT against the evaluation-at-odd-powers definition, for a
    ciphertext prime (64-bit words) and tensor-base primes (32-bit words);
    inverse round trip."""
    import torch
    api, S = mods
    ctx = gpu_ctx(N, L, 1)
    rng = np.random.default_rng(N)
    for pi in (0, L, L + ctx.K - 1):
        q = (ctx.q + ctx.b)[pi]
        a = rng.integers(0, q, size=(3, N), dtype=np.uint64)
        a[1] = 0
        a[1, 0] = 1                       # NTT(1) = all ones
        a[2, : N // 2] = q - 1            # top of the range
        if pi < L:
            dev = torch.from_numpy(a.view(np.int64)).cuda()
            view = api.to_numpy_u64
        else:
            dev = torch.from_numpy(a.astype(np.uint32).view(np.int32)).cuda()
            view = api.to_numpy_u32
        out = torch.empty_like(dev)
        S.sfhe_ntt(ctx.h, pi, False, dev, 3, out)
        got = view(out).astype(np.uint64)
        assert (got[1] == 1).all()
        assert (got[0] == O.ntt_naive(q, a[0])).all()
        back = torch.empty_like(dev)
        S.sfhe_ntt(ctx.h, pi, True, out, 3, back)
        assert (view(back).astype(np.uint64) == a).all()


@pytest.mark.parametrize("N,L", RINGS + [(16384, 8)])
def test_encrypt_matches_oracle(mods, N, L):
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    vals = np.array([0, 1, -1, 16, -16, 32768, -32768, 65536, 123456], dtype=np.int64)
    coords = np.array([(i, 3 * i + 1) for i in range(len(vals))], dtype=np.int32).reshape(-1)
    n = len(vals)
    import torch
    ct = torch.empty((n, 2, L, N), dtype=torch.int64, device="cuda")
    S.sfhe_encrypt(ctx.h, vals, coords, 77, ct)
    ctx.check()
    got = api.to_coeff(ctx, ct, n)
    count = n if N < 16384 else 2   # the oracle's schoolbook encryption is slow at N = 16384
    for k in range(count):
        assert (got[k] == octx.encrypt(int(vals[k]), 77, k, 3 * k + 1)).all(), k


def _lift_reference(coeff, q, b):
    """centred lift of every coefficient, reduced mod the tensor-base primes (big ints)."""
    Q = tb.prod(q)
    out = np.zeros((coeff.shape[0], 2, len(b), coeff.shape[-1]), dtype=np.uint64)
    for n in range(coeff.shape[0]):
        for pl in range(2):
            xs = [tb.centred(x, Q) for x in tb.to_int_poly(coeff[n, pl], q)]
            for k, bk in enumerate(b):
                out[n, pl, k] = [x % bk for x in xs]
    return out


@pytest.mark.parametrize("N,L", [(4096, 2), (4096, 3)])
def test_lift_is_exact_centred_extension(mods, N, L):
    """Lifted ciphertext = centred lift mod every b_k (big integers), also for
    the lift boundaries (Q-1)/2 and (Q+1)/2 and values next to them."""
    import torch
    api, S = mods
    ctx = gpu_ctx(N, L, 1)
    Q = tb.prod(ctx.q)
    rng = np.random.default_rng(3)
    ints = [[int(rng.integers(0, 2**62)) * int(rng.integers(0, 2**62)) % Q for _ in range(N)] for _ in range(4)]
    specials = [(Q - 1) // 2, (Q + 1) // 2, (Q - 3) // 2, (Q + 3) // 2, 0, 1, Q - 1]
    for k, v in enumerate(specials * 20):
        ints[k % 4][(k * 37) % N] = v
    coeff = np.stack([np.stack([tb.from_int_poly(ints[2 * n], ctx.q), tb.from_int_poly(ints[2 * n + 1], ctx.q)])
                      for n in range(2)])
    M = api.import_coeff(ctx, coeff)
    Bc = api.ext_to_coeff(ctx, M.ext).astype(np.uint64)
    assert (Bc == _lift_reference(coeff, ctx.q, ctx.b)).all()


def _tensor_scale_gpu(api, S, ctx, A_ext, a, b):
    import torch
    d = torch.empty((3, ctx.L, ctx.N), dtype=torch.int64, device="cuda")
    work = torch.empty(3 * ctx.K * ctx.N * 4, dtype=torch.uint8, device="cuda")
    S.sfhe_ct_tensor_scale(ctx.h, A_ext[a], A_ext[b], d, work)
    return api.to_numpy_u64(d)


@pytest.mark.parametrize("N,L", RINGS)
def test_tensor_scale_matches_oracle(mods, N, L):
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    vals = np.array([[5, -7, 16, -16]], dtype=np.int64)
    M = api.encrypt_matrix(ctx, vals, "dense", 11)
    for a, b in [(0, 1), (2, 3), (1, 1)]:
        got = _tensor_scale_gpu(api, S, ctx, M.ext, a, b)
        ref = octx.tensor_scale(octx.encrypt(int(vals[0, a]), 11, 0, a), octx.encrypt(int(vals[0, b]), 11, 0, b))
        assert (got == ref).all()


@pytest.mark.parametrize("N,L", [(4096, 2), (4096, 3)])
def test_tensor_scale_rounding_boundaries(mods, N, L):
    """Tensor coefficients with t x / Q = n + 1/2 +- 1/(2Q) and lift
    boundaries: the exact fallbacks of both roundings are exercised."""
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    a, b = boundary_pair(ctx.q, T, N, seed=7)
    M = api.import_coeff(ctx, np.stack([a, b]))
    got = _tensor_scale_gpu(api, S, ctx, M.ext, 0, 1)
    ref = octx.tensor_scale(a, b)
    assert (got == ref).all()


@pytest.mark.parametrize("N,L", RINGS)
def test_mul_relin_matches_oracle(mods, N, L):
    import torch
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    vals = np.array([[3, -11]], dtype=np.int64)
    M = api.encrypt_matrix(ctx, vals, "dense", 12)
    out = torch.empty((1, 2, L, N), dtype=torch.int64, device="cuda")
    need = ((3 * ctx.K * N * 4 + 255) // 256) * 256 + (3 * L + (L + 2) * L) * N * 8
    work = torch.empty(need, dtype=torch.uint8, device="cuda")
    S.sfhe_ct_mul_relin(ctx.h, M.ext[0], M.ext[1], out[0], work)
    got = api.to_coeff(ctx, out, 1)[0]
    ref = octx.mul_relin(octx.encrypt(3, 12, 0, 0), octx.encrypt(-11, 12, 0, 1))
    assert (got == ref).all()
    assert octx.decrypt(got)[0] == -33


@pytest.mark.parametrize("N,L", RINGS)
def test_decrypt_matches_oracle(mods, N, L):
    api, S = mods
    ctx, octx = gpu_ctx(N, L, 1), oracle_ctx(N, L, 1)
    vals = np.array([[0, 1, -1, 32768, -32768, 40000, 7, -9]], dtype=np.int64)
    M = api.encrypt_matrix(ctx, vals, "dense", 13, lift=False)
    got = api.decrypt(ctx, M)[0]
    want = ((vals[0] + T // 2) % T) - T // 2
    assert (got == want).all()
    coeff = coeff_of(api, ctx, M)
    assert [octx.decrypt(coeff[k])[0] for k in range(vals.shape[1])] == list(got)


def test_measured_mulmod_rate_is_below_the_derived_peak():
    """sfhe_measure_mulmod32: a positive rate whose three 32-bit multiplies
    per modular multiply stay below 152 SMs x 64 multiplies per clock at the
    GPU's maximum clock (the derived integer peak)."""
    import torch
    api, S = gpu_modules()
    ctx = gpu_ctx(8192, 4, 0)
    r = S.sfhe_measure_mulmod32(ctx.h, torch.cuda.current_stream())
    props = torch.cuda.get_device_properties(0)
    peak = props.multi_processor_count * 64 * 2.07e9
    assert 0 < 3 * r <= 1.05 * peak, (r, peak)
