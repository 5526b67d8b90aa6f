"""Convenience layer over the C ABI: contexts, encrypted matrices held in
torch device tensors, matmul plans.  Argument marshalling only; all
arithmetic runs in libsfhe.so's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import sfhe as S

PLAIN, PERSISTENT, GRAPH, LAZY = S.SFHE_EXEC_PLAIN, S.SFHE_EXEC_PERSISTENT, S.SFHE_EXEC_GRAPH, S.SFHE_EXEC_LAZY


def _dev_u64(shape) -> torch.Tensor:
    """uint64 words in an int64 device tensor (same bits)."""
    return torch.empty(shape, dtype=torch.int64, device="cuda")


def _dev_u32(shape) -> torch.Tensor:
    """uint32 words in an int32 device tensor (same bits)."""
    return torch.empty(shape, dtype=torch.int32, device="cuda")


def to_numpy_u64(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def to_numpy_u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


class Context:
    def __init__(self, N: int, L: int, t: int = 65537, sigma: float = 3.2, seed: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.h = S.sfhe_ctx_create(N, L, t, sigma, seed)
        info = S.sfhe_ctx_info(self.h)
        self.N, self.L, self.K, self.t = info.N, info.L, info.K, info.t
        self.q = [int(x) for x in info.q[: self.L]]
        self.b = [int(x) for x in info.b[: self.K]]
        self.ct_words, self.ext_words, self.num_sms = int(info.ct_words), int(info.ext_words), info.num_sms
        self.ext_interleave = int(info.ext_interleave)
        self.lazy_group = int(info.lazy_group)
        self.l2_window, self.l2_hit_ratio = int(info.l2_window), float(info.l2_hit_ratio)
        self.seed = seed

    def close(self):
        if getattr(self, "h", None):
            S.sfhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, stream=None):
        S.sfhe_ctx_check(self.h, stream)


class EncMatrix:
    """An encoded, encrypted matrix: host structure arrays + device storage."""

    def __init__(self, rows, cols, encoding, nct, ell_width=0, mask=None, row_ptr=None, col_idx=None, ell_col=None,
                 ct=None, ext=None):
        self.rows, self.cols, self.encoding, self.nct, self.ell_width = rows, cols, encoding, nct, ell_width
        self.mask, self.row_ptr, self.col_idx, self.ell_col = mask, row_ptr, col_idx, ell_col
        self.ct, self.ext = ct, ext

    def desc(self) -> S.sfhe_matrix_view:
        def p(a):
            return None if a is None else S._ptr(a)
        return S.sfhe_matrix_view(self.rows, self.cols, self.encoding, self.nct, self.ell_width, p(self.mask),
                              p(self.row_ptr), p(self.col_idx), p(self.ell_col), p(self.ct), p(self.ext))

    def memory(self, ctx: "Context") -> dict:
        """bytes of the ciphertexts, of their lift and of the plaintext
        structure this encoding holds (sfhe_matrix_bytes)."""
        return S.sfhe_matrix_bytes(ctx.N, ctx.L, self.desc())


def encrypt_matrix(ctx: Context, values: np.ndarray, encoding: int | str, matrix_id: int, lift: bool = True,
                   stream=None, col_offset: int = 0) -> EncMatrix:
    """col_offset: the matrix is a column block of a larger one starting at
    that column; elements are encrypted under their coordinates in the larger
    matrix (the same ciphertexts as encrypting it whole)."""
    if isinstance(encoding, str):
        encoding = S.ENCODINGS[encoding]
    values = np.ascontiguousarray(values, dtype=np.int64)
    rows, cols = values.shape
    f = S.sfhe_encode_fill(values, encoding)
    if col_offset:
        if encoding != S.SFHE_ENC_DENSE:
            raise ValueError("column blocks of DENSE matrices only")
        f["ct_coords"][1::2] += col_offset
    nct = f["nct"]
    M = EncMatrix(rows, cols, encoding, nct, f["ell_width"], f["mask"], f["row_ptr"], f["col_idx"], f["ell_col"])
    M.ct = _dev_u64((max(nct, 1), 2, ctx.L, ctx.N))
    S.sfhe_encrypt(ctx.h, f["ct_values"], f["ct_coords"], matrix_id, M.ct, stream)
    if lift:
        lift_matrix(ctx, M, stream)
    return M


def lift_matrix(ctx: Context, M: EncMatrix, stream=None):
    M.ext = _dev_u32((max(M.nct, 1), 2, ctx.K, ctx.N))
    if M.nct:
        work = torch.empty(S.sfhe_lift_workspace_size(ctx.h, M.nct), dtype=torch.uint8, device="cuda")
        S.sfhe_lift(ctx.h, M.ct, M.nct, M.ext, work, stream)
        # keep the workspace alive until the stream has consumed it
        (torch.cuda.current_stream() if stream is None else stream).synchronize()


def result_matrix(ctx: Context, rows: int, cols: int) -> EncMatrix:
    C = EncMatrix(rows, cols, S.SFHE_ENC_DENSE, rows * cols)
    C.ct = _dev_u64((max(rows * cols, 1), 2, ctx.L, ctx.N))
    return C


def import_coeff(ctx: Context, coeff: np.ndarray, lift: bool = True, stream=None) -> EncMatrix:
    """Ciphertexts given in coefficient form [n][2][L][N] as a 1 x n DENSE row."""
    coeff = np.ascontiguousarray(coeff, dtype=np.uint64)
    n = coeff.shape[0]
    src = torch.from_numpy(coeff.view(np.int64)).cuda()
    M = EncMatrix(1, n, S.SFHE_ENC_DENSE, n)
    M.ct = _dev_u64(coeff.shape)
    S.sfhe_from_coeff(ctx.h, src, 2 * n, M.ct, stream)
    if lift:
        lift_matrix(ctx, M, stream)
    return M


def ext_to_coeff(ctx: Context, ext: torch.Tensor) -> np.ndarray:
    """coefficient form of lifted ciphertexts: [n][2][K][N] uint32 residues mod b_k
    (the lifted layout is undone first: slot i is stored at (i mod R)(N/R) + i/R)."""
    n = ext.shape[0]
    R = ctx.ext_interleave
    out = np.zeros((n, 2, ctx.K, ctx.N), dtype=np.uint32)
    for k in range(ctx.K):
        src = ext[:, :, k].reshape(n, 2, R, ctx.N // R).transpose(-1, -2).contiguous().reshape(n, 2, ctx.N)
        dst = torch.empty_like(src)
        S.sfhe_ntt(ctx.h, ctx.L + k, True, src, 2 * n, dst)
        out[:, :, k] = to_numpy_u32(dst)
    return out


def to_coeff(ctx: Context, ct: torch.Tensor, n: int, stream=None) -> np.ndarray:
    out = _dev_u64((n, 2, ctx.L, ctx.N))
    S.sfhe_to_coeff(ctx.h, ct, 2 * n, out, stream)
    return to_numpy_u64(out)


def decrypt(ctx: Context, M: EncMatrix, stream=None) -> np.ndarray:
    out = torch.empty(max(M.nct, 1), dtype=torch.int64, device="cuda")
    S.sfhe_decrypt(ctx.h, M.ct, M.nct, out, stream)
    vals = out.cpu().numpy()[: M.nct]
    if M.encoding in (S.SFHE_ENC_DENSE, S.SFHE_ENC_MASK):
        return vals.reshape(M.rows, M.cols)
    return vals


def _flags(mode: str, graph: bool = False) -> int:
    """mode: "persistent", "plain" or "lazy" (persistent, grouped accumulate-then-round)."""
    f = {"persistent": PERSISTENT, "plain": PLAIN, "lazy": PERSISTENT | LAZY}[mode]
    return f | (GRAPH if graph else 0)


def workspace(ctx: Context, As, Bs, flags: int) -> torch.Tensor:
    n = S.sfhe_matmul_workspace_size(ctx.h, [a.desc() for a in As], [b.desc() for b in Bs], flags)
    return torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")


def matmul(ctx: Context, A: EncMatrix, B: EncMatrix, *, dense: bool = False, mode: str = "persistent",
           stream=None, work: torch.Tensor | None = None) -> EncMatrix:
    """C = A x B: the dense loop (Alg. 1) or the loop over A's nonzeros as
    A's encoding lists them."""
    C = result_matrix(ctx, A.rows, B.cols)
    dense = dense or A.encoding == S.SFHE_ENC_DENSE
    flags = _flags(mode)
    if work is None:
        work = workspace(ctx, [A], [B], flags)
    Ad, Bd, Cd = A.desc(), B.desc(), C.desc()
    if dense:
        S.sfhe_matmul_dense_view(ctx.h, Ad, Bd, Cd, flags, work, stream)
    else:
        S.sfhe_matmul_sparse_view(ctx.h, Ad, Bd, A.encoding, Cd, flags, work, stream)
    C._work = work
    return C


def matmul_batch(ctx: Context, As, Bs, *, mode: str = "persistent", stream=None) -> list[EncMatrix]:
    Cs = [result_matrix(ctx, a.rows, b.cols) for a, b in zip(As, Bs)]
    flags = _flags(mode)
    work = workspace(ctx, As, Bs, flags)
    S.sfhe_matmul_batch_view(ctx.h, [a.desc() for a in As], [b.desc() for b in Bs], [c.desc() for c in Cs], flags, work,
                        stream)
    for c in Cs:
        c._work = work
    return Cs


class Plan:
    """A matmul plan (work list uploaded once); execute() only launches."""

    def __init__(self, ctx: Context, As, Bs, *, mode: str = "persistent", graph: bool = False, stream=None,
                 Cs=None):
        self.ctx = ctx
        self.As, self.Bs = list(As), list(Bs)
        self.Cs = Cs if Cs is not None else [result_matrix(ctx, a.rows, b.cols) for a, b in zip(As, Bs)]
        flags = _flags(mode, graph)
        self.work = workspace(ctx, self.As, self.Bs, flags)
        self.h = S.sfhe_plan_create(ctx.h, [a.desc() for a in self.As], [b.desc() for b in self.Bs],
                                    [c.desc() for c in self.Cs], flags, self.work, stream)
        self.stats = S.sfhe_plan_stats(self.h)

    def execute(self, stream=None):
        S.sfhe_plan_execute(self.h, stream)

    def close(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            S.sfhe_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------ slot-packed chunks -------
class ChunkedMatrix:
    """A matrix stored as Alg. 1's chunks (Sec. 3.2): element e of the
    row-major order in slot e mod c of chunk ciphertext e / c."""

    def __init__(self, rows: int, cols: int, c: int, ct: torch.Tensor, zero: np.ndarray | None = None):
        self.rows, self.cols, self.c, self.ct, self.zero = rows, cols, c, ct, zero

    @property
    def nchunks(self) -> int:
        return -(-(self.rows * self.cols) // self.c)


def encrypt_chunked(ctx: Context, values: np.ndarray, c: int, matrix_id: int, stream=None) -> ChunkedMatrix:
    """chunk q encrypted under the stream object (matrix_id, q, 0)"""
    values = np.ascontiguousarray(values, dtype=np.int64)
    flat = values.reshape(-1)
    n = -(-flat.size // c)
    polys = np.zeros((max(n, 1), ctx.N), dtype=np.int64)
    for q in range(n):
        v = np.zeros(ctx.N, dtype=np.int64)
        part = flat[q * c:(q + 1) * c]
        v[:part.size] = part
        polys[q] = S.sfhe_slots_encode(ctx.N, ctx.t, v)
    coords = np.zeros((max(n, 1), 2), dtype=np.int32)
    coords[:, 0] = np.arange(max(n, 1))
    ct = _dev_u64((max(n, 1), 2, ctx.L, ctx.N))
    if n:
        S.sfhe_encrypt_poly(ctx.h, polys[:n], coords[:n], matrix_id, ct, stream)
    return ChunkedMatrix(values.shape[0], values.shape[1], c, ct, (values == 0).astype(np.uint8))


def decrypt_chunked(ctx: Context, M: ChunkedMatrix, stream=None) -> np.ndarray:
    """the matrix, centred mod t"""
    n = M.nchunks
    out = torch.empty((max(n, 1), ctx.N), dtype=torch.int64, device="cuda")
    S.sfhe_decrypt_poly(ctx.h, M.ct, n, out, stream)
    (torch.cuda.current_stream() if stream is None else stream).synchronize()
    polys = out.cpu().numpy()
    vals = []
    for q in range(n):
        vals.extend(int(x) for x in S.sfhe_slots_decode(ctx.N, ctx.t, polys[q])[:M.c])
    t = ctx.t
    flat = np.array(vals[:M.rows * M.cols], dtype=np.int64)
    return (((flat + t // 2) % t) - t // 2).reshape(M.rows, M.cols)


class RotationKeys:
    """Galois keys of the left and right rotations by 1 .. c-1."""

    def __init__(self, ctx: Context, c: int, stream=None):
        self.ctx, self.c = ctx, c
        self.h = S.sfhe_rotkeys_create(ctx.h, c, stream)

    def close(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize()
            S.sfhe_rotkeys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def matmul_chunked(ctx: Context, A: ChunkedMatrix, B: ChunkedMatrix, rk: RotationKeys, *, skip_zeros: bool = False,
                   fused: bool = False, stream=None, work: torch.Tensor | None = None) -> tuple[ChunkedMatrix, int]:
    """C = A x B by Alg. 1 over chunks; skip_zeros: the naive sparse scheme's
    two masks (products where A[i][k] or B[k][j] is zero are skipped); fused:
    operand rotations once per element, inner sums on the persistent kernel,
    mask and result rotation per entry (same decryption, other ciphertext).
    Returns (C, products performed)."""
    assert A.c == B.c == rk.c and A.cols == B.rows
    c = A.c
    nC = -(-(A.rows * B.cols) // c)
    C = ChunkedMatrix(A.rows, B.cols, c, _dev_u64((max(nC, 1), 2, ctx.L, ctx.N)))
    az = np.ascontiguousarray(A.zero.reshape(-1)) if skip_zeros else None
    bz = np.ascontiguousarray(B.zero.reshape(-1)) if skip_zeros else None
    if fused:
        if work is None:
            n_bytes = S.sfhe_matmul_chunked_fused_workspace_size(ctx.h, c, A.rows, A.cols, B.cols, az, bz)
            work = torch.empty(n_bytes, dtype=torch.uint8, device="cuda")
        n = S.sfhe_matmul_chunked_fused(ctx.h, rk.h, A.rows, A.cols, B.cols, A.ct, B.ct, C.ct, az, bz, work, stream)
    else:
        if work is None:
            work = torch.empty(S.sfhe_matmul_chunked_workspace_size(ctx.h), dtype=torch.uint8, device="cuda")
        n = S.sfhe_matmul_chunked(ctx.h, rk.h, A.rows, A.cols, B.cols, A.ct, B.ct, C.ct, az, bz, work, stream)
    C._work = work
    return C, n
