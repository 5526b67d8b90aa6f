"""Thin Python binding of the C ABI in include/sfhe.h (libsfhe.so).

Functions keep the C names and only marshal arguments: every step of the
computation runs in the library's CUDA kernels.  Device buffers are torch
tensors (int64 storage holding the uint64 words); streams are torch CUDA
streams.  Loading fails loudly when the compiled library is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfhe.so")

SFHE_OK, SFHE_EINVAL, SFHE_ESHAPE, SFHE_ENOMEM, SFHE_ECUDA = 0, 1, 2, 3, 4
SFHE_ETIMEOUT, SFHE_EBUDGET, SFHE_EUNSUPPORTED, SFHE_EDEVICE = 5, 6, 7, 8
SFHE_ENC_DENSE, SFHE_ENC_MASK, SFHE_ENC_CSR, SFHE_ENC_ELL = 0, 1, 2, 3
SFHE_EXEC_PLAIN, SFHE_EXEC_PERSISTENT, SFHE_EXEC_GRAPH, SFHE_EXEC_LAZY = 1, 2, 4, 8
ENCODINGS = {"dense": SFHE_ENC_DENSE, "mask": SFHE_ENC_MASK, "csr": SFHE_ENC_CSR, "ell": SFHE_ENC_ELL}


class SfheError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"sfhe status {status}: {message}")
        self.status = status


class sfhe_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("t", ctypes.c_uint64), ("sigma", ctypes.c_double)]


class sfhe_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("K", ctypes.c_uint32),
                ("t", ctypes.c_uint64), ("q", ctypes.c_uint64 * 8), ("b", ctypes.c_uint32 * 32),
                ("ct_words", ctypes.c_uint64), ("ext_words", ctypes.c_uint64), ("num_sms", ctypes.c_int32),
                ("ext_interleave", ctypes.c_uint32), ("lazy_group", ctypes.c_int32),
                ("l2_window", ctypes.c_uint64), ("l2_hit_ratio", ctypes.c_float)]


class sfhe_matrix_view(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("encoding", ctypes.c_int32),
                ("nct", ctypes.c_int32), ("ell_width", ctypes.c_int32),
                ("mask", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("ell_col", ctypes.c_void_p), ("ct", ctypes.c_void_p), ("ext", ctypes.c_void_p)]


class sfhe_ckks_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("L", ctypes.c_uint32), ("bits", ctypes.c_uint32 * 8),
                ("special_bits", ctypes.c_uint32), ("log_scale", ctypes.c_uint32), ("sigma", ctypes.c_double)]


_vp, _u32, _u64, _i32, _i64, _sz = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.c_int64, ctypes.c_size_t)
_P = ctypes.POINTER

# name -> (argtypes, restype)
_SIGS = {
    "sfhe_ctx_create": ([_P(sfhe_params), _u64, _P(_vp)], ctypes.c_int),
    "sfhe_ctx_destroy": ([_vp], None),
    "sfhe_ctx_info": ([_vp, _P(sfhe_info)], ctypes.c_int),
    "sfhe_ctx_check": ([_vp, _vp], ctypes.c_int),
    "sfhe_last_error": ([], ctypes.c_char_p),
    "sfhe_select_primes": ([_u32, _u32, _vp, _vp, _P(_i32)], ctypes.c_int),
    "sfhe_cdt_table": ([ctypes.c_double, _vp], ctypes.c_int),
    "sfhe_encode_count": ([_vp, _i32, _i32, _i32, _P(_i32), _P(_i32)], ctypes.c_int),
    "sfhe_encode_fill": ([_vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sfhe_matrix_bytes": ([_u32, _u32, _P(sfhe_matrix_view), _P(_u64), _P(_u64), _P(_u64)], ctypes.c_int),
    "sfhe_encrypt": ([_vp, _vp, _vp, _i64, _u64, _vp, _vp], ctypes.c_int),
    "sfhe_lift_workspace_size": ([_vp, _i64, _P(_sz)], ctypes.c_int),
    "sfhe_lift": ([_vp, _vp, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_decrypt": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_to_coeff": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_from_coeff": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_export_secret": ([_vp, _vp], ctypes.c_int),
    "sfhe_export_relin_key": ([_vp, _vp, _vp], ctypes.c_int),
    "sfhe_matmul_workspace_size": ([_vp, _i32, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _u32, _P(_sz)], ctypes.c_int),
    "sfhe_matmul_workspace_bound": ([_vp, _i32, _i64, _i64, _u32, _P(_sz)], ctypes.c_int),
    "sfhe_matmul_dense_view": ([_vp, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _P(sfhe_matrix_view), _u32, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_matmul_sparse_view": ([_vp, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _i32, _P(sfhe_matrix_view), _u32, _vp, _sz, _vp],
                           ctypes.c_int),
    "sfhe_matmul_batch_view": ([_vp, _i32, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _P(sfhe_matrix_view), _u32, _vp, _sz, _vp],
                          ctypes.c_int),
    "sfhe_plan_create": ([_vp, _i32, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _P(sfhe_matrix_view), _u32, _vp, _sz, _vp, _P(_vp)],
                         ctypes.c_int),
    "sfhe_plan_execute": ([_vp, _vp], ctypes.c_int),
    "sfhe_plan_set_stop": ([_vp, _vp], ctypes.c_int),
    "sfhe_plan_progress": ([_vp, _P(_i64), _vp], ctypes.c_int),
    "sfhe_plan_resume": ([_vp, _vp], ctypes.c_int),
    "sfhe_slots_encode": ([_u32, _u64, _vp, _vp], ctypes.c_int),
    "sfhe_slots_decode": ([_u32, _u64, _vp, _vp], ctypes.c_int),
    "sfhe_rotation_element": ([_u32, _i32], _u32),
    "sfhe_encrypt_poly": ([_vp, _vp, _vp, _i64, _u64, _vp, _vp], ctypes.c_int),
    "sfhe_decrypt_poly": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_galois_keygen": ([_vp, _u32, _vp, _vp, _vp], ctypes.c_int),
    "sfhe_rotate_workspace_size": ([_vp, _P(_sz)], ctypes.c_int),
    "sfhe_rotate": ([_vp, _vp, _i64, _u32, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_plain_ntt": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "sfhe_mul_plain": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_add": ([_vp, _vp, _vp, _i64, _vp], ctypes.c_int),
    "sfhe_rotkeys_create": ([_vp, _i32, _vp, _P(_vp)], ctypes.c_int),
    "sfhe_rotkeys_destroy": ([_vp], None),
    "sfhe_matmul_chunked_workspace_size": ([_vp, _P(_sz)], ctypes.c_int),
    "sfhe_matmul_chunked": ([_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _P(_i64)],
                            ctypes.c_int),
    "sfhe_matmul_chunked_fused_workspace_size": ([_vp, _i32, _i32, _i32, _i32, _vp, _vp, _P(_sz)], ctypes.c_int),
    "sfhe_matmul_chunked_fused": ([_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _P(_i64)],
                                  ctypes.c_int),
    "sfhe_measure_mulmod32": ([_vp, _P(ctypes.c_double), _vp], ctypes.c_int),
    "sfhe_plan_stats": ([_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i64)], ctypes.c_int),
    "sfhe_ctx_tuning": ([_vp, _P(_i32), _P(_i32), _vp], ctypes.c_int),
    "sfhe_ctx_set_variant": ([_vp, _i32], ctypes.c_int),
    "sfhe_ctx_variant_name": ([_vp, _i32], ctypes.c_char_p),
    "sfhe_matmul_check": ([_vp, _vp], ctypes.c_int),
    "sfhe_selftest_wait_bound": ([_vp, _u32, _u32, _vp], ctypes.c_int),
    "sfhe_plan_destroy": ([_vp], None),
    "sfhe_ct_tensor_scale": ([_vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_ct_mul_relin": ([_vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_ct_mul_relin_static": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sfhe_ntt": ([_vp, _i32, _i32, _vp, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_prng_words": ([_u64, _u32, _u64, _u64, _u64, _u64, _i64, _vp, _vp], ctypes.c_int),
    # library-owned matrices and matmuls over them
    "sfhe_ctx_get_primes": ([_vp, _vp, _vp], ctypes.c_int),
    "sfhe_matrix_encrypt": ([_vp, _vp, _i32, _i32, ctypes.c_int, _u64, _vp, _P(_vp)], ctypes.c_int),
    "sfhe_matrix_import": ([_vp, _vp, _vp, _i32, _i32, ctypes.c_int, _vp, _P(_vp)], ctypes.c_int),
    "sfhe_matrix_export": ([_vp, _vp, _vp], ctypes.c_int),
    "sfhe_matrix_decrypt": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "sfhe_matrix_destroy": ([_vp], None),
    "sfhe_matrix_info": ([_vp, _P(_i32), _P(_i32), _P(_i32), _P(_i32)], ctypes.c_int),
    "sfhe_matrix_view_of": ([_vp, _P(sfhe_matrix_view), _vp], ctypes.c_int),
    "sfhe_matmul_dense": ([_vp, _vp, _vp, _P(_vp), _vp], ctypes.c_int),
    "sfhe_matmul_sparse": ([_vp, _vp, _vp, ctypes.c_int, _P(_vp), _vp], ctypes.c_int),
    "sfhe_matmul_batch": ([_vp, _i32, _P(_vp), _P(_vp), _P(_vp), _u32, _vp], ctypes.c_int),
    # host-resident operands
    "sfhe_host_plan_create": ([_vp, _i32, _P(sfhe_matrix_view), _P(sfhe_matrix_view), _u32, _i32, _P(_vp)],
                              ctypes.c_int),
    "sfhe_matmul_host": ([_vp, _P(_vp), _P(_vp), _P(_vp), _vp], ctypes.c_int),
    "sfhe_host_plan_stats": ([_vp, _P(_i64), _P(_u64), _P(_u64), _P(_i64)], ctypes.c_int),
    "sfhe_host_plan_destroy": ([_vp], None),
    # CKKS
    "sfhe_ckks_ctx_create": ([_P(sfhe_ckks_params), _u64, _P(_vp)], ctypes.c_int),
    "sfhe_ckks_ctx_destroy": ([_vp], None),
    "sfhe_ckks_ctx_primes": ([_vp, _vp, _P(_u64), _P(ctypes.c_double)], ctypes.c_int),
    "sfhe_ckks_encode": ([_vp, _vp, _i32, ctypes.c_double, _vp], ctypes.c_int),
    "sfhe_ckks_decode": ([_vp, _vp, _i32, ctypes.c_double, _i32, _vp], ctypes.c_int),
    "sfhe_ckks_encrypt": ([_vp, _vp, _vp, _i64, _u64, _vp, _vp], ctypes.c_int),
    "sfhe_ckks_decrypt": ([_vp, _vp, _i32, _i64, ctypes.c_double, _i32, _vp, _vp], ctypes.c_int),
    "sfhe_ckks_to_coeff": ([_vp, _vp, _i32, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_ckks_workspace_size": ([_vp, _P(_sz)], ctypes.c_int),
    "sfhe_ckks_mul_relin": ([_vp, _vp, _vp, _i32, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_ckks_rescale": ([_vp, _vp, _i32, _i64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_ckks_rotkeys_create": ([_vp, _i32, _vp, _P(_vp)], ctypes.c_int),
    "sfhe_ckks_rotkeys_destroy": ([_vp], None),
    "sfhe_ckks_rotate": ([_vp, _vp, _vp, _i32, _i32, _vp, _vp, _sz, _vp], ctypes.c_int),
    "sfhe_ckks_plain_ntt": ([_vp, _vp, _i32, _vp, _vp], ctypes.c_int),
    "sfhe_ckks_mul_plain": ([_vp, _vp, _i32, _i64, _vp, _vp], ctypes.c_int),
    "sfhe_ckks_add": ([_vp, _vp, _vp, _i32, _i64, _vp], ctypes.c_int),
    "sfhe_ckks_matmul_chunked_workspace_size": ([_vp, _P(_sz)], ctypes.c_int),
    "sfhe_ckks_matmul_chunked": ([_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _P(_i64),
                                  _P(ctypes.c_double)], ctypes.c_int),
}

_lib = None


def lib(path: str = LIB_PATH):
    """The loaded libsfhe.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(path)
        for name, (argt, rest) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = argt
            f.restype = rest
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(status: int):
    if status != SFHE_OK:
        msg = lib().sfhe_last_error()
        raise SfheError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    """device/host address of a torch tensor or numpy array (None for None)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


# ---------------------------------------------------------------- context ---
def sfhe_ctx_create(N: int, L: int, t: int = 65537, sigma: float = 3.2, seed: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_ctx_create(ctypes.byref(sfhe_params(N, L, t, sigma)), seed, ctypes.byref(h)))
    return h.value


def sfhe_ctx_destroy(ctx: int) -> None:
    lib().sfhe_ctx_destroy(ctx)


def sfhe_ctx_info(ctx: int) -> sfhe_info:
    info = sfhe_info()
    _check(lib().sfhe_ctx_info(ctx, ctypes.byref(info)))
    return info


def sfhe_ctx_check(ctx: int, stream=None) -> None:
    _check(lib().sfhe_ctx_check(ctx, _stream(stream)))


def sfhe_select_primes(N: int, L: int) -> tuple[list[int], list[int]]:
    """(ciphertext primes q, tensor-base primes b)."""
    q = np.zeros(8, dtype=np.uint64)
    b = np.zeros(32, dtype=np.uint32)
    K = ctypes.c_int32()
    _check(lib().sfhe_select_primes(N, L, _ptr(q), _ptr(b), ctypes.byref(K)))
    return [int(x) for x in q[:L]], [int(x) for x in b[:K.value]]


def sfhe_cdt_table(sigma: float = 3.2) -> list[int]:
    T = np.zeros(20, dtype=np.uint64)
    _check(lib().sfhe_cdt_table(sigma, _ptr(T)))
    return [int(x) for x in T]


# --------------------------------------------------------------- operands ---
def sfhe_encode_count(values: np.ndarray, encoding: int) -> tuple[int, int]:
    v = np.ascontiguousarray(values, dtype=np.int64)
    nct, w = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sfhe_encode_count(_ptr(v), v.shape[0], v.shape[1], encoding, ctypes.byref(nct), ctypes.byref(w)))
    return nct.value, w.value


def sfhe_encode_fill(values: np.ndarray, encoding: int) -> dict:
    v = np.ascontiguousarray(values, dtype=np.int64)
    rows, cols = v.shape
    nct, width = sfhe_encode_count(v, encoding)
    out = {"nct": nct, "ell_width": width, "mask": None, "row_ptr": None, "col_idx": None, "ell_col": None,
           "ct_values": np.zeros(nct, dtype=np.int64), "ct_coords": np.zeros(2 * max(nct, 1), dtype=np.int32)}
    if encoding == SFHE_ENC_MASK:
        out["mask"] = np.zeros(rows * cols, dtype=np.uint8)
    if encoding == SFHE_ENC_CSR:
        out["row_ptr"] = np.zeros(rows + 1, dtype=np.int32)
        out["col_idx"] = np.zeros(max(nct, 1), dtype=np.int32)
    if encoding == SFHE_ENC_ELL:
        out["ell_col"] = np.zeros(max(rows * width, 1), dtype=np.int32)
    _check(lib().sfhe_encode_fill(_ptr(v), rows, cols, encoding, _ptr(out["mask"]), _ptr(out["row_ptr"]),
                                  _ptr(out["col_idx"]), _ptr(out["ell_col"]), _ptr(out["ct_values"]),
                                  _ptr(out["ct_coords"])))
    return out


def sfhe_matrix_bytes(N: int, L: int, M) -> dict:
    """{"ct", "ext", "meta"}: bytes of an encoded operand's ciphertexts, of
    their lift to the tensor base and of its plaintext structure."""
    v = [ctypes.c_uint64() for _ in range(3)]
    _check(lib().sfhe_matrix_bytes(N, L, ctypes.byref(M), *[ctypes.byref(x) for x in v]))
    return dict(zip(("ct", "ext", "meta"), (x.value for x in v)))


def sfhe_encrypt(ctx: int, values: np.ndarray, coords: np.ndarray, matrix_id: int, ct, stream=None) -> None:
    values = np.ascontiguousarray(values, dtype=np.int64)
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    _check(lib().sfhe_encrypt(ctx, _ptr(values), _ptr(coords), values.size, matrix_id, _ptr(ct), _stream(stream)))


def sfhe_lift_workspace_size(ctx: int, n: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_lift_workspace_size(ctx, n, ctypes.byref(b)))
    return b.value


def sfhe_lift(ctx: int, ct, n: int, ext, work, stream=None) -> None:
    _check(lib().sfhe_lift(ctx, _ptr(ct), n, _ptr(ext), _ptr(work), work.numel() * work.element_size(),
                           _stream(stream)))


def sfhe_decrypt(ctx: int, ct, n: int, out, stream=None) -> None:
    _check(lib().sfhe_decrypt(ctx, _ptr(ct), n, _ptr(out), _stream(stream)))


def sfhe_to_coeff(ctx: int, inp, npoly: int, out, stream=None) -> None:
    _check(lib().sfhe_to_coeff(ctx, _ptr(inp), npoly, _ptr(out), _stream(stream)))


def sfhe_from_coeff(ctx: int, inp, npoly: int, out, stream=None) -> None:
    _check(lib().sfhe_from_coeff(ctx, _ptr(inp), npoly, _ptr(out), _stream(stream)))


def sfhe_export_secret(ctx: int) -> np.ndarray:
    info = sfhe_ctx_info(ctx)
    s = np.zeros(info.N, dtype=np.int8)
    _check(lib().sfhe_export_secret(ctx, _ptr(s)))
    return s


def sfhe_export_relin_key(ctx: int, out, stream=None) -> None:
    _check(lib().sfhe_export_relin_key(ctx, _ptr(out), _stream(stream)))


# ----------------------------------------------------------------- matmul ---
def _mats(ms) -> ctypes.Array:
    arr = (sfhe_matrix_view * len(ms))()
    for k, m in enumerate(ms):
        arr[k] = m
    return arr


def sfhe_matmul_workspace_size(ctx: int, A: list, B: list, flags: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_matmul_workspace_size(ctx, len(A), _mats(A), _mats(B), flags, ctypes.byref(b)))
    return b.value


def sfhe_matmul_workspace_bound(ctx: int, max_matmuls: int, max_entries: int, max_products: int, flags: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_matmul_workspace_bound(ctx, max_matmuls, max_entries, max_products, flags, ctypes.byref(b)))
    return b.value


def sfhe_matmul_dense_view(ctx: int, A, B, C, flags: int, work, stream=None) -> None:
    _check(lib().sfhe_matmul_dense_view(ctx, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), flags, _ptr(work),
                                   work.numel() * work.element_size(), _stream(stream)))


def sfhe_matmul_sparse_view(ctx: int, A, B, encoding: int, C, flags: int, work, stream=None) -> None:
    _check(lib().sfhe_matmul_sparse_view(ctx, ctypes.byref(A), ctypes.byref(B), encoding, ctypes.byref(C), flags,
                                    _ptr(work), work.numel() * work.element_size(), _stream(stream)))


def sfhe_matmul_batch_view(ctx: int, A: list, B: list, C: list, flags: int, work, stream=None) -> None:
    _check(lib().sfhe_matmul_batch_view(ctx, len(A), _mats(A), _mats(B), _mats(C), flags, _ptr(work),
                                   work.numel() * work.element_size(), _stream(stream)))


def sfhe_plan_create(ctx: int, A: list, B: list, C: list, flags: int, work, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_plan_create(ctx, len(A), _mats(A), _mats(B), _mats(C), flags, _ptr(work),
                                  work.numel() * work.element_size(), _stream(stream), ctypes.byref(h)))
    return h.value


def sfhe_plan_execute(plan: int, stream=None) -> None:
    _check(lib().sfhe_plan_execute(plan, _stream(stream)))


def sfhe_plan_set_stop(plan: int, word) -> None:
    """word: a device tensor whose first 4 bytes are the stop word, or None"""
    _check(lib().sfhe_plan_set_stop(plan, None if word is None else _ptr(word)))


def sfhe_plan_progress(plan: int, stream=None) -> int:
    done = _i64()
    _check(lib().sfhe_plan_progress(plan, ctypes.byref(done), _stream(stream)))
    return done.value


def sfhe_plan_resume(plan: int, stream=None) -> None:
    _check(lib().sfhe_plan_resume(plan, _stream(stream)))


# ------------------------------------------------ slot-packed chunks ---
def sfhe_slots_encode(N: int, t: int, values) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.int64))
    out = np.zeros(N, dtype=np.int64)
    _check(lib().sfhe_slots_encode(N, t, _ptr(v), _ptr(out)))
    return out


def sfhe_slots_decode(N: int, t: int, poly) -> np.ndarray:
    p = np.ascontiguousarray(np.asarray(poly, dtype=np.int64))
    out = np.zeros(N, dtype=np.int64)
    _check(lib().sfhe_slots_decode(N, t, _ptr(p), _ptr(out)))
    return out


def sfhe_rotation_element(N: int, k: int) -> int:
    return int(lib().sfhe_rotation_element(N, k))


def sfhe_encrypt_poly(ctx: int, polys: np.ndarray, coords: np.ndarray, matrix_id: int, ct, stream=None) -> None:
    polys = np.ascontiguousarray(polys, dtype=np.int64)
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    _check(lib().sfhe_encrypt_poly(ctx, _ptr(polys), _ptr(coords), polys.shape[0], matrix_id, _ptr(ct),
                                   _stream(stream)))


def sfhe_decrypt_poly(ctx: int, ct, n: int, out, stream=None) -> None:
    _check(lib().sfhe_decrypt_poly(ctx, _ptr(ct), n, _ptr(out), _stream(stream)))


def sfhe_galois_keygen(ctx: int, g: int, key, key_sh, stream=None) -> None:
    _check(lib().sfhe_galois_keygen(ctx, g, _ptr(key), _ptr(key_sh), _stream(stream)))


def sfhe_rotate_workspace_size(ctx: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_rotate_workspace_size(ctx, ctypes.byref(b)))
    return b.value


def sfhe_rotate(ctx: int, ct_in, n: int, g: int, key, key_sh, ct_out, work, stream=None) -> None:
    _check(lib().sfhe_rotate(ctx, _ptr(ct_in), n, g, _ptr(key), _ptr(key_sh), _ptr(ct_out), _ptr(work),
                             work.numel() * work.element_size(), _stream(stream)))


def sfhe_plain_ntt(ctx: int, poly, pt, stream=None) -> None:
    p = np.ascontiguousarray(np.asarray(poly, dtype=np.int64))
    _check(lib().sfhe_plain_ntt(ctx, _ptr(p), _ptr(pt), _stream(stream)))


def sfhe_mul_plain(ctx: int, ct, n: int, pt, stream=None) -> None:
    _check(lib().sfhe_mul_plain(ctx, _ptr(ct), n, _ptr(pt), _stream(stream)))


def sfhe_add(ctx: int, acc, x, n: int, stream=None) -> None:
    _check(lib().sfhe_add(ctx, _ptr(acc), _ptr(x), n, _stream(stream)))


def sfhe_rotkeys_create(ctx: int, c: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_rotkeys_create(ctx, c, _stream(stream), ctypes.byref(h)))
    return h.value


def sfhe_rotkeys_destroy(rk: int) -> None:
    lib().sfhe_rotkeys_destroy(rk)


def sfhe_matmul_chunked_workspace_size(ctx: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_matmul_chunked_workspace_size(ctx, ctypes.byref(b)))
    return b.value


def sfhe_matmul_chunked(ctx: int, rk: int, M: int, K: int, Nc: int, A, B, C, a_zero, b_zero, work,
                        stream=None) -> int:
    n = ctypes.c_int64()
    _check(lib().sfhe_matmul_chunked(ctx, rk, M, K, Nc, _ptr(A), _ptr(B), _ptr(C), _ptr(a_zero), _ptr(b_zero),
                                     _ptr(work), work.numel() * work.element_size(), _stream(stream),
                                     ctypes.byref(n)))
    return n.value


def sfhe_matmul_chunked_fused_workspace_size(ctx: int, c: int, M: int, K: int, Nc: int, a_zero, b_zero) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_matmul_chunked_fused_workspace_size(ctx, c, M, K, Nc, _ptr(a_zero), _ptr(b_zero),
                                                          ctypes.byref(b)))
    return b.value


def sfhe_matmul_chunked_fused(ctx: int, rk: int, M: int, K: int, Nc: int, A, B, C, a_zero, b_zero, work,
                              stream=None) -> int:
    n = ctypes.c_int64()
    _check(lib().sfhe_matmul_chunked_fused(ctx, rk, M, K, Nc, _ptr(A), _ptr(B), _ptr(C), _ptr(a_zero), _ptr(b_zero),
                                           _ptr(work), work.numel() * work.element_size(), _stream(stream),
                                           ctypes.byref(n)))
    return n.value


def sfhe_measure_mulmod32(ctx: int, stream=None) -> float:
    """32-bit Shoup modular multiplies per second over all SMs."""
    r = ctypes.c_double()
    _check(lib().sfhe_measure_mulmod32(ctx, ctypes.byref(r), _stream(stream)))
    return r.value


def sfhe_plan_stats(plan: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().sfhe_plan_stats(plan, *[ctypes.byref(x) for x in v]))
    return dict(zip(("products", "entries", "launches", "ctas"), (x.value for x in v)))


def sfhe_ctx_tuning(ctx: int) -> dict:
    """{"variant", "variants", "ms", "names"}: the tile in use (-1 before the
    first persistent plan), how many exist, their calibration times and
    descriptions."""
    v, n = ctypes.c_int32(), ctypes.c_int32()
    ms = np.zeros(8, dtype=np.float32)
    _check(lib().sfhe_ctx_tuning(ctx, ctypes.byref(v), ctypes.byref(n), _ptr(ms)))
    names = [lib().sfhe_ctx_variant_name(ctx, i).decode() for i in range(n.value)]
    return {"variant": v.value, "variants": n.value, "ms": [float(x) for x in ms[:n.value]], "names": names}


def sfhe_ctx_set_variant(ctx: int, variant: int) -> None:
    _check(lib().sfhe_ctx_set_variant(ctx, variant))


def sfhe_ctx_variant_name(ctx: int, variant: int) -> str:
    return lib().sfhe_ctx_variant_name(ctx, variant).decode()


def sfhe_matmul_check(work, stream=None) -> None:
    _check(lib().sfhe_matmul_check(_ptr(work), _stream(stream)))


def sfhe_selftest_wait_bound(work, tries: int, limit_us: int = 1_000_000, stream=None) -> None:
    _check(lib().sfhe_selftest_wait_bound(_ptr(work), tries, limit_us, _stream(stream)))


def sfhe_plan_destroy(plan: int) -> None:
    lib().sfhe_plan_destroy(plan)


# ------------------------------------------------------------ stage calls ---
def sfhe_ct_tensor_scale(ctx: int, a_ext, b_ext, d, work, stream=None) -> None:
    _check(lib().sfhe_ct_tensor_scale(ctx, _ptr(a_ext), _ptr(b_ext), _ptr(d), _ptr(work),
                                      work.numel() * work.element_size(), _stream(stream)))


def sfhe_ct_mul_relin(ctx: int, a_ext, b_ext, out, work, stream=None) -> None:
    _check(lib().sfhe_ct_mul_relin(ctx, _ptr(a_ext), _ptr(b_ext), _ptr(out), _ptr(work),
                                   work.numel() * work.element_size(), _stream(stream)))


def sfhe_ct_mul_relin_static(ctx: int, a_ext, b_ext, out, stream=None) -> None:
    _check(lib().sfhe_ct_mul_relin_static(ctx, _ptr(a_ext), _ptr(b_ext), _ptr(out), _stream(stream)))


def sfhe_ntt(ctx: int, prime_index: int, inverse: bool, inp, npoly: int, out, stream=None) -> None:
    _check(lib().sfhe_ntt(ctx, prime_index, int(inverse), _ptr(inp), npoly, _ptr(out), _stream(stream)))


def sfhe_prng_words(seed: int, domain: int, o0: int, o1: int, o2: int, idx0: int, n: int, out, stream=None) -> None:
    _check(lib().sfhe_prng_words(seed, domain, o0, o1, o2, idx0, n, _ptr(out), _stream(stream)))


# --------------------------------------- library-owned matrices (handles) ---
def sfhe_ctx_get_primes(ctx: int) -> tuple[list[int], list[int]]:
    """(ciphertext primes q, extended-base primes p)."""
    info = sfhe_ctx_info(ctx)
    q = np.zeros(max(info.L, 1), dtype=np.uint64)
    p = np.zeros(max(info.K, 1), dtype=np.uint64)
    _check(lib().sfhe_ctx_get_primes(ctx, _ptr(q), _ptr(p)))
    return [int(x) for x in q[:info.L]], [int(x) for x in p[:info.K]]


def sfhe_matrix_encrypt(ctx: int, vals: np.ndarray, encoding: int, matrix_id: int, stream=None) -> int:
    v = np.ascontiguousarray(vals, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib().sfhe_matrix_encrypt(ctx, _ptr(v), v.shape[0], v.shape[1], encoding, matrix_id, _stream(stream),
                                     ctypes.byref(h)))
    return h.value


def sfhe_matrix_import(ctx: int, coeff_limbs: np.ndarray, idx, rows: int, cols: int, encoding: int,
                       stream=None) -> int:
    c = np.ascontiguousarray(coeff_limbs, dtype=np.uint64)
    ix = None if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().sfhe_matrix_import(ctx, _ptr(c), _ptr(ix), rows, cols, encoding, _stream(stream), ctypes.byref(h)))
    return h.value


def sfhe_matrix_info(M: int) -> dict:
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().sfhe_matrix_info(M, *[ctypes.byref(x) for x in v]))
    return dict(zip(("rows", "cols", "encoding", "nct"), (x.value for x in v)))


def sfhe_matrix_export(M: int, out: np.ndarray, stream=None) -> np.ndarray:
    """out: host uint64 [nct][2][L][N], filled in coefficient form."""
    assert out.dtype == np.uint64 and out.flags["C_CONTIGUOUS"]
    _check(lib().sfhe_matrix_export(M, _ptr(out), _stream(stream)))
    return out


def sfhe_matrix_decrypt(ctx: int, M: int, stream=None) -> np.ndarray:
    info = sfhe_matrix_info(M)
    out = np.zeros((max(info["rows"], 1), max(info["cols"], 1)), dtype=np.int64)
    _check(lib().sfhe_matrix_decrypt(ctx, M, _ptr(out), _stream(stream)))
    return out[:info["rows"], :info["cols"]]


def sfhe_matrix_destroy(M: int) -> None:
    lib().sfhe_matrix_destroy(M)


def sfhe_matrix_view_of(M: int, stream=None) -> sfhe_matrix_view:
    v = sfhe_matrix_view()
    _check(lib().sfhe_matrix_view_of(M, ctypes.byref(v), _stream(stream)))
    return v


def sfhe_matmul_dense(ctx: int, A: int, B: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_matmul_dense(ctx, A, B, ctypes.byref(h), _stream(stream)))
    return h.value


def sfhe_matmul_sparse(ctx: int, A: int, B: int, encoding: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_matmul_sparse(ctx, A, B, encoding, ctypes.byref(h), _stream(stream)))
    return h.value


def sfhe_matmul_batch(ctx: int, A: list, B: list, flags: int, stream=None) -> list[int]:
    n = len(A)
    Aa = (ctypes.c_void_p * max(n, 1))(*A)
    Ba = (ctypes.c_void_p * max(n, 1))(*B)
    Ca = (ctypes.c_void_p * max(n, 1))()
    _check(lib().sfhe_matmul_batch(ctx, n, Aa, Ba, Ca, flags, _stream(stream)))
    return [Ca[m] for m in range(n)]


# ------------------------------------------------ host-resident operands ---
def sfhe_host_plan_create(ctx: int, A: list, B: list, flags: int, depth: int = 2) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_host_plan_create(ctx, len(A), _mats(A), _mats(B), flags, depth, ctypes.byref(h)))
    return h.value


def sfhe_matmul_host(hp: int, A_ct: list, B_ct: list, C_ct: list, stream=None) -> None:
    """A_ct, B_ct, C_ct: host buffers (numpy arrays or CPU torch tensors,
    preferably pinned) of each matmul's ciphertexts in NTT form."""
    def arr(xs):
        return (ctypes.c_void_p * max(len(xs), 1))(*[_ptr(x) for x in xs])
    _check(lib().sfhe_matmul_host(hp, arr(A_ct), arr(B_ct), arr(C_ct), _stream(stream)))


def sfhe_host_plan_stats(hp: int) -> dict:
    p, l = ctypes.c_int64(), ctypes.c_int64()
    u, d = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sfhe_host_plan_stats(hp, ctypes.byref(p), ctypes.byref(u), ctypes.byref(d), ctypes.byref(l)))
    return {"products": p.value, "h2d_bytes": u.value, "d2h_bytes": d.value, "launches": l.value}


def sfhe_host_plan_destroy(hp: int) -> None:
    lib().sfhe_host_plan_destroy(hp)


# ------------------------------------------------------------------- CKKS ---
def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def sfhe_ckks_ctx_create(N: int = 8192, bits=(50, 40, 40, 40), special_bits: int = 40, log_scale: int = 40,
                         sigma: float = 3.2, seed: int = 0) -> int:
    b = (ctypes.c_uint32 * 8)(*list(bits))
    h = ctypes.c_void_p()
    _check(lib().sfhe_ckks_ctx_create(ctypes.byref(sfhe_ckks_params(N, len(bits), b, special_bits, log_scale, sigma)),
                                      seed, ctypes.byref(h)))
    return h.value


def sfhe_ckks_ctx_destroy(ctx: int) -> None:
    lib().sfhe_ckks_ctx_destroy(ctx)


def sfhe_ckks_ctx_primes(ctx: int, L: int) -> tuple[list[int], int, float]:
    q = np.zeros(8, dtype=np.uint64)
    p, sc = ctypes.c_uint64(), ctypes.c_double()
    _check(lib().sfhe_ckks_ctx_primes(ctx, _ptr(q), ctypes.byref(p), ctypes.byref(sc)))
    return [int(x) for x in q[:L]], p.value, sc.value


def sfhe_ckks_encode(ctx: int, N: int, values, scale: float) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    out = np.zeros(N, dtype=np.int64)
    _check(lib().sfhe_ckks_encode(ctx, _ptr(v) if v.size else None, v.size, scale, _ptr(out)))
    return out


def sfhe_ckks_decode(ctx: int, coeff: np.ndarray, level: int, scale: float, n: int) -> np.ndarray:
    c = np.ascontiguousarray(coeff, dtype=np.uint64)
    out = np.zeros(max(n, 1), dtype=np.float64)
    _check(lib().sfhe_ckks_decode(ctx, _ptr(c), level, scale, n, _ptr(out)))
    return out[:n]


def sfhe_ckks_encrypt(ctx: int, polys: np.ndarray, coords: np.ndarray, matrix_id: int, ct, stream=None) -> None:
    p = np.ascontiguousarray(polys, dtype=np.int64)
    c = np.ascontiguousarray(coords, dtype=np.int32)
    _check(lib().sfhe_ckks_encrypt(ctx, _ptr(p), _ptr(c), p.shape[0], matrix_id, _ptr(ct), _stream(stream)))


def sfhe_ckks_decrypt(ctx: int, ct, level: int, n: int, scale: float, slots: int, stream=None) -> np.ndarray:
    out = np.zeros((max(n, 1), max(slots, 1)), dtype=np.float64)
    _check(lib().sfhe_ckks_decrypt(ctx, _ptr(ct), level, n, scale, slots, _ptr(out), _stream(stream)))
    return out[:n, :slots]


def sfhe_ckks_to_coeff(ctx: int, ct, level: int, n: int, out, stream=None) -> None:
    _check(lib().sfhe_ckks_to_coeff(ctx, _ptr(ct), level, n, _ptr(out), _stream(stream)))


def sfhe_ckks_workspace_size(ctx: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_ckks_workspace_size(ctx, ctypes.byref(b)))
    return b.value


def sfhe_ckks_mul_relin(ctx: int, a, b, level: int, out, work, stream=None) -> None:
    _check(lib().sfhe_ckks_mul_relin(ctx, _ptr(a), _ptr(b), level, _ptr(out), _ptr(work), _nbytes(work),
                                     _stream(stream)))


def sfhe_ckks_rescale(ctx: int, inp, level: int, n: int, out, work, stream=None) -> None:
    _check(lib().sfhe_ckks_rescale(ctx, _ptr(inp), level, n, _ptr(out), _ptr(work), _nbytes(work), _stream(stream)))


def sfhe_ckks_rotkeys_create(ctx: int, c: int, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfhe_ckks_rotkeys_create(ctx, c, _stream(stream), ctypes.byref(h)))
    return h.value


def sfhe_ckks_rotkeys_destroy(rk: int) -> None:
    lib().sfhe_ckks_rotkeys_destroy(rk)


def sfhe_ckks_rotate(ctx: int, rk: int, inp, level: int, k: int, out, work, stream=None) -> None:
    _check(lib().sfhe_ckks_rotate(ctx, rk, _ptr(inp), level, k, _ptr(out), _ptr(work), _nbytes(work),
                                  _stream(stream)))


def sfhe_ckks_plain_ntt(ctx: int, poly, level: int, pt, stream=None) -> None:
    p = np.ascontiguousarray(np.asarray(poly, dtype=np.int64))
    _check(lib().sfhe_ckks_plain_ntt(ctx, _ptr(p), level, _ptr(pt), _stream(stream)))


def sfhe_ckks_mul_plain(ctx: int, ct, level: int, n: int, pt, stream=None) -> None:
    _check(lib().sfhe_ckks_mul_plain(ctx, _ptr(ct), level, n, _ptr(pt), _stream(stream)))


def sfhe_ckks_add(ctx: int, acc, x, level: int, n: int, stream=None) -> None:
    _check(lib().sfhe_ckks_add(ctx, _ptr(acc), _ptr(x), level, n, _stream(stream)))


def sfhe_ckks_matmul_chunked_workspace_size(ctx: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().sfhe_ckks_matmul_chunked_workspace_size(ctx, ctypes.byref(b)))
    return b.value


def sfhe_ckks_matmul_chunked(ctx: int, rk: int, M: int, K: int, Nc: int, A, B, C, a_zero, b_zero, work,
                             stream=None) -> tuple[int, float]:
    n, sc = ctypes.c_int64(), ctypes.c_double()
    _check(lib().sfhe_ckks_matmul_chunked(ctx, rk, M, K, Nc, _ptr(A), _ptr(B), _ptr(C), _ptr(a_zero), _ptr(b_zero),
                                          _ptr(work), _nbytes(work), _stream(stream), ctypes.byref(n),
                                          ctypes.byref(sc)))
    return n.value, sc.value
