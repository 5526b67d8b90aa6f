// handles.cu -- library-owned matrices (sfhe_matrix) and matmuls over
// host-resident operands (sfhe_host_plan).  Both are layers over the
// descriptor calls of api.cu: they own device memory and streams, and every
// step of the arithmetic runs in the same kernels.
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sfhe.h"
#include "api_internal.h"

using sfhe::set_error;

namespace {

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

#define CUDA_OR_FAIL(expr)                                                                         \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return set_error(SFHE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

struct CtxDims {
    int N, L, K;
    uint64_t t;
    uint64_t q[8];
};

sfhe_status dims_of(const sfhe_ctx* c, CtxDims& d)
{
    sfhe_info info;
    sfhe_status st = sfhe_ctx_info(c, &info);
    if (st != SFHE_OK) return st;
    d.N = (int)info.N;
    d.L = (int)info.L;
    d.K = (int)info.K;
    d.t = info.t;
    for (int i = 0; i < 8; i++) d.q[i] = info.q[i];
    return SFHE_OK;
}

}  // namespace

// An encoded, encrypted matrix whose device memory the library owns.  The
// plaintext structure is kept on the host (the work-list builder reads it
// there); `ext` (the lift to the tensor base) is filled when the matrix is
// made from inputs, and on first use as an operand for a matmul result.
struct sfhe_matrix {
    sfhe_ctx* ctx;
    int32_t rows, cols, encoding, nct, ell_width;
    std::vector<uint8_t> mask;
    std::vector<int32_t> row_ptr, col_idx, ell_col;
    uint64_t* ct;   // [max(nct, 1)][2][L][N]
    uint32_t* ext;  // [max(nct, 1)][2][K][N]
    bool lifted;
    size_t ct_bytes, ext_bytes;

    sfhe_matrix_view view() const
    {
        sfhe_matrix_view v;
        memset(&v, 0, sizeof(v));
        v.rows = rows;
        v.cols = cols;
        v.encoding = encoding;
        v.nct = nct;
        v.ell_width = ell_width;
        v.mask = mask.empty() ? nullptr : mask.data();
        v.row_ptr = row_ptr.empty() ? nullptr : row_ptr.data();
        v.col_idx = col_idx.empty() ? nullptr : col_idx.data();
        v.ell_col = ell_col.empty() ? nullptr : ell_col.data();
        v.ct = ct;
        v.ext = ext;
        return v;
    }
};

namespace {

// a handle with its ciphertext storage allocated (not yet written)
sfhe_status new_matrix(sfhe_ctx* c, int32_t rows, int32_t cols, int32_t enc, int32_t nct, int32_t width,
                       sfhe_matrix** out)
{
    CtxDims d;
    sfhe_status st = dims_of(c, d);
    if (st != SFHE_OK) return st;
    sfhe_matrix* M = new sfhe_matrix();
    M->ctx = c;
    M->rows = rows;
    M->cols = cols;
    M->encoding = enc;
    M->nct = nct;
    M->ell_width = width;
    M->ct = nullptr;
    M->ext = nullptr;
    M->lifted = false;
    M->ct_bytes = (size_t)std::max(nct, 1) * 2 * d.L * d.N * 8;
    M->ext_bytes = (size_t)std::max(nct, 1) * 2 * d.K * d.N * 4;
    if (cudaMalloc((void**)&M->ct, M->ct_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete M;
        return set_error(SFHE_ENOMEM, "device allocation of %zu bytes for a matrix failed", (size_t)M->ct_bytes);
    }
    *out = M;
    return SFHE_OK;
}

// lift to the tensor base on `stream` unless done already (a cache: the
// ciphertexts themselves do not change)
sfhe_status ensure_lifted(sfhe_matrix* M, cudaStream_t s)
{
    if (M->lifted) return SFHE_OK;
    if (!M->ext && cudaMalloc((void**)&M->ext, M->ext_bytes) != cudaSuccess) {
        cudaGetLastError();
        M->ext = nullptr;
        return set_error(SFHE_ENOMEM, "device allocation of %zu bytes for a lifted matrix failed", M->ext_bytes);
    }
    if (M->nct > 0) {
        size_t wb = 0;
        sfhe_status st = sfhe_lift_workspace_size(M->ctx, M->nct, &wb);
        if (st != SFHE_OK) return st;
        void* w = nullptr;
        CUDA_OR_FAIL(cudaMallocAsync(&w, wb, s));
        st = sfhe_lift(M->ctx, M->ct, M->nct, M->ext, w, wb, s);
        cudaFreeAsync(w, s);
        if (st != SFHE_OK) return st;
    }
    M->lifted = true;
    return SFHE_OK;
}

sfhe_status check_encoding(int32_t enc)
{
    if (enc < SFHE_ENC_DENSE || enc > SFHE_ENC_ELL) return set_error(SFHE_EINVAL, "unknown encoding %d", enc);
    return SFHE_OK;
}

}  // namespace

// ------------------------------------------------------------- context ---
extern "C" sfhe_status sfhe_ctx_get_primes(const sfhe_ctx* c, uint64_t* q, uint64_t* p)
{
    if (!c || !q || !p) return set_error(SFHE_EINVAL, "null argument");
    sfhe_info info;
    sfhe_status st = sfhe_ctx_info(c, &info);
    if (st != SFHE_OK) return st;
    for (uint32_t i = 0; i < info.L; i++) q[i] = info.q[i];
    for (uint32_t k = 0; k < info.K; k++) p[k] = info.b[k];
    return SFHE_OK;
}

// ------------------------------------------------------------ matrices ---
extern "C" void sfhe_matrix_destroy(sfhe_matrix* M)
{
    if (!M) return;
    cudaFree(M->ct);
    cudaFree(M->ext);
    delete M;
}

extern "C" sfhe_status sfhe_matrix_encrypt(sfhe_ctx* c, const int64_t* vals, int32_t rows, int32_t cols,
                                           sfhe_encoding encoding, uint64_t matrix_id, void* stream, sfhe_matrix** out)
{
    if (!out) return set_error(SFHE_EINVAL, "null output");
    *out = nullptr;
    if (!c) return set_error(SFHE_EINVAL, "null context");
    sfhe_status st = check_encoding(encoding);
    if (st != SFHE_OK) return st;
    int32_t nct = 0, width = 0;
    st = sfhe_encode_count(vals, rows, cols, encoding, &nct, &width);
    if (st != SFHE_OK) return st;
    std::vector<int64_t> ct_values(std::max(nct, 1));
    std::vector<int32_t> ct_coords(2 * (size_t)std::max(nct, 1));
    sfhe_matrix* M = nullptr;
    st = new_matrix(c, rows, cols, encoding, nct, width, &M);
    if (st != SFHE_OK) return st;
    if (encoding == SFHE_ENC_MASK) M->mask.resize((size_t)rows * cols);
    if (encoding == SFHE_ENC_CSR) {
        M->row_ptr.resize((size_t)rows + 1);
        M->col_idx.resize(std::max(nct, 1));
    }
    if (encoding == SFHE_ENC_ELL) M->ell_col.resize(std::max(nct, 1));
    st = sfhe_encode_fill(vals, rows, cols, encoding, M->mask.empty() ? nullptr : M->mask.data(),
                          M->row_ptr.empty() ? nullptr : M->row_ptr.data(),
                          M->col_idx.empty() ? nullptr : M->col_idx.data(),
                          M->ell_col.empty() ? nullptr : M->ell_col.data(), ct_values.data(), ct_coords.data());
    if (st == SFHE_OK && nct > 0)
        st = sfhe_encrypt(c, ct_values.data(), ct_coords.data(), nct, matrix_id, M->ct, stream);
    if (st == SFHE_OK) st = ensure_lifted(M, as_stream(stream));
    if (st != SFHE_OK) {
        sfhe_matrix_destroy(M);
        return st;
    }
    *out = M;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_import(sfhe_ctx* c, const uint64_t* coeff_limbs, const int32_t* idx, int32_t rows,
                                          int32_t cols, sfhe_encoding encoding, void* stream, sfhe_matrix** out)
{
    if (!out) return set_error(SFHE_EINVAL, "null output");
    *out = nullptr;
    if (!c) return set_error(SFHE_EINVAL, "null context");
    sfhe_status st = check_encoding(encoding);
    if (st != SFHE_OK) return st;
    if (rows < 0 || cols < 0) return set_error(SFHE_ESHAPE, "negative shape");
    CtxDims d;
    st = dims_of(c, d);
    if (st != SFHE_OK) return st;
    // the structure, read out of `idx` into a descriptor, then checked
    const int64_t cells = (int64_t)rows * cols;
    std::vector<uint8_t> mask;
    std::vector<int32_t> row_ptr, col_idx, ell_col;
    int64_t nct = 0;
    int32_t width = 0;
    switch (encoding) {
    case SFHE_ENC_DENSE: nct = cells; break;
    case SFHE_ENC_MASK:
        if (!idx && cells > 0) return set_error(SFHE_EINVAL, "MASK needs idx[rows*cols]");
        mask.resize(cells);
        for (int64_t e = 0; e < cells; e++) mask[e] = idx[e] != 0;
        nct = cells;
        break;
    case SFHE_ENC_CSR:
        if (!idx) return set_error(SFHE_EINVAL, "CSR needs idx = row_ptr[rows+1], col_idx[nnz]");
        row_ptr.assign(idx, idx + rows + 1);
        nct = row_ptr[rows];
        if (nct < 0 || nct > cells) return set_error(SFHE_EINVAL, "row_ptr[rows] = %lld out of range", (long long)nct);
        col_idx.assign(idx + rows + 1, idx + rows + 1 + nct);
        break;
    case SFHE_ENC_ELL:
        if (!idx) return set_error(SFHE_EINVAL, "ELL needs idx = ell_width, ell_col[rows*ell_width]");
        width = idx[0];
        if (width < 0 || width > cols) return set_error(SFHE_EINVAL, "ell_width %d out of range", width);
        nct = (int64_t)rows * width;
        ell_col.assign(idx + 1, idx + 1 + nct);
        break;
    }
    if (nct > INT32_MAX) return set_error(SFHE_EUNSUPPORTED, "too many ciphertexts");
    sfhe_matrix_view v;
    memset(&v, 0, sizeof(v));
    v.rows = rows;
    v.cols = cols;
    v.encoding = encoding;
    v.nct = (int32_t)nct;
    v.ell_width = width;
    v.mask = mask.empty() ? nullptr : mask.data();
    v.row_ptr = row_ptr.empty() ? nullptr : row_ptr.data();
    v.col_idx = col_idx.empty() ? nullptr : col_idx.data();
    v.ell_col = ell_col.empty() ? nullptr : ell_col.data();
    st = sfhe::validate_view(v, "imported matrix");
    if (st != SFHE_OK) return st;
    if (nct > 0 && !coeff_limbs) return set_error(SFHE_EINVAL, "null ciphertexts");
    // canonical residues: limb i below q_i
    const size_t N = d.N, L = d.L;
    for (int64_t n = 0; n < nct; n++)
        for (size_t p = 0; p < 2; p++)
            for (size_t i = 0; i < L; i++) {
                const uint64_t* w = coeff_limbs + (((size_t)n * 2 + p) * L + i) * N;
                for (size_t e = 0; e < N; e++)
                    if (w[e] >= d.q[i])
                        return set_error(SFHE_EINVAL, "ciphertext %lld, polynomial %zu, limb %zu: residue >= q_%zu",
                                         (long long)n, p, i, i);
            }
    sfhe_matrix* M = nullptr;
    st = new_matrix(c, rows, cols, encoding, (int32_t)nct, width, &M);
    if (st != SFHE_OK) return st;
    M->mask = std::move(mask);
    M->row_ptr = std::move(row_ptr);
    M->col_idx = std::move(col_idx);
    M->ell_col = std::move(ell_col);
    cudaStream_t s = as_stream(stream);
    if (nct > 0) {
        const size_t bytes = (size_t)nct * 2 * L * N * 8;
        void* tmp = nullptr;
        cudaError_t e = cudaMallocAsync(&tmp, bytes, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, coeff_limbs, bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) st = sfhe_from_coeff(c, (const uint64_t*)tmp, 2 * nct, M->ct, stream);
        if (tmp) cudaFreeAsync(tmp, s);
        // the caller may reuse its host array once the call returns
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = set_error(SFHE_ECUDA, "import: %s", cudaGetErrorString(e));
    }
    if (st == SFHE_OK) st = ensure_lifted(M, s);
    if (st != SFHE_OK) {
        sfhe_matrix_destroy(M);
        return st;
    }
    *out = M;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_export(const sfhe_matrix* M, uint64_t* coeff_limbs, void* stream)
{
    if (!M || (!coeff_limbs && M->nct > 0)) return set_error(SFHE_EINVAL, "null argument");
    if (M->nct == 0) return SFHE_OK;
    cudaStream_t s = as_stream(stream);
    const size_t bytes = (size_t)M->nct * (M->ct_bytes / std::max(M->nct, 1));
    void* tmp = nullptr;
    CUDA_OR_FAIL(cudaMallocAsync(&tmp, bytes, s));
    sfhe_status st = sfhe_to_coeff(M->ctx, M->ct, 2 * (int64_t)M->nct, (uint64_t*)tmp, stream);
    cudaError_t e = st == SFHE_OK ? cudaMemcpyAsync(coeff_limbs, tmp, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st != SFHE_OK) return st;
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "export: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_decrypt(sfhe_ctx* c, const sfhe_matrix* M, int64_t* out, void* stream)
{
    if (!c || !M || !out) return set_error(SFHE_EINVAL, "null argument");
    if (M->ctx != c) return set_error(SFHE_EINVAL, "matrix of another context");
    const int64_t cells = (int64_t)M->rows * M->cols;
    std::fill(out, out + cells, 0);
    if (M->nct == 0) return SFHE_OK;
    cudaStream_t s = as_stream(stream);
    std::vector<int64_t> vals(M->nct);
    void* tmp = nullptr;
    CUDA_OR_FAIL(cudaMallocAsync(&tmp, (size_t)M->nct * 8, s));
    sfhe_status st = sfhe_decrypt(c, M->ct, M->nct, (int64_t*)tmp, stream);
    cudaError_t e = st == SFHE_OK ? cudaMemcpyAsync(vals.data(), tmp, (size_t)M->nct * 8, cudaMemcpyDeviceToHost, s)
                                  : cudaSuccess;
    cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st != SFHE_OK) return st;
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "decrypt: %s", cudaGetErrorString(e));
    // back to the matrix's positions: the t-th stored element of the encoding
    switch (M->encoding) {
    case SFHE_ENC_DENSE:
    case SFHE_ENC_MASK:
        std::copy(vals.begin(), vals.end(), out);
        break;
    case SFHE_ENC_CSR:
        for (int32_t r = 0; r < M->rows; r++)
            for (int32_t t = M->row_ptr[r]; t < M->row_ptr[r + 1]; t++) out[(int64_t)r * M->cols + M->col_idx[t]] = vals[t];
        break;
    case SFHE_ENC_ELL:
        for (int32_t r = 0; r < M->rows; r++)
            for (int32_t sl = 0; sl < M->ell_width; sl++) {
                const int64_t t = (int64_t)r * M->ell_width + sl;
                if (M->ell_col[t] >= 0) out[(int64_t)r * M->cols + M->ell_col[t]] = vals[t];
            }
        break;
    }
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_info(const sfhe_matrix* M, int32_t* rows, int32_t* cols, int32_t* encoding,
                                        int32_t* nct)
{
    if (!M) return set_error(SFHE_EINVAL, "null matrix");
    if (rows) *rows = M->rows;
    if (cols) *cols = M->cols;
    if (encoding) *encoding = M->encoding;
    if (nct) *nct = M->nct;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_view_of(sfhe_matrix* M, sfhe_matrix_view* out, void* stream)
{
    if (!M || !out) return set_error(SFHE_EINVAL, "null argument");
    sfhe_status st = ensure_lifted(M, as_stream(stream));
    if (st != SFHE_OK) return st;
    *out = M->view();
    return SFHE_OK;
}

// --------------------------------------------------------- matmuls ---
namespace {

// kind 0: dense loop, 1: sparse over `enc`, 2: batch under `flags`
sfhe_status matmul_handles(sfhe_ctx* c, int32_t n, const sfhe_matrix* const* A, const sfhe_matrix* const* B,
                           sfhe_matrix** C, int kind, int32_t enc, uint32_t flags, void* stream)
{
    if (!c || !C || (n > 0 && (!A || !B))) return set_error(SFHE_EINVAL, "null argument");
    if (n < 0) return set_error(SFHE_ESHAPE, "negative matmul count");
    for (int32_t m = 0; m < n; m++) C[m] = nullptr;
    cudaStream_t s = as_stream(stream);
    std::vector<sfhe_matrix_view> Av(n), Bv(n), Cv(n);
    for (int32_t m = 0; m < n; m++) {
        if (!A[m] || !B[m]) return set_error(SFHE_EINVAL, "null operand %d", m);
        if (A[m]->ctx != c || B[m]->ctx != c) return set_error(SFHE_EINVAL, "operand %d of another context", m);
        if (A[m]->cols != B[m]->rows)
            return set_error(SFHE_ESHAPE, "A is %dx%d, B is %dx%d", A[m]->rows, A[m]->cols, B[m]->rows, B[m]->cols);
    }
    // results of earlier matmuls are lifted on first use as operands
    for (int32_t m = 0; m < n; m++) {
        sfhe_status st = ensure_lifted(const_cast<sfhe_matrix*>(A[m]), s);
        if (st == SFHE_OK) st = ensure_lifted(const_cast<sfhe_matrix*>(B[m]), s);
        if (st != SFHE_OK) return st;
        Av[m] = A[m]->view();
        Bv[m] = B[m]->view();
    }
    const uint32_t f = kind == 2 ? flags : (uint32_t)SFHE_EXEC_PERSISTENT;
    size_t wb = 0;
    sfhe_status st = sfhe_matmul_workspace_size(c, n, Av.data(), Bv.data(), f & ~(uint32_t)SFHE_EXEC_GRAPH, &wb);
    if (st != SFHE_OK) return st;
    std::vector<sfhe_matrix*> made(n, nullptr);
    auto undo = [&](sfhe_status e) {
        for (sfhe_matrix* M : made) sfhe_matrix_destroy(M);
        return e;
    };
    for (int32_t m = 0; m < n; m++) {
        const int32_t rows = A[m]->rows, cols = B[m]->cols;
        st = new_matrix(c, rows, cols, SFHE_ENC_DENSE, rows * cols, 0, &made[m]);
        if (st != SFHE_OK) return undo(st);
        Cv[m] = made[m]->view();
    }
    void* work = nullptr;
    if (cudaMallocAsync(&work, std::max<size_t>(wb, 256), s) != cudaSuccess) {
        cudaGetLastError();
        return undo(set_error(SFHE_ENOMEM, "matmul workspace of %zu bytes", wb));
    }
    if (kind == 0)
        st = sfhe_matmul_dense_view(c, &Av[0], &Bv[0], &Cv[0], f, work, wb, stream);
    else if (kind == 1)
        st = sfhe_matmul_sparse_view(c, &Av[0], &Bv[0], enc, &Cv[0], f, work, wb, stream);
    else
        st = sfhe_matmul_batch_view(c, n, Av.data(), Bv.data(), Cv.data(), f & ~(uint32_t)SFHE_EXEC_GRAPH, work, wb,
                                    stream);
    cudaFreeAsync(work, s);
    if (st != SFHE_OK) return undo(st);
    for (int32_t m = 0; m < n; m++) C[m] = made[m];
    return SFHE_OK;
}

}  // namespace

extern "C" sfhe_status sfhe_matmul_dense(sfhe_ctx* c, const sfhe_matrix* A, const sfhe_matrix* B, sfhe_matrix** C,
                                         void* stream)
{
    if (!C) return set_error(SFHE_EINVAL, "null output");
    *C = nullptr;
    return matmul_handles(c, 1, &A, &B, C, 0, 0, 0, stream);
}

extern "C" sfhe_status sfhe_matmul_sparse(sfhe_ctx* c, const sfhe_matrix* A, const sfhe_matrix* B,
                                          sfhe_encoding encoding, sfhe_matrix** C, void* stream)
{
    if (!C) return set_error(SFHE_EINVAL, "null output");
    *C = nullptr;
    return matmul_handles(c, 1, &A, &B, C, 1, encoding, 0, stream);
}

extern "C" sfhe_status sfhe_matmul_batch(sfhe_ctx* c, int32_t n, const sfhe_matrix* const* A,
                                         const sfhe_matrix* const* B, sfhe_matrix** C, uint32_t flags, void* stream)
{
    return matmul_handles(c, n, A, B, C, 2, 0, flags, stream);
}

// ------------------------------------------------ host-resident operands ---
struct sfhe_host_plan {
    sfhe_ctx* ctx;
    int32_t n, depth;
    uint32_t flags;
    // the structure, copied out of the caller's descriptors
    std::vector<sfhe_matrix_view> A, B;
    std::vector<std::vector<uint8_t>> masks;
    std::vector<std::vector<int32_t>> ints;
    std::vector<size_t> a_bytes, b_bytes, c_bytes;  // ciphertext bytes per matmul
    struct Set {
        std::vector<void*> bufs;  // every device allocation of the set
        std::vector<sfhe_matrix_view> A, B, C;
        void* lift_ws = nullptr;
        size_t lift_bytes = 0;
        void* work = nullptr;
        sfhe_plan* plan = nullptr;
        cudaEvent_t up_done = nullptr, comp_done = nullptr, down_done = nullptr;
    };
    std::vector<Set> sets;
    cudaStream_t s_up = nullptr, s_comp = nullptr, s_down = nullptr;
    int64_t calls = 0, products = 0, launches = 0;
    uint64_t h2d = 0, d2h = 0;
};

extern "C" void sfhe_host_plan_destroy(sfhe_host_plan* hp)
{
    if (!hp) return;
    for (cudaStream_t s : {hp->s_up, hp->s_comp, hp->s_down})
        if (s) cudaStreamSynchronize(s);
    for (auto& S : hp->sets) {
        if (S.plan) sfhe_plan_destroy(S.plan);
        for (void* p : S.bufs) cudaFree(p);
        for (cudaEvent_t e : {S.up_done, S.comp_done, S.down_done})
            if (e) cudaEventDestroy(e);
    }
    for (cudaStream_t s : {hp->s_up, hp->s_comp, hp->s_down})
        if (s) cudaStreamDestroy(s);
    delete hp;
}

extern "C" sfhe_status sfhe_host_plan_create(sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A,
                                             const sfhe_matrix_view* B, uint32_t flags, int32_t depth,
                                             sfhe_host_plan** out)
{
    if (!out) return set_error(SFHE_EINVAL, "null output");
    *out = nullptr;
    if (!c || (n > 0 && (!A || !B))) return set_error(SFHE_EINVAL, "null argument");
    if (n < 1) return set_error(SFHE_ESHAPE, "at least one matmul");
    if (depth < 1 || depth > 2) return set_error(SFHE_EINVAL, "depth must be 1 or 2");
    if (flags & SFHE_EXEC_GRAPH) return set_error(SFHE_EINVAL, "GRAPH is for caller-built plans");
    CtxDims d;
    sfhe_status st = dims_of(c, d);
    if (st != SFHE_OK) return st;
    sfhe_host_plan* hp = new sfhe_host_plan();
    hp->ctx = c;
    hp->n = n;
    hp->depth = depth;
    hp->flags = flags;
    auto bail = [&](sfhe_status e) {
        sfhe_host_plan_destroy(hp);
        return e;
    };
    // copy the structure (validated by the plan build below)
    auto keep = [&](const sfhe_matrix_view& v) {
        sfhe_matrix_view k = v;
        k.ct = nullptr;
        k.ext = nullptr;
        const int64_t cells = (int64_t)v.rows * v.cols;
        if (v.mask && cells > 0) {
            hp->masks.emplace_back(v.mask, v.mask + cells);
            k.mask = hp->masks.back().data();
        }
        if (v.row_ptr && v.rows >= 0) {
            hp->ints.emplace_back(v.row_ptr, v.row_ptr + v.rows + 1);
            k.row_ptr = hp->ints.back().data();
        }
        if (v.col_idx && v.nct > 0) {
            hp->ints.emplace_back(v.col_idx, v.col_idx + v.nct);
            k.col_idx = hp->ints.back().data();
        }
        if (v.ell_col && v.nct > 0) {
            hp->ints.emplace_back(v.ell_col, v.ell_col + v.nct);
            k.ell_col = hp->ints.back().data();
        }
        return k;
    };
    hp->masks.reserve(2 * (size_t)n);
    hp->ints.reserve(6 * (size_t)n);
    for (int32_t m = 0; m < n; m++) {
        st = sfhe::validate_view(A[m], "A");
        if (st == SFHE_OK) st = sfhe::validate_view(B[m], "B");
        if (st != SFHE_OK) return bail(st);
        hp->A.push_back(keep(A[m]));
        hp->B.push_back(keep(B[m]));
    }
    const size_t ctb = (size_t)2 * d.L * d.N * 8, extb = (size_t)2 * d.K * d.N * 4;
    for (int32_t m = 0; m < n; m++) {
        hp->a_bytes.push_back((size_t)hp->A[m].nct * ctb);
        hp->b_bytes.push_back((size_t)hp->B[m].nct * ctb);
        hp->c_bytes.push_back((size_t)hp->A[m].rows * hp->B[m].cols * ctb);
        hp->h2d += hp->a_bytes[m] + hp->b_bytes[m];
        hp->d2h += hp->c_bytes[m];
    }
    if (cudaStreamCreateWithFlags(&hp->s_up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp->s_comp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp->s_down, cudaStreamNonBlocking) != cudaSuccess)
        return bail(set_error(SFHE_ECUDA, "stream or event creation failed"));
    hp->sets.resize(depth);
    for (auto& S : hp->sets) {
        auto alloc = [&](size_t bytes) -> void* {
            void* p = nullptr;
            if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            S.bufs.push_back(p);
            return p;
        };
        int32_t nmax = 1;
        for (int32_t m = 0; m < n; m++) {
            sfhe_matrix_view a = hp->A[m], b = hp->B[m], cv;
            a.ct = (uint64_t*)alloc(hp->a_bytes[m]);
            a.ext = (uint32_t*)alloc((size_t)a.nct * extb);
            b.ct = (uint64_t*)alloc(hp->b_bytes[m]);
            b.ext = (uint32_t*)alloc((size_t)b.nct * extb);
            memset(&cv, 0, sizeof(cv));
            cv.rows = a.rows;
            cv.cols = b.cols;
            cv.encoding = SFHE_ENC_DENSE;
            cv.nct = a.rows * b.cols;
            cv.ct = (uint64_t*)alloc(hp->c_bytes[m]);
            if (!a.ct || !a.ext || !b.ct || !b.ext || !cv.ct)
                return bail(set_error(SFHE_ENOMEM, "device buffers of a host plan"));
            S.A.push_back(a);
            S.B.push_back(b);
            S.C.push_back(cv);
            nmax = std::max(nmax, std::max(a.nct, b.nct));
        }
        st = sfhe_lift_workspace_size(c, nmax, &S.lift_bytes);
        if (st != SFHE_OK) return bail(st);
        size_t wb = 0;
        st = sfhe_matmul_workspace_size(c, n, S.A.data(), S.B.data(), flags, &wb);
        if (st != SFHE_OK) return bail(st);
        S.lift_ws = alloc(S.lift_bytes);
        S.work = alloc(wb);
        if (!S.lift_ws || !S.work) return bail(set_error(SFHE_ENOMEM, "workspaces of a host plan"));
        st = sfhe_plan_create(c, n, S.A.data(), S.B.data(), S.C.data(), flags, S.work, std::max<size_t>(wb, 256),
                              hp->s_comp, &S.plan);
        if (st != SFHE_OK) return bail(st);
        if (cudaEventCreateWithFlags(&S.up_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S.comp_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S.down_done, cudaEventDisableTiming) != cudaSuccess)
            return bail(set_error(SFHE_ECUDA, "event creation failed"));
    }
    int64_t plan_launches = 0;
    st = sfhe_plan_stats(hp->sets[0].plan, &hp->products, nullptr, &plan_launches, nullptr);
    if (st != SFHE_OK) return bail(st);
    // three kernels per lift chunk of 256 ciphertexts
    int64_t lifts = 0;
    for (int32_t m = 0; m < n; m++) lifts += 3 * (((int64_t)hp->A[m].nct + 255) / 256 + ((int64_t)hp->B[m].nct + 255) / 256);
    hp->launches = plan_launches + lifts;
    if (cudaStreamSynchronize(hp->s_comp) != cudaSuccess) return bail(set_error(SFHE_ECUDA, "plan upload failed"));
    *out = hp;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_host(sfhe_host_plan* hp, const uint64_t* const* A_ct, const uint64_t* const* B_ct,
                                        uint64_t* const* C_ct, void* stream)
{
    if (!hp || !A_ct || !B_ct || !C_ct) return set_error(SFHE_EINVAL, "null argument");
    for (int32_t m = 0; m < hp->n; m++)
        if ((!A_ct[m] && hp->a_bytes[m]) || (!B_ct[m] && hp->b_bytes[m]) || (!C_ct[m] && hp->c_bytes[m]))
            return set_error(SFHE_EINVAL, "null host buffer of matmul %d", m);
    cudaStream_t s = as_stream(stream);
    auto& S = hp->sets[hp->calls % hp->depth];
    const bool reuse = hp->calls >= hp->depth;
    // uploads: once the set's previous inputs have been consumed (its lift
    // ran before its matmul finished).  They do not wait for `stream`: that
    // stream waits for the previous call's download, and waiting on it
    // would serialise every upload behind the previous call's whole matmul.
    if (reuse) CUDA_OR_FAIL(cudaStreamWaitEvent(hp->s_up, S.comp_done, 0));
    for (int32_t m = 0; m < hp->n; m++) {
        if (hp->a_bytes[m])
            CUDA_OR_FAIL(cudaMemcpyAsync(S.A[m].ct, A_ct[m], hp->a_bytes[m], cudaMemcpyHostToDevice, hp->s_up));
        if (hp->b_bytes[m])
            CUDA_OR_FAIL(cudaMemcpyAsync(S.B[m].ct, B_ct[m], hp->b_bytes[m], cudaMemcpyHostToDevice, hp->s_up));
    }
    CUDA_OR_FAIL(cudaEventRecord(S.up_done, hp->s_up));
    // compute: once the uploads landed and the set's previous C was read out
    CUDA_OR_FAIL(cudaStreamWaitEvent(hp->s_comp, S.up_done, 0));
    if (reuse) CUDA_OR_FAIL(cudaStreamWaitEvent(hp->s_comp, S.down_done, 0));
    for (int32_t m = 0; m < hp->n; m++) {
        sfhe_status st = sfhe_lift(hp->ctx, S.A[m].ct, S.A[m].nct, S.A[m].ext, S.lift_ws, S.lift_bytes, hp->s_comp);
        if (st == SFHE_OK)
            st = sfhe_lift(hp->ctx, S.B[m].ct, S.B[m].nct, S.B[m].ext, S.lift_ws, S.lift_bytes, hp->s_comp);
        if (st != SFHE_OK) return st;
    }
    sfhe_status st = sfhe_plan_execute(S.plan, hp->s_comp);
    if (st != SFHE_OK) return st;
    CUDA_OR_FAIL(cudaEventRecord(S.comp_done, hp->s_comp));
    // download, then the caller's stream waits for it
    CUDA_OR_FAIL(cudaStreamWaitEvent(hp->s_down, S.comp_done, 0));
    for (int32_t m = 0; m < hp->n; m++)
        if (hp->c_bytes[m])
            CUDA_OR_FAIL(cudaMemcpyAsync(C_ct[m], S.C[m].ct, hp->c_bytes[m], cudaMemcpyDeviceToHost, hp->s_down));
    CUDA_OR_FAIL(cudaEventRecord(S.down_done, hp->s_down));
    CUDA_OR_FAIL(cudaStreamWaitEvent(s, S.down_done, 0));
    hp->calls++;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_host_plan_stats(const sfhe_host_plan* hp, int64_t* products, uint64_t* h2d_bytes,
                                            uint64_t* d2h_bytes, int64_t* launches)
{
    if (!hp) return set_error(SFHE_EINVAL, "null plan");
    if (products) *products = hp->products;
    if (h2d_bytes) *h2d_bytes = hp->h2d;
    if (d2h_bytes) *d2h_bytes = hp->d2h;
    if (launches) *launches = hp->launches;
    return SFHE_OK;
}
