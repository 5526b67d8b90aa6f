// api.cu -- the C ABI (include/sfhe.h): contexts, operands, matmul plans.
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sfhe.h"
#include "api_internal.h"
#include "host_math.h"
#include "launch.h"
#include "chunk_launch.h"

using namespace sfhe;

namespace {

// an NVTX range over one entry point (visible to profilers; free otherwise)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

thread_local std::string g_last_error;

sfhe_status fail(sfhe_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return fail(SFHE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Scratch of sfhe_ct_mul_relin_static: a file-scope device array, so that the
// call needs no workspace from its caller and allocates nothing.  Its callers
// are those that cannot hand over device memory: a plain C caller with no
// device allocator of its own, code that runs while a stream is being
// captured (where cudaMalloc is not allowed), and a serving loop that must
// not enter an allocator between requests.  One copy exists per device; its
// address is looked up once per device, on the first call made there, and
// forgotten when a context of that device is destroyed (a device reset
// between contexts would move the array), so the next first call looks it up
// again.
namespace {
__device__ __align__(256) unsigned char g_static_scratch[SFHE_STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void* g_static_addr[64];  // per device ordinal; null until the first call there

void forget_static_scratch(int dev)
{
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(g_static_mu);
    g_static_addr[dev] = nullptr;
}
}  // namespace

struct sfhe_ctx {
    sfhe_params params;
    uint64_t seed;
    int device;
    int num_sms;
    RnsConsts rc;
    u64* d_tw;
    u32* d_twb;
    u64* d_s;
    signed char* d_s_coeff;
    u64* d_rlk;     // the key, followed in the same allocation by
    u64* d_rlk_sh;  // its Shoup companions
    int* d_err;
    // persisting-L2 window over the key and companions (bytes 0: none)
    size_t l2_bytes;
    float l2_hit;
    // tile tuning of the per-product persistent kernel
    std::mutex tune_mu;
    int n_variants;
    int forced_variant;  // -1: tuned on the first persistent plan
    int tuned_variant;   // -1 until tuned
    float variant_ms[8];
};

struct sfhe_plan {
    sfhe_ctx* ctx;
    uint32_t flags;
    std::vector<MmDesc> mms;
    std::vector<Entry> entries;
    std::vector<int2> rowlist;
    std::vector<size_t> c_words;  // per matmul: words of C
    int64_t products;
    // device regions inside the caller's workspace
    unsigned* d_queue;
    MmDesc* d_mms;
    Entry* d_entries;
    int2* d_rowlist;
    u64* d_scratch;
    size_t scratch_stride;
    int grid;
    u32* d_T;
    u64 *d_D, *d_U;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    int variant;  // tile variant of the persistent kernel
    const unsigned* d_stop;  // preemption word of the persistent launches (nullable)
    bool launched;           // an execution has set the entry counter
};

extern "C" const char* sfhe_last_error(void) { return g_last_error.c_str(); }

sfhe_status sfhe::set_error(sfhe_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

int sfhe::ctx_device(const sfhe_ctx* c) { return c->device; }

// ---------------------------------------------------------------- helpers ---
extern "C" sfhe_status sfhe_select_primes(uint32_t N, uint32_t L, uint64_t* q, uint32_t* b, int32_t* K)
{
    if (!q || !b || !K) return fail(SFHE_EINVAL, "null output");
    int logN = 0;
    while ((1u << logN) < N) logN++;
    if ((1u << logN) != N || logN < 1 || logN > 15 || L < 1 || L > SFHE_MAX_L)
        return fail(SFHE_EUNSUPPORTED, "N=%u L=%u", N, L);
    *K = tensor_base_size(logN, (int)L);
    if (*K > SFHE_MAX_K) return fail(SFHE_EUNSUPPORTED, "tensor base larger than %d primes", SFHE_MAX_K);
    std::vector<uint64_t> pq, pb;
    if (!ntt_primes(N, (int)L, pq, 54) || !ntt_primes(N, *K, pb, 30)) return fail(SFHE_EUNSUPPORTED, "not enough primes");
    for (uint32_t i = 0; i < L; i++) q[i] = pq[i];
    for (int k = 0; k < *K; k++) b[k] = (uint32_t)pb[k];
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_cdt_table(double sigma, uint64_t* T20)
{
    if (!T20) return fail(SFHE_EINVAL, "null output");
    if (!(sigma > 0.0)) return fail(SFHE_EINVAL, "sigma must be positive");
    cdt_table(sigma, T20);
    return SFHE_OK;
}

// ---------------------------------------------------------------- context ---
// Stage R reads the whole key once per output entry.  A persisting
// access-policy window over the key and its companions keeps them in L2
// between entries while the per-product scratch streams through: the
// context raises its persisting-L2 limit (a limit of this process's
// context, released with it) to the key's size or the device's maximum,
// and every persistent launch carries the window.  SFHE_L2_PERSIST=0 in the
// environment leaves both alone.
static void setup_l2_window(sfhe_ctx* c, size_t key_bytes)
{
    c->l2_bytes = 0;
    c->l2_hit = 0.f;
    const char* env = getenv("SFHE_L2_PERSIST");
    if (env && env[0] == '0') return;
    int max_persist = 0, max_window = 0;
    if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, c->device) != cudaSuccess ||
        max_persist <= 0 || max_window <= 0) {
        cudaGetLastError();
        return;
    }
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    const size_t want = std::min(key_bytes, (size_t)max_persist);
    if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    c->l2_bytes = std::min(key_bytes, (size_t)max_window);
    c->l2_hit = (float)std::min(1.0, (double)cur / (double)c->l2_bytes);
}

extern "C" void sfhe_ctx_destroy(sfhe_ctx* c)
{
    if (!c) return;
    forget_static_scratch(c->device);
    cudaFree(c->d_tw);
    cudaFree(c->d_twb);
    cudaFree(c->d_s);
    cudaFree(c->d_s_coeff);
    cudaFree(c->d_rlk);  // the companions share the allocation
    cudaFree(c->d_err);
    delete c;
}

extern "C" sfhe_status sfhe_ctx_create(const sfhe_params* params, uint64_t seed, sfhe_ctx** out)
{
    if (!params || !out) return fail(SFHE_EINVAL, "null argument");
    *out = nullptr;
    const uint32_t N = params->N, L = params->L;
    int logN = 0;
    while ((1u << logN) < N) logN++;
    if ((1u << logN) != N || !supported_ring(logN, (int)L))
        return fail(SFHE_EUNSUPPORTED, "ring N=%u L=%u not implemented (N in {4096, 8192, 16384}, L in {2,3,4,8})", N, L);
    if (params->t < 2 || params->t >= (1ULL << 32)) return fail(SFHE_EUNSUPPORTED, "t out of range");
    if (!(params->sigma > 0.0) || params->sigma > 8.0) return fail(SFHE_EUNSUPPORTED, "sigma out of range");

    sfhe_ctx* c = new sfhe_ctx();
    memset(&c->rc, 0, sizeof(c->rc));
    c->params = *params;
    c->seed = seed;
    auto bail = [&](sfhe_status st) {
        sfhe_ctx_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(SFHE_ECUDA, "no CUDA device"));
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);

    RnsConsts& rc = c->rc;
    rc.N = (int)N;
    rc.logN = logN;
    rc.L = (int)L;
    rc.K = tensor_base_size(logN, (int)L);
    rc.t = params->t;
    rc.seed = seed;
    std::vector<uint64_t> pq, pb;
    if (!ntt_primes(N, rc.L, pq, 54) || !ntt_primes(N, rc.K, pb, 30))
        return bail(fail(SFHE_EUNSUPPORTED, "not enough primes"));
    for (int i = 0; i < rc.L; i++) rc.m[i].q = pq[i];
    for (int k = 0; k < rc.K; k++) rc.mb[k].b = (u32)pb[k];
    if (!fill_constants(rc)) return bail(fail(SFHE_EUNSUPPORTED, "tensor base too small for these parameters"));
    cdt_table(params->sigma, rc.cdt);

    std::vector<uint64_t> tw((size_t)rc.L * 4 * N);
    for (int i = 0; i < rc.L; i++) twiddles(rc.m[i].q, N, tw.data() + (size_t)i * 4 * N, &rc.ninv[i], &rc.wlast[i]);
    std::vector<uint32_t> twb((size_t)rc.K * 4 * N);
    for (int k = 0; k < rc.K; k++)
        twiddles32(rc.mb[k].b, N, twb.data() + (size_t)k * 4 * N, &rc.ninv_b[k], &rc.wlast_b[k]);
    fold_tensor_scaling(rc);

    const size_t rlk_words = (size_t)L * 2 * L * N;
    if (cudaMalloc(&c->d_tw, tw.size() * 8) != cudaSuccess || cudaMalloc(&c->d_twb, twb.size() * 4) != cudaSuccess ||
        cudaMalloc(&c->d_s, (size_t)L * N * 8) != cudaSuccess ||
        cudaMalloc(&c->d_s_coeff, N) != cudaSuccess || cudaMalloc(&c->d_rlk, 2 * rlk_words * 8) != cudaSuccess ||
        cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess)
        return bail(fail(SFHE_ENOMEM, "device allocation of the context failed"));
    c->d_rlk_sh = c->d_rlk + rlk_words;
    rc.tw = c->d_tw;
    rc.twb = c->d_twb;
    if (cudaMemcpy(c->d_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_twb, twb.data(), twb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)
        return bail(fail(SFHE_ECUDA, "table upload failed"));
    cudaError_t e = launch_keygen(rc, c->d_s, c->d_s_coeff, c->d_rlk, c->d_rlk_sh, c->d_err, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(fail(SFHE_ECUDA, "key generation: %s", cudaGetErrorString(e)));
    int err = 0;
    cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return bail(fail(SFHE_EDEVICE, "key generation sampler failed"));
    setup_l2_window(c, 2 * rlk_words * 8);
    c->n_variants = persistent_variants(c->rc);
    c->forced_variant = -1;
    c->tuned_variant = -1;
    *out = c;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ctx_info(const sfhe_ctx* c, sfhe_info* out)
{
    if (!c || !out) return fail(SFHE_EINVAL, "null argument");
    memset(out, 0, sizeof(*out));
    out->N = (uint32_t)c->rc.N;
    out->L = (uint32_t)c->rc.L;
    out->K = (uint32_t)c->rc.K;
    out->t = c->rc.t;
    for (int i = 0; i < c->rc.L; i++) out->q[i] = c->rc.m[i].q;
    for (int k = 0; k < c->rc.K; k++) out->b[k] = c->rc.mb[k].b;
    out->ct_words = (uint64_t)2 * c->rc.L * c->rc.N;
    out->ext_words = (uint64_t)2 * c->rc.K * c->rc.N;
    out->num_sms = c->num_sms;
    out->ext_interleave = (uint32_t)ext_interleave(c->rc.logN);
    out->lazy_group = c->rc.lazy_group;
    out->l2_window = c->l2_bytes;
    out->l2_hit_ratio = c->l2_hit;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ctx_check(sfhe_ctx* c, void* stream)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return fail(SFHE_EDEVICE, "a sampler exhausted its retries");
    return SFHE_OK;
}

// --------------------------------------------------------------- operands ---
static sfhe_status check_values(const int64_t* v, int32_t rows, int32_t cols, int32_t enc)
{
    if (!v && rows > 0 && cols > 0) return fail(SFHE_EINVAL, "null values");
    if (rows < 0 || cols < 0) return fail(SFHE_ESHAPE, "negative shape");
    if (enc < SFHE_ENC_DENSE || enc > SFHE_ENC_ELL) return fail(SFHE_EINVAL, "unknown encoding %d", enc);
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_encode_count(const int64_t* values, int32_t rows, int32_t cols, int32_t encoding,
                                         int32_t* nct, int32_t* ell_width)
{
    sfhe_status st = check_values(values, rows, cols, encoding);
    if (st != SFHE_OK) return st;
    if (!nct || !ell_width) return fail(SFHE_EINVAL, "null output");
    int64_t nnz = 0;
    int32_t width = 0;
    for (int32_t r = 0; r < rows; r++) {
        int32_t row_nnz = 0;
        for (int32_t c = 0; c < cols; c++) row_nnz += values[(int64_t)r * cols + c] != 0;
        nnz += row_nnz;
        width = std::max(width, row_nnz);
    }
    int64_t n = (int64_t)rows * cols;
    if (encoding == SFHE_ENC_CSR) n = nnz;
    if (encoding == SFHE_ENC_ELL) n = (int64_t)rows * width;
    if (n > INT32_MAX) return fail(SFHE_EUNSUPPORTED, "too many ciphertexts");
    *nct = (int32_t)n;
    *ell_width = encoding == SFHE_ENC_ELL ? width : 0;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matrix_bytes(uint32_t N, uint32_t L, const sfhe_matrix_view* M, uint64_t* ct_bytes,
                                         uint64_t* ext_bytes, uint64_t* meta_bytes)
{
    if (!M || !ct_bytes || !ext_bytes || !meta_bytes) return fail(SFHE_EINVAL, "null argument");
    int logN = 0;
    while ((1u << logN) < N) logN++;
    if ((1u << logN) != N || logN < 1 || logN > 15 || L < 1 || L > SFHE_MAX_L)
        return fail(SFHE_EUNSUPPORTED, "N=%u L=%u", N, L);
    if (M->rows < 0 || M->cols < 0 || M->nct < 0 || M->ell_width < 0) return fail(SFHE_ESHAPE, "negative size");
    const uint64_t K = (uint64_t)tensor_base_size(logN, (int)L);
    const uint64_t nct = (uint64_t)M->nct, cells = (uint64_t)M->rows * (uint64_t)M->cols;
    *ct_bytes = nct * 2 * L * N * 8;
    *ext_bytes = nct * 2 * K * N * 4;
    switch (M->encoding) {
    case SFHE_ENC_DENSE: *meta_bytes = 0; break;
    case SFHE_ENC_MASK: *meta_bytes = cells; break;
    case SFHE_ENC_CSR: *meta_bytes = ((uint64_t)M->rows + 1 + nct) * 4; break;
    case SFHE_ENC_ELL: *meta_bytes = (uint64_t)M->rows * (uint64_t)M->ell_width * 4; break;
    default: return fail(SFHE_EINVAL, "bad encoding");
    }
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_encode_fill(const int64_t* values, int32_t rows, int32_t cols, int32_t encoding,
                                        uint8_t* mask, int32_t* row_ptr, int32_t* col_idx, int32_t* ell_col,
                                        int64_t* ct_values, int32_t* ct_coords)
{
    int32_t nct = 0, width = 0;
    sfhe_status st = sfhe_encode_count(values, rows, cols, encoding, &nct, &width);
    if (st != SFHE_OK) return st;
    if (!ct_values || !ct_coords) return fail(SFHE_EINVAL, "null output");
    int64_t t = 0;
    switch (encoding) {
    case SFHE_ENC_DENSE:
    case SFHE_ENC_MASK:
        if (encoding == SFHE_ENC_MASK && !mask) return fail(SFHE_EINVAL, "null mask");
        for (int32_t r = 0; r < rows; r++)
            for (int32_t c = 0; c < cols; c++, t++) {
                const int64_t v = values[(int64_t)r * cols + c];
                if (encoding == SFHE_ENC_MASK) mask[t] = v == 0;
                ct_values[t] = v;
                ct_coords[2 * t] = r;
                ct_coords[2 * t + 1] = c;
            }
        break;
    case SFHE_ENC_CSR:
        if (!row_ptr || (!col_idx && nct > 0)) return fail(SFHE_EINVAL, "null CSR arrays");
        row_ptr[0] = 0;
        for (int32_t r = 0; r < rows; r++) {
            for (int32_t c = 0; c < cols; c++) {
                const int64_t v = values[(int64_t)r * cols + c];
                if (!v) continue;
                col_idx[t] = c;
                ct_values[t] = v;
                ct_coords[2 * t] = r;
                ct_coords[2 * t + 1] = c;
                t++;
            }
            row_ptr[r + 1] = (int32_t)t;
        }
        break;
    case SFHE_ENC_ELL:
        if (!ell_col && nct > 0) return fail(SFHE_EINVAL, "null ELL column array");
        for (int32_t r = 0; r < rows; r++) {
            int32_t s = 0;
            for (int32_t c = 0; c < cols; c++) {
                const int64_t v = values[(int64_t)r * cols + c];
                if (!v) continue;
                t = (int64_t)r * width + s;
                ell_col[t] = c;
                ct_values[t] = v;
                ct_coords[2 * t] = r;
                ct_coords[2 * t + 1] = c;
                s++;
            }
            for (; s < width; s++) {  // encrypted zero padding
                t = (int64_t)r * width + s;
                ell_col[t] = -1;
                ct_values[t] = 0;
                ct_coords[2 * t] = r;
                ct_coords[2 * t + 1] = cols + s;
            }
        }
        break;
    }
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_encrypt(sfhe_ctx* c, const int64_t* values, const int32_t* coords, int64_t n,
                                    uint64_t matrix_id, uint64_t* ct, void* stream)
{
    Range range("sfhe_encrypt");
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!values || !coords || !ct) return fail(SFHE_EINVAL, "null argument");
    cudaStream_t s = as_stream(stream);
    long long* d_vals = nullptr;
    int* d_coords = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&d_vals, n * sizeof(long long), s));
    CUDA_TRY(cudaMallocAsync((void**)&d_coords, n * 2 * sizeof(int), s));
    CUDA_TRY(cudaMemcpyAsync(d_vals, values, n * sizeof(long long), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_coords, coords, n * 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_encrypt(c->rc, c->d_s, d_vals, d_coords, n, matrix_id, ct, c->d_err, s);
    cudaFreeAsync(d_vals, s);
    cudaFreeAsync(d_coords, s);
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "encrypt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

static const int64_t kLiftChunk = 256;

extern "C" sfhe_status sfhe_lift_workspace_size(const sfhe_ctx* c, int64_t n, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, kLiftChunk));
    *bytes = (size_t)chunk * 2 * c->rc.N * (c->rc.L * 8 + c->rc.K * 4);
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_lift(sfhe_ctx* c, const uint64_t* ct, int64_t n, uint32_t* ext, void* work,
                                 size_t work_bytes, void* stream)
{
    Range range("sfhe_lift");
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!ct || !ext || !work) return fail(SFHE_EINVAL, "null argument");
    const RnsConsts& rc = c->rc;
    const size_t N = rc.N, L = rc.L, K = rc.K;
    const size_t per_ct = 2 * N * (L * 8 + K * 4);
    const int64_t chunk = (int64_t)(work_bytes / per_ct);
    if (chunk < 1) return fail(SFHE_ENOMEM, "lift workspace too small");
    cudaStream_t s = as_stream(stream);
    u64* wq = (u64*)work;  // [2c][L][N] coefficient form over Q
    const size_t ctw = 2 * L * N, extw = 2 * K * N;
    for (int64_t n0 = 0; n0 < n; n0 += chunk) {
        const int64_t cnt = std::min(chunk, n - n0);
        u32* wb = (u32*)(wq + (size_t)cnt * 2 * L * N);  // [2c][K][N] coefficient form over B
        const u64* src = ct + n0 * ctw;
        u32* dst = ext + n0 * extw;
        cudaError_t e = launch_ntt(rc, true, src, L * N, 0, wq, L * N, 0, 0, (int)L, 2 * cnt, s);
        if (e == cudaSuccess) e = launch_lift_extend(rc, wq, wb, 2 * cnt, s);
        if (e == cudaSuccess) e = launch_ntt32(rc, false, wb, K * N, 0, dst, K * N, 0, 0, (int)K, 2 * cnt, true, s);
        if (e != cudaSuccess) return fail(SFHE_ECUDA, "lift: %s", cudaGetErrorString(e));
    }
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_decrypt(sfhe_ctx* c, const uint64_t* ct, int64_t n, int64_t* out, void* stream)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!ct || !out) return fail(SFHE_EINVAL, "null argument");
    cudaError_t e = launch_decrypt(c->rc, c->d_s, ct, n, (long long*)out, as_stream(stream));
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "decrypt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

static sfhe_status convert(sfhe_ctx* c, const uint64_t* in, int64_t npoly, uint64_t* out, void* stream, bool inverse)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (npoly < 0) return fail(SFHE_ESHAPE, "negative count");
    if (npoly == 0) return SFHE_OK;
    if (!in || !out) return fail(SFHE_EINVAL, "null argument");
    const size_t LN = (size_t)c->rc.L * c->rc.N;
    cudaError_t e = launch_ntt(c->rc, inverse, in, LN, 0, out, LN, 0, 0, c->rc.L, npoly, as_stream(stream));
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "ntt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_to_coeff(sfhe_ctx* c, const uint64_t* in, int64_t npoly, uint64_t* out, void* stream)
{
    return convert(c, in, npoly, out, stream, true);
}

extern "C" sfhe_status sfhe_from_coeff(sfhe_ctx* c, const uint64_t* in, int64_t npoly, uint64_t* out, void* stream)
{
    return convert(c, in, npoly, out, stream, false);
}

extern "C" sfhe_status sfhe_export_secret(sfhe_ctx* c, int8_t* s_host)
{
    if (!c || !s_host) return fail(SFHE_EINVAL, "null argument");
    CUDA_TRY(cudaMemcpy(s_host, c->d_s_coeff, c->rc.N, cudaMemcpyDeviceToHost));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_export_relin_key(sfhe_ctx* c, uint64_t* out, void* stream)
{
    if (!c || !out) return fail(SFHE_EINVAL, "null argument");
    return convert(c, c->d_rlk, 2 * c->rc.L, out, stream, true);
}

// ------------------------------------------------------------- work lists ---
namespace {

struct Layout {
    size_t queue, mms, entries, rowlist, scratch, T, D, U, total;
};

sfhe_status validate_matrix(const sfhe_matrix_view& m, const char* name)
{
    if (m.rows < 0 || m.cols < 0) return fail(SFHE_ESHAPE, "%s: negative shape", name);
    if (m.encoding < SFHE_ENC_DENSE || m.encoding > SFHE_ENC_ELL) return fail(SFHE_EINVAL, "%s: bad encoding", name);
    const int64_t dense = (int64_t)m.rows * m.cols;
    switch (m.encoding) {
    case SFHE_ENC_DENSE:
        if (m.nct != dense) return fail(SFHE_ESHAPE, "%s: DENSE needs rows*cols ciphertexts", name);
        break;
    case SFHE_ENC_MASK:
        if (m.nct != dense) return fail(SFHE_ESHAPE, "%s: MASK needs rows*cols ciphertexts", name);
        if (!m.mask && dense > 0) return fail(SFHE_EINVAL, "%s: null mask", name);
        break;
    case SFHE_ENC_CSR: {
        if (!m.row_ptr) return fail(SFHE_EINVAL, "%s: null row_ptr", name);
        if (m.row_ptr[0] != 0) return fail(SFHE_EINVAL, "%s: row_ptr[0] != 0", name);
        for (int32_t r = 0; r < m.rows; r++)
            if (m.row_ptr[r + 1] < m.row_ptr[r]) return fail(SFHE_EINVAL, "%s: row_ptr not monotone at %d", name, r);
        if (m.row_ptr[m.rows] != m.nct) return fail(SFHE_ESHAPE, "%s: row_ptr[rows] != nct", name);
        if (m.nct > 0 && !m.col_idx) return fail(SFHE_EINVAL, "%s: null col_idx", name);
        for (int32_t t = 0; t < m.nct; t++)
            if (m.col_idx[t] < 0 || m.col_idx[t] >= m.cols) return fail(SFHE_EINVAL, "%s: col_idx[%d] out of range", name, t);
        break;
    }
    case SFHE_ENC_ELL:
        if (m.ell_width < 0 || (int64_t)m.rows * m.ell_width != m.nct)
            return fail(SFHE_ESHAPE, "%s: ELL needs rows*ell_width ciphertexts", name);
        if (m.nct > 0 && !m.ell_col) return fail(SFHE_EINVAL, "%s: null ell_col", name);
        for (int32_t t = 0; t < m.nct; t++)
            if (m.ell_col[t] < -1 || m.ell_col[t] >= m.cols) return fail(SFHE_EINVAL, "%s: ell_col[%d] out of range", name, t);
        break;
    }
    return SFHE_OK;
}

// rows of (A ciphertext index, k) pairs listed by A's encoding
void row_pairs(const sfhe_matrix_view& A, int32_t i, bool dense_loop, std::vector<int2>& out)
{
    const int32_t K = A.cols;
    if (dense_loop) {
        for (int32_t k = 0; k < K; k++) out.push_back(make_int2(i * K + k, k));
        return;
    }
    switch (A.encoding) {
    case SFHE_ENC_DENSE:
        for (int32_t k = 0; k < K; k++) out.push_back(make_int2(i * K + k, k));
        break;
    case SFHE_ENC_MASK:
        for (int32_t k = 0; k < K; k++)
            if (!A.mask[(int64_t)i * K + k]) out.push_back(make_int2(i * K + k, k));
        break;
    case SFHE_ENC_CSR:
        for (int32_t t = A.row_ptr[i]; t < A.row_ptr[i + 1]; t++) out.push_back(make_int2(t, A.col_idx[t]));
        break;
    case SFHE_ENC_ELL:
        for (int32_t s = 0; s < A.ell_width; s++) {
            const int32_t k = A.ell_col[(int64_t)i * A.ell_width + s];
            if (k >= 0) out.push_back(make_int2(i * A.ell_width + s, k));
        }
        break;
    }
}

sfhe_status build(const sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B, const sfhe_matrix_view* C,
                  const bool* dense_loop, sfhe_plan& P)
{
    if (n < 0) return fail(SFHE_ESHAPE, "negative matmul count");
    if (n > 0 && (!A || !B)) return fail(SFHE_EINVAL, "null operands");
    P.mms.clear();
    P.entries.clear();
    P.rowlist.clear();
    P.c_words.clear();
    P.products = 0;
    const size_t ctw = (size_t)2 * c->rc.L * c->rc.N;
    for (int32_t m = 0; m < n; m++) {
        sfhe_status st = validate_matrix(A[m], "A");
        if (st == SFHE_OK) st = validate_matrix(B[m], "B");
        if (st != SFHE_OK) return st;
        if (B[m].encoding != SFHE_ENC_DENSE && B[m].encoding != SFHE_ENC_MASK)
            return fail(SFHE_EINVAL, "B must be DENSE- or MASK-encoded");
        if (A[m].cols != B[m].rows) return fail(SFHE_ESHAPE, "A is %dx%d, B is %dx%d", A[m].rows, A[m].cols, B[m].rows, B[m].cols);
        if (C) {
            if (C[m].rows != A[m].rows || C[m].cols != B[m].cols) return fail(SFHE_ESHAPE, "C shape mismatch");
            if (C[m].encoding != SFHE_ENC_DENSE || C[m].nct != C[m].rows * C[m].cols)
                return fail(SFHE_EINVAL, "C must be DENSE with rows*cols ciphertexts");
            if (!C[m].ct && C[m].nct > 0) return fail(SFHE_EINVAL, "null C storage");
        }
        if ((A[m].nct > 0 && !A[m].ext) || (B[m].nct > 0 && !B[m].ext))
            return fail(SFHE_EINVAL, "operands need lifted storage (sfhe_lift)");
        MmDesc d;
        d.A_ext = A[m].ext;
        d.B_ext = B[m].ext;
        d.C = C ? C[m].ct : nullptr;
        d.Nc = B[m].cols;
        d.group = (P.flags & SFHE_EXEC_LAZY) ? c->rc.lazy_group : 1;
        P.mms.push_back(d);
        P.c_words.push_back((size_t)A[m].rows * B[m].cols * ctw);
        // with a masked B the naive sparse scheme also skips k where B[k][j]
        // is zero (Sec. 3.3.2: a product is skipped when either mask is set),
        // so every entry gets its own list; otherwise the entries of a row
        // share the row's list
        const bool b_mask = B[m].encoding == SFHE_ENC_MASK && !dense_loop[m];
        const int32_t Nc = B[m].cols;
        std::vector<int2> row;
        for (int32_t i = 0; i < A[m].rows; i++) {
            row.clear();
            row_pairs(A[m], i, dense_loop[m], row);
            int first = (int)P.rowlist.size();
            if (!b_mask) P.rowlist.insert(P.rowlist.end(), row.begin(), row.end());
            for (int32_t j = 0; j < Nc; j++) {
                if (b_mask) {
                    first = (int)P.rowlist.size();
                    for (const int2& it : row)
                        if (!B[m].mask[(int64_t)it.y * Nc + j]) P.rowlist.push_back(it);
                }
                const int count = b_mask ? (int)P.rowlist.size() - first : (int)row.size();
                if (count > 1024) return fail(SFHE_EUNSUPPORTED, "more than 1024 products per output entry");
                Entry en;
                memset(&en, 0, sizeof(en));
                en.mm = m;
                en.row = i;
                en.col = j;
                en.count = count;
                en.first = first;
                P.entries.push_back(en);
                P.products += count;
            }
        }
    }
    // longest entries first: the persistent queue then approximates LPT
    std::stable_sort(P.entries.begin(), P.entries.end(), [](const Entry& a, const Entry& b) { return a.count > b.count; });
    return SFHE_OK;
}

Layout layout_of(const sfhe_ctx* c, const sfhe_plan& P, uint32_t flags, int* grid_out, size_t* stride_out)
{
    Layout Lo;
    memset(&Lo, 0, sizeof(Lo));
    size_t off = 0;
    Lo.queue = off;
    off += 256;
    Lo.mms = off;
    off += align256(P.mms.size() * sizeof(MmDesc));
    Lo.entries = off;
    off += align256(P.entries.size() * sizeof(Entry));
    Lo.rowlist = off;
    off += align256(P.rowlist.size() * sizeof(int2));
    const size_t N = c->rc.N, L = c->rc.L, K = c->rc.K;
    *grid_out = 0;
    *stride_out = 0;
    if (flags & SFHE_EXEC_PERSISTENT) {
        const int per_sm = persistent_ctas_per_sm(c->rc);
        int grid = per_sm * c->num_sms;
        grid = (int)std::min<size_t>((size_t)grid, std::max<size_t>(1, P.entries.size()));
        const size_t stride = persistent_scratch_words(c->rc);
        Lo.scratch = off;
        off += align256((size_t)grid * stride * 8);
        *grid_out = grid;
        *stride_out = stride;
    }
    if (flags & SFHE_EXEC_PLAIN) {
        Lo.T = off;
        off += align256(3 * K * N * 4);
        Lo.D = off;
        off += align256(3 * L * N * 8);
        Lo.U = off;
        off += align256((L + 2) * L * N * 8);
    }
    Lo.total = off;
    return Lo;
}

sfhe_status check_flags(uint32_t flags)
{
    const bool plain = flags & SFHE_EXEC_PLAIN, pers = flags & SFHE_EXEC_PERSISTENT;
    if (plain == pers) return fail(SFHE_EINVAL, "exactly one of PLAIN and PERSISTENT");
    if ((flags & SFHE_EXEC_GRAPH) && !pers) return fail(SFHE_EINVAL, "GRAPH needs PERSISTENT");
    if ((flags & SFHE_EXEC_LAZY) && !pers) return fail(SFHE_EINVAL, "LAZY needs PERSISTENT");
    if (flags & ~(uint32_t)(SFHE_EXEC_PLAIN | SFHE_EXEC_PERSISTENT | SFHE_EXEC_GRAPH | SFHE_EXEC_LAZY))
        return fail(SFHE_EINVAL, "unknown flags");
    return SFHE_OK;
}

PersistentArgs persistent_args(const sfhe_plan* P, int n_entries, int variant)
{
    const sfhe_ctx* c = P->ctx;
    PersistentArgs a;
    a.mms = P->d_mms;
    a.entries = P->d_entries;
    a.n_entries = n_entries;
    a.rowlist = P->d_rowlist;
    a.rlk = c->d_rlk;
    a.rlk_sh = c->d_rlk_sh;
    a.scratch = P->d_scratch;
    a.scratch_stride = P->scratch_stride;
    a.queue = P->d_queue;
    a.stop = P->d_stop;
    a.grid = P->grid;
    a.grouped = (P->flags & SFHE_EXEC_LAZY) != 0;
    a.variant = a.grouped ? 0 : variant;
    a.l2_base = c->d_rlk;
    a.l2_bytes = c->l2_bytes;
    a.l2_hit_ratio = c->l2_hit;
    return a;
}

// The tile tuner.  On the first per-product persistent plan of a context at
// a ring with several stage-S tiles, every tile runs on a calibration list
// built from the plan's own work: its first `grid` entries (the longest,
// one per CTA) cut to at most 4 products each, uploaded over the plan's
// entry list and replaced by the real list afterwards.  Each tile runs once
// to warm up and twice timed (CUDA events on the plan's stream); the fastest
// is kept for the context.  The calibration writes C of those entries, which
// every execution of the plan writes again.  Synchronises the stream.
sfhe_status tune_variants(sfhe_plan* P, cudaStream_t s)
{
    sfhe_ctx* c = P->ctx;
    const int nv = c->n_variants;
    std::vector<Entry> cal(P->entries.begin(), P->entries.begin() + std::min<size_t>(P->entries.size(), P->grid));
    for (Entry& e : cal) e.count = std::min(e.count, 4);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    cudaError_t e = cudaMemcpyAsync(P->d_entries, cal.data(), cal.size() * sizeof(Entry), cudaMemcpyHostToDevice, s);
    float best = 0.f;
    int best_v = 0;
    for (int v = 0; v < nv && e == cudaSuccess; v++) {
        float t = 0.f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
            e = cudaMemsetAsync(P->d_queue, 0, 2 * sizeof(unsigned), s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_persistent(c->rc, persistent_args(P, (int)cal.size(), v), s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 || (rep == 2 && ms < t)) t = ms;
        }
        if (v < 8) c->variant_ms[v] = t;
        if (v == 0 || t < best) best = t, best_v = v;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->d_entries, P->entries.data(), cal.size() * sizeof(Entry), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "tile tuning: %s", cudaGetErrorString(e));
    // a bounded wait that ran out during calibration is reported like one
    // during an execution
    unsigned err = 0;
    CUDA_TRY(cudaMemcpy(&err, P->d_queue + 1, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) return fail(SFHE_ETIMEOUT, "an operand copy did not complete within its wait bound (tile tuning)");
    c->tuned_variant = best_v;
    return SFHE_OK;
}

sfhe_status launch_plan(sfhe_plan* P, cudaStream_t s)
{
    const sfhe_ctx* c = P->ctx;
    const RnsConsts& rc = c->rc;
    if (P->flags & SFHE_EXEC_PERSISTENT) {
        if (P->gexec) {
            CUDA_TRY(cudaGraphLaunch(P->gexec, s));
            return SFHE_OK;
        }
        CUDA_TRY(cudaMemsetAsync(P->d_queue, 0, 2 * sizeof(unsigned), s));
        if (P->entries.empty()) return SFHE_OK;
        CUDA_TRY(launch_persistent(rc, persistent_args(P, (int)P->entries.size(), P->variant), s));
        return SFHE_OK;
    }
    // plain: C = 0, then one launch sequence per product
    for (size_t m = 0; m < P->mms.size(); m++)
        if (P->c_words[m]) CUDA_TRY(cudaMemsetAsync(P->mms[m].C, 0, P->c_words[m] * 8, s));
    const size_t N = rc.N, L = rc.L, K = rc.K;
    const size_t ctw = 2 * L * N, extw = 2 * K * N;
    for (const Entry& en : P->entries) {
        const MmDesc& mm = P->mms[en.mm];
        u64* Cout = mm.C + ((size_t)en.row * mm.Nc + en.col) * ctw;
        for (int p = 0; p < en.count; p++) {
            const int2 it = P->rowlist[en.first + p];
            const u32* a = mm.A_ext + (size_t)it.x * extw;
            const u32* b = mm.B_ext + ((size_t)it.y * mm.Nc + en.col) * extw;
            CUDA_TRY(launch_tensor_intt(rc, a, b, P->d_T, s));
            CUDA_TRY(launch_scale_round(rc, P->d_T, P->d_D, s));
            CUDA_TRY(launch_relin_ntt(rc, P->d_D, P->d_U, s));
            CUDA_TRY(launch_relin_accum(rc, P->d_U, c->d_rlk, c->d_rlk_sh, Cout, s));
        }
    }
    return SFHE_OK;
}

}  // namespace

sfhe_status sfhe::validate_view(const sfhe_matrix_view& m, const char* name) { return validate_matrix(m, name); }

extern "C" void sfhe_plan_destroy(sfhe_plan* P)
{
    if (!P) return;
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;
}

static sfhe_status plan_finish(sfhe_ctx* c, sfhe_plan* P, uint32_t flags, void* work, size_t work_bytes, void* stream,
                               sfhe_plan** out);

static sfhe_plan* new_plan(sfhe_ctx* c, uint32_t flags)
{
    sfhe_plan* P = new sfhe_plan();
    P->ctx = c;
    P->flags = flags;
    P->graph = nullptr;
    P->gexec = nullptr;
    P->d_stop = nullptr;
    P->launched = false;
    return P;
}

static sfhe_status plan_create_impl(sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                    sfhe_matrix_view* C, const bool* dense_loop, uint32_t flags, void* work,
                                    size_t work_bytes, void* stream, sfhe_plan** out)
{
    if (!c || !out) return fail(SFHE_EINVAL, "null argument");
    *out = nullptr;
    sfhe_status st = check_flags(flags);
    if (st != SFHE_OK) return st;
    if (n > 0 && !C) return fail(SFHE_EINVAL, "null C");
    sfhe_plan* P = new_plan(c, flags);
    st = build(c, n, A, B, C, dense_loop, *P);
    if (st != SFHE_OK) {
        delete P;
        return st;
    }
    return plan_finish(c, P, flags, work, work_bytes, stream, out);
}

// A plan whose work list is filled: lay it out in `work`, upload the list,
// pick the tile, capture the graph.  Takes P (deleted on error).
static sfhe_status plan_finish(sfhe_ctx* c, sfhe_plan* P, uint32_t flags, void* work, size_t work_bytes, void* stream,
                               sfhe_plan** out)
{
    Layout Lo = layout_of(c, *P, flags, &P->grid, &P->scratch_stride);
    if ((flags & SFHE_EXEC_PERSISTENT) && P->grid <= 0) {
        delete P;
        return fail(SFHE_ECUDA, "persistent kernel cannot be resident on this device");
    }
    if (!work || work_bytes < Lo.total) {
        delete P;
        return fail(SFHE_ENOMEM, "workspace of %zu bytes needed, %zu given", Lo.total, work_bytes);
    }
    char* w = (char*)work;
    P->d_queue = (unsigned*)(w + Lo.queue);
    P->d_mms = (MmDesc*)(w + Lo.mms);
    P->d_entries = (Entry*)(w + Lo.entries);
    P->d_rowlist = (int2*)(w + Lo.rowlist);
    P->d_scratch = (u64*)(w + Lo.scratch);
    P->d_T = (u32*)(w + Lo.T);
    P->d_D = (u64*)(w + Lo.D);
    P->d_U = (u64*)(w + Lo.U);
    cudaStream_t s = as_stream(stream);
    auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    cudaError_t e = up(P->d_mms, P->mms.data(), P->mms.size() * sizeof(MmDesc));
    if (e == cudaSuccess) e = up(P->d_entries, P->entries.data(), P->entries.size() * sizeof(Entry));
    if (e == cudaSuccess) e = up(P->d_rowlist, P->rowlist.data(), P->rowlist.size() * sizeof(int2));
    if (e != cudaSuccess) {
        delete P;
        return fail(SFHE_ECUDA, "work list upload: %s", cudaGetErrorString(e));
    }
    // tile variant: forced, tuned earlier, or tuned now on this plan
    P->variant = 0;
    if ((flags & SFHE_EXEC_PERSISTENT) && !(flags & SFHE_EXEC_LAZY) && c->n_variants > 1) {
        std::lock_guard<std::mutex> lock(c->tune_mu);
        if (c->forced_variant >= 0) {
            P->variant = c->forced_variant;
        } else {
            if (c->tuned_variant < 0 && !P->entries.empty()) {
                sfhe_status ts = tune_variants(P, s);
                if (ts != SFHE_OK) {
                    delete P;
                    return ts;
                }
            }
            P->variant = std::max(c->tuned_variant, 0);
        }
    }
    if (flags & SFHE_EXEC_GRAPH) {
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            sfhe_status ls = SFHE_OK;
            if (cudaMemsetAsync(P->d_queue, 0, 2 * sizeof(unsigned), cap) != cudaSuccess) ls = SFHE_ECUDA;
            if (ls == SFHE_OK && !P->entries.empty())
                if (launch_persistent(c->rc, persistent_args(P, (int)P->entries.size(), P->variant), cap) !=
                    cudaSuccess)
                    ls = SFHE_ECUDA;
            cudaError_t e2 = cudaStreamEndCapture(cap, &P->graph);
            if (ls != SFHE_OK || e2 != cudaSuccess) e = cudaErrorUnknown;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->gexec, P->graph, 0);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            sfhe_plan_destroy(P);
            return fail(SFHE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
    }
    *out = P;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_plan_create(sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                        sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream,
                                        sfhe_plan** out)
{
    std::vector<char> dl(std::max(n, 0), 0);
    return plan_create_impl(c, n, A, B, C, (const bool*)dl.data(), flags, work, work_bytes, stream, out);
}

extern "C" sfhe_status sfhe_plan_execute(sfhe_plan* P, void* stream)
{
    Range range("sfhe_plan_execute");
    if (!P) return fail(SFHE_EINVAL, "null plan");
    P->launched = true;
    return launch_plan(P, as_stream(stream));
}

extern "C" sfhe_status sfhe_plan_set_stop(sfhe_plan* P, const uint32_t* word)
{
    if (!P) return fail(SFHE_EINVAL, "null plan");
    if (!(P->flags & SFHE_EXEC_PERSISTENT)) return fail(SFHE_EINVAL, "a stop word needs a PERSISTENT plan");
    if (P->gexec) return fail(SFHE_EINVAL, "a stop word cannot be set on a GRAPH plan (its launch is captured)");
    if (reinterpret_cast<uintptr_t>(word) % alignof(uint32_t)) return fail(SFHE_EINVAL, "misaligned stop word");
    P->d_stop = reinterpret_cast<const unsigned*>(word);
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_plan_progress(const sfhe_plan* P, int64_t* done, void* stream)
{
    if (!P || !done) return fail(SFHE_EINVAL, "null argument");
    if (!(P->flags & SFHE_EXEC_PERSISTENT)) return fail(SFHE_EINVAL, "progress is kept by PERSISTENT plans");
    if (!P->launched) {
        *done = 0;
        return SFHE_OK;
    }
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    unsigned taken = 0;
    CUDA_TRY(cudaMemcpy(&taken, P->d_queue, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *done = std::min<int64_t>((int64_t)taken, (int64_t)P->entries.size());
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_plan_resume(sfhe_plan* P, void* stream)
{
    Range range("sfhe_plan_resume");
    if (!P) return fail(SFHE_EINVAL, "null plan");
    if (!(P->flags & SFHE_EXEC_PERSISTENT)) return fail(SFHE_EINVAL, "only PERSISTENT plans resume");
    if (!P->launched) return fail(SFHE_EINVAL, "resume before the plan's first execution");
    // the entry counter is left as the stopped launch left it: the entries
    // below it are complete, the rest are taken from it on
    if (P->entries.empty()) return SFHE_OK;
    CUDA_TRY(launch_persistent(P->ctx->rc, persistent_args(P, (int)P->entries.size(), P->variant), as_stream(stream)));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_selftest_wait_bound(void* work, uint32_t tries, uint32_t limit_us, void* stream)
{
    if (!work) return fail(SFHE_EINVAL, "null workspace");
    if (tries == 0 || tries > (1u << 30)) return fail(SFHE_EINVAL, "tries must be in 1 .. 2^30");
    if (limit_us == 0 || limit_us > 1000000u) return fail(SFHE_EINVAL, "limit_us must be in 1 .. 10^6");
    CUDA_TRY(launch_wait_selftest((unsigned*)work, tries, (u64)limit_us * 1000u, as_stream(stream)));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_check(void* work, void* stream)
{
    if (!work) return fail(SFHE_EINVAL, "null workspace");
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    unsigned err = 0;
    CUDA_TRY(cudaMemcpy(&err, (char*)work + sizeof(unsigned), sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) return fail(SFHE_ETIMEOUT, "an operand copy of the persistent kernel did not complete within its wait bound");
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_measure_mulmod32(sfhe_ctx* c, double* per_s, void* stream)
{
    if (!c || !per_s) return fail(SFHE_EINVAL, "null argument");
    const u32 b = c->rc.mb[0].b, w = b - 12345u;
    const u32 ws = (u32)(((u64)w << 32) / b);
    CUDA_TRY(measure_mulmod32(b, w, ws, per_s, as_stream(stream)));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_plan_stats(const sfhe_plan* P, int64_t* products, int64_t* entries, int64_t* launches,
                                       int64_t* ctas)
{
    if (!P) return fail(SFHE_EINVAL, "null plan");
    if (products) *products = P->products;
    if (entries) *entries = (int64_t)P->entries.size();
    if (launches) *launches = (P->flags & SFHE_EXEC_PERSISTENT) ? (P->entries.empty() ? 0 : 1) : 4 * P->products;
    if (ctas) *ctas = P->grid;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ctx_tuning(const sfhe_ctx* c, int32_t* variant, int32_t* n_variants, float* ms)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    sfhe_ctx* m = const_cast<sfhe_ctx*>(c);
    std::lock_guard<std::mutex> lock(m->tune_mu);
    if (variant) *variant = c->forced_variant >= 0 ? c->forced_variant : c->tuned_variant;
    if (n_variants) *n_variants = c->n_variants;
    if (ms)
        for (int v = 0; v < c->n_variants && v < 8; v++) ms[v] = c->tuned_variant >= 0 ? c->variant_ms[v] : 0.f;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ctx_set_variant(sfhe_ctx* c, int32_t variant)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (variant < -1 || variant >= c->n_variants)
        return fail(SFHE_EINVAL, "variant %d outside -1 .. %d", variant, c->n_variants - 1);
    std::lock_guard<std::mutex> lock(c->tune_mu);
    c->forced_variant = variant;
    return SFHE_OK;
}

extern "C" const char* sfhe_ctx_variant_name(const sfhe_ctx* c, int32_t variant)
{
    return c ? persistent_variant_name(c->rc, variant) : "";
}

static sfhe_status size_impl(const sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                             const bool* dense_loop, uint32_t flags, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    sfhe_status st = check_flags(flags);
    if (st != SFHE_OK) return st;
    sfhe_plan P;
    P.ctx = const_cast<sfhe_ctx*>(c);
    P.flags = flags;
    st = build(c, n, A, B, nullptr, dense_loop, P);
    if (st != SFHE_OK) return st;
    int grid;
    size_t stride;
    *bytes = layout_of(c, P, flags, &grid, &stride).total;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_workspace_bound(const sfhe_ctx* c, int32_t max_matmuls, int64_t max_entries,
                                                   int64_t max_products, uint32_t flags, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    if (max_matmuls < 0 || max_entries < 0 || max_products < 0) return fail(SFHE_ESHAPE, "negative bound");
    sfhe_status st = check_flags(flags);
    if (st != SFHE_OK) return st;
    // the layout of layout_of() with every list at its bound and the full grid
    size_t off = 256;
    off += align256((size_t)max_matmuls * sizeof(MmDesc));
    off += align256((size_t)max_entries * sizeof(Entry));
    off += align256((size_t)max_products * sizeof(int2));
    const size_t N = c->rc.N, L = c->rc.L, K = c->rc.K;
    if (flags & SFHE_EXEC_PERSISTENT)
        off += align256((size_t)persistent_ctas_per_sm(c->rc) * c->num_sms * persistent_scratch_words(c->rc) * 8);
    if (flags & SFHE_EXEC_PLAIN)
        off += align256(3 * K * N * 4) + align256(3 * L * N * 8) + align256((L + 2) * L * N * 8);
    *bytes = off;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_workspace_size(const sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A,
                                                  const sfhe_matrix_view* B, uint32_t flags, size_t* bytes)
{
    std::vector<char> dl(std::max(n, 0), 0);
    return size_impl(c, n, A, B, (const bool*)dl.data(), flags, bytes);
}

static sfhe_status one_shot(sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B, sfhe_matrix_view* C,
                            const bool* dense_loop, uint32_t flags, void* work, size_t work_bytes, void* stream)
{
    Range range("sfhe_matmul");
    sfhe_plan* P = nullptr;
    // a one-shot call launches directly; graphs are for replayed plans
    sfhe_status st = plan_create_impl(c, n, A, B, C, dense_loop, flags & ~(uint32_t)SFHE_EXEC_GRAPH, work, work_bytes,
                                      stream, &P);
    if (st != SFHE_OK) return st;
    st = launch_plan(P, as_stream(stream));
    sfhe_plan_destroy(P);
    return st;
}

extern "C" sfhe_status sfhe_matmul_dense_view(sfhe_ctx* c, const sfhe_matrix_view* A, const sfhe_matrix_view* B, sfhe_matrix_view* C,
                                         uint32_t flags, void* work, size_t work_bytes, void* stream)
{
    if (!A) return fail(SFHE_EINVAL, "null A");
    if (A->encoding != SFHE_ENC_DENSE && A->encoding != SFHE_ENC_MASK)
        return fail(SFHE_EINVAL, "the dense loop needs every element of A stored (DENSE or MASK)");
    const bool dl = true;
    return one_shot(c, 1, A, B, C, &dl, flags, work, work_bytes, stream);
}

extern "C" sfhe_status sfhe_matmul_sparse_view(sfhe_ctx* c, const sfhe_matrix_view* A, const sfhe_matrix_view* B, int32_t encoding,
                                          sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream)
{
    if (!A) return fail(SFHE_EINVAL, "null A");
    if (encoding != SFHE_ENC_MASK && encoding != SFHE_ENC_CSR && encoding != SFHE_ENC_ELL)
        return fail(SFHE_EINVAL, "sparse encoding must be MASK, CSR or ELL");
    if (A->encoding != encoding) return fail(SFHE_EINVAL, "A is encoded as %d, not %d", A->encoding, encoding);
    const bool dl = false;
    return one_shot(c, 1, A, B, C, &dl, flags, work, work_bytes, stream);
}

extern "C" sfhe_status sfhe_matmul_batch_view(sfhe_ctx* c, int32_t n, const sfhe_matrix_view* A, const sfhe_matrix_view* B,
                                         sfhe_matrix_view* C, uint32_t flags, void* work, size_t work_bytes, void* stream)
{
    std::vector<char> dl(std::max(n, 0), 0);
    return one_shot(c, n, A, B, C, (const bool*)dl.data(), flags, work, work_bytes, stream);
}

// ------------------------------------------------------ stage entry points ---
extern "C" sfhe_status sfhe_ct_tensor_scale(sfhe_ctx* c, const uint32_t* a_ext, const uint32_t* b_ext, uint64_t* d,
                                            void* work, size_t work_bytes, void* stream)
{
    if (!c || !a_ext || !b_ext || !d || !work) return fail(SFHE_EINVAL, "null argument");
    const size_t need = (size_t)3 * c->rc.K * c->rc.N * 4;
    if (work_bytes < need) return fail(SFHE_ENOMEM, "workspace of %zu bytes needed", need);
    cudaStream_t s = as_stream(stream);
    CUDA_TRY(launch_tensor_intt(c->rc, a_ext, b_ext, (u32*)work, s));
    CUDA_TRY(launch_scale_round(c->rc, (const u32*)work, d, s));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ct_mul_relin(sfhe_ctx* c, const uint32_t* a_ext, const uint32_t* b_ext, uint64_t* out,
                                         void* work, size_t work_bytes, void* stream)
{
    if (!c || !a_ext || !b_ext || !out || !work) return fail(SFHE_EINVAL, "null argument");
    const size_t N = c->rc.N, L = c->rc.L, K = c->rc.K;
    const size_t tw = align256(3 * K * N * 4);
    const size_t need = tw + (3 * L + (L + 2) * L) * N * 8;
    if (work_bytes < need) return fail(SFHE_ENOMEM, "workspace of %zu bytes needed", need);
    cudaStream_t s = as_stream(stream);
    u32* T = (u32*)work;
    u64* D = (u64*)((char*)work + tw);
    u64* U = D + 3 * L * N;
    CUDA_TRY(cudaMemsetAsync(out, 0, 2 * L * N * 8, s));
    CUDA_TRY(launch_tensor_intt(c->rc, a_ext, b_ext, T, s));
    CUDA_TRY(launch_scale_round(c->rc, T, D, s));
    CUDA_TRY(launch_relin_ntt(c->rc, D, U, s));
    CUDA_TRY(launch_relin_accum(c->rc, U, c->d_rlk, c->d_rlk_sh, out, s));
    return SFHE_OK;
}


extern "C" sfhe_status sfhe_ct_mul_relin_static(sfhe_ctx* c, const uint32_t* a_ext, const uint32_t* b_ext,
                                                uint64_t* out, void* stream)
{
    if (!c || !a_ext || !b_ext || !out) return fail(SFHE_EINVAL, "null argument");
    const size_t N = c->rc.N, L = c->rc.L, K = c->rc.K;
    const size_t tw = align256(3 * K * N * 4);
    const size_t need = tw + (3 * L + (L + 2) * L) * N * 8;
    if (need > SFHE_STATIC_SCRATCH_BYTES)
        return fail(SFHE_ENOMEM, "N = %zu, L = %zu needs %zu bytes of scratch; the static scratch holds %zu", N, L,
                    need, (size_t)SFHE_STATIC_SCRATCH_BYTES);
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != c->device) return fail(SFHE_EINVAL, "current device %d is not the context's device %d", dev, c->device);
    if (dev < 0 || dev >= 64) return fail(SFHE_EINVAL, "device ordinal %d out of range", dev);
    void* base;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[dev]) {
            void* p = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
            g_static_addr[dev] = p;
        }
        base = g_static_addr[dev];
    }
    cudaStream_t s = as_stream(stream);
    u32* T = (u32*)base;
    u64* D = (u64*)((char*)base + tw);
    u64* U = D + 3 * L * N;
    CUDA_TRY(cudaMemsetAsync(out, 0, 2 * L * N * 8, s));
    CUDA_TRY(launch_tensor_intt(c->rc, a_ext, b_ext, T, s));
    CUDA_TRY(launch_scale_round(c->rc, T, D, s));
    CUDA_TRY(launch_relin_ntt(c->rc, D, U, s));
    CUDA_TRY(launch_relin_accum(c->rc, U, c->d_rlk, c->d_rlk_sh, out, s));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ntt(sfhe_ctx* c, int32_t prime_index, int32_t inverse, const void* in, int64_t npoly,
                                void* out, void* stream)
{
    if (!c || !in || !out) return fail(SFHE_EINVAL, "null argument");
    if (prime_index < 0 || prime_index >= c->rc.L + c->rc.K) return fail(SFHE_EINVAL, "prime index out of range");
    if (npoly < 0) return fail(SFHE_ESHAPE, "negative count");
    const size_t N = c->rc.N;
    cudaError_t e = prime_index < c->rc.L
                        ? launch_ntt(c->rc, inverse != 0, (const u64*)in, N, 0, (u64*)out, N, 0, prime_index, 1, npoly,
                                     as_stream(stream))
                        : launch_ntt32(c->rc, inverse != 0, (const u32*)in, N, 0, (u32*)out, N, 0,
                                       prime_index - c->rc.L, 1, npoly, false, as_stream(stream));
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "ntt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_prng_words(uint64_t seed, uint32_t domain, uint64_t o0, uint64_t o1, uint64_t o2,
                                       uint64_t idx0, int64_t n, uint64_t* out, void* stream)
{
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n > 0 && !out) return fail(SFHE_EINVAL, "null output");
    CUDA_TRY(launch_prng(seed, domain, o0, o1, o2, idx0, n, out, as_stream(stream)));
    return SFHE_OK;
}

// ------------------------------------------------- slot-packed chunks ---
// Alg. 1 with chunk size c > 1 (Sec. 3.2): c values per ciphertext in its
// slots, rotations to and from slot 0, the slot-0 mask.

extern "C" sfhe_status sfhe_slots_encode(uint32_t N, uint64_t t, const int64_t* values, int64_t* poly)
{
    if (!values || !poly) return fail(SFHE_EINVAL, "null argument");
    if (!slots_encode(N, t, values, poly)) return fail(SFHE_EUNSUPPORTED, "N=%u t=%llu", N, (unsigned long long)t);
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_slots_decode(uint32_t N, uint64_t t, const int64_t* poly, int64_t* values)
{
    if (!values || !poly) return fail(SFHE_EINVAL, "null argument");
    if (!slots_decode(N, t, poly, values)) return fail(SFHE_EUNSUPPORTED, "N=%u t=%llu", N, (unsigned long long)t);
    return SFHE_OK;
}

extern "C" uint32_t sfhe_rotation_element(uint32_t N, int32_t k)
{
    if (N < 4 || (N & (N - 1))) return 0;
    const int64_t half = N / 2;
    const uint64_t e = (uint64_t)(((k % half) + half) % half);
    uint64_t g = 1;
    for (uint64_t i = 0; i < e; i++) g = g * 3 % (2ULL * N);
    return (uint32_t)g;
}

extern "C" sfhe_status sfhe_encrypt_poly(sfhe_ctx* c, const int64_t* polys, const int32_t* coords, int64_t n,
                                         uint64_t matrix_id, uint64_t* ct, void* stream)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!polys || !coords || !ct) return fail(SFHE_EINVAL, "null argument");
    cudaStream_t s = as_stream(stream);
    const size_t N = c->rc.N;
    long long* d_polys = nullptr;
    int* d_coords = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&d_polys, n * N * sizeof(long long), s));
    CUDA_TRY(cudaMallocAsync((void**)&d_coords, n * 2 * sizeof(int), s));
    CUDA_TRY(cudaMemcpyAsync(d_polys, polys, n * N * sizeof(long long), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_coords, coords, n * 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_encrypt_poly(c->rc, c->d_s, d_polys, d_coords, n, matrix_id, ct, c->d_err, s);
    cudaFreeAsync(d_polys, s);
    cudaFreeAsync(d_coords, s);
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "encrypt_poly: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_decrypt_poly(sfhe_ctx* c, const uint64_t* ct, int64_t n, int64_t* out, void* stream)
{
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!ct || !out) return fail(SFHE_EINVAL, "null argument");
    cudaStream_t s = as_stream(stream);
    u64* w = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&w, (size_t)n * c->rc.L * c->rc.N * 8, s));
    cudaError_t e = launch_decrypt_poly(c->rc, c->d_s, ct, n, w, (long long*)out, s);
    cudaFreeAsync(w, s);
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "decrypt_poly: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

static size_t key_words(const RnsConsts& rc) { return (size_t)rc.L * 2 * rc.L * rc.N; }

extern "C" sfhe_status sfhe_galois_keygen(sfhe_ctx* c, uint32_t g, uint64_t* key, uint64_t* key_sh, void* stream)
{
    if (!c || !key || !key_sh) return fail(SFHE_EINVAL, "null argument");
    if (!(g & 1) || g >= 2 * c->rc.N) return fail(SFHE_EINVAL, "g must be odd and below 2N");
    cudaError_t e = launch_galois_keygen(c->rc, c->d_s, g, key, key_sh, c->d_err, as_stream(stream));
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "galois keygen: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_rotate_workspace_size(const sfhe_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    *bytes = rotate_work_words(c->rc) * 8;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_rotate(sfhe_ctx* c, const uint64_t* in, int64_t n, uint32_t g, const uint64_t* key,
                                   const uint64_t* key_sh, uint64_t* out, void* work, size_t work_bytes, void* stream)
{
    Range range("sfhe_rotate");
    if (!c) return fail(SFHE_EINVAL, "null context");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!in || !key || !key_sh || !out || !work) return fail(SFHE_EINVAL, "null argument");
    if (in == out) return fail(SFHE_EINVAL, "in and out must not overlap");
    if (!(g & 1) || g >= 2 * c->rc.N) return fail(SFHE_EINVAL, "g must be odd and below 2N");
    if (work_bytes < rotate_work_words(c->rc) * 8) return fail(SFHE_ENOMEM, "rotation workspace too small");
    const size_t ctw = (size_t)2 * c->rc.L * c->rc.N;
    // as many ciphertexts per batched key switch as the workspace holds
    const long long batch = (long long)(work_bytes / (rotate_work_words(c->rc) * 8));
    cudaError_t e = launch_rotate_batch(c->rc, in, ctw, n, g, key, key_sh, out, ctw, (u64*)work,
                                        std::min<long long>(batch, 4096), as_stream(stream));
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "rotate: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_plain_ntt(sfhe_ctx* c, const int64_t* poly, uint64_t* pt, void* stream)
{
    if (!c || !poly || !pt) return fail(SFHE_EINVAL, "null argument");
    const RnsConsts& rc = c->rc;
    const size_t N = rc.N, L = rc.L;
    std::vector<u64> h(L * N);
    const int64_t t = (int64_t)rc.t;
    for (size_t k = 0; k < N; k++) {
        int64_t v = poly[k] % t;
        if (v < 0) v += t;
        if (v > t / 2) v -= t;  // centred representative
        for (size_t i = 0; i < L; i++) h[i * N + k] = v >= 0 ? (u64)v : rc.m[i].q - (u64)(-v);
    }
    cudaStream_t s = as_stream(stream);
    u64* d = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&d, L * N * 8, s));
    CUDA_TRY(cudaMemcpyAsync(d, h.data(), L * N * 8, cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_ntt(rc, false, d, L * N, 0, pt, L * N, 0, 0, (int)L, 1, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "plain ntt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_mul_plain(sfhe_ctx* c, uint64_t* ct, int64_t n, const uint64_t* pt, void* stream)
{
    if (!c || (n > 0 && (!ct || !pt))) return fail(SFHE_EINVAL, "null argument");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    cudaError_t e = n ? launch_mul_plain(c->rc, ct, n, pt, as_stream(stream)) : cudaSuccess;
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "mul_plain: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_add(sfhe_ctx* c, uint64_t* acc, const uint64_t* x, int64_t n, void* stream)
{
    if (!c || (n > 0 && (!acc || !x))) return fail(SFHE_EINVAL, "null argument");
    if (n < 0) return fail(SFHE_ESHAPE, "negative count");
    cudaError_t e = n ? launch_add_ct(c->rc, acc, x, n, as_stream(stream)) : cudaSuccess;
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "add: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

// rotation keys of one chunk size: left and right rotations by 1 .. c-1
struct sfhe_rotkeys {
    sfhe_ctx* ctx;
    int32_t c;
    u64* d_keys;  // [2 (left, right)][c - 1][2 (key, companions)][key_words]
};

static const u64* rotkey(const sfhe_rotkeys* rk, int right, int off, int sh)
{
    const size_t kw = key_words(rk->ctx->rc);
    return rk->d_keys + (((size_t)right * (rk->c - 1) + (off - 1)) * 2 + sh) * kw;
}

extern "C" sfhe_status sfhe_rotkeys_create(sfhe_ctx* c, int32_t chunk, void* stream, sfhe_rotkeys** out)
{
    if (!c || !out) return fail(SFHE_EINVAL, "null argument");
    *out = nullptr;
    if (chunk < 1 || chunk > (int32_t)(c->rc.N / 2)) return fail(SFHE_ESHAPE, "chunk size outside 1 .. N/2");
    sfhe_rotkeys* rk = new sfhe_rotkeys();
    rk->ctx = c;
    rk->c = chunk;
    rk->d_keys = nullptr;
    const size_t kw = key_words(c->rc), nkeys = 2 * (size_t)(chunk - 1);
    cudaStream_t s = as_stream(stream);
    if (nkeys) {
        if (cudaMalloc((void**)&rk->d_keys, nkeys * 2 * kw * 8) != cudaSuccess) {
            delete rk;
            return fail(SFHE_ENOMEM, "rotation keys: %zu bytes", nkeys * 2 * kw * 8);
        }
        for (int right = 0; right < 2; right++)
            for (int off = 1; off < chunk; off++) {
                const uint32_t g = sfhe_rotation_element(c->rc.N, right ? -off : off);
                cudaError_t e = launch_galois_keygen(c->rc, c->d_s, g, (u64*)rotkey(rk, right, off, 0),
                                                     (u64*)rotkey(rk, right, off, 1), c->d_err, s);
                if (e != cudaSuccess) {
                    cudaFree(rk->d_keys);
                    delete rk;
                    return fail(SFHE_ECUDA, "rotation keys: %s", cudaGetErrorString(e));
                }
            }
    }
    *out = rk;
    return SFHE_OK;
}

extern "C" void sfhe_rotkeys_destroy(sfhe_rotkeys* rk)
{
    if (!rk) return;
    if (rk->d_keys) cudaFree(rk->d_keys);
    delete rk;
}

// ciphertexts per batched key switch of the term-by-term product
static const long long kTermRotBatch = 128;

// The term-by-term chunked product runs its terms in batches of
// term_batch(c): three rounds of the persistent kernel's grid.
static int64_t term_batch(const sfhe_ctx* c)
{
    return 3 * (int64_t)std::max(1, persistent_ctas_per_sm(c->rc) * c->num_sms);
}

// workspace of sfhe_matmul_chunked: the batched rotation scratch; five
// ciphertexts a term (gathered chunks, the two turned operands, the
// product, the placed product); both operands lifted and the lift's
// scratch; the mask; the work list of one batch; the batch's index arrays
struct TermLayout {
    size_t rot, tmp, ra, rb, prod, rr, ea, eb, lift, mask, plan, idx, total, lift_bytes, plan_bytes;
    int64_t n;
};

static sfhe_status term_layout(const sfhe_ctx* c, TermLayout& Lo)
{
    const RnsConsts& rc = c->rc;
    const int64_t n = term_batch(c);
    const size_t ctb = (size_t)2 * rc.L * rc.N * 8, extb = (size_t)2 * rc.K * rc.N * 4;
    Lo.n = n;
    size_t off = 0;
    Lo.rot = off, off += align256(rotate_batch_words(rc, kTermRotBatch) * 8);
    Lo.tmp = off, off += align256((size_t)n * ctb);
    Lo.ra = off, off += align256((size_t)n * ctb);
    Lo.rb = off, off += align256((size_t)n * ctb);
    Lo.prod = off, off += align256((size_t)n * ctb);
    Lo.rr = off, off += align256((size_t)n * ctb);
    Lo.ea = off, off += align256((size_t)n * extb);
    Lo.eb = off, off += align256((size_t)n * extb);
    sfhe_status st = sfhe_lift_workspace_size(c, n, &Lo.lift_bytes);
    if (st != SFHE_OK) return st;
    Lo.lift = off, off += align256(Lo.lift_bytes);
    Lo.mask = off, off += align256((size_t)rc.L * rc.N * 8);
    // the batch's work list: one matmul, n entries of one product each
    sfhe_plan W;
    W.mms.resize(1);
    W.entries.resize((size_t)n);
    W.rowlist.resize((size_t)n);
    int grid = 0;
    size_t stride = 0;
    Lo.plan_bytes = layout_of(c, W, SFHE_EXEC_PERSISTENT, &grid, &stride).total;
    Lo.plan = off, off += align256(Lo.plan_bytes);
    Lo.idx = off, off += align256((size_t)(6 * n + 1) * sizeof(int));
    Lo.total = off;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_chunked_workspace_size(const sfhe_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    TermLayout Lo;
    sfhe_status st = term_layout(c, Lo);
    if (st != SFHE_OK) return st;
    *bytes = Lo.total;
    return SFHE_OK;
}

// descriptors of a chunked matrix's elements for the work-list builder:
// MASK-encoded where a zero mask is given (the products it lists skip those
// elements), DENSE otherwise
static sfhe_matrix_view element_desc(int32_t rows, int32_t cols, const uint8_t* zero, uint64_t* ct, uint32_t* ext);

// The chunked product term by term.  The product sets are the work list of
// the per-element matmul, built by the same builder from element
// descriptors (so both zero masks skip exactly as in the fused form).  Each
// listed product is one short launch sequence: the chunks holding its two
// elements are turned so that the elements sit in slot 0, lifted, multiplied
// and relinearised on the per-product kernels; the term is masked to slot 0,
// turned right to its entry's offset and added into the entry's chunk.
// The chunked product term by term (Alg. 1's placement): for every output
// entry and every product of its product set, the chunks holding the two
// elements are turned so that the elements sit in slot 0, multiplied and
// relinearised, masked to slot 0, turned right to the entry's offset and
// added into the entry's chunk.  The terms are independent until those
// additions, so they run in batches of term_batch(c): the chunks of the
// batch's operands gathered and turned (one batched key switch per offset),
// lifted, multiplied and relinearised by the persistent kernel over a work
// list of one-product entries (each product into its own ciphertext),
// masked, turned right (one batched key switch per offset), and added into
// their chunks in the terms' order.  Every ciphertext is the one the terms
// taken one after another give, limb for limb.
extern "C" sfhe_status sfhe_matmul_chunked(sfhe_ctx* c, const sfhe_rotkeys* rk, int32_t M, int32_t K, int32_t Nc,
                                          const uint64_t* A, const uint64_t* B, uint64_t* C, const uint8_t* a_zero,
                                          const uint8_t* b_zero, void* work, size_t work_bytes, void* stream,
                                          int64_t* products)
{
    Range range("sfhe_matmul_chunked");
    if (!c || !rk || !work) return fail(SFHE_EINVAL, "null argument");
    if (rk->ctx != c) return fail(SFHE_EINVAL, "rotation keys of another context");
    if (M < 0 || K < 0 || Nc < 0) return fail(SFHE_ESHAPE, "negative shape");
    TermLayout Lo;
    sfhe_status st = term_layout(c, Lo);
    if (st != SFHE_OK) return st;
    if (work_bytes < Lo.total) return fail(SFHE_ENOMEM, "chunked workspace of %zu bytes needed, %zu given", Lo.total,
                                           work_bytes);
    const RnsConsts& rc = c->rc;
    const int32_t ch = rk->c;
    const size_t ctw = (size_t)2 * rc.L * rc.N;
    const int64_t nC = ((int64_t)M * Nc + ch - 1) / ch;
    if (nC > 0 && (!A || !B || !C)) return fail(SFHE_EINVAL, "null operand");
    cudaStream_t s = as_stream(stream);
    char* w = (char*)work;
    u64* rot_work = (u64*)(w + Lo.rot);
    u64 *tmp = (u64*)(w + Lo.tmp), *ra = (u64*)(w + Lo.ra), *rb = (u64*)(w + Lo.rb), *prod = (u64*)(w + Lo.prod),
        *rr = (u64*)(w + Lo.rr), *mask = (u64*)(w + Lo.mask);
    u32 *ea = (u32*)(w + Lo.ea), *eb = (u32*)(w + Lo.eb);
    int* d_idx = (int*)(w + Lo.idx);
    {
        std::vector<int64_t> v(rc.N, 0), poly(rc.N);
        v[0] = 1;
        if (!slots_encode((uint32_t)rc.N, rc.t, v.data(), poly.data())) return fail(SFHE_EUNSUPPORTED, "slots");
        st = sfhe_plain_ntt(c, poly.data(), mask, stream);
        if (st != SFHE_OK) return st;
    }
    if (nC > 0) CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)nC * ctw * 8, s));
    // the terms in Alg. 1's order: entry (i, j), then k where neither
    // element is zero
    struct Term {
        int64_t ea, eb, r;
    };
    std::vector<Term> terms;
    for (int32_t i = 0; i < M; i++)
        for (int32_t j = 0; j < Nc; j++)
            for (int32_t k = 0; k < K; k++)
                if (!(a_zero && a_zero[(int64_t)i * K + k]) && !(b_zero && b_zero[(int64_t)k * Nc + j]))
                    terms.push_back({(int64_t)i * K + k, (int64_t)k * Nc + j, (int64_t)i * Nc + j});
    // turn the gathered ciphertexts src[0 .. n) (slots sorted by offset)
    // from `tmp` into out: a turn by 0 is a copy
    auto turn = [&](const std::vector<int>& offs, bool right, u64* out) -> cudaError_t {
        const int64_t n = (int64_t)offs.size();
        for (int64_t q0 = 0; q0 < n;) {
            int64_t q1 = q0;
            while (q1 < n && offs[q1] == offs[q0]) q1++;
            const int off = offs[q0];
            cudaError_t e;
            if (off == 0)
                e = cudaMemcpyAsync(out + q0 * ctw, tmp + q0 * ctw, (size_t)(q1 - q0) * ctw * 8, cudaMemcpyDeviceToDevice,
                                    s);
            else
                e = launch_rotate_batch(rc, tmp + q0 * ctw, ctw, q1 - q0, sfhe_rotation_element(rc.N, right ? -off : off),
                                        rotkey(rk, right, off, 0), rotkey(rk, right, off, 1), out + q0 * ctw, ctw,
                                        rot_work, kTermRotBatch, s);
            if (e != cudaSuccess) return e;
            q0 = q1;
        }
        return cudaSuccess;
    };
    std::vector<int> host_idx;
    for (size_t t0 = 0; t0 < terms.size(); t0 += (size_t)Lo.n) {
        const int n = (int)std::min<size_t>((size_t)Lo.n, terms.size() - t0);
        auto sorted_by = [&](auto off_of) {
            std::vector<int> perm(n);
            for (int p = 0; p < n; p++) perm[p] = p;
            std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return off_of(x) < off_of(y); });
            return perm;
        };
        const auto perm_a = sorted_by([&](int p) { return (int)(terms[t0 + p].ea % ch); });
        const auto perm_b = sorted_by([&](int p) { return (int)(terms[t0 + p].eb % ch); });
        const auto perm_c = sorted_by([&](int p) { return (int)(terms[t0 + p].r % ch); });
        std::vector<int> oa(n), ob(n), oc(n), pos_a(n), pos_b(n), pos_c(n);
        // index region: [0, n) A chunks, [n, 2n) B chunks, [2n, 3n) the
        // placement's sources, [3n, 4n) chunks, [4n, 5n + 1) list offsets,
        // [5n + 1, 6n + 1) the lists
        host_idx.assign((size_t)(6 * n + 1), 0);
        for (int q = 0; q < n; q++) {
            const Term& ta = terms[t0 + perm_a[q]];
            const Term& tb = terms[t0 + perm_b[q]];
            host_idx[q] = (int)(ta.ea / ch), oa[q] = (int)(ta.ea % ch), pos_a[perm_a[q]] = q;
            host_idx[n + q] = (int)(tb.eb / ch), ob[q] = (int)(tb.eb % ch), pos_b[perm_b[q]] = q;
            host_idx[2 * n + q] = perm_c[q], oc[q] = (int)(terms[t0 + perm_c[q]].r % ch), pos_c[perm_c[q]] = q;
        }
        // the chunks the batch adds into, each with its terms in order
        std::vector<int64_t> chunk_ids;
        std::vector<std::vector<int>> by_chunk;
        for (int p = 0; p < n; p++) {
            const int64_t chk = terms[t0 + p].r / ch;
            if (chunk_ids.empty() || chunk_ids.back() != chk) {
                size_t m = 0;
                while (m < chunk_ids.size() && chunk_ids[m] != chk) m++;
                if (m == chunk_ids.size()) chunk_ids.push_back(chk), by_chunk.emplace_back();
                by_chunk[m].push_back(pos_c[p]);
            } else {
                by_chunk.back().push_back(pos_c[p]);
            }
        }
        const int64_t mch = (int64_t)chunk_ids.size();
        int listed = 0;
        for (int64_t m = 0; m < mch; m++) {
            host_idx[3 * n + m] = (int)chunk_ids[m];
            host_idx[4 * n + m] = listed;
            for (int q : by_chunk[m]) host_idx[5 * n + 1 + listed++] = q;
        }
        host_idx[4 * n + mch] = listed;
        CUDA_TRY(cudaMemcpyAsync(d_idx, host_idx.data(), host_idx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        // both operands to slot 0 and lifted
        cudaError_t e = launch_gather_ct(rc, A, d_idx, n, tmp, s);
        if (e == cudaSuccess) e = turn(oa, false, ra);
        if (e == cudaSuccess) e = launch_gather_ct(rc, B, d_idx + n, n, tmp, s);
        if (e == cudaSuccess) e = turn(ob, false, rb);
        if (e != cudaSuccess) return fail(SFHE_ECUDA, "operand turns: %s", cudaGetErrorString(e));
        st = sfhe_lift(c, ra, n, ea, w + Lo.lift, Lo.lift_bytes, stream);
        if (st == SFHE_OK) st = sfhe_lift(c, rb, n, eb, w + Lo.lift, Lo.lift_bytes, stream);
        if (st != SFHE_OK) return st;
        // every product into its own ciphertext: a work list of one-product
        // entries over a matmul whose B "row" is the term (Nc = 1)
        sfhe_plan* P = new_plan(c, SFHE_EXEC_PERSISTENT);
        MmDesc mm;
        memset(&mm, 0, sizeof(mm));
        mm.A_ext = ea, mm.B_ext = eb, mm.C = prod, mm.Nc = 1, mm.group = 1;
        P->mms.push_back(mm);
        P->c_words.push_back((size_t)n * ctw);
        P->products = n;
        for (int p = 0; p < n; p++) {
            Entry en;
            memset(&en, 0, sizeof(en));
            en.mm = 0, en.row = p, en.col = 0, en.count = 1, en.first = p;
            P->entries.push_back(en);
            P->rowlist.push_back(make_int2(pos_a[p], pos_b[p]));
        }
        sfhe_plan* Pf = nullptr;
        st = plan_finish(c, P, SFHE_EXEC_PERSISTENT, w + Lo.plan, Lo.plan_bytes, stream, &Pf);
        if (st != SFHE_OK) return st;
        st = launch_plan(Pf, s);
        sfhe_plan_destroy(Pf);
        if (st != SFHE_OK) return st;
        // mask, turn right to the entries' offsets, add into the chunks
        e = launch_mul_plain(rc, prod, n, mask, s);
        if (e == cudaSuccess) e = launch_gather_ct(rc, prod, d_idx + 2 * n, n, tmp, s);
        if (e == cudaSuccess) e = turn(oc, true, rr);
        if (e == cudaSuccess) e = launch_add_lists(rc, C, rr, d_idx + 3 * n, d_idx + 4 * n, d_idx + 5 * n + 1, mch, s);
        if (e != cudaSuccess) return fail(SFHE_ECUDA, "chunked terms: %s", cudaGetErrorString(e));
    }
    if (products) *products = (int64_t)terms.size();
    return SFHE_OK;
}

// The chunked product with each entry's terms summed before placement.
// Every operand element is brought to slot 0 of its own ciphertext once
// (element q c + o of a matrix is chunk q turned left by o, so one batched
// key switch per offset covers a matrix), which turns the chunked operands
// into per-element ones; the entries' sums of relinearised products then
// run on the persistent kernel over the same work list, and each entry's
// sum is masked to slot 0 and turned right to its offset (one batched key
// switch per offset) before it is added into its chunk.  The terms are
// those of the term-by-term form; only the placement moves from the terms
// to their sum, so the result is another ciphertext with the same
// decryption.
namespace {
// ciphertexts per batched key switch (the rotation scratch holds this many)
const long long kRotBatch = 128;

struct FusedLayout {
    size_t rot, arot, brot, cel, rr, ea, eb, lift, mask, plan, total, lift_bytes, plan_bytes;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

sfhe_status fused_layout(const sfhe_ctx* c, int32_t M, int32_t K, int32_t Nc, int32_t c_chunk, const sfhe_matrix_view& Ad,
                         const sfhe_matrix_view& Bd, FusedLayout& Lo)
{
    const RnsConsts& rc = c->rc;
    const size_t ctb = (size_t)2 * rc.L * rc.N * 8, extb = (size_t)2 * rc.K * rc.N * 4;
    const size_t nA = (size_t)M * K, nB = (size_t)K * Nc, nC = (size_t)M * Nc;
    size_t off = 0;
    Lo.rot = off, off += al256(rotate_batch_words(rc, kRotBatch) * 8);
    Lo.arot = off, off += al256(std::max<size_t>(nA, 1) * ctb);
    Lo.brot = off, off += al256(std::max<size_t>(nB, 1) * ctb);
    Lo.cel = off, off += al256(std::max<size_t>(nC, 1) * ctb);
    Lo.rr = off, off += al256(std::max<size_t>((nC + (size_t)c_chunk - 1) / (size_t)c_chunk, 1) * ctb);
    Lo.ea = off, off += al256(std::max<size_t>(nA, 1) * extb);
    Lo.eb = off, off += al256(std::max<size_t>(nB, 1) * extb);
    sfhe_status st = sfhe_lift_workspace_size(c, (int64_t)std::max(nA, nB), &Lo.lift_bytes);
    if (st != SFHE_OK) return st;
    Lo.lift = off, off += al256(Lo.lift_bytes);
    Lo.mask = off, off += al256((size_t)rc.L * rc.N * 8);
    const bool dl = false;
    st = size_impl(c, 1, &Ad, &Bd, &dl, SFHE_EXEC_PERSISTENT, &Lo.plan_bytes);
    if (st != SFHE_OK) return st;
    Lo.plan = off, off += al256(Lo.plan_bytes);
    Lo.total = off;
    return SFHE_OK;
}

}  // namespace

static sfhe_matrix_view element_desc(int32_t rows, int32_t cols, const uint8_t* zero, uint64_t* ct, uint32_t* ext)
{
    sfhe_matrix_view d;
    memset(&d, 0, sizeof(d));
    d.rows = rows;
    d.cols = cols;
    d.encoding = zero ? SFHE_ENC_MASK : SFHE_ENC_DENSE;
    d.nct = rows * cols;
    d.mask = zero;
    d.ct = ct;
    d.ext = ext;
    return d;
}

extern "C" sfhe_status sfhe_matmul_chunked_fused_workspace_size(const sfhe_ctx* c, int32_t chunk, int32_t M, int32_t K,
                                                                int32_t Nc, const uint8_t* a_zero,
                                                                const uint8_t* b_zero, size_t* bytes)
{
    if (!c || !bytes) return fail(SFHE_EINVAL, "null argument");
    if (M < 0 || K < 0 || Nc < 0 || chunk < 1) return fail(SFHE_ESHAPE, "negative shape or chunk size");
    sfhe_matrix_view Ad = element_desc(M, K, a_zero, (uint64_t*)16, (uint32_t*)16);
    sfhe_matrix_view Bd = element_desc(K, Nc, b_zero, (uint64_t*)16, (uint32_t*)16);
    FusedLayout Lo;
    sfhe_status st = fused_layout(c, M, K, Nc, chunk, Ad, Bd, Lo);
    if (st != SFHE_OK) return st;
    *bytes = Lo.total;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_matmul_chunked_fused(sfhe_ctx* c, const sfhe_rotkeys* rk, int32_t M, int32_t K,
                                                int32_t Nc, const uint64_t* A, const uint64_t* B, uint64_t* C,
                                                const uint8_t* a_zero, const uint8_t* b_zero, void* work,
                                                size_t work_bytes, void* stream, int64_t* products)
{
    Range range("sfhe_matmul_chunked_fused");
    if (!c || !rk || !work) return fail(SFHE_EINVAL, "null argument");
    if (rk->ctx != c) return fail(SFHE_EINVAL, "rotation keys of another context");
    if (M < 0 || K < 0 || Nc < 0) return fail(SFHE_ESHAPE, "negative shape");
    const RnsConsts& rc = c->rc;
    const int32_t ch = rk->c;
    const size_t ctw = (size_t)2 * rc.L * rc.N;
    const int64_t nC = ((int64_t)M * Nc + ch - 1) / ch;
    if (nC > 0 && (!A || !B || !C)) return fail(SFHE_EINVAL, "null operand");
    char* w = (char*)work;
    sfhe_matrix_view Ad = element_desc(M, K, a_zero, nullptr, nullptr), Bd = element_desc(K, Nc, b_zero, nullptr, nullptr);
    Ad.ct = (uint64_t*)16, Ad.ext = (uint32_t*)16, Bd.ct = (uint64_t*)16, Bd.ext = (uint32_t*)16;
    FusedLayout Lo;
    sfhe_status st = fused_layout(c, M, K, Nc, ch, Ad, Bd, Lo);
    if (st != SFHE_OK) return st;
    if (work_bytes < Lo.total) return fail(SFHE_ENOMEM, "workspace of %zu bytes needed, %zu given", Lo.total, work_bytes);
    cudaStream_t s = as_stream(stream);
    u64* rot_work = (u64*)(w + Lo.rot);
    u64 *arot = (u64*)(w + Lo.arot), *brot = (u64*)(w + Lo.brot), *cel = (u64*)(w + Lo.cel), *rr = (u64*)(w + Lo.rr);
    u32 *ea = (u32*)(w + Lo.ea), *eb = (u32*)(w + Lo.eb);
    u64* mask = (u64*)(w + Lo.mask);
    {
        std::vector<int64_t> v(rc.N, 0), poly(rc.N);
        v[0] = 1;
        if (!slots_encode((uint32_t)rc.N, rc.t, v.data(), poly.data())) return fail(SFHE_EUNSUPPORTED, "slots");
        st = sfhe_plain_ntt(c, poly.data(), mask, stream);
        if (st != SFHE_OK) return st;
    }
    // every operand element rotated into slot 0 of its own ciphertext:
    // element q c + o of a matrix is chunk q rotated left by o, so each
    // offset o is one batched key switch over all chunks
    auto place_all = [&](const u64* chunks, int64_t n_el, u64* dst) -> cudaError_t {
        const int64_t nq = (n_el + ch - 1) / ch;
        for (int off = 0; off < ch; off++) {
            const int64_t cnt = off < n_el ? (n_el - off + ch - 1) / ch : 0;  // q with q c + off < n_el
            if (cnt == 0) continue;
            cudaError_t e;
            if (off == 0)
                e = cudaMemcpy2DAsync(dst, (size_t)ch * ctw * 8, chunks, ctw * 8, ctw * 8, (size_t)cnt,
                                      cudaMemcpyDeviceToDevice, s);
            else
                e = launch_rotate_batch(rc, chunks, ctw, cnt, sfhe_rotation_element(rc.N, off), rotkey(rk, 0, off, 0),
                                        rotkey(rk, 0, off, 1), dst + (size_t)off * ctw, (size_t)ch * ctw, rot_work,
                                        kRotBatch, s);
            if (e != cudaSuccess) return e;
        }
        (void)nq;
        return cudaSuccess;
    };
    cudaError_t err = place_all(A, (int64_t)M * K, arot);
    if (err == cudaSuccess) err = place_all(B, (int64_t)K * Nc, brot);
    if (err != cudaSuccess) return fail(SFHE_ECUDA, "rotation: %s", cudaGetErrorString(err));
    // skipped elements are never read: the work list leaves them out
    st = sfhe_lift(c, arot, (int64_t)M * K, ea, w + Lo.lift, Lo.lift_bytes, stream);
    if (st == SFHE_OK) st = sfhe_lift(c, brot, (int64_t)K * Nc, eb, w + Lo.lift, Lo.lift_bytes, stream);
    if (st != SFHE_OK) return st;
    Ad = element_desc(M, K, a_zero, arot, ea);
    Bd = element_desc(K, Nc, b_zero, brot, eb);
    sfhe_matrix_view Cd = element_desc(M, Nc, nullptr, cel, nullptr);
    const bool dl = false;
    sfhe_plan* P = nullptr;
    st = plan_create_impl(c, 1, &Ad, &Bd, &Cd, &dl, SFHE_EXEC_PERSISTENT, w + Lo.plan, Lo.plan_bytes, stream, &P);
    if (st != SFHE_OK) return st;
    st = launch_plan(P, s);
    const int64_t prods = P->products;
    sfhe_plan_destroy(P);
    if (st != SFHE_OK) return st;
    if (nC > 0) CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)nC * ctw * 8, s));
    const int64_t nel = (int64_t)M * Nc;
    cudaError_t e = nel > 0 ? launch_mul_plain(rc, cel, nel, mask, s) : cudaSuccess;
    // entry q c + o goes to slot o of chunk q: one batched rotation right by
    // o over the entries at offset o, then one add into the chunks
    for (int off = 0; e == cudaSuccess && off < ch; off++) {
        const int64_t cnt = off < nel ? (nel - off + ch - 1) / ch : 0;
        if (cnt == 0) continue;
        if (off == 0)
            e = cudaMemcpy2DAsync(rr, ctw * 8, cel, (size_t)ch * ctw * 8, ctw * 8, (size_t)cnt,
                                  cudaMemcpyDeviceToDevice, s);
        else
            e = launch_rotate_batch(rc, cel + (size_t)off * ctw, (size_t)ch * ctw, cnt,
                                    sfhe_rotation_element(rc.N, -off), rotkey(rk, 1, off, 0), rotkey(rk, 1, off, 1),
                                    rr, ctw, rot_work, kRotBatch, s);
        if (e == cudaSuccess) e = launch_add_ct(rc, C, rr, cnt, s);
    }
    if (e != cudaSuccess) return fail(SFHE_ECUDA, "chunked results: %s", cudaGetErrorString(e));
    if (products) *products = prods;
    return SFHE_OK;
}
