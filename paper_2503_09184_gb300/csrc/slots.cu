// slots.cu -- slot-packed ciphertexts for Alg. 1 with chunk size c > 1
// (Sec. 3.2): encryption of whole plaintext polynomials, decryption of every
// coefficient, Galois keys, rotations (automorphism + key switch),
// ciphertext x plaintext products and additions.
//
// Automorphisms act on the NTT form as a permutation: slot i holds the
// evaluation at psi^e_i, e_i = 2 bitrev(i) + 1, and X -> X^g evaluates the
// input at psi^(g e_i), which is the input's slot with e = g e_i mod 2N.
#include "launch.h"
#include "chunk_launch.h"
#include "launch_util.cuh"

namespace sfhe {

namespace {

// stream domains of the Galois keys (after those of rns.h: secret 1,
// relinearisation key 2 and 3, encryption 4 and 5)
constexpr u64 SFHE_DOM_GAL_A = 6, SFHE_DOM_GAL_E = 7;

#define SLOTS_DISPATCH_LOGN(logN, ...)              \
    switch (logN) {                                 \
    case 12: { constexpr int LG = 12; __VA_ARGS__; } \
    case 13: { constexpr int LG = 13; __VA_ARGS__; } \
    case 14: { constexpr int LG = 14; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;          \
    }

// the input slot whose evaluation point is psi^(g e_i)
template <int LOGN>
SFHE_DEV int galois_src(int i, u32 g)
{
    constexpr u64 twoN = 2ull << LOGN;
    const u64 e = 2ull * (__brev((unsigned)i) >> (32 - LOGN)) + 1ull;
    const u64 f = (e * g) & (twoN - 1);
    return (int)(__brev((unsigned)((f - 1) >> 1)) >> (32 - LOGN));
}

// Galois key for g, block (limb i, digit j), same layout as the
// relinearisation key ([L digit][2 (b, a)][L limb][N], NTT form, Shoup
// companions beside):  b_j = -a_j s + e_j + delta_ij s(X^g),  a_j uniform;
// a_j from the stream (DOM_GAL_A, g, j) at index i N + k (coefficient k),
// e_j from (DOM_GAL_E, g, j) at index k.
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_galois_keygen(const __grid_constant__ RnsConsts c,
                                                                       const u64* s_ntt, u32 g, u64* key, u64* key_sh,
                                                                       int* err)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int i = blockIdx.x, j = blockIdx.y, tid = threadIdx.x, L = c.L;
    const Mod m = c.m[i];
    const u64* tw = c.tw + (size_t)i * 4 * N;
    int fail = 0;
    const u64 ka = sm_key(c.seed, SFHE_DOM_GAL_A, (u64)g, (u64)j, 0);
    const u64 ke = sm_key(c.seed, SFHE_DOM_GAL_E, (u64)g, (u64)j, 0);
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)i * N + k, m.q, &fail);
        e[v] = to_residue(sample_gauss(ke, (u64)k, c.cdt), m.q);
    }
    NT_::forward(a, sm, tid, tw, m.q);
    NT_::forward(e, sm, tid, tw, m.q);
    u64* b_out = key + (((size_t)j * 2 + 0) * L + i) * N;
    u64* a_out = key + (((size_t)j * 2 + 1) * L + i) * N;
    u64* bs_out = key_sh + (((size_t)j * 2 + 0) * L + i) * N;
    u64* as_out = key_sh + (((size_t)j * 2 + 1) * L + i) * N;
    const u64* s = s_ntt + (size_t)i * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::run_idx(v, tid);
        const u64 av = barrett64(a[v], m), ev = barrett64(e[v], m);
        u64 bv = sub_mod(ev, mul_mod(av, s[k], m), m.q);
        if (i == j) bv = add_mod(bv, s[galois_src<LOGN>(k, g)], m.q);
        b_out[k] = bv;
        a_out[k] = av;
        bs_out[k] = (u64)(((unsigned __int128)bv << 64) / m.q);
        as_out[k] = (u64)(((unsigned __int128)av << 64) / m.q);
    }
    if (fail) atomicExch(err, 1);
}

// Secret-key encryption of plaintext polynomials polys[n][N] (every
// coefficient a message digit mod t), block (limb l, ciphertext n):
// c1 = a, c0 = -a s + e + Delta m; stream object (matrix_id, coords[2n],
// coords[2n+1]) as for one value in the constant coefficient.
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_encrypt_poly(const __grid_constant__ RnsConsts c,
                                                                      const u64* s_ntt, const long long* polys,
                                                                      const int* coords, u64 matrix_id, u64* ct, int* err)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, n = blockIdx.y, tid = threadIdx.x, L = c.L;
    const Mod m = c.m[l];
    const u64* tw = c.tw + (size_t)l * 4 * N;
    const u64 row = (u64)(unsigned)coords[2 * n], col = (u64)(unsigned)coords[2 * n + 1];
    const u64 ka = sm_key(c.seed, SFHE_DOM_ENC_A, matrix_id, row, col);
    const u64 ke = sm_key(c.seed, SFHE_DOM_ENC_E, matrix_id, row, col);
    const long long* msg = polys + (size_t)n * N;
    int fail = 0;
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)l * N + k, m.q, &fail);
        long long mt = msg[k] % (long long)c.t;
        if (mt < 0) mt += (long long)c.t;
        e[v] = add_mod(to_residue(sample_gauss(ke, (u64)k, c.cdt), m.q), mul_mod(c.delta_q[l], (u64)mt, m), m.q);
    }
    NT_::forward(a, sm, tid, tw, m.q);
    NT_::forward(e, sm, tid, tw, m.q);
    u64* c0 = ct + ((size_t)n * 2 * L + l) * N;
    u64* c1 = c0 + (size_t)L * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::run_idx(v, tid);
        const u64 av = barrett64(a[v], m);
        c0[k] = sub_mod(barrett64(e[v], m), mul_mod(av, s_ntt[(size_t)l * N + k], m), m.q);
        c1[k] = av;
    }
    if (fail) atomicExch(err, 1);
}

// w[n][l] = c0 + c1 s  (NTT form, canonical)
__global__ void __launch_bounds__(256) k_dec_phase(const __grid_constant__ RnsConsts c, const u64* s_ntt, const u64* ct,
                                                   u64* w)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, l = blockIdx.y, n = blockIdx.z;
    if (k >= N) return;
    const Mod m = c.m[l];
    const u64* c0 = ct + ((size_t)n * 2 * L + l) * N;
    const u64* c1 = c0 + (size_t)L * N;
    w[((size_t)n * L + l) * N + k] = add_mod(csub(c0[k], m.q), mul_mod(c1[k], s_ntt[(size_t)l * N + k], m), m.q);
}

// every coefficient of the message, from v = [c0 + c1 s] in coefficient form
// (canonical residues [n][L][N]): m = [sum_i floor(x~_i t / q_i) +
// round(sum_i y_i / q_i)]_t with x~_i = [v_i (Q/q_i)^-1]_{q_i},
// x~_i t = u_i q_i + y_i, in [0, t)
__global__ void __launch_bounds__(256) k_dec_round(const __grid_constant__ RnsConsts c, const u64* v, long long* out,
                                                   long long n_total)
{
    const int N = c.N, L = c.L;
    const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
    if (idx >= n_total) return;
    const long long n = idx / N;
    const int k = (int)(idx - n * N);
    u64 y[SFHE_MAX_L];
    u64 usum = 0;
    for (int i = 0; i < L; i++) {
        const u64 qi = c.m[i].q;
        const u64 xt = shoup(v[((size_t)n * L + i) * N + k], c.qhat_inv[i], qi);
        u64 quo;
        y[i] = shoup_quot(xt, c.t_q[i], qi, quo);
        usum += quo;
    }
    const u64 kk = crt_round<0>(y, c, L);
    out[idx] = (long long)((usum + kk) % c.t);
}

// out = ct with X -> X^g applied to both polynomials (NTT form: a gather)
template <int LOGN>
__global__ void __launch_bounds__(256) k_galois_apply(const __grid_constant__ RnsConsts c, const u64* in, u32 g, u64* out)
{
    constexpr int N = 1 << LOGN;
    const int k = blockIdx.x * 256 + threadIdx.x;
    const size_t poly = blockIdx.y;  // n * 2L + p L + l
    if (k >= N) return;
    out[poly * N + k] = in[poly * N + galois_src<LOGN>(k, g)];
}

// ct[n][p][l] *= pt[l] (NTT form)
__global__ void __launch_bounds__(256) k_mul_plain(const __grid_constant__ RnsConsts c, u64* ct, const u64* pt)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, l = blockIdx.y;
    if (k >= N) return;
    const Mod m = c.m[l];
    const size_t o = ((size_t)blockIdx.z * L + l) * N + k;  // z = n * 2 + p
    ct[o] = mul_mod(csub(ct[o], m.q), pt[(size_t)l * N + k], m);
}

// acc += x (mod q_l), [n][2][L][N]
__global__ void __launch_bounds__(256) k_add_ct(const __grid_constant__ RnsConsts c, u64* acc, const u64* x)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, l = blockIdx.y;
    if (k >= N) return;
    const u64 q = c.m[l].q;
    const size_t o = ((size_t)blockIdx.z * L + l) * N + k;
    acc[o] = add_mod(csub(acc[o], q), csub(x[o], q), q);
}

// out[q] = in[src[q]] over whole ciphertexts of `words` uint64 each; grid
// (ceil(words / 256), n)
__global__ void __launch_bounds__(256) k_gather_ct(const u64* in, const int* src, size_t words, u64* out)
{
    const size_t w = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (w >= words) return;
    const size_t q = blockIdx.y;
    out[q * words + w] = in[(size_t)src[q] * words + w];
}

// C[chunk[j]] += x[list[t]] for t in ptr[j] .. ptr[j+1], one after another in
// list order (the additions of k_add_ct); grid (N / 256, L, 2 m)
__global__ void __launch_bounds__(256) k_add_lists(const __grid_constant__ RnsConsts c, u64* C, const u64* x,
                                                   const int* chunk, const int* ptr, const int* list)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, l = blockIdx.y;
    if (k >= N) return;
    const int j = blockIdx.z >> 1, p = blockIdx.z & 1;
    const u64 q = c.m[l].q;
    const size_t ctw = (size_t)2 * L * N, o = ((size_t)p * L + l) * N + k;
    u64* a = C + (size_t)chunk[j] * ctw + o;
    u64 acc = *a;
    for (int t = ptr[j]; t < ptr[j + 1]; t++) acc = add_mod(csub(acc, q), csub(x[(size_t)list[t] * ctw + o], q), q);
    *a = acc;
}

// batched key switching: ciphertext z of a batch at its own stride
template <int LOGN>
__global__ void __launch_bounds__(256) k_galois_apply_b(const __grid_constant__ RnsConsts c, const u64* in,
                                                        size_t in_stride, u32 g, u64* out, size_t out_stride)
{
    constexpr int N = 1 << LOGN;
    const int k = blockIdx.x * 256 + threadIdx.x;
    const size_t poly = blockIdx.y;  // p L + l
    if (k >= N) return;
    out[blockIdx.z * out_stride + poly * N + k] = in[blockIdx.z * in_stride + poly * N + galois_src<LOGN>(k, g)];
}

// block (target limb i, source s, ciphertext z): forward NTT of d0 limb i
// (s = 0), of d1 limb i (s = 1), of digit j = s - 2 mod q_i (s >= 2)
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_ks_ntt(const __grid_constant__ RnsConsts c, const u64* D,
                                                                size_t d_stride, u64* U, size_t u_stride)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int i = blockIdx.x, s = blockIdx.y, tid = threadIdx.x, L = c.L;
    const Mod m = c.m[i];
    const u64* Dz = D + blockIdx.z * d_stride;
    const u64* src = s == 0 ? Dz + (size_t)i * N : (s == 1 ? Dz + ((size_t)L + i) * N : Dz + ((size_t)2 * L + (s - 2)) * N);
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = src[NT_::fwd_in_idx(v, tid)];
    NT_::forward(x, sm, tid, c.tw + (size_t)i * 4 * N, m.q);
    u64* dst = U + blockIdx.z * u_stride + ((size_t)s * L + i) * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::run_idx(v, tid)] = barrett64(x[v], m);
}

// out[p][i] = U[p][i] + sum_j U[2+j][i] key[j][p][i]   (p = 0: b, 1: a)
__global__ void __launch_bounds__(256) k_ks_accum(const __grid_constant__ RnsConsts c, const u64* U, size_t u_stride,
                                                  const u64* key, const u64* key_sh, u64* out, size_t out_stride)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const Mod m = c.m[i];
    const u64* Uz = U + blockIdx.z * u_stride;
    for (int p = 0; p < 2; p++) {
        u64 acc = Uz[((size_t)p * L + i) * N + k];
        for (int j = 0; j < L; j++) {
            const size_t ro = (((size_t)j * 2 + p) * L + i) * N + k;
            acc += shoup_lazy(Uz[((size_t)(2 + j) * L + i) * N + k], key[ro], key_sh[ro], m.q);
        }
        out[blockIdx.z * out_stride + ((size_t)p * L + i) * N + k] = barrett64(acc, m);
    }
}

template <int LOGN>
cudaError_t rotate_batch_impl(const RnsConsts& rc, const u64* in, size_t in_stride, long long n, u32 g, const u64* key,
                              const u64* key_sh, u64* out, size_t out_stride, u64* work, cudaStream_t s)
{
    const size_t LN = (size_t)rc.L * rc.N;
    const size_t pw = 2 * LN, dw = 3 * LN, uw = (size_t)(rc.L + 2) * LN;
    u64* P = work;
    u64* D = P + (size_t)n * pw;
    u64* U = D + (size_t)n * dw;
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    k_galois_apply_b<LOGN><<<dim3(bx, 2 * rc.L, (unsigned)n), 256, 0, s>>>(rc, in, in_stride, g, P, pw);
    cudaError_t e = cudaGetLastError();
    // d0 = sigma_g(c0), d1 = 0, d2 = sigma_g(c1), coefficient form (canonical)
    if (e == cudaSuccess) e = launch_ntt(rc, true, P, pw, 0, D, dw, 0, 0, rc.L, n, s);
    if (e == cudaSuccess) e = launch_ntt(rc, true, P, pw, rc.L, D, dw, 2 * rc.L, 0, rc.L, n, s);
    if (e == cudaSuccess) e = cudaMemset2DAsync(D + LN, dw * 8, 0, LN * 8, (size_t)n, s);
    if (e != cudaSuccess) return e;
    e = allow_smem(k_ks_ntt<LOGN>, smem_of<LOGN>());
    if (e != cudaSuccess) return e;
    k_ks_ntt<LOGN><<<dim3(rc.L, rc.L + 2, (unsigned)n), nt_of<LOGN>(), smem_of<LOGN>(), s>>>(rc, D, dw, U, uw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ks_accum<<<dim3(bx, rc.L, (unsigned)n), 256, 0, s>>>(rc, U, uw, key, key_sh, out, out_stride);
    return cudaGetLastError();
}

template <int LOGN>
cudaError_t galois_keygen_impl(const RnsConsts& rc, const u64* s_ntt, u32 g, u64* key, u64* key_sh, int* err,
                               cudaStream_t s)
{
    cudaError_t e = allow_smem(k_galois_keygen<LOGN>, smem_of<LOGN>());
    if (e != cudaSuccess) return e;
    k_galois_keygen<LOGN><<<dim3(rc.L, rc.L), nt_of<LOGN>(), smem_of<LOGN>(), s>>>(rc, s_ntt, g, key, key_sh, err);
    return cudaGetLastError();
}

template <int LOGN>
cudaError_t encrypt_poly_impl(const RnsConsts& rc, const u64* s_ntt, const long long* polys, const int* coords,
                              long long n, u64 matrix_id, u64* ct, int* err, cudaStream_t s)
{
    cudaError_t e = allow_smem(k_encrypt_poly<LOGN>, smem_of<LOGN>());
    if (e != cudaSuccess) return e;
    for (long long n0 = 0; n0 < n; n0 += 65535) {
        const long long cnt = n - n0 < 65535 ? n - n0 : 65535;
        k_encrypt_poly<LOGN><<<dim3(rc.L, (unsigned)cnt), nt_of<LOGN>(), smem_of<LOGN>(), s>>>(
            rc, s_ntt, polys + n0 * rc.N, coords + 2 * n0, matrix_id, ct + (size_t)n0 * 2 * rc.L * rc.N, err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_galois_keygen(const RnsConsts& rc, const u64* s_ntt, u32 g, u64* key, u64* key_sh, int* err,
                                 cudaStream_t s)
{
    SLOTS_DISPATCH_LOGN(rc.logN, return galois_keygen_impl<LG>(rc, s_ntt, g, key, key_sh, err, s));
}

cudaError_t launch_encrypt_poly(const RnsConsts& rc, const u64* s_ntt, const long long* polys, const int* coords,
                                long long n, u64 matrix_id, u64* ct, int* err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    SLOTS_DISPATCH_LOGN(rc.logN, return encrypt_poly_impl<LG>(rc, s_ntt, polys, coords, n, matrix_id, ct, err, s));
}

cudaError_t launch_decrypt_poly(const RnsConsts& rc, const u64* s_ntt, const u64* ct, long long n, u64* w,
                                long long* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    for (long long n0 = 0; n0 < n; n0 += 65535) {
        const long long cnt = n - n0 < 65535 ? n - n0 : 65535;
        k_dec_phase<<<dim3(bx, rc.L, (unsigned)cnt), 256, 0, s>>>(rc, s_ntt, ct + (size_t)n0 * 2 * rc.L * rc.N,
                                                                  w + (size_t)n0 * rc.L * rc.N);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_ntt(rc, true, w, (size_t)rc.L * rc.N, 0, w, (size_t)rc.L * rc.N, 0, 0, rc.L, n, s);
    if (e != cudaSuccess) return e;
    const long long total = n * rc.N;
    k_dec_round<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rc, w, out, total);
    return cudaGetLastError();
}

cudaError_t launch_galois_apply(const RnsConsts& rc, const u64* in, long long n, u32 g, u64* out, cudaStream_t s)
{
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    const long long polys = n * 2 * rc.L;
    for (long long p0 = 0; p0 < polys; p0 += 65535) {
        const long long cnt = polys - p0 < 65535 ? polys - p0 : 65535;
        SLOTS_DISPATCH_LOGN(rc.logN, {
            k_galois_apply<LG><<<dim3(bx, (unsigned)cnt), 256, 0, s>>>(rc, in + (size_t)p0 * rc.N, g,
                                                                        out + (size_t)p0 * rc.N);
            break;
        });
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_mul_plain(const RnsConsts& rc, u64* ct, long long n, const u64* pt, cudaStream_t s)
{
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    for (long long z0 = 0; z0 < 2 * n; z0 += 65535) {
        const long long cnt = 2 * n - z0 < 65535 ? 2 * n - z0 : 65535;
        k_mul_plain<<<dim3(bx, rc.L, (unsigned)cnt), 256, 0, s>>>(rc, ct + (size_t)z0 * rc.L * rc.N, pt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_add_ct(const RnsConsts& rc, u64* acc, const u64* x, long long n, cudaStream_t s)
{
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    for (long long z0 = 0; z0 < 2 * n; z0 += 65535) {
        const long long cnt = 2 * n - z0 < 65535 ? 2 * n - z0 : 65535;
        k_add_ct<<<dim3(bx, rc.L, (unsigned)cnt), 256, 0, s>>>(rc, acc + (size_t)z0 * rc.L * rc.N,
                                                               x + (size_t)z0 * rc.L * rc.N);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t rotate_batch_words(const RnsConsts& rc, long long n) { return (size_t)n * rotate_work_words(rc); }

cudaError_t launch_gather_ct(const RnsConsts& rc, const u64* in, const int* src, long long n, u64* out, cudaStream_t s)
{
    const size_t words = (size_t)2 * rc.L * rc.N;
    for (long long z0 = 0; z0 < n; z0 += 65535) {
        const long long cnt = n - z0 < 65535 ? n - z0 : 65535;
        k_gather_ct<<<dim3((unsigned)((words + 255) / 256), (unsigned)cnt), 256, 0, s>>>(in, src + z0, words,
                                                                                          out + (size_t)z0 * words);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_add_lists(const RnsConsts& rc, u64* C, const u64* x, const int* chunk, const int* ptr,
                             const int* list, long long m, cudaStream_t s)
{
    const unsigned bx = (unsigned)((rc.N + 255) / 256);
    for (long long z0 = 0; z0 < m; z0 += 32767) {
        const long long cnt = m - z0 < 32767 ? m - z0 : 32767;
        k_add_lists<<<dim3(bx, rc.L, (unsigned)(2 * cnt)), 256, 0, s>>>(rc, C, x, chunk + z0, ptr + z0, list);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// n ciphertexts at in + z in_stride -> out + z out_stride (words), in
// batches of at most `batch` (the workspace holds rotate_batch_words(batch))
cudaError_t launch_rotate_batch(const RnsConsts& rc, const u64* in, size_t in_stride, long long n, u32 g,
                                const u64* key, const u64* key_sh, u64* out, size_t out_stride, u64* work,
                                long long batch, cudaStream_t s)
{
    for (long long z0 = 0; z0 < n; z0 += batch) {
        const long long cnt = n - z0 < batch ? n - z0 : batch;
        cudaError_t e;
        SLOTS_DISPATCH_LOGN(rc.logN, {
            e = rotate_batch_impl<LG>(rc, in + z0 * in_stride, in_stride, cnt, g, key, key_sh, out + z0 * out_stride,
                                      out_stride, work, s);
            break;
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Rotation of one ciphertext: P = sigma_g(in) (NTT form); its two
// polynomials back to coefficient form give d0 = sigma_g(c0) and the digits
// D_j = [sigma_g(c1)]_{q_j} (canonical); with d1 = 0 the relinearisation
// kernels then form out = (d0 + sum_j D_j b_j, sum_j D_j a_j) with the
// Galois key in place of the relinearisation key.
// work: P [2][L][N], D [3][L][N], U [(L+2)][L][N] (uint64).
size_t rotate_work_words(const RnsConsts& rc) { return (size_t)(2 + 3 + rc.L + 2) * rc.L * rc.N; }

cudaError_t launch_rotate(const RnsConsts& rc, const u64* in, u32 g, const u64* key, const u64* key_sh, u64* out,
                          u64* work, cudaStream_t s)
{
    const size_t LN = (size_t)rc.L * rc.N;
    u64* P = work;
    u64* D = P + 2 * LN;
    u64* U = D + 3 * LN;
    cudaError_t e = launch_galois_apply(rc, in, 1, g, P, s);
    if (e == cudaSuccess) e = launch_ntt(rc, true, P, LN, 0, D, LN, 0, 0, rc.L, 1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(D + LN, 0, LN * 8, s);
    if (e == cudaSuccess) e = launch_ntt(rc, true, P + LN, LN, 0, D + 2 * LN, LN, 0, 0, rc.L, 1, s);
    if (e == cudaSuccess) e = launch_relin_ntt(rc, D, U, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 2 * LN * 8, s);
    if (e == cudaSuccess) e = launch_relin_accum(rc, U, key, key_sh, out, s);
    return e;
}

}  // namespace sfhe
