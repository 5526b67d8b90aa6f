// ckks.cu -- the CKKS parameter set of the paper (Sec. 3.1: ring degree
// 8192, a coefficient modulus of 50, 40, 40 and 40 bits with a 40-bit
// key-switching prime, scale 2^40) and the chunked matrix product of Alg. 1
// over it: encryption, the ciphertext product with relinearisation,
// rescaling, rotations, the slot-0 mask, additions.
//
// Ciphertexts: [2 (c0, c1)][L][N] uint64, NTT form, canonical residues; a
// ciphertext at level l uses limbs 0 .. l (the primes q_0 .. q_l).  Key
// switching (relinearisation and rotations) uses one digit per prime and the
// extra prime P: a key digit j is (-a_j s + e_j + P g_j w, a_j) over
// q_0 .. q_{L-1}, P with g_j = 1 mod q_j and 0 mod the other q_i, and the
// result of switching d is round(sum_j [d]_{q_j} k_j / P).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sfhe.h"
#include "api_internal.h"
#include "host_math.h"
#include "ntt.cuh"

using sfhe::set_error;

#define CK_MAX 9  // data primes plus the key-switching prime

// An n-bit prime q with mu = floor(2^(2n) / q) for the Barrett reduction of
// values below 2^(2n) (HAC 14.42: the quotient estimate
// floor(floor(x / 2^(n-1)) mu / 2^(n+1)) is at most 2 below floor(x / q)).
struct ModG {
    u64 q;
    u64 mu;
    int n;
    int pad;
};

struct CkksConsts {
    int N, logN, L;  // L data primes; index L is the key-switching prime P
    u64 seed;
    ModG m[CK_MAX];
    const u64* tw;  // [L + 1][4][N]
    ShoupC ninv[CK_MAX], wlast[CK_MAX];
    ShoupC pinv[CK_MAX];               // P^-1 mod q_i
    ShoupC qinv[CK_MAX][CK_MAX];       // q_l^-1 mod q_i (i < l)
    u64 cdt[20];
};

enum { CK_DOM_SECRET = 1, CK_DOM_KSK_A = 9, CK_DOM_KSK_E = 10, CK_DOM_ENC_A = 11, CK_DOM_ENC_E = 12 };

// ------------------------------------------------------------ device math ---
SFHE_DEV u64 barrett_g(u64 hi, u64 lo, const ModG& m)
{
    const u64 xs = (hi << (65 - m.n)) | (lo >> (m.n - 1));
    const u64 ph = mulhi(xs, m.mu), pl = xs * m.mu;
    const u64 qh = (ph << (63 - m.n)) | (pl >> (m.n + 1));
    u64 r = lo - qh * m.q;
    r = csub(r, m.q);
    return csub(r, m.q);
}
SFHE_DEV u64 reduce_g(u64 x, const ModG& m) { return barrett_g(0, x, m); }
SFHE_DEV u64 mulmod_g(u64 a, u64 b, const ModG& m) { return barrett_g(mulhi(a, b), a * b, m); }
// a residue mod p, centred, taken mod q (p, q odd primes)
SFHE_DEV u64 centred_mod(u64 x, u64 p, const ModG& m)
{
    if (x > p / 2) {
        const u64 d = reduce_g(p - x, m);
        return d ? m.q - d : 0;
    }
    return reduce_g(x, m);
}

// the NTT slot whose evaluation point is psi^(g e_i): the automorphism
// X -> X^g permutes the slots of NTT form (slot i at psi^(2 bitrev(i) + 1))
template <int LOGN>
SFHE_DEV int galois_src_ck(int i, u32 g)
{
    constexpr u64 twoN = 2ull << LOGN;
    const u64 e = 2ull * (__brev((unsigned)i) >> (32 - LOGN)) + 1ull;
    const u64 f = (e * g) & (twoN - 1);
    return (int)(__brev((unsigned)((f - 1) >> 1)) >> (32 - LOGN));
}

template <int LOGN>
struct CkGeom {
    using T = NttT<LOGN, 4, Arith64>;
};
template <>
struct CkGeom<6> {
    using T = NttT<6, 2, Arith64>;  // 16 threads at N = 64
};

// ------------------------------------------------------------------ kernels ---
// Batched transforms, block (l, g): polynomial g's limb l, prime
// prime_of(l) = primes[l] (a prime index, L for P).  Forward input: any
// values below 2^(2n) (reduced first); inverse input and every output
// canonical.
struct PrimeList {
    int idx[CK_MAX];
};

template <int LOGN>
__global__ void __launch_bounds__(CkGeom<LOGN>::T::NT) k_ck_ntt(const __grid_constant__ CkksConsts c, int inverse,
                                                                const u64* in, size_t in_gstride, size_t in_lstride,
                                                                u64* out, size_t out_gstride, size_t out_lstride,
                                                                PrimeList pl)
{
    using NT_ = typename CkGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pi = pl.idx[l];
    const ModG m = c.m[pi];
    const u64* src = in + g * in_gstride + (size_t)l * in_lstride;
    u64* dst = out + g * out_gstride + (size_t)l * out_lstride;
    const u64* tw = c.tw + (size_t)pi * 4 * NT_::N;
    u64 x[NT_::R];
    if (!inverse) {
#pragma unroll
        for (int v = 0; v < NT_::R; v++) x[v] = reduce_g(src[NT_::fwd_in_idx(v, tid)], m);
        NT_::forward(x, sm, tid, tw, m.q);
#pragma unroll
        for (int v = 0; v < NT_::R; v++) dst[NT_::run_idx(v, tid)] = reduce_g(x[v], m);
    } else {
#pragma unroll
        for (int v = 0; v < NT_::R; v++) x[v] = src[NT_::run_idx(v, tid)];
        NT_::inverse(x, sm, tid, tw, m.q, c.ninv[pi].w, c.ninv[pi].ws, c.wlast[pi].w, c.wlast[pi].ws);
#pragma unroll
        for (int v = 0; v < NT_::R; v++) dst[NT_::inv_out_idx(v, tid)] = csub(x[v], m.q);
    }
}

// Forward transforms of centred residues: block (t, g): input polynomial g
// is canonical mod prime `from`, its centred representatives are taken mod
// prime pl.idx[t] and transformed.  (The rescale and the division by P.)
template <int LOGN>
__global__ void __launch_bounds__(CkGeom<LOGN>::T::NT) k_ck_ntt_centred(const __grid_constant__ CkksConsts c,
                                                                        int from, const u64* in, size_t in_gstride,
                                                                        u64* out, size_t out_gstride,
                                                                        size_t out_lstride, PrimeList pl)
{
    using NT_ = typename CkGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int t = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pi = pl.idx[t];
    const ModG m = c.m[pi];
    const u64 p = c.m[from].q;
    const u64* src = in + g * in_gstride;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = centred_mod(src[NT_::fwd_in_idx(v, tid)], p, m);
    NT_::forward(x, sm, tid, c.tw + (size_t)pi * 4 * NT_::N, m.q);
    u64* dst = out + g * out_gstride + (size_t)t * out_lstride;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::run_idx(v, tid)] = reduce_g(x[v], m);
}

// the secret: ternary coefficients (stream (seed, 1, 0, 0, 0), slot k) mod
// every prime, NTT form; block (prime t)
template <int LOGN>
__global__ void __launch_bounds__(CkGeom<LOGN>::T::NT) k_ck_secret(const __grid_constant__ CkksConsts c, u64* s_ntt,
                                                                   int* err)
{
    using NT_ = typename CkGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int t = blockIdx.x, tid = threadIdx.x;
    const ModG m = c.m[t];
    const u64 key = sm_key(c.seed, CK_DOM_SECRET, 0, 0, 0);
    int fail = 0;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int s = sample_ternary(key, (u64)NT_::fwd_in_idx(v, tid), &fail);
        x[v] = s >= 0 ? (u64)s : m.q - 1;
    }
    NT_::forward(x, sm, tid, c.tw + (size_t)t * 4 * NT_::N, m.q);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) s_ntt[(size_t)t * NT_::N + NT_::run_idx(v, tid)] = reduce_g(x[v], m);
    if (fail) atomicExch(err, 1);
}

// Key digit j over prime t for w = s^2 (g = 0) or s(X^g), block (t, j):
// a uniform (stream (seed, 9, g, j, 0), slot t N + k), e Gaussian (stream
// (seed, 10, g, j, 0), slot k), b = -a s + e + [t = j] P w; NTT form with
// Shoup companions; layout [L digit][2 (b, a)][L + 1 prime][N].
template <int LOGN>
__global__ void __launch_bounds__(CkGeom<LOGN>::T::NT) k_ck_ksk(const __grid_constant__ CkksConsts c,
                                                                const u64* s_ntt, u32 g, u64* key, u64* key_sh,
                                                                int* err)
{
    using NT_ = typename CkGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int t = blockIdx.x, j = blockIdx.y, tid = threadIdx.x, L = c.L;
    const ModG m = c.m[t];
    const u64* tw = c.tw + (size_t)t * 4 * N;
    const u64 ka = sm_key(c.seed, CK_DOM_KSK_A, (u64)g, (u64)j, 0);
    const u64 ke = sm_key(c.seed, CK_DOM_KSK_E, (u64)g, (u64)j, 0);
    int fail = 0;
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)t * N + k, m.q, &fail);
        const int ev = sample_gauss(ke, (u64)k, c.cdt);
        e[v] = ev >= 0 ? (u64)ev : m.q - (u64)(-ev);
    }
    NT_::forward(a, sm, tid, tw, m.q);
    NT_::forward(e, sm, tid, tw, m.q);
    const u64* s = s_ntt + (size_t)t * N;
    const u64 Pm = reduce_g(c.m[L].q, m);
    const size_t ob = (((size_t)j * 2 + 0) * (L + 1) + t) * N, oa = (((size_t)j * 2 + 1) * (L + 1) + t) * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::run_idx(v, tid);
        const u64 av = reduce_g(a[v], m), ev = reduce_g(e[v], m);
        u64 bv = sub_mod(ev, mulmod_g(av, s[k], m), m.q);
        if (t == j) {
            const u64 w = g == 0 ? mulmod_g(s[k], s[k], m) : s[galois_src_ck<LOGN>(k, g)];
            bv = add_mod(bv, mulmod_g(Pm, w, m), m.q);
        }
        key[ob + k] = bv;
        key[oa + k] = av;
        key_sh[ob + k] = (u64)(((unsigned __int128)bv << 64) / m.q);
        key_sh[oa + k] = (u64)(((unsigned __int128)av << 64) / m.q);
    }
    if (fail) atomicExch(err, 1);
}

// Encryption of integer plaintext polynomials at the top level, block
// (limb i, ciphertext n): c1 = a (stream (seed, 11, id, row, col), slot
// i N + k), c0 = -a s + e + m (e from stream (seed, 12, id, row, col), slot k).
template <int LOGN>
__global__ void __launch_bounds__(CkGeom<LOGN>::T::NT) k_ck_encrypt(const __grid_constant__ CkksConsts c,
                                                                    const u64* s_ntt, const long long* polys,
                                                                    const int* coords, u64 matrix_id, u64* ct, int* err)
{
    using NT_ = typename CkGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int i = blockIdx.x, n = blockIdx.y, tid = threadIdx.x, L = c.L;
    const ModG m = c.m[i];
    const u64* tw = c.tw + (size_t)i * 4 * N;
    const u64 row = (u64)(unsigned)coords[2 * n], col = (u64)(unsigned)coords[2 * n + 1];
    const u64 ka = sm_key(c.seed, CK_DOM_ENC_A, matrix_id, row, col);
    const u64 ke = sm_key(c.seed, CK_DOM_ENC_E, matrix_id, row, col);
    const long long* mp = polys + (size_t)n * N;
    int fail = 0;
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)i * N + k, m.q, &fail);
        const long long em = (long long)sample_gauss(ke, (u64)k, c.cdt) + mp[k];
        const u64 r = reduce_g(em >= 0 ? (u64)em : (u64)(-em), m);
        e[v] = em >= 0 ? r : (r ? m.q - r : 0);
    }
    NT_::forward(a, sm, tid, tw, m.q);
    NT_::forward(e, sm, tid, tw, m.q);
    u64* c0 = ct + ((size_t)n * 2 * L + i) * N;
    u64* c1 = c0 + (size_t)L * N;
    const u64* s = s_ntt + (size_t)i * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::run_idx(v, tid);
        const u64 av = reduce_g(a[v], m);
        c0[k] = sub_mod(reduce_g(e[v], m), mulmod_g(av, s[k], m), m.q);
        c1[k] = av;
    }
    if (fail) atomicExch(err, 1);
}

// Elementwise kernels over limbs 0 .. l of [n][2][L][N] ciphertexts; grid
// (N / 256, l + 1, n).
// d0 = a0 b0, d1 = a0 b1 + a1 b0 into out; d2 = a1 b1 into d2[l'][N]
__global__ void __launch_bounds__(256) k_ck_tensor(const __grid_constant__ CkksConsts c, const u64* a, const u64* b,
                                                   u64* out, u64* d2)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const ModG m = c.m[i];
    const size_t o0 = (size_t)i * N + k, o1 = ((size_t)L + i) * N + k;
    const u64 a0 = a[o0], a1 = a[o1], b0 = b[o0], b1 = b[o1];
    out[o0] = mulmod_g(a0, b0, m);
    out[o1] = add_mod(mulmod_g(a0, b1, m), mulmod_g(a1, b0, m), m.q);
    d2[(size_t)i * N + k] = mulmod_g(a1, b1, m);
}

// Key products of a switch of n polynomials: for target t of the list
// (limbs 0 .. l, then P) and polynomial b,
// u_c[b][t] = sum_{j <= l} U[t][b][j] key_j[c][prime(t)], U the transforms
// of the digits mod the target's prime, key the polynomial's own key; grid
// (N / 256, l + 2, n).
__global__ void __launch_bounds__(256) k_ck_ks_accum(const __grid_constant__ CkksConsts c, int level, int n,
                                                     PrimeList pl, const u64* U, const u64* key0, const u64* key_sh0,
                                                     size_t key_stride, const int* key_of, u64* u)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, t = blockIdx.y, b = blockIdx.z;
    if (k >= N) return;
    // polynomial b's key: key0 + key_of[b] key_stride (key_of NULL: key0)
    const size_t ko = key_of ? (size_t)key_of[b] * key_stride : 0;
    const u64* key = key0 + ko;
    const u64* key_sh = key_sh0 + ko;
    const int pi = pl.idx[t];
    const ModG m = c.m[pi];
    const int nt = level + 2;
    u64 s0 = 0, s1 = 0;
    for (int j = 0; j <= level; j++) {
        const u64 x = U[(((size_t)t * n + b) * (level + 1) + j) * N + k];
        const size_t ob = (((size_t)j * 2 + 0) * (L + 1) + pi) * N + k, oa = (((size_t)j * 2 + 1) * (L + 1) + pi) * N + k;
        s0 += shoup_lazy(x, key[ob], key_sh[ob], m.q);  // < 2q each, at most 9 terms: below 2^64
        s1 += shoup_lazy(x, key[oa], key_sh[oa], m.q);
    }
    u[(((size_t)0 * n + b) * nt + t) * N + k] = reduce_g(s0, m);
    u[(((size_t)1 * n + b) * nt + t) * N + k] = reduce_g(s1, m);
}

// The division of a switch's sums by P: out_c[b][i] (+)= (u_c[b][i] -
// X_c[b][i]) P^-1 mod q_i, X the centred P-limb transformed mod q_i; out_c[b]
// is polynomial c of the ciphertext at out + b out_stride; bit c of
// add_mask: add into it, else store; grid (N / 256, l + 1, 2 n).
__global__ void __launch_bounds__(256) k_ck_moddown(const __grid_constant__ CkksConsts c, int level, int n,
                                                    const u64* u, const u64* X, u64* out, size_t out_stride,
                                                    int add_mask)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const int cc = blockIdx.z / n, b = blockIdx.z - cc * n;
    const ModG m = c.m[i];
    const int nt = level + 2;
    const size_t g = (size_t)cc * n + b;
    const u64 d = sub_mod(u[(g * nt + i) * N + k], X[(g * (level + 1) + i) * N + k], m.q);
    const u64 v = csub(shoup_lazy(d, c.pinv[i].w, c.pinv[i].ws, m.q), m.q);
    u64* o = out + b * out_stride + ((size_t)cc * L + i) * N + k;
    *o = ((add_mask >> cc) & 1) ? add_mod(*o, v, m.q) : v;
}

// Rescale from level l: out_c[i] = (in_c[i] - X_c[i]) q_l^-1 mod q_i, i < l,
// X the centred limb l transformed mod q_i; grid (N / 256, l, 2 n).
__global__ void __launch_bounds__(256) k_ck_rescale(const __grid_constant__ CkksConsts c, int level, const u64* in,
                                                    const u64* X, u64* out)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const size_t pz = blockIdx.z;  // n * 2 + c
    const ModG m = c.m[i];
    const u64 d = sub_mod(in[(pz * L + i) * N + k], X[(pz * level + i) * N + k], m.q);
    out[(pz * L + i) * N + k] = csub(shoup_lazy(d, c.qinv[level][i].w, c.qinv[level][i].ws, m.q), m.q);
}

// slots permuted by X -> X^g, limbs 0 .. l of [n][2][L][N]; grid (N / 256, l + 1, 2 n)
template <int LOGN>
__global__ void __launch_bounds__(256) k_ck_galois(const __grid_constant__ CkksConsts c, const u64* in, u32 g, u64* out)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const size_t base = ((size_t)blockIdx.z * L + i) * N;
    out[base + k] = in[base + galois_src_ck<LOGN>(k, g)];
}

// ct *= pt (NTT form [L][N]) over limbs 0 .. l; grid (N / 256, l + 1, 2 n)
__global__ void __launch_bounds__(256) k_ck_mul_plain(const __grid_constant__ CkksConsts c, u64* ct, const u64* pt)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const size_t o = ((size_t)blockIdx.z * L + i) * N + k;
    ct[o] = mulmod_g(ct[o], pt[(size_t)i * N + k], c.m[i]);
}

// acc += x over limbs 0 .. l; grid (N / 256, l + 1, 2 n)
__global__ void __launch_bounds__(256) k_ck_add(const __grid_constant__ CkksConsts c, u64* acc, const u64* x)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const size_t o = ((size_t)blockIdx.z * L + i) * N + k;
    acc[o] = add_mod(acc[o], x[o], c.m[i].q);
}

// c0 + c1 s over limbs 0 .. l of ciphertext n, NTT form, into v[n][L][N];
// grid (N / 256, l + 1, n)
__global__ void __launch_bounds__(256) k_ck_phase(const __grid_constant__ CkksConsts c, const u64* ct, const u64* s_ntt,
                                                  u64* v)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const size_t n = blockIdx.z;
    const u64 c0 = ct[(n * 2 * L + i) * N + k], c1 = ct[((n * 2 + 1) * L + i) * N + k];
    v[(n * L + i) * N + k] = add_mod(c0, mulmod_g(c1, s_ntt[(size_t)i * N + k], c.m[i]), c.m[i].q);
}

// Gathers of the batched chunked product (ciphertexts [2][L][N], limbs
// 0 .. l).  Slot q of out receives ciphertext src[q] of in with its slots
// permuted by X -> X^g[q] (g = 1: a copy); grid (N / 256, l + 1, 2 n).
template <int LOGN>
__global__ void __launch_bounds__(256) k_ck_galois_gather(const __grid_constant__ CkksConsts c, const u64* in,
                                                          const int* src, const int* gs, u64* out)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const int q = blockIdx.z >> 1, cc = blockIdx.z & 1;
    const u32 g = (u32)gs[q];
    const size_t ctw = (size_t)2 * L * N;
    out[(size_t)q * ctw + ((size_t)cc * L + i) * N + k] =
        in[(size_t)src[q] * ctw + ((size_t)cc * L + i) * N + galois_src_ck<LOGN>(k, g)];
}

// tensor of product p from ra slot pa[p] and rb slot pb[p]: d0, d1 into
// prod[p], d2 into d2[p] ([L][N] each); grid (N / 256, l + 1, n)
__global__ void __launch_bounds__(256) k_ck_tensor_gather(const __grid_constant__ CkksConsts c, const u64* ra,
                                                          const u64* rb, const int* pa, const int* pb, u64* prod,
                                                          u64* d2)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y, p = blockIdx.z;
    if (k >= N) return;
    const size_t ctw = (size_t)2 * L * N;
    const u64* a = ra + (size_t)pa[p] * ctw;
    const u64* b = rb + (size_t)pb[p] * ctw;
    const ModG m = c.m[i];
    const size_t o0 = (size_t)i * N + k, o1 = ((size_t)L + i) * N + k;
    const u64 a0 = a[o0], a1 = a[o1], b0 = b[o0], b1 = b[o1];
    u64* o = prod + (size_t)p * ctw;
    o[o0] = mulmod_g(a0, b0, m);
    o[o1] = add_mod(mulmod_g(a0, b1, m), mulmod_g(a1, b0, m), m.q);
    d2[(size_t)p * L * N + o0] = mulmod_g(a1, b1, m);
}

// C[chunk[j]] += the placed terms list[ptr[j] .. ptr[j+1]) (slots of
// placed); grid (N / 256, l + 1, 2 m)
__global__ void __launch_bounds__(256) k_ck_add_lists(const __grid_constant__ CkksConsts c, u64* C, const u64* placed,
                                                      const int* chunk, const int* ptr, const int* list)
{
    const int N = c.N, L = c.L, k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const int j = blockIdx.z >> 1, cc = blockIdx.z & 1;
    const size_t ctw = (size_t)2 * L * N, o = ((size_t)cc * L + i) * N + k;
    const u64 q = c.m[i].q;
    u64 acc = C[(size_t)chunk[j] * ctw + o];
    for (int t = ptr[j]; t < ptr[j + 1]; t++) acc = add_mod(acc, placed[(size_t)list[t] * ctw + o], q);
    C[(size_t)chunk[j] * ctw + o] = acc;
}

// =================================================================== host ===
struct sfhe_ckks_ctx {
    sfhe_ckks_params params;
    int device;
    CkksConsts cc;
    double scale;
    u64* d_tw;
    u64* d_s;       // [L + 1][N], NTT form
    u64* d_rlk;     // [L][2][L + 1][N] then the companions
    u64* d_rlk_sh;
    int* d_err;
    std::vector<double> cos_tab;  // cos(pi r / N), r < 2N
    std::vector<int64_t> slot_exp;  // 3^j mod 2N
};

struct sfhe_ckks_rotkeys {
    sfhe_ckks_ctx* ctx;
    int32_t c;
    u64* d_keys;  // [2 (left, right)][c - 1][2 (key, companions)][key words]
};

namespace {

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

#define CK_TRY(expr)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return set_error(SFHE_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

size_t key_words(const CkksConsts& c) { return (size_t)c.L * 2 * (c.L + 1) * c.N; }
// work of one key switch: digits [L][N], transforms [L + 1][L][N], sums
// [2][L + 1][N], the P-limb [2][N], its transforms [2][L][N]
size_t ks_words(const CkksConsts& c)
{
    const size_t N = c.N, L = c.L;
    return L * N + (L + 1) * L * N + 2 * (L + 1) * N + 2 * N + 2 * L * N;
}

PrimeList primes_upto(int l, int extra = -1)
{
    PrimeList p;
    for (int i = 0; i < CK_MAX; i++) p.idx[i] = 0;
    for (int i = 0; i <= l; i++) p.idx[i] = i;
    if (extra >= 0) p.idx[l + 1] = extra;
    return p;
}
PrimeList one_prime(int i)
{
    PrimeList p = primes_upto(0);
    p.idx[0] = i;
    return p;
}

template <int LOGN>
size_t ck_smem() { return (size_t)CkGeom<LOGN>::T::SMEM_WORDS * 8; }
template <int LOGN>
int ck_nt() { return CkGeom<LOGN>::T::NT; }

template <typename K>
cudaError_t ck_allow(K* kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define CK_DISPATCH(logN, ...)                       \
    switch (logN) {                                  \
    case 6: { constexpr int LG = 6; __VA_ARGS__; }   \
    case 13: { constexpr int LG = 13; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;           \
    }

cudaError_t ntt(const CkksConsts& c, bool inverse, const u64* in, size_t in_g, size_t in_l, u64* out, size_t out_g,
                size_t out_l, PrimeList pl, int nl, int ng, cudaStream_t s)
{
    if (nl <= 0 || ng <= 0) return cudaSuccess;
    CK_DISPATCH(c.logN, {
        cudaError_t e = ck_allow(k_ck_ntt<LG>, ck_smem<LG>());
        if (e != cudaSuccess) return e;
        k_ck_ntt<LG><<<dim3(nl, ng), ck_nt<LG>(), ck_smem<LG>(), s>>>(c, inverse ? 1 : 0, in, in_g, in_l, out, out_g,
                                                                     out_l, pl);
        return cudaGetLastError();
    });
}

cudaError_t ntt_centred(const CkksConsts& c, int from, const u64* in, size_t in_g, u64* out, size_t out_g,
                        size_t out_l, PrimeList pl, int nt, int ng, cudaStream_t s)
{
    if (nt <= 0 || ng <= 0) return cudaSuccess;
    CK_DISPATCH(c.logN, {
        cudaError_t e = ck_allow(k_ck_ntt_centred<LG>, ck_smem<LG>());
        if (e != cudaSuccess) return e;
        k_ck_ntt_centred<LG><<<dim3(nt, ng), ck_nt<LG>(), ck_smem<LG>(), s>>>(c, from, in, in_g, out, out_g, out_l,
                                                                             pl);
        return cudaGetLastError();
    });
}

dim3 ew_grid(const CkksConsts& c, int y, int z) { return dim3((unsigned)((c.N + 255) / 256), (unsigned)y, (unsigned)z); }

// Key switch of n polynomials d_b = d + b d_stride (NTT form, limbs 0 .. l
// of a [L][N] layout): bit c of add_mask set: add the result into
// polynomial c of the ciphertext at out + b out_stride, else store it
// there.  Polynomial b switches with key + key_of[b] key_stride (its Shoup
// companions at the same offset from key_sh); key_of NULL: every one with
// key.  Scratch w: n ks_words.  One launch per step covers all n.
cudaError_t keyswitch(const CkksConsts& c, const u64* d, size_t d_stride, int n, int l, const u64* key,
                      const u64* key_sh, u64* out, size_t out_stride, int add_mask, u64* w, cudaStream_t s,
                      const int* key_of = nullptr, size_t key_stride = 0)
{
    if (n <= 0) return cudaSuccess;
    const size_t N = c.N, L = c.L, nl = (size_t)l + 1, nt = (size_t)l + 2;
    u64* D = w;                       // [n][l + 1][N]: digits, coefficient form
    u64* U = D + n * L * N;           // [l + 2][n][l + 1][N]: digits mod every target
    u64* u = U + n * (L + 1) * L * N; // [2][n][l + 2][N]: key products
    u64* Pc = u + 2 * n * (L + 1) * N; // [2][n][N]: their P-limbs, coefficient form
    u64* X = Pc + 2 * n * N;          // [2][n][l + 1][N]: the P-limbs centred into every q_i
    cudaError_t e = ntt(c, true, d, d_stride, N, D, nl * N, N, primes_upto(l), l + 1, n, s);
    for (int t = 0; t <= l + 1 && e == cudaSuccess; t++) {
        const int p = t <= l ? t : (int)L;
        e = ntt(c, false, D, N, 0, U + (size_t)t * n * nl * N, N, 0, one_prime(p), 1, (int)(n * nl), s);
    }
    if (e != cudaSuccess) return e;
    k_ck_ks_accum<<<ew_grid(c, l + 2, n), 256, 0, s>>>(c, l, n, primes_upto(l, (int)L), U, key, key_sh, key_stride,
                                                        key_of, u);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the P-limb of every sum to coefficient form, centred into every q_i
    e = ntt(c, true, u + (size_t)(l + 1) * N, nt * N, 0, Pc, N, 0, one_prime((int)L), 1, 2 * n, s);
    if (e == cudaSuccess) e = ntt_centred(c, (int)L, Pc, N, X, nl * N, N, primes_upto(l), l + 1, 2 * n, s);
    if (e != cudaSuccess) return e;
    k_ck_moddown<<<ew_grid(c, l + 1, 2 * n), 256, 0, s>>>(c, l, n, u, X, out, out_stride, add_mask);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ context ---
extern "C" void sfhe_ckks_ctx_destroy(sfhe_ckks_ctx* c)
{
    if (!c) return;
    cudaFree(c->d_tw);
    cudaFree(c->d_s);
    cudaFree(c->d_rlk);
    cudaFree(c->d_err);
    delete c;
}

static sfhe_status ckks_keygen(sfhe_ckks_ctx* c, u32 g, u64* key, u64* key_sh, cudaStream_t s)
{
    auto launch = [&]() -> cudaError_t {
        CK_DISPATCH(c->cc.logN, {
            cudaError_t e = ck_allow(k_ck_ksk<LG>, ck_smem<LG>());
            if (e != cudaSuccess) return e;
            k_ck_ksk<LG><<<dim3(c->cc.L + 1, c->cc.L), ck_nt<LG>(), ck_smem<LG>(), s>>>(c->cc, c->d_s, g, key, key_sh,
                                                                                       c->d_err);
            return cudaGetLastError();
        });
    };
    const cudaError_t e = launch();
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "key generation: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_ctx_create(const sfhe_ckks_params* params, uint64_t seed, sfhe_ckks_ctx** out)
{
    if (!params || !out) return set_error(SFHE_EINVAL, "null argument");
    *out = nullptr;
    const uint32_t N = params->N, L = params->L;
    if (N != 8192 && N != 64) return set_error(SFHE_EUNSUPPORTED, "CKKS ring degree %u (8192, or 64 for tests)", N);
    if (L < 2 || L > CK_MAX - 1) return set_error(SFHE_EUNSUPPORTED, "CKKS data primes %u (2 .. %d)", L, CK_MAX - 1);
    if (params->special_bits < 20 || params->special_bits > 60 || params->log_scale < 10 || params->log_scale > 60)
        return set_error(SFHE_EUNSUPPORTED, "prime or scale size");
    for (uint32_t i = 0; i < L; i++)
        if (params->bits[i] < 20 || params->bits[i] > 60) return set_error(SFHE_EUNSUPPORTED, "prime size %u", params->bits[i]);
    sfhe_ckks_ctx* c = new sfhe_ckks_ctx();
    c->params = *params;
    auto bail = [&](sfhe_status st) {
        sfhe_ckks_ctx_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(set_error(SFHE_ECUDA, "no CUDA device"));
    CkksConsts& cc = c->cc;
    memset(&cc, 0, sizeof(cc));
    cc.N = (int)N;
    cc.logN = N == 8192 ? 13 : 6;
    cc.L = (int)L;
    cc.seed = seed;
    // the primes: per bit size, the largest ones 1 mod 2N not yet taken, in
    // the order of the list; the key-switching prime last
    std::vector<uint64_t> all;
    for (uint32_t i = 0; i <= L; i++) {
        const int bits = (int)(i < L ? params->bits[i] : params->special_bits);
        int before = 0;
        for (uint32_t k = 0; k < i; k++) before += (int)((k < L ? params->bits[k] : params->special_bits) == (uint32_t)bits);
        std::vector<uint64_t> pr;
        if (!sfhe::ntt_primes(N, before + 1, pr, bits)) return bail(set_error(SFHE_EUNSUPPORTED, "not enough primes"));
        all.push_back(pr[before]);
    }
    for (uint32_t i = 0; i <= L; i++) {
        ModG& m = cc.m[i];
        m.q = all[i];
        m.n = 64 - __builtin_clzll(m.q);
        m.mu = (u64)(((unsigned __int128)1 << (2 * m.n)) / m.q);
    }
    auto shoup_c = [](uint64_t w, uint64_t q) {
        ShoupC r;
        r.w = w % q;
        r.ws = (uint64_t)(((unsigned __int128)r.w << 64) / q);
        return r;
    };
    auto invm = [](uint64_t a, uint64_t q) {  // q prime
        unsigned __int128 r = 1, b = a % q;
        for (uint64_t e = q - 2; e; e >>= 1, b = b * b % q)
            if (e & 1) r = r * b % q;
        return (uint64_t)r;
    };
    for (uint32_t i = 0; i < L; i++) {
        cc.pinv[i] = shoup_c(invm(cc.m[L].q % cc.m[i].q, cc.m[i].q), cc.m[i].q);
        for (uint32_t l = i + 1; l < L; l++) cc.qinv[l][i] = shoup_c(invm(cc.m[l].q % cc.m[i].q, cc.m[i].q), cc.m[i].q);
    }
    sfhe::cdt_table(params->sigma > 0 ? params->sigma : 3.2, cc.cdt);
    std::vector<uint64_t> tw((size_t)(L + 1) * 4 * N);
    for (uint32_t i = 0; i <= L; i++) sfhe::twiddles(cc.m[i].q, N, tw.data() + (size_t)i * 4 * N, &cc.ninv[i], &cc.wlast[i]);
    const size_t kw = key_words(cc);
    if (cudaMalloc(&c->d_tw, tw.size() * 8) != cudaSuccess || cudaMalloc(&c->d_s, (size_t)(L + 1) * N * 8) != cudaSuccess ||
        cudaMalloc(&c->d_rlk, 2 * kw * 8) != cudaSuccess || cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess)
        return bail(set_error(SFHE_ENOMEM, "device allocation of the CKKS context failed"));
    c->d_rlk_sh = c->d_rlk + kw;
    cc.tw = c->d_tw;
    if (cudaMemcpy(c->d_tw, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess)
        return bail(set_error(SFHE_ECUDA, "table upload failed"));
    c->scale = ldexp(1.0, (int)params->log_scale);
    c->cos_tab.resize(2 * N);
    for (uint32_t r = 0; r < 2 * N; r++) c->cos_tab[r] = cos(3.14159265358979323846 * (double)r / (double)N);
    c->slot_exp.resize(N / 2);
    int64_t x = 1;
    for (uint32_t j = 0; j < N / 2; j++, x = x * 3 % (2 * (int64_t)N)) c->slot_exp[j] = x;
    cudaError_t e = cudaSuccess;
    auto secret = [&]() -> cudaError_t {
        CK_DISPATCH(cc.logN, {
            cudaError_t ee = ck_allow(k_ck_secret<LG>, ck_smem<LG>());
            if (ee != cudaSuccess) return ee;
            k_ck_secret<LG><<<L + 1, ck_nt<LG>(), ck_smem<LG>(), 0>>>(cc, c->d_s, c->d_err);
            return cudaGetLastError();
        });
    };
    e = secret();
    if (e != cudaSuccess) return bail(set_error(SFHE_ECUDA, "secret: %s", cudaGetErrorString(e)));
    sfhe_status st = ckks_keygen(c, 0, c->d_rlk, c->d_rlk_sh, 0);
    if (st != SFHE_OK) return bail(st);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(set_error(SFHE_ECUDA, "key generation: %s", cudaGetErrorString(e)));
    int err = 0;
    cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) return bail(set_error(SFHE_EDEVICE, "key generation sampler failed"));
    *out = c;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_ctx_primes(const sfhe_ckks_ctx* c, uint64_t* q, uint64_t* p, double* scale)
{
    if (!c) return set_error(SFHE_EINVAL, "null context");
    if (q)
        for (int i = 0; i < c->cc.L; i++) q[i] = c->cc.m[i].q;
    if (p) *p = c->cc.m[c->cc.L].q;
    if (scale) *scale = c->scale;
    return SFHE_OK;
}

// ------------------------------------------------------- encode / decode ---
extern "C" sfhe_status sfhe_ckks_encode(const sfhe_ckks_ctx* c, const double* values, int32_t n, double scale,
                                        int64_t* poly)
{
    if (!c || !poly || (n > 0 && !values)) return set_error(SFHE_EINVAL, "null argument");
    const int N = c->cc.N;
    if (n < 0 || n > N / 2) return set_error(SFHE_ESHAPE, "%d values for %d slots", n, N / 2);
    for (int k = 0; k < N; k++) {
        double acc = 0.0;
        for (int j = 0; j < n; j++) {
            if (values[j] == 0.0) continue;
            acc += values[j] * c->cos_tab[(size_t)((c->slot_exp[j] * (int64_t)k) % (2 * (int64_t)N))];
        }
        const double v = nearbyint(2.0 * scale / (double)N * acc);
        if (!(fabs(v) < 9.0e18)) return set_error(SFHE_EINVAL, "value too large for the scale");
        poly[k] = (int64_t)v;
    }
    return SFHE_OK;
}

namespace {
// the centred integer of residues v[0 .. l] by CRT, as a double
double crt_double(const CkksConsts& cc, const u64* v, size_t stride, int l)
{
    // multiword little-endian, 4 words (the product of at most 4 primes of 60 bits fits)
    const int W = 5;
    u64 Q[W] = {1, 0, 0, 0, 0};
    auto mul_small = [&](u64* a, u64 m) {
        unsigned __int128 carry = 0;
        for (int w = 0; w < W; w++) {
            const unsigned __int128 t = (unsigned __int128)a[w] * m + carry;
            a[w] = (u64)t;
            carry = t >> 64;
        }
    };
    for (int i = 0; i <= l; i++) mul_small(Q, cc.m[i].q);
    u64 acc[W] = {0, 0, 0, 0, 0};
    for (int i = 0; i <= l; i++) {
        const u64 q = cc.m[i].q;
        // Q_i = Q / q (exact division) and its residue mod q
        u64 Qi[W];
        unsigned __int128 rem = 0;
        for (int w = W - 1; w >= 0; w--) {
            const unsigned __int128 cur = (rem << 64) | Q[w];
            Qi[w] = (u64)(cur / q);
            rem = cur % q;
        }
        unsigned __int128 r = 0;
        for (int w = W - 1; w >= 0; w--) r = ((r << 64) | Qi[w]) % q;
        // y = v_i Q_i^-1 mod q
        unsigned __int128 inv = 1, b = r, e = q - 2;
        for (; e; e >>= 1, b = b * b % q)
            if (e & 1) inv = inv * b % q;
        const u64 y = (u64)((unsigned __int128)(v[(size_t)i * stride] % q) * inv % q);
        mul_small(Qi, y);
        unsigned __int128 carry = 0;
        for (int w = 0; w < W; w++) {
            const unsigned __int128 t = (unsigned __int128)acc[w] + Qi[w] + carry;
            acc[w] = (u64)t;
            carry = t >> 64;
        }
    }
    auto geq = [&](const u64* a, const u64* b) {
        for (int w = W - 1; w >= 0; w--)
            if (a[w] != b[w]) return a[w] > b[w];
        return true;
    };
    auto sub = [&](u64* a, const u64* b) {
        u64 br = 0;
        for (int w = 0; w < W; w++) {
            const u64 t = a[w] - b[w] - br;
            br = (a[w] < b[w] || (a[w] == b[w] && br)) ? 1 : 0;
            a[w] = t;
        }
    };
    while (geq(acc, Q)) sub(acc, Q);
    // centred: acc > Q / 2 means acc - Q
    u64 twice[W];
    unsigned __int128 carry = 0;
    for (int w = 0; w < W; w++) {
        const unsigned __int128 t = ((unsigned __int128)acc[w] << 1) + carry;
        twice[w] = (u64)t;
        carry = t >> 64;
    }
    bool neg = geq(twice, Q) && !(std::equal(twice, twice + W, Q));
    if (neg) {
        u64 t[W];
        std::copy(Q, Q + W, t);
        sub(t, acc);
        std::copy(t, t + W, acc);
    }
    double d = 0.0;
    for (int w = W - 1; w >= 0; w--) d = d * 18446744073709551616.0 + (double)acc[w];
    return neg ? -d : d;
}
}  // namespace

extern "C" sfhe_status sfhe_ckks_decode(const sfhe_ckks_ctx* c, const uint64_t* coeff, int32_t level, double scale,
                                        int32_t n, double* values)
{
    if (!c || !coeff || (n > 0 && !values)) return set_error(SFHE_EINVAL, "null argument");
    const int N = c->cc.N;
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (n < 0 || n > N / 2) return set_error(SFHE_ESHAPE, "%d values for %d slots", n, N / 2);
    std::vector<double> m(N);
    for (int k = 0; k < N; k++) m[k] = crt_double(c->cc, coeff + k, (size_t)N, level);
    for (int j = 0; j < n; j++) {
        double acc = 0.0;
        for (int k = 0; k < N; k++) acc += m[k] * c->cos_tab[(size_t)((c->slot_exp[j] * (int64_t)k) % (2 * (int64_t)N))];
        values[j] = acc / scale;
    }
    return SFHE_OK;
}

// ------------------------------------------------------------ operations ---
extern "C" sfhe_status sfhe_ckks_encrypt(sfhe_ckks_ctx* c, const int64_t* polys, const int32_t* coords, int64_t n,
                                         uint64_t matrix_id, uint64_t* ct, void* stream)
{
    if (!c) return set_error(SFHE_EINVAL, "null context");
    if (n < 0) return set_error(SFHE_ESHAPE, "negative count");
    if (n == 0) return SFHE_OK;
    if (!polys || !coords || !ct) return set_error(SFHE_EINVAL, "null argument");
    if (n > 65535) return set_error(SFHE_EUNSUPPORTED, "at most 65535 ciphertexts per call");
    cudaStream_t s = as_stream(stream);
    const size_t N = c->cc.N;
    long long* d_polys = nullptr;
    int* d_coords = nullptr;
    CK_TRY(cudaMallocAsync((void**)&d_polys, n * N * 8, s));
    CK_TRY(cudaMallocAsync((void**)&d_coords, n * 2 * sizeof(int), s));
    CK_TRY(cudaMemcpyAsync(d_polys, polys, n * N * 8, cudaMemcpyHostToDevice, s));
    CK_TRY(cudaMemcpyAsync(d_coords, coords, n * 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    cudaError_t e;
    {
        auto launch = [&]() -> cudaError_t {
            CK_DISPATCH(c->cc.logN, {
                cudaError_t ee = ck_allow(k_ck_encrypt<LG>, ck_smem<LG>());
                if (ee != cudaSuccess) return ee;
                k_ck_encrypt<LG><<<dim3(c->cc.L, (unsigned)n), ck_nt<LG>(), ck_smem<LG>(), s>>>(
                    c->cc, c->d_s, d_polys, d_coords, matrix_id, ct, c->d_err);
                return cudaGetLastError();
            });
        };
        e = launch();
    }
    cudaFreeAsync(d_polys, s);
    cudaFreeAsync(d_coords, s);
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "encrypt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_to_coeff(sfhe_ckks_ctx* c, const uint64_t* ct, int32_t level, int64_t n,
                                          uint64_t* out, void* stream)
{
    if (!c || (n > 0 && (!ct || !out))) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (n < 0 || 2 * n > 65535) return set_error(SFHE_ESHAPE, "count");
    const size_t LN = (size_t)c->cc.L * c->cc.N;
    if (n > 0) CK_TRY(cudaMemsetAsync(out, 0, 2 * n * LN * 8, as_stream(stream)));
    CK_TRY(ntt(c->cc, true, ct, LN, c->cc.N, out, LN, c->cc.N, primes_upto(level), level + 1, (int)(2 * n),
               as_stream(stream)));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_decrypt(sfhe_ckks_ctx* c, const uint64_t* ct, int32_t level, int64_t n, double scale,
                                         int32_t slots, double* values, void* stream)
{
    if (!c || (n > 0 && (!ct || !values))) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (n < 0 || n > 65535) return set_error(SFHE_ESHAPE, "count");
    if (slots < 0 || slots > c->cc.N / 2) return set_error(SFHE_ESHAPE, "slots");
    if (n == 0) return SFHE_OK;
    cudaStream_t s = as_stream(stream);
    const size_t N = c->cc.N, L = c->cc.L;
    u64 *v = nullptr, *vc = nullptr;
    CK_TRY(cudaMallocAsync((void**)&v, n * L * N * 8, s));
    CK_TRY(cudaMallocAsync((void**)&vc, n * L * N * 8, s));
    k_ck_phase<<<ew_grid(c->cc, level + 1, (int)n), 256, 0, s>>>(c->cc, ct, c->d_s, v);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = ntt(c->cc, true, v, L * N, N, vc, L * N, N, primes_upto(level), level + 1, (int)n, s);
    std::vector<u64> h(n * L * N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), vc, h.size() * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(v, s);
    cudaFreeAsync(vc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "decrypt: %s", cudaGetErrorString(e));
    for (int64_t i = 0; i < n; i++) {
        sfhe_status st = sfhe_ckks_decode(c, h.data() + i * L * N, level, scale, slots, values + i * slots);
        if (st != SFHE_OK) return st;
    }
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_workspace_size(const sfhe_ckks_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return set_error(SFHE_EINVAL, "null argument");
    *bytes = ks_words(c->cc) * 8;
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_mul_relin(sfhe_ckks_ctx* c, const uint64_t* a, const uint64_t* b, int32_t level,
                                           uint64_t* out, void* work, size_t work_bytes, void* stream)
{
    if (!c || !a || !b || !out || !work) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (work_bytes < (ks_words(c->cc) + (size_t)c->cc.L * c->cc.N) * 8)
        return set_error(SFHE_ENOMEM, "workspace too small");
    if (out == a || out == b) return set_error(SFHE_EINVAL, "out must not overlap the operands");
    cudaStream_t s = as_stream(stream);
    u64* d2 = (u64*)work;
    u64* w = d2 + (size_t)c->cc.L * c->cc.N;
    k_ck_tensor<<<ew_grid(c->cc, level + 1, 1), 256, 0, s>>>(c->cc, a, b, out, d2);
    CK_TRY(cudaGetLastError());
    CK_TRY(keyswitch(c->cc, d2, 0, 1, level, c->d_rlk, c->d_rlk_sh, out, 0, 3, w, s));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_rescale(sfhe_ckks_ctx* c, const uint64_t* in, int32_t level, int64_t n, uint64_t* out,
                                         void* work, size_t work_bytes, void* stream)
{
    if (!c || (n > 0 && (!in || !out || !work))) return set_error(SFHE_EINVAL, "null argument");
    if (level < 1 || level >= c->cc.L) return set_error(SFHE_EINVAL, "rescale from level %d", level);
    if (n < 0 || 2 * n > 65535) return set_error(SFHE_ESHAPE, "count");
    const size_t N = c->cc.N, L = c->cc.L;
    if (work_bytes < (2 * n * N + 2 * n * (size_t)level * N) * 8) return set_error(SFHE_ENOMEM, "workspace too small");
    if (n == 0) return SFHE_OK;
    cudaStream_t s = as_stream(stream);
    u64* Pc = (u64*)work;        // [2n][N]: limb `level` of every polynomial, coefficient form
    u64* X = Pc + 2 * n * N;     // [2n][level][N]
    CK_TRY(ntt(c->cc, true, in + (size_t)level * N, L * N, 0, Pc, N, 0, one_prime(level), 1, (int)(2 * n), s));
    CK_TRY(ntt_centred(c->cc, level, Pc, N, X, (size_t)level * N, N, primes_upto(level - 1), level, (int)(2 * n), s));
    k_ck_rescale<<<ew_grid(c->cc, level, (int)(2 * n)), 256, 0, s>>>(c->cc, level, in, X, out);
    CK_TRY(cudaGetLastError());
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_rotkeys_create(sfhe_ckks_ctx* c, int32_t chunk, void* stream, sfhe_ckks_rotkeys** out)
{
    if (!c || !out) return set_error(SFHE_EINVAL, "null argument");
    *out = nullptr;
    if (chunk < 1 || chunk > c->cc.N / 2) return set_error(SFHE_ESHAPE, "chunk size outside 1 .. N/2");
    sfhe_ckks_rotkeys* rk = new sfhe_ckks_rotkeys();
    rk->ctx = c;
    rk->c = chunk;
    rk->d_keys = nullptr;
    const size_t kw = key_words(c->cc), nkeys = 2 * (size_t)(chunk - 1);
    if (nkeys) {
        if (cudaMalloc((void**)&rk->d_keys, nkeys * 2 * kw * 8) != cudaSuccess) {
            delete rk;
            return set_error(SFHE_ENOMEM, "rotation keys");
        }
        for (int right = 0; right < 2; right++)
            for (int off = 1; off < chunk; off++) {
                const uint32_t g = sfhe_rotation_element((uint32_t)c->cc.N, right ? -off : off);
                u64* k = rk->d_keys + (((size_t)right * (chunk - 1) + (off - 1)) * 2) * kw;
                sfhe_status st = ckks_keygen(c, g, k, k + kw, as_stream(stream));
                if (st != SFHE_OK) {
                    cudaFree(rk->d_keys);
                    delete rk;
                    return st;
                }
            }
    }
    *out = rk;
    return SFHE_OK;
}

extern "C" void sfhe_ckks_rotkeys_destroy(sfhe_ckks_rotkeys* rk)
{
    if (!rk) return;
    cudaFree(rk->d_keys);
    delete rk;
}

namespace {
// slots of ciphertext `in` turned left by k (right for k < 0) into out (distinct)
sfhe_status rotate_one(sfhe_ckks_ctx* c, const sfhe_ckks_rotkeys* rk, const uint64_t* in, int level, int k,
                       uint64_t* out, u64* w, cudaStream_t s)
{
    const int right = k < 0 ? 1 : 0, off = k < 0 ? -k : k;
    if (off == 0 || off >= rk->c) return set_error(SFHE_EINVAL, "rotation by %d with keys for chunks of %d", k, rk->c);
    const size_t kw = key_words(c->cc), N = c->cc.N, L = c->cc.L;
    const u64* key = rk->d_keys + (((size_t)right * (rk->c - 1) + (off - 1)) * 2) * kw;
    const uint32_t g = sfhe_rotation_element((uint32_t)N, k);
    cudaError_t e = cudaSuccess;
    auto gal = [&]() -> cudaError_t {
        CK_DISPATCH(c->cc.logN, {
            k_ck_galois<LG><<<ew_grid(c->cc, level + 1, 2), 256, 0, s>>>(c->cc, in, g, out);
            return cudaGetLastError();
        });
    };
    e = gal();
    if (e == cudaSuccess) e = keyswitch(c->cc, out + L * N, 0, 1, level, key, key + kw, out, 0, 1, w, s);
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "rotate: %s", cudaGetErrorString(e));
    return SFHE_OK;
}
}  // namespace

extern "C" sfhe_status sfhe_ckks_rotate(sfhe_ckks_ctx* c, const sfhe_ckks_rotkeys* rk, const uint64_t* in, int32_t level,
                                        int32_t k, uint64_t* out, void* work, size_t work_bytes, void* stream)
{
    if (!c || !rk || !in || !out || !work) return set_error(SFHE_EINVAL, "null argument");
    if (rk->ctx != c) return set_error(SFHE_EINVAL, "rotation keys of another context");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (in == out) return set_error(SFHE_EINVAL, "in and out must not overlap");
    if (work_bytes < ks_words(c->cc) * 8) return set_error(SFHE_ENOMEM, "workspace too small");
    return rotate_one(c, rk, in, level, k, out, (u64*)work, as_stream(stream));
}

extern "C" sfhe_status sfhe_ckks_plain_ntt(sfhe_ckks_ctx* c, const int64_t* poly, int32_t level, uint64_t* pt,
                                           void* stream)
{
    if (!c || !poly || !pt) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    const size_t N = c->cc.N;
    std::vector<u64> h((size_t)(level + 1) * N);
    for (int i = 0; i <= level; i++) {
        const u64 q = c->cc.m[i].q;
        for (size_t k = 0; k < N; k++) {
            const int64_t v = poly[k];
            const u64 r = (u64)(v >= 0 ? v : -v) % q;
            h[(size_t)i * N + k] = v >= 0 ? r : (r ? q - r : 0);
        }
    }
    cudaStream_t s = as_stream(stream);
    u64* d = nullptr;
    CK_TRY(cudaMallocAsync((void**)&d, h.size() * 8, s));
    CK_TRY(cudaMemcpyAsync(d, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s));
    cudaError_t e = ntt(c->cc, false, d, 0, N, pt, 0, N, primes_upto(level), level + 1, 1, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // h is released on return
    if (e != cudaSuccess) return set_error(SFHE_ECUDA, "plain ntt: %s", cudaGetErrorString(e));
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_mul_plain(sfhe_ckks_ctx* c, uint64_t* ct, int32_t level, int64_t n, const uint64_t* pt,
                                           void* stream)
{
    if (!c || (n > 0 && (!ct || !pt))) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (n < 0 || 2 * n > 65535) return set_error(SFHE_ESHAPE, "count");
    if (n == 0) return SFHE_OK;
    k_ck_mul_plain<<<ew_grid(c->cc, level + 1, (int)(2 * n)), 256, 0, as_stream(stream)>>>(c->cc, ct, pt);
    CK_TRY(cudaGetLastError());
    return SFHE_OK;
}

extern "C" sfhe_status sfhe_ckks_add(sfhe_ckks_ctx* c, uint64_t* acc, const uint64_t* x, int32_t level, int64_t n,
                                     void* stream)
{
    if (!c || (n > 0 && (!acc || !x))) return set_error(SFHE_EINVAL, "null argument");
    if (level < 0 || level >= c->cc.L) return set_error(SFHE_EINVAL, "level %d", level);
    if (n < 0 || 2 * n > 65535) return set_error(SFHE_ESHAPE, "count");
    if (n == 0) return SFHE_OK;
    k_ck_add<<<ew_grid(c->cc, level + 1, (int)(2 * n)), 256, 0, as_stream(stream)>>>(c->cc, acc, x);
    CK_TRY(cudaGetLastError());
    return SFHE_OK;
}

// ----------------------------------------------- the chunked matrix product ---
namespace {
// products per batch of the chunked product (the workspace holds one batch)
const int kCkBatch = 128;
// ints of the batch's index arrays per product
const int kCkIdx = 8;

struct CkChunkedLayout {
    u64 *ks, *ra, *rb, *prod, *d2, *rs, *mask;
    int* idx;
    size_t words;
};

// ks: kCkBatch key switches; ra, rb: the turned operands (ra later holds the
// placed terms); prod; d2; rs: a batch's rescale; mask; idx: the batch's
// index arrays (kCkIdx ints a product, plus one)
CkChunkedLayout chunked_layout(const CkksConsts& c, u64* base)
{
    const size_t N = c.N, L = c.L, ctw = 2 * L * N, n = kCkBatch;
    CkChunkedLayout Lo;
    u64* w = base;
    Lo.ks = w, w += n * ks_words(c);
    Lo.ra = w, w += n * ctw;
    Lo.rb = w, w += n * ctw;
    Lo.prod = w, w += n * ctw;
    Lo.d2 = w, w += n * L * N;
    Lo.rs = w, w += 2 * n * N + 2 * n * L * N;
    Lo.mask = w, w += L * N;
    Lo.idx = reinterpret_cast<int*>(w), w += (kCkIdx * n + 2) / 2;
    Lo.words = (size_t)(w - base);
    return Lo;
}
}  // namespace

extern "C" sfhe_status sfhe_ckks_matmul_chunked_workspace_size(const sfhe_ckks_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return set_error(SFHE_EINVAL, "null argument");
    *bytes = chunked_layout(c->cc, nullptr).words * 8;
    return SFHE_OK;
}

// The chunked product term by term (the placement of Alg. 1) under CKKS:
// for every output entry and every product of its product set, the two
// chunks holding the elements are turned so that the elements sit in slot
// 0, multiplied and relinearised at the top level and rescaled; the term is
// multiplied by the one-hot slot-0 mask (encoded at the scale of the next
// prime, so that the rescale after it keeps the scale at D^2 / q_top),
// rescaled, turned right to the entry's offset and added into the entry's
// chunk, two levels below the operands.
// The terms are independent until that addition, which is exact modular
// addition, so they run in batches of kCkBatch products, each step of the
// term one batched launch sequence (a turn is one gather and one key switch
// over the batch, each ciphertext with the key of its own offset; a turn by
// 0 is a copy), and each batch's terms are added into their chunks by one
// gather: the result is the same, limb for limb, as taking the terms one
// after another.
extern "C" sfhe_status sfhe_ckks_matmul_chunked(sfhe_ckks_ctx* c, const sfhe_ckks_rotkeys* rk, int32_t M, int32_t K,
                                                int32_t Nc, const uint64_t* A, const uint64_t* B, uint64_t* C,
                                                const uint8_t* a_zero, const uint8_t* b_zero, void* work,
                                                size_t work_bytes, void* stream, int64_t* products,
                                                double* result_scale)
{
    nvtxRangePushA("sfhe_ckks_matmul_chunked");
    struct Pop {
        ~Pop() { nvtxRangePop(); }
    } pop;
    if (!c || !rk || !work) return set_error(SFHE_EINVAL, "null argument");
    if (rk->ctx != c) return set_error(SFHE_EINVAL, "rotation keys of another context");
    if (M < 0 || K < 0 || Nc < 0) return set_error(SFHE_ESHAPE, "negative shape");
    const CkksConsts& cc = c->cc;
    if (cc.L < 3) return set_error(SFHE_EUNSUPPORTED, "the term's two rescales need at least 3 data primes");
    const CkChunkedLayout Lo = chunked_layout(cc, (u64*)work);
    if (work_bytes < Lo.words * 8) return set_error(SFHE_ENOMEM, "workspace too small");
    const int ch = rk->c, top = cc.L - 1;
    const size_t N = cc.N, L = cc.L, ctw = 2 * L * N, kw = key_words(cc);
    const int64_t nC = ((int64_t)M * Nc + ch - 1) / ch;
    if (nC > 0 && (!A || !B || !C)) return set_error(SFHE_EINVAL, "null operand");
    cudaStream_t s = as_stream(stream);
    // the one-hot slot-0 mask at the scale of q_{top-1}
    {
        std::vector<int64_t> poly(N);
        const double one = 1.0;
        sfhe_status st = sfhe_ckks_encode(c, &one, 1, (double)cc.m[top - 1].q, poly.data());
        if (st == SFHE_OK) st = sfhe_ckks_plain_ntt(c, poly.data(), top - 1, Lo.mask, stream);
        if (st != SFHE_OK) return st;
    }
    if (nC > 0) CK_TRY(cudaMemsetAsync(C, 0, (size_t)nC * ctw * 8, s));
    // the terms: entry (i, j) takes the k where neither mask is set
    struct Term {
        int64_t ea, eb, r;
    };
    std::vector<Term> terms;
    for (int32_t i = 0; i < M; i++)
        for (int32_t j = 0; j < Nc; j++)
            for (int32_t k = 0; k < K; k++)
                if (!(a_zero && a_zero[(int64_t)i * K + k]) && !(b_zero && b_zero[(int64_t)k * Nc + j]))
                    terms.push_back({(int64_t)i * K + k, (int64_t)k * Nc + j, (int64_t)i * Nc + j});
    // the rotation keys [2][c - 1][2][kw]: left turns by 1 .. c-1, then right
    // turns; key (right, off) has index right (c - 1) + off - 1
    auto key_index = [&](bool right, int off) { return (right ? 1 : 0) * (ch - 1) + (off - 1); };
    // Turn ciphertexts src[q] of `in` into out's slots q, slot q by offs[q]
    // (left, or right), the slots sorted by offset: one gather for all, then
    // one key switch over the slots with a nonzero offset, each with its own
    // key.  idx: src, then the Galois elements, then the key indices.
    auto turn = [&](const u64* in, const int* d_idx, const std::vector<int>& offs, int level,
                    u64* out) -> cudaError_t {
        const int n = (int)offs.size();
        int z = 0;
        while (z < n && offs[z] == 0) z++;
        cudaError_t e = cudaSuccess;
        CK_DISPATCH(cc.logN, {
            k_ck_galois_gather<LG><<<ew_grid(cc, level + 1, 2 * n), 256, 0, s>>>(cc, in, d_idx, d_idx + n, out);
            e = cudaGetLastError();
            break;
        });
        if (e == cudaSuccess && z < n)
            e = keyswitch(cc, out + (size_t)z * ctw + L * N, ctw, n - z, level, rk->d_keys, rk->d_keys + kw,
                          out + (size_t)z * ctw, ctw, 1, Lo.ks, s, d_idx + 2 * n + z, 2 * kw);
        return e;
    };
    // the index arrays of one turn: src, Galois element, key index per slot
    auto turn_arrays = [&](int* dst, const std::vector<int>& src, const std::vector<int>& offs, bool right) {
        const int n = (int)offs.size();
        for (int q = 0; q < n; q++) {
            dst[q] = src[q];
            dst[n + q] = offs[q] ? (int)sfhe_rotation_element((uint32_t)N, right ? -offs[q] : offs[q]) : 1;
            dst[2 * n + q] = offs[q] ? key_index(right, offs[q]) : 0;
        }
    };
    std::vector<int> host_idx;
    for (size_t t0 = 0; t0 < terms.size(); t0 += kCkBatch) {
        const int n = (int)std::min<size_t>(kCkBatch, terms.size() - t0);
        auto sorted_by = [&](auto off_of) {
            std::vector<int> perm(n);
            for (int p = 0; p < n; p++) perm[p] = p;
            std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return off_of(x) < off_of(y); });
            return perm;
        };
        const auto perm_a = sorted_by([&](int p) { return (int)(terms[t0 + p].ea % ch); });
        const auto perm_b = sorted_by([&](int p) { return (int)(terms[t0 + p].eb % ch); });
        const auto perm_c = sorted_by([&](int p) { return (int)(terms[t0 + p].r % ch); });
        std::vector<int> src_a(n), src_b(n), oa(n), ob(n), pos_a(n), pos_b(n);
        for (int q = 0; q < n; q++) {
            const Term& ta = terms[t0 + perm_a[q]];
            const Term& tb = terms[t0 + perm_b[q]];
            src_a[q] = (int)(ta.ea / ch), oa[q] = (int)(ta.ea % ch), pos_a[perm_a[q]] = q;
            src_b[q] = (int)(tb.eb / ch), ob[q] = (int)(tb.eb % ch), pos_b[perm_b[q]] = q;
        }
        // index region: [0, 3n) the turn of A, [3n, 6n) of B, [6n, 7n) and
        // [7n, 8n) the slots of each product's turned operands
        host_idx.assign((size_t)kCkIdx * kCkBatch + 1, 0);
        turn_arrays(host_idx.data(), src_a, oa, false);
        turn_arrays(host_idx.data() + 3 * n, src_b, ob, false);
        for (int p = 0; p < n; p++) host_idx[6 * n + p] = pos_a[p], host_idx[7 * n + p] = pos_b[p];
        CK_TRY(cudaMemcpyAsync(Lo.idx, host_idx.data(), 8 * (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s));
        // both operands to slot 0, multiply, relinearise
        CK_TRY(turn(A, Lo.idx, oa, top, Lo.ra));
        CK_TRY(turn(B, Lo.idx + 3 * n, ob, top, Lo.rb));
        k_ck_tensor_gather<<<ew_grid(cc, top + 1, n), 256, 0, s>>>(cc, Lo.ra, Lo.rb, Lo.idx + 6 * n, Lo.idx + 7 * n,
                                                                    Lo.prod, Lo.d2);
        CK_TRY(cudaGetLastError());
        CK_TRY(keyswitch(cc, Lo.d2, L * N, n, top, c->d_rlk, c->d_rlk_sh, Lo.prod, ctw, 3, Lo.ks, s));
        // rescale, the slot-0 mask, rescale
        const size_t rs_bytes = (2 * (size_t)n * N + 2 * (size_t)n * L * N) * 8;
        sfhe_status st = sfhe_ckks_rescale(c, Lo.prod, top, n, Lo.prod, Lo.rs, rs_bytes, stream);
        if (st == SFHE_OK) st = sfhe_ckks_mul_plain(c, Lo.prod, top - 1, n, Lo.mask, stream);
        if (st == SFHE_OK) st = sfhe_ckks_rescale(c, Lo.prod, top - 1, n, Lo.prod, Lo.rs, rs_bytes, stream);
        if (st != SFHE_OK) return st;
        // turn right to the entries' offsets (placed terms in ra's slots),
        // then add each chunk's terms into it
        std::vector<int> src_c(n), oc(n), chunk_of, ptr(1, 0), list;
        {
            std::vector<std::vector<int>> by_chunk;
            std::vector<int64_t> chunk_ids;
            for (int q = 0; q < n; q++) {
                src_c[q] = perm_c[q];
                oc[q] = (int)(terms[t0 + perm_c[q]].r % ch);
                const int64_t chk = terms[t0 + perm_c[q]].r / ch;
                size_t m = 0;
                while (m < chunk_ids.size() && chunk_ids[m] != chk) m++;
                if (m == chunk_ids.size()) chunk_ids.push_back(chk), by_chunk.emplace_back();
                by_chunk[m].push_back(q);
            }
            for (size_t m = 0; m < chunk_ids.size(); m++) {
                chunk_of.push_back((int)chunk_ids[m]);
                for (int q : by_chunk[m]) list.push_back(q);
                ptr.push_back((int)list.size());
            }
        }
        const int mch = (int)chunk_of.size();
        // index region again: [0, 3n) the placement turn, [3n, 3n + mch) the
        // chunks, [4n, 4n + mch + 1) list offsets, [5n + 1, 6n + 1) the lists
        host_idx.assign((size_t)kCkIdx * kCkBatch + 1, 0);
        turn_arrays(host_idx.data(), src_c, oc, true);
        for (int m = 0; m < mch; m++) host_idx[3 * n + m] = chunk_of[m];
        for (int m = 0; m <= mch; m++) host_idx[4 * n + m] = ptr[m];
        for (int q = 0; q < n; q++) host_idx[5 * n + 1 + q] = list[q];
        CK_TRY(cudaMemcpyAsync(Lo.idx, host_idx.data(), (6 * (size_t)n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
        CK_TRY(turn(Lo.prod, Lo.idx, oc, top - 2, Lo.ra));
        k_ck_add_lists<<<ew_grid(cc, top - 1, 2 * mch), 256, 0, s>>>(cc, C, Lo.ra, Lo.idx + 3 * n, Lo.idx + 4 * n,
                                                                     Lo.idx + 5 * n + 1);
        CK_TRY(cudaGetLastError());
    }
    if (products) *products = (int64_t)terms.size();
    if (result_scale) *result_scale = c->scale * c->scale / (double)cc.m[top].q;
    return SFHE_OK;
}
