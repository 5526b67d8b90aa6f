// kernels.cuh -- device code of the encrypted sparse matmul.
//
// Storage (canonical residues):
//   ciphertext, base Q, NTT form:          [2 (c0, c1)][L][N]  uint64
//   lifted ciphertext, base B, NTT form:   [2][K][N]           uint32 (lane-interleaved, NttT::lane_idx)
//   relinearisation key, base Q, NTT form: [L digit j][2 (b, a)][L limb i][N] uint64 (+ Shoup companions)
// Per product (Alg. 1's inner loop: multiply, relinearise, add):
//   tensor d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 over B (NTT form, 30-bit
//   arithmetic), inverse NTT: the exact integer tensor x in B (|x| < B / 4);
//   exact scale-and-round by t/Q straight from B (the result in Q);
//   digits D_j = [d2]_{q_j}; relinearise with the key; add into C.
#pragma once
#include <type_traits>

#include "ntt.cuh"
#include "worklist.h"

template <int LOGN, int L>
struct Cfg {
    static constexpr int K = tensor_base_size(LOGN, L);
    using NQ = typename NttGeom<LOGN>::T;     // 64-bit transforms (ciphertext primes)
    using NB = typename NttGeom<LOGN>::T32;   // 32-bit transforms (tensor base)
};

// ------------------------------------------------------------------------
// elementwise pieces
// ------------------------------------------------------------------------
// coefficient e of tensor polynomial `poly` (0: a0 b0, 1: a0 b1 + a1 b0,
// 2: a1 b1) times 2^-32 mod b, in [0, 2b) (Montgomery form: the tensor
// stage's inverse NTT multiplies the 2^32 back in with its last-stage
// constants); a, b point at limb k of c0 of lifted ciphertexts, off1 is the
// distance to the same limb of c1.
SFHE_DEV u32 tensor_coeff32(int poly, const u32* __restrict__ a, const u32* __restrict__ b, size_t off1, int e,
                            Mod32 m)
{
    if (poly == 0) return redc32((u64)__ldg(a + e) * __ldg(b + e), m);
    if (poly == 2) return redc32((u64)__ldg(a + off1 + e) * __ldg(b + off1 + e), m);
    return redc32((u64)__ldg(a + e) * __ldg(b + off1 + e) + (u64)__ldg(a + off1 + e) * __ldg(b + e), m);
}

// Exact decision of round(F) + K near a half-integer: with the words of
// Z = sum_k x~_k r_k - v r_B + K Q  (Z = (F + K) Q >= 0), the result is the
// candidate m-1, m or m+1 for which (2c - 1) Q <= 2 Z < (2c + 1) Q.  The
// x~_k are read again from xt32[k * stride] (memory), so that the caller's
// fast path keeps them in registers.
template <int K>
__device__ __noinline__ u64 scale_round_fallback(const u32* xt32, size_t stride, u32 v, u64 m, const RnsConsts& c)
{
    const int W = c.Qwords + 1;
    u64 Z[SFHE_MAX_L + 2], R[SFHE_MAX_L + 2];
    // Z = K Q
    u64 carry = 0;
    for (int w = 0; w <= W; w++) {
        const u64 qw = w < c.Qwords ? c.Qw[w] : 0;
        const u64 lo = qw * (u64)K + carry;
        carry = mulhi(qw, (u64)K) + (lo < carry ? 1 : 0);
        Z[w] = lo;
    }
    // + sum_k x~_k r_k
    for (int k = 0; k < K; k++) {
        const u64 xt = xt32[(size_t)k * stride];
        u64 cy = 0;
        for (int w = 0; w <= W; w++) {
            const u64 rw = w <= SFHE_MAX_L ? c.r_w[k][w] : 0;
            u64 lo = rw * xt, hi = mulhi(rw, xt);
            lo += cy;
            hi += lo < cy ? 1 : 0;
            const u64 s = Z[w] + lo;
            hi += s < lo ? 1 : 0;
            Z[w] = s;
            cy = hi;
        }
    }
    // - v r_B
    {
        u64 cy = 0, borrow = 0;
        for (int w = 0; w <= W; w++) {
            const u64 rw = w <= SFHE_MAX_L ? c.rB_w[w] : 0;
            u64 lo = rw * v, hi = mulhi(rw, (u64)v);
            lo += cy;
            hi += lo < cy ? 1 : 0;
            cy = hi;
            const u64 z = Z[w];
            const u64 d = z - lo - borrow;
            borrow = (z < lo) || (z - lo < borrow) ? 1 : 0;
            Z[w] = d;
        }
    }
    // 2Z
    for (int w = W; w > 0; w--) Z[w] = (Z[w] << 1) | (Z[w - 1] >> 63);
    Z[0] <<= 1;
    // count how many of (2m - 1) Q and (2m + 1) Q are <= 2Z
    u64 res = m - 1;
    for (int s = 0; s < 2; s++) {
        const long long f = 2 * (long long)m - 1 + 2 * s;
        if (f < 0) {
            res += 1;
            continue;
        }
        u64 cyf = 0;
        for (int w = 0; w <= W; w++) {
            const u64 qw = w < c.Qwords ? c.Qw[w] : 0;
            const u64 lo = qw * (u64)f + cyf;
            cyf = mulhi(qw, (u64)f) + (lo < cyf ? 1 : 0);
            R[w] = lo;
        }
        bool ge = true;
        for (int w = W; w >= 0; w--) {
            if (Z[w] != R[w]) {
                ge = Z[w] > R[w];
                break;
            }
        }
        res += ge ? 1 : 0;
    }
    return res;
}

// Exact round(t x / Q) mod q_i for M tensor coefficients x, each given by
// x~_k = [x_k (B/b_k)^-1]_{b_k} at xt32[m][k * stride] (canonical, k < K; the
// tensor stage's inverse NTT produces them):
//   x = sum_k x~_k (B/b_k) - v B,
//   v = round(sum_k x~_k / b_k)  (sum_k x~_k / b_k = v + x / B, |x| / B < 1/4);
//   with t (B/b_k) = alpha_k Q + r_k and t B = alpha_B Q + r_B,
//   t x / Q = sum_k x~_k alpha_k - v alpha_B + F,  F = (sum_k x~_k r_k - v r_B) / Q,
// so round(t x / Q) = sum_k x~_k alpha_k - v alpha_B + round(F).  F + K > 0
// is estimated as G / 2^64 with G = sum_k x~_k rho_k - v rho_B + K 2^64,
// rho = floor(r 2^64 / Q); with the exact rho_k the true value lies in
// (G - K, G + K 2^30) / 2^64,
// so round(F) + K = floor((G + 2^63) / 2^64) unless that interval crosses
// the rounding point, where the decision is taken exactly (Q is odd: no ties).
// Every product is one 32x32-bit multiply into a 64-bit sum without carries:
// G takes rho_k without its low 6 bits, in two 29-bit parts (products below
// 2^59), which widens the band to (G - K, G + K 2^37); the 54-bit
// [alpha_k]_{q_i} is split at bit 27 (below 2^62).  The M coefficients are
// independent; they are interleaved for instruction-level parallelism.
// LAZY: d[m][i] in [0, 3 q_i) (congruent, one Barrett step without the final
// subtractions) instead of canonical.
// The first half of the rounding: the x~_k of M coefficients into registers,
// v and round(F) + K of each.
template <int K, int M>
SFHE_DEV void scale_round_est(const u32* const (&x32)[M], size_t stride, const RnsConsts& c, u32 (&xt)[M][K],
                              u32 (&v)[M], u64 (&mK)[M])
{
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
        for (int m = 0; m < M; m++) xt[m][k] = x32[m][(size_t)k * stride];
    }
#pragma unroll
    for (int m = 0; m < M; m++) {
        v[m] = round_b<K>(xt[m], c);
        u64 s0 = 0, s1 = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
            s0 += (u64)xt[m][k] * c.rho_s[k][0];
            s1 += (u64)xt[m][k] * c.rho_s[k][1];
        }
        // G = s0 2^6 + s1 2^35 + K 2^64 + 2^63 - v rho_B   (mod 2^128)
        u64 ghi = (u64)K + (s0 >> 58) + (s1 >> 29), glo = s0 << 6;
        add128(ghi, glo, s1 << 35);
        add128(ghi, glo, 1ULL << 63);
        const u64 p0 = (u64)v[m] * c.rhoB_lo, p1 = (u64)v[m] * c.rhoB_hi;
        const u64 sub = p0 + (p1 << 32);
        const u64 subhi = (p1 >> 32) + (sub < p0 ? 1 : 0);
        ghi -= subhi + (glo < sub ? 1 : 0);
        glo -= sub;
        mK[m] = ghi;  // round(F) + K, unless glo sits in the uncertainty band
        if (glo < (u64)K || glo >= 0ULL - ((u64)K << 37)) mK[m] = scale_round_fallback<K>(x32[m], stride, v[m], mK[m], c);
    }
}

// The second half: round(t x / Q) mod q_i for the primes i = I0 .. I0+NI-1.
template <int K, int M, int NI, bool LAZY>
SFHE_DEV void scale_round_out(const u32 (&xt)[M][K], const u32 (&v)[M], const u64 (&mK)[M], const RnsConsts& c,
                              int I0, u64 (&d)[M][NI])
{
#pragma unroll
    for (int ii = 0; ii < NI; ii++) {
        const int i = I0 + ii;
#pragma unroll
        for (int m = 0; m < M; m++) {
            // sum_k x~_k alpha_k - v alpha_B + round(F) = shi 2^27 + slo (mod q_i)
            u64 slo = (u64)v[m] * c.negalphaB_q[i] + mK[m] + c.negK_q[i], shi = 0;
#pragma unroll
            for (int k = 0; k < K; k++) {
                slo += (u64)xt[m][k] * c.alpha_q_lo[k][i];
                shi += (u64)xt[m][k] * c.alpha_q_hi[k][i];
            }
            u64 hi = shi >> 37, lo = shi << 27;
            add128(hi, lo, slo);
            d[m][ii] = LAZY ? barrett_lazy(hi, lo, c.m[i]) : barrett(hi, lo, c.m[i]);
        }
    }
}

// Exact round(t x / Q) mod q_i for M tensor coefficients x, each given by
// x~_k = [x_k (B/b_k)^-1]_{b_k} at xt32[m][k * stride] (canonical, k < K; the
// tensor stage's inverse NTT produces them):
//   x = sum_k x~_k (B/b_k) - v B,
//   v = round(sum_k x~_k / b_k)  (sum_k x~_k / b_k = v + x / B, |x| / B < 1/4);
//   with t (B/b_k) = alpha_k Q + r_k and t B = alpha_B Q + r_B,
//   t x / Q = sum_k x~_k alpha_k - v alpha_B + F,  F = (sum_k x~_k r_k - v r_B) / Q,
// so round(t x / Q) = sum_k x~_k alpha_k - v alpha_B + round(F).  F + K > 0
// is estimated as G / 2^64 with G = sum_k x~_k rho_k - v rho_B + K 2^64,
// rho = floor(r 2^64 / Q); with the exact rho_k the true value lies in
// (G - K, G + K 2^30) / 2^64,
// so round(F) + K = floor((G + 2^63) / 2^64) unless that interval crosses
// the rounding point, where the decision is taken exactly (Q is odd: no ties).
// Every product is one 32x32-bit multiply into a 64-bit sum without carries:
// G takes rho_k without its low 6 bits, in two 29-bit parts (products below
// 2^59), which widens the band to (G - K, G + K 2^37); the 54-bit
// [alpha_k]_{q_i} is split at bit 27 (below 2^62).  The M coefficients are
// independent; they are interleaved for instruction-level parallelism.
// LAZY: d[m][i] in [0, 3 q_i) (congruent, one Barrett step without the final
// subtractions) instead of canonical.
template <int L, int K, int M, bool LAZY = false>
SFHE_DEV void scale_round_m(const u32* const (&x32)[M], size_t stride, const RnsConsts& c, u64 (&d)[M][L])
{
    u32 xt[M][K];
    u32 v[M];
    u64 mK[M];
    scale_round_est<K, M>(x32, stride, c, xt, v, mK);
    scale_round_out<K, M, L, LAZY>(xt, v, mK, c, 0, d);
}

template <int L, int K>
SFHE_DEV void scale_round_b(const u32* x32, size_t stride, const RnsConsts& c, u64* d)
{
    const u32* src[1] = {x32};
    u64 dd[1][L];
    scale_round_m<L, K, 1>(src, stride, c, dd);
#pragma unroll
    for (int i = 0; i < L; i++) d[i] = dd[0][i];
}

// ------------------------------------------------------------------------
// generic NTT kernels over batches of polynomials
// ------------------------------------------------------------------------
// Polynomial (g, l): input at in + g * in_gstride + (in_l0 + l) * N, output
// at out + g * out_gstride + (out_l0 + l) * N, prime index prime0 + l of Q.
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_ntt_fwd(const __grid_constant__ RnsConsts c, const u64* in,
                                                                 size_t in_gstride, int in_l0, u64* out,
                                                                 size_t out_gstride, int out_l0, int prime0)
{
    using NT_ = typename NttGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pi = prime0 + l;
    const Mod m = c.m[pi];
    const u64* src = in + g * in_gstride + (size_t)(in_l0 + l) * NT_::N;
    u64* dst = out + g * out_gstride + (size_t)(out_l0 + l) * NT_::N;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = src[NT_::fwd_in_idx(v, tid)];
    NT_::forward(x, sm, tid, c.tw + (size_t)pi * 4 * NT_::N, m.q);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::run_idx(v, tid)] = barrett64(x[v], m);
}

template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_ntt_inv(const __grid_constant__ RnsConsts c, const u64* in,
                                                                 size_t in_gstride, int in_l0, u64* out,
                                                                 size_t out_gstride, int out_l0, int prime0)
{
    using NT_ = typename NttGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pi = prime0 + l;
    const Mod m = c.m[pi];
    const u64* src = in + g * in_gstride + (size_t)(in_l0 + l) * NT_::N;
    u64* dst = out + g * out_gstride + (size_t)(out_l0 + l) * NT_::N;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = csub(src[NT_::run_idx(v, tid)], m.q);
    NT_::inverse(x, sm, tid, c.tw + (size_t)pi * 4 * NT_::N, m.q, c.ninv[pi].w, c.ninv[pi].ws, c.wlast[pi].w,
                 c.wlast[pi].ws);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::inv_out_idx(v, tid)] = csub(x[v], m.q);
}

// Same over the tensor base (32-bit words, prime index into B).
// ILV: the NTT-form side (forward output, inverse input) is stored
// lane-interleaved (NttT::lane_idx), the layout of lifted operands.
template <int LOGN, bool ILV>
__global__ void __launch_bounds__(NttGeom<LOGN>::T32::NT) k_ntt32_fwd(const __grid_constant__ RnsConsts c,
                                                                     const u32* in, size_t in_gstride, int in_l0,
                                                                     u32* out, size_t out_gstride, int out_l0,
                                                                     int prime0)
{
    using NT_ = typename NttGeom<LOGN>::T32;
    extern __shared__ u64 sm64[];
    u32* sm = reinterpret_cast<u32*>(sm64);
    const int l = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pk = prime0 + l;
    const Mod32 m = c.mb[pk];
    const u32* src = in + g * in_gstride + (size_t)(in_l0 + l) * NT_::N;
    u32* dst = out + g * out_gstride + (size_t)(out_l0 + l) * NT_::N;
    u32 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = src[NT_::fwd_in_idx(v, tid)];  // < b: a valid forward input
    NT_::forward(x, sm, tid, c.twb + (size_t)pk * 4 * NT_::N, m.b);
#pragma unroll
    for (int v = 0; v < NT_::R; v++)
        dst[ILV ? NT_::lane_idx(v, tid) : NT_::run_idx(v, tid)] = csub32(csub32(x[v], 2 * m.b), m.b);
}

template <int LOGN, bool ILV>
__global__ void __launch_bounds__(NttGeom<LOGN>::T32::NT) k_ntt32_inv(const __grid_constant__ RnsConsts c,
                                                                     const u32* in, size_t in_gstride, int in_l0,
                                                                     u32* out, size_t out_gstride, int out_l0,
                                                                     int prime0)
{
    using NT_ = typename NttGeom<LOGN>::T32;
    extern __shared__ u64 sm64[];
    u32* sm = reinterpret_cast<u32*>(sm64);
    const int l = blockIdx.x, g = blockIdx.y, tid = threadIdx.x, pk = prime0 + l;
    const Mod32 m = c.mb[pk];
    const u32* src = in + g * in_gstride + (size_t)(in_l0 + l) * NT_::N;
    u32* dst = out + g * out_gstride + (size_t)(out_l0 + l) * NT_::N;
    u32 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = csub32(src[ILV ? NT_::lane_idx(v, tid) : NT_::run_idx(v, tid)], m.b);
    NT_::inverse(x, sm, tid, c.twb + (size_t)pk * 4 * NT_::N, m.b, c.ninv_b[pk].w, c.ninv_b[pk].ws, c.wlast_b[pk].w,
                 c.wlast_b[pk].ws);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::inv_out_idx(v, tid)] = csub32(x[v], m.b);
}

// ------------------------------------------------------------------------
// key generation and encryption
// ------------------------------------------------------------------------
// Secret: ternary coefficients; block l writes s mod q_l in NTT form; block 0
// also writes the coefficients as int8.
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_keygen_secret(const __grid_constant__ RnsConsts c, u64* s_ntt,
                                                                       signed char* s_coeff, int* err)
{
    using NT_ = typename NttGeom<LOGN>::T;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, tid = threadIdx.x;
    const Mod m = c.m[l];
    const u64 key = sm_key(c.seed, SFHE_DOM_SECRET, 0, 0, 0);
    int fail = 0;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int e = NT_::fwd_in_idx(v, tid);
        const int s = sample_ternary(key, (u64)e, &fail);
        if (l == 0) s_coeff[e] = (signed char)s;
        x[v] = to_residue(s, m.q);
    }
    NT_::forward(x, sm, tid, c.tw + (size_t)l * 4 * NT_::N, m.q);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) s_ntt[(size_t)l * NT_::N + NT_::run_idx(v, tid)] = barrett64(x[v], m);
    if (fail) atomicExch(err, 1);
}

// Relinearisation key, block (i limb, j digit):
//   a uniform (coefficient form, NTT'd), e_j Gaussian,
//   b = -a s + e_j + delta_ij s^2  (NTT form), plus Shoup companions.
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_keygen_rlk(const __grid_constant__ RnsConsts c, const u64* s_ntt,
                                                                    u64* rlk, u64* rlk_sh, int* err)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int i = blockIdx.x, j = blockIdx.y, tid = threadIdx.x, L = c.L;
    const Mod m = c.m[i];
    const u64* tw = c.tw + (size_t)i * 4 * N;
    int fail = 0;
    const u64 ka = sm_key(c.seed, SFHE_DOM_RLK_A, (u64)j, 0, 0);
    const u64 ke = sm_key(c.seed, SFHE_DOM_RLK_E, (u64)j, 0, 0);
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)i * N + k, m.q, &fail);
        e[v] = to_residue(sample_gauss(ke, (u64)k, c.cdt), m.q);
    }
    NT_::forward(a, sm, tid, tw, m.q);
    NT_::forward(e, sm, tid, tw, m.q);
    u64* b_out = rlk + (((size_t)j * 2 + 0) * L + i) * N;
    u64* a_out = rlk + (((size_t)j * 2 + 1) * L + i) * N;
    u64* bs_out = rlk_sh + (((size_t)j * 2 + 0) * L + i) * N;
    u64* as_out = rlk_sh + (((size_t)j * 2 + 1) * L + i) * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::run_idx(v, tid);
        const u64 av = barrett64(a[v], m), ev = barrett64(e[v], m);
        const u64 sv = s_ntt[(size_t)i * N + k];
        u64 bv = sub_mod(ev, mul_mod(av, sv, m), m.q);
        if (i == j) bv = add_mod(bv, mul_mod(sv, sv, m), m.q);
        b_out[k] = bv;
        a_out[k] = av;
        bs_out[k] = (u64)(((unsigned __int128)bv << 64) / m.q);
        as_out[k] = (u64)(((unsigned __int128)av << 64) / m.q);
    }
    if (fail) atomicExch(err, 1);
}

// Secret-key encryption of vals[n] (value in the constant coefficient), block
// (limb l, ciphertext n): c1 = a, c0 = -a s + e + Delta [m]_t.  Stream object
// (matrix_id, coords[2n], coords[2n+1]).
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_encrypt(const __grid_constant__ RnsConsts c, const u64* s_ntt,
                                                                 const long long* vals, const int* coords, u64 matrix_id,
                                                                 u64* ct, int* err)
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
    long long mt = vals[n] % (long long)c.t;
    if (mt < 0) mt += (long long)c.t;
    int fail = 0;
    u64 a[NT_::R], e[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) {
        const int k = NT_::fwd_in_idx(v, tid);
        a[v] = sample_uniform(ka, (u64)l * N + k, m.q, &fail);
        u64 ev = to_residue(sample_gauss(ke, (u64)k, c.cdt), m.q);
        if (k == 0) ev = add_mod(ev, mul_mod(c.delta_q[l], (u64)mt, m), m.q);
        e[v] = ev;
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

// Decryption of the constant coefficient: v_l(0) = N^-1 sum_k (c0 + c1 s)[k]
// (NTT slots), then m = [sum_i floor(x~_i t / q_i) + round(sum_i y_i/q_i)]_t
// with x~_i = [v_i (Q/q_i)^-1]_{q_i}, x~_i t = u_i q_i + y_i; centred.
template <int LOGN>
__global__ void __launch_bounds__(256) k_decrypt(const __grid_constant__ RnsConsts c, const u64* s_ntt, const u64* ct,
                                                 long long* out)
{
    constexpr int N = 1 << LOGN;
    __shared__ u64 red[SFHE_MAX_L][8];
    __shared__ u64 v0[SFHE_MAX_L];
    const int n = blockIdx.x, tid = threadIdx.x, L = c.L;
    const int lane = tid & 31, warp = tid >> 5;
    for (int l = 0; l < L; l++) {
        const Mod m = c.m[l];
        const u64* c0 = ct + ((size_t)n * 2 * L + l) * N;
        const u64* c1 = c0 + (size_t)L * N;
        u64 acc = 0;
        for (int k = tid; k < N; k += 256) {
            u64 vv = add_mod(csub(c0[k], m.q), mul_mod(c1[k], s_ntt[(size_t)l * N + k], m), m.q);
            acc = add_mod(acc, vv, m.q);
        }
        for (int o = 16; o > 0; o >>= 1) acc = add_mod(acc, __shfl_xor_sync(0xffffffffu, acc, o), m.q);
        if (lane == 0) red[l][warp] = acc;
    }
    __syncthreads();
    if (tid < L) {
        const Mod m = c.m[tid];
        u64 s = 0;
        for (int w = 0; w < 8; w++) s = add_mod(s, red[tid][w], m.q);
        v0[tid] = shoup(s, c.ninv[tid], m.q);
    }
    __syncthreads();
    if (tid == 0) {
        u64 y[SFHE_MAX_L];
        u64 usum = 0;
        for (int i = 0; i < L; i++) {
            const u64 qi = c.m[i].q;
            const u64 xt = shoup(v0[i], c.qhat_inv[i], qi);
            u64 quo;
            y[i] = shoup_quot(xt, c.t_q[i], qi, quo);
            usum += quo;
        }
        const u64 k = crt_round<0>(y, c, L);
        const long long mt = (long long)((usum + k) % c.t);
        out[n] = mt > (long long)(c.t / 2) ? mt - (long long)c.t : mt;
    }
}

// ------------------------------------------------------------------------
// lift: base Q -> B (centred)
// ------------------------------------------------------------------------
// coefficient form in: [g][L][N] uint64 (canonical), out: [g][K][N] uint32.
//   a = sum_i a~_i (Q/q_i) - v Q,  a~_i = [a_i (Q/q_i)^-1]_{q_i},
//   v = round(sum_i a~_i / q_i) (exact: fixed-point estimate, multiword
//   decision near a half-integer), a mod b_k from the same sum.
template <int L, int K>
__global__ void __launch_bounds__(256) k_lift_extend(const __grid_constant__ RnsConsts c, const u64* in, u32* out,
                                                     int ngroups)
{
    const int N = c.N;
    const size_t idx = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= (size_t)ngroups * N) return;
    const size_t g = idx / N, e = idx % N;
    u64 at[L];
    u32 alo[L], ahi[L];
#pragma unroll
    for (int i = 0; i < L; i++) {
        at[i] = shoup(in[(g * L + i) * N + e], c.qhat_inv[i], c.m[i].q);
        alo[i] = (u32)(at[i] & ((1u << 27) - 1));
        ahi[i] = (u32)(at[i] >> 27);
    }
    const u64 v = crt_round<L>(at, c, L);
#pragma unroll
    for (int k = 0; k < K; k++) {
        u64 V = v * c.negQ_b[k];
#pragma unroll
        for (int i = 0; i < L; i++) V += (u64)alo[i] * c.qhat_b[i][k] + (u64)ahi[i] * c.qhat_b27[i][k];
        out[(g * K + k) * N + e] = reduce64b(V, c.mb[k]);
    }
}

// ------------------------------------------------------------------------
// plain per-product path
// ------------------------------------------------------------------------
// block (k limb of B, poly p): tensor polynomial p mod b_k, inverse NTT,
// coefficient form to T[p][k][N]
template <int LOGN, int L>
__global__ void __launch_bounds__(NttGeom<LOGN>::T32::NT) k_tensor_intt(const __grid_constant__ RnsConsts c, const u32* a,
                                                                       const u32* b, u32* T)
{
    using CF = Cfg<LOGN, L>;
    using NB = typename CF::NB;
    constexpr int N = NB::N, K = CF::K;
    extern __shared__ u64 sm64[];
    u32* sm = reinterpret_cast<u32*>(sm64);
    const int k = blockIdx.x, p = blockIdx.y, tid = threadIdx.x;
    const Mod32 m = c.mb[k];
    const size_t off1 = (size_t)K * N;
    const u32* ak = a + (size_t)k * N;
    const u32* bk = b + (size_t)k * N;
    u32 x[NB::R];
#pragma unroll
    for (int v = 0; v < NB::R; v++) x[v] = tensor_coeff32(p, ak, bk, off1, NB::lane_idx(v, tid), m);
    NB::inverse(x, sm, tid, c.twb + (size_t)k * 4 * N, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws, c.wlast_bx[k].w,
                c.wlast_bx[k].ws);
    u32* dst = T + ((size_t)p * K + k) * N;
#pragma unroll
    for (int v = 0; v < NB::R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[v], m.b);
}

// T [3][K][N] uint32 -> D [3][L][N] uint64 (coefficient form, canonical)
template <int LOGN, int L>
__global__ void __launch_bounds__(128) k_scale_round(const __grid_constant__ RnsConsts c, const u32* T, u64* D)
{
    using CF = Cfg<LOGN, L>;
    constexpr int N = 1 << LOGN, K = CF::K;
    const int e = blockIdx.x * 128 + threadIdx.x, p = blockIdx.y;
    if (e >= N) return;
    u64 d[L];
    scale_round_b<L, K>(T + (size_t)p * K * N + e, N, c, d);
#pragma unroll
    for (int i = 0; i < L; i++) D[((size_t)p * L + i) * N + e] = d[i];
}

// block (target limb i, source s): s = 0: d0_i, 1: d1_i, 2+j: [D_j]_{q_i}
// (digit j = d2 mod q_j); forward NTT into U[s][i][N]
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_relin_ntt(const __grid_constant__ RnsConsts c, const u64* D,
                                                                   u64* U)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int i = blockIdx.x, s = blockIdx.y, tid = threadIdx.x, L = c.L;
    const Mod m = c.m[i];
    const u64* src = s == 0 ? D + (size_t)i * N : (s == 1 ? D + ((size_t)L + i) * N : D + ((size_t)2 * L + (s - 2)) * N);
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = src[NT_::fwd_in_idx(v, tid)];  // < 2^54: fine as lazy input
    NT_::forward(x, sm, tid, c.tw + (size_t)i * 4 * N, m.q);
    u64* dst = U + ((size_t)s * L + i) * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::run_idx(v, tid)] = barrett64(x[v], m);
}

#ifdef SFHE_KERNELS_TU
// C[p][i] += U[p][i] + sum_j U[2+j][i] rlk[j][p][i]   (p = 0: b, 1: a)
__global__ void __launch_bounds__(256) k_relin_accum(const __grid_constant__ RnsConsts c, const u64* U, const u64* rlk,
                                                     const u64* rlk_sh, u64* C)
{
    const int N = c.N, L = c.L;
    const int k = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y;
    if (k >= N) return;
    const Mod m = c.m[i];
    for (int p = 0; p < 2; p++) {
        u64 acc = U[((size_t)p * L + i) * N + k];
        for (int j = 0; j < L; j++) {
            const size_t ro = (((size_t)j * 2 + p) * L + i) * N + k;
            acc += shoup_lazy(U[((size_t)(2 + j) * L + i) * N + k], rlk[ro], rlk_sh[ro], m.q);
        }
        u64* cp = C + ((size_t)p * L + i) * N + k;
        *cp = add_mod(*cp, barrett64(acc, m), m.q);
    }
}

// raw generator words (stream-equality checks against the oracle)
__global__ void k_prng_words(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, u64 idx0, long long n, u64* out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out[t] = sm_word(sm_key(seed, dom, o0, o1, o2), idx0 + (u64)t);
}
#endif

// ------------------------------------------------------------------------
// fused persistent matmul
// ------------------------------------------------------------------------
// Shared-memory plan of the persistent kernel.  Up to N = 8192 the operand
// limbs are staged: four 4N-byte slots (a0, a1, b0, b1 of one tensor-base
// prime) filled by TMA bulk copies behind the exchange buffers of the three
// 32-bit inverse NTTs that run together.  At N = 16384 two slots fit behind
// one exchange buffer: a prime's tensor is formed in four rounds of two
// staged limbs.  The 64-bit NTTs of stage R reuse the bytes from offset 0.
template <int LOGN, int L>
struct PersistentPlan {
    using CF = Cfg<LOGN, L>;
    static constexpr bool STAGED = LOGN <= 13;   // four slots, three polynomials per pass
    static constexpr bool STAGED2 = LOGN == 14;  // two slots, one polynomial per pass
    static constexpr int NPT = STAGED ? 3 : 1;   // polynomials per inverse-NTT pass in stage T
    static constexpr int NSLOT = STAGED ? 4 : 2;
    static constexpr size_t SLOT = (size_t)4 << LOGN;
    static constexpr size_t EXB = ((size_t)NPT * CF::NB::SMEM_WORDS * 4 + 127) & ~(size_t)127;
    static constexpr size_t NQB = (size_t)CF::NQ::SMEM_WORDS * 8;
    static constexpr size_t STAGE_B = EXB + NSLOT * SLOT;
    static constexpr size_t SMEM = (STAGED || STAGED2) ? (NQB > STAGE_B ? NQB : STAGE_B) : NQB;
    static_assert(SMEM <= 227 * 1024 - 256, "shared-memory plan too large");
};

// Tile of the persistent kernel, one per variant V that the run-time tuner
// can pick.  Stage S (the exact scale-and-round): SM coefficients per thread
// at a time (interleaved for instruction-level parallelism) and the output
// primes in chunks of LS (fewer live registers per chunk).  Stage T: the
// code form of the inverse NTT (NttT's FORM).  V = 0 is the default;
// variants 1 and 2 (stage-S tiles) exist for the rings
// persistent_variants() lists, variants 3 and 4 (tile 1 with the lean and
// with the shuffle-stage inverse NTT) at N = 8192, L = 4.
template <int LOGN, int L, int V>
struct PersistentTile {
    static constexpr int K = tensor_base_size(LOGN, L);
    static constexpr int R = NttGeom<LOGN>::T32::R;
    static constexpr int VS = V >= 3 ? 1 : V;  // the stage-S tile
    static constexpr int NTT_FORM = V == 3 ? 1 : (V == 4 ? 2 : 0);
    static constexpr int SMD = (K <= 16 && R <= 16) ? 2 : 1;
    static constexpr int SM = (VS == 2 && SMD == 2) ? 1 : SMD;
    static constexpr int LS = VS == 1 ? (L >= 2 ? L / 2 : L) : ((VS == 2 && SMD == 1) ? (L >= 4 ? L / 4 : L) : L);
    static_assert(L % LS == 0, "output primes in whole chunks");
    using NB = NttT<LOGN, NttGeom<LOGN>::T32::LOGR, Arith32, NTT_FORM>;  // stage T's transforms
};

// bounds of every mbarrier wait: one second of real time (a 64 KB bulk copy
// lands within microseconds), and at most 2^26 attempts
#define SFHE_WAIT_TRIES (1u << 26)
#define SFHE_WAIT_NS 1000000000ull

// One CTA per output entry at a time, taken from a queue in descending
// product count.  Per product (per rounding group of mm.group products in the
// grouped accumulate-then-round mode): stage T (tensor + 3K inverse NTTs over B into
// the CTA's scratch), stage S (exact scale-and-round to Q, then the sums of
// d0, d1 and of the digits D_j over the entry's products).  Per entry,
// stage R: since the NTT and the key product are linear mod q_i,
//   sum_k [NTT(d0_k) + sum_j NTT([D_jk]_{q_i}) b_j]
//     = NTT([sum_k d0_k]_{q_i}) + sum_j NTT([sum_k D_jk]_{q_i}) b_j   (mod q_i),
// so the relinearisation NTTs run once per entry; the result is identical,
// limb for limb, to relinearising every product and adding.
// Scratch per CTA: acc [3][L][N] uint64 (plain 64-bit sums: of the digits
// D_j, canonical, exact for up to 1024 products; of d0 and d1 in [0, 3 q_i),
// folded to canonical every 256 products), cacc [2][N] uint64, T [3][K][N]
// uint32 (x~_k, the inverse NTT's output).  queue[0] is the entry counter, queue[1] the error word (1: a
// bulk copy did not complete within the wait bound).  mbarriers 0 and 1
// track the operand pairs of stage T.
template <int LOGN, int L, bool GROUPED, int V>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_matmul_persistent(
    const __grid_constant__ RnsConsts c, const MmDesc* __restrict__ mms, const Entry* __restrict__ entries, int n_entries,
    const int2* __restrict__ rowlist, const u64* __restrict__ rlk, const u64* __restrict__ rlk_sh, u64* scratch,
    size_t scratch_stride, unsigned* queue, const unsigned* stop)
{
    using CF = Cfg<LOGN, L>;
    using NQ = typename CF::NQ;
    using NB = typename PersistentTile<LOGN, L, V>::NB;
    using PP = PersistentPlan<LOGN, L>;
    static_assert(NQ::NT == NB::NT, "both transforms use the same CTA");
    constexpr int N = NQ::N, NTH = NQ::NT, K = CF::K, R = NB::R;
    extern __shared__ __align__(128) u64 sm[];
    u32* sm32 = reinterpret_cast<u32*>(sm);
    unsigned char* smb = reinterpret_cast<unsigned char*>(sm);
    __shared__ int s_entry;
    __shared__ __align__(8) u64 mbar[2];
    const int tid = threadIdx.x;
    u64* base = scratch + (size_t)blockIdx.x * scratch_stride;
    u64* acc = base;                                        // [3][L][N] u64
    u64* cacc = acc + (size_t)3 * L * N;                    // [2][N] u64
    u32* T = reinterpret_cast<u32*>(cacc + (size_t)2 * N);  // [3][K][N] u32
    const size_t ext_words = (size_t)2 * K * N;
    const size_t ct_words = (size_t)2 * L * N;
    // staged operand slots: 0 a0, 1 a1, 2 b0, 3 b1 (limb k of the tensor base)
    auto slot = [&](int s) { return reinterpret_cast<u32*>(smb + PP::EXB + (size_t)s * PP::SLOT); };
    // per mbarrier: parity of the phase to wait for next, and whether a copy
    // is in flight (kept alike in every thread: issues and waits are uniform)
    u32 phbits = 0, pend = 0;
    if constexpr (PP::STAGED || PP::STAGED2) {
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < 2; i++) mbar_init(&mbar[i], 1);
            fence_mbar_init();
        }
    }
    // bounded wait on mbarrier bi by every thread; false (in every thread) if
    // any thread's wait ran out
    auto wait_bar = [&](int bi) -> bool {
        const bool ok = mbar_wait(&mbar[bi], (phbits >> bi) & 1u, SFHE_WAIT_TRIES, SFHE_WAIT_NS);
        if (ok) {
            phbits ^= 1u << bi;
            pend &= ~(1u << bi);
        }
        return !__syncthreads_or(!ok);
    };
    // the same wait without the block-wide vote: the caller votes on the
    // result at its next barrier
    auto wait_own = [&](int bi) -> bool {
        const bool ok = mbar_wait(&mbar[bi], (phbits >> bi) & 1u, SFHE_WAIT_TRIES, SFHE_WAIT_NS);
        if (ok) {
            phbits ^= 1u << bi;
            pend &= ~(1u << bi);
        }
        return ok;
    };
    // error exit: flag it, let the copies still in flight land, leave
    auto abort_cta = [&]() {
        if (tid == 0) {
            atomicExch(queue + 1, 1u);
            for (int bi = 0; bi < 2; bi++)
                if (pend & (1u << bi)) mbar_wait(&mbar[bi], (phbits >> bi) & 1u, SFHE_WAIT_TRIES, SFHE_WAIT_NS);
        }
    };

    for (;;) {
        __syncthreads();
        // a set stop word ends the launch at this entry boundary: the CTA
        // takes no entry (it is never waited on), so queue[0] stays the
        // number of entries taken and a later launch resumes from there
        if (tid == 0)
            s_entry = (stop && *reinterpret_cast<const volatile unsigned*>(stop)) ? n_entries
                                                                                   : (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int e = s_entry;
        if (e >= n_entries) break;
        const Entry en = entries[e];
        const MmDesc mm = mms[en.mm];
        u64* Cout = mm.C + ((size_t)en.row * mm.Nc + en.col) * ct_words;
        if (en.count == 0) {
            for (size_t w = tid; w < ct_words; w += NTH) Cout[w] = 0;
            continue;
        }
        auto operands = [&](int pr, const u32*& a, const u32*& b) {
            const int2 it = rowlist[en.first + pr];
            a = mm.A_ext + (size_t)it.x * ext_words;
            b = mm.B_ext + ((size_t)it.y * mm.Nc + en.col) * ext_words;
        };
        // stage S: scale-and-round every tensor coefficient and add the result
        // into the entry's sums, SM coefficients per thread at a time.  d0 and
        // d1 only need to be congruent (stage R reduces their sums), so they
        // stay in [0, 3 q_i); the digits of d2 must be canonical.
        auto stage_s = [&](int pr) {
            using TL = PersistentTile<LOGN, L, V>;
            constexpr int SM = TL::SM, LS = TL::LS;
            constexpr bool HOIST = K <= 16;
            const bool fold = pr != 0 && (pr & 255) == 0;  // sums below 2^64: fold every 256 products
            auto poly = [&](int p, int k, auto lazy) {
                constexpr bool LZ = decltype(lazy)::value;
                const u32* src[SM];
#pragma unroll
                for (int m = 0; m < SM; m++) src[m] = T + (size_t)p * K * N + k + m * NTH;
                // the sums so far of one chunk of output primes; with K <= 16
                // the first chunk's are loaded ahead of the arithmetic so that
                // their latency overlaps it (with more primes the registers
                // they would hold across the estimate are needed for x~)
                u64 prev[SM][LS];
                auto load_prev = [&](int i0) {
#pragma unroll
                    for (int m = 0; m < SM; m++) {
#pragma unroll
                        for (int ii = 0; ii < LS; ii++)
                            prev[m][ii] = pr == 0 ? 0 : acc[((size_t)p * L + i0 + ii) * N + k + m * NTH];
                    }
                };
                if constexpr (HOIST) load_prev(0);
                u32 xt[SM][K];
                u32 v[SM];
                u64 mK[SM];
                scale_round_est<K, SM>(src, N, c, xt, v, mK);
#pragma unroll
                for (int i0 = 0; i0 < L; i0 += LS) {
                    if (i0 > 0 || !HOIST) load_prev(i0);
                    u64 d[SM][LS];
                    scale_round_out<K, SM, LS, LZ>(xt, v, mK, c, i0, d);
#pragma unroll
                    for (int m = 0; m < SM; m++) {
#pragma unroll
                        for (int ii = 0; ii < LS; ii++) {
                            const int i = i0 + ii;
                            const u64 base = LZ && fold ? barrett64(prev[m][ii], c.m[i]) : prev[m][ii];
                            acc[((size_t)p * L + i) * N + k + m * NTH] = base + d[m][ii];
                        }
                    }
                }
            };
            for (int k = tid; k < N; k += SM * NTH) {
#pragma unroll 1
                for (int p = 0; p < 2; p++) poly(p, k, std::true_type{});
                poly(2, k, std::false_type{});
            }
        };
        if constexpr (PP::STAGED) {
            // stage T with TMA-staged operands: per tensor-base prime, the
            // three tensor polynomials are formed from the four staged limbs
            // and inverse-transformed together; the next limbs stream into the
            // slots meanwhile.  Products are taken in rounding groups of G
            // (G = 1: each product rounded on its own, Alg. 1): steps run
            // group by group, prime by prime, product by product, and a
            // group's tensor is summed over its products before the inverse
            // NTT (the NTT is linear), so stage S rounds it once.
            const int G = GROUPED ? mm.group : 1;
            if constexpr (!GROUPED) {
                const int total = en.count * K;
                auto issue = [&](int s, int pair) {
                    if (tid == 0) {
                        const int pr = s / K, k = s - pr * K;
                        const u32 *a, *b;
                        operands(pr, a, b);
                        const size_t off = (size_t)pair * K * N + (size_t)k * N;
                        fence_proxy_async();
                        mbar_arrive_expect_tx(&mbar[pair], (u32)(2 * PP::SLOT));
                        tma_load_1d(slot(pair), a + off, (u32)PP::SLOT, &mbar[pair]);
                        tma_load_1d(slot(2 + pair), b + off, (u32)PP::SLOT, &mbar[pair]);
                    }
                    pend |= 1u << pair;
                };
                issue(0, 0);
                issue(0, 1);
                for (int s = 0; s < total; s++) {
                    const int pr = s / K, k = s - pr * K;
                    const Mod32 m = c.mb[k];
                    const u32* tw = c.twb + (size_t)k * 4 * N;
                    const u32 ni = c.ninv_bx[k].w, nis = c.ninv_bx[k].ws, wl = c.wlast_bx[k].w, wls = c.wlast_bx[k].ws;
                    if (!wait_bar(0) || !wait_bar(1)) {
                        abort_cta();
                        return;
                    }
                    u32 x[3][R];
                    {
                        const u32* s0 = slot(0);
                        const u32* s1 = slot(1);
                        const u32* s2 = slot(2);
                        const u32* s3 = slot(3);
    #pragma unroll
                        for (int v = 0; v < R; v++) {
                            const int i = NB::lane_idx(v, tid);
                            const u64 a0 = s0[i], a1 = s1[i], b0 = s2[i], b1 = s3[i];
                            x[0][v] = redc32(a0 * b0, m);
                            x[1][v] = redc32(a0 * b1 + a1 * b0, m);
                            x[2][v] = redc32(a1 * b1, m);
                        }
                    }
                    __syncthreads();  // every thread has read the slots
                    if (s + 1 < total) {
                        issue(s + 1, 0);
                        issue(s + 1, 1);
                    }
                    NB::template inverse_m<3>(x, sm32, tid, tw, m.b, ni, nis, wl, wls);
    #pragma unroll
                    for (int p = 0; p < 3; p++) {
                        u32* dst = T + ((size_t)p * K + k) * N;
    #pragma unroll
                        for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[p][v], m.b);
                    }
                    if (k == K - 1) {
                        __syncthreads();
                        stage_s(pr);
                        __syncthreads();
                    }
                }
            } else {
            // The operand limbs stream in parts: part h of a step is the
            // lane-interleaved words [h N/NP, (h+1) N/NP) of its four limbs
            // (every thread's register slots h R/NP .. (h+1) R/NP - 1), copied
            // into buffer h (four limb parts) and tracked by mbarrier h; a
            // buffer is refilled with the next step's part as soon as it has
            // been summed, so NP - 1 parts' copies are in flight meanwhile.
            constexpr int NP = 2;  // one mbarrier per part
            constexpr int RH = R / NP;
            constexpr int HW = N / NP;  // words of a limb part
            static_assert(RH * NB::NT == HW && RH * NP == R, "a part is a contiguous slice of each limb");
            constexpr size_t PB = PP::SLOT / NP;  // bytes of a limb part
            auto hslot = [&](int h, int limb) {  // limbs 0 a0, 1 a1, 2 b0, 3 b1
                return reinterpret_cast<u32*>(smb + PP::EXB + (size_t)(h * 4 + limb) * PB);
            };
            // position of the next copy: group, prime, product in group
            int ig = 0, ik = 0, ip = 0, iGg = min(G, en.count);
            auto issue_part = [&](int h) {
                if (tid == 0) {
                    const u32 *a, *b;
                    operands(ig * G + ip, a, b);
                    const size_t o0 = (size_t)ik * N + (size_t)h * HW, o1 = (size_t)K * N + o0;
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&mbar[h], (u32)(4 * PB));
                    tma_load_1d(hslot(h, 0), a + o0, (u32)PB, &mbar[h]);
                    tma_load_1d(hslot(h, 1), a + o1, (u32)PB, &mbar[h]);
                    tma_load_1d(hslot(h, 2), b + o0, (u32)PB, &mbar[h]);
                    tma_load_1d(hslot(h, 3), b + o1, (u32)PB, &mbar[h]);
                }
                pend |= 1u << h;
            };
            auto advance = [&]() {  // false once every step has been issued
                if (++ip < iGg) return true;
                ip = 0;
                if (++ik < K) return true;
                ik = 0;
                ++ig;
                iGg = min(G, en.count - ig * G);
                return iGg > 0;
            };
#pragma unroll
            for (int h = 0; h < NP; h++) issue_part(h);
            bool more = advance();
            for (int g = 0; g * G < en.count; g++) {
                const int Gg = min(G, en.count - g * G);
                for (int k = 0; k < K; k++) {
                    const Mod32 m = c.mb[k];
                    // the group's tensor polynomials are summed in the idle
                    // exchange buffers (each thread at its own interleaved
                    // positions), not in registers kept across the copy waits
                    u32* acc3 = sm32;
                    __syncthreads();  // every thread is past the last transform's exchanges
                    for (int p = 0; p < Gg; p++) {
#pragma unroll
                        for (int h = 0; h < NP; h++) {
                            // each thread waits for buffer h by itself; whether
                            // any wait ran out is voted at the barrier that
                            // also releases the buffer for its next copy
                            const bool ok = wait_own(h);
                            if (ok) {
                                const u32* s0 = hslot(h, 0);
                                const u32* s1 = hslot(h, 1);
                                const u32* s2 = hslot(h, 2);
                                const u32* s3 = hslot(h, 3);
#pragma unroll
                                for (int vv = 0; vv < RH; vv++) {
                                    const int i = NB::lane_idx(h * RH + vv, tid);
                                    const int li = i - h * HW;
                                    const u64 a0 = s0[li], a1 = s1[li], b0 = s2[li], b1 = s3[li];
                                    const u32 t0 = redc32(a0 * b0, m), t1 = redc32(a0 * b1 + a1 * b0, m),
                                              t2 = redc32(a1 * b1, m);
                                    u32* q0 = acc3 + i;
                                    u32* q1 = acc3 + NB::SMEM_WORDS + i;
                                    u32* q2 = acc3 + 2 * NB::SMEM_WORDS + i;
                                    *q0 = p == 0 ? t0 : csub32(*q0 + t0, 2 * m.b);
                                    *q1 = p == 0 ? t1 : csub32(*q1 + t1, 2 * m.b);
                                    *q2 = p == 0 ? t2 : csub32(*q2 + t2, 2 * m.b);
                                }
                            }
                            if (__syncthreads_or(!ok)) {  // every thread has read buffer h
                                abort_cta();
                                return;
                            }
                            if (more) {
                                issue_part(h);
                                if (h == NP - 1) more = advance();
                            }
                        }
                    }
                    u32 x[3][R];
#pragma unroll
                    for (int j = 0; j < 3; j++) {
#pragma unroll
                        for (int v = 0; v < R; v++) x[j][v] = acc3[j * NB::SMEM_WORDS + NB::lane_idx(v, tid)];
                    }
                    const u32* tw = c.twb + (size_t)k * 4 * N;
                    NB::template inverse_m<3>(x, sm32, tid, tw, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws,
                                              c.wlast_bx[k].w, c.wlast_bx[k].ws);
#pragma unroll
                    for (int p = 0; p < 3; p++) {
                        u32* dst = T + ((size_t)p * K + k) * N;
#pragma unroll
                        for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[p][v], m.b);
                    }
                }
                __syncthreads();
                stage_s(g);
                __syncthreads();
            }
            }
        } else {
            // operands read from global memory; rounding groups of G products
            // as in the staged path
            const int G = GROUPED ? mm.group : 1;
            if constexpr (!GROUPED && PP::STAGED2) {
                // rounds of two staged limbs per prime: 0 (a0, b0) -> d0,
                // 1 (a1, b1) -> d2, 2 (a0, b1) and 3 (a1, b0) -> d1; each
                // round's copy streams in during the previous inverse NTT
                const int total = en.count * K * 4;
                auto issue2 = [&](int st) {
                    if (tid == 0) {
                        const int r = st & 3, q = st >> 2, pr = q / K, k = q - pr * K;
                        const u32 *a, *b;
                        operands(pr, a, b);
                        const size_t ca = (r == 1 || r == 3) ? 1 : 0, cb = (r == 1 || r == 2) ? 1 : 0;
                        fence_proxy_async();
                        mbar_arrive_expect_tx(&mbar[0], (u32)(2 * PP::SLOT));
                        tma_load_1d(slot(0), a + ca * K * N + (size_t)k * N, (u32)PP::SLOT, &mbar[0]);
                        tma_load_1d(slot(1), b + cb * K * N + (size_t)k * N, (u32)PP::SLOT, &mbar[0]);
                    }
                    pend |= 1u;
                };
                issue2(0);
                int st = 0;
                for (int pr = 0; pr < en.count; pr++) {
                    for (int k = 0; k < K; k++) {
                        const Mod32 m = c.mb[k];
                        const u32* tw = c.twb + (size_t)k * 4 * N;
                        u32 x[R];
                        for (int r = 0; r < 4; r++, st++) {
                            if (!wait_bar(0)) {
                                abort_cta();
                                return;
                            }
                            const u32* sa = slot(0);
                            const u32* sb = slot(1);
#pragma unroll
                            for (int v = 0; v < R; v++) {
                                const int i = NB::lane_idx(v, tid);
                                const u32 t = redc32((u64)sa[i] * sb[i], m);
                                x[v] = r == 3 ? csub32(x[v] + t, 2 * m.b) : t;
                            }
                            __syncthreads();  // every thread has read the slots
                            if (st + 1 < total) issue2(st + 1);
                            if (r == 2) continue;
                            NB::inverse(x, sm32, tid, tw, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws, c.wlast_bx[k].w,
                                        c.wlast_bx[k].ws);
                            u32* dst = T + ((size_t)(r == 0 ? 0 : (r == 1 ? 2 : 1)) * K + k) * N;
#pragma unroll
                            for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[v], m.b);
                        }
                    }
                    __syncthreads();
                    stage_s(pr);
                    __syncthreads();
                }
            } else if constexpr (GROUPED && PP::STAGED2) {
                // the same rounds, each over the group's products (the
                // group's tensor polynomial is summed before its inverse NTT)
                int ig = 0, ik = 0, ir = 0, ip = 0, iGg = min(G, en.count);
                auto issue2 = [&]() {
                    if (tid == 0) {
                        const u32 *a, *b;
                        operands(ig * G + ip, a, b);
                        const size_t ca = (ir == 1 || ir == 3) ? 1 : 0, cb = (ir == 1 || ir == 2) ? 1 : 0;
                        fence_proxy_async();
                        mbar_arrive_expect_tx(&mbar[0], (u32)(2 * PP::SLOT));
                        tma_load_1d(slot(0), a + ca * K * N + (size_t)ik * N, (u32)PP::SLOT, &mbar[0]);
                        tma_load_1d(slot(1), b + cb * K * N + (size_t)ik * N, (u32)PP::SLOT, &mbar[0]);
                    }
                    pend |= 1u;
                };
                auto advance = [&]() {  // false once every step has been issued
                    if (++ip < iGg) return true;
                    ip = 0;
                    if (++ir < 4) return true;
                    ir = 0;
                    if (++ik < K) return true;
                    ik = 0;
                    ++ig;
                    iGg = min(G, en.count - ig * G);
                    return iGg > 0;
                };
                issue2();
                bool more = advance();
                for (int g = 0; g * G < en.count; g++) {
                    const int Gg = min(G, en.count - g * G);
                    for (int k = 0; k < K; k++) {
                        const Mod32 m = c.mb[k];
                        const u32* tw = c.twb + (size_t)k * 4 * N;
                        u32 x[R];
                        for (int r = 0; r < 4; r++) {
                            for (int p = 0; p < Gg; p++) {
                                if (!wait_bar(0)) {
                                    abort_cta();
                                    return;
                                }
                                const u32* sa = slot(0);
                                const u32* sb = slot(1);
                                const bool fresh = p == 0 && r != 3;
#pragma unroll
                                for (int v = 0; v < R; v++) {
                                    const int i = NB::lane_idx(v, tid);
                                    const u32 t = redc32((u64)sa[i] * sb[i], m);
                                    x[v] = fresh ? t : csub32(x[v] + t, 2 * m.b);
                                }
                                __syncthreads();  // every thread has read the slots
                                if (more) {
                                    issue2();
                                    more = advance();
                                }
                            }
                            if (r == 2) continue;
                            NB::inverse(x, sm32, tid, tw, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws, c.wlast_bx[k].w,
                                        c.wlast_bx[k].ws);
                            u32* dst = T + ((size_t)(r == 0 ? 0 : (r == 1 ? 2 : 1)) * K + k) * N;
#pragma unroll
                            for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[v], m.b);
                        }
                    }
                    __syncthreads();
                    stage_s(g);
                    __syncthreads();
                }
            } else if constexpr (!GROUPED) {
                for (int pr = 0; pr < en.count; pr++) {
                    const u32 *a, *b;
                    operands(pr, a, b);
                    // stage T
                    for (int k = 0; k < K; k++) {
                        const Mod32 m = c.mb[k];
                        const u32* ak = a + (size_t)k * N;
                        const u32* bk = b + (size_t)k * N;
                        const u32* tw = c.twb + (size_t)k * 4 * N;
                        for (int p = 0; p < 3; p++) {
                            u32 x[R];
    #pragma unroll
                            for (int v = 0; v < R; v++) x[v] = tensor_coeff32(p, ak, bk, (size_t)K * N, NB::lane_idx(v, tid), m);
                            NB::inverse(x, sm32, tid, tw, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws, c.wlast_bx[k].w,
                                        c.wlast_bx[k].ws);
                            u32* dst = T + ((size_t)p * K + k) * N;
    #pragma unroll
                            for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[v], m.b);
                        }
                    }
                    __syncthreads();
                    stage_s(pr);
                    __syncthreads();
                }
            } else {
            for (int g = 0; g * G < en.count; g++) {
                const int g0 = g * G, Gg = min(G, en.count - g0);
                // stage T
                for (int k = 0; k < K; k++) {
                    const Mod32 m = c.mb[k];
                    const u32* tw = c.twb + (size_t)k * 4 * N;
                    for (int p = 0; p < 3; p++) {
                        u32 x[R];
                        for (int q = 0; q < Gg; q++) {
                            const u32 *a, *b;
                            operands(g0 + q, a, b);
#pragma unroll
                            for (int v = 0; v < R; v++) {
                                const u32 t = tensor_coeff32(p, a + (size_t)k * N, b + (size_t)k * N, (size_t)K * N,
                                                             NB::lane_idx(v, tid), m);
                                x[v] = q == 0 ? t : csub32(x[v] + t, 2 * m.b);
                            }
                        }
                        NB::inverse(x, sm32, tid, tw, m.b, c.ninv_bx[k].w, c.ninv_bx[k].ws, c.wlast_bx[k].w,
                                    c.wlast_bx[k].ws);
                        u32* dst = T + ((size_t)p * K + k) * N;
#pragma unroll
                        for (int v = 0; v < R; v++) dst[NB::inv_out_idx(v, tid)] = csub32(x[v], m.b);
                    }
                }
                __syncthreads();
                stage_s(g);
                __syncthreads();
            }
            }
        }
        // stage R.  The forward NTT leaves slot tid * R + v of every polynomial
        // with thread tid, so the key products and the output are private to
        // a thread, and the key and C are accessed with 16-byte vectors.  Up
        // to N = 8192 the sums [2][N] live in the idle operand slots (element
        // v of thread tid at v * NTH + tid, free of bank conflicts).  At
        // N = 16384 they do not fit: the L + 2 transforms of a limb go to the
        // idle tensor scratch and one pass forms both sums in registers.
        if constexpr (PP::STAGED) {
            u64* cs = PP::STAGED ? reinterpret_cast<u64*>(smb + PP::EXB) : cacc;
            auto cpos = [&](int v) -> size_t {
                return PP::STAGED ? (size_t)v * NTH + tid : (size_t)NQ::run_idx(v, tid);
            };
            for (int i = 0; i < L; i++) {
                const Mod m = c.m[i];
                const u64* tw = c.tw + (size_t)i * 4 * N;
                for (int s = 0; s < L + 2; s++) {
                    // s = 0: sum d0 (limb i), 1: sum d1 (limb i), 2 + j: sum of digits j
                    const u64* src = s < 2 ? acc + ((size_t)s * L + i) * N : acc + ((size_t)2 * L + (s - 2)) * N;
                    u64 x[NQ::R];
#pragma unroll
                    for (int v = 0; v < NQ::R; v++) x[v] = barrett64(src[NQ::fwd_in_idx(v, tid)], m);
                    NQ::forward(x, sm, tid, tw, m.q);
                    if (s < 2) {
#pragma unroll
                        for (int v = 0; v < NQ::R; v++) cs[(size_t)s * N + cpos(v)] = x[v];
                    } else {
                        const int j = s - 2;
                        const size_t ob = (((size_t)j * 2 + 0) * L + i) * N + (size_t)tid * NQ::R;
                        const size_t oa = (((size_t)j * 2 + 1) * L + i) * N + (size_t)tid * NQ::R;
#pragma unroll
                        for (int v = 0; v < NQ::R; v += 2) {
                            const ulonglong2 wb = __ldg(reinterpret_cast<const ulonglong2*>(rlk + ob + v));
                            const ulonglong2 sb = __ldg(reinterpret_cast<const ulonglong2*>(rlk_sh + ob + v));
                            const ulonglong2 wa = __ldg(reinterpret_cast<const ulonglong2*>(rlk + oa + v));
                            const ulonglong2 sa = __ldg(reinterpret_cast<const ulonglong2*>(rlk_sh + oa + v));
                            cs[cpos(v)] += shoup_lazy(x[v], wb.x, sb.x, m.q);
                            cs[cpos(v + 1)] += shoup_lazy(x[v + 1], wb.y, sb.y, m.q);
                            cs[N + cpos(v)] += shoup_lazy(x[v], wa.x, sa.x, m.q);
                            cs[N + cpos(v + 1)] += shoup_lazy(x[v + 1], wa.y, sa.y, m.q);
                        }
                    }
                }
                u64* c0 = Cout + (size_t)i * N + (size_t)tid * NQ::R;
                u64* c1 = Cout + ((size_t)L + i) * N + (size_t)tid * NQ::R;
#pragma unroll
                for (int v = 0; v < NQ::R; v += 2) {
                    *reinterpret_cast<ulonglong2*>(c0 + v) =
                        make_ulonglong2(barrett64(cs[cpos(v)], m), barrett64(cs[cpos(v + 1)], m));
                    *reinterpret_cast<ulonglong2*>(c1 + v) =
                        make_ulonglong2(barrett64(cs[N + cpos(v)], m), barrett64(cs[N + cpos(v + 1)], m));
                }
            }
        } else {
            // the L + 2 forward transforms of a limb run with 16 words per
            // thread (two virtual threads of the 16-word geometry per thread,
            // the data in shared memory between passes), which keeps stage R
            // within the registers the CTA is launched with
            using NH = NttT<LOGN, 4, Arith64>;
            constexpr int VT = NH::NT / NTH;
            static_assert(NH::SMEM_WORDS * 8 <= PP::SMEM, "shared memory of the looped transform");
            u64* U = reinterpret_cast<u64*>(T);  // [L + 2][N], slot e at its place
            for (int i = 0; i < L; i++) {
                const Mod m = c.m[i];
                const u64* tw = c.tw + (size_t)i * 4 * N;
                for (int s = 0; s < L + 2; s++) {
                    const u64* src = s < 2 ? acc + ((size_t)s * L + i) * N : acc + ((size_t)2 * L + (s - 2)) * N;
                    u64* dst = U + (size_t)s * N;
                    NH::template forward_looped<VT>(
                        sm, tid, tw, m.q, [&](int e) { return barrett64(src[e], m); },
                        [&](int vt, const u64(&x)[NH::R]) {
#pragma unroll
                            for (int v = 0; v < NH::R; v += 2)
                                *reinterpret_cast<ulonglong2*>(dst + (size_t)vt * NH::R + v) = make_ulonglong2(x[v], x[v + 1]);
                        });
                }
                // every thread reads back the slots its virtual threads wrote
#pragma unroll 1
                for (int jv = 0; jv < VT; jv++) {
                const size_t e0 = (size_t)(tid + jv * NTH) * NH::R;
                u64* c0 = Cout + (size_t)i * N + e0;
                u64* c1 = Cout + ((size_t)L + i) * N + e0;
#pragma unroll 1
                for (int v = 0; v < NH::R; v += 2) {
                    const ulonglong2 u0 = *reinterpret_cast<const ulonglong2*>(U + e0 + v);
                    const ulonglong2 u1 = *reinterpret_cast<const ulonglong2*>(U + N + e0 + v);
                    u64 b0 = u0.x, b1 = u0.y, a0 = u1.x, a1 = u1.y;
#pragma unroll
                    for (int j = 0; j < L; j++) {
                        const ulonglong2 d = *reinterpret_cast<const ulonglong2*>(U + (size_t)(2 + j) * N + e0 + v);
                        const size_t ob = (((size_t)j * 2 + 0) * L + i) * N + e0 + v;
                        const size_t oa = (((size_t)j * 2 + 1) * L + i) * N + e0 + v;
                        const ulonglong2 wb = __ldg(reinterpret_cast<const ulonglong2*>(rlk + ob));
                        const ulonglong2 sb = __ldg(reinterpret_cast<const ulonglong2*>(rlk_sh + ob));
                        const ulonglong2 wa = __ldg(reinterpret_cast<const ulonglong2*>(rlk + oa));
                        const ulonglong2 sa = __ldg(reinterpret_cast<const ulonglong2*>(rlk_sh + oa));
                        b0 += shoup_lazy(d.x, wb.x, sb.x, m.q);
                        b1 += shoup_lazy(d.y, wb.y, sb.y, m.q);
                        a0 += shoup_lazy(d.x, wa.x, sa.x, m.q);
                        a1 += shoup_lazy(d.y, wa.y, sa.y, m.q);
                    }
                    *reinterpret_cast<ulonglong2*>(c0 + v) = make_ulonglong2(barrett64(b0, m), barrett64(b1, m));
                    *reinterpret_cast<ulonglong2*>(c1 + v) = make_ulonglong2(barrett64(a0, m), barrett64(a1, m));
                }
                }
            }
        }
        // the slots are refilled by bulk copies (async proxy) for the next entry
        if constexpr (PP::STAGED || PP::STAGED2) fence_proxy_async();
    }
}
