// kernels.cuh -- device code of the encrypted sparse matmul.
//
// Storage (all uint64, canonical residues):
//   ciphertext, base Q, NTT form:      [2 (c0, c1)][L][N]
//   lifted ciphertext, base Q u P, NTT: [2][L + Lp][N]  (Q limbs first)
//   relinearisation key, NTT form:      [L digit j][2 (b, a)][L limb i][N] (+ Shoup companions)
// Per product (Alg. 1, "a <- a x b; fhe_relin; fhe_add"):
//   tensor d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1 over Q u P (NTT form),
//   inverse NTT, exact scale-and-round by t/Q (result in base Q), digits
//   D_j = [d2]_{q_j}, relinearise with the key, add into C.
#pragma once
#include "ntt.cuh"
#include "worklist.h"

// ------------------------------------------------------------------------
// elementwise pieces
// ------------------------------------------------------------------------
// one coefficient of tensor polynomial `poly` (0: a0 b0, 1: a0 b1 + a1 b0,
// 2: a1 b1) in limb l; a, b point at [2][L+Lp][N] lifted ciphertexts
SFHE_DEV u64 tensor_coeff(int poly, const u64* __restrict__ a, const u64* __restrict__ b, size_t off1, size_t e,
                          Mod m)
{
    // off1: distance between c0 and c1 of a lifted ciphertext
    if (poly == 0) return mul_mod(__ldg(a + e), __ldg(b + e), m);
    if (poly == 2) return mul_mod(__ldg(a + off1 + e), __ldg(b + off1 + e), m);
    u64 a0 = __ldg(a + e), a1 = __ldg(a + off1 + e), b0 = __ldg(b + e), b1 = __ldg(b + off1 + e);
    u64 hi = mulhi(a0, b1), lo = a0 * b1;
    mac(hi, lo, a1, b0);
    return barrett(hi, lo, m);
}

// Exact round(t x / Q) for a tensor coefficient x given over Q u P
// (x: L residues mod q_i, xp: Lp residues mod p_j, canonical); writes the
// result's residues mod q_i.  Step 1 gives the result in base P:
//   x~_i = [x_i (QP/q_i)^-1]_{q_i},  x~_i [tP]_{q_i} = u_i q_i + y_i,
//   r = sum u_i + round(sum y_i / q_i),
//   d_j = [x_j [tQ^-1]_{p_j} + sum_i x~_i [floor(tP/q_i)]_{p_j} + r]_{p_j};
// step 2 converts the centred d from P to Q (|d| < P 2^-24, so the rounding
// of sum d~_j / p_j is never near a half-integer).
template <int L>
SFHE_DEV void scale_round(const u64* x, const u64* xp, const RnsConsts& c, u64* d)
{
    constexpr int LP = L + 1;
    u64 xt[L], y[L];
    u64 usum = 0;
#pragma unroll
    for (int i = 0; i < L; i++) {
        const u64 qi = c.m[i].q;
        xt[i] = shoup(x[i], c.qphat_inv[i], qi);
        u64 quo;
        y[i] = shoup_quot(xt[i], c.tP_q[i], qi, quo);
        usum += quo;
    }
    const u64 r = usum + crt_round<L>(y, c, L);
    u64 dt[LP];
#pragma unroll
    for (int j = 0; j < LP; j++) {
        const Mod pm = c.m[L + j];
        u64 hi = 0, lo = 0;
#pragma unroll
        for (int i = 0; i < L; i++) mac(hi, lo, xt[i], c.omega[i][j]);
        add128(hi, lo, shoup_lazy(xp[j], c.tQinv_p[j], pm.q));
        add128(hi, lo, r);
        const u64 dj = barrett(hi, lo, pm);
        dt[j] = shoup(dj, c.phat_inv[j], pm.q);
    }
    const u64 v = crt_round_p_nearint(dt, c);
#pragma unroll
    for (int i = 0; i < L; i++) {
        u64 hi = 0, lo = 0;
#pragma unroll
        for (int j = 0; j < LP; j++) mac(hi, lo, dt[j], c.phat_mod_q[j][i]);
        add128(hi, lo, v * c.negP_mod_q[i]);
        d[i] = barrett(hi, lo, c.m[i]);
    }
}

// ------------------------------------------------------------------------
// generic NTT kernels over batches of polynomials
// ------------------------------------------------------------------------
// Polynomial (g, l): input at in + g * in_gstride + (in_l0 + l) * N, output
// at out + g * out_gstride + (out_l0 + l) * N, prime index prime0 + l.
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
    NT_::inverse(x, sm, tid, c.tw + (size_t)pi * 4 * NT_::N, m.q, c.ninv[pi], c.wlast[pi]);
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::inv_out_idx(v, tid)] = csub(x[v], m.q);
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
// lift: base Q -> Q u P (centred)
// ------------------------------------------------------------------------
#ifdef SFHE_KERNELS_TU
// coefficient form in: [g][L][N] (canonical), out: [g][Lp][N]
__global__ void __launch_bounds__(256) k_lift_extend(const __grid_constant__ RnsConsts c, const u64* in, u64* out,
                                                     int ngroups)
{
    const int N = c.N, L = c.L, Lp = c.Lp;
    const size_t idx = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= (size_t)ngroups * N) return;
    const size_t g = idx / N, k = idx % N;
    u64 at[SFHE_MAX_L];
    for (int i = 0; i < L; i++) at[i] = shoup(in[(g * L + i) * N + k], c.qhat_inv[i], c.m[i].q);
    const u64 v = crt_round<0>(at, c, L);
    for (int j = 0; j < Lp; j++) {
        const Mod pm = c.m[L + j];
        u64 hi = 0, lo = 0;
        for (int i = 0; i < L; i++) mac(hi, lo, at[i], c.qhat_mod_p[i][j]);
        add128(hi, lo, v * c.negQ_mod_p[j]);
        out[(g * Lp + j) * N + k] = barrett(hi, lo, pm);
    }
}
#endif

// ------------------------------------------------------------------------
// plain per-product path
// ------------------------------------------------------------------------
// block (limb l, poly p): tensor polynomial p in limb l, inverse NTT,
// coefficient form to T[p][l][N]
template <int LOGN>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_tensor_intt(const __grid_constant__ RnsConsts c, const u64* a,
                                                                     const u64* b, u64* T)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N;
    extern __shared__ u64 sm[];
    const int l = blockIdx.x, p = blockIdx.y, tid = threadIdx.x;
    const int LQP = c.L + c.Lp;
    const Mod m = c.m[l];
    const size_t off1 = (size_t)LQP * N;
    const u64* al = a + (size_t)l * N;
    const u64* bl = b + (size_t)l * N;
    u64 x[NT_::R];
#pragma unroll
    for (int v = 0; v < NT_::R; v++) x[v] = tensor_coeff(p, al, bl, off1, NT_::run_idx(v, tid), m);
    NT_::inverse(x, sm, tid, c.tw + (size_t)l * 4 * N, m.q, c.ninv[l], c.wlast[l]);
    u64* dst = T + ((size_t)p * LQP + l) * N;
#pragma unroll
    for (int v = 0; v < NT_::R; v++) dst[NT_::inv_out_idx(v, tid)] = csub(x[v], m.q);
}

// T [3][L+Lp][N] -> D [3][L][N] (coefficient form, canonical)
template <int L>
__global__ void __launch_bounds__(128) k_scale_round(const __grid_constant__ RnsConsts c, const u64* T, u64* D)
{
    const int N = c.N, LQP = L + L + 1;
    const int k = blockIdx.x * 128 + threadIdx.x, p = blockIdx.y;
    if (k >= N) return;
    u64 x[L], xp[L + 1], d[L];
#pragma unroll
    for (int i = 0; i < L; i++) x[i] = T[((size_t)p * LQP + i) * N + k];
#pragma unroll
    for (int j = 0; j < L + 1; j++) xp[j] = T[((size_t)p * LQP + L + j) * N + k];
    scale_round<L>(x, xp, c, d);
#pragma unroll
    for (int i = 0; i < L; i++) D[((size_t)p * L + i) * N + k] = d[i];
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
#endif

// ------------------------------------------------------------------------
// fused persistent matmul
// ------------------------------------------------------------------------
// One CTA per output entry at a time, taken from a queue in descending
// product count.  Per product: stage T (tensor + inverse NTT of the 3 (L+Lp)
// polynomials into the CTA's scratch), stage S (scale-and-round, then the
// sums of d0, d1 and of the digits D_j over the entry's products).  Per
// entry, stage R: since the NTT and the key product are linear mod q_i,
//   sum_k [NTT(d0_k) + sum_j NTT([D_jk]_{q_i}) b_j]
//     = NTT([sum_k d0_k]_{q_i}) + sum_j NTT([sum_k D_jk]_{q_i}) b_j   (mod q_i),
// so the relinearisation NTTs run once per entry; the result is identical,
// limb for limb, to relinearising every product and adding.
// Scratch per CTA: T [3][L+Lp][N], acc [3][L][N] (plain 64-bit sums of
// canonical residues: exact for up to 1024 products), cacc [2][N].
template <int LOGN, int L>
__global__ void __launch_bounds__(NttGeom<LOGN>::T::NT) k_matmul_persistent(
    const __grid_constant__ RnsConsts c, const MmDesc* __restrict__ mms, const Entry* __restrict__ entries, int n_entries,
    const int2* __restrict__ rowlist, const u64* __restrict__ rlk, const u64* __restrict__ rlk_sh, u64* scratch,
    size_t scratch_stride, unsigned* queue)
{
    using NT_ = typename NttGeom<LOGN>::T;
    constexpr int N = NT_::N, R = NT_::R, NTH = NT_::NT;
    constexpr int LP = L + 1, LQP = L + LP;
    extern __shared__ u64 sm[];
    __shared__ int s_entry;
    const int tid = threadIdx.x;
    u64* T = scratch + (size_t)blockIdx.x * scratch_stride;
    u64* acc = T + (size_t)3 * LQP * N;
    u64* cacc = acc + (size_t)3 * L * N;
    const size_t ext_words = (size_t)2 * LQP * N;
    const size_t ct_words = (size_t)2 * L * N;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_entry = (int)atomicAdd(queue, 1u);
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
        for (int pr = 0; pr < en.count; pr++) {
            const int2 it = rowlist[en.first + pr];
            const u64* a = mm.A_ext + (size_t)it.x * ext_words;
            const u64* b = mm.B_ext + ((size_t)it.y * mm.Nc + en.col) * ext_words;
            // stage T
            for (int l = 0; l < LQP; l++) {
                const Mod m = c.m[l];
                const u64* al = a + (size_t)l * N;
                const u64* bl = b + (size_t)l * N;
                const u64* tw = c.tw + (size_t)l * 4 * N;
                for (int p = 0; p < 3; p++) {
                    u64 x[R];
#pragma unroll
                    for (int v = 0; v < R; v++) x[v] = tensor_coeff(p, al, bl, (size_t)LQP * N, NT_::run_idx(v, tid), m);
                    NT_::inverse(x, sm, tid, tw, m.q, c.ninv[l], c.wlast[l]);
                    u64* dst = T + ((size_t)p * LQP + l) * N;
#pragma unroll
                    for (int v = 0; v < R; v++) dst[NT_::inv_out_idx(v, tid)] = csub(x[v], m.q);
                }
            }
            __syncthreads();
            // stage S
            for (int k = tid; k < N; k += NTH) {
#pragma unroll 1
                for (int p = 0; p < 3; p++) {
                    u64 x[L], xp[LP], d[L];
#pragma unroll
                    for (int i = 0; i < L; i++) x[i] = T[((size_t)p * LQP + i) * N + k];
#pragma unroll
                    for (int j = 0; j < LP; j++) xp[j] = T[((size_t)p * LQP + L + j) * N + k];
                    scale_round<L>(x, xp, c, d);
#pragma unroll
                    for (int i = 0; i < L; i++) {
                        u64* ap = acc + ((size_t)p * L + i) * N + k;
                        *ap = pr == 0 ? d[i] : *ap + d[i];
                    }
                }
            }
            __syncthreads();
        }
        // stage R
        for (int i = 0; i < L; i++) {
            const Mod m = c.m[i];
            const u64* tw = c.tw + (size_t)i * 4 * N;
            for (int s = 0; s < L + 2; s++) {
                // s = 0: sum d0 (limb i), 1: sum d1 (limb i), 2 + j: sum of digits j
                const u64* src = s < 2 ? acc + ((size_t)s * L + i) * N : acc + ((size_t)2 * L + (s - 2)) * N;
                u64 x[R];
#pragma unroll
                for (int v = 0; v < R; v++) x[v] = barrett64(src[NT_::fwd_in_idx(v, tid)], m);
                NT_::forward(x, sm, tid, tw, m.q);
#pragma unroll
                for (int v = 0; v < R; v++) {
                    const int k = NT_::run_idx(v, tid);
                    if (s == 0) {
                        cacc[k] = x[v];
                    } else if (s == 1) {
                        cacc[N + k] = x[v];
                    } else {
                        const int j = s - 2;
                        const size_t rb = (((size_t)j * 2 + 0) * L + i) * N + k;
                        const size_t ra = (((size_t)j * 2 + 1) * L + i) * N + k;
                        cacc[k] += shoup_lazy(x[v], __ldg(rlk + rb), __ldg(rlk_sh + rb), m.q);
                        cacc[N + k] += shoup_lazy(x[v], __ldg(rlk + ra), __ldg(rlk_sh + ra), m.q);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < R; v++) {
                const int k = NT_::run_idx(v, tid);
                Cout[(size_t)i * N + k] = barrett64(cacc[k], m);
                Cout[((size_t)L + i) * N + k] = barrett64(cacc[N + k], m);
            }
        }
    }
}

#ifdef SFHE_KERNELS_TU
// raw generator words (stream-equality checks against the oracle)
__global__ void k_prng_words(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, u64 idx0, long long n, u64* out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out[t] = sm_word(sm_key(seed, dom, o0, o1, o2), idx0 + (u64)t);
}
#endif
