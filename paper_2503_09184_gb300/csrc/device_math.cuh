// device_math.cuh -- 64-bit modular arithmetic for 54-bit primes, the exact
// CRT rounding used by every base conversion, and the counter-based
// generator.  All moduli satisfy 2^53 < q < 2^54.
#pragma once
#include <stdint.h>
#include "rns.h"

#define SFHE_DEV __device__ __forceinline__

// ---------------------------------------------------------------- scalar ---
SFHE_DEV u64 mulhi(u64 a, u64 b) { return __umul64hi(a, b); }

// a + b mod q for a, b < q
SFHE_DEV u64 add_mod(u64 a, u64 b, u64 q)
{
    u64 s = a + b;
    return s >= q ? s - q : s;
}
// a - b mod q for a, b < q
SFHE_DEV u64 sub_mod(u64 a, u64 b, u64 q)
{
    return a >= b ? a - b : a + q - b;
}
SFHE_DEV u64 csub(u64 a, u64 q) { return a >= q ? a - q : a; }

// Shoup: a * w mod q in [0, 2q) for any a < 2^64 (Harvey's lazy form).
SFHE_DEV u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q)
{
    return a * w - mulhi(a, ws) * q;
}
SFHE_DEV u64 shoup_lazy(u64 a, ShoupC c, u64 q) { return shoup_lazy(a, c.w, c.ws, q); }
SFHE_DEV u64 shoup(u64 a, ShoupC c, u64 q) { return csub(shoup_lazy(a, c.w, c.ws, q), q); }

// Shoup with the exact quotient: a * w = quo * q + rem, rem in [0, q),
// for a < q.
SFHE_DEV u64 shoup_quot(u64 a, ShoupC c, u64 q, u64& quo)
{
    u64 qh = mulhi(a, c.ws);
    u64 r = a * c.w - qh * q;
    if (r >= q) {
        r -= q;
        qh += 1;
    }
    quo = qh;
    return r;
}

// Barrett reduction of x = hi:lo < 2^114 with mu = floor(2^114 / q):
// qhat = floor(floor(x / 2^50) * mu / 2^64) is at most 2 below floor(x/q),
// so x - qhat q < 3q and two conditional subtractions finish it.
SFHE_DEV u64 barrett(u64 hi, u64 lo, Mod m)
{
    u64 xs = (hi << 14) | (lo >> 50);
    u64 qh = mulhi(xs, m.mu);
    u64 r = lo - qh * m.q;
    r = csub(r, m.q);
    return csub(r, m.q);
}
SFHE_DEV u64 barrett64(u64 x, Mod m) { return barrett(0, x, m); }
// the same without the final subtractions: a value in [0, 3q) congruent to x
SFHE_DEV u64 barrett_lazy(u64 hi, u64 lo, Mod m)
{
    const u64 xs = (hi << 14) | (lo >> 50);
    return lo - mulhi(xs, m.mu) * m.q;
}

// (hi:lo) += a * b
SFHE_DEV void mac(u64& hi, u64& lo, u64 a, u64 b)
{
    u64 l = a * b;
    u64 h = mulhi(a, b);
    lo += l;
    hi += h + (lo < l ? 1 : 0);
}
SFHE_DEV void add128(u64& hi, u64& lo, u64 a)
{
    lo += a;
    hi += (lo < a ? 1 : 0);
}

// a * b mod q for variable a, b < 2^54
SFHE_DEV u64 mul_mod(u64 a, u64 b, Mod m)
{
    return barrett(mulhi(a, b), a * b, m);
}

// ------------------------------------------------------ exact CRT rounding ---
// round(sum_{i<L} y_i / q_i) for residues y_i in [0, q_i), exactly.
//
// Estimate: e_i = floor((y_i 2^10) mu_i / 2^64) with mu_i = floor(2^114/q_i)
// lies in (y_i 2^60 / q_i - 2, y_i 2^60 / q_i], so with E = sum e_i the true
// value V satisfies V 2^60 in [E, E + 2L).  floor((E + 2^59) / 2^60) is
// exact unless (E + 2^59) mod 2^60 >= 2^60 - 2L; in that band the decision
// V >= k0 + 1/2 is taken exactly as 2 S >= (2 k0 + 1) Q with the multiword
// S = sum_i y_i (Q/q_i)  (V = S / Q; Q is odd, so there are no ties).
SFHE_DEV bool crt_round_fallback(const u64* y, const RnsConsts& c, u64 k0)
{
    const int W = c.Qwords + 1;
    u64 S[SFHE_MAX_L + 2];
    u64 R[SFHE_MAX_L + 2];
    for (int w = 0; w <= W; w++) { S[w] = 0; R[w] = 0; }
    for (int i = 0; i < c.L; i++) {
        u64 carry = 0;
        for (int w = 0; w < W; w++) {
            u64 lo = y[i] * c.Qhat_w[i][w];
            u64 hi = mulhi(y[i], c.Qhat_w[i][w]);
            lo += carry;
            hi += (lo < carry ? 1 : 0);
            u64 s = S[w] + lo;
            hi += (s < lo ? 1 : 0);
            S[w] = s;
            carry = hi;
        }
        S[W] += carry;
    }
    // 2S
    for (int w = W; w > 0; w--) S[w] = (S[w] << 1) | (S[w - 1] >> 63);
    S[0] <<= 1;
    // (2 k0 + 1) Q
    u64 f = 2 * k0 + 1, carry = 0;
    for (int w = 0; w < W; w++) {
        u64 qw = w < c.Qwords ? c.Qw[w] : 0;
        u64 lo = qw * f + carry;
        u64 hi = mulhi(qw, f) + (lo < carry ? 1 : 0);
        R[w] = lo;
        carry = hi;
    }
    R[W] = carry;
    for (int w = W; w >= 0; w--) {
        if (S[w] != R[w]) return S[w] > R[w];
    }
    return true;  // unreachable: 2S is even, (2k0+1)Q is odd
}

template <int L_STATIC>
SFHE_DEV u64 crt_round(const u64* y, const RnsConsts& c, int L)
{
    u64 E = 0;
    const int n = L_STATIC > 0 ? L_STATIC : L;
#pragma unroll
    for (int i = 0; i < (L_STATIC > 0 ? L_STATIC : SFHE_MAX_L); i++) {
        if (i < n) E += mulhi(y[i] << 10, c.m[i].mu);
    }
    u64 Eh = E + (1ULL << 59);
    u64 k0 = Eh >> 60;
    u64 fr = Eh & ((1ULL << 60) - 1);
    if (fr >= (1ULL << 60) - 2 * (u64)n) {
        if (crt_round_fallback(y, c, k0)) k0 += 1;
    }
    return k0;
}

// ------------------------------------------------- 30-bit tensor base -------
SFHE_DEV u32 csub32(u32 a, u32 b) { return a >= b ? a - b : a; }

// Shoup for b < 2^30: a * w mod b in [0, 2b) for any a < 2^32.
SFHE_DEV u32 shoup32_lazy(u32 a, u32 w, u32 ws, u32 b) { return a * w - __umulhi(a, ws) * b; }
SFHE_DEV u32 shoup32(u32 a, Shoup32 c, u32 b) { return csub32(shoup32_lazy(a, c.w, c.ws, b), b); }

// x mod b for x < 2^61 with mu61 = floor(2^61 / b): the estimate
// floor(floor(x / 2^29) mu61 / 2^32) is at most 2 below floor(x / b), so the
// remainder is below 3b < 2^32 and two conditional subtractions finish it.
SFHE_DEV u32 reduce61(u64 x, Mod32 m)
{
    const u32 qh = __umulhi((u32)(x >> 29), m.mu61);
    u32 r = (u32)x - qh * m.b;
    r = csub32(r, m.b);
    return csub32(r, m.b);
}

// Montgomery reduction: x 2^-32 mod b, in [0, 2b), for x < b 2^32, with
// binv = -b^-1 mod 2^32 (x + q b is divisible by 2^32 for q = x binv mod 2^32).
SFHE_DEV u32 redc32(u64 x, Mod32 m)
{
    const u32 q = (u32)x * m.binv;
    return (u32)((x + (u64)q * m.b) >> 32);
}

// x mod b for any 64-bit x with mu64 = floor(2^64 / b) (estimate at most 1 low).
SFHE_DEV u32 reduce64b(u64 x, Mod32 m)
{
    const u64 qh = mulhi(x, m.mu64);
    return csub32((u32)(x - qh * m.b), m.b);
}

// round(sum_{k<n} y_k / b_k) for y_k in [0, b_k) when the sum is known to lie
// within 1/4 of an integer, in 32-bit products: with bfrac_k =
// floor(2^43 / b_k) < 2^14, the term floor(y_k / 2^16) bfrac_k is below
// y_k 2^27 / b_k < 2^27 by less than y_k / 2^16 + 2^43 / b_k < 2^15, so
// E = sum of the terms is below 2^27 sum_k y_k / b_k (and below 2^32 for
// n <= 31) by less than n 2^-12 units of 2^27: far from moving the sum
// across a half-integer.
template <int n>
SFHE_DEV u32 round_b(const u32* y, const RnsConsts& c)
{
    static_assert(n <= 31, "the 32-bit estimate holds up to 31 primes");
    u32 E = 0;
#pragma unroll
    for (int k = 0; k < n; k++) E += (y[k] >> 16) * c.bfrac[k];
    return (E + (1u << 26)) >> 27;
}

// ---------------------------------------------------------- generator ------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-style:
//   key  = absorb(absorb(absorb(absorb(mix(seed + G), domain), o0), o1), o2)
//   word = mix(key + (idx + 1) G),  absorb(h, x) = mix(h ^ mix(x + G)).
#define SFHE_GAMMA 0x9E3779B97F4A7C15ULL
SFHE_DEV u64 sm_mix(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
SFHE_DEV u64 sm_absorb(u64 h, u64 x) { return sm_mix(h ^ sm_mix(x + SFHE_GAMMA)); }
SFHE_DEV u64 sm_key(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2)
{
    u64 h = sm_mix(seed + SFHE_GAMMA);
    h = sm_absorb(h, dom);
    h = sm_absorb(h, o0);
    h = sm_absorb(h, o1);
    return sm_absorb(h, o2);
}
SFHE_DEV u64 sm_word(u64 key, u64 idx) { return sm_mix(key + (idx + 1) * SFHE_GAMMA); }

// uniform residue for slot: first of words slot*16+r (r < 16) below
// floor(2^64/q) q, reduced mod q; sets *fail when all 16 are rejected.
SFHE_DEV u64 sample_uniform(u64 key, u64 slot, u64 q, int* fail)
{
    u64 lim = (~0ULL / q) * q;
    for (u64 r = 0; r < 16; r++) {
        u64 w = sm_word(key, slot * 16 + r);
        if (w < lim) return w % q;
    }
    *fail = 1;
    return 0;
}
SFHE_DEV int sample_ternary(u64 key, u64 slot, int* fail)
{
    u64 lim = (~0ULL / 3) * 3;
    for (u64 r = 0; r < 16; r++) {
        u64 w = sm_word(key, slot * 16 + r);
        if (w < lim) {
            u64 v = w % 3;
            return v == 0 ? 0 : (v == 1 ? 1 : -1);
        }
    }
    *fail = 1;
    return 0;
}
SFHE_DEV int sample_gauss(u64 key, u64 slot, const u64* cdt)
{
    u64 w = sm_word(key, slot * 16);
    u64 u = w >> 1;
    int k = 0;
    while (k < 19 && u >= cdt[k]) k++;
    if (k == 0) return 0;
    return (w & 1) ? -k : k;
}
// signed small integer to its residue mod q
SFHE_DEV u64 to_residue(long long v, u64 q)
{
    if (v >= 0) return (u64)v % q;
    u64 r = (u64)(-v) % q;
    return r ? q - r : 0;
}

// ------------------------------------------------- TMA bulk copies ---------
// One-dimensional bulk copies global -> shared through the tensor memory
// accelerator, completed on an mbarrier (transaction count in bytes).
SFHE_DEV u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

SFHE_DEV void mbar_init(u64* bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the async proxy (before their first use)
SFHE_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the calling thread arrives and announces `bytes` of incoming transactions
SFHE_DEV void mbar_arrive_expect_tx(u64* bar, u32 bytes)
{
    u64 state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    (void)state;
}
// bytes (multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst
SFHE_DEV void tma_load_1d(void* dst, const void* src, u32 bytes, u64* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses
SFHE_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// the GPU's nanosecond clock (PTX %globaltimer)
SFHE_DEV u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the phase with the given parity: false once max_tries
// attempts have failed or max_ns nanoseconds have passed, whichever comes
// first (an attempt may itself suspend the thread for a hardware-defined
// time, so the time bound is the one that holds in real time)
SFHE_DEV bool mbar_wait(u64* bar, u32 parity, u32 max_tries, u64 max_ns)
{
    const u64 t0 = global_ns();
    for (u32 i = 0; i < max_tries; i++) {
        u32 done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > max_ns) return false;
    }
    return false;
}
