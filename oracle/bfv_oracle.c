/*
 * bfv_oracle.c -- plain, slow, CPU-only oracle for encrypted sparse matrix
 * multiplication under RNS BFV: one ciphertext per matrix element with the
 * value in the constant coefficient, and (at the end of the file) the
 * chunked form of Sec. 3.2 with c values per ciphertext in its slots,
 * rotations and the slot-0 mask.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference arm may load this library.  It shares
 * no code with the CUDA path and the CUDA path never calls it.
 *
 * What it computes (paper: "Exploiting Unstructured Sparsity in Fully
 * Homomorphic Encrypted DNNs", Alg. 1 and Sec. 3.3.2):
 *   C[i][j] = sum over k in S(i,j) of Relin(Mul(A[i][k], B[k][j]))
 * where S(i,j) is the product set an encoding lists (dense: every k; naive
 * sparse / CSR / ELLPACK: the k with A[i][k] != 0).  Per product, in the
 * order of Alg. 1's inner loop: multiply the two chunks, relinearise, add
 * into the result.  BFV replaces CKKS's rescale by the exact scale-and-round by
 * t/Q that is part of the BFV multiply (Sec. 3.1 names BFV as the integer
 * scheme).
 *
 * Everything is done in coefficient form, in the order the textbook states it:
 *   - polynomial products are schoolbook negacyclic convolutions (no NTT);
 *   - the exact integer tensor is obtained by CRT over an auxiliary prime
 *     base large enough to hold it, reconstructed as a multiword integer;
 *   - d = floor((2 t x + Q) / (2 Q)) is an exact multiword long division.
 * Arithmetic is unsigned __int128; multiword integers are plain arrays.
 *
 * The random words the scheme draws (secret, relinearisation key,
 * encryption masks and errors) come from one counter-based generator,
 * written here from its published definition (SplitMix64, Steele, Lea &
 * Flood, OOPSLA 2014) and keyed as documented at or_prng_word().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef unsigned __int128 u128;

#define OR_MAX_L 8
#define OR_MAX_AUX 24
#define OR_MAX_GROUP 1024 /* most exact tensors summed before one scale-and-round */
#define MW 18 /* words per multiword integer: 1152 bits, enough for 2t|x| at L <= 8, N <= 2^15 */

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic (moduli < 2^62)                            */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 addmod(u64 a, u64 b, u64 m) { u64 s = a + b; return s >= m ? s - m : s; }
static u64 submod(u64 a, u64 b, u64 m) { return a >= b ? a - b : a + (m - b); }
static u64 powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}
/* m prime: Fermat inverse */
static u64 invmod(u64 a, u64 m) { return powmod(a % m, m - 2, m); }

/* Deterministic Miller-Rabin with the first twelve prime bases, exact for
 * every n < 3.3e24 and so for every 64-bit n. */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* The `count` largest primes below 2^54 congruent to 1 mod 2N, descending.
 * The first L are the ciphertext primes Q, the next L+1 the extension P. */
int or_ntt_primes(int N, int count, u64 *out)
{
    u64 twoN = 2 * (u64)N;
    u64 k = ((1ULL << 54) - 2) / twoN;
    int got = 0;
    while (got < count && k > 0) {
        u64 p = k * twoN + 1;
        if (or_is_prime(p)) out[got++] = p;
        k--;
    }
    return got == count ? 0 : -1;
}

/* Smallest x in [1, q) with x^N == -1 (mod q): the smallest primitive
 * 2N-th root of unity. */
u64 or_psi(u64 q, int N)
{
    u64 psi0 = 0;
    for (u64 g = 2; g < q; g++) {
        u64 c = powmod(g, (q - 1) / (2 * (u64)N), q);
        if (powmod(c, (u64)N, q) == q - 1) { psi0 = c; break; }
    }
    if (!psi0) return 0;
    /* every primitive 2N-th root is psi0^k with k odd */
    u64 step = mulmod(psi0, psi0, q), x = psi0, best = psi0;
    for (int k = 1; k < N; k++) {
        x = mulmod(x, step, q);
        if (x < best) best = x;
    }
    return best;
}

static int bitrev(int x, int logn)
{
    int r = 0;
    for (int i = 0; i < logn; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* NTT form by definition: out[i] = sum_j in[j] * psi^((2*bitrev(i)+1)*j). */
void or_ntt_naive(u64 q, int N, const u64 *in, u64 *out)
{
    int logn = 0;
    while ((1 << logn) < N) logn++;
    u64 psi = or_psi(q, N);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        u64 root = powmod(psi, 2 * (u64)bitrev(i, logn) + 1, q);
        u64 acc = 0, pw = 1;
        for (int j = 0; j < N; j++) {
            acc = addmod(acc, mulmod(in[j] % q, pw, q), q);
            pw = mulmod(pw, root, q);
        }
        out[i] = acc;
    }
}

/* Inverse of the definition above:
 *   in[j] = N^-1 psi^-j sum_b out[bitrev(b)] (psi^-2j)^b. */
void or_intt_naive(u64 q, int N, const u64 *in, u64 *out)
{
    int logn = 0;
    while ((1 << logn) < N) logn++;
    u64 psi = or_psi(q, N);
    u64 psi_inv = invmod(psi, q);
    u64 ninv = invmod((u64)N, q);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < N; j++) {
        u64 g = powmod(psi_inv, 2 * (u64)j, q);
        u64 acc = 0, pw = 1;
        for (int b = 0; b < N; b++) {
            acc = addmod(acc, mulmod(in[bitrev(b, logn)] % q, pw, q), q);
            pw = mulmod(pw, g, q);
        }
        out[j] = mulmod(mulmod(acc, powmod(psi_inv, (u64)j, q), q), ninv, q);
    }
}

/* ------------------------------------------------------------------ */
/* schoolbook negacyclic product in Z_m[X]/(X^N + 1)                    */
/* ------------------------------------------------------------------ */
/* out[c] = sum_{i+j=c} a_i b_j - sum_{i+j=c+N} a_i b_j  (mod m).
 * a, b < m < 2^54: each product < 2^108 and at most N <= 2^15 of them are
 * summed, so the two 128-bit accumulators never wrap. */
static void negacyclic_acc(u64 m, int N, const u64 *a, const u64 *b, u64 *out, int accumulate)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < N; c++) {
        u128 pos = 0, neg = 0;
        for (int i = 0; i <= c; i++) pos += (u128)a[i] * b[c - i];
        for (int i = c + 1; i < N; i++) neg += (u128)a[i] * b[N + c - i];
        u64 v = submod((u64)(pos % m), (u64)(neg % m), m);
        out[c] = accumulate ? addmod(out[c], v, m) : v;
    }
}

void or_negacyclic(u64 m, int N, const u64 *a, const u64 *b, u64 *out)
{
    negacyclic_acc(m, N, a, b, out, 0);
}

/* ------------------------------------------------------------------ */
/* multiword unsigned integers, little-endian 64-bit words              */
/* ------------------------------------------------------------------ */
typedef struct { u64 w[MW]; } mw_t;

static void mw_zero(mw_t *a) { memset(a, 0, sizeof(*a)); }
static void mw_set(mw_t *a, u64 v) { mw_zero(a); a->w[0] = v; }
static int mw_cmp(const mw_t *a, const mw_t *b)
{
    for (int i = MW - 1; i >= 0; i--) {
        if (a->w[i] != b->w[i]) return a->w[i] > b->w[i] ? 1 : -1;
    }
    return 0;
}
static int mw_is_zero(const mw_t *a)
{
    for (int i = 0; i < MW; i++) if (a->w[i]) return 0;
    return 1;
}
/* r = a + b (no overflow past MW words is allowed by the callers) */
static void mw_add(mw_t *r, const mw_t *a, const mw_t *b)
{
    u64 carry = 0;
    for (int i = 0; i < MW; i++) {
        u128 s = (u128)a->w[i] + b->w[i] + carry;
        r->w[i] = (u64)s;
        carry = (u64)(s >> 64);
    }
}
/* r = a - b, requires a >= b */
static void mw_sub(mw_t *r, const mw_t *a, const mw_t *b)
{
    u64 borrow = 0;
    for (int i = 0; i < MW; i++) {
        u64 ai = a->w[i], bi = b->w[i];
        u64 d = ai - bi - borrow;
        borrow = (ai < bi) || (ai - bi < borrow) ? 1 : 0;
        r->w[i] = d;
    }
}
/* r = a * s */
static void mw_mul_u64(mw_t *r, const mw_t *a, u64 s)
{
    u64 carry = 0;
    for (int i = 0; i < MW; i++) {
        u128 p = (u128)a->w[i] * s + carry;
        r->w[i] = (u64)p;
        carry = (u64)(p >> 64);
    }
}
static int mw_bitlen(const mw_t *a)
{
    for (int i = MW - 1; i >= 0; i--) {
        if (a->w[i]) {
            int b = 64;
            while (!((a->w[i] >> (b - 1)) & 1)) b--;
            return i * 64 + b;
        }
    }
    return 0;
}
/* bitwise long division: quo = a / b, rem = a % b, b != 0 */
static void mw_divmod(const mw_t *a, const mw_t *b, mw_t *quo, mw_t *rem)
{
    mw_t q, r;
    mw_zero(&q);
    mw_zero(&r);
    for (int bit = mw_bitlen(a) - 1; bit >= 0; bit--) {
        /* r = 2r + bit */
        for (int i = MW - 1; i > 0; i--) r.w[i] = (r.w[i] << 1) | (r.w[i - 1] >> 63);
        r.w[0] = (r.w[0] << 1) | ((a->w[bit / 64] >> (bit % 64)) & 1);
        if (mw_cmp(&r, b) >= 0) {
            mw_sub(&r, &r, b);
            q.w[bit / 64] |= 1ULL << (bit % 64);
        }
    }
    if (quo) *quo = q;
    if (rem) *rem = r;
}
/* a mod m for a word-sized m (Horner from the top word) */
static u64 mw_mod_u64(const mw_t *a, u64 m)
{
    u64 r = 0;
    for (int i = MW - 1; i >= 0; i--) r = (u64)((((u128)r << 64) | a->w[i]) % m);
    return r;
}
/* quotient of a by a word-sized m */
static void mw_div_u64(mw_t *q, const mw_t *a, u64 m)
{
    u64 r = 0;
    for (int i = MW - 1; i >= 0; i--) {
        u128 cur = ((u128)r << 64) | a->w[i];
        q->w[i] = (u64)(cur / m);
        r = (u64)(cur % m);
    }
}

/* ------------------------------------------------------------------ */
/* CRT over a prime base                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    int K;
    u64 m[OR_MAX_AUX];
    mw_t M;                 /* product of the moduli */
    mw_t Mk[OR_MAX_AUX];    /* M / m_k */
    u64 inv[OR_MAX_AUX];    /* (M / m_k)^-1 mod m_k */
    mw_t half;              /* floor(M / 2) */
} crt_base;

static void crt_init(crt_base *b, int K, const u64 *m)
{
    b->K = K;
    mw_set(&b->M, 1);
    for (int k = 0; k < K; k++) {
        b->m[k] = m[k];
        mw_mul_u64(&b->M, &b->M, m[k]);
    }
    for (int k = 0; k < K; k++) {
        mw_div_u64(&b->Mk[k], &b->M, m[k]);
        b->inv[k] = invmod(mw_mod_u64(&b->Mk[k], m[k]), m[k]);
    }
    mw_zero(&b->half);
    for (int i = 0; i < MW; i++)
        b->half.w[i] = (b->M.w[i] >> 1) | (i + 1 < MW ? b->M.w[i + 1] << 63 : 0);
}

/* The unique X in [0, M) with X == r_k (mod m_k) for every k. */
static void crt_reconstruct(const crt_base *b, const u64 *r, mw_t *X)
{
    mw_t acc, term;
    mw_zero(&acc);
    for (int k = 0; k < b->K; k++) {
        u64 y = mulmod(r[k] % b->m[k], b->inv[k], b->m[k]);
        mw_mul_u64(&term, &b->Mk[k], y);
        mw_add(&acc, &acc, &term);
    }
    while (mw_cmp(&acc, &b->M) >= 0) mw_sub(&acc, &acc, &b->M);
    *X = acc;
}

/* ------------------------------------------------------------------ */
/* counter-based generator (SplitMix64)                                 */
/* ------------------------------------------------------------------ */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL
static u64 sm_mix(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static u64 sm_absorb(u64 h, u64 x) { return sm_mix(h ^ sm_mix(x + SM_GAMMA)); }

enum { DOM_SECRET = 1, DOM_RLK_A = 2, DOM_RLK_E = 3, DOM_ENC_A = 4, DOM_ENC_E = 5, DOM_GAL_A = 6, DOM_GAL_E = 7 };

/* Key of the stream for (seed, domain, object) and its word number idx:
 *   key  = absorb(absorb(absorb(absorb(mix(seed + G), domain), o0), o1), o2)
 *   word = mix(key + (idx + 1) G)        (the (idx+1)-th SplitMix64 output)
 * with absorb(h, x) = mix(h ^ mix(x + G)), G = 0x9E3779B97F4A7C15. */
static u64 sm_key(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2)
{
    u64 h = sm_mix(seed + SM_GAMMA);
    h = sm_absorb(h, dom);
    h = sm_absorb(h, o0);
    h = sm_absorb(h, o1);
    return sm_absorb(h, o2);
}
static u64 sm_word(u64 key, u64 idx) { return sm_mix(key + (idx + 1) * SM_GAMMA); }

u64 or_prng_word(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, u64 idx)
{
    return sm_word(sm_key(seed, dom, o0, o1, o2), idx);
}

/* Uniform residue mod q for slot `slot`: words (slot*16 + r), r = 0..15, the
 * first one below floor(2^64/q)*q is taken mod q.  Returns -1 if all 16 are
 * rejected (probability below 2^-150 for 54-bit q). */
static int sample_uniform(u64 key, u64 slot, u64 q, u64 *out)
{
    u64 lim = (UINT64_MAX / q) * q; /* floor(2^64-1 / q) * q == floor(2^64/q)*q for q not a power of 2 */
    for (u64 r = 0; r < 16; r++) {
        u64 w = sm_word(key, slot * 16 + r);
        if (w < lim) { *out = w % q; return 0; }
    }
    return -1;
}
/* Ternary {0, 1, -1} for slot: first word below floor(2^64/3)*3, w mod 3 ->
 * 0 -> 0, 1 -> 1, 2 -> -1. */
static int sample_ternary(u64 key, u64 slot, int *out)
{
    u64 lim = (UINT64_MAX / 3) * 3;
    for (u64 r = 0; r < 16; r++) {
        u64 w = sm_word(key, slot * 16 + r);
        if (w < lim) {
            u64 v = w % 3;
            *out = v == 0 ? 0 : (v == 1 ? 1 : -1);
            return 0;
        }
    }
    return -1;
}

/* Cumulative table of |e| for the rounded Gaussian of width sigma, tail cut
 * at 19: rho(k) = exp(-k^2 / (2 sigma^2)), S = rho(0) + 2 (rho(1)+...+rho(19))
 * (partial sums in ascending k), CDF(k) = (rho(0) + 2 (rho(1)+...+rho(k))) / S,
 * T[k] = floor(CDF(k) * 2^63) for k < 19, T[19] = 2^63.  Plain IEEE double,
 * no contraction (the build passes -ffp-contract=off). */
void or_cdt(double sigma, u64 *T)
{
    double rho[20], S = 0.0, part = 0.0, two_s2 = 2.0 * sigma * sigma;
    for (int k = 0; k < 20; k++) rho[k] = exp(-((double)(k * k)) / two_s2);
    for (int k = 1; k < 20; k++) part = part + rho[k];
    S = rho[0] + 2.0 * part;
    part = 0.0;
    for (int k = 0; k < 19; k++) {
        if (k > 0) part = part + rho[k];
        double cdf = (rho[0] + 2.0 * part) / S;
        T[k] = (u64)ldexp(cdf, 63);
    }
    T[19] = 1ULL << 63;
}
/* Gaussian error for slot: w = word(slot*16); sign = w & 1, u = w >> 1,
 * |e| = min{k : u < T[k]}, e = |e| with the sign applied when |e| > 0. */
static int64_t sample_gauss(u64 key, u64 slot, const u64 *T)
{
    u64 w = sm_word(key, slot * 16);
    u64 u = w >> 1;
    int k = 0;
    while (u >= T[k]) k++;
    if (k == 0) return 0;
    return (w & 1) ? -(int64_t)k : (int64_t)k;
}

/* ------------------------------------------------------------------ */
/* context                                                              */
/* ------------------------------------------------------------------ */
typedef struct {
    int N, L, nP, nA;
    u64 t, seed;
    double sigma;
    u64 q[OR_MAX_L], p[OR_MAX_L + 1], aux[OR_MAX_AUX];
    crt_base Qb, Ab;
    mw_t Delta;                 /* floor(Q / t) */
    u64 delta_q[OR_MAX_L];      /* Delta mod q_i */
    u64 cdt[20];
    int64_t *s;                 /* secret, N ternary coefficients */
    u64 *s_mod;                 /* [L][N] s mod q_i */
    u64 *rlk;                   /* [L digit j][2 (b, a)][L limb i][N] */
} or_ctx;

static u64 *rlk_poly(or_ctx *c, int j, int ba, int i)
{
    return c->rlk + ((((size_t)j * 2 + ba) * c->L + i) * (size_t)c->N);
}

void or_ctx_free(void *vc)
{
    or_ctx *c = (or_ctx *)vc;
    if (!c) return;
    free(c->s);
    free(c->s_mod);
    free(c->rlk);
    free(c);
}

/* Key generation (secret-key BFV, relinearisation key with one digit per
 * ciphertext prime and no special prime):
 *   s ternary;  rlk_j = (b_j, a_j),  b_j = -a_j s + e_j + g_j s^2 (mod Q),
 * with the gadget g_j = (Q/q_j) [(Q/q_j)^-1]_{q_j}, so g_j == delta_ij mod q_i. */
void *or_ctx_create(int N, int L, u64 t, double sigma, u64 seed)
{
    if (N < 2 || (N & (N - 1)) || L < 1 || L > OR_MAX_L) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->N = N; c->L = L; c->nP = L + 1; c->t = t; c->seed = seed; c->sigma = sigma;
    u64 primes[2 * OR_MAX_L + 1];
    if (or_ntt_primes(N, 2 * L + 1, primes)) { free(c); return NULL; }
    for (int i = 0; i < L; i++) c->q[i] = primes[i];
    for (int j = 0; j < L + 1; j++) c->p[j] = primes[L + j];
    crt_init(&c->Qb, L, c->q);

    /* auxiliary base: the largest primes below 2^53, as many as needed for
     * a product above 4 N Q^2 OR_MAX_GROUP (twice the largest |coefficient|
     * of a sum of up to OR_MAX_GROUP tensors, with margin); tensors and their
     * sums are reconstructed exactly over it. */
    mw_t bound, prod;
    mw_set(&bound, 4ULL * (u64)N * OR_MAX_GROUP);
    {
        mw_t tmp;
        for (int i = 0; i < L; i++) { mw_mul_u64(&tmp, &bound, c->q[i]); bound = tmp; }
        for (int i = 0; i < L; i++) { mw_mul_u64(&tmp, &bound, c->q[i]); bound = tmp; }
    }
    mw_set(&prod, 1);
    int nA = 0;
    for (u64 cand = (1ULL << 53) - 1; nA < OR_MAX_AUX && cand > 3; cand -= 2) {
        if (!or_is_prime(cand)) continue;
        c->aux[nA++] = cand;
        mw_mul_u64(&prod, &prod, cand);
        if (mw_cmp(&prod, &bound) > 0) break;
    }
    c->nA = nA;
    crt_init(&c->Ab, nA, c->aux);

    mw_div_u64(&c->Delta, &c->Qb.M, t);
    for (int i = 0; i < L; i++) c->delta_q[i] = mw_mod_u64(&c->Delta, c->q[i]);
    or_cdt(sigma, c->cdt);

    /* secret */
    c->s = (int64_t *)malloc(sizeof(int64_t) * N);
    c->s_mod = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    u64 ks = sm_key(seed, DOM_SECRET, 0, 0, 0);
    for (int k = 0; k < N; k++) {
        int v;
        if (sample_ternary(ks, (u64)k, &v)) { or_ctx_free(c); return NULL; }
        c->s[k] = v;
    }
    for (int i = 0; i < L; i++)
        for (int k = 0; k < N; k++)
            c->s_mod[(size_t)i * N + k] = c->s[k] >= 0 ? (u64)c->s[k] : c->q[i] - (u64)(-c->s[k]);

    /* s^2 over the integers (coefficients bounded by N in magnitude) */
    int64_t *s2 = (int64_t *)calloc(N, sizeof(int64_t));
    for (int a = 0; a < N; a++) {
        if (!c->s[a]) continue;
        for (int b = 0; b < N; b++) {
            int64_t pr = c->s[a] * c->s[b];
            int idx = a + b;
            if (idx < N) s2[idx] += pr;
            else s2[idx - N] -= pr;
        }
    }

    c->rlk = (u64 *)malloc(sizeof(u64) * (size_t)L * 2 * L * N);
    u64 *tmp = (u64 *)malloc(sizeof(u64) * N);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int j = 0; j < L; j++) {
        u64 ka = sm_key(seed, DOM_RLK_A, (u64)j, 0, 0);
        u64 ke = sm_key(seed, DOM_RLK_E, (u64)j, 0, 0);
        for (int k = 0; k < N; k++) e[k] = sample_gauss(ke, (u64)k, c->cdt);
        for (int i = 0; i < L; i++) {
            u64 qi = c->q[i];
            u64 *a = rlk_poly(c, j, 1, i), *b = rlk_poly(c, j, 0, i);
            for (int k = 0; k < N; k++) {
                if (sample_uniform(ka, (u64)i * N + k, qi, &a[k])) { or_ctx_free(c); return NULL; }
            }
            or_negacyclic(qi, N, a, c->s_mod + (size_t)i * N, tmp);
            for (int k = 0; k < N; k++) {
                u64 ek = e[k] >= 0 ? (u64)e[k] : qi - (u64)(-e[k]);
                u64 v = submod(ek, tmp[k], qi);
                if (i == j) {
                    u64 s2k = s2[k] >= 0 ? (u64)s2[k] % qi : qi - ((u64)(-s2[k]) % qi);
                    v = addmod(v, s2k % qi, qi);
                }
                b[k] = v;
            }
        }
    }
    free(tmp);
    free(e);
    free(s2);
    return c;
}

int or_ctx_info(void *vc, int *N, int *L, int *nP, int *nA, u64 *q, u64 *p, u64 *aux)
{
    or_ctx *c = (or_ctx *)vc;
    *N = c->N; *L = c->L; *nP = c->nP; *nA = c->nA;
    for (int i = 0; i < c->L; i++) q[i] = c->q[i];
    for (int j = 0; j < c->nP; j++) p[j] = c->p[j];
    for (int k = 0; k < c->nA; k++) aux[k] = c->aux[k];
    return 0;
}

void or_get_secret(void *vc, int64_t *s)
{
    or_ctx *c = (or_ctx *)vc;
    memcpy(s, c->s, sizeof(int64_t) * c->N);
}

void or_get_rlk(void *vc, u64 *out)
{
    or_ctx *c = (or_ctx *)vc;
    memcpy(out, c->rlk, sizeof(u64) * (size_t)c->L * 2 * c->L * c->N);
}

void or_get_cdt(void *vc, u64 *T)
{
    or_ctx *c = (or_ctx *)vc;
    memcpy(T, c->cdt, sizeof(c->cdt));
}

/* Delta = floor(Q/t) written as L words (little-endian) */
void or_get_delta(void *vc, u64 *words, int nwords)
{
    or_ctx *c = (or_ctx *)vc;
    for (int i = 0; i < nwords && i < MW; i++) words[i] = c->Delta.w[i];
}

/* ------------------------------------------------------------------ */
/* encrypt / decrypt                                                    */
/* ------------------------------------------------------------------ */
/* Secret-key encryption of the integer m in the constant coefficient:
 *   c1 = a,  c0 = -a s + e + Delta [m]_t   (mod each q_i)
 * a uniform per limb, e Gaussian (shared by all limbs).  The stream object
 * is (matrix_id, row, col).  ct layout: [2][L][N], coefficient form. */
/* The same with a whole plaintext polynomial m (coefficients in [0, t)):
 *   c0 = -a s + e + Delta m  (mod each q_i), every coefficient carrying its
 * own message digit (the slot-packed encoding of Sec. 3.2's chunks). */
int or_encrypt_poly(void *vc, const u64 *m, u64 mid, u64 row, u64 col, u64 *ct)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 ka = sm_key(c->seed, DOM_ENC_A, mid, row, col);
    u64 ke = sm_key(c->seed, DOM_ENC_E, mid, row, col);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * N);
    u64 *as = (u64 *)malloc(sizeof(u64) * N);
    for (int k = 0; k < N; k++) e[k] = sample_gauss(ke, (u64)k, c->cdt);
    int rc = 0;
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        u64 *c0 = ct + (size_t)i * N, *c1 = ct + ((size_t)L + i) * N;
        for (int k = 0; k < N; k++)
            if (sample_uniform(ka, (u64)i * N + k, qi, &c1[k])) rc = -1;
        or_negacyclic(qi, N, c1, c->s_mod + (size_t)i * N, as);
        for (int k = 0; k < N; k++) {
            u64 ek = e[k] >= 0 ? (u64)e[k] : qi - (u64)(-e[k]);
            u64 v = submod(ek, as[k], qi);
            if (m[k]) v = addmod(v, mulmod(c->delta_q[i], m[k] % c->t, qi), qi);
            c0[k] = v;
        }
    }
    free(e);
    free(as);
    return rc;
}

int or_encrypt(void *vc, int64_t m, u64 mid, u64 row, u64 col, u64 *ct)
{
    or_ctx *c = (or_ctx *)vc;
    u64 *poly = (u64 *)calloc((size_t)c->N, sizeof(u64));
    int64_t mt = m % (int64_t)c->t;
    if (mt < 0) mt += (int64_t)c->t;
    poly[0] = (u64)mt;
    int rc = or_encrypt_poly(vc, poly, mid, row, col, ct);
    free(poly);
    return rc;
}

/* v = [c0 + c1 s]_Q in [0, Q);  m = floor((t v + floor(Q/2)) / Q) mod t,
 * returned centred in (-t/2, t/2].  noise_bits = bit length of
 * |[v - Delta [m]_t]_Q| (centred).  Only the constant coefficient carries
 * the message; *noise_bits is the maximum over all N coefficients. */
int or_decrypt(void *vc, const u64 *ct, int64_t *m_out, int *noise_bits)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 *v = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        or_negacyclic(qi, N, ct + ((size_t)L + i) * N, c->s_mod + (size_t)i * N, v + (size_t)i * N);
        for (int k = 0; k < N; k++) v[(size_t)i * N + k] = addmod(v[(size_t)i * N + k], ct[(size_t)i * N + k] % qi, qi);
    }
    int maxbits = 0;
    int64_t m0 = 0;
    for (int k = 0; k < N; k++) {
        u64 r[OR_MAX_L];
        for (int i = 0; i < L; i++) r[i] = v[(size_t)i * N + k];
        mw_t V, num, quo, halfQ, tmp;
        crt_reconstruct(&c->Qb, r, &V);
        mw_mul_u64(&num, &V, c->t);
        halfQ = c->Qb.half;
        mw_add(&num, &num, &halfQ);
        mw_divmod(&num, &c->Qb.M, &quo, NULL);
        u64 mu = mw_mod_u64(&quo, c->t);
        if (k == 0) m0 = mu > c->t / 2 ? (int64_t)mu - (int64_t)c->t : (int64_t)mu;
        /* noise: [V - Delta m(X)]_Q centred; the message sits in the
         * constant coefficient only, so m(X)'s other coefficients are 0 */
        mw_t dm;
        mw_mul_u64(&dm, &c->Delta, k == 0 ? mu : 0);
        while (mw_cmp(&dm, &c->Qb.M) >= 0) mw_sub(&dm, &dm, &c->Qb.M);
        if (mw_cmp(&V, &dm) >= 0) mw_sub(&tmp, &V, &dm);
        else { mw_sub(&tmp, &c->Qb.M, &dm); mw_add(&tmp, &tmp, &V); }
        if (mw_cmp(&tmp, &c->Qb.half) > 0) mw_sub(&tmp, &c->Qb.M, &tmp);
        int bits = mw_bitlen(&tmp);
        if (bits > maxbits) maxbits = bits;
    }
    *m_out = m0;
    if (noise_bits) *noise_bits = maxbits;
    free(v);
    return 0;
}

/* ------------------------------------------------------------------ */
/* multiply, relinearise, accumulate                                    */
/* ------------------------------------------------------------------ */
/* Centred lift of one coefficient given by its residues over Q, reduced mod
 * every auxiliary prime: X in (-Q/2, Q/2), out[k] = X mod aux_k. */
int or_tensor_scale_sum(void *vc, int n, const u64 *const *a, const u64 *const *b, u64 *d);

static void lift_centered_to_aux(const or_ctx *c, const u64 *r, u64 *out)
{
    mw_t X, mag;
    crt_reconstruct(&c->Qb, r, &X);
    int neg = mw_cmp(&X, &c->Qb.half) > 0;
    if (neg) mw_sub(&mag, &c->Qb.M, &X);
    else mag = X;
    for (int k = 0; k < c->nA; k++) {
        u64 v = mw_mod_u64(&mag, c->aux[k]);
        out[k] = (neg && v) ? c->aux[k] - v : v;
    }
}

/* d = floor((2 t X + Q) / (2 Q)) (floor toward -inf) for X given by its
 * residues over the auxiliary base, centred; writes d mod q_i, i < L. */
static void scale_round_coeff(const or_ctx *c, const u64 *xr, u64 *d_out)
{
    mw_t X, mag, num, twoQ, quo, rem;
    crt_reconstruct(&c->Ab, xr, &X);
    int neg = mw_cmp(&X, &c->Ab.half) > 0;
    if (neg) mw_sub(&mag, &c->Ab.M, &X);
    else mag = X;
    mw_add(&twoQ, &c->Qb.M, &c->Qb.M);
    mw_mul_u64(&num, &mag, 2 * c->t);          /* 2 t |X| */
    int dneg;
    if (!neg) {                                /* 2tX + Q >= 0 */
        mw_add(&num, &num, &c->Qb.M);
        mw_divmod(&num, &twoQ, &quo, NULL);
        dneg = 0;
    } else if (mw_cmp(&num, &c->Qb.M) <= 0) { /* -2t|X| + Q >= 0 */
        mw_sub(&num, &c->Qb.M, &num);
        mw_divmod(&num, &twoQ, &quo, NULL);
        dneg = 0;
    } else {                                   /* negative numerator n: floor(n/2Q) = -ceil(|n|/2Q) */
        mw_sub(&num, &num, &c->Qb.M);          /* |n| = 2t|X| - Q > 0 */
        mw_divmod(&num, &twoQ, &quo, &rem);
        if (!mw_is_zero(&rem)) {
            mw_t one;
            mw_set(&one, 1);
            mw_add(&quo, &quo, &one);
        }
        dneg = 1;
    }
    for (int i = 0; i < c->L; i++) {
        u64 v = mw_mod_u64(&quo, c->q[i]);
        d_out[i] = (dneg && v) ? c->q[i] - v : v;
    }
}

/* Exact integer tensor of one product, as residues over the auxiliary base:
 *   x0 = a0 b0, x1 = a0 b1 + a1 b0, x2 = a1 b1  (negacyclic products of the
 *   centred lifts).  a, b: [2][L][N]; x: [3][nA][N], added into x when
 *   accumulate is set. */
static void tensor_aux(const or_ctx *c, const u64 *a, const u64 *b, u64 *x, int accumulate)
{
    int N = c->N, L = c->L, nA = c->nA;
    /* lifts: [poly 4][aux k][N] */
    u64 *lift = (u64 *)malloc(sizeof(u64) * 4 * (size_t)nA * N);
    const u64 *src[4] = {a, a + (size_t)L * N, b, b + (size_t)L * N};
#pragma omp parallel for schedule(static)
    for (int idx = 0; idx < 4 * N; idx++) {
        int pi = idx / N, k = idx % N;
        u64 r[OR_MAX_L], o[OR_MAX_AUX];
        for (int i = 0; i < L; i++) r[i] = src[pi][(size_t)i * N + k];
        lift_centered_to_aux(c, r, o);
        for (int m = 0; m < nA; m++) lift[((size_t)pi * nA + m) * N + k] = o[m];
    }
    for (int m = 0; m < nA; m++) {
        u64 rm = c->aux[m];
        const u64 *A0 = lift + ((size_t)0 * nA + m) * N, *A1 = lift + ((size_t)1 * nA + m) * N;
        const u64 *B0 = lift + ((size_t)2 * nA + m) * N, *B1 = lift + ((size_t)3 * nA + m) * N;
        u64 *X0 = x + ((size_t)0 * nA + m) * N, *X1 = x + ((size_t)1 * nA + m) * N, *X2 = x + ((size_t)2 * nA + m) * N;
        negacyclic_acc(rm, N, A0, B0, X0, accumulate);
        negacyclic_acc(rm, N, A0, B1, X1, accumulate);
        negacyclic_acc(rm, N, A1, B0, X1, 1);
        negacyclic_acc(rm, N, A1, B1, X2, accumulate);
    }
    free(lift);
}

/* d_k = round(t x_k / Q) mod Q for x given over the auxiliary base. */
static void scale_round_aux(const or_ctx *c, const u64 *x, u64 *d)
{
    int N = c->N, L = c->L, nA = c->nA;
#pragma omp parallel for schedule(static)
    for (int idx = 0; idx < 3 * N; idx++) {
        int pi = idx / N, k = idx % N;
        u64 xr[OR_MAX_AUX], dd[OR_MAX_L];
        for (int m = 0; m < nA; m++) xr[m] = x[((size_t)pi * nA + m) * N + k];
        scale_round_coeff(c, xr, dd);
        for (int i = 0; i < L; i++) d[((size_t)pi * L + i) * N + k] = dd[i];
    }
}

/* BFV tensor product and scale-and-round, coefficient form:
 *   d_k = round(t x_k / Q) mod Q with the exact tensor x of a and b.
 * a, b: [2][L][N]; d: [3][L][N]. */
int or_tensor_scale(void *vc, const u64 *a, const u64 *b, u64 *d)
{
    return or_tensor_scale_sum(vc, 1, &a, &b, d);
}

/* The same for the sum of n exact tensors (n <= OR_MAX_GROUP):
 *   d_k = round(t (x_k(a_0, b_0) + ... + x_k(a_{n-1}, b_{n-1})) / Q) mod Q,
 * one rounding for the whole sum (the grouped accumulate-then-round order). */
int or_tensor_scale_sum(void *vc, int n, const u64 *const *a, const u64 *const *b, u64 *d)
{
    or_ctx *c = (or_ctx *)vc;
    if (n < 1 || n > OR_MAX_GROUP) return 1;
    u64 *x = (u64 *)malloc(sizeof(u64) * 3 * (size_t)c->nA * c->N);
    for (int m = 0; m < n; m++) tensor_aux(c, a[m], b[m], x, m > 0);
    scale_round_aux(c, x, d);
    free(x);
    return 0;
}

/* Relinearisation of (d0, d1, d2), coefficient form: with the unsigned
 * digits D_j = [d2]_{q_j} in [0, q_j),
 *   c0 = d0 + sum_j D_j b_j,   c1 = d1 + sum_j D_j a_j   (mod each q_i). */
int or_relin(void *vc, const u64 *d, u64 *out)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 *Dm = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        u64 *c0 = out + (size_t)i * N, *c1 = out + ((size_t)L + i) * N;
        memcpy(c0, d + ((size_t)0 * L + i) * N, sizeof(u64) * N);
        memcpy(c1, d + ((size_t)1 * L + i) * N, sizeof(u64) * N);
        for (int j = 0; j < L; j++) {
            const u64 *Dj = d + ((size_t)2 * L + j) * N; /* digit j: d2's residue mod q_j */
            for (int k = 0; k < N; k++) Dm[k] = Dj[k] % qi;
            negacyclic_acc(qi, N, Dm, rlk_poly(c, j, 0, i), c0, 1);
            negacyclic_acc(qi, N, Dm, rlk_poly(c, j, 1, i), c1, 1);
        }
    }
    free(Dm);
    return 0;
}

/* One product of Alg. 1's inner loop: multiply then relinearise. */
int or_mul_relin(void *vc, const u64 *a, const u64 *b, u64 *out)
{
    or_ctx *c = (or_ctx *)vc;
    u64 *d = (u64 *)malloc(sizeof(u64) * 3 * (size_t)c->L * c->N);
    or_tensor_scale(vc, a, b, d);
    or_relin(vc, d, out);
    free(d);
    return 0;
}

/* acc += x (mod q_i), both [2][L][N]: Alg. 1's accumulation into the result. */
void or_add(void *vc, u64 *acc, const u64 *x)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < L; i++)
            for (int k = 0; k < N; k++) {
                size_t o = ((size_t)p * L + i) * N + k;
                acc[o] = addmod(acc[o], x[o], c->q[i]);
            }
}

/* One output entry: its products f0 .. f0+count-1 in order, in groups of
 * `group` consecutive products; each group's exact tensors are summed,
 * scaled and rounded once and relinearised, and the groups are added.  With
 * group = 1 this is Alg. 1's inner loop (multiply, relinearise, add per
 * product). */
static void entry_grouped(void *vc, int f0, int count, const u64 *const *a_ptr, const u64 *const *b_ptr, u64 *acc,
                          int group, u64 *d, u64 *prod)
{
    for (int p = 0; p < count; p += group) {
        int n = count - p < group ? count - p : group;
        or_tensor_scale_sum(vc, n, a_ptr + f0 + p, b_ptr + f0 + p, d);
        or_relin(vc, d, prod);
        or_add(vc, acc, prod);
    }
}

/* Paper's multithreaded scheme (Sec. 3.4): result value (row, col) is
 * computed by thread (row * col) mod nthreads, each thread running the
 * product loop of Alg. 1 for its entries.  Entries e = 0..n_entries-1 list
 * (row, col, first, count) into the flat product arrays a_ptr / b_ptr, which
 * point at [2][L][N] coefficient-form ciphertexts.  out: [n_entries][2][L][N].
 * group: products per rounding (1 = per product, as in Alg. 1; see
 * entry_grouped).  Inner parallelism is switched off for the duration. */
int or_matmul_entries_grouped(void *vc, int n_entries, const int32_t *ent /* [n][4] */,
                              const u64 *const *a_ptr, const u64 *const *b_ptr, u64 *out, int nthreads, int group)
{
    or_ctx *c = (or_ctx *)vc;
    if (group < 1 || group > OR_MAX_GROUP) return 1;
    size_t ctw = 2 * (size_t)c->L * c->N;
    memset(out, 0, sizeof(u64) * ctw * (size_t)n_entries);
#ifdef _OPENMP
    int saved = omp_get_max_threads();
    if (nthreads < 1) nthreads = saved;
    omp_set_max_active_levels(1);
#pragma omp parallel num_threads(nthreads)
    {
        int tid = omp_get_thread_num(), nt = omp_get_num_threads();
        u64 *prod = (u64 *)malloc(sizeof(u64) * ctw);
        u64 *d = (u64 *)malloc(sizeof(u64) * 3 * (size_t)c->L * c->N);
        for (int e = 0; e < n_entries; e++) {
            long long row = ent[4 * e], col = ent[4 * e + 1];
            if ((int)((row * col) % nt) != tid) continue;
            entry_grouped(vc, ent[4 * e + 2], ent[4 * e + 3], a_ptr, b_ptr, out + ctw * e, group, d, prod);
        }
        free(prod);
        free(d);
    }
#else
    (void)nthreads;
    u64 *prod = (u64 *)malloc(sizeof(u64) * ctw);
    u64 *d = (u64 *)malloc(sizeof(u64) * 3 * (size_t)c->L * c->N);
    for (int e = 0; e < n_entries; e++)
        entry_grouped(vc, ent[4 * e + 2], ent[4 * e + 3], a_ptr, b_ptr, out + ctw * e, group, d, prod);
    free(prod);
    free(d);
#endif
    return 0;
}

int or_matmul_entries(void *vc, int n_entries, const int32_t *ent, const u64 *const *a_ptr, const u64 *const *b_ptr,
                      u64 *out, int nthreads)
{
    return or_matmul_entries_grouped(vc, n_entries, ent, a_ptr, b_ptr, out, nthreads, 1);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}


/* ------------------------------------------------------------------ */
/* slot packing, rotations and the slot-zero mask (Sec. 3.2, Alg. 1      */
/* with chunk size c > 1)                                               */
/* ------------------------------------------------------------------ */
/* Slots of a plaintext polynomial m in Z_t[X]/(X^N + 1), t prime with
 * t = 1 mod 2N: slot s = (r, j), r = s / (N/2), j = s mod (N/2), holds
 * m(zeta^e_s) with e_s = 3^j mod 2N for r = 0 and -3^j mod 2N for r = 1,
 * zeta the smallest primitive 2N-th root of unity mod t.  X -> X^(3^k)
 * then moves slot (r, j + k) to slot (r, j): a left rotation by k of each
 * row of N/2 slots. */
static int slot_exp(int N, int s)
{
    int half = N / 2, j = s % half, r = s / half;
    u64 e = 1;
    for (int i = 0; i < j; i++) e = e * 3 % (2 * (u64)N);
    return r == 0 ? (int)e : (int)(2 * (u64)N - e);
}

/* vals[s] = m(zeta^e_s), by direct evaluation */
int or_slots_decode(int N, u64 t, const u64 *poly, u64 *vals)
{
    u64 zeta = or_psi(t, N);
    if (!zeta) return 1;
    u64 *zp = (u64 *)malloc(sizeof(u64) * 2 * (size_t)N);  /* zeta^x, x < 2N */
    zp[0] = 1;
    for (int x = 1; x < 2 * N; x++) zp[x] = mulmod(zp[x - 1], zeta, t);
#pragma omp parallel for schedule(static)
    for (int s = 0; s < N; s++) {
        u64 e = (u64)slot_exp(N, s), acc = 0;
        for (int k = 0; k < N; k++) acc = addmod(acc, mulmod(poly[k] % t, zp[(e * (u64)k) % (2 * (u64)N)], t), t);
        vals[s] = acc;
    }
    free(zp);
    return 0;
}

/* the polynomial with the given slots: m_k = N^-1 sum_s vals[s] zeta^(-e_s k)
 * (the e_s run over every odd residue mod 2N, and zeta^2 is a primitive
 * N-th root, so this inverts the evaluation above) */
int or_slots_encode(int N, u64 t, const u64 *vals, u64 *poly)
{
    u64 zeta = or_psi(t, N);
    if (!zeta) return 1;
    u64 zinv = invmod(zeta, t), ninv = invmod((u64)N % t, t);
    u64 *zm = (u64 *)malloc(sizeof(u64) * 2 * (size_t)N);  /* zeta^-x, x < 2N */
    int *ex = (int *)malloc(sizeof(int) * (size_t)N);
    zm[0] = 1;
    for (int x = 1; x < 2 * N; x++) zm[x] = mulmod(zm[x - 1], zinv, t);
    for (int s = 0; s < N; s++) ex[s] = slot_exp(N, s);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < N; k++) {
        u64 acc = 0;
        for (int s = 0; s < N; s++) acc = addmod(acc, mulmod(vals[s] % t, zm[((u64)ex[s] * (u64)k) % (2 * (u64)N)], t), t);
        poly[k] = mulmod(acc, ninv, t);
    }
    free(zm);
    free(ex);
    return 0;
}

/* every coefficient of the message: m_k = floor((t v_k + floor(Q/2)) / Q)
 * mod t in [0, t), v = [c0 + c1 s]_Q; noise_bits as in or_decrypt, against
 * the whole polynomial Delta m */
int or_decrypt_poly(void *vc, const u64 *ct, u64 *m_out, int *noise_bits)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 *v = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        or_negacyclic(qi, N, ct + ((size_t)L + i) * N, c->s_mod + (size_t)i * N, v + (size_t)i * N);
        for (int k = 0; k < N; k++) v[(size_t)i * N + k] = addmod(v[(size_t)i * N + k], ct[(size_t)i * N + k] % qi, qi);
    }
    int maxbits = 0;
    for (int k = 0; k < N; k++) {
        u64 r[OR_MAX_L];
        for (int i = 0; i < L; i++) r[i] = v[(size_t)i * N + k];
        mw_t V, num, quo, dm, tmp;
        crt_reconstruct(&c->Qb, r, &V);
        mw_mul_u64(&num, &V, c->t);
        mw_add(&num, &num, &c->Qb.half);
        mw_divmod(&num, &c->Qb.M, &quo, NULL);
        u64 mu = mw_mod_u64(&quo, c->t);
        m_out[k] = mu;
        mw_mul_u64(&dm, &c->Delta, mu);
        while (mw_cmp(&dm, &c->Qb.M) >= 0) mw_sub(&dm, &dm, &c->Qb.M);
        if (mw_cmp(&V, &dm) >= 0) mw_sub(&tmp, &V, &dm);
        else { mw_sub(&tmp, &c->Qb.M, &dm); mw_add(&tmp, &tmp, &V); }
        if (mw_cmp(&tmp, &c->Qb.half) > 0) mw_sub(&tmp, &c->Qb.M, &tmp);
        int bits = mw_bitlen(&tmp);
        if (bits > maxbits) maxbits = bits;
    }
    if (noise_bits) *noise_bits = maxbits;
    free(v);
    return 0;
}

/* sigma_g: X -> X^g (g odd) on one polynomial mod q in coefficient form:
 * coefficient k moves to k g mod 2N, negated when that lands at or past N */
static void automorphism(int N, u64 q, u64 g, const u64 *in, u64 *out)
{
    for (int k = 0; k < N; k++) {
        u64 d = ((u64)k * g) % (2 * (u64)N);
        if (d < (u64)N) out[d] = in[k] % q;
        else out[d - N] = submod(0, in[k] % q, q);
    }
}

/* Galois key for g, same layout as the relinearisation key
 * ([L digit j][2 (b, a)][L limb i][N]):
 *   b_j = -a_j s + e_j + g_j sigma_g(s),  a_j uniform,
 * g_j the gadget of or_ctx_create (g_j == delta_ij mod q_i).  a_j from the
 * stream (DOM_GAL_A, g, j) at index i N + k, e_j from (DOM_GAL_E, g, j). */
int or_galois_key(void *vc, u64 g, u64 *key)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    if (!(g & 1)) return 1;
    u64 *tmp = (u64 *)malloc(sizeof(u64) * N);
    u64 *sg = (u64 *)malloc(sizeof(u64) * N);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * N);
    int rc = 0;
    for (int j = 0; j < L; j++) {
        u64 ka = sm_key(c->seed, DOM_GAL_A, g, (u64)j, 0);
        u64 ke = sm_key(c->seed, DOM_GAL_E, g, (u64)j, 0);
        for (int k = 0; k < N; k++) e[k] = sample_gauss(ke, (u64)k, c->cdt);
        for (int i = 0; i < L; i++) {
            u64 qi = c->q[i];
            u64 *a = key + (((size_t)j * 2 + 1) * L + i) * N, *b = key + (((size_t)j * 2 + 0) * L + i) * N;
            for (int k = 0; k < N; k++)
                if (sample_uniform(ka, (u64)i * N + k, qi, &a[k])) rc = -1;
            or_negacyclic(qi, N, a, c->s_mod + (size_t)i * N, tmp);
            automorphism(N, qi, g, c->s_mod + (size_t)i * N, sg);
            for (int k = 0; k < N; k++) {
                u64 ek = e[k] >= 0 ? (u64)e[k] : qi - (u64)(-e[k]);
                u64 v = submod(ek, tmp[k], qi);
                if (i == j) v = addmod(v, sg[k], qi);
                b[k] = v;
            }
        }
    }
    free(tmp);
    free(sg);
    free(e);
    return rc;
}

/* Rotation: (c0', c1') = (sigma_g(c0), sigma_g(c1)) decrypts under
 * sigma_g(s); switch it back to s with the Galois key, digits
 * D_j = [c1']_{q_j} in [0, q_j):
 *   out = (c0' + sum_j D_j b_j,  sum_j D_j a_j)   (mod each q_i). */
int or_rotate(void *vc, const u64 *ct, u64 g, const u64 *key, u64 *out)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 *c1g = (u64 *)malloc(sizeof(u64) * (size_t)L * N);
    u64 *Dm = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < L; i++) {
        automorphism(N, c->q[i], g, ct + (size_t)i * N, out + (size_t)i * N);
        automorphism(N, c->q[i], g, ct + ((size_t)L + i) * N, c1g + (size_t)i * N);
        memset(out + ((size_t)L + i) * N, 0, sizeof(u64) * N);
    }
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        u64 *c0 = out + (size_t)i * N, *c1 = out + ((size_t)L + i) * N;
        for (int j = 0; j < L; j++) {
            const u64 *Dj = c1g + (size_t)j * N;
            for (int k = 0; k < N; k++) Dm[k] = Dj[k] % qi;
            negacyclic_acc(qi, N, Dm, key + (((size_t)j * 2 + 0) * L + i) * N, c0, 1);
            negacyclic_acc(qi, N, Dm, key + (((size_t)j * 2 + 1) * L + i) * N, c1, 1);
        }
    }
    free(c1g);
    free(Dm);
    return 0;
}

/* ciphertext times plaintext polynomial pt (coefficients in [0, t), lifted
 * to their centred representatives in (-t/2, t/2]): (c0 pt, c1 pt) mod q_i;
 * it decrypts to the slot-wise product of the two messages */
int or_mul_plain(void *vc, const u64 *ct, const u64 *pt, u64 *out)
{
    or_ctx *c = (or_ctx *)vc;
    int N = c->N, L = c->L;
    u64 *pm = (u64 *)malloc(sizeof(u64) * N);
    for (int i = 0; i < L; i++) {
        u64 qi = c->q[i];
        for (int k = 0; k < N; k++) {
            u64 v = pt[k] % c->t;
            pm[k] = v > c->t / 2 ? qi - (c->t - v) : v;
        }
        for (int p = 0; p < 2; p++)
            or_negacyclic(qi, N, ct + ((size_t)p * L + i) * N, pm, out + ((size_t)p * L + i) * N);
    }
    free(pm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* helpers of the CKKS oracle (oracle/ckks.py, the parameter set of      */
/* Sec. 3.1): prime lists of other sizes, the generator's samplers as     */
/* whole polynomials, scalar products                                    */
/* ------------------------------------------------------------------ */
/* The primes p = 1 mod 2N below 2^bits in descending order, the first
 * `skip` of them left out, `count` of them into out. */
int or_ntt_primes_bits(int N, int bits, int skip, int count, u64 *out)
{
    u64 twoN = 2 * (u64)N;
    u64 k = ((1ULL << bits) - 2) / twoN;
    int seen = 0, got = 0;
    while (got < count && k > 0) {
        u64 p = k * twoN + 1;
        if (or_is_prime(p)) {
            if (seen >= skip) out[got++] = p;
            seen++;
        }
        k--;
    }
    return got == count ? 0 : -1;
}

/* One polynomial of the stream (seed, dom, o0, o1, o2), as residues mod q:
 * kind 0: uniform residues mod q, coefficient k from slot limb N + k;
 * kind 1: ternary, coefficient k from slot k;
 * kind 2: the rounded Gaussian of the table T20 (or_cdt), slot k.
 * Returns -1 if a rejection sampler ran out of words. */
int or_sample_poly(u64 seed, u64 dom, u64 o0, u64 o1, u64 o2, int kind, u64 q, int limb, int N, const u64 *T20,
                   u64 *out)
{
    u64 key = sm_key(seed, dom, o0, o1, o2);
    int rc = 0;
    for (int k = 0; k < N; k++) {
        if (kind == 0) {
            if (sample_uniform(key, (u64)limb * N + k, q, &out[k])) rc = -1;
        } else if (kind == 1) {
            int v = 0;
            if (sample_ternary(key, (u64)k, &v)) rc = -1;
            out[k] = v >= 0 ? (u64)v : q - 1;
        } else {
            int64_t e = sample_gauss(key, (u64)k, T20);
            out[k] = e >= 0 ? (u64)e : q - (u64)(-e);
        }
    }
    return rc;
}

/* out = a * s mod q, coefficient by coefficient (a < q, any s) */
void or_mul_scalar(u64 q, int N, const u64 *a, u64 s, u64 *out)
{
    s %= q;
    for (int k = 0; k < N; k++) out[k] = mulmod(a[k], s, q);
}
