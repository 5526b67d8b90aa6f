// host_math.cpp -- number theory on the host for the RNS bases.
#include "host_math.h"

#include <utility>

#include <math.h>
#include <string.h>

namespace sfhe {

typedef unsigned __int128 u128;

static inline uint64_t mulm(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

static uint64_t powm(uint64_t base, uint64_t exp, uint64_t m)
{
    uint64_t acc = 1 % m;
    base %= m;
    for (; exp; exp >>= 1) {
        if (exp & 1) acc = mulm(acc, base, m);
        base = mulm(base, base, m);
    }
    return acc;
}

static uint64_t invm(uint64_t a, uint64_t m) { return powm(a % m, m - 2, m); }  // m prime

static ShoupC shoup_of(uint64_t w, uint64_t q)
{
    ShoupC c;
    c.w = w;
    c.ws = (uint64_t)(((u128)w << 64) / q);
    return c;
}

static Shoup32 shoup32_of(uint64_t w, uint64_t b)
{
    Shoup32 c;
    c.w = (uint32_t)w;
    c.ws = (uint32_t)((w << 32) / b);
    return c;
}

bool is_prime_u64(uint64_t n)
{
    static const uint64_t witnesses[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t w : witnesses) {
        if (n % w == 0) return n == w;
    }
    int s = 0;
    uint64_t d = n - 1;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : witnesses) {
        uint64_t x = powm(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness_of_composite = true;
        for (int r = 1; r < s && witness_of_composite; ++r) {
            x = mulm(x, x, n);
            if (x == n - 1) witness_of_composite = false;
        }
        if (witness_of_composite) return false;
    }
    return true;
}

bool ntt_primes(uint32_t N, int count, std::vector<uint64_t>& out, int bits)
{
    out.clear();
    const uint64_t step = 2ULL * N;
    // largest candidate of the form k 2N + 1 below 2^bits
    uint64_t cand = (((1ULL << bits) - 1) / step) * step + 1;
    if (cand >= (1ULL << bits)) cand -= step;
    while ((int)out.size() < count && cand > step) {
        if (is_prime_u64(cand)) out.push_back(cand);
        cand -= step;
    }
    return (int)out.size() == count;
}

uint64_t min_primitive_2n_root(uint64_t q, uint32_t N)
{
    const uint64_t order = 2ULL * N;
    uint64_t root = 0;
    for (uint64_t g = 2; g < q && !root; ++g) {
        uint64_t r = powm(g, (q - 1) / order, q);
        if (powm(r, N, q) == q - 1) root = r;  // r^N = -1: order exactly 2N
    }
    // the primitive 2N-th roots are root^k, k odd; keep the smallest
    uint64_t best = root, r2 = mulm(root, root, q), cur = root;
    for (uint32_t k = 1; k < N; ++k) {
        cur = mulm(cur, r2, q);
        if (cur < best) best = cur;
    }
    return best;
}

// ------------------------------------------------------------- slots ---
// slot s = (r, j) = (s / (N/2), s mod (N/2)) holds m(zeta^e_s), e_s = 3^j
// (r = 0) or -3^j (r = 1) mod 2N, zeta the smallest primitive 2N-th root of
// unity mod t; the e_s are the odd residues mod 2N, so the slots are the
// negacyclic transform m(zeta^(2i+1)), i = (e_s - 1) / 2, reordered.
static void slot_positions(uint32_t N, std::vector<uint32_t>& pos)
{
    pos.resize(N);
    uint64_t x = 1;
    for (uint32_t j = 0; j < N / 2; ++j) {
        pos[j] = (uint32_t)((x - 1) / 2);
        pos[N / 2 + j] = (uint32_t)((2ULL * N - x - 1) / 2);
        x = x * 3 % (2ULL * N);
    }
}

// y_i = sum_k a_k w^(ik), natural order, w of order N (radix-2, in place)
static void cyclic_dft(std::vector<uint64_t>& a, uint64_t w, uint64_t t)
{
    const uint32_t N = (uint32_t)a.size();
    int bits = 0;
    while ((1u << bits) < N) ++bits;
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t r = 0;
        for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1u) << (bits - 1 - b);
        if (i < r) std::swap(a[i], a[r]);
    }
    for (uint32_t len = 2; len <= N; len <<= 1) {
        const uint64_t wl = powm(w, N / len, t);
        for (uint32_t i = 0; i < N; i += len) {
            uint64_t x = 1;
            for (uint32_t k = 0; k < len / 2; ++k) {
                const uint64_t u = a[i + k], v = mulm(a[i + k + len / 2], x, t);
                a[i + k] = (u + v) % t;
                a[i + k + len / 2] = (u + t - v) % t;
                x = mulm(x, wl, t);
            }
        }
    }
}

static bool slot_params(uint32_t N, uint64_t t, uint64_t& zeta)
{
    if (N < 4 || (N & (N - 1)) || t < 3 || (t - 1) % (2ULL * N) || !is_prime_u64(t)) return false;
    zeta = min_primitive_2n_root(t, N);
    return zeta != 0;
}

bool slots_decode(uint32_t N, uint64_t t, const int64_t* poly, int64_t* vals)
{
    uint64_t zeta;
    if (!slot_params(N, t, zeta)) return false;
    std::vector<uint64_t> a(N);
    uint64_t z = 1;
    for (uint32_t k = 0; k < N; ++k) {
        const int64_t m = poly[k] % (int64_t)t;
        a[k] = mulm(m < 0 ? (uint64_t)(m + (int64_t)t) : (uint64_t)m, z, t);
        z = mulm(z, zeta, t);
    }
    cyclic_dft(a, mulm(zeta, zeta, t), t);
    std::vector<uint32_t> pos;
    slot_positions(N, pos);
    for (uint32_t s = 0; s < N; ++s) vals[s] = (int64_t)a[pos[s]];
    return true;
}

bool slots_encode(uint32_t N, uint64_t t, const int64_t* vals, int64_t* poly)
{
    uint64_t zeta;
    if (!slot_params(N, t, zeta)) return false;
    std::vector<uint32_t> pos;
    slot_positions(N, pos);
    std::vector<uint64_t> y(N);
    for (uint32_t s = 0; s < N; ++s) {
        const int64_t v = vals[s] % (int64_t)t;
        y[pos[s]] = v < 0 ? (uint64_t)(v + (int64_t)t) : (uint64_t)v;
    }
    const uint64_t zi = invm(zeta, t);
    cyclic_dft(y, mulm(zi, zi, t), t);
    const uint64_t ninv = invm(N % t, t);
    uint64_t z = 1;
    for (uint32_t k = 0; k < N; ++k) {
        poly[k] = (int64_t)mulm(mulm(y[k], ninv, t), z, t);
        z = mulm(z, zi, t);
    }
    return true;
}

void cdt_table(double sigma, uint64_t* T)
{
    // rho(k) = exp(-k^2 / (2 sigma^2)); S = rho(0) + 2 (rho(1) + ... + rho(19));
    // T[k] = floor(2^63 (rho(0) + 2 (rho(1) + ... + rho(k))) / S), T[19] = 2^63
    double rho[20];
    const double den = 2.0 * sigma * sigma;
    for (int k = 0; k < 20; ++k) rho[k] = exp(-((double)(k * k)) / den);
    double tail = 0.0;
    for (int k = 1; k < 20; ++k) tail = tail + rho[k];
    const double S = rho[0] + 2.0 * tail;
    double run = 0.0;
    for (int k = 0; k < 19; ++k) {
        if (k) run = run + rho[k];
        T[k] = (uint64_t)ldexp((rho[0] + 2.0 * run) / S, 63);
    }
    T[19] = 1ULL << 63;
}

static uint32_t bit_reverse(uint32_t x, int bits)
{
    uint32_t r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

// psi^(+-bitrev(k)) for k < N
static void root_tables(uint64_t q, uint32_t N, std::vector<uint64_t>& fwd, std::vector<uint64_t>& inv)
{
    int logn = 0;
    while ((1u << logn) < N) ++logn;
    const uint64_t psi = min_primitive_2n_root(q, N);
    const uint64_t ipsi = invm(psi, q);
    std::vector<uint64_t> pw(N), ipw(N);
    pw[0] = ipw[0] = 1;
    for (uint32_t k = 1; k < N; ++k) {
        pw[k] = mulm(pw[k - 1], psi, q);
        ipw[k] = mulm(ipw[k - 1], ipsi, q);
    }
    fwd.resize(N);
    inv.resize(N);
    for (uint32_t k = 0; k < N; ++k) {
        const uint32_t r = bit_reverse(k, logn);
        fwd[k] = pw[r];
        inv[k] = ipw[r];
    }
}

void twiddles(uint64_t q, uint32_t N, uint64_t* out, ShoupC* ninv, ShoupC* wlast)
{
    std::vector<uint64_t> f, g;
    root_tables(q, N, f, g);
    for (uint32_t k = 0; k < N; ++k) {
        const ShoupC a = shoup_of(f[k], q), b = shoup_of(g[k], q);
        out[k] = a.w;
        out[N + k] = a.ws;
        out[2 * N + k] = b.w;
        out[3 * N + k] = b.ws;
    }
    const uint64_t ni = invm(N, q);
    *ninv = shoup_of(ni, q);
    *wlast = shoup_of(mulm(g[1], ni, q), q);
}

void twiddles32(uint32_t b, uint32_t N, uint32_t* out, Shoup32* ninv, Shoup32* wlast)
{
    std::vector<uint64_t> f, g;
    root_tables(b, N, f, g);
    for (uint32_t k = 0; k < N; ++k) {
        const Shoup32 x = shoup32_of(f[k], b), y = shoup32_of(g[k], b);
        out[k] = x.w;
        out[N + k] = x.ws;
        out[2 * N + k] = y.w;
        out[3 * N + k] = y.ws;
    }
    const uint64_t ni = invm(N, b);
    *ninv = shoup32_of(ni, b);
    *wlast = shoup32_of(mulm(g[1], ni, b), b);
}

// --------------------------------------------------------- multiword ---
namespace {
const int MWW = 20;  // 1280 bits
struct Big {
    uint64_t w[MWW];
};
Big big(uint64_t v)
{
    Big r;
    memset(&r, 0, sizeof(r));
    r.w[0] = v;
    return r;
}
void mul_small(Big& a, uint64_t f)
{
    u128 carry = 0;
    for (int k = 0; k < MWW; ++k) {
        u128 p = (u128)a.w[k] * f + carry;
        a.w[k] = (uint64_t)p;
        carry = p >> 64;
    }
}
void shl(Big& a, int bits)
{
    for (; bits > 0; --bits) {
        for (int k = MWW - 1; k > 0; --k) a.w[k] = (a.w[k] << 1) | (a.w[k - 1] >> 63);
        a.w[0] <<= 1;
    }
}
bool greater(const Big& a, const Big& b)
{
    for (int k = MWW - 1; k >= 0; --k)
        if (a.w[k] != b.w[k]) return a.w[k] > b.w[k];
    return false;
}
void sub(Big& a, const Big& b)  // a -= b, a >= b
{
    uint64_t borrow = 0;
    for (int k = 0; k < MWW; ++k) {
        const uint64_t ak = a.w[k], bk = b.w[k];
        a.w[k] = ak - bk - borrow;
        borrow = (ak < bk) || (ak - bk < borrow);
    }
}
// bitwise long division: a = quo * b + rem
void divmod(const Big& a, const Big& b, Big& quo, Big& rem)
{
    quo = big(0);
    rem = big(0);
    for (int bit = MWW * 64 - 1; bit >= 0; --bit) {
        shl(rem, 1);
        rem.w[0] |= (a.w[bit / 64] >> (bit % 64)) & 1;
        if (!greater(b, rem)) {
            sub(rem, b);
            quo.w[bit / 64] |= 1ULL << (bit % 64);
        }
    }
}
uint64_t mod_small(const Big& a, uint64_t m)
{
    uint64_t r = 0;
    for (int k = MWW - 1; k >= 0; --k) r = (uint64_t)((((u128)r << 64) | a.w[k]) % m);
    return r;
}
}  // namespace

// product of the chosen moduli (mod m), skipping index `skip`
static uint64_t prod_q(const RnsConsts& rc, int skip, uint64_t m)
{
    uint64_t acc = 1 % m;
    for (int i = 0; i < rc.L; ++i)
        if (i != skip) acc = mulm(acc, rc.m[i].q % m, m);
    return acc;
}
static uint64_t prod_b(const RnsConsts& rc, int count, int skip, uint64_t m)
{
    uint64_t acc = 1 % m;
    for (int k = 0; k < count; ++k)
        if (k != skip) acc = mulm(acc, rc.mb[k].b % m, m);
    return acc;
}

bool fill_constants(RnsConsts& rc)
{
    const int L = rc.L, K = rc.K;
    const uint64_t t = rc.t;
    // exact size margin: B > 2 N Q^2 (the centred tensor |x| < N Q^2 / 2)
    Big Qbig = big(1), Bbig = big(1);
    for (int i = 0; i < L; ++i) mul_small(Qbig, rc.m[i].q);
    for (int k = 0; k < K; ++k) mul_small(Bbig, rc.mb[k].b);
    {
        Big need_b = big(rc.N);
        for (int i = 0; i < L; ++i) {
            mul_small(need_b, rc.m[i].q);
            mul_small(need_b, rc.m[i].q);
        }
        shl(need_b, 1);
        if (!greater(Bbig, need_b)) return false;
        // products one rounding may take (grouped accumulate-then-round): a
        // sum of G tensors keeps |x| < B / 4 while G 2 N Q^2 <= B
        Big g, r;
        divmod(Bbig, need_b, g, r);
        bool big_g = g.w[0] > 1024;
        for (int w = 1; w < MWW; ++w) big_g = big_g || g.w[w] != 0;
        rc.lazy_group = big_g ? 1024 : (g.w[0] < 1 ? 1 : (int)g.w[0]);
    }
    for (int i = 0; i < L; ++i) rc.m[i].mu = (uint64_t)(((u128)1 << 114) / rc.m[i].q);
    for (int k = 0; k < K; ++k) {
        const uint64_t b = rc.mb[k].b;
        rc.mb[k].mu61 = (uint32_t)((1ULL << 61) / b);
        rc.mb[k].mu64 = (uint64_t)(((u128)1 << 64) / b);
        uint32_t inv = 1;  // b^-1 mod 2^32 by Newton's iteration (b odd)
        for (int it = 0; it < 5; ++it) inv *= 2u - (uint32_t)b * inv;
        rc.mb[k].binv = 0u - inv;
        rc.mb[k].pad = 0;
    }

    // ---- Q side, lift Q -> B and the exact-rounding words
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = rc.m[i].q;
        const uint64_t qhat = prod_q(rc, i, qi);
        rc.qhat_inv[i] = shoup_of(invm(qhat, qi), qi);
        rc.t_q[i] = shoup_of(t % qi, qi);
        for (int k = 0; k < K; ++k) {
            const uint64_t b = rc.mb[k].b;
            const uint64_t c = prod_q(rc, i, b);
            rc.qhat_b[i][k] = (uint32_t)c;
            rc.qhat_b27[i][k] = (uint32_t)mulm(c, (1ULL << 27) % b, b);
        }
    }
    for (int k = 0; k < K; ++k) {
        const uint64_t b = rc.mb[k].b;
        rc.negQ_b[k] = (uint32_t)((b - prod_q(rc, -1, b)) % b);
    }
    const int W = SFHE_MAX_L + 1;
    memset(rc.Qw, 0, sizeof(rc.Qw));
    rc.Qw[0] = 1;
    auto mul_words = [](uint64_t* w, int n, uint64_t f) {
        u128 carry = 0;
        for (int k = 0; k < n; ++k) {
            u128 p = (u128)w[k] * f + carry;
            w[k] = (uint64_t)p;
            carry = p >> 64;
        }
    };
    for (int i = 0; i < L; ++i) mul_words(rc.Qw, W, rc.m[i].q);
    int words = W;
    while (words > 1 && rc.Qw[words - 1] == 0) --words;
    rc.Qwords = words;
    for (int i = 0; i < L; ++i) {
        memset(rc.Qhat_w[i], 0, sizeof(rc.Qhat_w[i]));
        rc.Qhat_w[i][0] = 1;
        for (int k = 0; k < L; ++k)
            if (k != i) mul_words(rc.Qhat_w[i], W, rc.m[k].q);
    }

    // ---- tensor from B to Q
    for (int k = 0; k < K; ++k) {
        const uint64_t b = rc.mb[k].b;
        rc.bhat_inv[k] = shoup32_of(invm(prod_b(rc, K, k, b), b), b);
        rc.bfrac[k] = (uint32_t)((1ULL << 43) / b);
    }

    // ---- scale and round directly from B: t (B/b_k) = alpha_k Q + r_k, t B = alpha_B Q + r_B
    auto split_const = [&](const Big& c, Big& alpha, Big& rem, uint64_t& rho) {
        divmod(c, Qbig, alpha, rem);
        Big shifted = rem, quo, r2;
        shl(shifted, 64);
        divmod(shifted, Qbig, quo, r2);  // floor(rem 2^64 / Q) < 2^64
        rho = quo.w[0];
    };
    for (int k = 0; k < K; ++k) {
        Big ck = big(t);
        for (int j = 0; j < K; ++j)
            if (j != k) mul_small(ck, rc.mb[j].b);
        Big alpha, rem;
        uint64_t rho;
        split_const(ck, alpha, rem, rho);
        // the estimate of F uses rho_k without its low 6 bits, in two
        // 29-bit parts: each product with a 30-bit residue stays below 2^59,
        // so the sums of up to 31 of them need no carries
        rc.rho_s[k][0] = (uint32_t)((rho >> 6) & ((1ULL << 29) - 1));
        rc.rho_s[k][1] = (uint32_t)(rho >> 35);
        for (int i = 0; i < L; ++i) {
            const uint64_t a = mod_small(alpha, rc.m[i].q);
            rc.alpha_q_lo[k][i] = (uint32_t)(a & ((1ULL << 27) - 1));
            rc.alpha_q_hi[k][i] = (uint32_t)(a >> 27);
        }
        for (int w = 0; w < SFHE_MAX_L + 1; ++w) rc.r_w[k][w] = rem.w[w];
    }
    {
        Big cB = Bbig;
        mul_small(cB, t);
        Big alpha, rem;
        uint64_t rho;
        split_const(cB, alpha, rem, rho);
        rc.rhoB_lo = (uint32_t)rho;
        rc.rhoB_hi = (uint32_t)(rho >> 32);
        for (int i = 0; i < L; ++i) {
            const uint64_t qi = rc.m[i].q;
            rc.negalphaB_q[i] = (qi - mod_small(alpha, qi)) % qi;
            rc.negK_q[i] = qi - (uint64_t)K;
        }
        for (int w = 0; w < SFHE_MAX_L + 1; ++w) rc.rB_w[w] = rem.w[w];
    }

    // ---- encryption: Delta = floor(Q/t) = (Q - [Q]_t) / t, and Q = 0 mod q_i
    const uint64_t Q_mod_t = prod_q(rc, -1, t);
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = rc.m[i].q;
        rc.delta_q[i] = mulm((qi - Q_mod_t % qi) % qi, invm(t % qi, qi), qi);
    }
    return true;
}

void fold_tensor_scaling(RnsConsts& rc)
{
    for (int k = 0; k < rc.K; ++k) {
        const uint64_t b = rc.mb[k].b, h = mulm(rc.bhat_inv[k].w, (1ULL << 32) % b, b);
        rc.ninv_bx[k] = shoup32_of(mulm(rc.ninv_b[k].w, h, b), b);
        rc.wlast_bx[k] = shoup32_of(mulm(rc.wlast_b[k].w, h, b), b);
    }
}

}  // namespace sfhe
