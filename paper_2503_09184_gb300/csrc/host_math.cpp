// host_math.cpp -- number theory on the host for the RNS bases.
#include "host_math.h"

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

bool ntt_primes(uint32_t N, int count, std::vector<uint64_t>& out)
{
    out.clear();
    const uint64_t step = 2ULL * N;
    // largest candidate of the form k 2N + 1 below 2^54
    uint64_t cand = (((1ULL << 54) - 1) / step) * step + 1;
    if (cand >= (1ULL << 54)) cand -= step;
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

void twiddles(uint64_t q, uint32_t N, uint64_t* out, ShoupC* ninv, ShoupC* wlast)
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
    for (uint32_t k = 0; k < N; ++k) {
        const uint32_t r = bit_reverse(k, logn);
        const ShoupC f = shoup_of(pw[r], q), g = shoup_of(ipw[r], q);
        out[k] = f.w;
        out[N + k] = f.ws;
        out[2 * N + k] = g.w;
        out[3 * N + k] = g.ws;
    }
    const uint64_t ni = invm(N, q);
    *ninv = shoup_of(ni, q);
    *wlast = shoup_of(mulm(out[2 * N + 1], ni, q), q);
}

// product of the moduli in [lo, hi) except `skip`, mod m
static uint64_t prod_mod(const RnsConsts& rc, int lo, int hi, int skip, uint64_t m)
{
    uint64_t acc = 1 % m;
    for (int k = lo; k < hi; ++k)
        if (k != skip) acc = mulm(acc, rc.m[k].q % m, m);
    return acc;
}

void fill_constants(RnsConsts& rc)
{
    const int L = rc.L, Lp = rc.Lp;
    const uint64_t t = rc.t;
    for (int k = 0; k < L + Lp; ++k) rc.m[k].mu = (uint64_t)(((u128)1 << 114) / rc.m[k].q);

    for (int i = 0; i < L; ++i) {
        const uint64_t qi = rc.m[i].q;
        // (Q/q_i)^-1, (QP/q_i)^-1 mod q_i
        const uint64_t qhat = prod_mod(rc, 0, L, i, qi);
        rc.qhat_inv[i] = shoup_of(invm(qhat, qi), qi);
        const uint64_t P_mod = prod_mod(rc, L, L + Lp, -1, qi);
        rc.qphat_inv[i] = shoup_of(invm(mulm(qhat, P_mod, qi), qi), qi);
        rc.tP_q[i] = shoup_of(mulm(t % qi, P_mod, qi), qi);
        rc.negP_mod_q[i] = (qi - P_mod) % qi;
        rc.t_q[i] = shoup_of(t % qi, qi);
        for (int j = 0; j < Lp; ++j) {
            const uint64_t pj = rc.m[L + j].q;
            // [Q/q_i]_{p_j}
            rc.qhat_mod_p[i][j] = prod_mod(rc, 0, L, i, pj);
            // floor(tP/q_i) = (tP - [tP]_{q_i}) / q_i, and tP = 0 mod p_j
            const uint64_t c = rc.tP_q[i].w % pj;
            rc.omega[i][j] = mulm((pj - c) % pj, invm(qi % pj, pj), pj);
        }
    }
    for (int j = 0; j < Lp; ++j) {
        const uint64_t pj = rc.m[L + j].q;
        const uint64_t Q_mod = prod_mod(rc, 0, L, -1, pj);
        rc.negQ_mod_p[j] = (pj - Q_mod) % pj;
        rc.tQinv_p[j] = shoup_of(mulm(t % pj, invm(Q_mod, pj), pj), pj);
        const uint64_t phat_p = prod_mod(rc, L, L + Lp, L + j, pj);
        rc.phat_inv[j] = shoup_of(invm(phat_p, pj), pj);
        for (int i = 0; i < L; ++i) rc.phat_mod_q[j][i] = prod_mod(rc, L, L + Lp, L + j, rc.m[i].q);
    }
    // Q and Q/q_i as little-endian words
    auto mul_words = [](uint64_t* w, int n, uint64_t f) {
        u128 carry = 0;
        for (int k = 0; k < n; ++k) {
            u128 p = (u128)w[k] * f + carry;
            w[k] = (uint64_t)p;
            carry = p >> 64;
        }
    };
    const int W = SFHE_MAX_L + 1;
    memset(rc.Qw, 0, sizeof(rc.Qw));
    rc.Qw[0] = 1;
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
    // Delta = floor(Q/t) = (Q - [Q]_t) / t, and Q = 0 mod q_i
    const uint64_t Q_mod_t = [&] {
        uint64_t a = 1 % t;
        for (int i = 0; i < L; ++i) a = mulm(a, rc.m[i].q % t, t);
        return a;
    }();
    for (int i = 0; i < L; ++i) {
        const uint64_t qi = rc.m[i].q;
        rc.delta_q[i] = mulm((qi - Q_mod_t % qi) % qi, invm(t % qi, qi), qi);
    }
}

}  // namespace sfhe
