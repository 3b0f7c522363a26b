/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for the combinatorial
 * pi(x) method of Staple, "The combinatorial algorithm for computing pi(x)"
 * (arXiv:1503.01839).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) shares no code, header, table or helper with this file.
 *
 * Everything here is written from the mathematics, in exact integers, with no
 * blocking, fusion or reordering beyond what each definition states:
 *
 *   O-A  brute force: segmented sieve of Eratosthenes (Section 1) for pi(x),
 *        and a direct count of n <= x coprime to p_1..p_a for phi(x, a)
 *        (phi defined in Section 3).
 *   O-B  Meissel-Lehmer: pi(x) = phi(x, a) + a - 1 - P2(x, a), with phi(x, a)
 *        evaluated by the naive recursion of Eq. (4.1), cut off only by the
 *        textbook cases phi(v,0)=v, phi(0,k)=0, v < p_{k+1} -> 1 and the
 *        Legendre case of Section 4 (p_k <= v < p_{k+1}^2 -> pi(v) - k + 1).
 *   O-C  per-term brute force of the leaf decomposition the paper builds on
 *        (Section 2 refers to Deleglise-Rivat for it): ordinary leaves S1,
 *        special leaves split into trivial / easy / hard, and P2.  Every
 *        special leaf phi(u, b-1) is read from an incremental full sieve of
 *        [1, z] (Section 3: the main sieve exposes phi(m, b) for all m, b).
 *
 * Readings of the paper used here (the paper defers the formulas to [DR96]):
 *   - x/n always means floor(x/n); nested floors floor(floor(x/p)/m).
 *   - lpf(1) = infinity, mu(1) = 1, phi(v,0) = v, phi(0,a) = 0.
 *   - special leaf (b, m): c < b <= a, m squarefree, lpf(m) > p_b,
 *     gpf(m) <= p_a, floor(y/p_b) < m <= y; u = floor(x/(p_b m)).
 *     trivial: u < p_b; easy: p_b <= u < min(p_b^2, y); hard: otherwise.
 *   - P2(x, a) = sum_{a < b <= pi(isqrt x)} (pi(x/p_b) - b + 1).
 *
 * All 128-bit results are returned as (lo, hi) pairs of int64_t, value =
 * hi * 2^64 + (uint64_t)lo (two's complement).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- roots */

static int bitlen64(uint64_t n) { int k = 0; while (n) { k++; n >>= 1; } return k; }

/* floor(sqrt(n)) by integer Newton iteration from an upper bound. */
uint64_t orc_isqrt(uint64_t n)
{
    if (n < 2) return n;
    uint64_t x = (uint64_t)1 << ((bitlen64(n) + 1) / 2); /* x >= sqrt(n) */
    for (;;) {
        uint64_t y = (x + n / x) >> 1;
        if (y >= x) break;
        x = y;
    }
    return x;
}

static u128 cube128(uint64_t r) { return (u128)r * r * r; }

/* floor(cbrt(n)) by integer Newton iteration plus an exact correction. */
uint64_t orc_iroot3(uint64_t n)
{
    if (n < 8) return n ? 1 : 0;
    uint64_t x = (uint64_t)1 << ((bitlen64(n) + 2) / 3); /* x >= cbrt(n) */
    for (;;) {
        uint64_t y = (2 * x + n / (x * x)) / 3;
        if (y >= x) break;
        x = y;
    }
    while (cube128(x) > n) x--;
    while (cube128(x + 1) <= n) x++;
    return x;
}

/* -------------------------------------------------------- simple sieves */

/* is_prime[0..limit] as bytes (plain Eratosthenes). Caller frees. */
static uint8_t *prime_flags(uint64_t limit)
{
    uint8_t *f = (uint8_t *)malloc(limit + 1);
    if (!f) return NULL;
    memset(f, 1, limit + 1);
    f[0] = 0;
    if (limit >= 1) f[1] = 0;
    for (uint64_t p = 2; p * p <= limit; p++)
        if (f[p])
            for (uint64_t q = p * p; q <= limit; q += p) f[q] = 0;
    return f;
}

/* primes <= limit, 1-indexed: P[1] = 2.  *count = pi(limit).  P has a
 * sentinel slot P[count+1] = next prime above limit. */
static uint64_t *prime_list(uint64_t limit, uint64_t *count)
{
    uint64_t hi = limit < 2 ? 16 : 2 * limit + 16; /* Bertrand: next prime < 2*limit */
    uint8_t *f = prime_flags(hi);
    if (!f) return NULL;
    uint64_t n = 0;
    for (uint64_t i = 2; i <= limit; i++) n += f[i];
    uint64_t *P = (uint64_t *)malloc((n + 2) * sizeof(uint64_t));
    uint64_t k = 0;
    P[0] = 1;
    for (uint64_t i = 2; i <= limit; i++) if (f[i]) P[++k] = i;
    uint64_t nxt = limit + 1;
    while (!f[nxt]) nxt++;
    P[n + 1] = nxt;
    free(f);
    *count = n;
    return P;
}

/* ------------------------------------------------------------------ O-A */

/* pi(x): segmented sieve of Eratosthenes over the odd numbers (Section 1). */
uint64_t orc_pi_sieve(uint64_t x)
{
    if (x < 2) return 0;
    uint64_t r = orc_isqrt(x);
    uint64_t np;
    uint64_t *P = prime_list(r, &np);
    const uint64_t SEG = 1u << 20; /* odd numbers per segment */
    uint8_t *seg = (uint8_t *)malloc(SEG);
    uint64_t count = 1; /* the prime 2 */
    /* odd number 2*i+1, i >= 1 */
    for (uint64_t lo = 1; 2 * lo + 1 <= x; lo += SEG) {
        uint64_t hi = lo + SEG; /* exclusive index */
        uint64_t imax = (x - 1) / 2 + 1;
        if (hi > imax) hi = imax;
        memset(seg, 1, hi - lo);
        for (uint64_t k = 2; k <= np; k++) { /* odd primes */
            uint64_t p = P[k];
            if (p * p > 2 * (hi - 1) + 1) break;
            uint64_t start = p * p; /* first odd multiple >= max(p^2, 2lo+1) */
            uint64_t lown = 2 * lo + 1;
            if (start < lown) {
                start = (lown + p - 1) / p * p;
                if (start % 2 == 0) start += p;
            }
            for (uint64_t m = start; m <= 2 * (hi - 1) + 1; m += 2 * p) seg[(m - 1) / 2 - lo] = 0;
        }
        for (uint64_t i = 0; i < hi - lo; i++) count += seg[i];
    }
    free(seg);
    free(P);
    return count;
}

/* phi(x, a): count of 1 <= n <= x with no prime factor among p_1..p_a,
 * by direct marking (definition of phi in Section 3). */
uint64_t orc_phi_brute(uint64_t x, uint64_t a)
{
    if (x == 0) return 0;
    if (a == 0) return x;
    uint64_t np = 0, lim = 64;
    uint64_t *P = NULL;
    for (;;) { /* find at least a primes */
        P = prime_list(lim, &np);
        if (np >= a) break;
        free(P);
        lim *= 2;
    }
    const uint64_t SEG = 1u << 20;
    uint8_t *seg = (uint8_t *)malloc(SEG);
    uint64_t count = 0;
    for (uint64_t lo = 1; lo <= x; lo += SEG) {
        uint64_t hi = lo + SEG; if (hi > x + 1) hi = x + 1;
        memset(seg, 1, hi - lo);
        for (uint64_t k = 1; k <= a; k++) {
            uint64_t p = P[k];
            uint64_t start = (lo + p - 1) / p * p;
            for (uint64_t m = start; m < hi; m += p) seg[m - lo] = 0;
        }
        for (uint64_t i = 0; i < hi - lo; i++) count += seg[i];
    }
    free(seg);
    free(P);
    return count;
}

/* ------------------------------------------------------------------ O-B */

typedef struct {
    uint64_t *P;      /* primes, 1-indexed, with sentinel */
    uint64_t np;
    uint32_t *pi;     /* pi[v] for v <= L */
    uint64_t L;
} phi_ctx;

static int phi_ctx_init(phi_ctx *c, uint64_t a, uint64_t L)
{
    uint64_t lim = 64;
    for (;;) {
        c->P = prime_list(lim, &c->np);
        if (c->np >= a + 1) break;
        free(c->P);
        lim *= 2;
    }
    if (L < lim) L = lim;
    c->L = L;
    uint8_t *f = prime_flags(L);
    c->pi = (uint32_t *)malloc((L + 1) * sizeof(uint32_t));
    uint32_t s = 0;
    for (uint64_t v = 0; v <= L; v++) { s += f[v]; c->pi[v] = s; }
    free(f);
    return 0;
}

static void phi_ctx_free(phi_ctx *c) { free(c->P); free(c->pi); }

/* Naive recursion phi(v,k) = phi(v,k-1) - phi(floor(v/p_k), k-1), Eq. (4.1).
 * The first term is unrolled into a loop (same recurrence, applied again). */
static int64_t phi_rec(const phi_ctx *c, uint64_t v, uint64_t k)
{
    int64_t acc = 0;
    for (;;) {
        if (k == 0) return acc + (int64_t)v;
        if (v == 0) return acc;
        if (v < c->P[k + 1]) return acc + 1;           /* only n = 1 left */
        if (v <= c->L && (u128)v < (u128)c->P[k + 1] * c->P[k + 1])
            return acc + (int64_t)c->pi[v] - (int64_t)k + 1; /* Legendre case, Section 4 */
        acc -= phi_rec(c, v / c->P[k], k - 1);
        k -= 1;
    }
}

/* phi(x, a) by the naive recursion with a pi table up to L (L = 0: auto). */
uint64_t orc_phi_rec(uint64_t x, uint64_t a, uint64_t L)
{
    if (L == 0) {
        L = orc_isqrt(x) + 1;
        if (L < (1u << 16)) L = 1u << 16;
        if (L > (1u << 26)) L = 1u << 26;
    }
    phi_ctx c;
    phi_ctx_init(&c, a, L);
    int64_t r = phi_rec(&c, x, a);
    phi_ctx_free(&c);
    return (uint64_t)r;
}

/* P2(x, a) = sum over a < b <= pi(isqrt x) of (pi(x / p_b) - b + 1).
 * The pi values are collected in ascending order of x/p_b by one plain
 * segmented sieve of [1, x / p_{a+1}]. */
int orc_p2(uint64_t x, uint64_t a, int64_t *out)
{
    uint64_t r = orc_isqrt(x);
    uint64_t np;
    uint64_t *P = prime_list(r, &np); /* all primes <= isqrt(x) */
    i128 sum = 0;
    if (np > a) {
        uint64_t top = x / P[a + 1];
        uint64_t rt = orc_isqrt(top);
        uint64_t ns;
        uint64_t *S = prime_list(rt, &ns);
        const uint64_t SEG = 1u << 20;
        uint8_t *seg = (uint8_t *)malloc(SEG);
        uint64_t b = np;          /* next query: v = x / P[b], ascending */
        uint64_t count = 0;       /* primes < lo */
        for (uint64_t lo = 0; lo <= top && b > a; lo += SEG) {
            uint64_t hi = lo + SEG; if (hi > top + 1) hi = top + 1;
            memset(seg, 1, hi - lo);
            if (lo == 0) { seg[0] = 0; if (hi > 1) seg[1] = 0; }
            for (uint64_t k = 1; k <= ns; k++) {
                uint64_t p = S[k];
                if (p * p >= hi) break;
                uint64_t start = p * p;
                if (start < lo) start = (lo + p - 1) / p * p;
                for (uint64_t m = start; m < hi; m += p) seg[m - lo] = 0;
            }
            /* answer every query whose v lies in [lo, hi) */
            uint64_t run = count, pos = lo;
            while (b > a) {
                uint64_t v = x / P[b];
                if (v >= hi) break;
                while (pos <= v) { run += seg[pos - lo]; pos++; }
                sum += (i128)run - (i128)b + 1;
                b--;
            }
            for (uint64_t i = pos; i < hi; i++) run += seg[i - lo];
            count = run;
        }
        free(seg);
        free(S);
    }
    free(P);
    out[0] = (int64_t)(uint64_t)(u128)sum;
    out[1] = (int64_t)(uint64_t)((u128)sum >> 64);
    return 0;
}

/* pi(x) = phi(x, a) + a - 1 - P2(x, a), a = pi(y), for any y with
 * iroot3(x) <= y <= isqrt(x) (then P3 = 0).  y = 0 means y = iroot3(x). */
uint64_t orc_pi_meissel(uint64_t x, uint64_t y)
{
    if (x < 2) return 0;
    if (x < 8) { uint64_t c = 0; for (uint64_t n = 2; n <= x; n++) c += (n == 2 || n == 3 || n == 5 || n == 7); return c; }
    if (y == 0) y = orc_iroot3(x);
    uint64_t na;
    uint64_t *Py = prime_list(y, &na);
    free(Py);
    uint64_t a = na;
    uint64_t phi = orc_phi_rec(x, a, 0);
    int64_t p2[2];
    orc_p2(x, a, p2);
    i128 P2 = ((i128)p2[1] << 64) | (uint64_t)p2[0];
    i128 r = (i128)phi + (i128)a - 1 - P2;
    return (uint64_t)r;
}

/* ------------------------------------------------------------------ O-C */

/* Fenwick tree over the 64-bit words of a bitset of [0, n]. */
typedef struct {
    uint64_t *bits;
    int64_t *fw;   /* 1-indexed Fenwick over word popcounts */
    uint64_t nw;
} bitcount;

static void bc_add(bitcount *t, uint64_t w, int64_t d)
{
    for (uint64_t i = w + 1; i <= t->nw; i += i & (~i + 1)) t->fw[i] += d;
}

static int64_t bc_wordprefix(const bitcount *t, uint64_t w) /* sum of words < w */
{
    int64_t s = 0;
    for (uint64_t i = w; i > 0; i -= i & (~i + 1)) s += t->fw[i];
    return s;
}

/* number of set bits at positions 0..v */
static int64_t bc_prefix(const bitcount *t, uint64_t v)
{
    uint64_t w = v >> 6;
    uint64_t mask = (v & 63) == 63 ? ~0ull : ((1ull << ((v & 63) + 1)) - 1);
    return bc_wordprefix(t, w) + __builtin_popcountll(t->bits[w] & mask);
}

static void bc_clear(bitcount *t, uint64_t v)
{
    uint64_t w = v >> 6, m = 1ull << (v & 63);
    if (t->bits[w] & m) { t->bits[w] &= ~m; bc_add(t, w, -1); }
}

static void put128(int64_t *o, i128 v)
{
    o[0] = (int64_t)(uint64_t)(u128)v;
    o[1] = (int64_t)(uint64_t)((u128)v >> 64);
}

/* phi(v, c) for c <= 7 by inclusion-exclusion over the divisors of
 * p_1 * ... * p_c (Legendre's formula). */
static i128 phi_small(uint64_t v, uint32_t c, const uint64_t *P)
{
    i128 s = 0;
    for (uint32_t mask = 0; mask < (1u << c); mask++) {
        uint64_t d = 1; int sg = 1;
        for (uint32_t i = 0; i < c; i++) if (mask & (1u << i)) { d *= P[i + 1]; sg = -sg; }
        s += (i128)sg * (i128)(v / d);
    }
    return s;
}

/*
 * Leaf decomposition of phi(x, a) for a <= pi(y), and P2(x, a):
 *   out[0..1]  S1      ordinary leaves  sum mu(n) phi(x/n, c)
 *   out[2..3]  S2_triv trivial special leaves
 *   out[4..5]  S2_easy easy special leaves
 *   out[6..7]  S2_hard hard special leaves
 *   out[8..9]  P2(x, a)
 *   out[10] a, out[11] number of trivial, out[12] easy, out[13] hard leaves,
 *   out[14] number of ordinary leaves, out[15] z = floor(x/y),
 *   out[16] B = pi(isqrt z).
 * a_in = 0 selects a = pi(y).  Requires 1 <= y <= isqrt(x), c <= 7,
 * c <= a, p_a <= y.  Returns 0, or -1 on a domain error.
 */
int orc_leaf_sums(uint64_t x, uint64_t y, uint32_t c, uint64_t a_in, int64_t *out)
{
    if (y < 1 || y > orc_isqrt(x) || c > 7) return -1;
    uint64_t z = x / y;
    uint64_t lim = y;
    if (orc_isqrt(x) > lim) lim = orc_isqrt(x);
    if (lim < 32) lim = 32;
    uint64_t np;
    uint64_t *P = prime_list(lim, &np);
    uint64_t piy = 0;
    while (piy < np && P[piy + 1] <= y) piy++;
    uint64_t a = a_in ? a_in : piy;
    if (a > piy || c > a) { free(P); return -1; }

    /* lpf, mu and gpf of every n <= y (plain smallest-factor sieve). */
    uint32_t *lpf = (uint32_t *)calloc(y + 1, sizeof(uint32_t)); /* prime index */
    for (uint64_t k = 1; k <= np && P[k] <= y; k++)
        for (uint64_t q = P[k]; q <= y; q += P[k])
            if (!lpf[q]) lpf[q] = (uint32_t)k;
    int8_t *mu = (int8_t *)malloc(y + 1);
    uint32_t *gpf = (uint32_t *)calloc(y + 1, sizeof(uint32_t));
    mu[1] = 1; gpf[1] = 0;
    for (uint64_t n = 2; n <= y; n++) {
        uint64_t p = P[lpf[n]];
        uint64_t r = n / p;
        if (r % p == 0) mu[n] = 0; else mu[n] = (int8_t)(-mu[r]);
        gpf[n] = r == 1 ? lpf[n] : gpf[r];
    }

    /* ordinary leaves (n <= y, n = 1 or lpf(n) > p_c, gpf(n) <= p_a) */
    i128 S1 = 0; int64_t nord = 0;
    for (uint64_t n = 1; n <= y; n++) {
        if (mu[n] == 0) continue;
        if (n > 1 && (lpf[n] <= c || gpf[n] > a)) continue;
        S1 += (i128)mu[n] * phi_small(x / n, c, P);
        nord++;
    }

    /* special leaves from an incremental sieve of [1, z] */
    bitcount t;
    t.nw = z / 64 + 1;
    t.bits = (uint64_t *)malloc(t.nw * sizeof(uint64_t));
    t.fw = (int64_t *)calloc(t.nw + 1, sizeof(int64_t));
    for (uint64_t w = 0; w < t.nw; w++) t.bits[w] = ~0ull;
    t.bits[0] &= ~1ull; /* 0 is not counted */
    for (uint64_t v = z + 1; v < t.nw * 64; v++) t.bits[v >> 6] &= ~(1ull << (v & 63));
    for (uint64_t w = 0; w < t.nw; w++) bc_add(&t, w, __builtin_popcountll(t.bits[w]));

    i128 triv = 0, easy = 0, hard = 0;
    int64_t ntriv = 0, neasy = 0, nhard = 0;
    for (uint64_t b = 1; b <= a; b++) {
        uint64_t p = P[b];
        if (b > c) {
            /* the state now is phi(., b-1) */
            for (uint64_t m = y / p + 1; m <= y; m++) {
                if (mu[m] == 0 || lpf[m] <= b || gpf[m] > a) continue;
                uint64_t u = (x / p) / m;
                int64_t ph = bc_prefix(&t, u);
                i128 term = -(i128)mu[m] * ph;
                if (u < p) { triv += term; ntriv++; }
                else if ((u128)u < (u128)p * p && u < y) { easy += term; neasy++; }
                else { hard += term; nhard++; }
            }
        }
        /* sieve out p_b itself and its multiples */
        if (b < a)
            for (uint64_t q = p; q <= z; q += p) bc_clear(&t, q);
    }
    free(t.bits); free(t.fw);
    free(lpf); free(mu); free(gpf);

    int64_t p2[2];
    orc_p2(x, a, p2);

    put128(out + 0, S1);
    put128(out + 2, triv);
    put128(out + 4, easy);
    put128(out + 6, hard);
    out[8] = p2[0]; out[9] = p2[1];
    out[10] = (int64_t)a;
    out[11] = ntriv; out[12] = neasy; out[13] = nhard; out[14] = nord;
    out[15] = (int64_t)z;
    uint64_t sz = orc_isqrt(z), B = 0;
    while (B < np && P[B + 1] <= sz) B++;
    out[16] = (int64_t)B;
    free(P);
    return 0;
}

/* Enumerate the special leaves of phi(x, a) for tiny inputs: for each leaf,
 * writes (b, m, u, class) with class 0 trivial, 1 easy, 2 hard.  The value
 * phi(u, b-1) of each leaf is left to the caller (tests compute it by brute
 * force).  Returns the number of leaves, or -1 if cap is too small. */
int64_t orc_list_leaves(uint64_t x, uint64_t y, uint32_t c, uint64_t a_in,
                        int64_t *rows, int64_t cap)
{
    if (y < 1 || y > orc_isqrt(x) || c > 7) return -1;
    uint64_t lim = y < 32 ? 32 : y;
    uint64_t np;
    uint64_t *P = prime_list(lim, &np);
    uint64_t piy = 0;
    while (piy < np && P[piy + 1] <= y) piy++;
    uint64_t a = a_in ? a_in : piy;
    if (a > piy || c > a) { free(P); return -1; }
    int64_t n = 0;
    for (uint64_t b = c + 1; b <= a; b++) {
        uint64_t p = P[b];
        for (uint64_t m = y / p + 1; m <= y; m++) {
            /* factor m by trial division: squarefree, lpf > p_b, gpf <= p_a */
            uint64_t r = m; int ok = 1, k = 0; uint64_t small = 0, big = 0;
            for (uint64_t d = 2; d * d <= r; d++) {
                if (r % d == 0) {
                    r /= d; k++;
                    if (r % d == 0) { ok = 0; break; }
                    if (!small) small = d;
                    big = d;
                }
            }
            if (!ok) continue;
            if (r > 1) { k++; if (!small) small = r; big = r; }
            if (m == 1 || small <= p || big > P[a]) continue;
            uint64_t u = x / (p * m);
            int cls = u < p ? 0 : (((u128)u < (u128)p * p && u < y) ? 1 : 2);
            if (n >= cap) { free(P); return -1; }
            rows[4 * n + 0] = (int64_t)b;
            rows[4 * n + 1] = (int64_t)m;
            rows[4 * n + 2] = (int64_t)u;
            rows[4 * n + 3] = (int64_t)((k & 1) ? -1 : 1) * (cls + 1); /* sign carries mu */
            n++;
        }
    }
    free(P);
    return n;
}

/* p_k for 1 <= k (the k-th prime), plain sieve. */
/* The hard leaves with u in [lo, hi) only, the way one shard of the hard-leaf
 * sum sees them (Section 4): the interval [lo, hi) alone is sieved by
 * p_1, p_2, ... in order, and phi(u, b-1) of a hard leaf (b, m) is the
 * starting value phi(lo - 1, b - 1), from the recursion of Eq. (4.1), plus the
 * integers of [lo, u] still unsieved after p_{b-1}.  Same leaf classes as
 * orc_leaf_sums, a = pi(y): a leaf is hard unless u < p_b (trivial) or
 * p_b <= u < min(p_b^2, y) (easy).  The sums over any split of [1, z + 1]
 * into ranges add up to the S2_hard of orc_leaf_sums.  out[0..1]: the sum
 * (i128), out[2]: the number of leaves.  Returns 0, or -1 on a domain error. */
int orc_s2_hard_range(uint64_t x, uint64_t y, uint32_t c, uint64_t lo, uint64_t hi, int64_t *out)
{
    if (y < 1 || y > orc_isqrt(x) || c > 7 || lo < 1 || hi < lo) return -1;
    const uint64_t z = x / y;
    if (hi > z + 1) hi = z + 1;
    if (lo > hi) lo = hi;
    uint64_t lim = y;
    if (orc_isqrt(x) > lim) lim = orc_isqrt(x);
    if (lim < 32) lim = 32;
    uint64_t np;
    uint64_t *P = prime_list(lim, &np);
    uint64_t a = 0;
    while (a < np && P[a + 1] <= y) a++;
    if (c > a) { free(P); return -1; }
    uint32_t *lpf = (uint32_t *)calloc(y + 1, sizeof(uint32_t));
    for (uint64_t k = 1; k <= np && P[k] <= y; k++)
        for (uint64_t q = P[k]; q <= y; q += P[k])
            if (!lpf[q]) lpf[q] = (uint32_t)k;
    int8_t *mu = (int8_t *)malloc(y + 1);
    mu[1] = 1;
    for (uint64_t n = 2; n <= y; n++) {
        uint64_t p = P[lpf[n]], r = n / p;
        mu[n] = (r % p == 0) ? 0 : (int8_t)(-mu[r]);
    }
    /* bit v - lo of the bitset stands for the integer v, lo <= v < hi */
    const uint64_t n = hi - lo;
    bitcount t;
    t.nw = n / 64 + 1;
    t.bits = (uint64_t *)malloc(t.nw * sizeof(uint64_t));
    t.fw = (int64_t *)calloc(t.nw + 1, sizeof(int64_t));
    for (uint64_t w = 0; w < t.nw; w++) t.bits[w] = ~0ull;
    for (uint64_t v = n; v < t.nw * 64; v++) t.bits[v >> 6] &= ~(1ull << (v & 63));
    for (uint64_t w = 0; w < t.nw; w++) bc_add(&t, w, __builtin_popcountll(t.bits[w]));
    phi_ctx pc;
    uint64_t L = orc_isqrt(lo) + 1;   /* pi table of the recursion's Legendre cut-off */
    if (L < (1u << 16)) L = 1u << 16;
    if (L > (1u << 26)) L = 1u << 26;
    phi_ctx_init(&pc, a, L);
    i128 hard = 0;
    int64_t nhard = 0;
    for (uint64_t b = 1; b <= a && n > 0; b++) {
        const uint64_t p = P[b];
        if (b > c) {
            int64_t start = -1;   /* phi(lo - 1, b - 1), computed when a leaf needs it */
            for (uint64_t m = y / p + 1; m <= y; m++) {
                if (mu[m] == 0 || lpf[m] <= b) continue;
                const uint64_t u = (x / p) / m;
                if (u < lo || u >= hi) continue;
                if (u < p || ((u128)u < (u128)p * p && u < y)) continue;   /* trivial or easy */
                if (start < 0) start = phi_rec(&pc, lo - 1, b - 1);
                hard -= (i128)mu[m] * (start + bc_prefix(&t, u - lo));
                nhard++;
            }
        }
        /* sieve p_b (itself included) out of [lo, hi) */
        uint64_t q = lo <= p ? p : ((lo + p - 1) / p) * p;
        for (; q < hi; q += p) bc_clear(&t, q - lo);
    }
    phi_ctx_free(&pc);
    free(t.bits); free(t.fw);
    free(lpf); free(mu); free(P);
    put128(out, hard);
    out[2] = nhard;
    return 0;
}

uint64_t orc_nth_prime(uint64_t k)
{
    uint64_t lim = 64, np;
    for (;;) {
        uint64_t *P = prime_list(lim, &np);
        if (np >= k) { uint64_t r = P[k]; free(P); return r; }
        free(P);
        lim *= 2;
    }
}
