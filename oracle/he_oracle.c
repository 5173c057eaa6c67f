/*
 * he_oracle.c -- plain CPU reference for the RNS-CKKS arithmetic that the
 * quadratic-gradient NAG training iteration runs on (arXiv 2406.13221).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Everything here is written for obviousness, not speed: every modular
 * product is a 128-bit product followed by the C `%` operator, polynomials are
 * kept in coefficient form, and ring products go through a textbook NTT whose
 * output is pinned against the O(N^2) definition and against schoolbook
 * negacyclic convolution in the test-suite.
 *
 * The paper (Sec. 2.1) uses HEAAN's approximate scheme and lists the operations
 * Enc, Dec, Add, cAdd, Mul, cMul and rotation with rescaling; it delegates their
 * internals to HEAAN.  This file implements those operations in the RNS form of
 * the same approximate scheme (residue-number-system limbs, NTT-friendly
 * primes, hybrid key switching with one special prime), which is the reading
 * taken for the whole project.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

#define ORC_MAXQ 40

/* ------------------------------------------------------------------ */
/* scalar arithmetic modulo a prime q < 2^62                           */
/* ------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { uint64_t s = a + b; return s >= q ? s - q : s; }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + (q - b); }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); } /* q prime */

/* x mod q for a signed 64-bit x, result in [0, q) */
static uint64_t smod(int64_t x, uint64_t q)
{
    if (x >= 0) return (uint64_t)x % q;
    uint64_t r = (uint64_t)(-(x + 1)) % q; /* -x-1 never overflows */
    return q - 1 - r;
}
/* centred representative of x in (-q/2, q/2) for odd q */
static int64_t center(uint64_t x, uint64_t q) { return x > q / 2 ? (int64_t)x - (int64_t)q : (int64_t)x; }

/* ------------------------------------------------------------------ */
/* primes                                                             */
/* ------------------------------------------------------------------ */
/* Deterministic Miller-Rabin for 64-bit n (the first 12 prime bases). */
int orc_is_prime(uint64_t n)
{
    static const uint64_t base[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++)
        if (n % base[i] == 0) return n == base[i];
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(base[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* largest prime p < 2^bits with p = 1 (mod m), p >= 2^(bits-1), not in taken[] */
static uint64_t prime_below(int bits, uint64_t m, const uint64_t *taken, int ntaken)
{
    uint64_t bound = 1ull << bits, lo = 1ull << (bits - 1);
    uint64_t v = ((bound - 2) / m) * m + 1;
    for (; v >= lo; v -= m) {
        int used = 0;
        for (int i = 0; i < ntaken; i++) used |= (taken[i] == v);
        if (!used && orc_is_prime(v)) return v;
        if (v < m) break;
    }
    return 0;
}

/* Chain q_0 (q0_bits), q_1..q_{nq-1} (qi_bits, descending), then the special
 * prime P (p_bits); every prime is = 1 mod 2N and all are distinct.
 * out has nq+1 entries. Returns 0 on success. */
int orc_gen_primes(int logn, int nq, int q0_bits, int qi_bits, int p_bits, uint64_t *out)
{
    uint64_t m = 2ull << logn;
    int k = 0;
    if (nq < 1 || nq >= ORC_MAXQ) return -1;
    out[k] = prime_below(q0_bits, m, out, k); if (!out[k]) return -2; k++;
    for (int i = 1; i < nq; i++) { out[k] = prime_below(qi_bits, m, out, k); if (!out[k]) return -2; k++; }
    out[k] = prime_below(p_bits, m, out, k); if (!out[k]) return -2;
    return 0;
}

/* The same with a bit width per ciphertext prime: q_i the largest unused prime
 * below 2^bits[i] that is 1 mod 2N, taken in the order i = 0..nq-1, then P. */
int orc_gen_primes_bits(int logn, int nq, const int *bits, int p_bits, uint64_t *out)
{
    uint64_t m = 2ull << logn;
    if (nq < 1 || nq >= ORC_MAXQ) return -1;
    for (int k = 0; k < nq; k++) {
        if (bits[k] < 20 || bits[k] > 60) return -1;
        out[k] = prime_below(bits[k], m, out, k);
        if (!out[k]) return -2;
    }
    out[nq] = prime_below(p_bits, m, out, nq);
    return out[nq] ? 0 : -2;
}

/* psi = h^((q-1)/2N) for the smallest h >= 2 with psi^N = -1 (a primitive 2N-th root) */
uint64_t orc_find_psi(uint64_t q, int logn)
{
    uint64_t twon = 2ull << logn;
    for (uint64_t h = 2;; h++) {
        uint64_t psi = powmod(h, (q - 1) / twon, q);
        if (powmod(psi, twon / 2, q) == q - 1) return psi;
    }
}

/* ------------------------------------------------------------------ */
/* negacyclic NTT over Z_q[X]/(X^N+1)                                  */
/* ------------------------------------------------------------------ */
/* Definition: A_k = sum_j a_j psi^(j(2k+1)),  k = 0..N-1 (natural order).
 * O(N^2) evaluation of the definition, used only to pin orc_ntt. */
void orc_ntt_direct(int n, uint64_t q, uint64_t psi, const uint64_t *a, uint64_t *out)
{
    uint64_t *pp = (uint64_t *)malloc(sizeof(uint64_t) * 2 * n);
    pp[0] = 1;
    for (int e = 1; e < 2 * n; e++) pp[e] = mulmod(pp[e - 1], psi, q);
    for (int k = 0; k < n; k++) {
        uint64_t acc = 0;
        for (int j = 0; j < n; j++) {
            uint64_t e = ((uint64_t)j * (uint64_t)(2 * k + 1)) % (uint64_t)(2 * n);
            acc = addmod(acc, mulmod(a[j] % q, pp[e], q), q);
        }
        out[k] = acc;
    }
    free(pp);
}

/* c = a * b in Z_q[X]/(X^N+1) by schoolbook convolution (X^N = -1) */
void orc_polymul_schoolbook(int n, uint64_t q, const uint64_t *a, const uint64_t *b, uint64_t *c)
{
    uint64_t *t = (uint64_t *)calloc(n, sizeof(uint64_t));
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            uint64_t p = mulmod(a[i] % q, b[j] % q, q);
            if (i + j < n) t[i + j] = addmod(t[i + j], p, q);
            else t[i + j - n] = submod(t[i + j - n], p, q);
        }
    memcpy(c, t, sizeof(uint64_t) * n);
    free(t);
}

/* per-prime tables for the textbook transform */
typedef struct {
    uint64_t q, psi;
    uint64_t *psipow;   /* psi^j, j < N */
    uint64_t *ipsipow;  /* N^-1 psi^-j, j < N */
    uint64_t *w;        /* omega^j, omega = psi^2, j < N/2 */
    uint64_t *iw;       /* omega^-j */
} prime_tab;

static void tab_init(prime_tab *t, uint64_t q, uint64_t psi, int n)
{
    t->q = q; t->psi = psi;
    t->psipow = (uint64_t *)malloc(sizeof(uint64_t) * n);
    t->ipsipow = (uint64_t *)malloc(sizeof(uint64_t) * n);
    t->w = (uint64_t *)malloc(sizeof(uint64_t) * (n / 2 + 1));
    t->iw = (uint64_t *)malloc(sizeof(uint64_t) * (n / 2 + 1));
    uint64_t ipsi = invmod(psi, q), ninv = invmod((uint64_t)n % q, q);
    uint64_t om = mulmod(psi, psi, q), iom = invmod(om, q);
    t->psipow[0] = 1; t->ipsipow[0] = ninv;
    for (int j = 1; j < n; j++) {
        t->psipow[j] = mulmod(t->psipow[j - 1], psi, q);
        t->ipsipow[j] = mulmod(t->ipsipow[j - 1], ipsi, q);
    }
    t->w[0] = 1; t->iw[0] = 1;
    for (int j = 1; j <= n / 2; j++) {
        t->w[j] = mulmod(t->w[j - 1], om, q);
        t->iw[j] = mulmod(t->iw[j - 1], iom, q);
    }
}
static void tab_free(prime_tab *t)
{
    free(t->psipow); free(t->ipsipow); free(t->w); free(t->iw);
}

static void bitrev_u64(int n, uint64_t *a)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* textbook radix-2 decimation-in-time cyclic DFT, bit-reversed input, natural output */
static void dft_cyclic(int n, uint64_t q, const uint64_t *w, uint64_t *a)
{
    bitrev_u64(n, a);
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < half; j++) {
                uint64_t u = a[i + j], v = mulmod(a[i + j + half], w[j * step], q);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
}

/* forward: twist by psi^j, then the cyclic DFT with omega = psi^2 */
static void ntt_fwd(int n, const prime_tab *t, uint64_t *a)
{
    for (int j = 0; j < n; j++) a[j] = mulmod(a[j], t->psipow[j], t->q);
    dft_cyclic(n, t->q, t->w, a);
}
/* inverse: cyclic inverse DFT, then multiply by N^-1 psi^-j */
static void ntt_inv(int n, const prime_tab *t, uint64_t *a)
{
    dft_cyclic(n, t->q, t->iw, a);
    for (int j = 0; j < n; j++) a[j] = mulmod(a[j], t->ipsipow[j], t->q);
}

/* ------------------------------------------------------------------ */
/* counter-based randomness (splitmix64, Steele-Lea-Flood 2014)        */
/* ------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
/* The splitmix64 state after k steps from state s0 is s0 + k*GOLDEN and the
 * output is mix64(state).  Word idx of stream `stream` under `seed` is the
 * output at step k = (stream << 40) + idx + 1 from the state mix64(seed). */
uint64_t orc_rand_word(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t k = (stream << 40) + idx + 1;
    return mix64(mix64(seed) + k * 0x9E3779B97F4A7C15ull);
}
/* plain splitmix64 output sequence from a state, for the published test vector */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ull;
    return mix64(*state);
}

/* stream identifiers */
#define ST_SK 1ull
#define ST_SK_SPARSE 7ull
#define ST_PK_A 2ull
#define ST_PK_E 3ull
#define ST_ENC_V 4ull
#define ST_ENC_E0 5ull
#define ST_ENC_E1 6ull
static uint64_t st_ksk_a(uint64_t gal, int digit) { return (1ull << 24) | (gal << 6) | (uint64_t)digit; }
static uint64_t st_ksk_e(uint64_t gal, int digit) { return (2ull << 24) | (gal << 6) | (uint64_t)digit; }

static int64_t sample_ternary(uint64_t seed, uint64_t st, uint64_t i) { return (int64_t)(orc_rand_word(seed, st, i) % 3) - 1; }
/* uniform in [0,q): the 128-bit integer (w_{2i} * 2^64 + w_{2i+1}) reduced mod q */
static uint64_t sample_uniform(uint64_t seed, uint64_t st, uint64_t i, uint64_t q)
{
    u128 x = ((u128)orc_rand_word(seed, st, 2 * i) << 64) | orc_rand_word(seed, st, 2 * i + 1);
    return (uint64_t)(x % q);
}

/* Discrete Gaussian by cumulative-distribution table over |x| <= K, K = ceil(6 sigma):
 * P(x) proportional to exp(-x^2 / (2 sigma^2)).  cdt[k] = floor(2^63 * P(|X| <= k)),
 * cdt[K] = 2^63.  A sample draws w; u = w >> 1 picks |x| as the first k with u < cdt[k];
 * bit 0 of w is the sign. */
int orc_cdt_table(double sigma, uint64_t *cdt, int maxlen)
{
    int K = (int)ceil(6.0 * sigma);
    if (K + 1 > maxlen) return -1;
    double z = 0.0;
    for (int k = 0; k <= K; k++) {
        double p = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        z += (k == 0) ? p : 2.0 * p;
    }
    double acc = 0.0;
    for (int k = 0; k < K; k++) {
        double p = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        acc += (k == 0) ? p : 2.0 * p;
        cdt[k] = (uint64_t)(acc / z * 9223372036854775808.0);
    }
    cdt[K] = 1ull << 63;
    return K + 1;
}

typedef struct {
    int logn, n, nslots, nq; /* nq = number of ciphertext primes q_0..q_{nq-1} */
    uint64_t q[ORC_MAXQ + 1]; /* q[nq] = special prime P */
    prime_tab tab[ORC_MAXQ + 1];
    double sigma;
    uint64_t cdt[64];
    int cdt_len;
    /* canonical-embedding tables */
    double *zre, *zim; /* zeta^k = exp(i pi k / N), k < 2N */
    int *sidx;         /* slot j -> DFT index (5^j mod 2N - 1)/4 */
    /* keys */
    int secret_hw;     /* 0: every coefficient of s uniform in {-1,0,1}; h > 0: exactly h nonzeros */
    int have_sk;
    int64_t *sk;       /* ternary secret, N */
    uint64_t *pk;      /* [2][nq][N] (b, a) */
    int nksk;
    uint64_t ksk_gal[128];
    uint64_t *ksk[128]; /* [nq digits][2][nq+1 limbs][N], limb nq = P */
} orc_ctx;

static int64_t sample_gauss(const orc_ctx *c, uint64_t seed, uint64_t st, uint64_t i)
{
    uint64_t w = orc_rand_word(seed, st, i);
    uint64_t u = w >> 1;
    int k = 0;
    while (k < c->cdt_len - 1 && u >= c->cdt[k]) k++;
    return ((w & 1) && k) ? -(int64_t)k : (int64_t)k;
}

void orc_sample(uint64_t seed, uint64_t stream, int kind, uint64_t q, double sigma, int64_t n, int64_t *out)
{
    /* kind 0 ternary, 1 gaussian, 2 uniform mod q (values returned as int64) */
    orc_ctx tmp;
    if (kind == 1) { tmp.sigma = sigma; tmp.cdt_len = orc_cdt_table(sigma, tmp.cdt, 64); }
    for (int64_t i = 0; i < n; i++) {
        if (kind == 0) out[i] = sample_ternary(seed, stream, (uint64_t)i);
        else if (kind == 1) out[i] = sample_gauss(&tmp, seed, stream, (uint64_t)i);
        else out[i] = (int64_t)sample_uniform(seed, stream, (uint64_t)i, q);
    }
}

/* ------------------------------------------------------------------ */
/* context                                                            */
/* ------------------------------------------------------------------ */
static orc_ctx *ctx_from_primes(int logn, int nq, orc_ctx *c, double sigma);
orc_ctx *orc_ctx_new(int logn, int nq, int q0_bits, int qi_bits, int p_bits, double sigma)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (orc_gen_primes(logn, nq, q0_bits, qi_bits, p_bits, c->q)) { free(c); return NULL; }
    return ctx_from_primes(logn, nq, c, sigma);
}
/* a context whose ciphertext primes have the bit widths bits[0..nq-1] */
orc_ctx *orc_ctx_new_bits(int logn, int nq, const int *bits, int p_bits, double sigma)
{
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (orc_gen_primes_bits(logn, nq, bits, p_bits, c->q)) { free(c); return NULL; }
    return ctx_from_primes(logn, nq, c, sigma);
}
static orc_ctx *ctx_from_primes(int logn, int nq, orc_ctx *c, double sigma)
{
    c->logn = logn; c->n = 1 << logn; c->nslots = c->n / 2; c->nq = nq;
    for (int i = 0; i <= nq; i++) tab_init(&c->tab[i], c->q[i], orc_find_psi(c->q[i], logn), c->n);
    c->sigma = sigma;
    c->cdt_len = orc_cdt_table(sigma, c->cdt, 64);
    int n = c->n;
    c->zre = (double *)malloc(sizeof(double) * 2 * n);
    c->zim = (double *)malloc(sizeof(double) * 2 * n);
    for (int k = 0; k < 2 * n; k++) {
        double th = (M_PI * (double)k) / (double)n;
        c->zre[k] = cos(th);
        c->zim[k] = sin(th);
    }
    c->sidx = (int *)malloc(sizeof(int) * c->nslots);
    uint64_t g = 1, twon = 2ull * n;
    for (int j = 0; j < c->nslots; j++) { c->sidx[j] = (int)((g - 1) / 4); g = (g * 5) % twon; }
    return c;
}

/* secret with exactly h nonzero coefficients at the next orc_keygen (0 = dense ternary) */
int orc_set_secret_weight(orc_ctx *c, int h)
{
    if (h < 0 || h > c->n) return -1;
    c->secret_hw = h;
    return 0;
}

void orc_ctx_free(orc_ctx *c)
{
    if (!c) return;
    for (int i = 0; i <= c->nq; i++) tab_free(&c->tab[i]);
    free(c->zre); free(c->zim); free(c->sidx);
    free(c->sk); free(c->pk);
    for (int i = 0; i < c->nksk; i++) free(c->ksk[i]);
    free(c);
}

void orc_get_primes(const orc_ctx *c, uint64_t *out) { for (int i = 0; i <= c->nq; i++) out[i] = c->q[i]; }
void orc_get_psi(const orc_ctx *c, uint64_t *out) { for (int i = 0; i <= c->nq; i++) out[i] = c->tab[i].psi; }
void orc_get_zeta_table(const orc_ctx *c, double *re, double *im)
{
    memcpy(re, c->zre, sizeof(double) * 2 * c->n);
    memcpy(im, c->zim, sizeof(double) * 2 * c->n);
}
int orc_get_cdt(const orc_ctx *c, uint64_t *out) { memcpy(out, c->cdt, sizeof(uint64_t) * c->cdt_len); return c->cdt_len; }
void orc_get_sk(const orc_ctx *c, int64_t *out) { memcpy(out, c->sk, sizeof(int64_t) * c->n); }

/* modulus of limb t for a value at level `level`: t <= level -> q_t, t == level+1 -> P */
static const prime_tab *limb_tab(const orc_ctx *c, int level, int t) { return t <= level ? &c->tab[t] : &c->tab[c->nq]; }

/* transform wrappers on one limb of prime index pi (pi == nq means P) */
void orc_ntt(const orc_ctx *c, int pi, uint64_t *a) { ntt_fwd(c->n, &c->tab[pi], a); }
void orc_intt(const orc_ctx *c, int pi, uint64_t *a) { ntt_inv(c->n, &c->tab[pi], a); }

/* ring product of one limb: out = a * b mod (X^N+1, q) through the transform */
static void ring_mul(int n, const prime_tab *t, const uint64_t *a, const uint64_t *b, uint64_t *out)
{
    uint64_t *x = (uint64_t *)malloc(sizeof(uint64_t) * n), *y = (uint64_t *)malloc(sizeof(uint64_t) * n);
    memcpy(x, a, sizeof(uint64_t) * n); memcpy(y, b, sizeof(uint64_t) * n);
    ntt_fwd(n, t, x); ntt_fwd(n, t, y);
    for (int i = 0; i < n; i++) x[i] = mulmod(x[i], y[i], t->q);
    ntt_inv(n, t, x);
    memcpy(out, x, sizeof(uint64_t) * n);
    free(x); free(y);
}
void orc_polymul(const orc_ctx *c, int pi, const uint64_t *a, const uint64_t *b, uint64_t *out) { ring_mul(c->n, &c->tab[pi], a, b, out); }

/* ------------------------------------------------------------------ */
/* canonical embedding (encode / decode)                               */
/* ------------------------------------------------------------------ */
/* Length-n complex DFT, radix-2 decimation in time with bit-reversed input:
 * X_s = sum_k x_k w^(sign*s*k), w = exp(2 pi i / n) = zeta^4.  Every butterfly
 * multiplies data (a) by twiddle (b) as (a.re*b.re - a.im*b.im, a.re*b.im + a.im*b.re)
 * and the file is compiled without floating-point contraction. */
static void fft_c(const orc_ctx *c, int n, double *re, double *im, int inverse)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, tstep = n / len;
        for (int i = 0; i < n; i += len)
            for (int j = 0; j < half; j++) {
                int idx = 4 * j * tstep;
                double br = c->zre[idx], bi = inverse ? -c->zim[idx] : c->zim[idx];
                double ar = re[i + j + half], ai = im[i + j + half];
                double yr = ar * br - ai * bi;
                double yi = ar * bi + ai * br;
                double xr = re[i + j], xi = im[i + j];
                re[i + j] = xr + yr; im[i + j] = xi + yi;
                re[i + j + half] = xr - yr; im[i + j + half] = xi - yi;
            }
    }
}

/* Real coefficient vector of the inverse canonical embedding, before scaling:
 * for slot values z_j (slot j <-> root zeta^(5^j)), u_k = (1/n) zeta^-k sum_s V_s w^-sk with
 * V_(s(j)) = z_j, and coeff_k = Re u_k, coeff_(k+n) = Im u_k. */
void orc_embed_inv(const orc_ctx *c, const double *zr, const double *zi, double *coef)
{
    int n = c->nslots;
    double *vr = (double *)calloc(n, sizeof(double)), *vi = (double *)calloc(n, sizeof(double));
    for (int j = 0; j < n; j++) { vr[c->sidx[j]] = zr[j]; vi[c->sidx[j]] = zi[j]; }
    fft_c(c, n, vr, vi, 1);
    double inv_n = 1.0 / (double)n;
    for (int k = 0; k < n; k++) {
        double ar = vr[k] * inv_n, ai = vi[k] * inv_n;
        double br = c->zre[k], bi = -c->zim[k];
        coef[k] = ar * br - ai * bi;
        coef[k + n] = ar * bi + ai * br;
    }
    free(vr); free(vi);
}

/* Slot values of a real coefficient vector m: z_j = m(zeta^(5^j)) */
void orc_embed(const orc_ctx *c, const double *coef, double *zr, double *zi)
{
    int n = c->nslots;
    double *vr = (double *)malloc(sizeof(double) * n), *vi = (double *)malloc(sizeof(double) * n);
    for (int k = 0; k < n; k++) {
        double ar = coef[k], ai = coef[k + n];
        double br = c->zre[k], bi = c->zim[k];
        vr[k] = ar * br - ai * bi;
        vi[k] = ar * bi + ai * br;
    }
    fft_c(c, n, vr, vi, 0);
    for (int j = 0; j < n; j++) { zr[j] = vr[c->sidx[j]]; zi[j] = vi[c->sidx[j]]; }
    free(vr); free(vi);
}

/* Encode: m_k = round_half_away(scale * coef_k), reduced into limbs q_0..q_level.
 * Returns -1 if a coefficient leaves (-2^62, 2^62). out: [level+1][N]. */
int orc_encode(const orc_ctx *c, const double *zr, const double *zi, int level, double scale, uint64_t *out)
{
    int n = c->n;
    double *coef = (double *)malloc(sizeof(double) * n);
    orc_embed_inv(c, zr, zi, coef);
    int rc = 0;
    for (int k = 0; k < n; k++) {
        double x = coef[k] * scale;
        if (!(fabs(x) < 4611686018427387904.0)) { rc = -1; x = 0.0; }
        int64_t m = llround(x);
        for (int j = 0; j <= level; j++) out[(size_t)j * n + k] = smod(m, c->q[j]);
    }
    free(coef);
    return rc;
}

/* Decode: centred lift of limb 0 (mod q_0) as the integer coefficient, evaluate
 * the embedding, divide by scale.  Valid while |scale * z| stays below q_0 / 2. */
void orc_decode(const orc_ctx *c, const uint64_t *pt, double scale, double *zr, double *zi)
{
    int n = c->n;
    double *coef = (double *)malloc(sizeof(double) * n);
    for (int k = 0; k < n; k++) coef[k] = (double)center(pt[k], c->q[0]);
    orc_embed(c, coef, zr, zi);
    for (int j = 0; j < c->nslots; j++) { zr[j] = zr[j] / scale; zi[j] = zi[j] / scale; }
    free(coef);
}

/* ------------------------------------------------------------------ */
/* keys                                                               */
/* ------------------------------------------------------------------ */
/* a(X) -> a(X^g) in coefficient form, g odd; X^N = -1 */
static void automorph(int n, uint64_t q, uint64_t g, const uint64_t *a, uint64_t *out)
{
    uint64_t twon = 2ull * n;
    for (int k = 0; k < n; k++) {
        uint64_t e = ((uint64_t)k * g) % twon;
        if (e < (uint64_t)n) out[e] = a[k];
        else out[e - n] = a[k] ? q - a[k] : 0;
    }
}
void orc_automorph(const orc_ctx *c, int pi, uint64_t g, const uint64_t *a, uint64_t *out)
{
    automorph(c->n, c->q[pi], g, a, out);
}

/* Key-switching key from s' to s, digits i = 0..nq-1 (one per ciphertext prime):
 * over every modulus t in {q_0..q_{nq-1}, P}:  b_i = -a_i s + e_i + [t == q_i] P s',  a_i uniform.
 * Only s' (as a small integer polynomial) is needed. */
static uint64_t *make_ksk(orc_ctx *c, uint64_t seed, uint64_t gal, const int64_t *sprime)
{
    int n = c->n, nq = c->nq, nl = nq + 1;
    uint64_t *k = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nq * 2 * nl * n);
    for (int d = 0; d < nq; d++) {
        int64_t *e = (int64_t *)malloc(sizeof(int64_t) * n);
        for (int i = 0; i < n; i++) e[i] = sample_gauss(c, seed, st_ksk_e(gal, d), (uint64_t)i);
        #pragma omp parallel for schedule(dynamic)
        for (int t = 0; t < nl; t++) {
            const prime_tab *tb = &c->tab[t];
            uint64_t q = tb->q;
            uint64_t *b = k + (((size_t)d * 2 + 0) * nl + t) * n;
            uint64_t *a = k + (((size_t)d * 2 + 1) * nl + t) * n;
            uint64_t *sv = (uint64_t *)malloc(sizeof(uint64_t) * n), *as = (uint64_t *)malloc(sizeof(uint64_t) * n);
            for (int i = 0; i < n; i++) {
                a[i] = sample_uniform(seed, st_ksk_a(gal, d), (uint64_t)t * n + i, q);
                sv[i] = smod(c->sk[i], q);
            }
            ring_mul(n, tb, a, sv, as);
            uint64_t pq = c->q[nq] % q; /* P mod q_t (zero when t is P) */
            for (int i = 0; i < n; i++) {
                uint64_t v = submod(smod(e[i], q), as[i], q);
                if (t == d) v = addmod(v, mulmod(pq, smod(sprime[i], q), q), q);
                b[i] = v;
            }
            free(sv); free(as);
        }
        free(e);
    }
    return k;
}

/* s^2 as an integer polynomial: exact negacyclic square of a ternary polynomial
 * (|coefficients| <= N, computed directly in int64). */
static void square_small(int n, const int64_t *s, int64_t *out)
{
    memset(out, 0, sizeof(int64_t) * n);
    for (int i = 0; i < n; i++) {
        if (!s[i]) continue;
        for (int j = 0; j < n; j++) {
            int64_t p = s[i] * s[j];
            if (i + j < n) out[i + j] += p; else out[i + j - n] -= p;
        }
    }
}

static void automorph_small(int n, uint64_t g, const int64_t *a, int64_t *out)
{
    uint64_t twon = 2ull * n;
    for (int k = 0; k < n; k++) {
        uint64_t e = ((uint64_t)k * g) % twon;
        if (e < (uint64_t)n) out[e] = a[k]; else out[e - n] = -a[k];
    }
}

static uint64_t *find_ksk(const orc_ctx *c, uint64_t gal)
{
    for (int i = 0; i < c->nksk; i++) if (c->ksk_gal[i] == gal) return c->ksk[i];
    return NULL;
}

/* Secret s ternary; public key (b, a) = (-a s + e, a) over q_0..q_{nq-1};
 * relinearisation key (galois tag 0) for s' = s^2; one rotation key per galois
 * element g in gals for s' = s(X^g). */
int orc_keygen(orc_ctx *c, uint64_t seed, const uint64_t *gals, int ngal)
{
    int n = c->n, nq = c->nq;
    free(c->sk); free(c->pk);
    for (int i = 0; i < c->nksk; i++) free(c->ksk[i]);
    c->nksk = 0;
    c->sk = (int64_t *)malloc(sizeof(int64_t) * n);
    if (c->secret_hw > 0) {
        /* exactly h nonzero coefficients: word k of the stream picks position
         * word % N (skipped when already taken) and the sign from bit 32 */
        memset(c->sk, 0, sizeof(int64_t) * n);
        for (uint64_t k = 0, placed = 0; placed < (uint64_t)c->secret_hw; k++) {
            uint64_t w = orc_rand_word(seed, ST_SK_SPARSE, k);
            uint64_t pos = w % (uint64_t)n;
            if (c->sk[pos]) continue;
            c->sk[pos] = (w >> 32) & 1 ? 1 : -1;
            placed++;
        }
    } else {
        for (int i = 0; i < n; i++) c->sk[i] = sample_ternary(seed, ST_SK, (uint64_t)i);
    }
    c->have_sk = 1;
    c->pk = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)nq * n);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int i = 0; i < n; i++) e[i] = sample_gauss(c, seed, ST_PK_E, (uint64_t)i);
    #pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nq; j++) {
        uint64_t q = c->q[j];
        uint64_t *b = c->pk + (size_t)j * n, *a = c->pk + ((size_t)nq + j) * n;
        uint64_t *sv = (uint64_t *)malloc(sizeof(uint64_t) * n), *as = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int i = 0; i < n; i++) { a[i] = sample_uniform(seed, ST_PK_A, (uint64_t)j * n + i, q); sv[i] = smod(c->sk[i], q); }
        ring_mul(n, &c->tab[j], a, sv, as);
        for (int i = 0; i < n; i++) b[i] = submod(smod(e[i], q), as[i], q);
        free(sv); free(as);
    }
    free(e);
    int64_t *sp = (int64_t *)malloc(sizeof(int64_t) * n);
    square_small(n, c->sk, sp);
    c->ksk_gal[c->nksk] = 0;
    c->ksk[c->nksk++] = make_ksk(c, seed, 0, sp);
    for (int r = 0; r < ngal; r++) {
        if (find_ksk(c, gals[r])) continue;
        if (c->nksk >= 128) { free(sp); return -1; }
        automorph_small(n, gals[r], c->sk, sp);
        c->ksk_gal[c->nksk] = gals[r];
        c->ksk[c->nksk++] = make_ksk(c, seed, gals[r], sp);
    }
    free(sp);
    return 0;
}

/* ------------------------------------------------------------------ */
/* encryption                                                         */
/* ------------------------------------------------------------------ */
/* ct = (v b + e0 + m, v a + e1) over q_0..q_level; v ternary, e0, e1 Gaussian.
 * pt, ct in coefficient form: pt [level+1][N], ct [2][level+1][N]. */
void orc_encrypt(const orc_ctx *c, const uint64_t *pt, int level, uint64_t seed, uint64_t *ct)
{
    int n = c->n, nl = level + 1, nq = c->nq;
    #pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nl; j++) {
        uint64_t q = c->q[j];
        uint64_t *v = (uint64_t *)malloc(sizeof(uint64_t) * n), *t = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int i = 0; i < n; i++) v[i] = smod(sample_ternary(seed, ST_ENC_V, (uint64_t)i), q);
        uint64_t *c0 = ct + (size_t)j * n, *c1 = ct + ((size_t)nl + j) * n;
        ring_mul(n, &c->tab[j], v, c->pk + (size_t)j * n, t);
        for (int i = 0; i < n; i++)
            c0[i] = addmod(addmod(t[i], smod(sample_gauss(c, seed, ST_ENC_E0, (uint64_t)i), q), q), pt[(size_t)j * n + i], q);
        ring_mul(n, &c->tab[j], v, c->pk + ((size_t)nq + j) * n, t);
        for (int i = 0; i < n; i++) c1[i] = addmod(t[i], smod(sample_gauss(c, seed, ST_ENC_E1, (uint64_t)i), q), q);
        free(v); free(t);
    }
}

/* pt = c0 + c1 s over q_0..q_level */
void orc_decrypt(const orc_ctx *c, const uint64_t *ct, int level, uint64_t *pt)
{
    int n = c->n, nl = level + 1;
    #pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nl; j++) {
        uint64_t q = c->q[j];
        uint64_t *sv = (uint64_t *)malloc(sizeof(uint64_t) * n), *t = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int i = 0; i < n; i++) sv[i] = smod(c->sk[i], q);
        ring_mul(n, &c->tab[j], ct + ((size_t)nl + j) * n, sv, t);
        for (int i = 0; i < n; i++) pt[(size_t)j * n + i] = addmod(ct[(size_t)j * n + i], t[i], q);
        free(sv); free(t);
    }
}

/* decrypt a three-component tensor (d0, d1, d2) with (1, s, s^2) */
void orc_decrypt3(const orc_ctx *c, const uint64_t *d, int level, uint64_t *pt)
{
    int n = c->n, nl = level + 1;
    int64_t *s2 = (int64_t *)malloc(sizeof(int64_t) * n);
    square_small(n, c->sk, s2);
    for (int j = 0; j < nl; j++) {
        uint64_t q = c->q[j];
        uint64_t *sv = (uint64_t *)malloc(sizeof(uint64_t) * n), *t = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int i = 0; i < n; i++) sv[i] = smod(c->sk[i], q);
        ring_mul(n, &c->tab[j], d + ((size_t)nl + j) * n, sv, t);
        for (int i = 0; i < n; i++) pt[(size_t)j * n + i] = addmod(d[(size_t)j * n + i], t[i], q);
        for (int i = 0; i < n; i++) sv[i] = smod(s2[i], q);
        ring_mul(n, &c->tab[j], d + ((size_t)2 * nl + j) * n, sv, t);
        for (int i = 0; i < n; i++) pt[(size_t)j * n + i] = addmod(pt[(size_t)j * n + i], t[i], q);
        free(sv); free(t);
    }
    free(s2);
}

/* ------------------------------------------------------------------ */
/* homomorphic operations (all on coefficient-form limbs)              */
/* ------------------------------------------------------------------ */
/* out = a + b (or a - b), npoly polynomials of level+1 limbs each */
void orc_add(const orc_ctx *c, int level, int npoly, const uint64_t *a, const uint64_t *b, uint64_t *out, int subtract)
{
    int n = c->n, nl = level + 1;
    for (int p = 0; p < npoly; p++)
        for (int j = 0; j < nl; j++) {
            uint64_t q = c->q[j];
            size_t o = ((size_t)p * nl + j) * n;
            for (int i = 0; i < n; i++) out[o + i] = subtract ? submod(a[o + i], b[o + i], q) : addmod(a[o + i], b[o + i], q);
        }
}

/* tensor product (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1) */
void orc_tensor(const orc_ctx *c, int level, const uint64_t *a, const uint64_t *b, uint64_t *d)
{
    int n = c->n, nl = level + 1;
    #pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nl; j++) {
        const prime_tab *t = &c->tab[j];
        uint64_t q = t->q;
        const uint64_t *a0 = a + (size_t)j * n, *a1 = a + ((size_t)nl + j) * n;
        const uint64_t *b0 = b + (size_t)j * n, *b1 = b + ((size_t)nl + j) * n;
        uint64_t *d0 = d + (size_t)j * n, *d1 = d + ((size_t)nl + j) * n, *d2 = d + ((size_t)2 * nl + j) * n;
        uint64_t *x = (uint64_t *)malloc(sizeof(uint64_t) * n);
        ring_mul(n, t, a0, b0, d0);
        ring_mul(n, t, a0, b1, d1);
        ring_mul(n, t, a1, b0, x);
        for (int i = 0; i < n; i++) d1[i] = addmod(d1[i], x[i], q);
        ring_mul(n, t, a1, b1, d2);
        free(x);
    }
}

/* Hybrid key switching (Sec. 2.1, relinearisation and rotation keys) in two
 * halves.  ks_inner_add: ModUp and inner product of one polynomial d at
 * `level` with `key`: digit i = centred limb i of d, reduced into every
 * modulus t in {q_0..q_level, P}; acc_t += sum_i digit_i * key_(i,t) for both
 * key polynomials (acc: [2][level+2][N], t = level+1 standing for P).
 * ks_moddown: out_j = (acc_j - centred(acc_P) mod q_j) * P^-1 mod q_j. */
static void ks_inner_add(const orc_ctx *c, int level, const uint64_t *key, const uint64_t *d, uint64_t *acc)
{
    int n = c->n, nl = level + 1, nql = c->nq + 1, nt = level + 2;
    #pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < nt; t++) {
        const prime_tab *tb = limb_tab(c, level, t);
        uint64_t q = tb->q;
        int key_limb = t <= level ? t : c->nq;
        uint64_t *x = (uint64_t *)malloc(sizeof(uint64_t) * n), *y = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int i = 0; i < nl; i++) {
            uint64_t qi = c->q[i];
            const uint64_t *di = d + (size_t)i * n;
            for (int k = 0; k < n; k++) x[k] = smod(center(di[k], qi), q);
            for (int p = 0; p < 2; p++) {
                const uint64_t *kl = key + (((size_t)i * 2 + p) * nql + key_limb) * n;
                ring_mul(n, tb, x, kl, y);
                uint64_t *ac = acc + ((size_t)p * nt + t) * n;
                for (int k = 0; k < n; k++) ac[k] = addmod(ac[k], y[k], q);
            }
        }
        free(x); free(y);
    }
}
static void ks_moddown(const orc_ctx *c, int level, const uint64_t *acc, uint64_t *out)
{
    int n = c->n, nl = level + 1, nt = level + 2;
    uint64_t P = c->q[c->nq];
    for (int p = 0; p < 2; p++) {
        const uint64_t *ap = acc + ((size_t)p * nt + level + 1) * n;
        for (int j = 0; j <= level; j++) {
            uint64_t q = c->q[j], pinv = invmod(P % q, q);
            const uint64_t *aj = acc + ((size_t)p * nt + j) * n;
            uint64_t *oj = out + ((size_t)p * nl + j) * n;
            for (int k = 0; k < n; k++) oj[k] = mulmod(submod(aj[k], smod(center(ap[k], P), q), q), pinv, q);
        }
    }
}

/* key switching of one polynomial d at `level` under the key tagged gal; out: [2][level+1][N] */
int orc_keyswitch(const orc_ctx *c, int level, uint64_t gal, const uint64_t *d, uint64_t *out)
{
    const uint64_t *key = find_ksk(c, gal);
    if (!key) return -1;
    uint64_t *acc = (uint64_t *)calloc((size_t)2 * (level + 2) * c->n, sizeof(uint64_t));
    ks_inner_add(c, level, key, d, acc);
    ks_moddown(c, level, acc, out);
    free(acc);
    return 0;
}

/* relinearise (d0, d1, d2) -> (d0, d1) + KS_{s^2 -> s}(d2) */
int orc_relin(const orc_ctx *c, int level, const uint64_t *d, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    uint64_t *ks = (uint64_t *)malloc(sizeof(uint64_t) * 2 * nl * n);
    int rc = orc_keyswitch(c, level, 0, d + (size_t)2 * nl * n, ks);
    if (!rc) orc_add(c, level, 2, d, ks, out, 0);
    free(ks);
    return rc;
}

/* rotation by galois element g: (sigma_g(c0), sigma_g(c1)) then key-switch
 * the second component from s(X^g) back to s. */
int orc_rotate_gal(const orc_ctx *c, int level, uint64_t g, const uint64_t *ct, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    uint64_t *r = (uint64_t *)malloc(sizeof(uint64_t) * 2 * nl * n);
    uint64_t *ks = (uint64_t *)malloc(sizeof(uint64_t) * 2 * nl * n);
    for (int p = 0; p < 2; p++)
        for (int j = 0; j < nl; j++)
            automorph(n, c->q[j], g, ct + ((size_t)p * nl + j) * n, r + ((size_t)p * nl + j) * n);
    int rc = orc_keyswitch(c, level, g, r + (size_t)nl * n, ks);
    if (!rc) {
        for (int j = 0; j < nl; j++) {
            uint64_t q = c->q[j];
            for (int k = 0; k < n; k++) {
                size_t o = (size_t)j * n + k;
                out[o] = addmod(r[o], ks[o], q);
                out[(size_t)nl * n + o] = ks[(size_t)nl * n + o];
            }
        }
    }
    free(r); free(ks);
    return rc;
}

/* galois element for a left rotation of the slot vector by r (negative = right) */
uint64_t orc_galois_elt(const orc_ctx *c, int64_t r)
{
    int64_t ns = c->nslots;
    int64_t rr = ((r % ns) + ns) % ns;
    return powmod(5, (uint64_t)rr, 2ull * c->n);
}

int orc_rotate(const orc_ctx *c, int level, int64_t r, const uint64_t *ct, uint64_t *out)
{
    return orc_rotate_gal(c, level, orc_galois_elt(c, r), ct, out);
}

/* Sum of a ciphertext and several of its rotations with one shared ModUp and
 * one ModDown (hoisted rotations): out = ct + sum_j Rot_{g_j}(ct).  Rotation j
 * key-switches sigma_{g_j}(c1) with the key for s(X^{g_j}); since the centred
 * digit decomposition commutes with the automorphism (a signed permutation of
 * coefficients), every rotation reuses the digits of c1, and the inner
 * products of all rotations are added over {q_0..q_level, P} before a single
 * division by P.  c0 contributes c0 + sum_j sigma_{g_j}(c0).  With one
 * rotation the result equals ct + Rot(ct) word for word. */
int orc_rotsum_gal(const orc_ctx *c, int level, const uint64_t *gals, int ngal, const uint64_t *ct, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    for (int j = 0; j < ngal; j++)
        if (!find_ksk(c, gals[j])) return -1;
    uint64_t *acc = (uint64_t *)calloc((size_t)2 * (level + 2) * n, sizeof(uint64_t));
    uint64_t *r = (uint64_t *)malloc(sizeof(uint64_t) * nl * n);
    uint64_t *ks = (uint64_t *)malloc(sizeof(uint64_t) * 2 * nl * n);
    memcpy(out, ct, sizeof(uint64_t) * 2 * nl * n);
    for (int j = 0; j < ngal; j++) {
        for (int i = 0; i < nl; i++) {
            uint64_t q = c->q[i];
            /* sigma_j(c0) into out_0, sigma_j(c1) into r */
            automorph(n, q, gals[j], ct + (size_t)i * n, r + (size_t)i * n);
            uint64_t *o = out + (size_t)i * n;
            for (int k = 0; k < n; k++) o[k] = addmod(o[k], r[(size_t)i * n + k], q);
            automorph(n, q, gals[j], ct + ((size_t)nl + i) * n, r + (size_t)i * n);
        }
        ks_inner_add(c, level, find_ksk(c, gals[j]), r, acc);
    }
    ks_moddown(c, level, acc, ks);
    for (int p = 0; p < 2; p++)
        for (int i = 0; i < nl; i++) {
            uint64_t q = c->q[i];
            uint64_t *o = out + ((size_t)p * nl + i) * n;
            const uint64_t *b = ks + ((size_t)p * nl + i) * n;
            for (int k = 0; k < n; k++) o[k] = addmod(o[k], b[k], q);
        }
    free(acc); free(r); free(ks);
    return 0;
}

/* rescale: drop q_level with rounding, c_j <- (c_j - [c_level]_centred) * q_level^-1 mod q_j.
 * in [npoly][level+1][N] -> out [npoly][level][N] */
void orc_rescale(const orc_ctx *c, int level, int npoly, const uint64_t *in, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    uint64_t ql = c->q[level];
    for (int p = 0; p < npoly; p++) {
        const uint64_t *last = in + ((size_t)p * nl + level) * n;
        for (int j = 0; j < level; j++) {
            uint64_t q = c->q[j], inv = invmod(ql % q, q);
            const uint64_t *src = in + ((size_t)p * nl + j) * n;
            uint64_t *dst = out + ((size_t)p * level + j) * n;
            for (int k = 0; k < n; k++) dst[k] = mulmod(submod(src[k], smod(center(last[k], ql), q), q), inv, q);
        }
    }
}

/* mod-drop: keep limbs 0..target of each polynomial (scale unchanged) */
void orc_moddrop(const orc_ctx *c, int level, int target, int npoly, const uint64_t *in, uint64_t *out)
{
    int n = c->n, nl = level + 1, nt = target + 1;
    for (int p = 0; p < npoly; p++)
        for (int j = 0; j < nt; j++) memcpy(out + ((size_t)p * nt + j) * n, in + ((size_t)p * nl + j) * n, sizeof(uint64_t) * n);
}

/* multiply every polynomial by the integer constant k */
void orc_cmul_int(const orc_ctx *c, int level, int npoly, const uint64_t *in, int64_t k, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    for (int p = 0; p < npoly; p++)
        for (int j = 0; j < nl; j++) {
            uint64_t q = c->q[j], kk = smod(k, q);
            size_t o = ((size_t)p * nl + j) * n;
            for (int i = 0; i < n; i++) out[o + i] = mulmod(in[o + i], kk, q);
        }
}

/* add the integer constant k to the constant coefficient of c0 */
void orc_cadd_int(const orc_ctx *c, int level, const uint64_t *in, int64_t k, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    memcpy(out, in, sizeof(uint64_t) * 2 * nl * n);
    for (int j = 0; j < nl; j++) out[(size_t)j * n] = addmod(out[(size_t)j * n], smod(k, c->q[j]), c->q[j]);
}

/* multiply both components by a plaintext polynomial pt [level+1][N] */
void orc_ptmul(const orc_ctx *c, int level, const uint64_t *ct, const uint64_t *pt, uint64_t *out)
{
    int n = c->n, nl = level + 1;
    #pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nl; j++)
        for (int p = 0; p < 2; p++)
            ring_mul(n, &c->tab[j], ct + ((size_t)p * nl + j) * n, pt + (size_t)j * n, out + ((size_t)p * nl + j) * n);
}
