// helr_ctx.cu -- context, tables, keys and the C ABI of the scheme operations
// (Sec. 2.1: Enc, Dec, Add, cAdd, Mul, cMul, rotation, rescaling).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <math.h>
#include <algorithm>
#include <stdlib.h>

#include "helr_internal.cuh"
#include "ntt_core.cuh"

typedef unsigned __int128 u128;

std::atomic<unsigned long long> g_helr_launches{0};

void prof_start(he_ctx *c, int cls, cudaStream_t s)
{
    if (!c->prof.on) return;
    ProfClass &p = c->prof.cls[cls];
    while (p.ev.size() < 2 * (p.used + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p.ev.push_back(e);
    }
    cudaEventRecord(p.ev[2 * p.used], s);
}
void prof_stop(he_ctx *c, int cls, cudaStream_t s, double units, int launches, double units2, double units3)
{
    if (!c->prof.on) return;
    ProfClass &p = c->prof.cls[cls];
    if (p.ev.size() < 2 * (p.used + 1)) return;
    cudaEventRecord(p.ev[2 * p.used + 1], s);
    p.used++;
    p.units += units;
    p.units2 += units2;
    p.units3 += units3;
    p.launches += launches;
}

extern "C" uint64_t he_launch_count(void) { return g_helr_launches.load(); }

extern "C" int he_prof_enable(he_ctx *c, int on)
{
    if (!c) return HE_EINVAL;
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    c->prof.on = on;
    for (auto &p : c->prof.cls) p.used = 0, p.units = 0, p.units2 = 0, p.units3 = 0, p.launches = 0;
    for (double &k : c->prof.ks_by_limbs) k = 0;
    return HE_OK;
}

extern "C" int he_set_rotation_radix(he_ctx *c, int log2_radix)
{
    if (!c) return HE_EINVAL;
    if (log2_radix < 1 || (1 << log2_radix) - 1 > HELR_MAX_HOIST)
        return helr_fail(c, HE_EINVAL, "rotation radix 2^%d unsupported (1..3)", log2_radix);
    c->rot_radix_log = log2_radix;
    return HE_OK;
}

extern "C" int he_set_hoist_form(he_ctx *c, int form)
{
    if (!c) return HE_EINVAL;
    if (form < -1 || form > 1) return helr_fail(c, HE_EINVAL, "hoisted inner-product form %d (0, 1, -1 = tuned)", form);
    c->hoist_form = form;
    return HE_OK;
}

extern "C" unsigned long long he_hoist_tensor_launches(const he_ctx *c) { return c ? c->hoist_tensor_launches : 0; }

// One thread waits on an mbarrier of expected count 1 with the kernels' bounded
// wait; when `arrive` is 0 nothing arrives, the wait runs out after one second
// and bit 0 of the status word is set.
__global__ void k_selftest_wait(int arrive, int *status)
{
    __shared__ uint64_t bar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
    if (!mbar_wait_bounded(mb, 0)) atomicOr(status, 1);
}

extern "C" int he_selftest_bounded_wait(he_ctx *c, int arrive)
{
    if (!c) return HE_EINVAL;
    HELR_LAUNCH(k_selftest_wait<<<1, 1, 0, c->stream>>>(arrive ? 1 : 0, c->d_status));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

extern "C" int he_check_device(he_ctx *c)
{
    if (!c) return HE_EINVAL;
    int st = 0;
    HELR_CUDA(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st == 0) return HE_OK;
    HELR_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    return helr_fail(c, HE_ETIMEOUT, "a bounded device-side wait expired (status %#x)", st);
}

extern "C" int he_prof_keyswitches(he_ctx *c, double *by_limbs, size_t n)
{
    if (!c || !by_limbs) return HE_EINVAL;
    for (size_t i = 0; i < n; i++) by_limbs[i] = i < HELR_MAXQ + 2 ? c->prof.ks_by_limbs[i] : 0;
    return HE_OK;
}

extern "C" int he_prof_read2(he_ctx *c, int cls, double *units2, double *dram_limbs)
{
    if (!c || cls < 0 || cls >= PROF_NCLASS || !units2) return HE_EINVAL;
    *units2 = c->prof.cls[cls].units2;
    if (dram_limbs) *dram_limbs = c->prof.cls[cls].units3;
    return HE_OK;
}

extern "C" int he_prof_read(he_ctx *c, int cls, double *ms, double *units, uint64_t *launches)
{
    if (!c || cls < 0 || cls >= PROF_NCLASS) return HE_EINVAL;
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    ProfClass &p = c->prof.cls[cls];
    double tot = 0;
    for (size_t i = 0; i < p.used; i++) {
        float x = 0;
        HELR_CUDA(c, cudaEventElapsedTime(&x, p.ev[2 * i], p.ev[2 * i + 1]));
        tot += x;
    }
    if (ms) *ms = tot;
    if (units) *units = p.units;
    if (launches) *launches = p.launches;
    return HE_OK;
}

// ------------------------------------------------------------------ errors / memory
int helr_fail(he_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err.code = code;
        c->err.msg = buf;
    }
    return code;
}

int helr_alloc(he_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return helr_fail(c, e == cudaErrorMemoryAllocation ? HE_ENOMEM : HE_ECUDA, "device allocation of %zu bytes: %s",
                         bytes, cudaGetErrorString(e));
    }
    return HE_OK;
}
void helr_free(he_ctx *c, void *p)
{
    if (p) cudaFreeAsync(p, c->stream);
}

// ------------------------------------------------------------------ host number theory
static uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }
static uint64_t h_pow(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    for (; e; e >>= 1, a = h_mulmod(a, a, q))
        if (e & 1) r = h_mulmod(r, a, q);
    return r;
}
static uint64_t h_inv(uint64_t a, uint64_t q) { return h_pow(a % q, q - 2, q); }
static uint64_t h_shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Miller-Rabin with the prime bases below 40 (deterministic for 64-bit inputs)
static bool h_is_prime(uint64_t n)
{
    const uint64_t B[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : B)
        if (n % b == 0) return n == b;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) d >>= 1, s++;
    for (uint64_t b : B) {
        uint64_t x = h_pow(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s && comp; i++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

// largest unused prime below 2^bits (and at least 2^(bits-1)) that is 1 mod 2N
static uint64_t h_next_prime(int bits, uint64_t twon, const std::vector<uint64_t> &used)
{
    uint64_t top = (1ull << bits) - 1;
    uint64_t cand = top - (top % twon) + 1;
    if (cand > top) cand -= twon;
    for (; cand >= (1ull << (bits - 1)); cand -= twon) {
        if (std::find(used.begin(), used.end(), cand) != used.end()) continue;
        if (h_is_prime(cand)) return cand;
    }
    return 0;
}

static unsigned bitrev(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

int helr_build_cdt(double sigma, uint64_t *out, int cap)
{
    int K = (int)ceil(6.0 * sigma);
    if (K + 1 > cap) return -1;
    const double two_s2 = 2.0 * sigma * sigma;
    double z = 0.0;
    for (int k = 0; k <= K; k++) {
        double p = exp(-(double)(k * k) / two_s2);
        z += k ? 2.0 * p : p;
    }
    double run = 0.0;
    for (int k = 0; k < K; k++) {
        double p = exp(-(double)(k * k) / two_s2);
        run += k ? 2.0 * p : p;
        out[k] = (uint64_t)(run / z * 9223372036854775808.0);
    }
    out[K] = 1ull << 63;
    return K + 1;
}

static void zeta_table(int logn, double *re, double *im)
{
    const int n = 1 << logn;
    for (int k = 0; k < 2 * n; k++) {
        double th = (M_PI * (double)k) / (double)n;
        re[k] = cos(th);
        im[k] = sin(th);
    }
}

// ------------------------------------------------------------------ context
static int upload(he_ctx *c, void **dst, const void *src, size_t bytes)
{
    HELR_TRY(helr_alloc(c, dst, bytes));
    HELR_CUDA(c, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return HE_OK;
}

// The transform runs as a column pass over the first K1 = floor(log N / 2)
// stages and a row pass over the last K2 = log N - K1 stages; inside the row pass
// a row of R2 = 2^K2 words is held by T2 = 2^floor(K2/2) threads.  On the
// row-pass stages after the register exchange (local stage S >= ceil(K2/2),
// m = 2^S twiddles per row starting at m (R1 + row)), thread l uses twiddles
// l gpt + g (gpt = m / T2); those blocks are stored transposed, at g T2 + l, so
// that the threads of a row load adjacent pairs.  All other entries keep the
// bit-reversed order psi^bitrev(k).
static void row_pass_layout(uint64_t *pairs, int logn)
{
    const int K1 = logn / 2, K2 = logn - K1, R1 = 1 << K1, T2 = 1 << (K2 / 2), LE2 = (K2 + 1) / 2;
    std::vector<uint64_t> blk;
    for (int S = LE2; S < K2; S++) {
        const int m = 1 << S, gpt = m / T2;
        blk.resize((size_t)m * 2);
        for (int row = 0; row < R1; row++) {
            uint64_t *b = pairs + ((size_t)m * (R1 + row)) * 2;
            std::copy(b, b + (size_t)m * 2, blk.begin());
            for (int l = 0; l < T2; l++)
                for (int g = 0; g < gpt; g++) {
                    b[(size_t)(g * T2 + l) * 2] = blk[(size_t)(l * gpt + g) * 2];
                    b[(size_t)(g * T2 + l) * 2 + 1] = blk[(size_t)(l * gpt + g) * 2 + 1];
                }
        }
    }
}

static int ctx_init(he_ctx *c, const he_params *p)
{
    c->logn = p->log_n;
    c->n = 1 << p->log_n;
    c->nslots = c->n / 2;
    c->nq = p->n_q;
    c->nprime = p->n_q + 1;
    c->sigma = p->sigma;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            c->sms = sms;
    }
    const uint64_t twon = 2ull * c->n;
    std::vector<uint64_t> used;
    uint64_t v;
    for (int i = 0; i < c->nq; i++) {
        const int b = p->bits ? p->bits[i] : (i ? p->qi_bits : p->q0_bits);
        v = h_next_prime(b, twon, used);
        if (!v) return helr_fail(c, HE_EINVAL, "not enough %d-bit primes = 1 mod 2N", b);
        used.push_back(v);
    }
    c->secret_hw = p->secret_hw;
    v = h_next_prime(p->p_bits, twon, used);
    if (!v) return helr_fail(c, HE_EINVAL, "no special prime");
    used.push_back(v);
    // the key inner product accumulates up to n_q products below 20 q^2 (primes
    // under 2^58, unreduced butterflies) or 4 q^2 exactly in 128 bits
    for (int i = 0; i < c->nprime; i++) {
        const u128 q2 = (u128)used[i] * used[i];
        const unsigned f = (unsigned)c->nq * (used[i] < HELR_LZ_QMAX ? 20u : 4u);
        if (q2 > ~(u128)0 / f)
            return helr_fail(c, HE_EINVAL, "prime %d (%llu): %u 128-bit key products could overflow", i,
                             (unsigned long long)used[i], f);
    }
    for (int i = 0; i < c->nprime; i++) {
        uint64_t q = used[i];
        c->q[i] = q;
        int bits = 64 - __builtin_clzll(q);
        c->modh[i].q = q;
        c->modh[i].s = (uint32_t)(bits - 2);
        c->modh[i].mu = (uint64_t)(((u128)1 << (bits - 2 + 64)) / q);
        c->modh[i].pad = 0;
        uint64_t inv = q;  // Newton iteration for q^-1 mod 2^64 (q odd: correct to 3 bits, doubling each step)
        for (int it = 0; it < 6; it++) inv *= 2 - q * inv;
        c->modh[i].qinv = inv;
        // primitive 2N-th root: first h >= 2 whose (q-1)/2N-th power has order exactly 2N
        for (uint64_t h = 2;; h++) {
            uint64_t psi = h_pow(h, (q - 1) / twon, q);
            if (h_pow(psi, c->n, q) == q - 1) {
                c->psi[i] = psi;
                break;
            }
        }
    }
    c->cdt_len = helr_build_cdt(c->sigma, c->cdt_host, 64);
    if (c->cdt_len < 0) return helr_fail(c, HE_EINVAL, "sigma too large");

    // transform tables: psi^(bitrev(k)) and psi^-(bitrev(k)), k < N, Shoup pairs
    const int n = c->n, np = c->nprime;
    std::vector<uint64_t> tw((size_t)np * n * 2), itw((size_t)np * n * 2), ninv((size_t)np * 2);
    std::vector<uint64_t> pw(n), ipw(n);
    for (int i = 0; i < np; i++) {
        uint64_t q = c->q[i], psi = c->psi[i], ipsi = h_inv(psi, q);
        pw[0] = 1;
        ipw[0] = 1;
        for (int k = 1; k < n; k++) {
            pw[k] = h_mulmod(pw[k - 1], psi, q);
            ipw[k] = h_mulmod(ipw[k - 1], ipsi, q);
        }
        for (int k = 0; k < n; k++) {
            unsigned e = bitrev((unsigned)k, c->logn);
            size_t o = ((size_t)i * n + k) * 2;
            tw[o] = pw[e];
            tw[o + 1] = h_shoup(pw[e], q);
            itw[o] = ipw[e];
            itw[o + 1] = h_shoup(ipw[e], q);
        }
        row_pass_layout(tw.data() + (size_t)i * n * 2, c->logn);
        row_pass_layout(itw.data() + (size_t)i * n * 2, c->logn);
        uint64_t ni = h_inv((uint64_t)n % q, q);
        ninv[2 * i] = ni;
        ninv[2 * i + 1] = h_shoup(ni, q);
    }
    std::vector<double> zr(2 * n), zi(2 * n), zeta(4 * (size_t)n);
    zeta_table(c->logn, zr.data(), zi.data());
    for (int k = 0; k < 2 * n; k++) zeta[2 * k] = zr[k], zeta[2 * k + 1] = zi[k];
    std::vector<int> sidx(c->nslots);
    uint64_t g = 1;
    for (int j = 0; j < c->nslots; j++) {
        sidx[j] = (int)((g - 1) / 4);
        g = g * 5 % twon;
    }
    // rescale and ModDown inverses
    const int nq = c->nq;
    std::vector<uint64_t> qinv((size_t)nq * nq * 2, 0), pinv((size_t)nq * 2);
    for (int l = 0; l < nq; l++)
        for (int j = 0; j < l; j++) {
            uint64_t x = h_inv(c->q[l] % c->q[j], c->q[j]);
            qinv[((size_t)l * nq + j) * 2] = x;
            qinv[((size_t)l * nq + j) * 2 + 1] = h_shoup(x, c->q[j]);
        }
    for (int j = 0; j < nq; j++) {
        uint64_t x = h_inv(c->q[nq] % c->q[j], c->q[j]);
        pinv[2 * j] = x;
        pinv[2 * j + 1] = h_shoup(x, c->q[j]);
    }
    HELR_TRY(upload(c, (void **)&c->t.mod, c->modh, sizeof(ModQ) * np));
    HELR_TRY(upload(c, (void **)&c->t.tw, tw.data(), tw.size() * 8));
    HELR_TRY(upload(c, (void **)&c->t.itw, itw.data(), itw.size() * 8));
    HELR_TRY(upload(c, (void **)&c->t.ninv, ninv.data(), ninv.size() * 8));
    HELR_TRY(upload(c, (void **)&c->t.zeta, zeta.data(), zeta.size() * 8));
    HELR_TRY(upload(c, (void **)&c->t.sidx, sidx.data(), sidx.size() * sizeof(int)));
    HELR_TRY(upload(c, (void **)&c->t.cdt, c->cdt_host, sizeof(uint64_t) * c->cdt_len));
    HELR_TRY(upload(c, (void **)&c->d_qinv, qinv.data(), qinv.size() * 8));
    HELR_TRY(upload(c, (void **)&c->d_pinv, pinv.data(), pinv.size() * 8));
    HELR_TRY(helr_alloc(c, (void **)&c->d_sk, sizeof(uint64_t) * np * n));
    HELR_TRY(helr_alloc(c, (void **)&c->d_pk, sizeof(uint64_t) * 2 * nq * n));
    HELR_TRY(helr_alloc(c, (void **)&c->d_status, sizeof(int)));
    HELR_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    c->h_sk = (int64_t *)calloc(n, sizeof(int64_t));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    return HE_OK;
}

extern "C" int he_ctx_create(const he_params *p, void *stream, he_ctx **out)
{
    if (!out) return HE_EINVAL;
    *out = nullptr;
    if (!p || p->log_n < HELR_MIN_LOGN || p->log_n > HELR_MAX_LOGN || p->n_q < 2 || p->n_q + 1 > HELR_MAXQ ||
        p->q0_bits < 30 || p->q0_bits > 60 || p->qi_bits < 30 || p->qi_bits > 60 || p->p_bits < 30 || p->p_bits > 60 ||
        !(p->sigma > 0.0) || p->secret_hw < 0 || p->secret_hw > (1 << p->log_n))
        return HE_EINVAL;
    if (p->bits)
        for (int i = 0; i < p->n_q; i++)
            if (p->bits[i] < 30 || p->bits[i] > 60) return HE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return HE_ECUDA;
    }
    he_ctx *c = new he_ctx();
    c->stream = (cudaStream_t)stream;
    if (const char *w = getenv("HELR_KS_WAVE")) c->ks_wave = atoi(w);
    // keep freed stream-ordered memory in the pool between iterations
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    int rc = ctx_init(c, p);
    if (rc != HE_OK) {
        fprintf(stderr, "he_ctx_create: %s\n", c->err.msg.c_str());
        he_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return HE_OK;
}

extern "C" int he_ctx_destroy(he_ctx *c)
{
    if (!c) return HE_EINVAL;
    cudaStreamSynchronize(c->stream);
    for (auto &p : c->prof.cls)
        for (auto e : p.ev) cudaEventDestroy(e);
    void *ptrs[] = {c->t.mod, c->t.tw, c->t.itw, c->t.ninv, c->t.zeta, c->t.sidx, c->t.cdt, c->d_qinv, c->d_pinv, c->d_sk, c->d_pk,
                    c->d_status};
    for (void *p : ptrs) helr_free(c, p);
    for (auto &k : c->ksk) helr_free(c, k.d);
    for (auto &d : c->boot_diag) helr_free(c, d.second);
    cudaStreamSynchronize(c->stream);
    free(c->h_sk);
    delete c;
    return HE_OK;
}

extern "C" const char *he_last_error(const he_ctx *c) { return c ? c->err.msg.c_str() : "null context"; }

extern "C" int he_ctx_primes(const he_ctx *c, uint64_t *out, size_t n)
{
    if (!c || !out || n < (size_t)c->nprime) return HE_EINVAL;
    memcpy(out, c->q, sizeof(uint64_t) * c->nprime);
    return HE_OK;
}

extern "C" int he_gauss_table(double sigma, uint64_t *out, size_t cap, size_t *len)
{
    if (!out || !len || !(sigma > 0)) return HE_EINVAL;
    int k = helr_build_cdt(sigma, out, (int)std::min(cap, (size_t)1 << 20));
    if (k < 0) return HE_EINVAL;
    *len = (size_t)k;
    return HE_OK;
}

extern "C" int he_zeta_table(int log_n, double *re, double *im)
{
    if (!re || !im || log_n < 1 || log_n > 20) return HE_EINVAL;
    zeta_table(log_n, re, im);
    return HE_OK;
}

extern "C" uint64_t he_galois_elt(const he_ctx *c, int64_t r)
{
    const int64_t ns = c->nslots;
    int64_t rr = ((r % ns) + ns) % ns;
    return h_pow(5, (uint64_t)rr, 2ull * c->n);
}

// ------------------------------------------------------------------ keys
const uint64_t *helr_find_key(const he_ctx *c, uint64_t gal)
{
    for (auto &k : c->ksk)
        if (k.gal == gal) return k.d;
    return nullptr;
}

int helr_add_key(he_ctx *c, uint64_t gal)
{
    if (helr_find_key(c, gal)) return HE_OK;
    const int n = c->n, np = c->nprime, nq = c->nq;
    const size_t lw = (size_t)np * n;
    uint64_t *sp = nullptr, *key = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&sp, sizeof(uint64_t) * lw));
    HELR_TRY(helr_alloc(c, (void **)&key, sizeof(uint64_t) * (size_t)nq * 2 * lw));
    if (gal == 0) HELR_TRY(helr_square_dev(c, sp, c->d_sk, np));
    else k_automorph(c, sp, c->d_sk, np, gal, c->stream);
    HELR_TRY(helr_make_ksk(c, gal, sp, key));
    HELR_TRY(helr_to_montgomery(c, key, (size_t)nq * 2 * np, np));
    HELR_TRY(helr_ks_key_layout(c, key, (size_t)nq * 2 * np));
    HELR_CUDA(c, cudaGetLastError());
    helr_free(c, sp);
    c->ksk.push_back({gal, key});
    return HE_OK;
}

extern "C" int he_keygen(he_ctx *c, uint64_t seed, const int64_t *rot, size_t nrot)
{
    if (!c || (nrot && !rot)) return HE_EINVAL;
    if (!c->have_keys || c->key_seed != seed) {
        for (auto &k : c->ksk) helr_free(c, k.d);
    for (auto &d : c->boot_diag) helr_free(c, d.second);
        c->ksk.clear();
        HELR_TRY(helr_keygen_base(c, seed));
        HELR_TRY(helr_add_key(c, 0));
    }
    for (size_t i = 0; i < nrot; i++) HELR_TRY(helr_add_key(c, he_galois_elt(c, rot[i])));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    return HE_OK;
}

extern "C" int he_keygen_galois(he_ctx *c, const uint64_t *gals, size_t n)
{
    if (!c || (n && !gals)) return HE_EINVAL;
    if (!c->have_keys) return helr_fail(c, HE_EKEY, "he_keygen first");
    for (size_t i = 0; i < n; i++)
        if (!(gals[i] & 1) || gals[i] >= 2ull * c->n)
            return helr_fail(c, HE_EINVAL, "galois element %llu is not an odd residue below 2N",
                             (unsigned long long)gals[i]);
    for (size_t i = 0; i < n; i++) HELR_TRY(helr_add_key(c, gals[i]));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    return HE_OK;
}

// ------------------------------------------------------------------ handles
int helr_new_ct(he_ctx *c, int level, double scale, he_ct **out)
{
    he_ct *ct = new he_ct();
    ct->ctx = c;
    ct->level = level;
    ct->scale = scale;
    int rc = helr_alloc(c, (void **)&ct->d, sizeof(uint64_t) * 2 * (level + 1) * (size_t)c->n);
    if (rc) {
        delete ct;
        return rc;
    }
    *out = ct;
    return HE_OK;
}
static int new_pt(he_ctx *c, int level, double scale, he_pt **out)
{
    he_pt *pt = new he_pt();
    pt->ctx = c;
    pt->level = level;
    pt->scale = scale;
    int rc = helr_alloc(c, (void **)&pt->d, sizeof(uint64_t) * (level + 1) * (size_t)c->n);
    if (rc) {
        delete pt;
        return rc;
    }
    *out = pt;
    return HE_OK;
}

extern "C" int he_ct_free(he_ct *ct)
{
    if (!ct) return HE_EINVAL;
    helr_free(ct->ctx, ct->d);
    delete ct;
    return HE_OK;
}
extern "C" int he_pt_free(he_pt *pt)
{
    if (!pt) return HE_EINVAL;
    helr_free(pt->ctx, pt->d);
    delete pt;
    return HE_OK;
}
extern "C" int he_ct_level(const he_ct *ct, int *level, double *scale)
{
    if (!ct) return HE_EINVAL;
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    return HE_OK;
}
extern "C" int he_set_scale(he_ct *ct, double scale)
{
    if (!ct || !(scale > 0)) return HE_EINVAL;
    ct->scale = scale;
    return HE_OK;
}

extern "C" int he_encode(he_ctx *c, const double *re, const double *im, size_t nslots, int level, double scale, he_pt **out)
{
    if (!c || !out || !re || nslots > (size_t)c->nslots || level < 0 || level >= c->nq || !(scale > 0)) return HE_EINVAL;
    *out = nullptr;
    double *d = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&d, sizeof(double) * 2 * c->nslots));
    HELR_CUDA(c, cudaMemsetAsync(d, 0, sizeof(double) * 2 * c->nslots, c->stream));
    HELR_CUDA(c, cudaMemcpyAsync(d, re, sizeof(double) * nslots, cudaMemcpyHostToDevice, c->stream));
    if (im) HELR_CUDA(c, cudaMemcpyAsync(d + c->nslots, im, sizeof(double) * nslots, cudaMemcpyHostToDevice, c->stream));
    he_pt *pt = nullptr;
    HELR_TRY(new_pt(c, level, scale, &pt));
    int rc = helr_encode_dev(c, d, d + c->nslots, 1, 0, level, scale, pt->d, 0);
    helr_free(c, d);
    if (rc) {
        he_pt_free(pt);
        return rc;
    }
    *out = pt;
    return HE_OK;
}

extern "C" int he_decode(he_ctx *c, const he_pt *pt, double *re, double *im, size_t nslots)
{
    if (!c || !pt || !re || nslots > (size_t)c->nslots) return HE_EINVAL;
    double *d = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&d, sizeof(double) * 2 * c->nslots));
    HELR_TRY(helr_decode_dev(c, pt->d, pt->scale, d, d + c->nslots));
    HELR_CUDA(c, cudaMemcpyAsync(re, d, sizeof(double) * nslots, cudaMemcpyDeviceToHost, c->stream));
    if (im) HELR_CUDA(c, cudaMemcpyAsync(im, d + c->nslots, sizeof(double) * nslots, cudaMemcpyDeviceToHost, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, d);
    return HE_OK;
}

extern "C" int he_encrypt(he_ctx *c, const he_pt *pt, uint64_t seed, he_ct **out)
{
    if (!c || !pt || !out) return HE_EINVAL;
    he_ct *ct = nullptr;
    HELR_TRY(helr_new_ct(c, pt->level, pt->scale, &ct));
    int rc = helr_encrypt_dev(c, pt->d, pt->level, seed, ct->d);
    if (rc) {
        he_ct_free(ct);
        return rc;
    }
    *out = ct;
    return HE_OK;
}

extern "C" int he_decrypt(he_ctx *c, const he_ct *ct, he_pt **out)
{
    if (!c || !ct || !out) return HE_EINVAL;
    he_pt *pt = nullptr;
    HELR_TRY(new_pt(c, ct->level, ct->scale, &pt));
    int rc = helr_decrypt_dev(c, ct->d, ct->level, pt->d);
    if (rc) {
        he_pt_free(pt);
        return rc;
    }
    *out = pt;
    return HE_OK;
}

extern "C" int he_ct_export(const he_ct *ct, uint64_t *words, size_t nw, int *level, double *scale)
{
    if (!ct || !words) return HE_EINVAL;
    he_ctx *c = ct->ctx;
    const size_t need = 2 * (size_t)(ct->level + 1) * c->n;
    if (nw < need) return helr_fail(c, HE_EINVAL, "export buffer too small");
    uint64_t *tmp = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&tmp, need * 8));
    LimbMap lm = limbmap_ct(ct->level);
    HELR_TRY(helr_ntt_inv_oop(c, ct->d, tmp, 2 * (size_t)(ct->level + 1), lm, c->stream));
    HELR_CUDA(c, cudaMemcpyAsync(words, tmp, need * 8, cudaMemcpyDeviceToHost, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, tmp);
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    return HE_OK;
}

extern "C" int he_pt_export(const he_pt *pt, uint64_t *words, size_t nw, int *level, double *scale)
{
    if (!pt || !words) return HE_EINVAL;
    he_ctx *c = pt->ctx;
    const size_t need = (size_t)(pt->level + 1) * c->n;
    if (nw < need) return helr_fail(c, HE_EINVAL, "export buffer too small");
    uint64_t *tmp = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&tmp, need * 8));
    HELR_TRY(helr_ntt_inv_oop(c, pt->d, tmp, pt->level + 1, limbmap_ct(pt->level), c->stream));
    HELR_CUDA(c, cudaMemcpyAsync(words, tmp, need * 8, cudaMemcpyDeviceToHost, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, tmp);
    if (level) *level = pt->level;
    if (scale) *scale = pt->scale;
    return HE_OK;
}

extern "C" int he_ct_import(he_ctx *c, const uint64_t *words, size_t nw, int level, double scale, he_ct **out)
{
    if (!c || !words || !out || level < 0 || level >= c->nq) return HE_EINVAL;
    const size_t need = 2 * (size_t)(level + 1) * c->n;
    if (nw < need) return helr_fail(c, HE_EINVAL, "import buffer too small");
    for (size_t k = 0; k < need; k++)
        if (words[k] >= c->q[(k / c->n) % (size_t)(level + 1)])
            return helr_fail(c, HE_EINVAL, "import word not reduced modulo its prime");
    he_ct *ct = nullptr;
    HELR_TRY(helr_new_ct(c, level, scale, &ct));
    HELR_CUDA(c, cudaMemcpyAsync(ct->d, words, need * 8, cudaMemcpyHostToDevice, c->stream));
    HELR_TRY(helr_ntt_fwd(c, ct->d, 2 * (size_t)(level + 1), limbmap_ct(level), c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = ct;
    return HE_OK;
}

// ------------------------------------------------------------------ key switching
// d_in: [batch][nl][N] evaluation form; d_out: [batch][2][nl][N].
int helr_keyswitch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level, const uint64_t *key,
                   KsScratch *ws, const KsOut *o)
{
    const int nl = level + 1, nt = nl + 1;
    const size_t N = c->n;
    const size_t in_items = (size_t)batch * nl;
    KsScratch local;
    if (!ws) {
        HELR_TRY(helr_ks_scratch_alloc(c, batch, level, &local));
        ws = &local;
    }
    cudaStream_t s = c->stream;
    prof_start(c, PROF_KS, s);
    // 1. row pass of the inverse transform of every limb (the column pass runs inside ModUp)
    HELR_TRY(helr_ntt_inv_rows(c, d_in, 2 * N, N, ws->drow, in_items, limbmap_ct(level), s));
    // 2-3. ModUp fused with the transforms and the inner product, in waves
    // (the wave of this limb count, within the scratch's capacity)
    const size_t per_item = (size_t)nl * nt * N;
    const int wave = (int)std::max<size_t>(
        1, std::min({(size_t)(ws->wave > 0 ? ws->wave : helr_ks_wave(c, nl)), (size_t)batch, ws->ext_cap / per_item}));
    for (int b0 = 0; b0 < batch; b0 += wave) {
        int cnt = std::min(wave, batch - b0);
        HELR_TRY(helr_ks_fused(c, d_in + (size_t)b0 * nl * N, ws->drow + (size_t)b0 * nl * N, ws->ext, key,
                               ws->acc + (size_t)b0 * 2 * nt * N, cnt, nl, s));
    }
    // 4. ModDown: subtract the centred P-part and divide by P
    HELR_TRY(helr_ntt_inv_rows(c, ws->acc + (size_t)nl * N, 2 * (size_t)nt * N, (size_t)nt * N, ws->pl, (size_t)batch * 2,
                               limbmap_single(c->nq), s));
    KsOut plain;
    plain.out = Str{d_out, 2 * (size_t)nl * N, (size_t)nl * N};
    HELR_TRY(helr_ks_down(c, o ? *o : plain, ws->acc, 2 * (size_t)nt * N, (size_t)nt * N, ws->pl, c->nq, ws->lift, batch,
                          nl, c->d_pinv, s));
    HELR_CUDA(c, cudaGetLastError());
    const double waves = (double)((batch + wave - 1) / wave);
    prof_stop(c, PROF_KS, s, (double)batch, 0, (double)batch * nl,
              3.0 * nl * batch + waves * 2.0 * nl * (nl + 1));
    if (c->prof.on) c->prof.ks_by_limbs[nl] += batch;
    if (ws == &local) helr_ks_scratch_free(c, &local);
    return HE_OK;
}

// Hoisted rotation sum: out = a + sum_j Rot_{gal_j}(a) for every item of the
// batch.  The second polynomials are decomposed once (inverse row pass, ModUp
// with the column passes, the row passes of the lifted digits), the inner
// products of all rotations are summed over {q_0..q_l, P} (the automorphisms
// act on the transformed digits), and one ModDown forms
//   out_0 = a_0 + sum_j sigma_j(a_0) + KS_0,  out_1 = a_1 + KS_1
// in its output stage.  out must not alias a.
int helr_rotsum(he_ctx *c, const uint64_t *a, size_t a_item, int batch, int level, const HoistKeys &hk, KsScratch *ws,
                Str out)
{
    const int nl = level + 1, nt = nl + 1;
    const size_t N = c->n, lw = (size_t)nl * N;
    if (hk.n < 1 || hk.n > HELR_MAX_HOIST) return helr_fail(c, HE_EINVAL, "%d rotations in one hoisted sum", hk.n);
    // the summed 128-bit products must not overflow: hk.n * nl terms below q^2,
    // or below 20 q^2 where the digits' row pass leaves its words unreduced
    for (int t = 0; t <= nl; t++) {
        const uint64_t q = t < nl ? c->q[t] : c->q[c->nq];
        const unsigned f = (unsigned)hk.n * (unsigned)nl * (q < HELR_LZ_QMAX ? 20u : 1u);
        if ((u128)q * q > ~(u128)0 / f)
            return helr_fail(c, HE_EINVAL, "%d rotations x %d digits overflow the 128-bit sums", hk.n, nl);
    }
    cudaStream_t s = c->stream;
    prof_start(c, PROF_KS, s);
    // 1. row pass of the inverse transform of every second-polynomial limb
    HELR_TRY(helr_ntt_inv_rows(c, a + lw, a_item, N, ws->drow, (size_t)batch * nl, limbmap_ct(level), s, nl));
    // 2. ModUp, the digits' transforms and the summed inner products, in waves
    const size_t per_item = (size_t)nl * nt * N;
    const int wave = (int)std::max<size_t>(
        1, std::min({(size_t)(ws->wave > 0 ? ws->wave : helr_ks_wave(c, nl)), (size_t)batch, ws->ext_cap / per_item}));
    for (int b0 = 0; b0 < batch; b0 += wave) {
        const int cnt = std::min(wave, batch - b0);
        HELR_TRY(helr_ks_hoisted(c, a + (size_t)b0 * a_item + lw, a_item, ws->drow + (size_t)b0 * nl * N, ws->ext, hk,
                                 ws->acc + (size_t)b0 * 2 * nt * N, cnt, nl, s));
    }
    // 3. one ModDown, with the c0 terms of every rotation and a itself
    HELR_TRY(helr_ntt_inv_rows(c, ws->acc + (size_t)nl * N, 2 * (size_t)nt * N, (size_t)nt * N, ws->pl, (size_t)batch * 2,
                               limbmap_single(c->nq), s));
    KsOut o;
    o.out = out;
    o.rot = a;
    o.rot_item = a_item;
    for (int j = 0; j < hk.n; j++) o.gals[j] = hk.gal[j];
    o.ngal = hk.n;
    o.acc = a;
    o.acc_item = a_item;
    o.acc_poly = lw;
    HELR_TRY(helr_ks_down(c, o, ws->acc, 2 * (size_t)nt * N, (size_t)nt * N, ws->pl, c->nq, ws->lift, batch, nl, c->d_pinv, s));
    HELR_CUDA(c, cudaGetLastError());
    const double waves = (double)((batch + wave - 1) / wave);
    // algorithmic DRAM: input read once, output written once, the keys of every rotation once per wave
    prof_stop(c, PROF_KS, s, (double)batch * hk.n, 0, (double)batch * hk.n * nl,
              3.0 * nl * batch + waves * hk.n * 2.0 * nl * (nl + 1));
    if (c->prof.on) c->prof.ks_by_limbs[nl] += (double)batch * hk.n;
    return HE_OK;
}

int helr_ks_scratch_alloc(he_ctx *c, int batch, int level, KsScratch *ws)
{
    const int nl = level + 1, nt = nl + 1;
    const size_t N = c->n;
    // ext holds one wave at any limb count up to nl, each with its own wave size
    size_t ext = 0;
    for (int k = 1; k <= nl; k++)
        ext = std::max(ext, (size_t)std::min(helr_ks_wave(c, k), batch) * k * (k + 1) * N);
    size_t words = (size_t)batch * (nl * N + 2 * nt * N + 2 * N + 2 * (size_t)nl * N) + ext;
    uint64_t *base = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&base, words * 8));
    ws->base = base;
    ws->drow = base;
    ws->acc = ws->drow + (size_t)batch * nl * N;
    ws->pl = ws->acc + (size_t)batch * 2 * nt * N;
    ws->lift = ws->pl + (size_t)batch * 2 * N;
    ws->ext = ws->lift + (size_t)batch * 2 * nl * N;
    ws->batch = batch;
    ws->level = level;
    ws->wave = 0;
    ws->ext_cap = ext;
    return HE_OK;
}
void helr_ks_scratch_free(he_ctx *c, KsScratch *ws)
{
    helr_free(c, ws->base);
    ws->base = nullptr;
}

extern "C" int he_keyswitch_batch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level, uint64_t gal)
{
    if (!c || !d_in || !d_out || batch <= 0 || level < 0 || level >= c->nq) return HE_EINVAL;
    const uint64_t *key = helr_find_key(c, gal);
    if (!key) return helr_fail(c, HE_EKEY, "no key-switching key for galois element %llu", (unsigned long long)gal);
    return helr_keyswitch(c, d_in, d_out, batch, level, key, nullptr);
}

extern "C" int he_rotsum_batch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level, const int64_t *rots,
                               size_t n_rot)
{
    if (!c || !d_in || !d_out || !rots || batch <= 0 || level < 0 || level >= c->nq || n_rot < 1 ||
        n_rot > HELR_MAX_HOIST || d_in == d_out)
        return HE_EINVAL;
    HoistKeys hk{};
    hk.n = (int)n_rot;
    for (size_t j = 0; j < n_rot; j++) {
        hk.gal[j] = he_galois_elt(c, rots[j]);
        hk.key[j] = helr_find_key(c, hk.gal[j]);
        if (!hk.key[j]) return helr_fail(c, HE_EKEY, "no rotation key for %lld", (long long)rots[j]);
    }
    const size_t ct = 2 * (size_t)(level + 1) * c->n;
    KsScratch ws;
    HELR_TRY(helr_ks_scratch_alloc(c, batch, level, &ws));
    const int rc = helr_rotsum(c, d_in, ct, batch, level, hk, &ws, Str{d_out, ct, (size_t)(level + 1) * c->n});
    helr_ks_scratch_free(c, &ws);
    return rc;
}

static int limbmap_from(const he_ctx *c, const int *prime_of, int period, LimbMap *m)
{
    if (!prime_of || period <= 0 || period > HELR_MAXQ + 1) return HE_EINVAL;
    m->period = period;
    for (int i = 0; i < period; i++) {
        if (prime_of[i] < 0 || prime_of[i] >= c->nprime) return HE_EINVAL;
        m->p[i] = (unsigned char)prime_of[i];
    }
    return HE_OK;
}
extern "C" int he_ntt_forward(he_ctx *c, uint64_t *d, size_t nlimbs, const int *prime_of, int period)
{
    LimbMap m;
    if (!c || !d || limbmap_from(c, prime_of, period, &m)) return HE_EINVAL;
    return helr_ntt_fwd(c, d, nlimbs, m, c->stream);
}
extern "C" int he_ntt_inverse(he_ctx *c, uint64_t *d, size_t nlimbs, const int *prime_of, int period)
{
    LimbMap m;
    if (!c || !d || limbmap_from(c, prime_of, period, &m)) return HE_EINVAL;
    return helr_ntt_inv(c, d, nlimbs, m, c->stream);
}
