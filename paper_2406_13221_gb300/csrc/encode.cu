// encode.cu -- canonical-embedding encode/decode (FP64), sampling, encryption
// and key generation kernels (Sec. 2.1: Enc, Dec; Sec. 4.3 Steps 2 and 8).
//
// Encoding: slot j <-> evaluation at zeta^(5^j) (zeta = exp(i pi / N)).  With
// n = N/2, s(j) = (5^j mod 2N - 1) / 4 and w = zeta^4:
//   u_k = (1/n) zeta^-k sum_s V_s w^(-s k),  V_(s(j)) = z_j,
//   coefficient k = Re u_k, coefficient k + n = Im u_k, rounded half away from zero
// after multiplying by the scale.  Decoding runs the same transform forwards.
// The DFT is radix-2 decimation in time over bit-reversed input; every complex
// product is (a.re b.re - a.im b.im, a.re b.im + a.im b.re) with explicitly
// rounded double operations (no contraction), so results are reproducible.
//
// Randomness: splitmix64 (Steele, Lea & Flood 2014) used as a counter-based
// generator: word idx of stream st under seed is mix64(mix64(seed) + k GOLDEN)
// with k = (st << 40) + idx + 1.
#include "helr_internal.cuh"

#define GS_LOOP(i, n) for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

namespace {

inline unsigned grid_for(size_t work, int threads = 256)
{
    size_t b = (work + threads - 1) / threads;
    if (b > (size_t)152 * 64) b = (size_t)152 * 64;
    return (unsigned)(b ? b : 1);
}

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t rand_word(uint64_t seedm, uint64_t st, uint64_t idx)
{
    return mix64(seedm + ((st << 40) + idx + 1) * 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ uint64_t smod_dev(int64_t x, const ModQ m)
{
    if (x >= 0) return reduce64((uint64_t)x, m);
    uint64_t r = reduce64((uint64_t)(-x), m);
    return r ? m.q - r : 0;
}

// kind 0: ternary, 1: Gaussian (CDT), 2: uniform mod q (128-bit word pair)
__global__ void k_sample_kernel(uint64_t *out, size_t nwords, int logn, LimbMap lm, uint64_t seedm, uint64_t st, int kind,
                                const uint64_t *cdt, int cdt_len, const ModQ *mods)
{
    const int n = 1 << logn;
    GS_LOOP(i, nwords) {
        size_t limb = i >> logn;
        uint64_t k = i & (n - 1);
        int p = limb_prime(lm, limb);
        ModQ m = mods[p];
        uint64_t v;
        if (kind == 0) {
            int64_t t = (int64_t)(rand_word(seedm, st, k) % 3) - 1;
            v = smod_dev(t, m);
        } else if (kind == 1) {
            uint64_t w = rand_word(seedm, st, k), u = w >> 1;
            int j = 0;
            while (j < cdt_len - 1 && u >= cdt[j]) j++;
            int64_t x = ((w & 1) && j) ? -(int64_t)j : (int64_t)j;
            v = smod_dev(x, m);
        } else {
            uint64_t idx = (uint64_t)p * (uint64_t)n + k;
            uint64_t hi = rand_word(seedm, st, 2 * idx), lo = rand_word(seedm, st, 2 * idx + 1);
            uint64_t r64 = reduce64(~0ull, m) + 1;  // 2^64 mod q
            if (r64 == m.q) r64 = 0;
            v = addmod(mulmod(reduce64(hi, m), r64, m), reduce64(lo, m), m.q);
        }
        out[i] = v;
    }
}

// out = a - b * s  (+ optional): used for keys  b = e - a s
__global__ void k_e_minus_as(uint64_t *out, const uint64_t *e, const uint64_t *a, const uint64_t *s, size_t nwords,
                             int logn, LimbMap lm, const ModQ *mods)
{
    GS_LOOP(i, nwords) {
        size_t limb = i >> logn;
        int p = limb_prime(lm, limb);
        ModQ m = mods[p];
        uint64_t k = i & ((1u << logn) - 1);
        uint64_t as = mulmod(a[i], s[((size_t)p << logn) + k], m);
        out[i] = submod(e[i], as, m.q);
    }
}

// out[limb d] += f * sp[prime d] for the digit limb of a key-switching key
__global__ void k_add_scaled(uint64_t *out, const uint64_t *sp, uint64_t f, int n, const ModQ *mods, int p)
{
    ModQ m = mods[p];
    GS_LOOP(k, (size_t)n) out[k] = addmod(out[k], mulmod(f, sp[k], m), m.q);
}

// c = a * b + e (+ m when m != NULL); all [nl][N] evaluation form, limb j mod q_j
__global__ void k_mul_add(uint64_t *c, const uint64_t *a, const uint64_t *b, const uint64_t *e, const uint64_t *msg,
                          size_t nwords, int logn, const ModQ *mods)
{
    GS_LOOP(i, nwords) {
        int j = (int)(i >> logn);
        ModQ m = mods[j];
        uint64_t v = addmod(mulmod(a[i], b[i], m), e[i], m.q);
        if (msg) v = addmod(v, msg[i], m.q);
        c[i] = v;
    }
}

__global__ void k_square(uint64_t *out, const uint64_t *in, size_t nwords, int logn, const ModQ *mods)
{
    GS_LOOP(i, nwords) {
        ModQ m = mods[i >> logn];
        out[i] = mulmod(in[i], in[i], m);
    }
}

// ---------------------------------------------------------------- FFT
__device__ __forceinline__ void cmul_rn(double ar, double ai, double br, double bi, double &cr, double &ci)
{
    cr = __dsub_rn(__dmul_rn(ar, br), __dmul_rn(ai, bi));
    ci = __dadd_rn(__dmul_rn(ar, bi), __dmul_rn(ai, br));
}

__global__ void k_enc_scatter(const double *re, const double *im, double *vr, double *vi, int ns, int logns,
                              const int *sidx, int batch, size_t in_stride)
{
    GS_LOOP(u, (size_t)batch * ns) {
        size_t b = u / ns;
        int j = (int)(u % ns);
        int pos = (int)(__brev((unsigned)sidx[j]) >> (32 - logns));
        vr[b * ns + pos] = re[b * in_stride + j];
        vi[b * ns + pos] = im ? im[b * in_stride + j] : 0.0;
    }
}

__global__ void k_fft_stage(double *vr, double *vi, int ns, int batch, int len, int inverse, const double *zeta)
{
    const int half = len >> 1, tstep = ns / len;
    GS_LOOP(u, (size_t)batch * (ns / 2)) {
        size_t b = u / (ns / 2);
        int v = (int)(u % (ns / 2));
        int grp = v / half, j = v % half;
        size_t i0 = b * ns + (size_t)grp * len + j, i1 = i0 + half;
        int idx = 4 * j * tstep;
        double br = zeta[2 * idx], bi = zeta[2 * idx + 1];
        if (inverse) bi = -bi;
        double yr, yi;
        cmul_rn(vr[i1], vi[i1], br, bi, yr, yi);
        double xr = vr[i0], xi = vi[i0];
        vr[i0] = __dadd_rn(xr, yr);
        vi[i0] = __dadd_rn(xi, yi);
        vr[i1] = __dsub_rn(xr, yr);
        vi[i1] = __dsub_rn(xi, yi);
    }
}

// u = (v / n) * conj(zeta^k); coefficients round_half_away(scale * u) into limbs
__global__ void k_enc_finish(const double *vr, const double *vi, uint64_t *out, int ns, int logn, int nl, double scale,
                             const double *zeta, const ModQ *mods, int batch, size_t out_stride, int *err)
{
    const double inv_n = 1.0 / (double)ns;
    GS_LOOP(u, (size_t)batch * ns) {
        size_t b = u / ns;
        int k = (int)(u % ns);
        double ar = __dmul_rn(vr[b * ns + k], inv_n), ai = __dmul_rn(vi[b * ns + k], inv_n);
        double cr, ci;
        cmul_rn(ar, ai, zeta[2 * k], -zeta[2 * k + 1], cr, ci);
        double x0 = __dmul_rn(cr, scale), x1 = __dmul_rn(ci, scale);
        const double lim = 4611686018427387904.0;
        if (!(fabs(x0) < lim) || !(fabs(x1) < lim)) {
            atomicExch(err, 1);
            x0 = 0.0;
            x1 = 0.0;
        }
        int64_t m0 = llround(x0), m1 = llround(x1);
        uint64_t *o = out + b * out_stride;
        for (int j = 0; j < nl; j++) {
            ModQ m = mods[j];
            o[((size_t)j << logn) + k] = smod_dev(m0, m);
            o[((size_t)j << logn) + k + ns] = smod_dev(m1, m);
        }
    }
}

// v_k = (centred m_k + i centred m_(k+n)) * zeta^k, written at bitrev(k)
__global__ void k_dec_start(const uint64_t *coef, double *vr, double *vi, int ns, int logns, uint64_t q0, const double *zeta)
{
    GS_LOOP(u, (size_t)ns) {
        int k = (int)u;
        uint64_t a = coef[k], b = coef[k + ns];
        int64_t ca = a > (q0 >> 1) ? (int64_t)a - (int64_t)q0 : (int64_t)a;
        int64_t cb = b > (q0 >> 1) ? (int64_t)b - (int64_t)q0 : (int64_t)b;
        double yr, yi;
        cmul_rn(__ll2double_rn(ca), __ll2double_rn(cb), zeta[2 * k], zeta[2 * k + 1], yr, yi);
        int pos = (int)(__brev((unsigned)k) >> (32 - logns));
        vr[pos] = yr;
        vi[pos] = yi;
    }
}

__global__ void k_dec_finish(const double *vr, const double *vi, double *re, double *im, int ns, const int *sidx, double scale)
{
    GS_LOOP(u, (size_t)ns) {
        int s = sidx[u];
        re[u] = __ddiv_rn(vr[s], scale);
        im[u] = __ddiv_rn(vi[s], scale);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
int helr_sample(he_ctx *c, uint64_t *out, size_t nlimbs, const LimbMap &lm, uint64_t seed, uint64_t stream, int kind)
{
    size_t nw = nlimbs << c->logn;
    if (!nw) return HE_OK;
    HELR_LAUNCH(k_sample_kernel<<<grid_for(nw), 256, 0, c->stream>>>(out, nw, c->logn, lm, mix64(seed), stream, kind, c->t.cdt,
                                                        c->cdt_len, c->t.mod));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// Encode `batch` slot vectors (device doubles, row stride in_stride) at `level`
// into evaluation-form plaintexts d_out [batch][level+1][N] (row stride out_stride).
int helr_encode_dev(he_ctx *c, const double *d_re, const double *d_im, int batch, size_t in_stride, int level,
                    double scale, uint64_t *d_out, size_t out_stride)
{
    const int ns = c->nslots, logns = c->logn - 1;
    double *v = nullptr;
    int *err = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&v, sizeof(double) * 2 * (size_t)batch * ns + 256));
    err = (int *)(v + 2 * (size_t)batch * ns);
    double *vr = v, *vi = v + (size_t)batch * ns;
    HELR_CUDA(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
    size_t work = (size_t)batch * ns;
    HELR_LAUNCH(k_enc_scatter<<<grid_for(work), 256, 0, c->stream>>>(d_re, d_im, vr, vi, ns, logns, c->t.sidx, batch, in_stride));
    for (int len = 2; len <= ns; len <<= 1)
        HELR_LAUNCH(k_fft_stage<<<grid_for(work / 2), 256, 0, c->stream>>>(vr, vi, ns, batch, len, 1, c->t.zeta));
    HELR_LAUNCH(k_enc_finish<<<grid_for(work), 256, 0, c->stream>>>(vr, vi, d_out, ns, c->logn, level + 1, scale, c->t.zeta,
                                                       c->t.mod, batch, out_stride, err));
    HELR_CUDA(c, cudaGetLastError());
    int herr = 0;
    HELR_CUDA(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, v);
    if (herr) return helr_fail(c, HE_EINVAL, "encoded coefficient outside (-2^62, 2^62)");
    // coefficient form -> evaluation form, limb by limb
    for (int b = 0; b < batch; b++)
        HELR_TRY(helr_ntt_fwd(c, d_out + (size_t)b * out_stride, level + 1, limbmap_ct(level), c->stream));
    return HE_OK;
}

// Decode limb 0 of an evaluation-form plaintext into device slot vectors.
int helr_decode_dev(he_ctx *c, const uint64_t *d_pt, double scale, double *d_re, double *d_im)
{
    const int ns = c->nslots, logns = c->logn - 1;
    uint64_t *coef = nullptr;
    double *v = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&coef, sizeof(uint64_t) * c->n));
    HELR_TRY(helr_alloc(c, (void **)&v, sizeof(double) * 2 * ns));
    HELR_TRY(helr_ntt_inv_oop(c, d_pt, coef, 1, limbmap_single(0), c->stream));
    HELR_LAUNCH(k_dec_start<<<grid_for(ns), 256, 0, c->stream>>>(coef, v, v + ns, ns, logns, c->q[0], c->t.zeta));
    for (int len = 2; len <= ns; len <<= 1)
        HELR_LAUNCH(k_fft_stage<<<grid_for(ns / 2), 256, 0, c->stream>>>(v, v + ns, ns, 1, len, 0, c->t.zeta));
    HELR_LAUNCH(k_dec_finish<<<grid_for(ns), 256, 0, c->stream>>>(v, v + ns, d_re, d_im, ns, c->t.sidx, scale));
    HELR_CUDA(c, cudaGetLastError());
    helr_free(c, coef);
    helr_free(c, v);
    return HE_OK;
}

// ct = (v b + e0 + m, v a + e1) at `level` (streams: v 4, e0 5, e1 6)
int helr_encrypt_dev(he_ctx *c, const uint64_t *d_pt, int level, uint64_t seed, uint64_t *d_ct)
{
    if (!c->have_keys) return helr_fail(c, HE_EKEY, "no public key: call he_keygen first");
    const int nl = level + 1;
    const size_t lw = (size_t)nl << c->logn;
    uint64_t *tmp = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&tmp, sizeof(uint64_t) * 3 * lw));
    uint64_t *v = tmp, *e0 = tmp + lw, *e1 = tmp + 2 * lw;
    LimbMap lm = limbmap_ct(level);
    HELR_TRY(helr_sample(c, v, nl, lm, seed, 4, 0));
    HELR_TRY(helr_sample(c, e0, nl, lm, seed, 5, 1));
    HELR_TRY(helr_sample(c, e1, nl, lm, seed, 6, 1));
    HELR_TRY(helr_ntt_fwd(c, tmp, 3 * (size_t)nl, lm, c->stream));
    const uint64_t *pk0 = c->d_pk, *pk1 = c->d_pk + ((size_t)c->nq << c->logn);
    HELR_LAUNCH(k_mul_add<<<grid_for(lw), 256, 0, c->stream>>>(d_ct, v, pk0, e0, d_pt, lw, c->logn, c->t.mod));
    HELR_LAUNCH(k_mul_add<<<grid_for(lw), 256, 0, c->stream>>>(d_ct + lw, v, pk1, e1, nullptr, lw, c->logn, c->t.mod));
    HELR_CUDA(c, cudaGetLastError());
    helr_free(c, tmp);
    return HE_OK;
}

// pt = c0 + c1 s
int helr_decrypt_dev(he_ctx *c, const uint64_t *d_ct, int level, uint64_t *d_pt)
{
    if (!c->have_keys) return helr_fail(c, HE_EKEY, "no secret key");
    const size_t lw = (size_t)(level + 1) << c->logn;
    HELR_LAUNCH(k_mul_add<<<grid_for(lw), 256, 0, c->stream>>>(d_pt, d_ct + lw, c->d_sk, d_ct, nullptr, lw, c->logn, c->t.mod));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// secret (stream 1), public key (a: stream 2, e: stream 3)
int helr_keygen_base(he_ctx *c, uint64_t seed)
{
    const int n = c->n, nq = c->nq, np = c->nprime;
    LimbMap all;
    all.period = np;
    for (int j = 0; j < np; j++) all.p[j] = (unsigned char)j;
    if (c->secret_hw > 0) {
        // exactly h nonzero coefficients: word k of stream 7 picks position
        // word mod N (skipped when taken) and the sign from bit 32
        std::vector<int64_t> sk((size_t)n, 0);
        const uint64_t seedm = mix64(seed);
        for (uint64_t k = 0, placed = 0; placed < (uint64_t)c->secret_hw; k++) {
            const uint64_t w = mix64(seedm + ((7ull << 40) + k + 1) * 0x9E3779B97F4A7C15ull);
            const uint64_t pos = w % (uint64_t)n;
            if (sk[pos]) continue;
            sk[pos] = (w >> 32) & 1 ? 1 : -1;
            placed++;
        }
        std::vector<uint64_t> limbs((size_t)np * n);
        for (int j = 0; j < np; j++)
            for (int i = 0; i < n; i++)
                limbs[(size_t)j * n + i] = sk[i] >= 0 ? (uint64_t)sk[i] : c->q[j] - 1;
        HELR_CUDA(c, cudaMemcpyAsync(c->d_sk, limbs.data(), sizeof(uint64_t) * limbs.size(), cudaMemcpyHostToDevice,
                                     c->stream));
        HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    } else {
        HELR_TRY(helr_sample(c, c->d_sk, np, all, seed, 1, 0));
    }
    // host copy of the ternary secret: limb 0 in coefficient form, centred
    std::vector<uint64_t> h((size_t)n);
    HELR_CUDA(c, cudaMemcpyAsync(h.data(), c->d_sk, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, c->stream));
    HELR_TRY(helr_ntt_fwd(c, c->d_sk, np, all, c->stream));
    uint64_t *tmp = nullptr;
    const size_t lw = (size_t)nq * n;
    HELR_TRY(helr_alloc(c, (void **)&tmp, sizeof(uint64_t) * 2 * lw));
    LimbMap lq = limbmap_ct(nq - 1);
    HELR_TRY(helr_sample(c, tmp, nq, lq, seed, 2, 2));        // a
    HELR_TRY(helr_sample(c, tmp + lw, nq, lq, seed, 3, 1));   // e
    HELR_TRY(helr_ntt_fwd(c, tmp, 2 * (size_t)nq, lq, c->stream));
    HELR_LAUNCH(k_e_minus_as<<<grid_for(lw), 256, 0, c->stream>>>(c->d_pk, tmp + lw, tmp, c->d_sk, lw, c->logn, lq, c->t.mod));
    HELR_CUDA(c, cudaMemcpyAsync(c->d_pk + lw, tmp, sizeof(uint64_t) * lw, cudaMemcpyDeviceToDevice, c->stream));
    HELR_CUDA(c, cudaGetLastError());
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, tmp);
    for (int i = 0; i < n; i++) c->h_sk[i] = h[i] == 0 ? 0 : (h[i] == 1 ? 1 : -1);
    c->have_keys = 1;
    c->key_seed = seed;
    return HE_OK;
}

// Key-switching key for s' (evaluation form over all primes, [nprime][N]) with
// galois tag gal: digit d, limb t: b = e_d - a_dt s + [t == d] (P mod q_d) s'.
// Streams: a (1 << 24 | gal << 6 | d), e (2 << 24 | gal << 6 | d).
int helr_make_ksk(he_ctx *c, uint64_t gal, const uint64_t *sprime, uint64_t *out)
{
    const int n = c->n, nq = c->nq, np = c->nprime;
    const size_t lw = (size_t)np * n;
    LimbMap all;
    all.period = np;
    for (int j = 0; j < np; j++) all.p[j] = (unsigned char)j;
    uint64_t *e = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&e, sizeof(uint64_t) * lw));
    for (int d = 0; d < nq; d++) {
        uint64_t sta = (1ull << 24) | (gal << 6) | (uint64_t)d, ste = (2ull << 24) | (gal << 6) | (uint64_t)d;
        uint64_t *b = out + (size_t)d * 2 * lw, *a = b + lw;
        HELR_TRY(helr_sample(c, a, np, all, c->key_seed, sta, 2));
        HELR_TRY(helr_sample(c, e, np, all, c->key_seed, ste, 1));
        HELR_TRY(helr_ntt_fwd(c, a, np, all, c->stream));
        HELR_TRY(helr_ntt_fwd(c, e, np, all, c->stream));
        HELR_LAUNCH(k_e_minus_as<<<grid_for(lw), 256, 0, c->stream>>>(b, e, a, c->d_sk, lw, c->logn, all, c->t.mod));
        uint64_t pmod = c->q[nq] % c->q[d];
        HELR_LAUNCH(k_add_scaled<<<grid_for(n), 256, 0, c->stream>>>(b + (size_t)d * n, sprime + (size_t)d * n, pmod, n, c->t.mod, d));
        HELR_CUDA(c, cudaGetLastError());
    }
    helr_free(c, e);
    return HE_OK;
}

// x <- x 2^64 mod q for nlimbs limbs, limb i modulo prime i % period
__global__ void k_to_mont(uint64_t *x, size_t nwords, int logn, int period, const ModQ *mods)
{
    GS_LOOP(i, nwords) {
        const ModQ m = mods[(i >> logn) % period];
        uint64_t r64 = reduce64(~0ull, m) + 1;
        if (r64 == m.q) r64 = 0;
        x[i] = mulmod(x[i], r64, m);
    }
}

int helr_to_montgomery(he_ctx *c, uint64_t *x, size_t nlimbs, int period)
{
    size_t nw = nlimbs << c->logn;
    HELR_LAUNCH(k_to_mont<<<grid_for(nw), 256, 0, c->stream>>>(x, nw, c->logn, period, c->t.mod));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int helr_square_dev(he_ctx *c, uint64_t *out, const uint64_t *in, size_t nlimbs)
{
    size_t nw = nlimbs << c->logn;
    HELR_LAUNCH(k_square<<<grid_for(nw), 256, 0, c->stream>>>(out, in, nw, c->logn, c->t.mod));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}
