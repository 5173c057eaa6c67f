// helr_lr.cu -- encrypted logistic-regression training with quadratic-gradient
// NAG (arXiv 2406.13221): client precompute (Sec. 4.3 Steps 1-3), the encrypted
// iteration (Steps 4-6: gradient, quadratic gradient, NAG update of
// Algorithm 1) and the refresh between iterations (Step 7).
//
// Circuit per data block Z_i (all at the top level L, scale Delta):
//  1  t  = Rescale(Relin(Z_i (x) W))                   z_rc w_c
//  2  t += Rot(t, 2^k), k < log2 g                     row sums into column 0
//  3/5 s = (1 - c0) M - c1 (M t) - c3 t^2 (M t)        sigmoid term (Sec. 4.1) with
//          the column-0 mask M inside the plaintext products: t^2 and
//          (-c3 M) t in parallel, then their product; zero outside column 0
//  4  s += Rot(s, -2^k), k < log2 g                    s_r in every column
//  6  grad_i = Rescale(Relin(s (x) Z_i))               s_r z_rc
// then once:
//  7  acc = sum_i grad_i; acc += Rot(acc, g 2^k), k < log2 m   column sums
//  8  nG = Rescale(Relin(acc (x) B))                   n Bbar_c g_c (quadratic gradient)
//  9  V' = W + alpha nG/n,  W' = (1 - eta) V' + eta V  Algorithm 1 update
// The multiplier on G is alpha = F2(t) (the learning rate 2 - (t/81)^2.5 of the
// experiments), applied with the public scalar 1/n; Bbar and g are unnormalised
// sums and n Bbar is encrypted.  The circuit of Han et al. that the paper builds
// on is not given: folding the mask into the polynomial computes the same
// function as masking ip before the sigmoid, with one level less.
#include <math.h>
#include <string.h>
#include <thread>
#include <chrono>
#include <algorithm>
#include "helr_internal.cuh"

static const double G8[3] = {0.5, 0.15, -0.0015};
static const double G16[3] = {0.5, 0.0843, -0.0002};
static const double BBAR_EPS = 1e-8;
static const int ITER_DEPTH = 6;  // levels one iteration consumes
static const int ITER_DEPTH_FO = 5;  // the first-order baseline: no Bbar product

static uint64_t obj_seed(uint64_t base, uint64_t kind, uint64_t index) { return base + (kind << 48) + index; }

// ------------------------------------------------------------------ client precompute
// Bbar_c = 1 / (eps + 1/4 sum_k |(Z^T Z)_ck|) over rows [r0, r0 + rows) of Z = y [1 | X]
static void bbar_rows(const double *X, const double *y, size_t f, size_t r0, size_t rows, size_t g, double *out)
{
    const size_t f1 = f + 1;
    std::vector<double> H(f1 * f1, 0.0), z(f1);
    for (size_t r = r0; r < r0 + rows; r++) {
        z[0] = y[r];
        for (size_t c = 0; c < f; c++) z[c + 1] = y[r] * X[r * f + c];
        for (size_t a = 0; a < f1; a++) {
            double za = z[a];
            double *h = &H[a * f1];
            for (size_t b = a; b < f1; b++) h[b] += za * z[b];
        }
    }
    for (size_t a = 0; a < g; a++) out[a] = 0.0;
    for (size_t a = 0; a < f1; a++) {
        double s = 0.0;
        for (size_t b = 0; b < f1; b++) s += fabs(a <= b ? H[a * f1 + b] : H[b * f1 + a]);
        out[a] = 1.0 / (BBAR_EPS + 0.25 * s);
    }
}

extern "C" int he_lr_bbar(const double *X, const double *y, size_t n, size_t f, size_t row0, size_t rows, size_t g,
                          double *out)
{
    if (!X || !y || !out || g < f + 1 || row0 + rows > n) return HE_EINVAL;
    bbar_rows(X, y, f, row0, rows, g, out);
    return HE_OK;
}

// Bbar_k of every mini-batch k on the GPU (the same client precompute).  One
// CTA per (batch, 16 rows a of H = Z_k^T Z_k), one thread per column b: each
// Gram entry is accumulated over the rows in row order and each absolute row
// sum over the columns in column order, with separate multiplies and adds (no
// contraction), so the result equals bbar_rows bit for bit.
static const int BB_TA = 16, BB_RC = 32;
__global__ void __launch_bounds__(256) k_bbar(const double *__restrict__ X, const double *__restrict__ y, size_t n, int f,
                                              size_t batch_rows, int g, double *__restrict__ out)
{
    extern __shared__ double bsm[];
    const int f1 = f + 1, k = blockIdx.y, a0 = blockIdx.x * BB_TA, b = threadIdx.x;
    double *zs = bsm;                  // [BB_RC][f1]: rows of Z_k
    double *Hs = bsm + BB_RC * f1;     // [BB_TA][f1]: rows a0.. of H
    const size_t r0 = (size_t)k * batch_rows, r1 = min(n, r0 + batch_rows);
    double acc[BB_TA];
#pragma unroll
    for (int a = 0; a < BB_TA; a++) acc[a] = 0.0;
    for (size_t rc = r0; rc < r1; rc += BB_RC) {
        const int cnt = (int)min((size_t)BB_RC, r1 - rc);
        for (int idx = threadIdx.x; idx < cnt * f1; idx += blockDim.x) {
            const int rr = idx / f1, c = idx % f1;
            const double yr = y[rc + rr];
            zs[idx] = c == 0 ? yr : __dmul_rn(yr, X[(rc + rr) * f + c - 1]);
        }
        __syncthreads();
        if (b < f1)
            for (int rr = 0; rr < cnt; rr++) {
                const double zb = zs[rr * f1 + b];
#pragma unroll
                for (int a = 0; a < BB_TA; a++)
                    if (a0 + a < f1) acc[a] = __dadd_rn(acc[a], __dmul_rn(zs[rr * f1 + a0 + a], zb));
            }
        __syncthreads();
    }
    if (b < f1)
#pragma unroll
        for (int a = 0; a < BB_TA; a++) Hs[a * f1 + b] = acc[a];
    __syncthreads();
    const int a = a0 + (int)threadIdx.x;
    if (threadIdx.x < BB_TA && a < f1) {
        double s = 0.0;
        for (int bb = 0; bb < f1; bb++) s = __dadd_rn(s, fabs(Hs[threadIdx.x * f1 + bb]));
        out[(size_t)k * g + a] = 1.0 / __dadd_rn(BBAR_EPS, __dmul_rn(0.25, s));
    }
}

// Bbar_k for the mini-batches of batch_rows rows of Z = y [1 | X] (n x f host
// arrays) into out[nbatch][g] (host), computed on the device
static int bbar_batches_dev(he_ctx *c, const double *X, const double *y, size_t n, size_t f, size_t batch_rows, size_t g,
                            double *out)
{
    const size_t nbatch = (n + batch_rows - 1) / batch_rows, f1 = f + 1;
    const size_t smem = (size_t)(BB_RC + BB_TA) * f1 * sizeof(double);
    double *dX = nullptr, *dy = nullptr, *dout = nullptr;
    auto run = [&]() -> int {
        HELR_TRY(helr_alloc(c, (void **)&dX, sizeof(double) * n * f));
        HELR_TRY(helr_alloc(c, (void **)&dy, sizeof(double) * n));
        HELR_TRY(helr_alloc(c, (void **)&dout, sizeof(double) * nbatch * g));
        HELR_CUDA(c, cudaMemcpyAsync(dX, X, sizeof(double) * n * f, cudaMemcpyHostToDevice, c->stream));
        HELR_CUDA(c, cudaMemcpyAsync(dy, y, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        HELR_CUDA(c, cudaMemsetAsync(dout, 0, sizeof(double) * nbatch * g, c->stream));  // padded columns
        HELR_CUDA(c, cudaFuncSetAttribute(k_bbar, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const dim3 grid((unsigned)((f1 + BB_TA - 1) / BB_TA), (unsigned)nbatch);
        HELR_LAUNCH(k_bbar<<<grid, 256, smem, c->stream>>>(dX, dy, n, (int)f, batch_rows, (int)g, dout));
        HELR_CUDA(c, cudaGetLastError());
        HELR_CUDA(c, cudaMemcpyAsync(out, dout, sizeof(double) * nbatch * g, cudaMemcpyDeviceToHost, c->stream));
        HELR_CUDA(c, cudaStreamSynchronize(c->stream));
        return HE_OK;
    };
    const int rc = run();
    helr_free(c, dX);
    helr_free(c, dy);
    helr_free(c, dout);
    return rc;
}

extern "C" int he_lr_bbar_batches(he_ctx *c, const double *X, const double *y, size_t n, size_t f, size_t batch_rows,
                                  size_t g, double *out)
{
    if (!c || !X || !y || !out || n == 0 || f == 0 || batch_rows == 0 || g < f + 1 || f + 1 > 256) return HE_EINVAL;
    return bbar_batches_dev(c, X, y, n, f, batch_rows, g, out);
}

// ------------------------------------------------------------------ job
struct he_lr_job {
    he_ctx *c;
    int mode;                   // HE_LR_FULL_BATCH or HE_LR_MINI_BATCH
    bool first_order;           // first-order NAG baseline: no Bbar, depth 6
    double poly[3];
    size_t n, f;
    int g, m, lg, lm, L;
    int nblocks, bpb, nbatch;
    size_t batch_rows;
    double scale0;
    uint64_t enc_seed;
    size_t ctw;                 // words per top-level ciphertext
    uint64_t *Z;                // [nblocks][2][L+1][N]
    std::vector<he_ct *> B;     // Enc(n Bbar) per mini-batch, or one for the full batch (none first-order)
    std::vector<double> inv_n;
    he_ct *W, *V;
    uint64_t *sig;              // masked sigmoid plaintexts (see SigPts), evaluation form
    double p1_scale;
    Eval ev;
    int chunk, chunk_max;
    uint64_t *buf;              // work ciphertexts
    uint64_t *T0, *T1, *T2, *T3, *T4, *acc;
    he_lr_stats st;
    double upd_total, iter_total;
    int iters_done;
    // per-iteration CUDA graph (optional)
    int graph;
    cudaStream_t gstream;
    cudaGraphExec_t gexec;
    // refresh by bootstrapping (optional; otherwise decrypt and re-encrypt)
    int boot;
    he_boot_params bp;
    uint64_t *boot_buf;         // [2][2][L+1][N] in, then out
};

static double f2(const he_lr_sched &s, double t) { return s.max - (s.max - s.min) * pow(t / s.T, s.power); }

// Algorithm 1: eta_t from the alpha recurrence started at alpha_0 = 0.01
static double nag_eta(int t)
{
    double a0 = 0.01, a1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * a0 * a0)), eta = 0;
    for (int k = 0; k <= t; k++) {
        eta = (1.0 - a0) / a1;
        a0 = a1;
        a1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * a0 * a0));
    }
    return eta;
}

static int encrypt_slots(he_ctx *c, const double *h_slots, int count, int level, double scale, uint64_t seed_base_kind,
                         uint64_t enc_seed, int first_index, uint64_t *dst, size_t dst_item)
{
    const size_t ns = c->nslots, N = c->n, nl = level + 1;
    const int step = 32;
    double *d = nullptr;
    uint64_t *pt = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&d, sizeof(double) * ns * step));
    HELR_TRY(helr_alloc(c, (void **)&pt, sizeof(uint64_t) * nl * N * step));
    for (int b0 = 0; b0 < count; b0 += step) {
        int cnt = std::min(step, count - b0);
        HELR_CUDA(c, cudaMemcpyAsync(d, h_slots + (size_t)b0 * ns, sizeof(double) * ns * cnt, cudaMemcpyHostToDevice, c->stream));
        HELR_TRY(helr_encode_dev(c, d, nullptr, cnt, ns, level, scale, pt, nl * N));
        for (int b = 0; b < cnt; b++)
            HELR_TRY(helr_encrypt_dev(c, pt + (size_t)b * nl * N, level, obj_seed(enc_seed, seed_base_kind, first_index + b0 + b),
                                      dst + (size_t)(b0 + b) * dst_item));
    }
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, d);
    helr_free(c, pt);
    return HE_OK;
}

// The three plaintexts of Steps 3/5 for row width g, at the levels and scales
// the circuit reaches from data blocks at scale z_scale and weights at scale
// w_scale (level L): p3 = -c3 M at level L-1, scale w_scale; p1 = -c1 M at level
// L-1 with the scale that rescales (M t) to the scale of the cube; p0 = (1 - c0) M
// at level L-3 and the cube's scale.  M has ones in column 0 of every row.
// *out holds [p3 (L limbs) | p1 (L limbs) | p0 (L-2 limbs)] x N words.
struct SigPts {
    const uint64_t *p3, *p1, *p0;
};
static SigPts sig_pts(const uint64_t *buf, int L, size_t N)
{
    return SigPts{buf, buf + (size_t)L * N, buf + 2 * (size_t)L * N};
}
static int make_sigmoid_pts(he_ctx *c, int L, int g, double z_scale, double w_scale, const double poly[3], uint64_t **out,
                            double *p1_scale)
{
    const size_t N = c->n, ns = c->nslots;
    const double q = (double)c->q[L], q1 = (double)c->q[L - 1], q2 = (double)c->q[L - 2];
    const double t_scale = z_scale * w_scale / q;        // Step 1
    const double sq_scale = t_scale * t_scale / q1;      // t^2
    const double c3_scale = t_scale * w_scale / q1;      // (-c3 M) t
    const double s_scale = sq_scale * c3_scale / q2;     // the cube, and s
    *p1_scale = s_scale * q1 / t_scale;
    std::vector<double> v(3 * ns, 0.0);
    for (size_t i = 0; i < ns; i += g) {
        v[i] = -poly[2];
        v[ns + i] = -poly[1];
        v[2 * ns + i] = 1.0 - poly[0];
    }
    double *d = nullptr;
    uint64_t *buf = nullptr;
    auto run = [&]() -> int {
        HELR_TRY(helr_alloc(c, (void **)&d, sizeof(double) * 3 * ns));
        HELR_TRY(helr_alloc(c, (void **)&buf, sizeof(uint64_t) * (3 * (size_t)L - 2) * N));
        HELR_CUDA(c, cudaMemcpyAsync(d, v.data(), sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, c->stream));
        const SigPts p = sig_pts(buf, L, N);
        HELR_TRY(helr_encode_dev(c, d, nullptr, 1, 0, L - 1, w_scale, const_cast<uint64_t *>(p.p3), 0));
        HELR_TRY(helr_encode_dev(c, d + ns, nullptr, 1, 0, L - 1, *p1_scale, const_cast<uint64_t *>(p.p1), 0));
        HELR_TRY(helr_encode_dev(c, d + 2 * ns, nullptr, 1, 0, L - 3, s_scale, const_cast<uint64_t *>(p.p0), 0));
        HELR_CUDA(c, cudaStreamSynchronize(c->stream));
        return HE_OK;
    };
    const int rc = run();
    helr_free(c, d);
    if (rc) {
        helr_free(c, buf);
        return rc;
    }
    *out = buf;
    return HE_OK;
}

extern "C" int he_lr_job_free(he_lr_job *j)
{
    if (!j) return HE_EINVAL;
    he_ctx *c = j->c;
    cudaStreamSynchronize(c->stream);
    helr_free(c, j->Z);
    for (auto *b : j->B) he_ct_free(b);
    if (j->W) he_ct_free(j->W);
    if (j->V) he_ct_free(j->V);
    helr_free(c, j->sig);
    helr_free(c, j->buf);
    helr_free(c, j->boot_buf);
    ev_free(&j->ev);
    cudaStreamSynchronize(c->stream);
    if (j->gexec) cudaGraphExecDestroy(j->gexec);
    if (j->gstream) cudaStreamDestroy(j->gstream);
    delete j;
    return HE_OK;
}

extern "C" int he_lr_job_create(he_ctx *c, const double *X, const double *y, size_t n, size_t f, int mode,
                                size_t batch_rows, int poly, double log_scale, uint64_t enc_seed, uint64_t key_seed,
                                int batch_blocks, he_lr_job **out)
{
    const bool fo = (mode & HE_LR_FIRST_ORDER) != 0;
    mode &= ~HE_LR_FIRST_ORDER;
    if (!c || !X || !y || !out || n == 0 || f == 0 || (mode != HE_LR_FULL_BATCH && mode != HE_LR_MINI_BATCH) ||
        (poly != HE_LR_G8 && poly != HE_LR_G16) || !(log_scale > 0 && log_scale < 62))
        return HE_EINVAL;
    *out = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    // fresh ciphertexts sit at the iteration depth: the iteration ends at level 0
    // and any primes of the chain above it stay unused
    const int L = fo ? ITER_DEPTH_FO : ITER_DEPTH;
    if (c->nq - 1 < L) return helr_fail(c, HE_ELEVEL, "the iteration needs %d levels (n_q >= %d)", L, L + 1);
    int g = 1;
    while ((size_t)g < f + 1) g <<= 1;
    if (g > c->nslots) return helr_fail(c, HE_EINVAL, "too many features for N/2 slots");
    const int m = c->nslots / g;
    if (batch_rows == 0) batch_rows = 1024;
    if (batch_rows % m) return helr_fail(c, HE_EINVAL, "batch_rows must be a multiple of the %d rows per block", m);

    he_lr_job *j = new he_lr_job();
    j->c = c;
    j->mode = mode;
    j->first_order = fo;
    memcpy(j->poly, poly == HE_LR_G8 ? G8 : G16, sizeof j->poly);
    j->n = n;
    j->f = f;
    j->g = g;
    j->m = m;
    j->lg = __builtin_ctz(g);
    j->lm = __builtin_ctz(m);
    j->L = L;
    j->nblocks = (int)((n + m - 1) / m);
    j->batch_rows = batch_rows;
    j->bpb = (int)(batch_rows / m);
    j->nbatch = (int)((n + batch_rows - 1) / batch_rows);
    j->scale0 = ldexp(1.0, 0) * pow(2.0, log_scale);
    j->enc_seed = enc_seed;
    const size_t N = c->n, ns = c->nslots;
    j->ctw = 2 * (size_t)(L + 1) * N;
    int rc = HE_OK;
#define JTRY(x)                       \
    do {                              \
        rc = (x);                     \
        if (rc) {                     \
            he_lr_job_free(j);        \
            return rc;                \
        }                             \
    } while (0)

    // keys for the rotations of Steps 2, 4 and 7 (hoisted groups)
    std::vector<int64_t> rots;
    int64_t amt[HELR_MAX_HOIST];
    const int rho = c->rot_radix_log;
    for (int e = 0; e < j->lg; e += rho) {
        const int n = (1 << rot_group_amounts(e, j->lg, rho, 1, amt)) - 1;
        for (int k = 0; k < n; k++) rots.push_back(amt[k]), rots.push_back(-amt[k]);
    }
    for (int e = 0; e < j->lm; e += rho) {
        const int n = (1 << rot_group_amounts(e, j->lm, rho, g, amt)) - 1;
        rots.insert(rots.end(), amt, amt + n);
    }
    JTRY(he_keygen(c, key_seed, rots.data(), rots.size()));

    // Step 1: Z = y [1 | X], blocks of m rows x g columns, row-major in the slots
    std::vector<double> slots((size_t)j->nblocks * ns, 0.0);
    for (size_t r = 0; r < n; r++) {
        double *row = &slots[(r / m) * ns + (r % m) * g];
        row[0] = y[r];
        for (size_t k = 0; k < f; k++) row[k + 1] = y[r] * X[r * f + k];
    }
    // Bbar per mini-batch (threads over batches), full batch by 1 / sum_k (1 / Bbar_k);
    // the first-order baseline needs only the 1/n scalars
    // (on the device for up to 256 columns; wider data on the host threads,
    // with the same arithmetic)
    std::vector<double> bk(fo ? 0 : (size_t)j->nbatch * g);
    if (!fo && f + 1 <= 256) {
        JTRY(bbar_batches_dev(c, X, y, n, f, batch_rows, g, bk.data()));
    } else if (!fo) {
        unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nth; t++)
            th.emplace_back([&, t]() {
                for (int k = (int)t; k < j->nbatch; k += (int)nth) {
                    size_t r0 = (size_t)k * batch_rows, rows = std::min(batch_rows, n - r0);
                    bbar_rows(X, y, f, r0, rows, g, &bk[(size_t)k * g]);
                }
            });
        for (auto &x : th) x.join();
    }
    std::vector<std::vector<double>> bvec;
    if (fo) {
        if (mode == HE_LR_FULL_BATCH)
            j->inv_n.push_back(1.0 / (double)n);
        else
            for (int k = 0; k < j->nbatch; k++)
                j->inv_n.push_back(1.0 / (double)std::min(batch_rows, n - (size_t)k * batch_rows));
    } else if (mode == HE_LR_FULL_BATCH) {
        std::vector<double> full(g, 0.0);
        for (size_t a = 0; a <= f; a++) {
            double s = 0.0;
            for (int k = 0; k < j->nbatch; k++) s += 1.0 / bk[(size_t)k * g + a];
            full[a] = 1.0 / s;
        }
        std::vector<double> v(ns);
        for (size_t i = 0; i < ns; i++) v[i] = (double)n * full[i % g];
        bvec.push_back(v);
        j->inv_n.push_back(1.0 / (double)n);
    } else {
        for (int k = 0; k < j->nbatch; k++) {
            double nk = (double)std::min(batch_rows, n - (size_t)k * batch_rows);
            std::vector<double> v(ns);
            for (size_t i = 0; i < ns; i++) v[i] = nk * bk[(size_t)k * g + (i % g)];
            bvec.push_back(v);
            j->inv_n.push_back(1.0 / nk);
        }
    }
    // Step 2: encrypt blocks, n Bbar, W0 = V0 = 0
    JTRY(helr_alloc(c, (void **)&j->Z, sizeof(uint64_t) * j->ctw * j->nblocks));
    JTRY(encrypt_slots(c, slots.data(), j->nblocks, L, j->scale0, 1, enc_seed, 0, j->Z, j->ctw));
    slots.clear();
    slots.shrink_to_fit();
    for (size_t k = 0; k < bvec.size(); k++) {
        he_ct *ct = nullptr;
        JTRY(helr_new_ct(c, L, j->scale0, &ct));
        j->B.push_back(ct);
        JTRY(encrypt_slots(c, bvec[k].data(), 1, L, j->scale0, 2, enc_seed, (int)k, ct->d, j->ctw));
    }
    std::vector<double> zero(ns, 0.0);
    JTRY(helr_new_ct(c, L, j->scale0, &j->W));
    JTRY(encrypt_slots(c, zero.data(), 1, L, j->scale0, 3, enc_seed, 0, j->W->d, j->ctw));
    JTRY(helr_new_ct(c, L, j->scale0, &j->V));
    JTRY(encrypt_slots(c, zero.data(), 1, L, j->scale0, 4, enc_seed, 0, j->V->d, j->ctw));
    // Steps 3/5: the masked plaintexts of the sigmoid polynomial
    JTRY(make_sigmoid_pts(c, L, g, j->scale0, j->scale0, j->poly, &j->sig, &j->p1_scale));
    // work buffers: chunk of blocks per launch
    int chunk = batch_blocks > 0 ? batch_blocks : 256;  // tuned on GB300 at N = 2^16
    chunk = std::min(chunk, mode == HE_LR_FULL_BATCH ? j->nblocks : j->bpb);
    j->chunk = std::max(1, chunk);
    j->chunk_max = j->chunk;
    JTRY(ev_init(c, &j->ev, j->chunk, L));
    JTRY(helr_alloc(c, (void **)&j->buf, sizeof(uint64_t) * j->ctw * (5 * (size_t)j->chunk + 3)));
    j->T0 = j->buf;
    j->T1 = j->T0 + j->ctw * j->chunk;
    j->T2 = j->T1 + j->ctw * j->chunk;
    j->T3 = j->T2 + j->ctw * j->chunk;
    j->T4 = j->T3 + j->ctw * j->chunk;
    j->acc = j->T4 + j->ctw * j->chunk;
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    j->st.sec_setup = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    j->st.n_blocks = j->nblocks;
    j->st.g = g;
    j->st.m = m;
    *out = j;
    return HE_OK;
#undef JTRY
}

// cMul by c at the constant scale that makes the rescaled result carry `target`
static int cmul_to(Eval *ev, const CtB &a, double cval, double target, CtB &tmp, CtB &out)
{
    he_ctx *c = ev->c;
    double q = (double)c->q[a.level];
    double S = (target * q) / a.scale;
    HELR_TRY(ev_cmul_int(ev, a, round_half_away(cval * S), a.scale * S, tmp));
    HELR_TRY(ev_rescale(ev, tmp, out));
    out.scale = target;
    return HE_OK;
}

// Work buffers shared by the circuit functions: five ciphertext arrays of `cap`
// top-level ciphertexts each.
struct WorkSet {
    Eval *ev;
    uint64_t *T[5];
    size_t ctw;
    int L;
    double scale0;
    const double *poly;
};

// A run of data blocks that share W, the row width g and its masked sigmoid
// plaintexts (p1 at scale p1_scale).
struct Seg {
    int start, count, lg;
    const uint64_t *W;
    SigPts sig;
    double p1_scale;
};

int rot_group_amounts(int e, int nbits, int rho, int64_t step, int64_t *out)
{
    const int w = std::min(rho, nbits - e);
    for (int m = 1; m < (1 << w); m++) out[m - 1] = step * ((int64_t)m << e);
    return w;
}

// Group e of a rotate-and-sum (Sec. 2.2 SumColVec and its replication), as one
// hoisted rotation sum per run of items that share the group's width: an item
// of row width 2^lg takes width min(rho, lg - e) (segments are ordered by
// decreasing lg, so equal widths are contiguous); items with lg <= e are
// carried over unchanged.  Ping-pong: the result ends in Bt, R takes the input.
static int rot_group(const WorkSet &ws, CtB &Bt, CtB &R, int e, int64_t step, const Seg *segs, int nseg, int cnt)
{
    Eval *ev = ws.ev;
    const int rho = ev->c->rot_radix_log;
    auto width = [&](int i) { return std::max(0, std::min(rho, segs[i].lg - e)); };
    for (int i = 0; i < nseg;) {
        const int w = width(i);
        int k = i + 1;
        while (k < nseg && width(k) == w) k++;
        const int start = segs[i].start, end = segs[k - 1].start + segs[k - 1].count;
        CtB a = Bt, o = R;
        a.d = Bt.d + (size_t)start * ws.ctw;
        a.batch = end - start;
        o.d = R.d + (size_t)start * ws.ctw;
        if (w > 0) {
            int64_t rots[HELR_MAX_HOIST];
            const int n = (1 << rot_group_amounts(e, segs[i].lg, rho, step, rots)) - 1;
            HELR_TRY(ev_rotsum(ev, a, rots, n, o));
        } else {
            HELR_TRY(ev_moddrop(ev, a, a.level, o));
        }
        i = k;
    }
    R.level = Bt.level;
    R.scale = Bt.scale;
    R.batch = cnt;
    std::swap(Bt, R);
    return HE_OK;
}

// Steps 1-6 on `cnt` blocks at Z (item stride ctw) described by segments;
// result (level L-4) in g_out (buffer T2)
static int block_grads_seg(const WorkSet &ws, const uint64_t *Z, int cnt, const Seg *segs, int nseg, double w_scale,
                           CtB &g_out)
{
    Eval *ev = ws.ev;
    const int L = ws.L;
    const size_t w = ws.ctw;
    CtB Zc{const_cast<uint64_t *>(Z), cnt, L, ws.scale0, w};
    CtB A{ws.T[0], cnt, 0, 0, w}, Bt{ws.T[1], cnt, 0, 0, w}, R{ws.T[2], cnt, 0, 0, w};
    std::vector<const uint64_t *> wp(nseg);
    std::vector<int> st(nseg), ct(nseg);
    int lgmax = 0;
    for (int i = 0; i < nseg; i++) {
        wp[i] = segs[i].W, st[i] = segs[i].start, ct[i] = segs[i].count;
        lgmax = std::max(lgmax, segs[i].lg);
    }
    auto slice = [&](const CtB &x, int i) {
        CtB y = x;
        y.d = x.d + (size_t)segs[i].start * w;
        y.batch = segs[i].count;
        return y;
    };
    // per segment: out = Rescale-ready product of x with that segment's plaintext
    auto ptmul_segs = [&](const CtB &x, const uint64_t *SigPts::*which, double scale, CtB &out) -> int {
        for (int i = 0; i < nseg; i++) {
            CtB y = slice(out, i);
            HELR_TRY(ev_ptmul(ev, slice(x, i), segs[i].sig.*which, scale, y));
        }
        out.level = x.level;
        out.scale = x.scale * scale;
        out.batch = cnt;
        return HE_OK;
    };
    // 1
    HELR_TRY(ev_mul_relin_seg(ev, Zc, wp.data(), st.data(), ct.data(), nseg, w_scale, A));
    HELR_TRY(ev_rescale(ev, A, Bt));
    // 2: row sums, t += sum_m Rot(t, m 2^e) per hoisted group, ping-pong between T1 and T2
    const int rho = ev->c->rot_radix_log;
    for (int e = 0; e < lgmax; e += rho) HELR_TRY(rot_group(ws, Bt, R, e, 1, segs, nseg, cnt));
    const CtB t = Bt;  // level L-1; R is the other of T1 / T2
    // 3/5: s = (1 - c0) M - c1 (M t) - c3 t^2 (M t)
    CtB sq{ws.T[3], cnt, 0, 0, w}, c3{ws.T[4], cnt, 0, 0, w}, cube{ws.T[0], cnt, 0, 0, w};
    HELR_TRY(ev_mul_relin(ev, t, t, A));
    HELR_TRY(ev_rescale(ev, A, sq));
    HELR_TRY(ptmul_segs(t, &SigPts::p3, ws.scale0, A));
    HELR_TRY(ev_rescale(ev, A, c3));
    HELR_TRY(ev_mul_relin(ev, sq, c3, R));
    HELR_TRY(ev_rescale(ev, R, cube));
    CtB lin{ws.T[3], cnt, 0, 0, w}, lind{ws.T[4], cnt, 0, 0, w};
    HELR_TRY(ptmul_segs(t, &SigPts::p1, segs[0].p1_scale, R));
    HELR_TRY(ev_rescale(ev, R, lin));
    lin.scale = cube.scale;  // p1's scale was chosen for this
    HELR_TRY(ev_moddrop(ev, lin, cube.level, lind));
    CtB s{t.d, cnt, 0, 0, w};
    HELR_TRY(ev_add(ev, cube, lind, s, 0));
    for (int i = 0; i < nseg; i++) {
        CtB y = slice(s, i);
        HELR_TRY(ev_ptadd(ev, y, segs[i].sig.p0));
    }
    // 4: s += sum_m Rot(s, -m 2^e) per hoisted group, ping-pong between T1 and T2
    Bt = s;
    R.d = t.d == ws.T[1] ? ws.T[2] : ws.T[1];
    for (int e = 0; e < lgmax; e += rho) HELR_TRY(rot_group(ws, Bt, R, e, -1, segs, nseg, cnt));
    if (Bt.d != ws.T[1]) {
        CtB t1{ws.T[1], cnt, 0, 0, w};
        HELR_TRY(ev_moddrop(ev, Bt, Bt.level, t1));
        Bt = t1;
    }
    // 6
    CtB zd{ws.T[3], cnt, 0, 0, w};
    HELR_TRY(ev_moddrop(ev, Zc, Bt.level, zd));
    HELR_TRY(ev_mul_relin(ev, Bt, zd, A));
    g_out.d = ws.T[2];
    g_out.item = w;
    HELR_TRY(ev_rescale(ev, A, g_out));
    return HE_OK;
}

static WorkSet job_ws(he_lr_job *j)
{
    return WorkSet{&j->ev, {j->T0, j->T1, j->T2, j->T3, j->T4}, j->ctw, j->L, j->scale0, j->poly};
}

// Steps 1-6 on `cnt` consecutive blocks of one job
static int block_grads(he_lr_job *j, const uint64_t *Z, int cnt, const CtB &W, CtB &g_out)
{
    Seg sg{0, cnt, j->lg, W.d, sig_pts(j->sig, j->L, j->c->n), j->p1_scale};
    return block_grads_seg(job_ws(j), Z, cnt, &sg, 1, W.scale, g_out);
}

// Steps 7-9 on the accumulated gradient of one job (row width g = 2^lg... column
// sums over m = 2^lm rows); W', V' at level L-7 into Wn, Vn
static int finish_ws(const WorkSet &ws, CtB acc, const he_ct *Bct, const he_ct *W, const he_ct *V, int g, int lm, double alpha,
                     double eta, double inv_n, CtB &Wn, CtB &Vn)
{
    Eval *ev = ws.ev;
    const size_t w = ws.ctw;
    CtB R{ws.T[0], 1, 0, 0, w}, A{ws.T[1], 1, 0, 0, w}, Bd{ws.T[2], 1, 0, 0, w};
    // 7: column sums, acc += sum_m Rot(acc, g m 2^e) per hoisted group, ping-pong between acc and R
    const int rho = ev->c->rot_radix_log;
    for (int e = 0; e < lm; e += rho) {
        int64_t rots[HELR_MAX_HOIST];
        const int n = (1 << rot_group_amounts(e, lm, rho, g, rots)) - 1;
        HELR_TRY(ev_rotsum(ev, acc, rots, n, R));
        std::swap(acc, R);
    }
    // 8: n Bbar_c g_c; the first-order baseline (no Bbar) takes g_c itself
    CtB nG{ws.T[3], 1, 0, 0, w};
    if (Bct) {
        CtB Bv{Bct->d, 1, Bct->level, Bct->scale, 0};
        HELR_TRY(ev_moddrop(ev, Bv, acc.level, Bd));
        HELR_TRY(ev_mul_relin(ev, acc, Bd, A));
        HELR_TRY(ev_rescale(ev, A, nG));
    } else {
        HELR_TRY(ev_moddrop(ev, acc, acc.level, nG));  // a copy out of the buffers Step 9 reuses
    }
    // 9
    const int lv = nG.level;
    const double tgt = W->scale;
    CtB Wv{W->d, 1, W->level, W->scale, 0}, Vv{V->d, 1, V->level, V->scale, 0};
    CtB G{ws.T[4], 1, 0, 0, w}, Wd{ws.T[0], 1, 0, 0, w};
    HELR_TRY(cmul_to(ev, nG, alpha * inv_n, tgt, A, G));
    HELR_TRY(ev_moddrop(ev, Wv, lv - 1, Wd));
    HELR_TRY(ev_add(ev, Wd, G, Vn, 0));
    CtB x1{ws.T[4], 1, 0, 0, w}, x2{ws.T[0], 1, 0, 0, w};
    HELR_TRY(ev_moddrop(ev, Wv, lv, Bd));
    HELR_TRY(cmul_to(ev, Bd, 1.0 - eta, tgt, A, x1));
    HELR_TRY(ev_moddrop(ev, Vv, lv, Bd));
    HELR_TRY(cmul_to(ev, Bd, eta, tgt, A, x2));
    HELR_TRY(ev_add(ev, x1, x2, x1, 0));
    HELR_TRY(cmul_to(ev, nG, (1.0 - eta) * alpha * inv_n, tgt, A, x2));
    HELR_TRY(ev_add(ev, x1, x2, Wn, 0));
    return HE_OK;
}

static int finish(he_lr_job *j, CtB acc, const he_ct *Bct, double alpha, double eta, double inv_n, CtB &Wn, CtB &Vn)
{
    return finish_ws(job_ws(j), acc, Bct, j->W, j->V, j->g, j->lm, alpha, eta, inv_n, Wn, Vn);
}

// decrypt, keep the real part of every slot, re-encode at new_level, encrypt
static int refresh_dev(he_ctx *c, const uint64_t *ct, int level, double scale, int new_level, double new_scale,
                       uint64_t seed, uint64_t *dst)
{
    const size_t N = c->n, ns = c->nslots;
    uint64_t *pt = nullptr, *pt2 = nullptr;
    double *z = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&pt, sizeof(uint64_t) * (level + 1) * N));
    HELR_TRY(helr_alloc(c, (void **)&pt2, sizeof(uint64_t) * (new_level + 1) * N));
    HELR_TRY(helr_alloc(c, (void **)&z, sizeof(double) * 2 * ns));
    HELR_TRY(helr_decrypt_dev(c, ct, level, pt));
    HELR_TRY(helr_decode_dev(c, pt, scale, z, z + ns));
    HELR_TRY(helr_encode_dev(c, z, nullptr, 1, 0, new_level, new_scale, pt2, 0));
    HELR_TRY(helr_encrypt_dev(c, pt2, new_level, seed, dst));
    helr_free(c, pt);
    helr_free(c, pt2);
    helr_free(c, z);
    return HE_OK;
}

// Steps 1-9 of iteration t into Wn, Vn (device work only: no allocation, no synchronisation)
static int job_update(he_lr_job *j, int t, const he_lr_sched &sched, CtB &Wn, CtB &Vn)
{
    const double alpha = f2(sched, (double)t), eta = nag_eta(t);
    int b0 = 0, b1 = j->nblocks, k = 0;
    if (j->mode == HE_LR_MINI_BATCH) {
        k = t % j->nbatch;
        b0 = k * j->bpb;
        b1 = std::min(j->nblocks, b0 + j->bpb);
    }
    j->ev.keyswitches = 0;
    const CtB W{j->W->d, 1, j->L, j->W->scale, 0};
    double gscale = 0;
    int glevel = 0;
    for (int b = b0; b < b1; b += j->chunk) {
        int cnt = std::min(j->chunk, b1 - b);
        CtB g{};
        HELR_TRY(block_grads(j, j->Z + (size_t)b * j->ctw, cnt, W, g));
        HELR_TRY(ev_sum_items(&j->ev, g, j->acc, b != b0));
        gscale = g.scale;
        glevel = g.level;
    }
    CtB acc{j->acc, 1, glevel, gscale, 0};
    Wn = CtB{j->acc + j->ctw, 1, 0, 0, 0};
    Vn = CtB{j->acc + 2 * j->ctw, 1, 0, 0, 0};
    return finish(j, acc, j->first_order ? nullptr : j->B[k], alpha, eta, j->inv_n[k], Wn, Vn);
}

// Steps 1-9 recorded into a CUDA graph on the job's stream and launched as one unit
static int job_update_graph(he_lr_job *j, int t, const he_lr_sched &sched, CtB &Wn, CtB &Vn)
{
    he_ctx *c = j->c;
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaStream_t saved = c->stream;
    const int prof_on = c->prof.on;
    c->stream = j->gstream;
    c->prof.on = 0;  // no timing events inside the graph
    cudaGraph_t g = nullptr;
    int rc = HE_OK;
    cudaError_t e = cudaStreamBeginCapture(j->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = job_update(j, t, sched, Wn, Vn);
        e = cudaStreamEndCapture(j->gstream, &g);
    }
    c->stream = saved;
    c->prof.on = prof_on;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return helr_fail(c, HE_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    bool updated = false;
    if (j->gexec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(j->gexec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(j->gexec);
            j->gexec = nullptr;
        }
    }
    if (!j->gexec) e = cudaGraphInstantiate(&j->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return helr_fail(c, HE_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    HELR_CUDA(c, cudaGraphLaunch(j->gexec, j->gstream));
    HELR_CUDA(c, cudaStreamSynchronize(j->gstream));
    return HE_OK;
}

extern "C" int he_lr_job_set_graph(he_lr_job *j, int on)
{
    if (!j) return HE_EINVAL;
    if (on && !j->gstream) HELR_CUDA(j->c, cudaStreamCreateWithFlags(&j->gstream, cudaStreamNonBlocking));
    j->graph = on ? 1 : 0;
    return HE_OK;
}

// The refresh of W' and V' (Sec. 4.3 Step 7): one bootstrap over both when the
// job refreshes by bootstrapping, else decryption and re-encryption with the
// seeds of iteration t.
static int job_refresh(he_lr_job *j, int t, const CtB &Wn, const CtB &Vn)
{
    he_ctx *c = j->c;
    if (!j->boot) {
        HELR_TRY(refresh_dev(c, Wn.d, Wn.level, Wn.scale, j->L, j->scale0, obj_seed(j->enc_seed, 5, t), j->W->d));
        HELR_TRY(refresh_dev(c, Vn.d, Vn.level, Vn.scale, j->L, j->scale0, obj_seed(j->enc_seed, 6, t), j->V->d));
        j->W->scale = j->scale0;
        j->V->scale = j->scale0;
        return HE_OK;
    }
    if (Wn.level != 0 || Vn.level != 0) return helr_fail(c, HE_EINTERNAL, "the iteration should end at level 0");
    const size_t N = c->n, win = 2 * N, wout = 2 * (size_t)(j->L + 1) * N;
    HELR_CUDA(c, cudaMemcpyAsync(j->boot_buf, Wn.d, win * 8, cudaMemcpyDeviceToDevice, c->stream));
    HELR_CUDA(c, cudaMemcpyAsync(j->boot_buf + win, Vn.d, win * 8, cudaMemcpyDeviceToDevice, c->stream));
    uint64_t *out = j->boot_buf + 2 * win;
    HELR_TRY(he_bootstrap_batch(c, j->boot_buf, Wn.level, out, 2, &j->bp));
    HELR_CUDA(c, cudaMemcpyAsync(j->W->d, out, wout * 8, cudaMemcpyDeviceToDevice, c->stream));
    HELR_CUDA(c, cudaMemcpyAsync(j->V->d, out + wout, wout * 8, cudaMemcpyDeviceToDevice, c->stream));
    j->W->scale = j->V->scale = j->scale0;
    return HE_OK;
}

extern "C" int he_lr_job_set_refresh(he_lr_job *j, const he_boot_params *p)
{
    if (!j) return HE_EINVAL;
    he_ctx *c = j->c;
    if (!p) {
        j->boot = 0;
        return HE_OK;
    }
    if (p->level_out != j->L || p->scale_out != j->scale0 || p->slots != j->g)
        return helr_fail(c, HE_EINVAL, "the bootstrap must return slots of period g = %d at level %d, scale 2^%g", j->g,
                         j->L, log2(j->scale0));
    size_t nr = 0;
    HELR_TRY(he_boot_keys(c, p, nullptr, 0, &nr));
    std::vector<int64_t> rots(nr);
    HELR_TRY(he_boot_keys(c, p, rots.data(), nr, &nr));
    HELR_TRY(he_keygen(c, c->key_seed, rots.data(), nr));
    const uint64_t conj = 2ull * c->n - 1;
    HELR_TRY(he_keygen_galois(c, &conj, 1));
    if (!j->boot_buf) {
        const size_t N = c->n;
        HELR_TRY(helr_alloc(c, (void **)&j->boot_buf, 8 * (4 * (size_t)(j->L + 1) * N + 4 * N)));
    }
    j->bp = *p;
    j->boot = 1;
    return HE_OK;
}

extern "C" int he_lr_job_step(he_lr_job *j, int t, he_lr_sched sched)
{
    if (!j || t < 0 || !(sched.T > 0)) return HE_EINVAL;
    he_ctx *c = j->c;
    auto t0 = std::chrono::steady_clock::now();
    CtB Wn{}, Vn{};
    if (j->graph) HELR_TRY(job_update_graph(j, t, sched, Wn, Vn));
    else HELR_TRY(job_update(j, t, sched, Wn, Vn));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    auto t1 = std::chrono::steady_clock::now();
    // Step 7: refresh W and V
    HELR_TRY(job_refresh(j, t, Wn, Vn));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    auto t2 = std::chrono::steady_clock::now();
    j->upd_total += std::chrono::duration<double>(t1 - t0).count();
    j->iter_total += std::chrono::duration<double>(t2 - t0).count();
    j->iters_done++;
    j->st.keyswitches = j->ev.keyswitches;
    j->st.sec_update_avg = j->upd_total / j->iters_done;
    j->st.sec_iter_avg = j->iter_total / j->iters_done;
    return HE_OK;
}

extern "C" int he_lr_job_set_batch(he_lr_job *j, int b)
{
    if (!j || b < 1 || b > j->chunk_max) return HE_EINVAL;
    j->chunk = b;
    return HE_OK;
}

extern "C" int he_lr_job_step_io(he_lr_job *j, int t, he_lr_sched sched, const uint64_t *in, uint64_t *out)
{
    if (!j) return HE_EINVAL;
    he_ctx *c = j->c;
    const size_t nl = j->L + 1, lw = 2 * nl;  // limbs per ciphertext
    if (in) {
        HELR_CUDA(c, cudaMemcpyAsync(j->W->d, in, j->ctw * 8, cudaMemcpyHostToDevice, c->stream));
        HELR_CUDA(c, cudaMemcpyAsync(j->V->d, in + j->ctw, j->ctw * 8, cudaMemcpyHostToDevice, c->stream));
        HELR_TRY(helr_ntt_fwd(c, j->W->d, lw, limbmap_ct(j->L), c->stream));
        HELR_TRY(helr_ntt_fwd(c, j->V->d, lw, limbmap_ct(j->L), c->stream));
        j->W->scale = j->V->scale = j->scale0;
    }
    HELR_TRY(he_lr_job_step(j, t, sched));
    if (out) {
        uint64_t *tmp = j->acc;  // free after the step
        HELR_TRY(helr_ntt_inv_oop(c, j->W->d, tmp, lw, limbmap_ct(j->L), c->stream));
        HELR_CUDA(c, cudaMemcpyAsync(out, tmp, j->ctw * 8, cudaMemcpyDeviceToHost, c->stream));
        HELR_TRY(helr_ntt_inv_oop(c, j->V->d, tmp, lw, limbmap_ct(j->L), c->stream));
        HELR_CUDA(c, cudaMemcpyAsync(out + j->ctw, tmp, j->ctw * 8, cudaMemcpyDeviceToHost, c->stream));
        HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return HE_OK;
}

extern "C" int he_lr_job_weights(he_lr_job *j, int row, double *w, size_t len)
{
    if (!j || !w || row < 0 || row >= j->m || len < (size_t)j->g) return HE_EINVAL;
    he_ctx *c = j->c;
    he_pt *pt = nullptr;
    HELR_TRY(he_decrypt(c, j->W, &pt));
    std::vector<double> re(c->nslots);
    int rc = he_decode(c, pt, re.data(), nullptr, c->nslots);
    he_pt_free(pt);
    if (rc) return rc;
    memcpy(w, &re[(size_t)row * j->g], sizeof(double) * j->g);
    return HE_OK;
}

extern "C" int he_lr_job_state(he_lr_job *j, const he_ct **W, const he_ct **V)
{
    if (!j) return HE_EINVAL;
    if (W) *W = j->W;
    if (V) *V = j->V;
    return HE_OK;
}

extern "C" int he_lr_job_input(he_lr_job *j, int kind, int index, he_ct **out)
{
    if (!j || !out) return HE_EINVAL;
    he_ctx *c = j->c;
    const uint64_t *src;
    double scale = j->scale0;
    if (kind == 0 && index >= 0 && index < j->nblocks) src = j->Z + (size_t)index * j->ctw;
    else if (kind == 1 && index >= 0 && index < (int)j->B.size()) src = j->B[index]->d;
    else return HE_EINVAL;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, j->L, scale, &o));
    HELR_CUDA(c, cudaMemcpyAsync(o->d, src, sizeof(uint64_t) * j->ctw, cudaMemcpyDeviceToDevice, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = o;
    return HE_OK;
}

extern "C" int he_lr_job_block_grad(he_lr_job *j, int block, he_ct **out)
{
    if (!j || !out || block < 0 || block >= j->nblocks) return HE_EINVAL;
    he_ctx *c = j->c;
    const CtB W{j->W->d, 1, j->L, j->W->scale, 0};
    // the chunk of the step's launch sequence that holds `block`
    int b0 = 0, b1 = j->nblocks;
    if (j->mode == HE_LR_MINI_BATCH) {
        b0 = (block / j->bpb) * j->bpb;
        b1 = std::min(j->nblocks, b0 + j->bpb);
    }
    int start = b0 + ((block - b0) / j->chunk) * j->chunk;
    int cnt = std::min(j->chunk, b1 - start);
    CtB g{};
    HELR_TRY(block_grads(j, j->Z + (size_t)start * j->ctw, cnt, W, g));
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, g.level, g.scale, &o));
    HELR_CUDA(c, cudaMemcpyAsync(o->d, g.d + (size_t)(block - start) * g.item, sizeof(uint64_t) * 2 * (g.level + 1) * c->n,
                                 cudaMemcpyDeviceToDevice, c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = o;
    return HE_OK;
}

extern "C" int he_lr_job_info(const he_lr_job *j, he_lr_stats *st)
{
    if (!j || !st) return HE_EINVAL;
    *st = j->st;
    return HE_OK;
}

extern "C" int he_lr_train(he_ctx *c, const double *X, const double *y, size_t n, size_t f, int iters, he_lr_sched sched,
                           int mode, size_t batch_rows, int poly, uint64_t enc_seed, uint64_t key_seed, double *w_out,
                           size_t w_len, he_lr_stats *stats)
{
    if (!c || iters < 0 || !w_out) return HE_EINVAL;
    he_lr_job *j = nullptr;
    HELR_TRY(he_lr_job_create(c, X, y, n, f, mode, batch_rows, poly, 40.0, enc_seed, key_seed, 0, &j));
    int rc = HE_OK;
    for (int t = 0; t < iters && !rc; t++) rc = he_lr_job_step(j, t, sched);
    if (!rc) rc = he_lr_job_weights(j, 0, w_out, w_len);
    if (!rc && stats) rc = he_lr_job_info(j, stats);
    he_lr_job_free(j);
    return rc;
}

// ------------------------------------------------------------------ cloud-only iteration / refresh
extern "C" int he_lr_iteration(he_ctx *c, he_ct *const *Z, size_t nb, const he_ct *B, const he_ct *W, const he_ct *V, int g,
                               int m, double alpha, double eta, double inv_n, const double poly[3], he_ct **W_out,
                               he_ct **V_out)
{
    if (!c || !Z || !nb || !W || !V || !poly || !W_out || !V_out || g * m != c->nslots || (g & (g - 1)) || g < 1)
        return HE_EINVAL;
    const int L = W->level;
    const int depth = B ? ITER_DEPTH : ITER_DEPTH_FO;  // no B: the first-order baseline
    if (L < depth) return helr_fail(c, HE_ELEVEL, "the iteration needs %d levels", depth);
    for (size_t i = 0; i < nb; i++)
        if (Z[i]->level != L) return helr_fail(c, HE_ELEVEL, "data blocks must share the level of W");
    // a temporary job around the caller's ciphertexts
    he_lr_job j{};
    j.c = c;
    memcpy(j.poly, poly, sizeof j.poly);
    j.g = g;
    j.m = m;
    j.lg = __builtin_ctz(g);
    j.lm = __builtin_ctz(m);
    j.L = L;
    j.scale0 = W->scale;
    const size_t N = c->n;
    j.ctw = 2 * (size_t)(L + 1) * N;
    j.chunk = (int)std::min<size_t>(nb, 64);
    int rc = HE_OK;
    uint64_t *zbuf = nullptr;
    he_ct *Wo = nullptr, *Vo = nullptr;
    if ((rc = ev_init(c, &j.ev, std::max(j.chunk, 3), L))) goto out;
    if ((rc = helr_alloc(c, (void **)&j.buf, sizeof(uint64_t) * j.ctw * (5 * (size_t)std::max(j.chunk, 3) + 3)))) goto out;
    j.T0 = j.buf;
    j.T1 = j.T0 + j.ctw * std::max(j.chunk, 3);
    j.T2 = j.T1 + j.ctw * std::max(j.chunk, 3);
    j.T3 = j.T2 + j.ctw * std::max(j.chunk, 3);
    j.T4 = j.T3 + j.ctw * std::max(j.chunk, 3);
    j.acc = j.T4 + j.ctw * std::max(j.chunk, 3);
    if ((rc = make_sigmoid_pts(c, L, g, Z[0]->scale, W->scale, j.poly, &j.sig, &j.p1_scale))) goto out;
    if ((rc = helr_alloc(c, (void **)&zbuf, sizeof(uint64_t) * j.ctw * j.chunk))) goto out;
    j.W = const_cast<he_ct *>(W);
    j.V = const_cast<he_ct *>(V);
    {
        const CtB Wb{W->d, 1, L, W->scale, 0};
        double gscale = 0;
        int glevel = 0;
        for (size_t b = 0; b < nb && !rc; b += j.chunk) {
            int cnt = (int)std::min<size_t>(j.chunk, nb - b);
            for (int i = 0; i < cnt && !rc; i++)
                if (cudaMemcpyAsync(zbuf + (size_t)i * j.ctw, Z[b + i]->d, j.ctw * 8, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                    rc = helr_fail(c, HE_ECUDA, "gather");
            CtB gg{};
            if (!rc) rc = block_grads(&j, zbuf, cnt, Wb, gg);
            if (!rc) rc = ev_sum_items(&j.ev, gg, j.acc, b != 0);
            gscale = gg.scale;
            glevel = gg.level;
        }
        if (rc) goto out;
        if ((rc = helr_new_ct(c, L - depth, 0, &Wo))) goto out;
        if ((rc = helr_new_ct(c, L - depth, 0, &Vo))) goto out;
        CtB acc{j.acc, 1, glevel, gscale, 0};
        CtB Wn{Wo->d, 1, 0, 0, 0}, Vn{Vo->d, 1, 0, 0, 0};
        if ((rc = finish(&j, acc, B, alpha, eta, inv_n, Wn, Vn))) goto out;
        Wo->level = Wn.level;
        Wo->scale = Wn.scale;
        Vo->level = Vn.level;
        Vo->scale = Vn.scale;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = helr_fail(c, HE_ECUDA, "iteration");
    }
out:
    helr_free(c, zbuf);
    helr_free(c, j.sig);
    helr_free(c, j.buf);
    ev_free(&j.ev);
    cudaStreamSynchronize(c->stream);
    if (rc) {
        if (Wo) he_ct_free(Wo);
        if (Vo) he_ct_free(Vo);
        return rc;
    }
    *W_out = Wo;
    *V_out = Vo;
    return HE_OK;
}

extern "C" int he_refresh(he_ctx *c, const he_ct *in, int level, double scale, uint64_t seed, he_ct **out)
{
    if (!c || !in || !out || !(scale > 0) || level < 0 || level >= c->nq) return HE_EINVAL;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, level, scale, &o));
    int rc = refresh_dev(c, in->d, in->level, in->scale, level, scale, seed, o->d);
    if (!rc) rc = cudaStreamSynchronize(c->stream) == cudaSuccess ? HE_OK : helr_fail(c, HE_ECUDA, "refresh");
    if (rc) {
        he_ct_free(o);
        return rc;
    }
    *out = o;
    return HE_OK;
}

// ------------------------------------------------------------------ several jobs at once
// Independent full-batch jobs of one context stepped together: the data blocks
// of all jobs are ordered by decreasing row width g and Steps 1-6 run over
// chunks of that order, so every key switch is batched across jobs (segments
// carry each job's W and sigmoid plaintexts; rotations a narrower job does not need run on a
// prefix of the chunk).  Steps 7-9 and the refresh run per job.
struct he_lr_multi {
    he_ctx *c;
    std::vector<he_lr_job *> jobs;
    std::vector<std::pair<int, int>> order;  // (job, block)
    int L, chunk;
    size_t ctw;
    double scale0;
    double poly[3];
    Eval ev;
    uint64_t *buf;  // 5 x chunk work ciphertexts, chunk staged blocks, njobs accumulators, W' and V'
    uint64_t *T[5], *Zs, *accs, *wv;
};

extern "C" int he_lr_multi_free(he_lr_multi *m)
{
    if (!m) return HE_EINVAL;
    cudaStreamSynchronize(m->c->stream);
    helr_free(m->c, m->buf);
    ev_free(&m->ev);
    cudaStreamSynchronize(m->c->stream);
    delete m;
    return HE_OK;
}

extern "C" int he_lr_multi_create(he_ctx *c, he_lr_job *const *jobs, size_t njobs, int blocks_per_launch,
                                  he_lr_multi **out)
{
    if (!c || !jobs || !njobs || !out) return HE_EINVAL;
    *out = nullptr;
    for (size_t i = 0; i < njobs; i++) {
        const he_lr_job *j = jobs[i];
        if (!j || j->c != c) return helr_fail(c, HE_EINVAL, "job %zu belongs to another context", i);
        if (j->mode != HE_LR_FULL_BATCH) return helr_fail(c, HE_EINVAL, "job %zu is not a full-batch job", i);
        if (j->L != jobs[0]->L || j->scale0 != jobs[0]->scale0 || memcmp(j->poly, jobs[0]->poly, sizeof j->poly) ||
            j->first_order != jobs[0]->first_order)
            return helr_fail(c, HE_EINVAL, "job %zu differs from job 0 in level, scale, polynomial or method", i);
    }
    he_lr_multi *m = new he_lr_multi();
    m->c = c;
    m->jobs.assign(jobs, jobs + njobs);
    m->L = jobs[0]->L;
    m->ctw = jobs[0]->ctw;
    m->scale0 = jobs[0]->scale0;
    memcpy(m->poly, jobs[0]->poly, sizeof m->poly);
    std::vector<int> idx(njobs);
    for (size_t i = 0; i < njobs; i++) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return jobs[a]->lg > jobs[b]->lg; });
    for (int i : idx)
        for (int b = 0; b < jobs[i]->nblocks; b++) m->order.push_back({i, b});
    m->chunk = std::max(1, std::min(blocks_per_launch > 0 ? blocks_per_launch : 256, (int)m->order.size()));
    int rc = ev_init(c, &m->ev, m->chunk, m->L);
    const size_t cts = 6 * (size_t)m->chunk + njobs + 2;
    if (!rc) rc = helr_alloc(c, (void **)&m->buf, sizeof(uint64_t) * m->ctw * cts);
    if (rc) {
        he_lr_multi_free(m);
        return rc;
    }
    for (int k = 0; k < 5; k++) m->T[k] = m->buf + (size_t)k * m->chunk * m->ctw;
    m->Zs = m->buf + (size_t)5 * m->chunk * m->ctw;
    m->accs = m->Zs + (size_t)m->chunk * m->ctw;
    m->wv = m->accs + njobs * m->ctw;
    *out = m;
    return HE_OK;
}

extern "C" int he_lr_multi_step(he_lr_multi *m, int t, he_lr_sched sched)
{
    if (!m || t < 0 || !(sched.T > 0)) return HE_EINVAL;
    he_ctx *c = m->c;
    const double alpha = f2(sched, (double)t), eta = nag_eta(t);
    const WorkSet ws{&m->ev, {m->T[0], m->T[1], m->T[2], m->T[3], m->T[4]}, m->ctw, m->L, m->scale0, m->poly};
    std::vector<char> started(m->jobs.size(), 0);
    double gscale = 0;
    int glevel = 0;
    m->ev.keyswitches = 0;
    for (size_t p = 0; p < m->order.size(); p += m->chunk) {
        const int cnt = (int)std::min<size_t>(m->chunk, m->order.size() - p);
        std::vector<Seg> segs;
        for (int i = 0; i < cnt; i++) {
            const int jb = m->order[p + i].first, blk = m->order[p + i].second;
            he_lr_job *j = m->jobs[jb];
            HELR_CUDA(c, cudaMemcpyAsync(m->Zs + (size_t)i * m->ctw, j->Z + (size_t)blk * m->ctw, m->ctw * 8,
                                         cudaMemcpyDeviceToDevice, c->stream));
            if (i == 0 || m->order[p + i - 1].first != jb)
                segs.push_back(Seg{i, 0, j->lg, j->W->d, sig_pts(j->sig, j->L, c->n), j->p1_scale});
            segs.back().count++;
        }
        CtB g{};
        HELR_TRY(block_grads_seg(ws, m->Zs, cnt, segs.data(), (int)segs.size(), m->scale0, g));
        for (const Seg &sg : segs) {
            const int jb = m->order[p + sg.start].first;
            CtB sub{g.d + (size_t)sg.start * m->ctw, sg.count, g.level, g.scale, m->ctw};
            HELR_TRY(ev_sum_items(&m->ev, sub, m->accs + (size_t)jb * m->ctw, started[jb]));
            started[jb] = 1;
        }
        gscale = g.scale;
        glevel = g.level;
    }
    for (size_t jb = 0; jb < m->jobs.size(); jb++) {
        he_lr_job *j = m->jobs[jb];
        CtB acc{m->accs + jb * m->ctw, 1, glevel, gscale, 0};
        CtB Wn{m->wv, 1, 0, 0, 0}, Vn{m->wv + m->ctw, 1, 0, 0, 0};
        HELR_TRY(finish_ws(ws, acc, j->first_order ? nullptr : j->B[0], j->W, j->V, j->g, j->lm, alpha, eta, j->inv_n[0],
                           Wn, Vn));
        HELR_TRY(refresh_dev(c, Wn.d, Wn.level, Wn.scale, j->L, j->scale0, obj_seed(j->enc_seed, 5, t), j->W->d));
        HELR_TRY(refresh_dev(c, Vn.d, Vn.level, Vn.scale, j->L, j->scale0, obj_seed(j->enc_seed, 6, t), j->V->d));
        j->W->scale = j->V->scale = j->scale0;
    }
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    return HE_OK;
}
