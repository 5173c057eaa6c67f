// autotune.cu -- choice of the key-switch wave and kernel tiles per (N, limbs),
// measured on the device and kept in a table file.
//
// Hybrid key switching (Sec. 2.1: the relinearisation inside Mul and the key
// switch inside every rotation) runs its ModUp and inner product in waves of
// items that share one DRAM read of each key row.  The wave is the one tile of
// the fused path that is chosen at run time: a larger wave amortises the key
// read over more items but needs [wave][nl][nl+1][N] words of scratch and a
// larger L2 footprint per key row.  The kernel tiles come in four variants
// (tile bit 0: the column kernel of ModUp and ModDown with half as many
// columns per CTA; bit 1: the row kernels of ModDown and of the hoisted
// digits with half as many rows per CTA); the words per thread of a pass
// (2^ceil(K/2) of a row or column of 2^K words) are fixed by the transform's
// register layout.
//
// he_autotune times batched key switches at every limb count nl = 1..n_q:
// first every wave candidate with tile 0, keeping the smallest wave within 1%
// of the fastest, then the other tiles at that wave, keeping a variant only
// when it beats tile 0 by more than 1%; helr_ks_wave and helr_ks_tile consult
// the result.  Where the tensor-core form of the hoisted inner product applies
// (ks_tensor.cu), it also times a hoisted sum of seven rotations in both forms
// at that wave and keeps the tensor-core form only when it is more than 1%
// faster (helr_hoist_form).  The table file holds one header line naming the
// device and the parameters, then one line per limb count:
//     he_lr ks-wave table v3
//     key <device> <SMs> <log N> <n_q> <hash of the primes>
//     nl <nl> wave <items> tile <variant> us_per_keyswitch <time> hoist <form> us_per_rotation <time>
// (a v2 file, without the last four fields, is read with form 0).  A file
// whose header names another device or parameter set is measured anew and
// overwritten.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "helr_internal.cuh"

namespace {

constexpr int kWaves[] = {16, 32, 64, 128, 256};
constexpr int kTiles = 4;

// uniform words below q_j for limb j of every item (the values only need to be
// valid residues; their distribution does not change the work)
__global__ void k_fill_residues(uint64_t *out, size_t nwords, int logn, int nl, const ModQ *mods, uint64_t seed)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)((i >> logn) % (size_t)nl);
        uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        out[i] = reduce64(z, mods[j]);
    }
}

struct TuneKey {
    char dev[256];
    int sms, logn, nq;
    unsigned long long qhash;
};

TuneKey key_of(const he_ctx *c)
{
    TuneKey k{};
    cudaDeviceProp p;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
        snprintf(k.dev, sizeof k.dev, "%s", p.name);
        k.sms = p.multiProcessorCount;
    } else {
        snprintf(k.dev, sizeof k.dev, "unknown");
    }
    for (char *s = k.dev; *s; s++)
        if (*s == ' ' || *s == '\t') *s = '_';
    k.logn = c->logn;
    k.nq = c->nq;
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the primes q_0..q_{nq-1}, P
    for (int i = 0; i <= c->nq; i++)
        for (int b = 0; b < 8; b++) h = (h ^ ((c->q[i] >> (8 * b)) & 0xff)) * 1099511628211ull;
    k.qhash = h;
    return k;
}

struct TuneRow {
    int wave = 0, tile = 0, hoist = 0;
    double us = 0, us_rot = 0;
};

// entries of a table file whose header matches `k` (row.wave = 0: none)
bool load_table(const char *path, const TuneKey &k, TuneRow *rows)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512], dev[256];
    int sms, logn, nq, nl, wave, tile, hoist;
    unsigned long long qh;
    double t, tr;
    int ver = 0;
    if (fgets(line, sizeof line, f)) {
        if (strncmp(line, "he_lr ks-wave table v3", 22) == 0) ver = 3;
        else if (strncmp(line, "he_lr ks-wave table v2", 22) == 0) ver = 2;
    }
    bool ok = ver && fgets(line, sizeof line, f) &&
              sscanf(line, "key %255s %d %d %d %llx", dev, &sms, &logn, &nq, &qh) == 5 && strcmp(dev, k.dev) == 0 &&
              sms == k.sms && logn == k.logn && nq == k.nq && qh == k.qhash;
    while (ok && fgets(line, sizeof line, f)) {
        const int got = sscanf(line, "nl %d wave %d tile %d us_per_keyswitch %lf hoist %d us_per_rotation %lf", &nl,
                               &wave, &tile, &t, &hoist, &tr);
        if ((got == 6 || (ver == 2 && got == 4)) && nl >= 1 && nl <= k.nq && wave > 0 && tile >= 0 && tile < kTiles) {
            rows[nl].wave = wave, rows[nl].tile = tile, rows[nl].us = t;
            rows[nl].hoist = got == 6 && hoist == 1 ? 1 : 0;
            rows[nl].us_rot = got == 6 ? tr : 0;
        }
    }
    fclose(f);
    return ok;
}

bool save_table(const char *path, const TuneKey &k, const TuneRow *rows)
{
    FILE *f = fopen(path, "w");
    if (!f) return false;
    fprintf(f, "he_lr ks-wave table v3\nkey %s %d %d %d %llx\n", k.dev, k.sms, k.logn, k.nq, k.qhash);
    for (int nl = 1; nl <= k.nq; nl++)
        if (rows[nl].wave > 0)
            fprintf(f, "nl %d wave %d tile %d us_per_keyswitch %.3f hoist %d us_per_rotation %.3f\n", nl, rows[nl].wave,
                    rows[nl].tile, rows[nl].us, rows[nl].hoist, rows[nl].us_rot);
    return fclose(f) == 0;
}

// fastest wave, then fastest tile variant, for key switches of `items` inputs
// at nl limbs; *us = time per key switch
int measure(he_ctx *c, const uint64_t *key, int items, int nl, int *best, int *best_tile, double *us, int *hoist,
            double *us_rot)
{
    const size_t N = c->n;
    int maxw = 0;
    for (int w : kWaves)
        if (w <= items) maxw = w;
    uint64_t *din = nullptr, *dout = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&din, (size_t)items * nl * N * 8));
    int rc = helr_alloc(c, (void **)&dout, (size_t)items * 2 * nl * N * 8);
    KsScratch ws{};
    ws.base = nullptr;
    // scratch sized for the largest candidate that fits
    const int saved = c->ks_wave, saved_tile = c->ks_tile;
    while (rc == HE_OK) {
        c->ks_wave = maxw;
        rc = helr_ks_scratch_alloc(c, items, nl - 1, &ws);
        c->ks_wave = saved;
        if (rc != HE_ENOMEM || maxw <= kWaves[0]) break;
        maxw /= 2;
        rc = HE_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == HE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = helr_fail(c, HE_ECUDA, "event creation failed");
    if (rc == HE_OK) {
        const size_t nw = (size_t)items * nl * N;
        k_fill_residues<<<(unsigned)std::min<size_t>((nw + 255) / 256, 152 * 32), 256, 0, c->stream>>>(
            din, nw, c->logn, nl, c->t.mod, 0x5eedull + nl);
        if (cudaGetLastError() != cudaSuccess) rc = helr_fail(c, HE_ECUDA, "fill kernel launch failed");
    }
    // one warm-up, then the faster of two timed runs
    auto time_ks = [&](int w, int tile, double *ms) {
        ws.wave = w;
        c->ks_tile = tile;
        for (int r = 0; r < 3 && rc == HE_OK; r++) {
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) rc = helr_fail(c, HE_ECUDA, "event record failed");
            if (rc == HE_OK) rc = helr_keyswitch(c, din, dout, items, nl - 1, key, &ws, nullptr);
            float t = 0;
            if (rc == HE_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                rc = helr_fail(c, HE_ECUDA, "event timing failed");
            if (r == 1 || (r == 2 && t < *ms)) *ms = t;
        }
        c->ks_tile = saved_tile;
    };
    double msw[sizeof kWaves / sizeof kWaves[0]] = {};
    int nw = 0;
    for (int w : kWaves) {
        if (rc != HE_OK || w > maxw) break;
        double ms = 0;
        time_ks(w, 0, &ms);
        if (rc == HE_OK) msw[nw++] = ms;
    }
    // the smallest wave within 1% of the fastest: less scratch, and timing noise
    // does not flip the choice between near-equal waves
    double best_ms = 0;
    *best = 0;
    *best_tile = 0;
    for (int i = 0; i < nw; i++)
        if (i == 0 || msw[i] < best_ms) best_ms = msw[i];
    for (int i = 0; i < nw && !*best; i++)
        if (msw[i] <= 1.01 * best_ms) *best = kWaves[i], best_ms = msw[i];
    // the other tile variants at that wave: kept only when more than 1% faster
    for (int tile = 1; tile < kTiles && rc == HE_OK && *best; tile++) {
        double ms = 0;
        time_ks(*best, tile, &ms);
        if (rc == HE_OK && ms < best_ms / 1.01) *best_tile = tile, best_ms = ms;
    }
    // the hoisted inner product's two forms, on a sum of seven rotations of
    // `items` ciphertexts (the relinearisation key stands in for the rotation
    // keys: the timing does not depend on the key words)
    *hoist = 0;
    *us_rot = 0;
    int t_lo, t_hi;
    if (rc == HE_OK && *best && helr_hoist_tensor_range(c, nl, HELR_MAX_HOIST, &t_lo, &t_hi)) {
        HoistKeys hk{};
        hk.n = HELR_MAX_HOIST;
        uint64_t g = 1;
        for (int j = 0; j < HELR_MAX_HOIST; j++) {
            g = g * 5 % (2 * (uint64_t)N);
            hk.gal[j] = g;
            hk.key[j] = key;
        }
        const size_t ct = 2 * (size_t)nl * N;
        uint64_t *cin = nullptr, *cout = nullptr;
        rc = helr_alloc(c, (void **)&cin, (size_t)items * ct * 8);
        if (rc == HE_OK) rc = helr_alloc(c, (void **)&cout, (size_t)items * ct * 8);
        if (rc == HE_OK) {
            const size_t nw = (size_t)items * ct;
            k_fill_residues<<<(unsigned)std::min<size_t>((nw + 255) / 256, 152 * 32), 256, 0, c->stream>>>(
                cin, nw, c->logn, nl, c->t.mod, 0x7eedull + nl);
            if (cudaGetLastError() != cudaSuccess) rc = helr_fail(c, HE_ECUDA, "fill kernel launch failed");
        }
        const int saved_form = c->hoist_form;
        double ms_form[2] = {0, 0};
        ws.wave = *best;
        c->ks_tile = *best_tile;
        for (int form = 0; form < 2 && rc == HE_OK; form++) {
            c->hoist_form = form;
            for (int r = 0; r < 3 && rc == HE_OK; r++) {
                if (cudaEventRecord(e0, c->stream) != cudaSuccess) rc = helr_fail(c, HE_ECUDA, "event record failed");
                if (rc == HE_OK)
                    rc = helr_rotsum(c, cin, ct, items, nl - 1, hk, &ws, Str{cout, ct, (size_t)nl * N});
                float t = 0;
                if (rc == HE_OK &&
                    (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                     cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                    rc = helr_fail(c, HE_ECUDA, "event timing failed");
                if (r == 1 || (r == 2 && t < ms_form[form])) ms_form[form] = t;
            }
        }
        c->hoist_form = saved_form;
        c->ks_tile = saved_tile;
        if (rc == HE_OK) {
            *hoist = ms_form[1] < ms_form[0] / 1.01 ? 1 : 0;
            *us_rot = ms_form[*hoist] * 1000.0 / ((double)items * HELR_MAX_HOIST);
        }
        helr_free(c, cout);
        helr_free(c, cin);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ws.base) helr_ks_scratch_free(c, &ws);
    helr_free(c, dout);
    helr_free(c, din);
    if (rc == HE_OK) *us = best_ms * 1000.0 / items;
    return rc;
}

}  // namespace

int helr_ks_wave(const he_ctx *c, int nl)
{
    if (c->ks_wave > 0) return c->ks_wave;
    if (nl >= 1 && nl <= HELR_MAXQ && c->ks_wave_tab[nl] > 0) return c->ks_wave_tab[nl];
    // measured on GB300 at N = 2^16: each key row is read from DRAM once per
    // wave, and 128 items keep the scratch of [wave][nl][nl+1][N] words at
    // 3.7 GB for 7 limbs
    return 128;
}

int helr_ks_tile(const he_ctx *c, int nl)
{
    if (c->ks_tile >= 0) return c->ks_tile;
    if (nl >= 1 && nl <= HELR_MAXQ) return c->ks_tile_tab[nl];
    return 0;
}

int helr_hoist_form(const he_ctx *c, int nl)
{
    if (c->hoist_form >= 0) return c->hoist_form;
    if (nl >= 1 && nl <= HELR_MAXQ) return c->hoist_form_tab[nl];
    return 0;
}

extern "C" int he_autotune(he_ctx *c, const char *path, int items, int *measured)
{
    if (!c || items < 0 || (items > 0 && items < kWaves[0])) return HE_EINVAL;
    if (items == 0) items = 256;
    const uint64_t *key = helr_find_key(c, 0);
    if (!key) return helr_fail(c, HE_EKEY, "autotuning needs the relinearisation key (he_keygen first)");
    const TuneKey k = key_of(c);
    TuneRow rows[HELR_MAXQ + 1];
    if (path) load_table(path, k, rows);
    int n = 0;
    for (int nl = 1; nl <= c->nq; nl++) {
        if (rows[nl].wave > 0) continue;
        TuneRow &r = rows[nl];
        HELR_TRY(measure(c, key, items, nl, &r.wave, &r.tile, &r.us, &r.hoist, &r.us_rot));
        n++;
    }
    for (int nl = 1; nl <= c->nq; nl++)
        c->ks_wave_tab[nl] = rows[nl].wave, c->ks_tile_tab[nl] = rows[nl].tile, c->hoist_form_tab[nl] = rows[nl].hoist;
    if (path && n && !save_table(path, k, rows)) return helr_fail(c, HE_EINVAL, "cannot write %s", path);
    if (measured) *measured = n;
    return HE_OK;
}

extern "C" int he_ks_wave(const he_ctx *c, int level)
{
    if (!c || level < 0 || level >= c->nq) return -HE_EINVAL;
    return helr_ks_wave(c, level + 1);
}

extern "C" int he_ks_tile(const he_ctx *c, int level)
{
    if (!c || level < 0 || level >= c->nq) return -HE_EINVAL;
    return helr_ks_tile(c, level + 1);
}

extern "C" int he_hoist_form(const he_ctx *c, int level)
{
    if (!c || level < 0 || level >= c->nq) return -HE_EINVAL;
    return helr_hoist_form(c, level + 1);
}

extern "C" int he_set_ks_tile(he_ctx *c, int tile)
{
    if (!c || tile < -1 || tile >= kTiles) return c ? helr_fail(c, HE_EINVAL, "tile variant %d (0..3, -1 = tuned)", tile)
                                                     : HE_EINVAL;
    c->ks_tile = tile;
    return HE_OK;
}
