// eval.cu -- batched homomorphic operations (Sec. 2.1) over many ciphertexts at
// once, and the single-ciphertext C ABI built on them.
//
// Scale rule: Mul and plaintext products multiply scales; Rescale at level l
// divides by q_l; cMul by the integer k at constant scale S multiplies by S;
// cAdd adds round_half_away(c * scale); Add needs scales equal to 2^-40.
#include <math.h>
#include "helr_internal.cuh"

#define GS_LOOP(i, n) for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

namespace {
inline unsigned grid_for(size_t work, int threads = 256)
{
    size_t b = (work + threads - 1) / threads;
    if (b > (size_t)152 * 64) b = (size_t)152 * 64;
    return (unsigned)(b ? b : 1);
}

// acc[p][j][k] (+)= sum_b a[b][p][j][k]
__global__ void k_sum_items_kernel(uint64_t *acc, const uint64_t *a, size_t item, int batch, size_t nwords, int logn,
                                   int nl, const ModQ *mods, int accumulate)
{
    GS_LOOP(i, nwords) {
        int j = (int)((i >> logn) % nl);
        uint64_t q = mods[j].q;
        uint64_t s = accumulate ? acc[i] : 0;
        for (int b = 0; b < batch; b++) s = addmod(s, a[b * item + i], q);
        acc[i] = s;
    }
}
}  // namespace

bool scales_match(double a, double b) { return fabs(a - b) <= a * 0x1p-40; }

int64_t round_half_away(double x) { return llround(x); }

static KP shoup_consts(const he_ctx *c, int nl, int64_t k)
{
    KP kp;
    for (int j = 0; j < nl; j++) {
        uint64_t q = c->q[j];
        uint64_t v = k >= 0 ? (uint64_t)k % q : (q - (uint64_t)(-(k + 1)) % q - 1);
        kp.w[j][0] = v;
        kp.w[j][1] = (uint64_t)(((unsigned __int128)v << 64) / q);
    }
    return kp;
}

static inline Str S(const CtB &x, he_ctx *c) { return Str{x.d, x.item, (size_t)(x.level + 1) * c->n}; }

int ev_init(he_ctx *c, Eval *ev, int maxb, int maxlevel)
{
    ev->c = c;
    ev->maxb = maxb;
    ev->maxlevel = maxlevel;
    ev->keyswitches = 0;
    const size_t nl = maxlevel + 1, N = c->n, B = maxb;
    HELR_TRY(helr_ks_scratch_alloc(c, maxb, maxlevel, &ev->ks));
    size_t words = 3 * B * nl * N + 2 * B * nl * N + B * nl * N + 2 * B * N + 2 * B * nl * N;
    uint64_t *p = nullptr;
    HELR_TRY(helr_alloc(c, (void **)&p, words * 8));
    ev->tens = p;
    ev->ksout = ev->tens + 3 * B * nl * N;
    ev->rot1 = ev->ksout + 2 * B * nl * N;
    ev->last = ev->rot1 + B * nl * N;
    ev->lift = ev->last + 2 * B * N;
    return HE_OK;
}
void ev_free(Eval *ev)
{
    if (!ev->c) return;
    helr_ks_scratch_free(ev->c, &ev->ks);
    helr_free(ev->c, ev->tens);
    ev->tens = nullptr;
}

static int check_batch(Eval *ev, const CtB &a)
{
    if (a.batch > ev->maxb || a.level > ev->maxlevel)
        return helr_fail(ev->c, HE_EINTERNAL, "batch %d / level %d exceeds evaluator capacity", a.batch, a.level);
    return HE_OK;
}

// out = Relin(a (x) b); b may broadcast.  out.level = a.level, scale = product.
// The relinearisation sum (d0, d1) + KS(d2) is formed in the key switch's output stage.
int ev_mul_relin(Eval *ev, const CtB &a, const CtB &b, CtB &out)
{
    he_ctx *c = ev->c;
    HELR_TRY(check_batch(ev, a));
    if (a.level != b.level) return helr_fail(c, HE_ELEVEL, "Mul: levels %d and %d differ", a.level, b.level);
    const int B = a.batch, lv = a.level, nl = lv + 1;
    const size_t N = c->n, lw = (size_t)nl * N;
    const uint64_t *key = helr_find_key(c, 0);
    if (!key) return helr_fail(c, HE_EKEY, "no relinearisation key");
    k_tensor(c, a.d, b.d, ev->tens, B, lv, a.item, b.item, lw, (size_t)B * lw, c->stream);
    out.level = lv;
    out.batch = B;
    out.scale = a.scale * b.scale;
    KsOut o;
    o.out = S(out, c);
    o.rel = ev->tens;
    o.rel_item = lw;
    o.rel_poly = (size_t)B * lw;
    HELR_TRY(helr_keyswitch(c, ev->tens + 2 * (size_t)B * lw, nullptr, B, lv, key, &ev->ks, &o));
    ev->keyswitches += B;
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// out = Relin(a (x) b_s) where item i of segment s (items start_s .. start_s + count_s - 1)
// is multiplied by the single ciphertext bptr[s]; one key switch over the whole batch.
int ev_mul_relin_seg(Eval *ev, const CtB &a, const uint64_t *const *bptr, const int *start, const int *count, int nseg,
                     double bscale, CtB &out)
{
    he_ctx *c = ev->c;
    HELR_TRY(check_batch(ev, a));
    const int B = a.batch, lv = a.level, nl = lv + 1;
    const size_t N = c->n, lw = (size_t)nl * N;
    const uint64_t *key = helr_find_key(c, 0);
    if (!key) return helr_fail(c, HE_EKEY, "no relinearisation key");
    for (int sg = 0; sg < nseg; sg++)
        k_tensor(c, a.d + (size_t)start[sg] * a.item, bptr[sg], ev->tens + (size_t)start[sg] * lw, count[sg], lv, a.item, 0, lw,
                 (size_t)B * lw, c->stream);
    out.level = lv;
    out.batch = B;
    out.scale = a.scale * bscale;
    KsOut o;
    o.out = S(out, c);
    o.rel = ev->tens;
    o.rel_item = lw;
    o.rel_poly = (size_t)B * lw;
    HELR_TRY(helr_keyswitch(c, ev->tens + 2 * (size_t)B * lw, nullptr, B, lv, key, &ev->ks, &o));
    ev->keyswitches += B;
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// divide by q_level with rounding: out at level - 1
int ev_rescale(Eval *ev, const CtB &a, CtB &out)
{
    he_ctx *c = ev->c;
    HELR_TRY(check_batch(ev, a));
    const int lv = a.level;
    if (lv < 1) return helr_fail(c, HE_ELEVEL, "Rescale: no level left");
    const int B = a.batch, nl = lv + 1;
    const size_t N = c->n;
    cudaStream_t s = c->stream;
    const size_t item = a.item ? a.item : 2 * (size_t)nl * N;
    // the dropped limb q_lv of both polynomials: inverse row pass, then the
    // fused column passes and the output stage (value - centred lift) * q_lv^-1
    HELR_TRY(helr_ntt_inv_rows(c, a.d + (size_t)lv * N, item, (size_t)nl * N, ev->last, 2 * (size_t)B, limbmap_single(lv), s));
    out.level = lv - 1;
    out.batch = B;
    out.scale = a.scale / (double)c->q[lv];
    KsOut o;
    o.out = S(out, c);
    HELR_TRY(helr_ks_down(c, o, a.d, item, (size_t)nl * N, ev->last, lv, ev->lift, B, lv, c->d_qinv + (size_t)lv * c->nq * 2,
                          s));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// left rotation by r slots (accumulate: out = a + Rot(a, r)); out must not alias a
int ev_rotate_acc(Eval *ev, const CtB &a, int64_t r, CtB &out, int accumulate)
{
    he_ctx *c = ev->c;
    const uint64_t gal = he_galois_elt(c, r);
    if (!helr_find_key(c, gal)) return helr_fail(c, HE_EKEY, "no rotation key for %lld", (long long)r);
    return ev_rotate_gal(ev, a, gal, out, accumulate);
}

// the automorphism X -> X^gal of both polynomials and the key switch of the
// second back to s (gal = 5^r mod 2N: rotation by r slots; gal = 2N - 1: the
// slot-wise complex conjugation); accumulate: out = a + sigma_gal(a)
int ev_rotate_gal(Eval *ev, const CtB &a, uint64_t gal, CtB &out, int accumulate)
{
    he_ctx *c = ev->c;
    HELR_TRY(check_batch(ev, a));
    const uint64_t *key = helr_find_key(c, gal);
    if (!key) return helr_fail(c, HE_EKEY, "no key-switching key for galois element %llu", (unsigned long long)gal);
    const int B = a.batch, lv = a.level, nl = lv + 1;
    const size_t N = c->n, lw = (size_t)nl * N;
    cudaStream_t s = c->stream;
    k_automorph_items(c, ev->rot1, lw, a.d + lw, a.item, B, nl, gal, s);
    out.level = lv;
    out.batch = B;
    out.scale = a.scale;
    KsOut o;
    o.out = S(out, c);
    o.rot = a.d;
    o.rot_item = a.item;
    o.gals[0] = gal;
    o.ngal = 1;
    if (accumulate) {
        o.acc = a.d;
        o.acc_item = a.item;
        o.acc_poly = lw;
    }
    HELR_TRY(helr_keyswitch(c, ev->rot1, nullptr, B, lv, key, &ev->ks, &o));
    ev->keyswitches += B;
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}
int ev_rotate(Eval *ev, const CtB &a, int64_t r, CtB &out) { return ev_rotate_acc(ev, a, r, out, 0); }
// out = a + sum_j Rot(a, rots[j]) with one ModUp and one ModDown per item
// (hoisted rotations); out must not alias a
int ev_rotsum(Eval *ev, const CtB &a, const int64_t *rots, int nrot, CtB &out)
{
    he_ctx *c = ev->c;
    HELR_TRY(check_batch(ev, a));
    if (nrot < 1 || nrot > HELR_MAX_HOIST) return helr_fail(c, HE_EINVAL, "%d rotations in one hoisted sum", nrot);
    HoistKeys hk{};
    hk.n = nrot;
    for (int j = 0; j < nrot; j++) {
        hk.gal[j] = he_galois_elt(c, rots[j]);
        hk.key[j] = helr_find_key(c, hk.gal[j]);
        if (!hk.key[j]) return helr_fail(c, HE_EKEY, "no rotation key for %lld", (long long)rots[j]);
    }
    out.level = a.level;
    out.batch = a.batch;
    out.scale = a.scale;
    HELR_TRY(helr_rotsum(c, a.d, a.item, a.batch, a.level, hk, &ev->ks, S(out, c)));
    ev->keyswitches += (uint64_t)a.batch * nrot;
    return HE_OK;
}

int ev_add(Eval *ev, const CtB &a, const CtB &b, CtB &out, int sub)
{
    he_ctx *c = ev->c;
    if (a.level != b.level) return helr_fail(c, HE_ELEVEL, "Add: levels %d and %d differ", a.level, b.level);
    if (!scales_match(a.scale, b.scale)) return helr_fail(c, HE_ESCALE, "Add: scales %.17g and %.17g differ", a.scale, b.scale);
    out.level = a.level;
    out.batch = a.batch;
    out.scale = a.scale;
    k_ew(c, sub ? EW_SUB : EW_ADD, S(out, c), S(a, c), S(b, c), a.batch, 2, a.level + 1, nullptr, c->stream);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int ev_cmul_int(Eval *ev, const CtB &a, int64_t k, double out_scale, CtB &out)
{
    he_ctx *c = ev->c;
    KP kp = shoup_consts(c, a.level + 1, k);
    out.level = a.level;
    out.batch = a.batch;
    out.scale = out_scale;
    k_ew(c, EW_CMUL, S(out, c), S(a, c), S(a, c), a.batch, 2, a.level + 1, &kp, c->stream);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// c0 += k (the constant polynomial k is k in every evaluation)
int ev_cadd_int(Eval *ev, CtB &a, int64_t k)
{
    he_ctx *c = ev->c;
    KP kp = shoup_consts(c, a.level + 1, k);
    Str x{a.d, a.item, 0};
    k_ew(c, EW_CADD, x, x, x, a.batch, 1, a.level + 1, &kp, c->stream);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int ev_ptmul(Eval *ev, const CtB &a, const uint64_t *pt, double pt_scale, CtB &out)
{
    he_ctx *c = ev->c;
    out.level = a.level;
    out.batch = a.batch;
    out.scale = a.scale * pt_scale;
    Str p{const_cast<uint64_t *>(pt), 0, 0};
    k_ew(c, EW_MUL, S(out, c), S(a, c), p, a.batch, 2, a.level + 1, nullptr, c->stream);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// c0 += m in place for a plaintext m (evaluation form) at the level and scale of a
int ev_ptadd(Eval *ev, CtB &a, const uint64_t *pt)
{
    he_ctx *c = ev->c;
    Str p{const_cast<uint64_t *>(pt), 0, 0};
    k_ew(c, EW_ADD, S(a, c), S(a, c), p, a.batch, 1, a.level + 1, nullptr, c->stream);  // polynomial 0 only
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int ev_moddrop(Eval *ev, const CtB &a, int target, CtB &out)
{
    he_ctx *c = ev->c;
    if (target > a.level || target < 0) return helr_fail(c, HE_ELEVEL, "ModDrop to %d from %d", target, a.level);
    Str in{a.d, a.item, (size_t)(a.level + 1) * c->n};
    out.level = target;
    out.batch = a.batch;
    out.scale = a.scale;
    k_ew(c, EW_COPY, S(out, c), in, in, a.batch, 2, target + 1, nullptr, c->stream);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int ev_sum_items(Eval *ev, const CtB &a, uint64_t *acc, int accumulate)
{
    he_ctx *c = ev->c;
    const int nl = a.level + 1;
    size_t nw = 2 * (size_t)nl * c->n;
    HELR_LAUNCH(k_sum_items_kernel<<<grid_for(nw), 256, 0, c->stream>>>(acc, a.d, a.item, a.batch, nw, c->logn, nl, c->t.mod, accumulate));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

// ------------------------------------------------------------------ single-ciphertext C ABI
static int one_eval(he_ctx *c, int level, Eval *ev) { return ev_init(c, ev, 1, level); }

static CtB view(const he_ct *x) { return CtB{x->d, 1, x->level, x->scale, 0}; }

extern "C" int he_add(he_ctx *c, const he_ct *a, const he_ct *b, he_ct **out)
{
    if (!c || !a || !b || !out) return HE_EINVAL;
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, a->level, a->scale, &o));
    CtB ob{o->d, 1, a->level, a->scale, 0};
    int rc = ev_add(&ev, view(a), view(b), ob, 0);
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}
extern "C" int he_sub(he_ctx *c, const he_ct *a, const he_ct *b, he_ct **out)
{
    if (!c || !a || !b || !out) return HE_EINVAL;
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, a->level, a->scale, &o));
    CtB ob{o->d, 1, a->level, a->scale, 0};
    int rc = ev_add(&ev, view(a), view(b), ob, 1);
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_mul(he_ctx *c, const he_ct *a, const he_ct *b, he_ct **out)
{
    if (!c || !a || !b || !out) return HE_EINVAL;
    Eval ev{};
    HELR_TRY(one_eval(c, a->level, &ev));
    he_ct *o = nullptr;
    int rc = helr_new_ct(c, a->level, a->scale * b->scale, &o);
    if (!rc) {
        CtB ob{o->d, 1, a->level, 0, 0};
        rc = ev_mul_relin(&ev, view(a), view(b), ob);
        if (!rc) o->scale = ob.scale;
    }
    ev_free(&ev);
    if (rc) { if (o) he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_rescale(he_ctx *c, const he_ct *a, he_ct **out)
{
    if (!c || !a || !out) return HE_EINVAL;
    if (a->level < 1) return helr_fail(c, HE_ELEVEL, "Rescale: no level left");
    Eval ev{};
    HELR_TRY(one_eval(c, a->level, &ev));
    he_ct *o = nullptr;
    int rc = helr_new_ct(c, a->level - 1, 0, &o);
    if (!rc) {
        CtB ob{o->d, 1, a->level - 1, 0, 0};
        rc = ev_rescale(&ev, view(a), ob);
        o->scale = ob.scale;
    }
    ev_free(&ev);
    if (rc) { if (o) he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_moddrop(he_ctx *c, const he_ct *a, int level, he_ct **out)
{
    if (!c || !a || !out) return HE_EINVAL;
    if (level < 0 || level > a->level) return helr_fail(c, HE_ELEVEL, "ModDrop to %d from %d", level, a->level);
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, level, a->scale, &o));
    CtB ob{o->d, 1, level, a->scale, 0};
    int rc = ev_moddrop(&ev, view(a), level, ob);
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_rotate(he_ctx *c, const he_ct *a, int64_t r, he_ct **out)
{
    if (!c || !a || !out) return HE_EINVAL;
    Eval ev{};
    HELR_TRY(one_eval(c, a->level, &ev));
    he_ct *o = nullptr;
    int rc = helr_new_ct(c, a->level, a->scale, &o);
    if (!rc) {
        CtB ob{o->d, 1, a->level, a->scale, 0};
        rc = ev_rotate(&ev, view(a), r, ob);
    }
    ev_free(&ev);
    if (rc) { if (o) he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_rotsum(he_ctx *c, const he_ct *a, const int64_t *rots, size_t n_rot, he_ct **out)
{
    if (!c || !a || !out || !rots || n_rot < 1 || n_rot > HELR_MAX_HOIST) return HE_EINVAL;
    Eval ev{};
    HELR_TRY(one_eval(c, a->level, &ev));
    he_ct *o = nullptr;
    int rc = helr_new_ct(c, a->level, a->scale, &o);
    if (!rc) {
        CtB ob{o->d, 1, a->level, a->scale, 0};
        rc = ev_rotsum(&ev, view(a), rots, (int)n_rot, ob);
    }
    ev_free(&ev);
    if (rc) { if (o) he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

// Batched Mul (with relinearisation), Rescale and Rotation on device buffers:
// `batch` ciphertexts [batch][2][level+1][N] of NTT-form words, the output
// in its own buffer (no overlap with an operand).  The scale is the caller's:
// these calls move words only.
static int batch_args(he_ctx *c, const void *in, const void *out, int batch, int level)
{
    if (!c || !in || !out || batch <= 0 || level < 0 || level >= c->nq) return HE_EINVAL;
    if (in == out) return helr_fail(c, HE_EINVAL, "the output must not overlap the input");
    return HE_OK;
}

extern "C" int he_mul_relin_batch(he_ctx *c, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out, int batch,
                                  int level)
{
    HELR_TRY(batch_args(c, d_a, d_out, batch, level));
    if (!d_b || d_b == d_out) return HE_EINVAL;
    Eval ev{};
    HELR_TRY(ev_init(c, &ev, batch, level));
    const size_t item = 2 * (size_t)(level + 1) * c->n;
    CtB a{const_cast<uint64_t *>(d_a), batch, level, 1.0, item}, b{const_cast<uint64_t *>(d_b), batch, level, 1.0, item};
    CtB o{d_out, batch, level, 0, item};
    const int rc = ev_mul_relin(&ev, a, b, o);
    ev_free(&ev);
    return rc;
}

extern "C" int he_rescale_batch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level)
{
    HELR_TRY(batch_args(c, d_in, d_out, batch, level));
    if (level < 1) return helr_fail(c, HE_ELEVEL, "Rescale: no level left");
    Eval ev{};
    HELR_TRY(ev_init(c, &ev, batch, level));
    const size_t N = c->n;
    CtB a{const_cast<uint64_t *>(d_in), batch, level, 1.0, 2 * (size_t)(level + 1) * N};
    CtB o{d_out, batch, level - 1, 0, 2 * (size_t)level * N};
    const int rc = ev_rescale(&ev, a, o);
    ev_free(&ev);
    return rc;
}

extern "C" int he_rotate_batch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level, int64_t r)
{
    HELR_TRY(batch_args(c, d_in, d_out, batch, level));
    Eval ev{};
    HELR_TRY(ev_init(c, &ev, batch, level));
    const size_t item = 2 * (size_t)(level + 1) * c->n;
    CtB a{const_cast<uint64_t *>(d_in), batch, level, 1.0, item}, o{d_out, batch, level, 1.0, item};
    const int rc = ev_rotate(&ev, a, r, o);
    ev_free(&ev);
    return rc;
}

extern "C" int he_cmul(he_ctx *c, const he_ct *a, double v, double const_scale, he_ct **out)
{
    if (!c || !a || !out || !(const_scale > 0)) return HE_EINVAL;
    double x = v * const_scale;
    if (!(fabs(x) < 9.2e18)) return helr_fail(c, HE_EINVAL, "cMul constant out of range");
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, a->level, a->scale * const_scale, &o));
    CtB ob{o->d, 1, a->level, 0, 0};
    int rc = ev_cmul_int(&ev, view(a), round_half_away(x), a->scale * const_scale, ob);
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_cadd(he_ctx *c, const he_ct *a, double v, he_ct **out)
{
    if (!c || !a || !out) return HE_EINVAL;
    double x = v * a->scale;
    if (!(fabs(x) < 9.2e18)) return helr_fail(c, HE_EINVAL, "cAdd constant out of range");
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, a->level, a->scale, &o));
    HELR_CUDA(c, cudaMemcpyAsync(o->d, a->d, sizeof(uint64_t) * 2 * (a->level + 1) * (size_t)c->n,
                                 cudaMemcpyDeviceToDevice, c->stream));
    CtB ob{o->d, 1, a->level, a->scale, 0};
    int rc = ev_cadd_int(&ev, ob, round_half_away(x));
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}

extern "C" int he_ptmul(he_ctx *c, const he_ct *a, const he_pt *pt, he_ct **out)
{
    if (!c || !a || !pt || !out) return HE_EINVAL;
    if (pt->level != a->level) return helr_fail(c, HE_ELEVEL, "plaintext level %d vs %d", pt->level, a->level);
    Eval ev{};
    ev.c = c;
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, a->level, a->scale * pt->scale, &o));
    CtB ob{o->d, 1, a->level, 0, 0};
    int rc = ev_ptmul(&ev, view(a), pt->d, pt->scale, ob);
    if (rc) { he_ct_free(o); return rc; }
    *out = o;
    return HE_OK;
}
