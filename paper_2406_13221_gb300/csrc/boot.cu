// boot.cu -- bootstrapping of the weight ciphertexts: the refresh of W and V
// that the paper performs by bootstrapping (Sec. 2.1, Sec. 4.3 Step 7).
//
// For a ciphertext at level 0 whose slot vector repeats with period n (W and V
// hold the g weights in every row of the block, Sec. 2.2), with G = N / 2n and
// Y = X^G (so the message lies in Z[Y] up to noise):
//   ModRaise    the q0 words of both polynomials as centred integers modulo
//               every prime of the chain (inverse transform, lift, forward
//               transform): the decryption becomes m + e + q0 I, I small
//               because the secret is sparse;
//   SubSum      the trace to Z[Y]: hoisted sums of the rotations by n 2^k;
//   CoeffToSlot E^-1 = E^H / n (E_jk = xi^(5^j k), xi = zeta^G) by
//               baby-step/giant-step diagonals, scaled by 1 / (2 G q0 K'),
//               split into real and imaginary parts with the conjugation
//               X -> X^-1 and the monomial X^(3N/2) (times -i);
//   EvalMod     x -> sin(2 pi K' x): the Taylor polynomial of
//               cos(2 pi (K' x - 1/4) / 2^r) on the powers of x, then r
//               double angles y -> 2 y^2 - 1 (both halves as one batch);
//   SlotToCoeff q0 E / (2 pi Delta) on y_re + i y_im (i = X^(N/2)).
// Every constant comes from +, -, *, / in a fixed order and the encoder's
// zeta table, and every step is a batched operation of the evaluator (key
// switching, rescale, products) or a transform kernel of this library.
#include <math.h>
#include <algorithm>
#include <vector>

#include "helr_internal.cuh"

namespace {

constexpr double PI = 3.141592653589793;
constexpr int SUBSUM_RHO = 3;  // the trace's rotations summed in hoisted groups of 2^3 positions

struct Plan {
    int n, K, r, deg, out_level, n1, n2;
    double Kp, delta_out;
};

// cos b and sin b by their Taylor series, summed in the order k = 0, 1, ...
void taylor_cos_sin(double b, double *cv, double *sv)
{
    double c = 0.0, s = 0.0, term = 1.0;
    for (int k = 0; k < 40; k++) {
        switch (k % 4) {
        case 0: c += term; break;
        case 1: s += term; break;
        case 2: c -= term; break;
        default: s -= term; break;
        }
        term = term * b / (double)(k + 1);
    }
    *cv = c;
    *sv = s;
}

// Taylor coefficients of cos(A x + B), A = 2 pi K' / 2^r, B = -pi / 2^(r+1)
std::vector<double> cos_coeffs(const Plan &p)
{
    const double A = 2.0 * PI * p.Kp / (double)(1 << p.r);
    const double B = -PI / (double)(1 << (p.r + 1));
    double cb, sb;
    taylor_cos_sin(B, &cb, &sb);
    const double f[4] = {cb, -sb, -cb, sb};
    std::vector<double> out;
    double a = 1.0;
    for (int k = 0; k <= p.deg; k++) {
        out.push_back(a * f[k % 4]);
        a = a * A / (double)(k + 1);
    }
    return out;
}

// E[j][k] = xi^(5^j k), xi = zeta^(N / 2n), from the encoder's zeta table
void encoding_matrix(const he_ctx *c, int n, std::vector<double> &Ere, std::vector<double> &Eim)
{
    std::vector<double> zr(2 * (size_t)c->n), zi(2 * (size_t)c->n);
    he_zeta_table(c->logn, zr.data(), zi.data());
    const uint64_t G = (uint64_t)c->n / (2 * (uint64_t)n), twon = 2ull * c->n;
    Ere.assign((size_t)n * n, 0.0);
    Eim.assign((size_t)n * n, 0.0);
    uint64_t p5 = 1;
    for (int j = 0; j < n; j++) {
        for (int k = 0; k < n; k++) {
            const uint64_t idx = (G * p5 * (uint64_t)k) % twon;
            Ere[(size_t)j * n + k] = zr[idx];
            Eim[(size_t)j * n + k] = zi[idx];
        }
        p5 = (p5 * 5) % twon;
    }
}

// device buffers of whole ciphertext batches (item stride = the top level's size)
struct Pool {
    he_ctx *c = nullptr;
    size_t item = 0;
    int batch = 0;
    std::vector<uint64_t *> bufs;
    int get(uint64_t **p)
    {
        HELR_TRY(helr_alloc(c, (void **)p, sizeof(uint64_t) * item * batch));
        bufs.push_back(*p);
        return HE_OK;
    }
    ~Pool()
    {
        for (uint64_t *p : bufs) helr_free(c, p);
    }
};

// out = a * X^k (exact): the evaluation form of the monomial times both polynomials
int monomial(Eval *ev, const CtB &a, int k, CtB &out, uint64_t *pt)
{
    he_ctx *c = ev->c;
    const int nl = a.level + 1, N = c->n;
    k %= 2 * N;
    std::vector<uint64_t> h((size_t)nl * N, 0);
    for (int j = 0; j < nl; j++) h[(size_t)j * N + (k % N)] = k < N ? 1 : c->q[j] - 1;
    HELR_CUDA(c, cudaMemcpyAsync(pt, h.data(), sizeof(uint64_t) * h.size(), cudaMemcpyHostToDevice, c->stream));
    HELR_TRY(helr_ntt_fwd(c, pt, (size_t)nl, limbmap_ct(a.level), c->stream));
    HELR_CUDA(c, cudaStreamSynchronize(c->stream));  // h leaves scope
    return ev_ptmul(ev, a, pt, 1.0, out);
}

// out = sum_r diag_r (.) Rot(a, r) for the n x n matrix M (row-major re/im)
// acting on period-n slot vectors, diag_r[k] = M[k][(k + r) mod n]; baby-step
// rotations by b < n1, giant steps by g n1 on the partial sums (diagonals
// pre-rotated right by g n1); plaintexts at pt_scale; one rescale.
int linear_transform(Eval *ev, Pool &pool, const CtB &a, int n, const std::vector<double> &Mre,
                     const std::vector<double> &Mim, double pt_scale, CtB &out)
{
    he_ctx *c = ev->c;
    const int nb = 31 - __builtin_clz((unsigned)n);
    const int n1 = 1 << ((nb + 1) / 2), n2 = n / n1, ns = c->nslots, nl = a.level + 1;
    const size_t N = c->n;
    // every diagonal, encoded at once; the plaintexts depend on the matrix, the
    // level and the scale only, so a context encodes each set once and keeps it
    uint64_t key = 1469598103934665603ull;  // FNV-1a
    auto mix = [&key](const void *p, size_t bytes) {
        const unsigned char *u = (const unsigned char *)p;
        for (size_t i = 0; i < bytes; i++) key = (key ^ u[i]) * 1099511628211ull;
    };
    mix(Mre.data(), sizeof(double) * Mre.size());
    mix(Mim.data(), sizeof(double) * Mim.size());
    mix(&pt_scale, sizeof pt_scale);
    mix(&n, sizeof n);
    mix(&nl, sizeof nl);
    uint64_t *pts = nullptr;
    for (const auto &d : c->boot_diag)
        if (d.first == key) pts = d.second;
    int rc = HE_OK;
    if (!pts) {
        std::vector<double> re((size_t)n * ns), im((size_t)n * ns);
        for (int g = 0; g < n2; g++)
            for (int b = 0; b < n1; b++) {
                const int r = g * n1 + b;
                double *zr = re.data() + (size_t)r * ns, *zi = im.data() + (size_t)r * ns;
                for (int s = 0; s < ns; s++) {
                    const int k = ((s % n) - g * n1 + n) % n;
                    zr[s] = Mre[(size_t)k * n + (k + r) % n];
                    zi[s] = Mim[(size_t)k * n + (k + r) % n];
                }
            }
        double *dz = nullptr;
        HELR_TRY(helr_alloc(c, (void **)&dz, sizeof(double) * 2 * re.size()));
        rc = helr_alloc(c, (void **)&pts, sizeof(uint64_t) * (size_t)n * nl * N);
        if (!rc) {
            cudaMemcpyAsync(dz, re.data(), sizeof(double) * re.size(), cudaMemcpyHostToDevice, c->stream);
            cudaMemcpyAsync(dz + re.size(), im.data(), sizeof(double) * im.size(), cudaMemcpyHostToDevice, c->stream);
            rc = helr_encode_dev(c, dz, dz + re.size(), n, (size_t)ns, a.level, pt_scale, pts, (size_t)nl * N);
        }
        helr_free(c, dz);
        if (rc) {
            helr_free(c, pts);
            return rc;
        }
        c->boot_diag.push_back({key, pts});
    }
    // baby steps
    std::vector<CtB> baby(n1, a);
    uint64_t *buf = nullptr;
    for (int b = 1; b < n1 && !rc; b++) {
        rc = pool.get(&buf);
        if (!rc) {
            baby[b] = CtB{buf, a.batch, 0, 0, pool.item};
            rc = ev_rotate(ev, a, b, baby[b]);
        }
    }
    uint64_t *tb = nullptr, *ib = nullptr, *rb = nullptr, *ab = nullptr;
    if (!rc) rc = pool.get(&tb);
    if (!rc) rc = pool.get(&ib);
    if (!rc) rc = pool.get(&rb);
    if (!rc) rc = pool.get(&ab);
    CtB acc{ab, a.batch, 0, 0, pool.item}, term{tb, a.batch, 0, 0, pool.item}, inner{ib, a.batch, 0, 0, pool.item},
        rot{rb, a.batch, 0, 0, pool.item};
    for (int g = 0; g < n2 && !rc; g++) {
        for (int b = 0; b < n1 && !rc; b++) {
            const uint64_t *pt = pts + (size_t)(g * n1 + b) * nl * N;
            if (b == 0) {
                rc = ev_ptmul(ev, baby[b], pt, pt_scale, inner);
            } else {
                rc = ev_ptmul(ev, baby[b], pt, pt_scale, term);
                if (!rc) rc = ev_add(ev, inner, term, inner, 0);
            }
        }
        if (rc) break;
        const CtB *part = &inner;
        if (g) {
            rc = ev_rotate(ev, inner, (int64_t)g * n1, rot);
            part = &rot;
        }
        if (!rc) rc = g ? ev_add(ev, acc, *part, acc, 0) : ev_moddrop(ev, *part, part->level, acc);
    }
    if (!rc) rc = ev_rescale(ev, acc, out);
    return rc;
}

// x (slots v / K', batch of items) -> sin(2 pi v): the cosine polynomial on the
// powers of x, r double angles
int eval_mod(Eval *ev, Pool &pool, const Plan &p, const CtB &x, CtB &y)
{
    he_ctx *c = ev->c;
    const std::vector<double> coef = cos_coeffs(p);
    std::vector<CtB> pw(p.deg + 1);
    pw[1] = x;
    uint64_t *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;
    HELR_TRY(pool.get(&b1));
    HELR_TRY(pool.get(&b2));
    HELR_TRY(pool.get(&b3));
    CtB t1{b1, x.batch, 0, 0, pool.item}, t2{b2, x.batch, 0, 0, pool.item}, t3{b3, x.batch, 0, 0, pool.item};
    for (int k = 2; k <= p.deg; k++) {
        int a = 1 << (31 - __builtin_clz((unsigned)k));
        if (a == k) a = k / 2;
        CtB u = pw[a], w = pw[k - a];
        if (u.level > w.level) {
            HELR_TRY(ev_moddrop(ev, u, w.level, t1));
            u = t1;
        } else if (w.level > u.level) {
            HELR_TRY(ev_moddrop(ev, w, u.level, t1));
            w = t1;
        }
        uint64_t *bk = nullptr;
        HELR_TRY(pool.get(&bk));
        HELR_TRY(ev_mul_relin(ev, u, w, t2));
        pw[k] = CtB{bk, x.batch, 0, 0, pool.item};
        HELR_TRY(ev_rescale(ev, t2, pw[k]));
    }
    int low = pw[1].level;
    for (int k = 2; k <= p.deg; k++) low = std::min(low, pw[k].level);
    const double target = (double)c->q[low - 1];
    CtB &acc = y;
    for (int k = 1; k <= p.deg; k++) {
        CtB xk = pw[k];
        if (xk.level != low) {
            HELR_TRY(ev_moddrop(ev, pw[k], low, t1));
            xk = t1;
        }
        // cMul at the constant scale that lands the rescaled term on `target`
        const double S = (target * (double)c->q[low]) / xk.scale;
        HELR_TRY(ev_cmul_int(ev, xk, round_half_away(coef[k] * S), xk.scale * S, t2));
        HELR_TRY(ev_rescale(ev, t2, k == 1 ? acc : t3));
        if (k == 1) {
            acc.scale = target;
        } else {
            t3.scale = target;
            HELR_TRY(ev_add(ev, acc, t3, acc, 0));
        }
    }
    HELR_TRY(ev_cadd_int(ev, acc, round_half_away(coef[0] * acc.scale)));
    for (int i = 0; i < p.r; i++) {
        HELR_TRY(ev_mul_relin(ev, acc, acc, t2));
        HELR_TRY(ev_rescale(ev, t2, t3));
        HELR_TRY(ev_cmul_int(ev, t3, 2, t3.scale, acc));
        HELR_TRY(ev_cadd_int(ev, acc, round_half_away(-1.0 * acc.scale)));
    }
    return HE_OK;
}

}  // namespace

// Bootstrap `batch` level-0 ciphertexts of period-n slot vectors (in: item
// stride in_item) into out (item stride out_item) at level p.out_level, scale
// p.delta_out.
static int helr_bootstrap(he_ctx *c, const Plan &p, const uint64_t *in, size_t in_item, int in_level, int batch,
                          uint64_t *out, size_t out_item)
{
    const int top = c->nq - 1, N = c->n, ns = c->nslots;
    const size_t item = 2 * (size_t)(top + 1) * N;
    Eval ev{};
    HELR_TRY(ev_init(c, &ev, 2 * batch, top));
    Pool pool;
    pool.c = c;
    pool.item = item;
    pool.batch = 2 * batch;  // the real and imaginary halves travel as one batch
    int rc = HE_OK;
    uint64_t *raised = nullptr, *tmp = nullptr, *pt = nullptr, *b1 = nullptr, *b2 = nullptr, *xs = nullptr, *ys = nullptr;
    if (!rc) rc = pool.get(&raised);
    if (!rc) rc = pool.get(&tmp);
    if (!rc) rc = pool.get(&b1);
    if (!rc) rc = pool.get(&b2);
    if (!rc) rc = pool.get(&xs);
    if (!rc) rc = pool.get(&ys);
    if (!rc) rc = helr_alloc(c, (void **)&pt, sizeof(uint64_t) * (size_t)(top + 1) * N);
    // ModRaise: the q0 limb of both polynomials -> coefficients -> centred lift -> all limbs
    if (!rc) {
        const size_t lw0 = (size_t)(in_level + 1) * N;
        for (int b = 0; b < batch && !rc; b++)
            for (int q = 0; q < 2 && !rc; q++)
                if (cudaMemcpyAsync(tmp + (2 * (size_t)b + q) * N, in + (size_t)b * in_item + q * lw0, sizeof(uint64_t) * N,
                                    cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                    rc = helr_fail(c, HE_ECUDA, "ModRaise copy failed");
    }
    if (!rc) rc = helr_ntt_inv(c, tmp, 2 * (size_t)batch, limbmap_single(0), c->stream);
    if (!rc) {
        k_lift(c, tmp, raised, 2 * batch, 0, N, limbmap_ct(top), (size_t)(top + 1) * N, c->stream);
        rc = helr_ntt_fwd(c, raised, 2 * (size_t)batch * (top + 1), limbmap_ct(top), c->stream);
    }
    CtB t{raised, batch, top, 1.0, item}, t2{b1, batch, 0, 0, item};
    // SubSum: the trace to Z[X^G] by hoisted groups of the rotations n 2^k
    const int bits = 31 - __builtin_clz((unsigned)(N / (2 * p.n)));
    for (int e = 0; e < bits && !rc; e += SUBSUM_RHO) {
        const int w = std::min(SUBSUM_RHO, bits - e);
        int64_t rots[HELR_MAX_HOIST];
        for (int m = 1; m < (1 << w); m++) rots[m - 1] = (int64_t)p.n * ((int64_t)m << e);
        rc = ev_rotsum(&ev, t, rots, (1 << w) - 1, t2);
        std::swap(t, t2);
    }
    // CoeffToSlot: u = E^H / (2 n G q0 K') z, then the real and imaginary parts
    std::vector<double> Ere, Eim;
    encoding_matrix(c, p.n, Ere, Eim);
    const int n = p.n, G = N / (2 * n);
    const double cs = 1.0 / (2.0 * (double)n * (double)G * (double)c->q[0] * p.Kp);
    std::vector<double> Mre((size_t)n * n), Mim((size_t)n * n);
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++) {
            Mre[(size_t)k * n + j] = Ere[(size_t)j * n + k] * cs;
            Mim[(size_t)k * n + j] = -Eim[(size_t)j * n + k] * cs;
        }
    CtB u{b2, batch, 0, 0, item};
    const double s_x = (double)c->q[top - 1];
    if (!rc) rc = linear_transform(&ev, pool, t, n, Mre, Mim, (double)c->q[top] * s_x, u);
    u.scale = s_x;
    // x_re in items 0..batch-1 of xs, x_im in items batch..2 batch-1
    CtB uc{tmp, batch, 0, 0, item}, xre{xs, batch, 0, 0, item}, xim{xs + (size_t)batch * item, batch, 0, 0, item};
    if (!rc) rc = ev_rotate_gal(&ev, u, 2ull * N - 1, uc, 0);
    if (!rc) rc = ev_add(&ev, u, uc, xre, 0);
    CtB d{b1, batch, 0, 0, item};
    if (!rc) rc = ev_add(&ev, u, uc, d, 1);
    if (!rc) rc = monomial(&ev, d, 3 * N / 2, xim, pt);
    // EvalMod on both halves as one batch
    CtB x{xs, 2 * batch, xre.level, xre.scale, item}, y{ys, 2 * batch, 0, 0, item};
    if (!rc) rc = eval_mod(&ev, pool, p, x, y);
    // SlotToCoeff: q0 E / (2 pi Delta) on y_re + i y_im
    CtB yre{ys, batch, y.level, y.scale, item}, yim{ys + (size_t)batch * item, batch, y.level, y.scale, item};
    CtB iy{tmp, batch, 0, 0, item}, ysum{b1, batch, 0, 0, item};
    if (!rc) rc = monomial(&ev, yim, N / 2, iy, pt);
    if (!rc) rc = ev_add(&ev, yre, iy, ysum, 0);
    const double c2 = (double)c->q[0] / (2.0 * PI * p.delta_out);
    std::vector<double> M2re((size_t)n * n), M2im((size_t)n * n);
    for (size_t i = 0; i < M2re.size(); i++) M2re[i] = Ere[i] * c2, M2im[i] = Eim[i] * c2;
    CtB res{b2, batch, 0, 0, item};
    if (!rc) rc = linear_transform(&ev, pool, ysum, n, M2re, M2im, p.delta_out * (double)c->q[ysum.level] / ysum.scale, res);
    res.scale = p.delta_out;
    if (!rc && res.level < p.out_level)
        rc = helr_fail(c, HE_ELEVEL, "the bootstrap ends at level %d, below %d", res.level, p.out_level);
    CtB o{out, batch, 0, 0, out_item};
    if (!rc) rc = ev_moddrop(&ev, res, p.out_level, o);
    if (!rc) HELR_CUDA(c, cudaStreamSynchronize(c->stream));
    helr_free(c, pt);
    ev_free(&ev);
    (void)ns;
    return rc;
}

static int plan_of(he_ctx *c, const he_boot_params *bp, Plan *p)
{
    if (!bp || bp->slots < 1 || (bp->slots & (bp->slots - 1)) || bp->slots > c->nslots || bp->K < 1 ||
        bp->double_angles < 0 || bp->double_angles > 20 || bp->degree < 2 || bp->degree > 63 || !(bp->scale_out > 0) ||
        bp->level_out < 0)
        return helr_fail(c, HE_EINVAL, "bootstrap parameters out of range");
    p->n = bp->slots;
    p->K = bp->K;
    p->r = bp->double_angles;
    p->deg = bp->degree;
    p->Kp = (double)bp->K + 0.5;
    p->delta_out = bp->scale_out;
    p->out_level = bp->level_out;
    const int nb = 31 - __builtin_clz((unsigned)p->n);
    p->n1 = 1 << ((nb + 1) / 2);
    p->n2 = p->n / p->n1;
    const int depth = 1 + (32 - __builtin_clz((unsigned)(p->deg - 1))) + 1 + p->r + 1;
    if (c->nq - 1 - depth < p->out_level)
        return helr_fail(c, HE_ELEVEL, "the chain's %d levels hold a bootstrap of depth %d above level %d only",
                         c->nq - 1, depth, c->nq - 1 - depth);
    return HE_OK;
}

extern "C" int he_boot_keys(he_ctx *c, const he_boot_params *bp, int64_t *rots, size_t cap, size_t *n_rots)
{
    if (!c || !n_rots) return HE_EINVAL;
    Plan p;
    HELR_TRY(plan_of(c, bp, &p));
    std::vector<int64_t> r;
    const int bits = 31 - __builtin_clz((unsigned)(c->n / (2 * p.n)));
    for (int e = 0; e < bits; e += SUBSUM_RHO)
        for (int m = 1; m < (1 << std::min(SUBSUM_RHO, bits - e)); m++) r.push_back((int64_t)p.n * ((int64_t)m << e));
    for (int b = 1; b < p.n1; b++) r.push_back(b);
    for (int g = 1; g < p.n2; g++) r.push_back((int64_t)g * p.n1);
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    *n_rots = r.size();
    if (rots)
        for (size_t i = 0; i < r.size() && i < cap; i++) rots[i] = r[i];
    return HE_OK;
}

extern "C" int he_bootstrap(he_ctx *c, const he_ct *in, const he_boot_params *bp, he_ct **out)
{
    if (!c || !in || !out) return HE_EINVAL;
    Plan p;
    HELR_TRY(plan_of(c, bp, &p));
    he_ct *o = nullptr;
    HELR_TRY(helr_new_ct(c, p.out_level, p.delta_out, &o));
    const int rc = helr_bootstrap(c, p, in->d, 0, in->level, 1, o->d, 0);
    if (rc) {
        he_ct_free(o);
        return rc;
    }
    *out = o;
    return HE_OK;
}

extern "C" int he_bootstrap_batch(he_ctx *c, const uint64_t *d_in, int in_level, uint64_t *d_out, int batch,
                                  const he_boot_params *bp)
{
    if (!c || !d_in || !d_out || batch < 1 || in_level < 0 || in_level >= c->nq) return HE_EINVAL;
    Plan p;
    HELR_TRY(plan_of(c, bp, &p));
    return helr_bootstrap(c, p, d_in, 2 * (size_t)(in_level + 1) * c->n, in_level, batch, d_out,
                          2 * (size_t)(p.out_level + 1) * c->n);
}
