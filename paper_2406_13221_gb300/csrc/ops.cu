// ops.cu -- elementwise and structural kernels of the scheme (Sec. 2.1 operations)
//
// All ciphertext kernels work on evaluation-form limbs ([..][limb][N] words)
// except the lifts, which read coefficient-form limbs produced by an inverse
// transform.  Words move as 16-byte pairs (two coefficients per thread).
#include "helr_internal.cuh"

#define GS_LOOP(i, n) for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

namespace {

inline unsigned grid_for(size_t work, int threads = 256)
{
    size_t b = (work + threads - 1) / threads;
    if (b > (size_t)152 * 64) b = (size_t)152 * 64;
    return (unsigned)(b ? b : 1);
}

__global__ void k_add_kernel(uint64_t *out, const uint64_t *a, const uint64_t *b, size_t npairs, int half_n,
                             const ModQ *mods, LimbMap lm, int sub)
{
    GS_LOOP(i, npairs) {
        size_t limb = i / half_n;
        uint64_t q = mods[limb_prime(lm, limb)].q;
        ulonglong2 x = reinterpret_cast<const ulonglong2 *>(a)[i];
        ulonglong2 y = reinterpret_cast<const ulonglong2 *>(b)[i];
        ulonglong2 z;
        if (sub) { z.x = submod(x.x, y.x, q); z.y = submod(x.y, y.y, q); }
        else { z.x = addmod(x.x, y.x, q); z.y = addmod(x.y, y.y, q); }
        reinterpret_cast<ulonglong2 *>(out)[i] = z;
    }
}

__global__ void k_mul_kernel(uint64_t *out, const uint64_t *a, const uint64_t *b, size_t npairs, int half_n,
                             const ModQ *mods, LimbMap lm)
{
    GS_LOOP(i, npairs) {
        size_t limb = i / half_n;
        ModQ m = mods[limb_prime(lm, limb)];
        ulonglong2 x = reinterpret_cast<const ulonglong2 *>(a)[i];
        ulonglong2 y = reinterpret_cast<const ulonglong2 *>(b)[i];
        ulonglong2 z;
        z.x = mulmod(x.x, y.x, m);
        z.y = mulmod(x.y, y.y, m);
        reinterpret_cast<ulonglong2 *>(out)[i] = z;
    }
}

// (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1); a, b: items of [2][L][N]; d_i at d + item * d_stride + i * d_poly.
// grid: (N/2 / 256, limbs, items)
__global__ void k_tensor_kernel(const uint64_t *a, const uint64_t *b, uint64_t *d, int half_n, int nl, size_t a_stride,
                                size_t b_stride, size_t d_stride, size_t d_poly, const ModQ *mods)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= half_n) return;
    const int limb = blockIdx.y;
    const size_t bt = blockIdx.z;
    const ModQ m = mods[limb];
    const size_t per = (size_t)nl * half_n, r = (size_t)limb * half_n + w;
    const ulonglong2 *A = reinterpret_cast<const ulonglong2 *>(a + bt * a_stride);
    const ulonglong2 *B = reinterpret_cast<const ulonglong2 *>(b + bt * b_stride);
    ulonglong2 a0 = A[r], a1 = A[per + r], b0 = B[r], b1 = B[per + r];
    ulonglong2 o0, o1, o2;
    o0.x = mulmod(a0.x, b0.x, m); o0.y = mulmod(a0.y, b0.y, m);
    o1.x = addmod(mulmod(a0.x, b1.x, m), mulmod(a1.x, b0.x, m), m.q);
    o1.y = addmod(mulmod(a0.y, b1.y, m), mulmod(a1.y, b0.y, m), m.q);
    o2.x = mulmod(a1.x, b1.x, m); o2.y = mulmod(a1.y, b1.y, m);
    reinterpret_cast<ulonglong2 *>(d + bt * d_stride)[r] = o0;
    reinterpret_cast<ulonglong2 *>(d + bt * d_stride + d_poly)[r] = o1;
    reinterpret_cast<ulonglong2 *>(d + bt * d_stride + 2 * d_poly)[r] = o2;
}

// out = in * k_j (Shoup pair per limb position j = limb % period)
__global__ void k_cmul_kernel(uint64_t *out, const uint64_t *in, const uint64_t *kp, size_t npairs, int half_n,
                              int period, const ModQ *mods)
{
    GS_LOOP(i, npairs) {
        int j = (int)((i / half_n) % period);
        uint64_t q = mods[j].q, w = kp[2 * j], wp = kp[2 * j + 1];
        ulonglong2 x = reinterpret_cast<const ulonglong2 *>(in)[i];
        x.x = shoup(x.x, w, wp, q);
        x.y = shoup(x.y, w, wp, q);
        reinterpret_cast<ulonglong2 *>(out)[i] = x;
    }
}

// c0 += k_j in every evaluation (adding a constant polynomial)
__global__ void k_cadd_kernel(uint64_t *c0, const uint64_t *kv, size_t npairs, int half_n, int nl, size_t stride,
                              const ModQ *mods)
{
    GS_LOOP(i, npairs) {
        size_t per = (size_t)nl * half_n;
        size_t bt = i / per, r = i % per;
        int j = (int)(r / half_n);
        uint64_t q = mods[j].q, k = kv[j];
        ulonglong2 *p = reinterpret_cast<ulonglong2 *>(c0 + bt * stride) + r;
        ulonglong2 x = *p;
        x.x = addmod(x.x, k, q);
        x.y = addmod(x.y, k, q);
        *p = x;
    }
}

// evaluation-form automorphism X -> X^g: position p holds the evaluation at
// psi^(2 bitrev(p) + 1); a(X^g) there equals a at psi^((2 bitrev(p) + 1) g).
__global__ void k_automorph_kernel(uint64_t *out, const uint64_t *in, size_t nwords, int logn, uint64_t gal)
{
    const uint64_t mask2n = (2ull << logn) - 1;
    const int n = 1 << logn;
    GS_LOOP(i, nwords) {
        size_t limb = i >> logn;
        uint32_t p = (uint32_t)(i & (n - 1));
        uint32_t k = __brev(p) >> (32 - logn);
        uint64_t e = ((2ull * k + 1) * gal) & mask2n;
        uint32_t ks = (uint32_t)((e - 1) >> 1);
        uint32_t ps = __brev(ks) >> (32 - logn);
        out[i] = in[(limb << logn) + ps];
    }
}

// out[b][t][k] = centred(in[b][k] mod q_src) reduced mod prime(t), t < dst.period; grid (N / 256, ndst, items)
__global__ void k_lift_kernel(const uint64_t *in, uint64_t *out, int n, int src_prime, size_t in_stride,
                              size_t out_stride, const ModQ *mods, LimbMap dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int t = blockIdx.y;
    const size_t bt = blockIdx.z;
    const ModQ mt = mods[map_prime(dst, t)];
    out[bt * out_stride + (size_t)t * n + k] = lift_centered(in[bt * in_stride + k], mods[src_prime].q, mt);
}


// grid: (N/2 / 256, npoly * nl, items)
__global__ void k_ew_kernel(int op, Str out, Str a, Str b, int half_n, int nl, const KP kp, const ModQ *mods)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= half_n) return;
    const int pl = blockIdx.y / nl, j = blockIdx.y % nl;
    const size_t bt = blockIdx.z;
    const ModQ m = mods[j];
    const size_t off = 2 * ((size_t)j * half_n + w);
    ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a.p + bt * a.item + pl * a.poly + off);
    ulonglong2 z;
    if (op == EW_COPY) {
        z = x;
    } else if (op == EW_NEG) {
        z.x = x.x ? m.q - x.x : 0;
        z.y = x.y ? m.q - x.y : 0;
    } else if (op == EW_CMUL) {
        uint64_t wv = kp.w[j][0], wp = kp.w[j][1];
        z.x = shoup(x.x, wv, wp, m.q);
        z.y = shoup(x.y, wv, wp, m.q);
    } else if (op == EW_CADD) {
        z.x = addmod(x.x, kp.w[j][0], m.q);
        z.y = addmod(x.y, kp.w[j][0], m.q);
    } else {
        ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(b.p + bt * b.item + pl * b.poly + off);
        if (op == EW_SUBMUL) {
            uint64_t wv = kp.w[j][0], wp = kp.w[j][1];
            z.x = shoup(submod(x.x, y.x, m.q), wv, wp, m.q);
            z.y = shoup(submod(x.y, y.y, m.q), wv, wp, m.q);
        } else if (op == EW_ADD) {
            z.x = addmod(x.x, y.x, m.q);
            z.y = addmod(x.y, y.y, m.q);
        } else if (op == EW_SUB) {
            z.x = submod(x.x, y.x, m.q);
            z.y = submod(x.y, y.y, m.q);
        } else {
            z.x = mulmod(x.x, y.x, m);
            z.y = mulmod(x.y, y.y, m);
        }
    }
    *reinterpret_cast<ulonglong2 *>(out.p + bt * out.item + pl * out.poly + off) = z;
}

// grid: (N / 256, nl, items)
__global__ void k_automorph_items_kernel(uint64_t *out, size_t out_item, const uint64_t *in, size_t in_item, int logn,
                                         uint64_t gal)
{
    const int n = 1 << logn;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const size_t limb = blockIdx.y, bt = blockIdx.z;
    const uint64_t mask2n = (2ull << logn) - 1;
    uint32_t k = __brev((uint32_t)p) >> (32 - logn);
    uint64_t e = ((2ull * k + 1) * gal) & mask2n;
    uint32_t ks = (uint32_t)((e - 1) >> 1);
    uint32_t ps = __brev(ks) >> (32 - logn);
    out[bt * out_item + (limb << logn) + p] = in[bt * in_item + (limb << logn) + ps];
}

}  // namespace

// ------------------------------------------------------------------ launchers
void k_ew(he_ctx *c, int op, Str out, Str a, Str b, int batch, int npoly, int nl, const KP *kp, cudaStream_t s)
{
    static const KP zero = {};
    const int hn = c->n / 2;
    dim3 grid((hn + 255) / 256, npoly * nl, batch);
    if (batch && npoly && nl) HELR_LAUNCH(k_ew_kernel<<<grid, 256, 0, s>>>(op, out, a, b, hn, nl, kp ? *kp : zero, c->t.mod));
}
void k_automorph_items(he_ctx *c, uint64_t *out, size_t out_item, const uint64_t *in, size_t in_item, int batch, int nl,
                       uint64_t gal, cudaStream_t s)
{
    dim3 grid((c->n + 255) / 256, nl, batch);
    if (batch && nl) HELR_LAUNCH(k_automorph_items_kernel<<<grid, 256, 0, s>>>(out, out_item, in, in_item, c->logn, gal));
}
void k_add(he_ctx *c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t nlimbs, const LimbMap &m, int sub, cudaStream_t s)
{
    size_t np = nlimbs * (size_t)(c->n / 2);
    if (np) HELR_LAUNCH(k_add_kernel<<<grid_for(np), 256, 0, s>>>(out, a, b, np, c->n / 2, c->t.mod, m, sub));
}
void k_mul(he_ctx *c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t nlimbs, const LimbMap &m, cudaStream_t s)
{
    size_t np = nlimbs * (size_t)(c->n / 2);
    if (np) HELR_LAUNCH(k_mul_kernel<<<grid_for(np), 256, 0, s>>>(out, a, b, np, c->n / 2, c->t.mod, m));
}
void k_tensor(he_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *d, int batch, int level,
              size_t a_stride, size_t b_stride, size_t d_stride, size_t d_poly, cudaStream_t s)
{
    const int hn = c->n / 2;
    dim3 grid((hn + 255) / 256, level + 1, batch);
    if (batch) HELR_LAUNCH(k_tensor_kernel<<<grid, 256, 0, s>>>(a, b, d, hn, level + 1, a_stride, b_stride, d_stride, d_poly, c->t.mod));
}
void k_cmul_const(he_ctx *c, uint64_t *out, const uint64_t *in, const uint64_t *kp, size_t nlimbs, int period, cudaStream_t s)
{
    size_t np = nlimbs * (size_t)(c->n / 2);
    if (np) HELR_LAUNCH(k_cmul_kernel<<<grid_for(np), 256, 0, s>>>(out, in, kp, np, c->n / 2, period, c->t.mod));
}
void k_cadd_const(he_ctx *c, uint64_t *ct0, const uint64_t *kv, int batch, int level, size_t stride, cudaStream_t s)
{
    size_t np = (size_t)batch * (level + 1) * (c->n / 2);
    if (np) HELR_LAUNCH(k_cadd_kernel<<<grid_for(np), 256, 0, s>>>(ct0, kv, np, c->n / 2, level + 1, stride, c->t.mod));
}
void k_automorph(he_ctx *c, uint64_t *out, const uint64_t *in, size_t nlimbs, uint64_t gal, cudaStream_t s)
{
    size_t nw = nlimbs << c->logn;
    if (nw) HELR_LAUNCH(k_automorph_kernel<<<grid_for(nw), 256, 0, s>>>(out, in, nw, c->logn, gal));
}
void k_lift(he_ctx *c, const uint64_t *in, uint64_t *out, int batch, int src_prime, size_t in_stride,
            const LimbMap &dst, size_t out_stride, cudaStream_t s)
{
    dim3 grid((c->n + 255) / 256, dst.period, batch);
    if (batch) HELR_LAUNCH(k_lift_kernel<<<grid, 256, 0, s>>>(in, out, c->n, src_prime, in_stride, out_stride, c->t.mod, dst));
}
