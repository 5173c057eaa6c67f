// helr_internal.cuh -- shared declarations of the GB300 library (not installed).
//
// Ciphertexts live on the device in evaluation (NTT) form, limb-major:
// [poly][limb][N] uint64 words, limb j reduced modulo q_j.  All ciphertext
// arithmetic is exact modular integer arithmetic on 64-bit words with primes
// below 2^60.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <vector>
#include <map>
#include <memory>
#include <atomic>

#include "../../include/he_lr.h"

#define HELR_MAXQ 40      // ciphertext primes + special prime
#define HELR_MAX_LOGN 16
#define HELR_MIN_LOGN 10

// ------------------------------------------------------------------ modular arithmetic
// Per-prime constants.  Barrett: s = bits(q) - 2, mu = floor(2^(s+64) / q) < 2^63.
// Montgomery: qinv = q^-1 mod 2^64 (R = 2^64).
struct ModQ {
    uint64_t q;
    uint64_t mu;
    uint32_t s;
    uint32_t pad;
    uint64_t qinv;
};

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// x mod q for x = hi*2^64 + lo < q^2 (or any x < 2^64 with hi = 0); result in [0, q).
__host__ __device__ __forceinline__ uint64_t barrett_reduce(uint64_t hi, uint64_t lo, const ModQ m)
{
    uint64_t y = m.s ? ((hi << (64 - m.s)) | (lo >> m.s)) : lo;
    uint64_t qh = mulhi64(y, m.mu);
    uint64_t r = lo - qh * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}
__host__ __device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b, const ModQ m)
{
    return barrett_reduce(mulhi64(a, b), a * b, m);
}
__host__ __device__ __forceinline__ uint64_t reduce64(uint64_t x, const ModQ m) { return barrett_reduce(0, x, m); }
// Montgomery product a * b * 2^-64 mod q for a, b < q: with a b = hi 2^64 + lo and
// m = lo q^-1 mod 2^64, a b - m q is divisible by 2^64 and equals (hi - mulhi(m, q)) 2^64.
// With b stored as b' = b 2^64 mod q it returns a b mod q.
__host__ __device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, const ModQ m)
{
    uint64_t lo = a * b, hi = mulhi64(a, b);
    uint64_t mh = mulhi64(lo * m.qinv, m.q);
    return hi >= mh ? hi - mh : hi - mh + m.q;
}
__host__ __device__ __forceinline__ uint64_t addmod(uint64_t a, uint64_t b, uint64_t q)
{
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}
__host__ __device__ __forceinline__ uint64_t submod(uint64_t a, uint64_t b, uint64_t q)
{
    return a >= b ? a - b : a + (q - b);
}
// Shoup product with a fixed operand w < q and wp = floor(w 2^64 / q):
// returns w*y mod q up to one q, i.e. a value in [0, 2q), for any 64-bit y.
__host__ __device__ __forceinline__ uint64_t shoup_lazy(uint64_t y, uint64_t w, uint64_t wp, uint64_t q)
{
    return w * y - mulhi64(wp, y) * q;
}
__host__ __device__ __forceinline__ uint64_t shoup(uint64_t y, uint64_t w, uint64_t wp, uint64_t q)
{
    uint64_t r = shoup_lazy(y, w, wp, q);
    return r >= q ? r - q : r;
}
// centred representative of x in [0, qi) reduced into [0, qt); the Barrett
// reduction is skipped when the magnitude is already below qt
__host__ __device__ __forceinline__ uint64_t lift_centered(uint64_t x, uint64_t qi, const ModQ t)
{
    if (x > (qi >> 1)) {
        uint64_t neg = qi - x;
        if (neg >= t.q) neg = reduce64(neg, t);
        return neg ? t.q - neg : 0;
    }
    return x < t.q ? x : reduce64(x, t);
}

// ------------------------------------------------------------------ limb maps
// Limb i of a batch uses prime index p[i % period] (index nq means the special prime P).
struct LimbMap {
    int period;
    unsigned char p[HELR_MAXQ + 2];
};

// ------------------------------------------------------------------ launch accounting
// Every kernel launch of the library goes through HELR_LAUNCH, which counts it.
extern std::atomic<unsigned long long> g_helr_launches;
#define HELR_LAUNCH(...)                                                  \
    do {                                                                  \
        g_helr_launches.fetch_add(1, std::memory_order_relaxed);          \
        __VA_ARGS__;                                                      \
    } while (0)

// Optional per-class kernel timing with CUDA events on the context stream.
// PROF_KS spans whole key switches (it overlaps the kernel classes): units =
// key switches, units2 = their summed limb counts, units3 = algorithmic DRAM
// limbs of a key switch at L limbs (input limb read, two output limbs written:
// 3L per item; the 2L(L+1) key limbs once per wave).
enum { PROF_NTT_FWD = 0, PROF_NTT_INV = 1, PROF_MODUP = 2, PROF_KS_INNER = 3, PROF_KS = 4, PROF_NCLASS = 5 };
struct ProfClass {
    std::vector<cudaEvent_t> ev;  // start/stop pairs
    size_t used = 0;
    double units = 0;             // work units (limbs for transforms)
    double units2 = 0;            // second work count (multiply-accumulate limbs of the key inner product)
    double units3 = 0;            // algorithmic DRAM limbs (reads + writes, shared operands once per launch)
    unsigned long long launches = 0;
};
struct Prof {
    int on = 0;
    ProfClass cls[PROF_NCLASS];
    double ks_by_limbs[HELR_MAXQ + 2] = {};  // key switches issued per input limb count
};
struct he_ctx;
void prof_start(he_ctx *c, int cls, cudaStream_t s);
void prof_stop(he_ctx *c, int cls, cudaStream_t s, double units, int launches, double units2 = 0, double units3 = 0);

// prime index of limb `limb` (an unrolled select: a dynamic index into a kernel
// parameter array would force the array into local memory)
__device__ __forceinline__ int limb_prime(const LimbMap &lm, size_t limb)
{
    const int i = (int)(limb % (size_t)lm.period);
    int v = lm.p[0];
#pragma unroll
    for (int k = 1; k < HELR_MAXQ + 2; k++)
        if (k == i) v = lm.p[k];
    return v;
}
__device__ __forceinline__ int map_prime(const LimbMap &lm, int i)
{
    int v = lm.p[0];
#pragma unroll
    for (int k = 1; k < HELR_MAXQ + 2; k++)
        if (k == i) v = lm.p[k];
    return v;
}

// A subset of the positions 0..period-1 of a limb map, ascending.  Transforms
// are launched once per subset of primes that share a butterfly form: primes
// below HELR_LZ_QMAX take the unreduced forward butterfly, larger ones Harvey's.
constexpr uint64_t HELR_LZ_QMAX = 1ull << 58;
struct PosList {
    int n;
    unsigned char pos[HELR_MAXQ + 2];
};
__device__ __forceinline__ int pos_at(const PosList &pl, int k)
{
    int v = pl.pos[0];
#pragma unroll
    for (int j = 1; j < HELR_MAXQ + 2; j++)
        if (j == k) v = pl.pos[j];
    return v;
}

// ------------------------------------------------------------------ error state
struct HeError {
    int code;
    std::string msg;
};

// ------------------------------------------------------------------ device tables per prime
struct DevTables {
    ModQ *mod;          // [nprime]
    uint64_t *tw;       // [nprime][N][2]  forward (psi_rev, shoup)
    uint64_t *itw;      // [nprime][N][2]  inverse (psi^-1 rev, shoup)
    uint64_t *ninv;     // [nprime][2]     N^-1 and its Shoup companion
    double *zeta;       // [2N][2]         exp(i pi k / N)
    int *sidx;          // [N/2]           slot j -> DFT index
    uint64_t *cdt;      // [cdt_len]
};

struct KeySwitchKey {
    uint64_t gal;       // 0 = relinearisation
    uint64_t *d;        // [nq digits][2][nq+1 limbs][N], evaluation form, Montgomery form (k 2^64 mod q),
                        // words reordered inside each transform row as k_ks_inner_rows reads them
};

struct he_ctx {
    int logn, n, nslots, nq;       // nq ciphertext primes q_0..q_{nq-1}
    int nprime;                    // nq + 1 (index nq = P)
    uint64_t q[HELR_MAXQ + 1];
    ModQ modh[HELR_MAXQ + 1];
    uint64_t psi[HELR_MAXQ + 1];
    double sigma;
    int cdt_len;
    uint64_t cdt_host[64];
    cudaStream_t stream;
    DevTables t;
    // inverse constants for rescale / ModDown (Shoup pairs), host copies
    // qinv[l][j] = q_l^-1 mod q_j, pinv[j] = P^-1 mod q_j
    uint64_t *d_qinv;              // [nq][nq][2]
    uint64_t *d_pinv;              // [nq][2]
    // keys
    int have_keys;
    uint64_t key_seed;
    int64_t *h_sk;                 // host copy of the ternary secret (client side)
    uint64_t *d_sk;                // [nprime][N] NTT form
    uint64_t *d_pk;                // [2][nq][N] NTT form
    std::vector<KeySwitchKey> ksk;
    HeError err;
    Prof prof;
    int ks_wave = 0;               // items per fused key-switch wave forced by HELR_KS_WAVE (0 = none)
    int ks_wave_tab[HELR_MAXQ + 1] = {};  // wave per limb count chosen by he_autotune (0 = default)
    int ks_tile = -1;              // tile variant forced by he_set_ks_tile (-1 = none)
    int ks_tile_tab[HELR_MAXQ + 1] = {};  // tile variant per limb count chosen by he_autotune
    int rot_radix_log = 3;         // rotate-and-sum steps as hoisted groups of 2^rot_radix_log positions
    int secret_hw = 0;             // 0: dense ternary secret; h > 0: exactly h nonzero coefficients
    int sms = 152;                 // SMs of the device (grid sizing)
    int hoist_form = -1;           // hoisted inner product forced: 0 CUDA cores, 1 tensor cores; -1 tuned
    int hoist_form_tab[HELR_MAXQ + 1] = {};  // the form per limb count chosen by he_autotune (0 by default)
    unsigned long long hoist_tensor_launches = 0;
    int *d_status = nullptr;       // device failure bits (bit 0: a bounded wait expired), he_check_device
    // encoded diagonal plaintexts of the bootstrap's linear transforms, keyed by
    // a hash of the matrix, the level, the plaintext scale and the slot period
    std::vector<std::pair<uint64_t, uint64_t *>> boot_diag;
};

struct he_ct {
    he_ctx *ctx;
    int level;
    double scale;
    uint64_t *d;    // [2][level+1][N]
};
struct he_pt {
    he_ctx *ctx;
    int level;
    double scale;
    uint64_t *d;    // [level+1][N] NTT form
};

// ------------------------------------------------------------------ helpers (host)
int helr_fail(he_ctx *c, int code, const char *fmt, ...);
#define HELR_CUDA(c, call)                                                              \
    do {                                                                                \
        cudaError_t e__ = (call);                                                       \
        if (e__ != cudaSuccess)                                                         \
            return helr_fail((c), HE_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,  \
                             cudaGetErrorString(e__));                                  \
    } while (0)
#define HELR_TRY(x)                      \
    do {                                 \
        int rc__ = (x);                  \
        if (rc__ != HE_OK) return rc__;  \
    } while (0)

int helr_alloc(he_ctx *c, void **p, size_t bytes);
void helr_free(he_ctx *c, void *p);

static inline LimbMap limbmap_ct(int level)
{
    LimbMap m;
    m.period = level + 1;
    for (int j = 0; j <= level; j++) m.p[j] = (unsigned char)j;
    return m;
}
static inline LimbMap limbmap_single(int prime)
{
    LimbMap m;
    m.period = 1;
    m.p[0] = (unsigned char)prime;
    return m;
}

// positions of a limb map whose prime takes the unreduced forward butterfly
// (lazy) or Harvey's (!lazy)
static inline PosList poslist_of(const he_ctx *c, const LimbMap &m, bool lazy)
{
    PosList pl{};
    for (int j = 0; j < m.period; j++)
        if ((c->q[m.p[j]] < HELR_LZ_QMAX) == lazy) pl.pos[pl.n++] = (unsigned char)j;
    return pl;
}
// number of limbs l < nlimbs with l mod period in pl
static inline size_t poslist_count(const PosList &pl, size_t nlimbs, int period)
{
    size_t n = nlimbs / (size_t)period * (size_t)pl.n;
    const int rem = (int)(nlimbs % (size_t)period);
    for (int j = 0; j < pl.n; j++) n += pl.pos[j] < rem;
    return n;
}

// ------------------------------------------------------------------ kernels (launchers)
// NTT over a batch of limbs: data [nlimbs][N]; values in [0, q) in and out.
int helr_ntt_fwd(he_ctx *c, uint64_t *data, size_t nlimbs, const LimbMap &m, cudaStream_t s);
int helr_ntt_inv(he_ctx *c, uint64_t *data, size_t nlimbs, const LimbMap &m, cudaStream_t s);
// out-of-place variants (in may equal out)
int helr_ntt_fwd_oop(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s);
int helr_ntt_inv_oop(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s);
// row pass of the inverse transform only (see ntt.cu)
// (input limb k is read at in + (k / per_item) in_item + (k % per_item) in_poly)
int helr_ntt_inv_rows(he_ctx *c, const uint64_t *in, size_t in_item, size_t in_poly, uint64_t *out, size_t nlimbs,
                      const LimbMap &m, cudaStream_t s, int per_item = 2);

// elementwise / structural kernels (ops.cu)
void k_add(he_ctx *c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t nlimbs, const LimbMap &m, int sub, cudaStream_t s);
void k_mul(he_ctx *c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t nlimbs, const LimbMap &m, cudaStream_t s);
void k_tensor(he_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *d, int batch, int level,
              size_t a_stride, size_t b_stride, size_t d_stride, size_t d_poly_stride, cudaStream_t s);
void k_cmul_const(he_ctx *c, uint64_t *out, const uint64_t *in, const uint64_t *kpairs_dev,
                  size_t nlimbs, int period, cudaStream_t s);
void k_cadd_const(he_ctx *c, uint64_t *ct0, const uint64_t *kvals_dev, int batch, int level,
                  size_t stride, cudaStream_t s);
void k_automorph(he_ctx *c, uint64_t *out, const uint64_t *in, size_t nlimbs, uint64_t gal, cudaStream_t s);
void k_lift(he_ctx *c, const uint64_t *in, uint64_t *out, int batch, int src_prime, size_t in_stride,
            const LimbMap &dst, size_t out_stride, cudaStream_t s);

// strided elementwise kernel: element (item b, poly p, limb j, k) of X lives at
// X.p + b * X.item + p * X.poly + j * N + k (limb j reduced modulo q_j)
struct Str {
    uint64_t *p;
    size_t item, poly;
};
enum { EW_ADD = 0, EW_SUB = 1, EW_MUL = 2, EW_CMUL = 3, EW_COPY = 4, EW_NEG = 5, EW_CADD = 6, EW_SUBMUL = 7 };
// per-limb constants passed by value: Shoup pairs (w, w') for EW_CMUL / EW_SUBMUL, w alone for EW_CADD
struct KP {
    uint64_t w[HELR_MAXQ + 1][2];
};
void k_ew(he_ctx *c, int op, Str out, Str a, Str b, int batch, int npoly, int nl, const KP *kp, cudaStream_t s);
void k_automorph_items(he_ctx *c, uint64_t *out, size_t out_item, const uint64_t *in, size_t in_item, int batch, int nl,
                       uint64_t gal, cudaStream_t s);

struct KsScratch {
    uint64_t *base, *drow, *ext, *acc, *pl, *lift;  // drow: input after the inverse row pass
    int batch, level;
    int wave;        // items per wave forced for every call (0: helr_ks_wave of the call's limb count)
    size_t ext_cap;  // words of ext: a wave of w items at nl limbs needs w nl (nl + 1) N
};
int helr_ks_fused(he_ctx *c, const uint64_t *dntt, const uint64_t *drow, uint64_t *mid, const uint64_t *key, uint64_t *acc,
                  int items, int nl, cudaStream_t s);
// items per fused key-switch wave at nl limbs: HELR_KS_WAVE, else the
// he_autotune table, else 128 (autotune.cu)
int helr_ks_wave(const he_ctx *c, int nl);
// tile variant of the key-switch kernels at nl limbs (bit 0: narrower column
// CTAs, bit 1: fewer rows per row CTA): he_set_ks_tile, else the he_autotune
// table, else 0 (autotune.cu)
int helr_ks_tile(const he_ctx *c, int nl);
// the hoisted inner product's form at nl limbs (0 CUDA cores, 1 tensor cores)
int helr_hoist_form(const he_ctx *c, int nl);
int helr_ks_scratch_alloc(he_ctx *c, int batch, int level, KsScratch *ws);
void helr_ks_scratch_free(he_ctx *c, KsScratch *ws);
// Output stage of a key switch (ModDown combined with the operation around it):
//   out_0 = KS_0 + [rel: rel_0] + [rot: sigma_gal(rot_0)] + [acc: acc_0]
//   out_1 = KS_1 + [rel: rel_1] + [acc: acc_1]
// rel: polynomials (d0, d1) of a tensor; rot: c0 of the rotated ciphertext;
// acc: a ciphertext added to the result (rotate-and-add). Views are strided
// [item][poly][limb][N]; out must not alias rot or acc.
// Rotations whose key switches share one ModUp and one ModDown (hoisted
// rotation sums) take at most this many Galois elements per call.
#define HELR_MAX_HOIST 7
struct KsOut {
    Str out;
    const uint64_t *rel = nullptr;
    size_t rel_item = 0, rel_poly = 0;
    const uint64_t *rot = nullptr;  // out_0 += sum_j sigma_gals[j](rot_0)
    size_t rot_item = 0;
    uint64_t gals[HELR_MAX_HOIST] = {};
    int ngal = 0;
    const uint64_t *acc = nullptr;
    size_t acc_item = 0, acc_poly = 0;
};
// keys and Galois elements of the rotations of one hoisted rotation sum
struct HoistKeys {
    const uint64_t *key[HELR_MAX_HOIST];
    uint64_t gal[HELR_MAX_HOIST];
    int n;
};
int helr_keyswitch(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level, const uint64_t *key,
                   KsScratch *ws, const KsOut *o = nullptr);
// Hoisted rotation sum over a batch: out = a + sum_j Rot_{gal_j}(a) for every
// item of a ([items][2][nl][N] at stride a_item), one ModUp and one ModDown per
// item (helr_ctx.cu); hk lists the keys and Galois elements.
int helr_rotsum(he_ctx *c, const uint64_t *a, size_t a_item, int batch, int level, const HoistKeys &hk, KsScratch *ws,
                Str out);
// The hoisted inner product of a group on the tensor cores (ks_tensor.cu):
// whether it applies at nl limbs with nrot rotations and to which targets
// [t_lo, t_hi) (a run of primes below 2^40), and its launch for them (acc as
// for k_ks_hoist_ip).
bool helr_hoist_tensor_range(const he_ctx *c, int nl, int nrot, int *t_lo, int *t_hi);
int helr_hoist_ip_tensor(he_ctx *c, const uint64_t *mid, const uint64_t *dntt, size_t din_item, const HoistKeys &hk,
                         uint64_t *acc, int items, int nl, int t_lo, int t_hi, cudaStream_t s);
// ModUp of the input's digits, their full forward transforms and the summed
// inner products of every rotation of hk (ks.cu): dntt = second polynomials in
// evaluation form (item stride din_item), drow = the same after the inverse row
// pass ([items][nl][N]), mid = scratch [items][nl][nl+1][N], acc = [items][2][nl+1][N].
int helr_ks_hoisted(he_ctx *c, const uint64_t *dntt, size_t din_item, const uint64_t *drow, uint64_t *mid,
                    const HoistKeys &hk, uint64_t *acc, int items, int nl, cudaStream_t s);
int helr_ks_down(he_ctx *c, const KsOut &o, const uint64_t *src, size_t src_item, size_t src_poly, const uint64_t *drow,
                 int src_prime, uint64_t *lift, int items, int nl, const uint64_t *inv, cudaStream_t s);
const uint64_t *helr_find_key(const he_ctx *c, uint64_t gal);
int helr_add_key(he_ctx *c, uint64_t gal);
int helr_new_ct(he_ctx *c, int level, double scale, he_ct **out);

int helr_build_cdt(double sigma, uint64_t *out, int cap);
int helr_sample(he_ctx *c, uint64_t *out, size_t nlimbs, const LimbMap &lm, uint64_t seed, uint64_t stream, int kind);
int helr_encode_dev(he_ctx *c, const double *d_re, const double *d_im, int batch, size_t in_stride, int level,
                    double scale, uint64_t *d_out, size_t out_stride);
int helr_decode_dev(he_ctx *c, const uint64_t *d_pt, double scale, double *d_re, double *d_im);
int helr_encrypt_dev(he_ctx *c, const uint64_t *d_pt, int level, uint64_t seed, uint64_t *d_ct);
int helr_decrypt_dev(he_ctx *c, const uint64_t *d_ct, int level, uint64_t *d_pt);
int helr_keygen_base(he_ctx *c, uint64_t seed);
int helr_make_ksk(he_ctx *c, uint64_t gal, const uint64_t *sprime, uint64_t *out);
int helr_square_dev(he_ctx *c, uint64_t *out, const uint64_t *in, size_t nlimbs);
int helr_to_montgomery(he_ctx *c, uint64_t *x, size_t nlimbs, int period);
int helr_ks_key_layout(he_ctx *c, uint64_t *key, size_t nlimbs);
cudaError_t helr_fit_carveout(const void *f, int threads, size_t smem);

// ------------------------------------------------------------------ batched evaluator (eval.cu)
// A batch of ciphertexts: item i at d + i * item, polynomials [2][level+1][N];
// item == 0 broadcasts one ciphertext to every item.
struct CtB {
    uint64_t *d;
    int batch;
    int level;
    double scale;
    size_t item;
};
struct Eval {
    he_ctx *c;
    int maxb, maxlevel;
    KsScratch ks;
    uint64_t *tens;   // [3][maxb][nl][N]
    uint64_t *ksout;  // [maxb][2][nl][N]
    uint64_t *rot1;   // [maxb][nl][N]
    uint64_t *last;   // [maxb][2][N]
    uint64_t *lift;   // [maxb][2][nl][N]
    uint64_t keyswitches;
};
int ev_init(he_ctx *c, Eval *ev, int maxb, int maxlevel);
void ev_free(Eval *ev);
int ev_mul_relin(Eval *ev, const CtB &a, const CtB &b, CtB &out);
int ev_rescale(Eval *ev, const CtB &a, CtB &out);
int ev_mul_relin_seg(Eval *ev, const CtB &a, const uint64_t *const *bptr, const int *start, const int *count, int nseg,
                     double bscale, CtB &out);
int ev_rotate(Eval *ev, const CtB &a, int64_t r, CtB &out);
int ev_rotate_acc(Eval *ev, const CtB &a, int64_t r, CtB &out, int accumulate);
int ev_rotsum(Eval *ev, const CtB &a, const int64_t *rots, int nrot, CtB &out);
int ev_rotate_gal(Eval *ev, const CtB &a, uint64_t gal, CtB &out, int accumulate);
// Rotate-and-sum over 2^nbits positions spaced `step` slots apart as hoisted
// groups of 2^rho positions: group e (e = 0, rho, 2 rho, ...) of width
// w = min(rho, nbits - e) sums the rotations by m 2^e step, 0 < m < 2^w.
// Appends the rotation amounts of group e to out; returns w.
int rot_group_amounts(int e, int nbits, int rho, int64_t step, int64_t *out);
int ev_add(Eval *ev, const CtB &a, const CtB &b, CtB &out, int sub);
int ev_cmul_int(Eval *ev, const CtB &a, int64_t k, double out_scale, CtB &out);
int ev_cadd_int(Eval *ev, CtB &a, int64_t k);
int ev_ptmul(Eval *ev, const CtB &a, const uint64_t *pt, double pt_scale, CtB &out);
int ev_ptadd(Eval *ev, CtB &a, const uint64_t *pt);
int ev_moddrop(Eval *ev, const CtB &a, int target, CtB &out);
int ev_sum_items(Eval *ev, const CtB &a, uint64_t *acc, int accumulate);
bool scales_match(double a, double b);
int64_t round_half_away(double x);
