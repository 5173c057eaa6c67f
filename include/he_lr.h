/*
 * he_lr.h -- C ABI of the GB300 library for encrypted logistic-regression
 * training with quadratic-gradient NAG (arXiv 2406.13221).
 *
 * The paper trains logistic regression on data encrypted under an approximate
 * homomorphic scheme (Sec. 2.1: Enc, Dec, Add, cAdd, Mul, cMul, rotation and
 * rescaling), with the client preparing Z and Bbar, encrypting Z, Bbar and the
 * initial weights, and the cloud running the iterations (Sec. 4.3, Steps 1-8).
 * This library implements the scheme in residue-number-system form (limbs
 * modulo NTT-friendly primes below 2^60, hybrid key switching with one special
 * prime P) on one GPU.
 *
 * Conventions for every call:
 *   - Return value: HE_OK (0) or one of the HE_E* codes below; no call throws.
 *     he_last_error(ctx) returns a message for the last failure on ctx
 *     (owned by ctx, valid until the next call on ctx).
 *   - Handles are opaque.  The library owns all device memory it allocates
 *     (stream-ordered allocations on the stream given at he_ctx_create);
 *     the caller owns every host buffer it passes and keeps it valid for the
 *     duration of the call only.  Calls on one context are not thread-safe.
 *   - "Slots": N/2 complex values per plaintext; slot j is the value of the
 *     message polynomial at zeta^(5^j), zeta = exp(i pi / N).
 *   - Levels: a ciphertext at level l has limbs q_0..q_l; fresh encryptions
 *     sit at level n_q - 1.
 *   - Words exchanged with the host (he_ct_export / he_ct_import) are in
 *     coefficient form, layout [2][level+1][N], limb j reduced modulo q_j
 *     (he_ct_import returns HE_EINVAL on a word >= q_j).
 *   - The library fails loudly: there is no CPU fallback for any call that
 *     computes on ciphertexts; without a usable CUDA device they return
 *     HE_ECUDA.
 */
#ifndef HE_LR_H
#define HE_LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = 1,    /* bad argument (null pointer, size, parameter range) */
    HE_ENOMEM = 2,    /* device or host allocation failed */
    HE_ELEVEL = 3,    /* not enough levels left for the operation */
    HE_ESCALE = 4,    /* scales of the operands do not match */
    HE_ECUDA = 5,     /* CUDA runtime error or no device */
    HE_ETIMEOUT = 6,  /* a bounded device-side wait expired */
    HE_EINTERNAL = 7, /* internal invariant violated */
    HE_EKEY = 8       /* a required key (secret, relinearisation or rotation) is missing */
};

typedef struct he_ctx he_ctx;
typedef struct he_ct he_ct;
typedef struct he_pt he_pt;

/* Scheme parameters (Sec. 5: the paper's runs use N = 2^16; the chain here is
 * one q0_bits prime, n_q - 1 primes of qi_bits, one special prime of p_bits,
 * all = 1 mod 2N, each the largest unused such prime below 2^bits; the secret
 * is ternary and errors are discrete Gaussians of width sigma). log_n in
 * [10, 16], 2 <= n_q <= 39, bit widths in [30, 60].
 * bits (may be NULL): a width for each ciphertext prime q_0..q_(n_q-1) in
 * place of q0_bits / qi_bits (chains that bootstrap mix widths); the array is
 * read during he_ctx_create only.
 * secret_hw: 0 = every secret coefficient uniform in {-1, 0, 1}; h > 0 =
 * exactly h nonzero coefficients (a sparse secret keeps the integer overflow
 * of a bootstrap's ModRaise small). */
typedef struct {
    int log_n;
    int n_q;
    int q0_bits;
    int qi_bits;
    int p_bits;
    double sigma;
    const int *bits;
    int secret_hw;
} he_params;

/* Create a context: generates the prime chain, transform tables and the
 * encoder tables on the device.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream); every kernel of this context runs on it. */
int he_ctx_create(const he_params *p, void *cuda_stream, he_ctx **out);
/* Waits for the context stream, then frees the tables and keys.  Ciphertexts,
 * plaintexts and jobs of the context must be freed first. */
int he_ctx_destroy(he_ctx *ctx);
/* Message of the last failing call on ctx (owned by ctx, valid until its next
 * call); "null context" for NULL. */
const char *he_last_error(const he_ctx *ctx);
/* Prime chain q_0..q_{n_q-1}, P (n >= n_q + 1 entries). */
int he_ctx_primes(const he_ctx *ctx, uint64_t *out, size_t n);
/* Host-only: the Gaussian sampler's cumulative table for width sigma
 * (floor(2^63 P(|x| <= k)), last entry 2^63); returns its length via *len. */
int he_gauss_table(double sigma, uint64_t *out, size_t cap, size_t *len);
/* Host-only: the canonical-embedding root table zeta^k = exp(i pi k / N),
 * k < 2N, as re/im doubles (2N entries each). */
int he_zeta_table(int log_n, double *re, double *im);

/* Key generation (Sec. 2.1, Sec. 4.3: the third party issues the keys).
 * The secret s is ternary, the public key is (-a s + e, a), the
 * relinearisation key switches s^2 -> s and one rotation key per entry of
 * `rotations` (a left rotation of the slot vector by r; negative r rotates
 * right) switches s(X^(5^r)) -> s.  Randomness is the splitmix64 stream of
 * `seed`.  May be called again to add rotation keys (same seed). */
int he_keygen(he_ctx *ctx, uint64_t seed, const int64_t *rotations, size_t n_rot);
/* Keys for raw Galois elements (odd residues below 2N; 2N - 1 is the slot-wise
 * complex conjugation X -> X^-1 the bootstrap uses), from the seed of the
 * last he_keygen (HE_EKEY before it, HE_EINVAL for an even or out-of-range
 * element). */
int he_keygen_galois(he_ctx *ctx, const uint64_t *gals, size_t n);

/* Encode n_slots <= N/2 complex values (re, im; im may be NULL) at `level`
 * with `scale`: the coefficients are round_half_away(scale * tau^-1(z)). */
int he_encode(he_ctx *ctx, const double *re, const double *im, size_t n_slots, int level,
              double scale, he_pt **out);
/* Decode to n_slots values (im may be NULL).  Valid while |scale * z| < q_0/2. */
int he_decode(he_ctx *ctx, const he_pt *pt, double *re, double *im, size_t n_slots);
/* Enc_pk (Sec. 2.1): (v b + e0 + m, v a + e1), v ternary, e0, e1 Gaussian, all
 * drawn from the splitmix64 stream of `seed`. */
int he_encrypt(he_ctx *ctx, const he_pt *pt, uint64_t seed, he_ct **out);
/* Dec_sk (Sec. 2.1): c0 + c1 s. */
int he_decrypt(he_ctx *ctx, const he_ct *ct, he_pt **out);

/* Ciphertext words to the host in coefficient form, [2][level+1][N]
 * (n_words >= 2 (level + 1) N, else HE_EINVAL); level and scale may be NULL.
 * Synchronises the context stream. */
int he_ct_export(const he_ct *ct, uint64_t *words, size_t n_words, int *level, double *scale);
/* A new ciphertext from host words in the layout of he_ct_export (copied;
 * the caller keeps `words`).  0 <= level < n_q; a word >= q_j in limb j is
 * HE_EINVAL.  Synchronises the context stream. */
int he_ct_import(he_ctx *ctx, const uint64_t *words, size_t n_words, int level, double scale,
                 he_ct **out);
/* Plaintext words in coefficient form, [level+1][N]. */
int he_pt_export(const he_pt *pt, uint64_t *words, size_t n_words, int *level, double *scale);
/* Level and scale of a ciphertext (either pointer may be NULL). */
int he_ct_level(const he_ct *ct, int *level, double *scale);
/* Free a ciphertext or plaintext (stream-ordered on its context's stream);
 * NULL is HE_EINVAL. */
int he_ct_free(he_ct *ct);
int he_pt_free(he_pt *pt);

/* Homomorphic operations of Sec. 2.1; each returns a new ciphertext.
 * Add/Sub need equal levels and scales (relative 2^-40).  Mul is the tensor
 * product followed by relinearisation; its scale is the product of scales
 * and it does not rescale.  Rescale divides by q_level with rounding.
 * cMul multiplies by round_half_away(c * const_scale); cAdd adds
 * round_half_away(c * scale) to every slot.  Rotate by r slots to the left
 * (HE_EKEY without its key).  ModDrop keeps the limbs q_0..q_level without
 * scaling (level <= the input's, else HE_ELEVEL).  PtMul multiplies by an
 * encoded plaintext of the same level (else HE_ELEVEL); the scales multiply.
 * Level and scale errors are HE_ELEVEL and HE_ESCALE; the output is owned by
 * the caller (he_ct_free). */
int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_sub(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_mul(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);
int he_rescale(he_ctx *ctx, const he_ct *a, he_ct **out);
int he_moddrop(he_ctx *ctx, const he_ct *a, int level, he_ct **out);
int he_rotate(he_ctx *ctx, const he_ct *a, int64_t r, he_ct **out);
/* a + sum_j Rot(a, rots[j]) for 1 <= n_rot <= 7 rotations whose key switches
 * share one ModUp and one ModDown (hoisted rotations; Sec. 2.1 rotation, used
 * by the rotate-and-sum of Sec. 2.2): the digits of a's second polynomial are
 * lifted and transformed once, the inner products of every rotation are
 * summed over {q_0..q_l, P} and divided by P once.  With one rotation the
 * result equals he_add(a, he_rotate(a, r)) word for word.  HE_EKEY when a
 * rotation key is missing, HE_EINVAL for n_rot outside 1..7. */
int he_rotsum(he_ctx *ctx, const he_ct *a, const int64_t *rots, size_t n_rot, he_ct **out);
int he_cmul(he_ctx *ctx, const he_ct *a, double c, double const_scale, he_ct **out);
int he_cadd(he_ctx *ctx, const he_ct *a, double c, he_ct **out);
int he_ptmul(he_ctx *ctx, const he_ct *a, const he_pt *pt, he_ct **out);
/* Set the declared scale of a ciphertext (used to align scales that agree up
 * to rounding of a constant, Sec. 2.1 rescaling). */
int he_set_scale(he_ct *ct, double scale);

/* Batched negacyclic NTT on device limbs (the transform under every ring
 * product of the scheme).  d_limbs: device pointer, [n_limbs][N] words in
 * [0, q); limb i is reduced modulo prime index prime_of[i % period]
 * (index n_q is P).  Output: evaluation form in the library's internal order
 * (bit-reversed evaluation index); he_ntt_inverse undoes it.  Runs on the
 * context stream. */
int he_ntt_forward(he_ctx *ctx, uint64_t *d_limbs, size_t n_limbs, const int *prime_of, int period);
int he_ntt_inverse(he_ctx *ctx, uint64_t *d_limbs, size_t n_limbs, const int *prime_of, int period);

/* Batched key switching of device polynomials, the hot primitive of every Mul
 * and rotation.  d_in: [batch][level+1][N] NTT-form words (modulo q_j);
 * d_out: [batch][2][level+1][N].  gal = 0 selects the relinearisation key,
 * otherwise the rotation key of galois element gal.  Device scratch is
 * allocated by the call. */
int he_keyswitch_batch(he_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int batch, int level,
                       uint64_t gal);
/* Batched hoisted rotation sums of device ciphertexts (he_rotsum for every
 * item): d_in and d_out [batch][2][level+1][N] NTT-form words, d_out[b] =
 * d_in[b] + sum_j Rot(d_in[b], rots[j]) for 1 <= n_rot <= 7 rotations whose
 * key switches share one ModUp and one ModDown per item.  d_out must not
 * overlap d_in (HE_EINVAL).  Device scratch is allocated by the call. */
int he_rotsum_batch(he_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int batch, int level,
                    const int64_t *rots, size_t n_rot);
/* Batched Mul, Rescale and Rotation (Sec. 2.1) on device ciphertexts: `batch`
 * items of [2][level+1][N] NTT-form words each, stored contiguously; the
 * output buffer must not overlap an input (HE_EINVAL).  Scales are the
 * caller's (the words are those of he_mul, he_rescale and he_rotate on each
 * item).  Device scratch is allocated by the call; each runs on the context
 * stream without synchronising.
 * he_mul_relin_batch: d_out[b] = Relin(d_a[b] (x) d_b[b]) at the same level
 *   (HE_EKEY without a relinearisation key).
 * he_rescale_batch: d_out[b] = d_in[b] divided by q_level with rounding, at
 *   level - 1 ([batch][2][level][N]); HE_ELEVEL at level 0.
 * he_rotate_batch: d_out[b] = Rot(d_in[b], r), a left rotation of the slots
 *   by r (HE_EKEY without its key). */
int he_mul_relin_batch(he_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out, int batch, int level);
int he_rescale_batch(he_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int batch, int level);
int he_rotate_batch(he_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int batch, int level, int64_t r);
/* Autotuning of the key switch (Sec. 2.1; the relinearisation inside every
 * Mul and the key switch inside every rotation): per level it picks
 *  - the wave: the number of items whose ModUp and inner product share one
 *    DRAM read of each key row (scratch [wave][level+1][level+2][N] words),
 *    timing `items` batched relinearisations (16 or more; 0 = 256) with waves
 *    of 16, 32, 64, 128 and 256 items (those <= items) and keeping the
 *    smallest wave within 1% of the fastest;
 *  - the tile variant of the kernels at that wave: bit 0 halves the columns
 *    per CTA of the ModUp/ModDown column kernel, bit 1 halves the rows per
 *    CTA of the ModDown and hoisted-digit row kernels; a variant other than 0
 *    is kept only when it is more than 1% faster;
 *  - where the tensor-core form of the hoisted inner product applies
 *    (he_set_hoist_form), its time against the CUDA-core form on a hoisted
 *    sum of seven rotations; it is kept only when more than 1% faster.
 * Later key switches of this context use the choices; results do not depend
 * on them (the words are the same for every wave, tile and form).
 * table_path (may be NULL): a text table keyed by device, SM count, log N,
 * n_q and the primes; levels it already holds are loaded instead of measured,
 * and the file is rewritten when anything was measured.  *measured (may be
 * NULL) receives the number of levels measured.  Needs he_keygen first
 * (HE_EKEY); device memory for the largest wave is allocated and freed by the
 * call (a wave that does not fit is skipped); HE_EINVAL when the table cannot
 * be written.  The environment variable HELR_KS_WAVE, when set, overrides
 * every wave. */
int he_autotune(he_ctx *ctx, const char *table_path, int items, int *measured);
/* The wave key switches at `level` use (> 0), or -HE_EINVAL. */
int he_ks_wave(const he_ctx *ctx, int level);
/* The tile variant key switches at `level` use (0..3), or -HE_EINVAL. */
int he_ks_tile(const he_ctx *ctx, int level);
/* Force the tile variant of every later key switch (0..3), or return to the
 * autotuned choice (-1); HE_EINVAL otherwise. */
int he_set_ks_tile(he_ctx *ctx, int tile);
/* Form of the hoisted inner product of rotation groups (he_rotsum,
 * he_rotsum_batch and the rotate-and-sum steps of a training iteration,
 * Sec. 2.2 / 3.3): -1 = the form he_autotune chose per limb count (the
 * default; the CUDA-core form until he_autotune has measured both);
 * 0 = CUDA cores; 1 = tensor cores (tcgen05.mma on
 * FP16 byte slices of the digits and keys, exact: the sum over the group's
 * rotations and digits is formed in 128 bits from the integer diagonal sums
 * the MMA accumulates).  Form 1 applies at a key switch whose target primes
 * q_0..q_(nl-1) are below 2^40, with rotations x limbs <= 51 and nl <= 8; the
 * special prime's target and every other case keep the CUDA-core form.  Both
 * forms give the same words.  HE_EINVAL for other values. */
int he_set_hoist_form(he_ctx *ctx, int form);
/* The form hoisted sums at `level` use (0 or 1; he_autotune's choice unless
 * he_set_hoist_form forced one), or -HE_EINVAL. */
int he_hoist_form(const he_ctx *ctx, int level);
/* Launches of the tensor-core form made by ctx so far. */
unsigned long long he_hoist_tensor_launches(const he_ctx *ctx);
/* Synchronise the context stream and read the device status word: HE_OK, or
 * HE_ETIMEOUT when a bounded device-side wait (the mbarrier waits of the
 * tensor-core form, 1 s each) expired since the last call; the word is then
 * cleared. */
int he_check_device(he_ctx *ctx);
/* Self-test of that path: one thread waits on a barrier with the kernels'
 * bounded wait.  arrive = 1: the thread arrives first and the wait ends at
 * once; arrive = 0: nothing arrives, the wait runs out after one second and
 * the next he_check_device returns HE_ETIMEOUT.  The context stays usable. */
int he_selftest_bounded_wait(he_ctx *ctx, int arrive);
/* Rescale without allocating (no counterpart in the paper: it exists for
 * callers that may not allocate device memory, such as code running under a
 * device-memory budget fixed in advance or inside a framework that owns every
 * allocation).  Same result as he_rescale on device buffers: d_in holds
 * `batch` ciphertexts [batch][2][level+1][N] in evaluation form; d_out
 * receives [batch][2][level][N] (it must not overlap d_in).  The work space is
 * a 16 MiB array that every device loading the library keeps until exit; one
 * ciphertext needs (2 + 2 level) N words of it, so larger sizes (at N = 2^16,
 * level > 15) return HE_EINVAL.  The first call on a device looks up the
 * array's device address (make it before capturing any stream).  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams or
 * contexts on the same device) race; calls on one stream do not.  The array
 * needs no clearing: every word a call reads it wrote first.  Runs on the
 * context stream and returns without synchronising. */
int he_rescale_noalloc(he_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int batch, int level);
/* Number of kernels this library has launched since it was loaded. */
uint64_t he_launch_count(void);
/* Per-class kernel timing with CUDA events on the context stream (adds two
 * event records per timed launch group).  Classes: 0 forward NTT, 1 inverse
 * NTT, 2 ModUp lift, 3 key-switch inner product, 4 whole key switches (spans
 * the launches of classes 0-3 that belong to a key switch; units = key
 * switches).  Enabling resets the sums;
 * he_prof_read synchronises the stream and returns the summed milliseconds,
 * the work units (limbs for transforms, digit x modulus limbs for ModUp,
 * key switches for the inner product) and the kernel launches of the class. */
int he_prof_enable(he_ctx *ctx, int on);
int he_prof_read(he_ctx *ctx, int cls, double *ms, double *units, uint64_t *launches);
/* Further work counts of a class: units2 = for the key-switch inner product
 * (class 3) the limbs of key products (2 keys x digits x targets), 0 for the
 * other classes (class 3's first count is the limbs that run the row pass of
 * the transform); dram_limbs (may be NULL) = algorithmic DRAM traffic of the
 * key-switch classes in limbs (operands shared by a launch counted once). */
int he_prof_read2(he_ctx *ctx, int cls, double *units2, double *dram_limbs);
/* Class 4's counts: units2 = summed input limbs of the key switches,
 * dram_limbs = their algorithmic DRAM traffic in limbs of N words (a key
 * switch at L limbs reads its input once and writes two polynomials: 3L; the
 * 2L(L+1) key limbs it uses are read once per wave of items).
 * he_prof_keyswitches writes the key switches issued since profiling was
 * enabled per input limb count: by_limbs[L] for L < n. */
int he_prof_keyswitches(he_ctx *ctx, double *by_limbs, size_t n);
/* The rotate-and-sum steps of the training circuit (the row sums and their
 * replication, Sec. 2.2 SumColVec, and the column sums of the full-batch
 * gradient, Sec. 3.3) over 2^k positions run as hoisted groups of 2^r
 * positions: each group sums the rotations by m 2^e (0 < m < 2^r) of one
 * ciphertext with one ModUp and one ModDown (Sec. 2.1 key switching shared by
 * the rotations), so r = 1 is the plain log-step sum.  Sets r for later jobs
 * and iterations of ctx (default 3; 1..3, else HE_EINVAL).  A job must run
 * with the r it was created with (its rotation keys depend on it). */
int he_set_rotation_radix(he_ctx *ctx, int log2_radix);
/* ------------------------------------------------------------------ bootstrapping
 * The refresh of the weight ciphertexts by bootstrapping (Sec. 2.1, Sec. 4.3
 * Step 7): a ciphertext at level 0 whose slot vector repeats with period
 * `slots` (W and V repeat the g weights in every row) comes back at
 * `level_out` with scale `scale_out` holding the same slots:
 *   ModRaise (the q0 words as centred integers modulo every prime), SubSum
 *   (the trace to Z[X^(N / 2 slots)] by hoisted rotations), CoeffToSlot
 *   (E^H / slots by baby-step/giant-step diagonals, real and imaginary parts
 *   split with the conjugation and X^(N/2)), EvalMod (the degree-`degree`
 *   Taylor polynomial of cos(2 pi (v - 1/4) / 2^double_angles) on
 *   |v| <= K + 1/2, then `double_angles` steps y -> 2y^2 - 1: sin(2 pi v)),
 *   SlotToCoeff (q0 E / (2 pi scale_out)).
 * It consumes 1 + ceil(log2 degree) + 1 + double_angles + 1 levels from the
 * top of the chain and needs: a sparse secret (he_params.secret_hw, so that
 * the ModRaise overflow |I| stays below K), a scale_out well below q0 (the
 * refreshed value carries a relative error of about (2 pi scale_out |m| /
 * q0)^2 / 6 from sin against its argument), the rotation keys he_boot_keys
 * lists and the conjugation key (he_keygen_galois, element 2N - 1).
 * HE_ELEVEL when the chain is too short for level_out, HE_EKEY for a missing
 * key, HE_EINVAL for parameters out of range. */
typedef struct {
    int slots;          /* period of the slot vector (a power of two <= N/2) */
    int K;              /* bound on the ModRaise overflow |I| */
    int double_angles;  /* r */
    int degree;         /* degree of the cosine polynomial, 2..63 */
    double scale_out;
    int level_out;
} he_boot_params;
/* The rotation amounts a bootstrap with these parameters needs (written to
 * rots[0..cap), the count to *n_rots). */
int he_boot_keys(he_ctx *ctx, const he_boot_params *p, int64_t *rots, size_t cap, size_t *n_rots);
/* Bootstrap one ciphertext into a new one (scratch allocated by the call). */
int he_bootstrap(he_ctx *ctx, const he_ct *in, const he_boot_params *p, he_ct **out);
/* Bootstrap `batch` device ciphertexts [batch][2][in_level+1][N] (NTT form)
 * into d_out [batch][2][level_out+1][N]; the slots are refreshed together
 * (every key switch of the bootstrap runs over the whole batch). */
int he_bootstrap_batch(he_ctx *ctx, const uint64_t *d_in, int in_level, uint64_t *d_out, int batch,
                       const he_boot_params *p);

/* Galois element of a left rotation by r. */
uint64_t he_galois_elt(const he_ctx *ctx, int64_t r);

/* ------------------------------------------------------------------ training */
/* Learning-rate schedule F2(t) = max - (max - min) (t / T)^power (Sec. 3.2);
 * the paper's runs use (2, 1, 81, 2.5). */
typedef struct {
    double max, min, T, power;
} he_lr_sched;

enum { HE_LR_FULL_BATCH = 0, HE_LR_MINI_BATCH = 1 };
/* OR-ed into the mode of he_lr_job_create / he_lr_train: the first-order NAG
 * baseline the paper compares against (Sec. 2.3, w' = v + gamma (1/n) g): the
 * same circuit without the Bbar product of Step 8, so one level shallower
 * (fresh ciphertexts at level 5, no Bbar ciphertexts); the schedule's F2(t)
 * is the rate gamma (a constant when max = min). */
enum { HE_LR_FIRST_ORDER = 0x100 };
enum { HE_LR_G8 = 0, HE_LR_G16 = 1 };

typedef struct {
    double sec_setup;        /* client precompute + encryption + key generation */
    double sec_iter_avg;     /* average seconds per iteration (update + refresh) */
    double sec_update_avg;   /* average seconds of the update alone (Steps 4-6) */
    uint64_t keyswitches;    /* key switches issued per iteration (last one) */
    int n_blocks;            /* encrypted data blocks */
    int g, m;                /* packing: g columns x m rows per block */
    double max_abs_ip;       /* unused by the library (0) */
} he_lr_stats;

typedef struct he_lr_job he_lr_job;

/* Client side of Sec. 4.3 Steps 1-3: build Z = y * [1 | X] (bias first),
 * Bbar per mini-batch of batch_rows rows (Sec. 3.1, 1/(eps + 1/4 sum |Z^T Z|),
 * eps = 1e-8) and the full-batch Bbar by the combination of Sec. 3.3, pack
 * m x g blocks (g = next power of two >= f + 1, m g = N/2; Sec. 2.2),
 * encrypt the blocks, n*Bbar (replicated per row) and W = V = 0 at level 6
 * (the depth of one iteration, which then ends at level 0; primes above q_6
 * stay unused; level 5 and no Bbar with HE_LR_FIRST_ORDER) with scale
 * 2^log_scale.  Object k of kind K is encrypted with seed
 * enc_seed + (K << 48) + k (K: 1 block, 2 Bbar, 3 W0, 4 V0, 5 W refresh at
 * iteration k, 6 V refresh).  X: n x f row-major doubles, y: n labels +/-1.
 * Keys for the needed rotations are generated from key_seed if missing.
 * batch_blocks: data blocks per kernel launch (0 = automatic). */
int he_lr_job_create(he_ctx *ctx, const double *X, const double *y, size_t n, size_t f,
                     int mode, size_t batch_rows, int poly, double log_scale, uint64_t enc_seed,
                     uint64_t key_seed, int batch_blocks, he_lr_job **out);
/* Cloud side, Sec. 4.3 Steps 4-7 for iteration t (t = 0, 1, ...): gradient,
 * quadratic gradient, NAG update (Algorithm 1) and the refresh of W and V
 * (decrypt + re-encrypt, standing in for bootstrapping). */
int he_lr_job_step(he_lr_job *job, int t, he_lr_sched sched);
/* he_lr_job_step with the job state on the host: when state_in is not NULL,
 * W and V are first loaded from coefficient words [2 ciphertexts][2][n_q][N]
 * (W then V, at the job's start level L = 6, or 5 first-order, scale
 * 2^log_scale; n_q is then L + 1 limbs); when state_out is not NULL, the
 * refreshed W and V are written back in the same layout.  Host buffers may be
 * pinned; the copies run on the context stream inside the call. */
int he_lr_job_step_io(he_lr_job *job, int t, he_lr_sched sched, const uint64_t *state_in, uint64_t *state_out);
/* Record Steps 1-9 of every later he_lr_job_step as one CUDA graph on a
 * stream owned by the job (re-recorded each iteration with that iteration's
 * constants and swapped into the executable graph) and launch it as a unit;
 * the refresh runs after it.  on = 0 returns to direct launches. */
int he_lr_job_set_graph(he_lr_job *job, int on);
/* Data blocks per kernel launch for later steps: 1 = the plain
 * one-ciphertext-per-launch form; at most the value the job was created with. */
int he_lr_job_set_batch(he_lr_job *job, int blocks_per_launch);
/* Refresh W and V after every later step by bootstrapping (Sec. 4.3 Step 7)
 * instead of decrypting and re-encrypting them: one he_bootstrap_batch over
 * both.  p must return slots of period g at the job's start level with its
 * scale (HE_EINVAL otherwise); the context needs the chain and the sparse
 * secret the bootstrap requires; the rotation and conjugation keys are
 * generated here from the context's key seed.  p = NULL returns to
 * decryption and re-encryption. */
int he_lr_job_set_refresh(he_lr_job *job, const he_boot_params *p);
/* Decrypted weights W (slots of row `row`, g values; padded columns are 0). */
int he_lr_job_weights(he_lr_job *job, int row, double *w, size_t len);
/* Access to the job's current W and V ciphertexts (owned by the job). */
int he_lr_job_state(he_lr_job *job, const he_ct **W, const he_ct **V);
/* A copy of one encrypted input of the job: kind 0 = data block `index`,
 * kind 1 = Enc(n Bbar) of mini-batch `index` (index 0 in full-batch mode; none
 * for a first-order job: HE_EINVAL). */
int he_lr_job_input(he_lr_job *job, int kind, int index, he_ct **out);
/* Gradient ciphertext of one block for the job's current W (Steps 1-6 alone:
 * s_r z_rc with s = 1 - g(z_r . w), computed in the same chunked launch that
 * he_lr_job_step uses for the chunk holding the block); returns a new
 * ciphertext. */
int he_lr_job_block_grad(he_lr_job *job, int block, he_ct **out);
int he_lr_job_info(const he_lr_job *job, he_lr_stats *stats);
int he_lr_job_free(he_lr_job *job);

/* Several independent full-batch jobs of one context trained in lockstep
 * (uneven job sizes and feature counts, Sec. 4.2's multi-owner usage run as
 * separate models): Steps 1-6 of all jobs' data blocks share launches, ordered
 * by decreasing row width; Steps 7-9 and the refresh run per job.  The jobs
 * must use one level, scale and sigmoid polynomial; they stay owned by the
 * caller and must outlive the handle.  blocks_per_launch 0 = 256. */
typedef struct he_lr_multi he_lr_multi;
int he_lr_multi_create(he_ctx *ctx, he_lr_job *const *jobs, size_t n_jobs, int blocks_per_launch, he_lr_multi **out);
/* Iteration t of every job (same schedule); results through he_lr_job_weights. */
int he_lr_multi_step(he_lr_multi *multi, int t, he_lr_sched sched);
int he_lr_multi_free(he_lr_multi *multi);

/* Whole training through one call: job_create + iters x job_step + weights
 * of row 0 (w_out holds g values).  stats may be NULL. */
int he_lr_train(he_ctx *ctx, const double *X, const double *y, size_t n, size_t f, int iters,
                he_lr_sched sched, int mode, size_t batch_rows, int poly, uint64_t enc_seed,
                uint64_t key_seed, double *w_out, size_t w_len, he_lr_stats *stats);

/* One encrypted iteration on caller-supplied ciphertexts (cloud only):
 * Z[0..n_blocks-1] data blocks at one level, B = Enc(n Bbar) at that level,
 * W, V at that level; g x m packing; alpha = F2(t), eta from Algorithm 1,
 * inv_n = 1/n; poly = (c0, c1, c3) of the sigmoid polynomial.  Returns
 * W', V' six levels down (before any refresh).  B = NULL runs the
 * first-order baseline (alpha = gamma, no Bbar product): five levels down. */
int he_lr_iteration(he_ctx *ctx, he_ct *const *Z, size_t n_blocks, const he_ct *B, const he_ct *W,
                    const he_ct *V, int g, int m, double alpha, double eta, double inv_n,
                    const double poly[3], he_ct **W_out, he_ct **V_out);
/* The refresh used between iterations (standing in for the bootstrapping of
 * Sec. 4.3 Step 7): decrypt, take the real part of every slot, re-encode at
 * `level` with `scale`, encrypt with `seed`. */
int he_refresh(he_ctx *ctx, const he_ct *in, int level, double scale, uint64_t seed, he_ct **out);

/* Host-only client precompute exposed for checking: Bbar (length g) for the
 * rows [row0, row0 + rows) of Z = y * [1 | X]. */
int he_lr_bbar(const double *X, const double *y, size_t n, size_t f, size_t row0, size_t rows,
               size_t g, double *out);
/* The same precompute for every mini-batch of batch_rows rows at once, on the
 * device (Sec. 3.1 Bbar_k, Algorithm 1; used by he_lr_job_create for f + 1 <=
 * 256): out[k][0..g) for k < ceil(n / batch_rows), host memory, padded columns
 * 0.  The Gram sums run in row order and the absolute row sums in column order
 * without fused multiply-adds, so the values equal he_lr_bbar's bit for bit.
 * Requires f + 1 <= 256 and g >= f + 1 (else HE_EINVAL). */
int he_lr_bbar_batches(he_ctx *ctx, const double *X, const double *y, size_t n, size_t f, size_t batch_rows,
                       size_t g, double *out);

#ifdef __cplusplus
}
#endif
#endif
