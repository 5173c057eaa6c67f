// ks.cu -- fused hybrid key switching (the relinearisation inside every Mul and
// the key switch inside every rotation, Sec. 2.1), and the division by a
// dropped prime shared by ModDown and rescale.
//
// Key switching of d (level l, L = l + 1 limbs) with one special prime P and
// one digit per ciphertext prime:
//   ModUp    digit i = centred limb i of d in coefficient form, reduced into
//            every target modulus t in {q_0..q_l, P};
//   inner    acc_t = sum_i NTT_t(digit i) * key_(i,t)   (two key polynomials);
//   ModDown  out_j = (acc_j - centred(acc_P) mod q_j) * P^-1.
// The transforms are split into a column pass and a row pass (see ntt.cu) and
// fused with their neighbours:
//   k_ntt_inv_rows   (ntt.cu) row pass of the inverse transform of the input;
//   k_ks_modup_cols  finishes the inverse transform of digit i (column pass,
//                    N^-1), then lifts it into every target t != i and runs
//                    the forward column pass (t = i is the evaluation-form
//                    input itself);
//   k_ks_inner_rows  finishes the row pass of every digit for one target and
//                    multiplies-accumulates with the key rows (128-bit sums in
//                    tensor memory), so the transformed digits are never stored;
//   k_ntt_inv_rows   row pass of the inverse transform of the P part;
//   k_ks_modup_cols  (ModDown mode) its column pass, the lift into q_0..q_l and
//                    their forward column passes;
//   k_ks_down_rows   the forward row passes fused with the output stage.
// Key switches run in waves of items; each key row is read from DRAM once per
// wave and served from L2 to the wave's items.
#include <stdlib.h>
#include "ntt_core.cuh"

namespace {
using namespace nttc;

// a centred residue s (signed, |s| <= q_src / 2) reduced into [0, q_t); the
// Barrett step only when |s| can reach q_t
__device__ __forceinline__ uint64_t lift_signed(uint64_t s, uint64_t q, const ModQ &mt, bool reduce)
{
    const bool neg = (int64_t)s < 0;
    if (!reduce) return neg ? s + q : s;
    uint64_t m = neg ? 0 - s : s;
    m = m < q ? m : reduce64(m, mt);
    return neg && m ? q - m : m;
}

// Second half of an inverse transform followed by a centred lift into several
// primes and the first half of their forward transforms.  A CTA takes C
// adjacent columns of one source limb (row pass of the inverse transform
// already applied), runs the inverse column pass and the factor N^-1, keeps the
// coefficients in shared memory, then for every target lifts the centred
// coefficients into q_t and runs the forward column pass.  Each source column
// is read once.
//   ModUp (DOWN = false): source (b, i) = digit i of item b, prime q_i, in
//     drow[b][i]; targets t = 0..nl except i (nl stands for P), out
//     mid[b][i][t] (t = i is the evaluation-form input itself).
//   ModDown / rescale (DOWN = true): source k = drow[k], prime src_prime;
//     targets t = 0..nl-1, out mid[k][t].
template <int K1, int K2, int C, bool DOWN>
__global__ void __launch_bounds__(C * Geo<K1>::T, 3)
    k_ks_modup_cols(const uint64_t *__restrict__ drow, uint64_t *__restrict__ mid, const uint64_t *__restrict__ twall,
                    const uint64_t *__restrict__ itwall, const ModQ *__restrict__ mods, const uint64_t *__restrict__ ninv,
                    int nl, int pidx, int src_prime)
{
    using G = Geo<K1>;
    constexpr int R2 = 1 << K2, N = G::R * R2, NG = R2 / C, E = G::E, T = G::T;
    extern __shared__ uint64_t smem[];
    int bid = blockIdx.x;
    const int grp = bid % NG;
    bid /= NG;
    const size_t src = (size_t)bid;                       // source limb index in drow
    const int i = DOWN ? -1 : bid % nl;                    // digit index (ModUp)
    const int sp = DOWN ? src_prime : i;                   // prime of the source limb
    const int jj = threadIdx.x % C, l = threadIdx.x / C;
    uint64_t *seg = smem + jj * G::SEG;
    uint64_t *coef = smem + C * G::SEG;  // [R1][C]: word (j1, jj); each thread reads back only its own words
    const uint64_t qi = mods[sp].q;
    const size_t col = src * N + grp * C + jj;
    {
        const uint64_t *itw = itwall + (size_t)sp * N * 2;
        uint64_t c[E];
        // words of this column arrive as j1 = E l + r (contiguous assignment)
#pragma unroll
        for (int r = 0; r < E; r++) c[r] = drow[col + (size_t)(E * l + r) * R2];
        inv_contig<K1, false>(c, itw, 1, l, qi, 2 * qi);
        to_strided<K1>(c, seg, l);
        inv_strided<K1>(c, itw, 1, qi, 2 * qi);
        const uint64_t ni = ninv[2 * sp], nip = ninv[2 * sp + 1];
#pragma unroll
        for (int r = 0; r < E; r++) {
            // the centred representative, stored as a signed 64-bit word
            const uint64_t v = shoup(c[r], ni, nip, qi);  // in [0, q_src)
            coef[(l + T * r) * C + jj] = v > (qi >> 1) ? v - qi : v;
        }
    }
    uint64_t *dst = mid + src * (DOWN ? nl : nl + 1) * N + grp * C + jj;
    for (int tt = 0; tt < nl; tt++) {
        const int t = DOWN ? tt : (tt < i ? tt : tt + 1);
        const int pt = DOWN ? t : (t < nl ? t : pidx);
        const ModQ mt = mods[pt];
        const uint64_t q = mt.q, q2 = 2 * q;
        const uint64_t *tw = twall + (size_t)pt * N * 2;
        const bool reduce = (qi >> 1) >= q;  // centred words may reach q_t (a 60-bit source into a 40-bit target)
        uint64_t x[E];
#pragma unroll
        for (int r = 0; r < E; r++) x[r] = lift_signed(coef[(l + T * r) * C + jj], q, mt, reduce);
        fwd_strided<K1, false, false, true>(x, tw, 1, q, q2);  // lifted words are below q
        __syncthreads();  // the previous exchange has been read
        to_contig<K1>(x, seg, l);
        fwd_contig<K1, false>(x, tw, 1, l, q, q2);
#pragma unroll
        for (int r = 0; r < E; r++) dst[(size_t)t * N + (size_t)(E * l + r) * R2] = x[r];
    }
}


// bulk prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global
// address into L2 (no data returned to the thread)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// read-only load that does not allocate in L1
__device__ __forceinline__ uint64_t ld_stream(const uint64_t *p)
{
    uint64_t v;
    asm("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

// Key rows in the order the row pass consumes them: inside each row of R2 words
// the word at E l + r (thread l's r-th word on the contiguous assignment) moves
// to r T + l.  One CTA per row; applied once when a key is generated.
template <int K2>
__global__ void __launch_bounds__(1 << K2) k_key_rows(uint64_t *__restrict__ key)
{
    using G = Geo<K2>;
    __shared__ uint64_t row[G::R];
    uint64_t *p = key + (size_t)blockIdx.x * G::R;
    const int j = threadIdx.x;
    row[j] = p[j];
    __syncthreads();
    const int r = j / G::T, l = j % G::T;
    p[j] = row[G::E * l + r];
}

// 16-byte asynchronous global -> shared copies (cp.async), grouped per digit
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- tensor memory (TMEM) as accumulator storage between digits
// Each of the CTA's 4 warps owns a quarter of the 128 TMEM lanes (warp w: lanes
// 32 w .. 32 w + 31), one lane per thread; the thread's 64-bit accumulators take
// two 32-bit columns each.  Allocation is per CTA, by warp 0, and is returned
// before the CTA exits.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }
// 16 consecutive 32-bit columns of this thread's lane <-> registers (four
// 128-bit accumulators).  No memory clobbers: TMEM traffic does not alias global
// or shared memory, and the key loads must stay free to move ahead of it.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15, %16};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
                 "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&w)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
                 "%15}, [%16];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]), "=r"(w[8]),
                   "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
                 : "r"(taddr));
}
// wait for the loads into a and b; the registers are operands so that no use of
// them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&a)[16], uint32_t (&b)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                   "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]), "+r"(a[15]),
                   "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                   "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]));
}

// 128-bit accumulator held as four 32-bit words (least significant first)
__device__ __forceinline__ void mac128(uint32_t *acc, uint64_t x, uint64_t k)
{
    const uint64_t lo = x * k, hi = __umul64hi(x, k);
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3])
        : "r"((uint32_t)lo), "r"((uint32_t)(lo >> 32)), "r"((uint32_t)hi), "r"((uint32_t)(hi >> 32)));
}
__device__ __forceinline__ void set128(uint32_t *acc, uint64_t x, uint64_t k)
{
    const uint64_t lo = x * k, hi = __umul64hi(x, k);
    acc[0] = (uint32_t)lo;
    acc[1] = (uint32_t)(lo >> 32);
    acc[2] = (uint32_t)hi;
    acc[3] = (uint32_t)(hi >> 32);
}

// One launch per butterfly form: `tl` lists the targets t (0..nl, nl standing
// for P) whose primes take the unreduced forward butterfly (LZ) or Harvey's.
//
// Inner product without per-digit reduction: with keys k' = k 2^64 mod q, the
// CTA accumulates T = sum_i x_i k'_i over the nl digits exactly in 128 bits
// (x_i below 20q for LZ, where q < 2^58, and below 4q otherwise: T < nl 20 q^2
// or nl 4 q^2, which he_ctx_create keeps below 2^128 for every prime of the
// chain and nl <= n_q; with primes of at most 60 bits that holds up to 39
// digits) and reduces once: T 2^-64 mod q = sum_i x_i k_i mod q
// (one Montgomery reduction, after reducing the high word below q).  The 128-bit accumulators of both key polynomials live
// in TMEM between digits (128 columns per thread), so the registers hold only
// the digit being transformed.
//
// The row twiddles depend on the target and the row, not on the digit: the CTA
// copies those of its rows into shared memory once and serves every digit from
// there.  One digit buffer (the next digit's rows are requested as soon as the
// exchange has read the current ones) keeps the CTA at 48 KB, 4 CTAs per SM.
// A digit's rows are one contiguous tile, copied by the TMA engine
// (cp.async.bulk, one thread, completion counted in bytes on an mbarrier);
// the wait for it is bounded (1 s) and sets bit 1 of *status when it expires.
template <int K1, int K2, int RPC, bool LZ>
__global__ void __launch_bounds__(RPC * Geo<K2>::T, 4)
    k_ks_inner_rows(const uint64_t *__restrict__ mid, const uint64_t *__restrict__ dntt, const uint64_t *__restrict__ key,
                    uint64_t *__restrict__ acc, const uint64_t *__restrict__ twall, const ModQ *__restrict__ mods, int nl,
                    int nq, int pidx, int items, PosList tl, int *status)
{
    using G = Geo<K2>;
    constexpr int R1 = 1 << K1, R2 = G::R, N = R1 * R2, NG = R1 / RPC, E = G::E, NT = RPC * G::T;
    constexpr int TILE = RPC * R2;  // words of one digit's rows handled by this CTA
    constexpr int CH = 4;           // accumulators of one key polynomial per TMEM transfer (16 columns)
    constexpr uint32_t TCOLS = 8 * E;  // a0[r]: columns 4r..4r+3; a1[r]: 4E + 4r..4E + 4r + 3
    static_assert(NT == 128 && E % CH == 0 && TCOLS >= 32 && TCOLS <= 128 && (TCOLS & (TCOLS - 1)) == 0, "TMEM layout");
    extern __shared__ uint64_t smem[];
    // [TILE]: the rows of one digit, which also serve as its exchange segments
    uint64_t *buf = smem;
    // [RPC][R2] twiddle pairs of the CTA's rows: stage block m at pairs m - 1 .. 2m - 2
    // of its row (the last pair unused), then the TMEM address slot
    uint64_t *tws = smem + TILE;
    int bid = blockIdx.x;
    const int b = bid % items;  // items sharing one key row are adjacent: the key row is read from L2
    bid /= items;
    const int grp = bid % NG;
    const int t = pos_at(tl, bid / NG);
    const int pt = t < nl ? t : pidx, kl = t < nl ? t : nq;
    const ModQ m = mods[pt];
    const uint64_t q = m.q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pt * N * 2;
    const int l = threadIdx.x % G::T, rl = threadIdx.x / G::T, warp = threadIdx.x / 32;
    const int row = grp * RPC + rl;
    const size_t roff = (size_t)row * R2, toff = (size_t)grp * RPC * R2;
    // rows of digit i: the column-pass output for target t, or the input itself when i == t
    auto src_of = [&](int i) -> const uint64_t * {
        return i == t ? dntt + ((size_t)b * nl + i) * N + toff : mid + (((size_t)b * nl + i) * (nl + 1) + t) * N + toff;
    };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tws + 2 * RPC * R2);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(tws + 2 * RPC * R2 + 1);
    // the whole tile of digit i (TILE words, 16-byte aligned on both sides)
    auto prefetch = [&](int i, uint64_t *dst) {
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(TILE * 8)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(dst)),
                         "l"(src_of(i)), "r"(TILE * 8), "r"(mbar)
                         : "memory");
        }
    };
    if (warp == 0) tmem_alloc(tmem_slot, TCOLS);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    prefetch(0, buf);
    // pair j of stage block m of row r sits at m (R1 + r) + j in the table
    for (int k = threadIdx.x; k < RPC * R2; k += NT) {
        const int pr = k % R2, rr = k / R2;
        if (pr == R2 - 1) continue;
        const int mm = 1 << (31 - __clz(pr + 1));
        cp_async16(tws + 2 * k, tw + 2 * (mm * (R1 + grp * RPC + rr) + (pr + 1 - mm)));
    }
    cp_async_commit();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = *tmem_slot + ((uint32_t)(32 * warp) << 16);
    // the transform indexes stage block m at m A + j: with A = 1 that is pair
    // m - 1 + j from the start of the row's copy
    const uint64_t *twr = tws + 2 * (rl * R2 - 1);
    uint64_t *o0 = acc + (((size_t)b * 2 + 0) * (nl + 1) + t) * N + roff + E * l;
    uint64_t *o1 = acc + (((size_t)b * 2 + 1) * (nl + 1) + t) * N + roff + E * l;
    bool ok = true;
    for (int i = 0; i < nl; i++) {
        if (i == 0) cp_async_wait<0>();          // the twiddles have landed
        ok &= mbar_wait_bounded(mbar, i & 1);  // and digit i
        __syncthreads();
        uint64_t x[E];
        uint64_t *rows = buf + rl * R2;
        if (i == t) {
#pragma unroll
            for (int r = 0; r < E; r++) x[r] = rows[E * l + r];
        } else {
#pragma unroll
            for (int r = 0; r < E; r++) x[r] = rows[l + G::T * r];
            fwd_strided<K2, LZ, true>(x, twr, 1, q, q2);
            __syncthreads();  // every thread has read its words of the row
            to_contig_swz<K2>(x, rows, l);
        }
        __syncthreads();  // the buffer is read: it takes the next digit
        if (i + 1 < nl) prefetch(i + 1, buf);
        if (i != t) {
            fwd_contig<K2, true, LZ, true>(x, twr, 1, l, q, q2);
            // words stay unreduced: below 4q, or below 20q with LZ (the column
            // pass leaves them below 4q)
        }
        // key rows are stored with word E l + r at r T + l (see k_key_rows): adjacent
        // threads read adjacent words; each key word is read once per CTA, so it
        // bypasses L1
        const uint64_t *kp0 = key + (((size_t)i * 2 + 0) * (nq + 1) + kl) * N + roff + l;
        const uint64_t *kp1 = key + (((size_t)i * 2 + 1) * (nq + 1) + kl) * N + roff + l;
        // key words of chunk c in flight while chunk c - 1 is accumulated
        uint64_t ka[2][CH], kb[2][CH];
        auto load_keys = [&](int c, uint64_t (&k0v)[CH], uint64_t (&k1v)[CH]) {
#pragma unroll
            for (int k = 0; k < CH; k++) {
                k0v[k] = ld_stream(kp0 + (c * CH + k) * G::T);
                k1v[k] = ld_stream(kp1 + (c * CH + k) * G::T);
            }
        };
        load_keys(0, ka[0], kb[0]);
        if (i > 0) tmem_wait_st();  // the previous digit's accumulators are in place
#pragma unroll
        for (int c = 0; c < E / CH; c++) {
            if (c + 1 < E / CH) load_keys(c + 1, ka[(c + 1) & 1], kb[(c + 1) & 1]);
            uint32_t s0[4 * CH], s1[4 * CH];
            const uint32_t c0 = tbase + 4 * CH * c, c1 = tbase + 4 * E + 4 * CH * c;
            if (i > 0) {
                tmem_ld16(c0, s0);
                tmem_ld16(c1, s1);
                tmem_wait_ld32(s0, s1);
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    mac128(s0 + 4 * k, x[c * CH + k], ka[c & 1][k]);
                    mac128(s1 + 4 * k, x[c * CH + k], kb[c & 1][k]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    set128(s0 + 4 * k, x[c * CH + k], ka[c & 1][k]);
                    set128(s1 + 4 * k, x[c * CH + k], kb[c & 1][k]);
                }
            }
            if (i + 1 < nl) {
                tmem_st16(c0, s0);
                tmem_st16(c1, s1);
            } else {
                uint64_t r0[CH], r1[CH];
#pragma unroll
                for (int k = 0; k < CH; k++) {
                    uint64_t h0 = ((uint64_t)s0[4 * k + 3] << 32) | s0[4 * k + 2];
                    uint64_t h1 = ((uint64_t)s1[4 * k + 3] << 32) | s1[4 * k + 2];
                    // the high word is below q unless q > 2^64 / (20 nl) (LZ) or 2^64 / (4 nl)
                    h0 = h0 >= q ? reduce64(h0, m) : h0;
                    h1 = h1 >= q ? reduce64(h1, m) : h1;
                    r0[k] = redc128(h0, ((uint64_t)s0[4 * k + 1] << 32) | s0[4 * k], m);
                    r1[k] = redc128(h1, ((uint64_t)s1[4 * k + 1] << 32) | s1[4 * k], m);
                }
#pragma unroll
                for (int k = 0; k < CH; k += 2) {
                    *reinterpret_cast<ulonglong2 *>(o0 + c * CH + k) = make_ulonglong2(r0[k], r0[k + 1]);
                    *reinterpret_cast<ulonglong2 *>(o1 + c * CH + k) = make_ulonglong2(r1[k], r1[k + 1]);
                }
            }
        }
    }
    if (!ok) atomicOr(status, 2);
    tmem_fence_before();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tbase, TCOLS);  // warp 0's lane offset is 0: tbase is the allocation
    }
}

// Output stage of ModDown (and of rescale) fused with the row pass of its
// forward transform: the CTA finishes the transform of RPC rows of the lifted
// part of limb j (column pass already applied), then forms
// (src_j - lift_j) * inv_j (inv: P^-1 or q_l^-1 mod q_j, Shoup pairs) and the
// operation around the key switch (KsOut: + rel, + sigma_gal(rot_0), + acc) for
// those rows, so the lifted limbs are never written in evaluation form.
// src limb j of polynomial p of item b: src + b src_item + p src_poly + j N.
// grid: items * 2 polys * nl limbs * (R1 / RPC).
template <int K1, int K2, int RPC>
__global__ void __launch_bounds__(RPC * Geo<K2>::T, 1024 / (RPC * Geo<K2>::T))
    k_ks_down_rows(KsOut o, const uint64_t *__restrict__ srcp, size_t src_item, size_t src_poly,
                   const uint64_t *__restrict__ lift, const uint64_t *__restrict__ twall, const ModQ *__restrict__ mods,
                   const uint64_t *__restrict__ inv, int nl)
{
    using G = Geo<K2>;
    constexpr int R1 = 1 << K1, R2 = G::R, N = R1 * R2, NG = R1 / RPC, E = G::E, T = G::T, LOGN = K1 + K2;
    extern __shared__ uint64_t smem[];
    int bid = blockIdx.x;
    const int grp = bid % NG;
    bid /= NG;
    const int j = bid % nl;
    bid /= nl;
    const int p = bid & 1;
    const size_t bt = (size_t)(bid >> 1);
    const int l = threadIdx.x % T, rl = threadIdx.x / T;
    const int row = grp * RPC + rl;
    const ModQ mq = mods[j];
    const uint64_t q = mq.q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)j * N * 2;
    const uint64_t *rowp = lift + ((bt * 2 + p) * nl + j) * N + (size_t)row * R2;
    const uint64_t *sv = srcp + bt * src_item + p * src_poly;
    if (threadIdx.x == 0) {
        // the output stage's operand rows of this CTA (contiguous RPC rows of
        // limb j) start their way into L2 while the transform runs
        const size_t tile = (size_t)j * N + (size_t)grp * RPC * R2;
        constexpr unsigned bytes = RPC * R2 * 8;
        prefetch_l2(sv + tile, bytes);
        if (o.rel) prefetch_l2(o.rel + bt * o.rel_item + p * o.rel_poly + tile, bytes);
        if (o.acc) prefetch_l2(o.acc + bt * o.acc_item + p * o.acc_poly + tile, bytes);
    }
    uint64_t *seg = smem + rl * G::SEG;
    uint64_t x[E];
#pragma unroll
    for (int r = 0; r < E; r++) x[r] = rowp[l + T * r];
    const int A = R1 + row;
    fwd_strided<K2>(x, tw, A, q, q2);
    to_contig<K2>(x, seg, l);
    fwd_contig<K2, true>(x, tw, A, l, q, q2);
    __syncthreads();
    to_strided<K2>(x, seg, l);  // word l + T r of the row: coalesced below
    const uint64_t pv = inv[2 * j], pvp = inv[2 * j + 1], q4 = 4 * q;
    // lazy arithmetic, one reduction at the end: src + 4q - w < 5q (w < 4q from
    // Harvey's butterflies), the Shoup product < 2q, each added term < q (rel,
    // acc and up to HELR_MAX_HOIST rotation terms): the sum stays below
    // (4 + 7) q < 2^64 for primes below 2^60
    const size_t rowk = (size_t)j * N + (size_t)row * R2 + l;
#pragma unroll
    for (int r = 0; r < E; r++) {
        uint64_t v = shoup_lazy(sv[rowk + T * r] + (q4 - x[r]), pv, pvp, q);
        if (o.rel) v += o.rel[bt * o.rel_item + p * o.rel_poly + rowk + T * r];
        x[r] = v;
    }
    if (o.rot && p == 0) {
        // one rotation at a time: the CTA's reads of a rotation stay within the
        // source rows of its own rows, so L1 serves the repeated lines
        const uint64_t *rot = o.rot + bt * o.rot_item + (size_t)j * N;
        for (int g = 0; g < o.ngal; g++) {
            uint64_t gal = o.gals[0];
#pragma unroll
            for (int x2 = 1; x2 < HELR_MAX_HOIST; x2++)
                if (x2 == g) gal = o.gals[x2];
#pragma unroll
            for (int r = 0; r < E; r++) x[r] += rot[auto_pos<LOGN>((uint32_t)(row * R2 + l + T * r), gal)];
        }
    }
#pragma unroll
    for (int r = 0; r < E; r++) {
        uint64_t v = x[r];
        if (o.acc) v += o.acc[bt * o.acc_item + p * o.acc_poly + rowk + T * r];
        o.out.p[bt * o.out.item + p * o.out.poly + rowk + T * r] = reduce64(v, mq);
    }
}

// Hoisted rotations, step 1: the forward row pass of every lifted digit
// (column pass already applied by k_ks_modup_cols in ModUp mode), in place in
// mid[b][i][t] for the targets t != i (t = nl standing for P).  Words are
// reduced to [0, q_t) for primes of 2^58 and above; below that the unreduced
// butterflies leave them below 20 q_t.  grid: items * nl digits * nl targets
// * (R1 / RPC).
template <int K1, int K2, int RPC>
__global__ void __launch_bounds__(RPC * Geo<K2>::T, 3)
    k_ks_digit_rows(uint64_t *__restrict__ mid, const uint64_t *__restrict__ twall, const ModQ *__restrict__ mods, int nl,
                    int pidx)
{
    using G = Geo<K2>;
    constexpr int R1 = 1 << K1, R2 = G::R, N = R1 * R2, NG = R1 / RPC, E = G::E, T = G::T;
    extern __shared__ uint64_t smem[];
    int bid = blockIdx.x;
    const int grp = bid % NG;
    bid /= NG;
    const int tt = bid % nl;
    bid /= nl;
    const int i = bid % nl;
    const size_t b = (size_t)(bid / nl);
    const int t = tt < i ? tt : tt + 1;
    const int pt = t < nl ? t : pidx;
    const uint64_t q = mods[pt].q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pt * N * 2;
    const int l = threadIdx.x % T, rl = threadIdx.x / T;
    const int row = grp * RPC + rl;
    uint64_t *rowp = mid + ((b * nl + i) * (nl + 1) + t) * N + (size_t)row * R2;
    uint64_t *seg = smem + rl * G::SEG;
    uint64_t x[E];
#pragma unroll
    for (int r = 0; r < E; r++) x[r] = rowp[l + T * r];
    const int A = R1 + row;
    if (q < HELR_LZ_QMAX) {
        // unreduced butterflies: the words stay below 20q (< 2^47 for the
        // 40-bit primes), which the inner product accepts as they are
        fwd_strided<K2, true>(x, tw, A, q, q2);
        to_contig<K2>(x, seg, l);
        fwd_contig<K2, true, true>(x, tw, A, l, q, q2);
    } else {
        fwd_strided<K2>(x, tw, A, q, q2);
        to_contig<K2>(x, seg, l);
        fwd_contig<K2, true>(x, tw, A, l, q, q2);
#pragma unroll
        for (int r = 0; r < E; r++) {
            uint64_t v = x[r];
            v = v >= q2 ? v - q2 : v;
            x[r] = v >= q ? v - q : v;
        }
    }
    __syncthreads();
    to_strided<K2>(x, seg, l);
#pragma unroll
    for (int r = 0; r < E; r++) rowp[l + T * r] = x[r];
}

// Hoisted rotations, step 2: the inner products of every rotation j of hk,
// summed over j before the one ModDown:
//   acc_t = sum_j sum_i sigma_j(D_(i,t)) * key_j(i,t)     (both key polynomials)
// with D_(i,t) digit i of the second polynomial lifted into target t and
// transformed (mid, or the input itself in evaluation form when t == i).  The
// automorphism acts on the evaluation form as a permutation that maps every
// row of R2 words onto one source row (the top bits of a position decide the
// top bits of its image), so each output row gathers from one row of each
// digit, which L1 keeps while the row's threads read it.  Keys are in
// Montgomery form and in the row order of k_key_rows (word E l + r of a row
// at r T + l): thread u takes key positions u, u + TPR, ..., coalesced, and
// the columns they stand for.  Sums are exact in 128 bits and reduced once:
// at most HELR_MAX_HOIST * nl terms x k with k < q and x < q (primes of 2^58
// and above) or x < 20q (below 2^58; helr_rotsum refuses chains where that
// could reach 2^128).  A thread computes items b and b + 1 at the same
// positions, so every key word it loads serves both items.
//
// 128-bit sum of products x k for primes below 2^41 (x < 2^47, k < 2^41)
// without 64 x 64-bit products: with x = xh 2^32 + xl and k = kh 2^32 + kl,
// A (+ carries cA 2^64) sums xl kl and B sums xl kh + xh kl + xh kh 2^32 (each
// term < 2^57, and < 2^55 for x < 20q: B holds the 7 x 39 terms the context
// admits at most); T = A + cA 2^64 + B 2^32.
struct Acc40 {
    uint64_t A, B;
    uint32_t cA;
};
__device__ __forceinline__ void mac40(Acc40 &a, uint64_t x, uint64_t k)
{
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32), kl = (uint32_t)k, kh = (uint32_t)(k >> 32);
    const uint64_t p0 = (uint64_t)xl * kl;
    a.A += p0;
    a.cA += a.A < p0;
    a.B += (uint64_t)xl * kh + (uint64_t)xh * kl + ((uint64_t)(xh * kh) << 32);
}
// T 2^-64 mod q for the sum held by a (keys in Montgomery form)
__device__ __forceinline__ uint64_t redc40(const Acc40 &a, const ModQ &m)
{
    const uint64_t lo = a.A + (a.B << 32);
    uint64_t hi = a.cA + (a.B >> 32) + (lo < a.A);
    hi = hi >= m.q ? reduce64(hi, m) : hi;
    return redc128(hi, lo, m);
}

// grid: ceil(items / 2) item pairs (fastest: the items of a wave share each
// key row through L2) * (nl + 1 - t0) targets t0..nl * (R1 / RPC).
template <int K1, int K2>
struct HoistGeo {
    static constexpr int R1 = 1 << K1, R2 = 1 << K2;
    static constexpr int TPR = R2 / 2 < 128 ? R2 / 2 : 128;          // threads per row
    static constexpr int PPT = R2 / TPR;                             // positions per thread and item
    static constexpr int RPC = (256 / TPR) < R1 ? (256 / TPR) : R1;  // rows per CTA
    static constexpr int THREADS = RPC * TPR;
};
template <int K1, int K2, bool F40>
__device__ __forceinline__ void hoist_ip_body(const uint64_t *__restrict__ mid, const uint64_t *__restrict__ dntt,
                                               size_t din_item, const HoistKeys &hk, uint64_t *__restrict__ acc,
                                               const ModQ &m, int nl, int nq, int b0, bool two, int t, int kl, int row)
{
    using G = Geo<K2>;
    using H = HoistGeo<K1, K2>;
    constexpr int R1 = 1 << K1, R2 = 1 << K2, N = R1 * R2, LOGN = K1 + K2;
    constexpr int TPR = H::TPR, PPT = H::PPT;
    const int u = threadIdx.x % TPR;
    const size_t roff = (size_t)row * R2;
    const int b1 = two ? b0 + 1 : b0;
    int col[PPT];
#pragma unroll
    for (int mm = 0; mm < PPT; mm++) {
        const int p = u + TPR * mm;
        col[mm] = G::E * (p % G::T) + p / G::T;
    }
    Acc40 f0[2][PPT], f1[2][PPT];
    uint32_t a0[2][PPT][4], a1[2][PPT][4];
#pragma unroll
    for (int it = 0; it < 2; it++)
#pragma unroll
        for (int mm = 0; mm < PPT; mm++) {
            f0[it][mm] = f1[it][mm] = Acc40{0, 0, 0};
#pragma unroll
            for (int w = 0; w < 4; w++) a0[it][mm][w] = a1[it][mm][w] = 0;
        }
    for (int j = 0; j < hk.n; j++) {
        const uint64_t *key = hk.key[0];
        uint64_t gal = hk.gal[0];
#pragma unroll
        for (int g = 1; g < HELR_MAX_HOIST; g++)
            if (g == j) key = hk.key[g], gal = hk.gal[g];
        uint32_t ps[PPT];
#pragma unroll
        for (int mm = 0; mm < PPT; mm++) ps[mm] = auto_pos<LOGN>((uint32_t)(roff + col[mm]), gal);
        for (int i = 0; i < nl; i++) {
            const uint64_t *s0 = i == t ? dntt + (size_t)b0 * din_item + (size_t)i * N
                                        : mid + (((size_t)b0 * nl + i) * (nl + 1) + t) * N;
            const uint64_t *s1 = i == t ? dntt + (size_t)b1 * din_item + (size_t)i * N
                                        : mid + (((size_t)b1 * nl + i) * (nl + 1) + t) * N;
            const uint64_t *k0 = key + (((size_t)i * 2 + 0) * (nq + 1) + kl) * N + roff + u;
            const uint64_t *k1 = key + (((size_t)i * 2 + 1) * (nq + 1) + kl) * N + roff + u;
#pragma unroll
            for (int mm = 0; mm < PPT; mm++) {
                const uint64_t x0 = __ldg(s0 + ps[mm]), x1 = __ldg(s1 + ps[mm]);
                const uint64_t ka = ld_stream(k0 + TPR * mm), kb = ld_stream(k1 + TPR * mm);
                if constexpr (F40) {
                    mac40(f0[0][mm], x0, ka);
                    mac40(f1[0][mm], x0, kb);
                    mac40(f0[1][mm], x1, ka);
                    mac40(f1[1][mm], x1, kb);
                } else {
                    mac128(a0[0][mm], x0, ka);
                    mac128(a1[0][mm], x0, kb);
                    mac128(a0[1][mm], x1, ka);
                    mac128(a1[1][mm], x1, kb);
                }
            }
        }
    }
#pragma unroll
    for (int it = 0; it < 2; it++) {
        if (it == 1 && !two) break;
        const int b = b0 + it;
        uint64_t *o0 = acc + (((size_t)b * 2 + 0) * (nl + 1) + t) * N + roff;
        uint64_t *o1 = acc + (((size_t)b * 2 + 1) * (nl + 1) + t) * N + roff;
#pragma unroll
        for (int mm = 0; mm < PPT; mm++) {
            if constexpr (F40) {
                o0[col[mm]] = redc40(f0[it][mm], m);
                o1[col[mm]] = redc40(f1[it][mm], m);
            } else {
                uint64_t h0 = ((uint64_t)a0[it][mm][3] << 32) | a0[it][mm][2];
                uint64_t h1 = ((uint64_t)a1[it][mm][3] << 32) | a1[it][mm][2];
                h0 = h0 >= m.q ? reduce64(h0, m) : h0;
                h1 = h1 >= m.q ? reduce64(h1, m) : h1;
                o0[col[mm]] = redc128(h0, ((uint64_t)a0[it][mm][1] << 32) | a0[it][mm][0], m);
                o1[col[mm]] = redc128(h1, ((uint64_t)a1[it][mm][1] << 32) | a1[it][mm][0], m);
            }
        }
    }
}

template <int K1, int K2>
__global__ void __launch_bounds__(HoistGeo<K1, K2>::THREADS, 3)
    k_ks_hoist_ip(const uint64_t *__restrict__ mid, const uint64_t *__restrict__ dntt, size_t din_item, HoistKeys hk,
                   uint64_t *__restrict__ acc, const ModQ *__restrict__ mods, int nl, int nq, int pidx, int items, int t0)
{
    using H = HoistGeo<K1, K2>;
    constexpr int R1 = 1 << K1, NG = R1 / H::RPC;
    const int npair = (items + 1) / 2;
    int bid = blockIdx.x;
    const int b0 = 2 * (bid % npair);
    bid /= npair;
    const int grp = bid % NG;
    const int t = t0 + bid / NG;
    const int pt = t < nl ? t : pidx, kl = t < nl ? t : nq;
    const ModQ m = mods[pt];
    const int row = grp * H::RPC + threadIdx.x / H::TPR;
    const bool two = b0 + 1 < items;
    if (m.q < (1ull << 41))
        hoist_ip_body<K1, K2, true>(mid, dntt, din_item, hk, acc, m, nl, nq, b0, two, t, kl, row);
    else
        hoist_ip_body<K1, K2, false>(mid, dntt, din_item, hk, acc, m, nl, nq, b0, two, t, kl, row);
}

template <int K1, int K2>
struct KsPlan {
    static constexpr int T1 = Geo<K1>::T, T2 = Geo<K2>::T;
    static constexpr int R1 = 1 << K1, R2 = 1 << K2;
    static constexpr int C = (256 / T1) < R2 ? (256 / T1) : R2;
    static constexpr int RPC = (128 / T2) < R1 ? (128 / T2) : R1;
    static constexpr int RPCD = (256 / T2) < R1 ? (256 / T2) : R1;
    // tile variants chosen per limb count by he_autotune (tile bit 0: half as
    // many columns per CTA in the column kernel; bit 1: half as many rows per
    // CTA in the row kernels of ModDown and of the hoisted digits)
    static constexpr int CB = C / 2 > 0 ? C / 2 : 1;
    static constexpr int RB = RPCD / 2 > 0 ? RPCD / 2 : 1;
    // a launch of fewer than two CTAs per SM (a wave of one or a few items)
    // takes the narrower tile, with twice the CTAs
    static bool small(const he_ctx *c, size_t ctas) { return ctas < 2 * (size_t)c->sms; }
    static constexpr size_t smd(int rr) { return (size_t)rr * Geo<K2>::SEG * 8; }
    static constexpr size_t sm1(int cc) { return (size_t)cc * Geo<K1>::SEG * 8 + (size_t)cc * R1 * 8; }
    static constexpr size_t SMD = smd(RPCD);
    static constexpr size_t SM1 = sm1(C);
    // one digit's rows, the row twiddle pairs, the TMEM address slot
    static constexpr size_t SM2 = (size_t)RPC * R2 * 8 + (size_t)RPC * R2 * 16 + 16;
    static cudaError_t prepare()
    {
        cudaError_t e = helr_fit_carveout((const void *)k_ks_modup_cols<K1, K2, C, false>, C * T1, SM1);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_modup_cols<K1, K2, C, true>, C * T1, SM1);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_inner_rows<K1, K2, RPC, false>, RPC * T2, SM2);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_inner_rows<K1, K2, RPC, true>, RPC * T2, SM2);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_down_rows<K1, K2, RPCD>, RPCD * T2, SMD);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_digit_rows<K1, K2, RPCD>, RPCD * T2, SMD);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_hoist_ip<K1, K2>, HoistGeo<K1, K2>::THREADS, 0);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_modup_cols<K1, K2, CB, false>, CB * T1, sm1(CB));
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_modup_cols<K1, K2, CB, true>, CB * T1, sm1(CB));
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_down_rows<K1, K2, RB>, RB * T2, smd(RB));
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ks_digit_rows<K1, K2, RB>, RB * T2, smd(RB));
        return e;
    }
    template <int CC, bool DOWN>
    static void cols(he_ctx *c, const uint64_t *drow, uint64_t *out, size_t nsrc, int nl, int src_prime, cudaStream_t s)
    {
        const unsigned grid = (unsigned)(nsrc * (R2 / CC));
        HELR_LAUNCH(k_ks_modup_cols<K1, K2, CC, DOWN><<<grid, CC * T1, sm1(CC), s>>>(drow, out, c->t.tw, c->t.itw, c->t.mod,
                                                                                      c->t.ninv, nl, c->nq, src_prime));
    }
    // hoisted rotations: row passes of the lifted digits, then the summed inner products
    static int hoisted(he_ctx *c, const uint64_t *dntt, size_t din_item, uint64_t *mid, const HoistKeys &hk, uint64_t *acc,
                       int items, int nl, cudaStream_t s)
    {
        if ((helr_ks_tile(c, nl) & 2) || small(c, (size_t)items * nl * nl * (R1 / RPCD))) {
            const unsigned g1 = (unsigned)((size_t)items * nl * nl * (R1 / RB));
            HELR_LAUNCH(k_ks_digit_rows<K1, K2, RB><<<g1, RB * T2, smd(RB), s>>>(mid, c->t.tw, c->t.mod, nl, c->nq));
        } else {
            const unsigned g1 = (unsigned)((size_t)items * nl * nl * (R1 / RPCD));
            HELR_LAUNCH(k_ks_digit_rows<K1, K2, RPCD><<<g1, RPCD * T2, SMD, s>>>(mid, c->t.tw, c->t.mod, nl, c->nq));
        }
        // the tensor-core form takes the run of 40-bit targets [a, b) where it
        // applies; the CUDA cores take targets [0, a) and [b, nl] (nl = P)
        using H = HoistGeo<K1, K2>;
        int a = nl + 1, b = nl + 1;
        if (helr_hoist_form(c, nl) == 1 && helr_hoist_tensor_range(c, nl, hk.n, &a, &b))
            HELR_TRY(helr_hoist_ip_tensor(c, mid, dntt, din_item, hk, acc, items, nl, a, b, s));
        const int runs[2][2] = {{0, a}, {b, nl + 1}};
        for (const auto &r : runs)
            if (r[1] > r[0]) {
                const unsigned g2 = (unsigned)((size_t)((items + 1) / 2) * (r[1] - r[0]) * (R1 / H::RPC));
                HELR_LAUNCH(k_ks_hoist_ip<K1, K2><<<g2, H::THREADS, 0, s>>>(mid, dntt, din_item, hk, acc, c->t.mod, nl,
                                                                              c->nq, c->nq, items, r[0]));
            }
        return HE_OK;
    }
    static void down(he_ctx *c, const KsOut &o, const uint64_t *src, size_t src_item, size_t src_poly, const uint64_t *lift,
                     int items, int nl, const uint64_t *inv, cudaStream_t s)
    {
        if ((helr_ks_tile(c, nl) & 2) || small(c, (size_t)items * 2 * nl * (R1 / RPCD))) {
            const unsigned grid = (unsigned)((size_t)items * 2 * nl * (R1 / RB));
            HELR_LAUNCH(k_ks_down_rows<K1, K2, RB><<<grid, RB * T2, smd(RB), s>>>(o, src, src_item, src_poly, lift, c->t.tw,
                                                                                  c->t.mod, inv, nl));
        } else {
            const unsigned grid = (unsigned)((size_t)items * 2 * nl * (R1 / RPCD));
            HELR_LAUNCH(k_ks_down_rows<K1, K2, RPCD><<<grid, RPCD * T2, SMD, s>>>(o, src, src_item, src_poly, lift, c->t.tw,
                                                                                  c->t.mod, inv, nl));
        }
    }
    static void down_cols(he_ctx *c, const uint64_t *drow, size_t nsrc, int src_prime, uint64_t *out, int nl, cudaStream_t s)
    {
        if ((helr_ks_tile(c, nl) & 1) || small(c, nsrc * (R2 / C)))
            cols<CB, true>(c, drow, out, nsrc, nl, src_prime, s);
        else
            cols<C, true>(c, drow, out, nsrc, nl, src_prime, s);
    }
    // targets 0..nl of a key switch at nl limbs (nl = P) whose prime takes (lz) or
    // does not take the unreduced forward butterfly
    static PosList targets(const he_ctx *c, int nl, bool lz)
    {
        LimbMap m = limbmap_ct(nl - 1);
        m.period = nl + 1;
        m.p[nl] = (unsigned char)c->nq;
        return poslist_of(c, m, lz);
    }
    static int modup(he_ctx *c, const uint64_t *drow, uint64_t *mid, int items, int nl, cudaStream_t s)
    {
        if ((helr_ks_tile(c, nl) & 1) || small(c, (size_t)items * nl * (R2 / C)))
            cols<CB, false>(c, drow, mid, (size_t)items * nl, nl, 0, s);
        else
            cols<C, false>(c, drow, mid, (size_t)items * nl, nl, 0, s);
        return 1;
    }
    static int inner(he_ctx *c, const uint64_t *mid, const uint64_t *dntt, const uint64_t *key, uint64_t *acc, int items,
                     int nl, cudaStream_t s)
    {
        int launches = 0;
        for (int lz = 0; lz < 2; lz++) {
            const PosList tl = targets(c, nl, lz);
            if (!tl.n) continue;
            const unsigned grid = (unsigned)((size_t)items * tl.n * (R1 / RPC));
            if (lz)
                HELR_LAUNCH(k_ks_inner_rows<K1, K2, RPC, true><<<grid, RPC * T2, SM2, s>>>(mid, dntt, key, acc, c->t.tw, c->t.mod,
                                                                                        nl, c->nq, c->nq, items, tl, c->d_status));
            else
                HELR_LAUNCH(k_ks_inner_rows<K1, K2, RPC, false><<<grid, RPC * T2, SM2, s>>>(mid, dntt, key, acc, c->t.tw, c->t.mod,
                                                                                         nl, c->nq, c->nq, items, tl, c->d_status));
            launches++;
        }
        return launches;
    }
};

template <int K1, int K2>
int run_fused(he_ctx *c, const uint64_t *dntt, const uint64_t *drow, uint64_t *mid, const uint64_t *key, uint64_t *acc,
              int items, int nl, cudaStream_t s)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, (KsPlan<K1, K2>::prepare()));
        prepared = true;
    }
    prof_start(c, PROF_MODUP, s);
    const int l1 = KsPlan<K1, K2>::modup(c, drow, mid, items, nl, s);
    // forward column passes of (digit, target != digit), inverse column passes of the digits;
    // DRAM: digits read once, column-pass limbs written
    prof_stop(c, PROF_MODUP, s, (double)items * nl * nl, l1, (double)items * nl, (double)items * nl * (nl + 1));
    prof_start(c, PROF_KS_INNER, s);
    const int l2 = KsPlan<K1, K2>::inner(c, mid, dntt, key, acc, items, nl, s);
    // row passes: nl - 1 digits for each ciphertext target, nl for P; products: 2 keys x nl digits x (nl + 1) targets
    // DRAM: every digit's rows read once per target, the two key polynomials once per launch, acc written
    prof_stop(c, PROF_KS_INNER, s, (double)items * nl * nl, l2, (double)items * 2 * nl * (nl + 1),
              (double)items * nl * (nl + 1) + 2.0 * nl * (nl + 1) + (double)items * 2 * (nl + 1));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

}  // namespace

// ModUp + transforms + inner product for `items` polynomials: dntt is the
// input [items][nl][N] in evaluation form, drow the same after the row pass of
// the inverse transform; mid is scratch of [items][nl][nl+1][N]; acc receives
// [items][2][nl+1][N].
int helr_ks_fused(he_ctx *c, const uint64_t *dntt, const uint64_t *drow, uint64_t *mid, const uint64_t *key, uint64_t *acc,
                  int items, int nl, cudaStream_t s)
{
    switch (c->logn) {
    case 10: return run_fused<5, 5>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 11: return run_fused<5, 6>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 12: return run_fused<6, 6>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 13: return run_fused<6, 7>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 14: return run_fused<7, 7>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 15: return run_fused<7, 8>(c, dntt, drow, mid, key, acc, items, nl, s);
    case 16: return run_fused<8, 8>(c, dntt, drow, mid, key, acc, items, nl, s);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}

template <int K1, int K2>
int run_hoisted(he_ctx *c, const uint64_t *dntt, size_t din_item, const uint64_t *drow, uint64_t *mid, const HoistKeys &hk,
                uint64_t *acc, int items, int nl, cudaStream_t s)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, (KsPlan<K1, K2>::prepare()));
        prepared = true;
    }
    prof_start(c, PROF_MODUP, s);
    const int l1 = KsPlan<K1, K2>::modup(c, drow, mid, items, nl, s);
    prof_stop(c, PROF_MODUP, s, (double)items * nl * nl, l1, (double)items * nl, (double)items * nl * (nl + 1));
    prof_start(c, PROF_KS_INNER, s);
    HELR_TRY((KsPlan<K1, K2>::hoisted(c, dntt, din_item, mid, hk, acc, items, nl, s)));
    // row passes of the nl x nl lifted digits; products: rotations x 2 keys x nl digits x (nl + 1) targets;
    // DRAM: digit rows read and written once, read once per rotation (gathers), keys once per launch, acc written
    prof_stop(c, PROF_KS_INNER, s, (double)items * nl * nl, 2, (double)items * hk.n * 2 * nl * (nl + 1),
              (double)items * nl * nl * 2 + (double)items * hk.n * nl * (nl + 1) + hk.n * 2.0 * nl * (nl + 1) +
                  (double)items * 2 * (nl + 1));
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int helr_ks_hoisted(he_ctx *c, const uint64_t *dntt, size_t din_item, const uint64_t *drow, uint64_t *mid,
                    const HoistKeys &hk, uint64_t *acc, int items, int nl, cudaStream_t s)
{
    if (hk.n < 1 || hk.n > HELR_MAX_HOIST) return helr_fail(c, HE_EINVAL, "%d rotations in one hoisted sum", hk.n);
    switch (c->logn) {
    case 10: return run_hoisted<5, 5>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 11: return run_hoisted<5, 6>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 12: return run_hoisted<6, 6>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 13: return run_hoisted<6, 7>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 14: return run_hoisted<7, 7>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 15: return run_hoisted<7, 8>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    case 16: return run_hoisted<8, 8>(c, dntt, din_item, drow, mid, hk, acc, items, nl, s);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}

// reorder the rows of nlimbs key limbs ([nlimbs][N], evaluation form) for k_ks_inner_rows
int helr_ks_key_layout(he_ctx *c, uint64_t *key, size_t nlimbs)
{
    const unsigned rows = (unsigned)(nlimbs * (size_t)c->n >> (c->logn - c->logn / 2));
    switch (c->logn - c->logn / 2) {
    case 5: HELR_LAUNCH(k_key_rows<5><<<rows, 1 << 5, 0, c->stream>>>(key)); break;
    case 6: HELR_LAUNCH(k_key_rows<6><<<rows, 1 << 6, 0, c->stream>>>(key)); break;
    case 7: HELR_LAUNCH(k_key_rows<7><<<rows, 1 << 7, 0, c->stream>>>(key)); break;
    case 8: HELR_LAUNCH(k_key_rows<8><<<rows, 1 << 8, 0, c->stream>>>(key)); break;
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

template <int K1, int K2>
int run_down(he_ctx *c, const KsOut *o, const uint64_t *src, size_t src_item, size_t src_poly, const uint64_t *drow,
             int src_prime, uint64_t *lift, int items, int nl, const uint64_t *inv, cudaStream_t s)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, (KsPlan<K1, K2>::prepare()));
        prepared = true;
    }
    if (drow) {
        // the column kernel is the one ModUp runs, timed with it: 2 nl forward
        // column halves and 2 inverse column halves per item; DRAM: 2 source
        // limbs read, 2 nl written
        prof_start(c, PROF_MODUP, s);
        KsPlan<K1, K2>::down_cols(c, drow, (size_t)items * 2, src_prime, lift, nl, s);
        prof_stop(c, PROF_MODUP, s, (double)items * 2 * nl, 1, (double)items * 2, (double)items * 2 * (nl + 1));
    }
    if (o) {
        prof_start(c, PROF_NTT_FWD, s);
        KsPlan<K1, K2>::down(c, *o, src, src_item, src_poly, lift, items, nl, inv, s);
        prof_stop(c, PROF_NTT_FWD, s, 0.5 * items * 2 * nl, 1);  // row halves of 2 nl transforms per item
    }
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

static int down_dispatch(he_ctx *c, const KsOut *o, const uint64_t *src, size_t src_item, size_t src_poly,
                         const uint64_t *drow, int src_prime, uint64_t *lift, int items, int nl, const uint64_t *inv,
                         cudaStream_t s)
{
    if (items <= 0) return HE_OK;
    switch (c->logn) {
    case 10: return run_down<5, 5>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 11: return run_down<5, 6>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 12: return run_down<6, 6>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 13: return run_down<6, 7>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 14: return run_down<7, 7>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 15: return run_down<7, 8>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    case 16: return run_down<8, 8>(c, o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}

// Division by a dropped prime with rounding, for ModDown (by P) and rescale (by
// q_l), after the inverse row pass of the dropped limbs: drow holds
// [items][2][N], the dropped limb of every polynomial (prime src_prime) after
// the row pass of its inverse transform.  The kernels finish its inverse
// transform, lift it centred into q_0..q_(nl-1), transform it forward
// (lift: [items][2][nl][N] scratch) and write o.out = (src - lift) * inv plus
// the KsOut terms, inv holding Shoup pairs of the inverse of the dropped prime
// modulo each q_j.
int helr_ks_down(he_ctx *c, const KsOut &o, const uint64_t *src, size_t src_item, size_t src_poly, const uint64_t *drow,
                 int src_prime, uint64_t *lift, int items, int nl, const uint64_t *inv, cudaStream_t s)
{
    return down_dispatch(c, &o, src, src_item, src_poly, drow, src_prime, lift, items, nl, inv, s);
}

