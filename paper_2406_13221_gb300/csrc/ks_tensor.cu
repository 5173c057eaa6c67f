// ks_tensor.cu -- the hoisted inner product of a rotation group on the tensor
// cores (tcgen05.mma, kind::f16), an alternative form of k_ks_hoist_ip chosen
// with he_set_hoist_form.
//
// The hoisted key switch of a group of r rotations (Sec. 2.1 rotations, summed
// as in Sec. 2.2 / 3.3) ends in, for every item b, target t and position p,
//   T_b,poly = sum over pairs (j, i) of x_b[j, i] * k[j, i, poly]
// with x_b[j, i] the word of lifted digit i of item b that rotation j moves to
// p, and k the key word (both polynomials).  The keys are the same for every
// item of a wave, so at one position this is a product of the items' digit
// matrix with the keys: a contraction over the pairs.  It is made exact on
// FP16 operands by splitting every word into bytes: with x = sum_s x_s 2^(8s)
// and k = sum_s' k_s' 2^(8s'),
//   T = sum_d 2^(8d) D_d,   D_d = sum over pairs and s + s' = d of x_s k_s'.
// One MMA per position computes every D_d at once, for 128 items (M) and both
// key polynomials (N = 2 x 16 columns, 10 of them used):
//   A[b][(pair, s)] = x_s    (8 FP16 values per pair, bytes 6, 7 zero),
//   B[(pair, s)][(poly, d)] = k_(d - s)   (the key bytes in Toeplitz order).
// Bytes are integers below 256, so every product is exact in FP16 x FP16 and
// every D_d is an integer below pairs x 5 x 255^2, exact in the FP32
// accumulator while pairs <= 51 (below 2^24; the accumulation is exact for
// integers in that range on sm_103a, pinned by the tests through bit-exact
// results).  The epilogue converts D_0..D_9 to integers, forms T in 128 bits
// and reduces it exactly as the CUDA-core form does (keys in Montgomery form:
// T 2^-64 mod q), so both forms give the same words.
//
// Conditions (helr_hoist_tensor_range): the targets taken are a run of primes
// below 2^40 (keys below 2^40: five bytes; lifted digits below 20 q < 2^48:
// six bytes), r * nl <= 51 and nl <= 8.  The other targets (the 60-bit q_0
// and P of the training chain) keep the CUDA-core form.
//
// Data movement.  A CTA owns 128 items of the wave, one target and one row of
// R2 positions, taken in groups of 4 positions: the automorphism maps 4
// consecutive positions onto the 4 words of one 32-byte sector of the source
// row (in a rotation-dependent order), so a group needs one sector per item,
// digit and rotation.  A round is one (group, rotation): its sectors (cp.async,
// 4 rounds ahead) are split into bytes and written into the items' TMEM lanes
// as the A operand; the key bytes (cp.async, 4 rounds ahead) are laid out in
// shared memory as B; one thread issues 4 positions x nl/2 MMAs that
// accumulate over the group's rotations in TMEM.  Operand buffers and
// accumulators are double-buffered; mbarriers (tcgen05.commit) release them.
// Every wait is bounded (1 s of the global timer); on expiry the kernel sets
// bit 0 of the context's device status word and carries on, so it always
// returns and frees its tensor memory.
//
// Measured on GB300 (7 rotations, 6 limbs, 128 items at N = 2^16) it is slower
// than the CUDA-core form, 27.2 against 11.8 ms per rotation sum.  The tensor
// pipe is active 4% of the time.  Splitting digit words into bytes, the
// Toeplitz key layout and two barriers per round of 4 positions cost more than
// the 32-bit partial products they replace.  The per-item sector gathers also
// read about 1.8 times the DRAM bytes.  he_autotune measures both forms and keeps
// this one only where it is faster.
#include <stdint.h>

#include "ntt_core.cuh"

namespace {

constexpr int MT = 128;        // items per CTA (MMA M, one TMEM lane each)
constexpr int THREADS = 256;   // two threads per item (each half of the digits)
constexpr int GP = 4;          // positions per group (one source sector)
constexpr int NCOL = 32;       // MMA N: 2 key polynomials x 16 diagonal columns
constexpr int ND = 10;         // diagonals used: 6 digit bytes + 5 key bytes - 1
constexpr int PD = 4;          // rounds of copies in flight ahead of the current one
constexpr int RING = PD + 1;
constexpr int KW = 64;         // key words per round (GP x 2 x nl, nl <= 8)
constexpr int BMAX = 3;        // B chunks per thread and round (GP x 2 x ND x nl <= 640)
constexpr int NLMAX = 8;
constexpr int PAIRS_MAX = 51;  // pairs x 5 x 255^2 < 2^24

// shared-memory matrix descriptor, canonical K-major layout without swizzle:
// 8 rows x 16 bytes per core matrix, lbo between core matrices along K, sbo
// between groups of 8 rows
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
    return d;
}
// two halves 0x64vv (1024 + v) minus 1024: the FP16 values v, exactly
__device__ __forceinline__ uint32_t unbias(uint32_t v)
{
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(v), "r"(0xE400E400u));
    return d;
}
__device__ __forceinline__ void cp16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t ta, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ta), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t (&w)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15}, [%16];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                   "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
                 : "r"(ta));
}
// T = sum_d D_d 2^(8d) from the diagonal sums (integers below 2^24 in FP32),
// then T 2^-64 mod q; T < 51 x 2^48 x 2^40, so its high word is below q
__device__ __forceinline__ uint64_t combine(const uint32_t (&w)[16], const ModQ &m)
{
    uint32_t u[ND];
#pragma unroll
    for (int d = 0; d < ND; d++) asm("cvt.rzi.u32.f32 %0, %1;" : "=r"(u[d]) : "f"(__uint_as_float(w[d])));
    const uint64_t lo = (uint64_t)u[0] + ((uint64_t)u[1] << 8) + ((uint64_t)u[2] << 16) + ((uint64_t)u[3] << 24) +
                        ((uint64_t)u[4] << 32);
    const uint64_t hi = (uint64_t)u[5] + ((uint64_t)u[6] << 8) + ((uint64_t)u[7] << 16) + ((uint64_t)u[8] << 24) +
                        ((uint64_t)u[9] << 32);
    const uint64_t tl = lo + (hi << 40);
    const uint64_t th = (hi >> 24) + (tl < lo);
    return redc128(th, tl, m);
}

// grid: (items / 128 rounded up) x R1 rows x the targets t_lo.. (every one
// with q_t < 2^40), items fastest.  mid, dntt, din_item, hk, acc as for
// k_ks_hoist_ip.  Dynamic shared memory: hoist_mma_smem(nl).
template <int K1, int K2>
__global__ void __launch_bounds__(THREADS, 1)
    k_ks_hoist_mma(const uint64_t *__restrict__ mid, const uint64_t *__restrict__ dntt, size_t din_item, HoistKeys hk,
                   uint64_t *__restrict__ acc, const ModQ *__restrict__ mods, int nl, int nq, int items, int t_lo,
                   int *status)
{
    constexpr int R1 = 1 << K1, R2 = 1 << K2, N = R1 * R2, LOGN = K1 + K2;
    constexpr int E = nttc::Geo<K2>::E, T = nttc::Geo<K2>::T;  // key rows: word E l + r at r T + l
    constexpr int NG = R2 / GP;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int nlp = (nl + 1) & ~1, nl2 = (nl + 1) / 2, nrot = hk.n;
    const int ntile = (items + MT - 1) / MT;
    int bid = blockIdx.x;
    const int tile = bid % ntile;
    bid /= ntile;
    const int row = bid % R1;
    const int t = t_lo + bid / R1;
    const ModQ m = mods[t];
    const size_t roff = (size_t)row * R2;
    // shared memory: copy ring [RING][nl][2 halves][MT] x 16 bytes; B [2][GP]
    // x 32 rows x nlp chunks of 16 bytes; key ring [RING][KW]; 2 mbarriers; TMEM slot
    uint8_t *ring = sm;
    uint8_t *bsm = ring + (size_t)RING * nl * 2 * MT * 16;
    const uint32_t bpos = 32u * (uint32_t)nlp * 16u;
    uint64_t *kring = (uint64_t *)(bsm + 2 * GP * bpos);
    uint64_t *mbar = kring + RING * KW;
    uint32_t *slot = (uint32_t *)(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int mi = quarter * 32 + lane;  // the item's TMEM lane
    const int b = tile * MT + mi;
    const bool live = b < items;
    const int i0 = half * nl2, i1 = min(nl, i0 + nl2);
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t bsm_s = (uint32_t)__cvta_generic_to_shared(bsm);
    const uint32_t kring_s = (uint32_t)__cvta_generic_to_shared(kring);
    const uint32_t mb0 = (uint32_t)__cvta_generic_to_shared(mbar);
    // this thread's B chunks (the same in every round): offset, key word, byte selectors
    const int nb = GP * 2 * ND * nl;
    uint32_t boff[BMAX], bkw[BMAX], bsel[BMAX][4];
#pragma unroll
    for (int x = 0; x < BMAX; x++) {
        int k = tid + x * THREADS < nb ? tid + x * THREADS : 0;
        const int i = k % nl;
        k /= nl;
        const int d = k % ND;
        k /= ND;
        const int poly = k & 1, e = k >> 1;
        const int n = poly * 16 + d;
        boff[x] = (uint32_t)(e * bpos + (n >> 3) * nlp * 128 + i * 128 + (n & 7) * 16);
        bkw[x] = (uint32_t)((e * 2 + poly) * nl + i);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            // halves s = 2 sp, 2 sp + 1 take key bytes d - s; byte 7 (zero) outside 0..4
            const int k0 = d - 2 * sp, k1 = d - 2 * sp - 1;
            const uint32_t s0 = (unsigned)k0 < 5u ? (uint32_t)k0 : 7u, s1 = (unsigned)k1 < 5u ? (uint32_t)k1 : 7u;
            bsel[x][sp] = s0 | 0x70u | (s1 << 8) | 0x7000u;
        }
    }
    for (uint32_t k = tid; k < 2 * GP * bpos / 16; k += THREADS) *(uint4 *)(bsm + 16 * k) = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(slot);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(sa) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * quarter) << 16);
    // TMEM columns: accumulators D[gb][e] at gb 128 + e 32; A operands at 256 +
    // (rb GP + e) nlp 4, one 16-byte chunk (4 columns) per pair
    auto acol = [&](int rb, int e) { return 256u + (uint32_t)((rb * GP + e) * nlp * 4); };
    if (half == 0 && (nl & 1))  // the pad pair of an odd digit count stays zero
        for (int rb = 0; rb < 2; rb++)
            for (int e = 0; e < GP; e++) tmem_st4(tlane + acol(rb, e) + 4 * nl, 0, 0, 0, 0);
    const int R = NG * nrot;  // rounds: (group, rotation), rotations fastest
    auto rot_of = [&](int j, uint64_t &gal, const uint64_t *&key) {
        gal = hk.gal[0];
        key = hk.key[0];
#pragma unroll
        for (int x = 1; x < HELR_MAX_HOIST; x++)
            if (x == j) gal = hk.gal[x], key = hk.key[x];
    };
    auto issue = [&](int r) {
        if (r < R) {
            const int g = r / nrot, j = r % nrot;
            uint64_t gal;
            const uint64_t *key;
            rot_of(j, gal, key);
            if (live) {
                const uint32_t sec = auto_pos<LOGN>((uint32_t)(roff + GP * g), gal) & ~3u;
                const uint32_t st = ring_s + (uint32_t)((r % RING) * nl * 2 * MT * 16);
                for (int i = i0; i < i1; i++) {
                    const uint64_t *src = (i == t ? dntt + (size_t)b * din_item + (size_t)i * N
                                                  : mid + (((size_t)b * nl + i) * (nl + 1) + t) * N) +
                                          sec;
                    cp16(st + (uint32_t)(((i * 2 + 0) * MT + mi) * 16), src);
                    cp16(st + (uint32_t)(((i * 2 + 1) * MT + mi) * 16), src + 2);
                }
            }
            if (tid < GP * 2 * nl) {
                const int i = tid % nl, poly = (tid / nl) & 1, e = tid / (2 * nl);
                const int c = GP * g + e;
                const uint64_t *src =
                    key + ((size_t)(i * 2 + poly) * (nq + 1) + t) * N + roff + (size_t)(c % E) * T + c / E;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(kring_s + (uint32_t)(((r % RING) * KW + tid) * 8)),
                             "l"(src)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto epilogue = [&](int g) {
        // this thread: its item, positions 2 half and 2 half + 1, both polynomials
        const uint32_t dcol = (uint32_t)((g & 1) * 128);
        uint32_t w[4][16];
#pragma unroll
        for (int x = 0; x < 4; x++)
            tmem_ld16(tlane + dcol + (uint32_t)((2 * half + (x >> 1)) * 32 + 16 * (x & 1)), w[x]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint64_t res[4];
#pragma unroll
        for (int x = 0; x < 4; x++) res[x] = combine(w[x], m);
        if (live) {
            const size_t pos = roff + GP * g + 2 * half;
            uint64_t *o0 = acc + (((size_t)b * 2 + 0) * (nl + 1) + t) * N + pos;
            uint64_t *o1 = acc + (((size_t)b * 2 + 1) * (nl + 1) + t) * N + pos;
            *(ulonglong2 *)o0 = make_ulonglong2(res[0], res[2]);
            *(ulonglong2 *)o1 = make_ulonglong2(res[1], res[3]);
        }
    };
    // f32 accumulators, f16 A and B, both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | ((uint32_t)(NCOL >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
    bool ok = true;
    for (int r = 0; r < PD; r++) issue(r);
    for (int r = 0; r < R; r++) {
        issue(r + PD);
        const int rb = r & 1;
        if (r >= 2) {
            // the MMAs of round r - 2 have read buffers rb; a group whose last
            // rotation that was is complete in TMEM
            ok &= mbar_wait_bounded(mb0 + 8 * rb, (uint32_t)((r - 2) >> 1) & 1u);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if ((r - 2) % nrot == nrot - 1) epilogue((r - 2) / nrot);
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(PD) : "memory");
        const int g = r / nrot, j = r % nrot;
        uint64_t gal;
        const uint64_t *key;
        rot_of(j, gal, key);
        // position e reads word brev2((c0 + gal brev2(e)) mod 4) of the sector,
        // c0 = brev2 of the word position 0 reads; word w goes to the columns of
        // the position that reads it
        uint32_t colw[4] = {0, 0, 0, 0};
        {
            const uint32_t w0 = auto_pos<LOGN>((uint32_t)(roff + GP * g), gal) & 3u, ga = (uint32_t)gal & 3u;
            const uint32_t c0 = ((w0 & 1u) << 1) | (w0 >> 1);
#pragma unroll
            for (int e = 0; e < GP; e++) {
                const uint32_t v = (c0 + ga * (uint32_t)(((e & 1) << 1) | (e >> 1))) & 3u;
                const uint32_t w = ((v & 1u) << 1) | (v >> 1);
#pragma unroll
                for (int x = 0; x < 4; x++)
                    if (w == (uint32_t)x) colw[x] = acol(rb, e);
            }
        }
        const uint32_t st = ring_s + (uint32_t)((r % RING) * nl * 2 * MT * 16);
        for (int i = i0; i < i1; i++) {
            uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
            if (live) {
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v0.x), "=r"(v0.y), "=r"(v0.z), "=r"(v0.w)
                             : "r"(st + (uint32_t)(((i * 2 + 0) * MT + mi) * 16)));
                asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v1.x), "=r"(v1.y), "=r"(v1.z), "=r"(v1.w)
                             : "r"(st + (uint32_t)(((i * 2 + 1) * MT + mi) * 16)));
            }
            const uint32_t lo[4] = {v0.x, v0.z, v1.x, v1.z}, hi[4] = {v0.y, v0.w, v1.y, v1.w};
#pragma unroll
            for (int x = 0; x < 4; x++) {
                // bytes 0..5 of the word as FP16 pairs (0x64 high bytes, then minus 1024)
                const uint32_t c0 = unbias(prmt(lo[x], 0x64646464u, 0x4140u));
                const uint32_t c1 = unbias(prmt(lo[x], 0x64646464u, 0x4342u));
                const uint32_t c2 = unbias(prmt(hi[x], 0x64646464u, 0x4140u));
                tmem_st4(tlane + colw[x] + 4 * i, c0, c1, c2, 0u);
            }
        }
        __syncthreads();  // every thread's key copies of round r have landed
        {
            const uint64_t *kr = kring + (r % RING) * KW;
            uint8_t *bb = bsm + (size_t)rb * GP * bpos;
#pragma unroll
            for (int x = 0; x < BMAX; x++) {
                if (tid + x * THREADS < nb) {
                    const uint64_t y = kr[bkw[x]];
                    const uint32_t ylo = (uint32_t)y, yhi = (uint32_t)(y >> 32);
                    uint4 ch;
                    ch.x = unbias(prmt(ylo, yhi, bsel[x][0]) | 0x64006400u);
                    ch.y = unbias(prmt(ylo, yhi, bsel[x][1]) | 0x64006400u);
                    ch.z = unbias(prmt(ylo, yhi, bsel[x][2]) | 0x64006400u);
                    ch.w = unbias(prmt(ylo, yhi, bsel[x][3]) | 0x64006400u);
                    *(uint4 *)(bb + boff[x]) = ch;
                }
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            for (int e = 0; e < GP; e++)
                for (int kk = 0; kk < nlp / 2; kk++) {
                    const uint64_t bd =
                        smem_desc(bsm_s + (uint32_t)((rb * GP + e) * bpos + kk * 256), 128, (uint32_t)nlp * 128);
                    const uint32_t accum = (j > 0 || kk > 0) ? 1u : 0u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(
                                     tmem + (uint32_t)((g & 1) * 128 + e * 32)),
                                 "r"(tmem + acol(rb, e) + 8 * kk), "l"(bd), "r"(idesc), "r"(accum)
                                 : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb0 + 8 * rb)
                         : "memory");
        }
    }
    for (int r = R >= 2 ? R - 2 : 0; r < R; r++) {
        ok &= mbar_wait_bounded(mb0 + 8 * (r & 1), (uint32_t)(r >> 1) & 1u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (r % nrot == nrot - 1) epilogue(r / nrot);
    }
    if (!ok) atomicOr(status, 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

size_t hoist_mma_smem(int nl)
{
    const int nlp = (nl + 1) & ~1;
    return (size_t)RING * nl * 2 * MT * 16 + 2 * (size_t)GP * 32 * nlp * 16 + RING * KW * 8 + 64;
}

template <int K1, int K2>
int run_mma(he_ctx *c, const uint64_t *mid, const uint64_t *dntt, size_t din_item, const HoistKeys &hk, uint64_t *acc,
            int items, int nl, int t_lo, int t_hi, cudaStream_t s)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, cudaFuncSetAttribute(k_ks_hoist_mma<K1, K2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)hoist_mma_smem(NLMAX)));
        prepared = true;
    }
    const unsigned grid = (unsigned)((size_t)((items + MT - 1) / MT) * (1 << K1) * (t_hi - t_lo));
    HELR_LAUNCH(k_ks_hoist_mma<K1, K2><<<grid, THREADS, hoist_mma_smem(nl), s>>>(mid, dntt, din_item, hk, acc, c->t.mod,
                                                                                nl, c->nq, items, t_lo, c->d_status));
    HELR_CUDA(c, cudaGetLastError());
    c->hoist_tensor_launches++;
    return HE_OK;
}

}  // namespace

bool helr_hoist_tensor_range(const he_ctx *c, int nl, int nrot, int *t_lo, int *t_hi)
{
    if (nl < 1 || nl > NLMAX || nrot < 1 || nrot * nl > PAIRS_MAX) return false;
    int a = 0;
    while (a < nl && c->q[a] >= (1ull << 40)) a++;
    int b = a;
    while (b < nl && c->q[b] < (1ull << 40)) b++;
    if (b == a) return false;
    *t_lo = a;
    *t_hi = b;
    return true;
}

int helr_hoist_ip_tensor(he_ctx *c, const uint64_t *mid, const uint64_t *dntt, size_t din_item, const HoistKeys &hk,
                         uint64_t *acc, int items, int nl, int t_lo, int t_hi, cudaStream_t s)
{
    switch (c->logn) {
    case 10: return run_mma<5, 5>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 11: return run_mma<5, 6>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 12: return run_mma<6, 6>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 13: return run_mma<6, 7>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 14: return run_mma<7, 7>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 15: return run_mma<7, 8>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    case 16: return run_mma<8, 8>(c, mid, dntt, din_item, hk, acc, items, nl, t_lo, t_hi, s);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}
