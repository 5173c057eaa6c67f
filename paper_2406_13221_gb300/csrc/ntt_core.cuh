// ntt_core.cuh -- device building blocks of the negacyclic transform, shared by
// the standalone transform kernels (ntt.cu) and the fused key-switch kernels
// (ks.cu).  See ntt.cu for the layout and the butterfly forms.
#pragma once
#include "helr_internal.cuh"

namespace nttc {


// Forward (Cooley-Tukey) butterfly.  Harvey's form keeps words in [0, 4q).  The
// unreduced form (LZ) drops the conditional subtraction: a butterfly adds less
// than 2q to each word, so after S stages on inputs below 4q every word is below
// (4 + 2S) q, which stays under 2^64 for the S <= 16 stages of a transform when
// q < 2^58 (HELR_LZ_QMAX).  The Shoup product accepts any 64-bit operand.
template <bool LZ = false>
__device__ __forceinline__ void ct_bfly(uint64_t &x, uint64_t &y, uint64_t w, uint64_t wp, uint64_t q, uint64_t q2)
{
    uint64_t a = LZ ? x : (x >= q2 ? x - q2 : x);
    uint64_t t = shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + q2;
}

__device__ __forceinline__ void gs_bfly(uint64_t &x, uint64_t &y, uint64_t w, uint64_t wp, uint64_t q, uint64_t q2)
{
    uint64_t a = x + y;
    a = a >= q2 ? a - q2 : a;
    uint64_t b = x - y + q2;
    y = shoup_lazy(b, w, wp, q);
    x = a;
}

// twiddle pair idx (w, Shoup companion) from the global table, or from a copy
// in shared memory (SH)
template <bool SH = false>
__device__ __forceinline__ ulonglong2 ldtw(const uint64_t *tw, int idx)
{
    if constexpr (SH)
        return reinterpret_cast<const ulonglong2 *>(tw)[idx];
    else
        return __ldg(reinterpret_cast<const ulonglong2 *>(tw) + idx);
}

// padded shared-memory position of word j inside one column/row segment
template <int LE>
__device__ __forceinline__ int spad(int j) { return j + (j >> LE); }

template <int K>
struct Geo {
    static constexpr int LE = (K + 1) / 2, LT = K / 2;
    static constexpr int E = 1 << LE, T = 1 << LT, R = 1 << K;
    static constexpr int SEG = R + (R >> LE) + 1;  // segment stride in words (odd)
};

// Stage loops are template recursions over the stage index with one flattened
// constant-trip loop per stage, so every index into x[] is a compile-time
// constant and x[] stays in registers.
//
// forward stages on the strided assignment (j = l + T r): local stages s < LE;
// at local stage m = 2^s the E words form m groups of 2 hr (hr = E / 2m).
// LT2: the words enter below 2q, so the first stage needs no correction
template <int K, bool LZ, bool SH, bool LT2, int S>
__device__ __forceinline__ void fwd_strided_st(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, uint64_t q, uint64_t q2)
{
    constexpr int E = Geo<K>::E, LE = Geo<K>::LE, m = 1 << S, hr = E >> (S + 1);
    ulonglong2 w[m];
#pragma unroll
    for (int g = 0; g < m; g++) w[g] = ldtw<SH>(tw, m * A + g);
#pragma unroll
    for (int bf = 0; bf < E / 2; bf++) {
        const int g = bf / hr, k = bf % hr;
        ct_bfly<LZ || (LT2 && S == 0)>(x[g * 2 * hr + k], x[g * 2 * hr + k + hr], w[g].x, w[g].y, q, q2);
    }
    if constexpr (S + 1 < LE) fwd_strided_st<K, LZ, SH, LT2, S + 1>(x, tw, A, q, q2);
}
template <int K, bool LZ = false, bool SH = false, bool LT2 = false>
__device__ __forceinline__ void fwd_strided(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, uint64_t q, uint64_t q2)
{
    fwd_strided_st<K, LZ, SH, LT2, 0>(x, tw, A, q, q2);
}

// Twiddle j of stage block m * A (j < m) for group g of thread l on the
// contiguous assignment, j = l gpt + g.  Blocks used by the row pass (ROW) are
// stored with that index transposed, at m A + g T + l, so that the T threads of a
// row read one contiguous run per load instead of runs gpt pairs apart (the host
// table builder applies the same permutation to those blocks).
template <int K, bool ROW>
__device__ __forceinline__ int tw_contig(int m, int A, int l, int gpt, int g)
{
    return ROW ? m * A + g * Geo<K>::T + l : m * A + l * gpt + g;
}

// forward stages on the contiguous assignment (j = E l + r): local stages s >= LE;
// half-span h = R / 2^(s+1) <= E/2, gpt = E / 2h groups per thread.
template <int K, bool ROW, bool LZ, bool SH, int S>
__device__ __forceinline__ void fwd_contig_st(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, int l, uint64_t q, uint64_t q2)
{
    constexpr int E = Geo<K>::E, R = Geo<K>::R, m = 1 << S, h = R >> (S + 1), gpt = E / (2 * h);
    ulonglong2 w[gpt];
#pragma unroll
    for (int g = 0; g < gpt; g++) w[g] = ldtw<SH>(tw, tw_contig<K, ROW>(m, A, l, gpt, g));
#pragma unroll
    for (int bf = 0; bf < E / 2; bf++) {
        const int g = bf / h, k = bf % h;
        ct_bfly<LZ>(x[g * 2 * h + k], x[g * 2 * h + k + h], w[g].x, w[g].y, q, q2);
    }
    if constexpr (S + 1 < K) fwd_contig_st<K, ROW, LZ, SH, S + 1>(x, tw, A, l, q, q2);
}
template <int K, bool ROW, bool LZ = false, bool SH = false>
__device__ __forceinline__ void fwd_contig(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, int l, uint64_t q, uint64_t q2)
{
    fwd_contig_st<K, ROW, LZ, SH, Geo<K>::LE>(x, tw, A, l, q, q2);
}

template <int K, bool ROW, int S>
__device__ __forceinline__ void inv_contig_st(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, int l, uint64_t q, uint64_t q2)
{
    constexpr int E = Geo<K>::E, R = Geo<K>::R, m = 1 << S, h = R >> (S + 1), gpt = E / (2 * h);
    ulonglong2 w[gpt];
#pragma unroll
    for (int g = 0; g < gpt; g++) w[g] = ldtw(tw, tw_contig<K, ROW>(m, A, l, gpt, g));
#pragma unroll
    for (int bf = 0; bf < E / 2; bf++) {
        const int g = bf / h, k = bf % h;
        gs_bfly(x[g * 2 * h + k], x[g * 2 * h + k + h], w[g].x, w[g].y, q, q2);
    }
    if constexpr (S - 1 >= Geo<K>::LE) inv_contig_st<K, ROW, S - 1>(x, tw, A, l, q, q2);
}
template <int K, bool ROW>
__device__ __forceinline__ void inv_contig(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, int l, uint64_t q, uint64_t q2)
{
    inv_contig_st<K, ROW, K - 1>(x, tw, A, l, q, q2);
}

template <int K, int S>
__device__ __forceinline__ void inv_strided_st(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, uint64_t q, uint64_t q2)
{
    constexpr int E = Geo<K>::E, m = 1 << S, hr = E >> (S + 1);
    ulonglong2 w[m];
#pragma unroll
    for (int g = 0; g < m; g++) w[g] = ldtw(tw, m * A + g);
#pragma unroll
    for (int bf = 0; bf < E / 2; bf++) {
        const int g = bf / hr, k = bf % hr;
        gs_bfly(x[g * 2 * hr + k], x[g * 2 * hr + k + hr], w[g].x, w[g].y, q, q2);
    }
    if constexpr (S > 0) inv_strided_st<K, S - 1>(x, tw, A, q, q2);
}
template <int K>
__device__ __forceinline__ void inv_strided(uint64_t (&x)[Geo<K>::E], const uint64_t *tw, int A, uint64_t q, uint64_t q2)
{
    inv_strided_st<K, Geo<K>::LE - 1>(x, tw, A, q, q2);
}

// exchange the E words of thread l inside one segment of shared memory
template <int K>
__device__ __forceinline__ void to_contig(uint64_t (&x)[Geo<K>::E], uint64_t *seg, int l)
{
    constexpr int E = Geo<K>::E, LE = Geo<K>::LE, T = Geo<K>::T;
#pragma unroll
    for (int r = 0; r < E; r++) seg[spad<LE>(l + T * r)] = x[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; r++) x[r] = seg[spad<LE>(E * l + r)];
}
template <int K>
__device__ __forceinline__ void to_strided(uint64_t (&x)[Geo<K>::E], uint64_t *seg, int l)
{
    constexpr int E = Geo<K>::E, LE = Geo<K>::LE, T = Geo<K>::T;
#pragma unroll
    for (int r = 0; r < E; r++) seg[spad<LE>(E * l + r)] = x[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; r++) x[r] = seg[spad<LE>(l + T * r)];
}

// The same exchange inside an unpadded row segment of R words: word w lives at
// w ^ ((w >> 4) & 15) (the low four bits XORed with the next four, within its
// 16-word block).  For the 64-bit words of a row held by 16 threads (one
// half-warp) both access patterns, l + T r and E l + r, then fall into 16
// distinct bank pairs.  The caller synchronises before the first write when the
// segment still holds data other threads are reading.
__device__ __forceinline__ int swz(int w) { return w ^ ((w >> 4) & 15); }
template <int K>
__device__ __forceinline__ void to_contig_swz(uint64_t (&x)[Geo<K>::E], uint64_t *seg, int l)
{
    constexpr int E = Geo<K>::E, T = Geo<K>::T;
#pragma unroll
    for (int r = 0; r < E; r++) seg[swz(l + T * r)] = x[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; r++) x[r] = seg[swz(E * l + r)];
}

}  // namespace nttc

// sigma_gal on the evaluation form: position k holds the evaluation at
// psi^(2 bitrev(k) + 1), so sigma_gal(x) takes at k the value x holds at the
// position of psi^((2 bitrev(k) + 1) gal).  The product is needed modulo 2N
// only, so 32-bit arithmetic suffices.
template <int LOGN>
__device__ __forceinline__ uint32_t auto_pos(uint32_t k, uint64_t gal)
{
    const uint32_t kk = __brev(k) >> (32 - LOGN);
    const uint32_t e = ((2u * kk + 1u) * (uint32_t)gal) & ((2u << LOGN) - 1u);
    return __brev((e - 1u) >> 1) >> (32 - LOGN);
}

// Montgomery reduction of T = hi 2^64 + lo: T 2^-64 mod q, for hi < q.
__device__ __forceinline__ uint64_t redc128(uint64_t hi, uint64_t lo, const ModQ &m)
{
    const uint64_t mh = __umul64hi(lo * m.qinv, m.q);
    return hi >= mh ? hi - mh : hi - mh + m.q;
}

// Wait for phase `parity` of the mbarrier at shared address mb, for at most
// one second of the global timer; false when the wait expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mb), "r"(parity)
                     : "memory");
        if (done) return true;
        uint64_t t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > 1000000000ull) return false;
    }
}
