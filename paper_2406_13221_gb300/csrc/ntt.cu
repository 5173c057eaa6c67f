// ntt.cu -- batched negacyclic NTT over Z_q[X]/(X^N + 1) for N = 2^10 .. 2^16.
//
// Every ring product of the scheme (Sec. 2.1 Mul, cMul by a plaintext, key
// switching inside Mul and rotation) is a pointwise product between forward
// transforms.  Transform: A[p] = sum_j a_j psi^(j (2 bitrev(p) + 1)), i.e. the
// evaluations at the odd powers of a primitive 2N-th root psi, stored in
// bit-reversed order (merged-twist Cooley-Tukey forward, Gentleman-Sande
// inverse; the inverse includes the factor N^-1).
//
// Layout: N = R1 * R2 with R1 = 2^K1, R2 = 2^K2, index j = j1 * R2 + j2.
//  * pass 1: the first K1 butterfly stages act along j1 ("columns", stride R2);
//    a CTA takes C adjacent columns so that global accesses are contiguous runs.
//  * pass 2: the last K2 stages act inside each contiguous row of R2 words.
// Inside a pass one column/row of R = 2^K words is held by T threads with E
// words each (E = 2^ceil(K/2), T = 2^floor(K/2)): the first log2(E) stages run in
// registers on the strided assignment j = l + T r, one shared-memory exchange
// regroups the words as j = E l + r, and the remaining log2(T) stages run in
// registers again.  Butterflies are Harvey's lazy forms (values in [0, 4q) in the
// forward and [0, 2q) in the inverse) with Shoup twiddle products.  Each kernel
// is bounded to 64 registers so that 4 CTAs (32 warps) share an SM: a pass does
// one transform per load, and the extra warps hide more of its load latency
// (2% over 3 CTAs at N = 2^16, measured).
#include <algorithm>

#include "helr_internal.cuh"

#include "ntt_core.cuh"

namespace {
using namespace nttc;

// ---------------------------------------------------------------- forward
// pass 1: columns. grid.x = nlimbs * (R2 / C); block = C * T1 threads.
template <int K1, int K2, int C>
__global__ void __launch_bounds__(C * Geo<K1>::T, 4) k_ntt_fwd_cols(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                                 const uint64_t *__restrict__ twall, const ModQ *__restrict__ mods,
                                                                 LimbMap lm)
{
    using G = Geo<K1>;
    constexpr int R2 = 1 << K2, N = G::R * R2, NG = R2 / C;
    extern __shared__ uint64_t smem[];
    const int limb = blockIdx.x / NG, grp = blockIdx.x % NG;
    const int jj = threadIdx.x % C, l = threadIdx.x / C;
    const int pr = limb_prime(lm, limb);
    const uint64_t q = mods[pr].q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pr * N * 2;
    const size_t base = (size_t)limb * N + grp * C + jj;
    uint64_t x[G::E];
#pragma unroll
    for (int r = 0; r < G::E; r++) x[r] = in[base + (size_t)(l + G::T * r) * R2];
    fwd_strided<K1>(x, tw, 1, q, q2);
    to_contig<K1>(x, smem + jj * G::SEG, l);
    fwd_contig<K1, false>(x, tw, 1, l, q, q2);
#pragma unroll
    for (int r = 0; r < G::E; r++) out[base + (size_t)(G::E * l + r) * R2] = x[r];
}

// pass 2: rows. grid.x = nlimbs * (R1 / RPC); block = RPC * T2 threads.
template <int K1, int K2, int RPC>
__global__ void __launch_bounds__(RPC * Geo<K2>::T, 4) k_ntt_fwd_rows(uint64_t *__restrict__ data, const uint64_t *__restrict__ twall,
                                                                   const ModQ *__restrict__ mods, LimbMap lm)
{
    using G = Geo<K2>;
    constexpr int R1 = 1 << K1, R2 = G::R, N = R1 * R2, NG = R1 / RPC;
    extern __shared__ uint64_t smem[];
    const int limb = blockIdx.x / NG, grp = blockIdx.x % NG;
    const int l = threadIdx.x % G::T, rl = threadIdx.x / G::T;
    const int row = grp * RPC + rl;
    const int pr = limb_prime(lm, limb);
    const uint64_t q = mods[pr].q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pr * N * 2;
    uint64_t *rowp = data + (size_t)limb * N + (size_t)row * R2;
    uint64_t *seg = smem + rl * G::SEG;
    uint64_t x[G::E];
#pragma unroll
    for (int r = 0; r < G::E; r++) x[r] = rowp[l + G::T * r];
    const int A = R1 + row;
    fwd_strided<K2>(x, tw, A, q, q2);
    to_contig<K2>(x, seg, l);
    fwd_contig<K2, true>(x, tw, A, l, q, q2);
#pragma unroll
    for (int r = 0; r < G::E; r++) {
        uint64_t v = x[r];
        v = v >= q2 ? v - q2 : v;
        x[r] = v >= q ? v - q : v;
    }
    __syncthreads();
    to_strided<K2>(x, seg, l);
#pragma unroll
    for (int r = 0; r < G::E; r++) rowp[l + G::T * r] = x[r];
}

// ---------------------------------------------------------------- inverse
// pass A: rows (last forward stages undone first).  Input limb k is read at
// in + (k / per_item) in_item + (k % per_item) in_poly (contiguous limbs:
// in_item = per_item N, in_poly = N); output limbs are contiguous.
template <int K1, int K2, int RPC>
__global__ void __launch_bounds__(RPC * Geo<K2>::T, 4) k_ntt_inv_rows(const uint64_t *__restrict__ in, size_t in_item,
                                                                   size_t in_poly, uint64_t *__restrict__ out,
                                                                   const uint64_t *__restrict__ twall, const ModQ *__restrict__ mods,
                                                                   LimbMap lm, int per_item)
{
    using G = Geo<K2>;
    constexpr int R1 = 1 << K1, R2 = G::R, N = R1 * R2, NG = R1 / RPC;
    extern __shared__ uint64_t smem[];
    const int limb = blockIdx.x / NG, grp = blockIdx.x % NG;
    const int l = threadIdx.x % G::T, rl = threadIdx.x / G::T;
    const int row = grp * RPC + rl;
    const int pr = limb_prime(lm, limb);
    const uint64_t q = mods[pr].q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pr * N * 2;
    const uint64_t *rin = in + (size_t)(limb / per_item) * in_item + (size_t)(limb % per_item) * in_poly + (size_t)row * R2;
    uint64_t *rout = out + (size_t)limb * N + (size_t)row * R2;
    uint64_t *seg = smem + rl * G::SEG;
    uint64_t x[G::E];
#pragma unroll
    for (int r = 0; r < G::E; r++) x[r] = rin[l + G::T * r];
    to_contig<K2>(x, seg, l);
    const int A = R1 + row;
    inv_contig<K2, true>(x, tw, A, l, q, q2);
    __syncthreads();
    to_strided<K2>(x, seg, l);
    inv_strided<K2>(x, tw, A, q, q2);
#pragma unroll
    for (int r = 0; r < G::E; r++) rout[l + G::T * r] = x[r];
}

// pass B: columns, then the factor N^-1 and the final reduction to [0, q).
template <int K1, int K2, int C>
__global__ void __launch_bounds__(C * Geo<K1>::T, 4) k_ntt_inv_cols(uint64_t *__restrict__ data, const uint64_t *__restrict__ twall,
                                                                 const ModQ *__restrict__ mods, const uint64_t *__restrict__ ninv,
                                                                 LimbMap lm)
{
    using G = Geo<K1>;
    constexpr int R2 = 1 << K2, N = G::R * R2, NG = R2 / C;
    extern __shared__ uint64_t smem[];
    const int limb = blockIdx.x / NG, grp = blockIdx.x % NG;
    const int jj = threadIdx.x % C, l = threadIdx.x / C;
    const int pr = limb_prime(lm, limb);
    const uint64_t q = mods[pr].q, q2 = 2 * q;
    const uint64_t *tw = twall + (size_t)pr * N * 2;
    const size_t base = (size_t)limb * N + grp * C + jj;
    uint64_t x[G::E];
    // words of this column arrive as j1 = E l + r (contiguous assignment)
#pragma unroll
    for (int r = 0; r < G::E; r++) x[r] = data[base + (size_t)(G::E * l + r) * R2];
    inv_contig<K1, false>(x, tw, 1, l, q, q2);
    to_strided<K1>(x, smem + jj * G::SEG, l);
    inv_strided<K1>(x, tw, 1, q, q2);
    const uint64_t ni = ninv[2 * pr], nip = ninv[2 * pr + 1];
#pragma unroll
    for (int r = 0; r < G::E; r++) data[base + (size_t)(l + G::T * r) * R2] = shoup(x[r], ni, nip, q);
}

template <int K1, int K2>
struct NttPlan {
    static constexpr int T1 = Geo<K1>::T, T2 = Geo<K2>::T;
    static constexpr int R1 = 1 << K1, R2 = 1 << K2, N = R1 * R2;
    static constexpr int C = (256 / T1) < R2 ? (256 / T1) : R2;
    static constexpr int RPC = (256 / T2) < R1 ? (256 / T2) : R1;
    static constexpr size_t SM1 = (size_t)C * Geo<K1>::SEG * 8;
    static constexpr size_t SM2 = (size_t)RPC * Geo<K2>::SEG * 8;

    static cudaError_t prepare()
    {
        cudaError_t e = helr_fit_carveout((const void *)k_ntt_fwd_cols<K1, K2, C>, C * T1, SM1);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ntt_inv_cols<K1, K2, C>, C * T1, SM1);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ntt_fwd_rows<K1, K2, RPC>, RPC * T2, SM2);
        if (e == cudaSuccess) e = helr_fit_carveout((const void *)k_ntt_inv_rows<K1, K2, RPC>, RPC * T2, SM2);
        return e;
    }
    static void fwd(const uint64_t *in, uint64_t *out, size_t nlimbs, const DevTables &t, const LimbMap &m, cudaStream_t s)
    {
        HELR_LAUNCH(k_ntt_fwd_cols<K1, K2, C><<<(unsigned)(nlimbs * (R2 / C)), C * T1, SM1, s>>>(in, out, t.tw, t.mod, m));
        HELR_LAUNCH(k_ntt_fwd_rows<K1, K2, RPC><<<(unsigned)(nlimbs * (R1 / RPC)), RPC * T2, SM2, s>>>(out, t.tw, t.mod, m));
    }
    static void inv_rows(const uint64_t *in, size_t in_item, size_t in_poly, uint64_t *out, size_t nlimbs, const DevTables &t,
                         const LimbMap &m, cudaStream_t s, int per_item)
    {
        HELR_LAUNCH(k_ntt_inv_rows<K1, K2, RPC><<<(unsigned)(nlimbs * (R1 / RPC)), RPC * T2, SM2, s>>>(in, in_item, in_poly, out,
                                                                                                 t.itw, t.mod, m, per_item));
    }
    static void inv(const uint64_t *in, uint64_t *out, size_t nlimbs, const DevTables &t, const LimbMap &m, cudaStream_t s)
    {
        HELR_LAUNCH(k_ntt_inv_rows<K1, K2, RPC><<<(unsigned)(nlimbs * (R1 / RPC)), RPC * T2, SM2, s>>>(in, 2 * (size_t)N, N, out,
                                                                                                 t.itw, t.mod, m, 2));
        HELR_LAUNCH(k_ntt_inv_cols<K1, K2, C><<<(unsigned)(nlimbs * (R2 / C)), C * T1, SM1, s>>>(out, t.itw, t.mod, t.ninv, m));
    }
};

template <int K1, int K2>
int run_inv_rows(he_ctx *c, const uint64_t *in, size_t in_item, size_t in_poly, uint64_t *out, size_t nlimbs,
                 const LimbMap &m, cudaStream_t s, int per_item)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, (NttPlan<K1, K2>::prepare()));
        prepared = true;
    }
    if (nlimbs == 0) return HE_OK;
    prof_start(c, PROF_NTT_INV, s);
    NttPlan<K1, K2>::inv_rows(in, in_item, in_poly, out, nlimbs, c->t, m, s, per_item);
    prof_stop(c, PROF_NTT_INV, s, 0.5 * (double)nlimbs, 1);  // half of each transform
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

template <int K1, int K2>
int run(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s, bool inverse)
{
    static bool prepared = false;
    if (!prepared) {
        HELR_CUDA(c, (NttPlan<K1, K2>::prepare()));
        prepared = true;
    }
    if (nlimbs == 0) return HE_OK;
    const int cls = inverse ? PROF_NTT_INV : PROF_NTT_FWD;
    prof_start(c, cls, s);
    if (inverse) {
        NttPlan<K1, K2>::inv(in, out, nlimbs, c->t, m, s);
    } else {
        NttPlan<K1, K2>::fwd(in, out, nlimbs, c->t, m, s);
    }
    prof_stop(c, cls, s, (double)nlimbs, 2);
    HELR_CUDA(c, cudaGetLastError());
    return HE_OK;
}

int dispatch(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s, bool inv)
{
    if (nlimbs > (size_t)1 << 24) return helr_fail(c, HE_EINVAL, "too many limbs in one transform batch");
    switch (c->logn) {
    case 10: return run<5, 5>(c, in, out, nlimbs, m, s, inv);
    case 11: return run<5, 6>(c, in, out, nlimbs, m, s, inv);
    case 12: return run<6, 6>(c, in, out, nlimbs, m, s, inv);
    case 13: return run<6, 7>(c, in, out, nlimbs, m, s, inv);
    case 14: return run<7, 7>(c, in, out, nlimbs, m, s, inv);
    case 15: return run<7, 8>(c, in, out, nlimbs, m, s, inv);
    case 16: return run<8, 8>(c, in, out, nlimbs, m, s, inv);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}

}  // namespace

// Allow `smem` bytes of dynamic shared memory and ask for the smallest
// shared-memory carveout that still holds as many CTAs per SM as registers and
// threads allow, so that the rest of the SM's on-chip memory serves as L1 (the
// transforms re-read their twiddles from L1).  The CTA count is the larger of
// the runtime's occupancy figure and one computed from the kernel's registers,
// threads and shared memory (the runtime reports 0 for some kernels).
cudaError_t helr_fit_carveout(const void *f, int threads, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int blocks = 0, dev = 0, maxsm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, f, threads, smem);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e != cudaSuccess || maxsm <= 0 || threads <= 0) return e;
    const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // registers are granted per warp in units of 256
    int own = std::min(regs_sm / std::max(1, warp_regs * ((threads + 31) / 32)), thr_sm / threads);
    own = std::min(own, (int)((size_t)maxsm / per_cta));
    blocks = std::max(blocks, own);
    // rounded down: the driver takes the supported configuration at or just
    // above the requested share, and the configurations are coarser than 1%
    int pct = (int)((size_t)blocks * per_cta * 100 / (size_t)maxsm);
    pct = pct < 1 ? 1 : pct > 100 ? 100 : pct;
    return cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

int helr_ntt_fwd(he_ctx *c, uint64_t *data, size_t nlimbs, const LimbMap &m, cudaStream_t s)
{
    return dispatch(c, data, data, nlimbs, m, s, false);
}
int helr_ntt_inv(he_ctx *c, uint64_t *data, size_t nlimbs, const LimbMap &m, cudaStream_t s)
{
    return dispatch(c, data, data, nlimbs, m, s, true);
}
int helr_ntt_fwd_oop(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s)
{
    return dispatch(c, in, out, nlimbs, m, s, false);
}
int helr_ntt_inv_oop(he_ctx *c, const uint64_t *in, uint64_t *out, size_t nlimbs, const LimbMap &m, cudaStream_t s)
{
    return dispatch(c, in, out, nlimbs, m, s, true);
}
// the row pass of the inverse transform only: the column pass (K1 stages, the
// factor N^-1) is left to a consumer that reads whole columns.  Input limb k is
// read at in + (k / per_item) in_item + (k % per_item) in_poly; output limbs
// are contiguous.
int helr_ntt_inv_rows(he_ctx *c, const uint64_t *in, size_t in_item, size_t in_poly, uint64_t *out, size_t nlimbs,
                      const LimbMap &m, cudaStream_t s, int per_item)
{
    if (nlimbs > (size_t)1 << 24) return helr_fail(c, HE_EINVAL, "too many limbs in one transform batch");
    if (per_item < 1) return helr_fail(c, HE_EINVAL, "limbs per item %d", per_item);
    switch (c->logn) {
    case 10: return run_inv_rows<5, 5>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 11: return run_inv_rows<5, 6>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 12: return run_inv_rows<6, 6>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 13: return run_inv_rows<6, 7>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 14: return run_inv_rows<7, 7>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 15: return run_inv_rows<7, 8>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    case 16: return run_inv_rows<8, 8>(c, in, in_item, in_poly, out, nlimbs, m, s, per_item);
    default: return helr_fail(c, HE_EINVAL, "log_n %d unsupported", c->logn);
    }
}
