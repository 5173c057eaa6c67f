// noalloc.cu -- a rescale entry point that allocates no memory.
//
// he_rescale allocates its work space (stream-ordered cudaMallocAsync) on every
// call.  Some callers cannot allow that: code that runs under a device-memory
// budget fixed before it starts, code embedded in a host framework that owns
// all device allocations, or latency-critical loops where an allocation could
// stall or fail mid-iteration.  he_rescale_noalloc gives them the same result
// with its work space in a fixed array that every device holds for as long as
// the library is loaded.
#include <mutex>
#include <algorithm>
#include "helr_internal.cuh"

// Work space of he_rescale_noalloc: 2^21 words (16 MiB) on every device that
// loads the library.  In host code the name is only a handle for the runtime;
// the device address comes from cudaGetSymbolAddress below.
#define NOALLOC_WORDS (1u << 21)
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS];

static std::mutex g_noalloc_mu;
static uint64_t *g_noalloc_ptr[64];  // device address of the array, per device ordinal

// Looks up (once per device, with that device current) the device address of
// the work-space array.
static int noalloc_scratch(he_ctx *c, uint64_t **out)
{
    int dev = 0;
    HELR_CUDA(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return helr_fail(c, HE_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return helr_fail(c, HE_ECUDA, "cudaGetSymbolAddress of the rescale work space: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (uint64_t *)p;
    }
    *out = g_noalloc_ptr[dev];
    return HE_OK;
}

extern "C" int he_rescale_noalloc(he_ctx *c, const uint64_t *d_in, uint64_t *d_out, int batch, int level)
{
    if (!c || !d_in || !d_out || batch < 0 || level < 1 || level >= c->nq) return c ? helr_fail(c, HE_EINVAL,
        "he_rescale_noalloc: bad argument (batch %d, level %d)", batch, level) : HE_EINVAL;
    if (batch == 0) return HE_OK;
    const size_t N = c->n, nl = (size_t)level + 1;
    const size_t per_item = (2 + 2 * (size_t)level) * N;  // last limbs + their lifts
    if (per_item > NOALLOC_WORDS)
        return helr_fail(c, HE_EINVAL,
                         "he_rescale_noalloc: one ciphertext at level %d needs %zu work words, more than the %u available",
                         level, per_item, NOALLOC_WORDS);
    uint64_t *ws = nullptr;
    HELR_TRY(noalloc_scratch(c, &ws));
    const int per_pass = (int)(NOALLOC_WORDS / per_item);
    cudaStream_t s = c->stream;
    KP kp;
    for (int j = 0; j < level; j++) {
        unsigned __int128 r = 1, b = c->q[level] % c->q[j];
        for (uint64_t e = c->q[j] - 2; e; e >>= 1, b = b * b % c->q[j])
            if (e & 1) r = r * b % c->q[j];
        kp.w[j][0] = (uint64_t)r;
        kp.w[j][1] = (uint64_t)(((unsigned __int128)(uint64_t)r << 64) / c->q[j]);
    }
    for (int b0 = 0; b0 < batch; b0 += per_pass) {
        const int cnt = std::min(per_pass, batch - b0);
        const uint64_t *in = d_in + (size_t)b0 * 2 * nl * N;
        uint64_t *out = d_out + (size_t)b0 * 2 * level * N;
        uint64_t *last = ws, *lift = ws + 2 * (size_t)cnt * N;
        // last limb of each polynomial -> coefficient form -> centred lift to q_0..q_(level-1)
        HELR_CUDA(c, cudaMemcpy2DAsync(last, N * 8, in + (size_t)level * N, nl * N * 8, N * 8, 2 * (size_t)cnt,
                                       cudaMemcpyDeviceToDevice, s));
        HELR_TRY(helr_ntt_inv(c, last, 2 * (size_t)cnt, limbmap_single(level), s));
        k_lift(c, last, lift, 2 * cnt, level, N, limbmap_ct(level - 1), (size_t)level * N, s);
        HELR_TRY(helr_ntt_fwd(c, lift, 2 * (size_t)cnt * level, limbmap_ct(level - 1), s));
        Str si{const_cast<uint64_t *>(in), 2 * nl * N, nl * N}, sc{lift, 2 * (size_t)level * N, (size_t)level * N},
            so{out, 2 * (size_t)level * N, (size_t)level * N};
        k_ew(c, EW_SUBMUL, so, si, sc, cnt, 2, level, &kp, s);
        HELR_CUDA(c, cudaGetLastError());
    }
    return HE_OK;
}
