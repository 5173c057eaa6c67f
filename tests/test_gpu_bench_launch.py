"""Word-for-word parity at the launch configuration the benchmark times.

The full-batch benchmark runs N = 2^16 with the full chain (60 + 8 x 40 bits
and a 60-bit P), Steps 1-6 on 256 data blocks per launch and key switches in
waves of 64-256 items chosen by the autotuner.  These tests run exactly that
configuration -- the N = 2^16 template instantiations of the fused kernels,
more than one wave per launch, the ragged last chunk -- and compare sampled
outputs with the oracle word for word (the FP64 twin alone cannot see a
non-canonical word or a one-unit slip in one item of a wave).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import qgnag  # noqa: E402
from oracle.ckks import Ckks, Ct as OCt  # noqa: E402
from paper_2406_13221_gb300 import binding, build, synth  # noqa: E402

build.build()
D = 2.0 ** 40


@pytest.fixture(scope="module")
def bench_pair():
    """The benchmark's parameters with keys from seed 2, the key-switch waves
    chosen by the autotuner as the benchmark chooses them (256 items)."""
    ctx = binding.Context(16, 9)
    he = Ckks(16, 9)
    circ = qgnag.Circuit(he, 256, 128, D)
    ctx.keygen(2, circ.rotations())
    he.keygen(2, circ.rotations())
    ctx.autotune(None, 256)
    return ctx, he


@pytest.mark.parametrize("level,r", [(6, 0), (3, -4)])
def test_keyswitch_256_items_at_tuned_waves(bench_pair, level, r):
    """he_keyswitch_batch on 256 polynomials (relinearisation at 7 limbs, a
    rotation key at 4 limbs): items at both ends of the first and of the last
    wave equal the oracle's key switch."""
    ctx, he = bench_pair
    batch, n = 256, ctx.n
    wave = ctx.ks_wave(level)
    assert 16 <= wave <= 256
    rng = np.random.default_rng(1000 + level)
    polys = np.empty((batch, level + 1, n), np.uint64)
    for j in range(level + 1):
        polys[:, j, :] = rng.integers(0, he.q[j], (batch, n), dtype=np.uint64)
    gal = 0 if r == 0 else he.galois_elt(r)
    dev = torch.from_numpy(polys.reshape(-1).view(np.int64)).cuda()
    ctx.ntt_forward(dev.data_ptr(), batch * (level + 1), list(range(level + 1)))
    out = torch.zeros(batch * 2 * (level + 1) * n, dtype=torch.int64, device="cuda")
    ctx.keyswitch_batch(dev.data_ptr(), out.data_ptr(), batch, level, gal)
    ctx.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64).reshape(batch, 2, level + 1, n)
    last = batch - 1
    for b in sorted({0, wave - 1, wave, last - wave + 1, last} & set(range(batch))):
        assert np.array_equal(got[b], he.keyswitch(level, gal, polys[b])), (b, wave)


def test_hoisted_rotation_sums_256_items(bench_pair):
    """he_rotsum_batch on 256 ciphertexts at 6 limbs with the seven rotations
    of one hoisted group of Step 2 (1..7): items at both ends of the first
    wave and the last item equal the oracle's hoisted rotation sum."""
    ctx, he = bench_pair
    batch, n, level = 256, ctx.n, 5
    rots = list(range(1, 8))
    wave = ctx.ks_wave(level)
    rng = np.random.default_rng(77)
    cts = np.empty((batch, 2, level + 1, n), np.uint64)
    for j in range(level + 1):
        cts[:, :, j, :] = rng.integers(0, he.q[j], (batch, 2, n), dtype=np.uint64)
    dev = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    ctx.ntt_forward(dev.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    out = torch.zeros_like(dev)
    ctx.rotsum_batch(dev.data_ptr(), out.data_ptr(), batch, level, rots)
    ctx.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64).reshape(batch, 2, level + 1, n)
    for b in sorted({0, wave - 1, batch - 1}):
        ref = he.rotsum(OCt(cts[b], level, D), rots)
        assert np.array_equal(got[b], ref.data), (b, wave)


def test_hoisted_rotation_sums_256_items_tensor_form(bench_pair):
    """The same sums with the inner product on the tensor cores
    (he_set_hoist_form(1)): items at both ends of each 128-item tile of the
    first wave and the last item equal the oracle's hoisted rotation sum."""
    ctx, he = bench_pair
    batch, n, level = 256, ctx.n, 5
    rots = list(range(1, 8))
    rng = np.random.default_rng(78)
    cts = np.empty((batch, 2, level + 1, n), np.uint64)
    for j in range(level + 1):
        cts[:, :, j, :] = rng.integers(0, he.q[j], (batch, 2, n), dtype=np.uint64)
    dev = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    ctx.ntt_forward(dev.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    out = torch.zeros_like(dev)
    n0 = ctx.hoist_tensor_launches()
    ctx.set_hoist_form(1)
    try:
        ctx.rotsum_batch(dev.data_ptr(), out.data_ptr(), batch, level, rots)
    finally:
        ctx.set_hoist_form(-1)
    ctx.check_device()
    assert ctx.hoist_tensor_launches() > n0
    ctx.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64).reshape(batch, 2, level + 1, n)
    for b in (0, 127, 128, batch - 1):
        ref = he.rotsum(OCt(cts[b], level, D), rots)
        assert np.array_equal(got[b], ref.data), b


def test_batched_mul_rescale_rotate_64_items(bench_pair):
    """he_mul_relin_batch, he_rescale_batch and he_rotate_batch on 64 ciphertexts at
    the Step 1 level (7 limbs) with the bench's keys: items 0, 31 and 63 equal the
    oracle's Mul, Rescale and Rotate (by 1 slot)."""
    ctx, he = bench_pair
    batch, n, level = 64, ctx.n, 6
    rng = np.random.default_rng(91)
    A = np.empty((batch, 2, level + 1, n), np.uint64)
    B = np.empty_like(A)
    for j in range(level + 1):
        A[:, :, j, :] = rng.integers(0, he.q[j], (batch, 2, n), dtype=np.uint64)
        B[:, :, j, :] = rng.integers(0, he.q[j], (batch, 2, n), dtype=np.uint64)
    primes = list(range(level + 1))

    def dev(x):
        t = torch.from_numpy(x.reshape(-1).view(np.int64)).cuda()
        ctx.ntt_forward(t.data_ptr(), batch * 2 * (level + 1), primes)
        return t

    def host(t, lv):
        ctx.ntt_inverse(t.data_ptr(), batch * 2 * (lv + 1), list(range(lv + 1)))
        torch.cuda.synchronize()
        return t.cpu().numpy().view(np.uint64).reshape(batch, 2, lv + 1, n)

    da, db = dev(A), dev(B)
    prod, rot = torch.zeros_like(da), torch.zeros_like(da)
    resc = torch.zeros(batch * 2 * level * n, dtype=torch.int64, device="cuda")
    ctx.mul_relin_batch(da.data_ptr(), db.data_ptr(), prod.data_ptr(), batch, level)
    ctx.rescale_batch(prod.data_ptr(), resc.data_ptr(), batch, level)
    ctx.rotate_batch(da.data_ptr(), rot.data_ptr(), batch, level, 1)
    got_p, got_s, got_r = host(prod, level), host(resc, level - 1), host(rot, level)
    for b in (0, 31, batch - 1):
        ref = he.mul(OCt(A[b], level, D), OCt(B[b], level, D))
        assert np.array_equal(got_p[b], ref.data), b
        assert np.array_equal(got_s[b], he.rescale(ref).data), b
        assert np.array_equal(got_r[b], he.rotate(OCt(A[b], level, D), 1).data), b


def test_block_gradients_300_blocks_256_per_launch(bench_pair):
    """A 300-block job at 256 blocks per launch (a full chunk, then a ragged
    chunk of 44): the gradient ciphertexts of Steps 1-6 for blocks 0, 128, 255
    (first chunk) and 299 (last block of the ragged chunk), taken from the
    job's own chunked launches, equal the oracle's Steps 1-6 on the job's own
    encrypted block and weights."""
    ctx, he = bench_pair
    X, y = synth.financial(seed=6, n=300 * 128 - 37)
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=11, key_seed=2,
                      batch_blocks=256)
    assert job.stats().n_blocks == 300
    job.step(0)  # a refreshed, non-zero W
    circ = qgnag.Circuit(he, 256, 128, D)
    L = circ.L
    (Ww, lw, sw), _ = job.state_words()
    W = OCt(Ww, lw, sw)
    for b in (0, 128, 255, 299):
        got = job.block_grad(b)
        Z = OCt(job.input(0, b).export(), L, D)
        ref = circ.block_grad(Z, W)
        assert (got.level, got.scale) == (ref.level, ref.scale), b
        assert np.array_equal(got.export(), ref.data), b
    job.close()
