"""The bootstrap on the GPU (he_bootstrap, he_bootstrap_batch) against the
oracle's, word for word, at N = 2^10 with a sparse secret and a mixed chain;
at N = 2^16 with the bootstrappable chain of the training (q0 50 bits, six
40-bit levels, fourteen 55-bit levels), the refreshed slots against the
message."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import boot  # noqa: E402
from oracle.ckks import Ckks, Ct as OCt  # noqa: E402
from paper_2406_13221_gb300 import binding, build  # noqa: E402

build.build()
D = 2.0 ** 40
BITS = [50, 45] + [55] * 12
PARAMS = dict(slots=8, K=8, r=4, deg=23, scale_out=D, level_out=1)


@pytest.fixture(scope="module")
def pair():
    ctx = binding.Context(10, len(BITS), bits=BITS, secret_weight=16)
    he = Ckks(10, len(BITS), bits=BITS, secret_weight=16)
    assert ctx.primes == he.primes
    p = boot.BootParams(n=8, K=8, r=4, deg=23, delta_out=D, out_level=1)
    rots, gals = boot.key_rotations(he, p)
    assert ctx.boot_keys(**PARAMS) == rots
    he.keygen(5, rots, gals)
    ctx.keygen(5, rots)
    ctx.keygen_galois(gals)
    return ctx, he, p


def periodic(nslots, n, seed, amp=1.0):
    z = np.random.default_rng(seed).uniform(-amp, amp, n)
    return np.tile(z, nslots // n)


def test_sparse_secret_encryption_bitwise(pair):
    ctx, he, _ = pair
    z = periodic(he.nslots, 8, 1)
    ref = he.encrypt(he.encode(z, 3, D), 21)
    ct = ctx.encrypt(ctx.encode(z, 3, D), 21)
    assert np.array_equal(ct.export(), ref.data)
    words, _, _ = ctx.decrypt(ct).export()
    assert np.array_equal(words, he.decrypt(ref).data)


@pytest.mark.parametrize("amp", [1.0, 8.0])
def test_bootstrap_bitwise(pair, amp):
    ctx, he, p = pair
    z = periodic(he.nslots, 8, 2, amp)
    ref_in = he.encrypt(he.encode(z, 0, D), 22)
    ref = boot.bootstrap(he, ref_in, p)
    got = ctx.bootstrap(ctx.import_ct(ref_in.data, 0, D), **PARAMS)
    assert (got.level, got.scale) == (ref.level, ref.scale) == (1, D)
    assert np.array_equal(got.export(), ref.data)


def test_bootstrap_batch_bitwise(pair):
    """Three ciphertexts through he_bootstrap_batch equal three oracle bootstraps;
    the input may sit above level 0 (it is dropped to level 0 first)."""
    ctx, he, p = pair
    n = ctx.n
    refs, words = [], []
    for i in range(3):
        z = periodic(he.nslots, 8, 30 + i)
        c = he.encrypt(he.encode(z, 2, D), 40 + i)
        refs.append(boot.bootstrap(he, c, p))
        w = c.data.copy()
        words.append(w)
    din = torch.from_numpy(np.stack(words).reshape(-1).view(np.int64)).cuda()
    ctx.ntt_forward(din.data_ptr(), 3 * 2 * 3, list(range(3)))
    dout = torch.zeros(3 * 2 * 2 * n, dtype=torch.int64, device="cuda")
    ctx.bootstrap_batch(din.data_ptr(), 2, dout.data_ptr(), 3, **PARAMS)
    ctx.ntt_inverse(dout.data_ptr(), 3 * 2 * 2, list(range(2)))
    torch.cuda.synchronize()
    got = dout.cpu().numpy().view(np.uint64).reshape(3, 2, 2, n)
    for i in range(3):
        assert np.array_equal(got[i], refs[i].data), i


def test_bootstrap_errors(pair):
    ctx, he, _ = pair
    ct = ctx.import_ct(he.encrypt(he.encode(np.zeros(4), 0, D), 5).data, 0, D)
    with pytest.raises(binding.HeError) as e:
        ctx.bootstrap(ct, **dict(PARAMS, level_out=3))  # 12 levels leave level 1 at most
    assert e.value.code == binding.HE_ELEVEL
    with pytest.raises(binding.HeError):
        ctx.bootstrap(ct, **dict(PARAMS, slots=6))
    bare = binding.Context(10, len(BITS), bits=BITS, secret_weight=16)
    bare.keygen(5, [1])
    with pytest.raises(binding.HeError) as e:
        bare.bootstrap(bare.import_ct(ct.export(), 0, D), **PARAMS)
    assert e.value.code == binding.HE_EKEY


def test_bootstrap_full_size_refreshes_weights():
    """N = 2^16, 256 slots per period (the g = 256 weights of the 128 x 256
    packing), the bootstrappable chain: the refreshed W lands at the training's
    start level 6 with scale 2^40, its slots within 1e-4 of the message."""
    bits = [50] + [40] * 6 + [55] * 14
    ctx = binding.Context(16, len(bits), bits=bits, secret_weight=64)
    prm = dict(slots=256, K=16, r=6, deg=19, scale_out=D, level_out=6)
    ctx.keygen(2, ctx.boot_keys(**prm))
    ctx.keygen_galois([2 * ctx.n - 1])
    z = periodic(ctx.nslots, 256, 7, 2.0)
    ct = ctx.encrypt(ctx.encode(z, 0, D), 9)
    out = ctx.bootstrap(ct, **prm)
    assert (out.level, out.scale) == (6, D)
    got = ctx.decode(ctx.decrypt(out))
    assert np.abs(got.real - z).max() < 1e-4
    assert np.abs(got.imag).max() < 1e-4


def test_job_refreshed_by_bootstrapping_bitwise():
    """A full-batch job refreshing W and V by bootstrapping on a bootstrappable
    chain at N = 2^12 (16-column blocks, 8 blocks): after each of two steps the
    state equals, word for word, the oracle's iteration followed by the
    oracle's bootstrap of W' and V'; the weights track the FP64 twin."""
    from oracle import plain, qgnag
    from paper_2406_13221_gb300 import synth
    bits = [50] + [40] * 6 + [55] * 13
    ctx = binding.Context(12, len(bits), bits=bits, secret_weight=32)
    he = Ckks(12, len(bits), bits=bits, secret_weight=32)
    X, y = synth.small(seed=17, n=1024, f=15)
    data = qgnag.TrainData(X, y, g=16, m=128, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 128, D)
    L = circ.L
    prm = dict(slots=16, K=12, r=5, deg=23, scale_out=D, level_out=L)
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=19, key_seed=2)
    job.set_refresh(prm)
    p = boot.BootParams(n=16, K=12, r=5, deg=23, delta_out=D, out_level=L)
    rots, gals = boot.key_rotations(he, p)
    he.keygen(2, sorted(set(circ.rotations()) | set(rots)), gals)
    nb = data.blocks.shape[0]
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(nb)]
    B = OCt(job.input(1, 0).export(), L, D)
    (Ww, _, _), (Vw, _, _) = job.state_words()
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    etas = qgnag.nag_scalars(2)
    for t in range(2):
        job.step(t)
        Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(t), etas[t], 1.0 / data.n)
        W, V = boot.bootstrap(he, Wn, p), boot.bootstrap(he, Vn, p)
        (Ww, lw, sw), (Vw, _, _) = job.state_words()
        assert (lw, sw) == (L, D)
        assert np.array_equal(Ww, W.data), t
        assert np.array_equal(Vw, V.data), t
    wp = plain.train(data, 2)
    assert np.abs(job.weights(0) - wp).max() < 1e-3
    job.set_refresh(None)
