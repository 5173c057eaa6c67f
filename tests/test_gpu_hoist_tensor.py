"""The tensor-core form of the hoisted inner product (he_set_hoist_form(1):
tcgen05.mma on FP16 byte slices) against the oracle, word for word: hoisted
rotation sums of batches that span the 128-item tile of the kernel, at even
and odd limb counts, a case where the form does not apply (it falls back to
the CUDA cores), and a whole training iteration.  The tests also check that
the tensor-core kernel ran (its launch counter) and that no bounded
device-side wait expired."""
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
ROTS = sorted({r for k in range(1, 8) for r in (k, -k)} | {16 * k for k in range(1, 8)} | {
    r for n, st in ((4, 1), (4, -1), (8, 16)) for rots in qgnag.rot_groups(n, st, 3) for r in rots})


@pytest.fixture(scope="module")
def pair():
    """N = 2^13, the chain 60 + 8 x 40 bits and a 60-bit P, keys from seed 2."""
    ctx = binding.Context(13, 9)
    he = Ckks(13, 9)
    ctx.keygen(2, ROTS)
    he.keygen(2, ROTS)
    return ctx, he


def rotsum_batch(ctx, he, batch, level, rots, seed, form):
    """random ciphertext words (coefficient form) -> he_rotsum_batch under the
    given form -> coefficient-form words [batch][2][level+1][N], and the inputs"""
    n = ctx.n
    rng = np.random.default_rng(seed)
    cts = np.empty((batch, 2, level + 1, n), np.uint64)
    for j in range(level + 1):
        cts[:, :, j, :] = rng.integers(0, he.q[j], (batch, 2, n), dtype=np.uint64)
    dev = torch.from_numpy(cts.reshape(-1).view(np.int64)).cuda()
    ctx.ntt_forward(dev.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    out = torch.zeros_like(dev)
    ctx.set_hoist_form(form)
    try:
        ctx.rotsum_batch(dev.data_ptr(), out.data_ptr(), batch, level, rots)
    finally:
        ctx.set_hoist_form(-1)
    ctx.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(batch, 2, level + 1, n), cts


@pytest.mark.parametrize("level,rots,batch", [
    (5, list(range(1, 8)), 150),           # 6 limbs x 7 rotations = 42 pairs, two tiles (128 + 22 items)
    (4, list(range(-7, 0)), 40),           # 5 limbs: an odd digit count (a zero pad pair)
    (3, [16, 32, 48], 130),                # 4 limbs, 3 rotations, a tile of 2 items after a full one
    (6, [1, 2, 3, 4, 5, 6, 7], 3),         # 7 limbs x 7 = 49 pairs (the bound is 51), few items
])
def test_tensor_form_rotation_sums_bitwise(pair, level, rots, batch):
    ctx, he = pair
    n0 = ctx.hoist_tensor_launches()
    got, cts = rotsum_batch(ctx, he, batch, level, rots, 500 + level, 1)
    ctx.check_device()
    assert ctx.hoist_tensor_launches() > n0  # the tensor-core kernel ran
    for b in sorted({0, 1, batch // 2, min(127, batch - 1), min(128, batch - 1), batch - 1}):
        ref = he.rotsum(OCt(cts[b], level, D), rots)
        assert np.array_equal(got[b], ref.data), b
    base, _ = rotsum_batch(ctx, he, batch, level, rots, 500 + level, 0)
    assert np.array_equal(got, base)  # every item: the CUDA-core form's words


def test_tensor_form_falls_back_where_it_does_not_apply(pair):
    """9 limbs x 7 rotations = 63 pairs exceed the exact FP32 range of the
    byte products: the CUDA-core form runs, with the oracle's words."""
    ctx, he = pair
    n0 = ctx.hoist_tensor_launches()
    got, cts = rotsum_batch(ctx, he, 2, 8, list(range(1, 8)), 77, 1)
    assert ctx.hoist_tensor_launches() == n0
    assert np.array_equal(got[1], he.rotsum(OCt(cts[1], 8, D), list(range(1, 8))).data)
    with pytest.raises(binding.HeError) as e:
        ctx.set_hoist_form(2)
    assert e.value.code == binding.HE_EINVAL


def test_iteration_with_tensor_form_bitwise(pair):
    """A full-batch iteration (16 x 256 blocks, start level 6) with every
    hoisted group that fits on the tensor cores equals the oracle's circuit."""
    ctx, he = pair
    X, y = synth.small()
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    L = 6
    circ = qgnag.Circuit(he, 16, 256, D, start_level=L)
    Z = [he.encrypt(he.encode(data.blocks[b], L, D), 100 + b) for b in range(data.blocks.shape[0])]
    B = he.encrypt(he.encode(np.tile(data.n * data.bbar_full, circ.m), L, D), 200)
    rng = np.random.default_rng(12)
    w0 = np.tile(np.r_[rng.uniform(-0.5, 0.5, data.f1), np.zeros(16 - data.f1)], circ.m)
    W = he.encrypt(he.encode(w0, L, D), 201)
    V = he.encrypt(he.encode(0.5 * w0, L, D), 202)
    alpha, eta = qgnag.schedule(1), qgnag.nag_scalars(2)[1]
    Wn, Vn = circ.iteration(Z, B, W, V, alpha, eta, 1.0 / data.n)
    g = lambda c: ctx.import_ct(c.data, c.level, c.scale)  # noqa: E731
    n0 = ctx.hoist_tensor_launches()
    ctx.set_hoist_form(1)
    try:
        gW, gV = binding.lr_iteration(ctx, [g(z) for z in Z], g(B), g(W), g(V), 16, 256, alpha, eta,
                                      1.0 / data.n, qgnag.G8)
    finally:
        ctx.set_hoist_form(-1)
    ctx.check_device()
    assert ctx.hoist_tensor_launches() > n0
    assert np.array_equal(gW.export(), Wn.data)
    assert np.array_equal(gV.export(), Vn.data)
