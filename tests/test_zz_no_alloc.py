"""he_rescale_noalloc: a rescale for callers that may not allocate device memory
(code running under a device-memory budget fixed in advance, or inside a host
framework that owns every allocation).  It must return exactly what he_rescale
returns, and what the oracle's rescale (rounded division by the dropped prime)
returns, on consecutive calls that share its fixed work space, and refuse
sizes the work space cannot hold.

This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.ckks import Ckks, Ct as OCt  # noqa: E402
from paper_2406_13221_gb300 import binding, build  # noqa: E402

build.build()


def random_ct_words(primes, level, batch, n, seed):
    rng = np.random.default_rng(seed)
    w = np.zeros((batch, 2, level + 1, n), np.uint64)
    for j in range(level + 1):
        w[:, :, j, :] = rng.integers(0, primes[j], (batch, 2, n), dtype=np.uint64)
    return w


def reference(ctx, words, level):
    """he_rescale (the allocating entry point) on each ciphertext, coefficient words."""
    out = []
    for w in words:
        ct = ctx.import_ct(w, level, 2.0 ** 40)
        out.append(ctx.rescale(ct).export())
    return np.stack(out)


def oracle_rescale(he, words, level):
    """The oracle's rescale of each ciphertext (coefficient words)."""
    return np.stack([he.rescale(OCt(w, level, 2.0 ** 40)).data for w in words])


def no_alloc(ctx, words, level):
    batch, n = words.shape[0], ctx.n
    dev_in = torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda()
    dev_out = torch.zeros(batch * 2 * level * n, dtype=torch.int64, device="cuda")
    ctx.ntt_forward(dev_in.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    ctx.rescale_noalloc(dev_in.data_ptr(), dev_out.data_ptr(), batch, level)
    ctx.ntt_inverse(dev_out.data_ptr(), batch * 2 * level, list(range(level)))
    torch.cuda.synchronize()
    return dev_out.cpu().numpy().view(np.uint64).reshape(batch, 2, level, n)


def test_no_alloc_rescale_matches_he_rescale_on_two_calls():
    ctx = binding.Context(13, 9)
    he = Ckks(13, 9)
    for call, (level, batch) in enumerate(((8, 3), (4, 5))):
        words = random_ct_words(ctx.primes, level, batch, ctx.n, seed=40 + call)
        got = no_alloc(ctx, words, level)
        assert np.array_equal(got, reference(ctx, words, level)), call
        assert np.array_equal(got, oracle_rescale(he, words, level)), call


def test_no_alloc_rescale_splits_large_batches_and_refuses_oversized_work():
    ctx = binding.Context(16, 17)
    level, batch = 7, 3  # 16 limbs of 2^16 words per ciphertext: two per pass of the work space
    words = random_ct_words(ctx.primes, level, batch, ctx.n, seed=50)
    got = no_alloc(ctx, words, level)
    assert np.array_equal(got, reference(ctx, words, level))
    assert np.array_equal(got, oracle_rescale(Ckks(16, 17), words, level))
    with pytest.raises(binding.HeError) as e:
        ctx.rescale_noalloc(1, 1, 1, 16)  # (2 + 2*16) * 2^16 words exceed the work space
    assert e.value.code == binding.HE_EINVAL
    assert "work" in str(e.value)
