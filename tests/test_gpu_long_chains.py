"""Parity on long chains and the other transform sizes of the primitive sweep:
N = 2^14 with 24 primes and N = 2^15 with 16 primes (60-bit q_0, 40-bit q_i,
60-bit P).  The batched Mul (with relinearisation), Rescale, Rotation and a
hoisted rotation sum at the top level, where every key switch has 16-24
digits, equal the oracle's word for word.  These are the sizes the sweep times
(key switches of up to 24 digits accumulate 24 x 20 q^2 in 128 bits)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.ckks import Ckks, Ct as OCt  # noqa: E402
from paper_2406_13221_gb300 import binding, build  # noqa: E402

build.build()
D = 2.0 ** 40


@pytest.mark.parametrize("logn,nq", [(14, 24), (15, 16)])
def test_long_chain_primitives_bitwise(logn, nq):
    ctx = binding.Context(logn, nq)
    he = Ckks(logn, nq)
    ctx.keygen(2, [1, 2, 3])
    he.keygen(2, [1, 2, 3])
    assert ctx.primes == he.primes
    n, level, batch = ctx.n, nq - 1, 3
    rng = np.random.default_rng(logn)
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
    prod, rot, rsum = torch.zeros_like(da), torch.zeros_like(da), torch.zeros_like(da)
    resc = torch.zeros(batch * 2 * level * n, dtype=torch.int64, device="cuda")
    ctx.mul_relin_batch(da.data_ptr(), db.data_ptr(), prod.data_ptr(), batch, level)
    ctx.rescale_batch(prod.data_ptr(), resc.data_ptr(), batch, level)
    ctx.rotate_batch(da.data_ptr(), rot.data_ptr(), batch, level, 1)
    ctx.rotsum_batch(da.data_ptr(), rsum.data_ptr(), batch, level, [1, 2, 3])
    got_p, got_s, got_r, got_h = host(prod, level), host(resc, level - 1), host(rot, level), host(rsum, level)
    for b in (0, batch - 1):
        a, bb = OCt(A[b], level, D), OCt(B[b], level, D)
        ref = he.mul(a, bb)
        assert np.array_equal(got_p[b], ref.data), b
        assert np.array_equal(got_s[b], he.rescale(ref).data), b
        assert np.array_equal(got_r[b], he.rotate(a, 1).data), b
        assert np.array_equal(got_h[b], he.rotsum(a, [1, 2, 3]).data), b
    ctx.check_device()
