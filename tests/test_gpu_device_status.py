"""The device status word (he_check_device): a bounded device-side wait that
runs out is reported as HE_ETIMEOUT, once, and the context keeps computing.
The wait is made to run out with a barrier that nothing arrives on
(he_selftest_bounded_wait(ctx, 0)); nothing faults, traps or hangs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle.ckks import Ckks  # noqa: E402
from paper_2406_13221_gb300 import binding, build  # noqa: E402

build.build()
D = 2.0 ** 40


def test_expired_wait_is_reported_and_the_context_survives():
    ctx = binding.Context(10, 4)
    he = Ckks(10, 4)
    ctx.keygen(2, [1])
    he.keygen(2, [1])
    ctx.selftest_bounded_wait(1)  # the barrier completes: nothing to report
    ctx.check_device()
    ctx.selftest_bounded_wait(0)  # nothing arrives: the wait runs out after 1 s
    with pytest.raises(binding.HeError) as e:
        ctx.check_device()
    assert e.value.code == binding.HE_ETIMEOUT
    ctx.check_device()  # reported once, then cleared
    z = np.random.default_rng(3).uniform(-1, 1, ctx.nslots)
    ref = he.encrypt(he.encode(z, 3, D), 5)
    got = ctx.rotate(ctx.import_ct(ref.data, 3, D), 1)
    assert np.array_equal(got.export(), he.rotate(ref, 1).data)
