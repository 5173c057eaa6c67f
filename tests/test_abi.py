"""The C-ABI library builds, loads and exports every symbol include/he_lr.h
declares; its host-only tables equal the oracle's bit for bit; without a GPU the
compute entry points fail loudly instead of falling back to the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_13221_gb300 import binding, build
    build.build()
    return binding.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "he_lr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(he_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2406_13221_gb300 import binding
    syms = declared_symbols()
    assert len(syms) >= 40
    for s in syms:
        assert hasattr(lib, s), s
        assert s in binding.SIGNATURES, s


def test_gauss_table_matches_oracle(lib, oracle_lib):
    from paper_2406_13221_gb300 import binding
    for sigma in (3.2, 1.0, 6.4):
        ours = binding.gauss_table(sigma)
        ref = np.zeros(64, np.uint64)
        k = oracle_lib.orc_cdt_table(sigma, ref.ctypes.data_as(ctypes.c_void_p), 64)
        assert np.array_equal(ours, ref[:k])


@pytest.mark.parametrize("logn", [10, 13, 16])
def test_zeta_table_matches_oracle(lib, logn):
    from oracle.ckks import Ckks
    from paper_2406_13221_gb300 import binding
    re_, im_ = binding.zeta_table(logn)
    he = Ckks(logn, 2)
    r2, i2 = np.zeros(2 << logn), np.zeros(2 << logn)
    he.L.orc_get_zeta_table(he.ctx, r2.ctypes.data_as(ctypes.c_void_p), i2.ctypes.data_as(ctypes.c_void_p))
    assert np.array_equal(re_.view(np.uint64), r2.view(np.uint64))
    assert np.array_equal(im_.view(np.uint64), i2.view(np.uint64))


def test_client_bbar_matches_oracle(lib):
    from oracle import qgnag
    from paper_2406_13221_gb300 import binding, synth
    X, y = synth.small(seed=3, n=3000, f=20)
    Z = qgnag.make_z(X, y)
    for r0, rows in ((0, 1024), (2048, 952)):
        ours = binding.lr_bbar(X, y, r0, rows, 32)
        ref = qgnag.bbar_rows(Z[r0:r0 + rows], 32)
        assert np.allclose(ours, ref, rtol=1e-12, atol=0)
        assert not ours[21:].any()


def test_invalid_arguments_are_rejected(lib):
    from paper_2406_13221_gb300 import binding
    h = ctypes.c_void_p()
    p = binding.he_params(9, 9, 60, 40, 60, 3.2)   # log_n below the supported range
    assert lib.he_ctx_create(ctypes.byref(p), None, ctypes.byref(h)) == binding.HE_EINVAL
    p = binding.he_params(13, 1, 60, 40, 60, 3.2)  # one prime is not a chain
    assert lib.he_ctx_create(ctypes.byref(p), None, ctypes.byref(h)) == binding.HE_EINVAL
    assert lib.he_ctx_create(None, None, ctypes.byref(h)) == binding.HE_EINVAL


def test_no_gpu_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2406_13221_gb300 import binding
    with pytest.raises(binding.HeError) as e:
        binding.Context(13, 9)
    assert e.value.code == binding.HE_ECUDA
