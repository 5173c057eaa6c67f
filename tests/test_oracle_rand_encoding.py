"""Pins for the oracle's randomness and canonical-embedding encoder."""
import ctypes
import os

import numpy as np
import pytest

from oracle.ckks import Ckks

HERE = os.path.dirname(os.path.abspath(__file__))


def P(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_splitmix64_published_vector(oracle_lib):
    want = [int(l, 16) for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    st = ctypes.c_uint64(0)
    got = [oracle_lib.orc_splitmix64_next(ctypes.byref(st)) for _ in want]
    assert got == want


def test_counter_words_are_splitmix64_positions(oracle_lib):
    # word(seed, stream, idx) is output number (stream << 40) + idx + 1 of
    # splitmix64 started at state mix64(seed); mix64(0) == 0, so for seed 0 and
    # stream 0 the words are the plain splitmix64 sequence from state 0.
    st = ctypes.c_uint64(0)
    seq = [oracle_lib.orc_splitmix64_next(ctypes.byref(st)) for _ in range(5)]
    assert [oracle_lib.orc_rand_word(0, 0, i) for i in range(5)] == seq


def _sample(oracle_lib, kind, n, q=0, sigma=3.2, seed=9, stream=77):
    out = np.zeros(n, np.int64)
    oracle_lib.orc_sample(seed, stream, kind, q, sigma, n, P(out))
    return out


def test_ternary_distribution(oracle_lib):
    x = _sample(oracle_lib, 0, 300000)
    assert set(np.unique(x)) == {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(x == v) - 1 / 3) < 0.005


def test_gaussian_distribution(oracle_lib):
    x = _sample(oracle_lib, 1, 400000)
    assert abs(x.mean()) < 0.03
    assert abs(x.var() - 3.2 ** 2) < 0.15
    assert np.abs(x).max() <= 20
    # discrete Gaussian: P(0) / P(1) = exp(1 / (2 sigma^2))
    r = np.mean(x == 0) / (np.mean(np.abs(x) == 1) / 2)
    assert abs(r - np.exp(1 / (2 * 3.2 ** 2))) < 0.03


def test_uniform_distribution(oracle_lib):
    q = 1099511627297
    x = _sample(oracle_lib, 2, 200000, q=q)
    assert x.min() >= 0 and x.max() < q
    assert abs(x.mean() / q - 0.5) < 0.005


def test_cdt_table_monotone(oracle_lib):
    cdt = np.zeros(64, np.uint64)
    k = oracle_lib.orc_cdt_table(3.2, P(cdt), 64)
    assert k == 21
    assert np.all(np.diff(cdt[:k].astype(np.float64)) > 0)
    assert int(cdt[k - 1]) == 1 << 63


# ---------------------------------------------------------------- encoding
def direct_embed_inv(z, n):
    """m_k = (2/N) Re(sum_j z_j zeta_j^-k), zeta_j = exp(i pi 5^j / N)."""
    ns = n // 2
    t = np.array([pow(5, j, 2 * n) for j in range(ns)])
    k = np.arange(n)
    zeta = np.exp(-1j * np.pi * np.outer(k, t) / n)  # [k, j]
    return (2.0 / n) * np.real(zeta @ z)


def direct_embed(coef, n):
    ns = n // 2
    t = np.array([pow(5, j, 2 * n) for j in range(ns)])
    k = np.arange(n)
    return np.exp(1j * np.pi * np.outer(t, k) / n) @ coef


@pytest.mark.parametrize("logn", [3, 5, 8])
def test_embedding_matches_direct(logn):
    he = Ckks(logn, 2)
    n = 1 << logn
    rng = np.random.default_rng(logn)
    z = rng.standard_normal(n // 2) + 1j * rng.standard_normal(n // 2)
    coef = he.embed_inv(z)
    assert np.allclose(coef, direct_embed_inv(z, n), atol=1e-12)
    c2 = rng.standard_normal(n)
    assert np.allclose(he.embed(c2), direct_embed(c2, n), atol=1e-9)
    assert np.allclose(he.embed(coef), z, atol=1e-12)


def test_encode_decode_roundtrip():
    he = Ckks(12, 4)
    rng = np.random.default_rng(5)
    z = rng.uniform(-4, 4, he.nslots) + 1j * rng.uniform(-4, 4, he.nslots)
    pt = he.encode(z, 3, 2.0 ** 40)
    # every limb holds the same integer coefficients
    q = he.q
    c0 = [int(x) if int(x) <= q[0] // 2 else int(x) - q[0] for x in pt.data[0][:64]]
    for j in range(1, 4):
        assert [int(x) for x in pt.data[j][:64]] == [c % q[j] for c in c0]
    assert np.abs(he.decode(pt) - z).max() < 2 ** -30


def test_encoding_is_multiplicative_and_rotation_is_galois(oracle_lib):
    """encode(z1) * encode(z2) decodes to z1 * z2 slotwise, and X -> X^(5^r)
    rotates the slot vector left by r: pins the slot ordering."""
    he = Ckks(10, 2)
    rng = np.random.default_rng(6)
    z1 = rng.uniform(-1, 1, he.nslots) + 1j * rng.uniform(-1, 1, he.nslots)
    z2 = rng.uniform(-1, 1, he.nslots) + 1j * rng.uniform(-1, 1, he.nslots)
    s = 2.0 ** 25
    p1, p2 = he.encode(z1, 0, s), he.encode(z2, 0, s)
    prod = np.zeros(he.n, np.uint64)
    oracle_lib.orc_polymul(he.ctx, 0, P(p1.data[0]), P(p2.data[0]), P(prod))
    from oracle.ckks import Pt
    got = he.decode(Pt(prod[None, :], 0, s * s))
    assert np.abs(got - z1 * z2).max() < 1e-5
    for r in (1, 3, 17):
        g = he.galois_elt(r)
        assert g == pow(5, r, 2 * he.n)
        rot = np.zeros(he.n, np.uint64)
        oracle_lib.orc_automorph(he.ctx, 0, g, P(p1.data[0]), P(rot))
        got = he.decode(Pt(rot[None, :], 0, s))
        assert np.abs(got - np.roll(z1, -r)).max() < 1e-6
