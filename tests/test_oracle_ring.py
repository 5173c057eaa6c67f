"""Pins for the oracle's modular arithmetic, primes and negacyclic NTT.

Each check compares the oracle with something other than itself: a library
primality test, the defining sums evaluated with Python integers, schoolbook
negacyclic convolution, or algebraic identities.
"""
import ctypes

import numpy as np
import pytest
import sympy

from oracle.ckks import Ckks


def P(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("logn,nq", [(4, 3), (13, 9), (16, 9)])
def test_prime_chain(oracle_lib, logn, nq):
    out = np.zeros(nq + 1, np.uint64)
    assert oracle_lib.orc_gen_primes(logn, nq, 60, 40, 60, P(out)) == 0
    ps = [int(x) for x in out]
    twon = 2 << logn
    assert len(set(ps)) == len(ps)
    for i, p in enumerate(ps):
        bits = 40 if 0 < i < nq else 60
        assert sympy.isprime(p)
        assert p % twon == 1
        assert p.bit_length() == bits
    # q_0 is the largest 60-bit candidate, q_1.. descend through the 40-bit ones
    def primes_desc(bits, count):
        v = ((1 << bits) - 2) // twon * twon + 1
        found = []
        while len(found) < count:
            if sympy.isprime(v):
                found.append(v)
            v -= twon
        return found
    sixty = primes_desc(60, 2)
    assert ps[0] == sixty[0] and ps[nq] == sixty[1]
    assert ps[1:nq] == primes_desc(40, nq - 1)


def test_miller_rabin_matches_sympy(oracle_lib):
    rng = np.random.default_rng(0)
    cands = [int(x) | 1 for x in rng.integers(1 << 40, 1 << 62, size=300, dtype=np.int64)]
    cands += [2, 3, 4, 561, 1105, 3215031751, 2152302898747, 3474749660383, 341550071728321]
    for c in cands:
        assert bool(oracle_lib.orc_is_prime(c)) == sympy.isprime(c), c


@pytest.mark.parametrize("logn", [3, 4, 13, 16])
def test_psi_primitive_2n_root(oracle_lib, logn):
    he = Ckks(logn, 3)
    n = 1 << logn
    psi = np.zeros(4, np.uint64)
    oracle_lib.orc_get_psi(he.ctx, P(psi))
    for p, s in zip(he.primes, psi):
        s = int(s)
        assert pow(s, n, p) == p - 1
        assert pow(s, 2 * n, p) == 1


def python_ntt(a, q, psi):
    n = len(a)
    return [sum(int(a[j]) * pow(psi, j * (2 * k + 1), q) for j in range(n)) % q for k in range(n)]


def test_ntt_matches_definition_python(oracle_lib):
    he = Ckks(3, 2)
    psi = np.zeros(3, np.uint64)
    oracle_lib.orc_get_psi(he.ctx, P(psi))
    rng = np.random.default_rng(1)
    for pi in range(3):
        q = he.primes[pi]
        a = np.array([int(x) % q for x in rng.integers(0, 1 << 62, 8, dtype=np.int64)], np.uint64)
        want = python_ntt(a, q, int(psi[pi]))
        b = a.copy()
        oracle_lib.orc_ntt(he.ctx, pi, P(b))
        assert [int(x) for x in b] == want
        d = np.zeros(8, np.uint64)
        oracle_lib.orc_ntt_direct(8, q, int(psi[pi]), P(a), P(d))
        assert [int(x) for x in d] == want


@pytest.mark.parametrize("logn", [4, 6, 10])
def test_ntt_matches_direct_and_inverts(oracle_lib, logn):
    he = Ckks(logn, 2)
    n = 1 << logn
    psi = np.zeros(3, np.uint64)
    oracle_lib.orc_get_psi(he.ctx, P(psi))
    rng = np.random.default_rng(logn)
    for pi in range(3):
        q = he.primes[pi]
        a = (rng.integers(0, 1 << 62, n, dtype=np.int64).astype(np.uint64) % np.uint64(q))
        fast = a.copy()
        oracle_lib.orc_ntt(he.ctx, pi, P(fast))
        direct = np.zeros(n, np.uint64)
        oracle_lib.orc_ntt_direct(n, q, int(psi[pi]), P(a), P(direct))
        assert np.array_equal(fast, direct)
        oracle_lib.orc_intt(he.ctx, pi, P(fast))
        assert np.array_equal(fast, a)


def python_negacyclic(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            p = int(a[i]) * int(b[j])
            if i + j < n:
                c[i + j] += p
            else:
                c[i + j - n] -= p
    return [x % q for x in c]


def test_schoolbook_matches_python(oracle_lib):
    rng = np.random.default_rng(2)
    q = 1152921504606845473
    a = rng.integers(0, q, 8, dtype=np.int64).astype(np.uint64)
    b = rng.integers(0, q, 8, dtype=np.int64).astype(np.uint64)
    c = np.zeros(8, np.uint64)
    oracle_lib.orc_polymul_schoolbook(8, q, P(a), P(b), P(c))
    assert [int(x) for x in c] == python_negacyclic(a, b, q)


@pytest.mark.parametrize("logn", [3, 4, 6, 10])
def test_ring_product_matches_schoolbook(oracle_lib, logn):
    he = Ckks(logn, 3)
    n = 1 << logn
    rng = np.random.default_rng(3 + logn)
    for pi in range(4):
        q = he.primes[pi]
        a = rng.integers(0, 1 << 62, n, dtype=np.int64).astype(np.uint64) % np.uint64(q)
        b = rng.integers(0, 1 << 62, n, dtype=np.int64).astype(np.uint64) % np.uint64(q)
        c1 = np.zeros(n, np.uint64)
        c2 = np.zeros(n, np.uint64)
        oracle_lib.orc_polymul(he.ctx, pi, P(a), P(b), P(c1))
        oracle_lib.orc_polymul_schoolbook(n, q, P(a), P(b), P(c2))
        assert np.array_equal(c1, c2)
        if n == 8:
            assert [int(x) for x in c1] == python_negacyclic(a, b, q)


def test_automorphism_definition_and_homomorphism(oracle_lib):
    he = Ckks(4, 2)
    n, q = 16, he.primes[1]
    rng = np.random.default_rng(4)
    a = rng.integers(0, q, n, dtype=np.int64).astype(np.uint64)
    b = rng.integers(0, q, n, dtype=np.int64).astype(np.uint64)
    for g in (5, 25, 3, 2 * n - 1):
        sa = np.zeros(n, np.uint64)
        oracle_lib.orc_automorph(he.ctx, 1, g, P(a), P(sa))
        # definition: X^k -> X^(k g) with X^N = -1
        want = [0] * n
        for k in range(n):
            e = (k * g) % (2 * n)
            if e < n:
                want[e] = int(a[k])
            else:
                want[e - n] = (-int(a[k])) % q
        assert [int(x) for x in sa] == want
        # sigma(a b) = sigma(a) sigma(b)
        ab = np.zeros(n, np.uint64)
        oracle_lib.orc_polymul(he.ctx, 1, P(a), P(b), P(ab))
        s_ab = np.zeros(n, np.uint64)
        oracle_lib.orc_automorph(he.ctx, 1, g, P(ab), P(s_ab))
        sb = np.zeros(n, np.uint64)
        oracle_lib.orc_automorph(he.ctx, 1, g, P(b), P(sb))
        prod = np.zeros(n, np.uint64)
        oracle_lib.orc_polymul(he.ctx, 1, P(sa), P(sb), P(prod))
        assert np.array_equal(s_ab, prod)
