"""Pins for the oracle's bootstrapping (oracle/boot.py), each against what the
mathematics fixes: the series against the library cosine, the polynomial and
the double angles against sin on their interval, E^H / n as the inverse of the
encoding, ModRaise's integer lift, the monomial X^(N/2) as multiplication by i,
the trace as G times the periodic part, and the whole bootstrap against the
message it refreshes."""
import math

import numpy as np
import pytest

from oracle import boot
from oracle.ckks import Ckks

D = 2.0 ** 40
BITS = [50, 45] + [55] * 12  # q0, the output level, 12 levels of the bootstrap


@pytest.fixture(scope="module")
def setup():
    he = Ckks(10, len(BITS), bits=BITS, secret_weight=16)
    p = boot.BootParams(n=8, K=8, r=4, deg=23, delta_out=D, out_level=1)
    rots, gals = boot.key_rotations(he, p)
    he.keygen(5, rots, gals)
    return he, p


def periodic(he, n, seed, amp=1.0):
    z = np.random.default_rng(seed).uniform(-amp, amp, n)
    return np.tile(z, he.nslots // n)


def test_chain_and_sparse_secret(setup):
    he, p = setup
    assert [q.bit_length() for q in he.primes] == BITS + [60]
    assert all(q % (2 * he.n) == 1 for q in he.primes)
    s = he.secret_key()
    assert np.count_nonzero(s) == 16 and set(np.unique(s)) <= {-1, 0, 1}
    assert p.depth() == 12 and he.max_level == 13


def test_series_match_the_library_cosine():
    for b in (-0.3, -math.pi / 32, 0.0, 0.7):
        c, s = boot.taylor_cos_sin(b)
        assert abs(c - math.cos(b)) < 1e-15 and abs(s - math.sin(b)) < 1e-15


@pytest.mark.parametrize("K,r,deg", [(8, 4, 23), (16, 6, 19)])
def test_cosine_polynomial_and_double_angles_against_sin(K, r, deg):
    """On |v| <= K + 1/2: the Taylor polynomial of cos(2 pi (v - 1/4) / 2^r)
    within its remainder bound, and after r double angles sin(2 pi v) within
    the bound amplified 4^r; near integers, sin(2 pi v) / 2 pi is v - round(v)."""
    p = boot.BootParams(n=8, K=K, r=r, deg=deg, delta_out=D, out_level=1)
    c = p.cos_coeffs()
    A = 2 * math.pi * p.Kp / 2 ** r
    v = np.linspace(-p.Kp, p.Kp, 20001)
    x = v / p.Kp
    poly = sum(ck * x ** k for k, ck in enumerate(c))
    exact = np.cos(2 * np.pi * (v - 0.25) / 2 ** r)
    bound = A ** (deg + 1) / math.factorial(deg + 1)
    assert np.abs(poly - exact).max() <= bound + 1e-13
    y = poly
    for _ in range(r):
        y = 2 * y * y - 1
    assert np.abs(y - np.sin(2 * np.pi * v)).max() <= 4 ** r * (bound + 1e-13)
    eps = np.linspace(-1e-3, 1e-3, 11)
    for I in (-K, -3, 0, 5, K):
        xv = (I + eps) / p.Kp
        yv = sum(ck * xv ** k for k, ck in enumerate(c))
        for _ in range(r):
            yv = 2 * yv * yv - 1
        assert np.abs(yv / (2 * np.pi) - eps).max() < 1e-8


def test_encoding_matrix_inverse_and_slots(setup):
    """E E^H = n I, and E maps the coefficient pairs (t_k + i t_(k+n)) of a
    subring element to its slots as the encoder places them."""
    he, p = setup
    n = p.n
    Ere, Eim = boot.encoding_matrix(he, n)
    E = Ere + 1j * Eim
    assert np.allclose(E @ E.conj().T, n * np.eye(n), atol=1e-12)
    rng = np.random.default_rng(3)
    G = he.n // (2 * n)
    t = np.zeros(he.n)
    t[::G] = rng.integers(-1000, 1000, 2 * n)  # an element of Z[Y], Y = X^G
    w = t[::G][:n] + 1j * t[::G][n:]
    # the oracle's decode of an exact (noise-free) plaintext with these coefficients
    pt = np.zeros((1, he.n), np.uint64)
    pt[0] = (t.astype(np.int64) % np.int64(he.q[0])).astype(np.uint64)
    from oracle.ckks import Pt
    z = he.decode(Pt(pt, 0, 1.0))
    assert np.allclose(z[:n], E @ w, atol=1e-6)
    assert np.allclose(z, np.tile(z[:n], he.nslots // n), atol=1e-6)  # period n


def test_mod_raise_is_an_integer_lift(setup):
    """Decrypting the raised ciphertext modulo Q gives m + e + q0 I: modulo q0 it
    is the level-0 decryption, and I is a small integer polynomial."""
    he, p = setup
    ct = he.encrypt(he.encode(periodic(he, p.n, 4), 0, D), 11)
    low = he.decrypt(ct).data[0].astype(np.int64)
    t = boot.mod_raise(he, ct, 3)
    dec = he.decrypt(t).data  # [4][N]
    q = [int(x) for x in he.q[:4]]
    Q = q[0] * q[1] * q[2] * q[3]
    for k in range(0, he.n, 37):
        # CRT of the four residues, centred
        x = 0
        for j in range(4):
            Mj = Q // q[j]
            x += int(dec[j][k]) * Mj * pow(Mj, -1, q[j])
        x %= Q
        x = x - Q if x > Q // 2 else x
        lo = int(low[k])
        lo = lo - q[0] if lo > q[0] // 2 else lo
        I, rem = divmod(x - lo, q[0])
        assert rem == 0 and abs(I) <= p.K


def test_monomial_is_multiplication_by_i(setup):
    he, p = setup
    z = periodic(he, p.n, 5) + 1j * periodic(he, p.n, 6)
    ct = he.encrypt(he.encode(z, 2, D), 12)
    got = he.decode(he.decrypt(boot.monomial(he, ct, he.n // 2)))
    assert np.abs(got - 1j * z).max() < 1e-6
    got = he.decode(he.decrypt(boot.monomial(he, ct, 3 * he.n // 2)))
    assert np.abs(got + 1j * z).max() < 1e-6


def test_subsum_is_g_times_the_periodic_part(setup):
    """The trace of a period-n slot vector is G times itself (G = N / 2n)."""
    he, p = setup
    z = periodic(he, p.n, 7)
    ct = he.encrypt(he.encode(z, 3, D), 13)
    for rots in boot.subsum_rotations(he.n, p.n):
        ct = he.rotsum(ct, rots)
    G = he.n // (2 * p.n)
    assert np.abs(he.decode(he.decrypt(ct)).real - G * z).max() < 1e-5


@pytest.mark.parametrize("amp", [1.0, 20.0])
def test_bootstrap_refreshes_the_message(setup, amp):
    """A level-0 ciphertext of a period-8 slot vector comes back at level 1,
    scale 2^40, with the same slots: within 1e-6 of the amplitude plus the
    error of sin(2 pi eps) / 2 pi against eps, a relative (2 pi eps)^2 / 6 with
    eps = amp Delta / q0 at most."""
    he, p = setup
    z = periodic(he, p.n, 8, amp)
    ct = he.encrypt(he.encode(z, 0, D), 14)
    out = boot.bootstrap(he, ct, p)
    assert (out.level, out.scale) == (1, D)
    got = he.decode(he.decrypt(out))
    eps = amp * D / he.q[0]
    tol = amp * (1e-6 + (2 * math.pi * eps) ** 2 / 6)
    assert np.abs(got.real - z).max() < tol
    assert np.abs(got.imag).max() < tol
    # and the refreshed ciphertext computes: one more product at level 1
    sq = he.rescale(he.mul(out, out))
    assert np.abs(he.decode(he.decrypt(sq)).real - z * z).max() < 2 * amp * tol + 1e-6 * amp * amp


def test_training_with_bootstrapped_refresh_tracks_the_twin():
    """The encrypted QG-NAG iteration with W and V refreshed by bootstrapping
    (no decryption between iterations) on a bootstrappable chain at N = 2^12
    (q0 50 bits, six 40-bit levels for the iteration, thirteen 55-bit levels
    for the bootstrap): the decrypted weights after two iterations within
    1e-3 of the FP64 plaintext run."""
    from oracle import plain, qgnag
    from paper_2406_13221_gb300 import synth
    bits = [50] + [40] * 6 + [55] * 13
    he = Ckks(12, len(bits), bits=bits, secret_weight=32)
    X, y = synth.small(seed=17, n=1024, f=15)
    data = qgnag.TrainData(X, y, g=16, m=128, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 128, D)
    p = boot.BootParams(n=16, K=12, r=5, deg=23, delta_out=D, out_level=circ.L)
    rots, gals = boot.key_rotations(he, p)
    he.keygen(2, sorted(set(circ.rotations()) | set(rots)), gals)
    L = circ.L
    Z = [he.encrypt(he.encode(data.blocks[b], L, D), 100 + b) for b in range(data.blocks.shape[0])]
    B = he.encrypt(he.encode(np.tile(data.n * data.bbar_full, circ.m), L, D), 200)
    W = he.encrypt(he.encode(np.zeros(he.nslots), L, D), 201)
    V = he.encrypt(he.encode(np.zeros(he.nslots), L, D), 202)
    etas = qgnag.nag_scalars(2)
    for t in range(2):
        Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(t), etas[t], 1.0 / data.n)
        assert Wn.level == 0
        W, V = boot.bootstrap(he, Wn, p), boot.bootstrap(he, Vn, p)
        assert (W.level, W.scale) == (L, D)
    w = he.decode(he.decrypt(W)).real.reshape(circ.m, circ.g)
    wp = plain.train(data, 2)
    assert np.abs(w[0] - wp).max() < 1e-3 and np.abs(w[-1] - wp).max() < 1e-3
