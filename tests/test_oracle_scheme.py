"""Pins for the oracle's encryption scheme: decryption equals the message within
the noise bound, homomorphic operations equal their plaintext counterparts, and
on tiny N the decryption equation is checked with Python integers."""
import ctypes

import numpy as np
import pytest

from oracle.ckks import Ckks, Ct, Pt, ScaleError

D = 2.0 ** 40


def P(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.fixture(scope="module")
def he():
    h = Ckks(11, 9)
    h.keygen(7, [1, -1, 2, -2, 4, 64, 300])
    return h


def rand_slots(he, seed, scale=1.0, cplx=True):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-scale, scale, he.nslots)
    if cplx:
        z = z + 1j * rng.uniform(-scale, scale, he.nslots)
    return z


def enc(he, z, seed, level=None):
    lv = he.max_level if level is None else level
    return he.encrypt(he.encode(z, lv, D), seed)


def dec(he, ct):
    return he.decode(he.decrypt(ct))


def test_secret_key_is_ternary(he):
    s = he.secret_key()
    assert set(np.unique(s)) <= {-1, 0, 1}
    assert 0.25 < np.mean(s == 0) < 0.42


def test_decrypt_equation_tiny_n():
    """c0 + c1 s computed with Python integers and schoolbook convolution."""
    h = Ckks(4, 3)
    h.keygen(3)
    s = [int(x) for x in h.secret_key()]
    pt = h.encode(np.arange(8) / 8.0, 2, 2.0 ** 20)
    ct = h.encrypt(pt, 5)
    got = h.decrypt(ct)
    n = 16
    for j in range(3):
        q = h.q[j]
        c0 = [int(x) for x in ct.data[0][j]]
        c1 = [int(x) for x in ct.data[1][j]]
        want = list(c0)
        for i in range(n):
            for k in range(n):
                if i + k < n:
                    want[i + k] += c1[i] * s[k]
                else:
                    want[i + k - n] -= c1[i] * s[k]
        assert [int(x) for x in got.data[j]] == [w % q for w in want]


def test_fresh_noise_bound(he):
    z = rand_slots(he, 1)
    err = np.abs(dec(he, enc(he, z, 11)) - z).max()
    # noise coefficients are a few hundred at most; the embedding sums N of them
    assert err < 64 * 3.2 * np.sqrt(he.n) * np.sqrt(he.n) / D
    assert err < 1e-7


def test_add_cmul_cadd_ptmul(he):
    z1, z2 = rand_slots(he, 2), rand_slots(he, 3)
    c1, c2 = enc(he, z1, 12), enc(he, z2, 13)
    assert np.abs(dec(he, he.add(c1, c2)) - (z1 + z2)).max() < 1e-7
    assert np.abs(dec(he, he.sub(c1, c2)) - (z1 - z2)).max() < 1e-7
    m = he.rescale(he.cmul(c1, -0.37, D))
    assert np.abs(dec(he, m) - (-0.37 * z1)).max() < 1e-7
    a = he.cadd(c1, 0.625)
    assert np.abs(dec(he, a) - (z1 + 0.625)).max() < 1e-7
    pt = he.encode(z2, he.max_level, float(he.q[he.max_level]))
    m = he.rescale(he.ptmul(c1, pt))
    assert np.abs(dec(he, m) - z1 * z2).max() < 1e-7
    with pytest.raises(ScaleError):
        he.add(c1, Ct(c2.data, c2.level, c2.scale * 1.001))


def test_tensor_decrypts_with_s_squared(he):
    """(d0, d1, d2) decrypts under (1, s, s^2) to the product message; inputs are
    encoded at 2^26 so the 2^52-scale product stays below q_0 / 2."""
    z1, z2 = rand_slots(he, 4), rand_slots(he, 5)
    s = 2.0 ** 26
    lv = he.max_level
    c1 = he.encrypt(he.encode(z1, lv, s), 14)
    c2 = he.encrypt(he.encode(z2, lv, s), 15)
    d = he.tensor(c1, c2)
    zz = he.decode(he.decrypt3(d, lv, s * s))
    assert np.abs(zz - z1 * z2).max() < 1e-2
    r = he.relin(d, lv, s * s)
    assert np.abs(dec(he, r) - z1 * z2).max() < 1e-2


def test_relin_and_rescale_levels(he):
    z1, z2 = rand_slots(he, 6, cplx=False), rand_slots(he, 7, cplx=False)
    c = enc(he, z1, 16)
    c2 = enc(he, z2, 17)
    acc_z = z1.copy()
    for step in range(5):
        c = he.rescale(he.mul(c, he.moddrop(c2, c.level)))
        acc_z = acc_z * z2
        assert c.level == he.max_level - step - 1
        assert np.abs(dec(he, c) - acc_z).max() < 1e-6


@pytest.mark.parametrize("r", [1, -1, 2, -2, 4, 64, 300])
def test_rotation_matches_plaintext_roll(he, r):
    z = rand_slots(he, 8)
    c = enc(he, z, 18)
    got = dec(he, he.rotate(c, r))
    assert np.abs(got - np.roll(z, -r)).max() < 1e-7


def test_keys_depend_on_the_galois_element_not_the_request(he):
    """A key is a function of (seed, galois element): a context asked for only
    the rotation by 2 switches keys to exactly the words of one asked for a
    longer list, so contexts built for different circuits share keys."""
    other = Ckks(11, 9)
    other.keygen(7, [2])
    c = enc(he, rand_slots(he, 21), 23)
    d = c.data[1]
    for gal in (0, he.galois_elt(2)):
        assert np.array_equal(other.keyswitch(c.level, gal, d), he.keyswitch(c.level, gal, d))
    assert np.array_equal(other.rotate(c, 2).data, he.rotate(c, 2).data)


def test_rotation_at_lower_level(he):
    z = rand_slots(he, 9)
    c = he.moddrop(enc(he, z, 19), 3)
    assert np.abs(dec(he, he.rotate(c, 2)) - np.roll(z, -2)).max() < 1e-7


def test_keyswitch_identity_key_noise(he):
    """Key-switching d from s^2 to s: decrypts to d * s^2 within a small bound."""
    z1 = rand_slots(he, 10)
    c = enc(he, z1, 20)
    d = he.tensor(c, c)
    ks = he.keyswitch(c.level, 0, d[2])
    # (d0 + ks0) + (d1 + ks1) s  ==  d0 + d1 s + d2 s^2 + small
    full = he.decrypt3(d, c.level, D * D)
    lin = he.decrypt(Ct(np.stack([(d[0] + ks[0]) % np.array(he.q[:c.level + 1], np.uint64)[:, None],
                                  (d[1] + ks[1]) % np.array(he.q[:c.level + 1], np.uint64)[:, None]]),
                        c.level, D * D))
    q0 = he.q[0]
    diff = (full.data[0].astype(object) - lin.data[0].astype(object)) % q0
    diff = np.array([int(x) if x <= q0 // 2 else int(x) - q0 for x in diff])
    assert np.abs(diff).max() < 2 ** 16


def test_rescale_rounds_to_nearest(he):
    """Rescale of a trivial ciphertext (c1 = 0) divides the constant by q_l with rounding."""
    lv = 2
    n = he.n
    rng = np.random.default_rng(11)
    vals = rng.integers(-(1 << 62), 1 << 62, n, dtype=np.int64)
    data = np.zeros((2, lv + 1, n), np.uint64)
    for j in range(lv + 1):
        data[0, j] = [int(v) % he.q[j] for v in vals]
    out = he.rescale(Ct(data, lv, D))
    ql = he.q[lv]
    for j in range(lv):
        want = [((int(v) - ((int(v) % ql) if (int(v) % ql) <= ql // 2 else (int(v) % ql) - ql)) // ql) % he.q[j]
                for v in vals[:64]]
        assert [int(x) for x in out.data[0, j, :64]] == want
    assert not out.data[1].any()


def test_ptadd_adds_the_message():
    """c0 + m decrypts to the sum of the messages (same level and scale)."""
    he = Ckks(10, 3)
    he.keygen(3, [])
    rng = np.random.default_rng(21)
    a, b = rng.uniform(-1, 1, he.nslots), rng.uniform(-1, 1, he.nslots)
    ct = he.encrypt(he.encode(a, 2, 2.0 ** 30), 5)
    out = he.ptadd(ct, he.encode(b, 2, 2.0 ** 30))
    # the encryption noise cancels in the difference: what is left is b up to encoding rounding
    diff = he.decode(he.decrypt(out)).real - he.decode(he.decrypt(ct)).real
    assert np.abs(diff - b).max() < 1e-7
    assert np.abs(he.decode(he.decrypt(out)).real - (a + b)).max() < 1e-4
    with pytest.raises(ValueError):
        he.ptadd(ct, he.encode(b, 1, 2.0 ** 30))


def test_hoisted_rotation_sum_single_rotation_is_add_of_rotate(he):
    """One rotation through the hoisted path is exactly ct + Rot(ct): the
    shared ModUp and ModDown reduce to the key switch of one rotation."""
    ct = enc(he, rand_slots(he, 41), 43)
    for r in (1, -2, 300):
        assert np.array_equal(he.rotsum(ct, [r]).data, he.add(ct, he.rotate(ct, r)).data), r
    low = he.moddrop(ct, 3)
    assert np.array_equal(he.rotsum(low, [4]).data, he.add(low, he.rotate(low, 4)).data)


def test_hoisted_rotation_sum_decrypts_to_the_slot_sum(he):
    """ct + sum_j Rot(ct, r_j) with the inner products summed before one
    ModDown decrypts to z + sum_j rot(z, r_j) within the key-switching noise,
    and differs in its words from the sequential sum (one rounding, not
    several)."""
    z = rand_slots(he, 42)
    ct = enc(he, z, 44)
    rots = [1, 2, -1, 64]
    got = he.rotsum(ct, rots)
    want = z + sum(np.roll(z, -r) for r in rots)
    assert np.abs(dec(he, got) - want).max() < 1e-6
    seq = ct
    for r in rots:
        seq = he.add(seq, he.rotate(ct, r))
    assert not np.array_equal(got.data, seq.data)
    assert np.abs(dec(he, got) - dec(he, seq)).max() < 1e-6
    with pytest.raises(KeyError):
        he.rotsum(ct, [1, 5])  # no key for 5
