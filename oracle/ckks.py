"""Ciphertext objects and scale bookkeeping over the C primitives of he_oracle.c.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 2.1) lists the approximate-HE operations its training loop uses:
Enc, Dec, Add, cAdd, Mul, cMul, rotation and rescaling.  Each method below is
one of those, on the RNS form of the scheme.  All ciphertext words are kept in
coefficient form as numpy uint64 arrays of shape [2][level+1][N].

Scale rule (identical in the CUDA library's host code):
  * Mul / plaintext product: scale_out = scale_a * scale_b
  * Rescale at level l:      scale_out = scale / q_l
  * cMul by a real c at constant scale S: the integer round_half_away(c * S)
    multiplies every limb and scale_out = scale * S
  * cAdd of a real c: the integer round_half_away(c * scale) is added to the
    constant coefficient of c0
  * Add: both scales must agree to a relative 2^-40; scale_out = scale_a
"""
import ctypes
import math

import numpy as np

from . import lib

P = ctypes.c_void_p


def _p(a):
    return a.ctypes.data_as(P)


def round_half_away(x):
    """Nearest integer to the double x, halfway cases away from zero (C llround)."""
    f = math.floor(x)
    d = x - f  # exact for |x| < 2^52
    if d > 0.5 or (d == 0.5 and x > 0):
        f += 1
    return int(f)


class Pt:
    def __init__(self, data, level, scale):
        self.data, self.level, self.scale = data, level, scale


class Ct:
    def __init__(self, data, level, scale):
        self.data, self.level, self.scale = data, level, scale

    def copy(self):
        return Ct(self.data.copy(), self.level, self.scale)


class ScaleError(ValueError):
    pass


class Ckks:
    """One parameter set: ring degree 2^logn, ciphertext primes q_0..q_{nq-1},
    one special prime P, error width sigma."""

    def __init__(self, logn, nq, q0_bits=60, qi_bits=40, p_bits=60, sigma=3.2, bits=None, secret_weight=0):
        """bits: one bit width per ciphertext prime q_0..q_{nq-1} (default: q0_bits,
        then qi_bits); secret_weight: h > 0 gives the secret exactly h nonzero
        ternary coefficients (0: every coefficient uniform in {-1, 0, 1})."""
        self.L = lib()
        if bits is None:
            self.ctx = self.L.orc_ctx_new(logn, nq, q0_bits, qi_bits, p_bits, sigma)
        else:
            if len(bits) != nq:
                raise ValueError("one bit width per ciphertext prime")
            b = np.asarray(bits, np.int32)
            self.ctx = self.L.orc_ctx_new_bits(logn, nq, _p(b), p_bits, sigma)
        if not self.ctx:
            raise ValueError("no prime chain for these parameters")
        if self.L.orc_set_secret_weight(self.ctx, int(secret_weight)):
            raise ValueError("secret weight out of range")
        self.logn, self.n, self.nslots, self.nq = logn, 1 << logn, 1 << (logn - 1), nq
        self.max_level = nq - 1
        pr = np.zeros(nq + 1, np.uint64)
        self.L.orc_get_primes(self.ctx, _p(pr))
        self.primes = [int(x) for x in pr]
        self.q = self.primes[:nq]
        self.P = self.primes[nq]

    def __del__(self):
        try:
            self.L.orc_ctx_free(self.ctx)
        except Exception:
            pass

    # ---------------- keys ----------------
    def galois_elt(self, r):
        return int(self.L.orc_galois_elt(self.ctx, int(r)))

    def keygen(self, seed, rotations=(), extra_gals=()):
        """Secret, public key, relinearisation key and one key-switching key per
        rotation amount (and per raw Galois element in extra_gals, e.g. 2N - 1
        for the conjugation X -> X^-1)."""
        gals = np.array([self.galois_elt(r) for r in rotations] + [int(g) for g in extra_gals], np.uint64)
        rc = self.L.orc_keygen(self.ctx, seed, _p(gals), len(gals))
        if rc:
            raise RuntimeError("keygen failed")

    def secret_key(self):
        s = np.zeros(self.n, np.int64)
        self.L.orc_get_sk(self.ctx, _p(s))
        return s

    # ---------------- encoding ----------------
    def encode(self, z, level, scale):
        if not 0 <= level <= self.max_level:
            raise ValueError("level out of range")
        z = np.asarray(z, np.complex128)
        zr = np.zeros(self.nslots)
        zi = np.zeros(self.nslots)
        zr[:len(z)] = z.real
        zi[:len(z)] = z.imag
        out = np.zeros((level + 1, self.n), np.uint64)
        if self.L.orc_encode(self.ctx, _p(zr), _p(zi), level, float(scale), _p(out)):
            raise OverflowError("encoded coefficient out of range")
        return Pt(out, level, float(scale))

    def decode(self, pt):
        zr = np.zeros(self.nslots)
        zi = np.zeros(self.nslots)
        self.L.orc_decode(self.ctx, _p(np.ascontiguousarray(pt.data)), pt.scale, _p(zr), _p(zi))
        return zr + 1j * zi

    def embed_inv(self, z):
        z = np.asarray(z, np.complex128)
        zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        coef = np.zeros(self.n)
        self.L.orc_embed_inv(self.ctx, _p(zr), _p(zi), _p(coef))
        return coef

    def embed(self, coef):
        coef = np.ascontiguousarray(coef, np.float64)
        zr = np.zeros(self.nslots)
        zi = np.zeros(self.nslots)
        self.L.orc_embed(self.ctx, _p(coef), _p(zr), _p(zi))
        return zr + 1j * zi

    # ---------------- encryption ----------------
    def encrypt(self, pt, seed):
        ct = np.zeros((2, pt.level + 1, self.n), np.uint64)
        self.L.orc_encrypt(self.ctx, _p(np.ascontiguousarray(pt.data)), pt.level, seed, _p(ct))
        return Ct(ct, pt.level, pt.scale)

    def decrypt(self, ct):
        pt = np.zeros((ct.level + 1, self.n), np.uint64)
        self.L.orc_decrypt(self.ctx, _p(np.ascontiguousarray(ct.data)), ct.level, _p(pt))
        return Pt(pt, ct.level, ct.scale)

    def decrypt3(self, d, level, scale):
        pt = np.zeros((level + 1, self.n), np.uint64)
        self.L.orc_decrypt3(self.ctx, _p(np.ascontiguousarray(d)), level, _p(pt))
        return Pt(pt, level, scale)

    # ---------------- arithmetic ----------------
    @staticmethod
    def _check_scales(a, b):
        if a.level != b.level:
            raise ValueError("level mismatch %d vs %d" % (a.level, b.level))
        if abs(a.scale - b.scale) > a.scale * 2.0 ** -40:
            raise ScaleError("scale mismatch %r vs %r" % (a.scale, b.scale))

    def add(self, a, b):
        self._check_scales(a, b)
        out = np.zeros_like(a.data)
        self.L.orc_add(self.ctx, a.level, 2, _p(a.data), _p(b.data), _p(out), 0)
        return Ct(out, a.level, a.scale)

    def sub(self, a, b):
        self._check_scales(a, b)
        out = np.zeros_like(a.data)
        self.L.orc_add(self.ctx, a.level, 2, _p(a.data), _p(b.data), _p(out), 1)
        return Ct(out, a.level, a.scale)

    def tensor(self, a, b):
        if a.level != b.level:
            raise ValueError("level mismatch")
        d = np.zeros((3, a.level + 1, self.n), np.uint64)
        self.L.orc_tensor(self.ctx, a.level, _p(a.data), _p(b.data), _p(d))
        return d

    def keyswitch(self, level, gal, poly):
        out = np.zeros((2, level + 1, self.n), np.uint64)
        if self.L.orc_keyswitch(self.ctx, level, gal, _p(np.ascontiguousarray(poly)), _p(out)):
            raise KeyError("no key-switching key for galois element %d" % gal)
        return out

    def relin(self, d, level, scale):
        out = np.zeros((2, level + 1, self.n), np.uint64)
        if self.L.orc_relin(self.ctx, level, _p(np.ascontiguousarray(d)), _p(out)):
            raise KeyError("no relinearisation key")
        return Ct(out, level, scale)

    def mul(self, a, b):
        """Mul = tensor + relinearisation (no rescale)."""
        return self.relin(self.tensor(a, b), a.level, a.scale * b.scale)

    def rotate(self, ct, r):
        out = np.zeros_like(ct.data)
        if self.L.orc_rotate(self.ctx, ct.level, int(r), _p(ct.data), _p(out)):
            raise KeyError("no rotation key for %d" % r)
        return Ct(out, ct.level, ct.scale)

    def rotsum(self, ct, rots):
        """ct + sum_j Rot(ct, r_j) with one shared ModUp and one ModDown
        (hoisted rotations; a single rotation equals add(ct, rotate(ct, r)))."""
        gals = np.array([self.galois_elt(r) for r in rots], np.uint64)
        out = np.zeros_like(ct.data)
        if self.L.orc_rotsum_gal(self.ctx, ct.level, _p(gals), len(gals), _p(ct.data), _p(out)):
            raise KeyError("no rotation key for one of %s" % (list(rots),))
        return Ct(out, ct.level, ct.scale)

    def rotate_gal(self, ct, gal):
        """The automorphism X -> X^gal on both polynomials, then the key switch
        of the second back to s (gal = 2N - 1: slot-wise complex conjugation)."""
        out = np.zeros_like(ct.data)
        if self.L.orc_rotate_gal(self.ctx, ct.level, int(gal), _p(ct.data), _p(out)):
            raise KeyError("no key-switching key for galois element %d" % gal)
        return Ct(out, ct.level, ct.scale)

    def rescale(self, ct):
        lv = ct.level
        if lv < 1:
            raise ValueError("no level left to rescale")
        out = np.zeros((2, lv, self.n), np.uint64)
        self.L.orc_rescale(self.ctx, lv, 2, _p(ct.data), _p(out))
        return Ct(out, lv - 1, ct.scale / float(self.q[lv]))

    def moddrop(self, ct, target):
        if target > ct.level:
            raise ValueError("cannot raise level")
        out = np.zeros((2, target + 1, self.n), np.uint64)
        self.L.orc_moddrop(self.ctx, ct.level, target, 2, _p(ct.data), _p(out))
        return Ct(out, target, ct.scale)

    def cmul_int(self, ct, k, out_scale):
        out = np.zeros_like(ct.data)
        self.L.orc_cmul_int(self.ctx, ct.level, 2, _p(ct.data), int(k), _p(out))
        return Ct(out, ct.level, out_scale)

    def cmul(self, ct, c, const_scale):
        """cMul by real c encoded at scale const_scale; scale_out = scale * const_scale."""
        return self.cmul_int(ct, round_half_away(c * const_scale), ct.scale * const_scale)

    def cadd(self, ct, c):
        out = np.zeros_like(ct.data)
        self.L.orc_cadd_int(self.ctx, ct.level, _p(ct.data), round_half_away(c * ct.scale), _p(out))
        return Ct(out, ct.level, ct.scale)

    def ptadd(self, ct, pt):
        """c0 + m for a plaintext m at the ciphertext's level and scale."""
        if pt.level != ct.level:
            raise ValueError("level mismatch")
        self._check_scales(ct, pt)
        out = ct.data.copy()
        c0 = np.zeros_like(ct.data[0])
        self.L.orc_add(self.ctx, ct.level, 1, _p(np.ascontiguousarray(ct.data[0])), _p(pt.data), _p(c0), 0)
        out[0] = c0
        return Ct(out, ct.level, ct.scale)

    def ptmul(self, ct, pt):
        if pt.level != ct.level:
            raise ValueError("level mismatch")
        out = np.zeros_like(ct.data)
        self.L.orc_ptmul(self.ctx, ct.level, _p(ct.data), _p(pt.data), _p(out))
        return Ct(out, ct.level, ct.scale * pt.scale)
