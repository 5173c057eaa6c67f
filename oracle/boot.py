"""Bootstrapping of the weight ciphertexts (test infrastructure: the oracle).

The paper refreshes W and V every iteration by bootstrapping (Sec. 2.1
"bootstrapping", Sec. 4.3 Step 7; Table 1's "weight-refreshing" time).  This
module restates it for the RNS scheme of ckks.py, step by step and slowly:

    ModRaise -> SubSum -> CoeffToSlot -> EvalMod -> SlotToCoeff

for a ciphertext at level 0 whose slot vector is periodic with period n (W and
V hold the g = n weights in every row of the block, Sec. 2.2).  With
Y = X^(N / 2n) such a message lies in Z[Y]/(Y^(2n) + 1) (up to noise), whose n
slots are the values at xi^(5^j), xi = zeta^(N / 2n):

* ModRaise reads the level-0 words as centred integers modulo every prime of
  the chain: the decryption becomes t = m + e + q0 I with a small integer
  polynomial I (|I| stays small because the secret is sparse).
* SubSum adds the rotations by n, 2n, ..., N/2 - n slots (the automorphisms
  fixing Z[Y]): the trace to Z[Y], G = N / 2n times its Z[Y] part.
* CoeffToSlot applies E^-1 = E^H / n (E_jk = xi^(5^j k), the encoding of the
  subring) through diagonals: slots w_k = (t_k + i t_(k+n)) / (G q0), split
  into real and imaginary parts with the conjugation X -> X^-1 and the
  monomial X^(N/2) (multiplication by i), each scaled into [-1, 1].
* EvalMod takes v -> sin(2 pi v) for |v| <= K + 1/2: the Taylor polynomial of
  cos(2 pi (v - 1/4) / 2^r) in x = v / (K + 1/2), then r double-angle steps
  y -> 2 y^2 - 1.  For v = I + eps with integer I, sin(2 pi v) = sin(2 pi eps)
  ~ 2 pi eps, eps = (m + e) / q0.
* SlotToCoeff applies q0 E / (2 pi Delta) to y_re + i y_im: the slots of m / Delta.

Every constant is built from +, -, *, / in a fixed order (no library cos or
sin): the Taylor coefficients, cos and sin of the phase by their series, and
the powers of zeta from the encoder's table, so an independent implementation
that follows the same definitions forms the same doubles.
"""
import numpy as np

from .ckks import Ct

PI = 3.141592653589793
SUBSUM_RHO = 3  # the trace's rotations are summed in hoisted groups of 2^3 positions


def taylor_cos_sin(b, terms=20):
    """cos b and sin b by their Taylor series, summed in the order k = 0, 1, ..."""
    c = s = 0.0
    term = 1.0  # b^k / k!
    for k in range(2 * terms):
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        term = term * b / (k + 1)
    return c, s


class BootParams:
    """n: slot period; K: bound on |I|; r: double-angle steps; deg: degree of
    the cosine polynomial; delta_out: scale of the result; out_level: its level."""

    def __init__(self, n, K, r, deg, delta_out, out_level):
        self.n, self.K, self.r, self.deg = n, K, r, deg
        self.Kp = K + 0.5
        self.delta_out, self.out_level = float(delta_out), out_level
        nb = n.bit_length() - 1
        self.n1 = 1 << ((nb + 1) // 2)   # baby steps of the diagonal products
        self.n2 = n // self.n1           # giant steps

    def cos_coeffs(self):
        """Taylor coefficients of cos(A x + B), A = 2 pi K' / 2^r, B = -pi / 2^(r+1):
        c_k = A^k / k! * (cos B, -sin B, -cos B, sin B)[k mod 4]."""
        A = 2.0 * PI * self.Kp / float(1 << self.r)
        B = -PI / float(1 << (self.r + 1))
        cb, sb = taylor_cos_sin(B)
        out, a = [], 1.0
        for k in range(self.deg + 1):
            out.append(a * (cb, -sb, -cb, sb)[k % 4])
            a = a * A / (k + 1)
        return out

    def depth(self):
        """levels consumed: CoeffToSlot 1, powers ceil(log2 deg), the coefficients 1,
        the double angles r, SlotToCoeff 1"""
        return 1 + (self.deg - 1).bit_length() + 1 + self.r + 1


def subsum_rotations(N, n):
    """hoisted groups of rotation amounts for the trace: n, 2n, ..., summed over log2(N/2n) doublings"""
    bits = (N // (2 * n)).bit_length() - 1
    out = []
    for e in range(0, bits, SUBSUM_RHO):
        w = min(SUBSUM_RHO, bits - e)
        out.append([n * (m << e) for m in range(1, 1 << w)])
    return out


def key_rotations(he, p):
    """rotation amounts and raw Galois elements the bootstrap needs"""
    rots = {r for grp in subsum_rotations(he.n, p.n) for r in grp}
    rots |= set(range(1, p.n1)) | {g * p.n1 for g in range(1, p.n2)}
    return sorted(rots), [2 * he.n - 1]


def mod_raise(he, ct, level):
    """the level-0 words of ct (modulo q0) as centred integers modulo q_0..q_level"""
    if ct.level != 0:
        ct = he.moddrop(ct, 0)
    q0 = he.q[0]
    out = np.zeros((2, level + 1, he.n), np.uint64)
    for p in range(2):
        c = ct.data[p][0].astype(np.int64)
        c = np.where(c > q0 // 2, c - np.int64(q0), c)
        for j in range(level + 1):
            out[p, j] = (c % np.int64(he.q[j])).astype(np.uint64)
    return Ct(out, level, ct.scale)


def monomial(he, ct, k):
    """ct * X^k in Z[X]/(X^N + 1), exact: coefficient i moves to (i + k) mod 2N,
    negated when that lands in [N, 2N); the slot values are multiplied by
    zeta^(k 5^j), which for k = N/2 is i and for k = 3N/2 is -i"""
    N = he.n
    idx = (np.arange(N) + k) % (2 * N)
    pos, neg = idx % N, idx >= N
    out = np.zeros_like(ct.data)
    for j in range(ct.level + 1):
        q = np.uint64(he.q[j])
        for p in range(2):
            a = ct.data[p][j]
            out[p, j, pos] = np.where(neg & (a != 0), q - a, a)
    return Ct(out, ct.level, ct.scale)


def zeta_powers(he):
    re = np.zeros(2 * he.n)
    im = np.zeros(2 * he.n)
    he.L.orc_get_zeta_table(he.ctx, re.ctypes.data_as(__import__("ctypes").c_void_p),
                            im.ctypes.data_as(__import__("ctypes").c_void_p))
    return re, im


def encoding_matrix(he, n):
    """E[j][k] = xi^(5^j k), xi = zeta^(N / 2n), as (re, im) from the encoder's table"""
    re, im = zeta_powers(he)
    G = he.n // (2 * n)
    twoN = 2 * he.n
    Ere = np.zeros((n, n))
    Eim = np.zeros((n, n))
    p5 = 1
    for j in range(n):
        for k in range(n):
            idx = (G * p5 * k) % twoN
            Ere[j, k], Eim[j, k] = re[idx], im[idx]
        p5 = (p5 * 5) % twoN
    return Ere, Eim


def linear_transform(he, ct, Mre, Mim, pt_scale):
    """sum_r diag_r (.) Rot(ct, r) for the n x n matrix M acting on period-n slot
    vectors, with baby-step/giant-step rotations; plaintexts at pt_scale; the
    product is rescaled once."""
    n = Mre.shape[0]
    nb = n.bit_length() - 1
    n1 = 1 << ((nb + 1) // 2)
    n2 = n // n1
    reps = he.nslots // n
    baby = [ct] + [he.rotate(ct, b) for b in range(1, n1)]
    acc = None
    for g in range(n2):
        inner = None
        for b in range(n1):
            r = g * n1 + b
            # diag_r[k] = M[k][(k + r) mod n], rotated right by g n1: value[k] = diag_r[(k - g n1) mod n]
            ks = (np.arange(n) - g * n1) % n
            vre = Mre[ks, (ks + r) % n]
            vim = Mim[ks, (ks + r) % n]
            z = np.tile(vre, reps) + 1j * np.tile(vim, reps)
            pt = he.encode(z, ct.level, pt_scale)
            term = he.ptmul(baby[b], pt)
            inner = term if inner is None else he.add(inner, term)
        if g:
            inner = he.rotate(inner, g * n1)
        acc = inner if acc is None else he.add(acc, inner)
    return he.rescale(acc)


def coeff_to_slot(he, ct, p):
    """(x_re, x_im): the slots (t_k + i t_(k+n)) / (G q0 K') split into real and
    imaginary parts, at scale q_(top-1)"""
    n, N = p.n, he.n
    G = N // (2 * n)
    Ere, Eim = encoding_matrix(he, n)
    # E^-1 / (2 G q0 K') = conj(E)^T / (2 n G q0 K')
    c = 1.0 / (2.0 * float(n) * float(G) * float(he.q[0]) * p.Kp)
    Mre = Ere.T * c
    Mim = -Eim.T * c
    top = ct.level
    s_x = float(he.q[top - 1])
    u = linear_transform(he, ct, Mre, Mim, float(he.q[top]) * s_x)
    u.scale = s_x
    uc = he.rotate_gal(u, 2 * N - 1)
    x_re = he.add(u, uc)
    x_im = monomial(he, he.sub(u, uc), 3 * N // 2)
    return x_re, x_im


def cmul_to(he, ct, c, target):
    q = float(he.q[ct.level])
    S = (target * q) / ct.scale
    out = he.rescale(he.cmul(ct, c, S))
    out.scale = target
    return out


def eval_mod(he, x, p):
    """sin(2 pi v) for the slots x = v / K' (|v| <= K')"""
    coeffs = p.cos_coeffs()
    deg = p.deg
    pw = {1: x}
    for k in range(2, deg + 1):
        a = 1 << (k.bit_length() - 1)
        if a == k:
            a = k // 2
        u, w = pw[a], pw[k - a]
        if u.level > w.level:
            u = he.moddrop(u, w.level)
        elif w.level > u.level:
            w = he.moddrop(w, u.level)
        pw[k] = he.rescale(he.mul(u, w))
    low = min(c.level for c in pw.values())
    target = float(he.q[low - 1])
    acc = None
    for k in range(1, deg + 1):
        xk = pw[k] if pw[k].level == low else he.moddrop(pw[k], low)
        term = cmul_to(he, xk, coeffs[k], target)
        acc = term if acc is None else he.add(acc, term)
    y = he.cadd(acc, coeffs[0])
    for _ in range(p.r):
        y2 = he.rescale(he.mul(y, y))
        y = he.cadd(he.cmul_int(y2, 2, y2.scale), -1.0)
    return y


def slot_to_coeff(he, y_re, y_im, p):
    """slots of m / Delta_out from y = sin(2 pi v) = 2 pi (m + e) / q0 per coefficient"""
    n, N = p.n, he.n
    y = he.add(y_re, monomial(he, y_im, N // 2))
    Ere, Eim = encoding_matrix(he, n)
    c = float(he.q[0]) / (2.0 * PI * p.delta_out)
    pt_scale = p.delta_out * float(he.q[y.level]) / y.scale
    out = linear_transform(he, y, Ere * c, Eim * c, pt_scale)
    out.scale = p.delta_out
    if out.level > p.out_level:
        out = he.moddrop(out, p.out_level)
    return out


def bootstrap(he, ct, p):
    """level-0 ciphertext of a period-n slot vector at scale delta_out -> the
    same slots at level p.out_level, scale p.delta_out"""
    top = he.max_level
    t = mod_raise(he, ct, top)
    for rots in subsum_rotations(he.n, p.n):
        t = he.rotsum(t, rots)
    x_re, x_im = coeff_to_slot(he, t, p)
    y_re = eval_mod(he, x_re, p)
    y_im = eval_mod(he, x_im, p)
    return slot_to_coeff(he, y_re, y_im, p)
