"""Client precompute and the encrypted quadratic-gradient NAG iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper passages followed (arXiv 2406.13221):
  * Sec. 2.2  -- Z = y * [1 | X] (labels folded into samples, bias column
    first), row-by-row SIMD packing of m x g sub-matrices with m*g = N/2,
    column filter by a mask with ones in column 0, SumColVec-style
    rotate-and-sum.
  * Sec. 3.1  -- quadratic gradient G = Bbar g with
    Bbar_jj = 1 / (eps + sum_i |hbar_ji|) built from the fixed Hessian bound
    -1/4 X^T X (Sec. 4.3 Step 1); NAG with quadratic gradient.
  * Sec. 3.2  -- learning-rate schedule F2(t) = max - (max-min)(t/T)^gamma and
    Algorithm 1 (alpha/eta recurrence, V_temp = W + (1+gamma) G,
    W = (1-eta) V_temp + eta V, V = V_temp).
  * Sec. 3.3  -- full batch over mini-batch-encrypted data; full-batch Bbar from
    the mini-batch Bbar_k by Bbar = 1 / sum_k (1 / Bbar_k).
  * Sec. 4.1  -- degree-3 sigmoid polynomials g8 and g16.
  * Sec. 4.3  -- Steps 4-6 (gradient, quadratic gradient, NAG update) and Step 7
    (refresh; here a decrypt + re-encrypt of W and V stands in for bootstrapping).

Readings where the paper is silent or ambiguous:
  * The multiplier on G is F2(t) itself (the experiment tables quote the learning
    rate as 2 - (t/81)^2.5, i.e. 1 + gamma with gamma running from 1 down to 0);
    Bbar and g are unnormalised sums, so n * Bbar is encrypted and 1/n is applied
    as a public scalar at the end.
  * The circuit of Han et al. that Sec. 2.2 builds on is not given.  Reading:
    row sums by rotate-and-add put ip_r in column 0 (the other columns hold
    partial sums); the column-0 mask M is folded into the plaintext products of
    the sigmoid polynomial, s = (1 - c0) M - c1 (M t) - c3 t^2 (M t), evaluated
    at depth 2 (t^2 and (-c3 M) t in parallel, then their product), which is
    zero outside column 0; s is then replicated across the row by rotate-and-
    add.  This is the same function as masking ip first, with one level less,
    and the replication runs at a lower level.
  * The multiplier on G, F2(t), is applied with the public scalars of the
    update (Algorithm 1: V_temp = W + (1 + gamma) G), together with 1/n.
  * t starts at 0; mini-batches are visited in order 0, 1, 2, ... without shuffling.
  * First-order NAG baseline (Sec. 2.3, the method the paper compares against):
    the same circuit without the Bbar product (Step 8), so one level less; its
    learning rate gamma takes the place of F2(t) (a constant schedule max = min
    = gamma), and V' = W + (1/n) gamma g.
"""
import math

import numpy as np

from .ckks import Ckks, Ct, round_half_away  # noqa: F401

G8 = (0.5, 0.15, -0.0015)     # g8(x) = 0.5 + 0.15 x - 0.0015 x^3 on [-8, 8]
G16 = (0.5, 0.0843, -0.0002)  # g16(x) = 0.5 + 0.0843 x - 0.0002 x^3 on [-16, 16]
EPS = 1e-8

# seed kinds for the per-object encryption seeds
SEED_BLOCK, SEED_BBAR, SEED_W0, SEED_V0, SEED_WREF, SEED_VREF = 1, 2, 3, 4, 5, 6
M64 = (1 << 64) - 1


def obj_seed(enc_seed, kind, index):
    return (enc_seed + (kind << 48) + index) & M64


# ------------------------------------------------------------------ client side
def make_z(X, y):
    """z_ij = y_i x_ij with a leading bias column of ones (Sec. 2.2)."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    return np.concatenate([y[:, None], y[:, None] * X], axis=1)


def pad_cols(f1):
    g = 1
    while g < f1:
        g *= 2
    return g


def bbar_rows(Z, g):
    """Bbar_cc = 1 / (eps + 1/4 sum_k |(Z^T Z)_ck|) for the given rows (Sec. 3.1,
    Sec. 4.3 Step 1); padded columns c >= f+1 get 0."""
    H = Z.T @ Z
    out = np.zeros(g)
    f1 = Z.shape[1]
    out[:f1] = 1.0 / (EPS + 0.25 * np.abs(H).sum(axis=1))
    return out


def bbar_full_from_batches(bbars):
    """Sec. 3.3: Bbar[i][i] = 1 / sum_k (1 / Bbar_k[i][i]) (padded columns stay 0)."""
    B = np.asarray(bbars)
    out = np.zeros(B.shape[1])
    nz = B[0] != 0
    out[nz] = 1.0 / (1.0 / B[:, nz]).sum(axis=0)
    return out


def pack_blocks(Z, g, m):
    """Split Z into m x g blocks, zero padded, row-major into slot vectors."""
    n, f1 = Z.shape
    nb = -(-n // m)
    blocks = np.zeros((nb, m, g))
    for b in range(nb):
        rows = Z[b * m:(b + 1) * m]
        blocks[b, :rows.shape[0], :f1] = rows
    return blocks.reshape(nb, m * g)


def schedule(t, smax=2.0, smin=1.0, T=81.0, power=2.5):
    """F2(t) = max - (max - min) (t / T)^gamma (Sec. 3.2)."""
    return smax - (smax - smin) * (t / T) ** power


def nag_scalars(iters):
    """Algorithm 1: alpha_0 = 0.01, alpha_1 = (1 + sqrt(1 + 4 alpha_0^2)) / 2;
    eta = (1 - alpha_0) / alpha_1 each iteration, then alpha_0 <- alpha_1 and
    alpha_1 <- (1 + sqrt(1 + 4 alpha_0^2)) / 2."""
    a0 = 0.01
    a1 = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a0 * a0))
    etas = []
    for _ in range(iters):
        etas.append((1.0 - a0) / a1)
        a0 = a1
        a1 = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a0 * a0))
    return etas


class TrainData:
    """Client-side data for one training job (Sec. 4.3 Steps 1-2)."""

    def __init__(self, X, y, g, m, batch_rows):
        Z = make_z(X, y)
        self.n, self.f1 = Z.shape
        self.g, self.m = g, m
        self.blocks = pack_blocks(Z, g, m)
        self.batch_rows = batch_rows
        self.blocks_per_batch = batch_rows // m
        self.nbatch = -(-self.n // batch_rows)
        self.bbar_k = np.array([bbar_rows(Z[k * batch_rows:(k + 1) * batch_rows], g)
                                for k in range(self.nbatch)])
        self.n_k = np.array([min(batch_rows, self.n - k * batch_rows) for k in range(self.nbatch)])
        self.bbar_full = bbar_full_from_batches(self.bbar_k)
        self.Z = Z


# ------------------------------------------------------------------ encrypted iteration
DEPTH = 6  # levels one iteration consumes
DEPTH_FIRST_ORDER = 5  # without the Bbar product of Step 8


def rot_groups(nbits, step, rho):
    """Rotation amounts of a rotate-and-sum over 2^nbits positions spaced `step`
    slots apart, taken 2^rho positions at a time: group e (e = 0, rho, 2 rho,
    ...) of width w = min(rho, nbits - e) adds the rotations by m 2^e step for
    0 < m < 2^w.  After the groups up to e, slot c holds the sum of the
    2^(e + w) slots c, c + step, c + 2 step, ... (rho = 1: the log-step sum of
    Sec. 2.2, one rotation per step)."""
    out = []
    for e in range(0, nbits, rho):
        w = min(rho, nbits - e)
        out.append([step * (m << e) for m in range(1, 1 << w)])
    return out


class Circuit:
    """The encrypted QG-NAG iteration on one parameter set.

    Levels: fresh inputs sit at level L (default: the iteration depth, 6, so the
    iteration ends at level 0; any higher primes of the chain stay unused); the
    iteration consumes 6 levels and ends at level L - 6.  With first_order=True
    the circuit is the first-order NAG baseline: no Bbar product, depth 5."""

    def __init__(self, he: Ckks, g, m, scale, poly=G8, start_level=None, first_order=False, rot_radix_log=3):
        self.he, self.g, self.m, self.scale, self.poly = he, g, m, float(scale), poly
        self.first_order = first_order
        self.rho = rot_radix_log
        depth = DEPTH_FIRST_ORDER if first_order else DEPTH
        if g * m != he.nslots:
            raise ValueError("m * g must equal N/2")
        self.L = min(depth, he.max_level) if start_level is None else start_level
        if self.L < depth or self.L > he.max_level:
            raise ValueError("the iteration needs %d levels" % depth)
        self.lg, self.lm = int(math.log2(g)), int(math.log2(m))
        c0, c1, c3 = poly
        mask = np.zeros(he.nslots)
        mask[::g] = 1.0
        # the scale chain of Steps 1-5 (fresh Z and W at `scale`), for the
        # masked polynomial plaintexts
        q = [float(x) for x in he.q]
        L = self.L
        t_scale = scale * scale / q[L]                       # Step 1
        sq_scale = t_scale * t_scale / q[L - 1]              # t^2
        c3_scale = t_scale * scale / q[L - 1]                # (-c3 M) t, plaintext at `scale`
        self.s_scale = sq_scale * c3_scale / q[L - 2]        # the cube and s
        self.p3 = he.encode(-c3 * mask, L - 1, scale)
        self.p1 = he.encode(-c1 * mask, L - 1, self.s_scale * q[L - 1] / t_scale)  # rescales to s_scale
        self.p0 = he.encode((1.0 - c0) * mask, L - 3, self.s_scale)

    def groups(self, nbits, step):
        return rot_groups(nbits, step, self.rho)

    def rotsum(self, ct, nbits, step):
        for rots in self.groups(nbits, step):
            ct = self.he.rotsum(ct, rots)
        return ct

    def rotations(self):
        rs = []
        for grp in self.groups(self.lg, 1) + self.groups(self.lg, -1) + self.groups(self.lm, self.g):
            rs += grp
        return rs

    def cmul_to(self, ct, c, target):
        """cMul by c at the constant scale that makes the rescaled result carry
        scale `target`; returns the rescaled ciphertext with that scale."""
        q = float(self.he.q[ct.level])
        S = (target * q) / ct.scale
        out = self.he.rescale(self.he.cmul(ct, c, S))
        out.scale = target
        return out

    def block_grad(self, Z, W):
        """Steps 1-6 for one data block: slotwise s_r * z_rc, s = 1 - g(z_r . w)."""
        he = self.he
        # Step 1: z_rc * w_c
        t = he.rescale(he.mul(Z, W))
        # Step 2: row sums into column 0
        t = self.rotsum(t, self.lg, 1)
        # Steps 3 and 5: s = (1 - c0) M - c1 (M t) - c3 t^2 (M t), zero outside column 0
        sq = he.rescale(he.mul(t, t))
        c3t = he.rescale(he.ptmul(t, self.p3))
        cube = he.rescale(he.mul(sq, c3t))
        lin = he.rescale(he.ptmul(t, self.p1))
        lin.scale = cube.scale  # p1's scale was chosen for this
        s = he.ptadd(he.add(cube, he.moddrop(lin, cube.level)), self.p0)
        # Step 4: replicate s_r across the row
        s = self.rotsum(s, self.lg, -1)
        # Step 6: s_r * z_rc
        return he.rescale(he.mul(s, he.moddrop(Z, s.level)))

    def finish(self, acc, B, W, V, alpha, eta, inv_n):
        """Steps 7-9 on the accumulated gradient ciphertext; alpha = F2(t)."""
        he = self.he
        # Step 7: column sums, every row gets g_c
        acc = self.rotsum(acc, self.lm, self.g)
        # Step 8: n Bbar_c g_c (the first-order baseline uses g_c itself)
        nG = acc if B is None else he.rescale(he.mul(acc, he.moddrop(B, acc.level)))
        # Step 9: V' = W + G, W' = (1 - eta) V' + eta V
        lv = nG.level
        tgt = W.scale
        G = self.cmul_to(nG, alpha * inv_n, tgt)
        Vn = he.add(he.moddrop(W, lv - 1), G)
        Wn = he.add(he.add(self.cmul_to(he.moddrop(W, lv), 1.0 - eta, tgt),
                           self.cmul_to(he.moddrop(V, lv), eta, tgt)),
                    self.cmul_to(nG, (1.0 - eta) * alpha * inv_n, tgt))
        return Wn, Vn

    def iteration(self, Zs, B, W, V, alpha, eta, inv_n):
        acc = None
        for Z in Zs:
            gct = self.block_grad(Z, W)
            acc = gct if acc is None else he_add(self.he, acc, gct)
        return self.finish(acc, B, W, V, alpha, eta, inv_n)

    def refresh(self, ct, seed):
        """Step 7 stand-in: decrypt, keep the real part of the slots, re-encode at
        the start level with the initial scale, encrypt with fresh randomness."""
        he = self.he
        z = he.decode(he.decrypt(ct))
        return he.encrypt(he.encode(z.real, self.L, self.scale), seed)


def he_add(he, a, b):
    return he.add(a, b)


def train(he, circ, data, iters, enc_seed, mode="full", sched=(2.0, 1.0, 81.0, 2.5),
          block_ids=None, return_trace=False):
    """Encrypt the job (Sec. 4.3 Step 2), run `iters` iterations, decrypt W.

    Returns the decrypted slot vector of W (real parts), reshaped [m, g]."""
    L, scale = circ.L, circ.scale
    nb = data.blocks.shape[0]
    bids = range(nb) if block_ids is None else block_ids
    Zct = {b: he.encrypt(he.encode(data.blocks[b], L, scale), obj_seed(enc_seed, SEED_BLOCK, b))
           for b in bids}
    if mode == "full":
        bvec = [np.tile(data.n * data.bbar_full, circ.m)]
        inv_ns = [1.0 / data.n]
    else:
        bvec = [np.tile(float(data.n_k[k]) * data.bbar_k[k], circ.m) for k in range(data.nbatch)]
        inv_ns = [1.0 / float(data.n_k[k]) for k in range(data.nbatch)]
    Bct = ([None] * len(bvec) if circ.first_order else
           [he.encrypt(he.encode(v, L, scale), obj_seed(enc_seed, SEED_BBAR, k)) for k, v in enumerate(bvec)])
    zero = np.zeros(he.nslots)
    W = he.encrypt(he.encode(zero, L, scale), obj_seed(enc_seed, SEED_W0, 0))
    V = he.encrypt(he.encode(zero, L, scale), obj_seed(enc_seed, SEED_V0, 0))
    etas = nag_scalars(iters)
    trace = []
    for t in range(iters):
        alpha = schedule(t, *sched)
        if mode == "full":
            blocks, k = [Zct[b] for b in bids], 0
        else:
            k = t % data.nbatch
            bpb = data.blocks_per_batch
            blocks = [Zct[b] for b in range(k * bpb, min((k + 1) * bpb, nb))]
        Wn, Vn = circ.iteration(blocks, Bct[k], W, V, alpha, etas[t], inv_ns[k])
        W = circ.refresh(Wn, obj_seed(enc_seed, SEED_WREF, t))
        V = circ.refresh(Vn, obj_seed(enc_seed, SEED_VREF, t))
        if return_trace:
            trace.append((Wn, Vn, W, V))
    w = he.decode(he.decrypt(W)).real.reshape(circ.m, circ.g)
    return (w, trace) if return_trace else w
