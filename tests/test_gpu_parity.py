"""Parity of the CUDA path with the CPU oracle, element by element.

Ciphertext, plaintext and transform words must be identical (integer work is
bit-exact); decoded doubles must be identical too, because both sides run the
same FP64 butterfly network without contraction.  Inputs are seeded and
synthetic.  All calls go through the C ABI (binding.py).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import qgnag  # noqa: E402
from oracle.ckks import Ckks, Ct as OCt  # noqa: E402
from paper_2406_13221_gb300 import binding, build, synth  # noqa: E402

build.build()
D = 2.0 ** 40


def bitrev(x, bits):
    return int(format(x, "0%db" % bits)[::-1], 2)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def from_dev(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("logn", [10, 11, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("nlimbs", [1, 3, 37])
def test_ntt_matches_oracle(logn, nlimbs):
    nq = 3
    ctx = binding.Context(logn, nq)
    he = Ckks(logn, nq)
    assert ctx.primes == he.primes
    n = 1 << logn
    rng = np.random.default_rng(logn * 100 + nlimbs)
    period = nq + 1
    prime_of = [(i * 3 + 1) % period for i in range(period)]
    data = np.zeros((nlimbs, n), np.uint64)
    for i in range(nlimbs):
        q = he.primes[prime_of[i % period]]
        data[i] = rng.integers(0, q, n, dtype=np.uint64)
    dev = to_dev(data)
    ctx.ntt_forward(dev.data_ptr(), nlimbs, prime_of)
    got = from_dev(dev).reshape(nlimbs, n)
    perm = np.array([bitrev(p, logn) for p in range(n)])
    check = range(nlimbs) if n <= 8192 else [0, nlimbs - 1]
    for i in check:
        ref = data[i].copy()
        he.L.orc_ntt(he.ctx, prime_of[i % period], ref.ctypes.data_as(__import__("ctypes").c_void_p))
        assert np.array_equal(got[i], ref[perm]), "limb %d" % i
    ctx.ntt_inverse(dev.data_ptr(), nlimbs, prime_of)
    assert np.array_equal(from_dev(dev).reshape(nlimbs, n), data)


# rotations of the tests, plus those of the 16 x 256 training circuit with its
# rotate-and-sum steps in hoisted groups of 2, 4 and 8 positions
PAIR_ROTATIONS = [1, 2, 4, 8, -1, -2, -4, -8, 3, 100, -77] + [16 << k for k in range(8)]
PAIR_ROTATIONS = sorted(set(PAIR_ROTATIONS) | {
    r for rho in (1, 2, 3) for n, st in ((4, 1), (4, -1), (8, 16)) for rots in qgnag.rot_groups(n, st, rho) for r in rots})


@pytest.fixture(scope="module")
def pair():
    """GPU context and oracle with identical parameters and keys (N = 2^13)."""
    logn, nq = 13, 9
    ctx = binding.Context(logn, nq)
    he = Ckks(logn, nq)
    ctx.keygen(2, PAIR_ROTATIONS)
    he.keygen(2, PAIR_ROTATIONS)
    return ctx, he


def rand_slots(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, n) + 1j * rng.uniform(-scale, scale, n)


def test_secret_key_and_encode_bitwise(pair):
    ctx, he = pair
    z = rand_slots(ctx.nslots, 1, 3.0)
    for level, scale in ((8, D), (3, 2.0 ** 35), (0, float(he.q[0]) / 7)):
        words, lv, sc = ctx.encode(z, level, scale).export()
        ref = he.encode(z, level, scale)
        assert lv == level and sc == scale
        assert np.array_equal(words, ref.data)


def test_ragged_and_empty_slot_vectors(pair):
    ctx, he = pair
    for k in (0, 1, 1000, ctx.nslots):
        z = rand_slots(k, 2) if k else np.zeros(0, complex)
        words, _, _ = ctx.encode(z, 2, D).export()
        assert np.array_equal(words, he.encode(z, 2, D).data)


def test_decode_bitwise(pair):
    ctx, he = pair
    z = rand_slots(ctx.nslots, 3)
    pt = ctx.encode(z, 4, D)
    words, lv, sc = pt.export()
    from oracle.ckks import Pt as OPt
    ref = he.decode(OPt(words, lv, sc))
    got = ctx.decode(pt)
    assert np.array_equal(got.real.view(np.uint64), ref.real.view(np.uint64))
    assert np.array_equal(got.imag.view(np.uint64), ref.imag.view(np.uint64))


def test_encrypt_decrypt_bitwise(pair):
    ctx, he = pair
    z = rand_slots(ctx.nslots, 4)
    for level in (8, 5):
        ct = ctx.encrypt(ctx.encode(z, level, D), 11)
        ref = he.encrypt(he.encode(z, level, D), 11)
        assert np.array_equal(ct.export(), ref.data)
        words, _, _ = ctx.decrypt(ct).export()
        assert np.array_equal(words, he.decrypt(ref).data)


def enc_pair(ctx, he, z, seed, level=8, scale=D):
    ref = he.encrypt(he.encode(z, level, scale), seed)
    return ctx.import_ct(ref.data, level, scale), ref


def test_add_sub_mul_rescale_bitwise(pair):
    ctx, he = pair
    a, ra = enc_pair(ctx, he, rand_slots(ctx.nslots, 5), 21)
    b, rb = enc_pair(ctx, he, rand_slots(ctx.nslots, 6), 22)
    assert np.array_equal(ctx.add(a, b).export(), he.add(ra, rb).data)
    assert np.array_equal(ctx.sub(a, b).export(), he.sub(ra, rb).data)
    m = ctx.mul(a, b)
    rm = he.mul(ra, rb)
    assert np.array_equal(m.export(), rm.data)
    assert m.scale == rm.scale
    r = ctx.rescale(m)
    rr = he.rescale(rm)
    assert np.array_equal(r.export(), rr.data)
    assert (r.level, r.scale) == (rr.level, rr.scale)
    # a chain down to level 1 exercises every limb count of the key switch
    x, rx = r, rr
    while x.level > 1:
        y = ctx.moddrop(b, x.level)
        x = ctx.rescale(ctx.mul(x, y))
        rx = he.rescale(he.mul(rx, he.moddrop(rb, rx.level)))
        assert np.array_equal(x.export(), rx.data), x.level


@pytest.mark.parametrize("r", [1, -1, 3, 100, -77, 16, 2048])
def test_rotation_bitwise(pair, r):
    ctx, he = pair
    a, ra = enc_pair(ctx, he, rand_slots(ctx.nslots, 7), 23)
    assert np.array_equal(ctx.rotate(a, r).export(), he.rotate(ra, r).data)
    a3 = ctx.moddrop(a, 3)
    assert np.array_equal(ctx.rotate(a3, r).export(), he.rotate(he.moddrop(ra, 3), r).data)


@pytest.mark.parametrize("rots", [[3], [1, 2, 3], [-4, -8, -12], [16, 32, 48, 64, 80, 96, 112], [1, -1]])
def test_hoisted_rotation_sum_bitwise(pair, rots):
    """he_rotsum (one ModUp and one ModDown for all the rotations) equals the
    oracle's hoisted rotation sum at levels 8 and 3; one rotation equals
    add(a, rotate(a, r))."""
    ctx, he = pair
    a, ra = enc_pair(ctx, he, rand_slots(ctx.nslots, 31), 33)
    for lv in (8, 3):
        x, rx = (a, ra) if lv == 8 else (ctx.moddrop(a, lv), he.moddrop(ra, lv))
        got = ctx.rotsum(x, rots).export()
        assert np.array_equal(got, he.rotsum(rx, rots).data), lv
        if len(rots) == 1:
            assert np.array_equal(got, ctx.add(x, ctx.rotate(x, rots[0])).export())
    with pytest.raises(binding.HeError) as e:
        ctx.rotsum(a, [1, 9])  # no key for 9
    assert e.value.code == binding.HE_EKEY
    with pytest.raises(binding.HeError):
        ctx.rotsum(a, list(range(1, 9)))  # more than 7 rotations


def test_batched_mul_rescale_rotate_bitwise(pair):
    """he_mul_relin_batch, he_rescale_batch and he_rotate_batch on five device
    ciphertexts equal the oracle's Mul, Rescale and Rotate of every item; the
    calls refuse an output that overlaps the input, a missing key and a
    rescale at level 0."""
    ctx, he = pair
    n, level, batch = ctx.n, 8, 5
    A = [enc_pair(ctx, he, rand_slots(ctx.nslots, 70 + i), 80 + i)[1] for i in range(batch)]
    B = [enc_pair(ctx, he, rand_slots(ctx.nslots, 90 + i), 100 + i)[1] for i in range(batch)]
    primes = list(range(level + 1))

    def dev(cts):
        t = torch.from_numpy(np.stack([c.data for c in cts]).reshape(-1).view(np.int64)).cuda()
        ctx.ntt_forward(t.data_ptr(), batch * 2 * (level + 1), primes)
        return t

    def host(t, lv):
        ctx.ntt_inverse(t.data_ptr(), batch * 2 * (lv + 1), list(range(lv + 1)))
        torch.cuda.synchronize()
        return t.cpu().numpy().view(np.uint64).reshape(batch, 2, lv + 1, n)

    da, db = dev(A), dev(B)
    prod = torch.zeros_like(da)
    ctx.mul_relin_batch(da.data_ptr(), db.data_ptr(), prod.data_ptr(), batch, level)
    resc = torch.zeros(batch * 2 * level * n, dtype=torch.int64, device="cuda")
    ctx.rescale_batch(prod.data_ptr(), resc.data_ptr(), batch, level)
    rot = torch.zeros_like(da)
    ctx.rotate_batch(da.data_ptr(), rot.data_ptr(), batch, level, 4)
    got_p, got_r, got_s = host(prod, level), host(rot, level), host(resc, level - 1)
    for i in range(batch):
        ref = he.mul(A[i], B[i])
        assert np.array_equal(got_p[i], ref.data), i
        assert np.array_equal(got_s[i], he.rescale(ref).data), i
        assert np.array_equal(got_r[i], he.rotate(A[i], 4).data), i
    for call in (lambda: ctx.rescale_batch(da.data_ptr(), da.data_ptr(), batch, level),
                 lambda: ctx.mul_relin_batch(da.data_ptr(), db.data_ptr(), db.data_ptr(), batch, level)):
        with pytest.raises(binding.HeError) as e:
            call()
        assert e.value.code == binding.HE_EINVAL
    with pytest.raises(binding.HeError) as e:
        ctx.rotate_batch(da.data_ptr(), rot.data_ptr(), batch, level, 9)  # no key for 9
    assert e.value.code == binding.HE_EKEY
    with pytest.raises(binding.HeError) as e:
        ctx.rescale_batch(da.data_ptr(), resc.data_ptr(), batch, 0)
    assert e.value.code == binding.HE_ELEVEL


@pytest.mark.parametrize("rho", [1, 2])
def test_iteration_bitwise_other_rotation_radix(small_job_inputs, rho):
    """The iteration with its rotate-and-sum steps in hoisted groups of 2 (the
    plain log-step sum) and of 4 positions equals the oracle's circuit with the
    same grouping."""
    ctx, he, data, _ = small_job_inputs
    L = 6
    circ = qgnag.Circuit(he, 16, 256, D, start_level=L, rot_radix_log=rho)
    Z = [he.encrypt(he.encode(data.blocks[b], L, D), 400 + b) for b in range(data.blocks.shape[0])]
    B = he.encrypt(he.encode(np.tile(data.n * data.bbar_full, circ.m), L, D), 410)
    rng = np.random.default_rng(13)
    w0 = np.tile(np.r_[rng.uniform(-0.5, 0.5, data.f1), np.zeros(16 - data.f1)], circ.m)
    W = he.encrypt(he.encode(w0, L, D), 411)
    V = he.encrypt(he.encode(0.5 * w0, L, D), 412)
    alpha, eta = qgnag.schedule(2), qgnag.nag_scalars(3)[2]
    Wn, Vn = circ.iteration(Z, B, W, V, alpha, eta, 1.0 / data.n)
    g = lambda c: ctx.import_ct(c.data, c.level, c.scale)  # noqa: E731
    ctx.set_rotation_radix(rho)
    try:
        gW, gV = binding.lr_iteration(ctx, [g(z) for z in Z], g(B), g(W), g(V), 16, 256, alpha, eta,
                                      1.0 / data.n, qgnag.G8)
    finally:
        ctx.set_rotation_radix(3)
    assert np.array_equal(gW.export(), Wn.data)
    assert np.array_equal(gV.export(), Vn.data)
    with pytest.raises(binding.HeError):
        ctx.set_rotation_radix(4)


def test_constants_and_plaintext_product_bitwise(pair):
    ctx, he = pair
    a, ra = enc_pair(ctx, he, rand_slots(ctx.nslots, 8), 24)
    for c, s in ((-0.37, D), (0.0015 * 2, D), (1e-6, float(he.q[8]))):
        x = ctx.cmul(a, c, s)
        rx = he.cmul(ra, c, s)
        assert np.array_equal(x.export(), rx.data)
        assert x.scale == rx.scale
    assert np.array_equal(ctx.cadd(a, 0.625).export(), he.cadd(ra, 0.625).data)
    assert np.array_equal(ctx.cadd(a, -3.25).export(), he.cadd(ra, -3.25).data)
    z = rand_slots(ctx.nslots, 9)
    p = ctx.encode(z, 8, float(he.q[8]))
    rp = he.encode(z, 8, float(he.q[8]))
    assert np.array_equal(ctx.ptmul(a, p).export(), he.ptmul(ra, rp).data)


def test_batched_keyswitch_bitwise(pair):
    """he_keyswitch_batch on 5 polynomials (ragged batch) equals the oracle's key switch."""
    ctx, he = pair
    level, batch = 6, 5
    rng = np.random.default_rng(10)
    n = ctx.n
    polys = np.zeros((batch, level + 1, n), np.uint64)
    for b in range(batch):
        for j in range(level + 1):
            polys[b, j] = rng.integers(0, he.q[j], n, dtype=np.uint64)
    gal = he.galois_elt(3)
    dev = to_dev(polys)
    ctx.ntt_forward(dev.data_ptr(), batch * (level + 1), list(range(level + 1)))
    out = torch.zeros(batch * 2 * (level + 1) * n, dtype=torch.int64, device="cuda")
    ctx.keyswitch_batch(dev.data_ptr(), out.data_ptr(), batch, level, gal)
    ctx.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    got = from_dev(out).reshape(batch, 2, level + 1, n)
    for b in range(batch):
        assert np.array_equal(got[b], he.keyswitch(level, gal, polys[b]))


def test_autotune_table_and_parity(pair, tmp_path):
    """he_autotune measures every level once and writes its table (wave, tile
    variant and hoisted inner-product form per limb count); a second context
    with the same parameters loads the table without measuring; key switches of
    more than one wave with the chosen waves and tiles, and a hoisted sum with
    the chosen form, equal the oracle's."""
    _, he = pair
    path = tmp_path / "ks_wave.txt"
    ctx = binding.Context(13, 9)
    ctx.keygen(2, [3])
    assert ctx.autotune(str(path), items=40) == 9
    lines = path.read_text().splitlines()
    assert lines[0] == "he_lr ks-wave table v3" and lines[1].startswith("key ")
    rows = [ln.split() for ln in lines[2:]]
    assert all(len(f) == 12 and f[8] == "hoist" for f in rows)
    waves = {int(f[1]): int(f[3]) for f in rows}
    tiles = {int(f[1]): int(f[5]) for f in rows}
    forms = {int(f[1]): int(f[9]) for f in rows}
    assert sorted(waves) == list(range(1, 10))
    assert set(waves.values()) <= {16, 32}  # the candidates up to 40 items
    assert set(tiles.values()) <= {0, 1, 2, 3}
    assert set(forms.values()) <= {0, 1}
    # the tensor-core form applies from 2 limbs (a 40-bit target) to 7 (7 x 7 <= 51 pairs)
    assert forms[1] == 0 and forms[8] == 0 and forms[9] == 0
    assert all(float(f[11]) > 0 for f in rows if 2 <= int(f[1]) <= 7)
    assert [ctx.ks_wave(lv) for lv in range(9)] == [waves[nl] for nl in range(1, 10)]
    assert [ctx.ks_tile(lv) for lv in range(9)] == [tiles[nl] for nl in range(1, 10)]
    assert [ctx.hoist_form(lv) for lv in range(9)] == [forms[nl] for nl in range(1, 10)]
    ctx2 = binding.Context(13, 9)
    ctx2.keygen(2, [3])
    assert ctx2.autotune(str(path), items=40) == 0
    assert [ctx2.ks_wave(lv) for lv in range(9)] == [waves[nl] for nl in range(1, 10)]
    assert [ctx2.ks_tile(lv) for lv in range(9)] == [tiles[nl] for nl in range(1, 10)]
    assert [ctx2.hoist_form(lv) for lv in range(9)] == [forms[nl] for nl in range(1, 10)]
    ctx2.keygen(2, PAIR_ROTATIONS)
    a, ra = enc_pair(ctx2, he, rand_slots(ctx2.nslots, 44), 45, level=5)
    assert np.array_equal(ctx2.rotsum(a, [1, 2, 3]).export(), he.rotsum(ra, [1, 2, 3]).data)
    level, batch = 5, 40
    rng = np.random.default_rng(14)
    n = ctx2.n
    polys = np.stack([np.stack([rng.integers(0, he.q[j], n, dtype=np.uint64) for j in range(level + 1)])
                      for _ in range(batch)])
    gal = he.galois_elt(3)
    dev = to_dev(polys)
    ctx2.ntt_forward(dev.data_ptr(), batch * (level + 1), list(range(level + 1)))
    out = torch.zeros(batch * 2 * (level + 1) * n, dtype=torch.int64, device="cuda")
    ctx2.keyswitch_batch(dev.data_ptr(), out.data_ptr(), batch, level, gal)
    ctx2.ntt_inverse(out.data_ptr(), batch * 2 * (level + 1), list(range(level + 1)))
    got = from_dev(out).reshape(batch, 2, level + 1, n)
    for b in (0, 17, batch - 1):  # first wave, a later wave, the ragged last one
        assert np.array_equal(got[b], he.keyswitch(level, gal, polys[b]))


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_every_tile_variant_bitwise(pair, tile):
    """Each tile variant of the key-switch kernels (narrower column CTAs, fewer
    rows per row CTA, both) gives the oracle's words: a batched key switch
    with a rescale, and a hoisted rotation sum."""
    ctx, he = pair
    ctx.set_ks_tile(tile)
    try:
        a, ra = enc_pair(ctx, he, rand_slots(ctx.nslots, 60 + tile), 61)
        b, rb = enc_pair(ctx, he, rand_slots(ctx.nslots, 62 + tile), 63)
        assert np.array_equal(ctx.rescale(ctx.mul(a, b)).export(), he.rescale(he.mul(ra, rb)).data)
        assert np.array_equal(ctx.rotsum(a, [1, 2, 3]).export(), he.rotsum(ra, [1, 2, 3]).data)
    finally:
        ctx.set_ks_tile(-1)
    with pytest.raises(binding.HeError):
        ctx.set_ks_tile(4)


def test_errors_are_reported(pair):
    ctx, he = pair
    a, _ = enc_pair(ctx, he, rand_slots(ctx.nslots, 11), 25)
    b = ctx.cmul(a, 1.0, 3.0)  # scale 3 * 2^40
    with pytest.raises(binding.HeError) as e:
        ctx.add(a, b)
    assert e.value.code == binding.HE_ESCALE
    with pytest.raises(binding.HeError) as e:
        ctx.rotate(a, 9)  # no key for 9
    assert e.value.code == binding.HE_EKEY
    low = ctx.moddrop(a, 0)
    with pytest.raises(binding.HeError) as e:
        ctx.rescale(low)
    assert e.value.code == binding.HE_ELEVEL
    with pytest.raises(binding.HeError) as e:
        ctx.add(a, low)
    assert e.value.code == binding.HE_ELEVEL
    # imported words must be reduced modulo their limb's prime
    lv, sc = a.info()
    words = a.export()
    bad = words.copy()
    bad[1, lv, 7] = ctx.primes[lv]
    with pytest.raises(binding.HeError) as e:
        ctx.import_ct(bad, lv, sc)
    assert e.value.code == binding.HE_EINVAL
    assert np.array_equal(ctx.import_ct(words, lv, sc).export(), words)


# ------------------------------------------------------------------ the iteration
@pytest.fixture(scope="module")
def small_job_inputs(pair):
    ctx, he = pair
    X, y = synth.small()
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, D)
    return ctx, he, data, circ


@pytest.mark.parametrize("L", [8, 6])
def test_iteration_bitwise(small_job_inputs, L):
    ctx, he, data, _ = small_job_inputs
    circ = qgnag.Circuit(he, 16, 256, D, start_level=L)
    Z = [he.encrypt(he.encode(data.blocks[b], L, D), 100 + b) for b in range(data.blocks.shape[0])]
    B = he.encrypt(he.encode(np.tile(data.n * data.bbar_full, circ.m), L, D), 200)
    rng = np.random.default_rng(12)
    w0 = np.tile(np.r_[rng.uniform(-0.5, 0.5, data.f1), np.zeros(16 - data.f1)], circ.m)
    v0 = np.tile(np.r_[rng.uniform(-0.5, 0.5, data.f1), np.zeros(16 - data.f1)], circ.m)
    W = he.encrypt(he.encode(w0, L, D), 201)
    V = he.encrypt(he.encode(v0, L, D), 202)
    alpha, eta = qgnag.schedule(1), qgnag.nag_scalars(2)[1]
    Wn, Vn = circ.iteration(Z, B, W, V, alpha, eta, 1.0 / data.n)
    g = lambda c: ctx.import_ct(c.data, c.level, c.scale)  # noqa: E731
    gW, gV = binding.lr_iteration(ctx, [g(z) for z in Z], g(B), g(W), g(V), 16, 256, alpha, eta,
                                  1.0 / data.n, qgnag.G8)
    assert (gW.level, gW.scale) == (Wn.level, Wn.scale)
    assert np.array_equal(gW.export(), Wn.data)
    assert np.array_equal(gV.export(), Vn.data)
    # refresh of both
    for x, rx, seed in ((gW, Wn, 301), (gV, Vn, 302)):
        assert np.array_equal(ctx.refresh(x, circ.L, D, seed).export(), circ.refresh(rx, seed).data)


@pytest.mark.parametrize("graph", [False, True])
def test_job_step_bitwise_and_weights(small_job_inputs, graph):
    ctx, he, data, circ = small_job_inputs
    X, y = synth.small()
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=3, key_seed=2)
    job.set_graph(graph)
    st = job.stats()
    assert (st.n_blocks, st.g, st.m) == (4, 16, 256)
    L = circ.L
    assert L == 6
    # encrypted data blocks equal the oracle's encryption of the same packing
    for b in range(4):
        ref = he.encrypt(he.encode(data.blocks[b], L, D), qgnag.obj_seed(3, qgnag.SEED_BLOCK, b))
        assert np.array_equal(job.input(0, b).export(), ref.data)
    Bg = job.input(1, 0)
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(4)]
    B = OCt(Bg.export(), L, D)
    (Ww, _, _), (Vw, _, _) = job.state_words()
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    etas = qgnag.nag_scalars(2)
    for t in range(2):
        job.step(t)
        Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(t), etas[t], 1.0 / data.n)
        W = circ.refresh(Wn, qgnag.obj_seed(3, qgnag.SEED_WREF, t))
        V = circ.refresh(Vn, qgnag.obj_seed(3, qgnag.SEED_VREF, t))
        (Ww, _, _), (Vw, _, _) = job.state_words()
        assert np.array_equal(Ww, W.data), t
        assert np.array_equal(Vw, V.data), t
    from oracle import plain
    wp = plain.train(data, 2)
    for row in (0, 255):
        assert np.abs(job.weights(row) - wp).max() < 1e-3


def test_first_order_job_bitwise(pair):
    """The first-order NAG baseline (no Bbar product, fresh ciphertexts at level
    5): job state word for word against the oracle's first-order circuit, the
    cloud-only iteration with no Bbar likewise, weights against the FP64 twin."""
    ctx, he = pair
    X, y = synth.small(seed=12, n=1024, f=15)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, D, first_order=True)  # its rotations are among the fixture's keys
    job = binding.Job(ctx, X, y, binding.FULL_BATCH | binding.FIRST_ORDER, 1024, binding.G8, 40.0, enc_seed=5,
                      key_seed=2)
    L = circ.L
    assert L == 5
    with pytest.raises(binding.HeError):
        job.input(1, 0)  # no Bbar ciphertext in a first-order job
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(4)]
    (Ww, lw, _), (Vw, _, _) = job.state_words()
    assert lw == L
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    sched = (1.0, 1.0, 81.0, 2.5)
    etas = qgnag.nag_scalars(2)
    for t in range(2):
        if t == 1:  # the cloud-only entry point on the same inputs
            imp = lambda c: ctx.import_ct(c.data, c.level, c.scale)  # noqa: E731
            gW, gV = binding.lr_iteration(ctx, [imp(z) for z in Z], None, imp(W), imp(V), 16, 256,
                                          qgnag.schedule(t, *sched), etas[t], 1.0 / data.n, qgnag.G8)
        job.step(t, sched)
        Wn, Vn = circ.iteration(Z, None, W, V, qgnag.schedule(t, *sched), etas[t], 1.0 / data.n)
        assert Wn.level == 0
        if t == 1:
            assert np.array_equal(gW.export(), Wn.data) and np.array_equal(gV.export(), Vn.data)
        W = circ.refresh(Wn, qgnag.obj_seed(5, qgnag.SEED_WREF, t))
        V = circ.refresh(Vn, qgnag.obj_seed(5, qgnag.SEED_VREF, t))
        (Ww, _, _), (Vw, _, _) = job.state_words()
        assert np.array_equal(Ww, W.data), t
        assert np.array_equal(Vw, V.data), t
    from oracle import plain
    wp = plain.train(data, 2, sched=sched, first_order=True)
    assert np.abs(job.weights(0) - wp).max() < 1e-3


def test_lr_train_whole_job(pair):
    """he_lr_train (job creation, two full-batch iterations and the decryption
    in one call) returns the weights the oracle's whole training run decrypts,
    bit for bit, and they lie within 1e-3 of the FP64 twin."""
    ctx, he = pair
    X, y = synth.small(seed=13, n=1024, f=15)
    w, st = binding.lr_train(ctx, X, y, 2, enc_seed=17, key_seed=2)
    assert (st.n_blocks, st.g, st.m) == (4, 16, 256)
    assert st.keyswitches > 0
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, D)
    he.keygen(2, sorted(set(PAIR_ROTATIONS) | set(circ.rotations())))
    ref = qgnag.train(he, circ, data, 2, enc_seed=17)
    assert np.array_equal(w.view(np.uint64), ref[0].view(np.uint64))
    from oracle import plain
    assert np.abs(w - plain.train(data, 2)).max() < 1e-3


@pytest.mark.parametrize("f", [37, 200])
def test_bbar_batches_on_device_equal_host(pair, f):
    """Bbar_k of every mini-batch (Sec. 3.1) computed on the device equals the
    host routine bit for bit (same summation orders) and the oracle's numpy
    computation within rounding; the last batch is ragged."""
    ctx, _ = pair
    X, y = synth.job(seed=f, n=5000, f=f, n_gauss=f // 2)
    g = qgnag.pad_cols(f + 1)
    dev = binding.lr_bbar_batches(ctx, X, y, 1024, g)
    assert dev.shape == (5, g)
    Z = qgnag.make_z(X, y)
    for k in range(5):
        rows = min(1024, 5000 - 1024 * k)
        assert np.array_equal(dev[k], binding.lr_bbar(X, y, 1024 * k, rows, g)), k
        ref = qgnag.bbar_rows(Z[1024 * k:1024 * k + rows], g)
        assert np.allclose(dev[k], ref, rtol=1e-12, atol=0), k
    assert not dev[:, f + 1:].any()
    with pytest.raises(binding.HeError):
        binding.lr_bbar_batches(ctx, np.zeros((10, 300)), np.ones(10), 1024, 512)  # more than 256 columns


def test_minibatch_job_bitwise(pair):
    """Algorithm 1 over 3 mini-batches of 1,024 rows (the last one ragged: 952
    rows), 4 iterations so batch 0 is revisited; the g16 polynomial."""
    ctx, he = pair
    X, y = synth.small(seed=11, n=3000, f=15)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, D, poly=qgnag.G16)
    job = binding.Job(ctx, X, y, binding.MINI_BATCH, 1024, binding.G16, 40.0, enc_seed=8, key_seed=2, batch_blocks=3)
    job.set_graph(True)
    L = circ.L
    nb = data.blocks.shape[0]
    assert job.stats().n_blocks == nb == 12
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(nb)]
    B = [OCt(job.input(1, k).export(), L, D) for k in range(data.nbatch)]
    (Ww, _, _), (Vw, _, _) = job.state_words()
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    sched = (1.0, 0.2, 10.0, 2.5)
    etas = qgnag.nag_scalars(4)
    for t in range(4):
        job.step(t, sched)
        k = t % data.nbatch
        blocks = Z[k * 4:(k + 1) * 4]
        Wn, Vn = circ.iteration(blocks, B[k], W, V, qgnag.schedule(t, *sched), etas[t], 1.0 / float(data.n_k[k]))
        W = circ.refresh(Wn, qgnag.obj_seed(8, qgnag.SEED_WREF, t))
        V = circ.refresh(Vn, qgnag.obj_seed(8, qgnag.SEED_VREF, t))
        (Ww, _, _), (Vw, _, _) = job.state_words()
        assert np.array_equal(Ww, W.data), t
        assert np.array_equal(Vw, V.data), t
    from oracle import plain
    wp = plain.train(data, 4, mode="mini", sched=sched, poly=qgnag.G16)
    assert np.abs(job.weights(0) - wp).max() < 1e-3


def test_multi_job_matches_single_jobs(pair):
    """Three full-batch jobs of different widths (g = 32, 16, 8) stepped together
    give, word for word, the state the oracle's circuit gives for each job on
    the job's own encrypted inputs, the words each job gives alone, and track
    their FP64 twins."""
    ctx, he = pair
    shapes = [(700, 5, 21), (1500, 15, 22), (400, 30, 23)]  # (n, f, enc_seed)
    data = [synth.job(seed=s, n=n, f=f) for n, f, s in shapes]
    multi_jobs = [binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=s, key_seed=2,
                              batch_blocks=2) for (X, y), (_, _, s) in zip(data, shapes)]
    alone = [binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=s, key_seed=2, batch_blocks=4)
             for (X, y), (_, _, s) in zip(data, shapes)]
    assert sorted(j.stats().g for j in multi_jobs) == [8, 16, 32]
    # the oracle side of every job: its circuit, its encrypted inputs, its start state
    circs, inputs, states = [], [], []
    rots = set(PAIR_ROTATIONS)
    for (X, y), jm in zip(data, multi_jobs):
        st = jm.stats()
        td = qgnag.TrainData(X, y, g=st.g, m=st.m, batch_rows=1024)
        circ = qgnag.Circuit(he, st.g, st.m, D)
        rots |= set(circ.rotations())
        L = circ.L
        Z = [OCt(jm.input(0, b).export(), L, D) for b in range(st.n_blocks)]
        B = OCt(jm.input(1, 0).export(), L, D)
        (Ww, _, _), (Vw, _, _) = jm.state_words()
        circs.append((circ, td))
        inputs.append((Z, B))
        states.append((OCt(Ww, L, D), OCt(Vw, L, D)))
    he.keygen(2, sorted(rots))  # keys depend on the seed and the Galois element only
    multi = binding.Multi(ctx, multi_jobs, blocks_per_launch=5)  # chunks straddle jobs
    etas = qgnag.nag_scalars(2)
    for t in range(2):
        multi.step(t)
        for j in alone:
            j.step(t)
        for i, (jm, ja) in enumerate(zip(multi_jobs, alone)):
            (Wm, _, _), (Vm, _, _) = jm.state_words()
            (Wa, _, _), (Va, _, _) = ja.state_words()
            assert np.array_equal(Wm, Wa) and np.array_equal(Vm, Va), t
            (circ, td), (Z, B), (W, V) = circs[i], inputs[i], states[i]
            Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(t), etas[t], 1.0 / td.n)
            seed = shapes[i][2]
            W = circ.refresh(Wn, qgnag.obj_seed(seed, qgnag.SEED_WREF, t))
            V = circ.refresh(Vn, qgnag.obj_seed(seed, qgnag.SEED_VREF, t))
            states[i] = (W, V)
            assert np.array_equal(Wm, W.data) and np.array_equal(Vm, V.data), (t, i)
    from oracle import plain
    for (circ, td), jm in zip(circs, multi_jobs):
        wp = plain.train(td, 2)
        assert np.abs(jm.weights(0) - wp).max() < 1e-3
    multi.close()


@pytest.fixture(scope="module")
def full_pair():
    """N = 2^16 with the full chain (60 + 8 x 40 bits + 60-bit P): the parameters
    of the 422,108 x 200 workload, 128 x 256 packing."""
    ctx = binding.Context(16, 9)
    he = Ckks(16, 9)
    return ctx, he


def test_full_shape_iteration_bitwise(full_pair):
    """One full-batch iteration at N = 2^16 on two 128 x 256 blocks of
    Financial-shaped data (201 columns padded to 256): the job's W' and V' after
    the refresh equal the oracle's word for word."""
    ctx, he = full_pair
    X, y = synth.financial(seed=3, n=256)
    data = qgnag.TrainData(X, y, g=256, m=128, batch_rows=1024)
    circ = qgnag.Circuit(he, 256, 128, D)
    he.keygen(2, circ.rotations())
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=7, key_seed=2)
    L = circ.L
    Z = [OCt(job.input(0, b).export(), L, D) for b in range(2)]
    B = OCt(job.input(1, 0).export(), L, D)
    (Ww, _, _), (Vw, _, _) = job.state_words()
    W, V = OCt(Ww, L, D), OCt(Vw, L, D)
    job.step(0)
    Wn, Vn = circ.iteration(Z, B, W, V, qgnag.schedule(0), qgnag.nag_scalars(1)[0], 1.0 / data.n)
    W = circ.refresh(Wn, qgnag.obj_seed(7, qgnag.SEED_WREF, 0))
    V = circ.refresh(Vn, qgnag.obj_seed(7, qgnag.SEED_VREF, 0))
    (Ww, _, _), (Vw, _, _) = job.state_words()
    assert np.array_equal(Ww, W.data)
    assert np.array_equal(Vw, V.data)


def test_full_shape_launch_configuration_against_twin(full_pair):
    """The launch configuration of the bench at N = 2^16 (256 blocks per launch,
    key switches in waves of 128 items) on 300 blocks, the last one ragged:
    decrypted weights within 1e-3 of the FP64 twin after 3 iterations."""
    ctx, _ = full_pair
    X, y = synth.financial(seed=4, n=300 * 128 - 37)
    data = qgnag.TrainData(X, y, g=256, m=128, batch_rows=1024)
    job = binding.Job(ctx, X, y, binding.FULL_BATCH, 1024, binding.G8, 40.0, enc_seed=9, key_seed=2)
    assert job.stats().n_blocks == 300
    for t in range(3):
        job.step(t)
    from oracle import plain
    wp = plain.train(data, 3)
    for row in (0, 64, 127):
        assert np.abs(job.weights(row) - wp).max() < 1e-3
