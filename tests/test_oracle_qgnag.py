"""Pins for the algorithm layer of the oracle: client precompute, schedule, NAG
scalars, the FP64 plaintext twin and the encrypted circuit against that twin."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import plain, qgnag
from oracle.ckks import Ckks, round_half_away
from paper_2406_13221_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_polys():
    out = {}
    for line in open(os.path.join(HERE, "golden", "sigmoid_polys.txt")):
        if line.strip() and not line.startswith("#"):
            name, R, c0, c1, c3 = line.split()
            out[name] = (float(R), (float(c0), float(c1), float(c3)))
    return out


def test_sigmoid_polys_are_the_papers_and_least_squares():
    gp = golden_polys()
    assert gp["g8"][1] == qgnag.G8
    assert gp["g16"][1] == qgnag.G16
    for name, (R, (c0, c1, c3)) in gp.items():
        x = np.linspace(-R, R, 100001)
        fit = np.polyfit(x, 1.0 / (1.0 + np.exp(-x)), 3)[::-1]
        assert abs(fit[0] - c0) < 1e-9 and abs(fit[2]) < 1e-9
        assert abs(fit[1] - c1) < 1e-3
        assert abs(fit[3] - c3) < 1e-4


def test_schedule_endpoints_from_table():
    g = {}
    for line in open(os.path.join(HERE, "golden", "paper_workload.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = float(v)
    args = (g["sched_max"], g["sched_min"], g["sched_T"], g["sched_power"])
    assert qgnag.schedule(0, *args) == 2.0
    assert abs(qgnag.schedule(81, *args) - 1.0) < 1e-15
    vals = [qgnag.schedule(t, *args) for t in range(82)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    # 2 - (t/81)^2.5 at t = 41 (the mini-batch iteration count of Table 1)
    assert abs(qgnag.schedule(41, *args) - (2 - (41 / 81) ** 2.5)) < 1e-15


def test_nag_scalars_recurrence():
    """alpha_{k+1} solves a^2 - a - alpha_k^2 = 0; eta_k = (1 - alpha_k)/alpha_{k+1}."""
    etas = qgnag.nag_scalars(30)
    a = [0.01]
    for _ in range(31):
        # positive root of x^2 - x - a^2 = 0
        a.append((1 + math.sqrt(1 + 4 * a[-1] ** 2)) / 2)
    for k in range(30):
        assert abs(a[k + 1] ** 2 - a[k + 1] - a[k] ** 2) < 1e-9
        assert abs(etas[k] - (1 - a[k]) / a[k + 1]) < 1e-15
    assert 0.98 < etas[0] < 0.99 and all(e < 0 for e in etas[1:])


def test_bbar_is_inverse_gershgorin_bound():
    rng = np.random.default_rng(0)
    Z = rng.uniform(-1, 1, (50, 5))
    b = qgnag.bbar_rows(Z, 8)
    for c in range(5):
        s = 0.0
        for k in range(5):
            s += abs(sum(Z[r, c] * Z[r, k] for r in range(50)))
        assert abs(b[c] - 1.0 / (qgnag.EPS + 0.25 * s)) < 1e-12 * b[c]
    assert not b[5:].any()
    # a diagonal Hessian bound: B = diag(1/(eps + |H_cc|/4)) inverts -H/4 up to eps
    Zd = np.zeros((4, 3))
    Zd[0, 0], Zd[1, 1], Zd[2, 2] = 2.0, 3.0, 1.0
    assert np.allclose(qgnag.bbar_rows(Zd, 4)[:3], [1 / (1e-8 + 1.0), 1 / (1e-8 + 2.25), 1 / (1e-8 + 0.25)])


def test_full_batch_bbar_harmonic_combination():
    """Sec. 3.3 combination: one batch gives back its own Bbar; with entries of a
    single sign the combination equals the direct full-data Bbar up to eps terms."""
    rng = np.random.default_rng(1)
    Z = rng.uniform(0, 1, (64, 4))
    one = qgnag.bbar_rows(Z, 4)
    assert np.allclose(qgnag.bbar_full_from_batches([one]), one, rtol=1e-15)
    parts = [qgnag.bbar_rows(Z[k * 16:(k + 1) * 16], 4) for k in range(4)]
    full = qgnag.bbar_full_from_batches(parts)
    assert np.allclose(full, one, rtol=1e-6)


def test_gradient_matches_finite_differences():
    X, y = synth.small(seed=3, n=200, f=5)
    Z = qgnag.make_z(X, y)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(6) * 0.3
    g = plain.gradient(w, Z, "exact")
    h = 1e-6
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        fd = (plain.loglik(w + e, Z) - plain.loglik(w - e, Z)) / (2 * h)
        assert abs(g[j] / Z.shape[0] - fd) < 1e-7


def test_twin_converges_to_independent_mle():
    """Exact-sigmoid QG-NAG reaches the maximiser that scipy's BFGS finds."""
    X, y = synth.small(seed=4, n=1024, f=7)
    data = qgnag.TrainData(X, y, g=8, m=128, batch_rows=1024)
    W = plain.train(data, 60, sigmoid="exact", sched=(1.0, 1.0, 81.0, 2.5))
    res = minimize(lambda w: -plain.loglik(w, data.Z), np.zeros(8), method="BFGS",
                   jac=lambda w: -plain.gradient(w, data.Z, "exact") / data.n, tol=1e-12)
    assert np.abs(W - res.x).max() < 1e-4
    assert plain.loglik(W, data.Z) >= plain.loglik(res.x, data.Z) - 1e-10


def test_round_half_away():
    assert round_half_away(2.5) == 3 and round_half_away(-2.5) == -3
    assert round_half_away(0.49999999999999994) == 0
    assert round_half_away(-0.5) == -1 and round_half_away(1e15 + 0.5) == 1000000000000001


def test_block_count_closed_form():
    """Sec. 2.2: (n+1)(1+f)/(m g) ciphertexts; 422,108 x (200+1) padded to g = 256
    with m g = 2^15 gives 3,298 blocks."""
    g = qgnag.pad_cols(201)
    m = (1 << 15) // g
    assert (g, m) == (256, 128)
    assert -(-422108 // m) == 3298


@pytest.fixture(scope="module")
def small_run():
    X, y = synth.small()
    he = Ckks(13, 9)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, 2.0 ** 40)
    he.keygen(2, circ.rotations())
    return he, circ, data


def test_encrypted_small_config_matches_fp64_twin(small_run):
    he, circ, data = small_run
    w, trace = qgnag.train(he, circ, data, 2, enc_seed=3, return_trace=True)
    wp, hist = plain.train(data, 2, trace=True)
    err = np.abs(w - wp[None, :]).max()
    assert err < 1e-3
    # the first iteration's W', V' before refresh as well
    Wn, Vn = trace[0][0], trace[0][1]
    assert Wn.level == 0 and Vn.level == 0
    zw = he.decode(he.decrypt(Wn)).real.reshape(circ.m, circ.g)
    assert np.abs(zw - hist[0][0][None, :]).max() < 1e-3


def test_encrypted_minibatch_mode_matches_fp64_twin():
    X, y = synth.small(seed=7, n=2048, f=15)
    he = Ckks(13, 9)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, 2.0 ** 40, poly=qgnag.G16)
    he.keygen(5, circ.rotations())
    sched = (1.0, 0.2, 10.0, 2.5)
    w = qgnag.train(he, circ, data, 3, enc_seed=9, mode="mini", sched=sched)
    wp = plain.train(data, 3, mode="mini", sched=sched, poly=qgnag.G16)
    assert np.abs(w - wp[None, :]).max() < 1e-3


def test_first_order_step_closed_form():
    """Sec. 2.3 first-order NAG from W0 = V0 = 0: V1 = (gamma/n) sum_i (1 - g8(0)) z_i
    with g8(0) = 1/2, W1 = (1 - eta_0) V1."""
    X, y = synth.small(seed=5, n=300, f=6)
    data = qgnag.TrainData(X, y, g=8, m=128, batch_rows=1024)
    lr = 0.7
    W1, hist = plain.train(data, 1, sched=(lr, lr, 81.0, 2.5), trace=True, first_order=True)
    V1 = np.zeros(8)
    V1[:7] = lr * 0.5 * data.Z.mean(axis=0)
    eta0 = qgnag.nag_scalars(1)[0]
    assert np.allclose(hist[0][1], V1, atol=1e-15)
    assert np.allclose(W1, (1 - eta0) * V1, atol=1e-15)


def test_first_order_twin_converges_to_independent_mle():
    """With the exact sigmoid and a constant rate, first-order NAG reaches the
    maximiser that scipy's BFGS finds (pins sign and 1/n normalisation)."""
    X, y = synth.small(seed=4, n=1024, f=7)
    data = qgnag.TrainData(X, y, g=8, m=128, batch_rows=1024)
    W = plain.train(data, 400, sigmoid="exact", sched=(2.0, 2.0, 81.0, 2.5), first_order=True)
    res = minimize(lambda w: -plain.loglik(w, data.Z), np.zeros(8), method="BFGS",
                   jac=lambda w: -plain.gradient(w, data.Z, "exact") / data.n, tol=1e-12)
    assert np.abs(W - res.x).max() < 1e-5


def test_encrypted_first_order_matches_fp64_twin():
    """The first-order circuit (no Bbar product, depth 6) against its FP64 twin."""
    X, y = synth.small(seed=6, n=1024, f=15)
    he = Ckks(13, 9)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, 2.0 ** 40, first_order=True)
    assert circ.L == qgnag.DEPTH_FIRST_ORDER == 5
    he.keygen(2, circ.rotations())
    sched = (1.0, 1.0, 81.0, 2.5)
    w, trace = qgnag.train(he, circ, data, 2, enc_seed=4, sched=sched, return_trace=True)
    assert trace[0][0].level == 0
    wp = plain.train(data, 2, sched=sched, first_order=True)
    assert np.abs(w - wp[None, :]).max() < 1e-3
    # the first-order and quadratic-gradient updates differ (Bbar is not the identity)
    assert np.abs(wp - plain.train(data, 2, sched=sched)).max() > 1e-3


def test_masked_polynomial_is_zero_outside_column_zero():
    """Reading of the Sec. 2.2 circuit: with the mask inside the plaintext
    products, s = (1 - c0) M - c1 (M t) - c3 t^2 (M t) decrypts to 1 - g8(ip_r)
    in column 0 of row r and to 0 elsewhere (although t holds partial sums
    there); after the replication every column of row r holds 1 - g8(ip_r)."""
    X, y = synth.small(seed=8, n=256, f=15)
    he = Ckks(13, 9)
    data = qgnag.TrainData(X, y, g=16, m=256, batch_rows=1024)
    circ = qgnag.Circuit(he, 16, 256, 2.0 ** 40)
    he.keygen(3, circ.rotations())
    L, D = circ.L, 2.0 ** 40
    rng = np.random.default_rng(8)
    w = rng.uniform(-1, 1, 16)
    Z = he.encrypt(he.encode(data.blocks[0], L, D), 1)
    W = he.encrypt(he.encode(np.tile(w, 256), L, D), 2)
    t = he.rescale(he.mul(Z, W))
    for k in range(circ.lg):
        t = he.add(t, he.rotate(t, 1 << k))
    sq = he.rescale(he.mul(t, t))
    cube = he.rescale(he.mul(sq, he.rescale(he.ptmul(t, circ.p3))))
    lin = he.rescale(he.ptmul(t, circ.p1))
    lin.scale = cube.scale
    s = he.ptadd(he.add(cube, he.moddrop(lin, cube.level)), circ.p0)
    got = he.decode(he.decrypt(s)).real.reshape(256, 16)
    ip = data.blocks[0].reshape(256, 16) @ w
    c0, c1, c3 = qgnag.G8
    want = 1.0 - (c0 + c1 * ip + c3 * ip ** 3)
    assert np.abs(got[:, 0] - want).max() < 1e-6
    assert np.abs(got[:, 1:]).max() < 1e-6
    for k in range(circ.lg):
        s = he.add(s, he.rotate(s, -(1 << k)))
    rep = he.decode(he.decrypt(s)).real.reshape(256, 16)
    assert np.abs(rep - want[:, None]).max() < 1e-6
