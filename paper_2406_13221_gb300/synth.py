"""Seeded synthetic training data shaped like the paper's workloads.

This module only draws inputs; it holds none of the method's arithmetic and is
shared by the tests, the benchmark and the CPU reference.

* ``small``     -- 1,024 samples x 15 features uniform in [-1, 1]; labels +/-1
  from a logistic model with weights ~ N(0, 1) (bias included).
* ``financial`` -- stands in for the paper's private credit dataset
  (Sec. 5.1: 422,108 training samples, 200 features): 150 columns N(0, 1)
  standardised, 50 binary columns Bernoulli(p), p ~ U(0.05, 0.5); every column
  min-max scaled to [-1, 1]; labels from a sparse logistic model with 20 nonzero
  weights ~ N(0, 1) plus a N(0, 1) bias.
* ``job``       -- one job of the uneven multi-job workload: n samples, f
  features, generated like ``financial`` (three quarters Gaussian columns).
* ``image_pair`` -- stands in for the paper's restructured MNIST task
  (Sec. 5.2: 11,982 training images of two digit classes, 14 x 14 = 196
  pixel features): two smooth random class templates on a 14 x 14 grid,
  each sample its class template shifted by up to one pixel, scaled by a
  random stroke intensity, plus Gaussian pixel noise, clipped to [0, 1] and
  min-max scaled to [-1, 1]; labels +/-1 by class, classes balanced.
"""
import numpy as np


def _labels(rng, X, w, b):
    logit = X @ w + b
    p = 1.0 / (1.0 + np.exp(-logit))
    return np.where(rng.random(X.shape[0]) < p, 1.0, -1.0)


def small(seed=1, n=1024, f=15):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(n, f))
    w = rng.standard_normal(f + 1)
    y = _labels(rng, X, w[1:], w[0])
    return X, y


def _scale_cols(X):
    lo, hi = X.min(axis=0), X.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    return (X - lo) / span * 2.0 - 1.0


def job(seed, n, f, n_gauss=None, nnz=20):
    rng = np.random.default_rng(seed)
    ng = (3 * f) // 4 if n_gauss is None else n_gauss
    nbin = f - ng
    Xg = rng.standard_normal((n, ng))
    Xg = (Xg - Xg.mean(axis=0)) / Xg.std(axis=0)
    p = rng.uniform(0.05, 0.5, size=nbin)
    Xb = (rng.random((n, nbin)) < p).astype(np.float64)
    X = _scale_cols(np.concatenate([Xg, Xb], axis=1))
    w = np.zeros(f)
    idx = rng.choice(f, size=min(nnz, f), replace=False)
    w[idx] = rng.standard_normal(len(idx))
    y = _labels(rng, X, w, rng.standard_normal())
    return X, y


def financial(seed=1, n=422108, f=200):
    return job(seed, n, f, n_gauss=150, nnz=20)


def image_pair(seed=7, n=11982, side=14, noise=0.15):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:side, 0:side] / (side - 1.0)
    templates = []
    for _ in range(2):
        t = np.zeros((side, side))
        for _ in range(6):  # a few Gaussian strokes per class
            cy, cx = rng.uniform(0.2, 0.8, 2)
            sy, sx = rng.uniform(0.05, 0.2, 2)
            t += np.exp(-((yy - cy) ** 2 / (2 * sy * sy) + (xx - cx) ** 2 / (2 * sx * sx)))
        templates.append(t / t.max())
    cls = rng.permutation(np.arange(n) % 2)
    X = np.empty((n, side * side))
    for k in range(n):
        img = np.roll(templates[cls[k]], tuple(rng.integers(-1, 2, 2)), axis=(0, 1))
        img = img * rng.uniform(0.7, 1.0) + noise * rng.standard_normal((side, side))
        X[k] = np.clip(img, 0.0, 1.0).ravel()
    return _scale_cols(X), np.where(cls == 1, 1.0, -1.0)


def multijob_shapes(seed=5, njobs=16, lo=5000, hi=100000):
    """(n_j, f_j) for the uneven multi-job workload: n_j log-uniform in
    [lo, hi], f_j uniform in {32, 64, 128, 200}."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(lo), np.log(hi), size=njobs)).astype(np.int64)
    fs = rng.choice([32, 64, 128, 200], size=njobs)
    return [(int(a), int(b)) for a, b in zip(ns, fs)]
