"""Quadratic-gradient NAG in FP64 on plaintext -- the twin of the encrypted run.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Algorithm 1 (Sec. 3.2) with the full-batch variant of Sec. 3.3, on the same
packed data and with the same polynomial sigmoid as the encrypted circuit.  The
decrypted weights of an encrypted run must stay within 1e-3 of this run.

With ``sigmoid='exact'`` the logistic function replaces the polynomial; that
mode exists to pin the algorithm (gradient sign and normalisation, update
order) against an independent logistic-regression solver.  With
``first_order=True`` the update is the first-order NAG baseline of Sec. 2.3,
w' = v + gamma (1/n) g, gamma taken from the schedule (constant when max = min).
"""
import math

import numpy as np

from .qgnag import G8, nag_scalars, schedule


def loglik(w, Z):
    """l(w) = -(1/n) sum_i ln(1 + exp(-z_i . w)) (Sec. 2.3)."""
    return -np.mean(np.logaddexp(0.0, -(Z @ w)))


def gradient(w, Z, sigmoid="poly", poly=G8):
    """Unnormalised gradient sum_i (1 - sigma(z_i . w)) z_i (Algorithm 1)."""
    ip = Z @ w
    if sigmoid == "exact":
        one_minus = 1.0 - 1.0 / (1.0 + np.exp(-ip))
    else:
        c0, c1, c3 = poly
        one_minus = 1.0 - (c0 + c1 * ip + c3 * ip ** 3)
    return Z.T @ one_minus


def train(data, iters, mode="full", sched=(2.0, 1.0, 81.0, 2.5), sigmoid="poly",
          poly=G8, trace=False, first_order=False):
    """Returns W (length g) after `iters` iterations; with trace=True also the
    list of (W, V) after each iteration."""
    g = data.g
    W = np.zeros(g)
    V = np.zeros(g)
    etas = nag_scalars(iters)
    hist = []
    for t in range(iters):
        alpha = schedule(t, *sched)
        if mode == "full":
            Zr, nbb, inv_n = data.Z, data.n * data.bbar_full, 1.0 / data.n
        else:
            k = t % data.nbatch
            Zr = data.Z[k * data.batch_rows:(k + 1) * data.batch_rows]
            nbb, inv_n = float(data.n_k[k]) * data.bbar_k[k], 1.0 / float(data.n_k[k])
        grad = np.zeros(g)
        grad[:data.f1] = alpha * gradient(W[:data.f1], Zr, sigmoid, poly)
        G = (grad if first_order else nbb * grad) * inv_n
        eta = etas[t]
        Vt = W + G
        W = (1.0 - eta) * Vt + eta * V
        V = Vt
        if trace:
            hist.append((W.copy(), V.copy()))
    return (W, hist) if trace else W


def step_from(W, V, Zr, nbb, inv_n, alpha, eta, poly=G8):
    """One iteration of the update from given (W, V): returns (W', V')."""
    g = W.shape[0]
    f1 = Zr.shape[1]
    grad = np.zeros(g)
    grad[:f1] = alpha * gradient(W[:f1], Zr, "poly", poly)
    Vt = W + nbb * grad * inv_n
    return (1.0 - eta) * Vt + eta * V, Vt


def max_abs_ip(W, Z):
    return float(np.max(np.abs(Z @ W[:Z.shape[1]]))) if len(Z) else 0.0


__all__ = ["loglik", "gradient", "train", "step_from", "max_abs_ip", "math"]
