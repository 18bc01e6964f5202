"""The scalar polynomial of IFNSO and its coefficient learner, FP64
(test infrastructure only; see oracle/__init__.py).

Parity unpinned: the paper prints no coefficient values, so the fitted w of
``learn`` are pinned only through determinism, descent, the gradient formula
and Adam's update rule (tests/test_oracle_coeffs.py).
"""
from __future__ import annotations

import math

import numpy as np


def f_term(x, l: int):
    """f_l(x) = x for l = 0, x (1 - x^2)^(2^(l-1)) for l >= 1 (Eq. final_polynomial_term)."""
    x = np.asarray(x, dtype=np.float64)
    if l == 0:
        return x.copy()
    return x * (1.0 - x * x) ** (2 ** (l - 1))


def f_term_prime(x, l: int):
    """f_l'(x) = (1 - x^2)^(2^(l-1) - 1) [1 - (2^l + 1) x^2] for l >= 1, 1 for l = 0
    (Eq. eq_gradient)."""
    x = np.asarray(x, dtype=np.float64)
    if l == 0:
        return np.ones_like(x)
    return (1.0 - x * x) ** (2 ** (l - 1) - 1) * (1.0 - (2 ** l + 1) * x * x)


def peak(l: int):
    """Extreme point of f_l on (0, 1): x* = 1/sqrt(2^l + 1),
    y* = x* (2^l/(2^l + 1))^(2^(l-1))  (Sec. 2.2)."""
    xs = 1.0 / math.sqrt(2 ** l + 1)
    ys = xs * (2 ** l / (2 ** l + 1)) ** (2 ** (l - 1))
    return xs, ys


def f_full(x, w):
    """f(x) = x + sum_{l=1}^L w_l f_l(x)  (Eq. sum_equation); w = (w_1..w_L)."""
    x = np.asarray(x, dtype=np.float64)
    y = x.copy()
    for l, wl in enumerate(w, start=1):
        y = y + wl * f_term(x, l)
    return y


def wL_exact(w_free, L: int) -> float:
    """w_L from the peak constraint f(1/sqrt(2^L + 1)) = 1 (Eq. peak), solved
    exactly (Sec. 2.3): (sqrt(2^L+1) - 1 - sum_k w_k r^(2^(k-1))) r^(-2^(L-1)),
    r = 2^L/(2^L + 1)."""
    r = 2.0 ** L / (2.0 ** L + 1.0)
    s = sum(wk * r ** (2 ** (k - 1)) for k, wk in enumerate(w_free, start=1))
    return (math.sqrt(2.0 ** L + 1.0) - 1.0 - s) * (1.0 / r) ** (2 ** (L - 1))


def wL_approx(w_free, L: int) -> float:
    """The printed approximation (Eq. b_approximation, used in Eq.
    overall_polynomial): w_L = e^(1/2) (2^(L/2) - 1) - sum_{l<L} w_l."""
    return math.exp(0.5) * (2.0 ** (L / 2.0) - 1.0) - float(np.sum(w_free))


def complete(w_free, L: int, form: str = "approx"):
    """(w_1..w_{L-1}) -> (w_1..w_L) with w_L from the chosen form."""
    w_free = [float(v) for v in w_free]
    assert len(w_free) == L - 1
    wl = wL_approx(w_free, L) if form == "approx" else wL_exact(w_free, L)
    return np.array(w_free + [wl])


def loss(w_free, x, L: int, form: str = "approx") -> float:
    """sum_j (f(x_j) - 1)^2 with f of Eq. overall_polynomial (Sec. 2.4)."""
    return float(np.sum((f_full(x, complete(w_free, L, form)) - 1.0) ** 2))


def dwL_dw(L: int, form: str = "approx"):
    """d w_L / d w_k for k = 1..L-1 under the chosen form of the constraint."""
    if form == "approx":
        return -np.ones(L - 1)
    r = 2.0 ** L / (2.0 ** L + 1.0)
    return np.array([-(r ** (2 ** (k - 1))) * (1.0 / r) ** (2 ** (L - 1)) for k in range(1, L)])


def grad(w_free, x, L: int, form: str = "approx"):
    """Gradient of ``loss`` in w_1..w_{L-1}: 2 sum_j (f(x_j) - 1) (f_k(x_j) + dw_L/dw_k f_L(x_j))."""
    x = np.asarray(x, dtype=np.float64)
    e = f_full(x, complete(w_free, L, form)) - 1.0
    fL = f_term(x, L)
    dl = dwL_dw(L, form)
    return np.array([2.0 * np.sum(e * (f_term(x, k) + dl[k - 1] * fL)) for k in range(1, L)])


def learn(L: int, sampler, iters: int = 20000, lr: float = 0.1, step_size: int = 10000,
          gamma: float = 0.5, betas=(0.9, 0.999), eps: float = 1e-8, form: str = "approx",
          w0=None, record: int = 0):
    """Coefficient learning of Algorithm 1 / Sec. 2.3, with the schedule of Sec. 3.1.1.

    Adam (D. P. Kingma, J. Ba, 2015) on w_1..w_{L-1}, initial learning rate 0.1
    halved every 10000 iterations, 20000 iterations, each minimising
    sum_j (f(x_j) - 1)^2 over the samples ``sampler(t)`` of iteration t (the
    paper draws 1000 uniform points of (0, 1) per iteration).  Adam's moments
    start at zero; the bias corrections use running products of the betas;
    the learning rate of iteration t is lr * gamma^floor(t / step_size).
    Returns (w_1..w_L, [(t, loss_t) every ``record`` iterations]).
    """
    b1, b2 = betas
    n = L - 1
    w = np.zeros(n) if w0 is None else np.array(w0, dtype=np.float64)
    m = np.zeros(n)
    v = np.zeros(n)
    p1 = 1.0
    p2 = 1.0
    hist = []
    for t in range(iters):
        x = sampler(t)
        if n > 0:
            g = grad(w, x, L, form)
            m = b1 * m + (1.0 - b1) * g
            v = b2 * v + (1.0 - b2) * g * g
            p1 *= b1
            p2 *= b2
            lr_t = lr * gamma ** (t // step_size)
            denom = np.sqrt(v) / math.sqrt(1.0 - p2) + eps
            w = w - (lr_t / (1.0 - p1)) * m / denom
        if record and t % record == 0:
            hist.append((t, loss(w, x, L, form)))
    return complete(w, L, form), hist
