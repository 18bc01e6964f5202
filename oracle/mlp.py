"""FP64 oracle of the coefficient-proposal MLP (test infrastructure only; see
oracle/__init__.py).

The paper names per-input ("dynamic") coefficients as future work (Sec. 4);
this network is that extension: 6 spectral features of a matrix -> two GELU
layers of 64 -> K coefficient slots (c_0, w_1..w_L; K = L + 1) and one
fallback head.  Definitions written out plainly:

features  z = standardise([log tr(D)/h, log tr(D^2)/h, log tr(D^4)/h,
          log h, log w, log ||A||_F]) with D = A A^T / ||A A^T||_F, whose
          eigenvalues are x_i^2 for the singular values x_i of X = A/sqrt(o).
network   a1 = W1 z + b1, h1 = gelu(a1), a2 = W2 h1 + b2, h2 = gelu(a2),
          out = W3 h2 + b3, gelu(t) = t Phi(t) (exact, erf form).
coeffs    c_0 = 1 (projection onto p(1) = 1: f(1) = c_0 for every w);
          w_l = wfix_l + s_l out_l, s_l = max(1, |wfix_l|) / 10, l = 1..L.
objective E(c) = (1/h) sum_i (f_c(x_i) - 1)^2, the squared distance to the
          polar factor, ||Y - U V^T||_F^2 / h, of the output of Algorithm 1
          with coefficients c (Y = U diag(f_c(x)) V^T, Sec. 2.1).
fallback  head r = out_K is trained towards log(E(c) + eps) - log(E(wfix) + eps)
          (c held fixed); at inference the fixed coefficients are used when r > 0.
loss      E(c) + lam (r - target)^2, averaged over the batch.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 64
N_FEAT = 6
EPS_LOG = 1e-12
LAM = 0.1


def gelu(t):
    from scipy.special import erf

    return 0.5 * t * (1.0 + erf(t / math.sqrt(2.0)))


def gelu_prime(t):
    from scipy.special import erf

    return 0.5 * (1.0 + erf(t / math.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / math.sqrt(2.0 * math.pi)


def raw_features(x, h, w, norm_a):
    """Unstandardised features of one matrix from its scaled singular values x."""
    s = np.asarray(x, dtype=np.float64) ** 2
    t1 = np.sum(s) / h
    t2 = np.sum(s ** 2) / h
    t4 = np.sum(s ** 4) / h
    return np.array([math.log(t1), math.log(t2), math.log(t4), math.log(h), math.log(w), math.log(norm_a)])


def n_out(K):
    return K + 1


def init_params(K, rng):
    """Gaussian init with 1/sqrt(fan_in) scale; last layer small."""
    p = {
        "W1": rng.standard_normal((HIDDEN, N_FEAT)) / math.sqrt(N_FEAT),
        "b1": np.zeros(HIDDEN),
        "W2": rng.standard_normal((HIDDEN, HIDDEN)) / math.sqrt(HIDDEN),
        "b2": np.zeros(HIDDEN),
        "W3": 0.01 * rng.standard_normal((n_out(K), HIDDEN)) / math.sqrt(HIDDEN),
        "b3": np.zeros(n_out(K)),
    }
    return p


def forward(p, z):
    a1 = p["W1"] @ z + p["b1"]
    h1 = gelu(a1)
    a2 = p["W2"] @ h1 + p["b2"]
    h2 = gelu(a2)
    out = p["W3"] @ h2 + p["b3"]
    return out, (z, a1, h1, a2, h2)


def backward(p, cache, d_out):
    """Gradients of a scalar loss with respect to every parameter, given dL/d out."""
    z, a1, h1, a2, h2 = cache
    g = {"W3": np.outer(d_out, h2), "b3": d_out.copy()}
    d_h2 = p["W3"].T @ d_out
    d_a2 = d_h2 * gelu_prime(a2)
    g["W2"] = np.outer(d_a2, h1)
    g["b2"] = d_a2
    d_h1 = p["W2"].T @ d_a2
    d_a1 = d_h1 * gelu_prime(a1)
    g["W1"] = np.outer(d_a1, z)
    g["b1"] = d_a1
    return g


def scales(wfix):
    return np.maximum(1.0, np.abs(np.asarray(wfix, dtype=np.float64))) / 10.0


def coefficients(out, wfix):
    """(c_0 = 1, w_1..w_L) from the network output (the first K entries)."""
    L = len(wfix)
    w = np.asarray(wfix, dtype=np.float64) + scales(wfix) * out[1:L + 1]
    return np.concatenate([[1.0], w])


def spectral_error(c, x):
    """E(c) = (1/h) sum_i (f_c(x_i) - 1)^2 and dE/dw_l (l = 1..L), with
    f_c(x) = c_0 x + sum_l w_l x (1 - x^2)^(2^(l-1)) (Eq. sum_equation)."""
    x = np.asarray(x, dtype=np.float64)
    h = len(x)
    L = len(c) - 1
    terms = np.stack([x * (1.0 - x * x) ** (2 ** (l - 1)) for l in range(1, L + 1)])
    f = c[0] * x + np.asarray(c[1:]) @ terms
    e = f - 1.0
    return float(np.sum(e * e) / h), 2.0 * (terms @ e) / h


def sample_loss(p, z, x, wfix, target=None):
    """Loss of one sample and dL/d out.  The fallback head's target is a
    constant of the gradient (computed from the current coefficients unless
    given)."""
    L = len(wfix)
    out, cache = forward(p, z)
    c = coefficients(out, wfix)
    E, dE_dw = spectral_error(c, x)
    Efix, _ = spectral_error(np.concatenate([[1.0], wfix]), x)
    if target is None:
        target = math.log(E + EPS_LOG) - math.log(Efix + EPS_LOG)
    r = out[L + 1]
    loss = E + LAM * (r - target) ** 2
    d_out = np.zeros_like(out)
    d_out[1:L + 1] = dE_dw * scales(wfix)
    d_out[L + 1] = 2.0 * LAM * (r - target)
    return loss, d_out, cache, E, Efix, r, target


def batch_loss_grad(p, Z, spectra, wfix, targets=None):
    """Mean loss over a batch, its parameter gradients and the head targets used."""
    tot = 0.0
    G = {k: np.zeros_like(v) for k, v in p.items()}
    used = []
    for i, (z, x) in enumerate(zip(Z, spectra)):
        loss, d_out, cache, _, _, _, t = sample_loss(p, z, x, wfix, None if targets is None else targets[i])
        used.append(t)
        tot += loss
        g = backward(p, cache, d_out)
        for k in G:
            G[k] += g[k]
    n = len(Z)
    return tot / n, {k: v / n for k, v in G.items()}, used


def propose(p, z, wfix):
    """Coefficients used at inference: the network's, or the fixed ones when
    the fallback head predicts a larger error."""
    out, _ = forward(p, z)
    L = len(wfix)
    if out[L + 1] > 0.0:
        return np.concatenate([[1.0], wfix]), True
    return coefficients(out, wfix), False
