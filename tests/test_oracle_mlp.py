"""Pins of the FP64 oracle of the coefficient-proposal MLP."""
import math

import numpy as np
import pytest

import synth
from oracle import ifnso as O
from oracle import mlp as MLP


def _sample(seed, L=4):
    h, w, sig, fam = synth.mlp_spectrum(seed)
    o = math.sqrt(np.sum(sig ** 4))
    x = sig / math.sqrt(o)
    f = MLP.raw_features(x, h, w, math.sqrt(np.sum(sig ** 2)))
    return h, w, sig, x, f


def test_gelu_closed_form():
    assert MLP.gelu(np.array([0.0]))[0] == 0.0
    assert abs(MLP.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(MLP.gelu(np.array([-10.0]))[0]) < 1e-12
    t = np.linspace(-4, 4, 81)
    fd = (MLP.gelu(t + 1e-6) - MLP.gelu(t - 1e-6)) / 2e-6
    assert np.allclose(MLP.gelu_prime(t), fd, atol=1e-8)


def test_spectral_error_is_polar_distance_of_algorithm1():
    # E(c) = ||Y - U V^T||_F^2 / h for Y of Algorithm 1 with coefficients c (Sec. 2.1)
    w = np.array([0.3, 1.9, -2.4, 5.1])
    for seed in (3, 4, 5):
        M = synth.mlp_matrix(seed)
        h = M.shape[0]
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        x = s / math.sqrt(math.sqrt(np.sum(s ** 4)))
        E, _ = MLP.spectral_error(np.r_[1.0, w], x)
        Y = O.ifnso_alg1(M, w)
        assert abs(E - np.linalg.norm(Y - U @ Vt) ** 2 / h) < 1e-9 * max(1.0, E)


def test_features_match_matrix_traces():
    M = synth.mlp_matrix(7)
    h, w = M.shape
    G = M @ M.T
    D = G / np.linalg.norm(G)
    s = np.linalg.svd(M, compute_uv=False)
    x = s / math.sqrt(math.sqrt(np.sum(s ** 4)))
    f = MLP.raw_features(x, h, w, np.linalg.norm(M))
    D2 = D @ D
    ref = [math.log(np.trace(D) / h), math.log(np.trace(D2) / h), math.log(np.trace(D2 @ D2) / h),
           math.log(h), math.log(w), math.log(np.linalg.norm(M))]
    assert np.allclose(f, ref, atol=1e-10)
    assert abs(f[1] + math.log(h)) < 1e-12   # tr(D^2) = ||D||_F^2 = 1


def test_projection_and_zero_output():
    wfix = np.array([0.1, 2.1, -2.8, 5.5])
    out = np.zeros(6)
    c = MLP.coefficients(out, wfix)
    assert c[0] == 1.0 and np.array_equal(c[1:], wfix)
    out = np.arange(6.0)
    c = MLP.coefficients(out, wfix)
    assert c[0] == 1.0
    assert np.allclose(c[1:], wfix + MLP.scales(wfix) * out[1:5])


@pytest.mark.parametrize("K", [5, 7])
def test_batch_gradient_finite_difference(K):
    L = K - 1
    rng = np.random.default_rng(K)
    p = MLP.init_params(K, rng)
    p["W3"] *= 30.0  # leave the neighbourhood of the fixed coefficients
    wfix = rng.uniform(-2, 2, L)
    samples = [_sample(s, L) for s in range(4)]
    Z = [(f - f.mean()) / (f.std() + 1.0) for (_, _, _, _, f) in samples]
    spectra = [x for (_, _, _, x, _) in samples]
    loss, G, targets = MLP.batch_loss_grad(p, Z, spectra, wfix)
    for key in p:
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            lp, _, _ = MLP.batch_loss_grad(p, Z, spectra, wfix, targets)
            flat[idx] = old - 1e-6
            lm, _, _ = MLP.batch_loss_grad(p, Z, spectra, wfix, targets)
            flat[idx] = old
            fd = (lp - lm) / 2e-6
            an = G[key].reshape(-1)[idx]
            assert abs(an - fd) <= 1e-5 * max(1.0, abs(fd)), (key, idx, an, fd)


def test_fallback_rule():
    K = 5
    rng = np.random.default_rng(0)
    p = MLP.init_params(K, rng)
    wfix = np.array([0.1, 2.1, -2.8, 5.5])
    z = rng.standard_normal(6)
    p["b3"][K] = 5.0   # head predicts a larger error: fixed coefficients are used
    c, fb = MLP.propose(p, z, wfix)
    assert fb and np.array_equal(c[1:], wfix)
    p["b3"][K] = -5.0
    c, fb = MLP.propose(p, z, wfix)
    assert not fb and c[0] == 1.0
