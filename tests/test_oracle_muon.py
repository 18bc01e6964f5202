"""Pins of the FP64 Muon step (oracle/muon.py): its special cases reduce it to
pieces pinned elsewhere (Algorithm 1 in test_oracle_ifnso.py)."""
import numpy as np

import synth
from oracle import ifnso as O
from oracle import muon as MU

W4 = np.array([0.5, 0.4, 0.9, 1.0])


def test_beta_zero_is_plain_orthogonalized_step():
    G = synth.gaussian(1, 12, 20)
    M = synth.gaussian(2, 12, 20)
    W = synth.gaussian(3, 12, 20)
    for nest in (False, True):
        M1, U, W1 = MU.muon_step(G, M, W, W4, 0.0, nest, 0.1)
        assert np.array_equal(M1, G) and np.array_equal(U, G)
        assert np.allclose(W1, W - 0.1 * O.ifnso_alg1(G, W4), rtol=0, atol=1e-15)


def test_nesterov_input_expands():
    G, M = synth.gaussian(4, 9, 7), synth.gaussian(5, 9, 7)
    beta = 0.9
    M1, U = MU.momentum(G, M, beta, True)
    assert np.allclose(U, (1 + beta) * G + beta ** 2 * M, rtol=0, atol=1e-14)
    M1b, Ub = MU.momentum(G, M, beta, False)
    assert np.array_equal(M1, M1b) and np.array_equal(Ub, M1b)


def test_zero_step_and_shape_factor():
    G, M, W = synth.gaussian(6, 16, 8), synth.gaussian(7, 16, 8), synth.gaussian(8, 16, 8)
    assert np.array_equal(MU.muon_step(G, M, W, W4, 0.9, True, 0.0)[2], W)
    assert MU.shape_factor(16, 8) == np.sqrt(2.0) and MU.shape_factor(8, 16) == 1.0
    # a tall W takes its update in its own shape, scaled by sqrt(rows / cols)
    U = synth.gaussian(9, 16, 8)
    assert np.allclose(MU.update(W, U, W4, 1.0), W - np.sqrt(2.0) * O.ifnso_alg1(U, W4), rtol=0, atol=1e-14)


def test_momentum_accumulates_geometrically():
    # with a constant gradient, M after n steps from 0 is G (1 - beta^n) / (1 - beta)
    G = synth.gaussian(10, 5, 6)
    M = np.zeros_like(G)
    beta = 0.95
    for _ in range(7):
        M, _ = MU.momentum(G, M, beta, False)
    assert np.allclose(M, G * (1 - beta ** 7) / (1 - beta), rtol=1e-14, atol=0)
