"""The seeded input generators: Philox known-answer vectors, exact BF16
rounding, and the structure of the low-rank-plus-noise recipe."""
import json
import os

import numpy as np
import pytest

import synth
from synth import philox4x32_10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        c = [np.array([int(x, 16)], dtype=np.uint64) for x in v["ctr"]]
        k = [int(x, 16) for x in v["key"]]
        out = philox4x32_10(*c, *k)
        assert ["%08x" % int(o[0]) for o in out] == v["out"]


def test_bf16_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(100000).astype(np.float32) * 1e3
    x[:4] = [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0]   # ties
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(synth.to_bf16_bits(x), ref)


def test_uniforms_open_interval():
    u = synth.learner_uniforms(0, 3, 100000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01


def test_lowrank_noise_structure():
    rows, cols = 48, 80
    S, N = synth.lowrank_noise_int(3, rows, cols)
    assert np.linalg.matrix_rank(S.astype(np.float64)) == synth.LOWRANK_RANK
    assert np.abs(S).max() < 2 ** 24 and np.abs(N).max() <= 131070
    # row slices regenerate the same rows
    S2, N2 = synth.lowrank_noise_int(3, rows, cols, row0=10, nrows=7)
    assert np.array_equal(S2, S[10:17]) and np.array_equal(N2, N[10:17])
    a = synth.lowrank_noise_f32(3, 512, 512).astype(np.float64)
    Sf, Nf = synth.lowrank_noise_int(3, 512, 512)
    alpha, beta = synth.lowrank_constants()
    sig = np.linalg.norm(alpha * beta * Sf)
    noi = np.linalg.norm(beta * Nf)
    assert 7.0 < sig / noi < 14.0          # 10:1 amplitude ratio in expectation
    assert abs(np.std(beta * Nf) - 1.0) < 0.02
    assert np.allclose(a, alpha * beta * Sf + beta * Nf, rtol=1e-5, atol=1e-4)


def test_lists():
    l1 = synth.list_1b()
    assert len(l1) == 168
    assert sum(r * c for _, r, c in l1) == 24 * (4 * 2048 * 2048 + 3 * 2048 * 5632)
    assert sum(1 for _, r, c in l1 if r > c) == 24
    l7 = synth.list_7b()
    assert len(l7) == 224
    assert l7[6] == ("l0.down", 14336, 4096)
