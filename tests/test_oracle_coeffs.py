"""Pins of the scalar polynomial, the peak constraint and the coefficient
learner of the oracle (Sec. 2.2, 2.3, 2.4, 3.1.1) and of the FLOP counts of
Table 1."""
import json
import math
import os

import numpy as np
import pytest

from oracle import coeffs as C
from oracle import flops
from synth import learner_uniforms

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("l", [1, 2, 3, 5, 8])
def test_term_derivative_closed_form(l):
    # P6: Eq. eq_gradient against a central difference of Eq. final_polynomial_term
    x = np.linspace(0.01, 0.99, 37)
    hstep = 1e-6
    fd = (C.f_term(x + hstep, l) - C.f_term(x - hstep, l)) / (2 * hstep)
    assert np.allclose(C.f_term_prime(x, l), fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("l", [1, 2, 4, 7, 10])
def test_term_peak(l):
    # P6: the extreme point x* = 1/sqrt(2^l + 1) and its value y* (Sec. 2.2)
    xs, ys = C.peak(l)
    assert abs(C.f_term_prime(xs, l)) < 1e-12
    grid = np.linspace(1e-5, 1 - 1e-5, 2_000_001)
    i = int(np.argmax(C.f_term(grid, l)))
    assert abs(grid[i] - xs) < 1e-5
    assert abs(C.f_term(xs, l) - ys) < 1e-15
    # y* -> e^(-1/2) x* for large l
    if l >= 7:
        assert abs(ys / xs - math.exp(-0.5)) < 3e-3


def test_f_fixed_points():
    w = np.array([0.4, -2.0, 3.1, 8.8, -1.5])
    assert C.f_full(1.0, w) == 1.0      # y -> 1 as x -> 1 (Eq. our_scalar_formula)
    assert C.f_full(0.0, w) == 0.0


@pytest.mark.parametrize("L", [2, 4, 9, 14])
def test_peak_constraint_exact(L):
    # P6: exact w_L makes f(1/sqrt(2^L + 1)) = 1 (Eq. peak)
    rng = np.random.default_rng(L)
    wf = rng.uniform(-1, 1, L - 1)
    w = C.complete(wf, L, "exact")
    xs, _ = C.peak(L)
    assert abs(C.f_full(xs, w) - 1.0) < 1e-10 * max(1.0, abs(w[-1]))


def test_peak_constraint_approximation():
    # Eq. b_approximation: with w_l = 0 (l < L) the printed form approaches the exact one
    errs = []
    for L in (6, 10, 14, 18):
        z = np.zeros(L - 1)
        ex, ap = C.wL_exact(z, L), C.wL_approx(z, L)
        errs.append(abs(ex - ap) / ex)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 2e-3
    # the printed form subtracts sum w_l with weight 1 ...
    L = 16
    rng = np.random.default_rng(2)
    wf = rng.uniform(-1, 1, L - 1)
    assert abs(C.wL_approx(wf, L) - C.wL_approx(np.zeros(L - 1), L) + wf.sum()) < 1e-12
    # ... while the exact solution of f(x*_L) = 1 weighs w_k by f_k(x*)/f_L(x*)
    xs, _ = C.peak(L)
    for k in (1, 8, 15):
        e = np.zeros(L - 1)
        e[k - 1] = 1.0
        dk = C.wL_exact(e, L) - C.wL_exact(np.zeros(L - 1), L)
        assert abs(dk + C.f_term(xs, k) / C.f_term(xs, L)) < 1e-9


@pytest.mark.parametrize("form", ["approx", "exact"])
def test_gradient_finite_difference(form):
    L = 6
    rng = np.random.default_rng(1)
    wf = rng.uniform(-1, 1, L - 1)
    x = learner_uniforms(0, 0, 200)
    g = C.grad(wf, x, L, form)
    for k in range(L - 1):
        e = np.zeros(L - 1)
        e[k] = 1e-6
        fd = (C.loss(wf + e, x, L, form) - C.loss(wf - e, x, L, form)) / 2e-6
        assert abs(g[k] - fd) < 1e-5 * max(1.0, abs(fd))


def test_adam_first_step_is_lr_sign():
    # Adam's bias corrections make the first step lr * g / (|g| + eps') per coordinate
    L = 5
    x = learner_uniforms(0, 0, 1000)
    g0 = C.grad(np.zeros(L - 1), x, L)
    w, _ = C.learn(L, lambda t: x, iters=1, lr=0.1)
    assert np.allclose(w[:-1], -0.1 * np.sign(g0), atol=1e-8)


def test_learner_deterministic_and_descends():
    L = 5
    samp = lambda t: learner_uniforms(0, t, 1000)   # noqa: E731
    w1, _ = C.learn(L, samp, iters=1500, step_size=700)
    w2, _ = C.learn(L, samp, iters=1500, step_size=700)
    assert np.array_equal(w1, w2)
    xe = np.linspace(1e-4, 1 - 1e-4, 20001)
    base = np.mean((C.f_full(xe, C.complete(np.zeros(L - 1), L)) - 1) ** 2)
    fit = np.mean((C.f_full(xe, w1) - 1) ** 2)
    assert fit < 0.8 * base
    # w_L is the printed constraint of the free coefficients
    assert abs(w1[-1] - C.wL_approx(w1[:-1], L)) < 1e-12


def test_stored_coefficients_are_the_learner_output():
    # the committed artefact is what tests/golden/make_coeffs.py writes from the oracle
    with open(os.path.join(GOLDEN, "ifnso_coeffs.json")) as f:
        art = json.load(f)
    L = 4
    w = np.array(art["L"][str(L)]["w"])
    samp = lambda t: learner_uniforms(art["seed"], t, art["samples"])  # noqa: E731
    ref, _ = C.learn(L, samp, iters=art["iters"])
    assert np.allclose(w, ref, rtol=0, atol=1e-12)
    xe = np.linspace(1e-4, 1 - 1e-4, 20001)
    for Ls, ent in art["L"].items():
        Lv = int(Ls)
        wv = np.array(ent["w"])
        assert len(wv) == Lv
        assert abs(wv[-1] - C.wL_approx(wv[:-1], Lv)) < 1e-9 * max(1, abs(wv[-1]))
        assert abs(ent["eval_mse"] - np.mean((C.f_full(xe, wv) - 1) ** 2)) < 1e-12


def test_table1_flops():
    # P8: all nine FLOP entries of Table 1 to four significant figures
    with open(os.path.join(GOLDEN, "table1_flops.json")) as f:
        t = json.load(f)

    def sf4(v):
        return float(f"{v:.3e}")

    for (h, w), on, mu, ours in zip(t["sizes"], t["original_ns"], t["muon_ns"], t["ifnso"]):
        assert sf4(flops.original_ns(h, w, t["original_ns_steps"])) == on
        assert sf4(flops.muon_ns(h, w)) == mu
        assert sf4(flops.ifnso(h, w, t["ifnso_L"])) == ours


def test_nominal_flop_helpers():
    """The product-only counts used for TFLOP/s, tied to Table 1 and to hand counts."""
    with open(os.path.join(GOLDEN, "table1_flops.json")) as f:
        t = json.load(f)
    L = t["ifnso_L"]
    for (h, w), ifn, mu in zip(t["sizes"], t["ifnso"], t["muon_ns"]):
        # IFNSO: Table 1's count less its L h^2 elementwise aggregation
        assert flops.ifnso_nominal(h, w, L) + L * h * h == flops.ifnso(h, w, L)
        assert float(f"{flops.ifnso_nominal(h, w, L) + L * h * h:.3e}") == ifn
    # NS5 with (X X^T)^2 X formed as S (S X): on a square input 4h^2 w + 2h^3 =
    # 6h^2 w, the product part of the printed Muon count; only its 5 x 5hw
    # elementwise terms differ (Table 1, 128 x 128: 6.332e7)
    h = 128
    assert flops.ns5_nominal(h, h) + 25 * h * h == flops.muon_ns(h, h)
    assert float(f"{flops.ns5_nominal(h, h) + 25 * h * h:.3e}") == t["muon_ns"][0]
    # hand counts: one step on a 2 x 3 input is X X^T (2*2*3*2 = 24), S S (2*2*2*2 = 16),
    # B X (24) = 64; an L = 1 IFNSO on 1 x 1 is the Gram and the apply, 2 + 2
    assert flops.ns5_nominal(2, 3, steps=1) == 64
    assert flops.ns5_nominal(2, 3) == 5 * 64
    assert flops.ifnso_nominal(1, 1, 1) == 4
    assert flops.ifnso_nominal(2, 3, 3) == 4 * 4 * 3 + 2 * 2 * 8
