"""Pins of the FP64 Newton-Schulz oracle (Sec. 1, Eqs. one_iteration_matrix,
one_iteration_scalar, general_eq_matrix, iteration_jordan, polynomial_unify)."""
import numpy as np
import pytest

from oracle import ifnso as I
from oracle import ns
from synth import gaussian, spectral


@pytest.mark.parametrize("steps", [1, 3, 8])
def test_cubic_spectral_map(steps):
    # P7: singular values evolve independently under g (Eq. one_iteration_scalar)
    sig = np.array([9.0, 4.0, 2.0, 1.0, 0.3, 0.05])
    M = spectral(2, 6, 15, sig)
    Y = ns.ns_cubic(M, steps)
    x = sig / np.linalg.norm(sig)
    for _ in range(steps):
        x = ns.cubic_scalar(x)
    assert np.allclose(np.sort(np.linalg.svd(Y, compute_uv=False)), np.sort(np.abs(x)), atol=1e-12)
    # U and V are unchanged: Y = U diag(g^N(x)) V^T
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    assert np.allclose(Y, (U * x) @ Vt, atol=1e-12)


def test_quintic_spectral_map():
    sig = np.array([5.0, 2.0, 1.0, 0.1])
    M = spectral(4, 4, 9, sig)
    Y = ns.ns_quintic(M, 5)
    x = ns.ns_scalar(sig / np.linalg.norm(sig), ns.MUON_ABC, 5)
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    assert np.allclose(Y, (U * x) @ Vt, atol=1e-12)


def test_muon_constants_and_slope():
    # a = 3.4445 multiplies X: the slope of the quintic map at 0
    a, b, c = ns.MUON_ABC
    assert (a, b, c) == (3.4445, -4.7750, 2.0315)
    eps = 1e-7
    assert abs(ns.ns_scalar(eps, ns.MUON_ABC, 1) / eps - 3.4445) < 1e-9


@pytest.mark.parametrize("steps", [2, 3])
def test_unified_polynomial(steps):
    # N steps equal one odd polynomial of degree 3^N (Eq. polynomial_unify / old_unified_formula)
    b = ns.unified_coefficients(ns.CUBIC, steps)
    assert len(b) - 1 == 3 ** steps
    assert np.all(b[0::2] == 0.0)
    M = gaussian(1, 5, 12)
    A = M / np.linalg.norm(M)
    S = A @ A.T
    Y = np.zeros_like(A)
    SnX = A
    for n in range(0, (len(b) - 1) // 2 + 1):
        if n > 0:
            SnX = S @ SnX
        Y += b[2 * n + 1] * SnX
    assert np.allclose(Y, ns.ns_cubic(M, steps), atol=1e-13)


def test_cubic_converges_to_polar():
    sig = np.array([1.0, 0.8, 0.5, 0.3])
    M = spectral(7, 4, 10, sig)
    Y = ns.ns_cubic(M, 40)
    assert np.allclose(Y, I.polar_factor(M), atol=1e-12)


def test_tall_input_shape_and_zero():
    M = gaussian(3, 20, 7)
    Y = ns.ns_quintic(M, 5)
    assert Y.shape == M.shape
    assert np.allclose(Y, ns.ns_quintic(M.T, 5).T, atol=1e-14)
    assert np.all(ns.ns_quintic(np.zeros((3, 5)), 5) == 0.0)
