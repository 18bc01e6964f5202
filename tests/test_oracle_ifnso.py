"""Pins of the FP64 IFNSO oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong scale) fails at least one of them.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from oracle import ifnso as I
from synth import gaussian, haar_stiefel, spectral

W4 = np.array([0.3, -0.7, 1.9, 2.4])       # arbitrary coefficients w_1..w_4
W6 = np.array([0.5, 0.4, 0.9, -1.1, 2.0, 7.5])


def _paths(M, w, scale="gram"):
    return (I.ifnso_alg1(M, w, scale), I.ifnso_dbasis(M, w, scale), I.ifnso_spectral(M, w, scale))


@pytest.mark.parametrize("shape", [(12, 30), (30, 12), (17, 17), (1, 9), (9, 1)])
@pytest.mark.parametrize("scale", ["gram", "frob", "gelfand2"])
def test_three_paths_agree(shape, scale):
    # P1: Algorithm 1 (T basis), the D basis and the SVD evaluation of f agree (Sec. 2.1, 2.4)
    M = gaussian(3, *shape)
    a, b, c = _paths(M, W6, scale)
    assert a.shape == M.shape
    assert I.rel_fro(b, a) < 1e-12
    assert I.rel_fro(c, a) < 1e-10


def test_three_paths_agree_ill_conditioned():
    sig = 10.0 ** np.linspace(-6, 0, 20)
    M = spectral(1, 20, 44, sig)
    a, b, c = _paths(M, W6)
    assert I.rel_fro(b, a) < 1e-10
    assert I.rel_fro(c, a) < 1e-10


def test_rank_one_returns_uv():
    # P2: sigma u v^T has a single singular value, x = 1 under both scalings, f(1) = 1
    rng = np.random.default_rng(5)
    u = rng.standard_normal(7)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(19)
    v /= np.linalg.norm(v)
    M = 3.7 * np.outer(u, v)
    for scale in ("gram", "frob", "gelfand2"):
        Y = I.ifnso_alg1(M, W6, scale)
        assert np.allclose(Y, np.outer(u, v), atol=1e-12)


@pytest.mark.parametrize("h,w", [(4, 10), (16, 16), (10, 4)])
def test_orthonormal_rows_closed_form(h, w):
    # P3: Q Q^T = I gives o = ||I||_F = sqrt(h), x = h^(-1/4) (gram); ||Q||_F = sqrt(h), x = h^(-1/2) (frob)
    rng = np.random.default_rng(h * 100 + w)
    hh, ww = min(h, w), max(h, w)
    Q = haar_stiefel(rng, ww, hh).T          # hh x ww, orthonormal rows
    M = Q if h <= w else Q.T
    Yg = I.ifnso_alg1(M, W4, "gram")
    Yf = I.ifnso_alg1(M, W4, "frob")
    xg = hh ** -0.25
    xf = hh ** -0.5
    assert np.allclose(Yg, C.f_full(xg, W4) * M, atol=1e-12)
    assert np.allclose(Yf, C.f_full(xf, W4) * M, atol=1e-12)
    # Gelfand q = 2: (Q Q^T)^2 = I, ||I||_F^(1/4) = h^(1/8), x = h^(-1/8)
    Y2 = I.ifnso_alg1(M, W4, "gelfand2")
    assert np.allclose(Y2, C.f_full(hh ** -0.125, W4) * M, atol=1e-12)


def test_single_row_is_normalised():
    # P4: h = 1: x = 1 under both scalings, Y = a/||a||
    a = gaussian(2, 1, 13)
    for scale in ("gram", "frob"):
        assert np.allclose(I.ifnso_alg1(a, W6, scale), a / np.linalg.norm(a), atol=1e-14)


@pytest.mark.parametrize("M", [
    np.array([[3, -1, 2], [0, 4, 1], [-2, 1, 5]], dtype=float),
    None,
])
def test_brute_force_mpmath(M):
    # P5: naive repeated multiplication of (I - X X^T) at 50 digits (Eq. generalized_matrix_formula)
    pytest.importorskip("mpmath")
    if M is None:
        M = gaussian(11, 4, 8)
    for scale in ("gram", "frob", "gelfand2"):
        ref = I.brute_force(M, W4, scale=scale)
        assert I.rel_fro(I.ifnso_alg1(M, W4, scale), ref) < 1e-12
        assert I.rel_fro(I.ifnso_dbasis(M, W4, scale), ref) < 1e-12
        ref_t = I.brute_force(M.T, W4, scale=scale)
        assert I.rel_fro(I.ifnso_alg1(M.T, W4, scale), ref_t) < 1e-12


def test_gelfand_bounds():
    # Eq. gelfand_formula: sigma_1 <= ||(A A^T)^q||_F^(1/(2q)), and the bound
    # tightens from q = 1 to q = 2; h equal singular values s give s h^(1/(4q))
    for seed, shape in [(1, (8, 20)), (2, (15, 15)), (3, (30, 6))]:
        A = I.orient(gaussian(seed, *shape))[0]
        s1 = np.linalg.svd(A, compute_uv=False)[0]
        g1, g2 = I.scale_of(A, "gram"), I.scale_of(A, "gelfand2")
        assert s1 <= g2 * (1 + 1e-14) and g2 <= g1 * (1 + 1e-14)
    rng = np.random.default_rng(4)
    Q = haar_stiefel(rng, 12, 5).T
    for q, name in [(1, "gram"), (2, "gelfand2")]:
        assert np.isclose(I.scale_of(2.5 * Q, name), 2.5 * 5 ** (1 / (4 * q)), rtol=1e-14)


def test_orientation_and_transpose():
    # Eq. 1: Y(M^T) = Y(M)^T; a tall input is processed as its transpose
    M = gaussian(4, 25, 9)
    assert np.allclose(I.ifnso_alg1(M.T, W6), I.ifnso_alg1(M, W6).T, atol=1e-13)


def test_orthogonal_equivariance():
    # Y(Q1 M Q2) = Q1 Y(M) Q2 for orthogonal Q1, Q2: fails for a transposed operand
    rng = np.random.default_rng(8)
    M = gaussian(9, 6, 11)
    Q1 = haar_stiefel(rng, 6, 6)
    Q2 = haar_stiefel(rng, 11, 11)
    assert np.allclose(I.ifnso_alg1(Q1 @ M @ Q2, W6), Q1 @ I.ifnso_alg1(M, W6) @ Q2, atol=1e-12)


def test_scale_invariance_and_zero():
    M = gaussian(6, 5, 9)
    assert np.allclose(I.ifnso_alg1(123.0 * M, W6), I.ifnso_alg1(M, W6), atol=1e-12)
    Z = np.zeros((5, 9))
    assert np.all(I.ifnso_alg1(Z, W6) == 0.0)
    assert np.all(I.ifnso_dbasis(Z, W6) == 0.0)


def test_polar_factor_and_errors():
    rng = np.random.default_rng(10)
    U = haar_stiefel(rng, 6, 6)
    V = haar_stiefel(rng, 14, 6)
    sig = np.array([5.0, 3.0, 1.0, 0.5, 0.1, 0.01])
    M = (U * sig) @ V.T
    assert np.allclose(I.polar_factor(M), U @ V.T, atol=1e-12)
    assert I.orth_error(U @ V.T) < 1e-13
    # error metric of Sec. 3.2 on c * (orthonormal rows) is |c^2 - 1| sqrt(h)
    assert abs(I.orth_error(0.5 * (U @ V.T)) - 0.75 * np.sqrt(6)) < 1e-12
    assert abs(I.polar_distance(2.0 * (U @ V.T), M) - np.sqrt(6)) < 1e-12


def test_exponents():
    assert I.exponents(4) == [0, 1, 2, 4, 8]
    assert I.exponents(1) == [0, 1]


def test_rel_fro_hand_computed():
    # the metric every parity assertion goes through, on values worked by hand
    assert I.rel_fro(np.array([3.0, 4.0]), np.array([0.0, 5.0])) == pytest.approx(np.sqrt(10.0) / 5.0, rel=1e-15)
    R = np.array([[1.0, -2.0], [2.0, 4.0]])            # ||R||_F = 5
    assert I.rel_fro(R, R) == 0.0
    assert I.rel_fro(2.0 * R, R) == pytest.approx(1.0, rel=1e-15)
    assert I.rel_fro(R + np.array([[0.0, 0.0], [0.0, 1.0]]), R) == pytest.approx(0.2, rel=1e-15)
    assert I.rel_fro(R.T, R) == pytest.approx(np.sqrt(32.0) / 5.0, rel=1e-15)   # not symmetric: a transposed operand shows
    # a zero reference gives the absolute error
    assert I.rel_fro(np.array([3.0, 4.0]), np.zeros(2)) == pytest.approx(5.0, rel=1e-15)
    # invariant under a common scale, and not symmetric in its arguments
    assert I.rel_fro(7.0 * np.array([1.0, 2.0]), 7.0 * np.array([1.0, 3.0])) == pytest.approx(1.0 / np.sqrt(10.0))
    assert I.rel_fro(np.array([1.0, 3.0]), np.array([1.0, 2.0])) == pytest.approx(1.0 / np.sqrt(5.0))
