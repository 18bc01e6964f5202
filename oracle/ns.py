"""Newton-Schulz iterations in FP64 (test infrastructure only; see oracle/__init__.py)."""
from __future__ import annotations

import numpy as np

from .ifnso import orient, _deorient

# Muon's quintic coefficients (a, b, c) multiplying X, (XX^T)X, (XX^T)^2 X
# (Eq. iteration_jordan, Sec. 1; the coefficient of X is written a_0 there and
# a_1 in Eq. general_eq_matrix: it is the first one).
MUON_ABC = (3.4445, -4.7750, 2.0315)
CUBIC = (1.5, -0.5)


def ns_generic(M, a, steps: int):
    """X_0 = A/||A||_F (Eq. constraint), then ``steps`` times
    X_{k+1} = sum_{n=0}^{len(a)-1} a[n] (X_k X_k^T)^n X_k  (Eq. general_eq_matrix).
    Output in M's shape.  A zero input returns zeros."""
    A, tr = orient(M)
    nrm = np.linalg.norm(A, "fro")
    if nrm == 0.0:
        return np.zeros_like(np.asarray(M, dtype=np.float64))
    X = A / nrm
    for _ in range(steps):
        S = X @ X.T
        acc = a[0] * X
        SnX = X
        for n in range(1, len(a)):
            SnX = S @ SnX
            acc = acc + a[n] * SnX
        X = acc
    return _deorient(X, tr)


def ns_cubic(M, steps: int):
    """Classical iteration X_{k+1} = 1/2 (3I - X_k X_k^T) X_k (Eq. one_iteration_matrix)."""
    return ns_generic(M, CUBIC, steps)


def ns_quintic(M, steps: int = 5, abc=MUON_ABC):
    """Muon's quintic iteration (Eq. iteration_jordan) for ``steps`` steps."""
    return ns_generic(M, abc, steps)


def ns_scalar(x, a, steps: int):
    """The scalar map p(x) = sum a[n] x^(2n+1) (Eq. general_eq_scalar) iterated
    ``steps`` times (Eq. N_fold)."""
    x = np.asarray(x, dtype=np.float64)
    for _ in range(steps):
        x = sum(c * x ** (2 * n + 1) for n, c in enumerate(a))
    return x


def cubic_scalar(s):
    """g(sigma) = 1.5 sigma - 0.5 sigma^3 (Eq. one_iteration_scalar)."""
    s = np.asarray(s, dtype=np.float64)
    return 1.5 * s - 0.5 * s ** 3


def unified_coefficients(a, steps: int):
    """Coefficients b_{2n+1} of the single odd polynomial that equals ``steps``
    iterations of p (Eq. polynomial_unify): composition of polynomials in
    exact integer-free FP64 arithmetic (numpy.polynomial)."""
    from numpy.polynomial import polynomial as P

    p = np.zeros(2 * len(a))
    for n, c in enumerate(a):
        p[2 * n + 1] = c
    q = np.array([0.0, 1.0])
    for _ in range(steps):
        # q <- p(q)
        r = np.zeros(1)
        qp = np.array([1.0])
        for k in range(len(p)):
            if p[k] != 0.0:
                r = P.polyadd(r, p[k] * qp)
            qp = P.polymul(qp, q)
        q = r
    return q
