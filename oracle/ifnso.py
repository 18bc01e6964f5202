"""IFNSO in FP64 on the CPU (test infrastructure only; see oracle/__init__.py).

Notation follows the paper: M is the input, A its orientation with h <= w,
T_l the Gram / complement sequence, o = ||T_0||_F, w_1..w_L the learned
coefficients, Y the output.
"""
from __future__ import annotations

import numpy as np


def orient(M):
    """Eq. 1 (Sec. 1) and the initialisation of Algorithm 1: A = M^T if
    h_input > w_input, else A = M (a square input is not transposed)."""
    M = np.asarray(M, dtype=np.float64)
    if M.shape[0] > M.shape[1]:
        return M.T.copy(), True
    return M.copy(), False


def exponents(L: int):
    """Exponential term selection (Sec. 2.2): n_0 = 0, n_l = 2^(l-1), l = 1..L."""
    return [0] + [2 ** (l - 1) for l in range(1, L + 1)]


def _deorient(Y, transposed):
    return Y.T.copy() if transposed else Y


def scale_of(A, scale: str = "gram"):
    """The scalar the input is divided by.

    "gram": ||A A^T||_F^(1/2), Gelfand's bound with q = 1 (Eq. new_scale_formula,
            Sec. 2), which Algorithm 1 uses through o = ||T_0||_F.
    "frob": ||A||_F, the classical Newton-Schulz scaling (Eq. constraint, Sec. 1).
    "gelfand2": ||(A A^T)^2||_F^(1/4), the bound of Eq. gelfand_formula with q = 2
            (the scaling of Eq. scale_formula_function before the paper sets q = 1).
    """
    if scale == "gram":
        return np.sqrt(np.linalg.norm(A @ A.T, "fro"))
    if scale == "frob":
        return np.linalg.norm(A, "fro")
    if scale == "gelfand2":
        G = A @ A.T
        return np.linalg.norm(G @ G, "fro") ** 0.25
    raise ValueError(scale)


def ifnso_alg1(M, w, scale: str = "gram"):
    """Algorithm 1 step by step, in the T basis.

    T_0 = A A^T, o = ||T_0||_F, T_1 = I - T_0/o, T_l = T_{l-1} T_{l-1} (l = 2..L),
    Y' = I + sum_l w_l T_l, Y = Y' A / sqrt(o)  (Sec. 2.4, T_l definition,
    aggregation and Algorithm 1).  ``w`` holds w_1..w_L.  With scale="frob" the
    divisor sqrt(o) is replaced by ||A||_F (so T_1 = I - A A^T/||A||_F^2); with
    scale="gelfand2" by ||T_0^2||_F^(1/4) (o = ||T_0^2||_F^(1/2)).
    The output has the shape of M.  A zero input returns zeros.
    """
    A, tr = orient(M)
    w = np.asarray(w, dtype=np.float64)
    L = len(w)
    h = A.shape[0]
    T0 = A @ A.T
    s2 = scale_of(A, scale) ** 2
    if s2 == 0.0:
        return np.zeros_like(np.asarray(M, dtype=np.float64))
    I = np.eye(h)
    T = I - T0 / s2
    Yp = I + w[0] * T
    for l in range(2, L + 1):
        T = T @ T
        Yp = Yp + w[l - 1] * T
    Y = Yp @ A / np.sqrt(s2)
    return _deorient(Y, tr)


def ifnso_dbasis(M, w, scale: str = "gram"):
    """The same polynomial written with D_l = I - T_l.

    D_1 = T_0/o and, since T_{l+1} = T_l^2, D_{l+1} = 2 D_l - D_l^2.  Then
    Y' = I + sum w_l (I - D_l) = (1 + sum w_l) I - sum w_l D_l  and
    Y = Y' A / sqrt(o).  Algebraically identical to ``ifnso_alg1``.
    """
    A, tr = orient(M)
    w = np.asarray(w, dtype=np.float64)
    L = len(w)
    h = A.shape[0]
    G = A @ A.T
    s2 = scale_of(A, scale) ** 2
    if s2 == 0.0:
        return np.zeros_like(np.asarray(M, dtype=np.float64))
    D = G / s2
    c0 = 1.0 + float(np.sum(w))
    P = c0 * np.eye(h) - w[0] * D
    for l in range(2, L + 1):
        D = 2.0 * D - D @ D
        P = P - w[l - 1] * D
    Y = P @ A / np.sqrt(s2)
    return _deorient(Y, tr)


def f_scalar(x, w):
    """f(x) = x + sum_{l=1}^L w_l x (1 - x^2)^(2^(l-1))  (Eq. sum_equation, Sec. 2.3;
    Eq. final_polynomial_term for the individual terms)."""
    x = np.asarray(x, dtype=np.float64)
    y = x.copy()
    for l, wl in enumerate(np.asarray(w, dtype=np.float64), start=1):
        y = y + wl * x * (1.0 - x * x) ** (2 ** (l - 1))
    return y


def ifnso_spectral(M, w, scale: str = "gram"):
    """Each singular value maps independently (Sec. 2.1): with A = U S V^T,
    x_i = s_i / scale, Y = U diag(f(x_i)) V^T."""
    A, tr = orient(M)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    sc = scale_of(A, scale)
    if sc == 0.0:
        return np.zeros_like(np.asarray(M, dtype=np.float64))
    y = f_scalar(s / sc, w)
    Y = (U * y[None, :]) @ Vt
    return _deorient(Y, tr)


def polar_factor(M):
    """U V^T from the thin SVD of the oriented input, returned in M's shape:
    the limit the Newton-Schulz iterations approach (Sec. 1)."""
    A, tr = orient(M)
    U, _, Vt = np.linalg.svd(A, full_matrices=False)
    return _deorient(U @ Vt, tr)


def orth_error(Y):
    """Error = ||Y Y^T - I||_F over the h x h product of the oriented output
    (Sec. 3.2, error metric)."""
    Yo, _ = orient(Y)
    h = Yo.shape[0]
    return float(np.linalg.norm(Yo @ Yo.T - np.eye(h), "fro"))


def polar_distance(Y, M):
    """||Y - U V^T||_F, U V^T the polar factor of M."""
    return float(np.linalg.norm(np.asarray(Y, dtype=np.float64) - polar_factor(M), "fro"))


def rel_fro(Y, Yref):
    """Relative Frobenius error ||Y - Yref||_F / ||Yref||_F."""
    Yref = np.asarray(Yref, dtype=np.float64)
    d = np.linalg.norm(np.asarray(Y, dtype=np.float64) - Yref)
    n = np.linalg.norm(Yref)
    return float(d / n) if n > 0 else float(d)


def brute_force(M, w, exps=None, scale: str = "gram", dps: int = 50):
    """Eq. generalized_matrix_formula, sum_l w_l (I - X X^T)^{n_l} X with w_0 = 1,
    evaluated in mpmath at ``dps`` digits by naive repeated multiplication
    (no squaring).  For tiny matrices only."""
    import mpmath as mp

    with mp.workdps(dps):
        A, tr = orient(M)
        h, wd = A.shape
        Am = mp.matrix([[mp.mpf(float(v)) for v in row] for row in A])
        G = Am * Am.T
        if scale == "gram":
            s2 = mp.sqrt(sum(G[i, j] ** 2 for i in range(h) for j in range(h)))
        elif scale == "gelfand2":
            G2 = G * G
            s2 = mp.sqrt(mp.sqrt(sum(G2[i, j] ** 2 for i in range(h) for j in range(h))))
        else:
            s2 = sum(Am[i, j] ** 2 for i in range(h) for j in range(wd))
        X = Am / mp.sqrt(s2)
        I = mp.eye(h)
        C = I - X * X.T
        L = len(w)
        if exps is None:
            exps = exponents(L)
        coeffs = [mp.mpf(1)] + [mp.mpf(float(v)) for v in w]
        Y = mp.zeros(h, wd)
        for n, c in zip(exps, coeffs):
            Pw = mp.eye(h)
            for _ in range(n):
                Pw = Pw * C
            Y = Y + c * (Pw * X)
        out = np.array([[float(Y[i, j]) for j in range(wd)] for i in range(h)])
    return _deorient(out, tr)
