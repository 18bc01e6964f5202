"""One Muon step around IFNSO in FP64 (test infrastructure only; see
oracle/__init__.py).

The paper trains with Muon (Sec. 3.3) but does not write out its momentum;
this follows Muon's published form.  For a gradient G, momentum buffer M and
weights W (rows x cols):

    M' = beta M + G
    U  = G + beta M'   (Nesterov)   or   M'
    W' = W - lr sqrt(max(1, rows / cols)) Y,    Y = Algorithm 1 applied to U.

Parity status: the momentum and update formulas have no printed values to pin
them; tests/test_oracle_muon.py pins the special cases that reduce them to
pinned pieces (beta = 0 gives W - lr s Y(G); lr = 0 leaves W; the Nesterov
input expands to (1 + beta) G + beta^2 M).
"""
from __future__ import annotations

import numpy as np

from .ifnso import ifnso_alg1


def shape_factor(rows: int, cols: int) -> float:
    """sqrt(max(1, rows / cols)): Muon's scale of the orthogonalized update."""
    return float(np.sqrt(max(1.0, rows / cols)))


def momentum(G, M, beta: float, nesterov: bool):
    """(M', U): the momentum buffer after the step and the matrix that is orthogonalized."""
    G = np.asarray(G, dtype=np.float64)
    M1 = beta * np.asarray(M, dtype=np.float64) + G
    U = G + beta * M1 if nesterov else M1
    return M1, U


def update(W, U, w, lr: float):
    """W - lr sqrt(max(1, rows / cols)) Y with Y = Algorithm 1 on U (coefficients w_1..w_L)."""
    W = np.asarray(W, dtype=np.float64)
    rows, cols = W.shape
    return W - lr * shape_factor(rows, cols) * ifnso_alg1(U, w)


def muon_step(G, M, W, w, beta: float, nesterov: bool, lr: float):
    """(M', U, W') of one step."""
    M1, U = momentum(G, M, beta, nesterov)
    return M1, U, update(W, U, w, lr)
