"""FLOP counts of Table 1 (Sec. 3.4), reconstructed so that all nine printed
entries are reproduced to four significant figures
(test infrastructure only; see oracle/__init__.py).

Convention: a product of an (m x k) and a (k x n) matrix costs 2mkn; adding
or scaling an m x n matrix costs mn.
"""
from __future__ import annotations


def original_ns(h: int, w: int, N: int = 8) -> int:
    """N cubic steps, each: X X^T (2h^2 w), 3I - S (h^2), (.)X (2h^2 w), the
    scalar 1/2 and ... (2hw): N (4h^2 w + 2hw + h^2)."""
    return N * (4 * h * h * w + 2 * h * w + h * h)


def muon_ns(h: int, w: int, steps: int = 5) -> int:
    """Quintic steps with (XX^T)^2 X formed as two more h x h by h x w
    products: steps * (6h^2 w + 5hw)."""
    return steps * (6 * h * h * w + 5 * h * w)


def ifnso(h: int, w: int, L: int = 14) -> int:
    """Gram (2h^2 w) + (L - 1) squarings (2h^3 each) + aggregation (L h^2) +
    apply (2h^2 w): 4h^2 w + 2(L - 1)h^3 + L h^2."""
    return 4 * h * h * w + 2 * (L - 1) * h ** 3 + L * h * h


def ifnso_nominal(h: int, w: int, L: int) -> int:
    """Matrix-product FLOPs of IFNSO only: 4h^2 w + 2(L - 1) h^3."""
    return 4 * h * h * w + 2 * (L - 1) * h ** 3


def ns5_nominal(h: int, w: int, steps: int = 5) -> int:
    """Matrix-product FLOPs of an efficient quintic step (X X^T, (XX^T)^2, B X):
    steps * (4h^2 w + 2h^3)."""
    return steps * (4 * h * h * w + 2 * h ** 3)
