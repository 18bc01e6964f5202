"""Seeded synthetic inputs shaped like the paper's workloads.

Nothing here computes any step of the orthogonalisation method: these
functions only build input matrices (and the lists of shapes they come in).
Both the FP64 oracle tests and the CUDA path take their inputs from here.

Recipes
-------
* ``gaussian``: i.i.d. N(0, 1) entries from ``numpy.random.default_rng(seed)``
  (the paper's "randomly generated" matrices, Sec. 3.2; the distribution is
  not stated there, N(0, 1) is the reading used).
* ``spectral``: U diag(sigma) V^T with Haar U (h x h) and a Haar-distributed
  Stiefel V (w x h), both from QR of Gaussian matrices with the sign fix of
  F. Mezzadri, "How to generate random matrices from the classical compact
  groups", Notices AMS 54 (2007).
* ``lowrank_noise``: rank-32 signal plus noise at a 10:1 amplitude ratio,
  built from Philox4x32-10 integers so that every element is produced by the
  same sequence of correctly rounded FP32 operations on the CPU and on the GPU
  (bit-identical after round-to-nearest-even to BF16).
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10, uniform24, uniform53

# Philox key tags (second key word) for the different streams.
TAG_LEFT = 0x4C524B31   # low-rank left factor
TAG_RIGHT = 0x4C524B32  # low-rank right factor
TAG_NOISE = 0x4E4F4953  # additive noise
TAG_LEARN = 0x4C45524E  # scalar samples of the coefficient objective

LOWRANK_RANK = 32
# variance of a sum of four uniform bytes / four uniform 16-bit halves
_VAR_BYTES4 = 4.0 * (256.0 ** 2 - 1.0) / 12.0
_VAR_HALF4 = 4.0 * (65536.0 ** 2 - 1.0) / 12.0


def gaussian(seed: int, rows: int, cols: int) -> np.ndarray:
    """i.i.d. N(0,1), FP64."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def haar_stiefel(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """n x k matrix with orthonormal columns, Haar distributed (Mezzadri 2007)."""
    z = rng.standard_normal((n, k))
    q, r = np.linalg.qr(z)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def spectral(seed: int, h: int, w: int, sigma: np.ndarray) -> np.ndarray:
    """U diag(sigma) V^T (h x w, h <= w), FP64."""
    assert h <= w and sigma.shape == (h,)
    rng = np.random.default_rng(seed)
    U = haar_stiefel(rng, h, h)
    V = haar_stiefel(rng, w, h)
    return (U * sigma[None, :]) @ V.T


def loguniform_sigma(seed: int, h: int, lo_exp: float = -4.0, hi_exp: float = 0.0,
                     scale: float = 1e3) -> np.ndarray:
    """sigma_i = scale * 10^U(lo_exp, hi_exp): log-uniform in [1e-4, 1] x 1e3."""
    rng = np.random.default_rng(seed + 7919)
    return scale * 10.0 ** rng.uniform(lo_exp, hi_exp, size=h)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest even (finite inputs)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + ((b >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)) >> np.uint64(16)
    return b.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Values of x after RN-even rounding to BF16, as FP64."""
    return bf16_bits_to_f64(to_bf16_bits(np.asarray(x, dtype=np.float32)))


def lowrank_constants(snr: float = 10.0):
    """(alpha, beta) FP32 constants of ``lowrank_noise``: signal std snr, noise std 1."""
    std_s = math.sqrt(LOWRANK_RANK * _VAR_BYTES4 * _VAR_BYTES4)
    std_n = math.sqrt(_VAR_HALF4)
    return np.float32(snr * std_n / std_s), np.float32(1.0 / std_n)


def _byte_sum(word: np.ndarray) -> np.ndarray:
    w = word.astype(np.int64)
    return (w & 0xFF) + ((w >> 8) & 0xFF) + ((w >> 16) & 0xFF) + ((w >> 24) & 0xFF) - 510


def lowrank_factor(seed: int, n: int, tag: int) -> np.ndarray:
    """n x 32 integer factor: entry (i, r) = sum of the 4 bytes of Philox word 0
    at counter (i, r, 0, 0), key (seed, tag), minus 510."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    r = np.arange(LOWRANK_RANK, dtype=np.uint64)[None, :]
    w0, _, _, _ = philox4x32_10(i, r, 0, 0, seed, tag)
    return _byte_sum(w0)


def lowrank_noise_int(seed: int, rows: int, cols: int, row0: int = 0, nrows: int | None = None):
    """Integer signal S = L R^T and noise N for rows [row0, row0 + nrows)."""
    if nrows is None:
        nrows = rows - row0
    Lf = lowrank_factor(seed, rows, TAG_LEFT)[row0:row0 + nrows]
    Rf = lowrank_factor(seed, cols, TAG_RIGHT)
    S = (Lf.astype(np.float64) @ Rf.astype(np.float64).T).astype(np.int64)  # exact: |S| < 2^24
    i = np.arange(row0, row0 + nrows, dtype=np.uint64)[:, None]
    j = np.arange(cols, dtype=np.uint64)[None, :]
    w0, w1, _, _ = philox4x32_10(j, i, 0, 0, seed, TAG_NOISE)
    a = w0.astype(np.int64)
    b = w1.astype(np.int64)
    N = (a & 0xFFFF) + (a >> 16) + (b & 0xFFFF) + (b >> 16) - 131070
    return S, N


def lowrank_noise_f32(seed: int, rows: int, cols: int, snr: float = 10.0,
                      row0: int = 0, nrows: int | None = None) -> np.ndarray:
    """FP32 values fl(fl(fl(alpha*S) + N) * beta); every operation correctly rounded."""
    alpha, beta = lowrank_constants(snr)
    S, N = lowrank_noise_int(seed, rows, cols, row0, nrows)
    t = (alpha * S.astype(np.float32)).astype(np.float32)
    t = (t + N.astype(np.float32)).astype(np.float32)
    return (t * beta).astype(np.float32)


def lowrank_noise_bf16(seed: int, rows: int, cols: int, snr: float = 10.0,
                       row0: int = 0, nrows: int | None = None) -> np.ndarray:
    """BF16 bit patterns (uint16) of ``lowrank_noise_f32``."""
    return to_bf16_bits(lowrank_noise_f32(seed, rows, cols, snr, row0, nrows))


# --- weight-gradient lists of synthetic transformers ------------------------

def transformer_list(layers: int, d: int, ffn: int, attn_mats: int = 4):
    """[(name, rows, cols)] in layer order: attention projections d x d,
    gate and up d x ffn, down ffn x d (tall)."""
    out = []
    for layer in range(layers):
        for nm in ("q", "k", "v", "o")[:attn_mats]:
            out.append((f"l{layer}.{nm}", d, d))
        out.append((f"l{layer}.gate", d, ffn))
        out.append((f"l{layer}.up", d, ffn))
        out.append((f"l{layer}.down", ffn, d))
    return out


def list_1b():
    """24 layers x {Q,K,V,O 2048^2; gate, up 2048x5632; down 5632x2048}: 168 matrices."""
    return transformer_list(24, 2048, 5632)


def list_7b():
    """32 layers x {4 x 4096^2; gate, up 4096x14336; down 14336x4096}: 224 matrices."""
    return transformer_list(32, 4096, 14336)


def learner_uniforms(seed: int, iteration: int, count: int) -> np.ndarray:
    """The `count` FP64 samples in (0, 1) that the coefficient learner draws at one
    iteration: Philox counter (j, iteration, 0, 0), key (seed, TAG_LEARN)."""
    j = np.arange(count, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(j, np.uint64(iteration), 0, 0, seed, TAG_LEARN)
    return uniform53(w0, w1)


# --- spectra of the coefficient-proposal training set -----------------------

MLP_FAMILIES = ("loguniform", "powerlaw", "clustered")


def mlp_spectrum(seed: int):
    """One synthetic matrix of the coefficient-proposal data set, as a spectrum.

    h ~ U{64..1024}; w = round(h r), r ~ U[1, 4]; family chosen uniformly:
      loguniform  sigma_i = 10^U(-4, 0)
      powerlaw    sigma_i = i^-alpha, alpha ~ U[0.5, 2]
      clustered   2..4 centres 10^U(-4, 0), sigma = centre * exp(0.1 N(0, 1))
    times an overall scale 10^U(-2, 2).  Returns (h, w, sigma sorted
    descending, family index).
    """
    rng = np.random.default_rng(seed)
    h = int(rng.integers(64, 1025))
    w = int(round(h * rng.uniform(1.0, 4.0)))
    fam = int(rng.integers(0, 3))
    if fam == 0:
        sig = 10.0 ** rng.uniform(-4.0, 0.0, size=h)
    elif fam == 1:
        alpha = rng.uniform(0.5, 2.0)
        sig = np.arange(1, h + 1, dtype=np.float64) ** (-alpha)
    else:
        k = int(rng.integers(2, 5))
        centres = 10.0 ** rng.uniform(-4.0, 0.0, size=k)
        which = rng.integers(0, k, size=h)
        sig = centres[which] * np.exp(0.1 * rng.standard_normal(h))
    sig = np.sort(sig)[::-1] * 10.0 ** rng.uniform(-2.0, 2.0)
    return h, w, sig.copy(), fam


def mlp_matrix(seed: int):
    """The matrix U diag(sigma) V^T (h x w) of ``mlp_spectrum(seed)``, FP64."""
    h, w, sig, fam = mlp_spectrum(seed)
    return spectral(seed + 17, h, w, sig)


__all__ = [
    "MLP_FAMILIES", "mlp_spectrum", "mlp_matrix",
    "gaussian", "haar_stiefel", "spectral", "loguniform_sigma", "to_bf16_bits",
    "bf16_bits_to_f64", "round_bf16", "lowrank_constants", "lowrank_factor",
    "lowrank_noise_int", "lowrank_noise_f32", "lowrank_noise_bf16", "transformer_list",
    "list_1b", "list_7b", "learner_uniforms", "uniform24", "LOWRANK_RANK",
    "TAG_LEFT", "TAG_RIGHT", "TAG_NOISE", "TAG_LEARN",
]
