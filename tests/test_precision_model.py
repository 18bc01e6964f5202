"""The precision model behind the FP16 final product, emulated in FP64 on the
CPU: rounding P (Y' in the D basis, Alg. 1) once to FP16 costs several times
less than rounding it to BF16, and the power-of-two-scaled FP16 copy of a BF16
input is exact.  These pin the reasoning the GPU path rests on; the GPU
outputs themselves are compared with the oracle in the -m gpu tests."""
import numpy as np

import synth
from oracle import ifnso as O
from tests.gpu_util import coeffs


def _p_and_scale(A, w):
    """P = (1 + sum w) I - sum_l w_l D_l with D_1 = A A^T / o, D_{l+1} = 2 D_l - D_l^2
    (the D basis of Alg. 1's T_l = I - D_l), and o = ||A A^T||_F."""
    T0 = A @ A.T
    o = np.linalg.norm(T0)
    D = T0 / o
    h = A.shape[0]
    P = (1.0 + np.sum(w)) * np.eye(h) - w[0] * D
    for wl in w[1:]:
        D = 2.0 * D - D @ D
        P -= wl * D
    return P, o


def _round_bf16(x):
    return synth.round_bf16(np.asarray(x, dtype=np.float64))


def test_fp16_p_costs_a_fraction_of_bf16_p():
    """Log-uniform spectra (the hardest inputs of the parity tests) at L = 14:
    one FP16 P costs 5-7e-3 relative (BF16 P about 8 times more, the ratio of
    the two unit roundoffs), inside half the BF16 plans' 2e-2 budget."""
    w = coeffs(14)
    for seed, (h, wd) in [(7, (256, 768)), (8, (512, 512)), (9, (128, 1024))]:
        A = _round_bf16(synth.spectral(seed, h, wd, synth.loguniform_sigma(seed, h)))
        P, o = _p_and_scale(A, w)
        Y = P @ A / np.sqrt(o)
        # the D-basis evaluation is Algorithm 1 itself
        assert O.rel_fro(Y, O.ifnso_alg1(A, w)) < 1e-9
        e16 = O.rel_fro(P.astype(np.float16).astype(np.float64) @ A / np.sqrt(o), Y)
        ebf = O.rel_fro(_round_bf16(P) @ A / np.sqrt(o), Y)
        assert e16 < 1e-2, (seed, e16)
        assert ebf > 6.0 * e16, (seed, ebf, e16)


def test_scaled_fp16_copy_of_a_bf16_input_is_exact():
    rng = np.random.default_rng(3)
    for mag in (1e-6, 1.0, 1e4):
        A = _round_bf16(mag * rng.standard_normal((64, 200)))
        nrm = np.linalg.norm(A)
        s = 2.0 ** int(np.clip(np.floor(np.log2(32768.0 / nrm)), -60, 60))
        As = A * s
        assert np.max(np.abs(As)) <= 32768.0
        copy = As.astype(np.float16).astype(np.float64)
        # exact wherever A s is a normal FP16 value (2^-14 and up); the rest is far below ||A s||
        normal = np.abs(As) >= 2.0 ** -14
        assert np.array_equal(copy[normal], As[normal])
        assert np.linalg.norm(copy - As) <= 2.0 ** -24 * np.sqrt(As.size) + 1e-30
