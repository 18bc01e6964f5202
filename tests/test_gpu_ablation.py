"""The L ablation on the Table 1 shapes (Sec. 3.4, Table 1) through the C ABI,
against the FP64 oracle: for each L the batch of 128 x {128, 512, 1024}
N(0,1) matrices goes through one FP32 call and one BF16 call (the runs that
`bench.py --ablation` times), and every result matches the oracle's."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from oracle import ns as ONS
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(128, 128), (128, 512), (128, 1024)]


def run(dtype, L):
    import torch

    F = lib()
    mats = [synth.gaussian(s, h, w) for s, (h, w) in enumerate(SHAPES)]
    xs = [to_dev(M, dtype) for M in mats]
    ys = [torch.empty_like(x) for x in xs]
    plan = F.Plan(128, 1024, dtype, L=L)
    w = coeffs(L)
    plan.orthogonalize(F.Batch(xs), np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    return [to_np(x) for x in xs], [to_np(y) for y in ys], w


def tol(dtype, L, h, w):
    """2e-2 for BF16.  FP32: 1e-5, except on the square N(0,1) input at large
    L.  Its smallest singular values are tiny, and there D_{l+1} ~ 2 D_l, so
    the FP32 rounding of D_1 (unit roundoff 2^-24) grows by up to 2^(L-1)
    before it reaches the result: 1.4e-5 at L = 14 and 2.6e-5 at L = 16 on
    128 x 128, while the well-conditioned wide shapes stay below 1e-5."""
    if dtype == "bf16":
        return 2e-2
    return 1e-5 if (w > h or L <= 10) else 2.0 ** (L - 1) * 2.0 ** -24


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("L", [2, 6, 10, 14, 16])
def test_ablation(L, dtype):
    xs, ys, w = run(dtype, L)
    for A, Y in zip(xs, ys):
        ref = O.ifnso_alg1(A, w)
        assert rel(Y, ref) < tol(dtype, L, *A.shape)


def test_ablation_ns_rows():
    """The two NS rows of Table 1 on the same inputs: cubic NS with 8 steps and
    Muon's quintic with 5 steps, FP32 plan, against the oracle."""
    import torch

    F = lib()
    for s, (h, w) in enumerate(SHAPES):
        x = to_dev(synth.gaussian(s, h, w), "f32")
        for poly, steps in [(ONS.CUBIC, 8), (ONS.MUON_ABC, 5)]:
            y = torch.empty_like(x)
            F.Plan(h, w, "f32", L=1).ns_iterate(F.Batch([x]), poly, steps, [y])
            torch.cuda.synchronize()
            ref = ONS.ns_generic(to_np(x), poly, steps)
            assert rel(to_np(y), ref) < 1e-5
