"""The on-chip Newton-Schulz baseline for matrices with h <= 128
(csrc/small.cu, small_ns_kernel): one CTA runs every step of the iteration
(Sec. 1, Eqs. one_iteration_matrix and iteration_jordan) per matrix.  Every
output is compared with the iteration in FP64 (the oracle) on the same BF16
input, and with the tiled passes on the same batch."""
import numpy as np
import pytest

import synth
from oracle import ns as ONS
from tests.gpu_util import lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

# Table 1 shapes, ragged wide, tall (processed transposed), h = 1, h <= 64
# (one K block of the product), widths that are not multiples of 8 or 64
SHAPES = [(128, 128), (128, 512), (128, 1024), (100, 300), (300, 100), (1, 40), (64, 64), (17, 33),
          (128, 129), (96, 1000), (40, 7), (65, 257)]
# BF16 storage of X, X X^T and B every step, as on the tiled passes
TOL = 5e-2


def run(F, mats, poly, steps, small):
    import torch

    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
    hmax = max(min(x.shape) for x in xs)
    wmax = max(max(x.shape) for x in xs)
    plan = F.Plan(hmax, wmax, "bf16", L=1)
    plan.set(F.IFNSO_OPT_SMALL_MATRICES, small)
    plan.ns_iterate(F.Batch(xs), poly, steps, ys)
    torch.cuda.synchronize()
    st, s2, _ = plan.device_status(len(xs))
    return xs, [to_np(y) for y in ys], st, s2


@pytest.mark.parametrize("poly,steps", [(ONS.MUON_ABC, 5), (ONS.CUBIC, 8), (ONS.MUON_ABC, 1),
                                        (ONS.CUBIC, 16)])
def test_small_ns_matches_oracle(poly, steps):
    F = lib()
    mats = [synth.gaussian(600 + i, r, c) for i, (r, c) in enumerate(SHAPES)]
    xs, ys, st, s2 = run(F, mats, poly, steps, small=1)
    assert np.all(st == 0)
    for x, y, n2 in zip(xs, ys, s2):
        A = to_np(x)
        ref = ONS.ns_generic(A, poly, steps)
        err = rel(y, ref)
        print(f"{len(poly)} terms, {steps} steps {A.shape}: rel err {err:.2e}")
        assert err < TOL, (A.shape, err)
        # ||A||_F^2, from the trace of the first Gram
        assert abs(n2 - np.sum(A * A)) <= 1e-5 * np.sum(A * A)


@pytest.mark.parametrize("poly,steps", [(ONS.MUON_ABC, 5), (ONS.CUBIC, 8)])
def test_small_ns_agrees_with_tiled_passes(poly, steps):
    F = lib()
    mats = [synth.gaussian(700 + i, r, c) for i, (r, c) in enumerate(SHAPES)]
    xs, y_small, st1, n1 = run(F, mats, poly, steps, small=1)
    _, y_tiled, st2, n2 = run(F, mats, poly, steps, small=2)
    assert np.all(st1 == 0) and np.all(st2 == 0)
    for x, a, b in zip(xs, y_small, y_tiled):
        ref = ONS.ns_generic(to_np(x), poly, steps)
        assert rel(a, ref) < TOL and rel(b, ref) < TOL
        assert rel(a, b) < TOL
    assert np.allclose(n1, n2, rtol=1e-5)


def test_small_ns_zero_input_and_scale():
    F = lib()
    M = synth.gaussian(9, 96, 300)
    mats = [np.zeros((50, 70)), M, 1000.0 * M, np.zeros((200, 3))]
    xs, ys, st, s2 = run(F, mats, ONS.MUON_ABC, 5, small=1)
    for i in (0, 3):
        assert st[i] & F.IFNSO_DEV_ZERO_INPUT
        assert np.all(ys[i] == 0.0)
    assert st[1] == 0 and st[2] == 0
    for i in (1, 2):
        assert rel(ys[i], ONS.ns_generic(to_np(xs[i]), ONS.MUON_ABC, 5)) < TOL


def test_small_ns_many_matrices():
    """300 small matrices of random shapes in one launch."""
    F = lib()
    rng = np.random.default_rng(11)
    shapes = [(int(rng.integers(1, 129)), int(rng.integers(1, 700))) for _ in range(300)]
    shapes = [(r, c) if rng.random() < 0.8 else (c, r) for r, c in shapes]
    mats = [synth.gaussian(2000 + i, r, c) for i, (r, c) in enumerate(shapes)]
    xs, ys, st, _ = run(F, mats, ONS.MUON_ABC, 5, small=1)
    assert np.all(st == 0)
    for i in range(0, 300, 17):
        A = to_np(xs[i])
        assert rel(ys[i], ONS.ns_generic(A, ONS.MUON_ABC, 5)) < TOL, (A.shape,)


def test_small_ns_one_launch():
    """The whole iteration is one kernel launch; the tiled passes take
    2 + 3 per step."""
    F = lib()
    mats = [synth.gaussian(800 + i, 128, c) for i, c in enumerate([128, 512, 1024])]
    import torch

    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    plan = F.Plan(128, 1024, "bf16", L=1)
    plan.ns_iterate(F.Batch(xs), ONS.MUON_ABC, 5, ys)
    torch.cuda.synchronize()
    before = F.launch_count()
    plan.ns_iterate(F.Batch(xs), ONS.MUON_ABC, 5, ys)
    torch.cuda.synchronize()
    assert F.launch_count() - before == 1
    plan.set(F.IFNSO_OPT_SMALL_MATRICES, 2)
    before = F.launch_count()
    plan.ns_iterate(F.Batch(xs), ONS.MUON_ABC, 5, ys)
    torch.cuda.synchronize()
    assert F.launch_count() - before == 2 + 3 * 5


def test_small_ns_long_matrices():
    """Long rows: many K blocks, product tiles and X round trips per step."""
    F = lib()
    mats = [synth.gaussian(910, 128, 12000), synth.gaussian(911, 11001, 100), synth.gaussian(912, 64, 8192)]
    xs, ys, st, _ = run(F, mats, ONS.MUON_ABC, 5, small=1)
    assert np.all(st == 0)
    for x, y in zip(xs, ys):
        A = to_np(x)
        assert rel(y, ONS.ns_generic(A, ONS.MUON_ABC, 5)) < TOL, A.shape
