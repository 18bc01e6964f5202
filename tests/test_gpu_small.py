"""The on-chip path for matrices with h <= 128 (csrc/small.cu): one CTA runs
the whole of Algorithm 1 (Sec. 2.4) per matrix.  Every output is compared
with Algorithm 1 evaluated in FP64 (the oracle) on the same BF16 input, and
with the tiled passes on the same batch."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

# Table 1 shapes, ragged wide, tall (processed transposed), h = 1, h = 64 and
# a width that is not a multiple of 8 (scalar stores of the output)
SHAPES = [(128, 128), (128, 512), (128, 1024), (100, 300), (300, 100), (1, 40), (64, 64), (17, 33),
          (128, 129), (96, 1000)]


def run(F, mats, L, small, scale="gram", precision="auto"):
    import torch

    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
    hmax = max(min(x.shape) for x in xs)
    wmax = max(max(x.shape) for x in xs)
    plan = F.Plan(hmax, wmax, "bf16", L=L, scale=scale, precision=precision)
    plan.set(F.IFNSO_OPT_SMALL_MATRICES, small)
    w = coeffs(L)
    b = F.Batch(xs)
    plan.orthogonalize(b, np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    st, o, tr = plan.device_status(len(xs))
    return plan, xs, [to_np(y) for y in ys], w, st, o, tr


@pytest.mark.parametrize("L", [1, 4, 10, 14])
def test_small_path_matches_oracle(L):
    """One call over every shape; L = 10 and 14 take split FP16 squarings
    (2 and 6 of them in the mixed precision), L = 4 plain ones."""
    F = lib()
    mats = [synth.gaussian(200 + i, r, c) for i, (r, c) in enumerate(SHAPES)]
    plan, xs, ys, w, st, o, tr = run(F, mats, L, small=1)
    assert np.all(st == 0)
    for x, y, oo, t in zip(xs, ys, o, tr):
        A = to_np(x)
        ref = O.ifnso_alg1(A, w)
        err = rel(y, ref)
        print(f"L={L} {A.shape}: rel err {err:.2e}")
        assert err < 2e-2, (A.shape, err)
        Ao = O.orient(A)[0]
        G = Ao @ Ao.T
        assert abs(oo - np.linalg.norm(G)) <= 1e-5 * np.linalg.norm(G)
        assert abs(t - np.trace(G)) <= 1e-5 * np.trace(G)


@pytest.mark.parametrize("L", [4, 14])
def test_small_path_agrees_with_tiled_passes(L):
    F = lib()
    mats = [synth.gaussian(300 + i, r, c) for i, (r, c) in enumerate(SHAPES)]
    _, xs, y_small, w, _, _, _ = run(F, mats, L, small=1)
    _, _, y_tiled, _, _, _, _ = run(F, mats, L, small=2)
    for x, a, b in zip(xs, y_small, y_tiled):
        ref = O.ifnso_alg1(to_np(x), w)
        # both within the BF16 tolerance of the oracle, and of each other
        assert rel(a, ref) < 2e-2 and rel(b, ref) < 2e-2
        assert rel(a, b) < 2e-2


def test_small_path_frobenius_scale_split_precision_and_zero_input():
    F = lib()
    mats = [synth.gaussian(7, 128, 384), np.zeros((40, 80)), synth.gaussian(8, 90, 90)]
    plan, xs, ys, w, st, o, tr = run(F, mats, 6, small=1, scale="frob", precision="split")
    assert st[0] == 0 and st[2] == 0
    assert st[1] & F.IFNSO_DEV_ZERO_INPUT
    assert np.all(ys[1] == 0.0)
    for i in (0, 2):
        ref = O.ifnso_alg1(to_np(xs[i]), w, scale="frob")
        assert rel(ys[i], ref) < 2e-2


def test_small_path_many_matrices_and_host_buffers():
    """300 small matrices of random shapes in one launch; the host-buffer
    entry point (grouped uploads and downloads) gives the same results."""
    import torch

    F = lib()
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(1, 129)), int(rng.integers(1, 700))) for _ in range(300)]
    shapes = [(r, c) if rng.random() < 0.8 else (c, r) for r, c in shapes]
    mats = [synth.gaussian(1000 + i, r, c) for i, (r, c) in enumerate(shapes)]
    L = 14
    plan, xs, ys, w, st, _, _ = run(F, mats, L, small=1)
    assert np.all(st == 0)
    for i in range(0, 300, 23):
        A = to_np(xs[i])
        assert rel(ys[i], O.ifnso_alg1(A, w)) < 2e-2, (A.shape,)
    hout = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
    dev_out = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    # the host copies of the inputs have the device tensors' layout (padded rows)
    hin = []
    for x in xs:
        r, c = x.shape
        buf = torch.empty((r, x.stride(0)), dtype=x.dtype, pin_memory=True)[:, :c]
        buf.copy_(x)
        hin.append(buf)
    plan.orthogonalize_host(hin, F.Batch(xs), np.r_[1.0, w], dev_out, hout, groups=4)
    torch.cuda.synchronize()
    for i in range(300):
        assert np.array_equal(to_np(hout[i]), ys[i]), i


def test_autotuner_measures_the_small_bucket():
    F = lib()
    mats = [synth.gaussian(400 + i, 128, c) for i, c in enumerate([128, 512, 1024] * 4)]
    import torch

    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    plan = F.Plan(128, 1024, "bf16", L=14)
    assert plan.get(F.IFNSO_OPT_SMALL_TUNED) == 0
    w = coeffs(14)
    plan.autotune(F.Batch(xs), np.r_[1.0, w], ys, reps=2)
    assert plan.get(F.IFNSO_OPT_SMALL_TUNED) in (1, 2)
    print("autotuner chose", {1: "on-chip path", 2: "tiled passes"}[plan.get(F.IFNSO_OPT_SMALL_TUNED)])
    for y in ys:
        y.fill_(float("nan"))
    plan.orthogonalize(F.Batch(xs), np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    for x, y in zip(xs, ys):
        assert rel(to_np(y), O.ifnso_alg1(to_np(x), w)) < 2e-2


@pytest.mark.parametrize("L", [4, 14])
def test_mixed_batch_small_on_chip_rest_tiled(L):
    """A batch mixing h <= 128 and larger matrices: the small ones go to the
    on-chip path, the tiled passes skip them; every output matches the
    oracle, and the same batch with the on-chip path off agrees."""
    import torch

    F = lib()
    shapes = [(128, 512), (300, 700), (64, 64), (256, 256), (640, 100), (96, 1000), (513, 1030), (17, 33),
              (129, 400)]
    mats = [synth.gaussian(500 + i, r, c) for i, (r, c) in enumerate(shapes)]
    plan, xs, ys, w, st, o, tr = run(F, mats, L, small=1)
    assert np.all(st == 0)
    _, _, yt, _, st2, o2, tr2 = run(F, mats, L, small=2)
    for x, y, z, oo, oo2 in zip(xs, ys, yt, o, o2):
        A = to_np(x)
        ref = O.ifnso_alg1(A, w)
        assert rel(y, ref) < 2e-2, A.shape
        assert rel(z, ref) < 2e-2, A.shape
        Ao = O.orient(A)[0]
        G = Ao @ Ao.T
        assert abs(oo - np.linalg.norm(G)) <= 1e-5 * np.linalg.norm(G)
        assert abs(oo2 - np.linalg.norm(G)) <= 1e-5 * np.linalg.norm(G)
    # the large ones took the same tiled passes either way
    for i, (r, c) in enumerate(shapes):
        if min(r, c) > 128:
            assert np.array_equal(ys[i], yt[i]), shapes[i]
    # grouped host-buffer path over the mixed batch
    hin = []
    for x in xs:
        r, c = x.shape
        buf = torch.empty((r, x.stride(0)), dtype=x.dtype, pin_memory=True)[:, :c]
        buf.copy_(x)
        hin.append(buf)
    hout = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
    dev_out = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    plan.orthogonalize_host(hin, F.Batch(xs), np.r_[1.0, w], dev_out, hout, groups=3)
    torch.cuda.synchronize()
    for i in range(len(xs)):
        assert rel(to_np(hout[i]), ys[i]) < 1e-6, shapes[i]


def test_small_path_long_matrices():
    """Long rows: the Gram streams 188 K blocks through the 8-stage ring and
    the product 47 tiles through the two TMEM accumulators (many phase
    wraps of every barrier); wide and tall, against the oracle."""
    F = lib()
    mats = [synth.gaussian(900, 128, 12000), synth.gaussian(901, 11001, 100), synth.gaussian(902, 64, 8192)]
    plan, xs, ys, w, st, o, tr = run(F, mats, 14, small=1)
    assert np.all(st == 0)
    for x, y in zip(xs, ys):
        A = to_np(x)
        assert rel(y, O.ifnso_alg1(A, w)) < 2e-2, A.shape
