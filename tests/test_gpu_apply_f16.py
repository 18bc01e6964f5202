"""The FP16 final product (IFNSO_OPT_APPLY_F16): P as one FP16 value times an
FP16 copy A s of the input (s a power of two from ||A||_F).  The copy is
checked element by element against its definition, the outputs against
Algorithm 1 evaluated in FP64 (the oracle) on the same BF16 input, and the
host-buffer entry point and the Muon step against the same plan's device
path and the BF16 hi + lo product."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = 2e-2  # the BF16 plans' bar


def f16_copy(A):
    """A s rounded to FP16, s = 2^floor(log2(32768 / ||A||_F)) within 2^-60..2^60
    (1 for a zero A): the definition the copy kernel follows."""
    nrm = np.sqrt(np.sum(np.asarray(A, dtype=np.float64) ** 2))
    if nrm == 0.0:
        s = 1.0
    else:
        s = 2.0 ** int(np.clip(np.floor(np.log2(32768.0 / nrm)), -60, 60))
    return (A * s).astype(np.float16), s


def run(F, mats, L, f16, cta_group=None, scale=None):
    import torch

    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
    hmax = max(min(x.shape) for x in xs)
    wmax = max(max(x.shape) for x in xs)
    plan = F.Plan(hmax, wmax, "bf16", L=L, scale=scale)
    plan.set(F.IFNSO_OPT_APPLY_F16, f16)
    plan.set(F.IFNSO_OPT_SMALL_MATRICES, 2)
    if cta_group:
        plan.set(F.IFNSO_OPT_CTA_GROUP, cta_group)
    b = F.Batch(xs)
    w = coeffs(L)
    plan.orthogonalize(b, np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    st, _, _ = plan.device_status(len(xs))
    return plan, b, xs, [to_np(y) for y in ys], w, st


SHAPES = [(256, 512), (392, 136), (200, 328), (512, 512), (130, 260), (700, 1030), (1, 64)]


# MIXED plans (AUTO for 5 <= L <= 14); SPLIT (L >= 15) keeps hi + lo and PLAIN (L <= 4) one BF16 P
@pytest.mark.parametrize("L,cg", [(14, 1), (14, 2), (6, 1), (5, 1)])
def test_f16_product_matches_oracle(L, cg):
    F = lib()
    mats = [synth.gaussian(60 + i, r, c) for i, (r, c) in enumerate(SHAPES)]
    plan, b, xs, ys, w, st = run(F, mats, L, 1, cta_group=cg)
    assert plan.get(F.IFNSO_OPT_APPLY_F16) == 1
    assert np.all(st == 0)
    _, _, _, ys_bf, _, _ = run(F, mats, L, 0, cta_group=cg)
    for x, y, yb in zip(xs, ys, ys_bf):
        ref = O.ifnso_alg1(to_np(x), w)
        e16, ebf = rel(y, ref), rel(yb, ref)
        print(f"L={L} CG {cg} {x.shape}: FP16 product {e16:.2e}, BF16 hi + lo {ebf:.2e}")
        assert e16 < TOL, (tuple(x.shape), e16)


def test_f16_copy_is_the_scaled_rounded_input():
    import torch

    F = lib()
    mats = [synth.gaussian(70, 256, 520), synth.gaussian(71, 600, 200), 1e4 * synth.gaussian(72, 128, 300),
            1e-6 * synth.gaussian(73, 260, 260)]
    plan, b, xs, ys, w, st = run(F, mats, 6, 1)
    assert plan.get(F.IFNSO_OPT_FP16_COPY_HOSTS) == 0  # too few tiles to fill the GPU: the copy kernel
    for i, x in enumerate(xs):
        A = to_np(x)
        want, s = f16_copy(A)
        ptr, ld = plan.workspace_view(b, i, 7)
        r, c = A.shape
        got = F.tensor_at(ptr, (r, ld), torch.float16, plan._last_ws.buf)[:, :c].cpu().numpy()
        assert np.array_equal(got.view(np.uint16), want.view(np.uint16)), i
        assert rel(ys[i], O.ifnso_alg1(A, w)) < TOL


@pytest.mark.parametrize("L,shapes,hosts", [
    # six split squarings carry the copies: wide with a ragged row end, tall, ragged square
    (14, [(2048, 2048)] * 3 + [(2048, 5630), (5632, 2040), (1530, 1536)], 6),
    # no split squaring: all five squarings carry them (square shapes, whose copies are short)
    (6, [(2048, 2048)] * 5 + [(2040, 2044)], 5),
])
def test_f16_copy_written_by_the_squarings(L, shapes, hosts):
    """Batches that fill the GPU have the FP16 copies written by the side
    warps of the squarings: the copy matches its definition bit for bit on
    every matrix (one of them scaled by 1e-4, so that s is not the same for
    all), and sampled outputs match the oracle."""
    import torch

    F = lib()
    mats = [synth.gaussian(140 + i, r, c) for i, (r, c) in enumerate(shapes)]
    mats[1] = 1e-4 * mats[1]
    plan, b, xs, ys, w, st = run(F, mats, L, 1)
    assert np.all(st == 0)
    assert plan.get(F.IFNSO_OPT_FP16_COPY_HOSTS) == hosts
    for i, x in enumerate(xs):
        A = to_np(x)
        want, s = f16_copy(A)
        ptr, ld = plan.workspace_view(b, i, 7)
        r, c = A.shape
        got = F.tensor_at(ptr, (r, ld), torch.float16, plan._last_ws.buf)[:, :c].cpu().numpy()
        assert np.array_equal(got.view(np.uint16), want.view(np.uint16)), i
    for i in (1, len(xs) - 3, len(xs) - 1):
        err = rel(ys[i], O.ifnso_alg1(to_np(xs[i]), w))
        print(f"L={L} {tuple(xs[i].shape)}: {err:.2e}")
        assert err < TOL, (i, err)


def test_f16_product_zero_input_and_frobenius_scale():
    F = lib()
    mats = [np.zeros((256, 300)), synth.gaussian(80, 300, 700)]
    plan, b, xs, ys, w, st = run(F, mats, 8, 1, scale="frob")
    assert st[0] & F.IFNSO_DEV_ZERO_INPUT
    assert np.all(ys[0] == 0.0)
    assert rel(ys[1], O.ifnso_alg1(to_np(xs[1]), w, scale="frob")) < TOL


def test_f16_product_host_buffers_and_groups():
    """The host-buffer entry point (groups of uploads, passes, downloads)
    gives the device path's results bit for bit under the FP16 product."""
    import torch

    F = lib()
    mats = [synth.gaussian(90 + i, *s) for i, s in enumerate([(512, 768), (768, 512), (256, 256), (300, 900)])]
    plan, b, xs, ys, w, st = run(F, mats, 14, 1)
    hin = []
    for x in xs:
        r, c = x.shape
        buf = torch.empty((r, x.stride(0)), dtype=x.dtype, pin_memory=True)[:, :c]
        buf.copy_(x)
        hin.append(buf)
    hout = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
    dev = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    plan.orthogonalize_host(hin, b, np.r_[1.0, w], dev, hout, groups=2)
    torch.cuda.synchronize()
    for y, h in zip(ys, hout):
        assert np.array_equal(to_np(h), y)


def test_f16_product_in_the_muon_step():
    """The Muon step's fused weight update with the FP16 product agrees with
    the BF16 hi + lo product within the update's own tolerance."""
    import torch

    F = lib()
    shapes = [(256, 512), (512, 256)]
    outs = []
    for f16 in (1, 0):
        gs = [to_dev(synth.gaussian(100 + i, r, c), "bf16") for i, (r, c) in enumerate(shapes)]
        ws_ = [to_dev(0.1 * synth.gaussian(110 + i, r, c), "bf16") for i, (r, c) in enumerate(shapes)]
        w0 = [to_np(x) for x in ws_]
        ms = [torch.zeros(g.shape, dtype=torch.float32, device="cuda") for g in gs]
        us = [torch.empty_like(g) for g in gs]
        plan = F.Plan(512, 512, "bf16", L=14)
        plan.set(F.IFNSO_OPT_APPLY_F16, f16)
        w = coeffs(14)
        plan.muon_step(F.Batch(gs), ms, us, ws_, np.r_[1.0, w], lr=0.02, beta=0.95, nesterov=True)
        torch.cuda.synchronize()
        outs.append([to_np(x) - a for x, a in zip(ws_, w0)])
    for d16, dbf in zip(*outs):
        assert rel(d16, dbf) < TOL


def test_two_plans_sharing_one_workspace():
    """Calls of two plans (FP16 product at L = 14, BF16 hi + lo at L = 6)
    alternate on one workspace: each call finds the other plan's metadata
    there and uploads its own again; every output matches the oracle."""
    import torch

    F = lib()
    mats = [synth.gaussian(120 + i, *s) for i, s in enumerate([(256, 512), (384, 300)])]
    xs = [to_dev(m, "bf16") for m in mats]
    b = F.Batch(xs)
    pa = F.Plan(384, 512, "bf16", L=14)
    pa.set(F.IFNSO_OPT_APPLY_F16, 1)
    pb = F.Plan(384, 512, "bf16", L=6)
    ws = F.Workspace(max(pa.workspace_bytes(b), pb.workspace_bytes(b)), device="cuda")
    for rnd in range(3):
        for plan, L in ((pa, 14), (pb, 6)):
            ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
            w = coeffs(L)
            plan.orthogonalize(b, np.r_[1.0, w], ys, ws=ws)
            torch.cuda.synchronize()
            for x, y in zip(xs, ys):
                assert rel(to_np(y), O.ifnso_alg1(to_np(x), w)) < TOL, (rnd, L)
