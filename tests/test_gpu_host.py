"""The host-memory entry point: uploads, passes and downloads of groups of
matrices overlap, and the results are those of the device entry point."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _host_copy(x):
    """Page-locked host copy of the storage behind a (possibly row-padded) device view."""
    import torch

    rows, ld = x.shape[0], x.stride(0)
    full = torch.as_strided(x, (rows, ld), (ld, 1))
    return full.cpu().pin_memory()


@pytest.mark.parametrize("groups,streams", [(1, 2), (2, 2), (3, 2), (0, 2), (3, 1), (0, 1)])
def test_host_matches_device_bf16(groups, streams):
    import torch

    F = lib()
    shapes = [(256, 512), (392, 136), (200, 328), (512, 512), (130, 260), (640, 1000)]
    mats = [synth.gaussian(60 + i, *s) for i, s in enumerate(shapes)]
    xs = [to_dev(m, "bf16") for m in mats]
    L = 6
    w = np.r_[1.0, coeffs(L)]
    hmax = max(min(s) for s in shapes)
    wmax = max(max(s) for s in shapes)
    plan = F.Plan(hmax, wmax, "bf16", L=L)
    plan.set(F.IFNSO_OPT_HOST_STREAMS, streams)  # 2: odd groups on the plan's second compute stream
    batch = F.Batch(xs)
    ref = [torch.empty(x.shape, dtype=x.dtype, device=x.device) for x in xs]
    plan.orthogonalize(batch, w, ref)
    torch.cuda.synchronize()
    ref_h = [to_np(y) for y in ref]
    # host inputs: the same values; the device inputs are overwritten by the upload
    hin = [_host_copy(x) for x in xs]
    for x in xs:
        x.zero_()
    outs = [torch.full(x.shape, float("nan"), dtype=x.dtype, device=x.device) for x in xs]
    hout = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in xs]
    for _ in range(2):  # the second call reuses the cached metadata
        for h in hout:
            h.fill_(float("nan"))
        plan.orthogonalize_host(hin, batch, w, outs, hout, groups=groups)
        torch.cuda.synchronize()
        st, _, _ = plan.device_status(len(xs))
        assert np.all(st == 0)
        for i, (h, m) in enumerate(zip(hout, mats)):
            got = h.double().numpy()
            # same kernels; only the order of the FP64 atomics of o = ||T_0||_F may differ
            assert rel(got, ref_h[i]) < 1e-5, (groups, streams, i)
            A = to_np(xs[i])
            assert rel(got, O.ifnso_alg1(A, w[1:])) < 2e-2


def test_host_f32():
    import torch

    F = lib()
    shapes = [(100, 300), (256, 96)]
    mats = [synth.gaussian(70 + i, *s) for i, s in enumerate(shapes)]
    xs = [to_dev(m, "f32") for m in mats]
    L = 4
    w = np.r_[1.0, coeffs(L)]
    plan = F.Plan(256, 300, "f32", L=L)
    batch = F.Batch(xs)
    hin = [x.cpu().pin_memory() for x in xs]
    outs = [torch.empty_like(x) for x in xs]
    hout = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in xs]
    plan.orthogonalize_host(hin, batch, w, outs, hout, groups=4)
    torch.cuda.synchronize()
    for h, x in zip(hout, xs):
        assert rel(h.double().numpy(), O.ifnso_alg1(to_np(x), w[1:])) < 1e-5
