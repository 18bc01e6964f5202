"""Failure detection without a GPU fault: a host-set testing flag makes the
first CTA of the Gram pass load nothing, so its bounded pipeline waits run
out.  The kernel must return (no hang), report IFNSO_DEV_TIMEOUT for the
matrix, and leave the context usable for the next call."""
import time

import numpy as np
import pytest

import synth
from oracle import ifnso as O
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cta_group", [1, 2])
def test_stalled_pipeline_times_out_and_context_survives(cta_group):
    """cta_group 1: each CTA's own waits run out.  cta_group 2: the even CTA
    never arms its stage barriers, so the odd CTA's copies (which complete on
    the even CTA's barrier) never complete a phase; both CTAs' waits run out
    and the pair meets at its final cluster barriers."""
    import torch

    F = lib()
    x = to_dev(synth.gaussian(0, 256, 512), "bf16")
    y = torch.empty(x.shape, dtype=x.dtype, device="cuda")
    w = coeffs(4)
    plan = F.Plan(256, 512, "bf16", L=4)
    plan.set(F.IFNSO_OPT_CTA_GROUP, cta_group)
    plan.set(F.IFNSO_OPT_WAIT_LIMIT_MS, 100)
    plan.set(F.IFNSO_OPT_INJECT_STALL, 1)
    b = F.Batch([x])
    t0 = time.time()
    plan.orthogonalize(b, np.r_[1.0, w], [y])
    st, _, _ = plan.device_status(1)
    elapsed = time.time() - t0
    assert st[0] & F.IFNSO_DEV_TIMEOUT
    assert elapsed < 10.0
    import ctypes as C

    s = (C.c_int32 * 1)()
    rc = F.ifnso_device_status(plan.handle, C.c_void_p(plan._last_ws.ptr), 1, s, None, None,
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == F.IFNSO_ERR_DEVICE_TIMEOUT
    # the same plan and context compute correctly once the stall is gone
    plan.set(F.IFNSO_OPT_INJECT_STALL, 0)
    plan.orthogonalize(b, np.r_[1.0, w], [y])
    st, _, _ = plan.device_status(1)
    assert st[0] == 0
    assert rel(to_np(y), O.ifnso_alg1(to_np(x), w)) < 2e-2
