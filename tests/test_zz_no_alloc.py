"""The no-allocation Frobenius norm (ifnso_frobenius_norm2_static).

Callers that cannot let a library allocate device memory (hosts that own all
device memory through their own pool, latency-critical code that cannot take
the synchronisation of cudaMalloc) use this entry point; its descriptors live
in a fixed array inside the library.  This file runs last so that a failure
here does not hide the result of any other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from tests.gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu


def _static_norm2(F, mats, dtype):
    import torch

    b = F.Batch(mats)
    out = torch.full((len(mats),), float("nan"), dtype=torch.float64, device=mats[0].device)
    st = F.ifnso_frobenius_norm2_static(b.ref(), dtype, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == F.IFNSO_OK, F.ifnso_last_error()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_static_norm_matches_allocating_entry_point(dtype):
    F = lib()
    code = F.IFNSO_BF16 if dtype == "bf16" else F.IFNSO_F32
    # two calls in a row with different batches: the shared array is rewritten
    # and the sums restart from zero
    first = [to_dev(synth.gaussian(1, 300, 1000), dtype), to_dev(synth.gaussian(2, 17, 3), dtype),
             to_dev(synth.gaussian(3, 2048, 5632), dtype)]
    second = [to_dev(synth.gaussian(4, 64, 640), dtype)]
    for mats in (first, second, first):
        got = _static_norm2(F, mats, code)
        ref = F.frobenius_norm2(mats).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=1e-5, atol=0.0), (got, ref)
        # and the plain FP64 sum of squares of the same stored values
        exact = np.array([float(np.sum(m.double().cpu().numpy() ** 2)) for m in mats])
        assert np.allclose(got, exact, rtol=1e-5, atol=0.0), (got, exact)


def test_static_norm_rejects_oversized_batch():
    import torch

    F = lib()
    n = F.IFNSO_STATIC_NORM_MAX_MATRICES + 1
    x = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    b = F.Batch([x] * n)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = F.ifnso_frobenius_norm2_static(b.ref(), F.IFNSO_F32, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == F.IFNSO_ERR_INVALID_ARG
    assert b"static maximum" in F.ifnso_last_error()
