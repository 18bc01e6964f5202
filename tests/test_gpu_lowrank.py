"""Parity on matrices of the benchmark's workload (rank-32 signal plus noise,
generated on the GPU by the Philox kernel and regenerated bit for bit on the
CPU), in the launch configuration bench.py times: the batched BF16 path at
L = 14 with the default (AUTO = mixed) precision."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from oracle import ns as ONS
from tests.gpu_util import coeffs, lib, rel, to_np

pytestmark = pytest.mark.gpu


def test_lowrank_batch_L14_parity_and_polar():
    import torch

    F = lib()
    shapes = [(2048, 2048), (2048, 5632), (5632, 2048), (1024, 3000)]
    alpha, beta = synth.lowrank_constants()
    xs = []
    for i, (r, c) in enumerate(shapes):
        ld = (c + 7) // 8 * 8
        buf = torch.empty((r, ld), dtype=torch.bfloat16, device="cuda")
        F.synth_lowrank_bf16(buf[:, :c], 100 + i, float(alpha), float(beta))
        xs.append(buf[:, :c])
    ys = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    L = 14
    w = coeffs(L)
    plan = F.Plan(2048, 5632, "bf16", L=L)
    plan.orthogonalize(F.Batch(xs), np.r_[1.0, w], ys)
    zs = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    nsplan = F.Plan(2048, 5632, "bf16", L=1)
    nsplan.ns_iterate(F.Batch(xs), ONS.MUON_ABC, 5, zs)
    torch.cuda.synchronize()
    for i, (r, c) in enumerate(shapes[:3]):
        M = synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(100 + i, r, c))
        assert np.array_equal(to_np(xs[i]), M)          # the GPU generator matches synth/
        ref = O.ifnso_alg1(M, w)
        assert rel(to_np(ys[i]), ref) < 2e-2
        # equal polar error: the GPU IFNSO result is no farther from U V^T than the GPU NS5 result
        h = min(r, c)
        P = O.polar_factor(M)
        d_ifnso = np.linalg.norm(to_np(ys[i]) - P) / np.sqrt(h)
        d_ns5 = np.linalg.norm(to_np(zs[i]) - P) / np.sqrt(h)
        assert d_ifnso <= d_ns5 * 1.01, (d_ifnso, d_ns5)
