"""Parity on the benchmark's own lists in the launch configuration bench.py
times: every matrix of the synthetic 1B (168) or 7B (224) list goes through one
ifnso_orthogonalize call with the bench's defaults (L = 14, AUTO precision,
autotuned MMA modes, the GPU learner's coefficients).  A deterministic sample
(first, middle and last layer; every oriented shape) is compared with Algorithm 1
evaluated in FP64 on the same BF16 input, regenerated bit for bit on the CPU."""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from tests.gpu_util import lib, rel, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("workload,samples", [
    ("muon_1b", [0, 4, 6, 84, 88, 90, 161, 165, 167]),   # q, gate, down of layers 0, 12, 23
    ("muon_7b", [0, 6]),                                   # q and down of layer 0
])
def test_list_in_bench_configuration(workload, samples):
    import torch

    import bench

    F = lib()
    wl = bench.WORKLOADS[workload]
    shapes = bench.workload_list(wl)
    L = wl["L"]
    dev = torch.device("cuda:0")
    xs = bench.make_inputs(F, torch, shapes, 0, dev)
    ys = [torch.empty_like(x) for x in xs]
    hw = [bench.oriented(r, c) for _, r, c in shapes]
    plan = F.Plan(max(h for h, _ in hw), max(w for _, w in hw), "bf16", L=L)
    batch = F.Batch(xs)
    w = F.learn_coefficients(L)
    coef = np.r_[1.0, w]
    plan.autotune(batch, coef, ys, reps=1)
    for y in ys:
        y.fill_(float("nan"))
    plan.orthogonalize(batch, coef, ys)
    torch.cuda.synchronize()
    st, _, _ = plan.device_status(len(xs))
    assert np.all(st == 0)
    alpha, beta = synth.lowrank_constants()
    for i in samples:
        _, r, c = shapes[i]
        M = synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(i, r, c))
        assert np.array_equal(to_np(xs[i]), M)  # the GPU generator matches synth/
        err = rel(to_np(ys[i]), O.ifnso_alg1(M, w))
        print(f"{workload} matrix {i} ({r}x{c}): relative error {err:.2e}")
        assert err < 2e-2
