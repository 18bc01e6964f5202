"""GPU tests of the building blocks through the C ABI: the Philox input
generator (bit-exact against synth/), the split-K Frobenius norm, the GPU
coefficient learner against the FP64 oracle learner."""
import numpy as np
import pytest

import synth
from oracle import coeffs as OC
from tests.gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu


def test_synth_lowrank_bit_exact():
    torch = pytest.importorskip("torch")
    F = lib()
    alpha, beta = synth.lowrank_constants()
    for seed, (r, c) in [(3, (48, 80)), (7, (300, 520)), (11, (130, 37))]:
        ld = (c + 7) // 8 * 8
        buf = torch.zeros((r, ld), dtype=torch.bfloat16, device="cuda")
        F.synth_lowrank_bf16(buf[:, :c], seed, alpha, beta)
        torch.cuda.synchronize()
        got = buf[:, :c].contiguous().view(torch.int16).cpu().numpy().view(np.uint16)
        ref = synth.lowrank_noise_bf16(seed, r, c)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_frobenius_norm2(dtype):
    torch = pytest.importorskip("torch")
    F = lib()
    mats = [synth.gaussian(1, 300, 1000), synth.gaussian(2, 17, 3), synth.gaussian(3, 2048, 5632)]
    ts = [to_dev(m, dtype) for m in mats]
    got = F.frobenius_norm2(ts).cpu().numpy()
    for g, t in zip(got, ts):
        ref = float(np.sum(t.double().cpu().numpy() ** 2))
        assert abs(g - ref) / ref < 1e-5


@pytest.mark.parametrize("L", [1, 4, 9])
def test_learner_matches_oracle(L):
    F = lib()
    iters = 3000
    gpu = F.learn_coefficients(L, iters=iters, samples=1000, lr=0.1, step_size=1500, gamma=0.5, seed=0)
    ref, _ = OC.learn(L, lambda t: synth.learner_uniforms(0, t, 1000), iters=iters, step_size=1500)
    # both sides run the same FP64 arithmetic on the same Philox samples; only
    # the order of the 1000-term gradient sums differs
    assert np.allclose(gpu, ref, rtol=1e-9, atol=1e-11), (gpu, ref)
