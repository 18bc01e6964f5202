"""ifnso_muon_step through the C ABI against the FP64 oracle (oracle/muon.py):
the momentum buffer (FP32), the BF16 input U it orthogonalizes, and the
weights after the update fused into the final product, over two steps."""
import numpy as np
import pytest

import synth
from oracle import muon as MU
from tests.gpu_util import coeffs, lib, rel, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(256, 512), (512, 256), (200, 328), (136, 392)]


def bf16(a, dev):
    import torch

    return torch.tensor(np.asarray(a, dtype=np.float32), device=dev).to(torch.bfloat16).contiguous()


@pytest.mark.parametrize("nesterov,cg", [(True, 0), (False, 0), (True, 2)])
def test_muon_step_matches_oracle(nesterov, cg):
    import torch

    F = lib()
    dev = torch.device("cuda:0")
    L, beta, lr = 6, 0.95, 0.05
    w = coeffs(L)
    G = [bf16(synth.gaussian(60 + i, r, c), dev) for i, (r, c) in enumerate(SHAPES)]
    M = [torch.tensor(0.1 * synth.gaussian(70 + i, r, c), dtype=torch.float32, device=dev)
         for i, (r, c) in enumerate(SHAPES)]
    # step 1 starts from zero weights (W' = -lr s Y), step 2 from the result
    W = [torch.zeros((r, c), dtype=torch.bfloat16, device=dev) for r, c in SHAPES]
    U = [torch.empty_like(g) for g in G]
    hmax = max(min(s) for s in SHAPES)
    wmax = max(max(s) for s in SHAPES)
    plan = F.Plan(hmax, wmax, "bf16", L=L)
    plan.set(F.IFNSO_OPT_CTA_GROUP, cg)  # 2: the fused update also on MMAs of the CTA pair
    batch = F.Batch(G)
    for step in range(2):
        M0 = [to_np(m) for m in M]
        W0 = [to_np(x) for x in W]
        plan.muon_step(batch, M, U, W, np.r_[1.0, w], beta=beta, nesterov=nesterov, lr=lr)
        torch.cuda.synchronize()
        st, _, _ = plan.device_status(len(SHAPES))
        assert np.all(st == 0)
        for i, (r, c) in enumerate(SHAPES):
            g = to_np(G[i])
            M1, Uref = MU.momentum(g, M0[i], beta, nesterov)
            # FP32 momentum: one fused multiply-add per element
            assert rel(to_np(M[i]), M1) < 1e-6
            # U rounded once to BF16 (8-bit significand: relative error at most 2^-8 per element)
            u = to_np(U[i])
            # (plus the FP32 rounding of the momentum arithmetic before it)
            assert np.all(np.abs(u - Uref) <= (2.0 ** -8 + 1e-6) * np.abs(Uref) + 1e-9)
            # the update of the BF16 U the library orthogonalized, against W0
            dW = to_np(W[i]) - W0[i]
            dref = MU.update(np.zeros((r, c)), u, w, lr)
            # BF16 rounding of the stored weights adds at most 2^-8 |W'| per element
            slack = 2.0 ** -8 * np.linalg.norm(to_np(W[i])) / max(np.linalg.norm(dref), 1e-30)
            assert rel(dW, dref) < 2e-2 + slack, (step, i, rel(dW, dref), slack)
