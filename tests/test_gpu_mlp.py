"""The coefficient-proposal MLP on the GPU: gradients of the hand-written
forward/backward kernels against the FP64 oracle, training on 100k synthetic
spectra, the gain over the fixed coefficients on 2k held-out matrices, and the
network inside ifnso_orthogonalize."""
import math

import numpy as np
import pytest

import synth
from oracle import ifnso as O
from oracle import mlp as MLP
from tests.gpu_util import coeffs, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def spectra_to_device(seeds):
    import torch

    hs, ws, sig, offs = [], [], [], [0]
    for s in seeds:
        h, w, sg, _ = synth.mlp_spectrum(s)
        hs.append(h)
        ws.append(w)
        sig.append(sg.astype(np.float32))
        offs.append(offs[-1] + h)
    dev = "cuda"
    return (torch.tensor(np.concatenate(sig), device=dev), torch.tensor(offs, dtype=torch.int64, device=dev),
            torch.tensor(hs, dtype=torch.int32, device=dev), torch.tensor(ws, dtype=torch.int32, device=dev),
            sig, hs, ws)


def oracle_params(flat, K):
    NO = K + 1
    o = 0
    p = {}
    for name, shape in [("W1", (64, 6)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (NO, 64)),
                        ("b3", (NO,))]:
        n = int(np.prod(shape))
        p[name] = flat[o:o + n].astype(np.float64).reshape(shape)
        o += n
    return p


def flatten(g):
    return np.concatenate([g[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


@pytest.mark.parametrize("K", [5, 15])
def test_gradients_match_oracle(K):
    import torch

    F = lib()
    L = K - 1
    wfix = coeffs(L)
    net = F.Mlp(K, wfix, seed=3)
    prm, _ = net.params()
    prm = prm.copy()
    prm[-(K + 1) * 65:] *= 30.0   # move the output layer away from zero
    net.set_params(prm)
    seeds = list(range(500, 540))
    sig_d, off_d, h_d, w_d, sig, hs, ws = spectra_to_device(seeds)
    net.set_data(sig_d, off_d, h_d, w_d, fit=True)
    idx = torch.arange(len(seeds), dtype=torch.int32, device="cuda")
    g, loss = net.loss_grad(idx)
    torch.cuda.synchronize()
    prm, stats = net.params()
    p = oracle_params(prm, K)
    Z, X = [], []
    for sg, h, w in zip(sig, hs, ws):
        sg = sg.astype(np.float64)
        o = math.sqrt(np.sum(sg ** 4))
        x = sg / math.sqrt(o)
        f = MLP.raw_features(x, h, w, math.sqrt(np.sum(sg ** 2)))
        Z.append((f - stats[:6]) / stats[6:])
        X.append(x)
    ref_loss, ref_g, _ = MLP.batch_loss_grad(p, Z, X, wfix)
    gg = g.cpu().numpy().astype(np.float64)
    rg = flatten(ref_g)
    assert abs(float(loss.item()) - ref_loss) <= 1e-4 * abs(ref_loss)
    assert np.linalg.norm(gg - rg) <= 1e-4 * np.linalg.norm(rg)
    # per tensor too, so that a small tensor cannot hide behind W2
    o = 0
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        n = ref_g[k].size
        a, b = gg[o:o + n], rg[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-4 * max(np.linalg.norm(b), 1e-8), k
        o += n


@pytest.fixture(scope="module")
def trained():
    """Config 4: 100k training spectra, 2k held-out, K = 5 over exponents {0, 1, 2, 4, 8}."""
    F = lib()
    K = 5
    wfix = coeffs(K - 1)
    net = F.Mlp(K, wfix, seed=0)
    tr = spectra_to_device(range(0, 100000))
    net.set_data(*tr[:4], fit=True)
    curve = net.train(4000, batch=512, lr=1e-3, seed=1)
    ho = spectra_to_device(range(1000000, 1002000))
    net.set_data(*ho[:4], fit=False)
    e_mlp, e_fix, cf, fb = net.evaluate(2000)
    return F, net, wfix, curve.cpu().numpy(), e_mlp.cpu().numpy(), e_fix.cpu().numpy(), cf.cpu().numpy(), \
        fb.cpu().numpy(), ho


def test_training_reduces_loss(trained):
    F, net, wfix, curve, *_ = trained
    assert np.mean(curve[-200:]) < 0.9 * np.mean(curve[:50])


def test_heldout_gain_over_fixed_coefficients(trained):
    F, net, wfix, curve, e_mlp, e_fix, cf, fb, ho = trained
    # mean squared distance to U V^T per h, proposal (after fallback) vs fixed
    gain = 1.0 - e_mlp.mean() / e_fix.mean()
    print(f"held-out E: proposal {e_mlp.mean():.5f}  fixed {e_fix.mean():.5f}  gain {gain:.3f}  "
          f"fallback {fb.mean():.3f}")
    assert gain > 0.02
    # the fixed-coefficient errors agree with the oracle's spectral evaluation
    for t in (0, 7, 1999):
        sg = ho[4][t].astype(np.float64)
        x = sg / math.sqrt(math.sqrt(np.sum(sg ** 4)))
        ref, _ = MLP.spectral_error(np.r_[1.0, wfix], x)
        assert abs(e_fix[t] - ref) <= 1e-4 * ref + 1e-7
        c = cf[t].astype(np.float64)
        ref_m, _ = MLP.spectral_error(c, x)
        assert abs(e_mlp[t] - ref_m) <= 1e-4 * ref_m + 1e-7


def test_network_inside_orthogonalize(trained):
    """Held-out matrices materialised as U diag(sigma) V^T in BF16 go through one
    ifnso_orthogonalize call with per-matrix proposed coefficients; each output
    matches Algorithm 1 (FP64 oracle) with the coefficients that call chose, and
    the proposal's distance to U V^T beats the fixed coefficients on average."""
    import torch

    F, net, wfix, *_ = trained
    K = 5
    seeds = [1000000 + i for i in range(12)]
    mats = [synth.mlp_matrix(s) for s in seeds]
    xs = [to_dev(M, "bf16") for M in mats]
    ys = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    zs = [torch.empty(x.shape, dtype=x.dtype, device="cuda") for x in xs]
    hmax = max(min(x.shape) for x in xs)
    wmax = max(max(x.shape) for x in xs)
    plan = F.Plan(hmax, wmax, "bf16", L=K - 1)
    b = F.Batch(xs)
    plan.orthogonalize(b, net, ys)
    torch.cuda.synchronize()
    rows = []
    for i in range(len(xs)):
        ptr, ld = plan.workspace_view(b, i, 5)
        rows.append(F.tensor_at(ptr, (K,), torch.float32, plan._last_ws.buf).double().cpu().numpy())
    plan2 = F.Plan(hmax, wmax, "bf16", L=K - 1)
    plan2.orthogonalize(b, np.r_[1.0, wfix], zs)
    torch.cuda.synchronize()
    d_mlp, d_fix = [], []
    for x, y, z, row in zip(xs, ys, zs, rows):
        A = to_np(x)
        assert row[0] == 1.0
        assert rel(to_np(y), O.ifnso_alg1(A, row[1:])) < 2e-2
        P = O.polar_factor(A)
        h = min(A.shape)
        d_mlp.append(np.linalg.norm(to_np(y) - P) ** 2 / h)
        d_fix.append(np.linalg.norm(to_np(z) - P) ** 2 / h)
    print("in-path distance^2/h: proposal", np.mean(d_mlp), "fixed", np.mean(d_fix))
    assert np.mean(d_mlp) < np.mean(d_fix)
