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
from tests.gpu_util import block_max_rel, coeffs, lib, rel, to_dev, to_np

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


def oracle_raw_features(A):
    """The network's six raw features of A in FP64 (Sec. 2.1 scaling, q = 1):
    eigenvalues x_i^2 of D = A A^T / ||A A^T||_F from the Gram matrix."""
    Ao, _ = O.orient(A)
    h, w = Ao.shape
    G = Ao @ Ao.T
    o = np.linalg.norm(G)
    lam = np.clip(np.linalg.eigvalsh(G), 0.0, None) / o
    return MLP.raw_features(np.sqrt(lam), h, w, np.linalg.norm(Ao))


def gpu_raw_features(scal, h, w):
    """The same six features from the FP64 scalars the call kept for the
    matrix (||T_0||_F^2, tr T_0, and tr D_1^4 summed by the first squaring)."""
    o2, tr, t4 = scal[0], scal[1], scal[6]
    oo = math.sqrt(o2)
    return np.array([math.log(tr / oo / h), math.log(o2 / (oo * oo) / h), math.log(t4 / h), math.log(h),
                     math.log(w), 0.5 * math.log(tr)])


# Feature tolerances (absolute, on the logarithms = relative on the traces).
# tr T_0 and ||T_0||_F^2 are FP64 sums of FP32 partial sums, each over the
# 4096 squares (or diagonal entries) one epilogue warp sees: the FP32
# rounding of such a sum is typically sqrt(4096) 2^-24 ~ 4e-6 relative and at
# worst 4096 2^-24 ~ 2.4e-4; 5e-5 sits between.  tr D_1^4 is summed by the
# first squaring, whose operand D_1 is rounded to FP16 (unit roundoff
# u = 2^-11) when that squaring is plain: each (D_1^2)_ij then carries a
# relative error up to about 2u, its square 4u, so 4u ~ 2e-3 bounds the sum;
# split operands (hi + lo) leave FP32 rounding only.
FEAT_TOL = 5e-5


def check_proposals(F, plan, b, xs, net, wfix, K, t4_tol):
    """Every matrix's features, coefficient row and fallback decision of the
    last call against the FP64 oracle network (oracle.mlp.propose).  Returns
    the rows."""
    import torch

    prm, stats = net.params()
    p = oracle_params(prm, K)
    mean, std = stats[:6].astype(np.float64), stats[6:12].astype(np.float64)
    rows = []
    n_decided = 0
    for i, x in enumerate(xs):
        ptr, _ = plan.workspace_view(b, i, 5)
        row = F.tensor_at(ptr, (K,), torch.float32, plan._last_ws.buf).double().cpu().numpy()
        ptr, _ = plan.workspace_view(b, i, 6)
        sc = F.tensor_at(ptr, (8,), torch.float64, plan._last_ws.buf).cpu().numpy()
        A = to_np(x)
        h, w = min(A.shape), max(A.shape)
        raw_g = gpu_raw_features(sc, h, w)
        raw_o = oracle_raw_features(A)
        tol = np.full(6, FEAT_TOL)
        tol[2] = t4_tol
        assert np.all(np.abs(raw_g - raw_o) <= tol), (i, raw_g - raw_o)
        # inference on the features the call used (rounded to FP32 as the kernel does)
        z_g = ((raw_g - mean) / std).astype(np.float32).astype(np.float64)
        c_g, fb_g = MLP.propose(p, z_g, wfix)
        out_g, _ = MLP.forward(p, z_g)
        r = out_g[K]
        fb_dev = sc[7] == 1.0
        assert row[0] == 1.0
        if abs(r) > 1e-3:
            n_decided += 1
            assert fb_dev == fb_g, (i, r)
            assert np.all(np.abs(row - c_g) <= 1e-4 * np.maximum(1.0, np.abs(c_g))), (i, row - c_g)
            # and on the features computed in FP64 from A itself
            z_o = (raw_o - mean) / std
            c_o, fb_o = MLP.propose(p, z_o, wfix)
            if fb_o == fb_g:
                assert np.all(np.abs(row - c_o) <= 1e-3 * np.maximum(1.0, np.abs(c_o))), (i, row - c_o)
        if fb_dev:
            assert np.array_equal(row[1:], np.asarray(wfix, dtype=np.float32).astype(np.float64))
        rows.append(row)
    print(f"{n_decided} of {len(xs)} proposals compared with the oracle network "
          f"(fallback {sum(1 for rw in rows if np.array_equal(rw[1:], np.float32(wfix).astype(np.float64)))})")
    assert n_decided >= len(xs) // 2
    return rows


def test_network_inside_orthogonalize(trained):
    """Held-out matrices materialised as U diag(sigma) V^T in BF16 go through one
    ifnso_orthogonalize call with per-matrix proposed coefficients.  The
    features, coefficient rows and fallback decisions the call made match the
    FP64 oracle network; each output matches Algorithm 1 (FP64 oracle) with
    the coefficients that call chose; and the proposal's distance to U V^T
    beats the fixed coefficients on average."""
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
    # L = 4: the first squaring is plain FP16 (2^-11 roundoff of D_1)
    rows = check_proposals(F, plan, b, xs, net, wfix, K, t4_tol=4 * 2.0 ** -11)
    plan2 = F.Plan(hmax, wmax, "bf16", L=K - 1)
    plan2.orthogonalize(b, np.r_[1.0, wfix], zs)
    torch.cuda.synchronize()
    d_mlp, d_fix = [], []
    for x, y, z, row in zip(xs, ys, zs, rows):
        A = to_np(x)
        assert rel(to_np(y), O.ifnso_alg1(A, row[1:])) < 2e-2
        P = O.polar_factor(A)
        h = min(A.shape)
        d_mlp.append(np.linalg.norm(to_np(y) - P) ** 2 / h)
        d_fix.append(np.linalg.norm(to_np(z) - P) ** 2 / h)
    print("in-path distance^2/h: proposal", np.mean(d_mlp), "fixed", np.mean(d_fix))
    assert np.mean(d_mlp) < np.mean(d_fix)


def test_network_inside_orthogonalize_7b_shapes():
    """Config 5's path on a sample of the 7B list (q 4096^2 and down
    14336 x 4096 of layer 0, regenerated on the CPU bit for bit) with a K = 15
    network at L = 14: the proposals against the oracle network, the outputs
    against Algorithm 1 with the chosen coefficients, whole and per tile.  The
    network's output layer is scaled up so that its proposals and fallback
    decisions differ from matrix to matrix."""
    import torch

    import bench

    F = lib()
    K = 15
    L = K - 1
    wfix = coeffs(L)
    net = F.Mlp(K, wfix, seed=7)
    prm, _ = net.params()
    prm = prm.copy()
    prm[-(K + 1) * 65:] *= 30.0
    net.set_params(prm)
    tr = spectra_to_device(range(0, 2000))
    net.set_data(*tr[:4], fit=True)   # feature standardisation from 2000 training spectra
    shapes = bench.workload_list(bench.WORKLOADS["muon_7b"])
    idx = [0, 1, 6]   # q, k (4096 x 4096) and down (14336 x 4096) of layer 0
    alpha, beta = synth.lowrank_constants()
    xs = []
    for i in idx:
        _, r, c = shapes[i]
        x = torch.empty((r, c), dtype=torch.bfloat16, device="cuda")
        F.synth_lowrank_bf16(x, i, float(alpha), float(beta))
        xs.append(x)
    ys = [torch.empty_like(x) for x in xs]
    plan = F.Plan(4096, 14336, "bf16", L=L)
    b = F.Batch(xs)
    plan.orthogonalize(b, net, ys)
    torch.cuda.synchronize()
    st, _, _ = plan.device_status(len(xs))
    assert np.all(st == 0)
    # L = 14 mixed precision: the first squaring has split operands
    rows = check_proposals(F, plan, b, xs, net, wfix, K, t4_tol=FEAT_TOL)
    for j, (i, x, y, row) in enumerate(zip(idx, xs, ys, rows)):
        _, r, c = shapes[i]
        M = synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(i, r, c))
        assert np.array_equal(to_np(x), M)
        ref = O.ifnso_alg1(M, row[1:])
        Y = to_np(y)
        err, tile = rel(Y, ref), block_max_rel(Y, ref)
        print(f"7B matrix {i} ({r}x{c}), proposed coefficients: rel err {err:.2e}, worst tile {tile:.2e}")
        assert err < 2e-2
        assert tile < 5e-2
