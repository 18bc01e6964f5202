"""GPU parity of the hot path through the C ABI against the FP64 oracle.

Tolerances (relative Frobenius error against Algorithm 1 evaluated in FP64 on
the same, already rounded input): 1e-5 for FP32 plans, 2e-2 for BF16 plans.
"""
import numpy as np
import pytest

import synth
from oracle import ifnso as O
from oracle import ns as ONS
from tests.gpu_util import coeffs, lib, rel, sym_upper, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 2e-2}


def run_ifnso(mats, L, dtype, precision=None, scale=None, stop_after=None, plan_shape=None, cta_group=None):
    import torch

    F = lib()
    xs = [to_dev(m, dtype) for m in mats]
    ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device=x.device) for x in xs]
    hmax = max(min(x.shape) for x in xs)
    wmax = max(max(x.shape) for x in xs)
    plan = F.Plan(*(plan_shape or (hmax, wmax)), dtype, L=L, precision=precision, scale=scale)
    if stop_after is not None:
        plan.set(F.IFNSO_OPT_STOP_AFTER, stop_after)
    if cta_group is not None:
        plan.set(F.IFNSO_OPT_CTA_GROUP, cta_group)
    b = F.Batch(xs)
    w = coeffs(L)
    plan.orthogonalize(b, np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    return F, plan, b, xs, ys, w


# --------------------------------------------------------------- FP32 path
@pytest.mark.parametrize("shape", [(256, 512), (512, 256), (100, 300), (64, 64), (1, 40)])
def test_f32_ifnso(shape):
    M = synth.gaussian(0, *shape)
    F, plan, b, xs, ys, w = run_ifnso([M], 4, "f32")
    ref = O.ifnso_alg1(to_np(xs[0]), w)
    assert rel(to_np(ys[0]), ref) < TOL["f32"]
    st, s2, tr = plan.device_status(1)
    assert st[0] == 0
    A = to_np(xs[0])
    assert abs(tr[0] - np.sum(A * A)) / np.sum(A * A) < 1e-6


@pytest.mark.parametrize("scale", ["gram", "frob", "gelfand2"])
def test_f32_scale_modes(scale):
    M = synth.gaussian(5, 96, 200)
    F, plan, b, xs, ys, w = run_ifnso([M], 6, "f32", scale=scale)
    assert rel(to_np(ys[0]), O.ifnso_alg1(to_np(xs[0]), w, scale)) < TOL["f32"]


@pytest.mark.parametrize("shape", [(256, 512), (300, 180)])
def test_f32_ns(shape):
    import torch

    F = lib()
    M = synth.gaussian(1, *shape)
    x = to_dev(M, "f32")
    for poly, steps in [(ONS.MUON_ABC, 5), (ONS.CUBIC, 8)]:
        y = torch.empty_like(x)
        plan = F.Plan(min(shape), max(shape), "f32", L=1)
        plan.ns_iterate(F.Batch([x]), poly, steps, [y])
        torch.cuda.synchronize()
        ref = ONS.ns_generic(to_np(x), poly, steps)
        assert rel(to_np(y), ref) < TOL["f32"]


# --------------------------------------------------------------- BF16 tcgen05 path
@pytest.mark.parametrize("shape", [(256, 512), (200, 328), (392, 136), (512, 512), (640, 1000)])
def test_bf16_gram(shape):
    """The symmetric tcgen05 Gram: T_0 = A A^T in FP32, sum T_0^2 and tr T_0."""
    import torch

    M = synth.gaussian(2, *shape)
    F, plan, b, xs, ys, w = run_ifnso([M], 4, "bf16", stop_after=0)
    ptr, ld = plan.workspace_view(b, 0, 0)
    G = sym_upper(F.tensor_at(ptr, (ld, ld), torch.float32, plan._last_ws.buf).double().cpu().numpy())
    A = O.orient(to_np(xs[0]))[0]
    h = A.shape[0]
    ref = A @ A.T
    assert rel(G[:h, :h], ref) < 1e-5
    assert np.all(G[h:, :] == 0) and np.all(G[:, h:] == 0)
    st, s2, tr = plan.device_status(1)
    assert abs(s2[0] - np.linalg.norm(ref)) / np.linalg.norm(ref) < 1e-5
    assert abs(tr[0] - np.trace(ref)) / np.trace(ref) < 1e-5


@pytest.mark.parametrize("precision", ["plain", "split"])
def test_bf16_prep(precision):
    import torch

    M = synth.gaussian(3, 300, 700)
    F, plan, b, xs, ys, w = run_ifnso([M], 4, "bf16", precision=precision, stop_after=1)
    ptr, ld = plan.workspace_view(b, 0, 1)
    D = F.tensor_at(ptr, (ld, ld), torch.float16, plan._last_ws.buf).double().cpu().numpy()
    if precision == "split":
        ptr2, _ = plan.workspace_view(b, 0, 2)
        D = D + F.tensor_at(ptr2, (ld, ld), torch.float16, plan._last_ws.buf).double().cpu().numpy()
    D = sym_upper(D)
    A = to_np(xs[0])
    G = A @ A.T
    ref = G / np.linalg.norm(G)
    # split: limited by the FP32 accumulation of T_0 (as in test_bf16_gram); plain: FP16 rounding
    tol = 1e-5 if precision == "split" else 1e-3
    assert rel(D[:300, :300], ref) < tol


@pytest.mark.parametrize("L,precision", [(4, "plain"), (4, "split"), (14, "split"), (9, "plain"),
                                         (14, "mixed"), (14, "auto"), (10, "mixed"), (2, "split"),
                                         (3, "plain"), (1, "split"), (5, "auto")])
@pytest.mark.parametrize("shape", [(256, 512), (200, 328), (392, 136), (512, 512), (640, 1000)])
def test_bf16_ifnso(shape, L, precision):
    M = synth.gaussian(4, *shape)
    F, plan, b, xs, ys, w = run_ifnso([M], L, "bf16", precision=precision)
    A = to_np(xs[0])
    ref = O.ifnso_alg1(A, w)
    err = rel(to_np(ys[0]), ref)
    assert err < TOL["bf16"], err


@pytest.mark.parametrize("L,precision", [(4, "plain"), (14, "mixed"), (3, "split")])
@pytest.mark.parametrize("shape", [(256, 512), (392, 136), (640, 1000), (1000, 640)])
def test_bf16_cta_groups(shape, L, precision):
    """Per-CTA MMAs (whole B tile per CTA) and MMAs of the CTA pair give the same
    products up to the rounding order of the accumulation."""
    M = synth.gaussian(40, *shape)
    out = {}
    for cg in (1, 2):
        F, plan, b, xs, ys, w = run_ifnso([M], L, "bf16", precision=precision, cta_group=cg)
        assert plan.get(F.IFNSO_OPT_CTA_GROUP) == cg
        st, _, _ = plan.device_status(1)
        assert st[0] == 0
        out[cg] = to_np(ys[0])
        assert rel(out[cg], O.ifnso_alg1(to_np(xs[0]), w)) < TOL["bf16"]
    assert rel(out[1], out[2]) < 1e-3


@pytest.mark.parametrize("cg", [1, 2])
def test_bf16_stage_limits_give_identical_results(cg):
    """The depth of the operand ring changes when stages are loaded, not what
    the MMAs add in which order: every pass kind limited to 2 or 3 stages
    gives the whole ring's outputs bit for bit (L = 14 mixed: Gram, split,
    plain and final squarings, FP16 product), and they match the oracle."""
    import torch

    F = lib()
    mats = [synth.gaussian(150 + i, *s) for i, s in enumerate([(512, 768), (768, 512), (300, 900), (1024, 1024)])]
    xs = [to_dev(m, "bf16") for m in mats]
    b = F.Batch(xs)
    w = coeffs(14)
    outs = []
    for lim in (0, 2, 3):
        plan = F.Plan(1024, 1024, "bf16", L=14)
        plan.set(F.IFNSO_OPT_CTA_GROUP, cg)
        plan.set(F.IFNSO_OPT_SMALL_MATRICES, 2)
        plan.set(F.IFNSO_OPT_STAGE_LIMITS, sum(lim << (4 * k) for k in range(5)))
        ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
        plan.orthogonalize(b, np.r_[1.0, w], ys)
        torch.cuda.synchronize()
        st, _, _ = plan.device_status(len(xs))
        assert np.all(st == 0)
        outs.append([to_np(y) for y in ys])
    for o in outs[1:]:
        for y0, y in zip(outs[0], o):
            assert np.array_equal(y0, y)
    for x, y in zip(xs, outs[0]):
        assert rel(y, O.ifnso_alg1(to_np(x), w)) < TOL["bf16"]


def test_autotune_chooses_stage_limits():
    """The autotuner keeps a depth per pass kind (0, 4 or 3 in each nibble)
    and the call with its choice gives the whole ring's outputs bit for bit."""
    import torch

    F = lib()
    mats = [synth.gaussian(160 + i, 1024, 2048) for i in range(6)]
    xs = [to_dev(m, "bf16") for m in mats]
    b = F.Batch(xs)
    w = np.r_[1.0, coeffs(14)]
    ref = [torch.empty_like(x) for x in xs]
    p0 = F.Plan(1024, 2048, "bf16", L=14)
    p0.orthogonalize(b, w, ref)
    plan = F.Plan(1024, 2048, "bf16", L=14)
    ys = [torch.empty_like(x) for x in xs]
    plan.autotune(b, w, ys, reps=1)
    lim = plan.get(F.IFNSO_OPT_STAGE_LIMITS)
    assert all(((lim >> (4 * k)) & 15) in (0, 3, 4) for k in range(5)) and lim >> 20 == 0
    ys = [torch.full(x.shape, float("nan"), dtype=x.dtype, device="cuda") for x in xs]
    plan.set(F.IFNSO_OPT_CTA_GROUP_KINDS, 0)  # the untuned MMA modes, as p0, with the tuned depths
    plan.orthogonalize(b, w, ys)
    torch.cuda.synchronize()
    for y0, y in zip(ref, ys):
        assert np.array_equal(to_np(y0), to_np(y))


@pytest.mark.parametrize("L,precision", [(14, "mixed"), (14, "plain"), (16, "mixed")])
def test_bf16_folded_squarings_stay_accurate(L, precision):
    """Every other squaring folds -2 D_l into its MMAs, which rounds the two
    entries (r, c) and (c, r) of a diagonal block at different points of the K
    sum.  The next squaring forms D D there (B read MN-major), under which that
    asymmetry decays; under D D^T it would double every pass.  On a
    well-conditioned input D_l converges early, and the late squarings must
    keep it exact: with the asymmetry doubling, this case reached 4.2e-2 (256 x
    512, L = 14, mixed); the unfolded squarings give 1.7e-3."""
    M = synth.gaussian(4, 256, 512)
    F, plan, b, xs, ys, w = run_ifnso([M], L, "bf16", precision=precision)
    err = rel(to_np(ys[0]), O.ifnso_alg1(to_np(xs[0]), w))
    assert err < 1e-2, err


@pytest.mark.parametrize("L,shape", [(1, (256, 512)), (4, (200, 328)), (10, (512, 256)), (14, (256, 512)),
                                     (14, (640, 1000))])
def test_bf16_gelfand2(L, shape):
    """Gelfand scaling with q = 2 (Eq. gelfand_formula): o = ||T_0^2||_F^(1/2)
    from a product of D_1 with itself, then Algorithm 1 as usual."""
    M = synth.gaussian(50 + L, *shape)
    F, plan, b, xs, ys, w = run_ifnso([M], L, "bf16", scale="gelfand2")
    assert plan.get(F.IFNSO_OPT_SCALE) == F.IFNSO_SCALE_GELFAND2
    A = to_np(xs[0])
    assert rel(to_np(ys[0]), O.ifnso_alg1(A, w, "gelfand2")) < TOL["bf16"]
    st, s2, _ = plan.device_status(1)
    assert st[0] == 0
    At = O.orient(A)[0]
    assert abs(s2[0] - O.scale_of(At, "gelfand2") ** 2) < 1e-3 * O.scale_of(At, "gelfand2") ** 2


def test_bf16_split_squarings_option():
    """IFNSO_OPT_SPLIT_SQUARINGS moves the split/plain boundary of the mixed
    precision: 5 split squarings or all 13, on a well-conditioned input where
    both stay within the tolerance (the precision margin itself is measured
    on hard inputs separately); the two results differ, so the option acts."""
    import torch

    M = synth.gaussian(3, 512, 768)
    F = lib()
    x = to_dev(M, "bf16")
    w = coeffs(14)
    ref = O.ifnso_alg1(to_np(x), w)
    out = {}
    for k in (5, 13):
        y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
        plan = F.Plan(512, 768, "bf16", L=14)
        plan.set(F.IFNSO_OPT_SPLIT_SQUARINGS, k)
        assert plan.get(F.IFNSO_OPT_SPLIT_SQUARINGS) == k
        plan.orthogonalize(F.Batch([x]), np.r_[1.0, w], [y])
        torch.cuda.synchronize()
        out[k] = to_np(y)
        assert rel(out[k], ref) < TOL["bf16"]
    assert not np.array_equal(out[5], out[13])


@pytest.mark.parametrize("cg", [1, 2])
def test_bf16_gelfand2_cta_groups(cg):
    M = synth.gaussian(61, 512, 768)
    F, plan, b, xs, ys, w = run_ifnso([M], 10, "bf16", scale="gelfand2", cta_group=cg)
    assert rel(to_np(ys[0]), O.ifnso_alg1(to_np(xs[0]), w, "gelfand2")) < TOL["bf16"]


def test_bf16_gelfand2_zero_and_batch():
    import torch

    Z = np.zeros((256, 512))
    M = synth.gaussian(7, 200, 328)
    F, plan, b, xs, ys, w = run_ifnso([Z, M], 6, "bf16", scale="gelfand2")
    st, _, _ = plan.device_status(2)
    assert st[0] & F.IFNSO_DEV_ZERO_INPUT and st[1] == 0
    assert torch.all(ys[0] == 0)
    assert rel(to_np(ys[1]), O.ifnso_alg1(to_np(xs[1]), w, "gelfand2")) < TOL["bf16"]


@pytest.mark.parametrize("cg", [1, 2])
def test_bf16_ns_cta_groups(cg):
    import torch

    F = lib()
    M = synth.gaussian(41, 392, 136)
    x = to_dev(M, "bf16")
    y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
    plan = F.Plan(136, 392, "bf16", L=1)
    plan.set(F.IFNSO_OPT_CTA_GROUP, cg)
    plan.ns_iterate(F.Batch([x]), ONS.MUON_ABC, 5, [y])
    torch.cuda.synchronize()
    assert rel(to_np(y), ONS.ns_generic(to_np(x), ONS.MUON_ABC, 5)) < 5e-2


def test_bf16_batch_heterogeneous():
    shapes = [(256, 512), (392, 136), (200, 328), (512, 512), (130, 260), (1, 64)]
    mats = [synth.gaussian(10 + i, *s) for i, s in enumerate(shapes)]
    F, plan, b, xs, ys, w = run_ifnso(mats, 6, "bf16")
    for x, y in zip(xs, ys):
        assert rel(to_np(y), O.ifnso_alg1(to_np(x), w)) < TOL["bf16"]


def test_bf16_zero_and_scale_invariance():
    import torch

    Z = np.zeros((128, 256))
    M = synth.gaussian(6, 128, 256)
    F, plan, b, xs, ys, w = run_ifnso([Z, M, 1000.0 * M], 4, "bf16")
    assert torch.all(ys[0] == 0)
    st, s2, tr = plan.device_status(3)
    assert st[0] & F.IFNSO_DEV_ZERO_INPUT and st[1] == 0 and st[2] == 0
    # the output does not depend on the scale of the input (up to BF16 rounding of 1000 M)
    assert rel(to_np(ys[2]), O.ifnso_alg1(to_np(xs[2]), w)) < TOL["bf16"]


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_nonfinite_input_is_flagged_and_isolated(dtype):
    """A matrix holding a NaN (or an Inf) gets IFNSO_DEV_NONFINITE; the other
    matrices of the same call are unaffected (their scalars, tiles and
    results are their own)."""
    M = synth.gaussian(8, 128, 256)
    bad_nan = M.copy()
    bad_nan[5, 7] = np.nan
    bad_inf = M.copy()
    bad_inf[100, 200] = np.inf
    F, plan, b, xs, ys, w = run_ifnso([bad_nan, M, bad_inf], 6, dtype)
    st, _, _ = plan.device_status(3)
    assert st[0] & F.IFNSO_DEV_NONFINITE and st[2] & F.IFNSO_DEV_NONFINITE and st[1] == 0
    assert rel(to_np(ys[1]), O.ifnso_alg1(to_np(xs[1]), w)) < TOL[dtype]


def test_empty_batch_is_a_no_op():
    import torch

    F = lib()
    plan = F.Plan(128, 256, "bf16", L=4)
    before = F.launch_count()
    plan.orthogonalize(F.Batch([]), np.r_[1.0, coeffs(4)], [], ws=F.Workspace(1024, device=torch.device("cuda")))
    torch.cuda.synchronize()
    assert F.launch_count() == before


@pytest.mark.parametrize("shape", [(256, 512), (392, 136)])
def test_bf16_ns(shape):
    import torch

    F = lib()
    M = synth.gaussian(7, *shape)
    x = to_dev(M, "bf16")
    for poly, steps in [(ONS.MUON_ABC, 5), (ONS.CUBIC, 8)]:
        y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
        plan = F.Plan(min(shape), max(shape), "bf16", L=1)
        plan.ns_iterate(F.Batch([x]), poly, steps, [y])
        torch.cuda.synchronize()
        ref = ONS.ns_generic(to_np(x), poly, steps)
        # BF16 storage of X, X X^T and B every step: 5e-2 relative
        assert rel(to_np(y), ref) < 5e-2


# --------------------------------------------------------------- E4M3 Gram (experiment)
def e4m3_round(x):
    """Round to the nearest E4M3 value, ties to even, saturating at +-448
    (E4M3: 3 mantissa bits, normals down to 2^-6, subnormal spacing 2^-9)."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    q = 2.0 ** (e - 3)
    r = np.round(a / q) * q
    return np.sign(x) * np.minimum(r, 448.0)


def e4m3_scale(amax):
    """The power of two s with amax * s in (224, 448]."""
    s = 2.0 ** np.floor(np.log2(448.0 / amax))
    return s / 2 if amax * s > 448.0 else s


@pytest.mark.parametrize("shape", [(256, 512), (392, 136), (640, 1000), (1000, 640)])
def test_bf16_gram_e4m3(shape):
    """T_0 from the E4M3 copy of A s equals the FP64 Gram of the rounded copy / s^2."""
    import torch

    F = lib()
    M = synth.gaussian(80, *shape)
    x = to_dev(M, "bf16")
    h, w = min(shape), max(shape)
    plan = F.Plan(h, w, "bf16", L=4)
    plan.set(F.IFNSO_OPT_GRAM_E4M3, 1)
    plan.set(F.IFNSO_OPT_STOP_AFTER, 0)
    b = F.Batch([x])
    y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
    plan.orthogonalize(b, np.r_[1.0, coeffs(4)], [y])
    torch.cuda.synchronize()
    ptr, ld = plan.workspace_view(b, 0, 0)
    G = sym_upper(F.tensor_at(ptr, (ld, ld), torch.float32, plan._last_ws.buf).double().cpu().numpy())
    A = O.orient(to_np(x))[0]
    s = e4m3_scale(np.max(np.abs(A)))
    Aq = e4m3_round(A * s)
    ref = (Aq @ Aq.T) / (s * s)
    assert rel(G[:h, :h], ref) < 1e-5
    st, s2, tr = plan.device_status(1)
    assert st[0] == 0 and abs(s2[0] - np.linalg.norm(ref)) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("shape", [(256, 512), (392, 136)])
def test_bf16_ifnso_gram_e4m3_end_to_end(shape):
    """The whole path with the E4M3 Gram, against Algorithm 1 on the BF16 input:
    the error the 3-bit mantissa of the first product costs (reported)."""
    M = synth.gaussian(81, *shape)
    F = lib()
    import torch

    x = to_dev(M, "bf16")
    y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
    plan = F.Plan(min(shape), max(shape), "bf16", L=4)
    plan.set(F.IFNSO_OPT_GRAM_E4M3, 1)
    w = coeffs(4)
    plan.orthogonalize(F.Batch([x]), np.r_[1.0, w], [y])
    torch.cuda.synchronize()
    err = rel(to_np(y), O.ifnso_alg1(to_np(x), w))
    print(f"E4M3 Gram {shape}: relative error {err:.3e}")
    assert err < 0.1


def test_autotune_keeps_results():
    """Autotuning picks a mode per pass kind; results stay those of the oracle
    and agree with the untuned plan to rounding order."""
    import torch

    F = lib()
    shapes = [(512, 1024), (768, 640), (256, 512)]
    mats = [synth.gaussian(90 + i, *s) for i, s in enumerate(shapes)]
    xs = [to_dev(m, "bf16") for m in mats]
    L = 10
    w = np.r_[1.0, coeffs(L)]
    plan = F.Plan(768, 1024, "bf16", L=L)
    b = F.Batch(xs)
    ref = [torch.empty(x.shape, dtype=x.dtype, device=x.device) for x in xs]
    plan.orthogonalize(b, w, ref)
    torch.cuda.synchronize()
    outs = [torch.empty(x.shape, dtype=x.dtype, device=x.device) for x in xs]
    chosen = plan.autotune(b, w, outs, reps=2)
    assert len(chosen) == 4 and all(c in (1, 2) for c in chosen)
    assert plan.get(F.IFNSO_OPT_CTA_GROUP) == 0
    plan.orthogonalize(b, w, outs)
    torch.cuda.synchronize()
    for x, y, r in zip(xs, outs, ref):
        assert rel(to_np(y), to_np(r)) < 1e-3
        assert rel(to_np(y), O.ifnso_alg1(to_np(x), w[1:])) < TOL["bf16"]


# --------------------------------------------------------------- pass timing
def test_pass_times_follow_the_latest_graph():
    """A captured call has no times before its graph's first replay (the
    query skips it); a second capture replaces the first in the query."""
    import torch

    F = lib()
    xs = [to_dev(synth.gaussian(50, 256, 512), "bf16")]
    ys = [torch.empty_like(xs[0])]
    w = coeffs(6)
    plan = F.Plan(256, 512, "bf16", L=6)
    plan.set(F.IFNSO_OPT_TIMING, 1)
    b = F.Batch(xs)
    plan.orthogonalize(b, np.r_[1.0, w], ys)
    torch.cuda.synchronize()
    ms, calls = plan.pass_times()
    assert calls == 1 and len(ms) >= 7 and all(t > 0 for t in ms[:7])
    graphs = []
    for _ in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.orthogonalize(b, np.r_[1.0, w], ys)
        torch.cuda.synchronize()
        ms, calls = plan.pass_times()  # not replayed yet: nothing to report, no error
        assert calls == 0
        g.replay()
        torch.cuda.synchronize()
        ms, calls = plan.pass_times()
        assert calls == 1 and all(t > 0 for t in ms[:7])
        graphs.append(g)
    graphs[0].replay()  # the first graph still replays; its events are not followed
    torch.cuda.synchronize()
    assert rel(to_np(ys[0]), O.ifnso_alg1(to_np(xs[0]), w)) < TOL["bf16"]
