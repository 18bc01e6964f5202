"""The C-ABI library loads and exports every entry point include/ifnso.h
declares; host-side validation and workspace sizing (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2602_02500_gb300 import _build

    _build.build()
    from paper_2602_02500_gb300 import ifnso

    return ifnso


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ifnso.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)))


def test_exports_every_declared_symbol(F):
    names = header_functions()
    assert "ifnso_orthogonalize" in names and "ns_iterate" in names and "ifnso_plan_create" in names
    lib = C.CDLL(F._LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(F.EXPORTED)


def _plan(F, h, w, L, dtype=1):
    K = L + 1
    ex = (C.c_int32 * K)(*([0] + [1 << (l - 1) for l in range(1, K)]))
    p = C.c_void_p()
    st = F.ifnso_plan_create(C.byref(p), h, w, dtype, ex, K)
    return st, p


def test_plan_validation(F):
    st, p = _plan(F, 128, 256, 4)
    assert st == F.IFNSO_OK
    F.ifnso_plan_destroy(p)
    # exponents must be 0, 1, 2, 4, ... (repeated squaring)
    ex = (C.c_int32 * 4)(0, 1, 3, 4)
    q = C.c_void_p()
    assert F.ifnso_plan_create(C.byref(q), 128, 256, 1, ex, 4) == F.IFNSO_ERR_INVALID_ARG
    assert b"repeated squaring" in F.ifnso_last_error()
    assert F.ifnso_plan_create(C.byref(q), 300, 256, 1, (C.c_int32 * 2)(0, 1), 2) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_create(C.byref(q), 8, 8, 1, (C.c_int32 * 1)(0), 1) == F.IFNSO_ERR_INVALID_ARG


def _fake_batch(F, shapes, ld=None, base=1 << 30):
    n = len(shapes)
    ptrs = (C.c_void_p * n)(*[base + (i << 24) for i in range(n)])
    rows = (C.c_int64 * n)(*[s[0] for s in shapes])
    cols = (C.c_int64 * n)(*[s[1] for s in shapes])
    lds = (C.c_int64 * n)(*(ld or [s[1] for s in shapes]))
    d = F.ifnso_batch_desc(n, ptrs, rows, cols, lds)
    return d, (ptrs, rows, cols, lds)


def test_workspace_sizes(F):
    st, p = _plan(F, 2048, 5632, 14)
    d, keep = _fake_batch(F, [(2048, 2048), (2048, 5632), (5632, 2048)])
    split = F.ifnso_workspace_bytes(p, C.byref(d))
    F.ifnso_plan_set(p, F.IFNSO_OPT_PRECISION, F.IFNSO_PREC_PLAIN)
    plain = F.ifnso_workspace_bytes(p, C.byref(d))
    hp2 = 2048 * 2048
    # the MIXED plan (L = 14) also holds the FP16 copy of every input for its
    # FP16 final product (on by default); PLAIN plans take one BF16 product
    a16 = 2 * (2048 * 2048 + 2048 * 5632 + 5632 * 2048)
    assert 3 * 12 * hp2 + a16 <= split < 3 * 12 * hp2 + a16 + (4 << 20)
    assert 3 * 8 * hp2 <= plain < 3 * 8 * hp2 + (4 << 20)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_PRECISION, C.byref(v)) == 0 and v.value == F.IFNSO_PREC_PLAIN
    F.ifnso_plan_destroy(p)


def test_batch_validation(F):
    st, p = _plan(F, 256, 512, 4)
    d, keep = _fake_batch(F, [(256, 500)], ld=[500])   # BF16 ld must be a multiple of 8
    assert F.ifnso_workspace_bytes(p, C.byref(d)) == 0
    assert b"multiple of 8" in F.ifnso_last_error()
    d, keep = _fake_batch(F, [(300, 512)])               # oriented 300 x 512 exceeds 256 x 512
    assert F.ifnso_workspace_bytes(p, C.byref(d)) == 0
    d, keep = _fake_batch(F, [(512, 200)])               # tall: oriented 200 x 512 fits
    assert F.ifnso_workspace_bytes(p, C.byref(d)) > 0
    d, keep = _fake_batch(F, [(0, 5)])
    assert F.ifnso_workspace_bytes(p, C.byref(d)) == 0
    F.ifnso_plan_destroy(p)


def test_learn_argument_checks(F):
    w = (C.c_double * 4)()
    assert F.ifnso_learn_coefficients(0, 10, 100, 0.1, 10, 0.5, 0, w) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_learn_coefficients(4, 10, 5000, 0.1, 10, 0.5, 0, w) == F.IFNSO_ERR_INVALID_ARG


def test_precision_resolution(F):
    # AUTO: plain for L <= 4, mixed (first L - 8 squarings split, P split) for 5..14, split above
    for L, mode in [(4, F.IFNSO_PREC_PLAIN), (5, F.IFNSO_PREC_MIXED), (14, F.IFNSO_PREC_MIXED),
                    (15, F.IFNSO_PREC_SPLIT)]:
        st, p = _plan(F, 256, 512, L)
        v = C.c_int64()
        assert F.ifnso_plan_get(p, F.IFNSO_OPT_PRECISION, C.byref(v)) == 0
        assert v.value == mode, (L, v.value)
        F.ifnso_plan_destroy(p)


def test_cta_group_option(F):
    # default: automatic choice per pass; 0, 1 and 2 are the only accepted values
    st, p = _plan(F, 256, 512, 4)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_CTA_GROUP, C.byref(v)) == 0 and v.value == 0
    for bad in (3, -1, 4):
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_CTA_GROUP, bad) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_CTA_GROUP, 2) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_CTA_GROUP, C.byref(v)) == 0 and v.value == 2
    F.ifnso_plan_destroy(p)


def test_apply_f16_option(F):
    # on by default for MIXED-precision BF16 plans (AUTO for 5 <= L <= 14; the
    # others keep their products); only 0 and 1; the workspace holds the FP16
    # copy of the input (2 bytes per element, rows padded to 8) only when it is on
    st, p = _plan(F, 256, 512, 14)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_APPLY_F16, C.byref(v)) == 0 and v.value == 1
    for bad in (2, -1):
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_APPLY_F16, bad) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_APPLY_F16, 0) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_APPLY_F16, C.byref(v)) == 0 and v.value == 0
    d, keep = _fake_batch(F, [(256, 504)])
    before = F.ifnso_workspace_bytes(p, C.byref(d))
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_APPLY_F16, 1) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_APPLY_F16, C.byref(v)) == 0 and v.value == 1
    after = F.ifnso_workspace_bytes(p, C.byref(d))
    assert before > 0 and after >= before + 256 * 504 * 2
    F.ifnso_plan_destroy(p)
    # where the last call wrote the copy: read only, 0 before any call
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_FP16_COPY_HOSTS, C.byref(v)) == 0 and v.value == 0
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_FP16_COPY_HOSTS, 6) == F.IFNSO_ERR_INVALID_ARG
    for L in (1, 4, 16):  # L = 1 has no squarings; L = 4 is PLAIN (one BF16 P), L = 16 SPLIT
        st, p = _plan(F, 256, 512, L)
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_APPLY_F16, 1) == 0
        assert F.ifnso_plan_get(p, F.IFNSO_OPT_APPLY_F16, C.byref(v)) == 0 and v.value == 0
        F.ifnso_plan_destroy(p)


def test_stage_limits_option(F):
    # 4 bits per pass kind (Gram, split, plain, product, final squaring); 0 is
    # the whole ring, 1 and anything beyond 20 bits are rejected
    st, p = _plan(F, 256, 512, 14)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_STAGE_LIMITS, C.byref(v)) == 0 and v.value == 0
    packed = 3 << 16 | 3 << 12 | 4 << 8
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_STAGE_LIMITS, packed) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_STAGE_LIMITS, C.byref(v)) == 0 and v.value == packed
    for bad in (1, 1 << 8, 1 << 20, -1):
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_STAGE_LIMITS, bad) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_STAGE_LIMITS, C.byref(v)) == 0 and v.value == packed
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_STAGE_LIMITS, 0) == 0
    F.ifnso_plan_destroy(p)


def test_host_entry_argument_checks(F):
    # NULL host buffers are rejected before any device work
    st, p = _plan(F, 256, 512, 4)
    w = (C.c_double * 5)(1.0, 0.1, 0.2, 0.3, 0.4)
    cf = F.ifnso_coeffs(5, w, None, None)
    ptrs = (C.c_void_p * 1)(16 * 1024)
    rows = (C.c_int64 * 1)(256)
    cols = (C.c_int64 * 1)(512)
    desc = F.ifnso_batch_desc(1, ptrs, rows, cols, None)
    outs = (C.c_void_p * 1)(32 * 1024)
    nulls = (C.c_void_p * 1)(None)
    assert F.ifnso_orthogonalize_host(p, None, C.byref(desc), C.byref(cf), outs, outs, None, 0, 0,
                                      None) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_orthogonalize_host(p, nulls, C.byref(desc), C.byref(cf), outs, outs, None, 0, 0,
                                      None) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_orthogonalize_host(None, nulls, C.byref(desc), C.byref(cf), outs, outs, None, 0, 0,
                                      None) == F.IFNSO_ERR_INVALID_ARG
    F.ifnso_plan_destroy(p)


def test_scale_option(F):
    st, p = _plan(F, 256, 512, 4)
    v = C.c_int64()
    for val in (F.IFNSO_SCALE_GRAM, F.IFNSO_SCALE_FROB, F.IFNSO_SCALE_GELFAND2):
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_SCALE, val) == 0
        assert F.ifnso_plan_get(p, F.IFNSO_OPT_SCALE, C.byref(v)) == 0 and v.value == val
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_SCALE, 3) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_SCALE, -1) == F.IFNSO_ERR_INVALID_ARG
    F.ifnso_plan_destroy(p)


def test_split_squarings_option(F):
    st, p = _plan(F, 256, 512, 14)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_SPLIT_SQUARINGS, C.byref(v)) == 0 and v.value == 6  # AUTO -> MIXED: L - 8
    for n, eff in [(0, 0), (3, 3), (13, 13), (30, 13), (-1, 6)]:
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_SPLIT_SQUARINGS, n) == 0
        assert F.ifnso_plan_get(p, F.IFNSO_OPT_SPLIT_SQUARINGS, C.byref(v)) == 0 and v.value == eff
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_SPLIT_SQUARINGS, -2) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_SPLIT_SQUARINGS, 31) == F.IFNSO_ERR_INVALID_ARG
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_SPLIT_SQUARINGS, 4) == 0
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_PRECISION, F.IFNSO_PREC_SPLIT) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_SPLIT_SQUARINGS, C.byref(v)) == 0 and v.value == 13
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_PRECISION, F.IFNSO_PREC_PLAIN) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_SPLIT_SQUARINGS, C.byref(v)) == 0 and v.value == 0
    F.ifnso_plan_destroy(p)


def test_host_streams_option(F):
    st, p = _plan(F, 256, 512, 6)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_HOST_STREAMS, C.byref(v)) == 0 and v.value == 2
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_HOST_STREAMS, 1) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_HOST_STREAMS, C.byref(v)) == 0 and v.value == 1
    for bad in (0, 3, -1):
        assert F.ifnso_plan_set(p, F.IFNSO_OPT_HOST_STREAMS, bad) == F.IFNSO_ERR_INVALID_ARG
    F.ifnso_plan_destroy(p)


def test_muon_step_argument_checks(F):
    # every argument error is reported before any device work
    st, p = _plan(F, 256, 512, 4)
    w = (C.c_double * 5)(1.0, 0.1, 0.2, 0.3, 0.4)
    cf = F.ifnso_coeffs(5, w, None, None)
    g = (C.c_void_p * 1)(16 * 1024)
    rows = (C.c_int64 * 1)(256)
    cols = (C.c_int64 * 1)(512)
    desc = F.ifnso_batch_desc(1, g, rows, cols, None)
    m = (C.c_void_p * 1)(32 * 1024)
    u = (C.c_void_p * 1)(48 * 1024)
    wt = (C.c_void_p * 1)(64 * 1024)
    bad = F.IFNSO_ERR_INVALID_ARG

    def call(plan=p, mom=m, stg=u, wts=wt, beta=0.95, nesterov=1, lr=0.02):
        return F.ifnso_muon_step(plan, C.byref(desc), mom, stg, wts, C.byref(cf), beta, nesterov, lr, None, 0, None)

    assert call(plan=None) == bad
    assert call(mom=None) == bad and call(stg=None) == bad and call(wts=None) == bad
    assert call(beta=1.0) == bad and call(beta=-0.1) == bad and call(beta=float("nan")) == bad
    assert call(lr=-1.0) == bad and call(lr=float("inf")) == bad
    assert call(nesterov=2) == bad
    assert call(wts=(C.c_void_p * 1)(48 * 1024)) == bad        # weights alias the staging buffer
    assert call(stg=(C.c_void_p * 1)(16 * 1024)) == bad        # staging aliases the gradient
    assert call(mom=(C.c_void_p * 1)(64 * 1024 + 8)) == bad    # misaligned momentum
    assert call(mom=(C.c_void_p * 1)(None)) == bad
    F.ifnso_plan_destroy(p)
    st, p = _plan(F, 256, 512, 4, dtype=0)  # F32 plans have no Muon step
    assert call(plan=p) == F.IFNSO_ERR_UNSUPPORTED
    F.ifnso_plan_destroy(p)


def test_gram_e4m3_option(F):
    st, p = _plan(F, 256, 512, 4)
    v = C.c_int64()
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_GRAM_E4M3, C.byref(v)) == 0 and v.value == 0
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_GRAM_E4M3, 1) == 0
    assert F.ifnso_plan_get(p, F.IFNSO_OPT_GRAM_E4M3, C.byref(v)) == 0 and v.value == 1
    F.ifnso_plan_destroy(p)
    st, p = _plan(F, 256, 512, 4, dtype=0)  # F32 plans have no E4M3 Gram
    assert F.ifnso_plan_set(p, F.IFNSO_OPT_GRAM_E4M3, 1) == F.IFNSO_ERR_UNSUPPORTED
    F.ifnso_plan_destroy(p)


def test_autotune_argument_checks(F):
    st, p = _plan(F, 256, 512, 4)
    w = (C.c_double * 5)(1.0, 0.1, 0.2, 0.3, 0.4)
    cf = F.ifnso_coeffs(5, w, None, None)
    ptrs = (C.c_void_p * 1)(16 * 1024)
    rows = (C.c_int64 * 1)(256)
    cols = (C.c_int64 * 1)(512)
    desc = F.ifnso_batch_desc(1, ptrs, rows, cols, None)
    outs = (C.c_void_p * 1)(32 * 1024)
    for reps in (0, 101):
        assert F.ifnso_plan_autotune(p, C.byref(desc), C.byref(cf), outs, None, 0, reps, None,
                                     None) == F.IFNSO_ERR_INVALID_ARG
    F.ifnso_plan_destroy(p)
    st, p = _plan(F, 256, 512, 4, dtype=0)
    assert F.ifnso_plan_autotune(p, C.byref(desc), C.byref(cf), outs, None, 0, 2, None,
                                 None) == F.IFNSO_ERR_UNSUPPORTED
    F.ifnso_plan_destroy(p)
