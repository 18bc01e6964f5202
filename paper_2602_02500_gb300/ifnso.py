"""Python binding of libifnso.so (include/ifnso.h): argument marshalling only.

Every function of the C ABI is exposed under its own name with plain
integers / device pointers, plus ``Plan``, a small convenience wrapper that
takes torch tensors (device memory and streams come from PyTorch; all
computation runs in the library's kernels).  Importing this module loads the
library and raises ImportError if it has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libifnso.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2602_02500_gb300._build.build() "
                      "(or __graft_entry__.build()); there is no non-CUDA fallback")
lib = C.CDLL(_LIB_PATH)

# status codes / enums (include/ifnso.h)
IFNSO_OK = 0
IFNSO_ERR_INVALID_ARG = 1
IFNSO_ERR_UNSUPPORTED = 2
IFNSO_ERR_OOM = 3
IFNSO_ERR_CUDA = 4
IFNSO_ERR_DEVICE_TIMEOUT = 5
IFNSO_ERR_WORKSPACE = 6
IFNSO_F32 = 0
IFNSO_BF16 = 1
IFNSO_OPT_PRECISION = 1
IFNSO_OPT_SCALE = 2
IFNSO_OPT_MAX_CTAS = 3
IFNSO_OPT_STOP_AFTER = 4
IFNSO_OPT_TIMING = 5
IFNSO_OPT_WAIT_LIMIT_MS = 6
IFNSO_OPT_INJECT_STALL = 7
IFNSO_OPT_CTA_GROUP = 8
IFNSO_OPT_GRAM_E4M3 = 9
IFNSO_OPT_SPLIT_SQUARINGS = 10
IFNSO_OPT_HOST_STREAMS = 11
IFNSO_OPT_SMALL_MATRICES = 12
IFNSO_OPT_SMALL_TUNED = 13
IFNSO_OPT_CTA_GROUP_KINDS = 14
IFNSO_OPT_APPLY_F16 = 15
IFNSO_OPT_FP16_COPY_HOSTS = 16
IFNSO_OPT_STAGE_LIMITS = 17
IFNSO_PREC_AUTO, IFNSO_PREC_PLAIN, IFNSO_PREC_SPLIT, IFNSO_PREC_MIXED = 0, 1, 2, 3
IFNSO_SCALE_GRAM, IFNSO_SCALE_FROB, IFNSO_SCALE_GELFAND2 = 0, 1, 2
IFNSO_DEV_ZERO_INPUT, IFNSO_DEV_NONFINITE, IFNSO_DEV_TIMEOUT = 1, 2, 4
IFNSO_STATIC_NORM_MAX_MATRICES = 1024

EXPORTED = [
    "ifnso_plan_create", "ifnso_plan_set", "ifnso_plan_get", "ifnso_plan_destroy",
    "ifnso_workspace_bytes", "ifnso_orthogonalize", "ifnso_orthogonalize_host", "ifnso_plan_autotune",
    "ifnso_muon_step", "ns_iterate",
    "ns_workspace_bytes",
    "ifnso_device_status", "ifnso_workspace_view", "ifnso_pass_times", "ifnso_host_timeline",
    "ifnso_frobenius_norm2",
    "ifnso_frobenius_norm2_static", "ifnso_learn_coefficients", "ifnso_synth_lowrank_bf16", "ifnso_last_error",
    "ifnso_launch_count", "ifnso_mlp_param_count", "ifnso_mlp_create", "ifnso_mlp_destroy",
    "ifnso_mlp_get_params", "ifnso_mlp_set_params", "ifnso_mlp_set_data", "ifnso_mlp_loss_grad",
    "ifnso_mlp_train", "ifnso_mlp_evaluate",
]


class ifnso_batch_desc(C.Structure):
    _fields_ = [("count", C.c_int32), ("in_", C.POINTER(C.c_void_p)), ("rows", C.POINTER(C.c_int64)),
                ("cols", C.POINTER(C.c_int64)), ("ld", C.POINTER(C.c_int64))]


class ifnso_coeffs(C.Structure):
    _fields_ = [("K", C.c_int32), ("host", C.POINTER(C.c_double)), ("device", C.c_void_p), ("mlp", C.c_void_p)]


_P = C.c_void_p
_sig = {
    "ifnso_plan_create": (C.c_int, [C.POINTER(_P), C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_int32), C.c_int32]),
    "ifnso_plan_set": (C.c_int, [_P, C.c_int, C.c_int64]),
    "ifnso_plan_get": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64)]),
    "ifnso_plan_destroy": (C.c_int, [_P]),
    "ifnso_workspace_bytes": (C.c_size_t, [_P, C.POINTER(ifnso_batch_desc)]),
    "ns_workspace_bytes": (C.c_size_t, [_P, C.POINTER(ifnso_batch_desc)]),
    "ifnso_orthogonalize": (C.c_int, [_P, C.POINTER(ifnso_batch_desc), C.POINTER(ifnso_coeffs),
                                      C.POINTER(_P), _P, C.c_size_t, _P]),
    "ifnso_plan_autotune": (C.c_int, [_P, C.POINTER(ifnso_batch_desc), C.POINTER(ifnso_coeffs), C.POINTER(_P), _P,
                                      C.c_size_t, C.c_int32, C.POINTER(C.c_int32), _P]),
    "ifnso_orthogonalize_host": (C.c_int, [_P, C.POINTER(_P), C.POINTER(ifnso_batch_desc), C.POINTER(ifnso_coeffs),
                                           C.POINTER(_P), C.POINTER(_P), _P, C.c_size_t, C.c_int32, _P]),
    "ifnso_muon_step": (C.c_int, [_P, C.POINTER(ifnso_batch_desc), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                  C.POINTER(ifnso_coeffs), C.c_double, C.c_int32, C.c_double, _P, C.c_size_t, _P]),
    "ns_iterate": (C.c_int, [_P, C.POINTER(ifnso_batch_desc), C.POINTER(C.c_double), C.c_int32, C.c_int32,
                             C.POINTER(_P), _P, C.c_size_t, _P]),
    "ifnso_device_status": (C.c_int, [_P, _P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), _P]),
    "ifnso_pass_times": (C.c_int, [_P, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "ifnso_host_timeline": (C.c_int, [_P, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32)]),
    "ifnso_workspace_view": (C.c_int, [_P, C.POINTER(ifnso_batch_desc), _P, C.c_int32, C.c_int32,
                                       C.POINTER(_P), C.POINTER(C.c_int64)]),
    "ifnso_frobenius_norm2": (C.c_int, [C.POINTER(ifnso_batch_desc), C.c_int, _P, _P]),
    "ifnso_frobenius_norm2_static": (C.c_int, [C.POINTER(ifnso_batch_desc), C.c_int, _P, _P]),
    "ifnso_learn_coefficients": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int32, C.c_double,
                                           C.c_uint32, C.POINTER(C.c_double)]),
    "ifnso_synth_lowrank_bf16": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, C.c_uint32, C.c_float, C.c_float, _P]),
    "ifnso_mlp_param_count": (C.c_int32, [C.c_int32]),
    "ifnso_mlp_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(C.c_double), _P, C.c_uint32]),
    "ifnso_mlp_destroy": (C.c_int, [_P]),
    "ifnso_mlp_get_params": (C.c_int, [_P, _P, _P]),
    "ifnso_mlp_set_params": (C.c_int, [_P, _P, _P]),
    "ifnso_mlp_set_data": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_int32, _P]),
    "ifnso_mlp_loss_grad": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P]),
    "ifnso_mlp_train": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_float, C.c_uint32, _P, _P]),
    "ifnso_mlp_evaluate": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P, _P]),
    "ifnso_last_error": (C.c_char_p, []),
    "ifnso_launch_count": (C.c_uint64, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class IfnsoError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where} failed with status {status}: {ifnso_last_error().decode()}")


def check(status, where):
    if status != IFNSO_OK:
        raise IfnsoError(status, where)


# ------------------------------------------------------------ torch helpers

def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.bfloat16:
        return IFNSO_BF16
    if t.dtype == torch.float32:
        return IFNSO_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


class Batch:
    """Keeps the ctypes arrays of an ifnso_batch_desc alive."""

    def __init__(self, mats):
        n = len(mats)
        for m in mats:
            if not m.is_cuda or m.dim() != 2 or m.stride(1) != 1:
                raise ValueError("matrices must be 2-D CUDA tensors with unit column stride")
        self.mats = list(mats)
        self.ptrs = (C.c_void_p * max(n, 1))(*[m.data_ptr() for m in mats])
        self.rows = (C.c_int64 * max(n, 1))(*[m.shape[0] for m in mats])
        self.cols = (C.c_int64 * max(n, 1))(*[m.shape[1] for m in mats])
        self.ld = (C.c_int64 * max(n, 1))(*[m.stride(0) for m in mats])
        self.desc = ifnso_batch_desc(n, self.ptrs, self.rows, self.cols, self.ld)

    def ref(self):
        return C.byref(self.desc)


class Workspace:
    """Device workspace with the 1024-byte alignment the library requires."""

    def __init__(self, nbytes, device=None):
        torch = _torch()
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes + 1024, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.ptr = (base + 1023) // 1024 * 1024

    def view(self, offset, count, dtype):
        """Tensor view of `count` elements of `dtype` at byte offset `offset`."""
        torch = _torch()
        esz = torch.empty((), dtype=dtype).element_size()
        start = self.ptr - self.buf.data_ptr() + offset
        return self.buf[start:start + count * esz].view(dtype)


class Plan:
    """ifnso_plan for oriented shapes up to h x w and depth L (exponents 0, 1, 2, ..., 2^(L-1))."""

    def __init__(self, h, w, dtype="bf16", L=4, precision=None, scale=None, max_ctas=None):
        self.L = int(L)
        K = self.L + 1
        ex = (C.c_int32 * K)(*([0] + [1 << (l - 1) for l in range(1, K)]))
        self.dtype = IFNSO_BF16 if dtype in ("bf16", IFNSO_BF16) else IFNSO_F32
        h_ = C.c_void_p()
        check(ifnso_plan_create(C.byref(h_), int(h), int(w), self.dtype, ex, K), "ifnso_plan_create")
        self.handle = h_
        if precision is not None:
            self.set(IFNSO_OPT_PRECISION, {"auto": 0, "plain": 1, "split": 2, "mixed": 3}.get(precision, precision))
        if scale is not None:
            self.set(IFNSO_OPT_SCALE, {"gram": 0, "frob": 1, "gelfand2": 2}.get(scale, scale))
        if max_ctas is not None:
            self.set(IFNSO_OPT_MAX_CTAS, max_ctas)
        self._ws = None

    def set(self, opt, value):
        check(ifnso_plan_set(self.handle, opt, int(value)), "ifnso_plan_set")

    def get(self, opt):
        v = C.c_int64()
        check(ifnso_plan_get(self.handle, opt, C.byref(v)), "ifnso_plan_get")
        return v.value

    def close(self):
        if getattr(self, "handle", None):
            ifnso_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- sizes
    def workspace_bytes(self, batch):
        n = ifnso_workspace_bytes(self.handle, batch.ref())
        if n == 0 and batch.desc.count > 0:
            raise IfnsoError(IFNSO_ERR_INVALID_ARG, "ifnso_workspace_bytes")
        return n

    def ns_workspace_bytes(self, batch):
        n = ns_workspace_bytes(self.handle, batch.ref())
        if n == 0 and batch.desc.count > 0:
            raise IfnsoError(IFNSO_ERR_INVALID_ARG, "ns_workspace_bytes")
        return n

    def workspace(self, nbytes):
        if self._ws is None or self._ws.nbytes < nbytes:
            self._ws = Workspace(nbytes)
        return self._ws

    # -------------------------------------------------------------- calls
    def _coeffs(self, batch, coeffs):
        torch = _torch()
        K = self.L + 1
        if isinstance(coeffs, torch.Tensor) and coeffs.is_cuda:
            if coeffs.dtype != torch.float32 or coeffs.shape != (batch.desc.count, K) or not coeffs.is_contiguous():
                raise ValueError("device coefficients must be contiguous float32 of shape (count, L + 1)")
            self._cf_keep = coeffs
            cf = ifnso_coeffs(K, None, C.c_void_p(coeffs.data_ptr()), None)
        elif isinstance(coeffs, Mlp):
            self._cf_keep = coeffs
            cf = ifnso_coeffs(K, None, None, coeffs.handle)
        else:
            arr = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
            if arr.shape != (K,):
                raise ValueError(f"host coefficients must have K = {K} values")
            self._cf_keep = arr
            cf = ifnso_coeffs(K, arr.ctypes.data_as(C.POINTER(C.c_double)), None, None)
        return cf

    def orthogonalize(self, batch, coeffs, outs, ws=None, stream=None):
        """Run Algorithm 1 on every matrix of `batch` (Batch) into `outs` (tensors).
        coeffs: host sequence of K = L + 1 FP64 values (slot 0 ignored) or a
        CUDA float32 tensor of shape (count, K)."""
        cf = self._coeffs(batch, coeffs)
        need = self.workspace_bytes(batch)
        if ws is None:
            ws = self.workspace(need)
        optr = (C.c_void_p * max(len(outs), 1))(*[o.data_ptr() for o in outs])
        check(ifnso_orthogonalize(self.handle, batch.ref(), C.byref(cf), optr, C.c_void_p(ws.ptr),
                                  ws.nbytes, _stream(stream)), "ifnso_orthogonalize")
        self._last_ws = ws
        return outs

    def muon_step(self, grads, momentum, staging, weights, coeffs, beta=0.95, nesterov=True, lr=0.02, ws=None,
                  stream=None):
        """One Muon step (ifnso_muon_step): momentum (FP32), staging (BF16,
        the orthogonalized input U) and weights (BF16) are lists of tensors
        matching `grads` (Batch of BF16 gradients); W <- W - lr s orth(U)."""
        cf = self._coeffs(grads, coeffs)
        need = self.workspace_bytes(grads)
        if ws is None:
            ws = self.workspace(need)

        def ptrs(ts):
            return (C.c_void_p * max(len(ts), 1))(*[t.data_ptr() for t in ts])

        check(ifnso_muon_step(self.handle, grads.ref(), ptrs(momentum), ptrs(staging), ptrs(weights), C.byref(cf),
                              float(beta), 1 if nesterov else 0, float(lr), C.c_void_p(ws.ptr), ws.nbytes,
                              _stream(stream)), "ifnso_muon_step")
        self._last_ws = ws
        return weights

    def autotune(self, batch, coeffs, outs, reps=3, ws=None, stream=None):
        """Time per-CTA and CTA-pair MMAs on this batch and keep the faster per
        pass kind, then the depth of the operand ring per kind
        (IFNSO_OPT_STAGE_LIMITS); returns the modes (Gram, split squaring,
        plain squaring, product)."""
        cf = self._coeffs(batch, coeffs)
        need = self.workspace_bytes(batch)
        if ws is None:
            ws = self.workspace(need)
        optr = (C.c_void_p * max(len(outs), 1))(*[o.data_ptr() for o in outs])
        chosen = (C.c_int32 * 4)()
        check(ifnso_plan_autotune(self.handle, batch.ref(), C.byref(cf), optr, C.c_void_p(ws.ptr), ws.nbytes,
                                  int(reps), chosen, _stream(stream)), "ifnso_plan_autotune")
        self._last_ws = ws
        return list(chosen)

    def orthogonalize_host(self, host_in, batch, coeffs, outs, host_out, groups=0, ws=None, stream=None):
        """Algorithm 1 on matrices in host memory: host_in[i] (page-locked CPU
        tensors laid out like batch's device tensors) are uploaded into the
        tensors of `batch`, the results come back from `outs` (device) into
        host_out (CPU tensors); uploads, passes and downloads of `groups`
        groups overlap.  Asynchronous on `stream`."""
        cf = self._coeffs(batch, coeffs)
        need = self.workspace_bytes(batch)
        if ws is None:
            ws = self.workspace(need)
        n = max(len(outs), 1)
        hin = (C.c_void_p * n)(*[t.data_ptr() for t in host_in])
        hout = (C.c_void_p * n)(*[t.data_ptr() for t in host_out])
        optr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        check(ifnso_orthogonalize_host(self.handle, hin, batch.ref(), C.byref(cf), optr, hout, C.c_void_p(ws.ptr),
                                       ws.nbytes, int(groups), _stream(stream)), "ifnso_orthogonalize_host")
        self._last_ws = ws
        return host_out

    def ns_iterate(self, batch, poly, steps, outs, ws=None, stream=None):
        poly = np.ascontiguousarray(np.asarray(poly, dtype=np.float64))
        degree = 5 if len(poly) == 3 else 3
        need = self.ns_workspace_bytes(batch)
        if ws is None:
            ws = self.workspace(need)
        optr = (C.c_void_p * max(len(outs), 1))(*[o.data_ptr() for o in outs])
        check(ns_iterate(self.handle, batch.ref(), poly.ctypes.data_as(C.POINTER(C.c_double)), degree, int(steps),
                         optr, C.c_void_p(ws.ptr), ws.nbytes, _stream(stream)), "ns_iterate")
        self._last_ws = ws
        return outs

    def device_status(self, count, ws=None, stream=None):
        """(status words, s2 = o or ||A||_F^2, tr T_0) of the last call (synchronises)."""
        ws = ws or self._last_ws
        st = (C.c_int32 * max(count, 1))()
        o = (C.c_double * max(count, 1))()
        tr = (C.c_double * max(count, 1))()
        rc = ifnso_device_status(self.handle, C.c_void_p(ws.ptr), count, st, o, tr, _stream(stream))
        if rc not in (IFNSO_OK, IFNSO_ERR_DEVICE_TIMEOUT):
            check(rc, "ifnso_device_status")
        return np.array(st[:count]), np.array(o[:count]), np.array(tr[:count])

    def pass_times(self, max_passes=64):
        """(per-pass milliseconds summed over the calls since the last query, number of calls)."""
        ms = (C.c_double * max_passes)()
        n = C.c_int32()
        calls = C.c_int32()
        check(ifnso_pass_times(self.handle, ms, max_passes, C.byref(n), C.byref(calls)), "ifnso_pass_times")
        return np.array(ms[:n.value]), calls.value

    def host_timeline(self, max_groups=64):
        """Per group of the last eager orthogonalize_host call (IFNSO_OPT_TIMING on):
        (array of [uploads done, passes done, downloads done] in ms since the
        call's start, first matrix of each group followed by the count)."""
        ms = (C.c_double * (3 * max_groups))()
        first = (C.c_int32 * (max_groups + 1))()
        n = C.c_int32()
        check(ifnso_host_timeline(self.handle, ms, max_groups, C.byref(n), first), "ifnso_host_timeline")
        g = min(n.value, max_groups)
        return np.array(ms[:3 * g]).reshape(g, 3), list(first[:g + 1])

    def workspace_view(self, batch, index, which, ws=None):
        """(device pointer, ld) of an intermediate h_pad x h_pad buffer."""
        ws = ws or self._last_ws
        p = C.c_void_p()
        ld = C.c_int64()
        check(ifnso_workspace_view(self.handle, batch.ref(), C.c_void_p(ws.ptr), index, which, C.byref(p),
                                   C.byref(ld)), "ifnso_workspace_view")
        return p.value, ld.value


class Mlp:
    """ifnso_mlp: the coefficient-proposal network (K = L + 1 slots)."""

    def __init__(self, K, wfix, params=None, seed=0):
        self.K = int(K)
        self.P = int(ifnso_mlp_param_count(self.K))
        wf = np.ascontiguousarray(np.asarray(wfix, dtype=np.float64))
        assert wf.shape == (self.K - 1,)
        h = C.c_void_p()
        pp = None
        if params is not None:
            self._p0 = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
            pp = C.c_void_p(self._p0.ctypes.data)
        check(ifnso_mlp_create(C.byref(h), self.K, wf.ctypes.data_as(C.POINTER(C.c_double)), pp, int(seed)),
              "ifnso_mlp_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            ifnso_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        p = np.zeros(self.P, dtype=np.float32)
        st = np.zeros(12, dtype=np.float32)
        check(ifnso_mlp_get_params(self.handle, C.c_void_p(p.ctypes.data), C.c_void_p(st.ctypes.data)),
              "ifnso_mlp_get_params")
        return p, st

    def set_params(self, params=None, stats=None):
        pp = None if params is None else np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        ss = None if stats is None else np.ascontiguousarray(np.asarray(stats, dtype=np.float32))
        check(ifnso_mlp_set_params(self.handle, None if pp is None else C.c_void_p(pp.ctypes.data),
                                   None if ss is None else C.c_void_p(ss.ctypes.data)), "ifnso_mlp_set_params")

    def set_data(self, sigma, offsets, h, w, fit=True, stream=None):
        """sigma: CUDA float32 (concatenated), offsets: CUDA int64 (n + 1), h, w: CUDA int32 (n)."""
        self._data = (sigma, offsets, h, w)
        check(ifnso_mlp_set_data(self.handle, int(h.numel()), C.c_void_p(sigma.data_ptr()),
                                 C.c_void_p(offsets.data_ptr()), C.c_void_p(h.data_ptr()), C.c_void_p(w.data_ptr()),
                                 1 if fit else 0, _stream(stream)), "ifnso_mlp_set_data")

    def loss_grad(self, idx, stream=None):
        torch = _torch()
        g = torch.empty(self.P, dtype=torch.float32, device=idx.device)
        loss = torch.empty(1, dtype=torch.float32, device=idx.device)
        check(ifnso_mlp_loss_grad(self.handle, C.c_void_p(idx.data_ptr()), int(idx.numel()), C.c_void_p(g.data_ptr()),
                                  C.c_void_p(loss.data_ptr()), _stream(stream)), "ifnso_mlp_loss_grad")
        return g, loss

    def train(self, steps, batch=256, lr=1e-3, seed=0, stream=None):
        torch = _torch()
        curve = torch.empty(max(int(steps), 1), dtype=torch.float32, device="cuda")
        check(ifnso_mlp_train(self.handle, int(steps), int(batch), float(lr), int(seed), C.c_void_p(curve.data_ptr()),
                              _stream(stream)), "ifnso_mlp_train")
        return curve[:steps]

    def evaluate(self, n, idx=None, stream=None):
        torch = _torch()
        e1 = torch.empty(n, dtype=torch.float32, device="cuda")
        e0 = torch.empty(n, dtype=torch.float32, device="cuda")
        cf = torch.empty((n, self.K), dtype=torch.float32, device="cuda")
        fb = torch.empty(n, dtype=torch.int32, device="cuda")
        check(ifnso_mlp_evaluate(self.handle, None if idx is None else C.c_void_p(idx.data_ptr()), int(n),
                                 C.c_void_p(e1.data_ptr()), C.c_void_p(e0.data_ptr()), C.c_void_p(cf.data_ptr()),
                                 C.c_void_p(fb.data_ptr()), _stream(stream)), "ifnso_mlp_evaluate")
        return e1, e0, cf, fb


def tensor_at(ptr, shape, dtype, owner):
    """Copy of the device buffer at `ptr` (inside the tensor `owner`) as a new tensor."""
    torch = _torch()
    esz = torch.empty((), dtype=dtype).element_size()
    off = ptr - owner.data_ptr()
    n = int(np.prod(shape))
    return owner[off:off + n * esz].view(dtype).view(*shape).clone()


def frobenius_norm2(mats, stream=None):
    torch = _torch()
    b = Batch(mats)
    out = torch.zeros(len(mats), dtype=torch.float64, device=mats[0].device)
    check(ifnso_frobenius_norm2(b.ref(), _dtype_code(mats[0]), C.c_void_p(out.data_ptr()), _stream(stream)),
          "ifnso_frobenius_norm2")
    return out


def learn_coefficients(L, iters=20000, samples=1000, lr=0.1, step_size=10000, gamma=0.5, seed=0):
    w = (C.c_double * L)()
    check(ifnso_learn_coefficients(int(L), int(iters), int(samples), float(lr), int(step_size), float(gamma),
                                   int(seed), w), "ifnso_learn_coefficients")
    return np.array(w[:L])


def synth_lowrank_bf16(out, seed, alpha, beta, stream=None):
    check(ifnso_synth_lowrank_bf16(C.c_void_p(out.data_ptr()), out.shape[0], out.shape[1], out.stride(0), int(seed),
                                   float(alpha), float(beta), _stream(stream)), "ifnso_synth_lowrank_bf16")
    return out


def launch_count():
    return int(ifnso_launch_count())
