"""The bench's end-to-end host buffers: page-locked tensors carved from one
huge-page-backed mapping that is registered with CUDA once.  The CUDA runtime
calls are replaced by a recorder, so the carving is checked on the CPU."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


class _Cudart:
    def __init__(self, register_rc=0):
        self.calls = []
        self.register_rc = register_rc

    def cudaHostRegister(self, ptr, nbytes, flags):
        self.calls.append(("register", ptr, nbytes, flags))
        return self.register_rc

    def cudaHostUnregister(self, ptr):
        self.calls.append(("unregister", ptr))
        return 0


def test_pinned_block_carves_disjoint_aligned_views(monkeypatch):
    import torch

    bench = _bench()
    rt = _Cudart()
    monkeypatch.setattr(torch.cuda, "cudart", lambda: rt)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    # (rows, row pitch, cols, dtype): an input with padded rows, outputs, an FP32 one
    specs = [(5, 8, 6, torch.bfloat16), (3, 4, 4, torch.bfloat16), (7, 9, 9, torch.bfloat16),
             (2, 4, 3, torch.float32)]
    ts, release = bench.pinned_block(torch, specs)
    assert len(ts) == len(specs)
    regs = [c for c in rt.calls if c[0] == "register"]
    assert len(regs) == 1  # one registration for the whole block
    base, total = regs[0][1], regs[0][2]
    hp = 1 << 21
    for t, (r, ld, c, dt) in zip(ts, specs):
        assert t.shape == (r, c) and t.dtype == dt and t.stride() == (ld, 1)
        off = t.data_ptr() - base
        assert off % hp == 0  # every tensor starts on its own 2 MB boundary
        assert off + r * ld * t.element_size() <= total
    # the views do not overlap: each keeps the values written to it
    for i, t in enumerate(ts):
        t.fill_(i + 1)
    for i, t in enumerate(ts):
        assert np.all(t.float().numpy() == i + 1)
    release()
    assert rt.calls[-1] == ("unregister", base)


def test_pinned_block_falls_back_when_registration_fails(monkeypatch):
    import torch

    bench = _bench()
    rt = _Cudart(register_rc=1)
    monkeypatch.setattr(torch.cuda, "cudart", lambda: rt)
    made = []
    real_empty = torch.empty

    def empty(*a, **k):
        # PyTorch's page-locked tensors need a CUDA device: record the request instead
        made.append(k.get("pin_memory", False))
        k.pop("pin_memory", None)
        return real_empty(*a, **k)

    monkeypatch.setattr(torch, "empty", empty)
    ts, release = bench.pinned_block(torch, [(4, 8, 5, torch.bfloat16), (2, 2, 2, torch.bfloat16)])
    assert made.count(True) == 2  # one page-locked tensor per spec
    assert [tuple(t.shape) for t in ts] == [(4, 5), (2, 2)] and ts[0].stride() == (8, 1)
    release()  # nothing to unregister
    assert [c[0] for c in rt.calls] == ["register"]
