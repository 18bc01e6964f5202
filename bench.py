#!/usr/bin/env python
"""Throughput of IFNSO on GB300: orthogonalized matrices/s (and TFLOP/s) of one
batched Muon step, next to a 5-step quintic Newton-Schulz on the same GPU.

Default workload (one step = one pass of the whole hot path over the list):
the weight-gradient list of a synthetic 1B-parameter transformer,
24 layers x {Q, K, V, O 2048x2048; gate, up 2048x5632; down 5632x2048},
168 BF16 matrices of rank-32 signal plus noise (10:1), seeds 0..167, at
L = 14 (the depth whose distance to U V^T matches the 5-step quintic NS on
these matrices).  Inputs (2.47 GB) are larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded
sample of the same workload per step).  Under torchrun every rank runs its
own copy of the list (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orthogonalized matrices/s & TFLOP/s vs 5-step NS at equal polar error, 1 GB300"
MUON_ABC = (3.4445, -4.7750, 2.0315)

WORKLOADS = {
    "muon_1b": {
        "desc": "synthetic 1B transformer weight-gradient list: 24 layers x {Q,K,V,O 2048x2048; gate, up "
                "2048x5632; down 5632x2048}, 168 BF16 rank-32 + noise (10:1) matrices, seeds 0..167",
        "kind": "lowrank", "list": "list_1b", "L": 14, "L_gelfand2": 13,
    },
    "muon_1b_4l": {
        "desc": "first 4 layers of the synthetic 1B list (28 BF16 matrices, 412 MB of input > L2): the "
                "small case used for ncu captures",
        "kind": "lowrank", "list": "list_1b_4l", "L": 14, "L_gelfand2": 13,
    },
    "muon_7b": {
        "desc": "synthetic 7B transformer weight-gradient list: 32 layers x {4 x 4096x4096; gate, up "
                "4096x14336; down 14336x4096}, 224 BF16 rank-32 + noise (10:1) matrices, seeds 0..223",
        "kind": "lowrank", "list": "list_7b", "L": 14, "L_gelfand2": 13,
    },
    "config1_f32": {
        "desc": "one 256x512 FP32 matrix of i.i.d. N(0,1) entries (seed 0), L = 4 (exponents {1, 2, 4, 8}), "
                "the FP32 path",
        "kind": "gaussian", "shapes": [(256, 512, 0)], "dtype": "f32", "L": 4, "L_gelfand2": 4,
    },
    "config2": {
        "desc": "the precision-path pair in one call: BF16 4096x4096 (seed 0) and 4096x11008 (seed 1), "
                "U diag(sigma) V^T with Haar U, V and sigma = 1e3 * 10^U(-4, 0)",
        "kind": "spectral", "shapes": [(4096, 4096, 0), (4096, 11008, 1)], "L": 14, "L_gelfand2": 13,
    },
    "heldout_2k": {
        "desc": "the 2000 shapes of the coefficient network's held-out set (seeds 1000000..1001999: h ~ "
                "U{64..1024}, w = round(h U[1, 4])), BF16 rank-32 + noise (10:1) entries from the GPU "
                "generator (the entries do not change the work), L = 4 (K = 5 slots)",
        "kind": "heldout", "n": 2000, "L": 4, "L_gelfand2": 4,
    },
    "table1": {
        "desc": "the Table 1 shapes 128x128, 128x512, 128x1024 (Sec. 3.4), 10 N(0,1) BF16 matrices of "
                "each (seeds 0..9), 30 in one call, L = 14",
        "kind": "gaussian", "shapes": [(128, c, s) for c in (128, 512, 1024) for s in range(10)], "L": 14,
        "L_gelfand2": 13,
    },
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="muon_1b", choices=sorted(WORKLOADS))
    ap.add_argument("--L", type=int, default=None)
    ap.add_argument("--precision", default="auto", choices=["auto", "plain", "split"])
    ap.add_argument("--split-squarings", type=int, default=-1,
                    help="leading squarings with split FP16 operands in the mixed precision (-1: L - 8)")
    ap.add_argument("--scale", default="gram", choices=["gram", "frob", "gelfand2"],
                    help="input scaling: Gram (q = 1, the paper's), Frobenius, or Gelfand's bound with q = 2")
    ap.add_argument("--cta-group", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core passes: MMAs of the CTA pair (2), per-CTA MMAs, each CTA loading its whole B tile (1), "
                         "or the library's choice per pass (0)")
    ap.add_argument("--coeffs", default="fixed", choices=["fixed", "mlp"],
                    help="fixed: the learner's w_1..w_L for every matrix; mlp: per-matrix coefficients "
                         "proposed inside the call by the coefficient network (trained here first)")
    ap.add_argument("--mlp-steps", type=int, default=2000)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip ifnso_plan_autotune (MMA mode per pass kind) before timing")
    ap.add_argument("--gram-e4m3", action="store_true",
                    help="experiment: the first product T_0 = A A^T from an E4M3 copy of A")
    ap.add_argument("--groups", type=int, default=0,
                    help="end-to-end run: groups whose copies overlap the passes (0: the library default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the polar-distance and orthogonality report of the outputs")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="time eager calls instead of a captured CUDA graph of one step")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: one list shared out over the ranks (LPT on FLOPs), results exchanged")
    ap.add_argument("--muon", action="store_true",
                    help="time a whole Muon step (momentum, orthogonalization, fused weight update) on the list")
    ap.add_argument("--ablation", action="store_true",
                    help="the L ablation on the Table 1 shapes (one JSON line of per-L rows) instead of the bench")
    ap.add_argument("--ablation-L", default="2-16", help="range of L for --ablation, e.g. 2-16")
    ap.add_argument("--ablation-seeds", type=int, default=10)
    return ap.parse_args()


def flops_ifnso(h, w, L):
    """Matrix-product FLOPs of Algorithm 1: Gram 2h^2 w, (L - 1) squarings 2h^3, apply 2h^2 w."""
    return 4 * h * h * w + 2 * (L - 1) * h ** 3


def flops_ns5(h, w, steps=5):
    return steps * (4 * h * h * w + 2 * h ** 3)


def workload_list(wl):
    """[(name, rows, cols)] of the workload's matrices, in call order."""
    import synth

    kind = wl.get("kind", "lowrank")
    if kind == "lowrank":
        if wl["list"] == "list_1b_4l":
            return synth.transformer_list(4, 2048, 5632)
        return getattr(synth, wl["list"])()
    if kind == "heldout":
        out = []
        for i in range(wl["n"]):
            h, w, _, _ = synth.mlp_spectrum(1000000 + i)
            out.append((f"heldout{i}", h, w))
        return out
    return [(f"m{i}", r, c) for i, (r, c, _) in enumerate(wl["shapes"])]


def workload_dtype(wl):
    return wl.get("dtype", "bf16")


def oriented(r, c):
    return (min(r, c), max(r, c))


def rank_seed0(rank):
    """First seed of rank `rank`'s list: every rank orthogonalises its own list
    of independent matrices (weak scaling, no data-path collective)."""
    return rank * 100000


def max_over_ranks_of(dist, value, device):
    """The largest of the ranks' values (the whole job ends with the slowest rank)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, ms_max):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank * steps / (ms_max / 1000.0)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def load_traffic():
    """Per-launch DRAM traffic from the committed ncu summary, or {} when the
    kernel source changed since the capture (the counters no longer apply)."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        src = os.path.join(ROOT, "paper_2602_02500_gb300", "csrc", "tc_gemm.cu")
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != t.get("tc_gemm_sha256_16"):
                return {}
        return t
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def host_matrix(wl, i):
    """Matrix i of a gaussian or spectral workload, FP64, from synth/ (as the
    parity tests build it)."""
    import synth

    r, c, seed = wl["shapes"][i]
    if wl["kind"] == "gaussian":
        return synth.gaussian(seed, r, c)
    h = min(r, c)
    M = synth.spectral(seed, r, c, synth.loguniform_sigma(seed, h))
    return synth.round_bf16(M) if workload_dtype(wl) == "bf16" else M


def pinned_block(torch, specs):
    """Page-locked host tensors carved from one anonymous mapping that asks
    for transparent huge pages (madvise) and is registered with CUDA once.
    specs: (rows, row_pitch, cols, dtype) per tensor, each view (rows, cols)
    with that row pitch.  On a Grace host (64 KB base pages, 512 MB huge
    pages) the copy engines then work through a few large translations;
    page-locked tensors allocated one by one after another large process had
    freed its memory copied at about a tenth of their speed for stretches of
    100-200 ms.  Falls back to PyTorch's page-locked tensors when the mapping
    cannot be advised or registered.  Returns (tensors, release): release()
    unregisters the block once the tensors are no longer used."""
    import mmap

    import numpy as np

    hp = 1 << 21
    nbytes = [r * ld * torch.empty((), dtype=dt).element_size() for r, ld, _, dt in specs]
    offs, total = [], 0
    for n in nbytes:
        offs.append(total)
        total += (n + hp - 1) // hp * hp
    try:
        mm = mmap.mmap(-1, max(total, hp), flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        mm.madvise(mmap.MADV_HUGEPAGE)
        raw = torch.from_numpy(np.frombuffer(mm, dtype=np.uint8))
        raw.fill_(0)  # touch every page before it is registered
        cudart = torch.cuda.cudart()
        if int(cudart.cudaHostRegister(raw.data_ptr(), raw.numel(), 0)) != 0:
            raise RuntimeError("cudaHostRegister failed")
    except Exception:
        ts = [torch.empty((r, ld), dtype=dt, pin_memory=True)[:, :c] for r, ld, c, dt in specs]
        return ts, (lambda: None)
    ts = [raw[o:o + n].view(dt).view(r, ld)[:, :c] for (r, ld, c, dt), o, n in zip(specs, offs, nbytes)]

    def release():
        torch.cuda.synchronize()
        cudart.cudaHostUnregister(raw.data_ptr())

    return ts, release


def make_inputs(F, torch, shapes, seed0, device, wl=None):
    """Device inputs of the workload.  Low-rank lists (and the held-out
    shapes) come from the library's Philox generator on the GPU, seeds
    seed0 + i; gaussian and spectral matrices from synth/ on the host."""
    import synth

    wl = wl or WORKLOADS["muon_1b"]
    kind = wl.get("kind", "lowrank")
    xs = []
    if kind in ("lowrank", "heldout"):
        alpha, beta = synth.lowrank_constants()
        for i, (_, r, c) in enumerate(shapes):
            ld = (c + 7) // 8 * 8
            buf = torch.empty((r, ld), dtype=torch.bfloat16, device=device)
            x = buf[:, :c]
            F.synth_lowrank_bf16(x, seed0 + i, float(alpha), float(beta))
            xs.append(x)
        return xs
    dt = torch.float32 if workload_dtype(wl) == "f32" else torch.bfloat16
    for i in range(len(shapes)):
        xs.append(torch.tensor(host_matrix(wl, i), dtype=torch.float32).to(device=device, dtype=dt))
    return xs


def oracle_input(wl, shapes, i, seed0=0):
    """Matrix i of the workload as the FP64 oracle sees it (the same values
    the device computes on)."""
    import synth

    if wl.get("kind", "lowrank") in ("lowrank", "heldout"):
        _, r, c = shapes[i]
        return synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(seed0 + i, r, c))
    return host_matrix(wl, i)


def cpu_oracle_sample(wl, shapes, L, budget_s=20.0):
    """Time the FP64 oracle (Algorithm 1) on one matrix of each distinct
    shape, in list order, until about budget_s seconds are spent; project the
    time of the whole list (per shape when every distinct shape was timed,
    else by Algorithm 1's FLOPs).  Returns (matrices/s, sample text, cores)."""
    import numpy as np

    from oracle import coeffs as OC
    from oracle import ifnso as O

    w = OC.complete(np.zeros(L - 1), L)  # timing does not depend on the coefficient values
    first = {}
    for i, (_, r, c) in enumerate(shapes):
        first.setdefault((r, c), i)
    timed = {}
    t_used = 0.0
    for (r, c), i in first.items():
        M = oracle_input(wl, shapes, i)
        t0 = time.perf_counter()
        O.ifnso_alg1(M, w)
        dt = time.perf_counter() - t0
        timed[(r, c)] = dt
        t_used += dt
        if t_used > budget_s:
            break
    fl = {k: flops_ifnso(*oriented(*k), L) for k in first}
    if len(timed) == len(first):
        total = sum(timed[(r, c)] for _, r, c in shapes)
        how = f"list time projected per shape over {len(shapes)} matrices"
    else:
        rate = sum(fl[k] for k in timed) / sum(timed.values())
        total = sum(fl[(r, c)] for _, r, c in shapes) / rate
        how = (f"{len(timed)} of {len(first)} distinct shapes timed; list time projected by Algorithm 1's "
               f"FLOPs over {len(shapes)} matrices")
    shown = list(timed.items())[:6]
    sample = ("FP64 oracle (Algorithm 1, numpy) on one matrix of each distinct shape "
              + ", ".join(f"{r}x{c}: {t:.2f}s" for (r, c), t in shown)
              + (", ..." if len(timed) > len(shown) else "") + f"; {how}")
    return len(shapes) / total, sample, os.cpu_count()


def run_ablation(args):
    """L ablation on the Table 1 shapes (Sec. 3.4, Table 1): N(0,1) matrices
    128 x {128, 512, 1024}, seeds 0..S-1.  For each L, the library's GPU
    learner fits w_1..w_L (Sec. 3.1.1 schedule) and the library orthogonalizes
    the batch in an FP32 and a BF16 plan; the error is ||Y Y^T - I||_F (the
    Table 1 metric), evaluated on the host in FP64 from the returned Y.  The
    cubic NS with 8 steps (the Table 1 "Original NS") and Muon's quintic NS
    with 5 steps run on the same inputs.  FLOPs follow Table 1's counting."""
    import numpy as np
    import torch

    import synth
    from paper_2602_02500_gb300 import ifnso as F

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    lo, hi = (int(v) for v in args.ablation_L.split("-"))
    shapes = [(128, 128), (128, 512), (128, 1024)]
    S = args.ablation_seeds
    mats = [(h, w, synth.gaussian(seed, h, w)) for h, w in shapes for seed in range(S)]

    def inputs(dtype):
        out = []
        for h, w, M in mats:
            t = torch.tensor(M, dtype=torch.float32, device=dev)
            out.append(t.to(torch.bfloat16) if dtype == "bf16" else t)
        return out

    def orth_err(ys):
        per = {}
        for (h, w, _), y in zip(mats, ys):
            Y = y.double().cpu().numpy()
            per.setdefault((h, w), []).append(float(np.linalg.norm(Y @ Y.T - np.eye(h))))
        return {f"{h}x{w}": float(np.mean(v)) for (h, w), v in per.items()}

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    xin = {d: inputs(d) for d in ("f32", "bf16")}
    rows = []
    for L in range(lo, hi + 1):
        w = F.learn_coefficients(L)
        row = {"L": L, "flops": {f"{h}x{wd}": 4 * h * h * wd + 2 * (L - 1) * h ** 3 + L * h * h for h, wd in shapes}}
        for d in ("f32", "bf16"):
            xs = xin[d]
            ys = [torch.empty_like(x) for x in xs]
            plan = F.Plan(128, 1024, d, L=L)
            b = F.Batch(xs)
            ws = F.Workspace(plan.workspace_bytes(b), device=dev)
            ms = timed(lambda: plan.orthogonalize(b, np.r_[1.0, w], ys, ws=ws))
            row[f"err_{d}"] = orth_err(ys)
            row[f"ms_{d}"] = ms
        rows.append(row)
    ns = {}
    for name, poly, steps, fl in (("original_ns_8", (1.5, -0.5), 8, lambda h, w: 8 * (4 * h * h * w + 2 * h * w + h * h)),
                                  ("muon_ns_5", MUON_ABC, 5, lambda h, w: 5 * (6 * h * h * w + 5 * h * w))):
        ent = {"flops": {f"{h}x{wd}": fl(h, wd) for h, wd in shapes}}
        for d in ("f32", "bf16"):
            xs = xin[d]
            zs = [torch.empty_like(x) for x in xs]
            plan = F.Plan(128, 1024, d, L=1)
            b = F.Batch(xs)
            ws = F.Workspace(plan.ns_workspace_bytes(b), device=dev)
            ms = timed(lambda: plan.ns_iterate(b, poly, steps, zs, ws=ws))
            ent[f"err_{d}"] = orth_err(zs)
            ent[f"ms_{d}"] = ms
        ns[name] = ent
    print(json.dumps({"metric": "L ablation: ||Y Y^T - I||_F and FLOPs on the Table 1 shapes", "impl": "ours",
                      "data": f"synthetic: N(0,1), seeds 0..{S - 1} per shape",
                      "shapes": [f"{h}x{w}" for h, w in shapes], "rows": rows, "ns": ns,
                      "ms": "one call over all shapes and seeds (FP32 or BF16 plan), CUDA events, mean of 5"}),
          flush=True)
    return 0


def run_muon(args):
    """A whole Muon step on the list (ifnso_muon_step): the momentum update
    and Nesterov input (one elementwise kernel per matrix), Algorithm 1 on
    that input, and the weight update fused into the final product, captured
    in one CUDA graph; beside it the orthogonalization alone on the same
    list.  Prints one JSON line."""
    import numpy as np
    import torch

    from paper_2602_02500_gb300 import ifnso as F

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    wl = WORKLOADS[args.workload]
    shapes = workload_list(wl)
    L = args.L or wl["L"]
    n = len(shapes)
    hw = [oriented(r, c) for _, r, c in shapes]
    xs = make_inputs(F, torch, shapes, 0, device)
    mom = [torch.zeros(x.shape, dtype=torch.float32, device=device) for x in xs]
    stg = [torch.empty_like(x) for x in xs]
    wts = [torch.zeros_like(x) for x in xs]
    ys = [torch.empty_like(x) for x in xs]
    batch = F.Batch(xs)
    coef = np.r_[1.0, F.learn_coefficients(L)]
    plan = F.Plan(max(h for h, _ in hw), max(w for _, w in hw), "bf16", L=L, precision=args.precision)
    plan.set(F.IFNSO_OPT_CTA_GROUP, args.cta_group)
    ws = F.Workspace(plan.workspace_bytes(batch), device=device)
    if args.autotune and args.cta_group == 0:
        plan.autotune(batch, coef, ys, reps=2, ws=ws)

    def graph(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        return g

    def timed(g):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    g_muon = graph(lambda: plan.muon_step(batch, mom, stg, wts, coef, beta=0.95, nesterov=True, lr=0.02, ws=ws))
    g_orth = graph(lambda: plan.orthogonalize(batch, coef, ys, ws=ws))
    ms_muon, ms_orth = timed(g_muon), timed(g_orth)
    print(json.dumps({
        "metric": "Muon steps/s over the list (momentum, IFNSO, fused weight update)", "value": 1000.0 / ms_muon,
        "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_muon,
        "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "L": L, "matrices": n, "beta": 0.95,
                   "nesterov": True, "momentum": "FP32", "weights": "BF16"},
        "orthogonalize_only_ms": ms_orth, "overhead_ms": ms_muon - ms_orth,
    }), flush=True)
    return 0


def run_shard(args):
    """Strong scaling over N ranks: every rank holds the same list (seeds
    0..n-1), orthogonalizes the share that greedy LPT on Algorithm 1's
    nominal FLOPs gives it, and the results are then exchanged by one
    all-gather of the ranks' packed results, so that every rank ends with all
    of them (a replicated Muon update).  The timed step is the library call
    plus the exchange."""
    import numpy as np
    import torch

    from paper_2602_02500_gb300 import ifnso as F
    from paper_2602_02500_gb300 import shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    wl = WORKLOADS[args.workload]
    shapes = workload_list(wl)
    L = args.L or wl["L"]
    n = len(shapes)
    parts = shard.lpt_partition([shard.ifnso_cost(r, c, L) for _, r, c in shapes], world)
    mine = parts[rank]
    xs = make_inputs(F, torch, shapes, 0, device)
    ys = [torch.empty_like(x) for x in xs]
    hw = [oriented(r, c) for _, r, c in shapes]
    sub = F.Batch([xs[i] for i in mine])
    sub_out = [ys[i] for i in mine]
    w_full = F.learn_coefficients(L)
    coef = np.r_[1.0, w_full]
    plan = F.Plan(max(hw[i][0] for i in mine), max(hw[i][1] for i in mine), "bf16", L=L,
                  precision=args.precision)
    plan.set(F.IFNSO_OPT_CTA_GROUP, args.cta_group)
    ws = F.Workspace(plan.workspace_bytes(sub), device=device)
    if args.autotune and args.cta_group == 0:
        plan.autotune(sub, coef, sub_out, reps=2, ws=ws)

    def run_local(_idx):
        plan.orthogonalize(sub, coef, sub_out, ws=ws)

    def step():
        shard.sharded_orthogonalize(run_local, ys, parts, rank, dist)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = max_over_ranks_of(dist, e0.elapsed_time(e1), device)
    loads = [sum(shard.ifnso_cost(shapes[i][1], shapes[i][2], L) for i in p) for p in parts]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * args.steps / (ms / 1000.0), "unit": "matrices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": args.workload + ": " + wl["desc"], "L": L,
                       "parallelism": f"list sharded over {world} ranks (greedy LPT on FLOPs), results "
                                      "exchanged by one all-gather of the packed shares",
                       "matrices_per_rank": [len(p) for p in parts],
                       "flop_share_max_over_mean": max(loads) / (sum(loads) / len(loads))},
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    from oracle import coeffs as OC
    from oracle import ifnso as O

    wl = WORKLOADS[args.workload]
    shapes = workload_list(wl)
    L = args.L or wl["L"]
    w = OC.complete(np.zeros(L - 1), L)
    distinct = {}
    for i, (nm, r, c) in enumerate(shapes):
        distinct.setdefault((r, c), []).append(i)
    # one step = one matrix of each of (at most 8) distinct shapes: a bounded sample of the list
    keys = list(distinct)[:8]
    mats = {k: oracle_input(wl, shapes, distinct[k][0]) for k in keys}
    times = {k: [] for k in keys}
    for s in range(args.warmup + max(1, args.steps)):
        for k in keys:
            t0 = time.perf_counter()
            O.ifnso_alg1(mats[k], w)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times[k].append(dt)
    mean = {k: float(np.mean(times[k])) for k in keys}
    if len(keys) == len(distinct):
        list_time = sum(mean[k] * len(distinct[k]) for k in keys)
        how = "per shape"
    else:
        rate = sum(flops_ifnso(*oriented(*k), L) for k in keys) / sum(mean.values())
        list_time = sum(flops_ifnso(*oriented(r, c), L) for _, r, c in shapes) / rate
        how = "by Algorithm 1's FLOPs"
    value = len(shapes) / list_time
    step_ms = 1000.0 * list_time  # the whole list, projected from the sample
    sample = (f"each step: FP64 oracle (Algorithm 1, numpy) on one matrix of {len(keys)} distinct shapes "
              + ", ".join(f"{r}x{c}: {mean[(r, c)]:.2f}s" for (r, c) in keys)
              + f"; the time of the {len(shapes)}-matrix list is projected from it {how} (ms_per_step)")
    line = {
        "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "L": L, "parallelism": "host cores",
                   "timing": "projected: each step times the FP64 oracle on one matrix of every distinct "
                             "shape; ms_per_step and value are the whole list's, projected from that sample"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def polar_quality(torch, shapes, xs, outs, max_shapes=3, max_h=2048):
    """Distance to the polar factor U V^T (Frobenius, per sqrt(h)) and the
    orthogonality error ||Y Y^T - I||_F of the GPU outputs, in FP64 on the
    host, for the first matrix of each distinct shape (at most max_shapes
    shapes with h <= max_h); U V^T from numpy's SVD of the same input.
    Not timed."""
    import numpy as np

    t0 = time.perf_counter()
    seen = {}
    for i, (_, r, c) in enumerate(shapes):
        if (r, c) not in seen and min(r, c) <= max_h:
            seen[(r, c)] = i
    res = {}
    for (r, c), i in list(seen.items())[:max_shapes]:
        A = xs[i].double().cpu().numpy()
        tr = r > c
        Ao = A.T if tr else A
        U, _, Vt = np.linalg.svd(Ao, full_matrices=False)
        Q = U @ Vt
        h = Ao.shape[0]
        entry = {}
        for name, ys_ in outs.items():
            Y = ys_[i].double().cpu().numpy()
            Yo = Y.T if tr else Y
            entry[name] = {"dist_polar": float(np.linalg.norm(Yo - Q) / np.sqrt(h)),
                           "orth_err": float(np.linalg.norm(Yo @ Yo.T - np.eye(h)))}
        res[f"{r}x{c}"] = entry
    return {"what": "first matrix of each distinct shape: ||Y - U V^T||_F / sqrt(h) and ||Y Y^T - I||_F "
                    "(oriented, h <= w), FP64 on the host from numpy's SVD of the input; not timed",
            "shapes": res, "secs": round(time.perf_counter() - t0, 1)}


def averaged_pass_times(plan, step, k):
    """Per-pass milliseconds of `step` (a call, or a graph replay, of a plan
    with IFNSO_OPT_TIMING on) averaged over k runs, each read back after a
    synchronize: the pass events are recorded inside the step, so they hold
    one step's passes at a time.  Returns (array, runs averaged)."""
    import numpy as np
    import torch

    plan.pass_times()
    acc, n = None, 0
    for _ in range(k):
        step()
        torch.cuda.synchronize()
        pm, c = plan.pass_times()
        if c < 1:
            continue
        pm = np.asarray(pm, dtype=np.float64) / c
        acc = pm if acc is None else acc + pm
        n += 1
    return (acc / n if n else np.zeros(0)), n


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.shard:
        return run_shard(args)
    if args.muon:
        return run_muon(args)

    import numpy as np
    import torch

    import synth
    from paper_2602_02500_gb300 import ifnso as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return max_over_ranks_of(dist, v, device)

    wl = WORKLOADS[args.workload]
    shapes = workload_list(wl)
    # the equal-polar-error depth of the scaling (tests/golden/equal_polar.json)
    L = args.L or (wl.get("L_gelfand2", wl["L"]) if args.scale == "gelfand2" else wl["L"])
    n = len(shapes)
    hw = [oriented(r, c) for _, r, c in shapes]
    hmax = max(h for h, _ in hw)
    wmax = max(w for _, w in hw)
    seed0 = rank_seed0(rank)
    dtype = workload_dtype(wl)
    xs = make_inputs(F, torch, shapes, seed0, device, wl)
    ys = [torch.empty(x.shape, dtype=x.dtype, device=device) for x in xs]  # outputs are dense (ld = cols)
    batch = F.Batch(xs)

    # fixed coefficients from the library's own GPU learner (Sec. 2.3 / 3.1.1)
    w_full = F.learn_coefficients(L)
    coef = np.r_[1.0, w_full]
    mlp_info = None
    if args.coeffs == "mlp":
        # per-matrix proposals (the coefficient network, K = L + 1 outputs), trained on
        # synthetic spectra; the timed step includes the features, the network
        # and the coefficient rows inside ifnso_orthogonalize
        import synth

        n_train = 20000
        hs_, ws_, sig_, offs_ = [], [], [], [0]
        for sd in range(n_train):
            h_, w_, sg_, _ = synth.mlp_spectrum(sd)
            hs_.append(h_)
            ws_.append(w_)
            sig_.append(sg_.astype(np.float32))
            offs_.append(offs_[-1] + h_)
        net = F.Mlp(L + 1, w_full, seed=0)
        net.set_data(torch.tensor(np.concatenate(sig_), device=device),
                     torch.tensor(offs_, dtype=torch.int64, device=device),
                     torch.tensor(hs_, dtype=torch.int32, device=device),
                     torch.tensor(ws_, dtype=torch.int32, device=device), fit=True)
        curve = net.train(args.mlp_steps, batch=512, lr=1e-3, seed=1).cpu().numpy()
        coef = net
        mlp_info = {"train_spectra": n_train, "steps": args.mlp_steps, "batch": 512,
                    "loss_first_50": float(np.mean(curve[:50])), "loss_last_50": float(np.mean(curve[-50:]))}

    plan = F.Plan(hmax, wmax, dtype, L=L, precision=args.precision, scale=args.scale)
    plan.set(F.IFNSO_OPT_SPLIT_SQUARINGS, args.split_squarings)
    plan.set(F.IFNSO_OPT_TIMING, 1)
    plan.set(F.IFNSO_OPT_CTA_GROUP, args.cta_group)
    plan.set(F.IFNSO_OPT_GRAM_E4M3, 1 if args.gram_e4m3 else 0)
    ws = F.Workspace(plan.workspace_bytes(batch), device=device)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.autotune and args.cta_group == 0 and dtype == "bf16":
        # untimed set-up: per-CTA vs CTA-pair MMAs per pass kind on this list
        modes = plan.autotune(batch, coef, ys, reps=2, ws=ws)
        tuned = dict(zip(["gram", "split_squaring", "plain_squaring", "product"], modes))
    for _ in range(max(args.warmup, 3)):
        plan.orthogonalize(batch, coef, ys, ws=ws)
    torch.cuda.synchronize()
    plan.pass_times()  # discard warm-up events
    st, _, _ = plan.device_status(n, ws=ws)
    if np.any(st & F.IFNSO_DEV_TIMEOUT):
        raise RuntimeError("device wait timed out during warm-up")

    def make_step(fn):
        """The step as a CUDA graph replay (captured once, after warm-up) or as
        eager calls; returns (callable, launches per step or None)."""
        if not args.graph:
            return fn, None
        n_before = F.launch_count()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        return g.replay, F.launch_count() - n_before

    ifnso_step, ifnso_launches = make_step(lambda: plan.orthogonalize(batch, coef, ys, ws=ws))
    ifnso_step()
    torch.cuda.synchronize()
    plan.pass_times()

    # Inputs smaller than twice L2 (129 MB) would stay cached from one step to
    # the next: such workloads write a 512 MB buffer before every step and time
    # the steps alone (a pair of events around each).
    in_bytes = sum(x.numel() * x.element_size() for x in xs)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device) if in_bytes < (258 << 20) else None

    per_step_ms = {}

    def timed_steps(step, k, name=None):
        """Milliseconds of k steps (max over ranks), the L2 flushed before each if needed.
        Events between the steps (recorded without a synchronize) give each step's time."""
        barrier()
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()  # no collector pause inside the timed region
        try:
            return _timed_steps(step, k, name)
        finally:
            gc.enable()

    def _timed_steps(step, k, name):
        if flush is None:
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
            evs[0].record(stream)
            for i in range(k):
                step()
                evs[i + 1].record(stream)
            torch.cuda.synchronize()
            barrier()
            if name:
                per_step_ms[name] = [round(evs[i].elapsed_time(evs[i + 1]), 3) for i in range(k)]
            return max_over_ranks(evs[0].elapsed_time(evs[k]))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in evs:
            flush.fill_(1)
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs))

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    n0 = F.launch_count()
    ms_total = timed_steps(ifnso_step, args.steps, "ifnso")
    # where the timed step's FP16 copy of the inputs was written (set when the step was enqueued)
    hosts = plan.get(F.IFNSO_OPT_FP16_COPY_HOSTS) if dtype == "bf16" else 0
    fp16_copy = (f"written by the side warps of {hosts} squarings" if hosts else
                 "written by its own kernel" if plan.get(F.IFNSO_OPT_APPLY_F16) else "not used")
    launches = ifnso_launches * args.steps if ifnso_launches is not None else F.launch_count() - n0
    clk = clocks.stop()
    ms_step = ms_total / args.steps
    # Per-pass durations.  The library's pass events are recorded inside the
    # step (graph record nodes, or eager records), so they hold one step's
    # passes at a time: after the timed region, K more steps run, each read
    # back after a synchronize, and every pass is averaged over those K steps.
    pass_ms, n_pass_steps = averaged_pass_times(plan, ifnso_step, args.steps)
    calls = 1
    value = whole_job_rate(world, n, args.steps, ms_total)
    fl = sum(flops_ifnso(h, w, L) for h, w in hw)
    tflops = world * fl * args.steps / (ms_total / 1000.0) / 1e12

    # The dominant kernel: the squaring instantiation with the most time per
    # step.  Squarings j = 1..L-1 take split operands for j <= k (the rest
    # plain FP16).  With fixed coefficients every squaring folds -2 D_l into
    # its MMAs and adds its own P term; with proposed coefficients the odd
    # ones from 3 on fold and the others read D_l for two P terms.
    peaks, peak_src = load_peaks()
    mode = plan.get(F.IFNSO_OPT_PRECISION)
    k_split = plan.get(F.IFNSO_OPT_SPLIT_SQUARINGS)
    per_step = [float(x) / max(1, calls) for x in pass_ms]
    sq = per_step[2:2 + (L - 1)] if L > 1 else []

    def folded(j):
        return True if args.coeffs == "fixed" else (j % 2 == 1 and j >= 3)

    variants = {}
    for j, t in enumerate(sq, start=1):
        key = ("split" if j <= k_split else "plain") + ("_fold" if folded(j) else "_p")
        variants.setdefault(key, []).append(t)
    sq_alg = sum(2 * h ** 3 for h, _ in hw)  # algorithmic FLOPs per squaring launch
    hp = [((h + 255) // 256) * 256 for h, _ in hw]
    exec_one = sum(((p // 256) * (p // 256 + 1) // 2) * 2 * (2 * 128 * 256 * p) for p in hp)
    dominant = max(variants, key=lambda k: sum(variants[k])) if variants else None
    roof = None
    if dominant:
        dom = variants[dominant]
        sq_launch_ms = float(np.mean(dom))
        split = dominant.startswith("split")
        sq_exec = exec_one * (3 if split else 1)
        if dominant.endswith("_fold"):
            # the identity products: one N = 16 MMA per K step and A source in
            # the four K blocks of each 128 x 256 tile's own columns
            sq_exec += sum(((p // 256) * (p // 256 + 1) // 2) * 2 * (2 * 128 * 16 * 256) for p in hp) * (2 if split else 1)
        traffic = load_traffic().get(f"{args.workload}:squaring_{dominant}")
        ach = sq_alg / (sq_launch_ms / 1000.0) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        what = ("D_{l+1} = 2 D_l - D_l^2, -2 D_l folded into the MMAs, its P term added in L2"
                if dominant.endswith("_fold") else "D_{l+1} = 2 D_l - D_l^2 with two P terms, D_l read")
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic,
                "kernel": f"tc_gemm_kernel squaring pass, {dominant.split('_')[0]} operands ({what})",
                "launch_ms": sq_launch_ms, "launches_per_step": len(dom),
                "algorithmic_flop_per_launch": sq_alg, "executed_flop_per_launch": sq_exec,
                "executed_tflops": sq_exec / (sq_launch_ms / 1000.0) / 1e12,
                "peak_source": f"bf16_tflops_sustained ({peak_src})",
                "squarings": {k: {"launches": len(v), "ms": float(np.mean(v))} for k, v in sorted(variants.items())},
                "pass_ms_per_step": per_step,
                "pass_timing": f"CUDA events on the launching stream around every pass, averaged over "
                               f"{n_pass_steps} steps run after the timed region (each read after a synchronize)",
                "pass_sum_ms": float(sum(per_step)),
                "pass_sum_over_step": float(sum(per_step)) / ms_step}

    kind = wl.get("kind", "lowrank")
    if dtype == "f32":
        # the FP32 path runs on the SIMT FP32 units (FFMA): 152 SMs x 128 lanes x 2 FLOP per clock
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = fl / (ms_step / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak,
                "traffic": None, "kernel": "whole step (every FP32 SIMT pass of Algorithm 1)",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 FLOP x {sm_mhz:.0f} MHz (max SM clock)",
                "pass_ms_per_step": per_step, "pass_sum_ms": float(sum(per_step)),
                "pass_sum_over_step": float(sum(per_step)) / ms_step}
    elif kind in ("heldout", "gaussian"):
        # many small matrices: the whole step against HBM or the tensor pipe, by
        # its intensity (Algorithm 1's FLOPs over the bytes of A read twice and Y written)
        alg_bytes = sum(3 * h * w * 2 for h, w in hw)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        tpk = float(peaks.get("bf16_tflops_sustained", 1700.0))
        intensity = fl / alg_bytes
        ridge = tpk * 1e12 / (hbm * 1e9)
        bw = alg_bytes / (ms_step / 1000.0) / 1e9
        tf = fl / (ms_step / 1000.0) / 1e12
        on_hbm = intensity < ridge
        roof = {"bound": "hbm" if on_hbm else "tensor", "achieved": bw if on_hbm else tf,
                "peak": hbm if on_hbm else tpk, "unit": "GB/s" if on_hbm else "TFLOP/s",
                "frac": bw / hbm if on_hbm else tf / tpk, "traffic": None,
                "kernel": "whole step (every pass of Algorithm 1 on the batch)",
                "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
                "hbm_frac": bw / hbm, "tensor_frac": tf / tpk, "algorithmic_bytes_per_step": alg_bytes,
                "peak_source": f"hbm_gbs and bf16_tflops_sustained ({peak_src})",
                "pass_ms_per_step": per_step, "pass_sum_ms": float(sum(per_step)),
                "pass_sum_over_step": float(sum(per_step)) / ms_step}

    # end to end through the C ABI with host buffers: ifnso_orthogonalize_host
    # uploads the inputs, runs the passes and downloads the results, group by
    # group on overlapping streams
    e2e = None
    if not args.no_e2e:
        # host copies of the inputs (same row pitch) and host outputs, page-locked
        # in one huge-page-backed block
        host, release_host = pinned_block(
            torch, [(x.shape[0], x.stride(0), x.shape[1], x.dtype) for x in xs]
            + [(x.shape[0], x.shape[1], x.shape[1], x.dtype) for x in xs])
        hin, hout = host[:len(xs)], host[len(xs):]
        for h_, x in zip(hin, xs):
            h_.copy_(x)
        bi = sum(x.numel() * x.element_size() for x in xs)

        def e2e_step():
            plan.orthogonalize_host(hin, batch, coef, ys, hout, groups=args.groups, ws=ws)

        for _ in range(max(args.warmup, 3)):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = timed_steps(e2e_step, args.steps, "e2e")
        # host time spent enqueueing one call (the GPU waits if this exceeds the call's device time)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        host_ms = 1000.0 * (time.perf_counter() - t0)
        torch.cuda.synchronize()
        # where the time goes: the last step's per-group timeline, and the
        # copies alone (each direction by itself, then both at once)
        tl, first = plan.host_timeline()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()
        e0.record(stream)
        for h_, x in zip(hin, xs):
            x.copy_(h_, non_blocking=True)
        e1.record(stream)
        for h_, y in zip(hout, ys):
            h_.copy_(y, non_blocking=True)
        e2.record(stream)
        torch.cuda.synchronize()
        h2d_ms, d2h_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        s_up.wait_stream(stream)
        s_dn.wait_stream(stream)
        t0 = time.perf_counter()
        with torch.cuda.stream(s_up):
            for h_, x in zip(hin, xs):
                x.copy_(h_, non_blocking=True)
        with torch.cuda.stream(s_dn):
            for h_, y in zip(hout, ys):
                h_.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        both_ms = 1000.0 * (time.perf_counter() - t0)
        e2e = {"value": whole_job_rate(world, n, args.steps, e2e_ms), "unit": "matrices/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bi, "ms_per_step": e2e_ms / args.steps,
               "api": "ifnso_orthogonalize_host, page-locked host buffers in one huge-page-backed block, "
                      + (f"{args.groups} groups" if args.groups > 0 else "default grouping"),
               "host_enqueue_ms": host_ms,
               "per_step_ms": per_step_ms.get("e2e"),
               "median_ms_per_step": (float(np.median(per_step_ms["e2e"])) if per_step_ms.get("e2e") else None),
               "copies_alone": {"h2d_ms": h2d_ms, "h2d_GBs": bi / h2d_ms / 1e6, "d2h_ms": d2h_ms,
                                "d2h_GBs": bi / d2h_ms / 1e6, "both_directions_at_once_ms": both_ms},
               "timeline": {"what": "last timed step, per group: [uploads done, passes done, downloads done] "
                                    "in ms since the call's start",
                            "group_first_matrix": first,
                            "ms": [[round(float(v), 3) for v in row] for row in tl]}}
        plan.pass_times()
        del hin, hout, host
        release_host()

    # 5-step quintic Newton-Schulz on the same list
    nsplan = F.Plan(hmax, wmax, dtype, L=1)
    nsplan.set(F.IFNSO_OPT_CTA_GROUP, args.cta_group)
    if dtype == "bf16" and plan.get(F.IFNSO_OPT_CTA_GROUP_KINDS):
        # the baseline runs its passes in the modes the autotuner chose for IFNSO's passes of the same shape
        nsplan.set(F.IFNSO_OPT_CTA_GROUP_KINDS, plan.get(F.IFNSO_OPT_CTA_GROUP_KINDS))
    nsplan.set(F.IFNSO_OPT_TIMING, 1)
    nsws = F.Workspace(nsplan.ns_workspace_bytes(batch), device=device)
    zs = [torch.empty(x.shape, dtype=x.dtype, device=device) for x in xs]
    for _ in range(max(args.warmup, 3)):
        nsplan.ns_iterate(batch, MUON_ABC, 5, zs, ws=nsws)
    torch.cuda.synchronize()
    ns_step, _ = make_step(lambda: nsplan.ns_iterate(batch, MUON_ABC, 5, zs, ws=nsws))
    ns_step()
    torch.cuda.synchronize()
    ns_ms = timed_steps(ns_step, args.steps)
    ns_pass, _ = averaged_pass_times(nsplan, ns_step, args.steps)
    ns_value = whole_job_rate(world, n, args.steps, ns_ms)
    ns_on_chip = dtype == "bf16" and hmax <= 128
    ns_tflops = world * sum(flops_ns5(h, w) for h, w in hw) * args.steps / (ns_ms / 1000.0) / 1e12
    quality = None
    if rank == 0 and not args.no_quality:
        quality = polar_quality(torch, shapes, xs, {"ifnso": ys, "ns5": zs})
    del nsws, zs


    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sample, cores = cpu_oracle_sample(wl, shapes, L)
        cpu = {"value": v, "unit": "matrices/s", "cores": cores, "kind": "oracle", "sample": sample}

    lim = plan.get(F.IFNSO_OPT_STAGE_LIMITS)
    stage_limits = {k: ((lim >> (4 * i)) & 15) or "whole ring"
                    for i, k in enumerate(["gram", "split_squaring", "plain_squaring", "product", "final_squaring"])}
    if dtype != "bf16":
        product_label = ""
    elif plan.get(F.IFNSO_OPT_APPLY_F16):
        product_label = "; product: P in FP16 times an FP16 copy of A scaled by a power of two"
    else:
        product_label = "; product: P as BF16 hi+lo" if mode != F.IFNSO_PREC_PLAIN else "; product: P in BF16"
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload + ": " + wl["desc"], "L": L,
                       "precision": {F.IFNSO_PREC_PLAIN: "plain FP16 squarings",
                                     F.IFNSO_PREC_SPLIT: "split FP16 hi+lo squarings",
                                     F.IFNSO_PREC_MIXED: f"mixed: first {k_split} squarings split FP16 hi+lo, "
                                                         f"last {L - 1 - k_split} plain FP16"}.get(mode, "")
                                    + product_label,
                       "matrices_per_gpu": n, "parallelism": f"dp{world} (independent lists per GPU)",
                       "l2": ("inputs larger than L2 (no flush)" if flush is None else
                              "inputs smaller than twice L2: a 512 MB buffer is written before every step, "
                              "and only the steps are timed (CUDA events around each)"),
                       "launch": "CUDA graph of one step, replayed" if args.graph else "eager calls",
                       "mma": ({k: ("CTA pair (M = 256)" if v == 2 else "per CTA (M = 128), whole B tile per CTA")
                                for k, v in tuned.items()} if tuned else
                               {0: "tcgen05 MMAs of the CTA pair (M = 256) for the split squarings, per-CTA "
                                   "MMAs (each CTA loading its whole B tile) for the other passes",
                                1: "per-CTA tcgen05 MMAs, each CTA loading its whole B tile",
                                2: "tcgen05 MMAs of the CTA pair (M = 256)"}[args.cta_group]),
                       "autotuned": tuned is not None,
                       "stage_limits": stage_limits,
                       "fp16_copy": fp16_copy,
                       "small_matrices": ({1: "on-chip path (one CTA per matrix, all of Algorithm 1 in one launch)",
                                           2: "tiled passes"}.get(plan.get(F.IFNSO_OPT_SMALL_TUNED),
                                                                  "not applicable (a matrix has h > 128)")
                                          if dtype == "bf16" else "FP32 SIMT passes"),
                       "coefficients": ("per-matrix proposals of the coefficient network, computed inside each "
                                        "call after the first squaring" if args.coeffs == "mlp" else
                                        "fixed, learned on the GPU by ifnso_learn_coefficients (Sec. 3.1.1 "
                                        "schedule)"),
                       "coefficient_network": mlp_info,
                       "gram": "E4M3 copy of A s, FP32 accumulation (experiment)" if args.gram_e4m3 else "BF16",
                       "scale": {"gram": "X = A / ||A A^T||_F^(1/2) (q = 1, the paper's)",
                                 "frob": "X = A / ||A||_F",
                                 "gelfand2": "X = A / ||(A A^T)^2||_F^(1/4) (Gelfand, q = 2)"}[args.scale]},
            "tflops": tflops,
            "ns5": {"value": ns_value, "unit": "matrices/s", "tflops": ns_tflops, "ms_per_step": ns_ms / args.steps,
                    "mma": ("on-chip path (one CTA per matrix, every step in one launch)" if ns_on_chip
                            else "the autotuned modes of IFNSO's Gram, plain squarings and product"
                            if dtype == "bf16" and plan.get(F.IFNSO_OPT_CTA_GROUP_KINDS) else "per-CTA MMAs"),
                    "ifnso_over_ns5": value / ns_value,
                    "pass_ms_per_step": [float(x) for x in ns_pass],
                    "passes": ("one launch: per step S = X X^T, B = b S + c S^2, X <- a X + B X" if ns_on_chip else
                               "norm and scalars, then per step: Gram S = X X^T, B = b S + c S^2, X <- a X + B X")},
            "quality": quality,
            "clocks": clk, "gpu_launches": int(launches), "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
