"""Write tests/golden/equal_polar.json: distance to the polar factor U V^T (per sqrt(h)) of
the 5-step quintic NS and of IFNSO at depths L = 4..20 on low-rank-plus-noise matrices of each
shape of the synthetic 1B list, by spectral evaluation in FP64 (oracle + synth only), under the
paper's scaling (q = 1) and under Gelfand's bound with q = 2.

For each shape the first matrix of that shape (list seed 0, 4 or 6) is written out in full, with
the matrix NS5 iteration beside its spectral evaluation, and a sweep over 8 matrices of the same
shape from 8 layers of the list (seeds s0 + 7k, k = 0..7) gives the spread: per seed, the NS5
distance and the IFNSO distance for every L, and their mean and standard deviation.  The depth
the benchmark uses is the smallest L whose IFNSO distance is at or below NS5's on every swept
matrix of every shape.

Run:  python tests/golden/make_equal_polar.py
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import synth  # noqa: E402
from oracle import ifnso as O, ns as ONS  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
art = json.load(open(os.path.join(HERE, "ifnso_coeffs.json")))
LS = range(4, 21)
SWEEP = 8


def distances(s, h):
    """Spectral distances per sqrt(h) from the singular values s of the oriented input."""
    out = {}
    x = s / np.sqrt(np.sqrt(np.sum(s ** 4)))          # q = 1: s / ||T_0||_F^(1/2)
    x2 = s / np.sum(s ** 8) ** 0.125                    # q = 2: s / ||T_0^2||_F^(1/4)
    for L in LS:
        w = np.array(art["L"][str(L)]["w"])
        out[f"ifnso_L{L}"] = float(np.sqrt(np.sum((O.f_scalar(x, w) - 1) ** 2) / h))
        out[f"ifnso_gelfand2_L{L}"] = float(np.sqrt(np.sum((O.f_scalar(x2, w) - 1) ** 2) / h))
    xf = s / np.sqrt(np.sum(s ** 2))                    # NS: s / ||A||_F
    out["ns5_spectral"] = float(np.sqrt(np.sum((ONS.ns_scalar(xf, ONS.MUON_ABC, 5) - 1) ** 2) / h))
    return out, x


res = {}
for name, r, c, seed0 in [("sq2048", 2048, 2048, 0), ("wide2048x5632", 2048, 5632, 4),
                          ("tall5632x2048", 5632, 2048, 6)]:
    t0 = time.time()
    sweep = []
    first = None
    for k in range(SWEEP):
        seed = seed0 + 7 * k
        M = synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(seed, r, c))
        A, _ = O.orient(M)
        h = A.shape[0]
        if k == 0:
            U, s, Vt = np.linalg.svd(A, full_matrices=False)
            P = U @ Vt
            out, x = distances(s, h)
            out = {"seed": seed, "sigma_max": float(s[0]), "sigma_33": float(s[32]), "sigma_min": float(s[-1]),
                   "x_signal_min": float(x[31]), "x_noise_max": float(x[32]), "x_min": float(x[-1]), **out}
            out["ns5"] = float(np.linalg.norm(O.orient(ONS.ns_quintic(M, 5))[0] - P) / np.sqrt(h))
            first = out
            d = out
        else:
            s = np.linalg.svd(A, compute_uv=False)
            d, _ = distances(s, h)
            d["seed"] = seed
        sweep.append(d)
    keys = ["ns5_spectral"] + [f"ifnso_L{L}" for L in LS] + [f"ifnso_gelfand2_L{L}" for L in LS]
    first["sweep"] = {
        "seeds": [d["seed"] for d in sweep],
        **{k: [d[k] for d in sweep] for k in keys},
        "mean": {k: float(np.mean([d[k] for d in sweep])) for k in keys},
        "std": {k: float(np.std([d[k] for d in sweep])) for k in keys},
    }
    first["secs"] = time.time() - t0
    res[name] = first
    print(name, json.dumps({k: first[k] for k in ("ns5", "ns5_spectral", "ifnso_L13", "ifnso_L14",
                                                    "ifnso_gelfand2_L13")}),
          json.dumps({k: first["sweep"]["mean"][k] for k in ("ns5_spectral", "ifnso_L14", "ifnso_gelfand2_L13")}),
          flush=True)
json.dump(res, open(os.path.join(HERE, "equal_polar.json"), "w"), indent=1)
