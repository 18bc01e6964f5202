"""Write tests/golden/equal_polar.json: distance to the polar factor U V^T (per sqrt(h)) of
the 5-step quintic NS and of IFNSO at depths L = 4..20 on one low-rank-plus-noise matrix of each
shape of the synthetic 1B list, by spectral evaluation in FP64 (oracle + synth only), under the
paper's scaling (q = 1) and under Gelfand's bound with q = 2.
The smallest L whose distance is at or below NS5 is the depth the benchmark uses.

Run:  python tests/golden/make_equal_polar.py
"""
import json
import os
import sys
import time

import numpy as np
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import synth
from oracle import ifnso as O, ns as ONS
art = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), 'ifnso_coeffs.json')))
res = {}
for name, r, c, seed in [("sq2048", 2048, 2048, 0), ("wide2048x5632", 2048, 5632, 4), ("tall5632x2048", 5632, 2048, 6)]:
    t0 = time.time()
    M = synth.bf16_bits_to_f64(synth.lowrank_noise_bf16(seed, r, c))
    A, tr = O.orient(M)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    P = U @ Vt
    h = A.shape[0]
    def pd(Y):
        Yo = O.orient(Y)[0]
        return float(np.linalg.norm(Yo - P) / np.sqrt(h))
    out = {"sigma_max": float(s[0]), "sigma_33": float(s[32]), "sigma_min": float(s[-1])}
    out["ns5"] = pd(ONS.ns_quintic(M, 5))
    # spectral evaluation (exact, from the SVD) for each L
    o = np.sqrt(np.sum(s**4))
    x = s / np.sqrt(o)
    out["x_signal_min"] = float(x[31]); out["x_noise_max"] = float(x[32]); out["x_min"] = float(x[-1])
    # Gelfand's bound with q = 2: x = s / ||T_0^2||_F^(1/4)
    x2 = s / np.sum(s**8) ** 0.125
    for L in range(4, 21):
        w = np.array(art["L"][str(L)]["w"])
        y = O.f_scalar(x, w)
        out[f"ifnso_L{L}"] = float(np.sqrt(np.sum((y - 1)**2) / h))
        y2 = O.f_scalar(x2, w)
        out[f"ifnso_gelfand2_L{L}"] = float(np.sqrt(np.sum((y2 - 1)**2) / h))
    # NS5 spectral (Frobenius scaling)
    xf = s / np.sqrt(np.sum(s**2))
    out["ns5_spectral"] = float(np.sqrt(np.sum((ONS.ns_scalar(xf, ONS.MUON_ABC, 5) - 1)**2) / h))
    out["secs"] = time.time() - t0
    res[name] = out
    print(name, json.dumps(out), flush=True)
json.dump(res, open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "equal_polar.json"), "w"), indent=1)
