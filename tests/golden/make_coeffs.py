"""Write tests/golden/ifnso_coeffs.json: the fixed IFNSO coefficients learned by
the FP64 oracle learner (Sec. 2.3 objective, Sec. 3.1.1 schedule) for every
depth L used by the tests.

Calls only oracle/ (the learner) and synth/ (the Philox samples it draws).
Run:  python tests/golden/make_coeffs.py
"""
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SEED = 0
ITERS = 20000
SAMPLES = 1000
LS = list(range(1, 21))


def _one(L):
    import numpy as np

    from oracle import coeffs as C
    from synth import learner_uniforms

    w, _ = C.learn(L, lambda t: learner_uniforms(SEED, t, SAMPLES), iters=ITERS)
    xe = np.linspace(1e-4, 1 - 1e-4, 20001)
    mse = float(np.mean((C.f_full(xe, w) - 1) ** 2))
    return L, [float(v) for v in w], mse


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_one, sorted(LS, reverse=True))
    out = {
        "source": "oracle.coeffs.learn: Adam lr 0.1, x0.5 every 10000 iterations, 20000 iterations, "
                  "1000 uniform samples of (0,1) per iteration (Sec. 3.1.1), w_L from Eq. b_approximation",
        "seed": SEED, "iters": ITERS, "samples": SAMPLES,
        "eval": "eval_mse = mean (f(x) - 1)^2 over 20001 points of [1e-4, 1 - 1e-4]",
        "L": {str(L): {"w": w, "eval_mse": mse} for L, w, mse in sorted(res)},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ifnso_coeffs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
