"""FP64 CPU oracle for IFNSO (Iteration-Free Newton-Schulz Orthogonalization,
arXiv 2602.02500) and for the Newton-Schulz iterations it is compared with.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct NumPy code in FP64,
each function citing the passage of the paper it follows.  It shares no code
with the CUDA library and imports nothing from it.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it; the product path never does.

Modules
-------
ifnso   Algorithm 1 literally (T basis), the algebraically equal D basis, the
        spectral evaluation through the SVD, the polar factor, error metrics.
ns      classical cubic Newton-Schulz and Muon's quintic iteration.
coeffs  the scalar polynomial f, the peak constraint on w_L (exact and the
        printed approximation), the Adam coefficient learner of Sec. 2.3/3.1.1.
flops   the FLOP counts behind Table 1.
mlp     FP64 forward/backward of the coefficient-proposal MLP.
muon    one Muon step (momentum, Nesterov input, scaled update) around Algorithm 1.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute force or printed values, except the learned
coefficient values themselves (the paper prints none): "parity unpinned" for
the fitted values of ``coeffs.learn``; its determinism, descent and optimality
conditions are pinned instead.
"""
