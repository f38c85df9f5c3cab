"""FP64 CPU oracle for the augmented subspace eigensolver (test infrastructure only).

This package is the independent reference that the CUDA path is checked against.
It is plain NumPy/SciPy in float64, written from the paper (Liao, Liu, Xie, Wang,
"PASE: A Massively Parallel Augmented Subspace Eigensolver", arXiv 2502.04589) and
from textbook definitions.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the library never does.  It shares no code
with the CUDA path: both only read their inputs from `pase_inputs`.

Modules
-------
spectrum   closed-form eigenvalues of the Q1 Laplace pencil (tensor product of 1D P1)
dense      brute-force dense generalized eigensolve (the plain definition, §2.1)
mg         damped-Jacobi multigrid V-cycle and per-column CG (the linear solves of
           Alg. 1 / Alg. 3 step 3)
smoother   the learned fine-level smoother: convolutional network, energy-norm loss,
           backward pass and Adam (growth item; not in the paper)
pase       the augmented subspace iteration (Alg. 1, Alg. 3), step by step, with
           a dense solve of the augmented pencil and the PRECOND-A congruence (§4)

Parity status: every function is pinned by a `-m "not gpu"` test (see tests/
test_oracle_pins.py) against a closed form, brute force, or an invariant.
"""
from . import spectrum, dense, mg, pase, smoother  # noqa: F401
