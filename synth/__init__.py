"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.

This package only draws random numbers and assembles data; it contains none
of the solver's arithmetic (no MTTKRP, Gram, gradient, step or objective).
Both the CUDA path and the FP64 oracle consume its outputs as inputs.

Recipe (following the simulation design of Section IV): ground-truth
nonnegative factors, the first L_n columns of mode n shared by every block
(Eq. tensormodel), the noise-free tensor Y^(k) = sum_r a_r^(1) o ... o a_r^(N),
additive Gaussian noise scaled to the requested SNR in dB as a power ratio,
X = Y + 10^(-SNR/20) ||Y||_F  E / ||E||_F with E standard normal, and
negative entries clipped to 0 (the tensors are nonnegative by assumption).
Initial factors are Uniform[0, 1] (Section IV: MATLAB ``rand``).
"""

from .generate import (  # noqa: F401
    WORKLOADS,
    Workload,
    ground_truth,
    init_cores,
    init_factors,
    init_lra_factors,
    make_tensors,
    workload,
)
