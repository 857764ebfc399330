"""The simulation design of Section IV-A on the GPU, with its performance
index: S = 20 coupled blocks of 100 x 100 x 100, R = 10, 20 dB noise, for
each coupling pattern of Table III (L = [10,10,10], [5,5,5], [10,10,0],
[5,5,0], [10,0,0], [5,0,0]); the fully coupled patterns also with the core
tensors (Section III-C).  CoNCPD-APG runs to the termination rule of
Section III-C on the library; the factors are scored against the ground
truth with the oracle's performance index (PI, Section IV settings) and the
global Fit.

The paper's printed Fit / PI values come from a noise model whose formula
is garbled and from MATLAB's random streams, so they are not reproduced
(parity unpinned); the checks are the ones the method guarantees on this
synthetic data: the Fit reaches the noise floor (about 1 - 10^(-20/20) =
0.9 at 20 dB) and the factors are recovered up to permutation and scaling
(small PI)."""

import numpy as np
import pytest

from oracle import cncpd_oracle as O
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


CASES = [("e1a_l10", False), ("e1a_l10", True), ("e1a_l5", False), ("e1a_l5", True),
         ("e1b_l10", False), ("e1b_l5", False), ("e1c_l10", False), ("e1c_l5", False)]


@pytest.mark.parametrize("name,use_core", CASES)
def test_simulation_design_fit_and_performance_index(name, use_core):
    import torch

    import paper_2302_05119_gb300 as P
    import synth
    w = synth.workload(name)
    assert w.K == 20 and w.dims[0] == (100, 100, 100) and w.R == 10
    Xs, A = synth.make_tensors(w, dtype=np.float32)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    m = P.CoupledNCP([torch.from_numpy(X).cuda() for X in Xs], w.R, w.L, use_core=use_core, eps=1e-8,
                     max_it=1000)
    m.set_factors(U0)
    if use_core:
        m.set_cores(synth.init_cores(w.K, w.R, w.seed))
    s = m.fit()
    U = m.factors()
    fit = m.global_fit()
    lam = [m.core(k) for k in range(w.K)] if use_core else None
    m.close()
    pis = [O.performance_index(U[k][n], A[k][n]) for k in range(w.K) for n in range(w.N)]
    print(f"{name} core={use_core}: {s['total_iters']} iterations, {s['reupdates']} re-updates, "
          f"Fit {fit:.4f}, PI median {np.median(pis):.4f} max {np.max(pis):.4f}")
    assert s["converged"] or s["total_iters"] == 1000
    assert 0.88 <= fit <= 0.92
    assert np.median(pis) < 0.05
    for n, Ln in enumerate(w.L):
        for k in range(1, w.K):
            assert np.array_equal(U[k][n][:, :Ln], U[0][n][:, :Ln])
    if lam is not None:
        assert all(np.all(l >= 0) for l in lam)
