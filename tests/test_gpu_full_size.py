"""The CUDA path at the benchmark's full sizes, in the configuration bench.py
times (CUDA graphs, profile events, the persistent TMA passes or the tensor-
core passes), against the FP64 oracle on sampled outputs:

* MTTKRP rows: for sampled rows i of mode n (the first, the last, the ragged
  tails, random ones) the oracle computes row i alone from the slice of X at
  i (the MTTKRP of that slice), compared with the GPU's full product;
* the objective after a few iterations: the GPU's F (Gram expansion, FP32
  factors) against the oracle's explicit reconstruction at the GPU's factors,
  plus nonnegativity and bitwise-shared common columns.
"""

import types

import numpy as np
import pytest

from oracle import cncpd_oracle as O
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _P():
    import paper_2302_05119_gb300 as P
    return P


def _bf16_exact(X):
    import torch
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _sample_rows(I, rng, extra=6):
    base = {0, 1, I // 2, max(0, I - 2), I - 1}
    base.update(int(v) for v in rng.integers(0, I, size=extra))
    return sorted(base)


def _row_oracle(X, U, n, i):
    """Row i of X_(n) U^{odot_-n}: the oracle's MTTKRP of the slice of X at i."""
    Xs = np.take(X, [i], axis=n).astype(np.float64)
    Us = [A.astype(np.float64) for A in U]
    Us[n] = Us[n][i:i + 1]
    return O.mttkrp(Xs, Us, n)[0]


@pytest.mark.parametrize("name,storage", [
    ("sim_256cube", "f32"),
    ("bf16_512x512x256", "bf16"),
    ("eeg_uneven_4th", "f32"),
])
def test_full_size_mttkrp_sampled_rows(name, storage):
    import torch

    import synth
    w = synth.workload(name)
    blocks = [0, w.K - 1] if w.K > 1 else [0]
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    if storage == "bf16":
        Xs = [_bf16_exact(X) for X in Xs]  # stored losslessly: the result is the FP32 accumulation alone
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    m = _P().CoupledNCP([torch.from_numpy(X).cuda() for X in Xs], w.R, w.L, storage=storage, profile=True)
    m.set_factors(U0)
    m.step(1)  # graphs and plans as in the timed region
    m.set_factors(U0)
    U = [[A.astype(np.float32) for A in Uk] for Uk in U0]
    Uc = O.couple_initial(types.SimpleNamespace(N=w.N, K=w.K, L=w.L), U)
    rng = np.random.default_rng(17)
    for k in blocks:
        for n in range(w.N):
            got = m.mttkrp(k, n, np.float64)
            for i in _sample_rows(w.dims[k][n], rng):
                want = _row_oracle(Xs[k], [A.astype(np.float32) for A in Uc[k]], n, i)
                err = np.linalg.norm(got[i] - want) / np.linalg.norm(want)
                assert err <= 2e-5, (name, k, n, i, err)
    m.close()


def test_full_size_objective_and_invariants_sim_256cube():
    import torch

    import synth
    w = synth.workload("sim_256cube")
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    m = _P().CoupledNCP([torch.from_numpy(X).cuda() for X in Xs], w.R, w.L, profile=True)
    m.set_factors(U0)
    s = m.step(9)  # one profiled sweep and eight plain replays
    U = m.factors(np.float64)
    m.close()
    for Uk in U:
        for A in Uk:
            assert A.min() >= 0.0
    for n, Ln in enumerate(w.L):
        for k in range(1, w.K):
            assert np.array_equal(U[k][n][:, :Ln], U[0][n][:, :Ln])
    F = O.objective([X.astype(np.float64) for X in Xs], U, [np.ones(w.R)] * w.K)
    # FP32 Gram expansion against FP64 reconstruction: F is about 5 % of
    # ||X||^2 here, so ~1e-7 relative errors in its terms give ~2e-6 in F
    assert s["F"] == pytest.approx(F, rel=2e-5)


_ORACLE_RUNS = {}


@pytest.mark.parametrize("name,storage,tol", [
    ("sim_256cube", "f32", 1e-5),
    ("bf16_512x512x256", "bf16", 3e-3),
    ("bf16_512x512x256", "bf16x2", 3e-4),
])
def test_full_size_first_iterations_match_oracle(name, storage, tol):
    """The first 10 iterations at the benchmark's full size, in its launch
    configuration (graphs, profile events, TMA or tensor-core passes):
    every factor after every iteration within the stated relative Frobenius
    error of the FP64 oracle (FP32 storage: 1e-5; BF16 storage: 3e-3; BF16
    hi + lo storage: 3e-4; the oracle running on the unquantised FP32 data),
    and the same re-update decisions."""
    import torch

    import synth
    from tests.gpu_common import rel_fro, run_oracle_steps
    w = synth.workload(name)
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    m = _P().CoupledNCP([torch.from_numpy(X).cuda() for X in Xs], w.R, w.L, storage=storage, profile=True)
    m.set_factors(U0)
    snaps_g, redo_g = [], []
    for _ in range(10):
        s = m.step(1)
        redo_g.append(s["reupdates"] > 0)
        snaps_g.append(m.factors(np.float64))
    m.close()
    torch.cuda.empty_cache()
    if name not in _ORACLE_RUNS:  # the BF16 and hi + lo arms share the oracle's run on the FP32 data
        X64 = [X.astype(np.float64) for X in Xs]
        del Xs
        _ORACLE_RUNS[name] = run_oracle_steps(X64, [w.R] * w.K, w.L, U0, 10)
        del X64
    snaps_o, res_o = _ORACLE_RUNS[name]
    assert redo_g == res_o["hist"]["redo"]
    worst = 0.0
    for it in range(10):
        for k in range(w.K):
            for n in range(w.N):
                e = rel_fro(snaps_g[it][k][n], snaps_o[it][0][k][n])
                worst = max(worst, e)
                assert e <= tol, (name, it, k, n, e)
    print(f"{name} ({storage}): worst factor error over 10 iterations {worst:.3e} (bound {tol:g})")
