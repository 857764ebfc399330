"""CUDA path against the FP64 oracle on the shapes beyond the benchmark's:
per-block ranks (Section III-C allows R^(s) to differ between blocks), the
ERP shape (42 fully coupled third-order blocks with cores, Section IV-C) and
the ongoing-EEG shape (14 blocks of 46 x 510 x 64 with ranks 33..44,
Section IV-D), which also take the update kernel's many-blocks branch (K
times the padded rank above 512); and ALS at a scaled-down face shape
(sparse first mode, R~ = 30 above R = 20)."""

import numpy as np
import pytest

from oracle import cncpd_oracle as O
from tests.gpu_common import coupled_inputs, need_gpu, rel_fro, run_oracle_steps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _P():
    import paper_2302_05119_gb300 as P
    return P


def _gpu_steps(Xs, R, L, U0, iters, dt, use_core=False, lam0=None, storage=None):
    m = _P().CoupledNCP([X.astype(dt) for X in Xs], R, L, use_core=use_core, storage=storage)
    m.set_factors(U0)
    if lam0 is not None:
        m.set_cores(lam0)
    snaps, lams, redo = [], [], []
    for _ in range(iters):
        s = m.step(1)
        redo.append(s["reupdates"] > 0)
        snaps.append(m.factors())
        lams.append([m.core(k) for k in range(len(Xs))])
    m.close()
    return snaps, lams, redo


def _compare(tag, snaps_g, snaps_o, iters, K, N, tol, lams_g=None):
    worst = 0.0
    for it in range(iters):
        for k in range(K):
            if lams_g is not None:
                e = rel_fro(lams_g[it][k], snaps_o[it][1][k])
                worst = max(worst, e)
                assert e <= tol, (tag, it, k, "core", e)
            for n in range(N):
                e = rel_fro(snaps_g[it][k][n], snaps_o[it][0][k][n])
                worst = max(worst, e)
                assert e <= tol, (tag, it, k, n, e)
    print(f"{tag}: worst error {worst:.3e} (bound {tol:g})")


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_unequal_ranks_per_block(dt, tol):
    """Blocks of ranks 3, 5 and 4 sharing L = [2, 1, 0] columns."""
    import synth
    dims = [(12, 10, 9), (12, 10, 9), (12, 10, 7)]
    R = [3, 5, 4]
    L = [2, 1, 0]
    w = synth.Workload("unequal_ranks", dims, R, L, 20.0, 31)
    Xs, _ = synth.make_tensors(w)
    U0 = synth.init_factors(dims, R, 31, tag=1)
    snaps_o, res_o = run_oracle_steps(Xs, R, L, U0, 8)
    snaps_g, _, redo = _gpu_steps(Xs, R, L, U0, 8, dt)
    assert redo == res_o["hist"]["redo"]
    _compare("unequal ranks", snaps_g, snaps_o, 8, 3, 3, tol)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_many_blocks_high_rank_update_branch(dt, tol):
    """K = 16 blocks at R = 40 (K * 40 > 512): the update walks the blocks
    with one CTA per row group (the kernel for wide problems)."""
    dims = [(30, 26, 24)] * 16
    Xs, _, U0 = coupled_inputs(dims, 40, [4, 0, 0], seed=32)
    snaps_o, res_o = run_oracle_steps(Xs, [40] * 16, [4, 0, 0], U0, 5)
    snaps_g, _, redo = _gpu_steps(Xs, 40, [4, 0, 0], U0, 5, dt)
    assert redo == res_o["hist"]["redo"]
    _compare("K=16, R=40", snaps_g, snaps_o, 5, 16, 3, tol)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_erp_shape_fully_coupled_with_cores(dt, tol):
    """ERP shape: 42 blocks of 9 x 71 x 60, R = 36, every column shared in
    every mode, so the blocks differ only by their cores (Section III-C:
    the core tensors are needed when all modes are coupled)."""
    import synth
    w = synth.workload("erp_42x9x71x60")
    Xs, _ = synth.make_tensors(w)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    lam0 = synth.init_cores(w.K, w.R, w.seed)
    snaps_o, res_o = run_oracle_steps(Xs, w.ranks(), w.L, U0, 4, use_core=True, lam0=lam0)
    snaps_g, lams_g, redo = _gpu_steps(Xs, w.R, w.L, U0, 4, dt, use_core=True, lam0=lam0)
    assert redo == res_o["hist"]["redo"]
    _compare("ERP 42x9x71x60", snaps_g, snaps_o, 4, w.K, w.N, tol, lams_g)


@pytest.mark.parametrize("dt,tol", [(np.float64, 1e-9), (np.float32, 1e-5)])
def test_ongoing_eeg_shape_per_block_ranks(dt, tol):
    """Ongoing-EEG shape: 14 blocks of 46 x 510 x 64 with per-block ranks
    drawn in [33, 44] and L = [26, 26, 0]."""
    import synth
    w = synth.workload("eeg_ongoing_14x46x510x64")
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    Xs = [X.astype(np.float64) for X in Xs]
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    snaps_o, res_o = run_oracle_steps(Xs, w.ranks(), w.L, U0, 3)
    snaps_g, _, redo = _gpu_steps(Xs, w.ranks(), w.L, U0, 3, dt)
    assert redo == res_o["hist"]["redo"]
    _compare("ongoing EEG 14x46x510x64", snaps_g, snaps_o, 3, w.K, w.N, tol)


# ------------------------------------------------------------------ LRA ---

@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_als_at_scaled_face_shape(storage):
    """ALS of the LRA step at a scaled-down face shape: 2 blocks of
    120 x 120 x 48 whose first-mode columns are 10 % sparse, R = 20, L_1 =
    8, R~ = 30 > R.  FP64 storage reproduces the oracle's ALS (same sweep
    count, the same approximation to 1e-6); FP32 and BF16 storage reach the
    same ALS relative error within 1e-3 of it.  After 10 collapsed APG
    iterations the global Fit against the original tensors is within 1e-4
    of the oracle's (Algorithm 2)."""
    import synth
    w = synth.Workload("face_small", [(120, 120, 48)] * 2, 20, [8, 0, 0], 20.0, 35, sparse_mode=0,
                       density=0.1, R_lra=30)
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    X64 = [X.astype(np.float64) for X in Xs]
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    Ut0 = synth.init_lra_factors(w.dims, 30, w.seed)
    res = O.lra_apg(X64, Ut0, [20] * 2, w.L, U0, max_it=10, eps=0.0)
    rel_o = float(np.mean([np.linalg.norm(X - O.kruskal(np.ones(30), Ut)) / np.linalg.norm(X)
                           for X, Ut in zip(X64, res["Ut"])]))
    m = _P().CoupledNCP(X64 if storage == "f64" else Xs, 20, w.L, storage=storage)
    m.set_factors(U0)
    st = m.lra(30, Ut0)
    if storage == "f64":
        assert st["lra_sweeps"] == max(res["als_sweeps"])
        for k in range(2):
            Xt_g = O.kruskal(np.ones(30), [m.lra_factor(k, n) for n in range(3)])
            Xt_o = O.kruskal(np.ones(30), res["Ut"][k])
            assert rel_fro(Xt_g, Xt_o) <= 1e-6, k
    assert abs(st["lra_relerr"] - rel_o) <= 1e-3 * rel_o, (st["lra_relerr"], rel_o)
    m.step(10)
    gfit = m.global_fit()
    print(f"ALS face shape ({storage}): sweeps {st['lra_sweeps']} vs {res['als_sweeps']}, relerr "
          f"{st['lra_relerr']:.6f} vs {rel_o:.6f}; global fit {gfit:.6f} vs {res['global_fit']:.6f}")
    assert abs(gfit - res["global_fit"]) <= 1e-4
    m.close()
