"""Trailing-mode contraction of FP32-stored third-order tensors on the TF32
tensor cores (opt-in: cncpd_opts.tf32).  X and the factor are each split into two TF32 parts (x = xb +
xs up to 2^-23 |x|), and all four part products accumulate in FP32, so the
MTTKRPs must match the FP64 oracle to FP32 accumulation accuracy (the same
2e-6 bound as the CUDA-core pass) on shapes with ragged row tiles, ragged K
(I3 not a multiple of 32) and ranks 1..32; and the APG iterations must match
the oracle as tightly as the CUDA-core path does.  The stats field
trail_tensor_cores shows which pass ran."""

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


@pytest.mark.parametrize("dims,R", [
    ([(70, 37, 150), (9, 64, 130)], 10),
    ([(33, 41, 200)], 20),
    ([(20, 30, 40)], 32),
    ([(17, 19, 33), (40, 8, 1)], 1),
    ([(300, 260, 97), (280, 260, 136)], 16),
    ([(64, 64, 256)] * 3, 7),
])
def test_tf32_trailing_mttkrp_matches_oracle(dims, R):
    rng = np.random.default_rng(70 + R + len(dims))
    Xs = [rng.random(d).astype(np.float32) for d in dims]
    U = [[rng.random((I, R)).astype(np.float32) for I in d] for d in dims]
    m = _P().CoupledNCP(Xs, R, [0, 0, 0], tensor_cores=True, tf32=True)
    m.set_factors(U)
    for k in range(len(dims)):
        for n in range(3):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= 2e-6, (k, n, rel_fro(got, want))
    assert m.step(1)["trail_tensor_cores"] == 1
    m.close()


def test_tf32_trailing_signed_and_wide_range_values():
    """Negative entries and values spread over 2^-20 .. 2^20: the parts are
    formed per element, so relative accuracy holds for every magnitude."""
    rng = np.random.default_rng(77)
    d = (48, 40, 72)
    X = (rng.standard_normal(d) * np.exp2(rng.integers(-20, 21, d))).astype(np.float32)
    U = [rng.standard_normal((I, 12)).astype(np.float32) for I in d]
    m = _P().CoupledNCP([X], 12, [0, 0, 0], tensor_cores=True, tf32=True, nonneg=[False] * 3)
    m.set_factors([U])
    for n in range(3):
        got = m.mttkrp(0, n)
        want = O.mttkrp(X.astype(np.float64), [A.astype(np.float64) for A in U], n)
        # entries of mixed sign cancel: bound each by the sum of magnitudes
        # (FP32 accumulation of up to 2 880 terms; a lost TF32 part would
        # leave errors near 2^-11)
        mag = O.mttkrp(np.abs(X.astype(np.float64)), [np.abs(A.astype(np.float64)) for A in U], n)
        assert np.max(np.abs(got - want) / mag) <= 1e-5, n
    m.close()


@pytest.mark.parametrize("R,L,dims", [
    (10, [3, 3, 0], [(40, 36, 70), (40, 36, 45), (40, 36, 90)]),
    (24, [0, 5, 2], [(40, 36, 70), (30, 36, 70), (50, 36, 70)]),
])
def test_tf32_trailing_apg_iterations_match_oracle(R, L, dims):
    Xs, _, U0 = coupled_inputs(dims, R, L, seed=78)
    snaps_o, res_o = run_oracle_steps(Xs, [R] * 3, L, U0, 8)
    m = _P().CoupledNCP([X.astype(np.float32) for X in Xs], R, L, tensor_cores=True, tf32=True)
    m.set_factors(U0)
    for it in range(8):
        s = m.step(1)
        assert s["trail_tensor_cores"] == 1
        assert (s["reupdates"] > 0) == res_o["hist"]["redo"][it]
        U = m.factors()
        for k in range(3):
            for n in range(3):
                e = rel_fro(U[k][n], snaps_o[it][0][k][n])
                assert e <= 1e-5, (it, k, n, e)
    m.close()


@pytest.mark.parametrize("kw", [dict(tensor_cores=False, tf32=True), dict()])
def test_tf32_is_opt_in(kw):
    """Without tf32 (the default), or with the tensor cores off, FP32 data
    keeps the CUDA-core pass; both paths give the same iterates."""
    Xs, _, U0 = coupled_inputs([(20, 18, 40)] * 2, 5, [1, 0, 0], seed=79)
    a = _P().CoupledNCP([X.astype(np.float32) for X in Xs], 5, [1, 0, 0], **kw)
    b = _P().CoupledNCP([X.astype(np.float32) for X in Xs], 5, [1, 0, 0], tensor_cores=True, tf32=True)
    a.set_factors(U0)
    b.set_factors(U0)
    assert a.step(3)["trail_tensor_cores"] == 0
    assert b.step(3)["trail_tensor_cores"] == 1
    for k in range(2):
        for n in range(3):
            assert rel_fro(a.factor(k, n), b.factor(k, n)) <= 1e-5
    a.close()
    b.close()


def test_huge_values_keep_the_cuda_core_pass():
    """The TF32 split multiplies X by 2^13 + 1, so a tensor whose norm
    reaches 2^114 stays on the CUDA-core pass (and is still exact)."""
    rng = np.random.default_rng(80)
    X = rng.random((20, 18, 40)).astype(np.float32)
    X[3, 4, 5] = 3e35
    U = [rng.random((I, 6)).astype(np.float32) for I in X.shape]
    m = _P().CoupledNCP([X], 6, [0, 0, 0], tensor_cores=True, tf32=True)
    m.set_factors([U])
    assert m.step(0)["trail_tensor_cores"] == 0  # no iteration: FP32 would overflow on such data
    for n in range(3):
        got = m.mttkrp(0, n)
        want = O.mttkrp(X.astype(np.float64), [A.astype(np.float64) for A in U], n)
        assert rel_fro(got, want) <= 2e-6, n
    m.close()
