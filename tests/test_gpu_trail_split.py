"""Column ranges of the trailing-mode contraction (FP32 / BF16 CUDA-core
pass).  When one block's rows are so long that a single 256-row tile would
outlast the average CTA, the tile is cut into ranges of whole stages along
its columns; each range leaves partial products that a second kernel adds in
range order.  The MTTKRPs and the APG iterations must still match the FP64
oracle, on shapes that take the cut (checked through the stats field
trail_ranges), with ragged last ranges and ragged row tiles."""

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


def _to_bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


# long-row fourth-order blocks of uneven sizes: rows I1*I2, columns I3*I4
UNEVEN = [(16, 17, 61, 89), (16, 17, 23, 40), (9, 31, 97, 70), (16, 16, 11, 13)]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("R", [7, 12, 20])
def test_split_trailing_mttkrp_matches_oracle(storage, R):
    rng = np.random.default_rng(60 + R)
    Xs = [rng.random(d).astype(np.float32) for d in UNEVEN]
    if storage == "bf16":
        Xs = [_to_bf16(X) for X in Xs]  # lossless in BF16 storage
    U = [[rng.random((I, R)).astype(np.float32) for I in d] for d in UNEVEN]
    m = _P().CoupledNCP(Xs, R, [0] * 4, storage=storage, tensor_cores=False)
    m.set_factors(U)
    for k in range(len(UNEVEN)):
        for n in range(4):
            got = m.mttkrp(k, n)
            want = O.mttkrp(Xs[k].astype(np.float64), [A.astype(np.float64) for A in U[k]], n)
            assert rel_fro(got, want) <= 2e-6, (k, n)
    s = m.step(1)
    assert s["trail_ranges"] > 1, s
    m.close()


@pytest.mark.parametrize("dt,tol", [(np.float32, 1e-5)])
def test_split_trailing_apg_iterations_match_oracle(dt, tol):
    """Six iterations of Algorithm 1 with coupled columns in the first two
    modes, every block's factors against the oracle's after each one."""
    R, L = 6, [2, 2, 0, 0]
    dims = [(16, 17, 61, 89), (16, 17, 23, 40), (16, 17, 97, 30)]
    Xs, _, U0 = coupled_inputs(dims, R, L, seed=61)
    snaps_o, res_o = run_oracle_steps(Xs, [R] * 3, L, U0, 6)
    m = _P().CoupledNCP([X.astype(dt) for X in Xs], R, L)
    m.set_factors(U0)
    for it in range(6):
        s = m.step(1)
        assert s["trail_ranges"] > 1
        assert (s["reupdates"] > 0) == res_o["hist"]["redo"][it]
        U = m.factors()
        for k in range(3):
            for n in range(4):
                e = rel_fro(U[k][n], snaps_o[it][0][k][n])
                assert e <= tol, (it, k, n, e)
    m.close()


def test_split_trailing_full_size_eeg_blocks():
    """The 16 uneven EEG-shaped blocks at full size (FP32 storage): the
    trailing pass takes column ranges, and the first-mode MTTKRP of the three
    longest-row blocks matches the oracle to FP32 accumulation accuracy."""
    import synth
    w = synth.workload("eeg_uneven_4th")
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    m = _P().CoupledNCP(Xs, w.R, w.L)
    m.set_factors(U0)
    U = m.factors()  # the shared columns as the library holds them (block 0's)
    J = [d[2] * d[3] for d in w.dims]
    for k in sorted(range(w.K), key=lambda k: -J[k])[:3]:
        got = m.mttkrp(k, 0)
        want = O.mttkrp(Xs[k].astype(np.float64), U[k], 0)
        assert rel_fro(got, want) <= 1e-5, k
    assert m.step(1)["trail_ranges"] > 1
    m.close()
