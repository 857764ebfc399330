"""Streamed X (cncpd_opts.stream_x): only one block's stored values are on
the device at a time.  The LRA step of lraCoNCPD-APG runs each block's ALS
with its tensor in the window, the collapsed iterations need no X, and the
global fit streams the blocks once more.  A block's results depend on the
other blocks only through the split-K plan of the lead pass, which a
streamed handle makes per block (each block runs alone): so the streamed
handle must reproduce the resident one up to FP32 summation order, in the
ALS sweeps and errors, the low-rank reconstruction, the objective and the
global fit.  Plain iterations, which need every block each sweep, are
refused before the LRA step."""

import numpy as np
import pytest

from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _face_small(seed=36):
    import synth
    w = synth.Workload("face_small_stream", [(120, 120, 48), (120, 120, 48), (120, 120, 48)], 20, [8, 0, 0], 20.0,
                       seed, sparse_mode=0, density=0.1, R_lra=30)
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    return w, Xs, synth.init_factors(w.dims, w.R, w.seed), synth.init_lra_factors(w.dims, 30, w.seed)


def _run(Xs, w, U0, Ut0, storage, stream_x):
    import paper_2302_05119_gb300 as P
    m = P.CoupledNCP(Xs, w.R, w.L, storage=storage, stream_x=stream_x)
    m.set_factors(U0)
    st = m.lra(30, Ut0)
    from oracle import cncpd_oracle as O
    Ut = [O.kruskal(np.ones(30), [m.lra_factor(k, n) for n in range(3)]) for k in range(w.K)]
    fit0 = m.global_fit()
    s = m.step(10)
    out = (st["lra_sweeps"], st["lra_relerr"], Ut, fit0, s["F"], m.factors(), m.global_fit())
    m.close()
    return out


@pytest.mark.parametrize("storage,source", [
    ("f32", "pageable"), ("f32", "pinned"), ("bf16", "pageable"), ("bf16", "pinned"),
    ("bf16x2", "pageable"), ("bf16x2", "pinned"), ("f64", "pageable"), ("f64", "pinned")])
def test_streamed_lra_reproduces_resident(storage, source):
    import torch
    w, Xs, U0, Ut0 = _face_small()
    if storage == "f64":  # FP64 storage from FP64 tensors (the generic contraction kernels)
        Xs = [X.astype(np.float64) for X in Xs]
    src = Xs if source == "pageable" else [torch.from_numpy(X).pin_memory() for X in Xs]
    a = _run(Xs, w, U0, Ut0, storage, False)
    b = _run(src, w, U0, Ut0, storage, True)
    assert abs(a[0] - b[0]) <= 1, (a[0], b[0])
    assert abs(a[1] - b[1]) <= 1e-5 * a[1], (a[1], b[1])
    # the low-rank tensors X~ (their factors are not unique): with R~ = 30
    # above the data's rank 20 the fit leaves directions free, along which
    # summation-order differences (~1e-7) grow over the ALS sweeps (2e-5
    # measured with BF16 storage); the ALS error and the Fit agree to 1e-5
    for k in range(w.K):
        assert np.linalg.norm(a[2][k] - b[2][k]) <= 1e-4 * np.linalg.norm(a[2][k]), k
    assert abs(a[3] - b[3]) <= 1e-5 and abs(a[6] - b[6]) <= 1e-5, (a[3], b[3], a[6], b[6])
    assert abs(a[4] - b[4]) <= 1e-5 * abs(a[4]), (a[4], b[4])
    for k in range(w.K):
        for n in range(3):
            e = np.linalg.norm(a[5][k][n] - b[5][k][n]) / np.linalg.norm(a[5][k][n])
            assert e <= 1e-4, ("factor", k, n, e)
    assert 0.0 < b[6] < 1.0  # ten collapsed iterations from the initial factors: far from converged


def test_streamed_handle_refuses_plain_iterations_and_holds_one_block():
    import torch

    import paper_2302_05119_gb300 as P
    w, Xs, U0, Ut0 = _face_small(seed=37)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    r = P.CoupledNCP(Xs, w.R, w.L, storage="f32")
    used_resident = free0 - torch.cuda.mem_get_info()[0]
    r.close()
    free0 = torch.cuda.mem_get_info()[0]
    m = P.CoupledNCP(Xs, w.R, w.L, storage="f32", stream_x=True)
    used_streamed = free0 - torch.cuda.mem_get_info()[0]
    block = int(np.prod(w.dims[0])) * 4
    # two of the three stored blocks are not held (allocation granularity aside)
    assert used_streamed <= used_resident - block, (used_resident, used_streamed, block)
    m.set_factors(U0)
    for call in (lambda: m.step(1), lambda: m.fit(), lambda: m.mttkrp(0, 0)):
        with pytest.raises(P.CncpdError) as e:
            call()
        assert e.value.code == -6 and "stream_x" in str(e.value)
    st = m.lra(30, Ut0)
    assert st["lra_sweeps"] >= 1
    s = m.step(3)
    assert np.isfinite(s["F"])
    m.close()
