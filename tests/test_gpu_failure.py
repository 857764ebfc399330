"""Failure detection through the C ABI, in forms that fault no GPU: bad
values made on the host (a NaN or Inf in an input tensor or an initial
factor) and a bounded device-side wait that is made to run out (a one-CTA
self-test kernel waits on an mbarrier nothing arrives at, with no copy or
MMA in flight).  Each must come back as its status code, and the handle must
stay usable."""

import time

import numpy as np
import pytest

from tests.gpu_common import coupled_inputs, need_gpu, rel_fro

pytestmark = pytest.mark.gpu

ENONFINITE, ETIMEOUT = -4, -5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _P():
    import paper_2302_05119_gb300 as P
    return P


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_nonfinite_input_tensor_reports_enonfinite(bad, dt):
    P = _P()
    Xs, _, U0 = coupled_inputs([(10, 9, 8)] * 2, 3, [1, 0, 0], seed=21)
    Xs = [X.astype(dt) for X in Xs]
    Xs[1][3, 4, 5] = bad
    m = P.CoupledNCP(Xs, 3, [1, 0, 0])
    m.set_factors(U0)
    with pytest.raises(P.CncpdError) as e:
        m.step(1)
    assert e.value.code == ENONFINITE, str(e.value)
    m.close()
    # a later handle on clean data is unaffected
    Xs[1][3, 4, 5] = 0.5
    ok = P.CoupledNCP(Xs, 3, [1, 0, 0])
    ok.set_factors(U0)
    s = ok.step(2)
    assert np.isfinite(s["F"])
    ok.close()


def test_nonfinite_initial_factor_reports_enonfinite():
    P = _P()
    Xs, _, U0 = coupled_inputs([(10, 9, 8)] * 2, 3, [1, 0, 0], seed=22)
    m = P.CoupledNCP([X.astype(np.float32) for X in Xs], 3, [1, 0, 0])
    U0[0][2] = U0[0][2].copy()
    U0[0][2][1, 1] = np.nan
    m.set_factors(U0)
    with pytest.raises(P.CncpdError) as e:
        m.step(1)
    assert e.value.code == ENONFINITE, str(e.value)
    # the same handle recovers once the factors are finite again
    U0[0][2][1, 1] = 0.25
    m.set_factors(U0)
    assert np.isfinite(m.step(2)["F"])
    m.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_bounded_wait_times_out_and_handle_recovers(use_graph):
    """The self-test wait is given 1 ms and no arrival: the call returns
    ETIMEOUT quickly, and afterwards the handle runs Algorithm 1 afresh from
    its current factors, exactly like a new handle given those factors."""
    P = _P()
    dims = [(20, 18, 16)] * 3
    Xs, _, U0 = coupled_inputs(dims, 4, [2, 0, 0], seed=23)
    X32 = [X.astype(np.float32) for X in Xs]
    m = P.CoupledNCP(X32, 4, [2, 0, 0], use_graph=use_graph)
    m.set_factors(U0)
    m.step(3)
    U3 = m.factors(np.float32)
    t0 = time.perf_counter()
    code, msg = m.check_wait_timeout(1.0)
    dt = time.perf_counter() - t0
    assert code == ETIMEOUT, msg
    assert "wait" in msg
    assert dt < 1.0, dt
    s = m.step(4)
    assert s["iters"] == 4 and np.isfinite(s["F"])
    ref = P.CoupledNCP(X32, 4, [2, 0, 0], use_graph=use_graph)
    ref.set_factors(U3)
    ref.step(4)
    for k in range(3):
        for n in range(3):
            assert rel_fro(m.factor(k, n), ref.factor(k, n)) <= 1e-6, (k, n)
    # a second timeout on the same handle behaves the same
    assert m.check_wait_timeout(0.01)[0] == ETIMEOUT
    assert np.isfinite(m.step(1)["F"])
    ref.close()
    m.close()


def test_wait_timeout_limit_is_validated():
    P = _P()
    Xs, _, U0 = coupled_inputs([(6, 5, 4)], 2, [0, 0, 0], seed=24)
    m = P.CoupledNCP(Xs, 2, [0, 0, 0])
    assert m.check_wait_timeout(0.0)[0] == -1
    assert m.check_wait_timeout(5000.0)[0] == -1
    m.close()
