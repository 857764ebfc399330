"""Upload paths of cncpd_create and the factor setters.  Page-locked host
tensors are read in place by the quantising kernel, pageable ones through a
staging copy, device ones directly: all three must store the same values
(bit-identical iterates).  cncpd_set_factors_all must equal one
cncpd_set_factors call per block and mode, shared columns included."""

import ctypes

import numpy as np
import pytest

from tests.gpu_common import coupled_inputs, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("storage", ["f32", "bf16", "bf16x2", "f64"])
def test_pinned_pageable_and_device_uploads_agree(storage):
    import torch

    import paper_2302_05119_gb300 as P
    Xs, _, U0 = coupled_inputs([(30, 20, 40), (30, 25, 17)], 4, [2, 0, 0], seed=90)
    X32 = [X.astype(np.float32) for X in Xs]
    srcs = {"pageable": X32,
            "pinned": [torch.from_numpy(X).pin_memory() for X in X32],
            "device": [torch.from_numpy(X).cuda() for X in X32]}
    assert all(t.is_pinned() for t in srcs["pinned"])
    out = {}
    for name, X in srcs.items():
        m = P.CoupledNCP(X, 4, [2, 0, 0], storage=storage)
        m.set_factors(U0)
        s = m.step(3)
        out[name] = (s["F"], m.factors())
        m.close()
    for name in ("pinned", "device"):
        assert out[name][0] == out["pageable"][0], name
        for k in range(2):
            for n in range(3):
                assert np.array_equal(out[name][1][k][n], out["pageable"][1][k][n]), (name, k, n)


def test_set_factors_all_equals_per_factor_calls():
    import paper_2302_05119_gb300 as P
    from paper_2302_05119_gb300 import _lib as C
    Xs, _, U0 = coupled_inputs([(12, 10, 9)] * 3, 4, [2, 1, 0], seed=91)
    # blocks 1 and 2 carry their own (different) values in the shared columns:
    # only block 0's may be used
    rng = np.random.default_rng(92)
    for k in (1, 2):
        for n in range(3):
            U0[k][n] = U0[k][n].copy()
            U0[k][n][:, :2] = rng.random((U0[k][n].shape[0], 2))
    a = P.CoupledNCP(Xs, 4, [2, 1, 0])
    a.set_factors(U0)
    b = P.CoupledNCP(Xs, 4, [2, 1, 0])
    keep = []
    for k in range(3):
        for n in range(3):
            arr = np.ascontiguousarray(U0[k][n], dtype=np.float64)
            keep.append(arr)
            C.check(C.cncpd_set_factors(b._h, k, n, ctypes.c_void_p(arr.ctypes.data), C.CNCPD_F64))
    Fa, Fb = a.factors(), b.factors()
    for k in range(3):
        for n in range(3):
            assert np.array_equal(Fa[k][n], Fb[k][n]), (k, n)
            Ln = [2, 1, 0][n]
            assert np.array_equal(Fa[k][n][:, :Ln], U0[0][n][:, :Ln])
            assert np.array_equal(Fa[k][n][:, Ln:], U0[k][n][:, Ln:])
    assert a.step(2)["F"] == b.step(2)["F"]
    a.close()
    b.close()
