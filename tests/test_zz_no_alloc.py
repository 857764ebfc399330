"""The allocation-free MTTKRP entry point (for callers that must not let the
library call cudaMalloc) against the library's regular MTTKRP entry point and
against the FP64 oracle's MTTKRP, through the C ABI, on two calls in a row.
Collected last on purpose."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_2302_05119_gb300 import build
    build.build()
    from paper_2302_05119_gb300 import _lib
    return torch, _lib


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,R", [((37, 29, 256), 10), ((64, 33, 129), 20), ((5, 3, 7), 1)])
def test_noalloc_matches_regular_mttkrp_twice(shape, R):
    torch, C = _setup()
    import paper_2302_05119_gb300 as P
    rng = np.random.default_rng(R + shape[0])
    X = rng.random(shape).astype(np.float32)
    U = [rng.random((I, R)).astype(np.float32) for I in shape]
    m = P.CoupledNCP([X], R, [0, 0, 0])
    m.set_factors([U])
    ref = m.mttkrp(0, 2, np.float32)
    m.close()
    from oracle import cncpd_oracle as O
    want = O.mttkrp(X.astype(np.float64), [A.astype(np.float64) for A in U], 2)

    dev = torch.device("cuda")
    Xd = torch.from_numpy(X).to(dev)
    U0 = torch.from_numpy(U[0]).to(dev)
    U1 = torch.from_numpy(U[1]).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        M = torch.full((shape[2], R), float("nan"), dtype=torch.float32, device=dev)
        rc = C.cncpd_mttkrp_last_mode_noalloc(ctypes.c_void_p(Xd.data_ptr()), shape[0], shape[1], shape[2],
                                              ctypes.c_void_p(U0.data_ptr()), ctypes.c_void_p(U1.data_ptr()),
                                              R, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, C.lib().cncpd_last_error()
        torch.cuda.synchronize()
        got = M.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= 2e-6
        assert _rel(got, want) <= 2e-6


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, C = _setup()
    dev = torch.device("cuda")
    x = torch.zeros(8, dtype=torch.float32, device=dev)
    # I2 * R = 2^21 + 64 floats exceeds the fixed 8 MiB scratch
    rc = C.cncpd_mttkrp_last_mode_noalloc(ctypes.c_void_p(x.data_ptr()), 1, 1, 32769,
                                          ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          64, ctypes.c_void_p(x.data_ptr()), None)
    assert rc == -1
    assert b"scratch" in C.lib().cncpd_last_error()


def test_noalloc_rejects_host_pointers():
    """Host memory is refused before any kernel runs (this entry point takes
    device memory only)."""
    torch, C = _setup()
    dev = torch.device("cuda")
    xd = torch.zeros(64, dtype=torch.float32, device=dev)
    xh = np.zeros(64, dtype=np.float32)
    rc = C.cncpd_mttkrp_last_mode_noalloc(ctypes.c_void_p(xh.ctypes.data), 2, 2, 2,
                                          ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                          2, ctypes.c_void_p(xd.data_ptr()), None)
    assert rc == -1
    assert b"device" in C.lib().cncpd_last_error()
