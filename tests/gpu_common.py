"""Helpers shared by the GPU tests: run the oracle and the CUDA path on the
same seeded inputs."""

import numpy as np
import pytest

from oracle import cncpd_oracle as O


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_2302_05119_gb300 import build
    build.build()


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def coupled_inputs(dims, R, L, seed, noise=0.1, dist="uniform"):
    """Small coupled problem from the shared generator (synthetic data)."""
    import synth
    w = synth.Workload("test", [tuple(d) for d in dims], R, list(L), 20.0 if noise else None, seed, dist=dist)
    if noise is None or noise == 0:
        w.snr_db = None
    Xs, A = synth.make_tensors(w)
    U0 = synth.init_factors(w.dims, R, seed, tag=1)
    return Xs, A, U0


def run_oracle_steps(Xs, R, L, U0, iters, nonneg=None, use_core=False, lam0=None, reupdate=True):
    """Oracle factors after each iteration (list of U[k][n]) and redo flags."""
    prob = O.Problem(Xs, R, L, nonneg)
    snaps = []
    res = O.apg(prob, U0, lam0, use_core=use_core, max_it=iters, eps=0.0, reupdate=reupdate,
                callback=lambda it, st, info: snaps.append(([[A.copy() for A in Uk] for Uk in st.U1],
                                                            [l.copy() for l in st.lam1])))
    return snaps, res
