"""The seeded synthetic inputs have the structure the workload table states:
shared columns equal across blocks, the sparse mode's support, per-block
ranks in range, the noise level of the stated SNR, the value distributions,
and determinism (the oracle, the GPU tests and the bench draw the same
inputs).  CPU only, on scaled-down copies of the workloads."""

import numpy as np
import pytest

import synth


def _small(name, **kw):
    w = synth.workload(name)
    d = dict(name=w.name + "_small", dims=[tuple(max(2, s // 8) for s in dd) for dd in w.dims], R=w.R, L=w.L,
             snr_db=w.snr_db, seed=w.seed, dist=w.dist, sparse_mode=w.sparse_mode, density=w.density,
             R_lra=w.R_lra)
    d.update(kw)
    return synth.Workload(d.pop("name"), d.pop("dims"), d.pop("R"), d.pop("L"), d.pop("snr_db"), d.pop("seed"), **d)


def test_every_workload_is_defined_and_seeded_apart():
    seeds = []
    for name in synth.WORKLOADS:
        w = synth.workload(name)
        assert w.K == len(w.dims) and len(w.L) == w.N
        for n, Ln in enumerate(w.L):
            assert 0 <= Ln <= min(w.ranks())
            if Ln:
                assert len({d[n] for d in w.dims}) == 1, (name, n)  # coupled modes share I_n
        seeds.append(w.seed)
    assert len(set(seeds)) == len(seeds)  # every workload draws its own inputs


@pytest.mark.parametrize("name", ["sim_256cube", "bf16_512x512x256", "eeg_uneven_4th", "erp_42x9x71x60"])
def test_shared_columns_equal_across_blocks(name):
    w = _small(name)
    A = synth.ground_truth(w.dims, w.R, w.L, w.seed, w.dist, w.sparse_mode, w.density)
    for n, Ln in enumerate(w.L):
        for k in range(1, w.K):
            if Ln:
                assert np.array_equal(A[k][n][:, :Ln], A[0][n][:, :Ln])
            if Ln < w.R and A[k][n].shape == A[0][n].shape:  # individual columns are drawn per block
                assert not np.array_equal(A[k][n][:, Ln:], A[0][n][:, Ln:])


def test_sparse_mode_support():
    """Face shape: each column of mode 0 has round(density * I) nonzeros;
    the shared columns share their support, the individual ones do not."""
    w = synth.workload("face_lra_400x400x160")
    A = synth.ground_truth(w.dims, w.R, w.L, w.seed, w.dist, w.sparse_mode, w.density)
    I = w.dims[0][0]
    nnz = int(round(w.density * I))
    for k in range(w.K):
        U = A[k][0]
        assert np.all((U != 0).sum(axis=0) == nnz), k
        assert np.all(U >= 0) and np.all(U < 1)
        for n in (1, 2):
            assert np.all(A[k][n] > 0)  # dense U[0,1] in the other modes (zero with probability 0)
    for r in range(w.L[0]):
        assert np.array_equal(A[1][0][:, r] != 0, A[0][0][:, r] != 0)
    diff = [not np.array_equal(A[1][0][:, r] != 0, A[0][0][:, r] != 0) for r in range(w.L[0], w.R)]
    assert any(diff)


def test_per_block_ranks_of_the_ongoing_eeg_shape():
    w = synth.workload("eeg_ongoing_14x46x510x64")
    R = w.ranks()
    assert len(R) == 14 and all(33 <= r <= 44 for r in R) and len(set(R)) > 1
    A = synth.ground_truth(w.dims, w.R, w.L, w.seed)
    assert all(A[k][n].shape == (w.dims[k][n], R[k]) for k in range(w.K) for n in range(w.N))


@pytest.mark.parametrize("name,dist", [("small_40cube", "uniform"), ("eeg_uneven_4th", "gamma")])
def test_factor_distributions(name, dist):
    w = _small(name) if name != "small_40cube" else synth.workload(name)
    assert w.dist == dist
    A = synth.ground_truth(w.dims, w.R, w.L, w.seed, w.dist)
    v = np.concatenate([M.ravel() for Ak in A for M in Ak])
    if dist == "uniform":
        assert v.min() >= 0 and v.max() < 1 and abs(v.mean() - 0.5) < 0.02
    else:  # Gamma(2, 1): mean 2, variance 2
        assert v.min() > 0 and abs(v.mean() - 2) < 0.15 and abs(v.var() - 2) < 0.4


@pytest.mark.parametrize("snr", [10.0, 20.0])
def test_noise_level_matches_the_snr(snr):
    """||X - [[A]]|| / ||[[A]]|| = 10^(-SNR/20) before the clip at 0; the clip
    only removes noise, and on these positive tensors almost never acts."""
    w = _small("sim_256cube", snr_db=snr, dims=[(24, 20, 16)] * 2, L=[3, 3, 0])
    Xs, A = synth.make_tensors(w)
    for k in range(w.K):
        Y = np.einsum("ir,jr,kr->ijk", *A[k])
        ratio = np.linalg.norm(Xs[k] - Y) / np.linalg.norm(Y)
        target = 10.0 ** (-snr / 20.0)
        assert target * 0.97 <= ratio <= target * (1 + 1e-12), (ratio, target)
        assert np.all(Xs[k] >= 0)


def test_inputs_are_deterministic_and_blockwise():
    w = _small("eeg_uneven_4th")
    X1, _ = synth.make_tensors(w, dtype=np.float32)
    X2, _ = synth.make_tensors(w, dtype=np.float32)
    assert all(np.array_equal(a, b) for a, b in zip(X1, X2))
    # one block alone is the same block as in the full draw
    X3, _ = synth.make_tensors(w, dtype=np.float32, blocks=[2])
    assert np.array_equal(X3[0], X1[2])
    U1 = synth.init_factors(w.dims, w.R, w.seed)
    U2 = synth.init_factors(w.dims, w.R, w.seed)
    assert all(np.array_equal(a, b) for Ua, Ub in zip(U1, U2) for a, b in zip(Ua, Ub))
    assert not np.array_equal(U1[0][0], U1[1][0])
