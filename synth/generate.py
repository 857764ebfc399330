"""Seeded generators for coupled nonnegative tensors (see package docstring).

Every draw uses numpy's counter-based Philox bit generator keyed by
(seed, purpose, block), so a block's data does not depend on how many other
blocks are drawn.
"""

from dataclasses import dataclass, field

import numpy as np

_PURPOSE = {"sizes": 1, "common": 2, "indiv": 3, "noise": 4, "init": 5,
            "core": 6, "lra": 7, "support": 8}


def _rng(seed, purpose, *extra):
    key = [int(seed) & 0xFFFFFFFF, _PURPOSE[purpose]] + [int(e) & 0xFFFFFFFF for e in extra]
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(key)))


@dataclass
class Workload:
    """One synthetic coupled-tensor problem.

    dims: per-block tensor sizes (K tuples of N ints), R: rank (one int, or
    K ints for per-block ranks), L: coupled columns per mode, snr_db: noise level, dist: factor distribution
    ("uniform" or "gamma"), sparse_mode: mode whose ground-truth columns are
    sparse (fraction ``density`` nonzero) or None, iters: iteration count
    the workload is run for, R_lra: LRA rank (0: no LRA step).
    """
    name: str
    dims: list
    R: int
    L: list
    snr_db: float
    seed: int
    dist: str = "uniform"
    sparse_mode: int = None
    density: float = 1.0
    iters: int = 200
    R_lra: int = 0
    nonneg: list = field(default=None)

    @property
    def K(self):
        return len(self.dims)

    @property
    def N(self):
        return len(self.dims[0])

    def elements(self):
        return [int(np.prod(d)) for d in self.dims]

    def ranks(self):
        """Per-block ranks R_k."""
        return [int(r) for r in self.R] if np.ndim(self.R) else [int(self.R)] * self.K


def _eeg_dims(seed, K):
    rng = _rng(seed, "sizes")
    i3 = rng.integers(40, 161, size=K)
    i4 = rng.integers(20, 121, size=K)
    return [(64, 71, int(a), int(b)) for a, b in zip(i3, i4)]


def _ongoing_ranks(seed, K):
    return [int(r) for r in _rng(seed, "sizes", 1).integers(33, 45, size=K)]


# Coupling patterns of the simulation design (Section IV-A, Table III) at
# R = 10: L = [10,10,10], [5,5,5] (all modes coupled), [10,10,0], [5,5,0]
# (two), [10,0,0], [5,0,0] (one).
E1_PATTERNS = {"e1a_l10": [10, 10, 10], "e1a_l5": [5, 5, 5], "e1b_l10": [10, 10, 0],
               "e1b_l5": [5, 5, 0], "e1c_l10": [10, 0, 0], "e1c_l5": [5, 0, 0]}


def workload(name):
    """The named synthetic workloads (shapes and distributions of the paper's
    simulation, face-image and EEG experiments; seeds fixed)."""
    base = 20230210
    if name.startswith("e1") and name.split("_s")[0] in E1_PATTERNS:
        # simulation design: S = 20 blocks of 100^3, R = 10, 20 dB; "_s<K>"
        # takes the first K blocks only (the same data as the full design)
        pat = name.split("_s")[0]
        K = int(name.split("_s")[1]) if "_s" in name else 20
        return Workload(name, [(100, 100, 100)] * K, 10, list(E1_PATTERNS[pat]), 20.0,
                        base + 10 + sorted(E1_PATTERNS).index(pat), iters=1000)
    if name == "face_lra_400x400x160":
        # the face shape scaled down (each mode by 2.5) so that the FP64 oracle
        # can be run to convergence for its time-to-fit target
        return Workload(name, [(400, 400, 160)] * 8, 20, [8, 0, 0], 20.0, base + 8,
                        sparse_mode=0, density=0.1, iters=200, R_lra=30)
    if name == "erp_42x9x71x60":
        # ERP shape (Section IV-C): 42 blocks of 9 channels x 71 frequency
        # bins x 60 time points, R = 36, every column shared in every mode
        # (the blocks differ only by their cores)
        return Workload(name, [(9, 71, 60)] * 42, 36, [36, 36, 36], 15.0, base + 6, iters=200)
    if name == "eeg_ongoing_14x46x510x64":
        # ongoing-EEG shape (Section IV-D): 14 blocks of 46 x 510 x 64,
        # per-block ranks in [33, 44], L = [26, 26, 0]
        return Workload(name, [(46, 510, 64)] * 14, _ongoing_ranks(base + 7, 14), [26, 26, 0], 15.0,
                        base + 7, iters=200)
    if name == "small_40cube":
        return Workload(name, [(40, 40, 40)] * 3, 5, [2, 0, 0], 20.0, base + 1, iters=200)
    if name == "sim_256cube":
        return Workload(name, [(256, 256, 256)] * 5, 10, [3, 3, 0], 10.0, base + 2, iters=500)
    if name == "bf16_512x512x256":
        return Workload(name, [(512, 512, 256)] * 4, 20, [5, 0, 0], 20.0, base + 3, iters=200)
    if name == "eeg_uneven_4th":
        return Workload(name, _eeg_dims(base + 4, 16), 12, [4, 4, 0, 0], 15.0, base + 4,
                        dist="gamma", iters=200)
    if name == "face_lra_1000x1000x400":
        return Workload(name, [(1000, 1000, 400)] * 8, 20, [8, 0, 0], 20.0, base + 5,
                        sparse_mode=0, density=0.1, iters=200, R_lra=30)
    raise KeyError(name)


WORKLOADS = ["small_40cube", "sim_256cube", "bf16_512x512x256", "eeg_uneven_4th",
             "face_lra_1000x1000x400", "face_lra_400x400x160", "erp_42x9x71x60", "eeg_ongoing_14x46x510x64"] + sorted(E1_PATTERNS)


def _draw(rng, shape, dist):
    if dist == "uniform":
        return rng.random(shape)
    if dist == "gamma":
        return rng.gamma(2.0, 1.0, size=shape)
    raise ValueError(dist)


def ground_truth(dims, R, L, seed, dist="uniform", sparse_mode=None, density=1.0):
    """Ground-truth factors A[k][n] (I_n x R_k): the first L[n] columns of
    mode n are drawn once and shared by every block; the rest per block.
    R is one rank or K per-block ranks."""
    K, N = len(dims), len(dims[0])
    Rs = [int(r) for r in R] if np.ndim(R) else [int(R)] * K
    common = []
    for n in range(N):
        if L[n] > 0:
            common.append(_draw(_rng(seed, "common", n), (dims[0][n], L[n]), dist))
        else:
            common.append(None)
    A = []
    for k in range(K):
        Ak = []
        for n in range(N):
            I = dims[k][n]
            M = _draw(_rng(seed, "indiv", k, n), (I, Rs[k]), dist)
            if L[n] > 0:
                M[:, :L[n]] = common[n]
            if sparse_mode is not None and n == sparse_mode and density < 1.0:
                keep = np.zeros((I, Rs[k]), dtype=bool)
                nnz = max(1, int(round(density * I)))
                for r in range(Rs[k]):
                    src = ("support", 0, r) if r < L[n] else ("support", k + 1, r)
                    rows = _rng(seed, *src).choice(I, size=nnz, replace=False)
                    keep[rows, r] = True
                M = np.where(keep, M, 0.0)
            Ak.append(M)
        A.append(Ak)
    return A


def _outer_sum(Ak):
    """sum_r a_r^(1) o ... o a_r^(N) (data synthesis only)."""
    N = len(Ak)
    letters = "abcdefgh"[:N]
    spec = ",".join(f"{c}z" for c in letters) + "->" + letters
    return np.einsum(spec, *Ak, optimize=True)


def make_tensors(w, dtype=np.float64, blocks=None):
    """Noisy nonnegative tensors of workload ``w`` (list of K arrays in
    C order, ``dtype``), plus the ground-truth factors."""
    A = ground_truth(w.dims, w.R, w.L, w.seed, w.dist, w.sparse_mode, w.density)
    Xs = []
    for k in (range(w.K) if blocks is None else blocks):
        Y = _outer_sum(A[k])
        if w.snr_db is not None and np.isfinite(w.snr_db):
            E = _rng(w.seed, "noise", k).standard_normal(Y.shape)
            Y = Y + (10.0 ** (-w.snr_db / 20.0)) * np.linalg.norm(Y) * E / np.linalg.norm(E)
            np.maximum(Y, 0.0, out=Y)
        Xs.append(np.ascontiguousarray(Y, dtype=dtype))
    return Xs, A


def _ranks(R, K):
    return [int(r) for r in R] if np.ndim(R) else [int(R)] * K


def init_factors(dims, R, seed, tag=0):
    """Initial factors U0[k][n] ~ Uniform[0, 1] (Section IV settings); R is
    one rank or per-block ranks."""
    Rs = _ranks(R, len(dims))
    return [[_rng(seed, "init", tag, k, n).random((d[n], Rs[k])) for n in range(len(d))]
            for k, d in enumerate(dims)]


def init_cores(K, R, seed, tag=0):
    """Initial super-diagonal cores lambda^(k) ~ Uniform[0, 1]."""
    Rs = _ranks(R, K)
    return [_rng(seed, "core", tag, k).random(Rs[k]) for k in range(K)]


def init_lra_factors(dims, R_lra, seed, tag=0):
    """Initial ALS factors for the low-rank approximation ~ Uniform[0, 1]."""
    return [[_rng(seed, "lra", tag, k, n).random((d[n], R_lra)) for n in range(len(d))]
            for k, d in enumerate(dims)]
