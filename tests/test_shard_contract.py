"""The block-sharding contract on CPU (gloo, world size 2).

The blocks are split over ranks by paper_2302_05119_gb300.shard; each rank
forms the per-block terms of its own blocks (taken from the FP64 oracle,
which acts as the checker here), adds them in block order, and an
all-reduce completes the two sums the shared columns need per mode, sum_k
G_hat_C^(n,k) and sum_k L_u^(n,k) (Eq. solUnC), and the objective's
sum_k F_k.  One extrapolated sweep done that way must give every block the
factors of the single-process oracle sweep, and the same F.  This checks the
partition and the reduction, not a GPU: the library runs on one GPU here
(unmeasured on multi-GPU hardware)."""

import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from paper_2302_05119_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_block_once_and_balances():
    import synth
    eeg = synth.workload("eeg_uneven_4th").dims
    for dims in (eeg, [(8, 8, 8)] * 5, [(4, 5, 6), (40, 5, 6)], [(3, 3, 3)]):
        cost = shard.block_costs(dims)
        for ws in (1, 2, 3, 8):
            parts = shard.partition_blocks(dims, ws)
            assert len(parts) == ws
            owner = shard.owner_of(parts)
            assert sorted(owner) == list(range(len(dims)))
            for blocks in parts:
                assert blocks == sorted(blocks)
            loads = [sum(cost[k] for k in b) for b in parts]
            # longest-first greedy: the heaviest rank exceeds the lightest by
            # at most one block
            assert max(loads) - min(loads) <= max(cost)
    with pytest.raises(ValueError):
        shard.owner_of([[0, 1], [1]])


def _problem():
    sys.path.insert(0, ROOT)
    from tests.gpu_common import coupled_inputs
    dims = [(9, 8, 7), (9, 8, 5), (9, 8, 11), (9, 8, 6), (9, 8, 9)]
    L = [2, 1, 0]
    Xs, _, U0 = coupled_inputs(dims, 3, L, seed=41)
    rng = np.random.default_rng(42)
    U2 = [[A * (0.8 + 0.4 * rng.random(A.shape)) for A in Uk] for Uk in U0]
    for n, Ln in enumerate(L):  # the shared columns agree across blocks
        for k in range(1, len(dims) if Ln else 1):
            U0[k][n][:, :Ln] = U0[0][n][:, :Ln]
            U2[k][n][:, :Ln] = U2[0][n][:, :Ln]
    Lprev = {}
    for n in range(3):
        for k in range(len(dims)):
            Lprev[("u", n, k)] = 0.5 + 0.1 * k + 0.05 * n
        Lprev[("c", n)] = 2.0 + n
    return Xs, U0, U2, L, Lprev


def _sharded_sweep(rank, ws, Xs, U1, U2, L, Lprev, w_hat, delta_w, allreduce):
    """One sweep over this rank's blocks; the shared columns from the
    all-reduced block sums."""
    from oracle import cncpd_oracle as O
    K, N = len(Xs), 3
    mine = shard.partition_blocks([X.shape for X in Xs], ws)[rank]
    U1 = {k: [A.copy() for A in U1[k]] for k in mine}
    U2 = {k: [A.copy() for A in U2[k]] for k in mine}
    for n in range(N):
        Ln = L[n]
        H, M, Lu = {}, {}, {}
        for k in mine:
            H[k] = O.hadamard_except([O.gram(A) for A in U1[k]], n)
            M[k] = O.mttkrp(Xs[k], U1[k], n)
            Lu[k] = O.spectral_norm(H[k])
        LC = float(allreduce(np.array([sum(Lu[k] for k in sorted(mine))]))[0])
        wC = O.extrapolation_weight(w_hat, Lprev.get(("c", n)), LC, delta_w)
        Uhat, G = {}, {}
        for k in mine:
            w = O.extrapolation_weight(w_hat, Lprev.get(("u", n, k)), Lu[k], delta_w)
            Uhat[k] = U1[k][n] + w * (U1[k][n] - U2[k][n])
            if Ln:
                Uhat[k][:, :Ln] = U1[k][n][:, :Ln] + wC * (U1[k][n][:, :Ln] - U2[k][n][:, :Ln])
            G[k] = Uhat[k] @ H[k] - M[k]
        I = Xs[0].shape[n]
        GC = allreduce(shard.local_sum({k: G[k][:, :Ln] for k in mine}, mine)
                       if mine else np.zeros((I, Ln))) if Ln else None
        for k in mine:
            new = U1[k][n].copy()
            new[:, Ln:] = O.project(Uhat[k][:, Ln:] - G[k][:, Ln:] / Lu[k], True)
            if Ln:
                new[:, :Ln] = O.project(Uhat[k][:, :Ln] - GC / LC, True)
            U2[k][n] = U1[k][n]
            U1[k][n] = new
    Fk = {k: O.objective([Xs[k]], [U1[k]], [np.ones(3)]) for k in mine}
    F = float(allreduce(np.array([sum(Fk[k] for k in sorted(mine))]))[0])
    return {k: U1[k] for k in mine}, F


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    Xs, U1, U2, L, Lprev = _problem()
    U, F = _sharded_sweep(rank, ws, Xs, U1, U2, L, Lprev, 0.6, 0.9999, allreduce)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, {k: [A.tolist() for A in v] for k, v in U.items()}, F))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_sweep_matches_single_rank_gloo():
    pytest.importorskip("torch")
    from oracle import cncpd_oracle as O
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Xs, U1, U2, L, Lprev = _problem()
    prob = O.Problem(Xs, [3] * len(Xs), L)
    st = O.State([[A.copy() for A in Uk] for Uk in U1], [[A.copy() for A in Uk] for Uk in U2],
                 [np.ones(3)] * len(Xs), [np.ones(3)] * len(Xs))
    ref, _ = O.sweep(prob, st, 0.6, Lprev, False, 0.9999)
    F_ref = O.objective(Xs, ref.U1, ref.lam1)
    seen = set()
    for rank, U, F in out:
        assert F == pytest.approx(F_ref, rel=1e-12)
        for k, Uk in U.items():
            seen.add(int(k))
            for n in range(3):
                np.testing.assert_allclose(np.array(Uk[n]), ref.U1[int(k)][n], rtol=1e-12, atol=1e-14)
    assert seen == set(range(len(Xs)))
