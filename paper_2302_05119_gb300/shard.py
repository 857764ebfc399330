"""Host-side plan for sharding the K coupled blocks over ranks.

The blocks of CoNCPD-APG are independent except through the shared first
L_n columns of each mode (Eq. solUnC): their update needs, per mode n, the
block sums sum_k G_hat_C^(n,k) (I_n x L_n) and sum_k L_u^(n,k), and the
objective needs sum_k F_k.  A rank that owns a subset of the blocks forms
those per-block terms for its blocks, adds them in block order, and an
all-reduce (sum) over ranks completes each sum; every rank then applies the
same shared-column step.

This module holds the partition and the fixed order of that reduction; it
has no arithmetic of the method.  This build runs on one GPU, so the
library itself runs every block in one process (no collective on the data
path).
"""

import numpy as np


def block_costs(dims):
    """Work of each block: its number of tensor elements (prod_n I_n), the
    bytes every tensor pass streams."""
    return [int(np.prod(d)) for d in dims]


def partition_blocks(dims, world_size):
    """Assign the K blocks to `world_size` ranks, balanced by prod_n I_n.

    Longest first, each block to the rank with the least work so far (ties:
    lowest rank); each rank's blocks are returned in increasing block order,
    which is the order its local sums are formed in.  Every block is owned by
    exactly one rank; a rank may own none when K < world_size.
    """
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cost = block_costs(dims)
    order = sorted(range(len(cost)), key=lambda k: (-cost[k], k))
    load = [0] * world_size
    owned = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        owned[r].append(k)
        load[r] += cost[k]
    return [sorted(b) for b in owned]


def owner_of(parts):
    """Block -> rank map of a partition."""
    out = {}
    for r, blocks in enumerate(parts):
        for k in blocks:
            if k in out:
                raise ValueError(f"block {k} owned twice")
            out[k] = r
    return out


def local_sum(terms, blocks):
    """sum over this rank's blocks (increasing block order) of terms[k]; the
    all-reduce of these partial sums over ranks gives the sum over all
    blocks."""
    acc = None
    for k in sorted(blocks):
        t = np.asarray(terms[k], dtype=np.float64)
        acc = t.copy() if acc is None else acc + t
    return acc
