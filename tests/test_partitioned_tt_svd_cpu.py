"""The partitioned TT-SVD on CPU ranks (gloo, world size 2): the split a
multi-GPU run of one large array would use, checked against the oracle's
TT-SVD (Alg. 1 with the cap of Sec. 5 (1)).

Each rank holds a contiguous block of samples, i.e. a block of columns of
every unfolding (the column index of the k-th unfolding is made of the high
bits).  Per level: local partial Gram W W^H, one all-reduce (sum) of the
m_k x m_k Gram, the same Hermitian eigen-decomposition on every rank (the
left singular vectors and the rank decision, replicated), the local
projection U_r^H W and its local reshape to the next unfolding.  When a
rank is left with one column per level, the small remainder is gathered.
Only the Gram (<= 2 R_max squared) crosses ranks: no sample moves.
"""
import os
import socket

import numpy as np
import pytest

from oracle import qtt as Q


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _partitioned_tt_svd(v_local, d, rmax, rank, world):
    import torch
    import torch.distributed as dist
    cores = []
    r_prev = 1
    W = v_local.reshape((2, -1), order="F")               # local columns of the first unfolding
    split = True                                          # columns still spread over the ranks
    for k in range(1, d):
        if split and W.shape[1] == 1:
            # one column left per rank: gather the small unfolding, go on alike
            parts = [torch.zeros(W.shape[0], dtype=torch.complex128) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(W[:, 0].copy()))
            W = np.stack([p.numpy() for p in parts], axis=1)
            split = False
        G = torch.from_numpy(W @ W.conj().T)
        if split:
            dist.all_reduce(G)
        _, U = np.linalg.eigh(G.numpy())
        U = U[:, ::-1]
        m = W.shape[0]
        r = max(1, min(rmax, m, W.shape[1] * (world if split else 1)))
        cores.append(U[:, :r].reshape((r_prev, 2, r), order="F"))
        P = U[:, :r].conj().T @ W                           # r x (local) columns
        W = P.reshape((2 * r, -1), order="F")
        r_prev = r
    if split:
        parts = [torch.zeros(W.shape[0], dtype=torch.complex128) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(W[:, 0].copy()))
        W = np.stack([p.numpy() for p in parts], axis=1)
    cores.append(W.reshape((r_prev, 2, 1), order="F"))
    return cores


def _rank_main(rank, world, port, d, rmax, v, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = v.size // world
    cores = _partitioned_tt_svd(v[rank * n:(rank + 1) * n].astype(np.complex128), d, rmax, rank, world)
    out[rank] = [c.copy() for c in cores]
    dist.barrier()
    dist.destroy_process_group()


def _run(d, rmax, v, world=2):
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank_main, args=(world, port, d, rmax, v, out), nprocs=world, join=True)
    return [out[r] for r in range(world)]


def _low_rank_line(rng, d, r):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    cores = [rng.standard_normal((ranks[k], 2, ranks[k + 1])) + 1j * rng.standard_normal((ranks[k], 2, ranks[k + 1]))
             for k in range(d)]
    return Q.full(cores)


def test_partitioned_equals_oracle_on_low_rank_data():
    rng = np.random.default_rng(17)
    d, rmax = 12, 8
    v = _low_rank_line(rng, d, 5)
    per_rank = _run(d, rmax, v)
    ref, _, _ = Q.tt_svd(v, d, 0.0, rmax)
    for cores in per_rank:
        assert [c.shape[2] for c in cores[:-1]] == [c.shape[2] for c in ref[:-1]]
        assert np.linalg.norm(Q.full(cores) - v) <= 1e-9 * np.linalg.norm(v)
    # the ranks hold the same cores (replicated decisions)
    for a, b in zip(per_rank[0], per_rank[1]):
        assert np.array_equal(a, b)


def test_partitioned_truncation_error_matches_oracle():
    """On noisy data the cap truncates: the partitioned decomposition's error
    equals the oracle's (the same subspaces, up to the Gram's rounding)."""
    rng = np.random.default_rng(18)
    d, rmax = 12, 6
    v = _low_rank_line(rng, d, 4)
    v = v + 0.05 * np.linalg.norm(v) / np.sqrt(v.size) * rng.standard_normal(v.size)
    cores = _run(d, rmax, v)[0]
    ref, _, _ = Q.tt_svd(v, d, 0.0, rmax)
    e_p = np.linalg.norm(Q.full(cores) - v)
    e_o = np.linalg.norm(Q.full(ref) - v)
    assert abs(e_p - e_o) <= 1e-6 * e_o
    assert np.linalg.norm(Q.full(cores) - Q.full(ref)) <= 1e-6 * np.linalg.norm(v)
