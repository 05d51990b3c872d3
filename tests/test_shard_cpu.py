"""Sharding of a screened quartet list over ranks (CPU, gloo, world size 2):
the cost-balanced partition covers every quartet exactly once, and the
per-rank partial energies (oracle) all-reduce to the single-rank energy."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
import paper_2506_12501_gb300 as eri
from paper_2506_12501_gb300 import opcount, shard


def _quartets():
    basis = synth.molecule_basis(natom=2, radius=1.5, seed=3)
    pairs, batches = synth.all_unique_quartets(basis)
    shells, costs = [], []
    for cls, (bra, ket, q) in batches.items():
        qs = synth.quartet_shells(bra, ket, q)
        for s in qs:
            Kb = basis.shell_K[s[0]] * basis.shell_K[s[1]]
            Kk = basis.shell_K[s[2]] * basis.shell_K[s[3]]
            costs.append(opcount.sparse_flops(cls, int(Kb), int(Kk)))
        shells.append(qs)
    return basis, np.concatenate(shells), np.asarray(costs, dtype=np.float64)


def _energy(basis, shells, D):
    off = np.concatenate([[0], np.cumsum((basis.shell_l + 1) * (basis.shell_l + 2) // 2)[:-1]])
    vals = oracle.eri_quartets(basis, shells, prec="d")
    e, pos = 0.0, 0
    for a, b, c, d in shells:
        n = [(basis.shell_l[x] + 1) * (basis.shell_l[x] + 2) // 2 for x in (a, b, c, d)]
        blk = vals[pos:pos + np.prod(n)].reshape(n)
        pos += int(np.prod(n))
        Dab = D[off[a]:off[a] + n[0], off[b]:off[b] + n[1]]
        Dcd = D[off[c]:off[c] + n[2], off[d]:off[d] + n[3]]
        e += float(np.einsum("abcd,ab,cd->", blk, Dab, Dcd))
    return e


def test_partition_balanced_and_complete():
    costs = np.random.default_rng(0).lognormal(0, 2, 5000)
    parts = shard.partition(costs, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(5000))
    loads = [costs[p].sum() for p in parts]
    assert max(loads) - min(loads) <= costs.max()


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        basis, shells, costs = _quartets()
        nbf = int(((basis.shell_l + 1) * (basis.shell_l + 2) // 2).sum())
        U = np.random.default_rng(1).uniform(-1, 1, (nbf, nbf))
        D = np.triu(U) + np.triu(U, 1).T
        mine = shard.partition(costs, world)[rank]
        part = _energy(basis, shells[mine], D)
        out[rank] = (shard.allreduce_sum(part, dist), len(mine), _energy(basis, shells, D) if rank == 0 else None)
    finally:
        dist.destroy_process_group()


def test_two_rank_energy_equals_single_rank():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    total, single = out[0][0], out[0][2]
    assert out[0][0] == out[1][0]
    assert abs(total - single) <= 1e-12 * max(1.0, abs(single))
    assert out[0][1] > 0 and out[1][1] > 0


def _partial_coulomb(basis, shells, D):
    """J' over a share of the unique quartets with the plans' weighting rule
    (2s, s = 1/2 per coincident pair or pair of pairs); J = J' + J'^T."""
    n = (basis.shell_l + 1) * (basis.shell_l + 2) // 2
    off = np.concatenate([[0], np.cumsum(n)[:-1]])
    nbf = int(n.sum())
    Jp = np.zeros((nbf, nbf))
    if len(shells) == 0:
        return Jp
    vals = oracle.eri_quartets(basis, shells, prec="d")
    pos = 0
    for a, b, c, d in shells:
        na, nb, nc_, nd = n[a], n[b], n[c], n[d]
        blk = vals[pos:pos + na * nb * nc_ * nd].reshape(na, nb, nc_, nd)
        pos += na * nb * nc_ * nd
        w = 2.0 * (0.5 if a == b else 1.0) * (0.5 if c == d else 1.0) * (0.5 if {a, b} == {c, d} else 1.0)
        sa, sb, sc, sd = (slice(off[x], off[x] + n[x]) for x in (a, b, c, d))
        Jp[sa, sb] += w * np.einsum("abcd,cd->ab", blk, D[sc, sd])
        Jp[sc, sd] += w * np.einsum("abcd,ab->cd", blk, D[sa, sb])
    return Jp


def _j_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        basis, shells, costs = _quartets()
        nbf = int(((basis.shell_l + 1) * (basis.shell_l + 2) // 2).sum())
        U = np.random.default_rng(2).uniform(-1, 1, (nbf, nbf))
        D = np.triu(U) + np.triu(U, 1).T
        mine = shard.partition(costs, world)[rank]
        Jp = shard.allreduce_sum(_partial_coulomb(basis, shells[mine], D).ravel(), dist).reshape(nbf, nbf)
        out[rank] = (Jp + Jp.T, (_partial_coulomb(basis, shells, D), D) if rank == 0 else None)
    finally:
        dist.destroy_process_group()


def test_two_rank_coulomb_matrix_equals_single_rank():
    """Sharded J digestion: per-rank J' over each rank's quartets, one
    all-reduce, then J = J' + J'^T equals the single-rank J."""
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_j_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    J0, J1 = out[0][0], out[1][0]
    Jp_single, _ = out[0][1]
    J_single = Jp_single + Jp_single.T
    assert np.array_equal(J0, J1)
    assert np.abs(J0 - J_single).max() <= 1e-12 * np.abs(J_single).max()


def _plan_items(basis, chunk=8):
    """Work items shaped like a plan's: one bra pair and a run of at most
    ``chunk`` of its kets within one class, costed like eri_plan_set_slice
    (FP64 work per quartet times the item's quartet count)."""
    pairs, batches = synth.all_unique_quartets(basis)
    items, costs = [], []
    for cls, (bra, ket, q) in batches.items():
        qs = synth.quartet_shells(bra, ket, q)
        for b in np.unique(q[:, 0]):
            sel = np.where(q[:, 0] == b)[0]
            for k0 in range(0, len(sel), chunk):
                part = qs[sel[k0:k0 + chunk]]
                Kb = basis.shell_K[part[0, 0]] * basis.shell_K[part[0, 1]]
                Kk = basis.shell_K[part[:, 2]] * basis.shell_K[part[:, 3]]
                items.append(part)
                costs.append(sum(opcount.sparse_flops(cls, int(Kb), int(k)) for k in Kk))
    return items, np.asarray(costs)


def _item_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        basis = synth.molecule_basis(natom=2, radius=1.5, seed=5)
        items, costs = _plan_items(basis)
        nbf = int(((basis.shell_l + 1) * (basis.shell_l + 2) // 2).sum())
        U = np.random.default_rng(3).uniform(-1, 1, (nbf, nbf))
        D = np.triu(U) + np.triu(U, 1).T
        owner, load = eri.partition(costs, world)
        mine = [items[i] for i in np.where(owner == rank)[0]]
        part = _energy(basis, np.concatenate(mine), D) if mine else 0.0
        single = _energy(basis, np.concatenate(items), D) if rank == 0 else None
        out[rank] = (shard.allreduce_sum(part, dist), sum(len(m) for m in mine), single, load.tolist(),
                     float(costs.max()), len(items))
    finally:
        dist.destroy_process_group()


def test_two_rank_plan_items_energy_equals_single_rank():
    """The partition eri_plan_set_slice applies (the library's eri_partition,
    called on the host) over plan-shaped work items of a molecule's screened
    unique quartets: two gloo ranks digest their items with the oracle, one
    all-reduce gives the single-rank energy, every quartet is counted once,
    and the loads differ by at most the largest item cost."""
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_item_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    total, single = out[0][0], out[0][2]
    assert out[0][0] == out[1][0]
    assert abs(total - single) <= 1e-12 * max(1.0, abs(single))
    nq_total = sum(len(x) for x in _plan_items(synth.molecule_basis(natom=2, radius=1.5, seed=5))[0])
    assert out[0][1] + out[1][1] == nq_total and out[0][1] > 0 and out[1][1] > 0
    load, cmax = out[0][3], out[0][4]
    assert abs(load[0] - load[1]) <= cmax
