"""Database sharding on the host (CPU only): the partition, the top-k merge
and the exchange step between ranks (two gloo processes).

The merge must give exactly the unsharded top-k, ties included (score
descending, then database index ascending): each shard's list is what
sw_search returns for that shard alone, i.e. oracle.top_k of the shard's
own score row, and the expected result is oracle.top_k of the whole row.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2203_11100_gb300 import binding, multigpu


def _shard_top_k(row, members, moff, k):
    """What each shard's own search returns: the top-k of its local row."""
    out = np.empty((len(moff) - 1, k), dtype=binding.HIT_DTYPE)
    for s in range(len(moff) - 1):
        sc, ix = oracle.top_k(row[members[moff[s]:moff[s + 1]]], k)
        out[s]["score"] = sc
        out[s]["reserved"] = 0
        out[s]["db_index"] = ix
    return out


@pytest.mark.parametrize("n_shards", [1, 2, 3, 8])
def test_shard_plan_partitions_and_balances(n_shards):
    rng = np.random.default_rng(3)
    lens = synth.lognormal_lengths(rng, 5000, 360.0, 2, 35_000)
    lens[17] = 35_000
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    members, moff = binding.sw_shard_plan(off, n_shards)
    assert moff[0] == 0 and moff[-1] == len(lens) and len(moff) == n_shards + 1
    assert np.array_equal(np.sort(members), np.arange(len(lens)))          # a partition
    res = []
    for s in range(n_shards):
        m = members[moff[s]:moff[s + 1]]
        assert np.all(np.diff(m) > 0)                                         # caller's order
        res.append(int(lens[m].sum()))
    assert max(res) - min(res) <= lens.max()                                 # residue balance
    # length strata: the n_shards longest sequences land on distinct shards
    shard_of = np.empty(len(lens), np.int64)
    for s in range(n_shards):
        shard_of[members[moff[s]:moff[s + 1]]] = s
    longest = np.argsort(-lens, kind="stable")[:n_shards]
    assert len(set(shard_of[longest].tolist())) == n_shards


def test_shard_plan_more_shards_than_sequences():
    off = np.array([0, 5, 5, 9], np.int64)                   # one empty sequence
    members, moff = binding.sw_shard_plan(off, 5)
    assert np.array_equal(np.sort(members), [0, 1, 2]) and moff[-1] == 3
    assert sum(1 for s in range(5) if moff[s + 1] == moff[s]) == 2          # two empty shards


def test_shard_plan_rejects_bad_arguments():
    with pytest.raises(binding.SwError):
        binding.sw_shard_plan(np.array([0, 3], np.int64), 0)
    with pytest.raises(binding.SwError):
        binding.sw_shard_plan(np.array([0, 3, 2], np.int64), 2)


@pytest.mark.parametrize("n_shards,k", [(2, 10), (3, 5), (5, 40), (4, 1)])
def test_merge_equals_unsharded_top_k_with_ties(n_shards, k):
    rng = np.random.default_rng(n_shards * 100 + k)
    n = 300
    off = np.zeros(n + 1, np.int64)
    np.cumsum(rng.integers(1, 50, n), out=off[1:])
    members, moff = binding.sw_shard_plan(off, n_shards)
    for trial in range(20):
        rows = rng.integers(0, 6 if trial % 2 else 1000, size=(3, n))       # many ties half the time
        rows[1, :] = 7                                                          # all equal
        shard_hits = np.stack([_shard_top_k(r, members, moff, k) for r in rows], axis=1)
        merged = binding.sw_hits_merge(shard_hits, members, moff, k)
        for q, r in enumerate(rows):
            s_, i_ = oracle.top_k(r, k)
            np.testing.assert_array_equal(merged[q]["score"], s_)
            np.testing.assert_array_equal(merged[q]["db_index"], i_)


def test_merge_pads_when_k_exceeds_the_database():
    off = np.array([0, 3, 6, 9], np.int64)
    members, moff = binding.sw_shard_plan(off, 2)
    row = np.array([5, 9, 5])
    merged = binding.sw_hits_merge(_shard_top_k(row, members, moff, 6)[:, None], members, moff, 6)[0]
    assert merged["score"].tolist() == [9, 5, 5, -1, -1, -1]
    assert merged["db_index"].tolist() == [1, 0, 2, -1, -1, -1]


def test_merge_rejects_an_index_outside_its_shard():
    off = np.array([0, 3, 6, 9, 12], np.int64)
    members, moff = binding.sw_shard_plan(off, 2)
    bad = _shard_top_k(np.arange(4), members, moff, 2)[:, None]
    bad[1, 0, 0]["db_index"] = 2                     # shard 1 holds 2 sequences
    with pytest.raises(binding.SwError):
        binding.sw_hits_merge(bad, members, moff, 2)


def test_scores_scatter_rebuilds_the_table():
    rng = np.random.default_rng(9)
    off = np.zeros(41, np.int64)
    np.cumsum(rng.integers(1, 30, 40), out=off[1:])
    members, moff = binding.sw_shard_plan(off, 3)
    full = rng.integers(-50, 50, size=(4, 40)).astype(np.int32)
    out = np.full_like(full, 12345)
    for s in range(3):
        m = members[moff[s]:moff[s + 1]]
        binding.sw_scores_scatter(np.ascontiguousarray(full[:, m]), m, out)
    np.testing.assert_array_equal(out, full)
    with pytest.raises(binding.SwError):
        binding.sw_scores_scatter(full[:, :1].copy(), np.array([40], np.int64), out)


# ---------------------------------------------------------------------------
# the exchange step between ranks: two gloo processes, one shard each

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_db():
    """A small database in which many sequences repeat, so equal scores fall
    on both shards."""
    rng = np.random.default_rng(77)
    base = [synth.random_residues(rng, int(n)) for n in rng.integers(5, 120, 40)]
    seqs = [base[int(i)] for i in rng.integers(0, 40, 160)]
    return synth.seqset_from_list(seqs), synth.seqset_from_lengths(rng, [60, 90, 15])


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo")
    db, qs = _sharded_db()
    S = synth.blosum62()
    k = 10
    members, moff = binding.sw_shard_plan(db.offsets, world)
    mine = members[moff[rank]:moff[rank + 1]]
    # this rank's shard searched alone (the oracle stands in for the GPU here)
    shard = synth.seqset_from_list([db.seq(int(i)) for i in mine])
    rows = oracle.all_scores(qs, shard, S, 10, 1)
    local = np.empty((qs.n, k), dtype=binding.HIT_DTYPE)
    for q in range(qs.n):
        local[q]["score"], local[q]["db_index"] = oracle.top_k(rows[q], k)
        local[q]["reserved"] = 0
    merged = multigpu.exchange_hits(dist, multigpu.hits_to_tensor(local), members, moff, k)
    out[rank] = (merged["score"].tolist(), merged["db_index"].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_exchange_and_merge():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    db, qs = _sharded_db()
    full = oracle.all_scores(qs, db, synth.blosum62(), 10, 1)
    ties = 0
    for q in range(qs.n):
        s_, i_ = oracle.top_k(full[q], 10)
        ties += int(len(np.unique(s_)) < len(s_))
        for r in range(world):
            assert out[r][0][q] == s_.tolist() and out[r][1][q] == i_.tolist()
    assert ties >= 1                                  # equal scores were ordered across shards
