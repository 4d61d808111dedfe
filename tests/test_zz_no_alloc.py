"""sw_search_no_alloc gives sw_search's scores without allocating.

The entry point exists for callers of this library that cannot allocate
device memory when they search: code running while a CUDA stream is being
captured into a graph, serving loops that must not touch the allocator after
start-up, and processes whose device memory belongs to another framework's
pool.  Its scratch is a fixed device array the library owns, shared by all
calls and keeping the previous call's contents, so this test makes two calls
in a row (the first one leaves saturated sequences in the shared overflow
list) and checks each against sw_search and against the CPU oracle, exactly
(scores are integers).

This file is named to be collected last, so that a run that stops at its
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _database(rng):
    W = synth.ALPHABET.index("W")
    seqs = [synth.random_residues(rng, int(n)) for n in rng.integers(1, 400, 300)]
    seqs[7] = np.full(3100, W, dtype=np.uint8)          # saturates int16 against a W query
    seqs[100] = np.concatenate([synth.random_residues(rng, 500), np.full(3000, W, np.uint8)])
    return synth.seqset_from_list(seqs)


def _reference_scores(gpu, handle, q, S, o, e, n):
    scores = np.empty((1, n), dtype=np.int32)
    gpu.sw_search(handle, q, np.array([0, len(q)], np.int64), S, o, e, 0, scores_out=scores)
    return scores[0]


def test_no_alloc_matches_sw_search_twice(gpu):
    import torch
    rng = np.random.default_rng(31)
    db = _database(rng)
    S = synth.blosum62()
    W = synth.ALPHABET.index("W")
    queries = [np.full(3100, W, dtype=np.uint8),            # multi-pass, saturating pairs
               synth.random_residues(rng, 97)]               # single pass
    with gpu.Database(db.residues, db.offsets, 24) as d:
        wants = [_reference_scores(gpu, d.handle, q, S, 10, 1, db.n) for q in queries]
        q_dev = [torch.from_numpy(q).cuda() for q in queries]
        out = [torch.full((db.n,), -7, dtype=torch.int32, device="cuda") for _ in queries]
        torch.cuda.synchronize()
        # first call: sets up the scratch address for this device
        gpu.sw_search_no_alloc(d.handle, q_dev[0], S, 10, 1, out[0])
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        gpu.sw_search_no_alloc(d.handle, q_dev[1], S, 10, 1, out[1])
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        np.testing.assert_array_equal(out[0].cpu().numpy(), wants[0])
        np.testing.assert_array_equal(out[1].cpu().numpy(), wants[1])
        assert free_after == free_before
        assert (wants[0] > 32767 - 11).sum() >= 2                  # saturation was exercised
    exact = oracle.all_scores(synth.seqset_from_list(queries), db, S, 10, 1)
    np.testing.assert_array_equal(out[0].cpu().numpy().astype(np.int64), exact[0])
    np.testing.assert_array_equal(out[1].cpu().numpy().astype(np.int64), exact[1])


def test_no_alloc_rejects_oversized_scratch(gpu):
    import torch
    rng = np.random.default_rng(32)
    big = synth.seqset_from_lengths(rng, np.full(9000, 1000))     # ~9 MB layout: 4x exceeds 32 MiB
    S = synth.blosum62()
    with gpu.Database(big.residues, big.offsets, 24) as d:
        q = torch.from_numpy(synth.random_residues(rng, 300)).cuda()
        out = torch.empty((big.n,), dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.SwError) as e:
            gpu.sw_search_no_alloc(d.handle, q, S, 10, 1, out)
        assert e.value.code == 1 and "scratch" in str(e.value)
        # a single-pass query needs no boundary rows and fits
        q1 = torch.from_numpy(synth.random_residues(rng, 100)).cuda()
        gpu.sw_search_no_alloc(d.handle, q1, S, 10, 1, out)
        torch.cuda.synchronize()
        want = _reference_scores(gpu, d.handle, q1.cpu().numpy(), S, 10, 1, big.n)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
