"""Failure detection on the GPU without a fault: the bounded wait of the
intra-task kernel gives up on a flag that nothing sets, records
SW_ERR_TIMEOUT, and the CUDA context stays usable (a search right after is
still bit-exact).  Nothing here traps, faults or hangs the GPU: the wait
ends by itself after its spin limit."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_records_timeout_and_context_survives(gpu):
    for spins in (100_000, 1_000_000):
        status, ms = gpu.sw_probe_wait_timeout(0, spins)
        assert status == 4, status                 # SW_ERR_TIMEOUT
        assert ms < 10_000
    rng = np.random.default_rng(5)
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 400, 60), [3500]]))
    qs = synth.seqset_from_lengths(rng, [120, 2500])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        scores, _, st = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=3, stats=True)
    assert st["long_sequences"] > 0                 # the kernel with the bounded waits ran
    np.testing.assert_array_equal(scores, oracle.all_scores(qs, db, S, 10, 1))


def test_async_search_reports_its_status_word(gpu):
    """An asynchronous search (device outputs, no stats) copies its device-side
    status word to status_out on the stream: 0 after a search in which the
    intra-task kernel's bounded waits all completed (the word is first set to
    a non-zero value, so the copy is seen), with graph capture too."""
    import torch
    rng = np.random.default_rng(6)
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 400, 60), [3500, 3900]]))
    qs = synth.seqset_from_lengths(rng, [120, 2500])
    S = synth.blosum62()
    want = oracle.all_scores(qs, db, S, 10, 1)
    with gpu.Database(db.residues, db.offsets, 24) as d:
        q_dev = torch.from_numpy(qs.residues).cuda()
        scores = torch.empty((qs.n, db.n), dtype=torch.int32, device="cuda")
        status = torch.full((1,), 77, dtype=torch.int32, device="cuda")
        pinned = torch.full((1,), 77, dtype=torch.int32).pin_memory()
        for graph in (False, True, True):
            status.fill_(77)
            pinned.fill_(77)
            gpu.sw_search(d.handle, q_dev, qs.offsets, S, 10, 1, 0, scores, None, status_out=status, graph=graph)
            gpu.sw_search(d.handle, q_dev, qs.offsets, S, 10, 1, 0, scores, None, status_out=pinned)
            torch.cuda.synchronize()
            assert int(status.item()) == 0 and int(pinned.item()) == 0
            np.testing.assert_array_equal(scores.cpu().numpy().astype(np.int64), want)
