"""The job-taking protocol of the fused chain's launch with job counters (`pick_job` in
csrc/kf_chain.cuh), modelled on the host: as many blocks as jobs, each block tries the
three kinds in its SM's order with one atomic increment per kind and takes the first
whose counter was still below the kind's job count. Under any interleaving of the
blocks' increments every job is taken exactly once and every block takes one (a block
passes over a kind only when that kind is exhausted, which stays so)."""
import random

import pytest


def run_protocol(counts, prefs, rng):
    """counts: jobs per kind; prefs: for each block, the order in which it tries the
    kinds. Blocks interleave their steps at random; returns the job each block took."""
    ctr = [0, 0, 0]
    taken = [None] * len(prefs)
    step = [0] * len(prefs)  # next kind index each block will try
    live = list(range(len(prefs)))
    while live:
        b = rng.choice(live)
        k = prefs[b][step[b]]
        t = ctr[k]
        ctr[k] += 1  # the atomic increment
        if t < counts[k]:
            taken[b] = (k, t)
            live.remove(b)
        else:
            step[b] += 1
            assert step[b] < 3, "a block found no job"
    return taken


@pytest.mark.parametrize("counts", [(2000, 4000, 16000), (0, 5, 3), (7, 0, 0), (1, 1, 1), (13, 2, 40)])
def test_every_job_is_taken_once(counts):
    rng = random.Random(sum(counts) + 7)
    n = sum(counts)
    inner = [2, 1, 0]
    outer = [0, 1, 2]
    for trial in range(3):
        prefs = [inner if rng.random() < 0.7 else outer for _ in range(n)]
        taken = run_protocol(counts, prefs, rng)
        assert all(t is not None for t in taken)
        jobs = sorted(taken)
        expect = sorted((k, t) for k in range(3) for t in range(counts[k]))
        assert jobs == expect


def test_a_block_with_no_job_left_would_be_a_contradiction():
    """More blocks than jobs (not how the launch is made) is the only way a block finds
    nothing: the model then reports it."""
    rng = random.Random(3)
    with pytest.raises(AssertionError, match="no job"):
        run_protocol((1, 1, 1), [[0, 1, 2]] * 4, rng)
