"""Host logic of the batched solve: the grouping of scenes into two-block
cluster jobs (no device needed)."""
import numpy as np
import pytest

from paper_1808_02558_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    return binding.load()


def check_cover(jobs, n):
    seen = [s for a, b in jobs for s in ((a,) if b == -2 else (a, b)) if s >= 0]
    assert sorted(seen) == list(range(n))


def estimate(job, cost):
    a, b = job
    return 0.5 * cost[a] if b == -2 else cost[a]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_automatic_split_takes_scenes_above_an_even_share(lib, seed):
    rng = np.random.default_rng(seed)
    sides = rng.integers(4, 17, size=256)
    cost = [int(4 * s * s * (s - 1) + s * s) for s in sides]
    jobs = binding.newton_batch_plan(cost, 152)
    check_cover(jobs, len(cost))
    share = sum(cost) / 152
    split = {a for a, b in jobs if b == -2}
    assert split == {i for i, c in enumerate(cost) if c > share}
    est = [estimate(j, cost) for j in jobs]
    assert est == sorted(est, reverse=True)
    for a, b in jobs:
        if b >= 0:
            assert cost[a] >= cost[b]
            # neighbours in decreasing cost: nothing unsplit lies strictly between them
            between = [c for i, c in enumerate(cost) if i not in split and cost[b] < c < cost[a]]
            assert not between


def test_modes_none_and_all(lib):
    cost = [5, 9, 1, 9, 3]
    none = binding.newton_batch_plan(cost, 4, split=1)
    check_cover(none, 5)
    assert all(b != -2 for _, b in none)
    # decreasing cost (ties in index order): 1, 3, 0, 4, 2 -> pairs (1, 3), (0, 4), (2, -1)
    assert none == [(1, 3), (0, 4), (2, -1)]
    every = binding.newton_batch_plan(cost, 4, split=2)
    assert every == [(1, -2), (3, -2), (0, -2), (4, -2), (2, -2)]


def test_small_batches_split_everything_large(lib):
    # one scene: its cost exceeds total / SMs, so it runs on both blocks
    assert binding.newton_batch_plan([100], 152) == [(0, -2)]
    assert binding.newton_batch_plan([], 152) == []
    # equal costs on one SM: none exceeds the share (the total), so they pair
    assert binding.newton_batch_plan([7, 7, 7], 1) == [(0, 1), (2, -1)]


def test_plan_rejects_bad_arguments(lib):
    with pytest.raises(binding.QPError) as e:
        binding.newton_batch_plan([1, 2], 152, split=3)
    assert e.value.code == binding.QP_INVALID_ARG
    with pytest.raises(binding.QPError) as e:
        binding.newton_batch_plan([1, -2], 152)
    assert e.value.code == binding.QP_INVALID_ARG
