"""Host logic of grouped batch waves: the CTA split of snn_plan_groups against
brute force (no GPU needed)."""
import itertools

import numpy as np
import pytest

from paper_1803_08833_gb300 import snn

F = 8.0  # microseconds of a step's fixed latency in the split's cost model


@pytest.fixture(scope="module")
def lib():
    from paper_1803_08833_gb300 import _build
    _build.build()
    return snn.load()


def _makespan(steps, work, cta):
    return max((s * (F + w / g) for s, w, g in zip(steps, work, cta) if s > 0), default=0.0)


def test_equal_networks_split_evenly(lib):
    assert list(snn.plan_groups([100, 100], [50.0, 50.0], 152)) == [76, 76]
    assert list(snn.plan_groups([7] * 4, [10.0] * 4, 10)) in ([3, 3, 2, 2], [3, 2, 3, 2], [2, 3, 3, 2],
                                                                [2, 2, 3, 3], [3, 2, 2, 3], [2, 3, 2, 3])


def test_idle_networks_get_nothing_and_all_ctas_are_used(lib):
    cta = snn.plan_groups([100, 0, 100, 0], [500.0, 9.0, 5.0, 0.0], 152)
    assert cta[1] == 0 and cta[3] == 0 and cta[0] >= 1 and cta[2] >= 1 and cta.sum() == 152
    assert list(snn.plan_groups([0, 0], [1.0, 1.0], 8)) == [0, 0]


@pytest.mark.parametrize("seed", range(40))
def test_split_is_optimal_against_brute_force(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 4))
    S = int(rng.integers(n, 11))
    steps = rng.integers(0, 4, n) * int(rng.integers(1, 500))
    work = rng.choice([0.0, 1.0, 10.0, 100.0, 1000.0], n) * rng.uniform(0.5, 2.0, n)
    cta = snn.plan_groups(steps, work, S)
    assert np.all((cta == 0) == (steps == 0))
    if np.any(steps > 0):
        assert cta.sum() == S
    ranges = [range(1, S + 1) if s > 0 else range(0, 1) for s in steps]
    best = min(_makespan(steps, work, g) for g in itertools.product(*ranges) if sum(g) <= S)
    assert _makespan(steps, work, cta) <= best * (1 + 1e-9) + 1e-12


def test_the_largest_work_gets_the_most(lib):
    cta = snn.plan_groups([1000] * 5, [2000.0, 100.0, 400.0, 10.0, 800.0], 152)
    assert list(np.argsort(-cta.astype(np.int64), kind="stable")[:3]) == [0, 4, 2]
    assert cta.min() >= 1


@pytest.mark.parametrize("steps,work,ctas", [
    ([1, 1, 1], [1.0, 1.0, 1.0], 2),           # more networks than CTAs
    ([1, 1], [1.0, -1.0], 8),                  # negative work
    ([1, 1], [1.0, float("nan")], 8),          # not finite
    ([1], [float("inf")], 8),
])
def test_bad_plans_are_refused(lib, steps, work, ctas):
    with pytest.raises(snn.SnnError):
        snn.plan_groups(steps, work, ctas)


def test_null_arguments(lib):
    assert lib.snn_plan_groups(None, None, 1, 8, None) == snn.SNN_EINVAL
    assert lib.snn_batch_set_mode(None, 0) == snn.SNN_EINVAL
    assert lib.snn_batch_groups(None, None) == snn.SNN_EINVAL
    assert lib.snn_set_resident_state(None, 1, None, None) == snn.SNN_EINVAL


@pytest.mark.parametrize("seed", range(5))
def test_large_split_is_locally_optimal(lib, seed):
    """A full wave (up to one network per SM): the split uses every CTA, and no
    single CTA moved from one group to the group that finishes last shortens
    the makespan."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 153))
    S = 152
    steps = rng.integers(1, 3000, n)
    work = rng.lognormal(3.0, 1.5, n)
    cta = snn.plan_groups(steps, work, S).astype(np.int64)
    assert cta.sum() == S and cta.min() >= 1
    t = steps * (F + work / cta)
    worst = int(np.argmax(t))
    for j in range(n):
        if j == worst or cta[j] == 1:
            continue
        c2 = cta.copy()
        c2[j] -= 1
        c2[worst] += 1
        assert _makespan(steps, work, c2) >= t.max() * (1 - 1e-12)
