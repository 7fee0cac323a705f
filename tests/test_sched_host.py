"""Admission policy of the serving form, replayed in virtual time on the host
(lb_sched_simulate; no GPU).  Checks: the budget and slot limits hold at
every instant, nothing starts before it arrives, every admissible request
finishes, strict FIFO when bypassing is off, bypass only within its window,
and requests above the budget are never admitted."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def lb():
    from paper_1912_01491_gb300 import build
    build.build()
    import paper_1912_01491_gb300 as lb
    return lb


def _check_invariants(arr, nb, svc, budget, slots, start, finish):
    ok = nb <= budget
    assert np.all(start[~ok] == -1) and np.all(finish[~ok] == -1)
    assert np.all(start[ok] >= arr[ok])
    assert np.allclose(finish[ok], start[ok] + svc[ok])
    # at every start instant, the running set respects budget and slots
    for t in np.unique(start[ok]):
        run = ok & (start <= t) & (finish > t)
        assert nb[run].sum() <= budget
        assert run.sum() <= slots


def test_everything_fits_starts_on_arrival(lb):
    arr = np.array([0.0, 1.0, 2.0, 5.0])
    nb = np.array([10, 10, 10, 10])
    svc = np.array([3.0, 3.0, 3.0, 3.0])
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=0.0)
    assert np.array_equal(s, arr)
    assert np.array_equal(f, arr + svc)


def test_budget_serialises(lb):
    arr = np.zeros(3)
    nb = np.array([60, 60, 60])
    svc = np.array([5.0, 7.0, 1.0])
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=0.0)
    assert list(s) == [0.0, 5.0, 12.0]
    assert list(f) == [5.0, 12.0, 13.0]


def test_slots_serialise(lb):
    arr = np.zeros(4)
    nb = np.ones(4, np.int64)
    svc = np.array([4.0, 4.0, 4.0, 4.0])
    s, _ = lb.sched_simulate(arr, nb, svc, budget=100, slots=2, bypass_ms=0.0)
    assert list(s) == [0.0, 0.0, 4.0, 4.0]


def test_bypass_window(lb):
    """A (50) runs; B (100, needs everything) arrives at 1; C (10) at 2.
    With a long window C passes B; with bypass off C waits for B."""
    arr = np.array([0.0, 1.0, 2.0])
    nb = np.array([50, 100, 10])
    svc = np.array([10.0, 10.0, 1.0])
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=1e9)
    assert s[2] == 2.0 and s[1] == 10.0
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=0.0)
    assert s[1] == 10.0 and s[2] == 20.0
    # window of 0.5 ms: at t = 2 B has waited 1 ms > 0.5, so C may not pass
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=0.5)
    assert s[2] == 20.0
    # window of 5 ms: C passes
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=8, bypass_ms=5.0)
    assert s[2] == 2.0


def test_oversize_never_admitted(lb):
    arr = np.array([0.0, 0.0, 1.0])
    nb = np.array([10, 500, 10])
    svc = np.array([1.0, 1.0, 1.0])
    s, f = lb.sched_simulate(arr, nb, svc, budget=100, slots=4, bypass_ms=0.0)
    assert s[1] == -1 and f[1] == -1
    assert s[0] == 0.0 and s[2] == 1.0


@pytest.mark.parametrize("bypass", [0.0, 50.0, 1e9])
def test_random_traces_invariants(lb, bypass):
    g = np.random.default_rng(int(bypass) % 97 + 3)
    n = 400
    arr = np.cumsum(g.exponential(5.0, n))
    sizes = np.array([1, 8, 64, 200, 800])
    nb = g.choice(sizes, n)
    svc = nb * g.uniform(0.05, 0.2, n)
    budget, slots = 1000, 6
    s, f = lb.sched_simulate(arr, nb, svc, budget, slots, bypass)
    _check_invariants(arr, nb, svc, budget, slots, s, f)
    if bypass == 0.0:
        assert np.all(np.diff(s) >= 0), "bypass off must admit in arrival order"


def test_rejects_unsorted_arrivals(lb):
    with pytest.raises(lb.LBError):
        lb.sched_simulate([1.0, 0.0], [1, 1], [1.0, 1.0], 10, 1, 0.0)
