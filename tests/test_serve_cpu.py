"""Host-side logic of the serving layer that needs no GPU: the autotuner's
choice rule and the synthetic request stream."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def serve():
    import __graft_entry__ as g
    g.build()
    from paper_1803_01190_gb300 import serve as s
    return s


def test_autotuner_explores_then_exploits(serve):
    t = serve.Autotuner(candidates=[(1, 1), (2, 1), (4, 1)], trials=2, recheck_every=5)
    cost = {(1, 1): 3.0, (2, 1): 1.0, (4, 1): 2.0}
    key = serve.Autotuner.bucket("fp64", 2.0 ** 31)
    assert serve.Autotuner.bucket("fp64", 2.0 ** 32) == key       # same factor-of-8 bucket
    seen = []
    for _ in range(6):                     # exploration: each candidate twice
        c = t.choose(key)
        seen.append(c)
        t.record(key, c, cost[c])
    assert sorted(seen) == sorted([(1, 1), (2, 1), (4, 1)] * 2)
    picks = []
    for _ in range(10):
        c = t.choose(key)
        picks.append(c)
        t.record(key, c, cost[c])
    assert picks.count((2, 1)) == 8 and picks.count((4, 1)) == 2    # best, runner-up re-checked
    assert t.best(key) == (2, 1)
    # buckets are separate: another load starts exploring again
    assert t.choose(serve.Autotuner.bucket("fp64", 1e12)) == (1, 1)
    assert serve.Autotuner.bucket("mixed", 2.0 ** 31) != key


def test_autotuner_follows_a_change(serve):
    t = serve.Autotuner(candidates=[(1, 1), (2, 1)], trials=1, recheck_every=2)
    key = ("fp64", 10)
    cost = {(1, 1): 1.0, (2, 1): 2.0}
    for _ in range(6):
        c = t.choose(key)
        t.record(key, c, cost[c])
    assert t.best(key) == (1, 1)
    cost = {(1, 1): 5.0, (2, 1): 2.0}      # the first shape became slow
    for _ in range(40):
        c = t.choose(key)
        t.record(key, c, cost[c])
    assert t.best(key) == (2, 1)


def test_poisson_requests(serve):
    reqs = serve.poisson_requests(4000, rate=200.0, seed=1)
    t = np.array([r.t_arrive for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(reqs) / t[-1] - 200.0) < 10.0
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 2 ** 10 and ns.max() <= 2 ** 16
    assert abs(np.mean(np.log2(ns)) - 13.0) < 0.2                # log-uniform on [2^10, 2^16]
    assert 0.45 < np.mean([r.mode == "mixed" for r in reqs]) < 0.55
    assert 0.45 < np.mean([r.eps == 0.02 for r in reqs]) < 0.55   # disk + halo half of the time
    p, v, m = reqs[0].make()
    assert p.shape == (reqs[0].n, 3) and m.shape == (reqs[0].n,)
