"""Host-side logic of the serving engine (admission by HBM budget, LRU eviction),
with the GPU hierarchy replaced by a fake; no GPU needed."""
import threading

import pytest

serve = pytest.importorskip("paper_2008_03885_gb300.serve")


class FakeHierarchy:
    closed = []

    def __init__(self, key, opts):
        self.key = key

    def close(self):
        FakeHierarchy.closed.append(self.key)


@pytest.fixture
def cache(monkeypatch):
    monkeypatch.setattr(serve, "Hierarchy", FakeHierarchy)
    FakeHierarchy.closed = []
    c = serve.HierarchyCache(budget_bytes=100, opts={})
    monkeypatch.setattr(c, "key_bytes", lambda key: key[0])  # key = (bytes, order, op)
    return c


def test_reuse_idle_hierarchy_without_new_memory(cache):
    a = cache.acquire((40, 2, "galerkin"))
    cache.release(a)
    b = cache.acquire((40, 2, "galerkin"))
    assert b is a and cache.created == 1 and cache.in_use == 40


def test_lru_eviction_makes_room(cache):
    x = cache.acquire((40, 2, "galerkin"))
    y = cache.acquire((50, 4, "galerkin"))
    cache.release(x)
    cache.release(y)  # x is least recently used
    z = cache.acquire((45, 2, "nongalerkin"))
    assert FakeHierarchy.closed == [(40, 2, "galerkin")]
    assert cache.in_use == 95 and cache.evicted == 1 and z.key == (45, 2, "nongalerkin")


def test_request_larger_than_budget_is_refused(cache):
    import paper_2008_03885_gb300 as mg
    with pytest.raises(mg.MGError) as e:
        cache.acquire((150, 2, "galerkin"))
    assert e.value.status == mg.MG_ERR_BUDGET


def test_admission_waits_until_memory_frees(cache):
    held = cache.acquire((70, 2, "galerkin"))
    got = []

    def later():
        got.append(cache.acquire((60, 4, "galerkin")))

    t = threading.Thread(target=later)
    t.start()
    t.join(timeout=0.3)
    assert t.is_alive() and not got  # 70 + 60 > 100 and nothing idle to evict
    cache.release(held)  # now idle: evictable
    t.join(timeout=5)
    assert got and got[0].key == (60, 4, "galerkin")
    assert cache.in_use == 60


def test_poisson_stream_is_seeded_and_shaped():
    import numpy as np
    a = serve.poisson_stream(3, 50, 2000.0, 4, 6, rhs=lambda n, s: np.zeros((n + 1, n + 1)))
    b = serve.poisson_stream(3, 50, 2000.0, 4, 6, rhs=lambda n, s: np.zeros((n + 1, n + 1)))
    assert [(r.n, r.order, r.coarse_op, r.arrival) for r in a] == [(r.n, r.order, r.coarse_op, r.arrival) for r in b]
    assert all(r.n in (16, 32, 64) for r in a)
    assert all(a[i].arrival < a[i + 1].arrival for i in range(49))
    gaps = np.diff([r.arrival for r in a])
    assert 0.2 / 2000 < gaps.mean() < 5.0 / 2000
