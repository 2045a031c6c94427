"""The seeded generators: shapes, ranges and determinism."""
import numpy as np

from paper_1401_0763_gb300 import workloads as wl


def test_random_edges_layout():
    n = 10
    u = wl.random_edges(n, 3)
    assert u.shape == (12, 12)
    assert np.all(u[1:-1, 1:-1] == 0)
    ring = np.concatenate([u[0, :], u[-1, :], u[1:-1, 0], u[1:-1, -1]])
    assert ring.size == 4 * (n + 2) - 4 and ring.min() >= 0 and ring.max() <= 100
    assert np.array_equal(u, wl.random_edges(n, 3)) and not np.array_equal(u, wl.random_edges(n, 4))


def test_gaussian_source_and_sizes():
    f = wl.gaussian_source(64, 1)
    assert f.shape == (64, 64) and np.isfinite(f).all() and np.abs(f).max() <= 8
    s = wl.batch_sizes(512, 0)
    assert s.min() >= 64 and s.max() <= 1024 and len(s) == 512
    reqs = wl.request_stream(100, 50.0, 0)
    t = [r.arrival_s for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert all(128 <= r.n <= 4096 and 1e-10 <= r.tol <= 1e-6 for r in reqs)


def test_heat_plate_edges():
    for e in ("north", "south", "west", "east"):
        u = wl.heat_plate(5, 100.0, e)
        assert u.sum() == 100.0 * 7


def _gaussian_source_unblocked(n, seed, count=8):
    """The Gaussian sum written term by term on whole arrays (the blocked
    generator must give the same bits)."""
    g = wl.rng(seed)
    a = g.uniform(-1.0, 1.0, size=count)
    s = g.uniform(0.02, 0.2, size=count)
    c = g.uniform(0.0, 1.0, size=(count, 2))
    xs = np.arange(1, n + 1, dtype=np.float64) * (1.0 / (n + 1))
    f = np.zeros((n, n))
    for k in range(count):
        ex = np.exp(-((xs - c[k, 0]) ** 2) / (2.0 * s[k] ** 2))
        ey = np.exp(-((xs - c[k, 1]) ** 2) / (2.0 * s[k] ** 2))
        f += a[k] * np.outer(ey, ex)
    return f


def test_gaussian_source_blocked_equals_unblocked():
    for n in (1, 7, 300, 4097):
        assert np.array_equal(wl.gaussian_source(n, n), _gaussian_source_unblocked(n, n))
