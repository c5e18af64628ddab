"""Host logic of the serving loop: the arena allocator and the request
stream (no GPU, no CUDA library needed)."""
import numpy as np
import pytest

from paper_1205_2584_gb300.serve import Arena, poisson_requests, Request


def test_arena_first_fit_alignment_and_exhaustion():
    ar = Arena(4096, base=512, align=256)
    a = ar.alloc(1)          # rounds up to one unit
    b = ar.alloc(700)        # three units
    assert (a, b) == (512, 768)
    assert ar.used == 256 + 768
    assert all(off % 256 == 0 for off in (a, b))
    c = ar.alloc(4096)       # larger than what is left
    assert c is None
    d = ar.alloc(4096 - 1024)
    assert d == 512 + 1024
    assert ar.alloc(1) is None
    assert ar.largest_free() == 0


def test_arena_free_coalesces_both_sides():
    ar = Arena(10 * 256, align=256)
    offs = [ar.alloc(256) for _ in range(10)]
    assert offs == [k * 256 for k in range(10)]
    for k in (3, 5):
        ar.free(offs[k])
    assert ar.largest_free() == 256
    ar.free(offs[4])                     # joins 3,4,5
    assert ar.largest_free() == 3 * 256
    assert ar.alloc(3 * 256) == 3 * 256  # first fit takes the joined hole
    for k in range(10):
        if k not in (3, 4, 5):
            ar.free(offs[k])
    ar.free(3 * 256)
    assert ar.largest_free() == 10 * 256 and ar.used == 0


def test_arena_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(1)
    ar = Arena(1 << 20, align=256)
    live = {}
    for _ in range(3000):
        if live and rng.uniform() < 0.45:
            off = list(live)[rng.integers(len(live))]
            ar.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 40000))
            off = ar.alloc(n)
            if off is None:
                continue
            live[off] = (n + 255) // 256 * 256
        spans = sorted(live.items())
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2
        assert ar.used == sum(live.values())
        assert all(0 <= o and o + s <= ar.size for o, s in spans)


def test_poisson_stream_is_seeded_and_mixed():
    r1 = poisson_requests(seed=3, rate=200.0, seconds=5.0)
    r2 = poisson_requests(seed=3, rate=200.0, seconds=5.0)
    assert [(r.arrival, r.seed, r.dims, r.R) for r in r1] == [(r.arrival, r.seed, r.dims, r.R) for r in r2]
    assert 800 < len(r1) < 1200                      # ~ rate * seconds
    arr = np.array([r.arrival for r in r1])
    assert np.all(np.diff(arr) > 0) and arr[-1] <= 5.0
    frac = np.mean([r.dims == (32, 32, 32) for r in r1])
    assert 0.6 < frac < 0.8
    assert {r.R for r in r1} <= {5, 16, 30}
    assert all(0.0 <= r.collinearity <= 0.95 for r in r1)
    assert Request(0, 0.0, (4, 5, 6), 3).cost == 360.0
