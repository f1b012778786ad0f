"""The server's admission allocator (faco_test_pool, host only, no GPU)
against a plain first-fit model of the same policy: 256-byte granules, the
lowest free range that fits, freed ranges merged with free neighbours.
Invariants checked on the library's answers: taken ranges never overlap,
stay inside the pool, and the bytes in use are their sum."""
import numpy as np
import pytest

from paper_2203_02228_gb300 import FacoError, pool_replay


def g256(b):
    return (b + 255) // 256 * 256


class FirstFit:
    def __init__(self, size):
        self.size = size // 256 * 256
        self.free = [(0, self.size)] if self.size else []

    def take(self, b):
        b = g256(b)
        for i, (o, n) in enumerate(self.free):
            if n >= b:
                self.free[i:i + 1] = [(o + b, n - b)] if n > b else []
                return o
        return -1

    def give(self, o, b):
        self.free.append((o, g256(b)))
        self.free.sort()
        merged = []
        for o2, n2 in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o2:
                merged[-1] = (merged[-1][0], merged[-1][1] + n2)
            else:
                merged.append((o2, n2))
        self.free = merged


@pytest.mark.parametrize("seed", range(5))
def test_pool_matches_first_fit(seed):
    rng = np.random.default_rng(seed)
    size = int(rng.integers(4096, 1 << 20))
    model = FirstFit(size)
    ops, held, expect = [], {}, []
    in_use = 0
    for i in range(400):
        if held and rng.random() < 0.45:
            j = int(rng.choice(list(held)))
            o, b = held.pop(j)
            model.give(o, b)
            in_use -= g256(b)
            ops.append((0, j))
            expect.append((0, in_use))
        else:
            b = int(rng.integers(1, size // 6 + 2))
            o = model.take(b)
            if o >= 0:
                held[i] = (o, b)
                in_use += g256(b)
            ops.append((b, 0))
            expect.append((o, in_use))
    out = pool_replay(size, np.array(ops))
    np.testing.assert_array_equal(out, np.array(expect))
    # the library's own ranges: disjoint and inside the pool
    live = {}
    for i, ((a, j), (o, _)) in enumerate(zip(ops, out)):
        if a > 0 and o >= 0:
            live[i] = (o, g256(a))
        elif a == 0:
            live.pop(j, None)
        spans = sorted(live.values())
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert all(o + n <= size // 256 * 256 for o, n in spans)


def test_pool_merges_neighbours_into_one_range():
    # three takes fill the pool; giving back the outer two then the middle
    # one must leave a single free range that the whole pool fits in again
    out = pool_replay(3 * 256, np.array([(256, 0), (256, 0), (256, 0), (0, 0), (0, 2), (0, 1), (768, 0)]))
    assert list(out[:3, 0]) == [0, 256, 512]
    assert out[6, 0] == 0 and out[6, 1] == 768


def test_pool_rejects_a_malformed_script():
    with pytest.raises(FacoError):
        pool_replay(4096, np.array([(0, 0)]))  # gives back before anything was taken
    with pytest.raises(FacoError):
        pool_replay(4096, np.array([(256, 0), (0, 0), (0, 0)]))  # gives back twice
