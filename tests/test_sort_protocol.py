"""Host check of the radix sort's single-launch pass (decoupled look-back, as
in Merrill and Garland's single-pass prefix scan): each tile publishes its own
per-digit counts, then walks back over earlier tiles' published words, summing
own counts until it meets a running (inclusive) count, and publishes its own
running count.  This model runs the tiles' steps in random interleavings
(blocks start in tile order, each step one poll or one publication) and
requires every tile's digit starts to equal the exclusive scan over tiles, and
the pass to equal a stable counting sort by that digit.  It checks the protocol
only (with 4-bit digits: each digit's look-back is independent of the
others); the GPU tests check the kernels."""
import random

import pytest

BITS = 4
RADIX = 1 << BITS
MASK = RADIX - 1


def _pass(keys, shift, tile, rng):
    n = len(keys)
    tiles = [keys[i:i + tile] for i in range(0, n, tile)]
    counts = [[0] * RADIX for _ in tiles]
    for t, ks in enumerate(tiles):
        for k in ks:
            counts[t][(k >> shift) & MASK] += 1
    total = [sum(c[d] for c in counts) for d in range(RADIX)]
    gstart = [0] * RADIX
    for d in range(1, RADIX):
        gstart[d] = gstart[d - 1] + total[d - 1]
    status = [[None] * RADIX for _ in tiles]  # None: unpublished; ('A', c) own; ('I', c) running
    before = [[0] * RADIX for _ in tiles]

    def block(t):
        for d in range(RADIX):  # own counts first (the running count at once for tile 0)
            status[t][d] = ('I' if t == 0 else 'A', counts[t][d])
        yield
        if t > 0:
            for d in range(RADIX):
                s, u = 0, t - 1
                while True:
                    w = status[u][d]
                    if w is None:
                        yield  # poll again later
                        continue
                    s += w[1]
                    if w[0] == 'I' or u == 0:
                        break
                    u -= 1
                before[t][d] = s
                status[t][d] = ('I', s + counts[t][d])
                yield

    # blocks start in tile order; a started block runs interleaved with the others
    running, started = [], 0
    while started < len(tiles) or running:
        if started < len(tiles) and (not running or rng.random() < 0.3):
            running.append(block(started))
            started += 1
            continue
        k = rng.randrange(len(running))
        try:
            next(running[k])
        except StopIteration:
            running.pop(k)
    out = [None] * n
    for t, ks in enumerate(tiles):
        seen = [0] * RADIX
        for k in ks:  # stable within the tile
            d = (k >> shift) & MASK
            out[gstart[d] + before[t][d] + seen[d]] = k
            seen[d] += 1
        for d in range(RADIX):
            assert before[t][d] == sum(c[d] for c in counts[:t])
    return out


@pytest.mark.parametrize("seed", range(4))
def test_lookback_pass_is_a_stable_counting_sort(seed):
    rng = random.Random(seed)
    for _ in range(8):
        n = rng.choice([1, 7, 100, 1000, 3000])
        tile = rng.choice([max(1, n // 64), 16, 64, 256, 2048])
        keys = [rng.getrandbits(rng.choice([4, 8, 24])) for _ in range(n)]
        shift = rng.choice([0, 4])
        got = _pass(keys, shift, tile, rng)
        assert got == sorted(keys, key=lambda k: (k >> shift) & MASK)  # Python's sort is stable
