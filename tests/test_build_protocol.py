"""Host check of the hierarchy build's handoff protocol (section 2.6: the
bottom-up construction of Apetrei).  The CUDA build completes a node whose two
children lie in one chunk of sorted leaves through that chunk's shared memory,
lists the arrivals at nodes whose range crosses a chunk boundary (a parent
split at the chunk's edge, or a first arrival whose sibling never came), and
completes those in a second pass through global flags.  This model replays
that protocol in random interleavings and requires the same children and root
as the plain climb (one arrival at a time, every handoff through one flag per
node), for random, duplicate and clustered 63-bit codes and chunk sizes down to
two leaves.  It checks the protocol only; the GPU tests check the kernels."""
import random

import pytest


def _delta(keys, i):
    a, b = keys[i], keys[i + 1]
    if a != b:
        return 64 - (a ^ b).bit_length()
    return 64 + 32 - ((i ^ (i + 1)) & 0xFFFFFFFF).bit_length()


def _parent(keys, l, r):
    n = len(keys)
    left = l == 0 or (r != n - 1 and _delta(keys, r) > _delta(keys, l - 1))
    return left, (r if left else l - 1)


def _plain_climb(keys, rng):
    n = len(keys)
    child = [[None, None] for _ in range(n - 1)]
    flag = [-1] * (n - 1)
    root = None
    for i in rng.sample(range(n), n):
        l = r = i
        code = ("leaf", i)
        while True:
            left, g = _parent(keys, l, r)
            child[g][0 if left else 1] = code
            other, flag[g] = flag[g], (l if left else r)
            if other < 0:
                break
            l, r = (l, other) if left else (other, r)
            code = ("node", g)
            if l == 0 and r == n - 1:
                root = g
                break
    return child, root


def _interleave(gens, rng):
    while gens:
        k = rng.randrange(len(gens))
        try:
            next(gens[k])
        except StopIteration:
            gens.pop(k)


def _chunked(keys, chunk, rng):
    n = len(keys)
    child = [[None, None] for _ in range(n - 1)]
    root = [None]
    listed = []

    for ch in rng.sample(range((n + chunk - 1) // chunk), (n + chunk - 1) // chunk):
        c0, c1 = ch * chunk, min(n, ch * chunk + chunk)
        sflag = {}

        def climb(i):
            l = r = i
            code = ("leaf", i)
            while True:
                left, g = _parent(keys, l, r)
                child[g][0 if left else 1] = code
                if (r >= c1 - 1) if left else (l <= c0):  # split at the chunk's edge
                    listed.append((g, l if left else r))
                    return
                yield
                other = sflag.get(g, -1)
                sflag[g] = l if left else r
                if other < 0:
                    return
                sflag[g] = -2
                l, r = (l, other) if left else (other, r)
                code = ("node", g)
                if l == 0 and r == n - 1:
                    root[0] = g
                    return
                yield

        _interleave([climb(i) for i in range(c0, c1)], rng)
        listed += [(j, sflag[j]) for j in range(c0, c1 - 1) if sflag.get(j, -1) >= 0]

    flag = [-1] * (n - 1)

    def global_climb(g, v):
        left = v <= g
        l, r = (v, g) if left else (g + 1, v)
        written = True
        while True:
            if not written:
                left, g = _parent(keys, l, r)
                child[g][0 if left else 1] = code
            written = False
            yield
            other, flag[g] = flag[g], (l if left else r)
            if other < 0:
                return
            l, r = (l, other) if left else (other, r)
            code = ("node", g)
            if l == 0 and r == n - 1:
                root[0] = g
                return
            yield

    _interleave([global_climb(g, v) for g, v in listed], rng)
    return child, root[0], len(listed)


@pytest.mark.parametrize("seed", range(6))
def test_chunked_handoff_equals_plain_climb(seed):
    rng = random.Random(seed)
    for _ in range(25):
        n = rng.choice([2, 3, 5, 17, 64, 100, 513, 1000])
        chunk = rng.choice([2, 4, 8, 16, 64, 512])
        kind = rng.choice(["random", "duplicates", "clustered"])
        if kind == "random":
            keys = sorted(rng.getrandbits(63) for _ in range(n))
        elif kind == "duplicates":
            keys = sorted(rng.choice([5, 7, 9, 1 << 40]) for _ in range(n))
        else:
            keys = sorted(rng.getrandbits(6) << 50 for _ in range(n))
        ref_child, ref_root = _plain_climb(keys, rng)
        child, root, nlisted = _chunked(keys, chunk, rng)
        assert child == ref_child, (n, chunk, kind)
        assert root == ref_root, (n, chunk, kind)
        # the list bound the build allocates: two arrivals per node on the
        # root path of each chunk boundary (at most 97 nodes deep)
        nchunks = (n + chunk - 1) // chunk
        assert nlisted <= min(2 * n, 2 * 97 * nchunks + 2)
