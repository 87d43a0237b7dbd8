"""Host check of the rule the DBSCAN union phase walks by (section 2.4,
FDBSCAN): a core point unites only with the neighbours that come before its own
sorted leaf position, and so skips every right child whose range starts at or
after that position (split + 1 >= its position, the split being the left
child's range end).  On radix trees over random 2D points (built on the host
from sorted Morton codes, the same hierarchy the GPU build makes), the pruned
walk from every point must meet exactly the leaves before it within eps, so
each pair within eps is met once, from its later point."""
import random

import numpy as np
import pytest


def _delta(keys, i):
    a, b = int(keys[i]), int(keys[i + 1])
    if a != b:
        return 64 - (a ^ b).bit_length()
    return 64 + 32 - ((i ^ (i + 1)) & 0xFFFFFFFF).bit_length()


def _tree(keys):
    """Children of each internal node g (split between sorted leaves g, g+1) and
    the root; a child is ('leaf', pos) or ('node', g), with its range."""
    n = len(keys)
    child = [[None, None] for _ in range(n - 1)]
    rng_of = {}
    flag = [-1] * (n - 1)
    root = None
    for i in range(n):
        l = r = i
        code = ("leaf", i)
        while True:
            left = l == 0 or (r != n - 1 and _delta(keys, r) > _delta(keys, l - 1))
            g = r if left else l - 1
            child[g][0 if left else 1] = code
            other, flag[g] = flag[g], (l if left else r)
            if other < 0:
                break
            l, r = (l, other) if left else (other, r)
            code = ("node", g)
            rng_of[g] = (l, r)
            if l == 0 and r == n - 1:
                root = g
                break
    return child, rng_of, root


def _box(code, child, pts, rng_of):
    if code[0] == "leaf":
        return pts[code[1]], pts[code[1]]
    l, r = rng_of[code[1]]
    return pts[l:r + 1].min(axis=0), pts[l:r + 1].max(axis=0)


def _box_d2(q, lo, hi):
    t = np.maximum(np.maximum(lo - q, 0.0), q - hi)
    return float((t * t).sum())


@pytest.mark.parametrize("seed", range(4))
def test_union_walk_meets_each_pair_once_from_its_later_point(seed):
    rs = np.random.default_rng(seed)
    n = int(rs.integers(2, 300))
    pts = rs.random((n, 2))
    cells = (pts * 65535).astype(np.uint64)
    codes = np.zeros(n, dtype=np.uint64)
    for b in range(16):
        for a in range(2):
            codes |= ((cells[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + a)
    order = np.argsort(codes, kind="stable")
    keys, spts = codes[order], pts[order]  # leaf position p holds point order[p]
    eps2 = float(rs.choice([0.0, 0.003, 0.02, 0.2]))
    if n == 1:
        return
    child, rng_of, root = _tree(keys)
    for posq in range(n):
        q = spts[posq]
        met, stack = set(), [("node", root)]
        while stack:
            g = stack.pop()[1]
            c0, c1 = child[g]
            split = c0[1] if c0[0] == "leaf" else rng_of[c0[1]][1]
            for side, c in enumerate((c0, c1)):
                if side == 1 and split >= posq - 1:
                    continue  # every leaf of the right child is at or after the query's own position
                lo, hi = _box(c, child, spts, rng_of)
                if _box_d2(q, lo, hi) > eps2:
                    continue
                if c[0] == "leaf":
                    if c[1] < posq:
                        met.add(c[1])
                else:
                    stack.append(c)
        want = {p for p in range(posq) if float(((spts[p] - q) ** 2).sum()) <= eps2}
        assert met == want, (n, posq)
