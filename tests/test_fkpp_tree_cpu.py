"""Host model of the Fisher-KPP scan tree (CPU, no GPU).

The replay kernel finds tile t's incoming vector by walking from the root to
leaf t: -r_0 at the root, and at each right turn into child c the left
sibling's aggregate is applied, z <- z + S_{c-1} z + b_{c-1} (the delta form
of the operator of eq. 3.3).  The up-sweep pairs the nodes of each level
(S = S2 + S1 + S2 S1, b = b1 + S2 b1 + b2; a lone last node is copied).  This
model uses the same level layout and indexing and checks the walk against
the definition of the exclusive scan: the leaf elements 0 .. t-1 applied in
order to -r_0.
"""
import numpy as np
import pytest


def build_tree(S_leaf, b_leaf):
    levels = [(S_leaf, b_leaf)]
    while len(levels[-1][0]) > 1:
        S, b = levels[-1]
        n = len(S)
        Sp, bp = [], []
        for m in range((n + 1) // 2):
            if 2 * m + 1 < n:
                S1, b1, S2, b2 = S[2 * m], b[2 * m], S[2 * m + 1], b[2 * m + 1]
                Sp.append(S2 + S1 + S2 @ S1)
                bp.append(b1 + S2 @ b1 + b2)
            else:
                Sp.append(S[2 * m].copy())
                bp.append(b[2 * m].copy())
        levels.append((np.array(Sp), np.array(bp)))
    return levels


def walk(levels, t, z0):
    L = len(levels) - 1
    z = z0.copy()
    for lv in range(L, 0, -1):
        c = t >> (lv - 1)
        if c & 1:
            S, b = levels[lv - 1]
            z = z + S[c - 1] @ z + b[c - 1]
    return z


@pytest.mark.parametrize("T", [1, 2, 3, 5, 8, 13, 64, 607])
def test_tree_walk_is_the_exclusive_scan(T):
    rng = np.random.default_rng(T)
    d = 6
    S_leaf = rng.uniform(-0.3, 0.3, (T, d, d)) / d
    b_leaf = rng.uniform(-1, 1, (T, d))
    z0 = rng.uniform(-1, 1, d)
    levels = build_tree(S_leaf, b_leaf)
    ref = z0.copy()
    for t in range(T):
        z = walk(levels, t, z0)
        assert np.allclose(z, ref, rtol=1e-12, atol=1e-12), t
        ref = ref + S_leaf[t] @ ref + b_leaf[t]


def test_walk_reads_only_left_siblings_below_the_root():
    # the up-sweep skips the root's compose: the walks read only even-indexed
    # nodes (left siblings) of the levels below the root
    T = 607
    L = len(build_tree(np.zeros((T, 1, 1)), np.zeros((T, 1)))) - 1
    read = set()
    for t in range(T):
        for lv in range(L, 0, -1):
            c = t >> (lv - 1)
            if c & 1:
                read.add((lv - 1, c - 1))
    assert read and all(i % 2 == 0 for _, i in read)
    assert max(lv for lv, _ in read) == L - 1
