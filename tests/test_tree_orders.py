"""The three shapes of the fixed pairwise summation tree that the fit uses
agree bit for bit on non-negative FP64 terms (CPU).

The oracle sums a list by halving it pair by pair and carrying an odd last
value; the device sums a 256-position chunk as the complete binary tree with
zero padding (a warp), and a leaf of at most 32 samples in sample order like
a binary counter (one lane).  Adding +0.0 to a term >= +0 is exact, so the
three agree; this checks it on random terms of every length up to 64.
"""
import numpy as np
import pytest


def halve_and_carry(t):
    p = list(t)
    if not p:
        return 0.0
    while len(p) > 1:
        q = [p[2 * i] + p[2 * i + 1] for i in range(len(p) // 2)]
        if len(p) & 1:
            q.append(p[-1])
        p = q
    return p[0]


def padded_complete_tree(t, width=256):
    p = list(t) + [0.0] * (width - len(t))
    while len(p) > 1:
        p = [p[2 * i] + p[2 * i + 1] for i in range(len(p) // 2)]
    return p[0]


def binary_counter(t):
    levels = {}
    for x in t:
        carry, k = x, 0
        while k in levels:
            carry = levels.pop(k) + carry
            k += 1
        levels[k] = carry
    acc = None
    for k in sorted(levels):
        acc = levels[k] if acc is None else levels[k] + acc
    return 0.0 if acc is None else acc


@pytest.mark.parametrize("seed", range(4))
def test_tree_shapes_agree(seed):
    rng = np.random.default_rng(seed)
    for m in range(1, 65):
        # mixed magnitudes, so that a different association would round differently
        t = [float(v) for v in rng.random(m) * 10.0 ** rng.integers(-8, 9, m)]
        a = halve_and_carry(t)
        b = padded_complete_tree(t)
        c = binary_counter(t)
        assert np.float64(a).tobytes() == np.float64(b).tobytes() == np.float64(c).tobytes(), m


def test_association_matters_for_these_terms():
    """Guard: the test above would catch a wrong shape (left-to-right differs)."""
    rng = np.random.default_rng(7)
    differs = 0
    for m in range(3, 65):
        t = [float(v) for v in rng.random(m) * 10.0 ** rng.integers(-8, 9, m)]
        seq = 0.0
        for x in t:
            seq += x
        differs += seq != halve_and_carry(t)
    assert differs > 10
